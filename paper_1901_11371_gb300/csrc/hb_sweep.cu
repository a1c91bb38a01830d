// Cooperative sweep kernel: precision dispatch and the barrier error readout.
// The kernel templates live in hb_sweep_impl.cuh; their instances are compiled
// in hb_sweep_f64.cu, hb_sweep_f32n.cu, hb_sweep_f32w.cu and hb_sweep_mix.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_device.h"
#include "hb_sweep_launch.h"

namespace hb {

int launch_sweep_coop(const DevFactor& df, Prec p, int which, void* vec, int64_t R, void* state, void* bar,
                      cudaStream_t st, long long spin_limit) {
  if (which < 0 || which > 3) return HB_EINVAL;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms > 0 ? sms : 1;
  // columns per CTA of the single-CTA runs
  const int64_t q = (R + grid - 1) / grid;
  if (p == PREC_F64) return sweep_coop_f64(df, which, vec, R, state, bar, st, spin_limit, q);
  if (p == PREC_F32) {
    if (q <= 2) return sweep_coop_f32_narrow(df, which, vec, R, state, bar, st, spin_limit, q);
    return sweep_coop_f32_wide(df, which, vec, R, state, bar, st, spin_limit, q);
  }
  return sweep_coop_mix(df, which, vec, R, state, bar, st, spin_limit, q);
}

int read_grid_error(void* bar, cudaStream_t st, int* err) {
  GridBar h;
  if (cudaMemcpyAsync(&h, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, st) != cudaSuccess) return HB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HB_ECUDA;
  *err = h.err;
  if (h.err) {
    int zero = 0;
    if (cudaMemcpyAsync((char*)bar + 2 * sizeof(unsigned int), &zero, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) return HB_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HB_ECUDA;
  }
  return HB_OK;
}

}  // namespace hb

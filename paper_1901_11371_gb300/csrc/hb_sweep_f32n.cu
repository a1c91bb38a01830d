// Sweep kernel instances: complex FP32, one or two columns per CTA.
#include "hb_sweep_impl.cuh"

namespace hb {

int sweep_coop_f32_narrow(const DevFactor& df, int which, void* vec, int64_t R, void* st, void* bar, cudaStream_t s,
                          long long spin_limit, int64_t q) {
  if (q == 2) return sweep_coop_impl<float, float2, 2>(df, which, vec, R, st, bar, s, spin_limit);
  return sweep_coop_impl<float, float2, 1>(df, which, vec, R, st, bar, s, spin_limit);
}

}  // namespace hb

// Sweep kernel instances: complex FP64 factors and arithmetic (HB_C128).
#include "hb_sweep_impl.cuh"

namespace hb {

int sweep_coop_f64(const DevFactor& df, int which, void* vec, int64_t R, void* st, void* bar, cudaStream_t s,
                   long long spin_limit, int64_t q) {
  if (q >= 3) return sweep_coop_impl<double, double2, 4>(df, which, vec, R, st, bar, s, spin_limit);
  if (q == 2) return sweep_coop_impl<double, double2, 2>(df, which, vec, R, st, bar, s, spin_limit);
  return sweep_coop_impl<double, double2, 1>(df, which, vec, R, st, bar, s, spin_limit);
}

}  // namespace hb

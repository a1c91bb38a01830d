// Launch entry points of the cooperative sweep kernel, one per precision and
// column-chunk width (each in its own translation unit), and the grid-barrier
// state they share with the host.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_device.h"

namespace hb {

// Bounded-spin grid barrier state + error flag (device memory, zeroed per launch
// except err, which hb_status reads and clears).
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

// Limit of the wait for a CTA's own bulk copies still in flight after another
// bounded wait gave up: at least 2^22 polls whatever the configured limit, so
// that no copy lands in shared memory after the CTA has left.
__host__ __device__ inline long long drain_limit(long long spin_limit) {
  return spin_limit > (1LL << 22) ? spin_limit : (1LL << 22);
}

// q = columns per CTA of the single-CTA runs (ceil(R / #SMs)); each function
// picks the column-chunk width RC for q and launches the kernel.
int sweep_coop_f64(const DevFactor& df, int which, void* vec, int64_t R, void* st, void* bar, cudaStream_t s,
                   long long spin_limit, int64_t q);
int sweep_coop_f32_narrow(const DevFactor& df, int which, void* vec, int64_t R, void* st, void* bar,
                          cudaStream_t s, long long spin_limit, int64_t q);   // q <= 2
int sweep_coop_f32_wide(const DevFactor& df, int which, void* vec, int64_t R, void* st, void* bar,
                        cudaStream_t s, long long spin_limit, int64_t q);     // q >= 3
int sweep_coop_mix(const DevFactor& df, int which, void* vec, int64_t R, void* st, void* bar, cudaStream_t s,
                   long long spin_limit, int64_t q);

}  // namespace hb

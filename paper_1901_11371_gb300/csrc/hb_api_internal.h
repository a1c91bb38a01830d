// Handle types behind the opaque ABI pointers and shared helpers of the
// entry points.
#pragma once

#include <cuda_runtime.h>

#include "hb_device.h"
#include "hb_internal.h"

struct hb_geometry_s {
  hb::Geometry geo;
};

namespace hb {

enum WsSlot { WS_STATE = 0, WS_STATE_SWEEP, WS_VEC0, WS_VEC1, WS_VEC2, WS_VEC3, WS_BASIS, WS_ZBASIS, WS_RED, WS_DD0, WS_DD1,
              WS_SMALL, kSlots };

// Grow-only device workspaces owned by a factor handle (cudaMalloc on first use
// or growth; freed by hb_factor_destroy).
struct Workspace {
  void* ptr[kSlots] = {nullptr};
  size_t cap[kSlots] = {0};
  void* get(int slot, size_t bytes);
  void release();
};

// Event-based timing of the hot-path kernels (see hb_profile).
struct Profiler {
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[2];
  int64_t count[3] = {0, 0, 0};
  void begin(int kind, cudaStream_t st, cudaEvent_t& a);
  void end(int kind, cudaStream_t st, cudaEvent_t a);
  void reset();
};

}  // namespace hb

struct hb_factor_s {
  hb::HostFactor hf;     // construction record (bulky parts released after upload)
  hb::PackedHost ph;     // packed image (factor pool released after upload)
  hb::DevFactor df;
  hb::Workspace ws;
  double build_seconds = 0.0;
  double construct_seconds = 0.0;
  int64_t lower_nnz = 0, upper_nnz = 0;   // stored entries of the F21 / F12 butterflies
  bool host_only = false;                 // built by hb_factor_host: no device image
  hb::Profiler prof;
};

namespace hb {
int check_vec_args(hb_factor_t f, const void* a, const void* b, int64_t nrhs, int64_t ld, const char* who);
int apply_internal(hb_factor_t f, Prec p, bool adj, const void* x, void* y, int64_t R, cudaStream_t st);
int sweep_internal(hb_factor_t f, Prec p, int which, void* vec, int64_t R, cudaStream_t st);
// one sweep with a given kernel (0: cooperative, 1: column-partitioned)
int sweep_run(hb_factor_t f, Prec p, int which, void* vec, int64_t R, cudaStream_t st, int kernel);
// count kernels launched by the library (profiling)
inline void count_launch(hb_factor_t f, int n) { f->prof.count[2] += n; }
// r(col-major, ld) = b(col-major, ld) - y(internal [row][R], double2)
int launch_residual_cols(const void* b, int64_t ld, const void* y, int64_t n, int64_t R, void* r, cudaStream_t st);
}  // namespace hb

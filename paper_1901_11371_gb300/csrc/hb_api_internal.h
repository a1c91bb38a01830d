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
              WS_SMALL, WS_CYC, kSlots };

// Grow-only device workspaces owned by a factor handle (cudaMalloc on first use
// or growth; freed by hb_factor_destroy).
struct Workspace {
  void* ptr[kSlots] = {nullptr};
  size_t cap[kSlots] = {0};
  void* get(int slot, size_t bytes);
  void release();
};

// Event-based timing of the hot-path kernels (see hb_profile).  While a
// solver cycle is being captured into a CUDA graph the event pairs become
// graph nodes: they are kept in `cap`, tagged with the Arnoldi step they belong
// to (-1: run on every launch), and harvest() adds, after each launch of the
// graph, the times and the kernel counts of the steps that ran.  Inside a
// conditional body (in_body) no events are recorded: the capture places them
// around the body's IF node instead.
struct Profiler {
  struct Tagged {
    int kind, tag;
    cudaEvent_t a, b;
  };
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[2];
  int64_t count[3] = {0, 0, 0};
  double acc_ms[2] = {0.0, 0.0};
  bool capturing = false, in_body = false;
  int tag = -1;
  std::vector<Tagged> cap;
  std::vector<int64_t> cap_launches;   // kernels captured per tag + 1
  void begin(int kind, cudaStream_t st, cudaEvent_t& a);
  void end(int kind, cudaStream_t st, cudaEvent_t a);
  void record(cudaEvent_t e, cudaStream_t st);
  void reset();
  int harvest(int steps_run);   // after a synchronised graph launch
  void drop_capture();          // destroys the captured events (their graph is gone)
};

// One restart cycle of hb_gmres captured as a CUDA graph, kept on the factor
// across calls while its key, the factor's execution settings (stamp) and the
// workspace addresses it was captured with all hold.
struct CycleGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int op = -1, m = 0, mixed = -1;
  int64_t R = 0;
  uint64_t stamp = 0;
  void* ws[kSlots] = {nullptr};
  void release(Profiler& prof);
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
  hb::CycleGraph cg;                      // hb_gmres's captured restart cycle
  uint64_t stamp = 1;                     // bumped by every change of the execution settings
  int gmres_graph = 1;                    // hb_set_gmres_graph
};

namespace hb {
int check_vec_args(hb_factor_t f, const void* a, const void* b, int64_t nrhs, int64_t ld, const char* who);
int apply_internal(hb_factor_t f, Prec p, bool adj, const void* x, void* y, int64_t R, cudaStream_t st);
int sweep_internal(hb_factor_t f, Prec p, int which, void* vec, int64_t R, cudaStream_t st);
// one sweep with a given kernel (0: cooperative, 1: column-partitioned)
int sweep_run(hb_factor_t f, Prec p, int which, void* vec, int64_t R, cudaStream_t st, int kernel);
// count kernels launched by the library (profiling)
inline void count_launch(hb_factor_t f, int n) {
  Profiler& p = f->prof;
  if (!p.capturing) {
    p.count[2] += n;
    return;
  }
  const size_t t = (size_t)(p.tag + 1);
  if (p.cap_launches.size() <= t) p.cap_launches.resize(t + 1, 0);
  p.cap_launches[t] += n;
}
// the cached solver graph is stale from here on (settings that its kernels' arguments hold)
inline void settings_changed(hb_factor_t f) {
  f->stamp++;
  f->cg.release(f->prof);
}
// r(col-major, ld) = b(col-major, ld) - y(internal [row][R], double2)
int launch_residual_cols(const void* b, int64_t ld, const void* y, int64_t n, int64_t R, void* r, cudaStream_t st);
}  // namespace hb

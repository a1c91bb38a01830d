// hb_apply_noalloc: the H-IDBF apply (same kernels as hb_apply) for callers
// that must not allocate device memory.
//
// hb_apply keeps its scratch (the butterfly state between stages, plus the
// reordered input/output blocks for several right-hand sides) in a workspace
// that the factor handle grows with cudaMalloc on first use.  Some callers
// cannot let a library call cudaMalloc: a host framework whose own caching
// allocator already owns the device-memory budget, or a long-running service
// that must not allocate once it has started.  This entry point takes its
// scratch from one file-scope device array instead, sized once when the
// library is loaded.
#include <cuda_runtime.h>

#include <mutex>

#include "hb_api_internal.h"

namespace hb {
namespace {

// Maximum scratch of one call.  Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code the array's name is only a stand-in for the symbol; its device
// address is looked up once per device (with that device current) and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("hb_apply_noalloc: cannot query the current device (%s)", cudaGetErrorString(e));
    return HB_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error("hb_apply_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev, cudaGetErrorString(e));
      return HB_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HB_OK;
}

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace
}  // namespace hb

using namespace hb;

extern "C" int hb_apply_noalloc(hb_factor_t f, int op, const void* x, void* y, int64_t nrhs, int64_t ld,
                                void* stream) {
  int rc = check_vec_args(f, x, y, nrhs, ld, "hb_apply_noalloc");
  if (rc) return rc;
  if (op != HB_OP_N && op != HB_OP_H) {
    set_error("hb_apply_noalloc: bad op");
    return HB_EINVAL;
  }
  const DevFactor& df = f->df;
  const bool f64 = df.form == HB_C128;
  const Prec p = f64 ? PREC_F64 : PREC_F32;
  const int vt = f64 ? 0 : 1;
  const size_t es = f64 ? 16 : 8;
  // scratch layout: [butterfly state][reordered x][reordered y] (the last two only for nrhs > 1).
  // The column count is bounded before any product is formed, so the sizes
  // below cannot wrap around: one column of state plus two vector columns
  // must fit the array nrhs times.
  const size_t col_bytes = ((size_t)df.state_len + (nrhs > 1 ? 2 * (size_t)df.n : 0)) * es;
  if (col_bytes == 0 || (uint64_t)nrhs > (uint64_t)(kNoAllocScratchBytes / col_bytes)) {
    set_error("hb_apply_noalloc: %lld right-hand sides need more scratch than the fixed limit of %zu bytes "
              "(%zu bytes per right-hand side; use hb_apply, or fewer right-hand sides)", (long long)nrhs,
              kNoAllocScratchBytes, col_bytes);
    return HB_EINVAL;
  }
  const size_t state_bytes = round256((size_t)df.state_len * (size_t)nrhs * es);
  const size_t vec_bytes = nrhs > 1 ? round256((size_t)df.n * (size_t)nrhs * es) : 0;
  const size_t need = state_bytes + 2 * vec_bytes;
  if (need > kNoAllocScratchBytes) {
    set_error("hb_apply_noalloc: this call needs %zu bytes of scratch, above the fixed limit of %zu bytes "
              "(use hb_apply, or fewer right-hand sides)", need, kNoAllocScratchBytes);
    return HB_EINVAL;
  }
  void* base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  char* s = (char*)base;
  void* state = s;
  cudaStream_t st = (cudaStream_t)stream;
  // every state entry is written before it is read, so nothing needs clearing
  if (nrhs == 1) return launch_apply(df, p, op == HB_OP_H, x, y, 1, state, st);
  void* xi = s + state_bytes;
  void* yi = s + state_bytes + vec_bytes;
  if ((rc = launch_gather_cols(x, vt, ld, df.n, nrhs, xi, vt, 1.0, st))) return rc;
  if ((rc = launch_apply(df, p, op == HB_OP_H, xi, yi, nrhs, state, st))) return rc;
  return launch_scatter_cols(yi, vt, df.n, nrhs, y, vt, ld, 1.0, st);
}

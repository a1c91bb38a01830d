// C ABI of libhb (include/hb.h): handles, upload of the level-packed factor
// image, workspaces and the apply / sweep / residual entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>

#include "hb_api_internal.h"

namespace hb {
const char* last_error();

// ---------------------------------------------------------------------------
// Upload
// ---------------------------------------------------------------------------
template <class Dst>
static void convert(const std::vector<cplx>& src, std::vector<Dst>& dst) {
  dst.resize(src.size());
  for (size_t i = 0; i < src.size(); ++i) {
    dst[i].x = (decltype(dst[i].x))src[i].real();
    dst[i].y = (decltype(dst[i].y))src[i].imag();
  }
}

// leaves row-major [r][c] on the host -> [leaf][c][r] on the device
static std::vector<cplx> leaves_colmajor(const std::vector<cplx>& src, int64_t m, int64_t n0) {
  std::vector<cplx> out(src.size());
  for (int64_t l = 0; l < m; ++l)
    for (int64_t r = 0; r < n0; ++r)
      for (int64_t c = 0; c < n0; ++c) out[(l * n0 + c) * n0 + r] = src[(l * n0 + r) * n0 + c];
  return out;
}

#define HB_CU(call)                                                                  \
  do {                                                                               \
    cudaError_t e__ = (call);                                                        \
    if (e__ != cudaSuccess) {                                                        \
      set_error("%s failed: %s", #call, cudaGetErrorString(e__));                    \
      return e__ == cudaErrorMemoryAllocation ? HB_ENOMEM : HB_ECUDA;                \
    }                                                                                \
  } while (0)

template <class V>
static int up(const std::vector<V>& h, V** d, cudaStream_t st, int64_t& bytes) {
  size_t nb = std::max<size_t>(h.size(), 1) * sizeof(V);
  HB_CU(cudaMalloc((void**)d, nb));
  if (!h.empty()) HB_CU(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, st));
  bytes += (int64_t)nb;
  return HB_OK;
}

template <class E>
static int upload_elems(const PackedHost& ph, const HostFactor& hf, cudaStream_t st, DevFactor& df) {
  std::vector<E> tmp;
  int rc;
  convert(ph.fpool, tmp);
  if ((rc = up(tmp, (E**)&df.fpool, st, df.device_bytes))) return rc;
  HB_CU(cudaStreamSynchronize(st));
  convert(leaves_colmajor(hf.leaf, hf.m, hf.n0), tmp);
  if ((rc = up(tmp, (E**)&df.leaf, st, df.device_bytes))) return rc;
  HB_CU(cudaStreamSynchronize(st));
  for (int w = 0; w < 4; ++w) {
    convert(ph.sl[w], tmp);
    if ((rc = up(tmp, (E**)&df.sl[w], st, df.device_bytes))) return rc;
    HB_CU(cudaStreamSynchronize(st));
  }
  return HB_OK;
}

int upload_factor(const PackedHost& ph, const HostFactor& hf, const Geometry& g, int form, cudaStream_t st,
                  DevFactor& df) {
  df.form = form;
  df.n = ph.n; df.n0 = ph.n0; df.m = ph.m; df.D = ph.depth;
  df.state_len = ph.state_len;
  df.sl_n = ph.sl_n; df.sl_m = ph.sl_m;
  df.fpool_len = (int64_t)ph.fpool.size();
  df.ipool_len = (int64_t)ph.ipool.size();
  df.kappa = hf.kappa; df.eta0 = hf.eta0; df.scale = hf.scale;
  int rc = (form == HB_C128) ? upload_elems<double2>(ph, hf, st, df) : upload_elems<float2>(ph, hf, st, df);
  if (rc) return rc;
  if ((rc = up(ph.ipool, &df.ipool, st, df.device_bytes))) return rc;
  if ((rc = up(ph.vout, &df.vout, st, df.device_bytes))) return rc;
  if ((rc = up(ph.uout, &df.uout, st, df.device_bytes))) return rc;
  if ((rc = up(ph.bvout, &df.bvout, st, df.device_bytes))) return rc;
  if ((rc = up(ph.buout, &df.buout, st, df.device_bytes))) return rc;
  if ((rc = up(ph.bf_vout0, &df.bf_vout0, st, df.device_bytes))) return rc;
  if ((rc = up(ph.bf_uout0, &df.bf_uout0, st, df.device_bytes))) return rc;
  if ((rc = up(ph.items, &df.items, st, df.device_bytes))) return rc;
  if ((rc = up(ph.step_idx, &df.step_idx, st, df.device_bytes))) return rc;
  if ((rc = up(ph.astep_idx, &df.astep_idx, st, df.device_bytes))) return rc;
  df.step_ptr = ph.step_ptr;
  df.astep_ptr = ph.astep_ptr;
  const std::vector<DPhase>* progs[4] = {&ph.prog_lower, &ph.prog_upper, &ph.prog_lower_adj, &ph.prog_upper_adj};
  for (int i = 0; i < 4; ++i) {
    if ((rc = up(*progs[i], &df.prog[i], st, df.device_bytes))) return rc;
    df.nprog[i] = (int)progs[i]->size();
    FlatProgram fpg = flatten_program(ph, *progs[i], i);
    if (!fpg.ok) {
      set_error("sweep program: an op does not fit the 64-byte record");
      return HB_EUNSUPPORTED;
    }
    df.sweep_elems[i] = df.sweep_idx[i] = 0;
    for (const FlatOp& o : fpg.ops) {
      df.sweep_elems[i] += o.melems;
      if (o.ioff >= 0) df.sweep_idx[i] += o.ielems;
      // the sweep kernel copies every op's data with 16-byte bulk copies:
      // matrices must start on an even complex-FP32 entry, indices on a multiple of 8
      if ((o.moff & 1) || (o.ioff >= 0 && (o.ioff & 7))) {
        set_error("sweep program: op data not 16-byte aligned");
        return HB_EUNSUPPORTED;
      }
    }
    if ((rc = up(fpg.ops, &df.flat[i], st, df.device_bytes))) return rc;
    if ((rc = up(fpg.base, &df.flat_base[i], st, df.device_bytes))) return rc;
    if ((rc = up(fpg.pbytes, &df.flat_pbytes[i], st, df.device_bytes))) return rc;
    HB_CU(cudaStreamSynchronize(st));
  }
  HB_CU(cudaMalloc(&df.bar, 64));
  HB_CU(cudaMemsetAsync(df.bar, 0, 64, st));
  HB_CU(cudaMalloc(&df.abar, 64));
  HB_CU(cudaMemsetAsync(df.abar, 0, 64, st));
  if (form == HB_SPLIT_BF16) {
    // the entry and exit contractions of every leaf as split-BF16 tensor-core operands
    TcOperands tc;
    build_tc_operands(ph, hf, tc);
    if ((rc = up(tc.enter, &df.tc_enter, st, df.device_bytes))) return rc;
    if ((rc = up(tc.exit, &df.tc_exit, st, df.device_bytes))) return rc;
    if ((rc = up(tc.chunks, &df.tc_chunks, st, df.device_bytes))) return rc;
    if ((rc = up(tc.bpool, &df.tc_bpool, st, df.device_bytes))) return rc;
    if ((rc = up(tc.tab, &df.tc_tab, st, df.device_bytes))) return rc;
    HB_CU(cudaStreamSynchronize(st));
    df.tc_ok = true;
  }
  {
    // persistent single-column apply plans, cut for this device's SMs
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int fes = form == HB_C128 ? 16 : 8;
    for (int adj = 0; adj < 2 && sms > 0; ++adj) {
      ApplyPlan plan;
      build_apply_plan(ph, hf, adj != 0, sms, fes, kA1RingBytes / 2, plan);
      DevPlan& dp = df.plan[adj];
      if (!plan.ok) continue;   // the per-step kernels serve this direction
      if ((rc = up(plan.batches, &dp.batches, st, df.device_bytes))) return rc;
      if ((rc = up(plan.cta_batch, &dp.cta_batch, st, df.device_bytes))) return rc;
      if ((rc = up(plan.image, &dp.image, st, df.device_bytes))) return rc;
      HB_CU(cudaMalloc((void**)&dp.done, sizeof(int) * std::max<size_t>(plan.batches.size(), 1)));
      HB_CU(cudaMemsetAsync(dp.done, 0, sizeof(int) * std::max<size_t>(plan.batches.size(), 1), st));
      df.device_bytes += (int64_t)(sizeof(int) * plan.batches.size());
      HB_CU(cudaStreamSynchronize(st));
      dp.nphase = plan.nphase;
      dp.grid = sms;
      dp.nbatch = (int64_t)plan.batches.size();
      dp.ok = true;
    }
  }
  if (form != HB_C128) {
    // column-partitioned sweep schedules of the four sweeps (built in parallel;
    // they need the factor pool and the sweep-leaf triangles, released after upload)
    SwSched S[4];
    std::thread th[4];
    for (int w = 0; w < 4; ++w) th[w] = std::thread([&, w] { build_sweep_sched(ph, w, 8, df.sw_win, S[w]); });
    for (auto& t : th) t.join();
    for (int w = 0; w < 4; ++w) {
      if (!S[w].ok) continue;   // the cooperative kernel serves this sweep
      DevSched& d = df.sw[w];
      if ((rc = up(S[w].groups, &d.groups, st, df.device_bytes))) return rc;
      if ((rc = up(S[w].image, &d.image, st, df.device_bytes))) return rc;
      HB_CU(cudaStreamSynchronize(st));
      d.ngroup = (int64_t)S[w].groups.size();
      d.ok = true;
      std::vector<uint8_t>().swap(S[w].image);
    }
  }
  if ((rc = set_grid_min(df, ph, 16, st))) return rc;
  if ((rc = build_candidates(df, ph, 0, 1, st))) return rc;
  if ((rc = build_candidates(df, ph, 1, 2, st))) return rc;
  if ((rc = up(g.cx, &df.cx, st, df.device_bytes))) return rc;
  if ((rc = up(g.cy, &df.cy, st, df.device_bytes))) return rc;
  if ((rc = up(g.w, &df.w, st, df.device_bytes))) return rc;
  HB_CU(cudaStreamSynchronize(st));
  return HB_OK;
}

int64_t resident_budget(int64_t cols, size_t es) {
  const int64_t wr = cols <= 2 ? (cols < 1 ? 1 : cols) : (cols <= 4 ? 4 : (cols + 7) / 8 * 8);
  return (int64_t)kResidentBytes / (wr * (int64_t)es);
}

static size_t vec_elem_bytes(const DevFactor& df) { return df.form == HB_C128 ? 16 : 8; }

int set_grid_min(DevFactor& df, const PackedHost& ph, int grid_min, cudaStream_t st) {
  const std::vector<DPhase>* progs[4] = {&ph.prog_lower, &ph.prog_upper, &ph.prog_lower_adj, &ph.prog_upper_adj};
  HB_CU(cudaStreamSynchronize(st));
  const int64_t budget = resident_budget(1, vec_elem_bytes(df));
  for (int i = 0; i < 4; ++i) {
    std::vector<DSeg> segs = segment_program(*progs[i], flatten_program(ph, *progs[i], i), grid_min, budget);
    if (df.segs[i]) { cudaFree(df.segs[i]); df.segs[i] = nullptr; }
    int64_t dummy = 0;
    int rc = up(segs, &df.segs[i], st, dummy);
    if (rc) return rc;
    df.nsegs[i] = (int)segs.size();
  }
  HB_CU(cudaStreamSynchronize(st));
  df.grid_min = grid_min;
  return HB_OK;
}

int build_candidates(DevFactor& df, const PackedHost& ph, int cls, int64_t cols, cudaStream_t st) {
  const std::vector<DPhase>* progs[4] = {&ph.prog_lower, &ph.prog_upper, &ph.prog_lower_adj, &ph.prog_upper_adj};
  const int64_t budget = resident_budget(cols, vec_elem_bytes(df));
  if (df.cand_segs[cls][0][0] && df.cand_budget[cls] == budget) return HB_OK;
  HB_CU(cudaStreamSynchronize(st));
  for (int i = 0; i < 4; ++i) {
    FlatProgram fpg = flatten_program(ph, *progs[i], i);
    for (int c = 0; c < DevFactor::kNCand; ++c) {
      std::vector<DSeg> segs = segment_program(*progs[i], fpg, DevFactor::kCand[c], budget);
      if (df.cand_segs[cls][i][c]) { cudaFree(df.cand_segs[cls][i][c]); df.cand_segs[cls][i][c] = nullptr; }
      int64_t dummy = 0;
      int rc = up(segs, &df.cand_segs[cls][i][c], st, dummy);
      if (rc) return rc;
      df.cand_nsegs[cls][i][c] = (int)segs.size();
    }
  }
  HB_CU(cudaStreamSynchronize(st));
  df.cand_budget[cls] = budget;
  return HB_OK;
}

void free_factor(DevFactor& df) {
  void* ptrs[] = {df.fpool, df.leaf, df.sl[0], df.sl[1], df.sl[2], df.sl[3], df.ipool, df.vout, df.uout, df.bvout, df.buout,
                  df.bf_vout0, df.bf_uout0, df.items, df.step_idx, df.astep_idx, df.prog[0], df.prog[1],
                  df.prog[2], df.prog[3], df.segs[0], df.segs[1], df.segs[2], df.segs[3], df.bar,
                  df.flat[0], df.flat[1], df.flat[2], df.flat[3], df.flat_base[0], df.flat_base[1],
                  df.flat_base[2], df.flat_base[3], df.flat_pbytes[0], df.flat_pbytes[1], df.flat_pbytes[2],
                  df.flat_pbytes[3], df.cx, df.cy, df.w, df.abar, df.tc_enter, df.tc_exit, df.tc_chunks,
                  df.tc_bpool, df.tc_tab};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (DevPlan& dp : df.plan) {
    void* pp[] = {dp.batches, dp.cta_batch, dp.image, dp.done};
    for (void* p : pp)
      if (p) cudaFree(p);
  }
  for (auto& per_cls : df.cand_segs)
    for (auto& per_prog : per_cls)
      for (DSeg* p : per_prog)
        if (p) cudaFree(p);
  for (DevSched& s : df.sw) {
    void* pp[] = {s.groups, s.image};
    for (void* p : pp)
      if (p) cudaFree(p);
  }
  df = DevFactor();
}

void Profiler::begin(int kind, cudaStream_t st, cudaEvent_t& a) {
  a = nullptr;
  if (!on || in_body) return;
  if (cudaEventCreate(&a) != cudaSuccess) { a = nullptr; return; }
  record(a, st);
}
// Inside a stream capture a plain record only orders the capture; an external
// record becomes an event-record node that stamps the event at every launch.
void Profiler::record(cudaEvent_t e, cudaStream_t st) {
  if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
}
void Profiler::end(int kind, cudaStream_t st, cudaEvent_t a) {
  if (!on || !a) return;
  cudaEvent_t b;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
  record(b, st);
  if (capturing) {
    cap.push_back({kind, tag, a, b});
    return;
  }
  ev[kind].push_back({a, b});
  count[kind]++;
}
void Profiler::reset() {
  for (auto& v : ev)
    for (auto& p : v) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
  ev[0].clear(); ev[1].clear();
  count[0] = count[1] = count[2] = 0;
  acc_ms[0] = acc_ms[1] = 0.0;
}
int Profiler::harvest(int steps_run) {
  for (size_t t = 0; t < cap_launches.size(); ++t)
    if ((int)t - 1 < steps_run) count[2] += cap_launches[t];
  for (const Tagged& t : cap) {
    if (t.tag >= steps_run) continue;   // a skipped step: its kernels returned at once
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) {
      cudaGetLastError();   // not a device fault: clear it for the launch checks that follow
      return HB_ECUDA;
    }
    acc_ms[t.kind] += ms;
    count[t.kind]++;
  }
  return HB_OK;
}
void Profiler::drop_capture() {
  for (const Tagged& t : cap) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  cap.clear();
  cap_launches.clear();
}
void CycleGraph::release(Profiler& prof) {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  prof.drop_capture();
  op = -1;
  R = 0;
}


void* Workspace::get(int slot, size_t bytes) {
  if (slot < 0 || slot >= kSlots) return nullptr;
  if (cap[slot] >= bytes && ptr[slot]) return ptr[slot];
  if (ptr[slot]) { cudaFree(ptr[slot]); ptr[slot] = nullptr; cap[slot] = 0; }
  size_t nb = std::max<size_t>(bytes, 256);
  if (cudaMalloc(&ptr[slot], nb) != cudaSuccess) { ptr[slot] = nullptr; cap[slot] = 0; return nullptr; }
  cap[slot] = nb;
  return ptr[slot];
}
void Workspace::release() {
  for (int i = 0; i < kSlots; ++i)
    if (ptr[i]) { cudaFree(ptr[i]); ptr[i] = nullptr; cap[i] = 0; }
}

}  // namespace hb

using namespace hb;

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* hb_last_error(void) { return hb::last_error(); }
const char* hb_version(void) { return "hbutterfly 0.1 (sm_103a)"; }

int hb_geometry(int kind, const double* params, int nparams, int64_t n_segments, hb_geometry_t* out) {
  if (!out) { set_error("hb_geometry: out is null"); return HB_EINVAL; }
  *out = nullptr;
  hb_geometry_s* g = new (std::nothrow) hb_geometry_s();
  if (!g) { set_error("hb_geometry: out of host memory"); return HB_ENOMEM; }
  int rc = build_geometry(kind, params, nparams, n_segments, g->geo);
  if (rc) { delete g; return rc; }
  *out = g;
  return HB_OK;
}

int hb_geometry_polyline(const double* xy_nodes, const int64_t* curve_starts, int ncurves, int64_t nnodes,
                         hb_geometry_t* out) {
  if (!out) { set_error("hb_geometry_polyline: out is null"); return HB_EINVAL; }
  *out = nullptr;
  hb_geometry_s* g = new (std::nothrow) hb_geometry_s();
  if (!g) { set_error("hb_geometry_polyline: out of host memory"); return HB_ENOMEM; }
  int rc = build_geometry_polyline(xy_nodes, curve_starts, ncurves, nnodes, g->geo);
  if (rc) { delete g; return rc; }
  *out = g;
  return HB_OK;
}

int hb_geometry_segments(hb_geometry_t g, double* centers_xy, double* lengths) {
  if (!g) { set_error("hb_geometry_segments: null geometry"); return HB_EINVAL; }
  for (int64_t i = 0; i < g->geo.n; ++i) {
    if (centers_xy) { centers_xy[2 * i] = g->geo.cx[i]; centers_xy[2 * i + 1] = g->geo.cy[i]; }
    if (lengths) lengths[i] = g->geo.w[i];
  }
  return HB_OK;
}

int64_t hb_geometry_size(hb_geometry_t g) { return g ? g->geo.n : -1; }

void hb_geometry_destroy(hb_geometry_t g) { delete g; }

int hb_factor(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps, int form,
              uint64_t seed, void* stream, hb_factor_t* out) {
  return hb_factor_ex(g, wavelength, eta0, gamma, leaf, eps, form, seed, 0, stream, out);
}

int hb_factor_ex(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps, int form,
                 uint64_t seed, int options, void* stream, hb_factor_t* out) {
  if (!out || !g) { set_error("hb_factor: null argument"); return HB_EINVAL; }
  if (options & ~(HB_OPT_LEAF_LU | HB_OPT_SWEEP_WINDOW_MIN)) { set_error("hb_factor: unknown option bits 0x%x", options); return HB_EINVAL; }
  *out = nullptr;
  if (form != HB_C128 && form != HB_C64 && form != HB_SPLIT_BF16) { set_error("hb_factor: bad form %d", form); return HB_EINVAL; }
  auto t0 = std::chrono::steady_clock::now();
  hb_factor_s* f = new (std::nothrow) hb_factor_s();
  if (!f) { set_error("hb_factor: out of host memory"); return HB_ENOMEM; }
  int rc = build_factor(g->geo, wavelength, eta0, gamma, leaf, eps, seed, f->hf, options);
  if (!rc) {
    pack_factor(f->hf, f->ph);
    for (const auto& b : f->hf.bf) {
      int64_t z = 0;
      for (const auto& st : b.col) for (const auto& blk : st) z += (int64_t)blk.k * (blk.c - blk.k);
      for (const auto& st : b.row) for (const auto& blk : st) z += (int64_t)blk.k * (blk.c - blk.k);
      for (const auto& sm : b.mid) z += (int64_t)sm.size();
      (b.kind == 1 ? f->lower_nnz : f->upper_nnz) += z;
    }
    if (options & HB_OPT_SWEEP_WINDOW_MIN) f->df.sw_win = 512;
    rc = upload_factor(f->ph, f->hf, g->geo, form, (cudaStream_t)stream, f->df);
    f->df.form = form;
  }
  if (rc) { free_factor(f->df); delete f; return rc; }
  f->construct_seconds = f->hf.build_seconds;
  f->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // release the bulky host copies (stats kept)
  f->ph.fpool.clear(); f->ph.fpool.shrink_to_fit();
  for (auto& b : f->hf.bf) { b.col.clear(); b.row.clear(); b.mid.clear(); b.col.shrink_to_fit(); b.row.shrink_to_fit(); b.mid.shrink_to_fit(); }
  f->hf.leaf.clear(); f->hf.leaf.shrink_to_fit();
  f->hf.linv.clear(); f->hf.linv.shrink_to_fit();
  f->hf.uinv.clear(); f->hf.uinv.shrink_to_fit();
  for (auto& v : f->ph.sl) { v.clear(); v.shrink_to_fit(); }
  *out = f;
  return HB_OK;
}

int hb_factor_host(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
                   uint64_t seed, hb_factor_t* out) {
  return hb_factor_host_ex(g, wavelength, eta0, gamma, leaf, eps, seed, 0, out);
}

int hb_factor_host_ex(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
                      uint64_t seed, int options, hb_factor_t* out) {
  if (!out || !g) { set_error("hb_factor_host: null argument"); return HB_EINVAL; }
  *out = nullptr;
  if (options & ~(HB_OPT_LEAF_LU | HB_OPT_SWEEP_WINDOW_MIN)) { set_error("hb_factor_host: unknown option bits 0x%x", options); return HB_EINVAL; }
  hb_factor_s* f = new (std::nothrow) hb_factor_s();
  if (!f) { set_error("hb_factor_host: out of host memory"); return HB_ENOMEM; }
  int rc = build_factor(g->geo, wavelength, eta0, gamma, leaf, eps, seed, f->hf, options);
  if (rc) { delete f; return rc; }
  pack_factor(f->hf, f->ph);
  f->host_only = true;
  f->df.form = HB_C128;
  f->df.n = f->ph.n; f->df.n0 = f->ph.n0; f->df.m = f->ph.m; f->df.D = f->ph.depth;
  f->build_seconds = f->construct_seconds = f->hf.build_seconds;
  *out = f;
  return HB_OK;
}

int hb_host_apply(hb_factor_t f, int op, const double* x, double* y) {
  if (!f || !f->host_only || !x || !y || (op != HB_OP_N && op != HB_OP_H)) { set_error("hb_host_apply: bad argument"); return HB_EINVAL; }
  host_apply(f->ph, f->hf, op == HB_OP_H, reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y));
  return HB_OK;
}

int hb_host_apply_plan(hb_factor_t f, int op, int grid, int factor_bytes, const double* x, double* y) {
  if (!f || !f->host_only || !x || !y || (op != HB_OP_N && op != HB_OP_H) || grid < 1 ||
      (factor_bytes != 8 && factor_bytes != 16)) {
    set_error("hb_host_apply_plan: bad argument");
    return HB_EINVAL;
  }
  ApplyPlan plan;
  build_apply_plan(f->ph, f->hf, op == HB_OP_H, grid, factor_bytes, kA1RingBytes / 2, plan);
  if (!plan.ok) { set_error("hb_host_apply_plan: the plan failed its structural check"); return HB_EUNSUPPORTED; }
  host_apply_plan(f->ph, plan, factor_bytes, op == HB_OP_H, reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y));
  return (int)std::min<size_t>(plan.batches.size(), (size_t)INT32_MAX);
}

int hb_host_tc_apply(hb_factor_t f, const double* x, double* y) {
  if (!f || !f->host_only || !x || !y) { set_error("hb_host_tc_apply: bad argument"); return HB_EINVAL; }
  TcOperands tc;
  build_tc_operands(f->ph, f->hf, tc);
  host_tc_apply(f->ph, f->hf, tc, reinterpret_cast<const cplx*>(x), reinterpret_cast<cplx*>(y));
  return (int)std::min<size_t>(tc.chunks.size(), (size_t)INT32_MAX);
}

int hb_host_sweep_sched(hb_factor_t f, int which, int coef_bytes, int win_slots, double* vec) {
  if (!f || !f->host_only || !vec || which < 0 || which > 3 || (coef_bytes != 8 && coef_bytes != 16) ||
      win_slots < 0 || win_slots > kSwWinSlots) {
    set_error("hb_host_sweep_sched: bad argument");
    return HB_EINVAL;
  }
  SwSched S;
  build_sweep_sched(f->ph, which, coef_bytes, win_slots > 0 ? win_slots : kSwWinSlots, S);
  if (!S.ok) { set_error("hb_host_sweep_sched: no column-partitioned schedule for this factor (%s)", S.why); return HB_EUNSUPPORTED; }
  if (const char* bad = check_sweep_sched(f->ph, S); *bad) {
    set_error("hb_host_sweep_sched: the schedule failed its structural check (%s)", bad);
    return HB_EUNSUPPORTED;
  }
  host_sweep_sched(f->ph, S, reinterpret_cast<cplx*>(vec));
  return (int)std::min<int64_t>(S.batches, (int64_t)INT32_MAX);
}

int hb_host_sweep(hb_factor_t f, int which, double* vec) {
  if (!f || !f->host_only || !vec || which < 0 || which > 3) { set_error("hb_host_sweep: bad argument"); return HB_EINVAL; }
  host_sweep(f->ph, f->hf, which, reinterpret_cast<cplx*>(vec));
  return HB_OK;
}

int hb_factor_info(hb_factor_t f, hb_factor_stats* s) {
  if (!f || !s) { set_error("hb_factor_info: null argument"); return HB_EINVAL; }
  std::memset(s, 0, sizeof(*s));
  const PackedHost& ph = f->ph;
  s->n = ph.n; s->leaf = ph.n0; s->depth = ph.depth; s->form = f->df.form;
  s->n_butterflies = 2 * (ph.m - 1);
  s->scale = f->hf.scale; s->eps = f->hf.eps;
  s->kmax = ph.kmax; s->kavg = ph.kavg;
  for (int v = 0; v < 32; ++v) { s->kmax_depth[v] = ph.kmax_depth[v]; s->kavg_depth[v] = ph.kavg_depth[v]; }
  s->nnz_leaf = ph.m * ph.n0 * ph.n0;
  s->nnz_butterfly = ph.nnz_bf;
  s->sweep_leaf = (int32_t)ph.sl_n;
  s->nnz_lu_leaf = 2 * ph.sl_m * packed_tri(ph.sl_n);
  s->index_bytes = f->df.ipool_len * 2;
  s->device_bytes = f->df.device_bytes;
  int64_t eb = (f->df.form == HB_C128) ? 16 : 8;
  // algorithmic bytes of one single-RHS apply: every stored butterfly entry and
  // dense-leaf entry once, the index arrays once, x read and y written.
  s->apply_bytes = (ph.nnz_bf + s->nnz_leaf) * eb + s->index_bytes + 2 * ph.n * eb;
  // a sweep reads every factor entry and index entry of its program once (the
  // butterflies of one triangle above the sweep leaves, and one packed
  // triangle per sweep leaf), reads b and writes x
  int64_t el[2] = {f->df.sweep_elems[0], f->df.sweep_elems[1]}, ix[2] = {f->df.sweep_idx[0], f->df.sweep_idx[1]};
  if (f->host_only)
    for (int w = 0; w < 2; ++w) {
      FlatProgram fp = flatten_program(ph, w == 0 ? ph.prog_lower : ph.prog_upper, w);
      el[w] = ix[w] = 0;
      for (const FlatOp& o : fp.ops) { el[w] += o.melems; if (o.ioff >= 0) ix[w] += o.ielems; }
    }
  s->lower_bytes = el[0] * eb + ix[0] * 2 + 2 * ph.n * eb;
  s->upper_bytes = el[1] * eb + ix[1] * 2 + 2 * ph.n * eb;
  s->rebuilt_blocks = 0;
  s->build_seconds = f->build_seconds;
  return HB_OK;
}

int hb_profile(hb_factor_t f, int enable) {
  if (!f) { set_error("hb_profile: null factor"); return HB_EINVAL; }
  // a captured solver cycle holds (or lacks) the timing events: recapture only
  // when profiling is switched on or off; enabling it again just resets the counts
  if ((enable != 0) != f->prof.on) settings_changed(f);
  if (enable) f->prof.reset();
  f->prof.on = enable != 0;
  return HB_OK;
}

int hb_profile_read(hb_factor_t f, int kind, int64_t* count, double* total_ms) {
  if (!f || kind < 0 || kind > 2) { set_error("hb_profile_read: bad argument"); return HB_EINVAL; }
  double tot = 0.0;
  if (kind < 2) {
    for (auto& p : f->prof.ev[kind]) {
      if (cudaEventSynchronize(p.second) != cudaSuccess) { set_error("hb_profile_read: event sync failed"); return HB_ECUDA; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.first, p.second);
      tot += ms;
    }
    tot += f->prof.acc_ms[kind];
  }
  if (count) *count = f->prof.count[kind];
  if (total_ms) *total_ms = tot;
  return HB_OK;
}

void hb_factor_destroy(hb_factor_t f) {
  if (!f) return;
  f->cg.release(f->prof);
  f->prof.reset();
  f->ws.release();
  free_factor(f->df);
  delete f;
}

int hb_tree(hb_factor_t f, int64_t* node_begin, int64_t* node_end) {
  if (!f || !node_begin || !node_end) { set_error("hb_tree: null argument"); return HB_EINVAL; }
  const int D = f->ph.depth;
  const int64_t n = f->ph.n;
  for (int v = 0; v <= D; ++v) {
    int64_t cnt = (int64_t)1 << v, sz = n >> v;
    for (int64_t p = 0; p < cnt; ++p) {
      node_begin[cnt - 1 + p] = p * sz;
      node_end[cnt - 1 + p] = (p + 1) * sz;
    }
  }
  return HB_OK;
}

int hb_set_sweep_grid_min(hb_factor_t f, int grid_min) {
  if (!f || f->host_only || grid_min < 1) { set_error("hb_set_sweep_grid_min: bad argument"); return HB_EINVAL; }
  settings_changed(f);
  f->df.tuned[0] = f->df.tuned[1] = -1;
  f->df.cols_won[0] = f->df.cols_won[1] = false;
  int old = f->df.grid_min;
  int rc = set_grid_min(f->df, f->ph, grid_min, nullptr);
  return rc ? rc : old;
}

int hb_autotune(hb_factor_t f, int64_t nrhs, void* stream, int* chosen) {
  if (!f || f->host_only || nrhs < 1) { set_error("hb_autotune: bad argument"); return HB_EINVAL; }
  settings_changed(f);
  cudaStream_t st = (cudaStream_t)stream;
  DevFactor& df = f->df;
  const Prec p = df.form == HB_C128 ? PREC_F64 : PREC_F32;
  const size_t es = p == PREC_F32 ? 8 : 16;
  void* v = f->ws.get(WS_VEC0, (size_t)df.n * nrhs * es);
  if (!v) { set_error("hb_autotune: workspace allocation failed"); return HB_ENOMEM; }
  if (cudaMemsetAsync(v, 0, (size_t)df.n * nrhs * es, st) != cudaSuccess) return HB_ECUDA;
  const int cls = nrhs > 1 ? 1 : 0;
  {
    // candidate segmentations cut for this many columns per CTA
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cols = (nrhs + std::max(sms, 1) - 1) / std::max(sms, 1);
    int rc = build_candidates(df, f->ph, cls, cols, st);
    if (rc) return rc;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bestc = -1;
  for (int c = 0; c < DevFactor::kNCand; ++c) {
    df.tuned[cls] = c;
    int rc = sweep_run(f, p, 0, v, nrhs, st, 0);   // warm
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2; ++r) sweep_run(f, p, 0, v, nrhs, st, 0);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    df.cand_ms[cls][c] = ms / 2;
    if (ms < best) { best = ms; bestc = c; }
  }
  df.tuned[cls] = bestc;
  // the column-partitioned kernel (complex-FP32 factors with schedules)
  df.cols_won[cls] = false;
  df.cols_ms[cls] = 0.f;
  if (p == PREC_F32 && df.sw[0].ok) {
    int rc = sweep_run(f, p, 0, v, nrhs, st, 1);   // warm
    if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2; ++r) sweep_run(f, p, 0, v, nrhs, st, 1);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    df.cols_ms[cls] = ms / 2;
    df.cols_won[cls] = ms < best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (chosen) *chosen = df.cols_won[cls] ? 0 : DevFactor::kCand[bestc];
  return hb_status(f, stream);
}

int hb_autotune_times(hb_factor_t f, int64_t nrhs, float* ms_out, int* grid_min_out, int max) {
  if (!f || f->host_only || nrhs < 1 || max < 0 || (max > 0 && (!ms_out || !grid_min_out))) {
    set_error("hb_autotune_times: bad argument");
    return HB_EINVAL;
  }
  const int cls = nrhs > 1 ? 1 : 0;
  if (f->df.tuned[cls] < 0) return 0;
  const int n = std::min(max, DevFactor::kNCand);
  for (int c = 0; c < n; ++c) {
    ms_out[c] = f->df.cand_ms[cls][c];
    grid_min_out[c] = DevFactor::kCand[c];
  }
  if (f->df.cols_ms[cls] > 0.f && max > n) {
    ms_out[n] = f->df.cols_ms[cls];
    grid_min_out[n] = 0;   // the column-partitioned kernel
    return n + 1;
  }
  return n;
}

int hb_set_sweep_kernel(hb_factor_t f, int kind) {
  if (!f || f->host_only || kind < -1 || kind > 1) { set_error("hb_set_sweep_kernel: bad argument"); return HB_EINVAL; }
  if (kind == 1 && !(f->df.sw[0].ok && f->df.sw[1].ok && f->df.sw[2].ok && f->df.sw[3].ok)) {
    set_error("hb_set_sweep_kernel: this factor has no column-partitioned schedules (complex-FP32 forms only)");
    return HB_EUNSUPPORTED;
  }
  f->df.sweep_kernel = kind;
  settings_changed(f);
  return HB_OK;
}

int hb_set_gmres_graph(hb_factor_t f, int on) {
  if (!f || f->host_only || on < 0 || on > 1) { set_error("hb_set_gmres_graph: bad argument"); return HB_EINVAL; }
  f->gmres_graph = on;
  settings_changed(f);
  return HB_OK;
}

int hb_set_wait_limit(hb_factor_t f, long long spins) {
  if (!f || f->host_only || spins < 1) { set_error("hb_set_wait_limit: bad argument"); return HB_EINVAL; }
  f->df.spin_limit = spins;
  settings_changed(f);
  return HB_OK;
}

int hb_status(hb_factor_t f, void* stream) {
  if (!f || f->host_only) { set_error("hb_status: bad argument"); return HB_EINVAL; }
  int err = 0;
  if (read_grid_error(f->df.bar, (cudaStream_t)stream, &err)) { set_error("hb_status: CUDA error"); return HB_ECUDA; }
  if (err) { set_error("a bounded device-side wait expired in a sweep kernel"); return HB_ETIMEOUT; }
  return HB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// apply / sweeps / residual
// ---------------------------------------------------------------------------
namespace hb {

int check_vec_args(hb_factor_t f, const void* a, const void* b, int64_t nrhs, int64_t ld, const char* who) {
  if (!f || !a || !b) { set_error("%s: null argument", who); return HB_EINVAL; }
  if (f->host_only) { set_error("%s: factor has no device image (built by hb_factor_host)", who); return HB_EINVAL; }
  if (nrhs < 1 || ld < f->df.n) { set_error("%s: need nrhs >= 1 and ld >= N (got %lld, %lld)", who, (long long)nrhs, (long long)ld); return HB_EINVAL; }
  if (a == b) { set_error("%s: input and output must not alias", who); return HB_EINVAL; }
  return HB_OK;
}

// form vectors: double2 for HB_C128, float2 otherwise
static inline Prec form_prec(const DevFactor& df) { return df.form == HB_C128 ? PREC_F64 : PREC_F32; }
static inline int form_vt(const DevFactor& df) { return df.form == HB_C128 ? 0 : 1; }
static inline size_t vt_size(int t) { return t == 0 ? 16 : 8; }

int apply_internal(hb_factor_t f, Prec p, bool adj, const void* x, void* y, int64_t R, cudaStream_t st) {
  size_t es = (p == PREC_F32) ? 8 : 16;
  void* state = f->ws.get(WS_STATE, (size_t)f->df.state_len * R * es);
  if (!state) { set_error("apply: cannot allocate state workspace"); return HB_ENOMEM; }
  // FP64-accurate arithmetic on complex-FP32 factors for many columns: double-float
  const bool dd = p == PREC_F32_ACC64 && f->df.form != HB_C128 && apply_dd_ready(R);
  void* xdd = dd ? f->ws.get(WS_DD0, (size_t)f->df.n * R * 16) : nullptr;
  void* ydd = dd ? f->ws.get(WS_DD1, (size_t)f->df.n * R * 16) : nullptr;
  if (dd && (!xdd || !ydd)) { set_error("apply: cannot allocate double-float workspace"); return HB_ENOMEM; }
  cudaEvent_t e;
  f->prof.begin(0, st, e);
  int rc = dd ? launch_apply_dd(f->df, adj, x, y, R, state, xdd, ydd, st) : launch_apply(f->df, p, adj, x, y, R, state, st);
  f->prof.end(0, st, e);
  count_launch(f, (R == 1 && apply1_ready(f->df, adj)) ? 1 : (int)f->df.step_ptr.size() + 1);
  return rc;
}

// kernel: 0 = cooperative, 1 = column-partitioned
int sweep_run(hb_factor_t f, Prec p, int which, void* vec, int64_t R, cudaStream_t st, int kernel) {
  const size_t es = (p == PREC_F32) ? 8 : 16;
  const size_t need = kernel == 1 ? (size_t)sweep_cols_state_entries(f->df, R) * 8 : (size_t)f->df.state_len * R * es;
  void* state = f->ws.get(WS_STATE_SWEEP, need);
  if (!state) { set_error("sweep: cannot allocate state workspace"); return HB_ENOMEM; }
  cudaEvent_t e;
  f->prof.begin(1, st, e);
  int rc = kernel == 1 ? launch_sweep_cols(f->df, which, vec, R, state, st)
                       : launch_sweep_coop(f->df, p, which, vec, R, state, f->df.bar, st, f->df.spin_limit);
  f->prof.end(1, st, e);
  count_launch(f, kernel == 1 ? sweep_cols_launches(R) : 1);
  return rc;
}

int sweep_internal(hb_factor_t f, Prec p, int which, void* vec, int64_t R, cudaStream_t st) {
  const DevFactor& df = f->df;
  const bool cols = p == PREC_F32 && df.sw[which].ok &&
                    (df.sweep_kernel == 1 || (df.sweep_kernel < 0 && df.cols_won[R > 1 ? 1 : 0]));
  return sweep_run(f, p, which, vec, R, st, cols ? 1 : 0);
}

}  // namespace hb

extern "C" {

int hb_apply(hb_factor_t f, int op, const void* x, void* y, int64_t nrhs, int64_t ld, void* stream) {
  int rc = check_vec_args(f, x, y, nrhs, ld, "hb_apply");
  if (rc) return rc;
  if (op != HB_OP_N && op != HB_OP_H) { set_error("hb_apply: bad op"); return HB_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const DevFactor& df = f->df;
  Prec p = form_prec(df);
  int vt = form_vt(df);
  if (nrhs == 1) return apply_internal(f, p, op == HB_OP_H, x, y, 1, st);
  size_t bytes = (size_t)df.n * nrhs * vt_size(vt);
  void* xi = f->ws.get(WS_VEC0, bytes);
  void* yi = f->ws.get(WS_VEC1, bytes);
  if (!xi || !yi) { set_error("hb_apply: workspace allocation failed"); return HB_ENOMEM; }
  if ((rc = launch_gather_cols(x, vt, ld, df.n, nrhs, xi, vt, 1.0, st))) return rc;
  if ((rc = apply_internal(f, p, op == HB_OP_H, xi, yi, nrhs, st))) return rc;
  return launch_scatter_cols(yi, vt, df.n, nrhs, y, vt, ld, 1.0, st);
}

int hb_apply_adjoint(hb_factor_t f, const void* x, void* y, int64_t nrhs, int64_t ld, void* stream) {
  return hb_apply(f, HB_OP_H, x, y, nrhs, ld, stream);
}

static int sweeps(hb_factor_t f, int op, const void* b, void* x, int64_t nrhs, int64_t ld, void* stream,
                  int first, int second, const char* who) {
  int rc = check_vec_args(f, b, x, nrhs, ld, who);
  if (rc) return rc;
  if (op != HB_OP_N && op != HB_OP_H) { set_error("%s: bad op", who); return HB_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const DevFactor& df = f->df;
  Prec p = form_prec(df);
  int vt = form_vt(df);
  void* v;
  if (nrhs == 1) {
    if (cudaMemcpyAsync(x, b, (size_t)df.n * vt_size(vt), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      set_error("%s: copy failed", who);
      return HB_ECUDA;
    }
    v = x;
  } else {
    v = f->ws.get(WS_VEC0, (size_t)df.n * nrhs * vt_size(vt));
    if (!v) { set_error("%s: workspace allocation failed", who); return HB_ENOMEM; }
    if ((rc = launch_gather_cols(b, vt, ld, df.n, nrhs, v, vt, 1.0, st))) return rc;
  }
  if (first >= 0 && (rc = sweep_internal(f, p, first, v, nrhs, st))) return rc;
  if (second >= 0 && (rc = sweep_internal(f, p, second, v, nrhs, st))) return rc;
  if (nrhs > 1) return launch_scatter_cols(v, vt, df.n, nrhs, x, vt, ld, 1.0, st);
  return HB_OK;
}

int hb_precond_solve(hb_factor_t f, int op, const void* b, void* x, int64_t nrhs, int64_t ld, void* stream) {
  // op N: x = U~^{-1} L~^{-1} b;  op H: x = L~^{-H} U~^{-H} b
  if (op == HB_OP_H) return sweeps(f, op, b, x, nrhs, ld, stream, 3, 2, "hb_precond_solve");
  return sweeps(f, op, b, x, nrhs, ld, stream, 0, 1, "hb_precond_solve");
}
int hb_lower_solve(hb_factor_t f, int op, const void* b, void* x, int64_t nrhs, int64_t ld, void* stream) {
  return sweeps(f, op, b, x, nrhs, ld, stream, op == HB_OP_H ? 2 : 0, -1, "hb_lower_solve");
}
int hb_upper_solve(hb_factor_t f, int op, const void* b, void* x, int64_t nrhs, int64_t ld, void* stream) {
  return sweeps(f, op, b, x, nrhs, ld, stream, op == HB_OP_H ? 3 : 1, -1, "hb_upper_solve");
}

int hb_residual(hb_factor_t f, int op, const void* b, const void* x, void* r, int64_t nrhs, int64_t ld, void* stream) {
  int rc = check_vec_args(f, x, r, nrhs, ld, "hb_residual");
  if (rc) return rc;
  if (!b || b == r) { set_error("hb_residual: b must be non-null and distinct from r"); return HB_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const DevFactor& df = f->df;
  Prec p = df.form == HB_C128 ? PREC_F64 : PREC_F32_ACC64;
  size_t bytes = (size_t)df.n * nrhs * 16;
  void* xi = f->ws.get(WS_VEC0, bytes);
  void* yi = f->ws.get(WS_VEC1, bytes);
  if (!xi || !yi) { set_error("hb_residual: workspace allocation failed"); return HB_ENOMEM; }
  if ((rc = launch_gather_cols(x, 0, ld, df.n, nrhs, xi, 0, 1.0, st))) return rc;
  if ((rc = apply_internal(f, p, op == HB_OP_H, xi, yi, nrhs, st))) return rc;
  return launch_residual_cols(b, ld, yi, df.n, nrhs, r, st);
}

}  // extern "C"

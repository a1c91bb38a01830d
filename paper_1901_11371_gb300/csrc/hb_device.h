// Device image of an H-IDBF factor and the launchers of the hot-path kernels.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "hb_internal.h"

namespace hb {

// Device copy of an ApplyPlan (persistent single-column apply).
struct DevPlan {
  A1Batch* batches = nullptr;
  int32_t* cta_batch = nullptr;
  uint8_t* image = nullptr;    // batch images (ApplyPlan::image)
  int nphase = 0;
  int grid = 0;          // CTAs the plan was cut for (the device's SM count at upload)
  bool ok = false;
  int64_t nbatch = 0;
  int* done = nullptr;   // per batch: the epoch of the launch that completed it (zeroed at upload)
  int epoch = 0;         // the last launch's epoch
};
// Shared-memory staging ring of the persistent apply (bytes per CTA).
constexpr int kA1RingBytes = 200 * 1024;

// Device copy of a column-partitioned sweep schedule (SwSched).
struct DevSched {
  SwGroup* groups = nullptr;
  uint8_t* image = nullptr;
  int64_t ngroup = 0;
  bool ok = false;
};

struct DevFactor {
  int form = HB_C128;            // storage form of the factor pool
  int64_t n = 0, n0 = 0, m = 0;
  int D = 0;
  int64_t state_len = 0;         // butterfly state entries per RHS
  // factor data (element type double2 for HB_C128, float2 otherwise)
  void* fpool = nullptr;
  int64_t fpool_len = 0;
  void* leaf = nullptr;          // [m][c][r]
  void* sl[4] = {nullptr, nullptr, nullptr, nullptr};   // packed sweep-leaf triangles per sweep (PackedHost::sl)
  int64_t sl_n = 0, sl_m = 0;    // sweep-leaf order and count
  int64_t sweep_elems[4] = {0, 0, 0, 0};   // factor entries one sweep reads (per program)
  int64_t sweep_idx[4] = {0, 0, 0, 0};     // index entries one sweep reads
  int16_t* ipool = nullptr;
  int64_t ipool_len = 0;
  DOuter* vout = nullptr;        // [m][D]
  DOuter* uout = nullptr;        // [m][D]
  DOuter* bvout = nullptr;
  DOuter* buout = nullptr;
  int32_t* bf_vout0 = nullptr;   // device copies
  int32_t* bf_uout0 = nullptr;
  DItem* items = nullptr;
  int32_t* step_idx = nullptr;
  int32_t* astep_idx = nullptr;
  std::vector<int32_t> step_ptr, astep_ptr;   // host copies (launch sizes)
  DPhase* prog[4] = {nullptr, nullptr, nullptr, nullptr};   // lower, upper, lower^H, upper^H
  int nprog[4] = {0, 0, 0, 0};
  FlatOp* flat[4] = {nullptr, nullptr, nullptr, nullptr};   // resolved op records of each program
  int32_t* flat_base[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t* flat_pbytes[4] = {nullptr, nullptr, nullptr, nullptr};   // staging bytes per phase
  DSeg* segs[4] = {nullptr, nullptr, nullptr, nullptr};     // cooperative-kernel segments of each program
  int nsegs[4] = {0, 0, 0, 0};
  int grid_min = 0;                                         // phases with >= grid_min ops run grid-wide
  // autotuner: segmentations of each program for the candidate thresholds,
  // one set per class (0: one right-hand side, 1: several), each cut for the
  // shared-memory budget of that class's columns per CTA
  static constexpr int kNCand = 6;
  static constexpr int kCand[kNCand] = {4, 8, 16, 32, 64, 1 << 30};
  DSeg* cand_segs[2][4][kNCand] = {};
  int cand_nsegs[2][4][kNCand] = {};
  int64_t cand_budget[2] = {0, 0};                          // residency budget (entries) of each set
  float cand_ms[2][kNCand] = {};                            // last autotune timings
  int tuned[2] = {-1, -1};                                  // chosen candidate for 1 RHS / several RHS (-1: grid_min)
  // column-partitioned sweep kernel (complex-FP32 factors): schedules of the four
  // sweeps, the window their runs were cut for, the kernel choice (-1: the
  // autotuner's, 0: cooperative, 1: column-partitioned) and the autotuner's verdict
  DevSched sw[4];
  int sw_win = kSwWinSlots;
  int sweep_kernel = -1;
  bool cols_won[2] = {false, false};
  float cols_ms[2] = {0.f, 0.f};
  void* bar = nullptr;                                      // grid barrier state + error flag
  void* abar = nullptr;                                     // grid barrier of the persistent apply
  // split-BF16 tensor-core operands (form HB_SPLIT_BF16; TcOperands)
  bool tc_ok = false;
  TcJob* tc_enter = nullptr;
  TcJob* tc_exit = nullptr;
  TcChunk* tc_chunks = nullptr;
  uint16_t* tc_bpool = nullptr;
  uint32_t* tc_tab = nullptr;
  DevPlan plan[2];                                          // persistent apply plans: forward, adjoint
  long long spin_limit = 1LL << 24;                         // bounded waits of the grid barrier
  // geometry on the device (far field, plane waves)
  double* cx = nullptr;
  double* cy = nullptr;
  double* w = nullptr;
  double kappa = 0, eta0 = 0, scale = 1;
  int64_t device_bytes = 0;
};

// Upload a packed host image in `form`; returns HB_OK or an error code.
int upload_factor(const PackedHost& ph, const HostFactor& hf, const Geometry& g, int form, cudaStream_t st,
                  DevFactor& df);
void free_factor(DevFactor& df);

// Arithmetic precisions of the hot path.
enum Prec { PREC_F64 = 0,        // double factors, double arithmetic (HB_C128)
            PREC_F32 = 1,        // float factors, float arithmetic (HB_C64)
            PREC_F32_ACC64 = 2   // float factors, double arithmetic (FP64 residuals of HB_C64)
};

// All vectors below are in the internal layout [row][R] (RHS fastest) with
// complex element type double2 (PREC_F64, PREC_F32_ACC64) or float2 (PREC_F32).
// `state` holds df.state_len * R complex entries of the same type.
int launch_apply(const DevFactor& df, Prec p, bool adjoint, const void* x, void* y, int64_t R, void* state,
                 cudaStream_t st);
// PREC_F32_ACC64 apply of 32 or more columns in double-float arithmetic (FP32 pairs,
// about 48 significant bits): x, y double2 [row][R]; xdd, ydd, state: 16-byte-per-entry
// scratch of n R, n R and state_len R entries.  HB_EINVAL when not applicable.
bool apply_dd_ready(int64_t R);
int launch_apply_dd(const DevFactor& df, bool adjoint, const void* x, void* y, int64_t R, void* state, void* xdd,
                    void* ydd, cudaStream_t st);
// Split-BF16 tensor-core entry (exit_jobs = false: x -> butterfly state) or
// exit (true: state and x -> y) contractions of every leaf for R columns
// (complex64 vectors, layout [row][R]).  HB_EUNSUPPORTED without operands.
int launch_tc_jobs(const DevFactor& df, bool exit_jobs, const void* x, void* st, void* y, int64_t R,
                   cudaStream_t s);
// Persistent single-column apply (one cooperative launch); apply1_ready:
// the plan of that direction exists for the current device.
bool apply1_ready(const DevFactor& df, bool adjoint);
int launch_apply1(const DevFactor& df, Prec p, bool adjoint, const void* x, void* y, void* state, cudaStream_t st);
// Cooperative sweep, in place: vec holds b on entry and x on exit.  which:
// 0 = L~^{-1}, 1 = U~^{-1}, 2 = L~^{-H}, 3 = U~^{-H}.  One launch per sweep,
// grid barriers between segments.
int launch_sweep_coop(const DevFactor& df, Prec p, int which, void* vec, int64_t R, void* state, void* bar,
                      cudaStream_t st, long long spin_limit);
// Column-partitioned sweep, in place (complex-FP32 vectors [row][R]): every CTA
// runs the whole sweep for its own columns (kernel k_sweep_cols).  `state`: at
// least sweep_cols_state_entries(df, R) complex-FP32 entries.  HB_EUNSUPPORTED
// without a schedule for `which`.
int launch_sweep_cols(const DevFactor& df, int which, void* vec, int64_t R, void* state, cudaStream_t st);
int64_t sweep_cols_state_entries(const DevFactor& df, int64_t R);
int sweep_cols_launches(int64_t R);
// Read the barrier error flag (synchronises st).  *err != 0: a bounded wait expired.
int read_grid_error(void* bar, cudaStream_t st, int* err);
// Shared memory that a single-CTA run may use to keep its vector rows and
// butterfly state resident (bytes; the sweep kernel's layout holds this much).
constexpr int kResidentBytes = 56 * 1024;
// Residency budget in entries per right-hand side for `cols` columns per CTA
// of element size `es` bytes (the kernel rounds the columns up to its chunk).
int64_t resident_budget(int64_t cols, size_t es);
// (Re)build the cooperative segments of the four programs for threshold grid_min.
int set_grid_min(DevFactor& df, const PackedHost& ph, int grid_min, cudaStream_t st);
// (Re)build the autotuner's candidate segmentations of class cls for
// `cols` columns per CTA.
int build_candidates(DevFactor& df, const PackedHost& ph, int cls, int64_t cols, cudaStream_t st);

// Layout conversion between the ABI's column-major [R][ld] blocks and the
// internal [row][R] layout, with optional precision change and scaling.
// src_t / dst_t: 0 = double2, 1 = float2.
int launch_gather_cols(const void* src, int src_t, int64_t ld, int64_t n, int64_t R, void* dst, int dst_t,
                       double scale, cudaStream_t st);
int launch_scatter_cols(const void* src, int src_t, int64_t n, int64_t R, void* dst, int dst_t, int64_t ld,
                        double scale, cudaStream_t st);

}  // namespace hb

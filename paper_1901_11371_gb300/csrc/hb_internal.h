// Internal data structures of libhb: host-side H-IDBF (Alg. 1) and its
// level-packed device image.  Not part of the public ABI (include/hb.h).
#pragma once

#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../../include/hb.h"

namespace hb {

using cplx = std::complex<double>;

void set_error(const char* fmt, ...);

// ---------------------------------------------------------------------------
// Geometry: N pulse segments (Sec. 3.1), geometric order.
// ---------------------------------------------------------------------------
struct Geometry {
  int kind = 0;
  std::vector<double> params;
  int64_t n = 0;
  std::vector<double> cx, cy, w;   // centres and lengths
};

// ---------------------------------------------------------------------------
// Host H-IDBF.
//
// One interpolative decomposition over a candidate list of c indices keeps
// k skeletons q[0..k) and expresses the c-k others p[0..c-k) through the
// k x (c-k) matrix T (row-major, T[i*(c-k)+j]):
//   column ID (V side):  K(:, p_j) ~ sum_i K(:, q_i) T[i][j]
//                        => z_i = cand[q_i] + sum_j T[i][j] cand[p_j]
//   row ID (U side):     K(p_j, :) ~ sum_i T[i][j] K(q_i, :)
//                        => out[q_i] = y_i, out[p_j] = sum_i T[i][j] y_i
// ---------------------------------------------------------------------------
struct IdBlock {
  int k = 0, c = 0;
  std::vector<int> q, p;            // positions in the candidate list
  std::vector<cplx> t;              // k x (c-k), row-major
  std::vector<int64_t> skel;        // global row/column indices of the skeletons
};

// Butterfly of one off-diagonal block (IDBF, Appendix), canonical reading:
//  column stage l (0..hc-1): pair (a at row level l, b at column level L-l),
//      stored at g = a * 2^(L-l) + b;
//  row stage l (0..hr-1): pair (a at row level L-l, b at column level l),
//      stored at g = b * 2^(L-l) + a;
//  middle: S(g) = K(rskel, cskel) for the column-stage-(hc-1) pairs g.
struct Butterfly {
  int depth = 0;          // hierarchical depth v of the parent node
  int64_t node = 0;       // node index p at depth v
  int kind = 0;           // 0 = F12 (upper-right), 1 = F21 (lower-left)
  int64_t row0 = 0, col0 = 0, n = 0;
  int L = 0, hc = 0, hr = 0;
  std::vector<std::vector<IdBlock>> col, row;
  std::vector<std::vector<cplx>> mid;   // k_r x k_c, row-major
  int rebuilt = 0;
};

struct HostFactor {
  int64_t n = 0, n0 = 0, m = 0;
  int depth = 0;
  double scale = 1.0, eps = 0.0, kappa = 0.0, eta0 = 0.0, gamma = 0.0;
  std::vector<Butterfly> bf;            // index = butterfly id (see bf_id)
  std::vector<cplx> leaf;               // m blocks, n0 x n0 row-major (scaled A)
  std::vector<cplx> linv, uinv;         // leaf triangle inverses, row-major
  bool leaf_lu = false;                 // leaf triangles are LU factors of A_leaf (HB_OPT_LEAF_LU)
  double build_seconds = 0.0;
};

// butterfly id of (depth v, node p, kind) : 2*(2^v - 1 + p) + kind
inline int64_t bf_id(int v, int64_t p, int kind) { return 2 * (((int64_t)1 << v) - 1 + p) + kind; }

int build_geometry(int kind, const double* params, int nparams, int64_t n, Geometry& g);
// Explicit node list (HB_POLYLINE): see hb_geometry_polyline.
int build_geometry_polyline(const double* xy, const int64_t* starts, int ncurves, int64_t nnodes, Geometry& g);
// options: HB_OPT_* bits of include/hb.h
int build_factor(const Geometry& g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
                 uint64_t seed, HostFactor& hf, int options = 0);

// ---------------------------------------------------------------------------
// Level-packed device image (built on the host, uploaded as flat arrays).
// ---------------------------------------------------------------------------

// One ID block on the device.  Matrix layout:
//   V-type (column ID): M[j*k + i] = T[i][j]   (output index i fastest)
//   U-type (row ID):    M[i*(c-k) + j] = T[i][j] (output index j fastest)
// Index pool at ioff: q[k], p[c-k], map[c] (map[r] = i if r = q_i, -1-j if r = p_j).
struct DBlk {
  int64_t moff;
  int32_t ioff;
  int16_t k, c;
};

// Inner-stage work item.  "A side": the candidate vector, two segments
// (a0: a_k[0] entries, a1: a_k[1] entries, concatenated).  "B side": two
// skeleton vectors, one per ID block blk[s] (b_k[s] = blk[s].k).
//   type 0 (V stage):  forward A -> B (gather + T), adjoint B -> A
//   type 2 (U stage):  forward B -> A (scatter + T), adjoint A -> B
//   type 1 (middle):   forward y(b_off[0]) = S z(a_off[0]); S at blk[0].moff,
//                      k_r = b_k[0], k_c = a_k[0]; adjoint z = S^H y.
struct DItem {
  int32_t type;
  int32_t a_off[2];
  int32_t b_off[2];
  int16_t a_k[2];
  int16_t b_k[2];
  DBlk blk[2];
};

// Outer op of one butterfly on one leaf: V0 (column leaf -> z_0 pair) or
// U0 (y_0 pair -> row leaf).  seg_off = offset of the pair vector in the
// state buffer; leaf = global leaf index of the rows/columns.
struct DOuter {
  DBlk blk;
  int32_t seg_off;
  int32_t leaf;
};

// A phase of a sweep program: `count` independent ops of one kind.
// Forward sweeps enter a butterfly through its V0 ops (PH_ENTER reads the
// solved x of the column leaves) and leave through its U0 ops (PH_EXIT
// subtracts from b on the row leaves).  Adjoint sweeps enter through U0^H
// (row leaves) and leave through V0^H (column leaves).
enum PhaseKind : int32_t {
  PH_LEAF = 0,       // arg0 = leaf index: x_leaf = Tinv_leaf b_leaf (or Tinv^H)
  PH_ENTER = 1,      // arg0 = butterfly id
  PH_ITEMS = 2,      // arg0 = first DItem index, count = #items (one stage of one butterfly)
  PH_EXIT = 3,       // arg0 = butterfly id
};
struct DPhase {
  int32_t kind;
  int32_t arg0;
  int32_t count;
  int32_t adj;       // 1 = adjoint direction of the ops
  int32_t mbytes;    // largest factor bytes (matrices + indices) of one op, complex128 storage
  int32_t vmax;      // largest vector operand (entries per right-hand side) of one op
};

// A segment of a sweep program for the cooperative sweep kernel: either one
// grid-wide phase (its ops spread over every CTA) or a run of consecutive
// small phases executed by a single CTA per group of right-hand sides; a grid
// barrier separates two segments unless both are single-CTA runs (a CTA only
// reads what it wrote itself there).
struct DSeg {
  int32_t grid;      // 1 = grid-wide phase, 0 = single-CTA run
  int32_t first;     // first phase index
  int32_t count;     // number of phases
  int32_t st_cross;  // 1 = the run reads butterfly state written outside it, or
                     //     writes state read after it: keep it in global memory
  // single-CTA runs: the vector rows and butterfly-state entries the run
  // touches ([row_lo, row_hi), [st_lo, st_hi)); the kernel keeps them in
  // shared memory for the whole run when they fit.
  int32_t row_lo, row_hi, st_lo, st_hi;
};

// A fully resolved sweep op (built on the host per program, in program order),
// so the kernel needs a single record per op.  Element offsets/counts refer to
// the factor pool (or, for leaf ops, the leaf-inverse array) in elements of the
// storage type and to the index pool in int16 entries.
enum FlatKind : int16_t { FK_GATHER = 0, FK_SCATTER = 1, FK_MIDDLE = 2, FK_LEAF = 3,
                          FK_DLEAF = 4 /* apply: columns [c1, c1 + k1) of a dense diagonal leaf block */ };
enum FlatFlag : int16_t { FF_CONJ = 1, FF_SUB = 2, FF_ADJ = 4, FF_SRC_VEC = 8, FF_OUT_VEC = 16, FF_TWO = 32,
                          FF_UPPER = 64 /* leaf op: packed upper triangle */,
                          FF_ACC = 128 /* apply: add to the staged output rows instead of overwriting them */ };
// Largest sweep leaf (rows) that pack_factor forms by merging subtrees.
constexpr int kSweepLeafMax = 128;
#ifdef __CUDACC__
#define HB_HD __host__ __device__
#else
#define HB_HD
#endif
HB_HD inline int64_t packed_tri(int64_t s) { return s * (s + 1) / 2; }
// offset of entry (r, c) in a column-packed triangle of order s
HB_HD inline int64_t tri_off_lower(int64_t s, int64_t r, int64_t c) { return c * s - c * (c - 1) / 2 + (r - c); }
HB_HD inline int64_t tri_off_upper(int64_t r, int64_t c) { return c * (c + 1) / 2 + r; }
struct FlatOp {
  int64_t moff;      // first element to stage
  int32_t melems;    // elements to stage (both blocks and the gap between them)
  int32_t m1;        // element offset of block 1 inside the staged matrices
  int32_t ioff;      // first index entry to stage (-1: none)
  int32_t src0, src1;               // vector operand segments (state entries or vec rows)
  int32_t out0, out1;               // outputs (state entries or vec rows)
  int32_t soff;      // byte offset of this op's staged data inside its phase's staging area
  int16_t ielems;    // index entries to stage
  int16_t i1;        // offset of block 1's indices
  int16_t kind, flags;
  int16_t k0, c0, k1, c1;   // FK_MIDDLE: k0 = k_r, c0 = k_c; FK_LEAF: c0 = n0
  int16_t n_s0, n_s1;       // lengths of the two operand segments
  int16_t split;            // scatter: split row between the two outputs
  int16_t pad;
};
static_assert(sizeof(FlatOp) == 64, "one op record is 64 bytes");
struct FlatProgram {
  std::vector<FlatOp> ops;
  std::vector<int32_t> base;     // base[ph] = first op of phase ph; base[nphase] = total
  std::vector<int32_t> pbytes;   // staging bytes of phase ph (complex-FP32 factor storage)
  bool ok = true;                // false: a field did not fit its record width
};
// Staging bytes of one op with complex-FP32 factors: matrices, then indices,
// each rounded up to 16 bytes.
inline int32_t flat_stage_bytes32(const FlatOp& f) {
  auto a16 = [](int64_t b) { return (b + 15) & ~(int64_t)15; };
  return (int32_t)(a16((int64_t)f.melems * 8) + (f.ioff >= 0 ? a16((int64_t)f.ielems * 2) : 0));
}


// ---------------------------------------------------------------------------
// Single-column apply plan (persistent kernel k_apply1).  Alg. 2 as phases:
// phase 0 = the V0 ops of every column leaf (one ENTER task per leaf) and the
// first column chunk of every dense leaf product; phases 1..S = the inner
// butterfly steps (one task per item), with further dense-leaf column chunks
// (each adds to the rows the previous chunk wrote); the last phases = the U0
// ops of every row leaf (EXIT tasks, added to the leaf product in the fixed
// order of the depths, cut into chained chunks when one leaf's ops do not fit
// a staging area).  Each CTA owns a contiguous range of every phase's tasks,
// cut into batches: one batch = one staging area holding the batch's factor
// and index blocks and its vector gather list (copied in by a producer warp
// with bulk copies), followed by the vector entries the batch's ops read
// (gathered by the compute warps after the phase barrier).
// ---------------------------------------------------------------------------
struct A1Task {
  int32_t op0, nops;   // FlatOp range; DLEAF / EXIT: executed in order by one warp
  int32_t kind;        // 0 ENTER, 1 ITEM (ops independent); 2 DLEAF, 3 EXIT (one warp)
  int32_t pad;         // first staged vector entry of the task (batch-relative)
};
// Staging area of a batch: [task records][op records][factor / index
// blocks][gather list][staged vector entries]; everything before the staged
// entries is copied in by the producer warp.
struct A1Batch {
  int32_t phase;
  int32_t task0, ntasks;
  int32_t op0, nops;   // op records of the batch (consecutive)
  int32_t rec_off;     // byte offset of the op records (after ntasks 16-byte task records)
  int32_t tma_bytes;   // bytes the producer copies
  int32_t area_bytes;  // staging area: tma_bytes + staged vector entries (16 bytes each)
  int32_t gl_off;      // byte offset of the gather list inside the area
  int32_t nvec;        // staged vector entries (= gather-list length)
  int32_t vec_off;     // byte offset of the staged vector entries inside the area
  int32_t npar;        // the first npar ops (of ENTER / ITEM tasks) are independent: one warp each;
                       // the tasks from task0 + nptask on (DLEAF / EXIT) take one warp per task
  int32_t nptask;
  int32_t ndep;        // batches (plan indices) whose outputs this batch reads: it waits for them
  int64_t gl_src;      // first gather-list entry in ApplyPlan::gl
  int64_t img;         // byte offset of the batch's image (its first tma_bytes bytes, ready to copy)
  int32_t dep_off;     // byte offset of the ndep producer indices (int32) inside the area
  int32_t dep_src;     // first of them in ApplyPlan::deps
};
static_assert(sizeof(A1Task) == 16, "task record");
static_assert(sizeof(A1Batch) == 80, "batch record");
// Largest number of tasks in one batch (the kernel's per-warp row table) and
// the number of compute warps of the persistent apply.
constexpr int kA1MaxTasks = 128;
constexpr int kA1Warps = 19;
// Gather-list entry: bit 31 set = row of the vector x (bits 0..30), else a
// butterfly-state entry; bit 30 set (with bit 31) = a row of the output y.
constexpr uint32_t kA1FromX = 0x80000000u;
constexpr uint32_t kA1FromY = 0xC0000000u;
struct ApplyPlan {
  std::vector<FlatOp> ops;      // soff: byte offset of the op's blocks in its batch area;
                                // pad: first staged vector entry of the op's inputs (batch-relative)
  std::vector<A1Task> tasks;
  std::vector<A1Batch> batches;
  std::vector<int32_t> cta_batch;   // [G + 1]: batches of CTA g are [cta_batch[g], cta_batch[g+1])
  std::vector<uint32_t> gl;         // gather lists of all batches
  std::vector<int32_t> deps;        // producer batches of all batches (A1Batch::dep_src)
  // Batch images: for every batch, in plan order, the bytes the producer copies into its
  // staging area (task and op records, factor and index blocks in the factor's element
  // type, gather list), so that one bulk copy fills a batch.
  std::vector<uint8_t> image;
  int nphase = 0;
  int max_area = 0;
  bool ok = true;
};

struct PackedHost {
  int64_t n = 0, n0 = 0, m = 0;
  int depth = 0;
  int kmax = 0;
  std::vector<cplx> fpool;          // factor matrices (ID T blocks + middle S), padded to even length
  std::vector<int16_t> ipool;       // indices
  int64_t state_len = 0;            // entries of the butterfly state buffer (per RHS)
  // apply (forward)
  std::vector<DOuter> vout;         // [m][D]: column leaf j, depth v (index j*D + v)
  std::vector<DOuter> uout;         // [m][D]: row leaf i, depth v
  std::vector<DItem> items;         // all inner items, ordered by (butterfly, step, pair)
  std::vector<int32_t> step_ptr;    // forward apply: items of step s at step_idx[step_ptr[s]..step_ptr[s+1])
  std::vector<int32_t> step_idx;
  std::vector<int32_t> astep_ptr;   // adjoint apply step lists
  std::vector<int32_t> astep_idx;
  int nsteps = 0;
  // per-butterfly ops for the sweeps
  std::vector<DOuter> bvout;        // per butterfly, its m_b V0 ops (contiguous)
  std::vector<DOuter> buout;        // per butterfly, its m_b U0 ops
  std::vector<int32_t> bf_vout0, bf_uout0, bf_mb;  // first op index / op count per butterfly
  // per butterfly b: forward inner step s (1..L+1) owns items
  // [bf_steps[bf_step_base[b] + s - 1], bf_steps[bf_step_base[b] + s]); the adjoint
  // runs the same ranges in reverse step order.
  std::vector<int32_t> bf_step_base, bf_steps, bf_L;
  // sweep programs
  std::vector<DPhase> prog_lower, prog_upper, prog_lower_adj, prog_upper_adj;
  // Sweep leaves ("super-leaves"): the sweeps treat each subtree of
  // sl_n = n0 2^sl_t rows as one dense triangle, the exact inverse of L~ (or
  // U~) restricted to that subtree, i.e. what Alg. 3 (Alg. 4) computes on it.
  // sl[w] holds, for sweep w (0: L~^{-1}, 1: U~^{-1}, 2: L~^{-H}, 3: U~^{-H}),
  // sl_m packed triangles of sl_n (sl_n + 1) / 2 entries, column by column:
  // lower triangles (w = 0, 3) store rows c..s-1 of column c, upper ones
  // (w = 1, 2) rows 0..c.
  int sl_t = 0;
  int64_t sl_n = 0, sl_m = 0;
  std::vector<cplx> sl[4];
  // statistics
  int64_t nnz_bf = 0;
  int32_t kmax_depth[32] = {0};
  double kavg_depth[32] = {0};
  double kavg = 0;
};

void pack_factor(const HostFactor& hf, PackedHost& ph);
// Flatten sweep program `which` (0: L~^{-1}, 1: U~^{-1}, 2: L~^{-H}, 3: U~^{-H}).
FlatProgram flatten_program(const PackedHost& ph, const std::vector<DPhase>& prog, int which);
// fill the row / state ranges of the single-CTA runs
void annotate_segments(std::vector<DSeg>& segs, const FlatProgram& fp);
// Limits of a single-CTA run that the sweep kernel keeps in shared memory
// (its op records and phase table are staged there as well); the segmenter
// cuts runs to stay within them when it cuts for residency.
constexpr int kRunMaxOps = 768;      // 48 KB of op records
constexpr int kRunMaxPhases = 511;   // (phases + 1) x 8 bytes of phase table <= 4 KB
// Split a program into segments: phases with at least grid_min ops (or
// operands too wide for a warp) run grid-wide; the runs of small phases
// between them go to single CTAs.  res_entries > 0 cuts those runs into
// pieces whose vector rows + state entries (one right-hand side) stay within
// res_entries, so that the kernel can keep a piece in shared memory.  The
// result is annotated (annotate_segments).
std::vector<DSeg> segment_program(const std::vector<DPhase>& prog, const FlatProgram& fp, int grid_min,
                                  int64_t res_entries);

// ---------------------------------------------------------------------------
// Split-BF16 tensor-core operands of the forward many-column apply (form
// HB_SPLIT_BF16).  The entry ops of a column leaf (its V0 blocks of every
// depth, stacked) and the exit ops of a row leaf (its U0 blocks of every
// depth side by side, then the dense diagonal block) are dense contractions
// W (outputs x inputs) times the leaf's vector block (inputs x columns).
// Each W is expanded to real form and cut into chunks of at most 64 complex
// outputs and 64 complex inputs; a chunk's B operand holds
//   rows n < nn:       [ Re W(n, :) | -Im W(n, :) ]
//   rows nn + n:       [ Im W(n, :) |  Re W(n, :) ]
// as kTcParts bf16 parts (W = W1 + W2 + W3, each part the bf16 rounding of
// what the earlier parts leave: 3 x 8 significant bits, the FP32 value's 24),
// each part a block in the canonical K-major, no-swizzle tensor-core layout
// (8 x 8 core matrices of 128 bytes, the K-adjacent ones contiguous, row
// groups (2 nk / 8) x 128 bytes apart).  The vectors are split the same way
// on the device and the kTcProducts products with part indices summing to at
// most 2 (0-based: 11, 12, 21, 13, 22, 31 in 1-based terms) are accumulated;
// the dropped ones are below 2^-24 relative.
// ---------------------------------------------------------------------------
constexpr int kTcParts = 3;
constexpr int kTcProducts = 6;
constexpr int kTcProdA[kTcProducts] = {0, 0, 1, 0, 1, 2};   // part of the vector operand
constexpr int kTcProdB[kTcProducts] = {0, 1, 0, 2, 1, 0};   // part of the factor operand
struct TcChunk {
  int64_t boff;      // bf16 offset of the chunk's B operand (kTcParts blocks of 2nn x 2nk each)
  int32_t nn, nk;    // complex outputs / inputs (multiples of 8, at most 64)
  int32_t in0, out0; // first entries of the chunk's input / output tables
  int32_t tcol;      // tensor-memory column of the chunk's accumulator
  int32_t flags;     // TC_ACC: add to the accumulator; TC_LAST: write the accumulator out after this chunk
};
static_assert(sizeof(TcChunk) == 32, "chunk record");
enum { TC_ACC = 1, TC_LAST = 2 };
struct TcJob {
  int32_t chunk0, nchunk;
  int32_t nreg;      // accumulator regions (output chunks, 1 or 2) the job's chunks use
  int32_t pad;
};
// table entries: a butterfly-state entry, kTcVec | row of the vector (x for inputs, y for outputs), or kTcNone
constexpr uint32_t kTcVec = 0x80000000u;
constexpr uint32_t kTcNone = 0xFFFFFFFFu;
struct TcOperands {
  std::vector<uint16_t> bpool;      // bf16 bit patterns
  std::vector<TcChunk> chunks;
  std::vector<TcJob> enter, exit;   // per leaf
  std::vector<uint32_t> tab;
};
void build_tc_operands(const PackedHost& ph, const HostFactor& hf, TcOperands& tc);
// Host emulation of the split-BF16 forward apply of one column: entry and exit
// contractions from the tensor-core operands with the device's bf16 hi/lo
// splitting of both operands and its three partial products (accumulated in
// FP64 here), the inner butterfly items in FP64 (verification without a GPU).
void host_tc_apply(const PackedHost& ph, const HostFactor& hf, const TcOperands& tc, const cplx* x, cplx* y);
// The inner butterfly steps of the packed program on a host state vector (FP64).
void host_apply_items(const PackedHost& ph, const HostFactor& hf, bool adj, std::vector<cplx>& st);
// offset (elements) of entry (r, k) of a bf16 operand block with kk columns in the layout above
inline int64_t tc_off(int64_t r, int64_t k, int64_t kk) {
  return (r / 8) * (kk / 8) * 64 + (k / 8) * 64 + (r % 8) * 8 + (k % 8);
}
// bf16 bit pattern of a float, round to nearest even (finite inputs)
inline uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
inline float bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// x = sum of kTcParts bf16 parts, each the rounding of the remainder (FP32 arithmetic)
inline void bf16_split(float x, uint16_t* parts) {
  float rem = x;
  for (int q = 0; q < kTcParts; ++q) {
    parts[q] = bf16_bits(rem);
    rem = rem - bf16_value(parts[q]);
  }
}

// Plan of the persistent single-column apply for G CTAs, factor entries of
// fes bytes, staging areas of at most max_area bytes (adj: A^H).
void build_apply_plan(const PackedHost& ph, const HostFactor& hf, bool adj, int G, int fes, int max_area,
                      ApplyPlan& plan);
// Structural check of a plan against the layout the kernel assumes (areas,
// offsets, alignment, gather-list ranges, op ranges); false on any violation.
bool check_apply_plan(const ApplyPlan& plan, const PackedHost& ph, int fes, int max_area);
// Execute a plan on the host in plan order, reading every record, block and
// gather list from the batch images as the kernel does (verification of the
// plan without a GPU): y = A^_F x or A^_F^H x.
void host_apply_plan(const PackedHost& ph, const ApplyPlan& plan, int fes, bool adj, const cplx* x, cplx* y);

// ---------------------------------------------------------------------------
// Column-partitioned sweep schedule (kernel k_sweep_cols).  Every CTA runs a
// whole sweep (Alg. 3 / Alg. 4, flattened as for the cooperative kernel) for
// its own one or two right-hand sides, so no CTA waits on another.  The
// program is cut into
//   * resident runs: subtrees whose vector rows and butterfly state fit the
//     CTA's shared-memory window (their first group loads the rows, their
//     last writes them back);
//   * global phases: the stages of the large butterflies, reading and
//     writing the vector rows and a CTA-private butterfly state in global
//     memory (each batch first gathers its distinct inputs into its warp's
//     slice of the window, which is free between runs).
// Every butterfly phase is a sparse product in row form (one output row =
// an output slot and a list of (input, coefficient) entries: the ID's
// identity entries, the T or S entries, conjugated and negated as the op
// requires); sweep-leaf phases are the packed triangles of the exact subtree
// inverse, applied in place.  The schedule is a sequence of staging groups,
// one bulk copy each: a header, a phase table, the batch descriptors, the
// batches' data.  A group holds several consecutive small phases of a resident
// run (a barrier among the compute warps after each), or one part of a large
// phase (the phase's last part ends with the barrier); a triangle is a group of
// its own.  A resident run is executed by the first kSwChain compute warps
// alone (their own barrier between phases; the other warps wait for the run's
// end), which keeps the per-phase instruction overhead of this dependent chain
// small; a global phase part's batches go round-robin to all compute warps.
// ---------------------------------------------------------------------------
constexpr int kSwWarps = 12;                 // compute warps (one more warp stages the groups)
constexpr int kSwChain = 8;                  // compute warps that execute the resident runs
constexpr int kSwWinBytes = 96 * 1024;       // resident window: rows + state of a run
constexpr int kSwRingBytes = 104 * 1024;     // staging ring of group images
constexpr int kSwPartBytes = 16 * 1024;      // partial sums of a triangle product
constexpr int kSwMaxCols = 2;                // right-hand sides per CTA
constexpr int kSwWinSlots = kSwWinBytes / (kSwMaxCols * 8);   // window slots (complex-FP32 entries per column)
constexpr int kSwGather = kSwWinSlots / (2 * kSwWarps);       // gathered inputs of a global batch (half a warp's
                                                              // slice: the next batch's gather fills the other half)
constexpr int kSwBatchBytes = 8 * 1024;      // target data bytes of one resident batch
constexpr int kSwGlobBytes = 6 * 1024;       // target data bytes of one global batch
constexpr int kSwGroupBytes = 32 * 1024;     // target bytes of a group
constexpr int kSwMaxPhases = 64;             // phases of one group
constexpr int32_t kSwAcc = (int32_t)0x80000000;  // output slot flag: add to the output instead of overwriting
enum SwGroupFlag : int32_t {
  SWG_RES = 4,      // group: batches on the window (int16 window slots)
  SWG_BEGIN = 8,    // group: load window rows [beg_lo, beg_hi) first
  SWG_ENDRUN = 16,  // group: write window rows [end_lo, end_hi) back after its last phase
};
enum SwPhaseFlag : int32_t {
  SWP_END = 1,      // the phase ends with this part: barrier among the compute warps
  SWP_TRI = 2,      // one triangle batch, taken by all compute warps
  SWP_UPPER = 4     // triangle: upper
};
struct SwGroup {     // one bulk copy
  int64_t img;       // byte offset of the group image
  int32_t bytes;     // multiple of 16
  int32_t pad;
};
struct SwGroupHdr {  // first 32 bytes of a group image; then nph phase entries (8 bytes)
  int32_t nph, flags;
  int32_t beg_lo, beg_hi, end_lo, end_hi;
  int32_t off_desc;  // byte offset of the descriptors (all phases' batches in order)
  int32_t aux;       // first group of a run (SWG_BEGIN): the run's group count; global
                     // group: the compute warp that takes its first batch
};
struct SwPhase {
  int32_t nb, flags;
};
// Batch descriptor; offsets relative to the batch start.  Row form: out[nrows]
// (int32 slot | kSwAcc; window slot for resident batches, else a global slot: a
// vector row r < n or n + a state entry), e0[nrows + 1], coef[nent] (complex, the
// factor's precision), in[nent] (int16: window slot, or position in the gather
// list), gl[ngl] (int32 global slots of the distinct inputs, global batches
// only).  Triangle: a packed lower triangle of order nrows, column by column
// (rows c..s-1 of column c), applied in place to window rows a0 .. a0 + nrows - 1;
// an upper triangle U is stored reversed (stored (r, c) = U(s-1-r, s-1-c), with
// SWP_UPPER: stored row / column i stands for window row a0 + s-1-i).
struct SwDesc {
  int32_t off;       // byte offset of the batch inside the group image
  int32_t nrows, nent, ngl;
  int32_t a0;
  int32_t off_e0, off_coef, off_in, off_gl;
  int16_t glog;      // log2 of the lanes that share one row (reduced by shuffles)
  int16_t pad;
};
static_assert(sizeof(SwGroupHdr) == 32, "group header");
static_assert(sizeof(SwPhase) == 8, "phase entry");
static_assert(sizeof(SwDesc) == 40, "batch descriptor");
struct SwSched {
  std::vector<SwGroup> groups;
  std::vector<uint8_t> image;
  int coef_bytes = 8;          // bytes of one complex coefficient (8: complex FP32, 16: FP64)
  int win_slots = kSwWinSlots; // resident window the runs were cut for
  int max_bytes = 0;           // largest group image
  int64_t res_phases = 0, glob_phases = 0, runs = 0, batches = 0;
  bool ok = true;
  const char* why = "";        // reason when !ok
};
// Schedule of sweep `which` (0: L~^{-1}, 1: U~^{-1}, 2: L~^{-H}, 3: U~^{-H}) with
// complex coefficients of coef_bytes (8 or 16) bytes, runs cut for a resident
// window of win_slots (<= kSwWinSlots) entries; needs the factor pool and the
// sweep-leaf triangles (before they are released after an upload).
void build_sweep_sched(const PackedHost& ph, int which, int coef_bytes, int win_slots, SwSched& S);
// Execute a schedule on the host for one right-hand side (FP64 arithmetic on the
// image's coefficients), reading headers, descriptors, rows, entries and slots
// from the group images as the kernel does: vec = sweep(vec) (verification of
// the schedule without a GPU).
void host_sweep_sched(const PackedHost& ph, const SwSched& S, cplx* vec);
// Structural check of a schedule against what the kernel assumes (group sizes
// within the ring, pieces inside their group, slots inside the window or the
// vector / state, gather lists within a warp's slice, run headers, triangle
// rows inside the window); returns "" or the first violation found.
const char* check_sweep_sched(const PackedHost& ph, const SwSched& S);

// FP64 host execution of the packed program (verification without a GPU).
void host_apply(const PackedHost& ph, const HostFactor& hf, bool adj, const cplx* x, cplx* y);
void host_sweep(const PackedHost& ph, const HostFactor& hf, int which, cplx* vec);

}  // namespace hb

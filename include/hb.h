/*
 * hb.h -- C ABI of the GB300-native H-IDBF-LU library (libhb.so).
 *
 * Method: Liu & Yang, "A hierarchical butterfly LU preconditioner for
 * two-dimensional electromagnetic scattering problems involving open
 * surfaces" (arXiv:1901.11371).  The library discretises an open PEC curve
 * (Sec. 3.1), compresses the TM_z EFIE impedance matrix into an H-IDBF
 * (Alg. 1 with the IDBF of Sec. 2 / Appendix), applies it (Alg. 2), applies
 * the approximate LU inverse  U~^{-1} L~^{-1}  (Eqs. (Lt), (Ut); Algs. 3, 4)
 * and solves  L~^{-1} A U~^{-1} y = L~^{-1} b,  U~ x = y  (Eqs. (Axb2), (Axb3))
 * iteratively, all on one CUDA device.
 *
 * Conventions shared by every entry point
 *  - Return value: HB_OK (0) or a negative HB_E* code.  hb_last_error()
 *    returns a thread-local message describing the last failure.  No entry
 *    point aborts the process.
 *  - Vectors are DEVICE pointers owned by the caller, column-major blocks of
 *    nrhs columns with leading dimension ld >= N (elements).  Element type:
 *    complex128 (interleaved double pairs) for form HB_C128 and for every
 *    FP64 outer vector (hb_gmres, hb_tfqmr, hb_residual, hb_rhs_plane_wave); complex64
 *    (interleaved float pairs) for hb_apply / hb_precond_solve of the
 *    HB_C64 and HB_SPLIT_BF16 forms.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - A factor handle owns the device workspaces its calls use (grown on
 *    demand, freed by hb_factor_destroy): calls on one handle must not
 *    overlap on the GPU (issue them on one stream, or serialise them);
 *    different handles are independent.
 *  - Unknowns follow the geometric order of the curve (Sec. 3.3.1); the
 *    operator acted on by hb_apply / hb_precond_solve is the RESCALED
 *    A^ = a A with a = 1 / max_i |A_ii| (Sec. 3.1 and Sec. 4).
 */
#ifndef HB_H
#define HB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define HB_OK 0
#define HB_EINVAL -1        /* invalid argument (null pointer, bad size, bad enum) */
#define HB_ENOMEM -2        /* host or device allocation failed */
#define HB_ECUDA -3         /* a CUDA runtime call failed */
#define HB_ENOCONV -4       /* iterative solver stopped before reaching rtol */
#define HB_ETIMEOUT -5      /* a bounded device-side wait expired */
#define HB_ENAN -6          /* NaN/Inf found in an input or a result */
#define HB_EUNSUPPORTED -7  /* valid request this build does not implement */

/* ---- enums ------------------------------------------------------------- */
enum { HB_STRIP = 0, HB_SPIRAL = 1, HB_ARC = 2, HB_PARALLEL_STRIPS = 3, HB_POLYLINE = 4 };
enum { HB_C128 = 0, HB_C64 = 1, HB_SPLIT_BF16 = 2 };
enum { HB_OP_N = 0, HB_OP_H = 1 };

typedef struct hb_geometry_s* hb_geometry_t;  /* opaque; freed by hb_geometry_destroy */
typedef struct hb_factor_s* hb_factor_t;      /* opaque; freed by hb_factor_destroy   */

/* Factor statistics (host struct filled by hb_factor_info). */
typedef struct {
  int64_t n;              /* unknowns N */
  int64_t leaf;           /* n0 */
  int32_t depth;          /* D = log2(N / n0): depths with off-diagonal blocks */
  int32_t form;           /* HB_C128 / HB_C64 / HB_SPLIT_BF16 */
  int64_t n_butterflies;  /* 2 (2^D - 1) */
  double scale;           /* a */
  double eps;             /* compression tolerance */
  int32_t kmax;           /* largest ID rank over all blocks */
  int32_t sweep_leaf;     /* rows s of the dense triangle blocks the sweeps apply (s = n0 2^t) */
  double kavg;            /* mean ID rank over all ID blocks */
  int32_t kmax_depth[32]; /* largest rank per hierarchical depth v */
  double kavg_depth[32];  /* mean rank per depth */
  int64_t nnz_leaf;       /* entries of the dense diagonal leaves (m n0^2) */
  int64_t nnz_butterfly;  /* stored entries of all butterfly factors (ID form) */
  int64_t nnz_lu_leaf;    /* entries of the packed triangle inverses of both sweeps (2 (N/s) s(s+1)/2) */
  int64_t index_bytes;    /* bytes of pivot / map indices on the device */
  int64_t device_bytes;   /* total device bytes held by the factor */
  int64_t apply_bytes;    /* algorithmic bytes one single-RHS hb_apply touches */
  int64_t lower_bytes;    /* algorithmic bytes of one single-RHS L~^{-1} sweep */
  int64_t upper_bytes;    /* algorithmic bytes of one single-RHS U~^{-1} sweep */
  int32_t rebuilt_blocks; /* butterflies rebuilt with eps/10 by the error probe */
  int32_t pad1;
  double build_seconds;   /* host wall time of construction + upload */
} hb_factor_stats;

/* Solver report (host struct).  Optional per-RHS arrays are caller-owned
 * host buffers of length nrhs; leave NULL to skip. */
typedef struct {
  int32_t iters;          /* total inner iterations (max over RHS) */
  int32_t restarts;       /* restart cycles (max over RHS) */
  int32_t ir_steps;       /* outer iterative-refinement steps (mixed forms) */
  int32_t converged;      /* number of RHS that reached rtol */
  double true_rel_res;    /* max over RHS of ||b^ - A^_F x|| / ||b^|| (FP64) */
  double precond_rel_res; /* max over RHS of the final preconditioned residual estimate */
  double seconds;         /* wall time of the call (host clock, synchronised) */
  int32_t* iters_per_rhs; /* optional out */
  double* res_per_rhs;    /* optional out */
  int32_t graph_launches; /* hb_gmres: restart cycles run as one CUDA graph launch each */
  int32_t pad;
} hb_gmres_info;

/* hb_geometry -- discretise an open PEC curve into n_segments pulse segments
 * (Sec. 3.1: w_i, rho_i are the length and centre of segment i).  Curves are
 * split at equal arc length; each segment is the chord between consecutive
 * nodes.  params: STRIP (x0,y0,x1,y1); SPIRAL (a, theta0, theta1) for
 * r = a theta; ARC (R, phi0, phi1); PARALLEL_STRIPS (n_strips, length,
 * spacing) with strip s at y = s*spacing, x in [0, length], ordered strip
 * after strip.  Lengths in wavelengths.  *out is owned by the library.
 * Errors: HB_EINVAL (bad kind, nparams, n_segments < 1), HB_ENOMEM. */
int hb_geometry(int kind, const double* params, int nparams, int64_t n_segments, hb_geometry_t* out);

/* hb_geometry_polyline -- an explicitly given scatterer (kind HB_POLYLINE):
 * nnodes nodes xy_nodes[2*i], xy_nodes[2*i+1] (host, wavelengths) on ncurves
 * open curves; curve c uses nodes curve_starts[c] .. curve_starts[c+1]-1 (the
 * last up to nnodes-1) and contributes one pulse segment per pair of
 * consecutive nodes (the chord: centre = midpoint, w = length, Sec. 3.1), so
 * N = nnodes - ncurves, in the order given (the geometric order of Sec.
 * 3.3.1 is the caller's).  Errors: HB_EINVAL (null pointers, curve_starts[0]
 * != 0 or not increasing, a curve with fewer than 2 nodes, a non-finite
 * coordinate, a zero-length segment), HB_ENOMEM. */
int hb_geometry_polyline(const double* xy_nodes, const int64_t* curve_starts, int ncurves, int64_t nnodes,
                         hb_geometry_t* out);

/* Host copies of the segment centres (2N doubles, x/y interleaved) and
 * lengths (N doubles) into caller-owned buffers.  Either may be NULL. */
int hb_geometry_segments(hb_geometry_t g, double* centers_xy, double* lengths);
int64_t hb_geometry_size(hb_geometry_t g);
void hb_geometry_destroy(hb_geometry_t g);

/* hb_factor -- build the H-IDBF of the rescaled TM EFIE matrix (Sec. 3.1:
 * A_ij = (k eta0 w_j / 4) H0^(2)(k |rho_i - rho_j|), A_ii = (k eta0 w_i / 4)
 * [1 - i (2/pi) ln(gamma k w_i / (4e))], k = 2 pi / wavelength) with leaf
 * size `leaf` (n0) and compression tolerance eps (Alg. 1, IDBF of the
 * Appendix with sampled IDs seeded by `seed`), then upload the level-packed
 * factors, dense leaves and the sweeps' packed triangles (the exact inverse
 * of L~ / U~ on every subtree of up to 128 rows, formed on the host by
 * running Algs. 3/4 on unit vectors) to the current device in the storage
 * `form`.  HB_SPLIT_BF16 stores the factors like HB_C64 and adds, for every
 * leaf, its entry contraction (the V0 blocks of all depths) and exit
 * contraction (the U0 blocks of all depths and the dense diagonal block) as
 * dense split-BF16 tensor-core operands: the forward hb_apply of 32 or more
 * columns runs those on the tensor cores (tcgen05, bf16 hi/lo parts of both
 * operands, three products accumulated in FP32) and the inner butterfly steps,
 * the adjoint and the sweeps in complex FP32.  Construction runs on the host and is
 * timed apart from the hot path.  Requires N = leaf * 2^D with D >= 1,
 * 8 <= leaf <= 256.
 * Errors: HB_EINVAL, HB_EUNSUPPORTED (N not leaf*2^D), HB_ENOMEM, HB_ECUDA. */
int hb_factor(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
              int form, uint64_t seed, void* stream, hb_factor_t* out);

/* Factor options (bit mask for hb_factor_ex / hb_factor_host_ex).
 * HB_OPT_LEAF_LU: the leaf blocks of L~ and U~ are the LU factors of the dense
 *   leaf block (A_leaf = L U, L unit lower, U upper, no pivoting) instead of
 *   the entry-wise triangles of Eqs. (Lt), (Ut); the off-diagonal blocks and
 *   Algs. 3/4 are unchanged.  A variant the paper implies (its leaf solves are
 *   LAPACK triangular solves); HB_EUNSUPPORTED on a zero pivot. */
#define HB_OPT_LEAF_LU 1
/* HB_OPT_SWEEP_WINDOW_MIN: the column-partitioned sweep kernel (hb_set_sweep_kernel)
 *   keeps only subtrees of at most 512 vector rows + butterfly-state entries
 *   resident in shared memory, so that every larger butterfly runs as global
 *   phases; a test and tuning aid for small problems (results are unchanged). */
#define HB_OPT_SWEEP_WINDOW_MIN 2

/* hb_factor_ex / hb_factor_host_ex -- hb_factor / hb_factor_host with an
 * options mask (0 = the defaults of hb_factor).  Errors as hb_factor, plus
 * HB_EINVAL for unknown option bits. */
int hb_factor_ex(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
                 int form, uint64_t seed, int options, void* stream, hb_factor_t* out);
int hb_factor_info(hb_factor_t f, hb_factor_stats* s);
void hb_factor_destroy(hb_factor_t f);

/* hb_tree -- cluster tree node ranges [begin, end) in BFS order (node (v,p)
 * at index 2^v - 1 + p), 2m - 1 nodes (Alg. 1 recursion).  Host buffers. */
int hb_tree(hb_factor_t f, int64_t* node_begin, int64_t* node_end);

/* hb_apply -- y = A^_F x (op = HB_OP_N, Alg. 2) or y = A^_F^H x (HB_OP_H),
 * for nrhs columns.  x and y must not overlap.  Element type per form (see
 * top).  Errors: HB_EINVAL (null, nrhs < 1, ld < N), HB_ECUDA. */
int hb_apply(hb_factor_t f, int op, const void* x, void* y, int64_t nrhs, int64_t ld, void* stream);

/* hb_apply_noalloc -- the same product as hb_apply (same kernels, same
 * arguments, same result), for callers that must not let the library
 * allocate device memory: for instance a framework whose caching allocator
 * owns the whole device-memory budget, or a service that may not allocate
 * after start-up.  The paper has no counterpart; this is an interface
 * convenience.  Scratch comes from one fixed 16 MiB device array that every
 * GPU loading the library holds until the process exits; the call performs
 * no cudaMalloc / cudaFree.  The first call on each device looks up that
 * array's device address (cudaGetSymbolAddress, with the device current);
 * make that first call before any stream capture.  All calls share the
 * array: calls that may overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller.  Requests needing more than
 * 16 MiB of scratch (butterfly state, plus two reordered blocks when
 * nrhs > 1) return HB_EINVAL with the required size in hb_last_error(). */
int hb_apply_noalloc(hb_factor_t f, int op, const void* x, void* y, int64_t nrhs, int64_t ld, void* stream);

/* hb_apply_adjoint -- y = A^_F^H x: conjugate-transposed factors applied in
 * reverse stage order (no counterpart in the paper; same as hb_apply with HB_OP_H). */
int hb_apply_adjoint(hb_factor_t f, const void* x, void* y, int64_t nrhs, int64_t ld, void* stream);

/* hb_precond_solve -- x = U~^{-1} L~^{-1} b (op = HB_OP_N; Algs. 3 then 4)
 * or x = L~^{-H} U~^{-H} b (HB_OP_H), with L~/U~ the entry-wise triangles of
 * the compressed operator (Eqs. (Lt), (Ut)).  b and x must not overlap.
 * Errors: HB_EINVAL, HB_ECUDA. */
int hb_precond_solve(hb_factor_t f, int op, const void* b, void* x, int64_t nrhs, int64_t ld, void* stream);

/* hb_lower_solve / hb_upper_solve -- one sweep: x = L~^{-1} b (Alg. 3) or
 * x = U~^{-1} b (Alg. 4); op = HB_OP_H gives L~^{-H} b / U~^{-H} b. */
int hb_lower_solve(hb_factor_t f, int op, const void* b, void* x, int64_t nrhs, int64_t ld, void* stream);
int hb_upper_solve(hb_factor_t f, int op, const void* b, void* x, int64_t nrhs, int64_t ld, void* stream);

/* hb_residual -- r = b - A^_F x (op N) or b - A^_F^H x (op H) in FP64
 * arithmetic on the stored factors; complex128 vectors.  b, x, r distinct. */
int hb_residual(hb_factor_t f, int op, const void* b, const void* x, void* r, int64_t nrhs, int64_t ld, void* stream);

/* hb_gmres -- solve A x = b_phys for nrhs right-hand sides (complex128, the
 * PHYSICAL excitation; the rescaling a is applied internally, x is invariant).
 * HB_C128: GMRES(restart) on the split-preconditioned system (Eqs. (Axb2),
 * (Axb3)).  HB_C64 / HB_SPLIT_BF16: flexible GMRES right-preconditioned by
 * U~^{-1} L~^{-1}, with the preconditioner, A and the Krylov basis in complex
 * FP32, inside FP64 iterative refinement (residual with FP64 arithmetic on
 * the stored factors; once every column is within 1e-3, updated as
 * r -= A dz with the FP32 apply on the correction, accumulated in FP64).
 * Stops when that FP64 relative residual ||b^ - A^_F x||/||b^|| <= rtol for
 * every column or after maxit inner iterations.  The
 * initial guess is zero; x is overwritten with the solution.  Synchronises
 * `stream` before returning; info may be NULL.
 * Errors: HB_EINVAL, HB_ENAN (non-finite b, or a residual that became
 * non-finite: overflow of the preconditioned iteration; info filled, its
 * residual NaN), HB_ENOCONV (info still filled),
 * HB_ETIMEOUT (a bounded wait of a sweep kernel expired; x undefined; the
 * flag is cleared, so the next call starts clean). */
int hb_gmres(hb_factor_t f, int op, const void* b_phys, void* x, int64_t nrhs, int64_t ld, int restart,
             double rtol, int maxit, hb_gmres_info* info, void* stream);

/* hb_set_gmres_graph -- 1 (default): for nrhs >= 2, hb_gmres runs each restart
 * cycle as ONE CUDA graph launch: the start vector, every Arnoldi step (the
 * preconditioner sweeps, the operator, CGS2 with its reductions), the Givens
 * rotations of every column's Hessenberg matrix, the convergence test and the
 * least-squares solve all run on the device; the test closes a device flag
 * that makes the graph's remaining steps return at once, so a cycle costs what
 * the host-driven loop's does without a host round trip per step.  The graph
 * is captured once and kept on the factor while the restart, nrhs, op, the
 * factor's execution settings (hb_autotune, hb_set_sweep_kernel,
 * hb_set_sweep_grid_min, hb_set_wait_limit, hb_profile) and its workspaces stay
 * the same.  0: the host-driven loop (a host synchronisation per step).  Both
 * compute the same iteration; info->graph_launches says which ran.  One
 * right-hand side always takes the host-driven loop.  Returns HB_OK or
 * HB_EINVAL.  Not in the paper: an execution choice. */
int hb_set_gmres_graph(hb_factor_t f, int on);

/* hb_tfqmr -- solve A x = b_phys (complex128, physical excitation, as for
 * hb_gmres) with transpose-free QMR, the Krylov solver of Sec. 4, on the
 * split-preconditioned system (Eqs. (Axb2), (Axb3)), every storage form: the
 * vectors and scalars are FP64; the products with A^_F, L~^{-1} and U~^{-1} use
 * FP64 arithmetic on the form's factors (complex128 for HB_C128, complex64 for
 * HB_C64 and HB_SPLIT_BF16).  rstar: the shadow vectors r* of the Lanczos biorthogonalisation,
 * complex128 device block laid out like b (nrhs columns, leading dimension
 * ld), caller-owned and not modified; NULL takes r* = L~^{-1} b^ (the paper
 * does not name one; on the split EFIE systems that choice can meet a
 * near-breakdown and stall near 1e-5, while a random r* converges in about as
 * many operator products as GMRES(30) takes iterations).  Columns run in
 * lockstep with their own scalars; each half step costs at most one product
 * with L~^{-1} A U~^{-1} (two per pair of half steps).  When the quasi-residual
 * bound tau sqrt(m+1) reaches rtol ||L~^{-1} b^|| the FP64 true residual
 * ||b^ - A^_F x||/||b^|| is formed; a column stops once it is <= rtol.  info:
 * iters = half steps, restarts = true-residual checks, precond_rel_res = the
 * largest final bound relative to ||L~^{-1} b^||.  x is overwritten;
 * synchronises `stream` before returning; info may be NULL.
 * Errors: HB_EINVAL, HB_ENAN (non-finite b or
 * rstar), HB_ENOCONV (maxit half steps or a breakdown; info still filled),
 * HB_ETIMEOUT (as hb_gmres). */
int hb_tfqmr(hb_factor_t f, int op, const void* b_phys, const void* rstar, void* x, int64_t nrhs, int64_t ld,
             double rtol, int maxit, hb_gmres_info* info, void* stream);

/* hb_rhs_plane_wave -- b_i = exp(-i k (x_i cos phi + y_i sin phi)) (the
 * incident field E^inc_z(rho_i) of Sec. 3.1, physical, unscaled) for nrhs
 * angles phi_deg (host array, degrees) into the complex128 device block b. */
int hb_rhs_plane_wave(hb_factor_t f, const double* phi_deg, int64_t nrhs, void* b, int64_t ld, void* stream);

/* hb_far_field -- E_far(phi_q) = C sum_n w_n x_n exp(+i k (x_n cos phi_q + y_n sin phi_q)),
 * C = -(k eta0/4) sqrt(2i/(pi k)), for every column of x (complex128, the
 * physical current) and every observation angle (host array, degrees).
 * out: complex128 device array [nrhs][nobs] (row-major).  Not in the paper:
 * the far zone of the scattered field of the same EFIE kernel. */
int hb_far_field(hb_factor_t f, const void* x, int64_t nrhs, int64_t ld, const double* phi_obs_deg, int64_t nobs,
                 void* out, void* stream);

/* hb_far_field_adjoint -- the conjugate transpose of hb_far_field:
 * out[:, r] = sum_q conj(C) w_n exp(-i k (x_n cos phi_q + y_n sin phi_q)) g[r][q]
 * for g a complex128 device array [nrhs][nobs]; out is a complex128 device
 * block [nrhs][ld].  Used by the gradient of far-field losses (no counterpart
 * in the paper). */
int hb_far_field_adjoint(hb_factor_t f, const void* g, int64_t nrhs, const double* phi_obs_deg, int64_t nobs,
                         void* out, int64_t ld, void* stream);

/* hb_monostatic -- backscatter for column r of x at its own incidence angle
 * phi_deg[r]: C sum_n w_n b_n(phi_r) x_n.  out: complex128 device [nrhs]. */
int hb_monostatic(hb_factor_t f, const void* x, int64_t nrhs, int64_t ld, const double* phi_deg, void* out,
                  void* stream);

/* hb_set_sweep_grid_min -- tuning knob of the cooperative sweep kernel:
 * program phases with at least grid_min independent ops are spread over all
 * CTAs, smaller ones run inside one CTA (default 16).  Synchronises the
 * legacy default stream.  Returns the previous value (>= 1) or an error code. */
int hb_set_sweep_grid_min(hb_factor_t f, int grid_min);

/* hb_autotune -- time the cooperative sweep kernel for nrhs right-hand sides
 * under each candidate split between grid-wide and single-CTA phases
 * (thresholds 4, 8, 16, 32, 64 ops, and "all single-CTA") and, for the
 * complex-FP32 forms, the column-partitioned sweep kernel; keep the fastest
 * for calls with one right-hand side (nrhs == 1) or with several (nrhs > 1),
 * and report the choice in *chosen (may be NULL): the threshold, or 0 for the
 * column-partitioned kernel.  Synchronises `stream`; uses the factor's
 * workspace.  hb_set_sweep_grid_min clears the tuned choice.
 * Not in the paper: launch-configuration tuning. */
int hb_autotune(hb_factor_t f, int64_t nrhs, void* stream, int* chosen);

/* hb_autotune_times -- the per-candidate sweep times (ms per sweep) of the
 * last hb_autotune call of the class of nrhs (one / several right-hand
 * sides), with the candidates' thresholds (2^30 = all single-CTA; 0 = the
 * column-partitioned kernel, timed for the complex-FP32 forms only).  Writes
 * at most max of the 6 or 7 entries to ms_out / grid_min_out (host arrays)
 * and returns the number written, 0 if that class was never tuned, or HB_EINVAL. */
int hb_autotune_times(hb_factor_t f, int64_t nrhs, float* ms_out, int* grid_min_out, int max);

/* hb_set_sweep_kernel -- which kernel runs the sweeps (L~^{-1}, U~^{-1} and the
 * adjoints; Algs. 3, 4): -1 = the last hb_autotune choice (default; the
 * cooperative kernel until tuned), 0 = the cooperative kernel (grid-wide phases
 * for large butterfly stages, single-CTA runs near the leaves), 1 = the
 * column-partitioned kernel (every CTA runs the whole sweep for its own one or
 * two right-hand sides from host-built schedules: no grid barriers;
 * complex-FP32 forms only).  Results agree to the rounding of the forms'
 * arithmetic.  Returns HB_OK, HB_EUNSUPPORTED (kind 1 for HB_C128, which has
 * no schedules) or HB_EINVAL.  Not in the paper: an execution choice. */
int hb_set_sweep_kernel(hb_factor_t f, int kind);

/* hb_set_wait_limit -- iteration limit of every bounded device-side wait
 * (the sweep kernel's grid barrier; default 2^24 polls, about a second).
 * hb_status -- synchronise `stream`, then return HB_ETIMEOUT (and clear the
 * flag) if a bounded wait expired since the last call, else HB_OK.  A timed
 * out sweep leaves its output undefined; the device stays usable. */
int hb_set_wait_limit(hb_factor_t f, long long spins);
int hb_status(hb_factor_t f, void* stream);

/* hb_profile -- enable (1) / disable (0) timing of the hot-path kernels of
 * this factor.  While enabled, every apply launch sequence and every sweep
 * kernel is bracketed by CUDA events on its stream (enabling resets the
 * record; enabling it again while on resets the record only).  Inside
 * hb_gmres's graph-captured restart cycle the events sit around the
 * conditional node of each sweep or apply and are counted for the steps
 * that ran; switching profiling on or off discards the cached graph.  Not in
 * the paper: measurement support.
 * hb_profile_read -- kind 0: apply (D+2 kernels per call), 1: sweep kernels,
 * 2: every kernel the library launched (count only).  Returns the number of
 * recorded calls/launches and their summed device time in ms (synchronises
 * the recorded events; total_ms is 0 for kind 2). */
int hb_profile(hb_factor_t f, int enable);
int hb_profile_read(hb_factor_t f, int kind, int64_t* count, double* total_ms);

/* ---- host-only verification entry points (no GPU needed) -------------
 * hb_factor_host builds the same H-IDBF and packed program as hb_factor but
 * keeps it in host memory only (no device image; the device entry points
 * reject such a handle with HB_EINVAL).  hb_host_apply / hb_host_sweep run
 * the packed program in FP64 on the host: y = A^_F x (op N) or A^_F^H x, and
 * in-place sweeps (which: 0 L~^{-1}, 1 U~^{-1}, 2 L~^{-H}, 3 U~^{-H}).
 * Vectors are host arrays of N complex128 (interleaved doubles). */
int hb_factor_host(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
                   uint64_t seed, hb_factor_t* out);
int hb_factor_host_ex(hb_geometry_t g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
                      uint64_t seed, int options, hb_factor_t* out);
int hb_host_apply(hb_factor_t f, int op, const double* x, double* y);
/* hb_host_apply_plan -- build the schedule of the persistent single-column
 * apply for `grid` CTAs and factor entries of factor_bytes (8: complex64,
 * 16: complex128), check its structure, and execute it on the host in FP64
 * exactly as the kernel stages it (y = A^_F x or A^_F^H x).  Verifies the
 * schedule without a GPU.  Returns the number of staging batches (>= 0),
 * HB_EUNSUPPORTED if the schedule failed its check, or HB_EINVAL. */
int hb_host_apply_plan(hb_factor_t f, int op, int grid, int factor_bytes, const double* x, double* y);
/* hb_host_tc_apply -- build the split-BF16 tensor-core operands of the
 * HB_SPLIT_BF16 form and emulate its forward apply of one column on the host:
 * entry and exit contractions from those operands with the device's bf16
 * hi/lo splitting of both operands and its three partial products, inner
 * butterfly items in FP64.  Verifies the operands without a GPU.  Returns the
 * number of operand chunks (>= 0) or HB_EINVAL. */
int hb_host_tc_apply(hb_factor_t f, const double* x, double* y);
int hb_host_sweep(hb_factor_t f, int which, double* vec);
/* hb_host_sweep_sched -- build the schedule of the column-partitioned sweep
 * kernel (sweep `which`; complex coefficients of coef_bytes: 8 = complex64 as
 * on the device, 16 = complex128; runs cut for a resident window of win_slots
 * entries, 0 = the kernel's full window) and execute it on the host in FP64 for
 * the one column in vec (in place), reading every row, coefficient and slot from
 * the batch images as the kernel does.  Verifies the schedule without a GPU.
 * Returns the number of batches (>= 0), HB_EUNSUPPORTED if this factor has no
 * such schedule, or HB_EINVAL. */
int hb_host_sweep_sched(hb_factor_t f, int which, int coef_bytes, int win_slots, double* vec);

const char* hb_last_error(void);
const char* hb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HB_H */

// Cooperative sweep kernel (sm_103a), templates shared by the per-precision
// translation units hb_sweep_f64.cu, hb_sweep_f32n.cu, hb_sweep_f32w.cu and
// hb_sweep_mix.cu (compiled in parallel): x = L~^{-1} b, U~^{-1} b and their
// adjoints (Algs. 3, 4), in place on the vector.
//
// The recursion of Alg. 3 / Alg. 4 is flattened on the host into a program
// of phases (sweep-leaf solves -- packed triangles of the exact inverse on
// subtrees of up to 128 rows --, butterfly entry ops, butterfly stages,
// butterfly exit ops); consecutive phases depend on each other, ops inside a
// phase do not.  The program is cut into segments:
//   * a grid segment is one large phase (a stage of a big butterfly); its
//     ops (or, with many right-hand sides, (op, column range) units, taken by
//     two-warp groups) are spread over all CTAs;
//   * a local segment is a run of small phases (a subtree near the leaves);
//     each CTA executes it for its own share of the right-hand sides, one op
//     per warp, a barrier between phases.  Runs that fit are resident in
//     shared memory and fed by a producer warp (see local_run_ring).
// A grid barrier (bounded spin; HB_ETIMEOUT instead of a hang) separates a
// grid segment from its neighbours; consecutive local segments need none.
// Ops outside resident runs stage their factor blocks and vector operands
// into shared memory with 16-byte cp.async copies, then compute from shared
// memory.  Vector and butterfly-state reads bypass L1 (ld.global.cg) because
// other CTAs write them inside the same launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_device.h"
#include "hb_sweep_launch.h"

namespace hb {

namespace {

template <class T> struct CT;
template <> struct CT<float> { using t = float2; };
template <> struct CT<double> { using t = double2; };

template <class T> __device__ __forceinline__ typename CT<T>::t z2() { return {(T)0, (T)0}; }
template <class T, class F> __device__ __forceinline__ typename CT<T>::t cv(const F v) { return {(T)v.x, (T)v.y}; }
template <class T, class F> __device__ __forceinline__ typename CT<T>::t cvc(const F v) { return {(T)v.x, -(T)v.y}; }
template <class C> __device__ __forceinline__ void fma2(C& acc, const C& a, const C& b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 ldcg2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg2(const double2* p) { return __ldcg(p); }

// ---- a group of threads cooperating on one op: a warp or the whole CTA
struct Grp {
  int t, nt;
  bool cta;
  int bar = 0;   // > 0: a group of whole warps synchronised on named barrier `bar`
  __device__ __forceinline__ void sync() const {
    if (bar > 0) asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "r"(nt) : "memory");
    else if (cta) __syncthreads();
    else __syncwarp();
  }
};

__device__ __forceinline__ void cp16(void* smem_dst, const void* gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// stage `bytes` (rounded up to 16) from 16-byte aligned global memory
__device__ __forceinline__ void stage(void* dst, const void* src, int64_t bytes, const Grp& g) {
  const int64_t n16 = (bytes + 15) >> 4;
  const char* s = (const char*)src;
  char* d = (char*)dst;
  for (int64_t e = g.t; e < n16; e += g.nt) cp16(d + 16 * e, s + 16 * e);
}

__device__ __forceinline__ int64_t align16(int64_t b) { return (b + 15) & ~(int64_t)15; }

// Bounded-spin grid barrier.  Returns false if the wait limit expired or
// another CTA reported a failure.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_sync(GridBar* gb, unsigned& my_gen, long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    unsigned g = my_gen;
    unsigned old = atomicAdd(&gb->count, 1u);
    if (old == gridDim.x - 1) {
      gb->count = 0;
      __threadfence();
      atomicExch(&gb->gen, g + 1);
    } else {
      long long spins = 0;
      while (ld_acquire_u32(&gb->gen) == g) {
        if (++spins > spin_limit || *(volatile int*)&gb->err) { ok = 0; break; }
        __nanosleep(64);
      }
    }
    if (!ok) atomicExch(&gb->err, 1);
    __threadfence();
    s_ok = ok && !*(volatile int*)&gb->err;
  }
  my_gen++;
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// compute kernels of one op from staged operands
// ---------------------------------------------------------------------------

// B side = gather + T * rest (V-type layout M[j*k+i]; or U-type adjoint conj(M[i*nr+j])).
// The group's threads take (output i, RHS chunk ch) pairs: chunk ch holds the
// right-hand sides r0 + ch*RC .. (< rend) at column ch*RC of the staged rows
// (row stride vs) and of `out` (row stride R, column offset r0).
template <class T, class F, int RC, bool UADJ>
__device__ __forceinline__ void vlike(const F* M, const int16_t* idx, int k, int c,
                                      const typename CT<T>::t* cand /* [c][vs] smem */, int vs,
                                      typename CT<T>::t* out, int64_t R, int64_t r0, int64_t rend, int nch,
                                      const Grp& g) {
  using C = typename CT<T>::t;
  const int nr = c - k;
  for (int e = g.t; e < k * nch; e += g.nt) {
    const int i = e % k, ch = e / k;
    const C* cb = cand + ch * RC;
    const int64_t rs = r0 + (int64_t)ch * RC;
    const int rc = (rend - rs) < RC ? (int)(rend - rs) : RC;
    C acc[RC];
    const int qi = idx[i];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr] = cb[qi * vs + rr];
#pragma unroll 8
    for (int j = 0; j < nr; ++j) {
      C m = UADJ ? cvc<T>(M[(int64_t)i * nr + j]) : cv<T>(M[(int64_t)j * k + i]);
      const C* sv = cb + idx[k + j] * vs;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], m, sv[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
      if (rr < rc) out[(int64_t)i * R + rs + rr] = acc[rr];
  }
}

// candidate entry r of one block (U-type layout M[i*nr+j]; or V-type adjoint conj(M[j*k+i]))
template <class T, class F, int RC, bool VADJ>
__device__ __forceinline__ void rowc(typename CT<T>::t (&acc)[RC], const F* M, const int16_t* idx, int k, int c,
                                     const typename CT<T>::t* y /* [k][vs] smem */, int vs, int r) {
  using C = typename CT<T>::t;
  const int code = idx[c + r];
  if (code >= 0) {
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) { acc[rr].x += y[code * vs + rr].x; acc[rr].y += y[code * vs + rr].y; }
  } else {
    const int j = -1 - code, nr = c - k;
#pragma unroll 8
    for (int i = 0; i < k; ++i) {
      C m = VADJ ? cvc<T>(M[(int64_t)j * k + i]) : cv<T>(M[(int64_t)i * nr + j]);
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], m, y[i * vs + rr]);
    }
  }
}

// Stage `cnt` vector entries, right-hand sides [r0, r0+width), from global
// (row stride R) into shared memory rows of stride W (>= width).  Rows that
// are 16-byte aligned and sized go through cp.async (asynchronous; completed by
// cp_commit_wait), other rows through L1-bypassing loads.
template <class C>
__device__ __forceinline__ void stage_vec(C* dst, const C* src, int cnt, int64_t R, int64_t r0, int width, int W,
                                          const Grp& g, bool noasync = false) {
  const int64_t rowb = (int64_t)width * sizeof(C);
  const bool vec16 = !noasync && ((rowb & 15) == 0) && ((((uintptr_t)(src + r0)) & 15) == 0) && (((R * sizeof(C)) & 15) == 0) &&
                     ((((int64_t)W * sizeof(C)) & 15) == 0);
  if (vec16) {
    const int per = (int)(rowb >> 4);
    for (int e = g.t; e < cnt * per; e += g.nt) {
      const int i = e / per, q = e % per;
      cp16((char*)(dst + (int64_t)i * W) + 16 * q, (const char*)(src + (int64_t)i * R + r0) + 16 * q);
    }
  } else {
    for (int e = g.t; e < cnt * width; e += g.nt) {
      const int i = e / width, rr = e % width;
      dst[(int64_t)i * W + rr] = ldcg2(src + (int64_t)i * R + r0 + rr);
    }
  }
}

struct SweepArgs {
  const DSeg* segs;
  int nseg;
  const DPhase* prog;
  const FlatOp* flat;
  const int32_t* flat_base;
  const int32_t* flat_pbytes;
  int64_t n0;
  const DOuter* bvout;
  const DOuter* buout;
  const int32_t* bf_vout0;
  const int32_t* bf_uout0;
  const DItem* items;
  const void* fp;
  const int16_t* ip;
  const void* tinv;
  void* vec;
  void* st;
  int64_t R;
  GridBar* bar;
  int smem_bytes;
  long long spin_limit;
  int use_pf;
};

// ---------------------------------------------------------------------------
// one op of a phase, executed by group g (warp or CTA) with staging area buf.
// The op's factor blocks are staged once; its vector operands for the RHS
// range [rb, re) are staged in one pass when they fit next to them (else one
// RC-wide chunk at a time), and the op is computed chunk by chunk from shared
// memory.
// ---------------------------------------------------------------------------
// Vector operand plan of one op for the RHS range [rb, re): either the whole
// range is staged at once in rows of stride W = nch*RC, or one RC-wide chunk
// at a time (stride RC).
template <class C, int RC>
struct VecPlan {
  int64_t rb, re, nch;
  bool once;
  int W;
  __device__ VecPlan(int64_t rb_, int64_t re_, int64_t base_bytes, int vcnt, int64_t buf_bytes) : rb(rb_), re(re_) {
    nch = (re - rb + RC - 1) / RC;
    once = base_bytes + nch * RC * (int64_t)vcnt * (int64_t)sizeof(C) <= buf_bytes;
    W = once ? (int)(nch * RC) : RC;
  }
  __device__ int rc(int64_t ch) const {
    int64_t r0 = rb + ch * RC;
    return (int)((re - r0) < RC ? (re - r0) : RC);
  }
};

// stage the vector operand segments (up to two, concatenated) for RHS [r0, r0+width)
template <class C>
__device__ __forceinline__ void load_segs(C* dst, const C* s0, int n0s, const C* s1, int n1s, int64_t R, int64_t r0,
                                          int width, int W, const Grp& g, bool noasync = false) {
  stage_vec<C>(dst, s0, n0s, R, r0, width, W, g, noasync);
  if (n1s > 0) stage_vec<C>(dst + (int64_t)n0s * W, s1, n1s, R, r0, width, W, g, noasync);
}

template <class T, class F, int RC>
__device__ void do_op(const SweepArgs& a, const FlatOp& f, char* buf, int64_t buf_bytes, const Grp& g, int64_t rb,
                      int64_t re, bool pre = false) {
  using C = typename CT<T>::t;
  C* vec = (C*)a.vec;
  C* st = (C*)a.st;
  const int64_t R = a.R;
  const int kind = f.kind;
  const bool conj_layout = (f.flags & FF_CONJ) != 0;
  const bool subtract = (f.flags & FF_SUB) != 0;
  const bool adj = (f.flags & FF_ADJ) != 0;
  const int nblk = (f.flags & FF_TWO) ? 2 : 1;
  const int k0 = f.k0, c0 = f.c0, k1 = f.k1, c1 = f.c1;
  const C* src0 = ((f.flags & FF_SRC_VEC) ? vec : st) + (int64_t)f.src0 * R;
  const C* src1 = st + (int64_t)f.src1 * R;
  const int n_s0 = f.n_s0, n_s1 = f.n_s1;
  C* out0 = ((f.flags & FF_OUT_VEC) ? vec : st) + (int64_t)f.out0 * R;
  C* out1 = st + (int64_t)f.out1 * R;
  const int split_r = f.split;
  const int kr = f.k0, kc = f.c0;
  const F* mstart = (const F*)a.fp + f.moff;
  const int16_t* istart = f.ioff >= 0 ? a.ip + f.ioff : nullptr;
  const int64_t mbytes = align16((int64_t)f.melems * (int64_t)sizeof(F));
  const int64_t ibytes = f.ioff >= 0 ? align16((int64_t)f.ielems * (int64_t)sizeof(int16_t)) : 0;
  // ---- staging
  const int vcnt = n_s0 + n_s1;
  const bool fit = pre || mbytes + ibytes + (int64_t)vcnt * RC * (int64_t)sizeof(C) <= buf_bytes;
  const F* Ms = mstart;
  const int16_t* Is = istart;
  C* v = (C*)buf;
  int64_t base = 0;
  if (fit) {
    if (!pre) {
      stage(buf, mstart, mbytes, g);
      if (ibytes) stage(buf + mbytes, istart, ibytes, g);
    }
    Ms = (const F*)buf;
    Is = (const int16_t*)(buf + mbytes);
    base = mbytes + ibytes;
    v = (C*)(buf + base);
  }
  const F* M0 = Ms;
  const int16_t* I0 = Is;
  const F* M1 = Ms + f.m1;
  const int16_t* I1 = Is ? Is + f.i1 : nullptr;
  VecPlan<C, RC> pl(rb, re, base, vcnt, buf_bytes);
  const int W = pl.W;
  if (pl.once) {
    load_segs<C>(v, src0, n_s0, src1, n_s1, R, rb, (int)(re - rb), W, g, pre);
    if (!pre) cp_commit_wait();
    g.sync();
  }
  // Whole range staged: the threads take (output, chunk) pairs over all
  // chunks in one pass.  Otherwise one chunk per pass.
  const int nst = pl.once ? (int)pl.nch : 1;
  const int npass = pl.once ? 1 : (int)pl.nch;
  for (int ps = 0; ps < npass; ++ps) {
    const int64_t r0 = rb + (int64_t)ps * RC;
    C* vv = v;
    if (!pl.once) {
      load_segs<C>(vv, src0, n_s0, src1, n_s1, R, r0, pl.rc(ps), W, g, pre);
      if (!pre) cp_commit_wait();
      g.sync();
    }
    if (kind == 0) {
      if (conj_layout) {
        vlike<T, F, RC, true>(M0, I0, k0, c0, vv, W, out0, R, r0, re, nst, g);
        if (nblk == 2) vlike<T, F, RC, true>(M1, I1, k1, c1, vv, W, out1, R, r0, re, nst, g);
      } else {
        vlike<T, F, RC, false>(M0, I0, k0, c0, vv, W, out0, R, r0, re, nst, g);
        if (nblk == 2) vlike<T, F, RC, false>(M1, I1, k1, c1, vv, W, out1, R, r0, re, nst, g);
      }
    } else if (kind == 1) {
      const int nrows = c0;   // candidate entries (both blocks of an item share the candidate list)
      for (int e = g.t; e < nrows * nst; e += g.nt) {
        const int r = e % nrows, ch = e / nrows;
        const int64_t rs = r0 + (int64_t)ch * RC;
        const int rc = (re - rs) < RC ? (int)(re - rs) : RC;
        const C* y0 = vv + ch * RC;
        const C* y1 = vv + (int64_t)n_s0 * W + ch * RC;
        C acc[RC];
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
        if (conj_layout) {
          rowc<T, F, RC, true>(acc, M0, I0, k0, c0, y0, W, r);
          if (nblk == 2) rowc<T, F, RC, true>(acc, M1, I1, k1, c1, y1, W, r);
        } else {
          rowc<T, F, RC, false>(acc, M0, I0, k0, c0, y0, W, r);
          if (nblk == 2) rowc<T, F, RC, false>(acc, M1, I1, k1, c1, y1, W, r);
        }
        C* d = (nblk == 1 || r < split_r) ? out0 + (int64_t)r * R + rs : out1 + (int64_t)(r - split_r) * R + rs;
#pragma unroll
        for (int rr = 0; rr < RC; ++rr)
          if (rr < rc) {
            if (subtract) {
              C cur = ldcg2(d + rr);
              d[rr] = C{cur.x - acc[rr].x, cur.y - acc[rr].y};
            } else {
              d[rr] = acc[rr];
            }
          }
      }
    } else {
      const int nin = adj ? kr : kc, nout = adj ? kc : kr;
      for (int e = g.t; e < nout * nst; e += g.nt) {
        const int oo = e % nout, ch = e / nout;
        const int64_t rs = r0 + (int64_t)ch * RC;
        const int rc = (re - rs) < RC ? (int)(re - rs) : RC;
        const C* vb = vv + ch * RC;
        C acc[RC];
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
#pragma unroll 8
        for (int i = 0; i < nin; ++i) {
          C sv = adj ? cvc<T>(Ms[(int64_t)oo * kr + i]) : cv<T>(Ms[(int64_t)i * kr + oo]);
#pragma unroll
          for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], sv, vb[(int64_t)i * W + rr]);
        }
#pragma unroll
        for (int rr = 0; rr < RC; ++rr)
          if (rr < rc) out0[(int64_t)oo * R + rs + rr] = acc[rr];
      }
    }
    if (!pl.once) g.sync();
  }
  if (pl.once) g.sync();
}

// Sweep-leaf product x = T b, T the packed triangle of order s of the op
// (lower, or upper with FF_UPPER), column-packed.  Thread (pair j, group g)
// owns rows j and s-1-j (together s+1 triangle entries, so every thread has
// the same share) and sums the columns c = g, g + ngrp, ... of each row inside
// the triangle; for a fixed column consecutive threads read consecutive
// entries.  part: ngrp * s * RC partial sums; b: the s input rows (stride W,
// columns of this pass); results replace the rows of out (stride Wo) after a
// barrier, so out may alias b.
template <class T, class F, int RC>
__device__ __forceinline__ void tri_pass(const F* Tm, int s, bool upper, const typename CT<T>::t* b, int64_t W,
                                         typename CT<T>::t* out, int64_t Wo, int rc, typename CT<T>::t* part,
                                         const Grp& gt) {
  using C = typename CT<T>::t;
  const int npair = s > 1 ? s / 2 : 1;
  const int ngrp = gt.nt / npair > 0 ? gt.nt / npair : 1;
  for (int e = gt.t; e < ngrp * npair; e += gt.nt) {
    const int j = e % npair, g = e / npair;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h == 0 ? j : s - 1 - j;
      if (h == 1 && r == j) break;   // s == 1
      C acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
      if (upper) {
        // row r: columns r .. s-1, entry (r, c) at c (c + 1) / 2 + r
        int c = r + ((g - r % ngrp) + ngrp) % ngrp;
#pragma unroll 4
        for (; c < s; c += ngrp) {
          const C m = cv<T>(Tm[(c * (c + 1) >> 1) + r]);
#pragma unroll
          for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], m, b[(int64_t)c * W + rr]);
        }
      } else {
        // row r: columns 0 .. r, entry (r, c) at c s - c (c - 1) / 2 + r - c
#pragma unroll 4
        for (int c = g; c <= r; c += ngrp) {
          const C m = cv<T>(Tm[c * s - ((c * (c - 1)) >> 1) + r - c]);
#pragma unroll
          for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], m, b[(int64_t)c * W + rr]);
        }
      }
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) part[(g * s + r) * RC + rr] = acc[rr];
    }
  }
  gt.sync();
  for (int e = gt.t; e < s * RC; e += gt.nt) {
    const int r = e / RC, rr = e % RC;
    C sum = z2<T>();
    for (int g = 0; g < ngrp; ++g) { sum.x += part[(g * s + r) * RC + rr].x; sum.y += part[(g * s + r) * RC + rr].y; }
    if (rr < rc) out[(int64_t)r * Wo + rr] = sum;
  }
  gt.sync();
}

// sweep-leaf solve of a run kept in global memory: whole CTA, columns [rb, re)
template <class T, class F, int RC>
__device__ void do_leaf(const SweepArgs& a, const FlatOp& f, char* buf, int64_t buf_bytes, int64_t rb, int64_t re) {
  using C = typename CT<T>::t;
  const int s = f.c0;
  const int64_t R = a.R;
  const Grp g{(int)threadIdx.x, (int)blockDim.x, true};
  const F* Tg = (const F*)a.tinv + f.moff;
  C* v = (C*)a.vec + (int64_t)f.src0 * R;
  const bool upper = (f.flags & FF_UPPER) != 0;
  const int npair = s > 1 ? s / 2 : 1;
  const int ngrp = g.nt / npair > 0 ? g.nt / npair : 1;
  const int64_t mb = align16((int64_t)f.melems * (int64_t)sizeof(F));
  const int64_t partb = align16((int64_t)ngrp * s * RC * (int64_t)sizeof(C));
  const int64_t vb = (int64_t)s * RC * (int64_t)sizeof(C);
  const F* Tm = Tg;
  char* area = buf;
  if (mb + partb + vb <= buf_bytes) {
    stage(buf, Tg, mb, g);
    Tm = (const F*)buf;
    area = buf + mb;
  }
  C* part = (C*)area;
  C* bb = (C*)(area + partb);
  for (int64_t r0 = rb; r0 < re; r0 += RC) {
    const int rc = (re - r0) < RC ? (int)(re - r0) : RC;
    stage_vec<C>(bb, v, s, R, r0, rc, RC, g, true);
    cp_commit_wait();
    __syncthreads();
    tri_pass<T, F, RC>(Tm, s, upper, bb, RC, v + r0, R, rc, part, g);
  }
}

// ---------------------------------------------------------------------------
// Resident single-CTA runs with a staging ring (complex FP32 factors, sweep
// leaves of <= 256 rows).  The run's vector rows and butterfly state live in
// shared memory for the whole run, and its op records and phase table are
// copied in once.  A producer warp copies the factor data of the coming phases
// (each phase's ops packed into one contiguous area, offsets precomputed on
// the host) into a ring buffer with cp.async.bulk, one mbarrier per phase slot,
// up to kLook phases ahead of the compute warps and as far as the ring has
// room; so only shared-memory work and barriers remain on the dependency chain.
// Shared-memory map: [ring | op records | phase table | sweep-leaf partial
// sums | resident rows + state].
// ---------------------------------------------------------------------------
constexpr int kSmemBytes = 224 * 1024;
constexpr int kAuxBytes = 16 * 1024;                                    // sweep-leaf partial sums
constexpr int kRecBytes = kRunMaxOps * 64;                              // the run's op records (48 KB)
constexpr int kPhBytes = (kRunMaxPhases + 1) * 8;                       // the run's phase table (4 KB)
constexpr int kRingBytes = kSmemBytes - kAuxBytes - kResidentBytes - kRecBytes - kPhBytes;   // 100 KB
constexpr int kLook = 7;                                                // phases in flight beyond the current one

// ---- mbarrier + bulk-copy helpers (one thread issues a phase's copies)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* b) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(b)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
  return ok != 0;
}
// OR of v over the nt threads of named barrier id (also a barrier among them)
__device__ __forceinline__ bool bar_red_or(bool v, int id, int nt) {
  unsigned r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
               : "=r"(r) : "r"((unsigned)v), "r"(id), "r"(nt) : "memory");
  return r != 0;
}
// bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned), completion on mbarrier b
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}

// issue the bulk copies of one phase's factor data (ops[0 .. nops), total
// `bytes`) into dst, completing on mbarrier b (one warp; lane o issues op o)
template <class F>
__device__ void ring_issue(const SweepArgs& a, const FlatOp* ops, int nops, char* dst, unsigned bytes, uint64_t* b,
                           int lane) {
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // earlier generic reads of the area come first
    mbar_arrive_tx(b, bytes);
  }
  __syncwarp();
  if (ops[0].kind == FK_LEAF) {
    if (lane == 0)
      bulk_g2s(dst, (const F*)a.tinv + ops[0].moff, (unsigned)align16((int64_t)ops[0].melems * (int64_t)sizeof(F)), b);
    return;
  }
  for (int o = lane; o < nops; o += 32) {
    const FlatOp& f = ops[o];
    char* d = dst + f.soff;
    const unsigned mb = (unsigned)align16((int64_t)f.melems * (int64_t)sizeof(F));
    bulk_g2s(d, (const F*)a.fp + f.moff, mb, b);
    if (f.ioff >= 0) bulk_g2s(d + mb, a.ip + f.ioff, (unsigned)align16((int64_t)f.ielems * (int64_t)sizeof(int16_t)), b);
  }
}

// An op of a resident run: operands and results live in shared memory (rows
// of stride Wr, columns = the CTA's right-hand sides), the factor data is
// either prefetched into `half` (pre) or read from global memory.
// SM: the factor data was staged into shared memory (pre); the compiler is
// told that every operand of the op is then a shared-memory address.
template <class T, class F, int RC, bool SM>
__device__ void do_op_res(const SweepArgs& a, const FlatOp& f, const char* half, bool pre,
                          typename CT<T>::t* rvec, int row_lo, typename CT<T>::t* rst, int st_lo, int Wr, int ncol,
                          const Grp& g) {
  using C = typename CT<T>::t;
  __builtin_assume(__isShared(rvec));
  __builtin_assume(__isShared(rst));
  if (SM) __builtin_assume(__isShared(half));
  const bool conj_layout = (f.flags & FF_CONJ) != 0;
  const bool subtract = (f.flags & FF_SUB) != 0;
  const bool adj = (f.flags & FF_ADJ) != 0;
  const int nblk = (f.flags & FF_TWO) ? 2 : 1;
  const C* src0 = (f.flags & FF_SRC_VEC) ? rvec + (int64_t)(f.src0 - row_lo) * Wr : rst + (int64_t)(f.src0 - st_lo) * Wr;
  const C* src1 = rst + (int64_t)(f.src1 - st_lo) * Wr;
  C* out0 = (f.flags & FF_OUT_VEC) ? rvec + (int64_t)(f.out0 - row_lo) * Wr : rst + (int64_t)(f.out0 - st_lo) * Wr;
  C* out1 = rst + (int64_t)(f.out1 - st_lo) * Wr;
  const int64_t mbytes = align16((int64_t)f.melems * (int64_t)sizeof(F));
  const F* Ms = pre ? (const F*)half : (const F*)a.fp + f.moff;
  const int16_t* Is = pre ? (const int16_t*)(half + mbytes) : (f.ioff >= 0 ? a.ip + f.ioff : nullptr);
  const F* M1 = Ms + f.m1;
  const int16_t* I1 = Is ? Is + f.i1 : nullptr;
  if (SM) {
    __builtin_assume(__isShared(Ms));
    __builtin_assume(__isShared(M1));
    if (Is) __builtin_assume(__isShared(Is));
    if (I1) __builtin_assume(__isShared(I1));
  }
  const int nch = (ncol + RC - 1) / RC;
  if (f.kind == FK_GATHER) {
    if (conj_layout) {
      vlike<T, F, RC, true>(Ms, Is, f.k0, f.c0, src0, Wr, out0, Wr, 0, ncol, nch, g);
      if (nblk == 2) vlike<T, F, RC, true>(M1, I1, f.k1, f.c1, src0, Wr, out1, Wr, 0, ncol, nch, g);
    } else {
      vlike<T, F, RC, false>(Ms, Is, f.k0, f.c0, src0, Wr, out0, Wr, 0, ncol, nch, g);
      if (nblk == 2) vlike<T, F, RC, false>(M1, I1, f.k1, f.c1, src0, Wr, out1, Wr, 0, ncol, nch, g);
    }
  } else if (f.kind == FK_SCATTER) {
    const int split_r = f.split;
    for (int e = g.t; e < f.c0 * nch; e += g.nt) {
      const int r = e % f.c0, ch = e / f.c0;
      const int r0 = ch * RC;
      const int rc = (ncol - r0) < RC ? (ncol - r0) : RC;
      C acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
      if (conj_layout) {
        rowc<T, F, RC, true>(acc, Ms, Is, f.k0, f.c0, src0 + r0, Wr, r);
        if (nblk == 2) rowc<T, F, RC, true>(acc, M1, I1, f.k1, f.c1, src1 + r0, Wr, r);
      } else {
        rowc<T, F, RC, false>(acc, Ms, Is, f.k0, f.c0, src0 + r0, Wr, r);
        if (nblk == 2) rowc<T, F, RC, false>(acc, M1, I1, f.k1, f.c1, src1 + r0, Wr, r);
      }
      C* d = (nblk == 1 || r < split_r) ? out0 + (int64_t)r * Wr + r0 : out1 + (int64_t)(r - split_r) * Wr + r0;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) {
          if (subtract) d[rr] = C{d[rr].x - acc[rr].x, d[rr].y - acc[rr].y};
          else d[rr] = acc[rr];
        }
    }
  } else {   // middle
    const int kr = f.k0, kc = f.c0;
    const int nin = adj ? kr : kc, nout = adj ? kc : kr;
    for (int e = g.t; e < nout * nch; e += g.nt) {
      const int oo = e % nout, ch = e / nout;
      const int r0 = ch * RC;
      const int rc = (ncol - r0) < RC ? (ncol - r0) : RC;
      C acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
#pragma unroll 8
      for (int i = 0; i < nin; ++i) {
        C sv = adj ? cvc<T>(Ms[(int64_t)oo * kr + i]) : cv<T>(Ms[(int64_t)i * kr + oo]);
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], sv, src0[(int64_t)i * Wr + r0 + rr]);
      }
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) out0[(int64_t)oo * Wr + r0 + rr] = acc[rr];
    }
  }
  g.sync();
}

// sweep-leaf solve of a resident run: rows in shared memory, triangle staged (or global)
template <class T, class F, int RC, bool SM>
__device__ void do_leaf_res(const SweepArgs& a, const FlatOp& f, const F* Tm, typename CT<T>::t* rvec, int row_lo,
                            int Wr, int ncol, typename CT<T>::t* part, const Grp& gt) {
  using C = typename CT<T>::t;
  __builtin_assume(__isShared(rvec));
  __builtin_assume(__isShared(part));
  if (SM) __builtin_assume(__isShared(Tm));
  const int s = f.c0;
  const bool upper = (f.flags & FF_UPPER) != 0;
  C* v = rvec + (int64_t)(f.src0 - row_lo) * Wr;
  // the pass reads all of b before any row is written (a barrier separates them)
  for (int r0 = 0; r0 < ncol; r0 += RC) {
    const int rc = (ncol - r0) < RC ? (ncol - r0) : RC;
    tri_pass<T, F, RC>(Tm, s, upper, v + r0, Wr, v + r0, Wr, rc, part, gt);
  }
}

// bring a run's op and phase records into L1 (static data, one round trip)
__device__ __forceinline__ void prefetch_records(const SweepArgs& a, const DSeg& sg) {
  const int32_t o_first = __ldg(a.flat_base + sg.first), o_last = __ldg(a.flat_base + sg.first + sg.count);
  const char* p0 = (const char*)(a.flat + o_first);
  const int64_t nb = (int64_t)(o_last - o_first) * (int64_t)sizeof(FlatOp);
  for (int64_t e = (int64_t)threadIdx.x * 128; e < nb; e += (int64_t)blockDim.x * 128)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p0 + e));
  const char* p1 = (const char*)(a.flat_base + sg.first);
  const char* p2 = (const char*)(a.flat_pbytes + sg.first);
  for (int64_t e = (int64_t)threadIdx.x * 128; e < (int64_t)(sg.count + 1) * 4; e += (int64_t)blockDim.x * 128) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p1 + e));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p2 + e));
  }
}

// resident run with the staging ring (columns [lb, le) of this CTA); the
// run's op records and phase table are copied to shared memory first, so no
// phase waits on a record load from L2
template <class T, class F, int RC>
__device__ bool local_run_ring(const SweepArgs& a, const DSeg& sg, char* smem, int64_t lb, int64_t le,
                               int32_t o_first, int32_t o_last) {
  using C = typename CT<T>::t;
  __shared__ int s_qoff[kLook + 1];   // ring offset of each phase in flight (-1: read from global memory)
  __shared__ __align__(8) uint64_t s_mbar[kLook + 1];   // completion of each phase slot's bulk copies
  __shared__ int s_done;    // phases finished by the compute warps
  __shared__ int s_abort;   // a bounded wait gave up
  __shared__ int s_issued;  // phases the producer issued
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  const int np = sg.count;
  char* ring = smem;
  FlatOp* recs = (FlatOp*)(smem + kRingBytes);
  int32_t* sbase = (int32_t*)(smem + kRingBytes + kRecBytes);   // [np + 1] first op of each phase
  int32_t* spb = sbase + (kRunMaxPhases + 1);                      // [np] staging bytes of each phase
  C* part = (C*)(smem + kRingBytes + kRecBytes + kPhBytes);
  C* rvec = (C*)(smem + kRingBytes + kRecBytes + kPhBytes + kAuxBytes);
  const int ncol = (int)(le - lb);
  const int Wr = ((ncol + RC - 1) / RC) * RC;
  C* rst = rvec + (int64_t)(sg.row_hi - sg.row_lo) * Wr;
  C* vecg = (C*)a.vec;
  {
    const Grp g{(int)threadIdx.x, (int)blockDim.x, true};
    stage(recs, a.flat + o_first, (int64_t)(o_last - o_first) * (int64_t)sizeof(FlatOp), g);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int p = threadIdx.x; p <= np; p += blockDim.x) {
    sbase[p] = __ldg(a.flat_base + sg.first + p) - o_first;
    if (p < np) spb[p] = __ldg(a.flat_pbytes + sg.first + p);
  }
  const int nrow = sg.row_hi - sg.row_lo;
  for (int e = threadIdx.x; e < nrow * ncol; e += blockDim.x) {
    const int r = e / ncol, c = e % ncol;
    rvec[(int64_t)r * Wr + c] = ldcg2(vecg + (int64_t)(sg.row_lo + r) * a.R + lb + c);
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k <= kLook; ++k) mbar_init(&s_mbar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) { s_done = 0; s_abort = 0; s_issued = 0; }
  __syncthreads();
  bool ok = true;
  const int cw = nw - 1;                 // compute warps; the last warp is the producer
  if (warp == cw) {
    // ---- producer: stage phases ahead of the compute warps.  Ring state:
    // next phase to issue, allocation head; phases [done, issued) are in
    // flight (their ring areas in use).
    int issued = 0, head = 0;
    long long spins = 0;
    while (issued < np) {
      const int done = *(volatile int*)&s_done;
      __threadfence_block();   // pairs with the compute warps' fence before they publish s_done
      if (*(volatile int*)&s_abort) break;
      bool go = issued - done <= kLook;
      int off = -1;
      const int pb = spb[issued];
      if (go && pb > 0 && pb <= kRingBytes) {
        // oldest staged phase still in use
        int tail = -1;
        for (int q = done; q < issued; ++q) {
          const int o2 = s_qoff[q % (kLook + 1)];
          if (o2 >= 0) { tail = o2; break; }
        }
        if (tail < 0) {
          head = 0;
          off = 0;
        } else if (head > tail) {
          if (head + pb <= kRingBytes) off = head;
          else if (pb <= tail) off = 0;
        } else if (head < tail) {
          if (head + pb <= tail) off = head;
        }
        go = off >= 0;
      }
      if (!go) {   // wait for the compute warps to release a phase (bounded)
        if (++spins > a.spin_limit) { if (lane == 0) atomicExch(&s_abort, 1); break; }
        __nanosleep(32);
        continue;
      }
      spins = 0;
      uint64_t* mb = &s_mbar[issued % (kLook + 1)];
      if (lane == 0) s_qoff[issued % (kLook + 1)] = off;   // published by the barrier arrive below
      __syncwarp();
      if (off >= 0) {
        ring_issue<F>(a, recs + sbase[issued], sbase[issued + 1] - sbase[issued], ring + off, (unsigned)pb, mb, lane);
        head = off + pb;
      } else if (lane == 0) {
        mbar_arrive_tx(mb, 0);   // nothing staged: complete the slot's phase
      }
      ++issued;
    }
    if (lane == 0) s_issued = issued;
    __syncwarp();
  } else {
    // ---- compute warps (named barrier 1 among them)
    const Grp gc{(int)threadIdx.x, cw * 32, false, 1};
    int ph = 0;
    for (; ph < np; ++ph) {
      uint64_t* mb = &s_mbar[ph % (kLook + 1)];
      const unsigned par = (unsigned)(ph / (kLook + 1)) & 1u;
      long long spins = 0;
      while (!mbar_try_wait(mb, par)) {
        if (++spins > a.spin_limit || *(volatile int*)&s_abort) { ok = false; break; }
      }
      // uniform decision among the compute warps (the OR-reduction is their barrier)
      if (bar_red_or(!ok, gc.bar, gc.nt)) {
        ok = false;
        if (threadIdx.x == 0) atomicExch(&s_abort, 1);
        break;
      }
      const int myoff = s_qoff[ph % (kLook + 1)];
      const FlatOp* ops = recs + sbase[ph];
      const int nops = sbase[ph + 1] - sbase[ph];
      if (ops[0].kind == FK_LEAF) {
        if (myoff >= 0)
          do_leaf_res<T, F, RC, true>(a, ops[0], (const F*)(ring + myoff), rvec, sg.row_lo, Wr, ncol, part, gc);
        else
          do_leaf_res<T, F, RC, false>(a, ops[0], (const F*)a.tinv + ops[0].moff, rvec, sg.row_lo, Wr, ncol, part, gc);
      } else {
        const Grp g{lane, 32, false};
        for (int o = warp; o < nops; o += cw) {
          const FlatOp& f = ops[o];
          if (myoff >= 0)
            do_op_res<T, F, RC, true>(a, f, ring + myoff + f.soff, true, rvec, sg.row_lo, rst, sg.st_lo, Wr, ncol, g);
          else
            do_op_res<T, F, RC, false>(a, f, ring, false, rvec, sg.row_lo, rst, sg.st_lo, Wr, ncol, g);
        }
      }
      gc.sync();
      if (threadIdx.x == 0) {
        __threadfence_block();
        *(volatile int*)&s_done = ph + 1;   // releases the phase's slot and ring area
      }
    }
  }
  __syncthreads();
  ok = *(volatile int*)&s_abort == 0;
  if (!ok) {
    // a wait gave up: report, then give the copies in flight a second bounded
    // wait before the shared memory is left
    if (threadIdx.x == 0) atomicExch(&a.bar->err, 1);
    const int done = s_done, iss = s_issued;
    for (int q = done; q < iss; ++q) {
      long long spins = 0;
      while (!mbar_try_wait(&s_mbar[q % (kLook + 1)], (unsigned)(q / (kLook + 1)) & 1u) && ++spins < drain_limit(a.spin_limit)) {
      }
    }
  }
  for (int e = threadIdx.x; e < nrow * ncol; e += blockDim.x) {
    const int r = e / ncol, c = e % ncol;
    vecg[(int64_t)(sg.row_lo + r) * a.R + lb + c] = rvec[(int64_t)r * Wr + c];
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k <= kLook; ++k) mbar_inval(&s_mbar[k]);
  __syncthreads();
  return ok;
}

// run kept in global memory: operands staged per op into warp slices
template <class T, class F, int RC>
__device__ void local_run_plain(const SweepArgs& a, const DSeg& sg, char* smem, int64_t slice, int64_t lb,
                                int64_t le) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  prefetch_records(a, sg);
  for (int ph = sg.first; ph < sg.first + sg.count; ++ph) {
    const int32_t ob = __ldg(a.flat_base + ph), oe = __ldg(a.flat_base + ph + 1);
    const FlatOp* ops = a.flat + ob;
    if (ops[0].kind == FK_LEAF) {
      do_leaf<T, F, RC>(a, ops[0], smem, a.smem_bytes, lb, le);
    } else {
      const Grp g{lane, 32, false};
      for (int o = warp; o < oe - ob; o += nw) do_op<T, F, RC>(a, ops[o], smem + warp * slice, slice, g, lb, le);
      __syncthreads();
    }
  }
}

template <class T, class F, int RC>
__global__ void __launch_bounds__(256, 1) k_sweep_coop(SweepArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  unsigned my_gen = 0;
  const int64_t slice = (a.smem_bytes / nw) & ~(int64_t)15;
  // local runs: the right-hand sides are split over the CTAs; CTA b owns
  // [lb, le) (q = ceil(R / #CTAs) columns).  With one right-hand side only CTA 0 works.
  const int64_t q = (a.R + gridDim.x - 1) / gridDim.x;
  const int64_t lb = (int64_t)blockIdx.x * q;
  const int64_t le = (lb + q < a.R) ? lb + q : a.R;
  for (int s = 0; s < a.nseg; ++s) {
    const DSeg sg = a.segs[s];
    if (sg.grid) {
      const DPhase P = a.prog[sg.first];
      const FlatOp* ops = a.flat + a.flat_base[sg.first];
      if (a.R <= 4 && (int64_t)P.mbytes / (16 / (int)sizeof(F)) + (int64_t)P.vmax * RC * (int64_t)sizeof(typename CT<T>::t) <= slice) {
        // few right-hand sides and ops that fit a warp's slice: one op per warp over the whole grid
        const Grp g{lane, 32, false};
        const int gw = blockIdx.x * nw + warp, tw = gridDim.x * nw;
        for (int o = gw; o < P.count; o += tw) do_op<T, F, RC>(a, ops[o], smem + warp * slice, slice, g, 0, a.R);
      } else {
        // (op, column range) units over the workers: with many right-hand
        // sides each CTA runs kGroups groups of two warps (named barriers,
        // own shared-memory slice), so several units' staging latencies
        // overlap; a unit's columns are cut so that its staged operands fit
        // the slice, and a phase with fewer ops than workers splits its
        // right-hand sides further (ranges of >= 16 columns)
        constexpr int kGroups = 4;
        const int G = a.R >= 32 ? kGroups : 1;
        const int gsz = (int)blockDim.x / G, gi = (int)threadIdx.x / gsz;
        const Grp g{(int)threadIdx.x % gsz, gsz, G == 1, G == 1 ? 0 : 1 + gi};
        const int64_t gslice = ((int64_t)a.smem_bytes / G) & ~(int64_t)15;
        const int64_t workers = (int64_t)gridDim.x * G;
        const int64_t mbf = (int64_t)P.mbytes / (16 / (int)sizeof(F)) + 64;
        const int64_t colb = (int64_t)(P.vmax > 0 ? P.vmax : 1) * (int64_t)sizeof(typename CT<T>::t);
        int64_t wfit = (gslice - mbf) / colb;
        wfit = wfit < RC ? RC : wfit / RC * RC;
        int64_t nu = (a.R + wfit - 1) / wfit;
        if ((int64_t)P.count * nu < workers && a.R >= 32) {
          int64_t want = (workers + P.count - 1) / P.count;
          const int64_t maxu = a.R / 16;
          if (want > maxu) want = maxu;
          if (want > nu) nu = want;
        }
        int64_t wg = ((a.R + nu - 1) / nu + RC - 1) / RC * RC;
        nu = (a.R + wg - 1) / wg;
        const int64_t units = (int64_t)P.count * nu;
        char* gbuf = smem + gi * gslice;
        for (int64_t u = (int64_t)blockIdx.x * G + gi; u < units; u += workers) {
          const int o = (int)(u / nu);
          const int64_t rb = (u % nu) * wg;
          const int64_t re = (rb + wg < a.R) ? rb + wg : a.R;
          do_op<T, F, RC>(a, ops[o], gbuf, gslice, g, rb, re);
        }
        if (G > 1) __syncthreads();
      }
    } else if (lb < le) {
      const int64_t ncol = le - lb, Wr = (ncol + RC - 1) / RC * RC;
      const int64_t res_need = ((int64_t)(sg.row_hi - sg.row_lo) + (sg.st_hi - sg.st_lo)) * Wr *
                               (int64_t)sizeof(typename CT<T>::t);
      bool ring = a.use_pf && !sg.st_cross && res_need <= kResidentBytes && sg.count <= kRunMaxPhases;
      int32_t o_first = 0, o_last = 0;
      if (ring) {
        o_first = __ldg(a.flat_base + sg.first);
        o_last = __ldg(a.flat_base + sg.first + sg.count);
        ring = o_last - o_first <= kRunMaxOps;
      }
      if (ring) {
        if (!local_run_ring<T, F, RC>(a, sg, smem, lb, le, o_first, o_last)) return;
      } else {
        local_run_plain<T, F, RC>(a, sg, smem, slice, lb, le);
      }
    }
    // Two consecutive single-CTA runs need no grid barrier: each CTA only
    // reads there the columns it wrote itself.  No barrier after the last segment.
    if (s + 1 < a.nseg && (sg.grid || a.segs[s + 1].grid))
      if (!grid_sync(a.bar, my_gen, a.spin_limit)) return;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------
static int coop_launch_dims(int& grid) {
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  grid = sms > 0 ? sms : 1;
  return HB_OK;
}

template <class T, class F, int RC>
static int sweep_coop_impl(const DevFactor& df, int which, void* vec, int64_t R, void* st, void* bar,
                           cudaStream_t s, long long spin_limit) {
  int grid = 0;
  coop_launch_dims(grid);
  const int smem = kSmemBytes;
  auto kern = k_sweep_coop<T, F, RC>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr_done = true;
  }
  SweepArgs a;
  const int cls = R > 1 ? 1 : 0;
  if (df.tuned[cls] >= 0) {
    a.segs = df.cand_segs[cls][which][df.tuned[cls]];
    a.nseg = df.cand_nsegs[cls][which][df.tuned[cls]];
  } else {
    a.segs = df.segs[which];
    a.nseg = df.nsegs[which];
  }
  a.prog = df.prog[which];
  a.flat = df.flat[which];
  a.flat_base = df.flat_base[which];
  a.flat_pbytes = df.flat_pbytes[which];
  a.n0 = df.n0;
  a.bvout = df.bvout;
  a.buout = df.buout;
  a.bf_vout0 = df.bf_vout0;
  a.bf_uout0 = df.bf_uout0;
  a.items = df.items;
  a.fp = df.fpool;
  a.ip = df.ipool;
  a.tinv = df.sl[which];
  a.vec = vec;
  a.st = st;
  a.R = R;
  a.bar = (GridBar*)bar;
  a.smem_bytes = 192 * 1024;
  a.spin_limit = spin_limit;
  // resident runs with the staging ring: complex FP32 factors, sweep leaves of
  // at most 256 rows, and the sweep-leaf product's partial sums (2 x 256 rows
  // of RC columns) within the scratch area
  a.use_pf = (sizeof(F) == 8 && df.sl_n <= 256 &&
              2 * 256 * RC * (int64_t)sizeof(typename CT<T>::t) <= kAuxBytes) ? 1 : 0;
  // reset count and generation; the error flag stays set until hb_status reads it
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) return HB_ECUDA;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, smem, s);
  if (e != cudaSuccess) {
    set_error("cooperative sweep launch failed: %s", cudaGetErrorString(e));
    return HB_ECUDA;
  }
  return HB_OK;
}

}  // namespace hb

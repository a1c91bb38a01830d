// Hot-path CUDA kernels (sm_103a): H-IDBF apply (Alg. 2), forward and adjoint.
// (The L~ / U~ sweeps of Algs. 3, 4 live in hb_sweep.cu.)
//
// Every butterfly factor is a set of small ID blocks (Sec. 2 / Appendix).  A
// warp owns one block op; lanes run over the op's OUTPUT entries and loop over
// its inputs, so factor loads are coalesced (the packer stores every matrix
// with the output index fastest) and input entries are warp-wide broadcasts.
//   vlike  (V stage, column ID):  z_i  = cand[q_i] + sum_j T_ij cand[p_j]
//   ulike  (U stage, row ID):     out_r = y_{map r}            (r skeleton)
//                                 out_r = sum_i T_i,j(r) y_i   (r redundant)
//   middle:                       y = S z
// Adjoint ops swap the two shapes and conjugate the entries.
// Vectors and the butterfly state use the layout [entry][R] (RHS fastest);
// one op handles RC right-hand sides per pass.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hb_device.h"

namespace hb {

template <class T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

// Double-float numbers (a pair of FP32 values, about 48 significant bits): the
// FP64-accurate arithmetic of the complex-FP32 factors' refinement residual at
// FP32 instruction rates (FP64 runs at a small fraction of them on this GPU).
// The product uses the exact FMA residual of the high parts (Dekker / Knuth
// two-product with FMA), the sum the two-sum of the high parts with the low
// parts added; both renormalised.
struct Dd {
  float h, l;
  __host__ __device__ Dd(float v = 0.f) : h(v), l(0.f) {}
  __host__ __device__ Dd(float hi, float lo) : h(hi), l(lo) {}
};
struct __align__(16) DdC {
  Dd x, y;
};
template <> struct C2<Dd> { using t = DdC; };
__device__ __forceinline__ Dd dd_norm(float s, float e) {
  const float t = s + e;
  return Dd(t, e - (t - s));
}
__device__ __forceinline__ Dd operator-(const Dd& a) { return Dd(-a.h, -a.l); }
__device__ __forceinline__ Dd dd_add(const Dd& a, const Dd& b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = ((a.h - (s - bb)) + (b.h - bb)) + (a.l + b.l);
  return dd_norm(s, e);
}
__device__ __forceinline__ Dd& operator+=(Dd& a, const Dd& b) { a = dd_add(a, b); return a; }
// c + a * b
__device__ __forceinline__ Dd dd_fma(const Dd& a, const Dd& b, const Dd& c) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return dd_add(c, dd_norm(p, e));
}

template <class T> __device__ __forceinline__ typename C2<T>::t mk(T a, T b) { return {a, b}; }

template <class T, class F>
__device__ __forceinline__ typename C2<T>::t ldf(const F* p) {
  F v = __ldg(p);
  return mk<T>((T)v.x, (T)v.y);
}
template <class T, class F>
__device__ __forceinline__ typename C2<T>::t ldf_conj(const F* p) {
  F v = __ldg(p);
  return mk<T>((T)v.x, -(T)v.y);
}
// acc += a * b
template <class C>
__device__ __forceinline__ void cfma(C& acc, const C& a, const C& b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(DdC& acc, const DdC& a, const DdC& b) {
  acc.x = dd_fma(a.x, b.x, acc.x);
  acc.x = dd_fma(-a.y, b.y, acc.x);
  acc.y = dd_fma(a.x, b.y, acc.y);
  acc.y = dd_fma(a.y, b.x, acc.y);
}
template <class C>
__device__ __forceinline__ void cadd(C& acc, const C& a) {
  acc.x += a.x;
  acc.y += a.y;
}

// ---------------------------------------------------------------------------
// Block ops (one warp).  R = row stride of the [entry][R] layout, r0 = first
// RHS of this pass, rc = number of valid RHS in the pass (<= RC).
// ---------------------------------------------------------------------------

// B side (k outputs) = gather + T * rest of the candidate vector cand =
// concat(a0[0..ka0), a1[..]).  UTYPE_ADJ: the block is a row ID used in
// adjoint (entries conj(T_ij) read from the U-type layout M[i*(c-k)+j]);
// otherwise a column ID (V-type layout M[j*k+i]).
template <class T, class F, int RC, bool UTYPE_ADJ>
__device__ __forceinline__ void op_vlike(const F* __restrict__ M, const int16_t* __restrict__ idx, int k, int c,
                                         const typename C2<T>::t* a0, int ka0, const typename C2<T>::t* a1,
                                         typename C2<T>::t* out, int64_t R, int64_t r0, int rc, int lane) {
  using C = typename C2<T>::t;
  const int nr = c - k;
  for (int i = lane; i < k; i += 32) {
    C acc[RC];
    const int qi = idx[i];
    const C* src = (qi < ka0) ? a0 + (int64_t)qi * R : a1 + (int64_t)(qi - ka0) * R;
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr] = (rr < rc) ? src[r0 + rr] : mk<T>(0, 0);
#pragma unroll 4
    for (int j = 0; j < nr; ++j) {
      C mij = UTYPE_ADJ ? ldf_conj<T>(M + (int64_t)i * nr + j) : ldf<T>(M + (int64_t)j * k + i);
      const int pj = idx[k + j];
      const C* s = (pj < ka0) ? a0 + (int64_t)pj * R : a1 + (int64_t)(pj - ka0) * R;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) cfma(acc[rr], mij, s[r0 + rr]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
      if (rr < rc) out[(int64_t)i * R + r0 + rr] = acc[rr];
  }
}

// Contribution of one block to candidate entry r: VTYPE_ADJ: the block is a
// column ID used in adjoint (conj(T_ij) from M[j*k+i]); otherwise a row ID
// (U-type layout M[i*(c-k)+j]).
template <class T, class F, int RC, bool VTYPE_ADJ>
__device__ __forceinline__ void row_contrib(typename C2<T>::t (&acc)[RC], const F* __restrict__ M,
                                            const int16_t* __restrict__ idx, int k, int c,
                                            const typename C2<T>::t* y, int64_t R, int64_t r0, int rc, int r) {
  using C = typename C2<T>::t;
  const int code = idx[c + r];
  if (code >= 0) {
    const C* s = y + (int64_t)code * R + r0;
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
      if (rr < rc) cadd(acc[rr], s[rr]);
  } else {
    const int j = -1 - code;
    const int nr = c - k;
#pragma unroll 4
    for (int i = 0; i < k; ++i) {
      C mij = VTYPE_ADJ ? ldf_conj<T>(M + (int64_t)j * k + i) : ldf<T>(M + (int64_t)i * nr + j);
      const C* s = y + (int64_t)i * R + r0;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) cfma(acc[rr], mij, s[rr]);
    }
  }
}

template <class T, class F, int RC>
__device__ __forceinline__ void op_middle(const F* __restrict__ S, int kr, int kc, bool adj,
                                          const typename C2<T>::t* in, typename C2<T>::t* out, int64_t R,
                                          int64_t r0, int rc, int lane) {
  using C = typename C2<T>::t;
  const int nout = adj ? kc : kr, nin = adj ? kr : kc;
  for (int o = lane; o < nout; o += 32) {
    C acc[RC];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr] = mk<T>(0, 0);
#pragma unroll 4
    for (int i = 0; i < nin; ++i) {
      C s = adj ? ldf_conj<T>(S + (int64_t)o * kr + i) : ldf<T>(S + (int64_t)i * kr + o);
      const C* v = in + (int64_t)i * R + r0;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) cfma(acc[rr], s, v[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
      if (rr < rc) out[(int64_t)o * R + r0 + rr] = acc[rr];
  }
}

// One inner item (two ID blocks or one middle block), one warp.
template <class T, class F, int RC, bool ADJ>
__device__ __forceinline__ void op_item(const DItem& it, const F* __restrict__ fp, const int16_t* __restrict__ ip,
                                        typename C2<T>::t* st, int64_t R, int64_t r0, int rc, int lane) {
  using C = typename C2<T>::t;
  if (it.type == 1) {
    const F* S = fp + it.blk[0].moff;
    if (!ADJ) op_middle<T, F, RC>(S, it.b_k[0], it.a_k[0], false, st + (int64_t)it.a_off[0] * R, st + (int64_t)it.b_off[0] * R, R, r0, rc, lane);
    else op_middle<T, F, RC>(S, it.b_k[0], it.a_k[0], true, st + (int64_t)it.b_off[0] * R, st + (int64_t)it.a_off[0] * R, R, r0, rc, lane);
    return;
  }
  const bool to_b = (it.type == 0) != ADJ;   // V forward or U adjoint: A (candidates) -> B (skeletons)
  if (to_b) {
    const C* a0 = st + (int64_t)it.a_off[0] * R;
    const C* a1 = st + (int64_t)it.a_off[1] * R;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const DBlk& b = it.blk[s];
      if (it.type == 0)
        op_vlike<T, F, RC, false>(fp + b.moff, ip + b.ioff, b.k, b.c, a0, it.a_k[0], a1, st + (int64_t)it.b_off[s] * R, R, r0, rc, lane);
      else
        op_vlike<T, F, RC, true>(fp + b.moff, ip + b.ioff, b.k, b.c, a0, it.a_k[0], a1, st + (int64_t)it.b_off[s] * R, R, r0, rc, lane);
    }
  } else {
    const int c = it.a_k[0] + it.a_k[1];
    for (int r = lane; r < c; r += 32) {
      C acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = mk<T>(0, 0);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const DBlk& b = it.blk[s];
        if (it.type == 2)
          row_contrib<T, F, RC, false>(acc, fp + b.moff, ip + b.ioff, b.k, b.c, st + (int64_t)it.b_off[s] * R, R, r0, rc, r);
        else
          row_contrib<T, F, RC, true>(acc, fp + b.moff, ip + b.ioff, b.k, b.c, st + (int64_t)it.b_off[s] * R, R, r0, rc, r);
      }
      C* dst = (r < it.a_k[0]) ? st + (int64_t)(it.a_off[0] + r) * R : st + (int64_t)(it.a_off[1] + r - it.a_k[0]) * R;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) dst[r0 + rr] = acc[rr];
    }
  }
}

// ---------------------------------------------------------------------------
// Apply kernels (Alg. 2): entry, D inner steps, exit.
// ---------------------------------------------------------------------------

// Forward: block = column leaf j; warp w handles depths v = w, w+W, ...:
// z_0 = V0 x_j.  Adjoint: block = row leaf i; y_0 = U0^H x_i.
template <class T, class F, int RC, bool ADJ>
__global__ void __launch_bounds__(256) k_apply_enter(const DOuter* __restrict__ ops, int D, int64_t n0,
                                                     const F* __restrict__ fp, const int16_t* __restrict__ ip,
                                                     const typename C2<T>::t* __restrict__ x,
                                                     typename C2<T>::t* st, int64_t R) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t leaf = blockIdx.x;
  const typename C2<T>::t* xl = x + leaf * n0 * R;
  for (int v = warp; v < D; v += nw) {
    const DOuter o = ops[leaf * D + v];
    for (int64_t r0 = 0; r0 < R; r0 += RC) {
      int rc = (int)(R - r0 < (int64_t)RC ? R - r0 : (int64_t)RC);
      op_vlike<T, F, RC, ADJ>(fp + o.blk.moff, ip + o.blk.ioff, o.blk.k, o.blk.c, xl, (int)n0, xl,
                              st + (int64_t)o.seg_off * R, R, r0, rc, lane);
    }
  }
}

template <class T, class F, int RC, bool ADJ>
__global__ void __launch_bounds__(256) k_apply_items(const DItem* __restrict__ items, const int32_t* __restrict__ idx,
                                                     int count, const F* __restrict__ fp,
                                                     const int16_t* __restrict__ ip, typename C2<T>::t* st,
                                                     int64_t R) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= count) return;
  const DItem it = items[idx[w]];
  for (int64_t r0 = 0; r0 < R; r0 += RC) {
    int rc = (int)(R - r0 < (int64_t)RC ? R - r0 : (int64_t)RC);
    op_item<T, F, RC, ADJ>(it, fp, ip, st, R, r0, rc, lane);
  }
}

// Forward: block = row leaf i, thread = row r: y_r = sum_v (U0 y_0)_r + (A_leaf x_i)_r,
// summed in the fixed order v = 0..D-1 then the dense leaf.  Adjoint: block =
// column leaf j: (A^H x)_j = sum_v (V0^H z_0) + A_leaf^H x_j.
template <class T, class F, int RC, bool ADJ>
__global__ void __launch_bounds__(256) k_apply_exit(const DOuter* __restrict__ ops, int D, int64_t n0,
                                                    const F* __restrict__ fp, const int16_t* __restrict__ ip,
                                                    const F* __restrict__ leafm,
                                                    const typename C2<T>::t* __restrict__ x,
                                                    const typename C2<T>::t* st, typename C2<T>::t* y,
                                                    int64_t R) {
  using C = typename C2<T>::t;
  const int64_t leaf = blockIdx.x;
  const F* A = leafm + leaf * n0 * n0;
  const C* xl = x + leaf * n0 * R;
  for (int r = threadIdx.x; r < n0; r += blockDim.x) {
    for (int64_t r0 = 0; r0 < R; r0 += RC) {
      int rc = (int)(R - r0 < (int64_t)RC ? R - r0 : (int64_t)RC);
      C acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = mk<T>(0, 0);
      for (int v = 0; v < D; ++v) {
        const DOuter o = ops[leaf * D + v];
        row_contrib<T, F, RC, ADJ>(acc, fp + o.blk.moff, ip + o.blk.ioff, o.blk.k, o.blk.c,
                                   st + (int64_t)o.seg_off * R, R, r0, rc, r);
      }
#pragma unroll 4
      for (int cc = 0; cc < n0; ++cc) {
        C a = ADJ ? ldf_conj<T>(A + (int64_t)r * n0 + cc) : ldf<T>(A + (int64_t)cc * n0 + r);
        const C* s = xl + (int64_t)cc * R + r0;
#pragma unroll
        for (int rr = 0; rr < RC; ++rr)
          if (rr < rc) cfma(acc[rr], a, s[rr]);
      }
      C* dst = y + (leaf * n0 + r) * R + r0;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) dst[rr] = acc[rr];
    }
  }
}

// ---------------------------------------------------------------------------
// Column-parallel apply for many right-hand sides (R >= kWideMin): a CTA owns
// one op and up to 256 consecutive right-hand sides, one thread per
// right-hand side.  Vector rows are read as whole coalesced rows of the
// [entry][R] layout; factor entries are warp-uniform loads (one broadcast per
// warp, L1-resident across the CTA's warps); each thread keeps KC outputs in
// registers and walks the op's inputs once per chunk of KC outputs.
// ---------------------------------------------------------------------------
constexpr int kWideMin = 32;

template <class T> struct KCw { static constexpr int v = 16; };
template <> struct KCw<double> { static constexpr int v = 8; };
template <> struct KCw<Dd> { static constexpr int v = 8; };

// B side of a V-type op (or a U-type op in adjoint): out_i = cand[q_i] + sum_j T_ij cand[p_j]
template <class T, class F, bool UTYPE_ADJ>
__device__ __forceinline__ void w_vlike(const F* __restrict__ M, const int16_t* __restrict__ idx, int k, int c,
                                        const typename C2<T>::t* a0, int ka0, const typename C2<T>::t* a1,
                                        typename C2<T>::t* out, int64_t R, int64_t col) {
  using C = typename C2<T>::t;
  constexpr int KC = KCw<T>::v;
  const int nr = c - k;
  for (int i0 = 0; i0 < k; i0 += KC) {
    C acc[KC];
#pragma unroll
    for (int ii = 0; ii < KC; ++ii) {
      acc[ii] = mk<T>(0, 0);
      if (i0 + ii < k) {
        const int q = idx[i0 + ii];
        acc[ii] = (q < ka0) ? a0[(int64_t)q * R + col] : a1[(int64_t)(q - ka0) * R + col];
      }
    }
    for (int j = 0; j < nr; ++j) {
      const int pj = idx[k + j];
      const C sv = (pj < ka0) ? a0[(int64_t)pj * R + col] : a1[(int64_t)(pj - ka0) * R + col];
#pragma unroll
      for (int ii = 0; ii < KC; ++ii)
        if (i0 + ii < k) {
          const C m = UTYPE_ADJ ? ldf_conj<T>(M + (int64_t)(i0 + ii) * nr + j) : ldf<T>(M + (int64_t)j * k + i0 + ii);
          cfma(acc[ii], m, sv);
        }
    }
#pragma unroll
    for (int ii = 0; ii < KC; ++ii)
      if (i0 + ii < k) out[(int64_t)(i0 + ii) * R + col] = acc[ii];
  }
}

// Candidate entries r0 .. r0+KC-1 (< c) of one block added to acc: a skeleton
// entry copies y_{map r}; a redundant one sums T_{i,j(r)} y_i (U-type layout
// M[i*(c-k)+j]; VTYPE_ADJ: a V-type block in adjoint, conj(M[j*k+i])).
template <class T, class F, bool VTYPE_ADJ>
__device__ __forceinline__ void w_rows(typename C2<T>::t (&acc)[KCw<T>::v], const F* __restrict__ M,
                                       const int16_t* __restrict__ idx, int k, int c, const typename C2<T>::t* y,
                                       int64_t R, int64_t col, int r0, int nrow) {
  using C = typename C2<T>::t;
  constexpr int KC = KCw<T>::v;
  const int nr = c - k;
  int code[KC];
  bool any_red = false;
#pragma unroll
  for (int ii = 0; ii < KC; ++ii) {
    code[ii] = (ii < nrow) ? idx[c + r0 + ii] : 0;
    if (ii < nrow) {
      if (code[ii] >= 0) cadd(acc[ii], y[(int64_t)code[ii] * R + col]);
      else any_red = true;
    }
  }
  if (!any_red) return;
  for (int i = 0; i < k; ++i) {
    const C yi = y[(int64_t)i * R + col];
#pragma unroll
    for (int ii = 0; ii < KC; ++ii)
      if (ii < nrow && code[ii] < 0) {
        const int j = -1 - code[ii];
        const C m = VTYPE_ADJ ? ldf_conj<T>(M + (int64_t)j * k + i) : ldf<T>(M + (int64_t)i * nr + j);
        cfma(acc[ii], m, yi);
      }
  }
}

template <class T, class F, bool ADJ>
__global__ void __launch_bounds__(256) k_wapply_enter(const DOuter* __restrict__ ops, int64_t n0,
                                                      const F* __restrict__ fp, const int16_t* __restrict__ ip,
                                                      const typename C2<T>::t* __restrict__ x,
                                                      typename C2<T>::t* st, int64_t R) {
  const int64_t col = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (col >= R) return;
  const DOuter o = ops[blockIdx.x];   // (leaf, depth) = (blockIdx.x / D, blockIdx.x % D)
  const typename C2<T>::t* xl = x + (int64_t)o.leaf * n0 * R;
  w_vlike<T, F, ADJ>(fp + o.blk.moff, ip + o.blk.ioff, o.blk.k, o.blk.c, xl, (int)n0, xl,
                     st + (int64_t)o.seg_off * R, R, col);
}

template <class T, class F, bool ADJ>
__global__ void __launch_bounds__(256) k_wapply_items(const DItem* __restrict__ items,
                                                      const int32_t* __restrict__ idx, const F* __restrict__ fp,
                                                      const int16_t* __restrict__ ip, typename C2<T>::t* st,
                                                      int64_t R) {
  using C = typename C2<T>::t;
  constexpr int KC = KCw<T>::v;
  const int64_t col = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (col >= R) return;
  const DItem it = items[idx[blockIdx.x]];
  if (it.type == 1) {   // middle: y = S z (or z = S^H y)
    const F* S = fp + it.blk[0].moff;
    const int kr = it.b_k[0], kc = it.a_k[0];
    const int nout = ADJ ? kc : kr, nin = ADJ ? kr : kc;
    const C* in = st + (int64_t)(ADJ ? it.b_off[0] : it.a_off[0]) * R;
    C* out = st + (int64_t)(ADJ ? it.a_off[0] : it.b_off[0]) * R;
    for (int o0 = 0; o0 < nout; o0 += KC) {
      C acc[KC];
#pragma unroll
      for (int ii = 0; ii < KC; ++ii) acc[ii] = mk<T>(0, 0);
      for (int i = 0; i < nin; ++i) {
        const C v = in[(int64_t)i * R + col];
#pragma unroll
        for (int ii = 0; ii < KC; ++ii)
          if (o0 + ii < nout) {
            const C sv = ADJ ? ldf_conj<T>(S + (int64_t)(o0 + ii) * kr + i) : ldf<T>(S + (int64_t)i * kr + o0 + ii);
            cfma(acc[ii], sv, v);
          }
      }
#pragma unroll
      for (int ii = 0; ii < KC; ++ii)
        if (o0 + ii < nout) out[(int64_t)(o0 + ii) * R + col] = acc[ii];
    }
    return;
  }
  const bool to_b = (it.type == 0) != ADJ;
  if (to_b) {
    const C* a0 = st + (int64_t)it.a_off[0] * R;
    const C* a1 = st + (int64_t)it.a_off[1] * R;
#pragma unroll
    for (int sb = 0; sb < 2; ++sb) {
      const DBlk& b = it.blk[sb];
      if (it.type == 0)
        w_vlike<T, F, false>(fp + b.moff, ip + b.ioff, b.k, b.c, a0, it.a_k[0], a1, st + (int64_t)it.b_off[sb] * R, R, col);
      else
        w_vlike<T, F, true>(fp + b.moff, ip + b.ioff, b.k, b.c, a0, it.a_k[0], a1, st + (int64_t)it.b_off[sb] * R, R, col);
    }
  } else {
    const int c = it.a_k[0] + it.a_k[1];
    for (int r0 = 0; r0 < c; r0 += KC) {
      const int nrow = (c - r0) < KC ? (c - r0) : KC;
      C acc[KC];
#pragma unroll
      for (int ii = 0; ii < KC; ++ii) acc[ii] = mk<T>(0, 0);
#pragma unroll
      for (int sb = 0; sb < 2; ++sb) {
        const DBlk& b = it.blk[sb];
        if (it.type == 2)
          w_rows<T, F, false>(acc, fp + b.moff, ip + b.ioff, b.k, b.c, st + (int64_t)it.b_off[sb] * R, R, col, r0, nrow);
        else
          w_rows<T, F, true>(acc, fp + b.moff, ip + b.ioff, b.k, b.c, st + (int64_t)it.b_off[sb] * R, R, col, r0, nrow);
      }
#pragma unroll
      for (int ii = 0; ii < KC; ++ii)
        if (ii < nrow) {
          const int r = r0 + ii;
          C* dst = (r < it.a_k[0]) ? st + (int64_t)(it.a_off[0] + r) * R : st + (int64_t)(it.a_off[1] + r - it.a_k[0]) * R;
          dst[col] = acc[ii];
        }
    }
  }
}

// y_leaf = sum_v U0_v y_0 + A_leaf x_leaf (fixed order: depths 0..D-1, then the leaf)
template <class T, class F, bool ADJ>
__global__ void __launch_bounds__(256) k_wapply_exit(const DOuter* __restrict__ ops, int D, int64_t n0,
                                                     const F* __restrict__ fp, const int16_t* __restrict__ ip,
                                                     const F* __restrict__ leafm,
                                                     const typename C2<T>::t* __restrict__ x,
                                                     const typename C2<T>::t* st, typename C2<T>::t* y,
                                                     int64_t R) {
  using C = typename C2<T>::t;
  constexpr int KC = KCw<T>::v;
  const int64_t col = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (col >= R) return;
  const int64_t leaf = blockIdx.x;
  const F* A = leafm + leaf * n0 * n0;
  const C* xl = x + leaf * n0 * R;
  for (int r0 = 0; r0 < (int)n0; r0 += KC) {
    const int nrow = ((int)n0 - r0) < KC ? ((int)n0 - r0) : KC;
    C acc[KC];
#pragma unroll
    for (int ii = 0; ii < KC; ++ii) acc[ii] = mk<T>(0, 0);
    for (int v = 0; v < D; ++v) {
      const DOuter o = ops[leaf * D + v];
      w_rows<T, F, ADJ>(acc, fp + o.blk.moff, ip + o.blk.ioff, o.blk.k, o.blk.c, st + (int64_t)o.seg_off * R, R,
                        col, r0, nrow);
    }
    for (int cc = 0; cc < (int)n0; ++cc) {
      const C xv = xl[(int64_t)cc * R + col];
#pragma unroll
      for (int ii = 0; ii < KC; ++ii)
        if (ii < nrow) {
          const C a = ADJ ? ldf_conj<T>(A + (int64_t)(r0 + ii) * n0 + cc) : ldf<T>(A + (int64_t)cc * n0 + r0 + ii);
          cfma(acc[ii], a, xv);
        }
    }
#pragma unroll
    for (int ii = 0; ii < KC; ++ii)
      if (ii < nrow) y[(leaf * n0 + r0 + ii) * R + col] = acc[ii];
  }
}

// ---------------------------------------------------------------------------
// Layout conversion kernels
// ---------------------------------------------------------------------------
template <class S, class D>
__global__ void k_gather_cols(const S* __restrict__ src, int64_t ld, int64_t n, int64_t R, D* __restrict__ dst,
                              double scale) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = n * R;
  for (; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t row = e / R, r = e % R;
    S v = src[r * ld + row];
    dst[e].x = (decltype(dst[e].x))(scale * (double)v.x);
    dst[e].y = (decltype(dst[e].y))(scale * (double)v.y);
  }
}
template <class S, class D>
__global__ void k_scatter_cols(const S* __restrict__ src, int64_t n, int64_t R, D* __restrict__ dst, int64_t ld,
                               double scale) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = n * R;
  for (; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t row = e / R, r = e % R;
    S v = src[e];
    dst[r * ld + row].x = (decltype(dst[0].x))(scale * (double)v.x);
    dst[r * ld + row].y = (decltype(dst[0].y))(scale * (double)v.y);
  }
}

static inline int grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

int launch_gather_cols(const void* src, int src_t, int64_t ld, int64_t n, int64_t R, void* dst, int dst_t,
                       double scale, cudaStream_t st) {
  int g = grid_for(n * R, 256);
  if (src_t == 0 && dst_t == 0) k_gather_cols<<<g, 256, 0, st>>>((const double2*)src, ld, n, R, (double2*)dst, scale);
  else if (src_t == 0 && dst_t == 1) k_gather_cols<<<g, 256, 0, st>>>((const double2*)src, ld, n, R, (float2*)dst, scale);
  else if (src_t == 1 && dst_t == 0) k_gather_cols<<<g, 256, 0, st>>>((const float2*)src, ld, n, R, (double2*)dst, scale);
  else k_gather_cols<<<g, 256, 0, st>>>((const float2*)src, ld, n, R, (float2*)dst, scale);
  return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
}
int launch_scatter_cols(const void* src, int src_t, int64_t n, int64_t R, void* dst, int dst_t, int64_t ld,
                        double scale, cudaStream_t st) {
  int g = grid_for(n * R, 256);
  if (src_t == 0 && dst_t == 0) k_scatter_cols<<<g, 256, 0, st>>>((const double2*)src, n, R, (double2*)dst, ld, scale);
  else if (src_t == 0 && dst_t == 1) k_scatter_cols<<<g, 256, 0, st>>>((const double2*)src, n, R, (float2*)dst, ld, scale);
  else if (src_t == 1 && dst_t == 0) k_scatter_cols<<<g, 256, 0, st>>>((const float2*)src, n, R, (double2*)dst, ld, scale);
  else k_scatter_cols<<<g, 256, 0, st>>>((const float2*)src, n, R, (float2*)dst, ld, scale);
  return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class T, class F, int RC>
static int apply_impl(const DevFactor& df, bool adj, const void* xv, void* yv, int64_t R, void* stv,
                      cudaStream_t s) {
  using C = typename C2<T>::t;
  const F* fp = (const F*)df.fpool;
  const C* x = (const C*)xv;
  C* y = (C*)yv;
  C* st = (C*)stv;
  int wpb = df.D < 8 ? df.D : 8;
  if (!adj) k_apply_enter<T, F, RC, false><<<(unsigned)df.m, 32 * wpb, 0, s>>>(df.vout, df.D, df.n0, fp, df.ipool, x, st, R);
  else k_apply_enter<T, F, RC, true><<<(unsigned)df.m, 32 * wpb, 0, s>>>(df.uout, df.D, df.n0, fp, df.ipool, x, st, R);
  const std::vector<int32_t>& ptr = adj ? df.astep_ptr : df.step_ptr;
  const int32_t* idx = adj ? df.astep_idx : df.step_idx;
  for (int stp = 0; stp + 1 < (int)ptr.size(); ++stp) {
    int cnt = ptr[stp + 1] - ptr[stp];
    if (cnt <= 0) continue;
    int blocks = (cnt + 7) / 8;
    if (!adj) k_apply_items<T, F, RC, false><<<blocks, 256, 0, s>>>(df.items, idx + ptr[stp], cnt, fp, df.ipool, st, R);
    else k_apply_items<T, F, RC, true><<<blocks, 256, 0, s>>>(df.items, idx + ptr[stp], cnt, fp, df.ipool, st, R);
  }
  int thr = (int)((df.n0 + 31) / 32 * 32);
  if (thr > 256) thr = 256;
  if (!adj) k_apply_exit<T, F, RC, false><<<(unsigned)df.m, thr, 0, s>>>(df.uout, df.D, df.n0, fp, df.ipool, (const F*)df.leaf, x, st, y, R);
  else k_apply_exit<T, F, RC, true><<<(unsigned)df.m, thr, 0, s>>>(df.vout, df.D, df.n0, fp, df.ipool, (const F*)df.leaf, x, st, y, R);
  return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
}

template <class T, class F>
static int apply_wide(const DevFactor& df, bool adj, const void* xv, void* yv, int64_t R, void* stv,
                      cudaStream_t s) {
  using C = typename C2<T>::t;
  const F* fp = (const F*)df.fpool;
  const C* x = (const C*)xv;
  C* y = (C*)yv;
  C* st = (C*)stv;
  const int thr = (int)(R < 256 ? (R + 31) / 32 * 32 : 256);
  const unsigned cb = (unsigned)((R + thr - 1) / thr);
  const dim3 g_enter((unsigned)(df.m * df.D), cb);
  if (!adj) k_wapply_enter<T, F, false><<<g_enter, thr, 0, s>>>(df.vout, df.n0, fp, df.ipool, x, st, R);
  else k_wapply_enter<T, F, true><<<g_enter, thr, 0, s>>>(df.uout, df.n0, fp, df.ipool, x, st, R);
  const std::vector<int32_t>& ptr = adj ? df.astep_ptr : df.step_ptr;
  const int32_t* idx = adj ? df.astep_idx : df.step_idx;
  for (int stp = 0; stp + 1 < (int)ptr.size(); ++stp) {
    int cnt = ptr[stp + 1] - ptr[stp];
    if (cnt <= 0) continue;
    const dim3 g((unsigned)cnt, cb);
    if (!adj) k_wapply_items<T, F, false><<<g, thr, 0, s>>>(df.items, idx + ptr[stp], fp, df.ipool, st, R);
    else k_wapply_items<T, F, true><<<g, thr, 0, s>>>(df.items, idx + ptr[stp], fp, df.ipool, st, R);
  }
  const dim3 g_exit((unsigned)df.m, cb);
  if (!adj) k_wapply_exit<T, F, false><<<g_exit, thr, 0, s>>>(df.uout, df.D, df.n0, fp, df.ipool, (const F*)df.leaf, x, st, y, R);
  else k_wapply_exit<T, F, true><<<g_exit, thr, 0, s>>>(df.vout, df.D, df.n0, fp, df.ipool, (const F*)df.leaf, x, st, y, R);
  return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
}

template <class T, class F>
static int apply_dispatch(const DevFactor& df, bool adj, const void* x, void* y, int64_t R, void* st,
                          cudaStream_t s) {
  if (R >= kWideMin) return apply_wide<T, F>(df, adj, x, y, R, st, s);
  if (R == 1) return apply_impl<T, F, 1>(df, adj, x, y, R, st, s);   // (the persistent kernel is tried first, in launch_apply)
  if (R <= 4) return apply_impl<T, F, 4>(df, adj, x, y, R, st, s);
  return apply_impl<T, F, 8>(df, adj, x, y, R, st, s);
}

// Forward many-column apply of the split-BF16 form: entry and exit contractions on the
// tensor cores (hb_tc.cu), the inner butterfly items on CUDA cores in complex FP32.
static int apply_wide_tc(const DevFactor& df, const void* xv, void* yv, int64_t R, void* stv, cudaStream_t s) {
  int rc = launch_tc_jobs(df, false, xv, stv, nullptr, R, s);
  if (rc) return rc;
  const int thr = (int)(R < 256 ? (R + 31) / 32 * 32 : 256);
  const unsigned cb = (unsigned)((R + thr - 1) / thr);
  for (int stp = 0; stp + 1 < (int)df.step_ptr.size(); ++stp) {
    int cnt = df.step_ptr[stp + 1] - df.step_ptr[stp];
    if (cnt <= 0) continue;
    const dim3 g((unsigned)cnt, cb);
    k_wapply_items<float, float2, false><<<g, thr, 0, s>>>(df.items, df.step_idx + df.step_ptr[stp],
                                                           (const float2*)df.fpool, df.ipool, (float2*)stv, R);
  }
  if (cudaGetLastError() != cudaSuccess) return HB_ECUDA;
  return launch_tc_jobs(df, true, xv, stv, yv, R, s);
}

// double2 <-> double-float vectors
__global__ void k_to_dd(const double2* __restrict__ x, DdC* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    const float rh = (float)v.x, ih = (float)v.y;
    y[i] = DdC{Dd(rh, (float)(v.x - (double)rh)), Dd(ih, (float)(v.y - (double)ih))};
  }
}
__global__ void k_from_dd(const DdC* __restrict__ x, double2* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const DdC v = x[i];
    y[i] = make_double2((double)v.x.h + (double)v.x.l, (double)v.y.h + (double)v.y.l);
  }
}

bool apply_dd_ready(int64_t R) { return R >= kWideMin; }

int launch_apply_dd(const DevFactor& df, bool adjoint, const void* x, void* y, int64_t R, void* state, void* xdd,
                    void* ydd, cudaStream_t st) {
  if (!apply_dd_ready(R) || df.form == HB_C128) return HB_EINVAL;
  const int64_t nn = df.n * R;
  const unsigned g = (unsigned)std::min<int64_t>((nn + 255) / 256, 152 * 16);
  k_to_dd<<<g, 256, 0, st>>>((const double2*)x, (DdC*)xdd, nn);
  int rc = apply_wide<Dd, float2>(df, adjoint, xdd, ydd, R, state, st);
  if (rc) return rc;
  k_from_dd<<<g, 256, 0, st>>>((const DdC*)ydd, (double2*)y, nn);
  return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
}

int launch_apply(const DevFactor& df, Prec p, bool adjoint, const void* x, void* y, int64_t R, void* state,
                 cudaStream_t st) {
  if (R == 1 && apply1_ready(df, adjoint)) return launch_apply1(df, p, adjoint, x, y, state, st);
  if (p == PREC_F32 && !adjoint && R >= kWideMin && df.form == HB_SPLIT_BF16 && df.tc_ok)
    return apply_wide_tc(df, x, y, R, state, st);
  if (p == PREC_F64) return apply_dispatch<double, double2>(df, adjoint, x, y, R, state, st);
  if (p == PREC_F32) return apply_dispatch<float, float2>(df, adjoint, x, y, R, state, st);
  return apply_dispatch<double, float2>(df, adjoint, x, y, R, state, st);
}

}  // namespace hb

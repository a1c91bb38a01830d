// Cooperative sweep kernel (sm_103a): x = L~^{-1} b, U~^{-1} b and their
// adjoints (Algs. 3, 4), in place on the vector.
//
// The recursion of Alg. 3 / Alg. 4 is flattened on the host into a program
// of phases (leaf solves, butterfly entry ops, butterfly stages, butterfly
// exit ops); consecutive phases depend on each other, ops inside a phase do
// not.  The program is cut into segments:
//   * a grid segment is one large phase (a stage of a big butterfly); its
//     ops are spread over all CTAs, one op per CTA at a time;
//   * a local segment is a run of small phases (a subtree near the leaves);
//     a single CTA executes it, one op per warp, __syncthreads between phases.
// A grid barrier (bounded spin; HB_ETIMEOUT instead of a hang) separates the
// segments.  Every op first stages its factor blocks into shared memory with
// 16-byte cp.async copies (one memory round trip for the whole op), then
// computes from shared memory.  Vector and butterfly-state reads bypass L1
// (ld.global.cg) because other CTAs write them inside the same launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_device.h"

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
  __device__ __forceinline__ void sync() const {
    if (cta) __syncthreads();
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
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

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

// B side = gather + T * rest (V-type layout M[j*k+i]; or U-type adjoint conj(M[i*nr+j]))
template <class T, class F, int RC, bool UADJ>
__device__ __forceinline__ void vlike(const F* M, const int16_t* idx, int k, int c,
                                      const typename CT<T>::t* cand /* [c][RC] smem */,
                                      typename CT<T>::t* out, int64_t R, int64_t r0, int rc, const Grp& g) {
  using C = typename CT<T>::t;
  const int nr = c - k;
  for (int i = g.t; i < k; i += g.nt) {
    C acc[RC];
    const int qi = idx[i];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr] = cand[qi * RC + rr];
#pragma unroll 8
    for (int j = 0; j < nr; ++j) {
      C m = UADJ ? cvc<T>(M[(int64_t)i * nr + j]) : cv<T>(M[(int64_t)j * k + i]);
      const C* s = cand + idx[k + j] * RC;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], m, s[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
      if (rr < rc) out[(int64_t)i * R + r0 + rr] = acc[rr];
  }
}

// candidate entry r of one block (U-type layout M[i*nr+j]; or V-type adjoint conj(M[j*k+i]))
template <class T, class F, int RC, bool VADJ>
__device__ __forceinline__ void rowc(typename CT<T>::t (&acc)[RC], const F* M, const int16_t* idx, int k, int c,
                                     const typename CT<T>::t* y /* [k][RC] smem */, int r) {
  using C = typename CT<T>::t;
  const int code = idx[c + r];
  if (code >= 0) {
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) { acc[rr].x += y[code * RC + rr].x; acc[rr].y += y[code * RC + rr].y; }
  } else {
    const int j = -1 - code, nr = c - k;
#pragma unroll 8
    for (int i = 0; i < k; ++i) {
      C m = VADJ ? cvc<T>(M[(int64_t)j * k + i]) : cv<T>(M[(int64_t)i * nr + j]);
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], m, y[i * RC + rr]);
    }
  }
}

// load `cnt` vector entries (stride R, RHS r0..r0+rc) into smem [cnt][RC] (zero padded)
template <class C, int RC>
__device__ __forceinline__ void load_vec(C* dst, const C* src, int cnt, int64_t R, int64_t r0, int rc, const Grp& g) {
  for (int e = g.t; e < cnt * RC; e += g.nt) {
    int i = e / RC, rr = e % RC;
    dst[e] = (rr < rc) ? ldcg2(src + (int64_t)i * R + r0 + rr) : C{0, 0};
  }
}

struct SweepArgs {
  const DSeg* segs;
  int nseg;
  const DPhase* prog;
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
};

// ---------------------------------------------------------------------------
// one op of a phase, executed by group g (warp or CTA) with staging area buf
// ---------------------------------------------------------------------------
template <class T, class F, int RC>
__device__ void do_op(const SweepArgs& a, const DPhase& P, int o, char* buf, int64_t buf_bytes, const Grp& g,
                      int64_t rb, int64_t re) {
  using C = typename CT<T>::t;
  const F* fp = (const F*)a.fp;
  C* vec = (C*)a.vec;
  C* st = (C*)a.st;
  const int64_t R = a.R, n0 = a.n0;
  if (P.kind == PH_ENTER || P.kind == PH_EXIT) {
    const bool enter = P.kind == PH_ENTER;
    // forward: enter = V0 (bvout), exit = U0 (buout); adjoint: enter = U0^H, exit = V0^H
    const bool use_u = (enter == (P.adj != 0));
    const DOuter op = use_u ? a.buout[a.bf_uout0[P.arg0] + o] : a.bvout[a.bf_vout0[P.arg0] + o];
    const int k = op.blk.k, c = op.blk.c;
    const int64_t mb = align16((int64_t)k * (c - k) * sizeof(F));
    const int64_t ib = align16((int64_t)2 * c * sizeof(int16_t));
    const int vcnt = enter ? c : k;
    const int64_t need = mb + ib + (int64_t)vcnt * RC * sizeof(C);
    const F* M;
    const int16_t* idx;
    C* v;
    if (need <= buf_bytes) {
      stage(buf, fp + op.blk.moff, mb, g);
      stage(buf + mb, a.ip + op.blk.ioff, ib, g);
      M = (const F*)buf;
      idx = (const int16_t*)(buf + mb);
      v = (C*)(buf + mb + ib);
    } else {
      M = fp + op.blk.moff;
      idx = a.ip + op.blk.ioff;
      v = (C*)buf;
    }
    const C* src = enter ? vec + (int64_t)op.leaf * n0 * R : st + (int64_t)op.seg_off * R;
    for (int64_t r0 = rb; r0 < re; r0 += RC) {
    const int rc = (int)((re - r0) < RC ? (re - r0) : RC);
    load_vec<C, RC>(v, src, vcnt, R, r0, rc, g);
    cp_commit_wait();
    g.sync();
    if (enter) {
      C* out = st + (int64_t)op.seg_off * R;
      if (P.adj) vlike<T, F, RC, true>(M, idx, k, c, v, out, R, r0, rc, g);
      else vlike<T, F, RC, false>(M, idx, k, c, v, out, R, r0, rc, g);
    } else {
      C* bl = vec + (int64_t)op.leaf * n0 * R;
      for (int r = g.t; r < c; r += g.nt) {
        C acc[RC];
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
        if (P.adj) rowc<T, F, RC, true>(acc, M, idx, k, c, v, r);
        else rowc<T, F, RC, false>(acc, M, idx, k, c, v, r);
        C* d = bl + (int64_t)r * R + r0;
#pragma unroll
        for (int rr = 0; rr < RC; ++rr)
          if (rr < rc) {
            C cur = ldcg2(d + rr);
            d[rr] = C{cur.x - acc[rr].x, cur.y - acc[rr].y};
          }
      }
    }
    g.sync();
    }
    return;
  }
  // ---- inner item
  const DItem it = a.items[P.arg0 + o];
  const bool adj = P.adj != 0;
  if (it.type == 1) {
    const int kr = it.b_k[0], kc = it.a_k[0];
    const int64_t mb = align16((int64_t)kr * kc * sizeof(F));
    const int nin = adj ? kr : kc, nout = adj ? kc : kr;
    const F* S;
    C* v;
    if (mb + (int64_t)nin * RC * sizeof(C) <= buf_bytes) {
      stage(buf, fp + it.blk[0].moff, mb, g);
      S = (const F*)buf;
      v = (C*)(buf + mb);
    } else {
      S = fp + it.blk[0].moff;
      v = (C*)buf;
    }
    C* out = st + (int64_t)(adj ? it.a_off[0] : it.b_off[0]) * R;
    for (int64_t r0 = rb; r0 < re; r0 += RC) {
    const int rc = (int)((re - r0) < RC ? (re - r0) : RC);
    load_vec<C, RC>(v, st + (int64_t)(adj ? it.b_off[0] : it.a_off[0]) * R, nin, R, r0, rc, g);
    cp_commit_wait();
    g.sync();
    for (int oo = g.t; oo < nout; oo += g.nt) {
      C acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
#pragma unroll 8
      for (int i = 0; i < nin; ++i) {
        C s = adj ? cvc<T>(S[(int64_t)oo * kr + i]) : cv<T>(S[(int64_t)i * kr + oo]);
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], s, v[i * RC + rr]);
      }
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) out[(int64_t)oo * R + r0 + rr] = acc[rr];
    }
    g.sync();
    }
    return;
  }
  // two ID blocks: matrices and index arrays are contiguous in their pools
  const DBlk& b0 = it.blk[0];
  const DBlk& b1 = it.blk[1];
  const int64_t m1off = (b1.moff - b0.moff) * (int64_t)sizeof(F);
  const int64_t mb = align16(m1off + (int64_t)b1.k * (b1.c - b1.k) * sizeof(F));
  const int64_t i1off = (int64_t)(b1.ioff - b0.ioff) * (int64_t)sizeof(int16_t);
  const int64_t ib = align16(i1off + (int64_t)2 * b1.c * sizeof(int16_t));
  const int ca = it.a_k[0] + it.a_k[1];
  const bool to_b = (it.type == 0) != adj;
  const int vcnt = to_b ? ca : (it.b_k[0] + it.b_k[1]);
  const int64_t need = mb + ib + (int64_t)vcnt * RC * sizeof(C);
  const F *M0, *M1;
  const int16_t *I0, *I1;
  C* v;
  if (need <= buf_bytes) {
    stage(buf, fp + b0.moff, mb, g);
    stage(buf + mb, a.ip + b0.ioff, ib, g);
    M0 = (const F*)buf;
    M1 = (const F*)(buf + m1off);
    I0 = (const int16_t*)(buf + mb);
    I1 = (const int16_t*)(buf + mb + i1off);
    v = (C*)(buf + mb + ib);
  } else {
    M0 = fp + b0.moff;
    M1 = fp + b1.moff;
    I0 = a.ip + b0.ioff;
    I1 = a.ip + b1.ioff;
    v = (C*)buf;
  }
  for (int64_t r0 = rb; r0 < re; r0 += RC) {
  const int rc = (int)((re - r0) < RC ? (re - r0) : RC);
  if (to_b) {
    load_vec<C, RC>(v, st + (int64_t)it.a_off[0] * R, it.a_k[0], R, r0, rc, g);
    load_vec<C, RC>(v + it.a_k[0] * RC, st + (int64_t)it.a_off[1] * R, it.a_k[1], R, r0, rc, g);
  } else {
    load_vec<C, RC>(v, st + (int64_t)it.b_off[0] * R, it.b_k[0], R, r0, rc, g);
    load_vec<C, RC>(v + it.b_k[0] * RC, st + (int64_t)it.b_off[1] * R, it.b_k[1], R, r0, rc, g);
  }
  cp_commit_wait();
  g.sync();
  if (to_b) {
    C* o0 = st + (int64_t)it.b_off[0] * R;
    C* o1 = st + (int64_t)it.b_off[1] * R;
    if (it.type == 0) {
      vlike<T, F, RC, false>(M0, I0, b0.k, b0.c, v, o0, R, r0, rc, g);
      vlike<T, F, RC, false>(M1, I1, b1.k, b1.c, v, o1, R, r0, rc, g);
    } else {
      vlike<T, F, RC, true>(M0, I0, b0.k, b0.c, v, o0, R, r0, rc, g);
      vlike<T, F, RC, true>(M1, I1, b1.k, b1.c, v, o1, R, r0, rc, g);
    }
  } else {
    const C* y0 = v;
    const C* y1 = v + it.b_k[0] * RC;
    for (int r = g.t; r < ca; r += g.nt) {
      C acc[RC];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
      if (it.type == 2) {
        rowc<T, F, RC, false>(acc, M0, I0, b0.k, b0.c, y0, r);
        rowc<T, F, RC, false>(acc, M1, I1, b1.k, b1.c, y1, r);
      } else {
        rowc<T, F, RC, true>(acc, M0, I0, b0.k, b0.c, y0, r);
        rowc<T, F, RC, true>(acc, M1, I1, b1.k, b1.c, y1, r);
      }
      C* d = (r < it.a_k[0]) ? st + (int64_t)(it.a_off[0] + r) * R : st + (int64_t)(it.a_off[1] + r - it.a_k[0]) * R;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
        if (rr < rc) d[r0 + rr] = acc[rr];
    }
  }
  g.sync();
  }
}

// leaf solve x_leaf = Tinv b_leaf (or Tinv^H b_leaf), whole CTA
template <class T, class F, int RC>
__device__ void do_leaf(const SweepArgs& a, const DPhase& P, char* buf, int64_t buf_bytes, int64_t rb, int64_t re) {
  using C = typename CT<T>::t;
  const int64_t n0 = a.n0, R = a.R;
  const Grp g{(int)threadIdx.x, (int)blockDim.x, true};
  const F* Tg = (const F*)a.tinv + (int64_t)P.arg0 * n0 * n0;
  C* v = (C*)a.vec + (int64_t)P.arg0 * n0 * R;
  const int64_t mb = align16(n0 * n0 * (int64_t)sizeof(F));
  const int ngrp = (int)(blockDim.x / n0) > 0 ? (int)(blockDim.x / n0) : 1;
  const int64_t need = mb + n0 * RC * (int64_t)sizeof(C) + (int64_t)ngrp * n0 * RC * sizeof(C);
  const F* Tm;
  C* bv;
  C* part;
  if (need <= buf_bytes) {
    stage(buf, Tg, mb, g);
    Tm = (const F*)buf;
    bv = (C*)(buf + mb);
  } else {
    Tm = Tg;
    bv = (C*)buf;
  }
  part = bv + n0 * RC;
  for (int64_t r0 = rb; r0 < re; r0 += RC) {
  const int rc = (int)((re - r0) < RC ? (re - r0) : RC);
  load_vec<C, RC>(bv, v, (int)n0, R, r0, rc, g);
  cp_commit_wait();
  __syncthreads();
  // thread (row r, column group q): partial sums over columns cc = q, q+ngrp, ...
  for (int e = threadIdx.x; e < ngrp * n0; e += blockDim.x) {
    const int r = e % n0, q = e / n0;
    C acc[RC];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr] = z2<T>();
    for (int cc = q; cc < n0; cc += ngrp) {
      C m = P.adj ? cvc<T>(Tm[(int64_t)r * n0 + cc]) : cv<T>(Tm[(int64_t)cc * n0 + r]);
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) fma2(acc[rr], m, bv[cc * RC + rr]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) part[(q * n0 + r) * RC + rr] = acc[rr];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n0 * RC; e += blockDim.x) {
    const int r = e / RC, rr = e % RC;
    C s = z2<T>();
    for (int q = 0; q < ngrp; ++q) { s.x += part[(q * n0 + r) * RC + rr].x; s.y += part[(q * n0 + r) * RC + rr].y; }
    if (rr < rc) v[(int64_t)r * R + r0 + rr] = s;
  }
  __syncthreads();
  }
}

template <class T, class F, int RC>
__global__ void __launch_bounds__(256, 1) k_sweep_coop(SweepArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  unsigned my_gen = 0;
  const int64_t slice = (a.smem_bytes / nw) & ~(int64_t)15;
  // local runs: the right-hand sides are split over the CTAs (chunks of RC);
  // CTA b owns [lb, le).  With a single chunk only CTA 0 works.
  const int64_t nchunk = (a.R + RC - 1) / RC;
  const int64_t cper = (nchunk + gridDim.x - 1) / gridDim.x;
  const int64_t lb = (int64_t)blockIdx.x * cper * RC;
  const int64_t le = (lb + cper * RC < a.R) ? lb + cper * RC : a.R;
  for (int s = 0; s < a.nseg; ++s) {
    const DSeg sg = a.segs[s];
    if (sg.grid) {
      const DPhase P = a.prog[sg.first];
      const Grp g{(int)threadIdx.x, (int)blockDim.x, true};
      for (int o = blockIdx.x; o < P.count; o += gridDim.x) do_op<T, F, RC>(a, P, o, smem, a.smem_bytes, g, 0, a.R);
    } else if (lb < le) {
      for (int ph = sg.first; ph < sg.first + sg.count; ++ph) {
        const DPhase P = a.prog[ph];
        if (P.kind == PH_LEAF) {
          do_leaf<T, F, RC>(a, P, smem, a.smem_bytes, lb, le);
        } else {
          const Grp g{lane, 32, false};
          for (int o = warp; o < P.count; o += nw) do_op<T, F, RC>(a, P, o, smem + warp * slice, slice, g, lb, le);
          __syncthreads();
        }
      }
    }
    if (!grid_sync(a.bar, my_gen, a.spin_limit)) return;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------
struct CoopState {
  int sms = 0;
  GridBar* bar = nullptr;
};

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
  const int smem = 192 * 1024;
  auto kern = k_sweep_coop<T, F, RC>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr_done = true;
  }
  SweepArgs a;
  a.segs = df.segs[which];
  a.nseg = df.nsegs[which];
  a.prog = df.prog[which];
  a.n0 = df.n0;
  a.bvout = df.bvout;
  a.buout = df.buout;
  a.bf_vout0 = df.bf_vout0;
  a.bf_uout0 = df.bf_uout0;
  a.items = df.items;
  a.fp = df.fpool;
  a.ip = df.ipool;
  a.tinv = (which == 0 || which == 2) ? df.linv : df.uinv;
  a.vec = vec;
  a.st = st;
  a.R = R;
  a.bar = (GridBar*)bar;
  a.smem_bytes = smem;
  a.spin_limit = spin_limit;
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

int launch_sweep_coop(const DevFactor& df, Prec p, int which, void* vec, int64_t R, void* state, void* bar,
                      cudaStream_t st, long long spin_limit) {
  if (which < 0 || which > 3) return HB_EINVAL;
  if (p == PREC_F64) {
    if (R >= 4) return sweep_coop_impl<double, double2, 4>(df, which, vec, R, state, bar, st, spin_limit);
    return sweep_coop_impl<double, double2, 1>(df, which, vec, R, state, bar, st, spin_limit);
  }
  if (p == PREC_F32) {
    if (R >= 8) return sweep_coop_impl<float, float2, 8>(df, which, vec, R, state, bar, st, spin_limit);
    if (R >= 4) return sweep_coop_impl<float, float2, 4>(df, which, vec, R, state, bar, st, spin_limit);
    return sweep_coop_impl<float, float2, 1>(df, which, vec, R, state, bar, st, spin_limit);
  }
  return sweep_coop_impl<double, float2, 1>(df, which, vec, R, state, bar, st, spin_limit);
}

int read_grid_error(void* bar, cudaStream_t st, int* err) {
  GridBar h;
  if (cudaMemcpyAsync(&h, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, st) != cudaSuccess) return HB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HB_ECUDA;
  *err = h.err;
  if (h.err) {
    int zero = 0;
    if (cudaMemcpyAsync((char*)bar + 2 * sizeof(unsigned int), &zero, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) return HB_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HB_ECUDA;
  }
  return HB_OK;
}

}  // namespace hb

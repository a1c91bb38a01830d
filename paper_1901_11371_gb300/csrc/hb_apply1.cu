// Persistent single-column apply (sm_103a): y = A^_F x or A^_F^H x for one
// right-hand side in one cooperative launch (Alg. 2).
//
// A column-at-a-time apply streams every factor entry once and does about
// one complex multiply-add per 8-16 bytes, so it is bound by HBM bandwidth
// -- provided enough bytes are in flight.  The host plan (hb_plan.cpp) cuts
// the apply into phases (entry ops V0 and dense-leaf products, the inner
// butterfly steps, the exit ops U0) and gives every CTA a balanced, ordered
// list of staging batches.  Per CTA:
//   * one producer warp copies each batch into a shared-memory ring with one
//     cp.async.bulk (completion on one mbarrier per batch slot): the host laid
//     out every batch's records, factor and index blocks and vector gather
//     list contiguously (the plan's batch image), so a batch is one large
//     transfer; the producer runs ahead of the compute warps across phase
//     boundaries, since factor data never depends on the vectors;
//   * nineteen compute warps take the batches in turn (batch q goes to warp
//     q mod 19, so no CTA-wide barrier separates batches): a warp waits for
//     its batch, gathers the vector entries the batch's ops read (state
//     written in earlier phases, x, or y) with L1-bypassing loads in one round
//     trip, then its lanes take the batch's output rows in turn (an entry of
//     a skeleton or candidate vector, a row of y; an exit row sums the depths'
//     contributions in order), computing from shared memory and writing to
//     global memory, and the warp releases the ring area;
//   * there is no grid barrier between the phases: every batch lists the
//     batches (of earlier phases, on any CTA) that wrote the entries it
//     gathers, waits (bounded) until their completion flags carry this
//     launch's epoch, and sets its own flag when its outputs are written, so
//     a subtree's butterfly steps start as soon as its inputs exist.  Every
//     CTA runs its batches in phase order and all CTAs are resident
//     (cooperative launch), so the waits always end.
// Every wait is bounded; a wait that gives up raises the factor's error
// flag (reported by hb_status / the solvers) and the kernel returns after a
// second bounded wait for the copies still in flight.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_device.h"
#include "hb_sweep_launch.h"

namespace hb {

namespace {

constexpr int kA1Threads = 640;
static_assert(kA1Threads / 32 - 1 == kA1Warps, "compute warps");
constexpr int kA1Cw = kA1Warps;         // compute warps; one more warp is the producer
constexpr int kA1Slots = 32;            // batches in flight per CTA

template <class T> struct CT1;
template <> struct CT1<float> { using t = float2; };
template <> struct CT1<double> { using t = double2; };
template <class T, class F> __device__ __forceinline__ typename CT1<T>::t cv1(const F v) { return {(T)v.x, (T)v.y}; }
template <class T, class F> __device__ __forceinline__ typename CT1<T>::t cvc1(const F v) { return {(T)v.x, -(T)v.y}; }
template <class C> __device__ __forceinline__ void fma1(C& acc, const C& a, const C& b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 ldcg1(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldcg1(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ int64_t al16(int64_t b) { return (b + 15) & ~(int64_t)15; }

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_inval(uint64_t* b) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mb_arrive_tx(uint64_t* b, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(su32(b)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(b)) : "memory");
}
__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct A1Args {
  const A1Batch* batches;
  const int32_t* cta_batch;
  const uint8_t* image;
  int nphase;
  int ring_bytes;
  const void* x;
  void* y;
  void* st;
  int64_t n0;
  GridBar* gb;        // abort flag of this launch (err), shared by the CTAs
  int* done;          // per batch: the epoch of the launch that completed it
  int epoch;
  int* err_out;       // the factor's sticky error flag (hb_status)
  long long spin_limit;
};

// ---------------------------------------------------------------------------
// Row-parallel execution of a batch by one warp.  Every task of the batch
// yields output rows (an entry of a skeleton vector, of a candidate vector or
// of y); the lanes take the batch's rows in turn, so tiny ops cost no
// per-op synchronisation.  Matrices, indices and inputs are in shared memory.
// ---------------------------------------------------------------------------
// rows of one task
__device__ __forceinline__ int task_rows(const A1Task& tk, const FlatOp* recs, int op_base, int n0) {
  if (tk.kind == 3) return n0;
  int r = 0;
  for (int o = 0; o < tk.nops; ++o) {
    const FlatOp& f = recs[tk.op0 - op_base + o];
    if (f.kind == FK_GATHER) r += f.k0 + ((f.flags & FF_TWO) ? f.k1 : 0);
    else if (f.kind == FK_SCATTER) r += f.c0;
    else if (f.kind == FK_MIDDLE) r += (f.flags & FF_ADJ) ? f.c0 : f.k0;
    else r += (f.flags & FF_ADJ) ? f.k1 : n0;
  }
  return r;
}

// out_i = cand[q_i] + sum_j M(i, j) cand[p_j]  (V layout M[j*k+i]; CJ: conj(M[i*nr+j]))
template <class T, class F>
__device__ __forceinline__ typename CT1<T>::t row_gather(const F* M, const int16_t* I, int k, int c, bool cj,
                                                         const typename CT1<T>::t* cand, int i) {
  using C = typename CT1<T>::t;
  const int nr = c - k;
  C acc = cand[I[i]], acc2 = {(T)0, (T)0};   // two chains: even and odd inputs, summed at the end
  int j = 0;
  if (cj) {
    for (; j + 1 < nr; j += 2) {
      fma1(acc, cvc1<T>(M[i * nr + j]), cand[I[k + j]]);
      fma1(acc2, cvc1<T>(M[i * nr + j + 1]), cand[I[k + j + 1]]);
    }
    if (j < nr) fma1(acc, cvc1<T>(M[i * nr + j]), cand[I[k + j]]);
  } else {
    for (; j + 1 < nr; j += 2) {
      fma1(acc, cv1<T>(M[j * k + i]), cand[I[k + j]]);
      fma1(acc2, cv1<T>(M[(j + 1) * k + i]), cand[I[k + j + 1]]);
    }
    if (j < nr) fma1(acc, cv1<T>(M[j * k + i]), cand[I[k + j]]);
  }
  acc.x += acc2.x;
  acc.y += acc2.y;
  return acc;
}

// contribution of one block to candidate entry r (U layout M[i*nr+j]; CJ: conj(M[j*k+i]))
template <class T, class F>
__device__ __forceinline__ void w_row(typename CT1<T>::t& acc, const F* M, const int16_t* I, int k, int c, bool cj,
                                      const typename CT1<T>::t* yv, int r) {
  const int code = I[c + r];
  if (code >= 0) {
    acc.x += yv[code].x;
    acc.y += yv[code].y;
  } else {
    const int j = -1 - code, nr = c - k;
    if (cj) {
      for (int i = 0; i < k; ++i) fma1(acc, cvc1<T>(M[j * k + i]), yv[i]);
    } else {
      for (int i = 0; i < k; ++i) fma1(acc, cv1<T>(M[i * nr + j]), yv[i]);
    }
  }
}

template <class T, class F>
__device__ __forceinline__ const int16_t* op_idx(const char* area, const FlatOp& f) {
  return (const int16_t*)(area + f.soff + al16((int64_t)f.melems * (int64_t)sizeof(F)));
}

// row lr of task tk
template <class T, class F>
__device__ void run_row(const A1Args& a, const A1Task& tk, const FlatOp* recs, int op_base, const char* area,
                        const typename CT1<T>::t* sv, int lr) {
  using C = typename CT1<T>::t;
  C* st = (C*)a.st;
  C* y = (C*)a.y;
  const int n0 = (int)a.n0;
  if (tk.kind == 3) {
    // EXIT: row lr of the leaf = the rows the previous phase left + each depth's contribution, in order
    C acc = sv[tk.pad + lr];
    int out = 0;
    for (int o = 0; o < tk.nops; ++o) {
      const FlatOp& f = recs[tk.op0 - op_base + o];
      w_row<T, F>(acc, (const F*)(area + f.soff), op_idx<T, F>(area, f), f.k0, f.c0, (f.flags & FF_CONJ) != 0,
                  sv + f.pad, lr);
      out = f.out0;
    }
    y[out + lr] = acc;
    return;
  }
  if (tk.kind == 0) {
    // ENTER: find the op (depth) of the row
    int o = 0;
    for (; o + 1 < tk.nops; ++o) {
      const int k = recs[tk.op0 - op_base + o].k0;
      if (lr < k) break;
      lr -= k;
    }
    const FlatOp& f = recs[tk.op0 - op_base + o];
    st[f.out0 + lr] = row_gather<T, F>((const F*)(area + f.soff), op_idx<T, F>(area, f), f.k0, f.c0,
                                       (f.flags & FF_CONJ) != 0, sv + f.pad, lr);
    return;
  }
  const FlatOp& f = recs[tk.op0 - op_base];
  const F* M = (const F*)(area + f.soff);
  const C* in = sv + f.pad;
  if (f.kind == FK_GATHER) {
    const int16_t* I = op_idx<T, F>(area, f);
    const bool cj = (f.flags & FF_CONJ) != 0;
    if (lr < f.k0) st[f.out0 + lr] = row_gather<T, F>(M, I, f.k0, f.c0, cj, in, lr);
    else st[f.out1 + lr - f.k0] = row_gather<T, F>(M + f.m1, I + f.i1, f.k1, f.c1, cj, in, lr - f.k0);
  } else if (f.kind == FK_SCATTER) {
    const int16_t* I = op_idx<T, F>(area, f);
    const bool cj = (f.flags & FF_CONJ) != 0;
    C acc = {(T)0, (T)0};
    w_row<T, F>(acc, M, I, f.k0, f.c0, cj, in, lr);
    if (f.flags & FF_TWO) w_row<T, F>(acc, M + f.m1, I + f.i1, f.k1, f.c1, cj, in + f.n_s0, lr);
    if (!(f.flags & FF_TWO) || lr < f.split) st[f.out0 + lr] = acc;
    else st[f.out1 + (lr - f.split)] = acc;
  } else if (f.kind == FK_MIDDLE) {   // y = S z (adjoint z = S^H y), S stored [c][r]
    const int kr = f.k0, kc = f.c0;
    C acc = {(T)0, (T)0};
    if (f.flags & FF_ADJ) {
      for (int i = 0; i < kr; ++i) fma1(acc, cvc1<T>(M[lr * kr + i]), in[i]);
    } else {
      for (int i = 0; i < kc; ++i) fma1(acc, cv1<T>(M[i * kr + lr]), in[i]);
    }
    st[f.out0 + lr] = acc;
  } else {   // dense-leaf column chunk, column-major [cc][r]
    const int cn = f.k1;
    if (!(f.flags & FF_ADJ)) {
      C acc = (f.flags & FF_ACC) ? in[f.n_s0 + lr] : C{(T)0, (T)0}, acc2 = {(T)0, (T)0};
      int cc = 0;
      for (; cc + 1 < cn; cc += 2) {
        fma1(acc, cv1<T>(M[cc * n0 + lr]), in[cc]);
        fma1(acc2, cv1<T>(M[(cc + 1) * n0 + lr]), in[cc + 1]);
      }
      if (cc < cn) fma1(acc, cv1<T>(M[cc * n0 + lr]), in[cc]);
      acc.x += acc2.x;
      acc.y += acc2.y;
      y[f.out0 + lr] = acc;
    } else {
      // output lr = a column of the chunk: the rows visited from a per-row offset so that
      // neighbouring lanes read different banks
      C acc = {(T)0, (T)0};
      for (int rr = 0; rr < n0; ++rr) {
        const int r = (rr + lr) % n0;
        fma1(acc, cvc1<T>(M[lr * n0 + r]), in[r]);
      }
      y[f.out0 + lr] = acc;
    }
  }
}

// all rows of a batch, one warp; pre: per-warp scratch of kA1MaxTasks + 1 ints
template <class T, class F>
__device__ void run_batch(const A1Args& a, const A1Batch& B, const char* area, const typename CT1<T>::t* sv,
                          int* pre, int lane) {
  const A1Task* tks = (const A1Task*)area;
  const FlatOp* recs = (const FlatOp*)(area + B.rec_off);
  const int n0 = (int)a.n0;
  // row offsets of the tasks: lane l sums tasks 4l .. 4l+3, then a warp scan
  int c[4], s = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int t = 4 * lane + u;
    c[u] = t < B.ntasks ? task_rows(tks[t], recs, B.op0, n0) : 0;
    s += c[u];
  }
  int incl = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  int run = incl - s;
  if (lane == 0) pre[0] = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    run += c[u];
    if (4 * lane + u < B.ntasks) pre[4 * lane + u + 1] = run;
  }
  __syncwarp();
  const int R = pre[B.ntasks];
  for (int r = lane; r < R; r += 32) {
    int lo = 0, hi = B.ntasks;   // pre[lo] <= r < pre[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pre[mid] <= r) lo = mid;
      else hi = mid;
    }
    run_row<T, F>(a, tks[lo], recs, B.op0, area, sv, r - pre[lo]);
  }
  __syncwarp();
}

template <class T, class F>
__global__ void __launch_bounds__(kA1Threads, 1) k_apply1(A1Args a) {
  using C = typename CT1<T>::t;
  extern __shared__ __align__(128) char ring[];
  __shared__ int s_off[kA1Slots];                 // ring offset of each batch in flight
  __shared__ int s_bdone[kA1Slots];               // q + 1 once batch q (slot q % kA1Slots) is consumed
  __shared__ __align__(8) uint64_t s_mbar[kA1Slots];
  __shared__ __align__(16) A1Batch s_brec[32];    // the producer's window of batch records
  __shared__ int s_abort, s_issued;
  __shared__ int s_pre[kA1Cw][kA1MaxTasks + 1];   // per-warp row offsets of a batch's tasks
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b0 = a.cta_batch[blockIdx.x], b1 = a.cta_batch[blockIdx.x + 1];
  const int nb = b1 - b0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kA1Slots; ++k) {
      mb_init(&s_mbar[k], 1);
      s_bdone[k] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();
  if (warp == kA1Cw) {
    // ---- producer: batches [b0, b1) in order into the ring; [oldest, q) in flight.
    // Batch q is consumed by compute warp q % kA1Cw; completions come out of order, the
    // ring space is recycled from the oldest batch not yet consumed.
    int head = 0, q = 0, oldest = 0;
    long long spins = 0;
    for (; q < nb; ++q) {
      if ((q & 31) == 0) {
        // next window of 32 batch records, one per lane
        __syncwarp();
        if (q + lane < nb) s_brec[lane] = a.batches[b0 + q + lane];
        __syncwarp();
      }
      const A1Batch B = s_brec[q & 31];
      int off = -1;
      for (;;) {
        while (oldest < q && *(volatile int*)&s_bdone[oldest % kA1Slots] == oldest + 1) ++oldest;
        __threadfence_block();
        if (*(volatile int*)&s_abort) break;
        if (q - oldest < kA1Slots) {
          if (oldest == q) {
            off = 0;
          } else {
            const int tail = s_off[oldest % kA1Slots];
            if (head > tail) {
              if (head + B.area_bytes <= a.ring_bytes) off = head;
              else if (B.area_bytes <= tail) off = 0;
            } else if (head < tail) {
              if (head + B.area_bytes <= tail) off = head;
            }
          }
        }
        if (off >= 0) break;
        if (++spins > a.spin_limit) {
          if (lane == 0) atomicExch(&s_abort, 1);
          break;
        }
        __nanosleep(20);
      }
      if (off < 0) break;
      spins = 0;
      uint64_t* mb = &s_mbar[q % kA1Slots];
      char* dst = ring + off;
      if (lane == 0) {
        s_off[q % kA1Slots] = off;
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mb_arrive_tx(mb, (unsigned)B.tma_bytes);
      }
      __syncwarp();
      if (lane == 0) bulk_copy(dst, a.image + B.img, (unsigned)B.tma_bytes, mb);   // the batch's image
      head = off + B.area_bytes;
    }
    if (lane == 0) s_issued = q;
    __syncwarp();
  } else {
    // ---- compute warp: its batches q = warp, warp + kA1Cw, ... (in phase order)
    bool bad = false;   // uniform within the warp
    for (int q = warp; q < nb && !bad; q += kA1Cw) {
      const A1Batch B = a.batches[b0 + q];
      uint64_t* mb = &s_mbar[q % kA1Slots];
      const unsigned par = (unsigned)(q / kA1Slots) & 1u;
      long long spins = 0;
      bool w_ok = true;
      while (!mb_try_wait(mb, par)) {
        if (++spins > a.spin_limit || *(volatile int*)&s_abort) { w_ok = false; break; }
      }
      if (__any_sync(0xffffffffu, !w_ok)) { bad = true; break; }
      const char* area = ring + s_off[q % kA1Slots];
      // the producers of the entries this batch gathers (lanes in parallel)
      const int32_t* dep = (const int32_t*)(area + B.dep_off);
      for (int k = lane; k < B.ndep; k += 32) {
        const unsigned* fl = (const unsigned*)(a.done + dep[k]);
        spins = 0;
        while (ld_acq(fl) != (unsigned)a.epoch) {
          if (++spins > a.spin_limit || *(volatile int*)&a.gb->err || *(volatile int*)&s_abort) { w_ok = false; break; }
          __nanosleep(32);
        }
        if (!w_ok) break;
      }
      if (__any_sync(0xffffffffu, !w_ok)) { bad = true; break; }
      const uint32_t* gl = (const uint32_t*)(area + B.gl_off);
      C* sv = (C*)(ring + s_off[q % kA1Slots] + B.vec_off);
      const C* xv = (const C*)a.x;
      const C* yv = (const C*)a.y;
      const C* stv = (const C*)a.st;
      for (int e = lane; e < B.nvec; e += 32) {
        const uint32_t s = gl[e];
        const C* src = ((s & kA1FromY) == kA1FromY) ? yv + (s & 0x3FFFFFFFu)
                       : (s & kA1FromX) ? xv + (s & 0x3FFFFFFFu) : stv + s;
        sv[e] = ldcg1(src);
      }
      __syncwarp();
      run_batch<T, F>(a, B, area, sv, s_pre[warp], lane);
      __syncwarp();
      if (lane == 0) {
        // outputs first (the warp's writes, ordered by the warp barrier and this
        // cumulative fence), then the completion flag
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(a.done + b0 + q), "r"((unsigned)a.epoch) : "memory");
        __threadfence_block();
        *(volatile int*)&s_bdone[q % kA1Slots] = q + 1;   // releases the batch's slot and ring area
      }
    }
    if (bad && lane == 0) {
      atomicExch(&s_abort, 1);
      atomicExch(a.err_out, 1);
      atomicExch(&a.gb->err, 1);
    }
  }
  __syncthreads();
  if (*(volatile int*)&s_abort) {
    // give the copies still in flight a second bounded wait before leaving
    const int iss = s_issued;
    for (int q = 0; q < iss; ++q) {
      if (s_bdone[q % kA1Slots] == q + 1 || q + kA1Slots < iss) continue;
      long long spins = 0;
      while (!mb_try_wait(&s_mbar[q % kA1Slots], (unsigned)(q / kA1Slots) & 1u) && ++spins < drain_limit(a.spin_limit)) {
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < kA1Slots; ++k) mb_inval(&s_mbar[k]);
}

template <class T, class F>
int launch1(const DevFactor& df, bool adj, const void* x, void* y, void* st, cudaStream_t s) {
  DevPlan& pl = const_cast<DevPlan&>(df.plan[adj ? 1 : 0]);   // the epoch counter advances per launch
  auto kern = k_apply1<T, F>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kA1RingBytes);
    attr_done = true;
  }
  A1Args a;
  a.batches = pl.batches;
  a.cta_batch = pl.cta_batch;
  a.image = pl.image;
  a.nphase = pl.nphase;
  a.ring_bytes = kA1RingBytes;
  a.x = x;
  a.y = y;
  a.st = st;
  a.n0 = df.n0;
  a.gb = (GridBar*)df.abar;
  a.done = pl.done;
  a.epoch = ++pl.epoch;
  a.err_out = &((GridBar*)df.bar)->err;
  a.spin_limit = df.spin_limit;
  if (cudaMemsetAsync(df.abar, 0, sizeof(GridBar), s) != cudaSuccess) return HB_ECUDA;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3(pl.grid), dim3(kA1Threads), args,
                                              kA1RingBytes, s);
  if (e != cudaSuccess) {
    set_error("persistent apply launch failed: %s", cudaGetErrorString(e));
    return HB_ECUDA;
  }
  return HB_OK;
}

}  // namespace

bool apply1_ready(const DevFactor& df, bool adj) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const DevPlan& pl = df.plan[adj ? 1 : 0];
  return pl.ok && pl.grid == sms && df.abar != nullptr;
}

int launch_apply1(const DevFactor& df, Prec p, bool adj, const void* x, void* y, void* st, cudaStream_t s) {
  if (p == PREC_F64) return launch1<double, double2>(df, adj, x, y, st, s);
  if (p == PREC_F32) return launch1<float, float2>(df, adj, x, y, st, s);
  return launch1<double, float2>(df, adj, x, y, st, s);
}

}  // namespace hb

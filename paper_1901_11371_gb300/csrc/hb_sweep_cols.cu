// Column-partitioned sweep kernel (sm_103a): x = L~^{-1} b, U~^{-1} b and
// their adjoints (Algs. 3, 4) for many right-hand sides, in place.
//
// The sweep is a long chain of small dependent phases (one sweep-leaf solve,
// then the butterfly that carries its result to the next subtree, ...).  Run
// grid-wide, every link costs a grid barrier; run by one CTA, every link is a
// shared-memory round trip.  So here each CTA runs the whole sweep for its own
// one or two right-hand sides and never waits on another CTA:
//   * a producer warp streams the schedule's batch images (host-built, see
//     hb_swsched.cpp) into a shared-memory ring with one cp.async.bulk each,
//     as far ahead as the ring allows -- the factor data never depends on the
//     vectors;
//   * resident runs (subtrees whose rows and butterfly state fit the 96 KB
//     window) start by loading their rows into shared memory and end by
//     writing them back; inside them every phase reads and writes the window;
//   * global phases (stages of the large butterflies) read and write the
//     vector rows and a CTA-private butterfly state in global memory;
//   * a butterfly phase is a sparse product in row form: compute warp w takes
//     the batches w, w + 16, ...; in a batch, groups of 2^glog lanes share a
//     row (entries strided over the lanes, then a shuffle reduction), so that
//     short dot products do not serialise on one lane;
//   * a sweep-leaf phase (packed triangle, in place on the window rows) is
//     taken by all compute warps: pairs of rows (j, s-1-j) times column
//     groups, partial sums, a barrier, the reduction written back.
// Consecutive phases are separated by one named barrier among the compute
// warps.  Every wait is bounded; a wait that gives up raises the factor's
// error flag (reported by hb_status / the solvers) and the CTA returns after a
// second bounded wait for its copies still in flight.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hb_device.h"
#include "hb_sweep_launch.h"

namespace hb {

namespace {

constexpr int kSwThreads = (kSwWarps + 1) * 32;
constexpr int kSwSlots = 64;   // batches in flight per CTA
constexpr int kSwSmem = kSwRingBytes + kSwWinBytes + kSwPartBytes;
static_assert(kSwSmem <= 224 * 1024, "dynamic shared memory of the column-partitioned sweep");

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
// non-blocking test: the consumers count polls, so that a wait limit of one poll
// gives up at once on a batch still in flight
__device__ __forceinline__ bool mb_test_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(b)) : "memory");
}
__device__ __forceinline__ void cw_sync() {   // named barrier 1 among the compute warps
  asm volatile("bar.sync 1, %0;\n" ::"n"(kSwWarps * 32) : "memory");
}
__device__ __forceinline__ bool cw_red_or(bool v) {
  unsigned r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
               : "=r"(r) : "r"((unsigned)v), "n"(kSwWarps * 32) : "memory");
  return r != 0;
}

struct SwArgs {
  const SwStep* steps;
  int nstep;
  const SwBatch* batches;
  int64_t nbatch;
  const uint8_t* image;
  float2* x;           // vectors, layout [row][R]
  int64_t R, n;
  int64_t col0;        // first column of this launch
  float2* st;          // CTA-private butterfly state: [CTA][state_len][NC]
  int64_t state_len;
  int* err_out;        // the factor's sticky error flag
  long long spin_limit;
};

template <int NC>
struct Cv {
  float2 v[NC];
};

__device__ __forceinline__ void cmac(float2& acc, const float2 a, const float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// NC window entries (16-byte vector load for two columns)
template <int NC>
__device__ __forceinline__ Cv<NC> win_load(const float2* p) {
  Cv<NC> r;
  if constexpr (NC == 2) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r.v[0] = make_float2(v.x, v.y);
    r.v[1] = make_float2(v.z, v.w);
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) r.v[c] = p[c];
  }
  return r;
}

// input slot of a global phase: a vector row (this CTA's columns of x) or a
// CTA-private state entry
template <int NC>
__device__ __forceinline__ Cv<NC> glob_load(const SwArgs& a, int32_t s, const float2* xb, const float2* stp, int ncol) {
  Cv<NC> r;
  if (s < a.n) {
    const float2* p = xb + (int64_t)s * a.R;
#pragma unroll
    for (int c = 0; c < NC; ++c) r.v[c] = c < ncol ? p[c] : make_float2(0.f, 0.f);
  } else {
    r = win_load<NC>(stp + (int64_t)(s - a.n) * NC);
  }
  return r;
}

// One batch of a butterfly phase in row form, one warp.  RES: slots are window
// positions (int16), else global slots (int32).
template <int NC, bool RES>
__device__ void run_rows(const SwArgs& a, const SwBatch& B, const char* area, float2* win, float2* xb, float2* stp,
                         int ncol, int lane) {
  const int32_t* out = reinterpret_cast<const int32_t*>(area);
  const int32_t* e0 = reinterpret_cast<const int32_t*>(area + B.off_e0);
  const float2* cf = reinterpret_cast<const float2*>(area + B.off_coef);
  const int16_t* in16 = reinterpret_cast<const int16_t*>(area + B.off_in);
  const int32_t* in32 = reinterpret_cast<const int32_t*>(area + B.off_in);
  const int glog = B.glog, G = 1 << glog, ng = 32 >> glog;
  const int q = lane >> glog, l = lane & (G - 1);
  for (int base = 0; base < B.nrows; base += ng) {
    const int r = base + q;
    float2 acc[NC], acc2[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = acc2[c] = make_float2(0.f, 0.f);
    if (r < B.nrows) {
      const int ea = e0[r], eb = e0[r + 1];
      int e = ea + l;
      // two independent accumulator chains
      for (; e + G < eb; e += 2 * G) {
        const float2 m0 = cf[e], m1 = cf[e + G];
        Cv<NC> v0, v1;
        if constexpr (RES) {
          v0 = win_load<NC>(win + (int)in16[e] * NC);
          v1 = win_load<NC>(win + (int)in16[e + G] * NC);
        } else {
          v0 = glob_load<NC>(a, in32[e], xb, stp, ncol);
          v1 = glob_load<NC>(a, in32[e + G], xb, stp, ncol);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          cmac(acc[c], m0, v0.v[c]);
          cmac(acc2[c], m1, v1.v[c]);
        }
      }
      if (e < eb) {
        const float2 m0 = cf[e];
        Cv<NC> v0;
        if constexpr (RES) v0 = win_load<NC>(win + (int)in16[e] * NC);
        else v0 = glob_load<NC>(a, in32[e], xb, stp, ncol);
#pragma unroll
        for (int c = 0; c < NC; ++c) cmac(acc[c], m0, v0.v[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      acc[c].x += acc2[c].x;
      acc[c].y += acc2[c].y;
    }
    // sum over the group's lanes (groups are aligned runs of G lanes)
    for (int d = G >> 1; d > 0; d >>= 1) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        acc[c].x += __shfl_xor_sync(0xffffffffu, acc[c].x, d);
        acc[c].y += __shfl_xor_sync(0xffffffffu, acc[c].y, d);
      }
    }
    if (l == 0 && r < B.nrows) {
      const int32_t o = out[r];
      const bool add = (o & kSwAcc) != 0;
      const int32_t s = o & ~kSwAcc;
      if (RES) {
        float2* d = win + (int64_t)s * NC;
#pragma unroll
        for (int c = 0; c < NC; ++c) d[c] = add ? make_float2(d[c].x + acc[c].x, d[c].y + acc[c].y) : acc[c];
      } else if (s < a.n) {
        float2* d = xb + (int64_t)s * a.R;
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < ncol) d[c] = add ? make_float2(d[c].x + acc[c].x, d[c].y + acc[c].y) : acc[c];
      } else {
        float2* d = stp + (int64_t)(s - a.n) * NC;
#pragma unroll
        for (int c = 0; c < NC; ++c) d[c] = add ? make_float2(d[c].x + acc[c].x, d[c].y + acc[c].y) : acc[c];
      }
    }
  }
}

// Sweep-leaf phase: window rows a0 .. a0 + s - 1 replaced by T times them (T the
// packed triangle), all compute threads (t < nct).  Thread (pair j, column
// group g) owns rows j and s-1-j (s + 1 entries together) and the columns
// c = g (mod ncg) of them.  The triangle is not read after the first barrier.
template <int NC>
__device__ void run_tri(const SwBatch& B, const float2* T, float2* win, float2* part, int t, int nct) {
  const int s = B.nrows;
  const bool up = (B.flags & SWF_UPPER) != 0;
  float2* b = win + (int64_t)B.a0 * NC;
  const int npair = s >> 1;
  int ncg = nct / npair;
  const int cap = kSwPartBytes / (s * NC * 8);
  if (ncg > cap) ncg = cap;
  if (ncg < 1) ncg = 1;
  if (t < npair * ncg) {
    const int j = t % npair, g = t / npair;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h == 0 ? j : s - 1 - j;
      float2 acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = make_float2(0.f, 0.f);
      if (up) {
        // row r: columns r .. s-1; entry (r, c) at c (c + 1) / 2 + r.  The lanes of a warp
        // share g and step through the same columns (a predicate skips c < r).
        for (int c = g; c < s; c += ncg) {
          if (c >= r) {
            const float2 m = T[((c * (c + 1)) >> 1) + r];
            const Cv<NC> v = win_load<NC>(b + (int64_t)c * NC);
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) cmac(acc[cc], m, v.v[cc]);
          }
        }
      } else {
        // row r: columns 0 .. r; entry (r, c) at c s - c (c - 1) / 2 + r - c
        for (int c = g; c <= r; c += ncg) {
          const float2 m = T[c * s - ((c * (c - 1)) >> 1) + r - c];
          const Cv<NC> v = win_load<NC>(b + (int64_t)c * NC);
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) cmac(acc[cc], m, v.v[cc]);
        }
      }
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) part[((int64_t)g * s + r) * NC + cc] = acc[cc];
    }
  }
  cw_sync();
  for (int e = t; e < s * NC; e += nct) {
    const int r = e / NC, cc = e % NC;
    float2 sum = make_float2(0.f, 0.f);
    for (int g = 0; g < ncg; ++g) {
      const float2 p = part[((int64_t)g * s + r) * NC + cc];
      sum.x += p.x;
      sum.y += p.y;
    }
    b[(int64_t)r * NC + cc] = sum;
  }
}

template <int NC>
__global__ void __launch_bounds__(kSwThreads, 1) k_sweep_cols(SwArgs a) {
  extern __shared__ __align__(128) char smem[];
  char* ring = smem;
  float2* win = reinterpret_cast<float2*>(smem + kSwRingBytes);
  float2* part = reinterpret_cast<float2*>(smem + kSwRingBytes + kSwWinBytes);
  __shared__ int s_off[kSwSlots];                 // ring offset of each batch in flight
  __shared__ int s_bdone[kSwSlots];               // q + 1 once batch q (slot q % kSwSlots) is consumed
  __shared__ __align__(8) uint64_t s_mbar[kSwSlots];
  __shared__ __align__(16) SwBatch s_brec[32];    // the producer's window of batch records
  __shared__ int s_abort, s_issued;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t lb = a.col0 + (int64_t)blockIdx.x * NC;
  const int ncol = (int)((a.R - lb) < NC ? (a.R - lb) : NC);
  float2* xb = a.x + lb;
  float2* stp = a.st + (int64_t)blockIdx.x * a.state_len * NC;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kSwSlots; ++k) {
      mb_init(&s_mbar[k], 1);
      s_bdone[k] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();
  if (warp == kSwWarps) {
    // ---- producer: every batch of the schedule, in order, into the ring; batches
    // [oldest, q) are in flight; the ring space is recycled from the oldest batch
    // not yet consumed (completions come out of order).  Lane 0 keeps the ring
    // state and issues the copies; the warp loads the batch records 32 at a time.
    int head = 0, oldest = 0;
    int64_t q = 0;
    for (; q < a.nbatch; ++q) {
      if ((q & 31) == 0) {
        __syncwarp();
        if (q + lane < a.nbatch) s_brec[lane] = a.batches[q + lane];
        __syncwarp();
      }
      int off = -1;
      if (lane == 0) {
        const SwBatch& B = s_brec[q & 31];
        const int bytes = B.bytes;
        long long spins = 0;
        for (;;) {
          while (oldest < q && *(volatile int*)&s_bdone[oldest % kSwSlots] == oldest + 1) ++oldest;
          __threadfence_block();
          if (*(volatile int*)&s_abort) break;
          if (q - oldest < kSwSlots) {
            if (oldest == q) {
              off = 0;
            } else {
              const int tail = s_off[oldest % kSwSlots];
              if (head > tail) {
                if (head + bytes <= kSwRingBytes) off = head;
                else if (bytes <= tail) off = 0;
              } else if (head < tail) {
                if (head + bytes <= tail) off = head;
              }
            }
          }
          if (off >= 0) break;
          if (++spins > a.spin_limit) {
            atomicExch(&s_abort, 1);
            break;
          }
          __nanosleep(20);
        }
        if (off >= 0) {
          uint64_t* mb = &s_mbar[q % kSwSlots];
          s_off[q % kSwSlots] = off;
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mb_arrive_tx(mb, (unsigned)bytes);
          bulk_copy(ring + off, a.image + B.img, (unsigned)bytes, mb);
          head = off + bytes;
        }
      }
      off = __shfl_sync(0xffffffffu, off, 0);
      if (off < 0) break;
    }
    if (lane == 0) s_issued = (int)q;
    __syncwarp();
  } else {
    const int t = threadIdx.x, nct = kSwWarps * 32;
    bool bad = false;   // uniform among the compute warps after each step
    for (int si = 0; si < a.nstep && !bad; ++si) {
      const SwStep S = a.steps[si];
      if (S.kind == SW_BEGIN) {
        const int nrow = S.a1 - S.a0;
        for (int e = t; e < nrow * NC; e += nct) {
          const int r = e / NC, c = e % NC;
          win[e] = c < ncol ? __ldcg(xb + (int64_t)(S.a0 + r) * a.R + c) : make_float2(0.f, 0.f);
        }
      } else if (S.kind == SW_END) {
        const int nrow = S.a1 - S.a0;
        for (int e = t; e < nrow * NC; e += nct) {
          const int r = e / NC, c = e % NC;
          if (c < ncol) xb[(int64_t)(S.a0 + r) * a.R + c] = win[e];
        }
      } else if (S.flags & SWF_TRI) {
        const int64_t q = S.a0;
        long long spins = 0;
        bool ok = true;
        while (!mb_test_wait(&s_mbar[q % kSwSlots], (unsigned)(q / kSwSlots) & 1u)) {
          if (++spins > a.spin_limit || *(volatile int*)&s_abort) { ok = false; break; }
        }
        if (cw_red_or(!ok)) { bad = true; break; }
        const SwBatch B = a.batches[q];
        run_tri<NC>(B, reinterpret_cast<const float2*>(ring + s_off[q % kSwSlots]), win, part, t, nct);
        if (t == 0) {
          __threadfence_block();
          *(volatile int*)&s_bdone[q % kSwSlots] = (int)q + 1;   // the triangle was read before run_tri's barrier
        }
      } else {
        const bool res = (S.flags & SWF_RES) != 0;
        for (int64_t q = S.a0 + warp; q < (int64_t)S.a0 + S.a1; q += kSwWarps) {
          const SwBatch B = a.batches[q];
          long long spins = 0;
          bool ok = true;
          while (!mb_test_wait(&s_mbar[q % kSwSlots], (unsigned)(q / kSwSlots) & 1u)) {
            if (++spins > a.spin_limit || *(volatile int*)&s_abort) { ok = false; break; }
          }
          if (__any_sync(0xffffffffu, !ok)) { bad = true; break; }
          const char* area = ring + s_off[q % kSwSlots];
          if (res) run_rows<NC, true>(a, B, area, win, xb, stp, ncol, lane);
          else run_rows<NC, false>(a, B, area, win, xb, stp, ncol, lane);
          __syncwarp();
          if (lane == 0) {
            __threadfence_block();
            *(volatile int*)&s_bdone[q % kSwSlots] = (int)q + 1;   // releases the batch's ring area
          }
        }
      }
      // end of the step: every compute warp's writes are visible to the next step
      if (cw_red_or(bad)) bad = true;
    }
    if (bad && t == 0) {
      atomicExch(&s_abort, 1);
      atomicExch(a.err_out, 1);
    }
  }
  __syncthreads();
  if (*(volatile int*)&s_abort) {
    // give the copies still in flight a second bounded wait before leaving
    const int iss = s_issued;
    for (int q = 0; q < iss; ++q) {
      if (s_bdone[q % kSwSlots] == q + 1 || q + kSwSlots < iss) continue;
      long long spins = 0;
      while (!mb_try_wait(&s_mbar[q % kSwSlots], (unsigned)(q / kSwSlots) & 1u) &&
             ++spins < drain_limit(a.spin_limit)) {
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < kSwSlots; ++k) mb_inval(&s_mbar[k]);
}

template <int NC>
int launch_nc(const DevFactor& df, const DevSched& sc, float2* vec, int64_t R, int64_t col0, int grid, float2* st,
              cudaStream_t s) {
  auto kern = k_sweep_cols<NC>;
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSwSmem) != cudaSuccess) {
      set_error("column-partitioned sweep: shared-memory attribute failed");
      return HB_ECUDA;
    }
    attr_done = true;
  }
  SwArgs a;
  a.steps = sc.steps;
  a.nstep = sc.nstep;
  a.batches = sc.batches;
  a.nbatch = sc.nbatch;
  a.image = sc.image;
  a.x = vec;
  a.R = R;
  a.n = df.n;
  a.col0 = col0;
  a.st = st;
  a.state_len = df.state_len;
  a.err_out = &((GridBar*)df.bar)->err;
  a.spin_limit = df.spin_limit;
  kern<<<grid, kSwThreads, kSwSmem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("column-partitioned sweep launch failed: %s", cudaGetErrorString(e));
    return HB_ECUDA;
  }
  return HB_OK;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

int64_t sweep_cols_state_entries(const DevFactor& df, int64_t R) {
  // launches cover 2 * sms columns at a time (one column per CTA when R <= sms)
  const int64_t sms = sm_count();
  if (R <= sms) return df.state_len * R;
  const int64_t cols = std::min<int64_t>(R, 2 * sms);
  return df.state_len * ((cols + 1) / 2) * 2;
}

int launch_sweep_cols(const DevFactor& df, int which, void* vec, int64_t R, void* state, cudaStream_t s) {
  if (which < 0 || which > 3 || !df.sw[which].ok) {
    set_error("column-partitioned sweep: no schedule for this sweep");
    return HB_EUNSUPPORTED;
  }
  const DevSched& sc = df.sw[which];
  const int64_t sms = sm_count();
  float2* v = static_cast<float2*>(vec);
  float2* st = static_cast<float2*>(state);
  if (R <= sms) return launch_nc<1>(df, sc, v, R, 0, (int)R, st, s);
  for (int64_t c0 = 0; c0 < R; c0 += 2 * sms) {
    const int64_t cols = std::min<int64_t>(R - c0, 2 * sms);
    const int rc = launch_nc<2>(df, sc, v, R, c0, (int)((cols + 1) / 2), st, s);
    if (rc) return rc;
  }
  return HB_OK;
}

int sweep_cols_launches(int64_t R) {
  const int64_t sms = sm_count();
  return R <= sms ? 1 : (int)((R + 2 * sms - 1) / (2 * sms));
}

}  // namespace hb

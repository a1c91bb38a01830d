// Column-partitioned sweep kernel (sm_103a): x = L~^{-1} b, U~^{-1} b and
// their adjoints (Algs. 3, 4) for many right-hand sides, in place.
//
// The sweep is a long chain of small dependent phases (one sweep-leaf solve,
// then the butterfly that carries its result to the next subtree, ...).  Run
// grid-wide, every link costs a grid barrier; run by one CTA, every link is a
// shared-memory round trip.  So here each CTA runs the whole sweep for its own
// one or two right-hand sides and never waits on another CTA:
//   * a producer warp streams the schedule's group images (host-built, see
//     hb_swsched.cpp: a header, batch descriptors, the batches' data) into a
//     shared-memory ring with one cp.async.bulk each, as far ahead as the
//     ring allows -- the factor data never depends on the vectors, and the
//     compute warps find every record they need in the ring;
//   * resident runs (subtrees whose rows and butterfly state fit the 96 KB
//     window) start by loading their rows into shared memory and end by
//     writing them back; inside them every phase reads and writes the window;
//   * global phases (stages of the large butterflies) read and write the
//     vector rows and a CTA-private butterfly state in global memory: a batch
//     first gathers its distinct inputs into its warp's slice of the window
//     (free between runs) in one round trip;
//   * the resident runs -- the long dependent chain -- are executed by eight
//     chain warps (two per scheduler) with their own barrier: a phase's rows
//     are spread over eight warps, and a sweep leaf's columns over 256 threads,
//     while the per-phase overhead is paid eight times, not twelve; the other
//     compute warps wait for the run's end; a global phase's batches go
//     round-robin to all twelve compute warps;
//   * a butterfly phase is a sparse product in row form; in a batch, groups of
//     2^glog lanes share a row (entries strided over the lanes, then a shuffle
//     reduction), so that short dot products do not serialise on one lane;
//   * a sweep-leaf phase (packed triangle, in place on the window rows) is
//     taken by all chain warps: pairs of rows (j, s-1-j) times column groups,
//     four independent accumulation chains, partial sums, a barrier, the
//     reduction written back.
// Consecutive phases are separated by one named barrier among the compute
// warps; the groups of one phase are not.  Every wait is bounded; a warp whose
// wait gives up stops computing but still meets the barriers up to the end of
// the phase, where all compute warps learn of it and stop; the factor's error
// flag is raised (reported by hb_status / the solvers) and the CTA returns
// after a second bounded wait for its copies still in flight.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hb_device.h"
#include "hb_sweep_launch.h"

namespace hb {

namespace {

constexpr int kSwThreads = (kSwWarps + 1) * 32;
// at most four warps per scheduler: every thread may hold 128 registers
static_assert((kSwWarps + 1 + 3) / 4 * 128 * 32 <= 16384, "registers per scheduler");
constexpr int kSwSlots = 64;   // groups in flight per CTA
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
// asynchronous global -> shared copy of `bytes` (8 or 16), the first `src_bytes` of
// them from src and the rest zero
__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes, int src_bytes) {
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(dst)), "l"(src), "r"(src_bytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(su32(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(b)) : "memory");
}
__device__ __forceinline__ void ch_sync() {   // named barrier 2 among the chain warps
  asm volatile("bar.sync 2, %0;\n" ::"n"(kSwChain * 32) : "memory");
}
__device__ __forceinline__ bool ch_red_or(bool v) {
  unsigned r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 2, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
               : "=r"(r) : "r"((unsigned)v), "n"(kSwChain * 32) : "memory");
  return r != 0;
}
__device__ __forceinline__ bool cw_red_or(bool v) {
  unsigned r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
               : "=r"(r) : "r"((unsigned)v), "n"(kSwWarps * 32) : "memory");
  return r != 0;
}

struct SwArgs {
  const SwGroup* groups;
  int64_t ngroup;
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

// NC consecutive shared-memory entries (16-byte vector load for two columns)
template <int NC>
__device__ __forceinline__ Cv<NC> sm_load(const float2* p) {
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

// address of a global slot: a vector row (this CTA's columns of x) or a
// CTA-private state entry
__device__ __forceinline__ float2* gaddr(const SwArgs& a, int32_t s, float2* xb, float2* stp, int nc) {
  return s < a.n ? xb + (int64_t)s * a.R : stp + (int64_t)(s - a.n) * nc;
}

// NC columns of global slot s into dst (shared, 8 * NC bytes) asynchronously; the
// columns beyond this CTA's ncol read as zero.  x rows are 16-byte aligned when the
// row stride and the CTA's first column are even (vec16).
template <int NC>
__device__ __forceinline__ void slot_async(const SwArgs& a, int32_t s, float2* dst, float2* xb, float2* stp, int ncol,
                                           bool vec16) {
  if (s < a.n) {
    const float2* src = xb + (int64_t)s * a.R;
    if (NC == 2 && vec16) {
      cp_async(dst, src, 16, 8 * ncol);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) cp_async(dst + c, c < ncol ? src + c : src, 8, c < ncol ? 8 : 0);
    }
  } else {
    const float2* src = stp + (int64_t)(s - a.n) * NC;
    cp_async(dst, src, 8 * NC, 8 * NC);
  }
}

// One batch in row form, one warp.  Inputs: `in` (the window for resident
// batches, the warp's gathered slice for global ones); outputs: window slots
// (RES) or global slots.
template <int NC, bool RES>
__device__ void run_rows(const SwArgs& a, const SwDesc& D, const char* bb, const float2* in, float2* win,
                         float2* xb, float2* stp, int ncol, int lane) {
  const int32_t* out = reinterpret_cast<const int32_t*>(bb);
  const int32_t* e0 = reinterpret_cast<const int32_t*>(bb + D.off_e0);
  const float2* cf = reinterpret_cast<const float2*>(bb + D.off_coef);
  const int16_t* ix = reinterpret_cast<const int16_t*>(bb + D.off_in);
  const int glog = D.glog, G = 1 << glog, ng = 32 >> glog;
  const int q = lane >> glog, l = lane & (G - 1);
  for (int base = 0; base < D.nrows; base += ng) {
    const int r = base + q;
    float2 acc[NC], acc2[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = acc2[c] = make_float2(0.f, 0.f);
    if (r < D.nrows) {
      const int ea = e0[r], eb = e0[r + 1];
      int e = ea + l;
      // two independent accumulator chains
      for (; e + G < eb; e += 2 * G) {
        const float2 m0 = cf[e], m1 = cf[e + G];
        const Cv<NC> v0 = sm_load<NC>(in + (int)ix[e] * NC);
        const Cv<NC> v1 = sm_load<NC>(in + (int)ix[e + G] * NC);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          cmac(acc[c], m0, v0.v[c]);
          cmac(acc2[c], m1, v1.v[c]);
        }
      }
      if (e < eb) {
        const float2 m0 = cf[e];
        const Cv<NC> v0 = sm_load<NC>(in + (int)ix[e] * NC);
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
    if (l == 0 && r < D.nrows) {
      const int32_t o = out[r];
      const bool add = (o & kSwAcc) != 0;
      const int32_t s = o & ~kSwAcc;
      if (RES) {
        float2* d = win + (int64_t)s * NC;
#pragma unroll
        for (int c = 0; c < NC; ++c) d[c] = add ? make_float2(d[c].x + acc[c].x, d[c].y + acc[c].y) : acc[c];
      } else {
        float2* d = gaddr(a, s, xb, stp, NC);
        const int nc = s < a.n ? ncol : NC;
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < nc) {
            if (add) {
              const float2 cur = __ldcg(d + c);
              d[c] = make_float2(cur.x + acc[c].x, cur.y + acc[c].y);
            } else {
              d[c] = acc[c];
            }
          }
      }
    }
  }
}

// Sweep-leaf phase: window rows a0 .. a0 + s - 1 replaced by T times them (T the
// packed triangle), all chain threads (t < nct).  T is stored as a lower
// triangle, column by column; an upper triangle U is stored reversed (entry
// (r, c) of the stored triangle is U(s-1-r, s-1-c)), so rev maps the stored
// rows and columns to window rows s-1-i.  Thread (pair j, column group g) owns
// stored rows j and s-1-j (s + 1 entries together) and their columns
// c = g (mod ncg); the lanes of a warp share g and read consecutive entries of
// one column.  The triangle is not read after the barrier inside.
template <int NC>
__device__ void run_tri(const SwDesc& D, bool rev, const float2* T, float2* win, float2* part, int t, int nct) {
  const int s = D.nrows;
  float2* b = win + (int64_t)D.a0 * NC;
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
      constexpr int U = 4;   // independent accumulator chains
      float2 acc[4][NC];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[u][c] = make_float2(0.f, 0.f);
      // entry (r, c) at c s - c (c - 1) / 2 + r - c; from c to c + ncg the offset grows by
      // d = ncg (s - c) - ncg (ncg + 1) / 2, and d shrinks by ncg^2 per step
      int c = g;
      int off = c * s - ((c * (c - 1)) >> 1) + r - c;
      int d = ncg * (s - c) - ((ncg * (ncg + 1)) >> 1);
      const int dd = ncg * ncg;
      for (; c + (U - 1) * ncg <= r; c += U * ncg) {
        float2 m[U];
        Cv<NC> v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          m[u] = T[off];
          const int cc = c + u * ncg;
          v[u] = sm_load<NC>(b + (int64_t)(rev ? s - 1 - cc : cc) * NC);
          off += d;
          d -= dd;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int k = 0; k < NC; ++k) cmac(acc[u][k], m[u], v[u].v[k]);
      }
      for (; c <= r; c += ncg) {
        const float2 m = T[off];
        const Cv<NC> v = sm_load<NC>(b + (int64_t)(rev ? s - 1 - c : c) * NC);
#pragma unroll
        for (int k = 0; k < NC; ++k) cmac(acc[0][k], m, v.v[k]);
        off += d;
        d -= dd;
      }
      const int ro = rev ? s - 1 - r : r;
#pragma unroll
      for (int k = 0; k < NC; ++k)
        part[((int64_t)g * s + ro) * NC + k] =
            make_float2(acc[0][k].x + acc[1][k].x + acc[2][k].x + acc[3][k].x,
                        acc[0][k].y + acc[1][k].y + acc[2][k].y + acc[3][k].y);
    }
  }
  ch_sync();
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
// The bound of 512 threads (above the 416 launched) caps the registers at 128 a
// thread, so that the scheduler that holds four of the 13 warps stays within its
// 16K registers.
__global__ void __launch_bounds__(512, 1) k_sweep_cols(SwArgs a) {
  extern __shared__ __align__(128) char smem[];
  char* ring = smem;
  float2* win = reinterpret_cast<float2*>(smem + kSwRingBytes);
  float2* part = reinterpret_cast<float2*>(smem + kSwRingBytes + kSwWinBytes);
  __shared__ int s_off[kSwSlots];                 // ring offset of each group in flight
  __shared__ int s_cnt[kSwSlots];                 // compute warps done with the slot's group
  __shared__ __align__(8) uint64_t s_mbar[kSwSlots];
  __shared__ __align__(16) SwGroup s_grec[32];    // the producer's window of group records
  __shared__ int s_abort, s_issued;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t lb = a.col0 + (int64_t)blockIdx.x * NC;
  const int ncol = (int)((a.R - lb) < NC ? (a.R - lb) : NC);
  float2* xb = a.x + lb;
  float2* stp = a.st + (int64_t)blockIdx.x * a.state_len * NC;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kSwSlots; ++k) {
      mb_init(&s_mbar[k], 1);
      s_cnt[k] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();
  if (warp == kSwWarps) {
    // ---- producer: every group of the schedule, in order, into the ring; groups
    // [oldest, g) are in flight; a group's ring area is free once every compute
    // warp is done with it, and space is recycled from the oldest group.  Lane 0
    // keeps the ring state and issues the copies; the warp loads the group
    // records 32 at a time.
    int head = 0;
    int64_t oldest = 0, g = 0;
    for (; g < a.ngroup; ++g) {
      if ((g & 31) == 0) {
        __syncwarp();
        if (g + lane < a.ngroup) s_grec[lane] = a.groups[g + lane];
        __syncwarp();
      }
      int off = -1;
      if (lane == 0) {
        const SwGroup& G = s_grec[g & 31];
        const int bytes = G.bytes;
        long long spins = 0;
        unsigned nap = 32;   // back-off while the ring is full (the compute warps keep the issue slots)
        for (;;) {
          while (oldest < g && *(volatile int*)&s_cnt[oldest % kSwSlots] == kSwWarps) ++oldest;
          __threadfence_block();
          if (*(volatile int*)&s_abort) break;
          if (g - oldest < kSwSlots) {
            if (oldest == g) {
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
          __nanosleep(nap);
          if (nap < 256) nap <<= 1;
        }
        if (off >= 0) {
          const int slot = (int)(g % kSwSlots);
          uint64_t* mb = &s_mbar[slot];
          s_off[slot] = off;
          s_cnt[slot] = 0;   // published with the arrive (release) below
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mb_arrive_tx(mb, (unsigned)bytes);
          bulk_copy(ring + off, a.image + G.img, (unsigned)bytes, mb);
          head = off + bytes;
        }
      }
      off = __shfl_sync(0xffffffffu, off, 0);
      if (off < 0) break;
    }
    if (lane == 0) s_issued = (int)g;
    __syncwarp();
  } else {
    const int t = threadIdx.x;
    const bool chain = warp < kSwChain;
    float2* slice = win + (int64_t)warp * 2 * kSwGather * NC;   // gather area of global batches (two halves)
    const bool vec16 = NC == 2 && (a.R % 2) == 0 && (lb % 2) == 0;
    bool bad = false;   // warp-uniform; after a failed wait the warp only follows the barriers
    // wait for group g (bounded); returns its image (ring, or global memory after a failure)
    auto group = [&](int64_t g) -> const char* {
      const int slot = (int)(g % kSwSlots);
      if (!bad) {
        long long spins = 0;
        bool ok = true;
        while (!mb_test_wait(&s_mbar[slot], (unsigned)(g / kSwSlots) & 1u)) {
          if (++spins > a.spin_limit || *(volatile int*)&s_abort) { ok = false; break; }
          if (spins > 4) __nanosleep(32);   // leave the issue slots to the producer warp
        }
        if (__any_sync(0xffffffffu, !ok)) {
          bad = true;
          if (lane == 0) atomicExch(&s_abort, 1);
        }
      }
      return bad ? reinterpret_cast<const char*>(a.image + a.groups[g].img) : ring + s_off[slot];
    };
    int64_t g = 0;
    while (g < a.ngroup) {
      const char* gimg = group(g);
      SwGroupHdr H = *reinterpret_cast<const SwGroupHdr*>(gimg);
      if (H.flags & SWG_RES) {
        // ---- a resident run: groups g .. g + H.aux - 1, executed by the chain warps
        const int64_t g0 = g, gend = g + H.aux;
        if (!chain) {
          // the other warps only read the run's length; they release their hold on the
          // first group's ring area, then wait for the run's end
          if (!bad) {
            __syncwarp();
            if (lane == 0) {
              __threadfence_block();
              atomicAdd(&s_cnt[(int)(g % kSwSlots)], 1);
            }
          }
          g = gend;
          if (cw_red_or(bad)) { bad = true; break; }   // the run is done, its rows written back
          continue;
        }
        const int ct = t, nct = kSwChain * 32;
        bool stop = false;
        for (; g < gend && !stop; ++g) {
          if (g > g0) {
            gimg = group(g);
            H = *reinterpret_cast<const SwGroupHdr*>(gimg);
          }
          const int slot = (int)(g % kSwSlots);
          const SwPhase* tab = reinterpret_cast<const SwPhase*>(gimg + 32);
          const SwDesc* desc = reinterpret_cast<const SwDesc*>(gimg + H.off_desc);
          if (H.flags & SWG_BEGIN) {
            if (!bad) {
              // the run's rows, all in flight at once
              for (int r = ct; r < H.beg_hi - H.beg_lo; r += nct) slot_async<NC>(a, H.beg_lo + r, win + r * NC, xb, stp, ncol, vec16);
              cp_commit();
              cp_wait<0>();
            }
            ch_sync();
          }
          int di = 0;
          bool last_end = false;
          for (int k = 0; k < H.nph; ++k) {
            const SwPhase PH = tab[k];
            last_end = (PH.flags & SWP_END) != 0;
            if (PH.flags & SWP_TRI) {
              if (!bad) {
                const SwDesc D = desc[di];
                run_tri<NC>(D, (PH.flags & SWP_UPPER) != 0, reinterpret_cast<const float2*>(gimg + D.off), win, part,
                            ct, nct);
              } else {
                ch_sync();   // the barrier inside run_tri
              }
            } else if (!bad) {
              for (int b = warp; b < PH.nb; b += kSwChain) {
                const SwDesc D = desc[di + b];
                run_rows<NC, true>(a, D, gimg + D.off, win, win, xb, stp, ncol, lane);
              }
            }
            di += PH.nb;
            if (PH.flags & SWP_END) {
              if (ch_red_or(bad)) { bad = true; stop = true; break; }
            }
          }
          if (stop) break;
          // a group that ends inside a phase (a large phase spread over several groups):
          // every chain warp must be done with it before it is released
          if (!last_end) ch_sync();
          // every chain warp has passed the group's last barrier: the group is consumed
          // (the run's first group: together with the other warps' holds)
          if (!bad && ct == 0) {
            __threadfence_block();
            if (g == g0) atomicAdd(&s_cnt[slot], kSwChain);
            else *(volatile int*)&s_cnt[slot] = kSwWarps;
          }
          if (H.flags & SWG_ENDRUN) {
            const int nrow = H.end_hi - H.end_lo;
            for (int e = ct; e < nrow * NC; e += nct) {
              const int r = e / NC, c = e % NC;
              if (c < ncol) xb[(int64_t)(H.end_lo + r) * a.R + c] = win[e];
            }
          }
        }
        g = gend;
        if (cw_red_or(bad)) { bad = true; break; }   // the run is done, its rows written back
        continue;
      }
      // ---- a part of a global phase: batches round-robin over all compute warps
      {
        const int slot = (int)(g % kSwSlots);
        const SwPhase PH = *reinterpret_cast<const SwPhase*>(gimg + 32);
        const SwDesc* desc = reinterpret_cast<const SwDesc*>(gimg + H.off_desc);
        if (!bad) {
          // this warp's batches b0, b0 + 12, ...: the gather of the next one (cp.async into
          // the other half of the warp's slice) is in flight while this one is computed
          const int b0 = (warp - H.aux + kSwWarps) % kSwWarps;
          auto gather = [&](int b, float2* dst) {
            const SwDesc& D = desc[b];
            const int32_t* gl = reinterpret_cast<const int32_t*>(gimg + D.off + D.off_gl);
            for (int k = lane; k < D.ngl; k += 32) slot_async<NC>(a, gl[k], dst + k * NC, xb, stp, ncol, vec16);
            cp_commit();
          };
          int buf = 0;
          if (b0 < PH.nb) gather(b0, slice);
          for (int b = b0; b < PH.nb; b += kSwWarps) {
            const int bn = b + kSwWarps;
            if (bn < PH.nb) {
              gather(bn, slice + (buf ^ 1) * kSwGather * NC);
              cp_wait<1>();
            } else {
              cp_wait<0>();
            }
            __syncwarp();
            const SwDesc D = desc[b];
            run_rows<NC, false>(a, D, gimg + D.off, slice + buf * kSwGather * NC, win, xb, stp, ncol, lane);
            __syncwarp();
            buf ^= 1;
          }
        }
        if (PH.flags & SWP_END) {
          // end of the phase: every compute warp's writes are visible to the next phase
          if (cw_red_or(bad)) { bad = true; break; }
          if (t == 0) {
            __threadfence_block();
            *(volatile int*)&s_cnt[slot] = kSwWarps;
          }
        } else if (!bad) {
          __syncwarp();
          if (lane == 0) {
            __threadfence_block();
            atomicAdd(&s_cnt[slot], 1);   // this warp no longer reads the group's ring area
          }
        }
        ++g;
      }
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
      if (q + kSwSlots < iss) continue;
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
  a.groups = sc.groups;
  a.ngroup = sc.ngroup;
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

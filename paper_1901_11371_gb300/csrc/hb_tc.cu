// Split-BF16 tensor-core contractions of the many-column apply (form
// HB_SPLIT_BF16, sm_103a tcgen05): the entry ops of a column leaf (the V0
// blocks of every depth, stacked) and the exit ops of a row leaf (the U0
// blocks of every depth, then the dense diagonal block) applied to 128-column
// tiles of the right-hand sides.  Each is a dense complex contraction
//   OUT (outputs x columns) = W (outputs x inputs) * V (inputs x columns),
// run as a real GEMM with the columns on M (128 per tile), the real-expanded
// outputs on N and the real-expanded inputs on K:
//   D[m][n'] = sum_k' A[m][k'] B[n'][k'],  A = [Re V^T | Im V^T],
//   B rows n < nn: [Re W(n,:) | -Im W(n,:)],  rows nn + n: [Im W(n,:) | Re W(n,:)]
// so D[m][n] = Re OUT(n, m) and D[m][nn + n] = Im OUT(n, m).  Both operands
// are split into three bf16 parts (x = x1 + x2 + x3, 24 significant bits in
// all) and the six products x_a y_b with a + b <= 4 (1-based) accumulate in
// FP32 in tensor memory -- the leading product x1 y1 in one accumulator, the
// five smaller ones in another, added in the epilogue, so that their
// accumulation rounds at their own (2^8 smaller) magnitude -- and the result
// carries FP32 accuracy.  The host built
// every W chunk's B operand (its three parts) in the canonical K-major,
// no-swizzle layout; a CTA
// copies it with one bulk copy, builds the A operand of each column tile from
// the vectors (x / butterfly state) while converting and splitting, one
// thread issues the MMAs (tcgen05.mma kind::f16, M = 128, N = 2 nn, K = 16
// per instruction), and the four warps read the accumulator back
// (tcgen05.ld) and write the outputs (state entries / rows of y).
// Every wait is bounded; a wait that gives up raises the factor's error flag.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hb_device.h"
#include "hb_sweep_launch.h"

namespace hb {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcMaxK = 128;                       // real-expanded inputs per chunk (2 x 64)
constexpr int kTcMaxN = 128;                       // real-expanded outputs per chunk (2 x 64)
constexpr int kTcABytes = 128 * kTcMaxK * 2;       // one bf16 A block (128 rows)
constexpr int kTcBBytes = kTcMaxN * kTcMaxK * 2;   // one bf16 B block
constexpr int kTcSmem = kTcParts * kTcABytes + kTcParts * kTcBBytes + 1024;

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// no-swizzle K-major shared-memory matrix descriptor: start address, byte
// offset between K-adjacent core matrices (LBO), between row groups (SBO)
__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
  return d;
}
// instruction descriptor: kind::f16 with bf16 A and B, FP32 accumulate, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mb_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
  return ok != 0;
}
// bounded wait on phase `parity` of mbarrier b (all calling threads)
__device__ __forceinline__ bool mb_wait(uint64_t* b, unsigned parity, long long limit) {
  long long spins = 0;
  while (!mb_try(b, parity))
    if (++spins > limit) return false;
  return true;
}
// three-part bf16 split of the pair (a, b) (elements k, k + 1): words[q] holds
// part q of both (element k in the low half), and (a, b) is left with the remainder
__device__ __forceinline__ void split3(float& a, float& b, uint32_t (&words)[kTcParts]) {
#pragma unroll
  for (int q = 0; q < kTcParts; ++q) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    words[q] = *reinterpret_cast<const uint32_t*>(&v);
    const float2 f = __bfloat1622float2(v);
    a -= f.x;
    b -= f.y;
  }
}

// parts of the vector / factor operand in product pq (the same pairs as
// kTcProdA / kTcProdB, which the host emulation uses)
__device__ __forceinline__ constexpr int prod_a(int pq) { return pq == 2 || pq == 4 ? 1 : pq == 5 ? 2 : 0; }
__device__ __forceinline__ constexpr int prod_b(int pq) { return pq == 1 || pq == 4 ? 1 : pq == 3 ? 2 : 0; }
static_assert(kTcProducts == 6 && kTcProdA[2] == 1 && kTcProdA[4] == 1 && kTcProdA[5] == 2 && kTcProdB[1] == 1 &&
                  kTcProdB[4] == 1 && kTcProdB[3] == 2, "product table");

// eight consecutive 32-bit accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(addr));
}

struct TcArgs {
  const TcJob* jobs;
  const TcChunk* chunks;
  const uint16_t* bpool;
  const uint32_t* tab;
  const float2* x;     // input vectors [row][R]
  float2* st;          // butterfly state [entry][R] (read by exit jobs, written by entry jobs)
  float2* y;           // output vectors [row][R]
  int64_t R;
  int* err;            // the factor's sticky error flag
  long long spin_limit;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_jobs(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sA = sm;                                   // the vector operand's three parts
  unsigned char* sB = sm + kTcParts * kTcABytes;            // the factor operand's three parts (as copied)
  uint64_t* mbar = (uint64_t*)(sm + kTcParts * kTcABytes + kTcParts * kTcBBytes);   // [0] B copy, [1] MMA done
  uint32_t* s_tmem = (uint32_t*)(mbar + 2);
  int* s_bad = (int*)(s_tmem + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcJob job = a.jobs[blockIdx.x];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(s_tmem)), "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mb_init(&mbar[0]);
    mb_init(&mbar[1]);
    *s_bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tbase = *s_tmem;
  unsigned ph_b = 0, ph_m = 0;   // phases of the two mbarriers
  const int64_t R = a.R;
  const int ntile = (int)((R + 127) / 128);
  bool ok = true;
  // tensor memory (512 columns): per tile and output chunk a leading-product
  // region and a correction region of 128 columns each
  const int tiles_per_pass = job.nreg > 1 ? 1 : 2;
  const uint32_t tile_cols = (uint32_t)(256 * job.nreg);
  for (int g0 = 0; g0 < ntile && ok; g0 += tiles_per_pass) {
    const int ng = (ntile - g0) < tiles_per_pass ? (ntile - g0) : tiles_per_pass;
    for (int ci = 0; ci < job.nchunk && ok; ++ci) {
      const TcChunk ch = a.chunks[job.chunk0 + ci];
      const int Kr = 2 * ch.nk, Nr = 2 * ch.nn;
      const unsigned bbytes = (unsigned)(kTcParts * Nr * Kr * 2);
      // B operand (its parts) of the chunk: one bulk copy
      if (tid == 0) {
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
                     ::"r"(su32(&mbar[0])), "r"(bbytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                     ::"r"(su32(sB)), "l"(a.bpool + ch.boff), "r"(bbytes), "r"(su32(&mbar[0])) : "memory");
      }
      bool b_ready = false;
      for (int t = 0; t < ng; ++t) {
        // ---- A operand of column tile g0 + t: thread = column m, 8 inputs per 16-byte store
        const int64_t col = (int64_t)(g0 + t) * 128 + tid;
        const bool live = col < R;
        const int rb = (tid >> 3) * (Kr >> 3) * 128 + (tid & 7) * 16;   // byte offset of row m, K group 0
        for (int k0 = 0; k0 < ch.nk; k0 += 8) {
          float re[8], im[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const uint32_t e = a.tab[ch.in0 + k0 + u];
            float2 v = make_float2(0.f, 0.f);
            if (live && e != kTcNone) v = (e & kTcVec) ? a.x[(int64_t)(e & ~kTcVec) * R + col] : a.st[(int64_t)e * R + col];
            re[u] = v.x;
            im[u] = v.y;
          }
          uint32_t wr[4][kTcParts], wi[4][kTcParts];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            split3(re[2 * u], re[2 * u + 1], wr[u]);
            split3(im[2 * u], im[2 * u + 1], wi[u]);
          }
          const int offr = rb + (k0 >> 3) * 128;                 // real part: K columns k0 .. k0+7
          const int offi = rb + ((ch.nk + k0) >> 3) * 128;       // imaginary part: K columns nk + k0 ..
#pragma unroll
          for (int q = 0; q < kTcParts; ++q) {
            unsigned char* aq = sA + q * kTcABytes;
            *reinterpret_cast<uint4*>(aq + offr) = make_uint4(wr[0][q], wr[1][q], wr[2][q], wr[3][q]);
            *reinterpret_cast<uint4*>(aq + offi) = make_uint4(wi[0][q], wi[1][q], wi[2][q], wi[3][q]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (!b_ready) {
          if (!mb_wait(&mbar[0], ph_b, a.spin_limit)) atomicExch(s_bad, 1);
          b_ready = true;
        }
        __syncthreads();
        if (*(volatile int*)s_bad) { ok = false; break; }
        // ---- MMAs: K/16 steps x the six part products into the tile's accumulator region
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t idesc = idesc_bf16(128, Nr);
          const unsigned sbo = (unsigned)(Kr >> 3) * 128;
          const unsigned a0 = su32(sA), b0 = su32(sB);
          const unsigned bpart = (unsigned)(Nr * Kr * 2);
          const uint32_t dmain = tbase + (uint32_t)t * tile_cols + (uint32_t)ch.tcol;
          const uint32_t dcorr = dmain + 128u * (uint32_t)job.nreg;
          for (int s = 0; s < Kr / 16; ++s) {
            const unsigned ko = (unsigned)s * 256;   // two K core matrices per step
#pragma unroll
            for (int pq = 0; pq < kTcProducts; ++pq) {
              const uint32_t acc = ((pq > 1) || s > 0 || (ch.flags & TC_ACC)) ? 1u : 0u;
              mma_bf16(pq == 0 ? dmain : dcorr, sdesc(a0 + (unsigned)prod_a(pq) * kTcABytes + ko, 128, sbo),
                       sdesc(b0 + (unsigned)prod_b(pq) * bpart + ko, 128, sbo), idesc, acc);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                       ::"r"(su32(&mbar[1])) : "memory");
        }
        if (!mb_wait(&mbar[1], ph_m, a.spin_limit)) atomicExch(s_bad, 1);
        ph_m ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // ---- epilogue of the tile's region after the chunk that completes it
        if (ch.flags & TC_LAST) {
          const uint32_t rowaddr = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)t * tile_cols + (uint32_t)ch.tcol;
          const uint32_t corr = 128u * (uint32_t)job.nreg;
          for (int n0 = 0; n0 < ch.nn; n0 += 8) {
            uint32_t vr[8], vi[8], cr[8], ci[8];
            tmem_ld8(rowaddr + (uint32_t)n0, vr);
            tmem_ld8(rowaddr + (uint32_t)(ch.nn + n0), vi);
            tmem_ld8(rowaddr + corr + (uint32_t)n0, cr);
            tmem_ld8(rowaddr + corr + (uint32_t)(ch.nn + n0), ci);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            const int64_t c = (int64_t)(g0 + t) * 128 + 32 * warp + lane;
            if (c < R) {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const uint32_t e = a.tab[ch.out0 + n0 + u];
                if (e == kTcNone) continue;
                float2* d = (e & kTcVec) ? a.y + (int64_t)(e & ~kTcVec) * R + c : a.st + (int64_t)e * R + c;
                *d = make_float2(__uint_as_float(vr[u]) + __uint_as_float(cr[u]),
                                 __uint_as_float(vi[u]) + __uint_as_float(ci[u]));
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();   // the A buffer and the accumulator region are free again
      }
      ph_b ^= 1u;
    }
  }
  if (!ok && tid == 0) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(512u) : "memory");
  if (tid == 0) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(su32(&mbar[0])) : "memory");
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(su32(&mbar[1])) : "memory");
  }
}

}  // namespace

int launch_tc_jobs(const DevFactor& df, bool exit_jobs, const void* x, void* st, void* y, int64_t R,
                   cudaStream_t s) {
  const int njobs = (int)df.m;
  if (!df.tc_ok || njobs < 1) return HB_EUNSUPPORTED;
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_tc_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    attr_done = true;
  }
  TcArgs a;
  a.jobs = exit_jobs ? df.tc_exit : df.tc_enter;
  a.chunks = df.tc_chunks;
  a.bpool = df.tc_bpool;
  a.tab = df.tc_tab;
  a.x = (const float2*)x;
  a.st = (float2*)st;
  a.y = (float2*)y;
  a.R = R;
  a.err = &((GridBar*)df.bar)->err;
  a.spin_limit = df.spin_limit;
  k_tc_jobs<<<njobs, kTcThreads, kTcSmem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
}

}  // namespace hb

// Host construction of the split-BF16 tensor-core operands (form
// HB_SPLIT_BF16): the entry and exit contractions of every leaf of Alg. 2,
// expanded from the packed ID blocks into dense real-form chunks (see
// TcOperands in hb_internal.h).
#include <algorithm>

#include "hb_internal.h"

namespace hb {

namespace {

struct Dense {
  int64_t rows = 0, cols = 0;
  std::vector<cplx> w;   // row-major
  std::vector<uint32_t> in, out;
  cplx& at(int64_t r, int64_t c) { return w[(size_t)(r * cols + c)]; }
};

int64_t up8(int64_t v) { return (v + 7) / 8 * 8; }

// cut W into chunks of <= 64 outputs x <= 64 inputs; for every output chunk the input
// chunks accumulate in order into one tensor-memory region
void emit(const Dense& d, TcOperands& tc, std::vector<TcJob>& jobs) {
  const int64_t nN = (d.rows + 63) / 64, nK = (d.cols + 63) / 64;
  TcJob job{(int32_t)tc.chunks.size(), 0, nN > 1 ? 2 : 1, 0};
  for (int64_t ni = 0; ni < nN; ++ni) {
    const int64_t r0 = ni * 64, rn = std::min<int64_t>(64, d.rows - r0), nn = up8(rn);
    for (int64_t ki = 0; ki < nK; ++ki) {
      const int64_t c0 = ki * 64, cn = std::min<int64_t>(64, d.cols - c0), nk = up8(cn);
      TcChunk ch{};
      ch.nn = (int32_t)nn;
      ch.nk = (int32_t)nk;
      ch.tcol = (int32_t)(128 * (ni % 2));
      ch.flags = (ki > 0 ? TC_ACC : 0) | (ki == nK - 1 ? TC_LAST : 0);
      ch.in0 = (int32_t)tc.tab.size();
      for (int64_t k = 0; k < nk; ++k) tc.tab.push_back(k < cn ? d.in[(size_t)(c0 + k)] : kTcNone);
      ch.out0 = (int32_t)tc.tab.size();
      for (int64_t n = 0; n < nn; ++n) tc.tab.push_back(n < rn ? d.out[(size_t)(r0 + n)] : kTcNone);
      while (tc.bpool.size() % 64) tc.bpool.push_back(0);   // 128-byte aligned operand blocks
      ch.boff = (int64_t)tc.bpool.size();
      const int64_t R = 2 * nn, K = 2 * nk, blk = R * K;
      tc.bpool.resize(tc.bpool.size() + (size_t)(kTcParts * blk), 0);
      uint16_t* part[kTcParts];
      for (int q = 0; q < kTcParts; ++q) part[q] = &tc.bpool[(size_t)(ch.boff + q * blk)];
      for (int64_t n = 0; n < rn; ++n)
        for (int64_t k = 0; k < cn; ++k) {
          const cplx v = d.w[(size_t)((r0 + n) * d.cols + c0 + k)];
          const double vals[4][3] = {{(double)n, (double)k, v.real()},
                                     {(double)n, (double)(nk + k), -v.imag()},
                                     {(double)(nn + n), (double)k, v.imag()},
                                     {(double)(nn + n), (double)(nk + k), v.real()}};
          for (const auto& e : vals) {
            uint16_t b[kTcParts];
            bf16_split((float)e[2], b);
            const int64_t o = tc_off((int64_t)e[0], (int64_t)e[1], K);
            for (int q = 0; q < kTcParts; ++q) part[q][o] = b[q];
          }
        }
      tc.chunks.push_back(ch);
      job.nchunk++;
    }
  }
  jobs.push_back(job);
}

}  // namespace

void build_tc_operands(const PackedHost& ph, const HostFactor& hf, TcOperands& tc) {
  tc = TcOperands();
  const int D = ph.depth;
  const int64_t m = ph.m, n0 = ph.n0;
  for (int64_t l = 0; l < m; ++l) {
    // entry: z0 pairs of every depth = V0_v x_l (rows (v, i), columns = the leaf's n0 entries)
    Dense e;
    for (int v = 0; v < D; ++v) e.rows += ph.vout[(size_t)(l * D + v)].blk.k;
    e.cols = n0;
    e.w.assign((size_t)(e.rows * e.cols), cplx(0.0));
    for (int64_t c = 0; c < n0; ++c) e.in.push_back(kTcVec | (uint32_t)(l * n0 + c));
    int64_t r = 0;
    for (int v = 0; v < D; ++v) {
      const DOuter& o = ph.vout[(size_t)(l * D + v)];
      const int k = o.blk.k, c = o.blk.c, nr = c - k;
      const cplx* M = &ph.fpool[(size_t)o.blk.moff];
      const int16_t* I = &ph.ipool[(size_t)o.blk.ioff];
      for (int i = 0; i < k; ++i) {
        e.at(r + i, I[i]) += 1.0;
        for (int j = 0; j < nr; ++j) e.at(r + i, I[k + j]) += M[(size_t)j * k + i];
        e.out.push_back((uint32_t)(o.seg_off + i));
      }
      r += k;
    }
    emit(e, tc, tc.enter);
    // exit: y_l = sum_v U0_v y0_v + A_l x_l (columns: the y0 pairs of every depth, then x_l)
    Dense x;
    x.rows = n0;
    for (int v = 0; v < D; ++v) x.cols += ph.uout[(size_t)(l * D + v)].blk.k;
    x.cols += n0;
    x.w.assign((size_t)(x.rows * x.cols), cplx(0.0));
    int64_t col = 0;
    for (int v = 0; v < D; ++v) {
      const DOuter& o = ph.uout[(size_t)(l * D + v)];
      const int k = o.blk.k, c = o.blk.c, nr = c - k;
      const cplx* M = &ph.fpool[(size_t)o.blk.moff];
      const int16_t* I = &ph.ipool[(size_t)o.blk.ioff];
      for (int i = 0; i < k; ++i) {
        x.at(I[i], col + i) += 1.0;
        for (int j = 0; j < nr; ++j) x.at(I[k + j], col + i) += M[(size_t)i * nr + j];
        x.in.push_back((uint32_t)(o.seg_off + i));
      }
      col += k;
    }
    for (int64_t cc = 0; cc < n0; ++cc) {
      for (int64_t rr = 0; rr < n0; ++rr) x.at(rr, col + cc) = hf.leaf[(size_t)((l * n0 + rr) * n0 + cc)];
      x.in.push_back(kTcVec | (uint32_t)(l * n0 + cc));
    }
    for (int64_t rr = 0; rr < n0; ++rr) x.out.push_back(kTcVec | (uint32_t)(l * n0 + rr));
    emit(x, tc, tc.exit);
  }
}

namespace {
// one chunk: outputs from inputs with the device's split products
void tc_chunk_host(const TcOperands& tc, const TcChunk& ch, const std::vector<cplx>& in, std::vector<cplx>& out) {
  const int64_t K = 2 * ch.nk, N = 2 * ch.nn, blk = N * K;
  const uint16_t* bp = &tc.bpool[(size_t)ch.boff];
  std::vector<double> av((size_t)(kTcParts * K));   // av[q * K + k]: part q of input k
  for (int64_t k = 0; k < ch.nk; ++k) {
    const float v[2] = {(float)in[(size_t)k].real(), (float)in[(size_t)k].imag()};
    for (int half = 0; half < 2; ++half) {
      uint16_t b[kTcParts];
      bf16_split(v[half], b);
      for (int q = 0; q < kTcParts; ++q) av[(size_t)(q * K + half * ch.nk + k)] = bf16_value(b[q]);
    }
  }
  out.assign((size_t)ch.nn, cplx(0.0));
  for (int64_t n = 0; n < ch.nn; ++n) {
    double d[2] = {0.0, 0.0};
    for (int half = 0; half < 2; ++half) {
      const int64_t row = half * ch.nn + n;
      for (int64_t k = 0; k < K; ++k) {
        const int64_t o = tc_off(row, k, K);
        for (int pq = 0; pq < kTcProducts; ++pq) {
          const int qa = kTcProdA[pq], qb = kTcProdB[pq];
          d[half] += av[(size_t)(qa * K + k)] * (double)bf16_value(bp[qb * blk + o]);
        }
      }
    }
    out[(size_t)n] = cplx(d[0], d[1]);
  }
}

void tc_jobs_host(const TcOperands& tc, const std::vector<TcJob>& jobs, const cplx* x, std::vector<cplx>& st, cplx* y) {
  for (const TcJob& j : jobs) {
    std::vector<cplx> acc;
    for (int32_t c = j.chunk0; c < j.chunk0 + j.nchunk; ++c) {
      const TcChunk& ch = tc.chunks[(size_t)c];
      std::vector<cplx> in((size_t)ch.nk), part;
      for (int64_t k = 0; k < ch.nk; ++k) {
        const uint32_t e = tc.tab[(size_t)(ch.in0 + k)];
        in[(size_t)k] = e == kTcNone ? cplx(0.0) : (e & kTcVec) ? x[e & ~kTcVec] : st[e];
      }
      tc_chunk_host(tc, ch, in, part);
      if (!(ch.flags & TC_ACC)) acc.assign((size_t)ch.nn, cplx(0.0));
      for (int64_t n = 0; n < ch.nn; ++n) acc[(size_t)n] += part[(size_t)n];
      if (ch.flags & TC_LAST)
        for (int64_t n = 0; n < ch.nn; ++n) {
          const uint32_t e = tc.tab[(size_t)(ch.out0 + n)];
          if (e == kTcNone) continue;
          if (e & kTcVec) y[e & ~kTcVec] = acc[(size_t)n];
          else st[e] = acc[(size_t)n];
        }
    }
  }
}
}  // namespace

void host_tc_apply(const PackedHost& ph, const HostFactor& hf, const TcOperands& tc, const cplx* x, cplx* y) {
  std::vector<cplx> st((size_t)ph.state_len, cplx(0.0));
  tc_jobs_host(tc, tc.enter, x, st, y);
  host_apply_items(ph, hf, false, st);
  tc_jobs_host(tc, tc.exit, x, st, y);
}

}  // namespace hb

// Column-partitioned sweep schedules (kernel k_sweep_cols): the flattened
// program of Alg. 3 / Alg. 4 as resident runs and global phases, every
// butterfly phase written out as a sparse product in row form, every
// sweep-leaf phase as its packed triangle; plus a host executor of the
// schedule for checks without a GPU.
#include <algorithm>
#include <cstring>

#include "hb_internal.h"

namespace hb {

namespace {

inline int64_t al16(int64_t b) { return (b + 15) & ~(int64_t)15; }

// One phase in row form: rows r = [start[r], start[r+1]) of (slot, coef).
struct PhaseRows {
  std::vector<int32_t> out, start;
  std::vector<int32_t> slot;
  std::vector<cplx> coef;
  void clear() {
    out.clear();
    start.clear();
    slot.clear();
    coef.clear();
  }
  void begin_row(int32_t o) {
    out.push_back(o);
    start.push_back((int32_t)slot.size());
  }
  void add(int32_t s, cplx v) {
    slot.push_back(s);
    coef.push_back(v);
  }
  int32_t nrows() const { return (int32_t)out.size(); }
  int32_t len(int32_t r) const {
    return (r + 1 < nrows() ? start[r + 1] : (int32_t)slot.size()) - start[r];
  }
};

// Slots: a vector row r -> r, a state entry e -> n + e (global phases); inside a
// resident run the window holds rows [row_lo, row_hi) then state [st_lo, st_hi).
struct SlotMap {
  int64_t n = 0;
  bool res = false;
  int32_t row_lo = 0, row_hi = 0, st_lo = 0, st_hi = 0;
  bool bad = false;
  int32_t vec(int32_t r) {
    if (!res) return r;
    if (r < row_lo || r >= row_hi) { bad = true; return 0; }
    return r - row_lo;
  }
  int32_t st(int32_t e) {
    if (!res) {
      if ((int64_t)e + n > INT32_MAX - 1) { bad = true; return 0; }
      return (int32_t)(n + e);
    }
    if (e < st_lo || e >= st_hi) { bad = true; return 0; }
    return (row_hi - row_lo) + (e - st_lo);
  }
};

// The rows of one flattened op (semantics of the op kinds as defined with
// FlatOp: the ID's identity entries, T or S entries, conjugated for the
// adjoint layouts, negated when the op subtracts from its outputs).
void expand_op(const PackedHost& ph, const FlatOp& f, SlotMap& sm, PhaseRows& P) {
  const cplx* M = ph.fpool.data() + f.moff;
  const int16_t* I = f.ioff >= 0 ? ph.ipool.data() + f.ioff : nullptr;
  const bool conj_layout = (f.flags & FF_CONJ) != 0;
  const bool two = (f.flags & FF_TWO) != 0;
  // candidate v of the concatenated operand segments [src0 (n_s0) | src1]
  auto cand = [&](int v) -> int32_t {
    if (v < f.n_s0) return (f.flags & FF_SRC_VEC) ? sm.vec(f.src0 + v) : sm.st(f.src0 + v);
    return sm.st(f.src1 + (v - f.n_s0));
  };
  auto out0 = [&](int i) -> int32_t { return (f.flags & FF_OUT_VEC) ? sm.vec(f.out0 + i) : sm.st(f.out0 + i); };
  if (f.kind == FK_GATHER) {
    // out_b[i] = cand[q_i] + sum_j T(i, j) cand[p_j]
    for (int b = 0; b < (two ? 2 : 1); ++b) {
      const cplx* Mb = M + (b ? f.m1 : 0);
      const int16_t* Ib = I + (b ? f.i1 : 0);
      const int k = b ? f.k1 : f.k0, c = b ? f.c1 : f.c0, nr = c - k;
      for (int i = 0; i < k; ++i) {
        P.begin_row(b ? sm.st(f.out1 + i) : out0(i));
        P.add(cand(Ib[i]), cplx(1.0, 0.0));
        for (int j = 0; j < nr; ++j) {
          const cplx m = conj_layout ? std::conj(Mb[(int64_t)i * nr + j]) : Mb[(int64_t)j * k + i];
          P.add(cand(Ib[k + j]), m);
        }
      }
    }
  } else if (f.kind == FK_SCATTER) {
    // candidate entry r: y[map(r)] (skeleton) or sum_i T(i, j) y[i]; both blocks add
    const bool sub = (f.flags & FF_SUB) != 0;
    const double sg = sub ? -1.0 : 1.0;
    for (int r = 0; r < f.c0; ++r) {
      int32_t o;
      if (!two || r < f.split) o = out0(r);
      else o = sm.st(f.out1 + (r - f.split));
      P.begin_row(sub ? (o | kSwAcc) : o);
      for (int b = 0; b < (two ? 2 : 1); ++b) {
        const cplx* Mb = M + (b ? f.m1 : 0);
        const int16_t* Ib = I + (b ? f.i1 : 0);
        const int k = b ? f.k1 : f.k0, c = b ? f.c1 : f.c0, nr = c - k;
        const int ybase = b ? f.n_s0 : 0;   // y_b = candidates [ybase, ybase + k)
        const int code = Ib[c + r];
        if (code >= 0) {
          P.add(cand(ybase + code), cplx(sg, 0.0));
        } else {
          const int j = -1 - code;
          for (int i = 0; i < k; ++i) {
            const cplx m = conj_layout ? std::conj(Mb[(int64_t)j * k + i]) : Mb[(int64_t)i * nr + j];
            P.add(cand(ybase + i), sg * m);
          }
        }
      }
    }
  } else if (f.kind == FK_MIDDLE) {
    // y = S z (S stored [c][r]); adjoint z = S^H y
    const int kr = f.k0, kc = f.c0;
    const bool adj = (f.flags & FF_ADJ) != 0;
    const int nin = adj ? kr : kc, nout = adj ? kc : kr;
    for (int oo = 0; oo < nout; ++oo) {
      P.begin_row(sm.st(f.out0 + oo));
      for (int i = 0; i < nin; ++i) {
        const cplx m = adj ? std::conj(M[(int64_t)oo * kr + i]) : M[(int64_t)i * kr + oo];
        P.add(sm.st(f.src0 + i), m);
      }
    }
  }
}

template <class R>
void put_coef(uint8_t* dst, cplx v) {
  const R p[2] = {(R)v.real(), (R)v.imag()};
  std::memcpy(dst, p, sizeof(p));
}

struct Builder {
  const PackedHost& ph;
  SwSched& S;
  int cb;
  Builder(const PackedHost& p, SwSched& s, int coef_bytes) : ph(p), S(s), cb(coef_bytes) {}

  int64_t alloc(int64_t bytes) {
    const int64_t at = (int64_t)S.image.size();
    S.image.resize((size_t)(at + al16(bytes)), 0);
    return at;
  }
  void coef_at(uint8_t* dst, cplx v) {
    if (cb == 8) put_coef<float>(dst, v);
    else put_coef<double>(dst, v);
  }

  // one batch: rows rows[r0 .. r1) of P, in that order
  void emit_batch(const PhaseRows& P, const std::vector<int32_t>& rows, size_t r0, size_t r1, int glog, bool res) {
    SwBatch B{};
    B.nrows = (int32_t)(r1 - r0);
    int64_t ne = 0;
    for (size_t q = r0; q < r1; ++q) ne += P.len(rows[q]);
    if (ne > INT32_MAX / 16) { S.ok = false; S.why = "batch too large"; return; }
    B.nent = (int32_t)ne;
    B.glog = (int16_t)glog;
    B.flags = (int16_t)(res ? SWF_RES : 0);
    B.off_e0 = (int32_t)al16(4 * (int64_t)B.nrows);
    B.off_coef = B.off_e0 + (int32_t)al16(4 * ((int64_t)B.nrows + 1));
    B.off_in = B.off_coef + (int32_t)al16((int64_t)cb * ne);
    const int64_t bytes = B.off_in + al16((res ? 2 : 4) * ne);
    B.bytes = (int32_t)bytes;
    B.img = alloc(bytes);
    uint8_t* base = S.image.data() + B.img;
    int32_t* out = (int32_t*)base;
    int32_t* e0 = (int32_t*)(base + B.off_e0);
    uint8_t* coef = base + B.off_coef;
    int32_t e = 0;
    for (size_t q = r0; q < r1; ++q) {
      const int32_t r = rows[q];
      out[q - r0] = P.out[r];
      e0[q - r0] = e;
      const int32_t s0 = P.start[r], n = P.len(r);
      for (int32_t t = 0; t < n; ++t, ++e) {
        coef_at(coef + (int64_t)e * cb, P.coef[s0 + t]);
        if (res) ((int16_t*)(base + B.off_in))[e] = (int16_t)P.slot[s0 + t];
        else ((int32_t*)(base + B.off_in))[e] = P.slot[s0 + t];
      }
    }
    e0[B.nrows] = e;
    S.max_bytes = std::max(S.max_bytes, B.bytes);
    S.batches.push_back(B);
  }

  // lanes per row: about eight entries per lane
  static int pick_glog(const PhaseRows& P) {
    const double avg = P.nrows() > 0 ? (double)P.slot.size() / P.nrows() : 1.0;
    int g = 0;
    while (g < 5 && (double)(8 << g) < avg) ++g;
    return g;
  }

  void emit_phase(const PhaseRows& P, bool res) {
    const int32_t nrows = P.nrows();
    const int glog = pick_glog(P);
    const int per_round = 32 >> glog;
    const int32_t b0 = (int32_t)S.batches.size();
    const int64_t rowb = (int64_t)cb + (res ? 2 : 4);
    int64_t tot = 16 * (int64_t)nrows;
    for (int32_t r = 0; r < nrows; ++r) tot += rowb * P.len(r);
    std::vector<int32_t> order(nrows);
    for (int32_t r = 0; r < nrows; ++r) order[r] = r;
    if (res) {
      // small dependent phase: at most one batch per compute warp (more if the
      // images would be too large), rows by decreasing length dealt round-robin
      int64_t nb = std::min<int64_t>(kSwWarps, (nrows + per_round - 1) / per_round);
      nb = std::max<int64_t>(nb, (tot + kSwBatchBytes - 1) / kSwBatchBytes);
      nb = std::max<int64_t>(1, std::min<int64_t>(nb, nrows));
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return P.len(a) > P.len(b); });
      std::vector<int32_t> dealt;
      dealt.reserve(nrows);
      std::vector<size_t> cut(nb + 1, 0);
      for (int64_t q = 0; q < nb; ++q) {
        cut[q] = dealt.size();
        for (int64_t i = q; i < nrows; i += nb) dealt.push_back(order[i]);
      }
      cut[nb] = dealt.size();
      for (int64_t q = 0; q < nb; ++q) emit_batch(P, dealt, cut[q], cut[q + 1], glog, true);
    } else {
      // wide phase: consecutive rows (inputs shared by an op's rows stay together),
      // batches of about kSwBatchBytes, the rows of a batch by decreasing length
      size_t r0 = 0;
      int64_t acc = 0;
      for (size_t r = 0; r <= (size_t)nrows; ++r) {
        const int64_t add = r < (size_t)nrows ? 16 + rowb * P.len((int32_t)r) : 0;
        if (r == (size_t)nrows || (acc + add > kSwBatchBytes && r > r0)) {
          if (r > r0) {
            std::stable_sort(order.begin() + r0, order.begin() + r,
                             [&](int32_t a, int32_t b) { return P.len(a) > P.len(b); });
            emit_batch(P, order, r0, r, glog, false);
          }
          r0 = r;
          acc = 0;
        }
        acc += add;
      }
    }
    S.steps.push_back(SwStep{SW_PHASE, b0, (int32_t)S.batches.size() - b0, res ? SWF_RES : 0});
  }

  void emit_tri(const FlatOp& f, int which, int32_t a0) {
    const int64_t s = f.c0;
    SwBatch B{};
    B.nrows = (int32_t)s;
    B.flags = (int16_t)(SWF_TRI | SWF_RES | ((f.flags & FF_UPPER) ? SWF_UPPER : 0));
    B.a0 = a0;
    const int64_t ne = packed_tri(s);
    B.nent = (int32_t)ne;
    B.bytes = (int32_t)al16(ne * cb);
    B.img = alloc(B.bytes);
    uint8_t* base = S.image.data() + B.img;
    const cplx* T = ph.sl[which].data() + f.moff;
    for (int64_t e = 0; e < ne; ++e) coef_at(base + e * cb, T[e]);
    S.max_bytes = std::max(S.max_bytes, B.bytes);
    S.steps.push_back(SwStep{SW_PHASE, (int32_t)S.batches.size(), 1, SWF_TRI | SWF_RES});
    S.batches.push_back(B);
  }
};

}  // namespace

void build_sweep_sched(const PackedHost& ph, int which, int coef_bytes, int win_slots, SwSched& S) {
  S = SwSched{};
  S.coef_bytes = coef_bytes;
  S.win_slots = std::max(1, std::min(win_slots, kSwWinSlots));
  const std::vector<DPhase>* progs[4] = {&ph.prog_lower, &ph.prog_upper, &ph.prog_lower_adj, &ph.prog_upper_adj};
  const std::vector<DPhase>& prog = *progs[which];
  if (ph.fpool.empty() || ph.sl[which].empty()) { S.ok = false; S.why = "factor data released"; return; }
  const FlatProgram fp = flatten_program(ph, prog, which);
  if (!fp.ok) { S.ok = false; S.why = "flattened program"; return; }
  const std::vector<DSeg> segs = segment_program(prog, fp, 1 << 30, S.win_slots);
  Builder bd(ph, S, coef_bytes);
  PhaseRows P;
  for (const DSeg& sg : segs) {
    const int64_t rows = sg.row_hi - sg.row_lo, nst = sg.st_hi - sg.st_lo;
    const bool res = !sg.grid && !sg.st_cross && rows + nst <= S.win_slots && rows > 0;
    SlotMap sm;
    sm.n = ph.n;
    sm.res = res;
    sm.row_lo = sg.row_lo; sm.row_hi = sg.row_hi; sm.st_lo = sg.st_lo; sm.st_hi = sg.st_hi;
    if (res) {
      S.steps.push_back(SwStep{SW_BEGIN, sg.row_lo, sg.row_hi, 0});
      S.runs++;
    }
    for (int p = sg.first; p < sg.first + sg.count; ++p) {
      const int32_t o0 = fp.base[p], o1 = fp.base[p + 1];
      if (o1 <= o0) continue;
      if (fp.ops[o0].kind == FK_LEAF) {
        // a sweep leaf always lies inside a resident run (its rows alone fit the window)
        if (!res) { S.ok = false; S.why = "sweep leaf outside a resident run"; return; }
        for (int32_t o = o0; o < o1; ++o) bd.emit_tri(fp.ops[o], which, sm.vec(fp.ops[o].src0));
      } else {
        P.clear();
        for (int32_t o = o0; o < o1; ++o) expand_op(ph, fp.ops[o], sm, P);
        bd.emit_phase(P, res);
      }
      if (res) S.res_phases++;
      else S.glob_phases++;
      if (sm.bad) { S.ok = false; S.why = "slot outside the run's window"; return; }
      if (!S.ok) return;
    }
    if (res) S.steps.push_back(SwStep{SW_END, sg.row_lo, sg.row_hi, 0});
  }
  // (the device stages complex-FP32 images; FP64 images serve host checks only)
  if (coef_bytes == 8 && S.max_bytes > kSwRingBytes) { S.ok = false; S.why = "batch image larger than the staging ring"; }
}

void host_sweep_sched(const PackedHost& ph, const SwSched& S, cplx* vec) {
  const int64_t n = ph.n;
  std::vector<cplx> st((size_t)ph.state_len, cplx(0.0, 0.0)), win(kSwWinSlots), tmp;
  auto coef = [&](const uint8_t* p, int64_t e) -> cplx {
    if (S.coef_bytes == 8) {
      float v[2];
      std::memcpy(v, p + e * 8, 8);
      return cplx(v[0], v[1]);
    }
    double v[2];
    std::memcpy(v, p + e * 16, 16);
    return cplx(v[0], v[1]);
  };
  struct Out { bool res; int32_t o; cplx v; };
  std::vector<Out> outs;
  for (const SwStep& s : S.steps) {
    if (s.kind == SW_BEGIN) {
      for (int32_t r = s.a0; r < s.a1; ++r) win[r - s.a0] = vec[r];
      continue;
    }
    if (s.kind == SW_END) {
      for (int32_t r = s.a0; r < s.a1; ++r) vec[r] = win[r - s.a0];
      continue;
    }
    // outputs of a phase never feed the same phase: compute every batch from the
    // values before the phase, then store (as the kernel's phase barrier implies)
    outs.clear();
    for (int32_t b = s.a0; b < s.a0 + s.a1; ++b) {
      const SwBatch& B = S.batches[b];
      const uint8_t* base = S.image.data() + B.img;
      if (B.flags & SWF_TRI) {
        const int64_t sz = B.nrows;
        tmp.assign((size_t)sz, cplx(0.0, 0.0));
        const bool up = (B.flags & SWF_UPPER) != 0;
        for (int64_t c = 0; c < sz; ++c)
          for (int64_t r = up ? 0 : c; r < (up ? c + 1 : sz); ++r) {
            const int64_t off = up ? tri_off_upper(r, c) : tri_off_lower(sz, r, c);
            tmp[r] += coef(base, off) * win[B.a0 + c];
          }
        for (int64_t r = 0; r < sz; ++r) win[B.a0 + r] = tmp[r];
        continue;
      }
      const int32_t* out = (const int32_t*)base;
      const int32_t* e0 = (const int32_t*)(base + B.off_e0);
      const uint8_t* cf = base + B.off_coef;
      const bool res = (B.flags & SWF_RES) != 0;
      auto in_val = [&](int64_t e) -> cplx {
        if (res) return win[((const int16_t*)(base + B.off_in))[e]];
        const int32_t sl = ((const int32_t*)(base + B.off_in))[e];
        return sl < n ? vec[sl] : st[sl - n];
      };
      for (int32_t r = 0; r < B.nrows; ++r) {
        cplx acc(0.0, 0.0);
        for (int32_t e = e0[r]; e < e0[r + 1]; ++e) acc += coef(cf, e) * in_val(e);
        outs.push_back(Out{res, out[r], acc});
      }
    }
    for (const Out& ov : outs) {
      const bool acc = (ov.o & kSwAcc) != 0;
      const int32_t sl = ov.o & ~kSwAcc;
      cplx* d = ov.res ? &win[sl] : (sl < n ? &vec[sl] : &st[sl - n]);
      *d = acc ? *d + ov.v : ov.v;
    }
  }
}

}  // namespace hb

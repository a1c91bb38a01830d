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

// A batch before layout: rows of one phase (indices into PhaseRows), or a triangle.
struct PBatch {
  std::vector<int32_t> rows;
  std::vector<int32_t> gl;   // global batches: distinct input slots
  int glog = 0;
  bool tri = false;
  int64_t tri_off = 0, tri_n = 0;   // triangle: offset in the sweep-leaf array, order
  int32_t a0 = 0;
};

struct Builder {
  const PackedHost& ph;
  SwSched& S;
  int cb, which;
  Builder(const PackedHost& p, SwSched& s, int coef_bytes, int w) : ph(p), S(s), cb(coef_bytes), which(w) {}

  void coef_at(uint8_t* dst, cplx v) {
    if (cb == 8) put_coef<float>(dst, v);
    else put_coef<double>(dst, v);
  }
  int64_t batch_bytes(const PhaseRows& P, const PBatch& B, bool res) const {
    if (B.tri) return al16(packed_tri(B.tri_n) * cb);
    int64_t ne = 0;
    for (int32_t r : B.rows) ne += P.len(r);
    const int64_t nr = (int64_t)B.rows.size();
    return al16(4 * nr) + al16(4 * (nr + 1)) + al16(cb * ne) + al16(2 * ne) + (res ? 0 : al16(4 * (int64_t)B.gl.size()));
  }

  // lay out one group: header, descriptors, the batches' data
  void emit_group(const PhaseRows& P, const std::vector<PBatch>& bs, size_t b0, size_t b1, int32_t flags,
                  int32_t beg_lo, int32_t beg_hi, int32_t end_lo, int32_t end_hi) {
    const bool res = (flags & SWG_RES) != 0;
    const int64_t nb = (int64_t)(b1 - b0);
    int64_t off = al16(32 + 40 * nb), bytes = off;
    for (size_t q = b0; q < b1; ++q) bytes += batch_bytes(P, bs[q], res);
    if (bytes > INT32_MAX / 2) { S.ok = false; S.why = "group too large"; return; }
    SwGroup G{(int64_t)S.image.size(), (int32_t)bytes, 0};
    S.image.resize((size_t)(G.img + bytes), 0);
    uint8_t* base = S.image.data() + G.img;
    SwGroupHdr H{(int32_t)nb, flags, beg_lo, beg_hi, end_lo, end_hi, 0, 0};
    std::memcpy(base, &H, sizeof(H));
    for (size_t q = b0; q < b1; ++q) {
      const PBatch& B = bs[q];
      SwDesc D{};
      D.off = (int32_t)off;
      D.glog = (int16_t)B.glog;
      uint8_t* d = base + off;
      if (B.tri) {
        D.nrows = (int32_t)B.tri_n;
        D.nent = (int32_t)packed_tri(B.tri_n);
        D.a0 = B.a0;
        const cplx* T = ph.sl[which].data() + B.tri_off;
        for (int64_t e = 0; e < D.nent; ++e) coef_at(d + e * cb, T[e]);
      } else {
        int64_t ne = 0;
        for (int32_t r : B.rows) ne += P.len(r);
        const int64_t nr = (int64_t)B.rows.size();
        D.nrows = (int32_t)nr;
        D.nent = (int32_t)ne;
        D.ngl = (int32_t)B.gl.size();
        D.off_e0 = (int32_t)al16(4 * nr);
        D.off_coef = D.off_e0 + (int32_t)al16(4 * (nr + 1));
        D.off_in = D.off_coef + (int32_t)al16(cb * ne);
        D.off_gl = D.off_in + (int32_t)al16(2 * ne);
        int32_t* out = (int32_t*)d;
        int32_t* e0 = (int32_t*)(d + D.off_e0);
        int16_t* in = (int16_t*)(d + D.off_in);
        int32_t* gl = (int32_t*)(d + D.off_gl);
        // global batches: input slot -> position in the gather list
        std::vector<std::pair<int32_t, int32_t>> pos;
        if (!res) {
          for (size_t k = 0; k < B.gl.size(); ++k) {
            gl[k] = B.gl[k];
            pos.emplace_back(B.gl[k], (int32_t)k);
          }
          std::sort(pos.begin(), pos.end());
        }
        int32_t e = 0;
        for (int64_t q2 = 0; q2 < nr; ++q2) {
          const int32_t r = B.rows[q2];
          out[q2] = P.out[r];
          e0[q2] = e;
          const int32_t s0 = P.start[r], n = P.len(r);
          for (int32_t t = 0; t < n; ++t, ++e) {
            coef_at(d + D.off_coef + (int64_t)e * cb, P.coef[s0 + t]);
            const int32_t sl = P.slot[s0 + t];
            if (res) {
              in[e] = (int16_t)sl;
            } else {
              auto it = std::lower_bound(pos.begin(), pos.end(), std::make_pair(sl, INT32_MIN));
              in[e] = (int16_t)it->second;
            }
          }
        }
        e0[nr] = e;
      }
      std::memcpy(base + 32 + 40 * (q - b0), &D, sizeof(D));
      off += batch_bytes(P, B, res);
      S.batches++;
    }
    S.max_bytes = std::max<int64_t>(S.max_bytes, bytes);
    S.groups.push_back(G);
  }

  // lanes per row: about eight entries per lane
  static int pick_glog(const PhaseRows& P) {
    const double avg = P.nrows() > 0 ? (double)P.slot.size() / P.nrows() : 1.0;
    int g = 0;
    while (g < 5 && (double)(8 << g) < avg) ++g;
    return g;
  }

  // batches -> groups of at most kSwGroupBytes (a group holds at least one batch)
  void emit_groups(const PhaseRows& P, const std::vector<PBatch>& bs, int32_t flags, bool begin, int32_t beg_lo,
                   int32_t beg_hi, bool endrun, int32_t end_lo, int32_t end_hi) {
    const bool res = (flags & SWG_RES) != 0;
    size_t g0 = 0;
    int64_t acc = 0;
    for (size_t q = 0; q <= bs.size(); ++q) {
      const int64_t add = q < bs.size() ? 40 + batch_bytes(P, bs[q], res) : 0;
      const bool last = q == bs.size();
      if (last || (acc + add > kSwGroupBytes && q > g0)) {
        int32_t fl = flags;
        if (g0 == 0 && begin) fl |= SWG_BEGIN;
        if (last) fl |= SWG_END | (endrun ? SWG_ENDRUN : 0);
        emit_group(P, bs, g0, q, fl, begin ? beg_lo : 0, begin ? beg_hi : 0, endrun ? end_lo : 0,
                   endrun ? end_hi : 0);
        if (!S.ok) return;
        g0 = q;
        acc = 0;
      }
      acc += add;
    }
  }

  void phase_batches(const PhaseRows& P, bool res, std::vector<PBatch>& bs) {
    bs.clear();
    const int32_t nrows = P.nrows();
    const int glog = pick_glog(P);
    const int per_round = 32 >> glog;
    std::vector<int32_t> order(nrows);
    for (int32_t r = 0; r < nrows; ++r) order[r] = r;
    if (res) {
      // a dependent phase: about one batch per compute warp (more if the data would
      // be too large), rows by decreasing length dealt round-robin
      int64_t tot = 0;
      for (int32_t r = 0; r < nrows; ++r) tot += 8 + (int64_t)(cb + 2) * P.len(r);
      int64_t nb = std::min<int64_t>(kSwWarps, (nrows + per_round - 1) / per_round);
      nb = std::max<int64_t>(nb, (tot + kSwBatchBytes - 1) / kSwBatchBytes);
      nb = std::max<int64_t>(1, std::min<int64_t>(nb, nrows));
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return P.len(a) > P.len(b); });
      bs.resize(nb);
      for (int64_t q = 0; q < nb; ++q) {
        bs[q].glog = glog;
        for (int64_t i2 = q; i2 < nrows; i2 += nb) bs[q].rows.push_back(order[i2]);
      }
      return;
    }
    // wide phase: consecutive rows (an op's rows share inputs), batches of about
    // kSwGlobBytes of data with at most kSwGather distinct inputs
    PBatch cur;
    cur.glog = glog;
    std::vector<int32_t> seen;   // sorted distinct inputs of cur
    int64_t acc = 0;
    std::vector<int32_t> fresh;
    for (int32_t r = 0; r < nrows; ++r) {
      fresh.clear();
      const int32_t s0 = P.start[r], n = P.len(r);
      for (int32_t t = 0; t < n; ++t) {
        const int32_t sl = P.slot[s0 + t];
        if (!std::binary_search(seen.begin(), seen.end(), sl) &&
            std::find(fresh.begin(), fresh.end(), sl) == fresh.end())
          fresh.push_back(sl);
      }
      const int64_t add = 8 + (int64_t)(cb + 2) * n + 4 * (int64_t)fresh.size();
      if (!cur.rows.empty() &&
          (acc + add > kSwGlobBytes || seen.size() + fresh.size() > (size_t)kSwGather)) {
        cur.gl = seen;
        bs.push_back(std::move(cur));
        cur = PBatch();
        cur.glog = glog;
        seen.clear();
        acc = 0;
        fresh.clear();
        for (int32_t t = 0; t < n; ++t) {
          const int32_t sl = P.slot[s0 + t];
          if (std::find(fresh.begin(), fresh.end(), sl) == fresh.end()) fresh.push_back(sl);
        }
      }
      if (fresh.size() > (size_t)kSwGather) { S.ok = false; S.why = "a row has too many inputs"; return; }
      cur.rows.push_back(r);
      for (int32_t sl : fresh) seen.insert(std::lower_bound(seen.begin(), seen.end(), sl), sl);
      acc += 8 + (int64_t)(cb + 2) * n + 4 * (int64_t)fresh.size();
    }
    if (!cur.rows.empty()) {
      cur.gl = seen;
      bs.push_back(std::move(cur));
    }
    // rows of a batch by decreasing length (the lanes' rounds stay balanced)
    for (PBatch& B : bs)
      std::stable_sort(B.rows.begin(), B.rows.end(), [&](int32_t a, int32_t b) { return P.len(a) > P.len(b); });
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
  Builder bd(ph, S, coef_bytes, which);
  PhaseRows P;
  std::vector<PBatch> bs;
  for (const DSeg& sg : segs) {
    const int64_t rows = sg.row_hi - sg.row_lo, nst = sg.st_hi - sg.st_lo;
    const bool res = !sg.grid && !sg.st_cross && rows + nst <= S.win_slots && rows > 0;
    SlotMap sm;
    sm.n = ph.n;
    sm.res = res;
    sm.row_lo = sg.row_lo; sm.row_hi = sg.row_hi; sm.st_lo = sg.st_lo; sm.st_hi = sg.st_hi;
    if (res) S.runs++;
    // phases of the segment that hold ops
    std::vector<int> phs;
    for (int p = sg.first; p < sg.first + sg.count; ++p)
      if (fp.base[p + 1] > fp.base[p]) phs.push_back(p);
    for (size_t k = 0; k < phs.size(); ++k) {
      const int p = phs[k];
      const int32_t o0 = fp.base[p], o1 = fp.base[p + 1];
      const bool first = k == 0, last = k + 1 == phs.size();
      P.clear();
      int32_t flags = res ? SWG_RES : 0;
      if (fp.ops[o0].kind == FK_LEAF) {
        // a sweep leaf always lies inside a resident run (its rows alone fit the window)
        if (!res || o1 - o0 != 1) { S.ok = false; S.why = "sweep leaf outside a resident run"; return; }
        const FlatOp& f = fp.ops[o0];
        bs.assign(1, PBatch());
        bs[0].tri = true;
        bs[0].tri_off = f.moff;
        bs[0].tri_n = f.c0;
        bs[0].a0 = sm.vec(f.src0);
        flags |= SWG_TRI | ((f.flags & FF_UPPER) ? SWG_UPPER : 0);
      } else {
        for (int32_t o = o0; o < o1; ++o) expand_op(ph, fp.ops[o], sm, P);
        bd.phase_batches(P, res, bs);
      }
      if (sm.bad) { S.ok = false; S.why = "slot outside the run's window"; return; }
      if (!S.ok) return;
      bd.emit_groups(P, bs, flags, res && first, sg.row_lo, sg.row_hi, res && last, sg.row_lo, sg.row_hi);
      if (!S.ok) return;
      if (res) S.res_phases++;
      else S.glob_phases++;
    }
  }
  // (the device stages complex-FP32 images; FP64 images serve host checks only)
  if (coef_bytes == 8 && S.max_bytes > kSwRingBytes) { S.ok = false; S.why = "group image larger than the staging ring"; }
}

void host_sweep_sched(const PackedHost& ph, const SwSched& S, cplx* vec) {
  const int64_t n = ph.n;
  std::vector<cplx> st((size_t)ph.state_len, cplx(0.0, 0.0)), win(kSwWinSlots), tmp, gv;
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
  auto gslot = [&](int32_t sl) -> cplx& { return sl < n ? vec[sl] : st[sl - n]; };
  // a phase's outputs are stored at its end (its groups never read them)
  struct Out { bool res; int32_t o; cplx v; };
  std::vector<Out> outs;
  for (const SwGroup& G : S.groups) {
    const uint8_t* gb = S.image.data() + G.img;
    SwGroupHdr H;
    std::memcpy(&H, gb, sizeof(H));
    if (H.flags & SWG_BEGIN)
      for (int32_t r = H.beg_lo; r < H.beg_hi; ++r) win[r - H.beg_lo] = vec[r];
    const bool res = (H.flags & SWG_RES) != 0;
    for (int32_t b = 0; b < H.nb; ++b) {
      SwDesc D;
      std::memcpy(&D, gb + 32 + 40 * b, sizeof(D));
      const uint8_t* base = gb + D.off;
      if (H.flags & SWG_TRI) {
        const int64_t sz = D.nrows;
        tmp.assign((size_t)sz, cplx(0.0, 0.0));
        const bool up = (H.flags & SWG_UPPER) != 0;
        for (int64_t c = 0; c < sz; ++c)
          for (int64_t r = up ? 0 : c; r < (up ? c + 1 : sz); ++r) {
            const int64_t off = up ? tri_off_upper(r, c) : tri_off_lower(sz, r, c);
            tmp[r] += coef(base, off) * win[D.a0 + c];
          }
        for (int64_t r = 0; r < sz; ++r) win[D.a0 + r] = tmp[r];
        continue;
      }
      const int32_t* out = (const int32_t*)base;
      const int32_t* e0 = (const int32_t*)(base + D.off_e0);
      const int16_t* in = (const int16_t*)(base + D.off_in);
      const int32_t* gl = (const int32_t*)(base + D.off_gl);
      if (!res) {   // gather the batch's distinct inputs
        gv.resize((size_t)D.ngl);
        for (int32_t k = 0; k < D.ngl; ++k) gv[k] = gslot(gl[k]);
      }
      for (int32_t r = 0; r < D.nrows; ++r) {
        cplx acc(0.0, 0.0);
        for (int32_t e = e0[r]; e < e0[r + 1]; ++e) acc += coef(base + D.off_coef, e) * (res ? win[in[e]] : gv[in[e]]);
        outs.push_back(Out{res, out[r], acc});
      }
    }
    if (H.flags & SWG_END) {
      for (const Out& ov : outs) {
        const bool add = (ov.o & kSwAcc) != 0;
        const int32_t sl = ov.o & ~kSwAcc;
        cplx* d = ov.res ? &win[sl] : &gslot(sl);
        *d = add ? *d + ov.v : ov.v;
      }
      outs.clear();
      if (H.flags & SWG_ENDRUN)
        for (int32_t r = H.end_lo; r < H.end_hi; ++r) vec[r] = win[r - H.end_lo];
    }
  }
}

}  // namespace hb

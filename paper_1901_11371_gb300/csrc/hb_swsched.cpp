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
      // subtracting from an output: in the window, add to it in place; in global
      // memory, read its old value as one more input (coefficient 1), so that the
      // kernel's store needs no dependent load
      if (sub && !sm.res) {
        P.begin_row(o);
        P.add(o, cplx(1.0, 0.0));
      } else {
        P.begin_row(sub ? (o | kSwAcc) : o);
      }
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

// One phase part laid out on its own: descriptors with offsets relative to the
// part's data, and the data.
struct Part {
  int32_t flags = 0;   // SWP_*
  std::vector<SwDesc> descs;
  std::vector<uint8_t> data;
};

// log2 of the lanes per row of a batch: as many lanes per row as the warp's 32
// allow for the batch's rows, but not more than half the average row length
int batch_glog(const PhaseRows& P, const std::vector<int32_t>& rows) {
  if (rows.empty()) return 0;
  int64_t ne = 0;
  for (int32_t r : rows) ne += P.len(r);
  const double avg = (double)ne / (double)rows.size();
  int g = 0;
  while (g < 5 && ((int64_t)rows.size() << (g + 1)) <= 32 && (double)(4 << g) <= avg) ++g;
  return g;
}

struct Builder {
  const PackedHost& ph;
  SwSched& S;
  int cb, which;
  // the group being collected
  std::vector<Part> pend;
  int64_t pend_bytes = 0;
  bool pend_res = false;
  int64_t glob_batches = 0;   // batches of the current global phase so far (warp rotation)
  Builder(const PackedHost& p, SwSched& s, int coef_bytes, int w) : ph(p), S(s), cb(coef_bytes), which(w) {}

  void coef_at(uint8_t* dst, cplx v) {
    if (cb == 8) put_coef<float>(dst, v);
    else put_coef<double>(dst, v);
  }

  // lay out batches bs[b0, b1) as one part
  Part make_part(const PhaseRows& P, const std::vector<PBatch>& bs, size_t b0, size_t b1, bool res, int32_t pflags) {
    Part pt;
    pt.flags = pflags;
    for (size_t q = b0; q < b1; ++q) {
      const PBatch& B = bs[q];
      SwDesc D{};
      D.off = (int32_t)pt.data.size();
      D.glog = (int16_t)B.glog;
      if (B.tri) {
        D.nrows = (int32_t)B.tri_n;
        D.nent = (int32_t)packed_tri(B.tri_n);
        D.a0 = B.a0;
        pt.data.resize(pt.data.size() + al16((int64_t)D.nent * cb), 0);
        uint8_t* d = pt.data.data() + D.off;
        // stored as a lower triangle, column by column; an upper triangle U reversed:
        // stored (r, c) = U(s-1-r, s-1-c)
        const cplx* T = ph.sl[which].data() + B.tri_off;
        const int64_t sz = B.tri_n;
        const bool up = which == 1 || which == 2;
        for (int64_t c = 0; c < sz; ++c)
          for (int64_t r = c; r < sz; ++r) {
            const cplx v = up ? T[tri_off_upper(sz - 1 - r, sz - 1 - c)] : T[tri_off_lower(sz, r, c)];
            coef_at(d + tri_off_lower(sz, r, c) * cb, v);
          }
        pt.descs.push_back(D);
        S.batches++;
        continue;
      }
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
      const int64_t bytes = D.off_gl + (res ? 0 : al16(4 * (int64_t)D.ngl));
      pt.data.resize(pt.data.size() + bytes, 0);
      uint8_t* d = pt.data.data() + D.off;
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
      pt.descs.push_back(D);
      S.batches++;
    }
    return pt;
  }
  int64_t batch_bytes(const PhaseRows& P, const PBatch& B, bool res) const {
    if (B.tri) return al16(packed_tri(B.tri_n) * cb);
    int64_t ne = 0;
    for (int32_t r : B.rows) ne += P.len(r);
    const int64_t nr = (int64_t)B.rows.size();
    return al16(4 * nr) + al16(4 * (nr + 1)) + al16(cb * ne) + al16(2 * ne) + (res ? 0 : al16(4 * (int64_t)B.gl.size()));
  }
  static int64_t part_bytes(const Part& pt) { return 8 + 40 * (int64_t)pt.descs.size() + (int64_t)pt.data.size(); }

  // write the collected parts as one group
  void flush(bool begin, int32_t beg_lo, int32_t beg_hi) {
    if (pend.empty()) return;
    const int64_t nph = (int64_t)pend.size();
    int64_t nd = 0;
    for (const Part& pt : pend) nd += (int64_t)pt.descs.size();
    const int64_t off_desc = al16(32 + 8 * nph);
    const int64_t off_data = al16(off_desc + 40 * nd);
    int64_t bytes = off_data;
    for (const Part& pt : pend) bytes += al16((int64_t)pt.data.size());
    if (bytes > INT32_MAX / 2) { S.ok = false; S.why = "group too large"; pend.clear(); return; }
    SwGroup G{(int64_t)S.image.size(), (int32_t)bytes, 0};
    S.image.resize((size_t)(G.img + bytes), 0);
    uint8_t* base = S.image.data() + G.img;
    SwGroupHdr H{(int32_t)nph, pend_res ? SWG_RES : 0, 0, 0, 0, 0, (int32_t)off_desc,
                 pend_res ? 0 : (int32_t)(glob_batches % kSwWarps)};
    if (!pend_res) glob_batches += nd;
    if (begin) {
      H.flags |= SWG_BEGIN;
      H.beg_lo = beg_lo;
      H.beg_hi = beg_hi;
    }
    std::memcpy(base, &H, sizeof(H));
    int64_t di = 0, dat = off_data;
    for (int64_t k = 0; k < nph; ++k) {
      const Part& pt = pend[k];
      const SwPhase ph_ent{(int32_t)pt.descs.size(), pt.flags};
      std::memcpy(base + 32 + 8 * k, &ph_ent, sizeof(ph_ent));
      for (SwDesc D : pt.descs) {
        D.off += (int32_t)dat;
        std::memcpy(base + off_desc + 40 * di, &D, sizeof(D));
        ++di;
      }
      if (!pt.data.empty()) std::memcpy(base + dat, pt.data.data(), pt.data.size());
      dat += al16((int64_t)pt.data.size());
    }
    S.max_bytes = std::max<int64_t>(S.max_bytes, bytes);
    S.groups.push_back(G);
    pend.clear();
    pend_bytes = 0;
  }

  void batches_of_phase(const PhaseRows& P, bool res, std::vector<PBatch>& bs) {
    bs.clear();
    const int32_t nrows = P.nrows();
    std::vector<int32_t> order(nrows);
    for (int32_t r = 0; r < nrows; ++r) order[r] = r;
    if (res) {
      // a dependent phase: one batch per compute warp (more if the data would be
      // too large), rows by decreasing length dealt round-robin
      int64_t tot = 0;
      for (int32_t r = 0; r < nrows; ++r) tot += 8 + (int64_t)(cb + 2) * P.len(r);
      int64_t nb = std::min<int64_t>(kSwChain, nrows);
      nb = std::max<int64_t>(nb, (tot + kSwBatchBytes - 1) / kSwBatchBytes);
      nb = std::max<int64_t>(1, std::min<int64_t>(nb, nrows));
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return P.len(a) > P.len(b); });
      bs.resize(nb);
      for (int64_t q = 0; q < nb; ++q) {
        for (int64_t i2 = q; i2 < nrows; i2 += nb) bs[q].rows.push_back(order[i2]);
        bs[q].glog = batch_glog(P, bs[q].rows);
      }
      return;
    }
    // wide phase: consecutive rows (an op's rows share inputs), batches of about
    // kSwGlobBytes of data with at most kSwGather distinct inputs
    PBatch cur;
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
    for (PBatch& B : bs) {
      std::stable_sort(B.rows.begin(), B.rows.end(), [&](int32_t a, int32_t b) { return P.len(a) > P.len(b); });
      int64_t ne = 0;
      for (int32_t r : B.rows) ne += P.len(r);
      const double avg = (double)ne / (double)B.rows.size();
      int g = 0;
      while (g < 5 && (double)(8 << g) < avg) ++g;   // about eight entries per lane
      B.glog = g;
    }
  }

  // add a phase's batches to the groups: parts of at most kSwGroupBytes, the last
  // one ending the phase; resident parts share groups, global ones do not
  void add_phase(const PhaseRows& P, const std::vector<PBatch>& bs, bool res, int32_t pflags, bool& begin,
                 int32_t beg_lo, int32_t beg_hi) {
    size_t b0 = 0;
    while (b0 < bs.size()) {
      size_t b1 = b0;
      int64_t acc = 0;
      while (b1 < bs.size()) {
        const int64_t add = 40 + batch_bytes(P, bs[b1], res);
        if (b1 > b0 && acc + add > kSwGroupBytes) break;
        acc += add;
        ++b1;
      }
      const bool last = b1 == bs.size();
      Part pt = make_part(P, bs, b0, b1, res, pflags & ~(last ? 0 : SWP_END));
      const int64_t pb = part_bytes(pt);
      if (!pend.empty() && (!res || !pend_res || (pflags & SWP_TRI) || pend_bytes + pb > kSwGroupBytes ||
                            (int)pend.size() >= kSwMaxPhases)) {
        flush(begin, beg_lo, beg_hi);
        begin = false;
      }
      pend_res = res;
      pend.push_back(std::move(pt));
      pend_bytes += pb;
      if (!res || (pflags & SWP_TRI)) {   // global parts and triangles form groups of their own
        flush(begin, beg_lo, beg_hi);
        begin = false;
      }
      b0 = b1;
    }
  }
};

}  // namespace

void build_sweep_sched(const PackedHost& ph, int which, int coef_bytes, int win_slots, SwSched& S) {
  // (resident runs: their groups are counted into the first one's header below)
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
    bool begin = res;   // the run's first group loads its rows
    if (res) S.runs++;
    const size_t run_g0 = S.groups.size();
    bd.glob_batches = 0;
    for (int p = sg.first; p < sg.first + sg.count; ++p) {
      const int32_t o0 = fp.base[p], o1 = fp.base[p + 1];
      if (o1 <= o0) continue;
      P.clear();
      int32_t pflags = SWP_END;
      if (fp.ops[o0].kind == FK_LEAF) {
        // a sweep leaf always lies inside a resident run (its rows alone fit the window)
        if (!res || o1 - o0 != 1) { S.ok = false; S.why = "sweep leaf outside a resident run"; return; }
        const FlatOp& f = fp.ops[o0];
        bs.assign(1, PBatch());
        bs[0].tri = true;
        bs[0].tri_off = f.moff;
        bs[0].tri_n = f.c0;
        bs[0].a0 = sm.vec(f.src0);
        pflags |= SWP_TRI | ((f.flags & FF_UPPER) ? SWP_UPPER : 0);
      } else {
        for (int32_t o = o0; o < o1; ++o) expand_op(ph, fp.ops[o], sm, P);
        bd.batches_of_phase(P, res, bs);
      }
      if (sm.bad) { S.ok = false; S.why = "slot outside the run's window"; return; }
      if (!S.ok) return;
      bd.add_phase(P, bs, res, pflags, begin, sg.row_lo, sg.row_hi);
      if (!S.ok) return;
      if (res) S.res_phases++;
      else S.glob_phases++;
      bd.glob_batches = 0;
    }
    bd.flush(begin, sg.row_lo, sg.row_hi);
    begin = false;
    if (res && S.groups.size() > run_g0) {
      // the run's last group writes the rows back after its last phase; its first
      // group tells how many groups the run has
      SwGroupHdr H;
      uint8_t* hb = S.image.data() + S.groups.back().img;
      std::memcpy(&H, hb, sizeof(H));
      H.flags |= SWG_ENDRUN;
      H.end_lo = sg.row_lo;
      H.end_hi = sg.row_hi;
      std::memcpy(hb, &H, sizeof(H));
      hb = S.image.data() + S.groups[run_g0].img;
      std::memcpy(&H, hb, sizeof(H));
      if (!(H.flags & SWG_BEGIN)) { S.ok = false; S.why = "resident run without its first group"; return; }
      H.aux = (int32_t)(S.groups.size() - run_g0);
      std::memcpy(hb, &H, sizeof(H));
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
  // a phase's outputs are stored when it ends (its parts never read them)
  struct Out { bool res; int32_t o; cplx v; };
  std::vector<Out> outs;
  for (const SwGroup& G : S.groups) {
    const uint8_t* gb = S.image.data() + G.img;
    SwGroupHdr H;
    std::memcpy(&H, gb, sizeof(H));
    if (H.flags & SWG_BEGIN)
      for (int32_t r = H.beg_lo; r < H.beg_hi; ++r) win[r - H.beg_lo] = vec[r];
    const bool res = (H.flags & SWG_RES) != 0;
    int64_t di = 0;
    for (int32_t k = 0; k < H.nph; ++k) {
      SwPhase PH;
      std::memcpy(&PH, gb + 32 + 8 * k, sizeof(PH));
      for (int32_t b = 0; b < PH.nb; ++b, ++di) {
        SwDesc D;
        std::memcpy(&D, gb + H.off_desc + 40 * di, sizeof(D));
        const uint8_t* base = gb + D.off;
        if (PH.flags & SWP_TRI) {
          // lower layout; reversed rows and columns for an upper triangle
          const int64_t sz = D.nrows;
          tmp.assign((size_t)sz, cplx(0.0, 0.0));
          const bool rev = (PH.flags & SWP_UPPER) != 0;
          for (int64_t c = 0; c < sz; ++c)
            for (int64_t r = c; r < sz; ++r) {
              const int64_t ro = rev ? sz - 1 - r : r, co = rev ? sz - 1 - c : c;
              tmp[ro] += coef(base, tri_off_lower(sz, r, c)) * win[D.a0 + co];
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
          for (int32_t q = 0; q < D.ngl; ++q) gv[q] = gslot(gl[q]);
        }
        for (int32_t r = 0; r < D.nrows; ++r) {
          cplx acc(0.0, 0.0);
          for (int32_t e = e0[r]; e < e0[r + 1]; ++e)
            acc += coef(base + D.off_coef, e) * (res ? win[in[e]] : gv[in[e]]);
          outs.push_back(Out{res, out[r], acc});
        }
      }
      if (PH.flags & SWP_END) {
        for (const Out& ov : outs) {
          const bool add = (ov.o & kSwAcc) != 0;
          const int32_t sl = ov.o & ~kSwAcc;
          cplx* d = ov.res ? &win[sl] : &gslot(sl);
          *d = add ? *d + ov.v : ov.v;
        }
        outs.clear();
      }
    }
    if (H.flags & SWG_ENDRUN)
      for (int32_t r = H.end_lo; r < H.end_hi; ++r) vec[r] = win[r - H.end_lo];
  }
}

const char* check_sweep_sched(const PackedHost& ph, const SwSched& S) {
  const int64_t n = ph.n;
  const int cb = S.coef_bytes;
  int64_t run_left = 0;   // groups of the current resident run still to come
  int32_t win_rows = 0;
  // per window slot: the last resident phase that wrote / read it (a resident
  // phase's batches run concurrently on the chain warps, so no slot may be
  // written twice in a phase, nor written and read by the same phase)
  std::vector<int64_t> wstamp((size_t)S.win_slots, -1), rstamp((size_t)S.win_slots, -1);
  int64_t pid = 0;
  for (size_t gi = 0; gi < S.groups.size(); ++gi) {
    const SwGroup& G = S.groups[gi];
    if (G.img % 16 || G.bytes % 16 || G.bytes <= 0) return "group not 16-byte aligned";
    if (cb == 8 && G.bytes > kSwRingBytes) return "group larger than the ring";
    if (G.img + G.bytes > (int64_t)S.image.size()) return "group outside the image";
    const uint8_t* gb = S.image.data() + G.img;
    SwGroupHdr H;
    std::memcpy(&H, gb, sizeof(H));
    const bool res = (H.flags & SWG_RES) != 0;
    if (H.nph < 1 || 32 + 8 * (int64_t)H.nph > H.off_desc) return "phase table";
    if (res) {
      if (run_left == 0) {
        if (!(H.flags & SWG_BEGIN) || H.aux < 1) return "run start without BEGIN or length";
        run_left = H.aux;
        win_rows = H.beg_hi - H.beg_lo;
        if (win_rows < 1 || win_rows > S.win_slots) return "run rows";
      } else if (H.flags & SWG_BEGIN) {
        return "BEGIN inside a run";
      }
      --run_left;
      if ((run_left == 0) != ((H.flags & SWG_ENDRUN) != 0)) return "ENDRUN not on the run's last group";
    } else {
      if (run_left != 0) return "global group inside a run";
      if (H.nph != 1) return "global group with several phases";
      if (H.aux < 0 || H.aux >= kSwWarps) return "warp rotation";
    }
    int64_t di = 0;
    for (int32_t k = 0; k < H.nph; ++k) {
      SwPhase PH;
      std::memcpy(&PH, gb + 32 + 8 * k, sizeof(PH));
      if (PH.nb < 1) return "empty phase part";
      if ((PH.flags & SWP_TRI) && (PH.nb != 1 || !res)) return "triangle part";
      if (res && !(PH.flags & SWP_END)) {
        // a resident phase split over groups: only its last part ends it
        if (k + 1 != H.nph) return "unfinished resident phase inside a group";
      }
      for (int32_t b = 0; b < PH.nb; ++b, ++di) {
        SwDesc D;
        if (H.off_desc + 40 * (di + 1) > G.bytes) return "descriptor outside the group";
        std::memcpy(&D, gb + H.off_desc + 40 * di, sizeof(D));
        if (D.off % 16 || D.off < H.off_desc) return "batch offset";
        if (PH.flags & SWP_TRI) {
          const int64_t s = D.nrows;
          if (s < 2 || (s & 1) || 2 * (s / 2) * 1 == 0) return "triangle order";
          if (D.off + al16(packed_tri(s) * cb) > G.bytes) return "triangle outside the group";
          if (D.a0 < 0 || D.a0 + s > win_rows) return "triangle rows outside the window rows";
          if (s * kSwMaxCols * 8 > kSwPartBytes) return "triangle partial sums";
          continue;
        }
        const int64_t end = D.off + D.off_gl + (res ? 0 : al16(4 * (int64_t)D.ngl));
        if (end > G.bytes) return "batch outside the group";
        if (D.glog < 0 || D.glog > 5) return "lanes per row";
        if (!res && (D.ngl < 0 || D.ngl > kSwGather)) return "gather list longer than a warp slice";
        const uint8_t* bb = gb + D.off;
        const int32_t* out = (const int32_t*)bb;
        const int32_t* e0 = (const int32_t*)(bb + D.off_e0);
        const int16_t* in = (const int16_t*)(bb + D.off_in);
        const int32_t* gl = (const int32_t*)(bb + D.off_gl);
        if (e0[0] != 0 || e0[D.nrows] != D.nent) return "row offsets";
        for (int32_t r = 0; r < D.nrows; ++r) {
          if (e0[r + 1] < e0[r]) return "row offsets";
          if (!res && (out[r] & kSwAcc)) return "global row that adds in place";
          const int32_t o = out[r] & ~kSwAcc;
          if (res ? (o < 0 || o >= S.win_slots) : (o < 0 || o >= n + ph.state_len)) return "output slot";
          if (res) {
            if (wstamp[o] == pid) return "window slot written twice in one phase";
            if (rstamp[o] == pid) return "window slot read and written in one phase";
            wstamp[o] = pid;
          }
        }
        for (int32_t e = 0; e < D.nent; ++e) {
          if (res ? (in[e] < 0 || in[e] >= S.win_slots) : (in[e] < 0 || in[e] >= D.ngl)) return "input slot";
          if (res) {
            if (wstamp[in[e]] == pid) return "window slot read and written in one phase";
            rstamp[in[e]] = pid;
          }
        }
        for (int32_t q = 0; q < D.ngl && !res; ++q)
          if (gl[q] < 0 || gl[q] >= n + ph.state_len) return "gathered slot";
      }
      if (res && (PH.flags & SWP_END)) ++pid;
    }
  }
  if (run_left != 0) return "run not closed";
  return "";
}

}  // namespace hb

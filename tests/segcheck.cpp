// Host-side checks of the sweep-program segmentation (test helper; built by
// tests/test_segmentation.py with g++ against the library's host code).
//
// For strip, arc, leaf-LU and polyline factors it verifies, for every sweep program and
// several thresholds / residency budgets:
//   * the segments cover the phases in order, without gaps or overlaps;
//   * a grid segment is exactly one phase with >= grid_min ops (or wide operands);
//   * a single-CTA run without st_cross produces every butterfly-state entry it
//     reads and nothing it writes is read by a later segment;
//   * a run cut for residency fits the budget unless it is a single atom;
//   * the flattened ops' staging areas tile each phase's staging size;
//   * executing the flattened records the way the sweep kernel reads them
//     (run_flat) gives the host interpreter's sweep, for all four programs.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "hb_internal.h"

using namespace hb;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { ++fails; if (fails < 20) { std::printf("FAIL: " __VA_ARGS__); std::printf("\n"); } } } while (0)

static void outputs(const FlatOp& f, int& n0, int& n1) {
  n0 = (f.kind == FK_GATHER) ? f.k0 : (f.kind == FK_SCATTER) ? ((f.flags & FF_TWO) ? f.split : f.c0)
     : (f.kind == FK_MIDDLE) ? ((f.flags & FF_ADJ) ? f.c0 : f.k0) : f.c0;
  n1 = (f.kind == FK_GATHER && (f.flags & FF_TWO)) ? f.k1 : (f.kind == FK_SCATTER && (f.flags & FF_TWO)) ? f.c0 - f.split : 0;
}

// Execute a flattened sweep program record by record (FP64, one right-hand side),
// reading every field the way the sweep kernel does: a gather indexes the
// concatenation of its two operand segments; a scatter forms each candidate
// row from one or two blocks and writes (or, with FF_SUB, subtracts) it into
// out0 below `split` and out1 above; a middle op multiplies by S (conjugate
// transposed with FF_ADJ); a leaf op multiplies by its packed triangle.
static void run_flat(const PackedHost& ph, const FlatProgram& fp, int which, std::vector<cplx>& vec) {
  std::vector<cplx> st((size_t)ph.state_len + 1, cplx(0.0));
  for (const FlatOp& f : fp.ops) {
    if (f.kind == FK_LEAF) {
      const int64_t s = f.c0;
      const cplx* T = ph.sl[which].data() + f.moff;
      cplx* v = vec.data() + f.src0;
      std::vector<cplx> y((size_t)s, cplx(0.0));
      for (int64_t r = 0; r < s; ++r) {
        if (f.flags & FF_UPPER) for (int64_t c = r; c < s; ++c) y[(size_t)r] += T[tri_off_upper(r, c)] * v[c];
        else for (int64_t c = 0; c <= r; ++c) y[(size_t)r] += T[tri_off_lower(s, r, c)] * v[c];
      }
      std::copy(y.begin(), y.end(), v);
      continue;
    }
    const cplx* s0 = ((f.flags & FF_SRC_VEC) ? vec.data() : st.data()) + f.src0;
    std::vector<cplx> cand(s0, s0 + f.n_s0);
    if (f.n_s1 > 0) cand.insert(cand.end(), st.data() + f.src1, st.data() + f.src1 + f.n_s1);
    const cplx* M0 = ph.fpool.data() + f.moff;
    const cplx* M1 = M0 + f.m1;
    const int16_t* I0 = f.ioff >= 0 ? ph.ipool.data() + f.ioff : nullptr;
    const int16_t* I1 = I0 ? I0 + f.i1 : nullptr;
    const bool cj = (f.flags & FF_CONJ) != 0, two = (f.flags & FF_TWO) != 0;
    cplx* out0 = ((f.flags & FF_OUT_VEC) ? vec.data() : st.data()) + f.out0;
    cplx* out1 = st.data() + f.out1;
    if (f.kind == FK_GATHER) {
      auto gather = [&](const cplx* M, const int16_t* I, int k, int c, cplx* out) {
        const int nr = c - k;
        for (int i = 0; i < k; ++i) {
          cplx acc = cand[(size_t)I[i]];
          for (int j = 0; j < nr; ++j)
            acc += (cj ? std::conj(M[(int64_t)i * nr + j]) : M[(int64_t)j * k + i]) * cand[(size_t)I[k + j]];
          out[i] = acc;
        }
      };
      gather(M0, I0, f.k0, f.c0, out0);
      if (two) gather(M1, I1, f.k1, f.c1, out1);
    } else if (f.kind == FK_SCATTER) {
      auto rowc = [&](const cplx* M, const int16_t* I, int k, int c, const cplx* y, int r) {
        const int code = I[c + r];
        if (code >= 0) return y[code];
        const int j = -1 - code, nr = c - k;
        cplx acc = 0.0;
        for (int i = 0; i < k; ++i) acc += (cj ? std::conj(M[(int64_t)j * k + i]) : M[(int64_t)i * nr + j]) * y[i];
        return acc;
      };
      for (int r = 0; r < f.c0; ++r) {
        cplx acc = rowc(M0, I0, f.k0, f.c0, cand.data(), r);
        if (two) acc += rowc(M1, I1, f.k1, f.c1, cand.data() + f.n_s0, r);
        cplx* d = (!two || r < f.split) ? out0 + r : out1 + (r - f.split);
        if (f.flags & FF_SUB) *d -= acc; else *d = acc;
      }
    } else {
      const bool adj = (f.flags & FF_ADJ) != 0;
      const int kr = f.k0, kc = f.c0, nin = adj ? kr : kc, nout = adj ? kc : kr;
      for (int o = 0; o < nout; ++o) {
        cplx acc = 0.0;
        for (int i = 0; i < nin; ++i)
          acc += (adj ? std::conj(M0[(int64_t)o * kr + i]) : M0[(int64_t)i * kr + o]) * cand[(size_t)i];
        out0[o] = acc;
      }
    }
  }
}

static void check_flat_execution(const PackedHost& ph, const HostFactor& hf, int which, const FlatProgram& fp) {
  std::vector<cplx> b((size_t)ph.n);
  for (int64_t i = 0; i < ph.n; ++i) b[(size_t)i] = cplx(std::sin(0.37 * i + which), std::cos(1.13 * i));
  std::vector<cplx> ref = b, got = b;
  host_sweep(ph, hf, which, ref.data());
  run_flat(ph, fp, which, got);
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < ph.n; ++i) { num += std::norm(got[(size_t)i] - ref[(size_t)i]); den += std::norm(ref[(size_t)i]); }
  CHECK(std::sqrt(num / den) <= 1e-13, "flat execution of sweep %d differs: %.3e", which, std::sqrt(num / den));
}

static void check_program(const PackedHost& ph, const HostFactor& hf, int which) {
  const std::vector<DPhase>& prog = which == 0 ? ph.prog_lower : which == 1 ? ph.prog_upper
                                  : which == 2 ? ph.prog_lower_adj : ph.prog_upper_adj;
  FlatProgram fp = flatten_program(ph, prog, which);
  CHECK(fp.ok, "flatten not ok");
  check_flat_execution(ph, hf, which, fp);
  // staging offsets tile each phase
  for (size_t p = 0; p < prog.size(); ++p) {
    int32_t off = 0;
    for (int32_t o = fp.base[p]; o < fp.base[p + 1]; ++o) {
      CHECK(fp.ops[o].soff == off, "soff mismatch phase %zu", p);
      off += flat_stage_bytes32(fp.ops[o]);
    }
    CHECK(fp.pbytes[p] == off, "pbytes mismatch phase %zu", p);
  }
  for (int gm : {1, 8, 32, 1 << 30})
    for (int64_t bud : {(int64_t)0, (int64_t)3584, (int64_t)7168}) {
      std::vector<DSeg> segs = segment_program(prog, fp, gm, bud);
      int next = 0;
      std::vector<int32_t> writer((size_t)ph.state_len + 1, -1);
      for (size_t si = 0; si < segs.size(); ++si) {
        const DSeg& sg = segs[si];
        CHECK(sg.first == next && sg.count >= 1, "coverage which %d gm %d seg %zu", which, gm, si);
        next = sg.first + sg.count;
        if (sg.grid) {
          const DPhase& P = prog[sg.first];
          CHECK(sg.count == 1 && P.kind != PH_LEAF && (P.count >= gm || P.vmax > 128), "grid seg rule %zu", si);
        } else if (bud > 0 && !sg.st_cross && sg.count > 1) {
          // a multi-atom run cut for residency fits the budget
          const int64_t foot = (int64_t)(sg.row_hi - sg.row_lo) + (sg.st_hi - sg.st_lo);
          bool multi_atom = false;
          for (int p = sg.first + 1; p < sg.first + sg.count; ++p)
            if (prog[p].kind == PH_LEAF || prog[p].kind == PH_ENTER) multi_atom = true;
          if (multi_atom) CHECK(foot <= bud, "budget which %d gm %d seg %zu foot %lld", which, gm, si, (long long)foot);
        }
        // state produced / consumed inside non-crossing runs
        for (int32_t o = fp.base[sg.first]; o < fp.base[sg.first + sg.count]; ++o) {
          const FlatOp& f = fp.ops[o];
          if (f.kind == FK_LEAF) continue;
          auto rd = [&](int32_t a, int32_t n) {
            for (int32_t e = a; e < a + n; ++e) {
              const int32_t w = writer[(size_t)e];
              if (!sg.grid && !sg.st_cross) CHECK(w == (int32_t)si, "run %zu reads state %d written by %d", si, e, w);
              if (w >= 0 && w != (int32_t)si && !segs[(size_t)w].grid)
                CHECK(segs[(size_t)w].st_cross, "run %d's state read later but not flagged", w);
            }
          };
          if (!(f.flags & FF_SRC_VEC)) rd(f.src0, f.n_s0);
          if (f.n_s1 > 0) rd(f.src1, f.n_s1);
          int n0, n1;
          outputs(f, n0, n1);
          if (!(f.flags & FF_OUT_VEC)) for (int32_t e = f.out0; e < f.out0 + n0; ++e) writer[(size_t)e] = (int32_t)si;
          for (int32_t e = f.out1; e < f.out1 + n1; ++e) writer[(size_t)e] = (int32_t)si;
        }
      }
      CHECK(next == (int)prog.size(), "coverage end which %d gm %d", which, gm);
    }
}

int main() {
  struct Case { int kind; double p[4]; int np; int64_t n; int64_t leaf; int options; };
  const Case cases[] = {
    {HB_STRIP, {0, 0, 204.8, 0}, 4, 4096, 64, 0},
    {HB_ARC, {2086.075670094090545 / 16.0, 0.0, M_PI, 0}, 3, 16384, 64, 0},
    {HB_STRIP, {0, 0, 51.2, 0}, 4, 1024, 32, 0},
    {HB_STRIP, {0, 0, 51.2, 0}, 4, 1024, 32, HB_OPT_LEAF_LU},
    {HB_POLYLINE, {0, 0, 0, 0}, 0, 2048, 64, 0},   // two wavy curves from explicit nodes
  };
  for (const Case& c : cases) {
    Geometry g;
    if (c.kind == HB_POLYLINE) {
      const int64_t per = c.n / 2;
      std::vector<double> xy;
      for (int curve = 0; curve < 2; ++curve)
        for (int64_t i = 0; i <= per; ++i) {
          const double t = (double)i / per;
          xy.push_back(51.2 * t);
          xy.push_back(curve == 0 ? 1.5 * std::sin(6 * M_PI * t) : 6.0 + 0.8 * std::cos(4 * M_PI * t));
        }
      const int64_t starts[2] = {0, per + 1};
      if (build_geometry_polyline(xy.data(), starts, 2, 2 * (per + 1), g)) { std::printf("FAIL: polyline\n"); return 1; }
    } else if (build_geometry(c.kind, c.p, c.np, c.n, g)) {
      std::printf("FAIL: geometry\n");
      return 1;
    }
    HostFactor hf;
    if (build_factor(g, 1.0, 376.730313668, 1.781072, c.leaf, 1e-6, 1, hf, c.options)) {
      std::printf("FAIL: factor\n");
      return 1;
    }
    PackedHost ph;
    pack_factor(hf, ph);
    CHECK(ph.sl_n == std::min<int64_t>(kSweepLeafMax, c.leaf << ph.depth) || ph.sl_n == c.leaf << ph.sl_t,
          "sweep leaf size");
    for (int w = 0; w < 4; ++w) check_program(ph, hf, w);
  }
  if (fails) { std::printf("%d failures\n", fails); return 1; }
  std::printf("OK\n");
  return 0;
}

// Host-side checks of the sweep-program segmentation (test helper; built by
// tests/test_segmentation.py with g++ against the library's host code).
//
// For a strip and an arc factor it verifies, for every sweep program and
// several thresholds / residency budgets:
//   * the segments cover the phases in order, without gaps or overlaps;
//   * a grid segment is exactly one phase with >= grid_min ops (or wide operands);
//   * a single-CTA run without st_cross produces every butterfly-state entry it
//     reads and nothing it writes is read by a later segment;
//   * a run cut for residency fits the budget unless it is a single atom;
//   * the flattened ops' staging areas tile each phase's staging size.
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

static void check_program(const PackedHost& ph, int which) {
  const std::vector<DPhase>& prog = which == 0 ? ph.prog_lower : which == 1 ? ph.prog_upper
                                  : which == 2 ? ph.prog_lower_adj : ph.prog_upper_adj;
  FlatProgram fp = flatten_program(ph, prog, which);
  CHECK(fp.ok, "flatten not ok");
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
  struct Case { int kind; double p[4]; int np; int64_t n; int64_t leaf; };
  const Case cases[] = {
    {HB_STRIP, {0, 0, 204.8, 0}, 4, 4096, 64},
    {HB_ARC, {2086.075670094090545 / 16.0, 0.0, M_PI, 0}, 3, 16384, 64},
    {HB_STRIP, {0, 0, 51.2, 0}, 4, 1024, 32},
  };
  for (const Case& c : cases) {
    Geometry g;
    if (build_geometry(c.kind, c.p, c.np, c.n, g)) { std::printf("FAIL: geometry\n"); return 1; }
    HostFactor hf;
    if (build_factor(g, 1.0, 376.730313668, 1.781072, c.leaf, 1e-6, 1, hf)) { std::printf("FAIL: factor\n"); return 1; }
    PackedHost ph;
    pack_factor(hf, ph);
    CHECK(ph.sl_n == std::min<int64_t>(kSweepLeafMax, c.leaf << ph.depth) || ph.sl_n == c.leaf << ph.sl_t,
          "sweep leaf size");
    for (int w = 0; w < 4; ++w) check_program(ph, w);
  }
  if (fails) { std::printf("%d failures\n", fails); return 1; }
  std::printf("OK\n");
  return 0;
}

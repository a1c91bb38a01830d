// Structural check of the column-partitioned sweep schedules (test helper; built by
// tests/test_sweep_sched.py with g++ against the library's host code).
//
// The schedules of an arc factor (all four sweeps, the full and the smallest resident
// window) pass the check as built.  Then one defect at a time is planted in a copy of a
// schedule, and the check must name it: a window slot written twice within one resident
// phase, a window slot written and read within one phase (the chain warps run a phase's
// batches concurrently, so either would race), an input outside the window, a group off
// its 16-byte alignment, a resident run whose last group lacks its ENDRUN flag, and a
// global row that adds in place.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hb_internal.h"

using namespace hb;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { ++fails; if (fails < 20) { std::printf("FAIL: " __VA_ARGS__); std::printf("\n"); } } } while (0)

namespace {

SwGroupHdr header(const SwSched& S, size_t gi) {
  SwGroupHdr H;
  std::memcpy(&H, S.image.data() + S.groups[gi].img, sizeof(H));
  return H;
}

// Locate the first batch (group index, byte offset of its descriptor) of a phase part
// that satisfies `want(H, PH, D)`; returns false if there is none.
template <class Want>
bool find_batch(const SwSched& S, Want want, size_t& gi_out, int64_t& desc_off) {
  for (size_t gi = 0; gi < S.groups.size(); ++gi) {
    const uint8_t* gb = S.image.data() + S.groups[gi].img;
    const SwGroupHdr H = header(S, gi);
    int64_t di = 0;
    for (int k = 0; k < H.nph; ++k) {
      SwPhase PH;
      std::memcpy(&PH, gb + 32 + 8 * k, sizeof(PH));
      for (int b = 0; b < PH.nb; ++b, ++di) {
        SwDesc D;
        std::memcpy(&D, gb + H.off_desc + 40 * di, sizeof(D));
        if (want(H, PH, D)) {
          gi_out = gi;
          desc_off = H.off_desc + 40 * di;
          return true;
        }
      }
    }
  }
  return false;
}

SwDesc desc_at(const SwSched& S, size_t gi, int64_t off) {
  SwDesc D;
  std::memcpy(&D, S.image.data() + S.groups[gi].img + off, sizeof(D));
  return D;
}

int32_t* outs(SwSched& S, size_t gi, const SwDesc& D) {
  return reinterpret_cast<int32_t*>(S.image.data() + S.groups[gi].img + D.off);
}
int16_t* ins(SwSched& S, size_t gi, const SwDesc& D) {
  return reinterpret_cast<int16_t*>(S.image.data() + S.groups[gi].img + D.off + D.off_in);
}

void expect(const PackedHost& ph, const SwSched& S, const char* reason, const char* what) {
  const std::string got = check_sweep_sched(ph, S);
  CHECK(got == reason, "%s: check said '%s', expected '%s'", what, got.c_str(), reason);
}

}  // namespace

int main() {
  Geometry g;
  const double prm[3] = {4096 / 40.0 / M_PI, 0.0, M_PI};
  if (build_geometry(HB_ARC, prm, 3, 4096, g)) { std::printf("FAIL: geometry\n"); return 1; }
  HostFactor hf;
  if (build_factor(g, 1.0, 376.730313668, 1.781072, 64, 1e-6, 1, hf, 0)) { std::printf("FAIL: factor\n"); return 1; }
  PackedHost ph;
  pack_factor(hf, ph);

  for (int which = 0; which < 4; ++which)
    for (int ws : {kSwWinSlots, 512}) {
      SwSched S;
      build_sweep_sched(ph, which, 8, ws, S);
      CHECK(S.ok, "schedule %d / %d not built: %s", which, ws, S.why);
      const std::string got = check_sweep_sched(ph, S);
      CHECK(got.empty(), "schedule %d / %d rejected: %s", which, ws, got.c_str());
    }

  SwSched base;
  build_sweep_sched(ph, 0, 8, kSwWinSlots, base);
  const auto res_rows = [](const SwGroupHdr& H, const SwPhase& PH, const SwDesc& D) {
    return (H.flags & SWG_RES) && !(PH.flags & SWP_TRI) && D.nrows >= 2 && D.nent >= 1;
  };
  size_t gi = 0;
  int64_t off = 0;
  CHECK(find_batch(base, res_rows, gi, off), "no resident batch with two rows");

  {   // two rows of one resident batch write the same window slot
    SwSched S = base;
    const SwDesc D = desc_at(S, gi, off);
    int32_t* o = outs(S, gi, D);
    o[1] = (o[0] & ~kSwAcc) | (o[1] & kSwAcc);
    expect(ph, S, "window slot written twice in one phase", "duplicate output");
  }
  {   // a resident batch reads a slot that its own phase writes
    SwSched S = base;
    const SwDesc D = desc_at(S, gi, off);
    ins(S, gi, D)[0] = (int16_t)(outs(S, gi, D)[0] & ~kSwAcc);
    expect(ph, S, "window slot read and written in one phase", "read of a slot written in the phase");
  }
  {   // an input outside the window
    SwSched S = base;
    const SwDesc D = desc_at(S, gi, off);
    ins(S, gi, D)[0] = (int16_t)S.win_slots;
    expect(ph, S, "input slot", "input outside the window");
  }
  {   // a group off its 16-byte alignment
    SwSched S = base;
    S.groups[1].img += 8;
    expect(ph, S, "group not 16-byte aligned", "misaligned group");
  }
  {   // the ENDRUN flag taken off a run's last group
    SwSched S = base;
    size_t last = S.groups.size();
    for (size_t k = 0; k < S.groups.size(); ++k)
      if (header(S, k).flags & SWG_ENDRUN) { last = k; break; }
    CHECK(last < S.groups.size(), "no ENDRUN group");
    if (last < S.groups.size()) {
      SwGroupHdr H = header(S, last);
      H.flags &= ~SWG_ENDRUN;
      std::memcpy(S.image.data() + S.groups[last].img, &H, sizeof(H));
      expect(ph, S, "ENDRUN not on the run's last group", "missing ENDRUN");
    }
  }
  {   // a global row that adds in place (the smallest window leaves global phases at this size)
    SwSched S;
    build_sweep_sched(ph, 0, 8, 512, S);
    size_t gg = 0;
    int64_t go = 0;
    const auto glob = [](const SwGroupHdr& H, const SwPhase&, const SwDesc& D) {
      return !(H.flags & SWG_RES) && D.nrows >= 1;
    };
    CHECK(find_batch(S, glob, gg, go), "no global batch");
    const SwDesc D = desc_at(S, gg, go);
    outs(S, gg, D)[0] |= kSwAcc;
    expect(ph, S, "global row that adds in place", "global accumulate");
  }
  if (fails) { std::printf("%d failures\n", fails); return 1; }
  std::printf("OK\n");
  return 0;
}

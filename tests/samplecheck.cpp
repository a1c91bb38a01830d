// Host-side check of the ID sampling (test helper; built by tests/test_segmentation.py
// with g++).  It includes the library's host source to reach its internal sampling
// policies and verifies that the k-d tree path (TreePool) picks exactly the samples
// and probe rows of the full scan (ListPool) over the same pool: the nearest half
// (smallest squared distance to the candidates' reference points, ties by position),
// then the Chebyshev and uniform picks, for contiguous and listed pools, several
// sample sizes and seeds, and with a previous sample removed (the probe).
#include "../paper_1901_11371_gb300/csrc/hb_host.cpp"

#include <cstdio>

using namespace hb;

int main() {
  int fails = 0;
  // a curve that turns back on itself (near field between turns) plus a straight part
  Geometry g;
  const int64_t n = 20000;
  for (int64_t i = 0; i < n; ++i) {
    const double t = 0.002 * (double)i;
    g.cx.push_back(i < 12000 ? t * std::cos(t) : 20.0 + 0.01 * (double)(i - 12000));
    g.cy.push_back(i < 12000 ? t * std::sin(t) : 0.25 * std::floor((double)(i - 12000) / 400.0));
    g.w.push_back(0.01);
  }
  g.n = n;
  uint64_t st = 12345;
  for (int trial = 0; trial < 300; ++trial) {
    // pool: a contiguous range, or an increasing list of indices
    const bool range = trial % 3 == 0;
    const int64_t M = 1500 + (int64_t)(splitmix(st) % 6000);
    const int64_t lo = (int64_t)(splitmix(st) % (uint64_t)(n - M));
    std::vector<int64_t> list;
    if (range) {
      for (int64_t p = 0; p < M; ++p) list.push_back(lo + p);
    } else {
      for (int64_t i = 0; i < n && (int64_t)list.size() < M; ++i)
        if (splitmix(st) % 3 == 0) list.push_back(i);
    }
    PoolTree tree;
    if (range) tree.build(g, nullptr, lo, M);
    else tree.build(g, list.data(), 0, (int64_t)list.size());
    const ListPool lp{g, list};
    const TreePool tp{tree};
    // candidates: a short run of nearby indices (as an ID's candidate list)
    const int c = 4 + (int)(splitmix(st) % 60);
    const int64_t c0 = (int64_t)(splitmix(st) % (uint64_t)(n - c));
    std::vector<int64_t> cand;
    for (int i = 0; i < c; ++i) cand.push_back(c0 + i);
    const int s = sample_count(c) << (splitmix(st) % 4);
    const uint64_t seed = splitmix(st);
    std::vector<int64_t> p1, p2, r1, r2;
    lp.sample(cand, s, seed, p1);
    tp.sample(cand, s, seed, p2);
    if (p1 != p2) { ++fails; std::printf("FAIL: sample differs (trial %d, M %lld, s %d)\n", trial, (long long)M, s); }
    const int sp = (int)std::min<int64_t>((int64_t)lp.size() - (int64_t)p1.size(), 16 + c / 2);
    if (sp > 0) {
      lp.probe(cand, p1, sp, seed ^ 0xFEEDull, r1);
      tp.probe(cand, p1, sp, seed ^ 0xFEEDull, r2);
      if (r1 != r2) { ++fails; std::printf("FAIL: probe differs (trial %d)\n", trial); }
    }
    for (size_t i = 0; i < p1.size(); ++i)
      if (lp.at(p1[i]) != tp.at(p1[i])) { ++fails; std::printf("FAIL: index map (trial %d)\n", trial); break; }
  }
  if (fails) { std::printf("%d failures\n", fails); return 1; }
  std::printf("OK\n");
  return 0;
}

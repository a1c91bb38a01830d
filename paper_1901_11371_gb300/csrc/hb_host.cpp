// Host side of libhb: geometry (Sec. 3.1), EFIE entries, H-IDBF construction
// (Alg. 1 with the IDBF of Sec. 2 / Appendix, sampled linear-scaling IDs) and
// packing of the factors into the level-packed device image.
//
// Construction is not on the measured hot path; it runs on the host cores
// with OpenMP and is timed separately (hb_factor_stats.build_seconds).
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <climits>
#include <numeric>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "hb_internal.h"

namespace hb {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

// ---------------------------------------------------------------------------
// Geometry: equal-arc-length nodes on the exact curve, chord segments.
// ---------------------------------------------------------------------------
static void chords(const std::vector<double>& nx, const std::vector<double>& ny, Geometry& g, int64_t off) {
  int64_t cnt = (int64_t)nx.size() - 1;
  for (int64_t i = 0; i < cnt; ++i) {
    g.cx[off + i] = 0.5 * (nx[i] + nx[i + 1]);
    g.cy[off + i] = 0.5 * (ny[i] + ny[i + 1]);
    g.w[off + i] = std::hypot(nx[i + 1] - nx[i], ny[i + 1] - ny[i]);
  }
}

// s(theta) = (a/2) [theta sqrt(1 + theta^2) + asinh(theta)] for r = a theta.
static double spiral_s(double a, double t) { return 0.5 * a * (t * std::sqrt(1.0 + t * t) + std::asinh(t)); }

int build_geometry(int kind, const double* params, int nparams, int64_t n, Geometry& g) {
  if (n < 1 || params == nullptr) {
    set_error("hb_geometry: n_segments must be >= 1 and params non-null");
    return HB_EINVAL;
  }
  g.kind = kind;
  g.n = n;
  g.cx.assign(n, 0.0);
  g.cy.assign(n, 0.0);
  g.w.assign(n, 0.0);
  std::vector<double> nx(n + 1), ny(n + 1);
  if (kind == HB_STRIP) {
    if (nparams != 4) { set_error("STRIP needs 4 params"); return HB_EINVAL; }
    for (int64_t i = 0; i <= n; ++i) {
      double t = (double)i / (double)n;
      nx[i] = params[0] + (params[2] - params[0]) * t;
      ny[i] = params[1] + (params[3] - params[1]) * t;
    }
    chords(nx, ny, g, 0);
  } else if (kind == HB_SPIRAL) {
    if (nparams != 3 || params[0] <= 0 || params[2] <= params[1]) { set_error("SPIRAL needs (a>0, th0<th1)"); return HB_EINVAL; }
    double a = params[0], t0 = params[1], t1 = params[2];
    double s0 = spiral_s(a, t0), s1 = spiral_s(a, t1);
    for (int64_t i = 0; i <= n; ++i) {
      double target = s0 + (s1 - s0) * (double)i / (double)n;
      double th = t0 + (t1 - t0) * (double)i / (double)n;
      for (int it = 0; it < 100; ++it) {   // Newton on s(theta) = target, s' = a sqrt(1+theta^2)
        double step = (spiral_s(a, th) - target) / (a * std::sqrt(1.0 + th * th));
        th -= step;
        if (std::fabs(step) <= 1e-15 * std::max(1.0, std::fabs(t1))) break;
      }
      if (i == 0) th = t0;
      if (i == n) th = t1;
      nx[i] = a * th * std::cos(th);
      ny[i] = a * th * std::sin(th);
    }
    chords(nx, ny, g, 0);
  } else if (kind == HB_ARC) {
    if (nparams != 3 || params[0] <= 0) { set_error("ARC needs (R>0, phi0, phi1)"); return HB_EINVAL; }
    for (int64_t i = 0; i <= n; ++i) {
      double ph = params[1] + (params[2] - params[1]) * (double)i / (double)n;
      nx[i] = params[0] * std::cos(ph);
      ny[i] = params[0] * std::sin(ph);
    }
    chords(nx, ny, g, 0);
  } else if (kind == HB_PARALLEL_STRIPS) {
    if (nparams != 3) { set_error("PARALLEL_STRIPS needs 3 params"); return HB_EINVAL; }
    int64_t ns = (int64_t)std::llround(params[0]);
    if (ns < 1 || n % ns) { set_error("PARALLEL_STRIPS: n_strips must divide n_segments"); return HB_EINVAL; }
    int64_t per = n / ns;
    std::vector<double> sx(per + 1), sy(per + 1);
    for (int64_t s = 0; s < ns; ++s) {
      for (int64_t i = 0; i <= per; ++i) {
        sx[i] = params[1] * (double)i / (double)per;
        sy[i] = (double)s * params[2];
      }
      chords(sx, sy, g, s * per);
    }
  } else {
    set_error("hb_geometry: unknown kind %d", kind);
    return HB_EINVAL;
  }
  g.params.assign(params, params + nparams);
  return HB_OK;
}

int build_geometry_polyline(const double* xy, const int64_t* starts, int ncurves, int64_t nnodes, Geometry& g) {
  if (!xy || !starts || ncurves < 1 || nnodes < 2) {
    set_error("hb_geometry_polyline: null pointer, ncurves < 1 or nnodes < 2");
    return HB_EINVAL;
  }
  if (starts[0] != 0) { set_error("hb_geometry_polyline: curve_starts[0] must be 0"); return HB_EINVAL; }
  for (int c = 0; c < ncurves; ++c) {
    const int64_t e = c + 1 < ncurves ? starts[c + 1] : nnodes;
    if (e - starts[c] < 2 || e > nnodes) {
      set_error("hb_geometry_polyline: curve %d needs at least 2 nodes inside the node list", c);
      return HB_EINVAL;
    }
  }
  for (int64_t i = 0; i < 2 * nnodes; ++i)
    if (!std::isfinite(xy[i])) { set_error("hb_geometry_polyline: non-finite coordinate"); return HB_EINVAL; }
  const int64_t n = nnodes - ncurves;
  g.kind = HB_POLYLINE;
  g.n = n;
  g.params.clear();
  g.cx.assign(n, 0.0);
  g.cy.assign(n, 0.0);
  g.w.assign(n, 0.0);
  int64_t off = 0;
  for (int c = 0; c < ncurves; ++c) {
    const int64_t b = starts[c], e = c + 1 < ncurves ? starts[c + 1] : nnodes;
    std::vector<double> nx((size_t)(e - b)), ny((size_t)(e - b));
    for (int64_t i = b; i < e; ++i) { nx[(size_t)(i - b)] = xy[2 * i]; ny[(size_t)(i - b)] = xy[2 * i + 1]; }
    chords(nx, ny, g, off);
    off += e - b - 1;
  }
  for (int64_t i = 0; i < n; ++i)
    if (!(g.w[i] > 0.0)) { set_error("hb_geometry_polyline: segment %lld has zero length", (long long)i); return HB_EINVAL; }
  return HB_OK;
}

// ---------------------------------------------------------------------------
// EFIE entries (Sec. 3.1), rescaled by a.  H0^(2) = J0 - i Y0 from the C
// library's j0 / y0.
// ---------------------------------------------------------------------------
struct Entries {
  const Geometry* g;
  double kappa, eta0, gamma, scale;
  std::vector<cplx> diag;

  void init(const Geometry& geo, double wavelength, double eta, double gam) {
    g = &geo;
    kappa = 2.0 * M_PI / wavelength;
    eta0 = eta;
    gamma = gam;
    diag.resize(geo.n);
    double mx = 0.0;
    for (int64_t i = 0; i < geo.n; ++i) {
      double w = geo.w[i];
      double c = kappa * eta0 * w / 4.0;
      diag[i] = cplx(c, -c * (2.0 / M_PI) * std::log(gamma * kappa * w / (4.0 * M_E)));
      mx = std::max(mx, std::abs(diag[i]));
    }
    scale = 1.0 / mx;
    for (auto& d : diag) d *= scale;
  }
  inline cplx operator()(int64_t i, int64_t j) const {
    if (i == j) return diag[i];
    double dx = g->cx[i] - g->cx[j], dy = g->cy[i] - g->cy[j];
    double x = kappa * std::sqrt(dx * dx + dy * dy);
    double c = scale * kappa * eta0 * g->w[j] * 0.25;
    return cplx(c * ::j0(x), -c * ::y0(x));
  }
};

// ---------------------------------------------------------------------------
// Interpolative decomposition: Householder QR with column pivoting of an
// s x c column-major matrix, truncated at the first k with |R_kk| <= tol |R_00|
// (reading of Eq. (req)); T = R11^{-1} R12.
// ---------------------------------------------------------------------------
static void column_id(std::vector<cplx>& M, int s, int c, double tol, IdBlock& out) {
  std::vector<int> perm(c);
  std::iota(perm.begin(), perm.end(), 0);
  int steps = std::min(s, c);
  int k = steps;
  double r00 = 0.0;
  std::vector<cplx> v(s);
  for (int j = 0; j < steps; ++j) {
    // pivot: largest trailing column norm, lowest index on ties
    int piv = j;
    double best = -1.0;
    for (int l = j; l < c; ++l) {
      double nr = 0.0;
      const cplx* col = &M[(size_t)l * s];
      for (int r = j; r < s; ++r) nr += std::norm(col[r]);
      if (nr > best) { best = nr; piv = l; }
    }
    if (piv != j) {
      std::swap_ranges(M.begin() + (size_t)j * s, M.begin() + (size_t)(j + 1) * s, M.begin() + (size_t)piv * s);
      std::swap(perm[j], perm[piv]);
    }
    double alpha = std::sqrt(std::max(best, 0.0));
    if (j == 0) r00 = alpha;
    if (alpha == 0.0 || (j > 0 && alpha <= tol * r00)) { k = j; break; }
    cplx* colj = &M[(size_t)j * s];
    cplx x0 = colj[j];
    cplx phase = (std::abs(x0) > 0) ? x0 / std::abs(x0) : cplx(1.0, 0.0);
    for (int r = j; r < s; ++r) v[r] = colj[r];
    v[j] += phase * alpha;
    double vn = 0.0;
    for (int r = j; r < s; ++r) vn += std::norm(v[r]);
    vn = std::sqrt(vn);
    for (int r = j; r < s; ++r) v[r] /= vn;
    for (int l = j; l < c; ++l) {
      cplx* col = &M[(size_t)l * s];
      cplx d = 0.0;
      for (int r = j; r < s; ++r) d += std::conj(v[r]) * col[r];
      d *= 2.0;
      for (int r = j; r < s; ++r) col[r] -= v[r] * d;
    }
  }
  k = std::max(k, 1);
  k = std::min(k, c);
  out.k = k;
  out.c = c;
  out.q.assign(perm.begin(), perm.begin() + k);
  out.p.assign(perm.begin() + k, perm.end());
  int nr = c - k;
  out.t.assign((size_t)k * nr, cplx(0.0));
  // back substitution R11 T = R12 (R stored in the top k rows of M)
  for (int j = 0; j < nr; ++j) {
    for (int i = k - 1; i >= 0; --i) {
      cplx acc = M[(size_t)(k + j) * s + i];
      for (int l = i + 1; l < k; ++l) acc -= M[(size_t)l * s + i] * out.t[(size_t)l * nr + j];
      out.t[(size_t)i * nr + j] = acc / M[(size_t)i * s + i];
    }
  }
}

// ---------------------------------------------------------------------------
// Seeded sampling for the IDs (Mock-Chebyshev grid + uniform fill + near field).
// ---------------------------------------------------------------------------
static inline uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline int sample_count(int c) { return 2 * c + 16; }

// Reference points of a candidate list: up to 8 evenly spaced candidates.
static int near_refs(const std::vector<int64_t>& cand, int64_t* refs) {
  const int nc = (int)cand.size();
  const int nref = std::min(nc, 8);
  for (int r = 0; r < nref; ++r) refs[r] = cand[(int64_t)r * (nc - 1) / std::max(1, nref - 1)];
  return nref;
}

// Squared distance of (px, py) to the nearest reference point.
static inline double near_d2(const Geometry& g, double px, double py, const int64_t* refs, int nref) {
  double dmin = 1e300;
  for (int r = 0; r < nref; ++r) {
    const double dx = px - g.cx[refs[r]], dy = py - g.cy[refs[r]];
    dmin = std::min(dmin, dx * dx + dy * dy);
  }
  return dmin;
}

// Chebyshev-spaced then uniform picks among M positions, skipping those in `used`,
// until `out` holds s entries (the fill shared by both sampling paths).
template <class Used>
static void fill_picks(int64_t M, int s, int nn, uint64_t seed, Used& used, std::vector<int64_t>& out) {
  const int nrest = s - nn;
  const int ncheb = nrest / 2;
  for (int i = 0; i < ncheb; ++i) {
    double x = 0.5 * (1.0 - std::cos(M_PI * (2.0 * i + 1.0) / (2.0 * ncheb)));
    int64_t idx = std::min<int64_t>(M - 1, (int64_t)std::llround(x * (double)(M - 1)));
    if (used.insert(idx)) out.push_back(idx);
  }
  uint64_t st = seed;
  while ((int)out.size() < s) {
    int64_t idx = (int64_t)(splitmix(st) % (uint64_t)M);
    if (used.insert(idx)) out.push_back(idx);
  }
}

struct FlagSet {   // dense membership over [0, M)
  std::vector<char> f;
  explicit FlagSet(int64_t M) : f((size_t)M, 0) {}
  bool insert(int64_t i) { if (f[(size_t)i]) return false; f[(size_t)i] = 1; return true; }
};
struct SmallSet {  // sparse membership (a few thousand entries at most)
  std::vector<int64_t> v;
  bool insert(int64_t i) {
    auto it = std::lower_bound(v.begin(), v.end(), i);
    if (it != v.end() && *it == i) return false;
    v.insert(it, i);
    return true;
  }
};

// Sample positions of `pool` for an ID over the candidate points `cand`: half
// of the sample is the pool entries geometrically nearest to the candidates
// (the near field across block boundaries and between adjacent turns, which a
// uniform or Chebyshev sample of a long pool can miss; ties by position), the
// rest a Mock-Chebyshev + uniform sample of the remaining entries.
static void sample_near(const Geometry& g, const std::vector<int64_t>& pool, const std::vector<int64_t>& cand,
                        int s, uint64_t seed, std::vector<int64_t>& out) {
  const int64_t M = (int64_t)pool.size();
  if (M <= s) {
    out.resize(M);
    std::iota(out.begin(), out.end(), 0);
    return;
  }
  int64_t refs[8];
  const int nref = near_refs(cand, refs);
  std::vector<std::pair<double, int64_t>> dist(M);
  for (int64_t e = 0; e < M; ++e) dist[e] = {near_d2(g, g.cx[pool[e]], g.cy[pool[e]], refs, nref), e};
  const int nn = s / 2;
  std::nth_element(dist.begin(), dist.begin() + nn, dist.end());
  FlagSet used(M);
  out.clear();
  for (int i = 0; i < nn; ++i) { used.insert(dist[i].second); out.push_back(dist[i].second); }
  fill_picks(M, s, nn, seed, used, out);
  std::sort(out.begin(), out.end());
}

// k-d tree over the segment centres of a pool: a contiguous range [lo, lo + M)
// (idx null) or an index list idx[0..M).  The pools of a butterfly stage are
// shared by many of its IDs (the first row stage samples the whole column
// range, the first column stage all row skeletons); nearest() returns the same
// entries as the full scan of sample_near (the nn smallest (squared distance,
// position) pairs) in O(nn log M) instead of O(M) per ID.
struct PoolTree {
  struct Node { double x0, y0, x1, y1; int32_t begin, end, left, right; };
  const Geometry* g = nullptr;
  const int64_t* idx = nullptr;
  int64_t lo = 0, M = 0;
  std::vector<int32_t> pts;   // pool positions in tree order
  std::vector<Node> nodes;
  int64_t global(int64_t p) const { return idx ? idx[p] : lo + p; }

  int32_t build_node(int32_t b, int32_t e) {
    Node nd{1e300, 1e300, -1e300, -1e300, b, e, -1, -1};
    for (int32_t i = b; i < e; ++i) {
      const double x = g->cx[global(pts[i])], y = g->cy[global(pts[i])];
      nd.x0 = std::min(nd.x0, x); nd.x1 = std::max(nd.x1, x);
      nd.y0 = std::min(nd.y0, y); nd.y1 = std::max(nd.y1, y);
    }
    const int32_t id = (int32_t)nodes.size();
    nodes.push_back(nd);
    if (e - b > 16) {
      const bool xs = (nd.x1 - nd.x0) >= (nd.y1 - nd.y0);
      const int32_t mid = b + (e - b) / 2;
      std::nth_element(pts.begin() + b, pts.begin() + mid, pts.begin() + e, [&](int32_t u, int32_t v) {
        const int64_t gu = global(u), gv = global(v);
        const double a = xs ? g->cx[gu] : g->cy[gu], c = xs ? g->cx[gv] : g->cy[gv];
        return a < c || (a == c && u < v);
      });
      const int32_t l = build_node(b, mid);
      const int32_t r = build_node(mid, e);
      nodes[id].left = l;
      nodes[id].right = r;
    }
    return id;
  }
  void build(const Geometry& geo, const int64_t* idx_, int64_t lo_, int64_t M_) {
    g = &geo; idx = idx_; lo = lo_; M = M_;
    pts.resize((size_t)M);
    std::iota(pts.begin(), pts.end(), 0);
    nodes.clear();
    nodes.reserve((size_t)(M / 8 + 2));
    build_node(0, (int32_t)M);
  }
  // the nn pool positions not in `skip` (sorted) with the smallest (near_d2, position)
  void nearest(const int64_t* refs, int nref, int nn, const std::vector<int64_t>& skip,
               std::vector<int64_t>& out) const {
    using Cand = std::pair<double, int64_t>;
    std::vector<Cand> best;   // max-heap of the nn best so far
    best.reserve((size_t)nn + 1);
    auto box_d2 = [&](const Node& nd) {
      double m = 1e300;
      for (int r = 0; r < nref; ++r) {
        const double px = g->cx[refs[r]], py = g->cy[refs[r]];
        const double dx = std::max(0.0, std::max(nd.x0 - px, px - nd.x1));
        const double dy = std::max(0.0, std::max(nd.y0 - py, py - nd.y1));
        m = std::min(m, dx * dx + dy * dy);
      }
      return m * (1.0 - 1e-12);   // a lower bound also under rounding
    };
    using QE = std::pair<double, int32_t>;
    std::vector<QE> queue;      // min-heap of nodes by lower bound
    auto qcmp = [](const QE& a, const QE& b) { return a.first > b.first; };
    queue.push_back({box_d2(nodes[0]), 0});
    while (!queue.empty()) {
      std::pop_heap(queue.begin(), queue.end(), qcmp);
      const QE top = queue.back();
      queue.pop_back();
      if ((int)best.size() == nn && top.first > best.front().first) break;
      const Node& nd = nodes[(size_t)top.second];
      if (nd.left < 0) {
        for (int32_t i = nd.begin; i < nd.end; ++i) {
          const int64_t p = pts[(size_t)i];
          if (!skip.empty() && std::binary_search(skip.begin(), skip.end(), p)) continue;
          const int64_t gp = global(p);
          const Cand cnd{near_d2(*g, g->cx[gp], g->cy[gp], refs, nref), p};
          if ((int)best.size() < nn) {
            best.push_back(cnd);
            std::push_heap(best.begin(), best.end());
          } else if (cnd < best.front()) {
            std::pop_heap(best.begin(), best.end());
            best.back() = cnd;
            std::push_heap(best.begin(), best.end());
          }
        }
      } else {
        for (int32_t ch : {nd.left, nd.right}) {
          queue.push_back({box_d2(nodes[(size_t)ch]), ch});
          std::push_heap(queue.begin(), queue.end(), qcmp);
        }
      }
    }
    out.clear();
    for (const Cand& c : best) out.push_back(c.second);
  }
};

// Explicit pool of indices: the full-scan sampling above.
struct ListPool {
  const Geometry& g;
  const std::vector<int64_t>& idx;
  int64_t size() const { return (int64_t)idx.size(); }
  int64_t at(int64_t p) const { return idx[(size_t)p]; }
  void sample(const std::vector<int64_t>& cand, int s, uint64_t seed, std::vector<int64_t>& pos) const {
    sample_near(g, idx, cand, s, seed, pos);
  }
  // probe rows: a sample of the unsampled entries (global indices, in pool order)
  void probe(const std::vector<int64_t>& cand, const std::vector<int64_t>& pos, int s, uint64_t seed,
             std::vector<int64_t>& rows) const {
    const int64_t M = size();
    std::vector<char> used((size_t)M, 0);
    for (int64_t e : pos) used[(size_t)e] = 1;
    std::vector<int64_t> rest;
    rest.reserve((size_t)(M - (int64_t)pos.size()));
    for (int64_t e = 0; e < M; ++e)
      if (!used[(size_t)e]) rest.push_back(idx[(size_t)e]);
    std::vector<int64_t> ppos;
    sample_near(g, rest, cand, s, seed, ppos);
    rows.clear();
    for (int64_t r : ppos) rows.push_back(rest[(size_t)r]);
  }
};

// Pool with its k-d tree: the same samples as ListPool over the same entries,
// without touching all M of them per ID.
struct TreePool {
  const PoolTree& tree;
  int64_t size() const { return tree.M; }
  int64_t at(int64_t p) const { return tree.global(p); }
  // sample_near over the pool with the (sorted) positions `skip` removed; the
  // result counts positions over the remaining entries, as sample_near would
  void sample_skip(const std::vector<int64_t>& cand, int s, uint64_t seed, const std::vector<int64_t>& skip,
                   std::vector<int64_t>& out) const {
    const int64_t M = tree.M - (int64_t)skip.size();
    out.clear();
    if (M <= s) {
      out.resize(M);
      std::iota(out.begin(), out.end(), 0);
      return;
    }
    int64_t refs[8];
    const int nref = near_refs(cand, refs);
    const int nn = s / 2;
    std::vector<int64_t> near;
    tree.nearest(refs, nref, nn, skip, near);
    SmallSet used;
    for (int64_t p : near) {   // pool position -> position among the remaining entries
      const int64_t r = p - (int64_t)(std::lower_bound(skip.begin(), skip.end(), p) - skip.begin());
      used.insert(r);
      out.push_back(r);
    }
    fill_picks(M, s, nn, seed, used, out);
    std::sort(out.begin(), out.end());
  }
  void sample(const std::vector<int64_t>& cand, int s, uint64_t seed, std::vector<int64_t>& pos) const {
    static const std::vector<int64_t> none;
    sample_skip(cand, s, seed, none, pos);
  }
  void probe(const std::vector<int64_t>& cand, const std::vector<int64_t>& pos, int s, uint64_t seed,
             std::vector<int64_t>& rows) const {
    std::vector<int64_t> rpos;
    sample_skip(cand, s, seed, pos, rpos);
    // position r among the unsampled entries -> pool position (pos is sorted)
    rows.clear();
    size_t k = 0;
    for (int64_t r : rpos) {   // rpos is sorted: walk pos once
      int64_t q = r + (int64_t)k;
      while (k < pos.size() && pos[k] <= q) { ++k; ++q; }
      rows.push_back(tree.global(q));
    }
  }
};

// ---------------------------------------------------------------------------
// Adaptive sampled ID.  cand: the c candidate indices; pool: the other
// dimension's indices to sample (ListPool / TreePool); ent(pool index,
// candidate index) gives the entry.  The ID is computed on a sample
// (sample_near), then checked on a probe of unsampled pool entries (nearest
// first, then uniform); while the probe residual ||M_P(:,p) - M_P(:,q) T||_F
// exceeds 10 tol ||M_P||_F the sample is doubled.
// ---------------------------------------------------------------------------
template <class Pool, class Ent>
static void adaptive_id(const Pool& pool, const std::vector<int64_t>& cand, double tol, uint64_t seed,
                        const Ent& ent, IdBlock& blk) {
  const int c = (int)cand.size();
  const int64_t M = pool.size();
  int s = sample_count(c);
  std::vector<int64_t> pos, rows;
  for (int attempt = 0;; ++attempt) {
    pool.sample(cand, s, seed + 0x51ull * attempt, pos);
    const int ns = (int)pos.size();
    std::vector<cplx> Mt((size_t)ns * c);
    for (int cc = 0; cc < c; ++cc)
      for (int r = 0; r < ns; ++r) Mt[(size_t)cc * ns + r] = ent(pool.at(pos[r]), cand[cc]);
    column_id(Mt, ns, c, tol, blk);
    if (ns >= M || blk.k >= c) return;          // whole pool used, or no compression: exact on the sample
    // probe: up to 16 + c/2 unsampled entries, the nearest half first
    pool.probe(cand, pos, (int)std::min<int64_t>(M - ns, 16 + c / 2), seed ^ 0xFEEDull, rows);
    const int np = (int)rows.size();
    double num = 0.0, den = 0.0;
    const int nr = c - blk.k;
    for (int r = 0; r < np; ++r) {
      std::vector<cplx> row(c);
      for (int cc = 0; cc < c; ++cc) { row[cc] = ent(rows[r], cand[cc]); den += std::norm(row[cc]); }
      for (int j = 0; j < nr; ++j) {
        cplx acc = row[blk.p[j]];
        for (int i = 0; i < blk.k; ++i) acc -= row[blk.q[i]] * blk.t[(size_t)i * nr + j];
        num += std::norm(acc);
      }
    }
    if (num <= 100.0 * tol * tol * den || s >= M || attempt >= 6) return;
    s = (int)std::min<int64_t>(M, 2 * (int64_t)s);
  }
}

// ---------------------------------------------------------------------------
// One butterfly: interleaved row / column stages (complementary
// skeletonization of the IDBF: column IDs sample the row skeletons of the
// same level, row IDs sample the column skeletons of the previous level).
// ---------------------------------------------------------------------------
static void build_butterfly(Butterfly& B, const Entries& K, int64_t n0, double tol, uint64_t seed, bool par) {
  const Geometry& geo = *K.g;
  const int L = B.L;
  const int64_t npairs = (int64_t)1 << L;
  B.col.assign(B.hc, std::vector<IdBlock>(npairs));
  B.row.assign(B.hr, std::vector<IdBlock>(npairs));
  const int dmax = std::max(B.hc, B.hr);
  // Sample pools are shared: the first row stage samples the whole column range,
  // and a stage's other pools depend on one node pair only.  Each distinct pool
  // is formed once per stage; pools of kTreeMin entries or more get a k-d tree.
  constexpr int64_t kTreeMin = 1024;
  std::vector<std::vector<int64_t>> lists;
  std::vector<PoolTree> trees;
  auto make_pools = [&](int64_t nkeys, const auto& fill) {
    lists.assign((size_t)nkeys, {});
    trees.assign((size_t)nkeys, PoolTree());
#pragma omp parallel for schedule(dynamic, 1) if (par)
    for (int64_t key = 0; key < nkeys; ++key) {
      fill(key, lists[(size_t)key]);
      const int64_t M = (int64_t)lists[(size_t)key].size();
      if (M >= kTreeMin) trees[(size_t)key].build(geo, lists[(size_t)key].data(), 0, M);
    }
  };
  PoolTree col_tree;   // row stage 0: the column range [col0, col0 + n)
  col_tree.build(geo, nullptr, B.col0, B.n);
  for (int d = 0; d < dmax; ++d) {
    // ---- row stage d: pairs (a at row level L-d, b at column level d), g = b*2^(L-d) + a
    if (d < B.hr) {
      const int64_t na = (int64_t)1 << (L - d);
      // d > 0: pool (ap, b) = column skeletons of column stage d-1 under column node b
      // (level d): pairs (ap = ancestor of a at row level d-1, b'' at column level L-d+1)
      const int sh = L - 2 * d + 1;
      const int64_t nbd = (int64_t)1 << d;
      if (d > 0) {
        const int64_t nbpp = (int64_t)1 << (L - d + 1);
        make_pools(((int64_t)1 << (d - 1)) * nbd, [&](int64_t key, std::vector<int64_t>& pool) {
          const int64_t ap = key / nbd, b = key % nbd;
          for (int64_t bb = b << sh; bb < ((b + 1) << sh); ++bb) {
            const IdBlock& cb = B.col[d - 1][ap * nbpp + bb];
            pool.insert(pool.end(), cb.skel.begin(), cb.skel.end());
          }
        });
      }
#pragma omp parallel for schedule(dynamic, 4) if (par)
      for (int64_t g = 0; g < npairs; ++g) {
        int64_t b = g / na, a = g % na;
        IdBlock& blk = B.row[d][g];
        std::vector<int64_t> cand;
        if (d == 0) {
          for (int64_t r = 0; r < n0; ++r) cand.push_back(B.row0 + a * n0 + r);
        } else {
          const int64_t nap = (int64_t)1 << (L - d + 1);
          const IdBlock& c0 = B.row[d - 1][(b >> 1) * nap + 2 * a];
          const IdBlock& c1 = B.row[d - 1][(b >> 1) * nap + 2 * a + 1];
          cand = c0.skel;
          cand.insert(cand.end(), c1.skel.begin(), c1.skel.end());
        }
        uint64_t sd = seed ^ (0x1000003ull * (uint64_t)(d + 1)) ^ (0x9E37ull * (uint64_t)g) ^ 0xABCDull;
        // row ID: entries K(candidate row, sampled column)
        auto ent = [&](int64_t col, int64_t row) { return K(row, col); };
        if (d == 0) {
          adaptive_id(TreePool{col_tree}, cand, tol, sd, ent, blk);
        } else {
          const size_t key = (size_t)((a >> sh) * nbd + b);
          if (trees[key].M > 0) adaptive_id(TreePool{trees[key]}, cand, tol, sd, ent, blk);
          else adaptive_id(ListPool{geo, lists[key]}, cand, tol, sd, ent, blk);
        }
        blk.skel.resize(blk.k);
        for (int i = 0; i < blk.k; ++i) blk.skel[i] = cand[blk.q[i]];
      }
    }
    // ---- column stage d: pairs (a at row level d, b at column level L-d), g = a*2^(L-d) + b
    if (d < B.hc) {
      const int64_t nb = (int64_t)1 << (L - d);
      // pool (a, bp) = row skeletons of row stage d under row node a (level d):
      // pairs (a'' at row level L-d below a, bp = ancestor of b at column level d)
      const int sh = L - 2 * d;
      const int64_t nad = (int64_t)1 << d;
      const int64_t na2 = (int64_t)1 << (L - d);
      make_pools(nad * nad, [&](int64_t key, std::vector<int64_t>& pool) {
        const int64_t a = key / nad, bp = key % nad;
        for (int64_t aa = a << sh; aa < ((a + 1) << sh); ++aa) {
          const IdBlock& rb = B.row[d][bp * na2 + aa];
          pool.insert(pool.end(), rb.skel.begin(), rb.skel.end());
        }
      });
#pragma omp parallel for schedule(dynamic, 4) if (par)
      for (int64_t g = 0; g < npairs; ++g) {
        int64_t a = g / nb, b = g % nb;
        IdBlock& blk = B.col[d][g];
        std::vector<int64_t> cand;
        if (d == 0) {
          for (int64_t j = 0; j < n0; ++j) cand.push_back(B.col0 + b * n0 + j);
        } else {
          const int64_t nbp = (int64_t)1 << (L - d + 1);
          const IdBlock& c0 = B.col[d - 1][(a >> 1) * nbp + 2 * b];
          const IdBlock& c1 = B.col[d - 1][(a >> 1) * nbp + 2 * b + 1];
          cand = c0.skel;
          cand.insert(cand.end(), c1.skel.begin(), c1.skel.end());
        }
        uint64_t sd = seed ^ (0x2000011ull * (uint64_t)(d + 1)) ^ (0x7F4Aull * (uint64_t)g) ^ 0x1234ull;
        // column ID: entries K(sampled row, candidate column)
        auto ent = [&](int64_t row, int64_t col) { return K(row, col); };
        const size_t key = (size_t)(a * nad + (b >> sh));
        if (trees[key].M > 0) adaptive_id(TreePool{trees[key]}, cand, tol, sd, ent, blk);
        else adaptive_id(ListPool{geo, lists[key]}, cand, tol, sd, ent, blk);
        blk.skel.resize(blk.k);
        for (int i = 0; i < blk.k; ++i) blk.skel[i] = cand[blk.q[i]];
      }
    }
  }
  // ---- middle: S(g) = K(rskel, cskel) on the column-stage-(hc-1) pairs
  const int64_t nbm = (int64_t)1 << (L - B.hc + 1);   // column nodes at level L-hc+1
  const int64_t nam = (int64_t)1 << (B.hc - 1);       // row nodes at level hc-1 (= L-hr+1)
  B.mid.assign(npairs, {});
#pragma omp parallel for schedule(dynamic, 8) if (par)
  for (int64_t g = 0; g < npairs; ++g) {
    int64_t a = g / nbm, b = g % nbm;
    const IdBlock& cb = B.col[B.hc - 1][g];
    const IdBlock& rb = B.row[B.hr - 1][b * nam + a];
    std::vector<cplx>& S = B.mid[g];
    S.resize((size_t)rb.k * cb.k);
    for (int r = 0; r < rb.k; ++r)
      for (int c = 0; c < cb.k; ++c) S[(size_t)r * cb.k + c] = K(rb.skel[r], cb.skel[c]);
  }
}

// inverse of a unit-lower (lower=true, strict lower part of A plus I) or upper
// (diagonal included) triangle of the n0 x n0 row-major block A
static void triangle_inverse(const cplx* A, int n0, bool lower, cplx* X) {
  for (int i = 0; i < n0 * n0; ++i) X[i] = 0.0;
  for (int col = 0; col < n0; ++col) {
    if (lower) {
      for (int i = 0; i < n0; ++i) {
        cplx acc = (i == col) ? cplx(1.0) : cplx(0.0);
        for (int l = 0; l < i; ++l) acc -= A[i * n0 + l] * X[l * n0 + col];
        X[i * n0 + col] = acc;
      }
    } else {
      for (int i = n0 - 1; i >= 0; --i) {
        cplx acc = (i == col) ? cplx(1.0) : cplx(0.0);
        for (int l = i + 1; l < n0; ++l) acc -= A[i * n0 + l] * X[l * n0 + col];
        X[i * n0 + col] = acc / A[i * n0 + i];
      }
    }
  }
}

// The sampled IDs truncate at eps / 10 (the tightened tolerance of the reading of
// Eq. (req)): per-ID errors of the sampled construction accumulate over the
// L + 3 factors of a butterfly and over the H-IDBF levels.
static constexpr double kIdTolFactor = 0.1;

// In-place LU without pivoting (Doolittle) of the n0 x n0 row-major block A:
// on return the strict lower part holds L (unit diagonal implied), the upper
// part U.  Returns false on a zero pivot.
static bool leaf_lu_inplace(cplx* A, int n0) {
  for (int k = 0; k < n0; ++k) {
    const cplx piv = A[k * n0 + k];
    if (piv == cplx(0.0)) return false;
    for (int i = k + 1; i < n0; ++i) {
      const cplx l = A[i * n0 + k] / piv;
      A[i * n0 + k] = l;
      for (int j = k + 1; j < n0; ++j) A[i * n0 + j] -= l * A[k * n0 + j];
    }
  }
  return true;
}

int build_factor(const Geometry& g, double wavelength, double eta0, double gamma, int64_t leaf, double eps,
                 uint64_t seed, HostFactor& hf, int options) {
  auto t0 = std::chrono::steady_clock::now();
  if (leaf < 8 || leaf > 256 || eps <= 0 || eps >= 1 || wavelength <= 0) {
    set_error("hb_factor: need 8 <= leaf <= 256, 0 < eps < 1, wavelength > 0");
    return HB_EINVAL;
  }
  int64_t n = g.n;
  if (n % leaf) { set_error("hb_factor: N=%lld is not leaf*2^D", (long long)n); return HB_EUNSUPPORTED; }
  int64_t m = n / leaf;
  int D = 0;
  while (((int64_t)1 << D) < m) ++D;
  if (((int64_t)1 << D) != m || D < 1) {
    set_error("hb_factor: N=%lld is not leaf*2^D with D>=1", (long long)n);
    return HB_EUNSUPPORTED;
  }
  if (D > 30) { set_error("hb_factor: depth too large"); return HB_EUNSUPPORTED; }
  Entries K;
  K.init(g, wavelength, eta0, gamma);
  hf.n = n; hf.n0 = leaf; hf.m = m; hf.depth = D;
  hf.scale = K.scale; hf.eps = eps; hf.kappa = K.kappa; hf.eta0 = eta0; hf.gamma = gamma;
  // dense leaves and their triangle inverses
  hf.leaf.assign((size_t)m * leaf * leaf, cplx(0.0));
  hf.linv.assign(hf.leaf.size(), cplx(0.0));
  hf.uinv.assign(hf.leaf.size(), cplx(0.0));
  // leaf triangles: the entry-wise triangles of A_leaf (Eqs. (Lt), (Ut)), or with
  // HB_OPT_LEAF_LU the LU factors of A_leaf (unit lower L, upper U, no pivoting)
  const bool leaf_lu = (options & HB_OPT_LEAF_LU) != 0;
  hf.leaf_lu = leaf_lu;
  int bad_pivot = 0;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t j = 0; j < m; ++j) {
    cplx* A = &hf.leaf[(size_t)j * leaf * leaf];
    for (int64_t r = 0; r < leaf; ++r)
      for (int64_t c = 0; c < leaf; ++c) A[r * leaf + c] = K(j * leaf + r, j * leaf + c);
    if (leaf_lu) {
      std::vector<cplx> lu(A, A + leaf * leaf);
      if (!leaf_lu_inplace(lu.data(), (int)leaf)) {
#pragma omp atomic write
        bad_pivot = 1;
        continue;
      }
      triangle_inverse(lu.data(), (int)leaf, true, &hf.linv[(size_t)j * leaf * leaf]);
      triangle_inverse(lu.data(), (int)leaf, false, &hf.uinv[(size_t)j * leaf * leaf]);
    } else {
      triangle_inverse(A, (int)leaf, true, &hf.linv[(size_t)j * leaf * leaf]);
      triangle_inverse(A, (int)leaf, false, &hf.uinv[(size_t)j * leaf * leaf]);
    }
  }
  if (bad_pivot) {
    set_error("hb_factor: LU of a leaf block without pivoting met a zero pivot");
    return HB_EUNSUPPORTED;
  }
  // butterflies: F12 and F21 of every internal node (Alg. 1)
  int64_t nbf = 2 * (m - 1);
  hf.bf.assign(nbf, Butterfly());
  for (int v = 0; v < D; ++v) {
    int64_t nodes = (int64_t)1 << v;
    int64_t half = n >> (v + 1);
    for (int64_t p = 0; p < nodes; ++p)
      for (int kind = 0; kind < 2; ++kind) {
        Butterfly& B = hf.bf[bf_id(v, p, kind)];
        B.depth = v; B.node = p; B.kind = kind; B.n = half;
        int64_t base = p * 2 * half;
        B.row0 = kind == 0 ? base : base + half;
        B.col0 = kind == 0 ? base + half : base;
        B.L = D - v - 1;
        B.hc = (B.L % 2 == 0) ? B.L / 2 + 1 : (B.L + 1) / 2;
        B.hr = B.L + 2 - B.hc;
      }
  }
#ifdef _OPENMP
  int nthr = omp_get_max_threads();
#else
  int nthr = 1;
#endif
  for (int v = 0; v < D; ++v) {
    int64_t first = bf_id(v, 0, 0), cnt = (int64_t)2 << v;
    bool outer = cnt >= 2 * nthr;
    uint64_t sdv = seed * 0x100000001B3ull;
#pragma omp parallel for schedule(dynamic, 1) if (outer)
    for (int64_t i = 0; i < cnt; ++i)
      build_butterfly(hf.bf[first + i], K, leaf, eps * kIdTolFactor, sdv ^ (uint64_t)(first + i) * 0xC2B2AE35ull, !outer);
  }
  hf.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return HB_OK;
}

// ---------------------------------------------------------------------------
// Packing into the level-packed device image.
// ---------------------------------------------------------------------------
namespace {
struct Packer {
  PackedHost& ph;
  explicit Packer(PackedHost& p) : ph(p) {}
  int64_t push_mat(const cplx* src, int64_t cnt) {
    if (ph.fpool.size() % 2) ph.fpool.push_back(cplx(0.0));     // 16-byte aligned starts for float2
    int64_t off = (int64_t)ph.fpool.size();
    ph.fpool.insert(ph.fpool.end(), src, src + cnt);
    return off;
  }
  DBlk push_block(const IdBlock& b, bool vtype) {
    DBlk d;
    d.k = (int16_t)b.k;
    d.c = (int16_t)b.c;
    int nr = b.c - b.k;
    std::vector<cplx> m((size_t)b.k * nr);
    for (int i = 0; i < b.k; ++i)
      for (int j = 0; j < nr; ++j) {
        cplx t = b.t[(size_t)i * nr + j];
        if (vtype) m[(size_t)j * b.k + i] = t; else m[(size_t)i * nr + j] = t;
      }
    d.moff = push_mat(m.data(), (int64_t)m.size());
    while (ph.ipool.size() % 8) ph.ipool.push_back(0);     // 16-byte aligned index blocks
    d.ioff = (int32_t)ph.ipool.size();
    for (int i = 0; i < b.k; ++i) ph.ipool.push_back((int16_t)b.q[i]);
    for (int j = 0; j < nr; ++j) ph.ipool.push_back((int16_t)b.p[j]);
    std::vector<int16_t> map(b.c);
    for (int i = 0; i < b.k; ++i) map[b.q[i]] = (int16_t)i;
    for (int j = 0; j < nr; ++j) map[b.p[j]] = (int16_t)(-1 - j);
    ph.ipool.insert(ph.ipool.end(), map.begin(), map.end());
    ph.nnz_bf += (int64_t)b.k * nr;
    return d;
  }
};
}  // namespace

// Dense sweep-leaf triangles (PackedHost::sl) from the subtree programs.
static void build_sweep_leaves(const HostFactor& hf, PackedHost& ph, const std::vector<std::vector<DPhase>> (&subs)[2]);

void pack_factor(const HostFactor& hf, PackedHost& ph) {
  Packer pk(ph);
  const int D = hf.depth;
  const int64_t m = hf.m, n0 = hf.n0;
  ph.n = hf.n; ph.n0 = n0; ph.m = m; ph.depth = D;
  ph.fpool.clear(); ph.ipool.clear(); ph.items.clear();
  ph.nnz_bf = 0;
  const int64_t nbf = (int64_t)hf.bf.size();
  ph.vout.assign((size_t)m * D, DOuter{});
  ph.uout.assign((size_t)m * D, DOuter{});
  ph.bf_vout0.assign(nbf, 0); ph.bf_uout0.assign(nbf, 0); ph.bf_mb.assign(nbf, 0);
  ph.bf_step_base.assign(nbf, 0); ph.bf_L.assign(nbf, 0);
  ph.bvout.clear(); ph.buout.clear(); ph.bf_steps.clear();
  int64_t state = 0;
  int64_t ksum = 0, kcnt = 0;
  int kmax = 0;
  std::vector<int64_t> ksum_d(D, 0), kcnt_d(D, 0);
  std::vector<int> kmax_d(D, 0);
  // per step item lists for the apply
  std::vector<std::vector<int32_t>> fsteps(D + 2), asteps(D + 2);
  // butterfly state in post-order of the cluster tree (both subtrees, then the
  // node's F12 and F21), so the state of every subtree is one contiguous range
  std::vector<int64_t> st_base(nbf, 0);
  {
    int64_t cur = 0;
    std::function<void(int, int64_t)> alloc = [&](int v, int64_t p) {
      if (v == D) return;
      alloc(v + 1, 2 * p);
      alloc(v + 1, 2 * p + 1);
      for (int kind = 0; kind < 2; ++kind) {
        int64_t id = bf_id(v, p, kind);
        const Butterfly& B = hf.bf[id];
        st_base[id] = cur;
        const int64_t np = (int64_t)1 << B.L;
        for (int l = 0; l < B.hc; ++l)
          for (int64_t g = 0; g < np; ++g) cur += B.col[l][g].k;
        for (int l = 0; l < B.hr; ++l)
          for (int64_t g = 0; g < np; ++g) cur += B.row[l][g].k;
      }
    };
    alloc(0, 0);
    state = cur;
  }
  for (int64_t id = 0; id < nbf; ++id) {
    const Butterfly& B = hf.bf[id];
    const int L = B.L;
    const int64_t np = (int64_t)1 << L;
    ph.bf_L[id] = L;
    int64_t sb = st_base[id];
    // state offsets of every pair vector
    std::vector<std::vector<int32_t>> zoff(B.hc, std::vector<int32_t>(np)), yoff(B.hr, std::vector<int32_t>(np));
    for (int l = 0; l < B.hc; ++l)
      for (int64_t g = 0; g < np; ++g) { zoff[l][g] = (int32_t)sb; sb += B.col[l][g].k; }
    for (int l = 0; l < B.hr; ++l)
      for (int64_t g = 0; g < np; ++g) { yoff[l][g] = (int32_t)sb; sb += B.row[l][g].k; }
    // rank statistics
    for (int l = 0; l < B.hc; ++l)
      for (auto& b : B.col[l]) { ksum += b.k; kcnt++; kmax = std::max(kmax, b.k); ksum_d[B.depth] += b.k; kcnt_d[B.depth]++; kmax_d[B.depth] = std::max(kmax_d[B.depth], b.k); }
    for (int l = 0; l < B.hr; ++l)
      for (auto& b : B.row[l]) { ksum += b.k; kcnt++; kmax = std::max(kmax, b.k); ksum_d[B.depth] += b.k; kcnt_d[B.depth]++; kmax_d[B.depth] = std::max(kmax_d[B.depth], b.k); }
    // V0 ops (column leaves) and U0 ops (row leaves)
    ph.bf_mb[id] = (int32_t)np;
    ph.bf_vout0[id] = (int32_t)ph.bvout.size();
    for (int64_t b = 0; b < np; ++b) {
      DOuter o;
      o.blk = pk.push_block(B.col[0][b], true);        // g = 0*2^L + b
      o.seg_off = zoff[0][b];
      o.leaf = (int32_t)(B.col0 / n0 + b);
      ph.bvout.push_back(o);
      ph.vout[(size_t)o.leaf * D + B.depth] = o;
    }
    ph.bf_uout0[id] = (int32_t)ph.buout.size();
    for (int64_t a = 0; a < np; ++a) {
      DOuter o;
      o.blk = pk.push_block(B.row[0][a], false);       // g = 0*2^L + a
      o.seg_off = yoff[0][a];
      o.leaf = (int32_t)(B.row0 / n0 + a);
      ph.buout.push_back(o);
      ph.uout[(size_t)o.leaf * D + B.depth] = o;
    }
    // inner steps: VIN l = 1..hc-1, MID, UIN l = hr-1..1
    ph.bf_step_base[id] = (int32_t)ph.bf_steps.size();
    int step = 0;
    auto open_step = [&]() { ph.bf_steps.push_back((int32_t)ph.items.size()); step++; };
    for (int l = 1; l < B.hc; ++l) {
      open_step();
      const int64_t nb = (int64_t)1 << (L - l), nbp = (int64_t)1 << (L - l + 1);
      for (int64_t ap = 0; ap < ((int64_t)1 << (l - 1)); ++ap)
        for (int64_t b = 0; b < nb; ++b) {
          DItem it{};
          it.type = 0;
          int64_t gi0 = ap * nbp + 2 * b, gi1 = gi0 + 1;
          int64_t go0 = (2 * ap) * nb + b, go1 = (2 * ap + 1) * nb + b;
          it.a_off[0] = zoff[l - 1][gi0]; it.a_k[0] = (int16_t)B.col[l - 1][gi0].k;
          it.a_off[1] = zoff[l - 1][gi1]; it.a_k[1] = (int16_t)B.col[l - 1][gi1].k;
          it.b_off[0] = zoff[l][go0]; it.b_k[0] = (int16_t)B.col[l][go0].k;
          it.b_off[1] = zoff[l][go1]; it.b_k[1] = (int16_t)B.col[l][go1].k;
          it.blk[0] = pk.push_block(B.col[l][go0], true);
          it.blk[1] = pk.push_block(B.col[l][go1], true);
          fsteps[step].push_back((int32_t)ph.items.size());
          asteps[L + 2 - step].push_back((int32_t)ph.items.size());
          ph.items.push_back(it);
        }
    }
    {
      open_step();
      const int64_t nbm = (int64_t)1 << (L - B.hc + 1), nam = (int64_t)1 << (B.hc - 1);
      for (int64_t g = 0; g < np; ++g) {
        int64_t a = g / nbm, b = g % nbm;
        int64_t gr = b * nam + a;
        DItem it{};
        it.type = 1;
        it.a_off[0] = zoff[B.hc - 1][g]; it.a_k[0] = (int16_t)B.col[B.hc - 1][g].k;
        it.b_off[0] = yoff[B.hr - 1][gr]; it.b_k[0] = (int16_t)B.row[B.hr - 1][gr].k;
        // S stored [c][r] (output index r fastest)
        const std::vector<cplx>& S = B.mid[g];
        int kr = it.b_k[0], kc = it.a_k[0];
        std::vector<cplx> sm((size_t)kr * kc);
        for (int r = 0; r < kr; ++r)
          for (int c = 0; c < kc; ++c) sm[(size_t)c * kr + r] = S[(size_t)r * kc + c];
        it.blk[0].moff = pk.push_mat(sm.data(), (int64_t)sm.size());
        it.blk[0].ioff = 0; it.blk[0].k = (int16_t)kr; it.blk[0].c = (int16_t)kc;
        ph.nnz_bf += (int64_t)kr * kc;
        fsteps[step].push_back((int32_t)ph.items.size());
        asteps[L + 2 - step].push_back((int32_t)ph.items.size());
        ph.items.push_back(it);
      }
    }
    for (int l = B.hr - 1; l >= 1; --l) {
      open_step();
      const int64_t na = (int64_t)1 << (L - l), nap = (int64_t)1 << (L - l + 1);
      for (int64_t bp = 0; bp < ((int64_t)1 << (l - 1)); ++bp)
        for (int64_t a = 0; a < na; ++a) {
          DItem it{};
          it.type = 2;
          int64_t gi0 = (2 * bp) * na + a, gi1 = (2 * bp + 1) * na + a;      // row stage l inputs
          int64_t go0 = bp * nap + 2 * a, go1 = go0 + 1;                       // row stage l-1 outputs
          it.a_off[0] = yoff[l - 1][go0]; it.a_k[0] = (int16_t)B.row[l - 1][go0].k;
          it.a_off[1] = yoff[l - 1][go1]; it.a_k[1] = (int16_t)B.row[l - 1][go1].k;
          it.b_off[0] = yoff[l][gi0]; it.b_k[0] = (int16_t)B.row[l][gi0].k;
          it.b_off[1] = yoff[l][gi1]; it.b_k[1] = (int16_t)B.row[l][gi1].k;
          it.blk[0] = pk.push_block(B.row[l][gi0], false);
          it.blk[1] = pk.push_block(B.row[l][gi1], false);
          fsteps[step].push_back((int32_t)ph.items.size());
          asteps[L + 2 - step].push_back((int32_t)ph.items.size());
          ph.items.push_back(it);
        }
    }
    ph.bf_steps.push_back((int32_t)ph.items.size());   // end of the last step
  }
  ph.state_len = state;
  ph.nsteps = D;
  ph.step_ptr.assign(1, 0); ph.step_idx.clear();
  ph.astep_ptr.assign(1, 0); ph.astep_idx.clear();
  for (int s = 1; s <= D; ++s) {
    ph.step_idx.insert(ph.step_idx.end(), fsteps[s].begin(), fsteps[s].end());
    ph.step_ptr.push_back((int32_t)ph.step_idx.size());
    ph.astep_idx.insert(ph.astep_idx.end(), asteps[s].begin(), asteps[s].end());
    ph.astep_ptr.push_back((int32_t)ph.astep_idx.size());
  }
  // sweep programs (recursion of Algs. 3 and 4, and their adjoints)
  auto blk_bytes = [](const DBlk& b) { return (int64_t)b.k * (b.c - b.k) * 16 + (int64_t)4 * b.c + 32; };
  auto outer_phase = [&](int kind, int64_t id, bool adj) {
    bool use_u = ((kind == PH_ENTER) == adj);
    const DOuter* ops = use_u ? &ph.buout[ph.bf_uout0[id]] : &ph.bvout[ph.bf_vout0[id]];
    int64_t mb = 0;
    int vm = 0;
    for (int o = 0; o < ph.bf_mb[id]; ++o) {
      mb = std::max(mb, blk_bytes(ops[o].blk));
      vm = std::max(vm, kind == PH_ENTER ? (int)ops[o].blk.c : (int)ops[o].blk.k);
    }
    return DPhase{kind, (int32_t)id, ph.bf_mb[id], adj ? 1 : 0, (int32_t)std::min<int64_t>(mb, INT32_MAX), vm};
  };
  auto emit_bf = [&](std::vector<DPhase>& prog, int64_t id, bool adj) {
    int L = ph.bf_L[id];
    int base = ph.bf_step_base[id];
    prog.push_back(outer_phase(PH_ENTER, id, adj));
    for (int t = 1; t <= L + 1; ++t) {
      int s = adj ? (L + 2 - t) : t;
      int32_t b0 = ph.bf_steps[base + s - 1], b1 = ph.bf_steps[base + s];
      int64_t mb = 0;
      int vm = 0;
      for (int32_t e = b0; e < b1; ++e) {
        const DItem& it = ph.items[e];
        if (it.type == 1) {
          mb = std::max(mb, (int64_t)it.a_k[0] * it.b_k[0] * 16 + 32);
          vm = std::max(vm, (int)std::max(it.a_k[0], it.b_k[0]));
        } else {
          mb = std::max(mb, blk_bytes(it.blk[0]) + blk_bytes(it.blk[1]));
          vm = std::max(vm, std::max(it.a_k[0] + it.a_k[1], it.b_k[0] + it.b_k[1]));
        }
      }
      prog.push_back(DPhase{PH_ITEMS, b0, b1 - b0, adj ? 1 : 0, (int32_t)std::min<int64_t>(mb, INT32_MAX), vm});
    }
    prog.push_back(outer_phase(PH_EXIT, id, adj));
  };
  ph.prog_lower.clear(); ph.prog_upper.clear(); ph.prog_lower_adj.clear(); ph.prog_upper_adj.clear();
  // sweep leaves: merge the lowest sl_t levels while the subtree has at most kSweepLeafMax rows
  ph.sl_t = 0;
  while (ph.sl_t < D && (n0 << (ph.sl_t + 1)) <= kSweepLeafMax) ++ph.sl_t;
  ph.sl_n = n0 << ph.sl_t;
  ph.sl_m = m >> ph.sl_t;
  const int vl = D - ph.sl_t;   // depth of the sweep leaves
  // lower: left child, F21, right child
  std::function<void(int, int64_t, std::vector<DPhase>&, int)> rec = [&](int v, int64_t p, std::vector<DPhase>& prog, int mode) {
    if (v == vl) {
      prog.push_back(DPhase{PH_LEAF, (int32_t)p, 1, (mode >= 2) ? 1 : 0,
                            (int32_t)std::min<int64_t>(packed_tri(ph.sl_n) * 16, INT32_MAX), (int32_t)ph.sl_n});
      return;
    }
    int64_t lo = 2 * p, hi = 2 * p + 1;
    switch (mode) {
      case 0:  rec(v + 1, lo, prog, mode); emit_bf(prog, bf_id(v, p, 1), false); rec(v + 1, hi, prog, mode); break;  // L~^{-1}
      case 1:  rec(v + 1, hi, prog, mode); emit_bf(prog, bf_id(v, p, 0), false); rec(v + 1, lo, prog, mode); break;  // U~^{-1}
      case 2:  rec(v + 1, hi, prog, mode); emit_bf(prog, bf_id(v, p, 1), true); rec(v + 1, lo, prog, mode); break;   // L~^{-H}
      default: rec(v + 1, lo, prog, mode); emit_bf(prog, bf_id(v, p, 0), true); rec(v + 1, hi, prog, mode); break;  // U~^{-H}
    }
  };
  rec(0, 0, ph.prog_lower, 0);
  rec(0, 0, ph.prog_upper, 1);
  rec(0, 0, ph.prog_lower_adj, 2);
  rec(0, 0, ph.prog_upper_adj, 3);
  // the full-depth programs (down to the n0 leaves) of every sweep-leaf subtree,
  // for L~^{-1} (mode 0) and U~^{-1} (mode 1); their results on unit vectors
  // are the columns of the sweep-leaf triangles
  std::vector<std::vector<DPhase>> subs[2];
  std::function<void(int, int64_t, std::vector<DPhase>&, int)> rec_full = [&](int v, int64_t p, std::vector<DPhase>& prog, int mode) {
    if (v == D) {
      prog.push_back(DPhase{PH_LEAF, (int32_t)p, 1, 0, 0, (int32_t)n0});
      return;
    }
    const int64_t lo = 2 * p, hi = 2 * p + 1;
    if (mode == 0) { rec_full(v + 1, lo, prog, mode); emit_bf(prog, bf_id(v, p, 1), false); rec_full(v + 1, hi, prog, mode); }
    else { rec_full(v + 1, hi, prog, mode); emit_bf(prog, bf_id(v, p, 0), false); rec_full(v + 1, lo, prog, mode); }
  };
  for (int mode = 0; mode < 2; ++mode) {
    subs[mode].resize((size_t)ph.sl_m);
    for (int64_t p = 0; p < ph.sl_m; ++p) rec_full(vl, p, subs[mode][(size_t)p], mode);
  }
  build_sweep_leaves(hf, ph, subs);
  // tail padding so 16-byte bulk copies of the last block stay inside the pools
  for (int i = 0; i < 4; ++i) ph.fpool.push_back(cplx(0.0));
  for (int i = 0; i < 16; ++i) ph.ipool.push_back(0);
  ph.kmax = kmax;
  ph.kavg = kcnt ? (double)ksum / (double)kcnt : 0.0;
  for (int v = 0; v < D && v < 32; ++v) {
    ph.kmax_depth[v] = kmax_d[v];
    ph.kavg_depth[v] = kcnt_d[v] ? (double)ksum_d[v] / (double)kcnt_d[v] : 0.0;
  }
}

}  // namespace hb

// ---------------------------------------------------------------------------
// Host interpreter of the packed program (FP64).  It walks exactly the
// records the device kernels walk (V0 / items / U0 / sweep phases) and is used
// to verify construction and packing on machines without a GPU.
// ---------------------------------------------------------------------------
namespace hb {

namespace {
struct HostExec {
  const PackedHost& ph;
  const HostFactor& hf;
  std::vector<cplx> st;
  HostExec(const PackedHost& p, const HostFactor& h) : ph(p), hf(h), st(p.state_len) {}

  // V-type (column ID) element T_ij from layout A; U-type from layout B
  cplx tv(const DBlk& b, int i, int j) const { return ph.fpool[b.moff + (int64_t)j * b.k + i]; }
  cplx tu(const DBlk& b, int i, int j) const { return ph.fpool[b.moff + (int64_t)i * (b.c - b.k) + j]; }
  const int16_t* idx(const DBlk& b) const { return &ph.ipool[b.ioff]; }

  // B = gather + T * rest of cand;  utype_adj: conj(T) from the U layout
  void vlike(const DBlk& b, const cplx* a0, int ka0, const cplx* a1, cplx* out, bool utype_adj) const {
    const int16_t* q = idx(b);
    const int16_t* p = q + b.k;
    for (int i = 0; i < b.k; ++i) {
      cplx acc = q[i] < ka0 ? a0[q[i]] : a1[q[i] - ka0];
      for (int j = 0; j < b.c - b.k; ++j) {
        cplx t = utype_adj ? std::conj(tu(b, i, j)) : tv(b, i, j);
        acc += t * (p[j] < ka0 ? a0[p[j]] : a1[p[j] - ka0]);
      }
      out[i] = acc;
    }
  }
  // contribution to candidate entry r;  vtype_adj: conj(T) from the V layout
  cplx row(const DBlk& b, const cplx* y, int r, bool vtype_adj) const {
    int code = idx(b)[b.c + r];
    if (code >= 0) return y[code];
    int j = -1 - code;
    cplx acc = 0.0;
    for (int i = 0; i < b.k; ++i) acc += (vtype_adj ? std::conj(tv(b, i, j)) : tu(b, i, j)) * y[i];
    return acc;
  }
  void item(const DItem& it, bool adj) {
    if (it.type == 1) {
      int kr = it.b_k[0], kc = it.a_k[0];
      const cplx* S = &ph.fpool[it.blk[0].moff];
      if (!adj)
        for (int r = 0; r < kr; ++r) {
          cplx acc = 0.0;
          for (int c = 0; c < kc; ++c) acc += S[(int64_t)c * kr + r] * st[it.a_off[0] + c];
          st[it.b_off[0] + r] = acc;
        }
      else
        for (int c = 0; c < kc; ++c) {
          cplx acc = 0.0;
          for (int r = 0; r < kr; ++r) acc += std::conj(S[(int64_t)c * kr + r]) * st[it.b_off[0] + r];
          st[it.a_off[0] + c] = acc;
        }
      return;
    }
    bool to_b = (it.type == 0) != adj;
    if (to_b) {
      for (int s = 0; s < 2; ++s)
        vlike(it.blk[s], &st[it.a_off[0]], it.a_k[0], &st[it.a_off[1]], &st[it.b_off[s]], it.type == 2);
    } else {
      int c = it.a_k[0] + it.a_k[1];
      std::vector<cplx> out(c);
      for (int r = 0; r < c; ++r)
        out[r] = row(it.blk[0], &st[it.b_off[0]], r, it.type == 0) + row(it.blk[1], &st[it.b_off[1]], r, it.type == 0);
      for (int r = 0; r < c; ++r) st[r < it.a_k[0] ? it.a_off[0] + r : it.a_off[1] + r - it.a_k[0]] = out[r];
    }
  }
  // leaf matrices are row-major [r][c] on the host
  void leaf_mv(const std::vector<cplx>& M, int64_t leaf, const cplx* x, cplx* y, bool adj) const {
    const int64_t n0 = ph.n0;
    const cplx* A = &M[leaf * n0 * n0];
    for (int64_t r = 0; r < n0; ++r) {
      cplx acc = 0.0;
      for (int64_t c = 0; c < n0; ++c) acc += (adj ? std::conj(A[c * n0 + r]) : A[r * n0 + c]) * x[c];
      y[r] = acc;
    }
  }

  void apply(bool adj, const cplx* x, cplx* y) {
    const int D = ph.depth;
    const int64_t n0 = ph.n0;
    const std::vector<DOuter>& enter = adj ? ph.uout : ph.vout;
    const std::vector<DOuter>& exitv = adj ? ph.vout : ph.uout;
    for (int64_t l = 0; l < ph.m; ++l)
      for (int v = 0; v < D; ++v) {
        const DOuter& o = enter[l * D + v];
        vlike(o.blk, x + l * n0, (int)n0, x + l * n0, &st[o.seg_off], adj);
      }
    const std::vector<int32_t>& ptr = adj ? ph.astep_ptr : ph.step_ptr;
    const std::vector<int32_t>& ix = adj ? ph.astep_idx : ph.step_idx;
    for (size_t s = 0; s + 1 < ptr.size(); ++s)
      for (int32_t e = ptr[s]; e < ptr[s + 1]; ++e) item(ph.items[ix[e]], adj);
    std::vector<cplx> tmp(n0);
    for (int64_t l = 0; l < ph.m; ++l) {
      for (int64_t r = 0; r < n0; ++r) {
        cplx acc = 0.0;
        for (int v = 0; v < D; ++v) {
          const DOuter& o = exitv[l * D + v];
          acc += row(o.blk, &st[o.seg_off], (int)r, adj);
        }
        y[l * n0 + r] = acc;
      }
      leaf_mv(hf.leaf, l, x + l * n0, tmp.data(), adj);
      for (int64_t r = 0; r < n0; ++r) y[l * n0 + r] += tmp[r];
    }
  }

  // x = T x for the packed sweep-leaf triangle p of sweep `which`
  void sl_mv(int which, int64_t p, cplx* x, cplx* y) const {
    const int64_t s = ph.sl_n;
    const cplx* T = &ph.sl[which][(size_t)(p * packed_tri(s))];
    const bool upper = (which == 1 || which == 2);
    for (int64_t r = 0; r < s; ++r) {
      cplx acc = 0.0;
      if (upper) for (int64_t c = r; c < s; ++c) acc += T[tri_off_upper(r, c)] * x[c];
      else for (int64_t c = 0; c <= r; ++c) acc += T[tri_off_lower(s, r, c)] * x[c];
      y[r] = acc;
    }
    std::copy(y, y + s, x);
  }

  // Run a sweep program in place.  sweep_leaves: its PH_LEAF phases are sweep
  // leaves (packed triangles of ph.sl[which]); otherwise n0 leaves (the leaf
  // triangle inverses, `which` 0 or 1).
  void run(const std::vector<DPhase>& prog, int which, cplx* vec, bool sweep_leaves) {
    const int64_t n0 = ph.n0;
    std::vector<cplx> tmp((size_t)std::max<int64_t>(n0, ph.sl_n));
    for (const DPhase& P : prog) {
      if (P.kind == PH_LEAF) {
        if (sweep_leaves) {
          sl_mv(which, P.arg0, vec + (int64_t)P.arg0 * ph.sl_n, tmp.data());
        } else {
          const std::vector<cplx>& tinv = (which == 0 || which == 2) ? hf.linv : hf.uinv;
          leaf_mv(tinv, P.arg0, vec + (int64_t)P.arg0 * n0, tmp.data(), P.adj != 0);
          std::copy(tmp.begin(), tmp.begin() + n0, vec + (int64_t)P.arg0 * n0);
        }
      } else if (P.kind == PH_ENTER) {
        const DOuter* ops = P.adj ? &ph.buout[ph.bf_uout0[P.arg0]] : &ph.bvout[ph.bf_vout0[P.arg0]];
        for (int o = 0; o < P.count; ++o) {
          const cplx* xl = vec + (int64_t)ops[o].leaf * n0;
          vlike(ops[o].blk, xl, (int)n0, xl, &st[ops[o].seg_off], P.adj != 0);
        }
      } else if (P.kind == PH_ITEMS) {
        for (int o = 0; o < P.count; ++o) item(ph.items[P.arg0 + o], P.adj != 0);
      } else {
        const DOuter* ops = P.adj ? &ph.bvout[ph.bf_vout0[P.arg0]] : &ph.buout[ph.bf_uout0[P.arg0]];
        for (int o = 0; o < P.count; ++o) {
          cplx* bl = vec + (int64_t)ops[o].leaf * n0;
          for (int64_t r = 0; r < n0; ++r) bl[r] -= row(ops[o].blk, &st[ops[o].seg_off], (int)r, P.adj != 0);
        }
      }
    }
  }

  void sweep(int which, cplx* vec) {
    const std::vector<DPhase>& prog = which == 0 ? ph.prog_lower : which == 1 ? ph.prog_upper
                                    : which == 2 ? ph.prog_lower_adj : ph.prog_upper_adj;
    run(prog, which, vec, true);
  }
};
}  // namespace

static void build_sweep_leaves(const HostFactor& hf, PackedHost& ph, const std::vector<std::vector<DPhase>> (&subs)[2]) {
  const int64_t s = ph.sl_n, P = packed_tri(s);
  for (int w = 0; w < 4; ++w) ph.sl[w].assign((size_t)(ph.sl_m * P), cplx(0.0));
#pragma omp parallel
  {
    HostExec ex(ph, hf);
    std::vector<cplx> vec((size_t)ph.n, cplx(0.0));
    std::vector<cplx> dense((size_t)(s * s));
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < ph.sl_m; ++p) {
      cplx* v = vec.data() + p * s;
      for (int mode = 0; mode < 2; ++mode) {
        // column j of the subtree's inverse triangle = the subtree sweep of e_j
        for (int64_t j = 0; j < s; ++j) {
          std::fill(v, v + s, cplx(0.0));
          v[j] = 1.0;
          ex.run(subs[mode][(size_t)p], mode, vec.data(), false);
          for (int64_t r = 0; r < s; ++r) dense[(size_t)(r * s + j)] = v[r];
        }
        // mode 0: T lower -> sl[0], T^H upper -> sl[2];  mode 1: T upper -> sl[1], T^H lower -> sl[3]
        cplx* a = &ph.sl[mode][(size_t)(p * P)];
        cplx* b = &ph.sl[mode + 2][(size_t)(p * P)];
        for (int64_t c = 0; c < s; ++c) {
          if (mode == 0) {
            for (int64_t r = c; r < s; ++r) a[tri_off_lower(s, r, c)] = dense[(size_t)(r * s + c)];
            for (int64_t r = 0; r <= c; ++r) b[tri_off_upper(r, c)] = std::conj(dense[(size_t)(c * s + r)]);
          } else {
            for (int64_t r = 0; r <= c; ++r) a[tri_off_upper(r, c)] = dense[(size_t)(r * s + c)];
            for (int64_t r = c; r < s; ++r) b[tri_off_lower(s, r, c)] = std::conj(dense[(size_t)(c * s + r)]);
          }
        }
      }
    }
  }
}

FlatProgram flatten_program(const PackedHost& ph, const std::vector<DPhase>& prog, int which) {
  FlatProgram fp;
  const int64_t n0 = ph.n0;
  const bool upper_tri = (which == 1 || which == 2);
  fp.base.reserve(prog.size() + 1);
  auto blkm = [](const DBlk& b) { return (int64_t)b.k * (b.c - b.k); };
  for (const DPhase& P : prog) {
    fp.base.push_back((int32_t)fp.ops.size());
    const bool adj = P.adj != 0;
    for (int o = 0; o < P.count; ++o) {
      FlatOp f{};
      if (P.kind == PH_LEAF) {
        // sweep leaf: packed triangle of order sl_n
        const int64_t s = ph.sl_n;
        f.kind = FK_LEAF;
        f.flags = (int16_t)(upper_tri ? FF_UPPER : 0);
        f.moff = (int64_t)P.arg0 * packed_tri(s);
        f.melems = (int32_t)packed_tri(s);
        f.ioff = -1;
        f.c0 = (int16_t)s;
        f.src0 = (int32_t)(P.arg0 * s);
        f.n_s0 = (int16_t)s;
        if (s > INT16_MAX) fp.ok = false;
        f.out0 = f.src0;
      } else if (P.kind == PH_ENTER || P.kind == PH_EXIT) {
        const bool enter = P.kind == PH_ENTER;
        const bool use_u = (enter == adj);
        const DOuter& op = use_u ? ph.buout[ph.bf_uout0[P.arg0] + o] : ph.bvout[ph.bf_vout0[P.arg0] + o];
        f.moff = op.blk.moff;
        f.melems = (int32_t)blkm(op.blk);
        f.ioff = op.blk.ioff;
        f.ielems = (int16_t)(2 * op.blk.c);
        f.k0 = op.blk.k;
        f.c0 = op.blk.c;
        if (enter) {
          f.kind = FK_GATHER;
          f.flags = (int16_t)((adj ? FF_CONJ : 0) | FF_SRC_VEC);
          f.src0 = (int32_t)(op.leaf * n0);
          f.n_s0 = op.blk.c;
          f.out0 = op.seg_off;
        } else {
          f.kind = FK_SCATTER;
          f.flags = (int16_t)((adj ? FF_CONJ : 0) | FF_SUB | FF_OUT_VEC);
          f.src0 = op.seg_off;
          f.n_s0 = op.blk.k;
          f.out0 = (int32_t)(op.leaf * n0);
          f.split = op.blk.c;
        }
      } else {
        const DItem& it = ph.items[P.arg0 + o];
        if (it.type == 1) {
          f.kind = FK_MIDDLE;
          f.flags = (int16_t)(adj ? FF_ADJ : 0);
          f.moff = it.blk[0].moff;
          f.melems = it.a_k[0] * it.b_k[0];
          f.ioff = -1;
          f.k0 = it.b_k[0];
          f.c0 = it.a_k[0];
          f.src0 = adj ? it.b_off[0] : it.a_off[0];
          f.n_s0 = adj ? it.b_k[0] : it.a_k[0];
          f.out0 = adj ? it.a_off[0] : it.b_off[0];
        } else {
          const DBlk& b0 = it.blk[0];
          const DBlk& b1 = it.blk[1];
          f.moff = b0.moff;
          f.m1 = (int32_t)(b1.moff - b0.moff);
          f.melems = (int32_t)(f.m1 + blkm(b1));
          f.ioff = b0.ioff;
          const int64_t i1 = (int64_t)b1.ioff - b0.ioff, ie = i1 + 2 * (int64_t)b1.c;
          if (i1 < 0 || ie > INT16_MAX) fp.ok = false;   // index blocks of an item must be adjacent
          f.i1 = (int16_t)i1;
          f.ielems = (int16_t)ie;
          f.k0 = b0.k; f.c0 = b0.c; f.k1 = b1.k; f.c1 = b1.c;
          const bool to_b = (it.type == 0) != adj;
          if (to_b) {
            f.kind = FK_GATHER;
            f.flags = (int16_t)(FF_TWO | (it.type == 2 ? FF_CONJ : 0));
            f.src0 = it.a_off[0]; f.n_s0 = it.a_k[0];
            f.src1 = it.a_off[1]; f.n_s1 = it.a_k[1];
            f.out0 = it.b_off[0]; f.out1 = it.b_off[1];
          } else {
            f.kind = FK_SCATTER;
            f.flags = (int16_t)(FF_TWO | (it.type == 0 ? FF_CONJ : 0));
            f.src0 = it.b_off[0]; f.n_s0 = it.b_k[0];
            f.src1 = it.b_off[1]; f.n_s1 = it.b_k[1];
            f.out0 = it.a_off[0]; f.out1 = it.a_off[1];
            f.split = it.a_k[0];
          }
        }
      }
      fp.ops.push_back(f);
    }
    // staging offsets of the phase's ops (one contiguous area per phase)
    int32_t off = 0;
    for (int32_t o = fp.base.back(); o < (int32_t)fp.ops.size(); ++o) {
      fp.ops[o].soff = off;
      off += flat_stage_bytes32(fp.ops[o]);
    }
    fp.pbytes.push_back(off);
  }
  fp.base.push_back((int32_t)fp.ops.size());
  return fp;
}

namespace {
// outputs (state entries or vector rows) of one op: [out0, out0+n0) and [out1, out1+n1)
void op_outputs(const FlatOp& f, int& n_out0, int& n_out1) {
  n_out0 = (f.kind == FK_GATHER) ? f.k0 : (f.kind == FK_SCATTER) ? ((f.flags & FF_TWO) ? f.split : f.c0)
         : (f.kind == FK_MIDDLE) ? ((f.flags & FF_ADJ) ? f.c0 : f.k0) : f.c0;
  n_out1 = (f.kind == FK_GATHER && (f.flags & FF_TWO)) ? f.k1
         : (f.kind == FK_SCATTER && (f.flags & FF_TWO)) ? f.c0 - f.split : 0;
}

// vector-row and state spans [lo, hi) touched by one phase (empty: lo = hi = 0)
struct Span { int32_t row_lo, row_hi, st_lo, st_hi; };
Span phase_span(const FlatProgram& fp, int ph) {
  Span sp{INT32_MAX, 0, INT32_MAX, 0};
  for (int32_t o = fp.base[ph]; o < fp.base[ph + 1]; ++o) {
    const FlatOp& f = fp.ops[o];
    auto row = [&](int32_t a, int32_t n) { sp.row_lo = std::min(sp.row_lo, a); sp.row_hi = std::max(sp.row_hi, a + n); };
    auto stt = [&](int32_t a, int32_t n) { if (n > 0) { sp.st_lo = std::min(sp.st_lo, a); sp.st_hi = std::max(sp.st_hi, a + n); } };
    int n_out0, n_out1;
    op_outputs(f, n_out0, n_out1);
    if (f.kind == FK_LEAF) { row(f.src0, f.n_s0); continue; }
    if (f.flags & FF_SRC_VEC) row(f.src0, f.n_s0); else stt(f.src0, f.n_s0);
    stt(f.src1, f.n_s1);
    if (f.flags & FF_OUT_VEC) row(f.out0, n_out0); else stt(f.out0, n_out0);
    stt(f.out1, n_out1);
  }
  if (sp.row_lo > sp.row_hi) sp.row_lo = sp.row_hi = 0;
  if (sp.st_lo > sp.st_hi) sp.st_lo = sp.st_hi = 0;
  return sp;
}
}  // namespace

void annotate_segments(std::vector<DSeg>& segs, const FlatProgram& fp) {
  // st_cross: a single-CTA run that keeps its state in shared memory must
  // produce every state entry it reads and consume every entry it writes.
  {
    int32_t st_len = 0;
    for (const FlatOp& f : fp.ops) {
      if (f.kind == FK_LEAF) continue;
      int n0o, n1o;
      op_outputs(f, n0o, n1o);
      if (!(f.flags & FF_SRC_VEC)) st_len = std::max(st_len, f.src0 + f.n_s0);
      if (f.n_s1 > 0) st_len = std::max(st_len, f.src1 + f.n_s1);
      if (!(f.flags & FF_OUT_VEC)) st_len = std::max(st_len, f.out0 + n0o);
      if (n1o > 0) st_len = std::max(st_len, f.out1 + n1o);
    }
    std::vector<int32_t> writer((size_t)st_len, -1);   // segment that last wrote each state entry
    for (size_t si = 0; si < segs.size(); ++si) segs[si].st_cross = 0;
    for (size_t si = 0; si < segs.size(); ++si) {
      DSeg& sg = segs[si];
      for (int32_t o = fp.base[sg.first]; o < fp.base[sg.first + sg.count]; ++o) {
        const FlatOp& f = fp.ops[o];
        if (f.kind == FK_LEAF) continue;
        auto rd = [&](int32_t a, int32_t n) {
          for (int32_t e = a; e < a + n; ++e) {
            const int32_t w = writer[(size_t)e];
            if (w != (int32_t)si) {
              sg.st_cross = 1;
              if (w >= 0) segs[(size_t)w].st_cross = 1;
            }
          }
        };
        if (!(f.flags & FF_SRC_VEC)) rd(f.src0, f.n_s0);
        if (f.n_s1 > 0) rd(f.src1, f.n_s1);
        int n0o, n1o;
        op_outputs(f, n0o, n1o);
        if (!(f.flags & FF_OUT_VEC)) for (int32_t e = f.out0; e < f.out0 + n0o; ++e) writer[(size_t)e] = (int32_t)si;
        for (int32_t e = f.out1; e < f.out1 + n1o; ++e) writer[(size_t)e] = (int32_t)si;
      }
    }
  }
  for (DSeg& sg : segs) {
    sg.row_lo = sg.st_lo = sg.row_hi = sg.st_hi = 0;
    if (sg.grid) continue;
    bool rows = false, st = false;
    for (int ph = sg.first; ph < sg.first + sg.count; ++ph) {
      const Span v = phase_span(fp, ph);
      if (v.row_hi > v.row_lo) {
        if (!rows) { sg.row_lo = v.row_lo; sg.row_hi = v.row_hi; rows = true; }
        else { sg.row_lo = std::min(sg.row_lo, v.row_lo); sg.row_hi = std::max(sg.row_hi, v.row_hi); }
      }
      if (v.st_hi > v.st_lo) {
        if (!st) { sg.st_lo = v.st_lo; sg.st_hi = v.st_hi; st = true; }
        else { sg.st_lo = std::min(sg.st_lo, v.st_lo); sg.st_hi = std::max(sg.st_hi, v.st_hi); }
      }
    }
  }
}

std::vector<DSeg> segment_program(const std::vector<DPhase>& prog, const FlatProgram& fp, int grid_min,
                                  int64_t res_entries) {
  std::vector<DSeg> segs;
  int n = (int)prog.size();
  int i = 0;
  // grid-wide: many ops, or vector operands too wide for a warp's staging slice
  auto big = [&](const DPhase& P) { return P.kind != PH_LEAF && (P.count >= grid_min || P.vmax > 128); };
  while (i < n) {
    if (big(prog[i])) {
      segs.push_back(DSeg{1, i, 1, 0, 0, 0, 0, 0});
      ++i;
      continue;
    }
    int j = i;
    while (j < n && !big(prog[j])) ++j;
    if (res_entries <= 0) {
      segs.push_back(DSeg{0, i, j - i, 0, 0, 0, 0, 0});
      i = j;
      continue;
    }
    // cut the run so that each piece's rows + state entries fit the budget;
    // cuts fall between atoms (a leaf solve, or a butterfly from its entry
    // phase to its exit phase), so that a piece holds whole butterflies (an
    // atom that alone exceeds the budget forms a piece of its own)
    auto atom_end = [&](int p) {
      if (prog[p].kind != PH_ENTER) return p + 1;
      int q = p + 1;
      while (q < j && !(prog[q].kind == PH_EXIT && prog[q].arg0 == prog[p].arg0)) ++q;
      return q < j ? q + 1 : j;
    };
    auto atom_span = [&](int p, int e) {
      Span u = phase_span(fp, p);
      for (int q = p + 1; q < e; ++q) {
        Span v = phase_span(fp, q);
        if (v.row_hi > v.row_lo) {
          if (u.row_hi <= u.row_lo) { u.row_lo = v.row_lo; u.row_hi = v.row_hi; }
          else { u.row_lo = std::min(u.row_lo, v.row_lo); u.row_hi = std::max(u.row_hi, v.row_hi); }
        }
        if (v.st_hi > v.st_lo) {
          if (u.st_hi <= u.st_lo) { u.st_lo = v.st_lo; u.st_hi = v.st_hi; }
          else { u.st_lo = std::min(u.st_lo, v.st_lo); u.st_hi = std::max(u.st_hi, v.st_hi); }
        }
      }
      return u;
    };
    int s0 = i;
    int ae = atom_end(i);
    Span cur = atom_span(i, ae);
    for (int p = ae; p <= j; p = ae) {
      bool cut = (p == j);
      Span nx{};
      if (!cut) {
        ae = atom_end(p);
        nx = atom_span(p, ae);
        auto lo = [](int32_t a, int32_t b, int32_t ha, int32_t hb) {
          if (ha <= a) return b;           // empty span a
          if (hb <= b) return a;
          return std::min(a, b);
        };
        auto hi = [](int32_t a, int32_t b, int32_t la, int32_t lb) {
          if (a <= la) return b;
          if (b <= lb) return a;
          return std::max(a, b);
        };
        Span u{lo(cur.row_lo, nx.row_lo, cur.row_hi, nx.row_hi), hi(cur.row_hi, nx.row_hi, cur.row_lo, nx.row_lo),
               lo(cur.st_lo, nx.st_lo, cur.st_hi, nx.st_hi), hi(cur.st_hi, nx.st_hi, cur.st_lo, nx.st_lo)};
        const int64_t foot = (int64_t)(u.row_hi - u.row_lo) + (int64_t)(u.st_hi - u.st_lo);
        const int64_t nops = (int64_t)fp.base[ae] - fp.base[s0];
        if (foot > res_entries || nops > kRunMaxOps || ae - s0 > kRunMaxPhases) cut = true;
        else cur = u;
      }
      if (cut) {
        segs.push_back(DSeg{0, s0, p - s0, 0, 0, 0, 0, 0});
        s0 = p;
        if (p < j) cur = nx;
      }
      if (p == j) break;
    }
    i = j;
  }
  annotate_segments(segs, fp);
  return segs;
}

void host_apply(const PackedHost& ph, const HostFactor& hf, bool adj, const cplx* x, cplx* y) {
  HostExec ex(ph, hf);
  ex.apply(adj, x, y);
}

void host_apply_items(const PackedHost& ph, const HostFactor& hf, bool adj, std::vector<cplx>& st) {
  HostExec ex(ph, hf);
  ex.st = st;
  const std::vector<int32_t>& ptr = adj ? ph.astep_ptr : ph.step_ptr;
  const std::vector<int32_t>& ix = adj ? ph.astep_idx : ph.step_idx;
  for (size_t s = 0; s + 1 < ptr.size(); ++s)
    for (int32_t e = ptr[s]; e < ptr[s + 1]; ++e) ex.item(ph.items[ix[e]], adj);
  st = ex.st;
}
void host_sweep(const PackedHost& ph, const HostFactor& hf, int which, cplx* vec) {
  HostExec ex(ph, hf);
  ex.sweep(which, vec);
}

}  // namespace hb

// Plan of the persistent single-column apply (Alg. 2 for one right-hand
// side) and its host executor.
//
// The plan lists, per CTA, the staging batches of every phase (see
// ApplyPlan in hb_internal.h).  Phases follow the data dependences of
// Alg. 2: the entry ops V0 (column leaves -> first butterfly stage), the
// inner butterfly stages one global step at a time, then the exit ops U0
// (last stage -> row leaves) summed over the depths v = 0..D-1 after the
// dense diagonal leaf product.  Inside a phase no op reads what another op
// of the same phase writes, except the chained chunks of one dense leaf or
// one row leaf, which are placed in consecutive phases.
#include <algorithm>
#include <cstring>

#include "hb_internal.h"

namespace hb {

namespace {

int64_t a16(int64_t b) { return (b + 15) & ~(int64_t)15; }

struct TaskDraft {
  std::vector<FlatOp> ops;
  std::vector<uint32_t> gl;     // gather-list entries of the task
  int kind = 0;
  int64_t fbytes = 0;           // factor / index bytes
};

// staging bytes of one op's blocks (matrix, then indices, each 16-byte aligned)
int64_t op_fbytes(const FlatOp& f, int fes) {
  return a16((int64_t)f.melems * fes) + (f.ioff >= 0 ? a16((int64_t)f.ielems * 2) : 0);
}

// area of a task: blocks + gather list (4 bytes per entry) + staged entries (16 bytes each)
int64_t task_area(const TaskDraft& t) { return t.fbytes + 4 * (int64_t)t.gl.size() + 16 * (int64_t)t.gl.size(); }

}  // namespace

void build_apply_plan(const PackedHost& ph, bool adj, int G, int fes, int max_area, ApplyPlan& plan) {
  plan = ApplyPlan();
  const int D = ph.depth;
  const int64_t m = ph.m, n0 = ph.n0;
  const std::vector<int32_t>& ptr = adj ? ph.astep_ptr : ph.step_ptr;
  const std::vector<int32_t>& sidx = adj ? ph.astep_idx : ph.step_idx;
  const int S = (int)ptr.size() - 1;                    // inner steps
  const int64_t task_max = std::max<int64_t>(max_area / 2, 4096);
  auto blkm = [](const DBlk& b) { return (int64_t)b.k * (b.c - b.k); };

  // ---- drafts per phase
  std::vector<std::vector<TaskDraft>> phases(1 + S);
  // entry ops (one task per leaf, split if its blocks do not fit a task area)
  for (int64_t j = 0; j < m; ++j) {
    TaskDraft t;
    t.kind = 0;
    auto flush = [&]() {
      if (!t.ops.empty()) phases[0].push_back(t);
      t = TaskDraft();
      t.kind = 0;
    };
    for (int v = 0; v < D; ++v) {
      const DOuter& o = adj ? ph.uout[(size_t)j * D + v] : ph.vout[(size_t)j * D + v];
      FlatOp f{};
      f.kind = FK_GATHER;
      f.flags = (int16_t)((adj ? FF_CONJ : 0) | FF_SRC_VEC);
      f.moff = o.blk.moff;
      f.melems = (int32_t)blkm(o.blk);
      f.ioff = o.blk.ioff;
      f.ielems = (int16_t)(2 * o.blk.c);
      f.k0 = o.blk.k;
      f.c0 = o.blk.c;
      f.src0 = (int32_t)(j * n0);
      f.n_s0 = (int16_t)n0;
      f.out0 = o.seg_off;
      const int64_t fb = op_fbytes(f, fes);
      if (!t.ops.empty() && t.fbytes + fb + 20 * n0 > task_max) flush();
      if (t.ops.empty())
        for (int64_t r = 0; r < n0; ++r) t.gl.push_back(kA1FromX | (uint32_t)(j * n0 + r));
      f.pad = 0;   // the leaf's x rows, staged once per task
      t.fbytes += fb;
      t.ops.push_back(f);
    }
    flush();
  }
  // dense leaves: column chunks, chunk c in phase c (forward chunks accumulate)
  int64_t nc = std::max<int64_t>(1, (int64_t)8192 / ((int64_t)fes * n0) * 2);   // <= 16 KB of matrix
  nc = std::min<int64_t>(nc, n0);
  nc = std::max<int64_t>(nc, (n0 + S) / (S + 1));
  const int64_t nchunk = (n0 + nc - 1) / nc;
  if (nchunk > S + 1) plan.ok = false;
  for (int64_t l = 0; l < m; ++l)
    for (int64_t c = 0; c < nchunk; ++c) {
      const int64_t cb = c * nc, cn = std::min<int64_t>(nc, n0 - cb);
      TaskDraft t;
      t.kind = 2;
      FlatOp f{};
      f.kind = FK_DLEAF;
      f.moff = l * n0 * n0 + cb * n0;
      f.melems = (int32_t)(cn * n0);
      f.ioff = -1;
      f.c0 = (int16_t)n0;
      f.c1 = (int16_t)cb;
      f.k1 = (int16_t)cn;
      f.flags = (int16_t)(FF_SRC_VEC | FF_OUT_VEC | (adj ? FF_ADJ : 0) | (!adj && c > 0 ? FF_ACC : 0));
      // inputs: forward x[cb, cb+cn) of the leaf; adjoint all n0 rows of x
      f.src0 = (int32_t)(l * n0 + (adj ? 0 : cb));
      f.n_s0 = (int16_t)(adj ? n0 : cn);
      f.out0 = (int32_t)(l * n0 + (adj ? cb : 0));
      for (int64_t r = 0; r < f.n_s0; ++r) t.gl.push_back(kA1FromX | (uint32_t)(f.src0 + r));
      f.pad = 0;
      if (f.flags & FF_ACC)   // the rows written by the previous chunk follow the inputs
        for (int64_t r = 0; r < n0; ++r) t.gl.push_back(kA1FromY | (uint32_t)(l * n0 + r));
      t.fbytes = op_fbytes(f, fes);
      t.ops.push_back(f);
      phases[(size_t)c].push_back(t);
    }
  // inner steps: one task per item
  for (int s = 0; s < S; ++s)
    for (int32_t q = ptr[s]; q < ptr[s + 1]; ++q) {
      const DItem& it = ph.items[sidx[q]];
      TaskDraft t;
      t.kind = 1;
      FlatOp f{};
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
        if (i1 < 0 || ie > INT16_MAX || f.m1 < 0) plan.ok = false;
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
      for (int r = 0; r < f.n_s0; ++r) t.gl.push_back((uint32_t)(f.src0 + r));
      for (int r = 0; r < f.n_s1; ++r) t.gl.push_back((uint32_t)(f.src1 + r));
      f.pad = 0;
      t.fbytes = op_fbytes(f, fes);
      t.ops.push_back(f);
      phases[(size_t)s + 1].push_back(t);
    }
  // exit ops: per row leaf, the depths in order, chained chunks in consecutive phases
  std::vector<std::vector<TaskDraft>> exits;
  for (int64_t i = 0; i < m; ++i) {
    int chunk = 0;
    TaskDraft t;
    t.kind = 3;
    auto flush = [&]() {
      if (t.ops.empty()) return;
      if ((int)exits.size() <= chunk) exits.resize((size_t)chunk + 1);
      exits[(size_t)chunk].push_back(t);
      ++chunk;
      t = TaskDraft();
      t.kind = 3;
    };
    for (int v = 0; v < D; ++v) {
      const DOuter& o = adj ? ph.vout[(size_t)i * D + v] : ph.uout[(size_t)i * D + v];
      FlatOp f{};
      f.kind = FK_SCATTER;
      f.flags = (int16_t)((adj ? FF_CONJ : 0) | FF_OUT_VEC | FF_ACC);
      f.moff = o.blk.moff;
      f.melems = (int32_t)blkm(o.blk);
      f.ioff = o.blk.ioff;
      f.ielems = (int16_t)(2 * o.blk.c);
      f.k0 = o.blk.k;
      f.c0 = o.blk.c;
      f.src0 = o.seg_off;
      f.n_s0 = o.blk.k;
      f.out0 = (int32_t)(i * n0);
      f.split = o.blk.c;
      const int64_t fb = op_fbytes(f, fes);
      if (!t.ops.empty() && t.fbytes + fb + 20 * (n0 + (int64_t)t.gl.size() + f.n_s0) > task_max) flush();
      if (t.ops.empty())   // the rows the leaf product (or the previous chunk) wrote
        for (int64_t r = 0; r < n0; ++r) t.gl.push_back(kA1FromY | (uint32_t)(i * n0 + r));
      f.pad = (int16_t)t.gl.size();
      for (int r = 0; r < f.n_s0; ++r) t.gl.push_back((uint32_t)(f.src0 + r));
      t.fbytes += fb;
      t.ops.push_back(f);
    }
    flush();
  }
  for (auto& e : exits) phases.push_back(std::move(e));
  plan.nphase = (int)phases.size();

  // ---- CTA ranges (balanced by area) and batches
  std::vector<std::vector<A1Batch>> per_cta((size_t)G);
  struct BatchDraft { int phase; std::vector<const TaskDraft*> tasks; };
  std::vector<std::vector<BatchDraft>> bd((size_t)G);
  const int64_t batch_target = std::max<int64_t>(max_area / 4, 8192);
  for (int p = 0; p < plan.nphase; ++p) {
    const std::vector<TaskDraft>& tl = phases[(size_t)p];
    int64_t total = 0;
    for (const TaskDraft& t : tl) {
      const int64_t a = task_area(t);
      if (a + 16 > max_area) plan.ok = false;
      total += a;
    }
    size_t ti = 0;
    int64_t acc = 0;
    for (int g = 0; g < G; ++g) {
      const int64_t goal = (total * (int64_t)(g + 1)) / G;
      BatchDraft cur{p, {}};
      int64_t cur_area = 0;
      while (ti < tl.size() && (acc < goal || g == G - 1)) {
        const int64_t a = task_area(tl[ti]);
        if (!cur.tasks.empty() && cur_area + a > batch_target) {
          bd[(size_t)g].push_back(cur);
          cur = BatchDraft{p, {}};
          cur_area = 0;
        }
        cur.tasks.push_back(&tl[ti]);
        cur_area += a + 64;
        acc += a;
        ++ti;
      }
      if (!cur.tasks.empty()) bd[(size_t)g].push_back(cur);
    }
  }
  // ---- flatten: ops, tasks, batches, gather lists with staging offsets
  plan.cta_batch.assign((size_t)G + 1, 0);
  for (int g = 0; g < G; ++g) {
    plan.cta_batch[(size_t)g] = (int32_t)plan.batches.size();
    for (const BatchDraft& b : bd[(size_t)g]) {
      A1Batch B{};
      B.phase = b.phase;
      B.task0 = (int32_t)plan.tasks.size();
      B.ntasks = (int32_t)b.tasks.size();
      int64_t off = 0;
      int32_t nvec = 0;
      for (const TaskDraft* t : b.tasks) {
        A1Task T{};
        T.op0 = (int32_t)plan.ops.size();
        T.nops = (int32_t)t->ops.size();
        T.kind = t->kind;
        T.pad = nvec;   // first staged entry of the task
        for (FlatOp f : t->ops) {
          f.soff = (int32_t)off;
          off += op_fbytes(f, fes);
          f.pad = (int16_t)(f.pad + 0);   // relative to the task's first staged entry
          plan.ops.push_back(f);
        }
        plan.tasks.push_back(T);
        for (uint32_t e : t->gl) plan.gl.push_back(e);
        nvec += (int32_t)t->gl.size();
      }
      while (plan.gl.size() % 4) plan.gl.push_back(0);   // 16-byte aligned lists (entry 0: a valid state index)
      B.gl_off = (int32_t)off;
      B.nvec = nvec;
      B.gl_src = (int64_t)plan.gl.size() - (int64_t)((nvec + 3) / 4 * 4);
      off += a16(4 * (int64_t)nvec);
      B.tma_bytes = (int32_t)off;
      B.vec_off = (int32_t)off;
      off += 16 * (int64_t)nvec;
      B.area_bytes = (int32_t)a16(off);
      if (B.area_bytes > max_area) plan.ok = false;
      plan.max_area = std::max(plan.max_area, B.area_bytes);
      plan.batches.push_back(B);
    }
  }
  plan.cta_batch[(size_t)G] = (int32_t)plan.batches.size();
  for (int i = 0; i < 16; ++i) plan.gl.push_back(0);     // tail: 16-byte bulk copies stay inside
}

// ---------------------------------------------------------------------------
// Host executor of a plan (FP64): runs every phase, CTA and batch in order,
// staging the vector entries through the gather lists exactly as the kernel
// does, so a wrong offset, list or chain order shows up against host_apply.
// ---------------------------------------------------------------------------
void host_apply_plan(const PackedHost& ph, const HostFactor& hf, const ApplyPlan& plan, bool adj, const cplx* x,
                     cplx* y) {
  const int64_t n0 = ph.n0;
  std::vector<cplx> st((size_t)ph.state_len, cplx(0.0));
  std::fill(y, y + ph.n, cplx(std::nan(""), 0.0));
  const int G = (int)plan.cta_batch.size() - 1;
  auto M = [&](const FlatOp& f, int64_t e) { return ph.fpool[(size_t)(f.moff + e)]; };
  auto I = [&](const FlatOp& f, int64_t e) { return ph.ipool[(size_t)(f.ioff + e)]; };
  auto leafm = [&](const FlatOp& f, int64_t r, int64_t c) {   // device layout: [leaf][c][r]
    const int64_t l = f.moff / (n0 * n0);
    return hf.leaf[(size_t)((l * n0 + r) * n0 + c)];
  };
  for (int p = 0; p < plan.nphase; ++p) {
    for (int g = 0; g < G; ++g) {
      for (int32_t b = plan.cta_batch[(size_t)g]; b < plan.cta_batch[(size_t)g + 1]; ++b) {
        const A1Batch& B = plan.batches[(size_t)b];
        if (B.phase != p) continue;
        std::vector<cplx> sv((size_t)B.nvec);
        for (int e = 0; e < B.nvec; ++e) {
          const uint32_t s = plan.gl[(size_t)(B.gl_src + e)];
          if ((s & kA1FromY) == kA1FromY) sv[(size_t)e] = y[s & 0x3FFFFFFFu];
          else if (s & kA1FromX) sv[(size_t)e] = x[s & 0x3FFFFFFFu];
          else sv[(size_t)e] = st[s];
        }
        for (int32_t t = B.task0; t < B.task0 + B.ntasks; ++t) {
          const A1Task& T = plan.tasks[(size_t)t];
          const cplx* tv = sv.data() + T.pad;
          std::vector<cplx> acc;
          for (int32_t o = T.op0; o < T.op0 + T.nops; ++o) {
            const FlatOp& f = plan.ops[(size_t)o];
            const cplx* in = tv + f.pad;
            if (f.kind == FK_DLEAF) {
              const int64_t cb = f.c1, cn = f.k1;
              if (!adj) {
                for (int64_t r = 0; r < n0; ++r) {
                  cplx a = (f.flags & FF_ACC) ? tv[f.n_s0 + r] : cplx(0.0);
                  for (int64_t c = 0; c < cn; ++c) a += leafm(f, r, cb + c) * in[c];
                  y[(size_t)(f.out0 + r)] = a;
                }
              } else {
                for (int64_t c = 0; c < cn; ++c) {
                  cplx a = 0.0;
                  for (int64_t r = 0; r < n0; ++r) a += std::conj(leafm(f, r, cb + c)) * in[r];
                  y[(size_t)(f.out0 + c)] = a;
                }
              }
            } else if (f.kind == FK_GATHER) {
              const bool cj = (f.flags & FF_CONJ) != 0;
              for (int s2 = 0; s2 < ((f.flags & FF_TWO) ? 2 : 1); ++s2) {
                const int k = s2 ? f.k1 : f.k0, c = s2 ? f.c1 : f.c0, nr = c - k;
                const int64_t mo = s2 ? f.m1 : 0, io = s2 ? f.i1 : 0;
                const int32_t out = s2 ? f.out1 : f.out0;
                for (int i = 0; i < k; ++i) {
                  cplx a = in[I(f, io + i)];
                  for (int j = 0; j < nr; ++j) {
                    cplx mm = cj ? std::conj(M(f, mo + (int64_t)i * nr + j)) : M(f, mo + (int64_t)j * k + i);
                    a += mm * in[I(f, io + k + j)];
                  }
                  st[(size_t)(out + i)] = a;
                }
              }
            } else if (f.kind == FK_SCATTER) {
              const bool cj = (f.flags & FF_CONJ) != 0;
              const int nrow = f.c0;
              if (f.flags & FF_ACC) {
                if (acc.empty()) acc.assign(tv, tv + n0);
              }
              for (int r = 0; r < nrow; ++r) {
                cplx a = 0.0;
                for (int s2 = 0; s2 < ((f.flags & FF_TWO) ? 2 : 1); ++s2) {
                  const int k = s2 ? f.k1 : f.k0, c = s2 ? f.c1 : f.c0, nr = c - k;
                  const int64_t mo = s2 ? f.m1 : 0, io = s2 ? f.i1 : 0;
                  const cplx* yy = in + (s2 ? f.n_s0 : 0);
                  const int code = I(f, io + c + r);
                  if (code >= 0) a += yy[code];
                  else {
                    const int j = -1 - code;
                    for (int i = 0; i < k; ++i) {
                      cplx mm = cj ? std::conj(M(f, mo + (int64_t)j * k + i)) : M(f, mo + (int64_t)i * nr + j);
                      a += mm * yy[i];
                    }
                  }
                }
                if (f.flags & FF_ACC) acc[(size_t)r] += a;
                else if (!(f.flags & FF_TWO) || r < f.split) st[(size_t)(f.out0 + r)] = a;
                else st[(size_t)(f.out1 + r - f.split)] = a;
              }
            } else {   // middle
              const int kr = f.k0, kc = f.c0;
              const bool a2 = (f.flags & FF_ADJ) != 0;
              const int nin = a2 ? kr : kc, nout = a2 ? kc : kr;
              for (int o2 = 0; o2 < nout; ++o2) {
                cplx a = 0.0;
                for (int i = 0; i < nin; ++i)
                  a += (a2 ? std::conj(M(f, (int64_t)o2 * kr + i)) : M(f, (int64_t)i * kr + o2)) * in[i];
                st[(size_t)(f.out0 + o2)] = a;
              }
            }
          }
          if (!acc.empty()) {
            const FlatOp& f0 = plan.ops[(size_t)T.op0];
            for (int64_t r = 0; r < n0; ++r) y[(size_t)(f0.out0 + r)] = acc[(size_t)r];
          }
        }
      }
    }
  }
}

}  // namespace hb

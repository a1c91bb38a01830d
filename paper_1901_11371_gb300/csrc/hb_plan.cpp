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
#include <functional>

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
int64_t task_area(const TaskDraft& t) {
  return 16 + 64 * (int64_t)t.ops.size() + t.fbytes + 4 * (int64_t)t.gl.size() + 16 * (int64_t)t.gl.size();
}

}  // namespace

void build_apply_plan(const PackedHost& ph, const HostFactor& hf, bool adj, int G, int fes, int max_area,
                      ApplyPlan& plan) {
  plan = ApplyPlan();
  const int D = ph.depth;
  const int64_t m = ph.m, n0 = ph.n0;
  const std::vector<int32_t>& ptr = adj ? ph.astep_ptr : ph.step_ptr;
  const std::vector<int32_t>& sidx = adj ? ph.astep_idx : ph.step_idx;
  const int S = (int)ptr.size() - 1;                    // inner steps
  // batches are consumed one per warp: a batch target of an eighth of the largest area lets
  // the compute warps hold several batches each while the producer fills the rest of the ring;
  // entry and exit tasks are cut to that size (a single larger op gets a batch of its own)
  const int64_t batch_target = std::max<int64_t>(max_area / 8, 4096);
  const int64_t task_max = batch_target;
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
  // (at most half a batch of matrix per chunk; at least four chunks when there are phases for them, so
  // that the independent leaf products spread over the first inner phases)
  int64_t nc = std::max<int64_t>(1, batch_target / 2 / ((int64_t)fes * n0));
  nc = std::min<int64_t>(nc, (n0 + 3) / 4);
  nc = std::max<int64_t>(nc, (n0 + S) / (S + 1));
  nc = std::max<int64_t>(1, std::min<int64_t>(nc, n0));
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
      // (exit tasks may fill half an area: their rows run in parallel, and every extra chunk
      // costs a phase)
      if (!t.ops.empty() && t.fbytes + fb + 20 * (n0 + (int64_t)t.gl.size() + f.n_s0) > max_area / 2) flush();
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

  // ---- CTA assignment and batches.  Every task goes to the CTA with the least work so far
  // (work = staging bytes plus a per-output-row charge), so that each CTA of a phase gets a
  // mix of the phase's task kinds and about the same time; a CTA's tasks are then cut into
  // batches of about batch_target bytes and at most kA1MaxTasks tasks.
  struct BatchDraft { int phase; std::vector<const TaskDraft*> tasks; };
  std::vector<std::vector<BatchDraft>> bd((size_t)G);
  auto task_rows = [&](const TaskDraft& t) {
    int64_t r = 0;
    for (const FlatOp& f : t.ops) {
      if (t.kind == 3) return (int64_t)n0;
      if (f.kind == FK_GATHER) r += f.k0 + ((f.flags & FF_TWO) ? f.k1 : 0);
      else if (f.kind == FK_SCATTER) r += f.c0;
      else if (f.kind == FK_MIDDLE) r += (f.flags & FF_ADJ) ? f.c0 : f.k0;
      else r += (f.flags & FF_ADJ) ? f.k1 : n0;
    }
    return r;
  };
  for (int p = 0; p < plan.nphase; ++p) {
    const std::vector<TaskDraft>& tl = phases[(size_t)p];
    std::vector<std::vector<const TaskDraft*>> mine((size_t)G);
    // min-heap of (work, cta)
    std::vector<std::pair<int64_t, int>> heap;
    for (int g = 0; g < G; ++g) heap.push_back({0, g});
    std::make_heap(heap.begin(), heap.end(), std::greater<std::pair<int64_t, int>>());
    for (const TaskDraft& t : tl) {
      const int64_t a = task_area(t);
      if (a + 16 > max_area) plan.ok = false;
      std::pop_heap(heap.begin(), heap.end(), std::greater<std::pair<int64_t, int>>());
      auto& top = heap.back();
      mine[(size_t)top.second].push_back(&t);
      top.first += a + 96 * task_rows(t);
      std::push_heap(heap.begin(), heap.end(), std::greater<std::pair<int64_t, int>>());
    }
    for (int g = 0; g < G; ++g) {
      // a phase with little work per CTA gets smaller batches, so that every compute warp
      // takes part (about two batches per warp)
      int64_t mine_area = 0;
      for (const TaskDraft* t : mine[(size_t)g]) mine_area += task_area(*t);
      const int64_t target = std::max<int64_t>(2048, std::min<int64_t>(batch_target, mine_area / (2 * kA1Warps)));
      BatchDraft cur{p, {}};
      int64_t cur_area = 0;
      for (const TaskDraft* t : mine[(size_t)g]) {
        const int64_t a = task_area(*t);
        if (!cur.tasks.empty() && (cur_area + a > target || (int)cur.tasks.size() >= kA1MaxTasks)) {
          bd[(size_t)g].push_back(cur);
          cur = BatchDraft{p, {}};
          cur_area = 0;
        }
        cur.tasks.push_back(t);
        cur_area += a;
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
      B.op0 = (int32_t)plan.ops.size();
      int32_t nops = 0;
      for (const TaskDraft* t : b.tasks) nops += (int32_t)t->ops.size();
      B.nops = nops;
      B.rec_off = (int32_t)(16 * (int64_t)B.ntasks);
      int64_t off = B.rec_off + 64 * (int64_t)nops;
      int32_t nvec = 0;
      // independent-op tasks first (their ops spread over the warps), then the one-warp tasks
      std::vector<const TaskDraft*> order;
      for (const TaskDraft* t : b.tasks) if (t->kind <= 1) order.push_back(t);
      B.nptask = (int32_t)order.size();
      B.npar = 0;
      for (const TaskDraft* t : order) B.npar += (int32_t)t->ops.size();
      for (const TaskDraft* t : b.tasks) if (t->kind > 1) order.push_back(t);
      for (const TaskDraft* t : order) {
        A1Task T{};
        T.op0 = (int32_t)plan.ops.size();
        T.nops = (int32_t)t->ops.size();
        T.kind = t->kind;
        T.pad = nvec;   // first staged entry of the task
        for (FlatOp f : t->ops) {
          f.soff = (int32_t)off;
          off += op_fbytes(f, fes);
          if (nvec + f.pad > INT16_MAX) plan.ok = false;
          f.pad = (int16_t)(nvec + f.pad);   // batch-relative
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
      B.dep_off = (int32_t)off;   // producer list, sized below
      plan.batches.push_back(B);
    }
  }
  plan.cta_batch[(size_t)G] = (int32_t)plan.batches.size();
  for (int i = 0; i < 16; ++i) plan.gl.push_back(0);     // tail: 16-byte bulk copies stay inside
  // ---- producers: a batch waits only for the batches (of earlier phases, any CTA) that
  // wrote the state entries and y rows it gathers, instead of for every CTA at a grid
  // barrier.  Writers are tracked phase by phase (the last writer before the phase).
  {
    const int64_t nb = (int64_t)plan.batches.size();
    std::vector<std::vector<int32_t>> byph((size_t)plan.nphase);
    for (int64_t b = 0; b < nb; ++b) byph[(size_t)plan.batches[(size_t)b].phase].push_back((int32_t)b);
    std::vector<int32_t> wst((size_t)std::max<int64_t>(ph.state_len, 1), -1), wy((size_t)ph.n, -1);
    std::vector<std::vector<int32_t>> dl((size_t)nb);
    for (int p = 0; p < plan.nphase; ++p) {
      for (int32_t b : byph[(size_t)p]) {
        const A1Batch& B = plan.batches[(size_t)b];
        std::vector<int32_t>& d = dl[(size_t)b];
        for (int32_t e = 0; e < B.nvec; ++e) {
          const uint32_t s = plan.gl[(size_t)(B.gl_src + e)];
          int32_t w = -1;
          if ((s & kA1FromY) == kA1FromY) w = wy[(size_t)(s & 0x3FFFFFFFu)];
          else if (!(s & kA1FromX)) w = wst[(size_t)s];
          if (w >= 0) d.push_back(w);
        }
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
      }
      for (int32_t b : byph[(size_t)p]) {
        const A1Batch& B = plan.batches[(size_t)b];
        auto st_range = [&](int64_t a, int64_t c) { for (int64_t i = a; i < a + c && i < (int64_t)wst.size(); ++i) wst[(size_t)i] = b; };
        auto y_range = [&](int64_t a, int64_t c) { for (int64_t i = a; i < a + c && i < ph.n; ++i) wy[(size_t)i] = b; };
        for (int32_t t = B.task0; t < B.task0 + B.ntasks; ++t) {
          const A1Task& T = plan.tasks[(size_t)t];
          if (T.kind == 3) {   // exit: the leaf's n0 rows of y
            y_range(plan.ops[(size_t)(T.op0 + T.nops - 1)].out0, n0);
            continue;
          }
          for (int32_t o = T.op0; o < T.op0 + T.nops; ++o) {
            const FlatOp& f = plan.ops[(size_t)o];
            const bool fadj = (f.flags & FF_ADJ) != 0;
            if (f.kind == FK_GATHER) {
              st_range(f.out0, f.k0);
              if (f.flags & FF_TWO) st_range(f.out1, f.k1);
            } else if (f.kind == FK_SCATTER) {
              const bool two = (f.flags & FF_TWO) != 0;
              st_range(f.out0, two ? f.split : f.c0);
              if (two) st_range(f.out1, f.c0 - f.split);
            } else if (f.kind == FK_MIDDLE) {
              st_range(f.out0, fadj ? f.c0 : f.k0);
            } else if (f.kind == FK_DLEAF) {
              y_range(f.out0, fadj ? f.k1 : n0);
            }
          }
        }
      }
    }
    for (int64_t b = 0; b < nb; ++b) {
      A1Batch& B = plan.batches[(size_t)b];
      B.dep_src = (int32_t)plan.deps.size();
      B.ndep = (int32_t)dl[(size_t)b].size();
      for (int32_t w : dl[(size_t)b]) plan.deps.push_back(w);
      int64_t off = B.dep_off + a16(4 * (int64_t)B.ndep);
      B.tma_bytes = (int32_t)off;
      B.vec_off = (int32_t)off;
      off += 16 * (int64_t)B.nvec;
      B.area_bytes = (int32_t)a16(off);
      if (B.area_bytes > max_area) plan.ok = false;
      plan.max_area = std::max(plan.max_area, B.area_bytes);
    }
  }
  if (plan.ok) plan.ok = check_apply_plan(plan, ph, fes, max_area);
  if (!plan.ok) return;
  // ---- batch images
  int64_t total = 0;
  for (A1Batch& B : plan.batches) {
    B.img = total;
    total += B.tma_bytes;
  }
  plan.image.assign((size_t)total, 0);
  auto put_elem = [&](uint8_t* dst, cplx v) {
    if (fes == 16) {
      const double d[2] = {v.real(), v.imag()};
      std::memcpy(dst, d, 16);
    } else {
      const float f[2] = {(float)v.real(), (float)v.imag()};
      std::memcpy(dst, f, 8);
    }
  };
  for (const A1Batch& B : plan.batches) {
    uint8_t* base = plan.image.data() + B.img;
    std::memcpy(base, &plan.tasks[(size_t)B.task0], 16 * (size_t)B.ntasks);
    std::memcpy(base + B.rec_off, &plan.ops[(size_t)B.op0], 64 * (size_t)B.nops);
    for (int32_t o = B.op0; o < B.op0 + B.nops; ++o) {
      const FlatOp& f = plan.ops[(size_t)o];
      uint8_t* d = base + f.soff;
      if (f.kind == FK_DLEAF) {
        // device layout [leaf][c][r]: the chunk's columns one after the other
        const int64_t l = f.moff / (ph.n0 * ph.n0), cb = f.c1;
        for (int64_t cc = 0; cc < f.k1; ++cc)
          for (int64_t r = 0; r < ph.n0; ++r)
            put_elem(d + (cc * ph.n0 + r) * fes, hf.leaf[(size_t)((l * ph.n0 + r) * ph.n0 + cb + cc)]);
      } else {
        for (int64_t e = 0; e < f.melems; ++e) put_elem(d + e * fes, ph.fpool[(size_t)(f.moff + e)]);
      }
      if (f.ioff >= 0)
        std::memcpy(d + a16((int64_t)f.melems * fes), &ph.ipool[(size_t)f.ioff], 2 * (size_t)f.ielems);
    }
    std::memcpy(base + B.gl_off, &plan.gl[(size_t)B.gl_src], 4 * (size_t)B.nvec);
    if (B.ndep > 0) std::memcpy(base + B.dep_off, &plan.deps[(size_t)B.dep_src], 4 * (size_t)B.ndep);
  }
}

bool check_apply_plan(const ApplyPlan& plan, const PackedHost& ph, int fes, int max_area) {
  const int64_t nst = ph.state_len, n = ph.n, n0 = ph.n0;
  const int G = (int)plan.cta_batch.size() - 1;
  if (G < 1 || plan.cta_batch[0] != 0 || plan.cta_batch[(size_t)G] != (int32_t)plan.batches.size()) return false;
  const int64_t fpool = (int64_t)ph.fpool.size(), ipool = (int64_t)ph.ipool.size(), leaf = ph.m * n0 * n0;
  for (int g = 0; g < G; ++g) {
    int last_phase = -1;
    for (int32_t b = plan.cta_batch[(size_t)g]; b < plan.cta_batch[(size_t)g + 1]; ++b) {
      const A1Batch& B = plan.batches[(size_t)b];
      if (B.phase < last_phase || B.phase >= plan.nphase) return false;   // phase order per CTA
      last_phase = B.phase;
      if (B.area_bytes > max_area || B.area_bytes < B.tma_bytes || (B.area_bytes & 15)) return false;
      if (B.rec_off != 16 * B.ntasks || (B.gl_off & 15) || (B.vec_off & 15)) return false;
      if (B.ntasks < 1 || B.ntasks > kA1MaxTasks || B.nvec > INT16_MAX) return false;
      if (B.vec_off + 16 * (int64_t)B.nvec > B.area_bytes || B.gl_off + 4 * (int64_t)B.nvec > B.tma_bytes) return false;
      if (B.gl_src < 0 || (B.gl_src & 3) || B.gl_src + (B.nvec + 3) / 4 * 4 + 16 > (int64_t)plan.gl.size()) return false;
      if (B.op0 < 0 || B.op0 + B.nops > (int32_t)plan.ops.size()) return false;
      int64_t bytes = B.rec_off + 64 * (int64_t)B.nops;
      int32_t op_next = B.op0;
      for (int32_t t = B.task0; t < B.task0 + B.ntasks; ++t) {
        const A1Task& T = plan.tasks[(size_t)t];
        if (T.op0 != op_next || T.nops < 1) return false;
        op_next += T.nops;
        for (int32_t o = T.op0; o < T.op0 + T.nops; ++o) {
          const FlatOp& f = plan.ops[(size_t)o];
          const int64_t mb = a16((int64_t)f.melems * fes), ib = f.ioff >= 0 ? a16((int64_t)f.ielems * 2) : 0;
          if (f.soff != bytes || (f.soff & 15)) return false;
          bytes += mb + ib;
          if (f.kind == FK_DLEAF) {
            if (f.moff < 0 || f.moff + a16((int64_t)f.melems * fes) / fes > leaf || ((f.moff * fes) & 15)) return false;
          } else if (f.moff < 0 || f.moff + mb / fes > fpool + 4 || ((f.moff * fes) & 15)) {
            return false;
          }
          if (f.ioff >= 0 && ((f.ioff & 7) || f.ioff + ib / 2 > ipool)) return false;
          const int64_t first = f.pad, cnt = f.n_s0 + f.n_s1 + ((f.flags & FF_ACC) && f.kind == FK_DLEAF ? n0 : 0);
          if ((T.kind <= 1) != (t < B.task0 + B.nptask)) return false;
          if (first < 0 || first + cnt > B.nvec) return false;
          // gather-list entries in range
          for (int64_t e = first; e < first + cnt; ++e) {
            const uint32_t s = plan.gl[(size_t)(B.gl_src + e)];
            if ((s & kA1FromY) == kA1FromY) { if ((int64_t)(s & 0x3FFFFFFFu) >= n) return false; }
            else if (s & kA1FromX) { if ((int64_t)(s & 0x3FFFFFFFu) >= n) return false; }
            else if ((int64_t)s >= nst) return false;
          }
          const bool outv = (f.flags & FF_OUT_VEC) != 0;
          const int64_t lim = outv ? n : nst;
          if (f.out0 < 0 || f.out0 >= lim || f.out1 < 0 || f.out1 >= std::max<int64_t>(nst, 1)) return false;
        }
      }
      if (op_next != B.op0 + B.nops || bytes != B.gl_off) return false;
      if (B.nptask < 0 || B.nptask > B.ntasks || B.npar < 0 || B.npar > B.nops) return false;
      // producer list: right after the gather list, earlier phases only
      if (B.dep_off != B.gl_off + a16(4 * (int64_t)B.nvec) || B.ndep < 0) return false;
      if (B.dep_off + 4 * (int64_t)B.ndep > B.tma_bytes || B.vec_off != B.tma_bytes) return false;
      if (B.dep_src < 0 || B.dep_src + (int64_t)B.ndep > (int64_t)plan.deps.size()) return false;
      for (int32_t k = 0; k < B.ndep; ++k) {
        const int32_t w = plan.deps[(size_t)(B.dep_src + k)];
        if (w < 0 || w >= (int32_t)plan.batches.size() || plan.batches[(size_t)w].phase >= B.phase) return false;
      }
      if (B.nptask < B.ntasks && plan.tasks[(size_t)(B.task0 + B.nptask)].op0 != B.op0 + B.npar) return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Host executor of a plan (FP64): runs every phase, CTA and batch in order,
// staging the vector entries through the gather lists exactly as the kernel
// does, so a wrong offset, list or chain order shows up against host_apply.
// ---------------------------------------------------------------------------
void host_apply_plan(const PackedHost& ph, const ApplyPlan& plan, int fes, bool adj, const cplx* x, cplx* y) {
  const int64_t n0 = ph.n0;
  std::vector<cplx> st((size_t)ph.state_len, cplx(0.0));
  std::fill(y, y + ph.n, cplx(std::nan(""), 0.0));
  const int G = (int)plan.cta_batch.size() - 1;
  auto elem = [&](const uint8_t* p) {
    if (fes == 16) {
      double d[2];
      std::memcpy(d, p, 16);
      return cplx(d[0], d[1]);
    }
    float f[2];
    std::memcpy(f, p, 8);
    return cplx(f[0], f[1]);
  };
  for (int p = 0; p < plan.nphase; ++p) {
    for (int g = 0; g < G; ++g) {
      for (int32_t b = plan.cta_batch[(size_t)g]; b < plan.cta_batch[(size_t)g + 1]; ++b) {
        const A1Batch& B = plan.batches[(size_t)b];
        if (B.phase != p) continue;
        const uint8_t* area = plan.image.data() + B.img;     // what the producer copies in
        std::vector<A1Task> tks((size_t)B.ntasks);
        std::vector<FlatOp> recs((size_t)B.nops);
        std::memcpy(tks.data(), area, 16 * (size_t)B.ntasks);
        std::memcpy(recs.data(), area + B.rec_off, 64 * (size_t)B.nops);
        std::vector<uint32_t> gl((size_t)B.nvec);
        std::memcpy(gl.data(), area + B.gl_off, 4 * (size_t)B.nvec);
        std::vector<cplx> sv((size_t)B.nvec);
        for (int e = 0; e < B.nvec; ++e) {
          const uint32_t s = gl[(size_t)e];
          if ((s & kA1FromY) == kA1FromY) sv[(size_t)e] = y[s & 0x3FFFFFFFu];
          else if (s & kA1FromX) sv[(size_t)e] = x[s & 0x3FFFFFFFu];
          else sv[(size_t)e] = st[s];
        }
        for (int32_t t = 0; t < B.ntasks; ++t) {
          const A1Task& T = tks[(size_t)t];
          const cplx* tv = sv.data() + T.pad;
          std::vector<cplx> acc;
          for (int32_t o = T.op0; o < T.op0 + T.nops; ++o) {
            const FlatOp& f = recs[(size_t)(o - B.op0)];
            const cplx* in = sv.data() + f.pad;
            const uint8_t* mb = area + f.soff;
            const int16_t* ib = (const int16_t*)(area + f.soff + a16((int64_t)f.melems * fes));
            auto M = [&](int64_t e) { return elem(mb + e * fes); };
            auto I = [&](int64_t e) { return ib[e]; };
            if (f.kind == FK_DLEAF) {
              const int64_t cn = f.k1;
              if (!adj) {
                for (int64_t r = 0; r < n0; ++r) {
                  cplx a = (f.flags & FF_ACC) ? in[f.n_s0 + r] : cplx(0.0);
                  for (int64_t c = 0; c < cn; ++c) a += M(c * n0 + r) * in[c];
                  y[(size_t)(f.out0 + r)] = a;
                }
              } else {
                for (int64_t c = 0; c < cn; ++c) {
                  cplx a = 0.0;
                  for (int64_t r = 0; r < n0; ++r) a += std::conj(M(c * n0 + r)) * in[r];
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
                  cplx a = in[I(io + i)];
                  for (int j = 0; j < nr; ++j) {
                    cplx mm = cj ? std::conj(M(mo + (int64_t)i * nr + j)) : M(mo + (int64_t)j * k + i);
                    a += mm * in[I(io + k + j)];
                  }
                  st[(size_t)(out + i)] = a;
                }
              }
            } else if (f.kind == FK_SCATTER) {
              const bool cj = (f.flags & FF_CONJ) != 0;
              const int nrow = f.c0;
              if ((f.flags & FF_ACC) && acc.empty()) acc.assign(tv, tv + n0);
              for (int r = 0; r < nrow; ++r) {
                cplx a = 0.0;
                for (int s2 = 0; s2 < ((f.flags & FF_TWO) ? 2 : 1); ++s2) {
                  const int k = s2 ? f.k1 : f.k0, c = s2 ? f.c1 : f.c0, nr = c - k;
                  const int64_t mo = s2 ? f.m1 : 0, io = s2 ? f.i1 : 0;
                  const cplx* yy = in + (s2 ? f.n_s0 : 0);
                  const int code = I(io + c + r);
                  if (code >= 0) a += yy[code];
                  else {
                    const int j = -1 - code;
                    for (int i = 0; i < k; ++i) {
                      cplx mm = cj ? std::conj(M(mo + (int64_t)j * k + i)) : M(mo + (int64_t)i * nr + j);
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
                  a += (a2 ? std::conj(M((int64_t)o2 * kr + i)) : M((int64_t)i * kr + o2)) * in[i];
                st[(size_t)(f.out0 + o2)] = a;
              }
            }
          }
          if (!acc.empty()) {
            const FlatOp& f0 = recs[(size_t)(T.op0 - B.op0)];
            for (int64_t r = 0; r < n0; ++r) y[(size_t)(f0.out0 + r)] = acc[(size_t)r];
          }
        }
      }
    }
  }
}

}  // namespace hb

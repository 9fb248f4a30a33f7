// hm_plan.cu -- host-side planning: front geometry, HODLR block layout, device arenas and
// the per-level task tables of the factorization and of the preconditioner apply.
// Integer bookkeeping only; all arithmetic of the method runs in the kernels.
#include <cstddef>
#include <algorithm>
#include <cstring>

#include "hm_internal.h"

namespace hm {

static inline void* at(void* base, int64_t off, int es) {
  return (void*)((char*)base + off * (int64_t)es);
}

static int hodlr_depth(int n, int leaf) {
  int L = 0;
  while (ceil_div(n, 1 << L) > leaf) ++L;
  return L;
}

static GemmTask gemm(const void* A, int lda, int opA, const void* B, int ldb, int opB, void* C,
                     int ldc, int m, int n, int k, double alpha, double beta, int lower = 0) {
  GemmTask t;
  t.A = A; t.B = B; t.C = C;
  t.m = m; t.n = n; t.k = k;
  t.lda = lda; t.ldb = ldb; t.ldc = ldc;
  t.opA = opA; t.opB = opB; t.lower = lower; t.pad = 0;
  t.alpha = alpha; t.beta = beta;
  return t;
}

// Splits the panel QRs of one launch group.  A panel that fits in shared memory whole
// (with its row-major reflector block) goes to the shared-memory kernel.  A larger one
// is cut into row blocks that fit: each block is factored by the same kernel (Q_b to
// scratch, R_b into a stack of the blocks' R factors), the stack is factored next
// (its Q in place, the panel's R), and Y_b = Q_b (rows b of the stack's Q) by a batched
// GEMM.  Panels whose stack would not fit either use the three-stage TSQR, else the
// global-memory kernel.
static QrBatch make_qr_batch(TaskBuf& tb, const std::vector<QrTask>& v, int es, int max_smem,
                             int64_t* scratch_need) {
  QrBatch b;
  std::vector<QrTask> plain, stack;
  std::vector<TsqrTask> ts;
  std::vector<TsqrBlock> blocks;
  std::vector<GemmTask> cmb;
  std::vector<int> plain_rel;  // plain tasks whose R and Q hold scratch offsets
  // TSQR blocks and stacks must leave room for the kernels' own static shared memory
  const size_t budget = (size_t)std::max(0, max_smem - 8192);
  const size_t over = qr_smem_overhead(es);
  auto smem_fits = [&](int64_t m, int k) {
    return ((size_t)((m * k + 15) / 16 * 16) + (size_t)8 * m) * es + over <= (size_t)max_smem;
  };
  auto scratch = [&](int64_t elems) { return (void*)(uintptr_t)(elems * es); };
  int64_t off = 0;
  for (const QrTask& t : v) {
    b.work += work_of(t, es);
    const int m = t.m, k = t.k;
    if (k <= 0 || smem_fits(m, k)) {
      plain.push_back(t);
      continue;
    }
    int mfit = (int)(((int64_t)max_smem - (int64_t)over) / es / (k + 8)) - 16;
    while (mfit > k && !smem_fits(mfit, k)) --mfit;
    const int nbr = mfit > 0 ? (m + mfit - 1) / mfit : 0;
    const int mb = nbr > 0 ? (m + nbr - 1) / nbr : 0;
    if (nbr >= 2 && m - (nbr - 1) * mb >= k && smem_fits((int64_t)nbr * k, k)) {
      const int64_t qoff = off, soff = off + (int64_t)m * k;
      off = soff + (int64_t)nbr * k * k;
      for (int bi = 0, r0 = 0; bi < nbr; ++bi, r0 += mb) {
        const int rows = std::min(mb, m - r0);
        QrTask bt{};
        bt.Y = (unsigned char*)t.Y + (size_t)r0 * es;
        bt.R = scratch(soff + (int64_t)bi * k);
        bt.m = rows;
        bt.k = k;
        bt.ld = t.ld;
        bt.Q = scratch(qoff + (int64_t)r0 * k);
        bt.ldr = nbr * k;
        bt.ldq = rows;
        plain_rel.push_back((int)plain.size());
        plain.push_back(bt);
        cmb.push_back(gemm(bt.Q, rows, 0, scratch(soff + (int64_t)bi * k), nbr * k, 0,
                           (unsigned char*)t.Y + (size_t)r0 * es, t.ld, rows, k, k, 1.0, 0.0));
      }
      QrTask st{};
      st.Y = scratch(soff);
      st.R = t.R;
      st.m = nbr * k;
      st.k = k;
      st.ld = nbr * k;
      stack.push_back(st);
      b.stack_maxm = std::max(b.stack_maxm, nbr * k);
      b.stack_maxmk = std::max(b.stack_maxmk, (int64_t)nbr * k * k);
      continue;
    }
    const size_t kk = (size_t)k * k * es;
    int nb = (m + std::max(256, 2 * k) - 1) / std::max(256, 2 * k);
    const int nb_stack = kk > 0 ? (int)((budget - std::min(budget, (size_t)k * es)) / kk) : 0;
    nb = std::min(nb, nb_stack);
    const bool fits = nb >= 1 && m / nb >= k && (size_t)((m + nb - 1) / nb) * k * es <= budget;
    if (!fits) {
      plain.push_back(t);
      continue;
    }
    for (int j = 0; j < nb; ++j) blocks.push_back(TsqrBlock{(int)ts.size(), j});
    ts.push_back(TsqrTask{t.Y, t.R, off, m, k, t.ld, nb});
    off += (int64_t)nb * k * k + (int64_t)nb * k;
    b.smem_block = std::max(b.smem_block, (size_t)((m + nb - 1) / nb) * k * es);
    b.smem_stack = std::max(b.smem_stack, ((size_t)nb * k * k + k) * es);
  }
  Sig sg;
  for (const QrTask& t : plain) {
    sg << t.m << t.k;
    b.plain_maxm = std::max(b.plain_maxm, t.m);
    b.plain_maxmk = std::max(b.plain_maxmk, (int64_t)t.m * t.k);
  }
  b.sig = sg.h;
  b.plain = tb.add(plain);
  for (int i : plain_rel) {
    const size_t base = b.plain.off + (size_t)i * sizeof(QrTask);
    tb.relocs.push_back(base + offsetof(QrTask, R));
    tb.relocs.push_back(base + offsetof(QrTask, Q));
  }
  b.stack = tb.add(stack);
  for (int i = 0; i < (int)stack.size(); ++i)
    tb.relocs.push_back(b.stack.off + (size_t)i * sizeof(QrTask) + offsetof(QrTask, Y));
  b.combine = tb.add_gemm(cmb);
  for (int i = 0; i < (int)cmb.size(); ++i) {
    const size_t base = b.combine.tasks.off + (size_t)i * sizeof(GemmTask);
    tb.relocs.push_back(base + offsetof(GemmTask, A));
    tb.relocs.push_back(base + offsetof(GemmTask, B));
  }
  b.ts = tb.add(ts);
  b.blocks = tb.add(blocks);
  *scratch_need = std::max(*scratch_need, off);
  return b;
}

// Dense fronts up to this size are factored by one sweep kernel (registers hold the
// front); larger ones by Cholesky, triangular solve, update and inverse launches.
constexpr int kSweepMaxN = 128;

int build_plan(hm_sys_s* sys) {
  Plan& P = sys->plan;
  const hm_opts& o = sys->ctx->opts;
  const int es = sys->precision == HM_PREC_FP64 ? 8 : 4;
  const int nf = sys->nf;
  const int S0 = o.samples;
  P.fg.assign(nf, FrontGeom());
  int maxlev = 0;
  for (int q = 0; q < nf; ++q) {
    FrontGeom& g = P.fg[q];
    g.np = sys->h_first[q + 1] - sys->h_first[q];
    g.nu = sys->h_nupd[q];
    g.nhat = g.np + g.nu;
    g.level = sys->h_level[q];
    maxlev = std::max(maxlev, g.level);
  }
  P.nlevels = maxlev + 1;
  P.level_fronts.assign(P.nlevels, {});
  for (int q = 0; q < nf; ++q) P.level_fronts[P.fg[q].level].push_back(q);
  P.level_front_begin.assign(P.nlevels, 0);
  P.level_front_end.assign(P.nlevels, 0);
  // Front storage: with reuse, the levels of even depth share one bank and those of odd
  // depth the other (a level is assembled while its children's level, of the other
  // parity, still holds their updates; the level two below is packed and dead by then);
  // otherwise every level has its own range, deepest first.
  P.reuse = o.keep_fronts == 0;
  std::vector<int64_t> lsum(P.nlevels, 0);
  for (int q = 0; q < nf; ++q) lsum[P.fg[q].level] += (int64_t)P.fg[q].nhat * P.fg[q].nhat;
  int64_t bank[2] = {0, 0};
  for (int l = 0; l < P.nlevels; ++l) bank[l & 1] = std::max(bank[l & 1], lsum[l]);
  int64_t off = 0;
  for (int l = P.nlevels - 1; l >= 0; --l) {
    if (P.reuse) off = (l & 1) ? bank[0] : 0;
    P.level_front_begin[l] = off;
    for (int q : P.level_fronts[l]) {
      P.fg[q].off = off;
      off += (int64_t)P.fg[q].nhat * P.fg[q].nhat;
    }
    P.level_front_end[l] = off;
  }
  P.front_total = P.reuse ? bank[0] + bank[1] : off;
  P.level_entries.assign(P.nlevels, 0);
  const double per_col = ((double)sys->nnz + sys->n) / (2.0 * std::max(sys->n, 1));
  for (int q = 0; q < nf; ++q) P.level_entries[P.fg[q].level] += (int64_t)(per_col * P.fg[q].np + 0.5);
  P.max_children = 0;
  for (int q = 0; q < nf; ++q) P.max_children = std::max(P.max_children, sys->children(q).size());

  // ---------------------------------------------------------------- HODLR fronts
  P.hf.clear();
  P.bo_total = P.w_total = P.t_total = P.p_total = P.g_total = 0;
  P.core_total = P.piv_total = P.comp_total = P.tb_total = 0;
  P.qr_scratch = 0;
  P.nrank = 0;
  for (int l = P.nlevels - 1; l >= 0; --l) {
    for (int q : P.level_fronts[l]) {
      FrontGeom& g = P.fg[q];
      if (g.np <= o.n_c) continue;
      if (g.np < 2) continue;
      HFront h;
      h.q = q;
      h.np = g.np;
      h.nu = g.nu;
      h.L = hodlr_depth(g.np, o.hodlr_leaf);
      const int S = sys->level_width.empty() ? S0 : sys->level_width[g.level];  // sketch width cap
      h.kf = g.nu > 0 ? std::min(S, std::min(g.nu, g.np)) : 0;
      // node ranges level by level
      std::vector<std::pair<int, int>> ranges = {{0, g.np}};
      h.kl.assign(h.L, 0);
      for (int lv = 0; lv < h.L; ++lv) {
        std::vector<std::pair<int, int>> next;
        for (size_t j = 0; j < ranges.size(); ++j) {
          const int lo = ranges[j].first, hi = ranges[j].second;
          const int mid = lo + (hi - lo) / 2;
          HNodeGeom nd;
          nd.level = lv;
          nd.index = (int)j;
          nd.lo = lo; nd.mid = mid; nd.hi = hi;
          nd.kb = std::min(S, std::min(mid - lo, hi - mid));
          h.kl[lv] = std::max(h.kl[lv], nd.kb);
          h.nodes.push_back(nd);
          next.push_back({lo, mid});
          next.push_back({mid, hi});
        }
        ranges.swap(next);
      }
      for (auto& r : ranges) { h.leaf_lo.push_back(r.first); h.leaf_hi.push_back(r.second); }
      if (o.compress_ff && g.nu > 0) {  // F_ff's HODLR tree (leaf hodlr_leaf), the same width
        std::vector<std::pair<int, int>> fr = {{0, g.nu}};
        const int Lf = hodlr_depth(g.nu, o.hodlr_leaf);
        for (int lv = 0; lv < Lf; ++lv) {
          std::vector<std::pair<int, int>> next;
          for (size_t j = 0; j < fr.size(); ++j) {
            const int lo = fr[j].first, hi = fr[j].second, mid = lo + (hi - lo) / 2;
            HNodeGeom nd;
            nd.level = lv;
            nd.index = (int)j;
            nd.lo = lo; nd.mid = mid; nd.hi = hi;
            nd.kb = std::min(S, std::min(mid - lo, hi - mid));
            nd.core_off = nd.piv_off = nd.tb_off = 0;
            h.ff_nodes.push_back(nd);
            next.push_back({lo, mid});
            next.push_back({mid, hi});
          }
          fr.swap(next);
        }
      }
      h.col.assign(h.L + 1, 0);
      h.col[0] = h.kf;
      for (int lv = 0; lv < h.L; ++lv) h.col[lv + 1] = h.col[lv] + h.kl[lv];
      h.xc = h.col[h.L];
      h.bo_off = P.bo_total;
      P.bo_total += (int64_t)h.np * h.xc;
      h.g_off = P.g_total;
      P.g_total += (int64_t)h.np * 2 * (h.xc - h.kf);
      h.w_off = P.w_total;
      P.w_total += (int64_t)h.nu * h.kf;
      h.t_off = P.t_total;
      P.t_total += (int64_t)h.kf * h.kf;
      h.p_off = P.p_total;
      P.p_total += (int64_t)h.nu * h.kf;
      h.rank_slot_f = P.nrank++;
      // F_fp compression scratch
      const int kf = h.kf;
      h.fom_off = P.comp_total; P.comp_total += (int64_t)h.np * kf;
      h.fy_off = P.comp_total; P.comp_total += (int64_t)h.nu * kf;
      h.fz_off = P.comp_total; P.comp_total += (int64_t)h.np * kf;
      h.fr_off = P.comp_total; P.comp_total += (int64_t)kf * kf;
      h.fuhs_off = P.comp_total; P.comp_total += (int64_t)kf * kf;
      h.fvh_off = P.comp_total; P.comp_total += (int64_t)kf * kf;
      for (auto& nd : h.nodes) {
        const int k = h.kl[nd.level];
        const int na = nd.mid - nd.lo, nb = nd.hi - nd.mid, kb = nd.kb;
        nd.core_off = P.core_total; P.core_total += (int64_t)2 * (2 * k) * (2 * k);
        nd.piv_off = P.piv_total; P.piv_total += 2 * k;
        nd.rank_slot = P.nrank++;
        nd.om_off = P.comp_total; P.comp_total += (int64_t)nb * kb;
        nd.y_off = P.comp_total; P.comp_total += (int64_t)na * kb;
        nd.z_off = P.comp_total; P.comp_total += (int64_t)nb * kb;
        nd.r_off = P.comp_total; P.comp_total += (int64_t)kb * kb;
        nd.uhs_off = P.comp_total; P.comp_total += (int64_t)kb * kb;
        nd.vh_off = P.comp_total; P.comp_total += (int64_t)kb * kb;
        nd.tb_off = P.tb_total; P.tb_total += (int64_t)2 * (2 * k) * h.col[nd.level];
      }
      for (auto& nd : h.ff_nodes) {
        const int na = nd.mid - nd.lo, nb = nd.hi - nd.mid, kb = nd.kb;
        nd.rank_slot = P.nrank++;
        nd.om_off = P.comp_total; P.comp_total += (int64_t)nb * kb;
        nd.y_off = P.comp_total; P.comp_total += (int64_t)na * kb;
        nd.z_off = P.comp_total; P.comp_total += (int64_t)nb * kb;
        nd.r_off = P.comp_total; P.comp_total += (int64_t)kb * kb;
        nd.uhs_off = P.comp_total; P.comp_total += (int64_t)kb * kb;
        nd.vh_off = P.comp_total; P.comp_total += (int64_t)kb * kb;
        nd.u_off = P.comp_total; P.comp_total += (int64_t)na * kb;
        nd.v_off = P.comp_total; P.comp_total += (int64_t)nb * kb;
      }
      g.hodlr = (int)P.hf.size();
      P.hf.push_back(std::move(h));
    }
  }

  host_mark("build_plan: geometry");
  // ---------------------------------------------------------------- capacity checks
  for (int q = 0; q < nf; ++q) {
    const FrontGeom& g = P.fg[q];
    if (g.hodlr < 0 && g.np > 128) {
      set_last_error("dense pivot block larger than 128 (lower n_c)");
      return HM_ERR_CAPACITY;
    }
  }

  // ---------------------------------------------------------------- packed factor
  P.dense_total = P.leaf_total = 0;
  for (int q = 0; q < nf; ++q) {
    FrontGeom& g = P.fg[q];
    if (g.hodlr < 0) {
      g.cf_off = P.dense_total;
      P.dense_total += packed_size(g.np, g.nhat, es);
      continue;
    }
    HFront& h = P.hf[g.hodlr];
    h.lmax = 0;
    for (size_t li = 0; li < h.leaf_lo.size(); ++li) h.lmax = std::max(h.lmax, h.leaf_hi[li] - h.leaf_lo[li]);
    h.lv_off = P.leaf_total;
    P.leaf_total += (int64_t)h.np * h.lmax;
  }

  // ---------------------------------------------------------------- allocations
  auto A = [&](void** p, int64_t elems, int size) -> int {
    return dev_alloc_ctx(sys->ctx, &sys->plan_allocs, p, (size_t)std::max<int64_t>(elems, 1) * size);
  };
  HM_TRY(A(&sys->d_front, P.front_total, es));
  HM_TRY(A(&sys->d_bo, P.bo_total, es));
  HM_TRY(A(&sys->d_x, P.bo_total, es));
  HM_TRY(A(&sys->d_g, P.g_total, es));
  HM_TRY(A(&sys->d_w, P.w_total, es));
  HM_TRY(A(&sys->d_tm, P.t_total, es));
  HM_TRY(A(&sys->d_pm, P.p_total, es));
  HM_TRY(A(&sys->d_core, P.core_total, es));
  HM_TRY(A((void**)&sys->d_piv, P.piv_total, 4));
  HM_TRY(A(&sys->d_comp, P.comp_total, es));
  HM_TRY(A(&sys->d_tb, P.tb_total, es));
  HM_TRY(A((void**)&sys->d_ranks, P.nrank, 4));
  HM_TRY(A((void**)&sys->d_pvals, sys->nnz, 8));
  HM_TRY(A((void**)&sys->d_pvals2, sys->nnz, 8));
  HM_TRY(A((void**)&P.d_front_off, nf, 8));
  HM_TRY(A((void**)&P.d_nhat, nf, 4));
  HM_TRY(A((void**)&P.d_np, nf, 4));
  HM_TRY(A((void**)&P.d_hkind, nf, 4));
  HM_TRY(A(&sys->d_dfac, P.dense_total, es));
  HM_TRY(A(&sys->d_leafinv, P.leaf_total, es));
  HM_TRY(A((void**)&P.d_cf_off, nf, 8));
  HM_TRY(A((void**)&P.d_flevel, nf, 4));
  {
    // the host copies live as long as the plan, so the uploads need no synchronization
    auto& fo = P.h_front_off;
    auto& nh = P.h_nhat;
    auto& npv = P.h_np;
    auto& hk = P.h_hkind;
    fo.resize(nf); nh.resize(nf); npv.resize(nf); hk.resize(nf);
    P.h_cf_off.resize(nf);
    P.h_flevel.resize(nf);
    for (int q = 0; q < nf; ++q) {
      fo[q] = P.fg[q].off; nh[q] = P.fg[q].nhat; npv[q] = P.fg[q].np; hk[q] = P.fg[q].hodlr;
      P.h_cf_off[q] = P.fg[q].cf_off;
      P.h_flevel[q] = P.fg[q].level;
    }
    cudaStream_t s = sys->ctx->stream;
    HM_CUDA(cudaMemcpyAsync(P.d_front_off, fo.data(), nf * 8, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(P.d_nhat, nh.data(), nf * 4, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(P.d_np, npv.data(), nf * 4, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(P.d_hkind, hk.data(), nf * 4, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(P.d_cf_off, P.h_cf_off.data(), nf * 8, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(P.d_flevel, P.h_flevel.data(), nf * 4, cudaMemcpyHostToDevice, s));
  }

  host_mark("build_plan: allocations");
  // ---------------------------------------------------------------- factor tasks
  void* F = sys->d_front;
  void* Bo = sys->d_bo;
  void* X = sys->d_x;
  void* W = sys->d_w;
  void* Tm = sys->d_tm;
  void* Pm = sys->d_pm;
  void* Gm = sys->d_g;
  void* Cm = sys->d_core;
  void* Cp = sys->d_comp;
  void* Tb = sys->d_tb;
  int* piv = sys->d_piv;
  int* ranks = sys->d_ranks;
  TaskBuf& tb = P.tb;
  tb.host.clear();
  tb.es = es;
  tb.split_target = 2 * sys->ctx->num_sms;
  P.levels.assign(P.nlevels, LevelFactorPlan());
  double fbytes = 0;
  for (int l = P.nlevels - 1; l >= 0; --l) {
    LevelFactorPlan& lp = P.levels[l];
    const auto& fr = P.level_fronts[l];
    // extend-add: per child slot, the parents that have a child in that slot
    int slots = 0;
    for (int q : fr) slots = std::max(slots, sys->children(q).size());
    for (int s = 0; s < slots; ++s) {
      std::vector<int> par;
      Work w;
      int max_nu = 0;
      for (int q : fr) {
        const auto ch = sys->children(q);
        if (s >= (int)ch.size()) continue;
        par.push_back(q);
        const int c = ch[s];
        const double nuc = P.fg[c].nu;
        max_nu = std::max(max_nu, P.fg[c].nu);
        w.flops += nuc * (nuc + 1) / 2;
        w.bytes += 3.0 * es * nuc * (nuc + 1) / 2 + 4.0 * nuc;
      }
      lp.ea_parents.push_back(tb.add(par));
      lp.ea_max_nu.push_back(max_nu);
      lp.ea_work.push_back(w);
    }
    // dense fronts
    std::vector<PotrfTask> pot;
    std::vector<TrsmTask> trs;
    std::vector<GemmTask> syrk;
    std::vector<CholInvTask> dinv;
    std::vector<SweepTask> sweep;
    for (int q : fr) {
      const FrontGeom& g = P.fg[q];
      if (g.hodlr >= 0) continue;
      lp.n_dense++;
      void* Fq = at(F, g.off, es);
      fbytes += es * ((double)g.np * g.np + 2.0 * g.nu * g.np);
      if (g.nhat <= kSweepMaxN) {
        sweep.push_back(SweepTask{Fq, at(sys->d_dfac, g.cf_off, es), g.np, g.nhat, q, 0, 0, 0});
        lp.sweep_maxn = std::max(lp.sweep_maxn, g.nhat);
        continue;
      }
      pot.push_back(PotrfTask{Fq, g.np, g.nhat, q, 0});
      lp.potrf_maxn = std::max(lp.potrf_maxn, g.np);
      if (g.nu > 0) {
        for (int r0 = 0; r0 < g.nu; r0 += 64)
          trs.push_back(TrsmTask{Fq, at(F, g.off + g.np, es), g.np, g.nhat, g.nu, g.nhat, r0, 0});
        lp.trsm_maxn = std::max(lp.trsm_maxn, g.np);
        syrk.push_back(gemm(at(F, g.off + g.np, es), g.nhat, 0, at(F, g.off + g.np, es), g.nhat, 1,
                            at(F, g.off + g.np + (int64_t)g.np * g.nhat, es), g.nhat, g.nu, g.nu,
                            g.np, -1.0, 1.0, 1));
      }
      // K = F_fp F_pp^{-1} below the pivot block and K^T beside it, so that both apply
      // passes read the front with rows on consecutive threads
      dinv.push_back(CholInvTask{Fq, at(F, g.off + g.np, es), g.np, g.nhat, g.nu, g.nhat,
                                 at(F, g.off + (int64_t)g.np * g.nhat, es), g.nhat, 0});
    }
    lp.potrf = tb.add(pot);
    lp.trsm = tb.add(trs);
    lp.syrk = tb.add_gemm(syrk);
    lp.dinv = tb.add(dinv);
    lp.sweep = tb.add(sweep);
    // HODLR fronts
    std::vector<OmegaTask> om;
    std::vector<GemmTask> gy, gz, gu, gv, ffx;
    std::vector<QrTask> qy, qz;
    std::vector<SvdTask> sv;
    std::vector<SweepTask> lsw;
    std::vector<GemmTask> lxg;
    std::vector<GemmTask> sT, sP, sF;
    std::vector<BdlrTask> bd;
    const bool bdlr = o.compressor == HM_COMP_BDLR;
    int maxL = 0;
    for (int q : fr) {
      const FrontGeom& g = P.fg[q];
      if (g.hodlr < 0) continue;
      lp.n_hodlr++;
      const HFront& h = P.hf[g.hodlr];
      maxL = std::max(maxL, h.L);
      const int np = h.np, nu = h.nu, nh = g.nhat;
      const int64_t fo = g.off;
      // pivot-block off-diagonal blocks: B = K[a, b] = K[b, a]^T (lower storage)
      for (const auto& nd : h.nodes) {
        const int na = nd.mid - nd.lo, nb = nd.hi - nd.mid, kb = nd.kb, k = h.kl[nd.level];
        const uint64_t blk = block_id(q, 0, nd.level, nd.index);
        void* Kba = at(F, fo + nd.mid + (int64_t)nd.lo * nh, es);  // nb x na
        if (bdlr) {
          const int64_t colb = (int64_t)h.col[nd.level] * np;
          bd.push_back(BdlrTask{at(F, fo, es), at(Bo, h.bo_off + colb + nd.lo, es),
                                at(Bo, h.bo_off + colb + nd.mid, es), ranks + nd.rank_slot, q, nh, nd.lo, na,
                                nd.mid, nb, 1, np, np, kb});
          lp.bdlr_maxnh = std::max(lp.bdlr_maxnh, nh);
          lp.bdlr_maxcap = std::max(lp.bdlr_maxcap, kb);
          fbytes += es * (3.0 * (na + nb) * k);
          continue;
        }
        om.push_back(OmegaTask{at(Cp, nd.om_off, es), blk, nb, kb, nb, 0});
        gy.push_back(gemm(Kba, nh, 1, at(Cp, nd.om_off, es), nb, 0, at(Cp, nd.y_off, es), na, na, kb,
                          nb, 1.0, 0.0));
        qy.push_back(QrTask{at(Cp, nd.y_off, es), nullptr, na, kb, na, 0});
        gz.push_back(gemm(Kba, nh, 0, at(Cp, nd.y_off, es), na, 0, at(Cp, nd.z_off, es), nb, nb, kb,
                          na, 1.0, 0.0));
        qz.push_back(QrTask{at(Cp, nd.z_off, es), at(Cp, nd.r_off, es), nb, kb, nb, 0});
        sv.push_back(SvdTask{at(Cp, nd.r_off, es), at(Cp, nd.uhs_off, es), at(Cp, nd.vh_off, es),
                             ranks + nd.rank_slot, kb, 0});
        lp.svd_maxk = std::max(lp.svd_maxk, kb);
        const int64_t colo = (int64_t)h.col[nd.level] * np;
        gu.push_back(gemm(at(Cp, nd.y_off, es), na, 0, at(Cp, nd.uhs_off, es), kb, 0,
                          at(Bo, h.bo_off + colo + nd.lo, es), np, na, kb, kb, 1.0, 0.0));
        gv.push_back(gemm(at(Cp, nd.z_off, es), nb, 0, at(Cp, nd.vh_off, es), kb, 0,
                          at(Bo, h.bo_off + colo + nd.mid, es), np, nb, kb, kb, 1.0, 0.0));
        fbytes += es * (3.0 * (na + nb) * k);  // the apply reads U / V (k) and G (2k) rows
      }
      if (nu > 0 && h.kf > 0) {
        const int kf = h.kf;
        const uint64_t blk = block_id(q, 1, 0, 0);
        void* Ffp = at(F, fo + np, es);  // nu x np, ld nh
        if (bdlr) {
          bd.push_back(BdlrTask{at(F, fo, es), at(W, h.w_off, es), at(Bo, h.bo_off, es), ranks + h.rank_slot_f, q,
                                nh, np, nu, 0, np, 0, nu, np, kf});
          lp.bdlr_maxnh = std::max(lp.bdlr_maxnh, nh);
          lp.bdlr_maxcap = std::max(lp.bdlr_maxcap, kf);
        } else {
        om.push_back(OmegaTask{at(Cp, h.fom_off, es), blk, np, kf, np, 0});
        gy.push_back(gemm(Ffp, nh, 0, at(Cp, h.fom_off, es), np, 0, at(Cp, h.fy_off, es), nu, nu, kf,
                          np, 1.0, 0.0));
        qy.push_back(QrTask{at(Cp, h.fy_off, es), nullptr, nu, kf, nu, 0});
        gz.push_back(gemm(Ffp, nh, 1, at(Cp, h.fy_off, es), nu, 0, at(Cp, h.fz_off, es), np, np, kf,
                          nu, 1.0, 0.0));
        qz.push_back(QrTask{at(Cp, h.fz_off, es), at(Cp, h.fr_off, es), np, kf, np, 0});
        sv.push_back(SvdTask{at(Cp, h.fr_off, es), at(Cp, h.fuhs_off, es), at(Cp, h.fvh_off, es),
                             ranks + h.rank_slot_f, kf, 0});
        lp.svd_maxk = std::max(lp.svd_maxk, kf);
        gu.push_back(gemm(at(Cp, h.fy_off, es), nu, 0, at(Cp, h.fuhs_off, es), kf, 0,
                          at(W, h.w_off, es), nu, nu, kf, kf, 1.0, 0.0));
        gv.push_back(gemm(at(Cp, h.fz_off, es), np, 0, at(Cp, h.fvh_off, es), kf, 0,
                          at(Bo, h.bo_off, es), np, np, kf, kf, 1.0, 0.0));
        }
        // Schur complement: T = Vf^T Vtilde, P = W T, F_ff -= P W^T
        sT.push_back(gemm(at(Bo, h.bo_off, es), np, 1, at(X, h.bo_off, es), np, 0, at(Tm, h.t_off, es),
                          kf, kf, kf, np, 1.0, 0.0));
        sP.push_back(gemm(at(W, h.w_off, es), nu, 0, at(Tm, h.t_off, es), kf, 0, at(Pm, h.p_off, es), nu,
                          nu, kf, kf, 1.0, 0.0));
        sF.push_back(gemm(at(Pm, h.p_off, es), nu, 0, at(W, h.w_off, es), nu, 1,
                          at(F, fo + np + (int64_t)np * nh, es), nh, nu, nu, kf, -1.0, 1.0, 1));
        fbytes += es * 4.0 * (double)(np + nu) * kf;
      }
      // compress_ff: F_ff's off-diagonal blocks (lower storage, nb x na at rows np + mid,
      // columns np + lo) by the same range finder, then written back as V U^T, before
      // the Schur update subtracts W T W^T
      for (const auto& nd : h.ff_nodes) {
        const int na = nd.mid - nd.lo, nb = nd.hi - nd.mid, kb = nd.kb;
        const uint64_t blk = block_id(q, 2, nd.level, nd.index);
        void* Kba = at(F, fo + np + nd.mid + (int64_t)(np + nd.lo) * nh, es);
        om.push_back(OmegaTask{at(Cp, nd.om_off, es), blk, nb, kb, nb, 0});
        gy.push_back(gemm(Kba, nh, 1, at(Cp, nd.om_off, es), nb, 0, at(Cp, nd.y_off, es), na, na, kb,
                          nb, 1.0, 0.0));
        qy.push_back(QrTask{at(Cp, nd.y_off, es), nullptr, na, kb, na, 0});
        gz.push_back(gemm(Kba, nh, 0, at(Cp, nd.y_off, es), na, 0, at(Cp, nd.z_off, es), nb, nb, kb,
                          na, 1.0, 0.0));
        qz.push_back(QrTask{at(Cp, nd.z_off, es), at(Cp, nd.r_off, es), nb, kb, nb, 0});
        sv.push_back(SvdTask{at(Cp, nd.r_off, es), at(Cp, nd.uhs_off, es), at(Cp, nd.vh_off, es),
                             ranks + nd.rank_slot, kb, 0});
        lp.svd_maxk = std::max(lp.svd_maxk, kb);
        gu.push_back(gemm(at(Cp, nd.y_off, es), na, 0, at(Cp, nd.uhs_off, es), kb, 0, at(Cp, nd.u_off, es), na,
                          na, kb, kb, 1.0, 0.0));
        gv.push_back(gemm(at(Cp, nd.z_off, es), nb, 0, at(Cp, nd.vh_off, es), kb, 0, at(Cp, nd.v_off, es), nb,
                          nb, kb, kb, 1.0, 0.0));
        ffx.push_back(gemm(at(Cp, nd.v_off, es), nb, 0, at(Cp, nd.u_off, es), na, 1, Kba, nh, nb, na, kb, 1.0,
                           0.0));
      }
      for (size_t li = 0; li < h.leaf_lo.size(); ++li) {
        const int lo = h.leaf_lo[li], n = h.leaf_hi[li] - lo;
        void* Lq = at(F, fo + lo + (int64_t)lo * nh, es);
        // the leaf's inverse in one sweep kernel, into the packed leaf store
        void* Lp = at(sys->d_leafinv, h.lv_off + lo, es);
        lsw.push_back(SweepTask{Lq, Lp, n, n, q, nh, np, 0});
        lp.leaf_maxn = std::max(lp.leaf_maxn, n);
        // X (leaf rows) = K_leaf^{-1} Bo (leaf rows), once the explicit inverse is formed
        if (h.xc > 0)
          lxg.push_back(gemm(Lp, np, 0, at(Bo, h.bo_off + lo, es), np, 0, at(X, h.bo_off + lo, es), np, n, h.xc,
                             n, 1.0, 0.0));
        fbytes += es * (double)n * n;
      }
    }
    lp.bdlr = tb.add(bd);
    lp.omega = tb.add(om);
    const bool tc = sys->precision == HM_PREC_MIXED_BF16;  // sampling products on tensor cores
    lp.sampY = tb.add_gemm(gy, tc);
    lp.qrY = make_qr_batch(tb, qy, es, sys->ctx->max_smem, &P.qr_scratch);
    lp.sampZ = tb.add_gemm(gz, tc);
    lp.qrZ = make_qr_batch(tb, qz, es, sys->ctx->max_smem, &P.qr_scratch);
    lp.svd = tb.add(sv);
    lp.formU = tb.add_gemm(gu);
    lp.formV = tb.add_gemm(gv);
    lp.ffx = tb.add_gemm(ffx);
    lp.leaf_sweep = tb.add(lsw);
    lp.leaf_x = tb.add_gemm(lxg);
    // Woodbury levels, bottom-up (height 1 = parents of the leaves)
    for (int ht = 1; ht <= maxL; ++ht) {
      std::vector<GemmTask> pre, sg, upd, gmv;
      std::vector<CoreLuTask> lu;
      for (int q : fr) {
        const FrontGeom& g = P.fg[q];
        if (g.hodlr < 0) continue;
        const HFront& h = P.hf[g.hodlr];
        if (h.L < ht) continue;
        const int lv = h.L - ht;
        const int np = h.np, k = h.kl[lv], A_ = h.col[lv];
        const int64_t colo = (int64_t)h.col[lv] * np;
        for (const auto& nd : h.nodes) {
          if (nd.level != lv) continue;
          const int na = nd.mid - nd.lo, nb = nd.hi - nd.mid;
          void* core = at(Cm, nd.core_off, es);
          void* cinv = at(Cm, nd.core_off + (int64_t)4 * k * k, es);
          void* Ua = at(Bo, h.bo_off + colo + nd.lo, es);
          void* Vb = at(Bo, h.bo_off + colo + nd.mid, es);
          void* Uh = at(X, h.bo_off + colo + nd.lo, es);
          void* Vh = at(X, h.bo_off + colo + nd.mid, es);
          pre.push_back(gemm(Ua, np, 1, Uh, np, 0, core, 2 * k, k, k, na, 1.0, 0.0));
          pre.push_back(gemm(Vb, np, 1, Vh, np, 0, at(Cm, nd.core_off + (int64_t)k * 2 * k + k, es),
                             2 * k, k, k, nb, 1.0, 0.0));
          lu.push_back(CoreLuTask{core, cinv, piv + nd.piv_off, k, q});
          {  // G for the apply: Zhat_a C^{-1}[0:k, :] and Zhat_b C^{-1}[k:2k, :]
            void* Gl = at(Gm, h.g_off + (int64_t)2 * (h.col[lv] - h.kf) * np, es);
            gmv.push_back(gemm(Uh, np, 0, cinv, 2 * k, 0, at(Gl, nd.lo, es), np, na, 2 * k, k, 1.0, 0.0));
            gmv.push_back(gemm(Vh, np, 0, at(cinv, k, es), 2 * k, 0, at(Gl, nd.mid, es), np, nb, 2 * k, k, 1.0,
                               0.0));
          }
          if (A_ > 0) {
            void* tbuf = at(Tb, nd.tb_off, es);
            void* sbuf = at(Tb, nd.tb_off + (int64_t)2 * k * A_, es);
            pre.push_back(gemm(Ua, np, 1, at(X, h.bo_off + nd.lo, es), np, 0, tbuf, 2 * k, k, A_, na,
                               1.0, 0.0));
            pre.push_back(gemm(Vb, np, 1, at(X, h.bo_off + nd.mid, es), np, 0,
                               at(Tb, nd.tb_off + k, es), 2 * k, k, A_, nb, 1.0, 0.0));
            sg.push_back(gemm(cinv, 2 * k, 0, tbuf, 2 * k, 0, sbuf, 2 * k, 2 * k, A_, 2 * k, 1.0, 0.0));
            upd.push_back(gemm(Uh, np, 0, sbuf, 2 * k, 0, at(X, h.bo_off + nd.lo, es), np, na, A_, k,
                               -1.0, 1.0));
            upd.push_back(gemm(Vh, np, 0, at(Tb, nd.tb_off + (int64_t)2 * k * A_ + k, es), 2 * k, 0,
                               at(X, h.bo_off + nd.mid, es), np, nb, A_, k, -1.0, 1.0));
          }
        }
      }
      LevelFactorPlan::Height H;
      H.pre = tb.add_gemm(pre);
      H.lu = tb.add(lu);
      for (const auto& c : lu) H.lu_maxk = std::max(H.lu_maxk, c.k);
      H.sg = tb.add_gemm(sg);
      H.upd = tb.add_gemm(upd);
      H.gm = tb.add_gemm(gmv);
      lp.heights.push_back(H);
    }
    lp.schurT = tb.add_gemm(sT);
    lp.schurP = tb.add_gemm(sP);
    lp.schurF = tb.add_gemm(sF);
    // pack the dense fronts factored in place (beyond the sweep kernel): [F_pp^-1 | K^T]
    // (np x nhat) and K (nu x np).  The sweep kernel writes its fronts and the HODLR
    // leaves' inverses to the packed stores itself.
    std::vector<CopyTask> pk;
    for (int q : fr) {
      const FrontGeom& g = P.fg[q];
      if (g.hodlr >= 0 || g.nhat <= kSweepMaxN) continue;
      pk.push_back(CopyTask{at(F, g.off, es), at(sys->d_dfac, g.cf_off, es), g.np, g.nhat, g.nhat, g.np});
      if (g.nu > 0)
        pk.push_back(CopyTask{at(F, g.off + g.np, es),
                              at(sys->d_dfac, g.cf_off + packed_k_offset(g.np, g.nhat, es), es), g.nu, g.np, g.nhat,
                              g.nu});
    }
    lp.pack = tb.add(pk);
  }
  P.factor_bytes = fbytes;
  P.stored_bytes = 0;
  for (int q = 0; q < nf; ++q) {
    const FrontGeom& g = P.fg[q];
    if (g.hodlr < 0) {  // F_pp^{-1}, K and K^T
      P.stored_bytes += es * ((double)g.np * g.np + 2.0 * g.np * g.nu);
      continue;
    }
    const HFront& h = P.hf[g.hodlr];
    double e = (double)h.np * h.xc + (double)h.np * h.kf + (double)h.np * 2 * (h.xc - h.kf) + (double)h.nu * h.kf;
    for (size_t li = 0; li < h.leaf_lo.size(); ++li) {
      const double n = h.leaf_hi[li] - h.leaf_lo[li];
      e += n * n;
    }
    P.stored_bytes += es * e;
  }
  host_mark("build_plan: tasks");
  HM_TRY(A(&sys->d_qrs, P.qr_scratch, es));
  tb.relocate(sys->d_qrs);  // row-block QR tasks address the scratch by offset until now
  HM_TRY(A(&P.d_split_ws, tb.split_ws, es));
  HM_TRY(A((void**)&P.d_split_cnt, tb.split_slots, (int)sizeof(unsigned)));
  HM_CUDA(cudaMemsetAsync(P.d_split_cnt, 0, sizeof(unsigned) * std::max(tb.split_slots, 1), sys->ctx->stream));
  HM_TRY(A((void**)&P.d_tasks, (int64_t)std::max<size_t>(tb.host.size(), 16), 1));
  HM_CUDA(cudaMemcpyAsync(P.d_tasks, tb.host.data(), tb.host.size(), cudaMemcpyHostToDevice,
                          sys->ctx->stream));
  return HM_OK;
}

// ------------------------------------------------------------------------------------
// Solve plan for nrhs right-hand sides.
// ------------------------------------------------------------------------------------
void release_solve_state(hm_sys_s* sys) {
  cudaStreamSynchronize(sys->ctx->stream);
  for (auto& kv : sys->solve_plans) dev_free_all(sys->ctx, &kv.second->allocs);
  sys->solve_plans.clear();
  dev_free_all(sys->ctx, &sys->gm.allocs);
  if (sys->gm.h_res) cudaFreeHost(sys->gm.h_res);
  sys->gm.h_res = nullptr;
  sys->gm.nrhs = 0;
  sys->gm.m = 0;
}

// The fused kernels of a level's HODLR fronts: one cluster of C CTAs per front (C a
// power of two, at most 8, about 64 pivot rows per CTA, at most the number of leaves of
// the shallowest front so that every CTA owns a node of depth log2 C), RB right-hand
// sides per cluster (the widest group whose shared memory fits; the autotuner may take
// a half or a quarter of it, for more clusters).
static void plan_hodlr_apply(hm_sys_s* sys, SolvePlan* sp, LevelSolvePlan& lp, const std::vector<int>& hod,
                             int nrhs, int es) {
  Plan& P = sys->plan;
  TaskBuf& tb = sp->tb;
  lp.ha_ok = false;
  if (hod.empty()) return;
  int max_np = 0, min_L = 1 << 20;
  for (int q : hod) {
    const HFront& h = P.hf[P.fg[q].hodlr];
    if (h.L > kHaMaxL || (int)h.leaf_lo.size() != (1 << h.L)) return;
    max_np = std::max(max_np, h.np);
    min_L = std::min(min_L, h.L);
  }
  int C = 1;
  while (C < 8 && C * 64 < max_np && 2 * C <= (1 << min_L)) C *= 2;
  int lc = 0;
  while ((1 << lc) < C) ++lc;
  std::vector<HApplyTask> tasks;
  std::vector<int> leafb;
  HaDims d{};
  double fbytes_up = 0, fbytes_down = 0, vbytes_up = 0, vbytes_down = 0;
  for (int q : hod) {
    const FrontGeom& g = P.fg[q];
    const HFront& h = P.hf[g.hodlr];
    HApplyTask t{};
    t.X = at(sys->d_x, h.bo_off, es);
    t.Bo = at(sys->d_bo, h.bo_off, es);
    t.G = at(sys->d_g, h.g_off, es);
    t.W = at(sys->d_w, h.w_off, es);
    t.F = at(sys->d_leafinv, h.lv_off, es);
    t.fv_off = sp->fv_off[q];
    t.q = q;
    t.first = sys->h_first[q];
    t.np = h.np;
    t.nu = h.nu;
    t.nhat = g.nhat;
    t.L = h.L;
    t.kf = h.kf;
    t.leaf_off = (int)leafb.size();
    t.ea_off = (int)sp->ea_total;
    sp->ea_total += (int64_t)C * sys->children(q).size();
    for (int l = 0; l < h.L; ++l) {
      t.kl[l] = h.kl[l];
      t.col[l] = h.col[l];
      d.kmax = std::max(d.kmax, h.kl[l]);
    }
    for (int lo : h.leaf_lo) leafb.push_back(lo);
    leafb.push_back(h.np);
    const int span = 1 << (h.L - lc);
    for (int c = 0; c < C; ++c) {
      const int j1 = (c + 1) * span;
      const int p1 = j1 < (int)h.leaf_lo.size() ? h.leaf_lo[j1] : h.np;
      d.rowsP = std::max(d.rowsP, p1 - h.leaf_lo[c * span]);
    }
    d.rowsU = std::max(d.rowsU, (h.nu + C - 1) / C);
    d.kf = std::max(d.kf, h.kf);
    tasks.push_back(t);
    // algorithmic bytes: every factor entry the pass reads, once; the vectors per RHS
    double leaves = 0, xc = 0;
    for (size_t i = 0; i < h.leaf_lo.size(); ++i) leaves += (double)(h.leaf_hi[i] - h.leaf_lo[i]) * (h.leaf_hi[i] - h.leaf_lo[i]);
    for (int l = 0; l < h.L; ++l) xc += h.kl[l];
    fbytes_up += (double)es * ((double)h.np * h.kf + (double)h.nu * h.kf);
    fbytes_down += (double)es * ((double)h.np * h.kf + (double)h.nu * h.kf + (double)h.np * 3.0 * xc + leaves);
    double child = 0;
    for (int c : sys->children(q)) child += (double)es * nrhs * P.fg[c].nu + 4.0 * P.fg[c].nu;
    vbytes_up += (double)es * nrhs * ((double)h.np + g.nhat) + child;
    vbytes_down += (double)es * nrhs * (2.0 * h.np + h.nu) + 4.0 * h.nu;
  }
  // widest right-hand-side group whose shared memory fits
  int RB = nrhs >= 16 ? 16 : nrhs > 4 ? 8 : nrhs > 2 ? 4 : nrhs;
  auto tstore = [&](int rb) {
    int m = 0;
    for (int q : hod) {
      const HFront& h = P.hf[P.fg[q].hodlr];
      for (int l = 0; l < h.L; ++l) {
        const int nodes = l >= lc ? (1 << (l - lc)) : 1;
        m = std::max(m, nodes * 2 * h.kl[l] * rb);
      }
    }
    return m;
  };
  const size_t cap = (size_t)sys->ctx->max_smem;
  for (; RB >= 1; RB /= 2) {
    d.tstore = tstore(RB);
    if (hodlr_apply_smem(d, RB, true, es) <= cap && hodlr_apply_smem(d, RB, false, es) <= cap) break;
  }
  if (RB < 1) return;
  lp.ha_C = C;
  lp.ha_RB = RB;
  lp.ha_dims = d;
  lp.ha_tasks = tb.add(tasks);
  lp.ha_leaf = tb.add(leafb);
  lp.ha_up_work = Work{0.0, fbytes_up + vbytes_up};
  lp.ha_down_work = Work{0.0, fbytes_down + vbytes_down};
  Sig sg;
  sg << nrhs << (int64_t)hod.size() << C << RB << d.rowsP << d.rowsU << d.kmax << d.kf;
  lp.ha_sig = sg.h;
  lp.ha_ok = true;
}

int get_solve_plan(hm_sys_s* sys, int nrhs, SolvePlan** out) {
  auto it = sys->solve_plans.find(nrhs);
  sys->ctx->last_nrhs = nrhs;
  if (it != sys->solve_plans.end()) {
    it->second->last_use = ++sys->plan_clock;
    *out = it->second.get();
    return HM_OK;
  }
  // keep at most kMaxSolvePlans right-hand-side counts: drop the least recently used
  if ((int)sys->solve_plans.size() >= kMaxSolvePlans) {
    auto lru = sys->solve_plans.begin();
    for (auto jt = sys->solve_plans.begin(); jt != sys->solve_plans.end(); ++jt)
      if (jt->second->last_use < lru->second->last_use) lru = jt;
    HM_CUDA(cudaStreamSynchronize(sys->ctx->stream));  // no launch of it may still run
    dev_free_all(sys->ctx, &lru->second->allocs);
    sys->solve_plans.erase(lru);
  }
  host_mark("solve plan: enter");
  Plan& P = sys->plan;
  const int es = sys->precision == HM_PREC_FP64 ? 8 : 4;
  const int nf = sys->nf;
  std::unique_ptr<SolvePlan> sp(new SolvePlan());
  sp->nrhs = nrhs;
  sp->fv_off.assign(nf, 0);
  int64_t fv = 0;
  for (int q = 0; q < nf; ++q) { sp->fv_off[q] = fv; fv += (int64_t)P.fg[q].nhat * nrhs; }
  sp->fv_total = fv;
  // scratch: per HODLR node t (2k x nrhs); per HODLR front tf (kf x nrhs).  A HODLR
  // front's pivot-block solution y lives in its own rows of the solution xfix (ld n), so
  // the downward pass needs no copy-out.
  std::vector<std::vector<int64_t>> node_sb(P.hf.size());
  std::vector<int64_t> front_sb(P.hf.size());
  int64_t sb = 0;
  for (size_t i = 0; i < P.hf.size(); ++i) {
    const HFront& h = P.hf[i];
    for (const auto& nd : h.nodes) { node_sb[i].push_back(sb); sb += (int64_t)2 * h.kl[nd.level] * nrhs; }
    front_sb[i] = sb;
    sb += (int64_t)h.kf * nrhs;
  }
  sp->sb_total = sb;
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, &sp->d_fv, (size_t)std::max<int64_t>(fv, 1) * es));
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, &sp->d_sb, (size_t)std::max<int64_t>(sb, 1) * es));
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, (void**)&sp->d_fvoff, (size_t)nf * 8));
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, &sp->d_xfix, (size_t)std::max<int64_t>((int64_t)sys->n * nrhs, 1) * es));
  HM_CUDA(cudaMemcpyAsync(sp->d_fvoff, sp->fv_off.data(), (size_t)nf * 8, cudaMemcpyHostToDevice,
                          sys->ctx->stream));
  void* XF = sp->d_xfix;
  const int n = sys->n;
  void* Bo = sys->d_bo;
  void* X = sys->d_x;
  void* W = sys->d_w;
  void* Gm = sys->d_g;
  void* FV = sp->d_fv;
  void* SB = sp->d_sb;
  TaskBuf& tb = sp->tb;
  tb.es = es;
  tb.split_target = 2 * sys->ctx->num_sms;
  sp->levels.assign(P.nlevels, LevelSolvePlan());
  for (int l = 0; l < P.nlevels; ++l) {
    LevelSolvePlan& lp = sp->levels[l];
    const auto& fr = P.level_fronts[l];
    std::vector<int> dense, hod;
    for (int q : fr) {
      const FrontGeom& g = P.fg[q];
      const auto ch = sys->children(q);
      const double np = g.np, nu = g.nu, nh = g.nhat, R = nrhs;
      double vec = es * R * (np + nh);  // read r(I_p), write fv
      for (int c : ch) vec += es * R * 3.0 * P.fg[c].nu + 4.0 * P.fg[c].nu;  // extend-add
      if (g.hodlr < 0) {
        dense.push_back(q);
        lp.dense_max_np = std::max(lp.dense_max_np, g.np);
        lp.dense_max_nhat = std::max(lp.dense_max_nhat, g.nhat);
        // up: vectors + K (nu x np); down: [b_p; -x(I_f)] in, x_p out, the first np rows
        lp.up_work.bytes += vec + es * nu * np;
        lp.up_work.flops += 2.0 * R * nu * np;
        lp.down_work.bytes += es * R * (2.0 * np + 2.0 * nu) + 4.0 * nu + es * np * nh;
        lp.down_work.flops += 2.0 * R * np * nh;
      } else {
        hod.push_back(q);
        lp.hodlr_max_nhat = std::max(lp.hodlr_max_nhat, g.nhat);
        lp.hodlr_max_nu = std::max(lp.hodlr_max_nu, g.nu);
        lp.hup_work.bytes += vec;
        lp.hdown_work.bytes += es * R * 2.0 * nu + 4.0 * nu;
      }
    }
    lp.dense = tb.add(dense);
    lp.hfronts = tb.add(hod);
    lp.n_hodlr = (int)hod.size();
    std::vector<GemmTask> ug, dg;
    std::vector<GemmTask> u2, d1, d2;
    int maxL = 0;
    for (int q : fr) {
      const FrontGeom& g = P.fg[q];
      if (g.hodlr < 0) continue;
      const HFront& h = P.hf[g.hodlr];
      maxL = std::max(maxL, h.L);
      const int64_t fvq = sp->fv_off[q], yq = sys->h_first[q];  // y = xfix rows of I_q
      for (size_t li = 0; li < h.leaf_lo.size(); ++li) {
        const int lo = h.leaf_lo[li], nl = h.leaf_hi[li] - lo;
        dg.push_back(gemm(at(sys->d_leafinv, h.lv_off + lo, es), h.np, 0, at(FV, fvq + lo, es),
                          g.nhat, 0, at(XF, yq + lo, es), n, nl, nrhs, nl, 1.0, 0.0));
      }
      if (h.kf > 0) {
        void* tf = at(SB, front_sb[g.hodlr], es);
        ug.push_back(gemm(at(X, h.bo_off, es), h.np, 1, at(FV, fvq, es), g.nhat, 0, tf, h.kf, h.kf,
                          nrhs, h.np, 1.0, 0.0));
        u2.push_back(gemm(at(W, h.w_off, es), h.nu, 0, tf, h.kf, 0, at(FV, fvq + h.np, es), g.nhat,
                          h.nu, nrhs, h.kf, -1.0, 1.0));
        d1.push_back(gemm(at(W, h.w_off, es), h.nu, 1, at(FV, fvq + h.np, es), g.nhat, 0, tf, h.kf,
                          h.kf, nrhs, h.nu, 1.0, 0.0));
        d2.push_back(gemm(at(X, h.bo_off, es), h.np, 0, tf, h.kf, 0, at(XF, yq, es), n, h.np,
                          nrhs, h.kf, 1.0, 1.0));
      }
    }
    lp.up_gemm = tb.add_gemm(ug);
    lp.up2 = tb.add_gemm(u2);
    lp.down_gemm = tb.add_gemm(dg);
    for (int ht = 1; ht <= maxL; ++ht) {
      std::vector<GemmTask> tt, upd;
      for (int q : fr) {
        const FrontGeom& g = P.fg[q];
        if (g.hodlr < 0) continue;
        const HFront& h = P.hf[g.hodlr];
        if (h.L < ht) continue;
        const int lv = h.L - ht, k = h.kl[lv], np = h.np;
        const int64_t colo = (int64_t)h.col[lv] * np, yq = sys->h_first[q];
        for (size_t ni = 0; ni < h.nodes.size(); ++ni) {
          const auto& nd = h.nodes[ni];
          if (nd.level != lv) continue;
          const int na = nd.mid - nd.lo, nb = nd.hi - nd.mid;
          void* tn = at(SB, node_sb[g.hodlr][ni], es);
          void* Gl = at(Gm, h.g_off + (int64_t)2 * (h.col[lv] - h.kf) * np, es);
          tt.push_back(gemm(at(Bo, h.bo_off + colo + nd.lo, es), np, 1, at(XF, yq + nd.lo, es), n, 0,
                            tn, 2 * k, k, nrhs, na, 1.0, 0.0));
          tt.push_back(gemm(at(Bo, h.bo_off + colo + nd.mid, es), np, 1, at(XF, yq + nd.mid, es), n, 0,
                            at(SB, node_sb[g.hodlr][ni] + k, es), 2 * k, k, nrhs, nb, 1.0, 0.0));
          // y_a -= Zhat_a s_a = (Zhat_a C^{-1}[0:k, :]) t, likewise y_b
          upd.push_back(gemm(at(Gl, nd.lo, es), np, 0, tn, 2 * k, 0, at(XF, yq + nd.lo, es), n, na, nrhs,
                             2 * k, -1.0, 1.0));
          upd.push_back(gemm(at(Gl, nd.mid, es), np, 0, tn, 2 * k, 0, at(XF, yq + nd.mid, es), n, nb, nrhs,
                             2 * k, -1.0, 1.0));
        }
      }
      LevelSolvePlan::Height H;
      H.t = tb.add_gemm(tt);
      H.upd = tb.add_gemm(upd);
      lp.heights.push_back(H);
    }
    lp.down1 = tb.add_gemm(d1);
    lp.down2 = tb.add_gemm(d2);
    plan_hodlr_apply(sys, sp.get(), lp, hod, nrhs, es);
  }
  host_mark("solve plan: tasks");
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, &sp->d_split_ws, (size_t)std::max<int64_t>(tb.split_ws, 1) * es));
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, (void**)&sp->d_split_cnt, sizeof(unsigned) * std::max(tb.split_slots, 1)));
  HM_CUDA(cudaMemsetAsync(sp->d_split_cnt, 0, sizeof(unsigned) * std::max(tb.split_slots, 1),
                          sys->ctx->stream));
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, (void**)&sp->d_tasks, std::max<size_t>(tb.host.size(), 16)));
  HM_CUDA(cudaMemcpyAsync(sp->d_tasks, tb.host.data(), tb.host.size(), cudaMemcpyHostToDevice,
                          sys->ctx->stream));
  HM_TRY(dev_alloc_ctx(sys->ctx, &sp->allocs, (void**)&sp->d_ea, sizeof(int4) * std::max<int64_t>(sp->ea_total, 1)));
  for (const auto& lp : sp->levels) HM_TRY(hodlr_child_ranges(lp, sp->d_tasks, sys, sp.get()));
  sp->last_use = ++sys->plan_clock;
  *out = sp.get();
  sys->solve_plans[nrhs] = std::move(sp);
  host_mark("solve plan: built");
  return HM_OK;
}

}  // namespace hm

namespace hm {

int rebuild_plan(hm_sys_s* sys) {
  HM_CUDA(cudaStreamSynchronize(sys->ctx->stream));
  release_solve_state(sys);
  dev_free_all(sys->ctx, &sys->plan_allocs);
  sys->plan = Plan();
  return build_plan(sys);
}

}  // namespace hm

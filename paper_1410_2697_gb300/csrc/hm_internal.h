// hm_internal.h -- host-side state of a context / system and the execution plan.
#pragma once

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "hm_common.cuh"
#include "hm_dense.cuh"

struct hm_ctx_s;
struct hm_sys_s;

namespace hm {

// Algorithmic work of one launch (minimum flops and HBM bytes of what it computes).
struct Work {
  double flops = 0, bytes = 0;
  Work& operator+=(const Work& o) { flops += o.flops; bytes += o.bytes; return *this; }
};

inline Work work_of(const GemmTask& t, int es) {
  Work w;
  const double m = t.m, n = t.n, k = t.k;
  w.flops = (t.lower ? 1.0 : 2.0) * m * n * k;
  w.bytes = es * (m * k + k * n + (t.lower ? 0.5 : 1.0) * m * n * (t.beta != 0.0 ? 2.0 : 1.0));
  return w;
}
inline Work work_of(const SweepTask& t, int es) {
  return Work{2.0 * t.np * (double)t.nhat * t.nhat, 2.0 * es * (double)t.nhat * t.nhat};
}
inline Work work_of(const PotrfTask& t, int es) {
  return Work{(double)t.n * t.n * t.n / 3.0, (double)es * t.n * (t.n + 1)};
}
inline Work work_of(const TrsmTask& t, int es) {
  const double rows = std::min(64, t.m - t.row0);
  return Work{rows * t.n * t.n, es * (2.0 * rows * t.n + 0.5 * t.n * t.n)};
}
inline Work work_of(const QrTask& t, int es) {
  return Work{4.0 * t.m * t.k * t.k, es * (3.0 * t.m * t.k + (t.R ? (double)t.k * t.k : 0.0))};
}
inline Work work_of(const BdlrTask& t, int es) {
  const double c = t.cap, mm = (double)t.mx + t.my;
  return Work{c * c * c + mm * c * c, es * (2.0 * mm * c + c * c)};
}
inline Work work_of(const SvdTask& t, int es) {
  return Work{12.0 * t.k * t.k * t.k, es * 3.0 * t.k * t.k};  // ~ per-sweep cost x 2
}
inline Work work_of(const OmegaTask& t, int es) { return Work{0.0, (double)es * t.rows * t.cols}; }
inline Work work_of(const CopyTask& t, int es) { return Work{0.0, 2.0 * es * t.rows * t.cols}; }
inline Work work_of(const CoreLuTask& t, int es) {
  const double n2 = 2.0 * t.k;
  return Work{2.0 * n2 * n2 * n2 / 3.0 + 2.0 * n2 * n2 * n2, es * 3.0 * n2 * n2};
}
inline Work work_of(const CholInvTask& t, int es) {
  const double n = t.n, m = t.m;
  return Work{n * n * n / 3.0 + n * n * n / 3.0 + m * n * n,
              es * (1.5 * n * n + 2.0 * m * n)};
}
template <typename TaskT>
inline Work work_of(const TaskT&, int) { return Work{}; }

// A typed span inside the uploaded task buffer.
template <typename TaskT>
struct Span {
  size_t off = 0;  // byte offset in the task buffer
  int count = 0;
  Work work;       // summed over the tasks
  const TaskT* dev(const unsigned char* base) const {
    return reinterpret_cast<const TaskT*>(base + off);
  }
};

struct GemmBatch {
  Span<GemmTask> tasks;
  Span<GemmTile> tiles;
  Span<GemmTile> tiles_big;  // 128 x 128 tiles for the FP32 large-tile variant (if eligible)
  Span<GemmTile> tiles_tc;   // 128 x 64 tiles for the FP32 tensor-core (3xTF32) variant
  int bn = 64;       // tile width of the batch
  int tc = 0;        // 1: tensor-core BF16 kernel (128 x 64 tiles)
  uint64_t sig = 0;  // shape signature (autotuner key)
};

// Shape signatures: FNV-1a over the integers that fix a launch's shape, so the same
// problem analysed again maps to the same autotuner choices.
struct Sig {
  uint64_t h = 1469598103934665603ull;
  Sig& operator<<(int64_t v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (uint64_t)((v >> (8 * i)) & 0xff);
      h *= 1099511628211ull;
    }
    return *this;
  }
};

// Tunable launch sites and their variants (variant 0 is the built-in default).
enum TuneSite { TS_GEMM = 1, TS_QR = 2, TS_DENSE_UP = 3, TS_DENSE_DOWN = 4, TS_HODLR_APPLY = 5 };
inline uint64_t tune_key(int site, uint64_t sig) { return sig ^ ((uint64_t)site * 0x9e3779b97f4a7c15ull); }

// Host builder of the task buffer (one upload after planning).
struct TaskBuf {
  std::vector<unsigned char> host;
  int es = 4;
  // Byte positions of pointer fields that hold byte offsets into an arena allocated
  // after planning (the panel-QR scratch); the base is added before the upload.
  std::vector<size_t> relocs;
  void relocate(const void* base) {
    for (size_t pos : relocs) {
      uintptr_t v;
      memcpy(&v, host.data() + pos, sizeof(v));
      v += (uintptr_t)base;
      memcpy(host.data() + pos, &v, sizeof(v));
    }
    relocs.clear();
  }
  template <typename TaskT>
  Span<TaskT> add(const std::vector<TaskT>& v) {
    Span<TaskT> s;
    size_t a = (host.size() + 15) & ~size_t(15);
    host.resize(a + v.size() * sizeof(TaskT));
    if (!v.empty()) memcpy(host.data() + a, v.data(), v.size() * sizeof(TaskT));
    s.off = a;
    s.count = (int)v.size();
    for (const auto& t : v) s.work += work_of(t, es);
    return s;
  }
  // Split-k bookkeeping: the largest workspace (elements) and slot count of any batch
  // (batches of one plan run one after another, so they share one workspace).
  int64_t split_ws = 0;
  int split_slots = 0;
  // A batch with fewer tiles than about two waves of the GPU (split_target = two tiles
  // per SM, set from the device's SM count) splits the k range of its long products
  // (parts of at least kSplitMinK) so that more SMs share the work.
  int split_target = 304;
  static constexpr int kSplitMinK = 128, kSplitMax = 16;
  GemmBatch add_gemm(const std::vector<GemmTask>& t, bool tc = false) {
    std::vector<GemmTile> tiles;
    GemmBatch b;
    b.tc = tc ? 1 : 0;
    b.bn = tc ? kTcBN : gemm_bn_for(t);
    const int bm = tc ? kTcBM : kGemmBM;
    int ntiles = 0;
    for (const auto& x : t) ntiles += gemm_tile_count(x, bm, b.bn);
    int slots = 0;
    int64_t ws = 0;
    for (size_t i = 0; i < t.size(); ++i) {
      int nsplit = 1;
      if (ntiles < split_target && t[i].k >= 2 * kSplitMinK)
        nsplit = std::min(std::min(split_target / std::max(ntiles, 1), t[i].k / kSplitMinK), kSplitMax);
      gemm_tiles_for(t[i], (int)i, bm, b.bn, nsplit, &tiles, &slots, &ws);
    }
    split_ws = std::max(split_ws, ws);
    split_slots = std::max(split_slots, slots);
    // FP32 batches with a product of at least one 128 x 128 tile also get the tiles of
    // the large-tile kernel (an autotuner variant)
    std::vector<GemmTile> big;
    bool eligible = !tc && es == 4 && b.bn == 64;
    bool large = false;
    for (const auto& x : t) large = large || (x.m >= kBigTile && x.n >= kBigTile && x.k >= 32);
    if (eligible && large) {
      int nbig = 0;
      for (const auto& x : t) nbig += gemm_tile_count(x, kBigTile, kBigTile);
      int bslots = 0;
      int64_t bws = 0;
      for (size_t i = 0; i < t.size(); ++i) {
        int nsplit = 1;
        if (nbig < split_target && t[i].k >= 2 * kSplitMinK)
          nsplit = std::min(std::min(split_target / std::max(nbig, 1), t[i].k / kSplitMinK), kSplitMax);
        gemm_tiles_for(t[i], (int)i, kBigTile, kBigTile, nsplit, &big, &bslots, &bws);
      }
      split_ws = std::max(split_ws, bws);
      split_slots = std::max(split_slots, bslots);
    }
    // FP32 batches holding a product of at least one 128 x 64 tile over 64 k also get the
    // tiles of the tensor-core 3xTF32 kernel (an autotuner variant)
    std::vector<GemmTile> tct;
    bool sizable = false;
    for (const auto& x : t) sizable = sizable || (x.m >= 64 && x.n >= 32 && x.k >= 64);
    if (!tc && es == 4 && sizable) {
      int ntc = 0;
      for (const auto& x : t) ntc += gemm_tile_count(x, kTcBM, kTcBN);
      int tslots = 0;
      int64_t tws = 0;
      for (size_t i = 0; i < t.size(); ++i) {
        int nsplit = 1;
        if (ntc < split_target && t[i].k >= 2 * kSplitMinK)
          nsplit = std::min(std::min(split_target / std::max(ntc, 1), t[i].k / kSplitMinK), kSplitMax);
        gemm_tiles_for(t[i], (int)i, kTcBM, kTcBN, nsplit, &tct, &tslots, &tws);
      }
      split_ws = std::max(split_ws, tws);
      split_slots = std::max(split_slots, tslots);
    }
    Sig sg;
    sg << b.bn << b.tc << (int64_t)t.size() << (int64_t)tiles.size();
    for (const auto& x : t) sg << x.m << x.n << x.k << (x.opA + 2 * x.opB + 4 * x.lower);
    b.sig = sg.h;
    b.tasks = add(t);
    b.tiles = add(tiles);
    b.tiles_big = add(big);
    b.tiles_tc = add(tct);
    return b;
  }
};

// ------------------------------------------------------------------------------------
// Launch profiler: when enabled, every launch is bracketed by a pair of CUDA events on
// its stream and tagged with a category and its algorithmic work.
// ------------------------------------------------------------------------------------
enum ProfCat {
  PC_ND = 0, PC_SYMBOLIC, PC_PERMUTE_CSR, PC_SCATTER, PC_EXTEND_ADD, PC_POTRF, PC_TRSM,
  PC_GEMM_FACTOR, PC_SKETCH, PC_QR, PC_SVD, PC_CHOL_SOLVE, PC_CORE_LU, PC_INVERSE,
  PC_UP, PC_DOWN, PC_GEMM_APPLY, PC_SPMV, PC_DOTS, PC_GS_UPDATE, PC_GMRES_SMALL, PC_VECTOR,
  PC_MEMSET, PC_SWEEP, PC_BDLR, PC_HODLR_UP, PC_HODLR_DOWN, PC_GEMM_TC, PC_PACK, PC_GROUP, PC_COUNT
};
const char* prof_cat_name(int c);

struct ProfRec {
  int cat;
  cudaEvent_t a, b;
  Work w;
  int kernels;  // kernel launches inside the bracket (0 for copies / memsets)
};

struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
};

// Autotuner state of a context: the chosen variant per (site, shape signature), and,
// while a tuning pass runs, the forced variant and one event pair per timed launch.
struct TuneRec {
  uint64_t key;
  cudaEvent_t a, b;
};
struct Tuner {
  std::unordered_map<uint64_t, int> choice;
  int force = -1;   // >= 0 while tuning: every tunable site takes this variant
  bool rec = false;
  std::vector<TuneRec> recs;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  cudaEvent_t get();
  int variant(int site, uint64_t sig) const {
    if (force >= 0) return force;
    auto it = choice.find(tune_key(site, sig));
    return it == choice.end() ? 0 : it->second;
  }
};

// Per-front geometry of the plan.
struct FrontGeom {
  int np = 0, nu = 0, nhat = 0;
  int level = 0;
  int hodlr = -1;          // index into Plan::hf, -1 for a dense front
  int64_t off = 0;         // element offset of the dense front (nhat x nhat) in the arena
  int64_t cf_off = -1;     // dense front: its packed factor (see Plan::dense_total)
};

struct HNodeGeom {
  int level, index, lo, mid, hi;
  int kb;                  // sketch width of this node's off-diagonal block
  int64_t core_off;        // C (LU) then C^{-1}: 2 (2 k_level)^2 elements in the core arena
  int64_t piv_off;         // 2 k_level ints
  int rank_slot;
  int64_t om_off, y_off, z_off, r_off, uhs_off, vh_off;  // compression scratch
  int64_t tb_off;          // factor-time t then s buffers, 2 x (2 k_level x A_level)
  int64_t u_off = 0, v_off = 0;  // F_ff nodes: the block's U (na x kb) and V (nb x kb)
};

struct HFront {
  int q;                   // front id
  int np, nu, L;
  int kf;                  // sketch width (capacity) of F_fp, 0 if nu == 0
  std::vector<int> kl;     // capacity per HODLR level
  std::vector<int> col;    // column offset of each level in Bo / X
  int xc;                  // total columns of Bo / X
  int64_t bo_off;          // np x xc (same offsets in the Bo and X arenas)
  int64_t g_off;           // np x 2 (xc - kf): G of every level (the apply's Zhat C^{-1})
  int64_t w_off;           // nu x kf
  int64_t t_off;           // kf x kf
  int64_t p_off;           // nu x kf
  int rank_slot_f;
  int64_t fom_off, fy_off, fz_off, fr_off, fuhs_off, fvh_off;
  std::vector<HNodeGeom> nodes;   // all internal nodes, level by level
  std::vector<int> leaf_lo, leaf_hi;
  std::vector<HNodeGeom> ff_nodes;  // compress_ff: internal nodes of F_ff's HODLR tree
  int64_t lv_off = 0;      // leaf inverses, packed: np x lmax (ld np), leaf [lo, hi) in rows
  int lmax = 0;            // lo..hi and columns 0..hi-lo
};

// Panel QRs of one launch group: shared-memory TSQR where the panel fits, the
// single-CTA global-memory kernel otherwise.
struct QrBatch {
  Span<QrTask> plain;
  int plain_maxm = 0;
  int64_t plain_maxmk = 0;  // largest m k of the plain panels (shared-memory-resident kernel)
  Span<TsqrTask> ts;
  Span<TsqrBlock> blocks;
  size_t smem_block = 0, smem_stack = 0;
  Work work;
  uint64_t sig = 0;  // shape signature of the plain panels (autotuner key)
  // Panels beyond shared memory, in row blocks: the blocks go with the plain panels
  // (Q_b to scratch, R_b stacked), then the stacks of R_b (stack), then
  // Y_b = Q_b Q_stack,b (combine).
  Span<QrTask> stack;
  int stack_maxm = 0;
  int64_t stack_maxmk = 0;
  GemmBatch combine;
};

struct LevelFactorPlan {
  std::vector<Span<int>> ea_parents;  // slot j: fronts of the level with more than j children
  std::vector<int> ea_max_nu;         // per slot, the largest update size of those children
  std::vector<Work> ea_work;
  Span<PotrfTask> potrf;       // dense fronts
  int potrf_maxn = 0;
  Span<TrsmTask> trsm;
  int trsm_maxn = 0;
  GemmBatch syrk;
  Span<CholInvTask> dinv;      // F_pp^{-1} and K = F_fp F_pp^{-1} of the dense fronts
  Span<SweepTask> sweep;       // dense fronts with nhat <= 128, factored in one pass
  int sweep_maxn = 0;
  Span<CopyTask> pack;         // the level's factor out of the fronts (dense and leaf inverses)
  // HODLR fronts
  Span<OmegaTask> omega;
  GemmBatch sampY, sampZ, formU, formV;
  GemmBatch ffx;               // compress_ff: F_ff's off-diagonal blocks <- V U^T
  QrBatch qrY, qrZ;
  Span<SvdTask> svd;
  int svd_maxk = 0;
  Span<BdlrTask> bdlr;         // BDLR compressor: every off-diagonal block of the level
  int bdlr_maxnh = 0, bdlr_maxcap = 0;
  int leaf_maxn = 0;
  Span<SweepTask> leaf_sweep;  // explicit leaf inverses (factorization and apply), one sweep each
  GemmBatch leaf_x;            // X (leaf rows) = K_leaf^{-1} Bo (leaf rows): the first Woodbury sweep
  struct Height {
    GemmBatch pre;            // core diagonal blocks and t = Z^T X_anc
    Span<CoreLuTask> lu;      // explicit inverse of the cores (Gauss-Jordan)
    int lu_maxk = 0;
    GemmBatch sg;             // s = C^{-1} t
    GemmBatch upd;            // X_anc -= Zhat s
    GemmBatch gm;             // G = [Zhat_a C^{-1}[0:k, :]; Zhat_b C^{-1}[k:2k, :]] for the apply
  };
  std::vector<Height> heights;
  GemmBatch schurT, schurP, schurF;
  int n_dense = 0, n_hodlr = 0;
};

// One HODLR front in the fused per-level apply kernels (hm_hodlr_apply.cu).
constexpr int kHaMaxL = 16;  // deepest HODLR tree the fused kernels take
struct HApplyTask {
  const void* X;    // np x xc (ld np): Vtilde = F_pp^{-1} V_f in the first kf columns
  const void* Bo;   // np x xc (ld np): [V_f | B_0 | ... | B_{L-1}], level l's U on the
                    // rows of each node's first child, V on the second's
  const void* G;    // np x 2 (xc - kf) (ld np): G_l = Zhat_l C_l^{-1} per level
  const void* W;    // nu x kf (ld nu): F_fp ~ W V_f^T
  const void* F;    // packed leaf inverses (np x lmax, ld np): leaf [lo, hi) in rows lo..hi
  int64_t fv_off;   // element offset of the front's vector block (nhat x nrhs)
  int q, first, np, nu, nhat, L, kf, leaf_off;  // leaf_off: its 2^L + 1 leaf boundaries
  int ea_off;       // its entries of the child-range table (C x children of them)
  int kl[kHaMaxL];  // sketch width (column capacity) per level
  int col[kHaMaxL]; // first column of each level in X / Bo
};
// Per-launch sizes of the fused kernels' shared memory (elements, maxima over the
// level's fronts).
struct HaDims {
  int rowsP, rowsU;  // pivot / update rows of one CTA
  int kmax, kf;      // widest level, widest F_fp
  int tstore;        // t of the nodes one CTA processes at once (RB columns)
};

// Solve-time plan for a given number of right-hand sides.
struct UpItem {
  int q;
};
struct LevelSolvePlan {
  Span<int> dense;             // dense fronts of the level (fused up / down kernels)
  int dense_max_np = 0, dense_max_nhat = 0;
  Work up_work, down_work;     // the fused dense kernels
  Span<int> hfronts;           // HODLR fronts of the level
  int n_hodlr = 0;
  int hodlr_max_nhat = 0, hodlr_max_nu = 0;
  Work hup_work, hdown_work;   // HODLR vector kernels (init + extend-add; gather)
  GemmBatch up_gemm;           // HODLR: tf = Vtilde^T b_p
  GemmBatch up2;               // HODLR: f -= W tf
  GemmBatch down_gemm;         // HODLR leaves: y = K^{-1} b
  struct Height {
    GemmBatch t;               // t = [U^T y_a; V^T y_b]
    GemmBatch upd;             // y -= G t  (G = Zhat C^{-1}, formed by the factorization)
  };
  std::vector<Height> heights;
  GemmBatch down1, down2;      // tf = W^T (-x_f) ; y += Vtilde tf
  // fused kernels: one cluster of ha_C CTAs per (HODLR front, group of ha_RB
  // right-hand sides), one launch per pass (ha_ok: the level fits them)
  bool ha_ok = false;
  int ha_C = 1, ha_RB = 1;
  HaDims ha_dims{};
  Span<HApplyTask> ha_tasks;
  Span<int> ha_leaf;
  uint64_t ha_sig = 0;         // autotuner key (fused kernels or the GEMM path)
  Work ha_up_work, ha_down_work;
};

struct SolvePlan {
  int nrhs = 0;
  std::vector<LevelSolvePlan> levels;
  std::vector<int64_t> fv_off;  // per front, element offset of its (nhat x nrhs) vector
  int64_t fv_total = 0;
  int64_t sb_total = 0;         // node t/s buffers + tf buffers
  TaskBuf tb;
  unsigned char* d_tasks = nullptr;
  void* d_split_ws = nullptr;       // T, split-k partial sums of the apply GEMMs
  unsigned* d_split_cnt = nullptr;
  void* d_fv = nullptr;         // T
  void* d_sb = nullptr;         // T
  void* d_xfix = nullptr;       // T, n x nrhs: the solution (task tables point into it)
  int64_t* d_fvoff = nullptr;
  int4* d_ea = nullptr;         // per (fused HODLR task, CTA, child): the child's relative-map
  int64_t ea_total = 0;         // ranges landing on the CTA's pivot and update rows
  // captured apply (graph of the launches for input graph_in) and the last input seen
  std::vector<void*> allocs;    // device memory of this plan (freed when it is dropped)
  int64_t last_use = 0;
  cudaGraphExec_t graph_exec = nullptr;
  const void* graph_in = nullptr;
  const void* last_in = nullptr;
  ~SolvePlan() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
  }
};

struct Plan {
  std::vector<FrontGeom> fg;
  std::vector<HFront> hf;
  std::vector<std::vector<int>> level_fronts;   // fronts per depth
  int nlevels = 0;
  int64_t front_total = 0, bo_total = 0, w_total = 0, t_total = 0, p_total = 0, g_total = 0;
  int64_t core_total = 0, piv_total = 0, comp_total = 0, tb_total = 0;
  int64_t qr_scratch = 0;  // elements of the TSQR scratch arena (reused by every QR launch)
  int nrank = 0;
  std::vector<int64_t> level_front_begin, level_front_end;   // element ranges per level
  std::vector<int64_t> level_entries;  // A's lower entries per level, estimated (grid sizes)
  std::vector<LevelFactorPlan> levels;
  TaskBuf tb;
  unsigned char* d_tasks = nullptr;
  void* d_split_ws = nullptr;       // T, split-k partial sums of the factor GEMMs
  unsigned* d_split_cnt = nullptr;  // split-k arrival counters (zero between launches)
  int64_t* d_front_off = nullptr;
  int* d_nhat = nullptr;
  int* d_np = nullptr;
  int* d_hkind = nullptr;  // per front: -1 dense, else HODLR index
  // host copies of the uploaded per-front arrays (kept while the copies may be in flight)
  std::vector<int64_t> h_front_off;
  std::vector<int> h_nhat, h_np, h_hkind;
  int max_children = 0;
  double factor_bytes = 0;
  double stored_bytes = 0;   // factor data the apply reads (see hm_factor_info)
  // Packed factor, written level by level as the fronts are factored (the apply reads
  // only these, so the front storage may be reused): per dense front [F_pp^-1 | K^T]
  // (np x nhat, ld np) then K (nu x np, ld nu); per HODLR front its leaf inverses.
  int64_t dense_total = 0, leaf_total = 0;
  bool reuse = false;               // front storage shared by the levels of each parity
  int64_t* d_cf_off = nullptr;      // per front: packed dense factor offset
  int* d_flevel = nullptr;          // per front: tree depth
  std::vector<int64_t> h_cf_off;
  std::vector<int> h_flevel;
};

struct DevArena {
  std::vector<void*> ptrs;
};

// A device-memory budget shared by several contexts (the serving workers, which also
// share one memory pool): every allocation and free of a context that points here, and
// every read or move of its allocation records, holds `mu`.
struct SharedBudget {
  std::mutex mu;
  size_t limit = 0;  // bytes the contexts may hold together; 0 = no limit
  size_t used = 0;   // bytes they hold now
};

}  // namespace hm

struct hm_ctx_s {
  hm_opts opts;
  hm::Profiler prof;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t allocated = 0;
  int max_smem = 0;
  int num_sms = 0;
  int last_nrhs = 0;             // right-hand-side count of the most recent apply plan
  hm::Tuner tune;
  cudaMemPool_t pool = nullptr;  // stream-ordered pool; freed memory is kept for reuse
  bool own_pool = true;          // false: the pool belongs to another context
  hm::SharedBudget* shared = nullptr;  // budget shared with other contexts, or null
  std::vector<void*> allocs;     // (bytes, pointer) pairs of the live allocations
  void* noalloc_scratch = nullptr;  // device address of the allocation-free apply's array
  // adaptive rank: sketch width per front level learned for an analysis (key: its shape
  // signature), so a later analysis of the same pattern starts from the grown widths
  std::unordered_map<uint64_t, std::vector<int>> level_widths;
};

struct hm_sys_s {
  hm_ctx_s* ctx = nullptr;
  int n = 0;
  int64_t nnz = 0;
  int nf = 0;
  int dim = 0;
  int precision = HM_PREC_MIXED;
  // pattern and ordering (device)
  int64_t* d_rowptr = nullptr;
  int32_t* d_colidx = nullptr;
  int32_t* d_perm = nullptr;
  int32_t* d_iperm = nullptr;
  int32_t* d_first = nullptr;
  int32_t* d_parent = nullptr;
  int32_t* d_node_of = nullptr;
  // independent blocks (batched meshes): unknowns [seg_ptr[b], seg_ptr[b+1]) in both
  // numberings; GMRES runs one instance per block and right-hand side
  int nseg = 1;
  std::vector<int32_t> h_seg_ptr;
  int32_t* d_seg_ptr = nullptr;
  int32_t* d_child_ptr = nullptr;
  int32_t* d_child_list = nullptr;
  int64_t* d_prowptr = nullptr;
  int32_t* d_pcol = nullptr;
  int64_t* d_psrc = nullptr;
  int64_t* d_amap = nullptr;
  // symbolic (device)
  int32_t* d_nupd = nullptr;
  int64_t* d_ifoff = nullptr;
  int32_t* d_iflist = nullptr;
  int32_t* d_relmap = nullptr;
  int64_t if_total = 0;
  // host copies
  std::vector<int32_t> h_first, h_parent, h_level, h_nupd;
  std::vector<int64_t> h_ifoff;
  std::vector<int32_t> h_child_ptr, h_child_list;  // children (ascending), CSR by parent
  struct Children {
    const int32_t* b;
    const int32_t* e;
    const int32_t* begin() const { return b; }
    const int32_t* end() const { return e; }
    int size() const { return (int)(e - b); }
    int32_t operator[](int i) const { return b[i]; }
  };
  Children children(int q) const {
    return Children{h_child_list.data() + h_child_ptr[q], h_child_list.data() + h_child_ptr[q + 1]};
  }
  // plan + numeric state
  hm::Plan plan;
  void* d_front = nullptr;   // T arena
  void* d_bo = nullptr;      // T
  void* d_x = nullptr;       // T
  void* d_g = nullptr;       // T, the apply's G = Zhat C^{-1} per HODLR level
  void* d_w = nullptr;       // T
  void* d_tm = nullptr;      // T
  void* d_pm = nullptr;      // T
  void* d_core = nullptr;    // T
  int* d_piv = nullptr;
  void* d_comp = nullptr;    // T
  void* d_qrs = nullptr;     // T, TSQR scratch
  void* d_dfac = nullptr;    // T, packed dense-front factors
  void* d_leafinv = nullptr; // T, packed HODLR leaf inverses
  // A's lower-triangle entries grouped by the tree depth of their front: value index and
  // element offset in the front storage; [lev_range[2 l], lev_range[2 l + 1]) per depth
  int64_t* d_scat_src = nullptr;
  int64_t* d_scat_dst = nullptr;
  int64_t* d_lev_range = nullptr;
  void* d_tb = nullptr;      // T
  int* d_ranks = nullptr;
  double* d_pvals = nullptr; // permuted A values (FP64) for SpMV
  float2* d_pvals2 = nullptr;  // the same split as FP32 hi + lo (double-float SpMV)
  int* d_err = nullptr;      // device error word (4 ints)
  bool factored = false;
  double tol = 0;
  std::map<int, std::unique_ptr<hm::SolvePlan>> solve_plans;
  int64_t plan_clock = 0;
  std::vector<void*> allocs;
  std::vector<void*> plan_allocs;     // device memory of the plan (rebuilt when widths grow)
  std::vector<int> level_width;       // sketch width per front level (empty: opts.samples)
  uint64_t shape_sig = 0;             // analysis signature (key of ctx->level_widths)
  // GMRES workspace (grown on demand)
  struct Gm {
    int nrhs = 0, m = 0;
    double *V = nullptr, *w = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;
    double *b = nullptr, *x = nullptr, *r = nullptr, *bnorm = nullptr, *res = nullptr, *y = nullptr;
    double *part = nullptr, *hv = nullptr;
    void* Z = nullptr;  // T, m x nrhs x n
    void* wT = nullptr; // T, n x nrhs (apply input)
    int* len = nullptr;
    double* h_res = nullptr;  // pinned
    std::vector<void*> allocs;
    int nchunks = 0;                          // row chunks (never straddling a block)
    int *crow = nullptr, *cseg = nullptr, *cptr = nullptr;  // chunk rows, block, chunks per block
    // slot session (serving): per column, occupied / tolerance / iterations / cap / ||b|| /
    // last true relative residual; `fresh` marks columns whose norms must be computed
    std::vector<char> on, fresh;
    std::vector<double> rtol, bnorm_h, relres;
    std::vector<int> iters, cap;
  } gm;
};

namespace hm {

// RAII launch bracket: records events around the launches in its scope when profiling.
struct ProfScope {
  hm_ctx_s* ctx;
  int cat;
  Work w;
  int nk;
  cudaEvent_t a = nullptr;
  ProfScope(hm_ctx_s* c, int category, Work work, int kernels = 1)
      : ctx(c), cat(category), w(work), nk(kernels) {
    if (ctx->prof.on) {
      a = ctx->prof.get();
      cudaEventRecord(a, ctx->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = ctx->prof.get();
      cudaEventRecord(b, ctx->stream);
      ctx->prof.recs.push_back(ProfRec{cat, a, b, w, nk});
    }
  }
};

// Times one tunable launch while a tuning pass runs (events on the context's stream).
struct TuneScope {
  hm_ctx_s* ctx;
  uint64_t key;
  cudaEvent_t a = nullptr;
  TuneScope(hm_ctx_s* c, int site, uint64_t sig) : ctx(c), key(tune_key(site, sig)) {
    if (ctx->tune.rec) {
      a = ctx->tune.get();
      cudaEventRecord(a, ctx->stream);
    }
  }
  ~TuneScope() {
    if (a) {
      cudaEvent_t b = ctx->tune.get();
      cudaEventRecord(b, ctx->stream);
      ctx->tune.recs.push_back(TuneRec{key, a, b});
    }
  }
};

int dev_alloc(hm_sys_s* sys, void** p, size_t bytes);
int dev_alloc_ctx(hm_ctx_s* ctx, std::vector<void*>* owner, void** p, size_t bytes);
void dev_free_all(hm_ctx_s* ctx, std::vector<void*>* owner);
std::unique_lock<std::mutex> alloc_lock(const hm_ctx_s* ctx);
int move_sys(hm_sys_s* sys, hm_ctx_s* to, cudaEvent_t ready);
size_t sys_bytes(const hm_sys_s* sys);  // device bytes a system holds (all its owners)
int check_device_error(hm_sys_s* sys, const char* where);
bool is_device_ptr(const void* p);
int copy_in(hm_sys_s* sys, void* dst, const void* src, size_t bytes);

int analyze_impl(hm_sys_s* sys, const int64_t* rowptr, const int32_t* colidx, int dim,
                 const int32_t* coords, const int32_t* perm_in, int nfronts_in,
                 const int32_t* first_in, const int32_t* parent_in, int nblocks,
                 const int32_t* block_ptr);
int build_plan(hm_sys_s* sys);
// Frees the plan's device memory and builds it again (after the sketch widths changed).
int rebuild_plan(hm_sys_s* sys);
int factor_impl(hm_sys_s* sys, const double* d_values, double tol);
// Apply plans are kept for at most this many right-hand-side counts per system.
constexpr int kMaxSolvePlans = 4;
int get_solve_plan(hm_sys_s* sys, int nrhs, SolvePlan** out);
// Frees the per-right-hand-side-count state of a system (apply plans, GMRES workspace);
// it is rebuilt on the next solve.
void release_solve_state(hm_sys_s* sys);
// z (T, n x nrhs, ld n, new numbering) = M^{-1} r (T, same layout)
int apply_impl(hm_sys_s* sys, int nrhs, const void* rT, void* zT);
// As apply_impl, always launched kernel by kernel: never captures or instantiates a
// CUDA graph (the driver allocates for those).
int apply_impl_eager(hm_sys_s* sys, int nrhs, const void* rT, void* zT);
// As apply_impl, with z written row-major (element (i, r) at i nrhs + r).
int apply_impl_rowmajor(hm_sys_s* sys, int nrhs, const void* rT, void* zT);
int solve_setup(int max_smem);
// The fused HODLR-front apply of one level (upward: down = false, input win; downward:
// solution rows of the level's fronts into xv).
// rb: right-hand sides per cluster (1, 2, 4, 8 or 16, at most lp.ha_RB); nt: threads per
// CTA (256, or 512 for rb <= 4).
template <typename T>
int launch_hodlr_apply(bool down, const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys,
                       SolvePlan* sp, int nrhs, const T* win, T* xv, int rb, int nt);
size_t hodlr_apply_smem(const HaDims& d, int RB, bool down, int es);
int hodlr_apply_setup(int max_smem);
int hodlr_child_ranges(const LevelSolvePlan& lp, const unsigned char* base, hm_sys_s* sys, SolvePlan* sp);
int direct_impl(hm_sys_s* sys, int nrhs, const double* d_b, int refine, double* d_x, hm_solve_info* info);
// Slot sessions of GMRES for serving: nslots columns, each its own instance.  A right-hand
// side enters a free slot between restart cycles (gm_session_put, host array in the
// original numbering) and leaves when taken (gm_session_take, x to a host array); each
// gm_session_cycle runs one restart cycle over the occupied, unconverged slots (one
// system, no batch of meshes).
int gm_session_begin(hm_sys_s* sys, int nslots);
int gm_session_put(hm_sys_s* sys, int slot, const double* b_host, double rtol, int max_iters);
int gm_session_cycle(hm_sys_s* sys, int* its);
// state of a slot: 1 = converged, 0 = running, -1 = its iteration cap was reached
int gm_session_state(const hm_sys_s* sys, int slot, double* relres, int* iters);
int gm_session_take(hm_sys_s* sys, int slot, double* x_host);
int gmres_impl(hm_sys_s* sys, int nrhs, const double* d_b, double rtol, int max_iters,
               double* d_x, hm_solve_info* info);
// permutation helpers (new <-> original numbering), FP64 n x nrhs
void launch_permute_in(const double* src, double* dst, const int32_t* perm, int n, int nrhs,
                       cudaStream_t s);
void launch_permute_out(const double* src, double* dst, const int32_t* perm, int n, int nrhs,
                        cudaStream_t s);
template <typename T>
void launch_cast_to(const double* src, T* dst, int64_t count, cudaStream_t s);
template <typename T>
void launch_cast_from(const T* src, double* dst, int64_t count, cudaStream_t s);

}  // namespace hm

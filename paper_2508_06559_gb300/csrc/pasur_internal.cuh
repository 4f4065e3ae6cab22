// Internal declarations of the Pasur GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pasur.h"

// ---------------------------------------------------------------------------------------------
// Cards (the paper's Fig. "Mapping Cards to Indices" and Table card index sets):
// id = 4*rank + suit; ranks Ace..Ten are the numeric cards 0..39, Jacks 40..43, Queens 44..47,
// Kings 48..51; clubs are the ids divisible by 4.
// ---------------------------------------------------------------------------------------------
namespace pasur {

constexpr uint64_t kNumeric = (1ULL << 40) - 1ULL;
constexpr uint64_t kJacks = 0xFULL << 40;
constexpr uint64_t kQueens = 0xFULL << 44;
constexpr uint64_t kKings = 0xFULL << 48;
constexpr uint64_t kClubs = 0x0001111111111111ULL;  // bits 0, 4, ..., 48
constexpr uint64_t kAces = 0xFULL;
constexpr int kTwoClubs = 4;
constexpr int kTenDiamonds = 37;

// Points of a captured set (Table "Pasur Scoring System"): Aces and Jacks 1, two of clubs 2,
// ten of diamonds 3.
__host__ __device__ __forceinline__ int set_points(uint64_t m) {
#ifdef __CUDA_ARCH__
    return __popcll(m & (kAces | kJacks)) + 2 * (int)((m >> kTwoClubs) & 1ULL) +
           3 * (int)((m >> kTenDiamonds) & 1ULL);
#else
    return __builtin_popcountll(m & (kAces | kJacks)) + 2 * (int)((m >> kTwoClubs) & 1ULL) +
           3 * (int)((m >> kTenDiamonds) & 1ULL);
#endif
}

__host__ __device__ __forceinline__ int set_clubs(uint64_t m) {
#ifdef __CUDA_ARCH__
    return __popcll(m & kClubs);
#else
    return __builtin_popcountll(m & kClubs);
#endif
}

// Running score of a round packed in bytes of a uint64 (Table "Column definitions for the
// running-score tensor"): [0] Alex clubs [1] Bob clubs [2] last picker (0/1/2) [3] Alex points
// [4] Alex surs [5] Bob points [6] Bob surs.
__host__ __device__ __forceinline__ int rus_get(uint64_t r, int f) { return (int)((r >> (8 * f)) & 0xFFULL); }
__host__ __device__ __forceinline__ uint64_t rus_add(uint64_t r, int f, int v) { return r + ((uint64_t)(uint32_t)v << (8 * f)); }
__host__ __device__ __forceinline__ uint64_t rus_set(uint64_t r, int f, int v) {
    return (r & ~(0xFFULL << (8 * f))) | ((uint64_t)(v & 0xFF) << (8 * f));
}
// Alex minus Bob points of the round, 5 per Sur.
__host__ __device__ __forceinline__ int rus_diff(uint64_t r) {
    return (rus_get(r, 3) + 5 * rus_get(r, 4)) - (rus_get(r, 5) + 5 * rus_get(r, 6));
}

struct __align__(16) GTState {
    uint64_t hand[2];  // Alex, Bob
    uint64_t pool;
    uint64_t rus;
};

// Score normalisation (section "Score Tensors"): a player with at least 7 clubs earns the bonus and
// both club counts reset to 0; with a bonus recorded clubs are not tracked.
__host__ __device__ __forceinline__ void normalize_score(int &ac, int &bc, int &bonus) {
    if (bonus == 0) {
        if (ac >= 7) { ac = 0; bc = 0; bonus = 1; }
        else if (bc >= 7) { ac = 0; bc = 0; bonus = 2; }
    } else {
        ac = 0;
        bc = 0;
    }
}

// CleanUp at the end of the final round (caption of Fig. game_0): the last picker takes what is
// left in the pool with its clubs and points; with no picker in the round the pool is discarded.
__host__ __device__ __forceinline__ uint64_t cleanup_rus(uint64_t r, uint64_t pool) {
    int L = rus_get(r, 2);
    if (L != 0 && pool != 0) {
        int w = L - 1;
        r = rus_add(r, w, set_clubs(pool));
        r = rus_add(r, 3 + 2 * w, set_points(pool));
    }
    return r;
}

// Owner of the 7-clubs bonus (0 none, 1 Alex, 2 Bob) after a round that ends with running score
// r from the root score (clubs carried, bonus recorded), and its points for Alex (eq. final_util).
__host__ __device__ __forceinline__ int bonus_after(int a_clubs, int b_clubs, int bonus, uint64_t r) {
    int ac = a_clubs + rus_get(r, 0), bc = b_clubs + rus_get(r, 1), bn = bonus;
    normalize_score(ac, bc, bn);
    return bn;
}
__host__ __device__ __forceinline__ int bonus_points(int bonus) { return bonus == 1 ? 7 : (bonus == 2 ? -7 : 0); }

// Sort key of a score: ascending key = lexicographic (a_clubs, b_clubs, delta, bonus), signed.
__host__ __device__ __forceinline__ uint32_t score_key(int ac, int bc, int delta, int bonus) {
    return ((uint32_t)ac << 22) | ((uint32_t)bc << 18) | ((uint32_t)(delta + 32768) << 2) | (uint32_t)bonus;
}
__host__ __device__ __forceinline__ void score_unkey(uint32_t k, int &ac, int &bc, int &delta, int &bonus) {
    ac = (int)(k >> 22);
    bc = (int)((k >> 18) & 0xF);
    delta = (int)((k >> 2) & 0xFFFF) - 32768;
    bonus = (int)(k & 3);
}
constexpr int kScoreKeyBits = 26;

}  // namespace pasur

// ---------------------------------------------------------------------------------------------
// Context and tree objects
// ---------------------------------------------------------------------------------------------
struct pasur_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the context's stream-ordered memory pool: freed blocks stay reserved for the next
    // allocation (a solve's arrays are reused by the next solve without new mappings) until
    // pasur_destroy returns them
    cudaMemPool_t pool = nullptr;
    // device-to-host copies of asynchronous exports (created on first use), after an event on
    // the context's stream; pasur_sync waits for them
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_after = nullptr;
    size_t budget = 0, in_use = 0, peak = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    std::string err;
    // capture table of numeric moves: per numeric card c, the picked sets completing it to 11,
    // ascending; tab_off[41]
    uint64_t *tab = nullptr;
    int32_t *tab_off = nullptr;
    int32_t *counter = nullptr;  // work-queue counters (device)
    int32_t *errflag = nullptr;  // device error word
    int64_t launches = 0;        // kernels launched through this context
    // forked streams for concurrent launches (created on first use): CFR classes 0..5, cluster
    // launches 6..9
    cudaStream_t aux[12] = {nullptr};
    cudaEvent_t fork = nullptr, join[12] = {nullptr}, cls_t0[12] = {nullptr}, cls_t1[12] = {nullptr};
    int64_t live_trees = 0;      // trees not yet freed (the context outlives them)
    bool cfr_smem_raised = false;  // CFR kernels' dynamic shared-memory limit raised
    float selfplay_ms = 0.f;     // device time of the last self-play launch
    int64_t selfplay_games = 0;  //   and its number of games
    // a batch's build workers each own a context with its own stream and error word; their
    // allocations are charged to (and limited by the budget of) the parent context
    pasur_ctx *acct = nullptr;
    std::mutex acct_mu;
};

// Host phases of a call under PASUR_VERBOSE: each mark waits for the context's stream and prints
// the wall time since the previous mark (a diagnostic; without the variable it does nothing).
struct PhaseTimer {
    cudaStream_t stream;
    const char *what;
    bool on;
    std::chrono::steady_clock::time_point t0;
    PhaseTimer(cudaStream_t s, const char *w) : stream(s), what(w), on(getenv("PASUR_VERBOSE") != nullptr) {
        if (on) {
            cudaStreamSynchronize(stream);
            t0 = std::chrono::steady_clock::now();
        }
    }
    void mark(const char *phase) {
        if (!on) return;
        cudaStreamSynchronize(stream);
        const auto t1 = std::chrono::steady_clock::now();
        fprintf(stderr, "[pasur] %s: %s %.2f ms\n", what, phase, std::chrono::duration<double, std::milli>(t1 - t0).count());
        t0 = t1;
    }
};

struct RootInfo {             // one GT root's subtree, level by level
    int64_t lvl_begin[9];     // first GT node of the root at level k
    int32_t lvl_count[9];     // its GT nodes at level k
    int32_t local_start[10];  // local (level-major) index of its first node at level k; [9] = nodes
    int64_t struct_off;       // offset of its internal nodes in the local structure arrays
    int32_t n_internal;       // nodes at levels 0..7
    int32_t pad;
};

// CFR view of one GT root's subtree.  Nodes whose whole subtree is a single path of forced moves
// ("chains") have a fixed value, sigma = 1 and zero regret on every edge below them, so the CFR
// state is kept only for the "local" nodes: the root and every child of an "active" node (a
// local node that is not a chain).  Local nodes are numbered level by level in GT order; chain
// nodes among them are "terminals" whose value is the leaf at the end of their chain.
struct CfrRoot {
    int32_t ls[10];           // first local index of level k; ls[9] = number of local nodes L
    int32_t as[10];           // first active entry of level k; as[8] = as[9] = active nodes
    int64_t loc_off;          // offset of the root's local nodes in the per-local arrays
    int64_t act_off;          // offset of the root's active entries in the per-active arrays
    int64_t locbase[9];       // global local-rank of the root's first node at level k
    int64_t actbase[9];       // global active-rank of the root's first node at level k
    int32_t W;                // slots per work item of this root
    int32_t cls;              // launch class of its items
    int64_t item0;            // index of its first work item
};

// A root subtree too large for one block's shared memory, split over a thread-block cluster:
// CTA 0 holds the top levels 0..ell-1 (and part 0), CTA r holds part r, a set of subtrees of
// active level-ell nodes.  Parts and top are pseudo-roots (CfrRoot records appended after the real
// roots) with their own local numbering; each active level-ell node has a ghost slot in its part
// for its parent's reach.
struct ClusterPart {
    int32_t root;             // pseudo-root
    int32_t pad;
    int64_t data_base;        // its regrets and strategy sums in R and S
};

struct ClusterItem {
    int32_t tree, root;       // launch tree index, real GT root
    int64_t s0;               // slot (one per cluster item)
    int64_t part0;            // cparts[part0] = top, cparts[part0 + 1 + r] = part r
    int64_t x0;               // exchange entries cx[x0 .. x0 + nx) (5 ints each)
    int32_t nx, nparts;
    int32_t ell, smem;        // split level; shared memory of its largest CTA
};

// Per-tree pointers of the CFR kernel (one entry per round tree of a launch).
struct TreeView {
    const CfrRoot *roots;
    const int32_t *act_li, *act_pl, *act_cs;
    const uint16_t *act_d;
    const int64_t *loc_tq;
    const float *leaf_v;
    const int64_t *fgt_off0;
    float *R, *S, *V, *X;
    double *uacc;
    const ClusterPart *cparts;   // cluster items: parts table
    const int32_t *cx;           // cluster items: (part, top node, top parent, part node, part ghost)
};

struct CfrItem {              // one work item of the CFR kernel: a root and a run of its slots
    int32_t root;
    int32_t tree;             // index into the launch's TreeView table
    int32_t ns;               // slots in the item
    int32_t width;            // largest number of (active node, slot) pairs of one level
    int64_t s0;               // first slot of the item within its root
    int64_t data_base;        // offset of the item's (local node, slot) table in R and S
    int64_t scratch_base;     // offset in the global transients, or -1 when the item is resident
    int64_t cost;             // active nodes * slots, for the schedule
};

// cluster items are launched in groups by their CTA count: clusters of 2, 4, 8 and 16 CTAs
constexpr int kCluGroups = 4;

// One item of the level-streaming sweep, resolved once per plan: its state arrays, its active
// entries (offsets applied), the level starts of its entries, its slot count (a power of two) and
// the index of its first slot in the per-slot arrays of the sweep.
struct StreamDesc {
    float *R, *S, *V, *X;
    const int32_t *li, *pl, *cs;
    const uint16_t *d;
    int32_t as[9];
    int32_t sh, ns;
    int64_t slot;
};

// A CFR launch plan: work items of one or more trees merged per shared-memory class.
struct CfrPlan {
    std::vector<CfrItem> items_h;       // ordered by class, then cost (largest first)
    CfrItem *items_d = nullptr;
    TreeView *views_d = nullptr;
    int64_t n_items = 0;
    int64_t cls_begin[8] = {0}, cls_end[8] = {0};
    size_t cls_smem[8] = {0};
    int cls_blocks[8] = {0};
    int cls_threads[8] = {0};
    float cls_ms[12] = {0};
    // cluster items (class 6 holds their pseudo-items, used for exports only), sorted by part
    // count into up to four launches of 2, 4, 8 and 16 CTAs per cluster
    std::vector<ClusterItem> clu_h;
    ClusterItem *clu_d = nullptr;
    int clu_threads = 0;
    int64_t clu_begin[kCluGroups] = {0}, clu_end[kCluGroups] = {0};
    int clu_ctas[kCluGroups] = {2, 4, 8, 16};
    size_t clu_smem[kCluGroups] = {0};
    // items of class 5 (state in device memory) run as a level-streaming sweep over every SM:
    // exclusive prefixes over those items of their (entry, slot) pairs per level [8][n + 1], of
    // their (local node, slot) pairs [n + 1] and of their slots [n + 1]; per slot the largest
    // |terminal value| (float bits) and the sum of the root values of the current call
    int64_t str_n = 0, str_nslots = 0;
    int64_t *str_pairs = nullptr, *str_locs = nullptr, *str_slots = nullptr;
    uint32_t *str_tu = nullptr;
    double *str_acc = nullptr;
    struct StreamDesc *str_desc = nullptr;  // per class-5 item: what its (entry, slot) pairs need
};

struct pasur_tree {
    pasur_ctx *ctx = nullptr;
    int round = 0;
    bool final_round = false;
    uint8_t deck[52];
    uint64_t hand_a = 0, hand_b = 0;
    int64_t n_roots = 0;
    int64_t M[9] = {0};
    // game tree, level by level (device)
    pasur::GTState *st[9] = {nullptr};
    int64_t *child_off[9] = {nullptr};  // levels 0..7: M[k]+1
    int64_t *parent[9] = {nullptr};     // levels 1..8
    int8_t *lay[9] = {nullptr};         // levels 1..8
    uint64_t *pick[9] = {nullptr};      // levels 1..8
    int32_t *root[9] = {nullptr};       // root id of every node
    std::vector<RootInfo> roots_h;
    int64_t *bounds_d = nullptr;        // [n_roots+1][9]: first GT node of root g at level k
    // full game tree
    bool unfolded = false;
    int64_t Q[9] = {0};
    int64_t *fgt_off[9] = {nullptr};    // M[k]+1
    int64_t *score_off_d = nullptr;
    pasur_score *scores_d = nullptr;
    std::vector<int64_t> score_off_h;
    std::vector<pasur_score> scores_h;
    // score slots the CFR solves.  Slots of one root whose leaf values coincide for every leaf
    // give identical CFR runs; with merging, the slots of a root that share (a_clubs, b_clubs,
    // bonus) -- which differ only in the inherited difference, which no utility contains (eq.
    // final_util, eq. passuputil) -- are solved once.  "Solved slots" are numbered per root in
    // order of their first full slot; without merging they are the full slots.
    bool merged = false;
    std::vector<int64_t> csoff_h;       // [n_roots+1] solved slots per root (prefix)
    int64_t *csoff_d = nullptr;
    int32_t *crep_d = nullptr;          // [cQ[0]] per solved slot: its first full slot within the root
    int64_t *cidx0_d = nullptr;         // [Q[0]] per full root slot: the global index of its solved slot
    int32_t *cmult_d = nullptr;         // [cQ[0]] per solved slot: the number of full slots it stands for
    int64_t *cfgt_off[9] = {nullptr};   // per GT node: first solved FGT node (= fgt_off unless merged)
    int64_t cQ[9] = {0};                // solved FGT level sizes
    int64_t swept_edges = 0;            // (local non-root node, solved slot) pairs: edges with CFR state
    int64_t swept_pairs = 0;            // (active node, solved slot) pairs: node updates per iteration
    // next round links
    bool has_next = false;
    int64_t *lnk_d = nullptr;           // Q[8]
    int64_t n_next_roots = 0;
    std::vector<uint64_t> next_pools_h;
    std::vector<int64_t> next_soff_h;
    std::vector<pasur_score> next_scores_h;
    // CFR state
    bool cfr_ready = false;
    int64_t iters_done = 0;
    float umax = 0.f;
    float *leaf_v = nullptr;            // cQ[8], solved FGT order
    std::vector<CfrRoot> croots_h;
    CfrRoot *croots_d = nullptr;
    int32_t *act_li = nullptr;          // per active entry: its local index
    int32_t *act_pl = nullptr;          //   local index of its parent (-1 at the root)
    int32_t *act_cs = nullptr;          //   local index of its first child
    uint16_t *act_d = nullptr;          //   number of children
    int64_t *act_gt = nullptr;          //   GT node index
    int64_t *loc_tq = nullptr;          // per local node: FGT index (slot 0) of its chain's leaf, -1 if active
    int64_t n_local = 0, n_active = 0;
    std::vector<ClusterPart> cparts_h;  // cluster items of this tree
    std::vector<int32_t> cx_h;
    ClusterPart *cparts_d = nullptr;
    int32_t *cx_d = nullptr;
    CfrPlan plan;                       // this tree alone
    TreeView view{};                    // its pointers for the CFR kernel
    int64_t data_size = 0, scratch_size = 0;
    float *R = nullptr, *S = nullptr;   // per (local node, slot) of every item
    float *V = nullptr, *X = nullptr;   // values and reaches of the non-resident items
    double *uacc = nullptr;             // cQ[0]

    int32_t variant = -1;
    // GT roots the CFR solves: [range_first, range_first + range_count) (the whole round unless a
    // caller shards the roots over several solvers)
    int64_t range_first = 0, range_count = -1;
    bool in_range(int64_t g) const { return range_count < 0 || (g >= range_first && g < range_first + range_count); }
    float last_ms = 0.f;
    int32_t last_launches = 0;
    std::vector<void *> allocs;
};

// ---------------------------------------------------------------------------------------------
// Helpers shared by the library's translation units
// ---------------------------------------------------------------------------------------------
namespace pasur {

int set_err(pasur_ctx *ctx, int code, const std::string &msg);
int cuda_err(pasur_ctx *ctx, cudaError_t e, const char *what);
int dev_alloc(pasur_ctx *ctx, void **p, size_t bytes);
void dev_free(pasur_ctx *ctx, void *p, size_t bytes);
int tree_alloc(pasur_tree *t, void **p, size_t bytes);  // freed with the tree
bool is_device_ptr(const void *p);

#define PASUR_CUDA(ctx, call)                                   \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::pasur::cuda_err((ctx), e_, #call); \
    } while (0)
#define PASUR_TRY(call)            \
    do {                           \
        int rc_ = (call);          \
        if (rc_ != PASUR_OK) return rc_; \
    } while (0)

// scan_sort.cu
// out[i] = sum_{j<i} in[i] for i in [0, n], out has n+1 entries (out[n] = total); in is int32
// or int64 (device).  Scratch is allocated from ctx.
int exclusive_scan_i32(pasur_ctx *ctx, const int32_t *in, int64_t *out, int64_t n);
int exclusive_scan_i64(pasur_ctx *ctx, const int64_t *in, int64_t *out, int64_t n);
// stable LSD radix sort of (key, value) pairs by the low `bits` bits of key (device, in place
// through ping-pong buffers allocated inside)
int radix_sort_pairs(pasur_ctx *ctx, uint64_t *keys, int64_t *vals, int64_t n, int bits);
int read_i64(pasur_ctx *ctx, const int64_t *dptr, int64_t *out);

// build.cu
int ensure_capture_table(pasur_ctx *ctx);
int build_levels(pasur_tree *t, const uint64_t *root_pools_dev);
int unfold_levels(pasur_tree *t);
int compute_leaf_values(pasur_tree *t, const float *next_util_dev);
int launch_leaf_values(pasur_tree *t, const float *next_util_dev, unsigned *umax_bits);
// the solved slots of an unfolded tree: merged per (a_clubs, b_clubs, bonus) when `merge`, else one
// per full slot; a non-final round given next_util_dev merges only if every merged slot's leaves
// equal its representative's (checked on the device); idempotent
int plan_solve_slots(pasur_tree *t, bool merge, const float *next_util_dev);
// full FGT leaf values from the solved ones (out: device, Q[8] floats)
int expand_leaf_values(const pasur_tree *t, float *out_dev);

// cfr.cu
int cfr_prepare(pasur_tree *t, const pasur_config *cfg);
int cfr_run(pasur_tree *t, const pasur_config *cfg);
// layout, per-root plan and state of one tree; its items (tagged with tree index `tree`) are
// appended per class to cls_items, the shared-memory need per class raised in need[]
// (cls_items / need: 8 classes; roots split over thread-block clusters append ClusterItems to clu)
int cfr_setup_tree(pasur_tree *t, const pasur_config *cfg, int tree, std::vector<CfrItem> *cls_items, size_t *need,
                   std::vector<ClusterItem> *clu);
// sort and upload merged items and the tree views; launch configuration per class
int cfr_finalize_plan(pasur_ctx *ctx, CfrPlan &plan, std::vector<CfrItem> *cls_items, const size_t *need,
                      const std::vector<TreeView> &views, const pasur_config *cfg, std::vector<std::pair<void *, size_t>> &owned,
                      const std::vector<ClusterItem> &clu);
// launch the plan's classes for cfg->iters iterations starting at iteration t0 (+1); no host
// synchronisation (capturable); per-class times are read by cfr_plan_times
int cfr_launch_plan(pasur_ctx *ctx, CfrPlan &plan, const pasur_config *cfg, int64_t t0, const float *dcfr);
void cfr_plan_times(pasur_ctx *ctx, CfrPlan &plan);
int cfr_dcfr_factors(pasur_ctx *ctx, const pasur_config *cfg, int64_t t0, float **out, size_t *bytes);
// blocks of a persistent CFR launch with this block size and shared memory (0 if it cannot run)
int cfr_occupancy(pasur_ctx *ctx, int threads, int cls, size_t smem, int64_t n_items, int *blocks);
int cfr_export_sigma(const pasur_tree *t, float *out_dev);
// average strategies of the solved slots only (levels 1..8, solved FGT order, sum of cQ[1..8])
int export_sigma_solved(const pasur_tree *t, float *out_dev);
// sum over every FGT edge of (a - b)^2 for two solved-order strategy vectors (each solved edge
// counted once per full slot it stands for), added to *acc_dev (device double)
int sigma_sqdiff(const pasur_tree *t, const float *a_dev, const float *b_dev, double *acc_dev);
int cfr_export_utilities(const pasur_tree *t, float *out_dev);
int cfr_export_utilities_n(const pasur_tree *t, int64_t iters, float *out_dev);
int ensure_aux(pasur_ctx *ctx);

// selfplay.cu: device view of one round tree for the self-play kernel
struct SpRound {
    const int64_t *child_off[8];   // GT CSR child offsets, levels 0..7
    const int64_t *fgt_off[9];     // first FGT node of every GT node, levels 0..8
    const float *sigma;            // strategy per FGT edge, levels 1..8 concatenated
    int64_t sig_base[9];           // offset of level k in sigma (k >= 1)
    const int64_t *lnk;            // FGT leaf -> next-round FGT root (non-final rounds)
    int64_t n_roots;               // GT roots
    const pasur::GTState *st8;     // final round: leaf states
    const int32_t *root8;          //   root id of every leaf
    const int64_t *score_off;      //   score slots of every root
    const pasur_score *scores;
};
void selfplay_view(const pasur_tree *t, const float *sigma_dev, SpRound *v);
// games of n_deals deals (views[d * n_rounds + i]); seeds_dev / roots_dev per deal; out_dev
// int16 [n_deals * n_games], deal-major; records the kernel's device time in ctx
int selfplay_launch(pasur_ctx *ctx, const SpRound *views_dev, int n_rounds, int64_t n_deals, int64_t n_games,
                    const uint64_t *seeds_dev, const int64_t *roots_dev, int16_t *out_dev);

// between.cu
int next_roots(pasur_tree *t, std::vector<uint64_t> &pools, std::vector<int64_t> &score_off,
               std::vector<pasur_score> &scores);

}  // namespace pasur

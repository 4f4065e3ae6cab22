// Batched exact solve of many seeded deals: every deal's rounds are built and unfolded up front,
// the work items of all deals' trees of one round are merged into one plan (one persistent
// launch per shared-memory class, largest subtrees first across all deals), an autotuner picks
// the block size of every class on the largest round, and the whole backward sweep (leaf values,
// CFR, root utilities, round 5 down to the first round) is captured once into a CUDA graph and
// replayed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>

#include "pasur_internal.cuh"

struct pasur_batch {
    pasur_ctx *ctx = nullptr;
    int first_round = 0, last_round = 5, n_rounds = 0;
    std::vector<float *> cut_util;        // per deal: surrogate values of the roots after last_round
    // per deal: the roots of first_round (pools, score offsets, scores); empty = the standalone
    // convention root (pool deck[0:4], score 0)
    std::vector<std::vector<uint64_t>> root_pools;
    std::vector<std::vector<int64_t>> root_soff;
    std::vector<std::vector<pasur_score>> root_scores;
    int64_t n_deals = 0;
    std::vector<pasur_tree *> trees;      // [deal * n_rounds + (round - first_round)]
    std::vector<CfrPlan> plans;           // per round (index round - first_round)
    std::vector<float *> util;            // per tree: average root utilities (device)
    std::vector<std::pair<void *, size_t>> owned;
    pasur_config cfg{};
    float *dcfr = nullptr;
    size_t dcfr_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_launches = 0, edges = 0, solved_edges = 0, swept_edges = 0, swept_pairs = 0;
    float last_ms = 0.f;
    bool solved = false;
};

namespace pasur {
namespace {

pasur_tree *tree_of(pasur_batch *b, int64_t d, int ri) { return b->trees[(size_t)(d * b->n_rounds + ri)]; }

void free_batch(pasur_batch *b) {
    pasur_ctx *ctx = b->ctx;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &o : b->owned) dev_free(ctx, o.first, o.second);
    b->owned.clear();
    for (pasur_tree *t : b->trees)
        if (t) pasur_tree_free(t);
    b->trees.clear();
    cudaStreamSynchronize(ctx->stream);
}

int batch_alloc(pasur_batch *b, void **p, size_t bytes) {
    PASUR_TRY(dev_alloc(b->ctx, p, bytes));
    b->owned.push_back({*p, bytes});
    return PASUR_OK;
}

// What one deal leaves for the merged plans: per round its work items by launch class, the
// shared memory each class needs and its cluster items.
struct DealPlan {
    std::vector<CfrItem> own[6][8];
    size_t need[6][8] = {};
    std::vector<ClusterItem> clu[6];
    int64_t edges = 0, solved_edges = 0, swept_edges = 0, swept_pairs = 0;
};

// One deal on the context wc: its rounds forward from the standalone convention root (pool
// deck[0:4], score 0), each tree unfolded and linked to the next, then every tree's CFR layout.
int build_deal(pasur_batch *b, pasur_ctx *wc, const uint8_t *deck, int64_t d, DealPlan &o) {
    uint64_t pool0 = 0;
    for (int i = 0; i < 4; i++) pool0 |= 1ULL << deck[i];
    std::vector<uint64_t> pools(1, pool0);
    std::vector<int64_t> soff = {0, 1};
    std::vector<pasur_score> scores(1, pasur_score{0, 0, 0, 0});
    if (!b->root_pools.empty()) {
        pools = b->root_pools[(size_t)d];
        soff = b->root_soff[(size_t)d];
        scores = b->root_scores[(size_t)d];
    }
    for (int ri = 0; ri < b->n_rounds; ri++) {
        pasur_tree *t = nullptr;
        PASUR_TRY(pasur_build_round(wc, deck, b->first_round + ri, pools.data(), (int64_t)pools.size(), &t));
        b->trees[(size_t)(d * b->n_rounds + ri)] = t;
        PASUR_TRY(pasur_unfold(t, soff.data(), scores.data(), nullptr));
        PASUR_TRY(tree_alloc(t, (void **)&b->util[(size_t)(d * b->n_rounds + ri)], sizeof(float) * (size_t)(t->Q[0] + 1)));
        if (b->first_round + ri < 5) {
            int64_t np = 0, nr = 0;
            PASUR_TRY(pasur_next_roots(t, nullptr, 0, nullptr, nullptr, 0, nullptr, &np, &nr));
            pools.assign((size_t)np, 0);
            soff.assign((size_t)np + 1, 0);
            scores.assign((size_t)nr, pasur_score{});
            PASUR_TRY(pasur_next_roots(t, pools.data(), np, soff.data(), scores.data(), nr, nullptr, &np, &nr));
        }
    }
    for (int ri = 0; ri < b->n_rounds; ri++) {
        pasur_tree *t = tree_of(b, d, ri);
        // slots that differ only in delta share one solve, except in a round whose leaves take the
        // surrogate's values (its input includes delta); the batch's own utilities of the next
        // round are exact and do not depend on delta
        const bool cut = ri == b->n_rounds - 1 && b->last_round < 5;
        PASUR_TRY(plan_solve_slots(t, b->cfg.merge_delta != 0 && !cut, nullptr));
        PASUR_TRY(tree_alloc(t, (void **)&t->leaf_v, sizeof(float) * (size_t)(t->cQ[8] + 1)));
        if (t->M[8] > 0) PASUR_CUDA(wc, cudaMemsetAsync(t->leaf_v, 0, sizeof(float) * (size_t)(t->cQ[8] + 1), wc->stream));
        PASUR_TRY(cfr_setup_tree(t, &b->cfg, (int)d, o.own[ri], o.need[ri], &o.clu[ri]));
        t->cfr_ready = true;
        t->variant = b->cfg.variant;
        // the tree keeps its own items for exporting its average strategy
        t->plan.items_h.clear();
        for (int c = 0; c < 8; c++) t->plan.items_h.insert(t->plan.items_h.end(), o.own[ri][c].begin(), o.own[ri][c].end());
        t->plan.n_items = (int64_t)t->plan.items_h.size();
        if (t->plan.n_items) {
            PASUR_TRY(tree_alloc(t, (void **)&t->plan.items_d, sizeof(CfrItem) * (size_t)t->plan.n_items));
            PASUR_CUDA(wc, cudaMemcpyAsync(t->plan.items_d, t->plan.items_h.data(), sizeof(CfrItem) * (size_t)t->plan.n_items,
                                           cudaMemcpyHostToDevice, wc->stream));
        }
        for (int k = 1; k < 9; k++) {
            o.edges += t->Q[k];
            o.solved_edges += t->cQ[k];
        }
        o.swept_edges += t->swept_edges;
        o.swept_pairs += t->swept_pairs;
    }
    PASUR_CUDA(wc, cudaStreamSynchronize(wc->stream));
    return PASUR_OK;
}

// A build worker's context: its own stream, work counter and error word on the parent's device,
// the parent's capture table, allocations charged to the parent.
int open_worker(pasur_ctx *parent, pasur_ctx *w) {
    w->device = parent->device;
    w->num_sms = parent->num_sms;
    w->smem_optin = parent->smem_optin;
    w->tab = parent->tab;
    w->tab_off = parent->tab_off;
    w->acct = parent;
    PASUR_CUDA(w, cudaSetDevice(w->device));
    PASUR_CUDA(w, cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
    w->own_stream = true;
    PASUR_TRY(dev_alloc(w, (void **)&w->counter, 64));
    PASUR_TRY(dev_alloc(w, (void **)&w->errflag, 64));
    PASUR_CUDA(w, cudaMemsetAsync(w->errflag, 0, 64, w->stream));
    return PASUR_OK;
}

void close_worker(pasur_ctx *w) {
    dev_free(w, w->counter, 64);
    dev_free(w, w->errflag, 64);
    if (w->stream) cudaStreamSynchronize(w->stream);
    if (w->own_stream) cudaStreamDestroy(w->stream);
}

// Build every deal, spread over up to 8 host threads, each on a context with its own stream so
// that the many small launches and synchronisations of different deals overlap.  Deals are taken
// in order from a shared counter; what each produces depends only on the deal, and the trees are
// handed to the batch's context afterwards.  PASUR_BUILD_WORKERS sets the number of threads.
int build_deals(pasur_batch *b, const uint8_t *decks, std::vector<DealPlan> &dp, int *n_used) {
    pasur_ctx *ctx = b->ctx;
    int nw = (int)std::min<int64_t>(b->n_deals, 8);
    const unsigned hw = std::thread::hardware_concurrency();
    if (hw > 0) nw = std::min<int>(nw, (int)hw);
    if (const char *e = getenv("PASUR_BUILD_WORKERS")) nw = std::max(1, std::min(nw, atoi(e)));
    *n_used = nw;
    if (nw <= 1) {
        for (int64_t d = 0; d < b->n_deals; d++) PASUR_TRY(build_deal(b, ctx, decks + 52 * d, d, dp[(size_t)d]));
        return PASUR_OK;
    }
    std::vector<std::unique_ptr<pasur_ctx>> ws;
    int rc = PASUR_OK;
    for (int i = 0; i < nw && rc == PASUR_OK; i++) {
        ws.emplace_back(new pasur_ctx());
        rc = open_worker(ctx, ws.back().get());
        if (rc != PASUR_OK) ctx->err = "pasur_batch_create: build worker: " + ws.back()->err;
    }
    std::atomic<int64_t> next{0};
    std::atomic<bool> failed{false};
    std::mutex mu;
    int64_t err_deal = -1;
    int err_rc = PASUR_OK;
    std::string err_msg;
    auto run = [&](pasur_ctx *w) {
        cudaSetDevice(w->device);
        for (;;) {
            const int64_t d = next.fetch_add(1);
            if (d >= b->n_deals || failed.load()) return;
            int r;
            try {
                r = build_deal(b, w, decks + 52 * d, d, dp[(size_t)d]);
            } catch (...) {  // host allocation inside the build: no exception leaves the library
                r = set_err(w, PASUR_ENOMEM, "host allocation failed");
            }
            if (r != PASUR_OK) {
                std::lock_guard<std::mutex> lk(mu);
                if (err_deal < 0 || d < err_deal) err_deal = d, err_rc = r, err_msg = w->err;
                failed.store(true);
                return;
            }
        }
    };
    if (rc == PASUR_OK) {
        std::vector<std::thread> th;
        for (auto &w : ws) {
            try {
                th.emplace_back(run, w.get());
            } catch (...) {
                break;  // fewer threads: the shared counter hands every deal to those running
            }
        }
        if (th.empty()) run(ws[0].get());
        for (auto &x : th) x.join();
    }
    // the trees (built or partly built) belong to the batch's context from here on
    for (pasur_tree *t : b->trees)
        if (t) t->ctx = ctx;
    for (auto &w : ws) {
        ctx->live_trees += w->live_trees;
        ctx->launches += w->launches;
        close_worker(w.get());
    }
    if (rc == PASUR_OK && err_deal >= 0) {
        ctx->err = "deal " + std::to_string(err_deal) + ": " + err_msg;
        rc = err_rc;
    }
    return rc;
}

// Time one class of a plan alone (no other class, no cluster item) for a few iterations at each
// candidate block size; keep the best.  Class 5 (the level-streaming sweep) and the cluster
// items have no block size to choose.
int autotune(pasur_batch *b, CfrPlan &plan) {
    pasur_ctx *ctx = b->ctx;
    pasur_config cfg = b->cfg;
    cfg.iters = 8;
    cudaEvent_t e0, e1;
    PASUR_CUDA(ctx, cudaEventCreate(&e0));
    PASUR_CUDA(ctx, cudaEventCreate(&e1));
    for (int c = 0; c < 5; c++) {
        if (plan.cls_end[c] == plan.cls_begin[c]) continue;
        const int def = plan.cls_threads[c];
        const int cand_small[3] = {64, 128, 256}, cand_wide[3] = {256, 512, 1024};
        const int *cand = def > 256 ? cand_wide : cand_small;
        CfrPlan one = plan;
        for (int o = 0; o < 8; o++)
            if (o != c) one.cls_begin[o] = one.cls_end[o] = 0;
        for (int o = 0; o < kCluGroups; o++) one.clu_begin[o] = one.clu_end[o] = 0;
        float best_ms = 1e30f;
        int best = def;
        for (int i = 0; i < 3; i++) {
            int blocks = 0;
            PASUR_TRY(cfr_occupancy(ctx, cand[i], c, one.cls_smem[c], one.cls_end[c] - one.cls_begin[c], &blocks));
            if (blocks <= 0) continue;
            one.cls_threads[c] = cand[i];
            one.cls_blocks[c] = blocks;
            PASUR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
            PASUR_TRY(cfr_launch_plan(ctx, one, &cfg, 0, nullptr));
            PASUR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
            PASUR_CUDA(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            PASUR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (getenv("PASUR_VERBOSE"))
                fprintf(stderr, "[pasur] autotune class %d alone: %d blocks x %d threads, %d iterations in %.3f ms\n", c, blocks,
                        cand[i], cfg.iters, ms);
            if (ms < best_ms) {
                best_ms = ms;
                best = cand[i];
            }
        }
        // apply to every round's plan
        for (CfrPlan &pl : b->plans) {
            if (pl.cls_end[c] == pl.cls_begin[c]) continue;
            int blocks = 0;
            PASUR_TRY(cfr_occupancy(ctx, best, c, pl.cls_smem[c], pl.cls_end[c] - pl.cls_begin[c], &blocks));
            if (blocks > 0) {
                pl.cls_threads[c] = best;
                pl.cls_blocks[c] = blocks;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return PASUR_OK;
}

// one backward sweep on ctx->stream without host synchronisation (captured into the graph)
int record_sweep(pasur_batch *b) {
    pasur_ctx *ctx = b->ctx;
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int32_t), ctx->stream));
    for (int ri = b->n_rounds - 1; ri >= 0; ri--) {
        for (int64_t d = 0; d < b->n_deals; d++) {
            pasur_tree *t = tree_of(b, d, ri);
            PASUR_CUDA(ctx, cudaMemsetAsync(t->R, 0, sizeof(float) * (size_t)(t->data_size + 1), ctx->stream));
            PASUR_CUDA(ctx, cudaMemsetAsync(t->S, 0, sizeof(float) * (size_t)(t->data_size + 1), ctx->stream));
            PASUR_CUDA(ctx, cudaMemsetAsync(t->uacc, 0, sizeof(double) * (size_t)(t->cQ[0] + 1), ctx->stream));
            const float *next = ri + 1 < b->n_rounds ? b->util[(size_t)(d * b->n_rounds + ri + 1)]
                                                     : (b->cut_util.empty() ? nullptr : b->cut_util[(size_t)d]);
            PASUR_TRY(launch_leaf_values(t, next, nullptr));
        }
        PASUR_TRY(cfr_launch_plan(ctx, b->plans[(size_t)ri], &b->cfg, 0, b->dcfr));
        for (int64_t d = 0; d < b->n_deals; d++)
            PASUR_TRY(cfr_export_utilities_n(tree_of(b, d, ri), b->cfg.iters, b->util[(size_t)(d * b->n_rounds + ri)]));
    }
    return PASUR_OK;
}

// Diagnostics (PASUR_VERBOSE): every round's merged plan per class, and the device time of each
// round's CFR launches run once outside the graph on zeroed state (the batch is re-zeroed by
// every pasur_batch_solve).
int print_batch(pasur_batch *b) {
    pasur_ctx *ctx = b->ctx;
    for (int ri = b->n_rounds - 1; ri >= 0; ri--) {
        CfrPlan &pl = b->plans[(size_t)ri];
        for (int64_t d = 0; d < b->n_deals; d++) {
            pasur_tree *t = tree_of(b, d, ri);
            const float *next = ri + 1 < b->n_rounds ? b->util[(size_t)(d * b->n_rounds + ri + 1)]
                                                     : (b->cut_util.empty() ? nullptr : b->cut_util[(size_t)d]);
            PASUR_TRY(launch_leaf_values(t, next, nullptr));
        }
        cudaEvent_t e0, e1;
        PASUR_CUDA(ctx, cudaEventCreate(&e0));
        PASUR_CUDA(ctx, cudaEventCreate(&e1));
        PASUR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        PASUR_TRY(cfr_launch_plan(ctx, pl, &b->cfg, 0, b->dcfr));
        PASUR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
        PASUR_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        PASUR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        cfr_plan_times(ctx, pl);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (int64_t d = 0; d < b->n_deals; d++)
            PASUR_TRY(cfr_export_utilities_n(tree_of(b, d, ri), b->cfg.iters, b->util[(size_t)(d * b->n_rounds + ri)]));
        fprintf(stderr, "[pasur] batch round %d: %lld items, %d iterations in %.3f ms\n", b->first_round + ri,
                (long long)pl.n_items, b->cfg.iters, ms);
        for (int bk = 0; bk < kCluGroups; bk++)
            if (pl.clu_end[bk] != pl.clu_begin[bk])
                fprintf(stderr, "[pasur]   cluster items: %lld, %d CTAs x %d threads, smem %zu B, %.3f ms\n",
                        (long long)(pl.clu_end[bk] - pl.clu_begin[bk]), pl.clu_ctas[bk], pl.clu_threads, pl.clu_smem[bk],
                        pl.cls_ms[6 + bk]);
        for (int c = 0; c < 8; c++) {
            const int64_t n = pl.cls_end[c] - pl.cls_begin[c];
            if (!n) continue;
            int64_t cost = 0, slots = 0, maxcost = 0;
            for (int64_t i = pl.cls_begin[c]; i < pl.cls_end[c]; i++) {
                cost += pl.items_h[(size_t)i].cost;
                slots += pl.items_h[(size_t)i].ns;
                maxcost = std::max(maxcost, pl.items_h[(size_t)i].cost);
            }
            fprintf(stderr, "[pasur]   class %d: items %lld (slots %lld), smem %zu B, blocks %d x %d threads, "
                            "active-node-slots %lld (largest item %lld), %.3f ms\n",
                    c, (long long)n, (long long)slots, pl.cls_smem[c], pl.cls_blocks[c], pl.cls_threads[c], (long long)cost,
                    (long long)maxcost, pl.cls_ms[c]);
        }
    }
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

}  // namespace
}  // namespace pasur

using namespace pasur;

extern "C" {

int pasur_batch_create(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, const pasur_config *cfg,
                       pasur_batch **out) {
    return pasur_batch_create_cut(ctx, decks, n_deals, first_round, 5, cfg, nullptr, out);
}

static int batch_create(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, int last_round,
                        const pasur_config *cfg, pasur_mlp *mlp, const int64_t *deal_roots, const uint64_t *pools,
                        const int64_t *score_offs, const pasur_score *scores, pasur_batch **out);

int pasur_batch_create_cut(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, int last_round,
                           const pasur_config *cfg, pasur_mlp *mlp, pasur_batch **out) {
    return batch_create(ctx, decks, n_deals, first_round, last_round, cfg, mlp, nullptr, nullptr, nullptr, nullptr, out);
}

int pasur_batch_create_roots(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, const int64_t *deal_roots,
                             const uint64_t *pools, const int64_t *score_offs, const pasur_score *scores,
                             const pasur_config *cfg, pasur_batch **out) {
    if (!deal_roots || !pools || !score_offs || !scores)
        return ctx ? set_err(ctx, PASUR_EINVAL, "pasur_batch_create_roots: NULL argument") : PASUR_EINVAL;
    return batch_create(ctx, decks, n_deals, first_round, 5, cfg, nullptr, deal_roots, pools, score_offs, scores, out);
}

int pasur_batch_set_cut_values(pasur_batch *b, int64_t deal, const float *values, int64_t n) {
    if (!b) return PASUR_EINVAL;
    pasur_ctx *ctx = b->ctx;
    if (b->cut_util.empty()) return set_err(ctx, PASUR_EINVAL, "pasur_batch_set_cut_values: the batch has no cut");
    if (deal < 0 || deal >= b->n_deals || !values) return set_err(ctx, PASUR_EINVAL, "pasur_batch_set_cut_values: bad deal or NULL");
    const pasur_tree *t = b->trees[(size_t)(deal * b->n_rounds + b->n_rounds - 1)];
    if (n != t->n_next_roots)
        return set_err(ctx, PASUR_EINVAL, "pasur_batch_set_cut_values: n must be the number of roots after the cut (" +
                                              std::to_string(t->n_next_roots) + ")");
    cudaSetDevice(ctx->device);
    PASUR_CUDA(ctx, cudaMemcpyAsync(b->cut_util[(size_t)deal], values, sizeof(float) * (size_t)n,
                                    is_device_ptr(values) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

static int batch_create(pasur_ctx *ctx, const uint8_t *decks, int64_t n_deals, int first_round, int last_round,
                        const pasur_config *cfg, pasur_mlp *mlp, const int64_t *deal_roots, const uint64_t *pools,
                        const int64_t *score_offs, const pasur_score *scores, pasur_batch **out) {
    if (!ctx || !out || !cfg || (n_deals > 0 && !decks)) return ctx ? set_err(ctx, PASUR_EINVAL, "pasur_batch_create: NULL argument") : PASUR_EINVAL;
    *out = nullptr;
    if (n_deals < 1 || n_deals > (1 << 20)) return set_err(ctx, PASUR_EINVAL, "pasur_batch_create: n_deals must be 1..2^20");
    if (first_round < 0 || first_round > 5) return set_err(ctx, PASUR_EINVAL, "pasur_batch_create: first_round must be 0..5");
    if (last_round < first_round || last_round > 5)
        return set_err(ctx, PASUR_EINVAL, "pasur_batch_create_cut: last_round must be first_round..5");
    if (last_round < 5 && !mlp) return set_err(ctx, PASUR_EINVAL, "pasur_batch_create_cut: a cut before round 5 needs the surrogate");
    if (cfg->iters < 1 || (cfg->variant != 0 && cfg->variant != 1))
        return set_err(ctx, PASUR_EINVAL, "pasur_batch_create: cfg.iters >= 1 and variant 0 or 1 required");
    cudaSetDevice(ctx->device);
    pasur_batch *b = new pasur_batch();
    b->ctx = ctx;
    b->first_round = first_round;
    b->last_round = last_round;
    b->n_rounds = last_round - first_round + 1;
    b->n_deals = n_deals;
    b->cfg = *cfg;
    b->trees.assign((size_t)(n_deals * b->n_rounds), nullptr);
    b->util.assign(b->trees.size(), nullptr);
    if (deal_roots) {
        // deal d's roots: pools[deal_roots[d] .. deal_roots[d+1]), their score slots from the
        // global score offsets (score_offs[i] .. score_offs[i+1] for pool i)
        b->root_pools.resize((size_t)n_deals);
        b->root_soff.resize((size_t)n_deals);
        b->root_scores.resize((size_t)n_deals);
        for (int64_t d = 0; d < n_deals; d++) {
            const int64_t a = deal_roots[d], e = deal_roots[d + 1];
            if (e < a) {
                delete b;
                return set_err(ctx, PASUR_EINVAL, "pasur_batch_create_roots: deal_roots must not decrease");
            }
            b->root_pools[(size_t)d].assign(pools + a, pools + e);
            b->root_soff[(size_t)d].assign(1, 0);
            for (int64_t i = a; i < e; i++) {
                if (score_offs[i + 1] < score_offs[i]) {
                    delete b;
                    return set_err(ctx, PASUR_EINVAL, "pasur_batch_create_roots: score_offs must not decrease");
                }
                for (int64_t x = score_offs[i]; x < score_offs[i + 1]; x++) b->root_scores[(size_t)d].push_back(scores[x]);
                b->root_soff[(size_t)d].push_back((int64_t)b->root_scores[(size_t)d].size());
            }
        }
    }
    int rc = PASUR_OK;
    const bool verbose = getenv("PASUR_VERBOSE") != nullptr;
    using clk = std::chrono::steady_clock;
    double ph_ms[4] = {0};  // rounds and layouts, surrogate, merged plans, autotune
    int n_workers = 1;
    auto lap = [&](clk::time_point &t0, int i) {
        if (!verbose) return;
        cudaStreamSynchronize(ctx->stream);
        const clk::time_point t1 = clk::now();
        ph_ms[i] += std::chrono::duration<double, std::milli>(t1 - t0).count();
        t0 = t1;
    };
    clk::time_point tp = clk::now();
    // every deal's rounds and CFR layouts, deals spread over the build workers
    std::vector<DealPlan> dp((size_t)n_deals);
    rc = ensure_capture_table(ctx);
    if (rc == PASUR_OK) rc = cudaStreamSynchronize(ctx->stream) == cudaSuccess ? PASUR_OK : set_err(ctx, PASUR_ECUDA, "pasur_batch_create: sync");
    if (rc == PASUR_OK) rc = build_deals(b, decks, dp, &n_workers);
    lap(tp, 0);
    // surrogate values of every deal's roots after the last round
    if (rc == PASUR_OK && last_round < 5) {
        b->cut_util.assign((size_t)n_deals, nullptr);
        for (int64_t d = 0; d < n_deals && rc == PASUR_OK; d++) {
            pasur_tree *t = tree_of(b, d, b->n_rounds - 1);
            rc = batch_alloc(b, (void **)&b->cut_util[(size_t)d], sizeof(float) * (size_t)(t->n_next_roots + 1));
            if (rc == PASUR_OK && t->n_next_roots > 0)
                rc = pasur_mlp_predict_next(mlp, t, b->cut_util[(size_t)d], t->n_next_roots);
        }
    }
    lap(tp, 1);
    // one merged plan per round, the deals' items in deal order
    b->plans.resize((size_t)b->n_rounds);
    for (int ri = 0; ri < b->n_rounds && rc == PASUR_OK; ri++) {
        std::vector<CfrItem> cls_items[8];
        size_t need[8] = {0};
        std::vector<TreeView> views;
        std::vector<ClusterItem> clu;
        for (int64_t d = 0; d < n_deals; d++) {
            DealPlan &o = dp[(size_t)d];
            for (int c = 0; c < 8; c++) {
                cls_items[c].insert(cls_items[c].end(), o.own[ri][c].begin(), o.own[ri][c].end());
                need[c] = std::max(need[c], o.need[ri][c]);
            }
            clu.insert(clu.end(), o.clu[ri].begin(), o.clu[ri].end());
            views.push_back(tree_of(b, d, ri)->view);
        }
        rc = cfr_finalize_plan(ctx, b->plans[(size_t)ri], cls_items, need, views, cfg, b->owned, clu);
    }
    for (const DealPlan &o : dp) {
        b->edges += o.edges;
        b->solved_edges += o.solved_edges;
        b->swept_edges += o.swept_edges;
        b->swept_pairs += o.swept_pairs;
    }
    lap(tp, 2);
    if (rc == PASUR_OK) rc = cfr_dcfr_factors(ctx, cfg, 0, &b->dcfr, &b->dcfr_bytes);
    if (rc == PASUR_OK && b->dcfr) b->owned.push_back({b->dcfr, b->dcfr_bytes});
    if (rc == PASUR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "pasur_batch_create: sync");
    lap(tp, 2);
    // autotune the block size of every class on the round with the most work
    if (rc == PASUR_OK && cfg->threads == 0) {
        int big = 0;
        int64_t best = -1;
        for (int ri = 0; ri < b->n_rounds; ri++) {
            int64_t cost = 0;
            for (const CfrItem &it : b->plans[(size_t)ri].items_h) cost += it.cost;
            if (cost > best) best = cost, big = ri;
        }
        rc = autotune(b, b->plans[(size_t)big]);
    }
    if (rc == PASUR_OK) rc = ensure_aux(ctx);
    lap(tp, 3);
    if (rc == PASUR_OK && verbose) {
        fprintf(stderr, "[pasur] batch create: rounds and layouts %.1f ms (%d build workers), surrogate %.1f, "
                        "merged plans %.1f, autotune %.1f\n", ph_ms[0], n_workers, ph_ms[1], ph_ms[2], ph_ms[3]);
        rc = print_batch(b);
    }
    if (rc != PASUR_OK) {
        free_batch(b);
        delete b;
        return rc;
    }
    *out = b;
    return PASUR_OK;
}

int pasur_batch_solve(pasur_batch *b, float *root_util_out, int64_t cap) {
    if (!b) return PASUR_EINVAL;
    pasur_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    if (root_util_out && cap < b->n_deals) return set_err(ctx, PASUR_EOVERFLOW, "pasur_batch_solve: cap < n_deals");
    if (!b->exec) {
        const int64_t before = ctx->launches;
        PASUR_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        int rc = record_sweep(b);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        if (rc != PASUR_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_err(ctx, e, "pasur_batch_solve: stream capture");
        b->graph = g;
        PASUR_CUDA(ctx, cudaGraphInstantiate(&b->exec, g, 0));
        b->graph_launches = ctx->launches - before;
    }
    cudaEvent_t e0, e1;
    PASUR_CUDA(ctx, cudaEventCreate(&e0));
    PASUR_CUDA(ctx, cudaEventCreate(&e1));
    PASUR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    PASUR_CUDA(ctx, cudaGraphLaunch(b->exec, ctx->stream));
    ctx->launches += b->graph_launches;
    PASUR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    int32_t ef = 0;
    PASUR_CUDA(ctx, cudaMemcpyAsync(&ef, ctx->errflag, sizeof ef, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    PASUR_CUDA(ctx, cudaEventElapsedTime(&b->last_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (pasur_tree *t : b->trees) t->iters_done = b->cfg.iters;
    b->solved = true;
    if (ef) return set_err(ctx, PASUR_ENUMERIC, "non-finite root value in the batched CFR sweep");
    if (root_util_out) {
        bool dev = is_device_ptr(root_util_out);
        for (int64_t d = 0; d < b->n_deals; d++)
            PASUR_CUDA(ctx, cudaMemcpyAsync(root_util_out + d, b->util[(size_t)(d * b->n_rounds)], sizeof(float),
                                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return PASUR_OK;
}

int pasur_batch_tree(const pasur_batch *b, int64_t deal, int round, pasur_tree **tree_out) {
    if (!b || !tree_out) return PASUR_EINVAL;
    if (deal < 0 || deal >= b->n_deals || round < b->first_round || round > b->last_round)
        return set_err(b->ctx, PASUR_EINVAL, "pasur_batch_tree: deal or round out of range");
    *tree_out = b->trees[(size_t)(deal * b->n_rounds + (round - b->first_round))];
    return PASUR_OK;
}

int pasur_batch_stats(const pasur_batch *b, float *ms, int64_t *edges, int64_t *launches) {
    if (!b) return PASUR_EINVAL;
    if (ms) *ms = b->last_ms;
    if (edges) *edges = b->edges;
    if (launches) *launches = b->graph_launches;
    return PASUR_OK;
}

int pasur_batch_work(const pasur_batch *b, int64_t *solved_edges, int64_t *swept_edges) {
    if (!b) return PASUR_EINVAL;
    if (solved_edges) *solved_edges = b->solved_edges;
    if (swept_edges) *swept_edges = b->swept_edges;
    return PASUR_OK;
}

int pasur_batch_pairs(const pasur_batch *b, int64_t *swept_pairs) {
    if (!b || !swept_pairs) return PASUR_EINVAL;
    *swept_pairs = b->swept_pairs;
    return PASUR_OK;
}

int pasur_batch_free(pasur_batch *b) {
    if (!b) return PASUR_EINVAL;
    cudaSetDevice(b->ctx->device);
    free_batch(b);
    delete b;
    return PASUR_OK;
}

}  // extern "C"

extern "C" int pasur_batch_selfplay(pasur_batch *b, int64_t n_games, const uint64_t *seeds, int16_t *out) {
    if (!b) return PASUR_EINVAL;
    pasur_ctx *ctx = b->ctx;
    if (!b->solved) return set_err(ctx, PASUR_EINVAL, "pasur_batch_selfplay: call pasur_batch_solve first");
    if (b->last_round != 5) return set_err(ctx, PASUR_EINVAL, "pasur_batch_selfplay: the batch must end with the final round");
    if (n_games < 0 || n_games > ((int64_t)1 << 40) / b->n_deals)
        return set_err(ctx, PASUR_EINVAL, "pasur_batch_selfplay: n_games out of range");
    if (n_games > 0 && (!seeds || !out)) return set_err(ctx, PASUR_EINVAL, "pasur_batch_selfplay: NULL seeds or out");
    cudaSetDevice(ctx->device);
    if (n_games == 0) {
        ctx->selfplay_ms = 0.f;
        ctx->selfplay_games = 0;
        return PASUR_OK;
    }
    std::vector<std::pair<void *, size_t>> tmp;
    auto alloc = [&](void **p, size_t bytes) {
        int rc = dev_alloc(ctx, p, bytes);
        if (rc == PASUR_OK) tmp.push_back({*p, bytes});
        return rc;
    };
    // every tree's average strategy, one buffer, tree after tree
    std::vector<int64_t> sig_off(b->trees.size() + 1, 0);
    for (size_t i = 0; i < b->trees.size(); i++) {
        const pasur_tree *t = b->trees[i];
        int64_t ne = 0;
        for (int k = 1; k < 9; k++) ne += t->Q[k];
        sig_off[i + 1] = sig_off[i] + ne;
    }
    float *sig = nullptr;
    SpRound *views_d = nullptr;
    uint64_t *seeds_d = nullptr;
    int64_t *roots_d = nullptr;
    int16_t *out_d = nullptr;
    const bool out_dev = is_device_ptr(out);
    const int64_t total = b->n_deals * n_games;
    int rc = alloc((void **)&sig, sizeof(float) * (size_t)(sig_off.back() + 1));
    std::vector<SpRound> views(b->trees.size());
    for (size_t i = 0; i < b->trees.size() && rc == PASUR_OK; i++) {
        rc = cfr_export_sigma(b->trees[i], sig + sig_off[i]);
        selfplay_view(b->trees[i], sig + sig_off[i], &views[i]);
    }
    if (rc == PASUR_OK) rc = alloc((void **)&views_d, sizeof(SpRound) * views.size());
    if (rc == PASUR_OK) rc = alloc((void **)&seeds_d, sizeof(uint64_t) * (size_t)b->n_deals);
    if (rc == PASUR_OK) rc = alloc((void **)&roots_d, sizeof(int64_t) * (size_t)b->n_deals);
    if (rc == PASUR_OK && !out_dev) rc = alloc((void **)&out_d, sizeof(int16_t) * (size_t)total);
    if (rc == PASUR_OK) {
        if (out_dev) out_d = out;
        if (cudaMemcpyAsync(views_d, views.data(), sizeof(SpRound) * views.size(), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(seeds_d, seeds, sizeof(uint64_t) * (size_t)b->n_deals, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
            cudaMemsetAsync(roots_d, 0, sizeof(int64_t) * (size_t)b->n_deals, ctx->stream) != cudaSuccess)
            rc = set_err(ctx, PASUR_ECUDA, "pasur_batch_selfplay: upload");
    }
    // the first round of every deal has a single FGT root (index 0)
    if (rc == PASUR_OK) rc = selfplay_launch(ctx, views_d, b->n_rounds, b->n_deals, n_games, seeds_d, roots_d, out_d);
    if (rc == PASUR_OK && !out_dev &&
        cudaMemcpyAsync(out, out_d, sizeof(int16_t) * (size_t)total, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        rc = set_err(ctx, PASUR_ECUDA, "pasur_batch_selfplay: copy results");
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == PASUR_OK) rc = set_err(ctx, PASUR_ECUDA, "pasur_batch_selfplay: sync");
    for (auto &x : tmp) dev_free(ctx, x.first, x.second);
    return rc;
}

// C ABI of the Pasur GB300 library: contexts, trees, argument checks, host/device marshalling.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "pasur_internal.cuh"

namespace pasur {

static thread_local std::string g_create_err;

int set_err(pasur_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return code;
}

int cuda_err(pasur_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    int code = (e == cudaErrorMemoryAllocation) ? PASUR_ENOMEM : PASUR_ECUDA;
    return set_err(ctx, code, m);
}

int dev_alloc(pasur_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    pasur_ctx *a = ctx->acct ? ctx->acct : ctx;
    {
        std::lock_guard<std::mutex> lk(a->acct_mu);
        if (a->budget && a->in_use + bytes > a->budget)
            return set_err(ctx, PASUR_ENOMEM, "device-memory budget exceeded (" + std::to_string(a->in_use + bytes) + " > " +
                                                  std::to_string(a->budget) + " bytes)");
        a->in_use += bytes;
        a->peak = std::max(a->peak, a->in_use);
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, a->pool, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        std::lock_guard<std::mutex> lk(a->acct_mu);
        a->in_use -= std::min(a->in_use, bytes);
        return set_err(ctx, PASUR_ENOMEM, std::string("cudaMallocFromPoolAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    return PASUR_OK;
}

void dev_free(pasur_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    cudaFreeAsync(p, ctx->stream);
    pasur_ctx *a = ctx->acct ? ctx->acct : ctx;
    std::lock_guard<std::mutex> lk(a->acct_mu);
    a->in_use -= std::min(a->in_use, bytes);
}

int tree_alloc(pasur_tree *t, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    PASUR_TRY(dev_alloc(t->ctx, p, bytes));
    t->allocs.push_back(*p);
    t->allocs.push_back((void *)(uintptr_t)bytes);
    return PASUR_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- the library's own seeded deal (SplitMix64 seeding, xoshiro256**, Lemire bounded draw) ----
struct Xoshiro {
    uint64_t s[4];
    static uint64_t mix(uint64_t &x) {
        x += 0x9E3779B97F4A7C15ULL;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    explicit Xoshiro(uint64_t seed) {
        uint64_t x = seed;
        for (auto &v : s) v = mix(x);
    }
    uint64_t next() {
        const uint64_t out = ((s[1] * 5ULL) << 7 | (s[1] * 5ULL) >> 57) * 9ULL;
        const uint64_t sh = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= sh;
        s[3] = (s[3] << 45) | (s[3] >> 19);
        return out;
    }
    uint64_t below(uint64_t n) {  // Lemire 2019
        unsigned __int128 prod = (unsigned __int128)next() * n;
        uint64_t low = (uint64_t)prod;
        if (low < n) {
            const uint64_t floor = (uint64_t)(-n) % n;
            while (low < floor) {
                prod = (unsigned __int128)next() * n;
                low = (uint64_t)prod;
            }
        }
        return (uint64_t)(prod >> 64);
    }
};

}  // namespace pasur

using namespace pasur;

namespace {

int check_tree(const pasur_tree *t) { return t && t->ctx ? PASUR_OK : PASUR_EINVAL; }

void set_device(pasur_ctx *ctx) { cudaSetDevice(ctx->device); }

template <typename T>
int copy_out(pasur_ctx *ctx, T *dst, const T *src_dev, int64_t n) {
    if (n <= 0) return PASUR_OK;
    cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    PASUR_CUDA(ctx, cudaMemcpyAsync(dst, src_dev, sizeof(T) * (size_t)n, kind, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

void free_tree_mem(pasur_tree *t) {
    for (size_t i = 0; i + 1 < t->allocs.size(); i += 2) dev_free(t->ctx, t->allocs[i], (size_t)(uintptr_t)t->allocs[i + 1]);
    t->allocs.clear();
}

}  // namespace

extern "C" {

int pasur_config_default(pasur_config *cfg) {
    if (!cfg) return PASUR_EINVAL;
    cfg->variant = 0;
    cfg->iters = 1000;
    cfg->rm_deadzone = 1e-6f;
    cfg->dcfr_alpha = 1.5f;
    cfg->dcfr_beta = 0.0f;
    cfg->dcfr_gamma = 2.0f;
    cfg->slots_per_item = 0;
    cfg->threads = 0;
    cfg->split_bytes = 0;
    cfg->stream_bytes = 0;
    cfg->merge_delta = 1;
    return PASUR_OK;
}

int pasur_create(pasur_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream) {
    if (!out) return set_err(nullptr, PASUR_EINVAL, "pasur_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev)
        return set_err(nullptr, PASUR_EINVAL, std::string("pasur_create: no CUDA device ") + std::to_string(device) +
                                                  (e != cudaSuccess ? std::string(" (") + cudaGetErrorString(e) + ")" : ""));
    pasur_ctx *ctx = new (std::nothrow) pasur_ctx();
    if (!ctx) return set_err(nullptr, PASUR_ENOMEM, "pasur_create: host allocation");
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ctx->smem_optin = (size_t)optin;
    if (e == cudaSuccess) {
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = true;
        }
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&ctx->pool, &props);
        uint64_t keep = UINT64_MAX;  // never trim at synchronisation: reuse instead of remapping
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        std::string m = std::string("pasur_create: ") + cudaGetErrorString(e);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return set_err(nullptr, PASUR_ECUDA, m);
    }
    int rc = dev_alloc(ctx, (void **)&ctx->counter, 64);
    if (rc == PASUR_OK) rc = dev_alloc(ctx, (void **)&ctx->errflag, 64);
    if (rc == PASUR_OK && cudaMemsetAsync(ctx->errflag, 0, 64, ctx->stream) != cudaSuccess) rc = PASUR_ECUDA;
    if (rc == PASUR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = PASUR_ECUDA;
    if (rc != PASUR_OK) {
        std::string m = ctx->err;
        cudaStreamSynchronize(ctx->stream);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return set_err(nullptr, rc, "pasur_create: " + m);
    }
    *out = ctx;
    return PASUR_OK;
}

int pasur_destroy(pasur_ctx *ctx) {
    if (!ctx) return PASUR_EINVAL;
    if (ctx->live_trees > 0)
        return set_err(ctx, PASUR_EINVAL, "pasur_destroy: " + std::to_string(ctx->live_trees) + " tree(s) still alive");
    set_device(ctx);
    dev_free(ctx, ctx->tab, 0);
    dev_free(ctx, ctx->tab_off, 0);
    dev_free(ctx, ctx->counter, 64);
    dev_free(ctx, ctx->errflag, 64);
    cudaStreamSynchronize(ctx->stream);
    for (int c = 0; c < 12; c++) {
        if (ctx->aux[c]) cudaStreamDestroy(ctx->aux[c]);
        if (ctx->join[c]) cudaEventDestroy(ctx->join[c]);
        if (ctx->cls_t0[c]) cudaEventDestroy(ctx->cls_t0[c]);
        if (ctx->cls_t1[c]) cudaEventDestroy(ctx->cls_t1[c]);
    }
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->copy_after) cudaEventDestroy(ctx->copy_after);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return PASUR_OK;
}

const char *pasur_last_error(const pasur_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int pasur_memory(const pasur_ctx *ctx, size_t *in_use, size_t *peak) {
    if (!ctx) return PASUR_EINVAL;
    if (in_use) *in_use = ctx->in_use;
    if (peak) *peak = ctx->peak;
    return PASUR_OK;
}

int pasur_launch_count(const pasur_ctx *ctx, int64_t *count) {
    if (!ctx || !count) return PASUR_EINVAL;
    *count = ctx->launches;
    return PASUR_OK;
}

int pasur_deal(uint64_t seed, uint8_t deck_out[52]) {
    if (!deck_out) return PASUR_EINVAL;
    Xoshiro g(seed);
    for (;;) {
        uint8_t d[52];
        for (int i = 0; i < 52; i++) d[i] = (uint8_t)i;
        for (int i = 51; i > 0; i--) std::swap(d[i], d[g.below((uint64_t)i + 1)]);
        int jacks = 0, at = -1;
        for (int i = 0; i < 4; i++)
            if (d[i] >= 40 && d[i] < 44) jacks++, at = i;
        bool ok = jacks == 0;
        if (jacks == 1 && !(d[4] >= 40 && d[4] < 44)) {
            std::swap(d[at], d[4]);
            ok = true;
        }
        if (ok) {
            memcpy(deck_out, d, 52);
            return PASUR_OK;
        }
    }
}

int pasur_build_round(pasur_ctx *ctx, const uint8_t deck[52], int round, const uint64_t *root_pools, int64_t n_pools,
                      pasur_tree **out) {
    if (!ctx || !out || !deck) return ctx ? set_err(ctx, PASUR_EINVAL, "pasur_build_round: NULL argument") : PASUR_EINVAL;
    *out = nullptr;
    set_device(ctx);
    if (round < 0 || round > 5) return set_err(ctx, PASUR_EINVAL, "pasur_build_round: round must be 0..5");
    if (n_pools < 0 || (n_pools > 0 && !root_pools)) return set_err(ctx, PASUR_EINVAL, "pasur_build_round: bad pools");
    if (n_pools >= INT32_MAX) return set_err(ctx, PASUR_EOVERFLOW, "pasur_build_round: too many roots");
    uint64_t seen = 0;
    for (int i = 0; i < 52; i++) {
        if (deck[i] >= 52 || (seen >> deck[i] & 1ULL)) return set_err(ctx, PASUR_EINVAL, "pasur_build_round: deck is not a permutation");
        seen |= 1ULL << deck[i];
    }
    uint64_t ha = 0, hb = 0;
    for (int i = 0; i < 4; i++) {
        ha |= 1ULL << deck[4 + 8 * round + i];
        hb |= 1ULL << deck[8 + 8 * round + i];
    }
    std::vector<uint64_t> hp;
    const uint64_t *pools_host = root_pools;
    bool dev = is_device_ptr(root_pools);
    if (dev && n_pools > 0) {
        hp.resize((size_t)n_pools);
        cudaError_t e = cudaMemcpy(hp.data(), root_pools, sizeof(uint64_t) * (size_t)n_pools, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(ctx, e, "pasur_build_round: reading root pools");
        pools_host = hp.data();
    }
    for (int64_t i = 0; i < n_pools; i++) {
        uint64_t p = pools_host[i];
        if (p >> 52) return set_err(ctx, PASUR_EINVAL, "pasur_build_round: pool has bits above 51");
        if (p & (ha | hb)) return set_err(ctx, PASUR_EINVAL, "pasur_build_round: pool overlaps the round's hands");
        if (i > 0 && p <= pools_host[i - 1]) return set_err(ctx, PASUR_EINVAL, "pasur_build_round: pools not strictly ascending");
    }
    pasur_tree *t = new (std::nothrow) pasur_tree();
    if (!t) return set_err(ctx, PASUR_ENOMEM, "pasur_build_round: host allocation");
    t->ctx = ctx;
    t->round = round;
    t->final_round = round == 5;
    memcpy(t->deck, deck, 52);
    t->hand_a = ha;
    t->hand_b = hb;
    t->n_roots = n_pools;
    uint64_t *dpools = nullptr;
    int rc = tree_alloc(t, (void **)&dpools, sizeof(uint64_t) * (size_t)(n_pools + 1));
    if (rc == PASUR_OK && n_pools > 0) {
        cudaError_t e = cudaMemcpyAsync(dpools, pools_host, sizeof(uint64_t) * (size_t)n_pools, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "pasur_build_round: copy pools");
    }
    if (rc == PASUR_OK) rc = build_levels(t, dpools);
    if (rc != PASUR_OK) {
        free_tree_mem(t);
        cudaStreamSynchronize(ctx->stream);
        delete t;
        return rc;
    }
    ctx->live_trees++;
    *out = t;
    return PASUR_OK;
}

int pasur_tree_free(pasur_tree *t) {
    if (!t) return PASUR_EINVAL;
    set_device(t->ctx);
    free_tree_mem(t);
    cudaStreamSynchronize(t->ctx->stream);
    t->ctx->live_trees--;
    delete t;
    return PASUR_OK;
}

int pasur_tree_sizes(const pasur_tree *t, int64_t gt_sizes[9], int64_t fgt_sizes[9]) {
    if (check_tree(t)) return PASUR_EINVAL;
    for (int k = 0; k < 9; k++) {
        if (gt_sizes) gt_sizes[k] = t->M[k];
        if (fgt_sizes) fgt_sizes[k] = t->unfolded ? t->Q[k] : -1;
    }
    return PASUR_OK;
}

int pasur_unfold(pasur_tree *t, const int64_t *score_offs, const pasur_score *scores, int64_t level_sizes_out[9]) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (!score_offs || (!scores && t->n_roots > 0)) return set_err(ctx, PASUR_EINVAL, "pasur_unfold: NULL argument");
    if (t->unfolded) return set_err(ctx, PASUR_EINVAL, "pasur_unfold: tree is already unfolded");
    int64_t nr = t->n_roots;
    if (score_offs[0] != 0) return set_err(ctx, PASUR_EINVAL, "pasur_unfold: score_offs[0] must be 0");
    for (int64_t g = 0; g < nr; g++) {
        if (score_offs[g + 1] < score_offs[g]) return set_err(ctx, PASUR_EINVAL, "pasur_unfold: score_offs must not decrease");
        for (int64_t s = score_offs[g]; s < score_offs[g + 1]; s++) {
            const pasur_score &x = scores[s];
            if (x.a_clubs < 0 || x.a_clubs > 13 || x.b_clubs < 0 || x.b_clubs > 13 || x.bonus < 0 || x.bonus > 2)
                return set_err(ctx, PASUR_EINVAL, "pasur_unfold: score field out of range");
            if (s > score_offs[g]) {
                const pasur_score &y = scores[s - 1];
                if (score_key(y.a_clubs, y.b_clubs, y.delta, y.bonus) >= score_key(x.a_clubs, x.b_clubs, x.delta, x.bonus))
                    return set_err(ctx, PASUR_EINVAL, "pasur_unfold: scores of a root must be strictly ascending");
            }
        }
    }
    int64_t ns = score_offs[nr];
    t->score_off_h.assign(score_offs, score_offs + nr + 1);
    t->scores_h.assign(scores, scores + ns);
    PASUR_TRY(tree_alloc(t, (void **)&t->score_off_d, sizeof(int64_t) * (size_t)(nr + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->scores_d, sizeof(pasur_score) * (size_t)(ns + 1)));
    PASUR_CUDA(ctx, cudaMemcpyAsync(t->score_off_d, score_offs, sizeof(int64_t) * (size_t)(nr + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (ns > 0)
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->scores_d, scores, sizeof(pasur_score) * (size_t)ns, cudaMemcpyHostToDevice, ctx->stream));
    PASUR_TRY(unfold_levels(t));
    t->unfolded = true;
    if (level_sizes_out)
        for (int k = 0; k < 9; k++) level_sizes_out[k] = t->Q[k];
    return PASUR_OK;
}

int pasur_cfr_iterate_roots(pasur_tree *t, const pasur_config *cfg, const float *next_root_util, int64_t root_first,
                            int64_t root_count) {
    if (check_tree(t)) return PASUR_EINVAL;
    if (root_first < 0 || root_count < 0 || root_first + root_count > t->n_roots)
        return set_err(t->ctx, PASUR_EINVAL, "pasur_cfr_iterate_roots: root range outside the tree's GT roots");
    if (t->cfr_ready && (t->range_first != root_first || t->range_count != root_count))
        return set_err(t->ctx, PASUR_EINVAL, "pasur_cfr_iterate_roots: the root range is fixed by the first call");
    if (!t->cfr_ready) {
        t->range_first = root_first;
        t->range_count = root_count;
    }
    return pasur_cfr_iterate(t, cfg, next_root_util);
}

int pasur_root_sizes(const pasur_tree *t, int64_t *gt_nodes_out, int64_t cap) {
    if (check_tree(t)) return PASUR_EINVAL;
    if (!gt_nodes_out || cap < t->n_roots) return set_err(t->ctx, PASUR_EOVERFLOW, "pasur_root_sizes: cap < GT roots");
    for (int64_t g = 0; g < t->n_roots; g++) {
        int64_t n = 0;
        for (int k = 0; k < 9; k++) n += t->roots_h[(size_t)g].lvl_count[k];
        gt_nodes_out[g] = n;
    }
    return PASUR_OK;
}

int pasur_cfr_iterate(pasur_tree *t, const pasur_config *cfg, const float *next_root_util) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (!cfg) return set_err(ctx, PASUR_EINVAL, "pasur_cfr_iterate: cfg is NULL");
    if (!t->unfolded) return set_err(ctx, PASUR_EINVAL, "pasur_cfr_iterate: tree is not unfolded");
    if (cfg->variant != 0 && cfg->variant != 1) return set_err(ctx, PASUR_EINVAL, "pasur_cfr_iterate: variant must be 0 or 1");
    if (cfg->iters < 0 || !(cfg->rm_deadzone >= 0.f)) return set_err(ctx, PASUR_EINVAL, "pasur_cfr_iterate: bad iters / rm_deadzone");
    if (t->variant >= 0 && t->variant != cfg->variant)
        return set_err(ctx, PASUR_EINVAL, "pasur_cfr_iterate: variant changed during a run");
    if (!t->cfr_ready) {
        float *nu = nullptr;
        size_t nb = 0;
        if (!t->final_round) {
            if (!t->has_next) return set_err(ctx, PASUR_EINVAL, "pasur_cfr_iterate: call pasur_next_roots first (non-final round)");
            if (!next_root_util) return set_err(ctx, PASUR_EINVAL, "pasur_cfr_iterate: next_root_util is required (non-final round)");
            if (is_device_ptr(next_root_util)) {
                nu = const_cast<float *>(next_root_util);
            } else {
                nb = sizeof(float) * (size_t)(t->n_next_roots + 1);
                PASUR_TRY(dev_alloc(ctx, (void **)&nu, nb));
                PASUR_CUDA(ctx, cudaMemcpyAsync(nu, next_root_util, sizeof(float) * (size_t)t->n_next_roots,
                                                cudaMemcpyHostToDevice, ctx->stream));
            }
        }
        PhaseTimer pt(ctx->stream, "cfr set-up");
        int rc = plan_solve_slots(t, cfg->merge_delta != 0, nu);
        pt.mark("solved slots");
        if (rc == PASUR_OK) rc = compute_leaf_values(t, nu);
        pt.mark("leaf values");
        if (nb) dev_free(ctx, nu, nb);
        if (rc != PASUR_OK) return rc;
        PASUR_TRY(cfr_prepare(t, cfg));
        pt.mark("layout and plan");
    }
    t->variant = cfg->variant;
    return cfr_run(t, cfg);
}

int pasur_avg_strategy(const pasur_tree *t, float *out, int64_t cap) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (!t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_avg_strategy: no CFR run yet");
    int64_t ne = 0;
    for (int k = 1; k < 9; k++) ne += t->Q[k];
    if (!out || cap < ne) return set_err(ctx, PASUR_EOVERFLOW, "pasur_avg_strategy: need " + std::to_string(ne) + " floats");
    if (is_device_ptr(out)) {
        PASUR_TRY(cfr_export_sigma(t, out));
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return PASUR_OK;
    }
    float *tmp = nullptr;
    size_t b = sizeof(float) * (size_t)(ne + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&tmp, b));
    int rc = cfr_export_sigma(t, tmp);
    if (rc == PASUR_OK) rc = copy_out(ctx, out, tmp, ne);
    dev_free(ctx, tmp, b);
    return rc;
}

int pasur_avg_strategy_async(const pasur_tree *t, float *out, int64_t cap) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (!t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_avg_strategy_async: no CFR run yet");
    int64_t ne = 0;
    for (int k = 1; k < 9; k++) ne += t->Q[k];
    if (!out || cap < ne) return set_err(ctx, PASUR_EOVERFLOW, "pasur_avg_strategy_async: need " + std::to_string(ne) + " floats");
    if (is_device_ptr(out)) return cfr_export_sigma(t, out);  // stream-ordered on the context's stream
    if (!ctx->copy_stream) {
        PASUR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        PASUR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->copy_after, cudaEventDisableTiming));
    }
    float *tmp = nullptr;
    const size_t b = sizeof(float) * (size_t)(ne + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&tmp, b));
    int rc = cfr_export_sigma(t, tmp);
    if (rc != PASUR_OK) {
        dev_free(ctx, tmp, b);
        return rc;
    }
    // the copy and the release of the staging buffer follow the export on the copy stream, so the
    // context's stream (the next round's CFR) runs on while the strategies travel to the host
    PASUR_CUDA(ctx, cudaEventRecord(ctx->copy_after, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_after, 0));
    PASUR_CUDA(ctx, cudaMemcpyAsync(out, tmp, sizeof(float) * (size_t)ne, cudaMemcpyDeviceToHost, ctx->copy_stream));
    PASUR_CUDA(ctx, cudaFreeAsync(tmp, ctx->copy_stream));
    pasur_ctx *a = ctx->acct ? ctx->acct : ctx;
    std::lock_guard<std::mutex> lk(a->acct_mu);
    a->in_use -= std::min(a->in_use, b);
    return PASUR_OK;
}

int pasur_sync(pasur_ctx *ctx) {
    if (!ctx) return PASUR_EINVAL;
    set_device(ctx);
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->copy_stream) PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->copy_stream));
    return PASUR_OK;
}

int pasur_round_utilities(const pasur_tree *t, float *out, int64_t cap) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (!t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_round_utilities: no CFR run yet");
    if (!out || cap < t->Q[0]) return set_err(ctx, PASUR_EOVERFLOW, "pasur_round_utilities: need " + std::to_string(t->Q[0]) + " floats");
    if (is_device_ptr(out)) {
        PASUR_TRY(cfr_export_utilities(t, out));
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return PASUR_OK;
    }
    float *tmp = nullptr;
    size_t b = sizeof(float) * (size_t)(t->Q[0] + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&tmp, b));
    int rc = cfr_export_utilities(t, tmp);
    if (rc == PASUR_OK) rc = copy_out(ctx, out, tmp, t->Q[0]);
    dev_free(ctx, tmp, b);
    return rc;
}

int pasur_next_roots(pasur_tree *t, uint64_t *pools_out, int64_t cap_pools, int64_t *score_offs_out, pasur_score *scores_out,
                     int64_t cap_roots, int64_t *lnk_out, int64_t *n_pools, int64_t *n_roots) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (t->final_round) return set_err(ctx, PASUR_EINVAL, "pasur_next_roots: the final round has no next round");
    if (!t->unfolded) return set_err(ctx, PASUR_EINVAL, "pasur_next_roots: tree is not unfolded");
    if (!t->has_next) PASUR_TRY(next_roots(t, t->next_pools_h, t->next_soff_h, t->next_scores_h));
    const std::vector<uint64_t> &pools = t->next_pools_h;
    const std::vector<int64_t> &soff = t->next_soff_h;
    const std::vector<pasur_score> &sc = t->next_scores_h;
    int64_t np = (int64_t)pools.size(), nr = (int64_t)sc.size();
    if (n_pools) *n_pools = np;
    if (n_roots) *n_roots = nr;
    if ((pools_out || score_offs_out) && cap_pools < np) return set_err(ctx, PASUR_EOVERFLOW, "pasur_next_roots: cap_pools too small");
    if (scores_out && cap_roots < nr) return set_err(ctx, PASUR_EOVERFLOW, "pasur_next_roots: cap_roots too small");
    if (pools_out) std::copy(pools.begin(), pools.end(), pools_out);
    if (score_offs_out) std::copy(soff.begin(), soff.end(), score_offs_out);
    if (scores_out) std::copy(sc.begin(), sc.end(), scores_out);
    if (lnk_out) PASUR_TRY(copy_out(ctx, lnk_out, t->lnk_d, t->Q[8]));
    return PASUR_OK;
}

int pasur_export_level(const pasur_tree *t, int k, int64_t cap, int64_t *parent, int32_t *nchild, int32_t *lay, uint64_t *pick,
                       uint64_t *state, int8_t *rus) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (k < 0 || k > 8) return set_err(ctx, PASUR_EINVAL, "pasur_export_level: k must be 0..8");
    int64_t n = t->M[k];
    if (cap < n) return set_err(ctx, PASUR_EOVERFLOW, "pasur_export_level: cap too small");
    if (parent) {
        if (k == 0) std::fill(parent, parent + n, (int64_t)-1);
        else PASUR_TRY(copy_out(ctx, parent, t->parent[k], n));
    }
    if (nchild) {
        if (k == 8) std::fill(nchild, nchild + n, 0);
        else {
            std::vector<int64_t> off((size_t)n + 1);
            PASUR_TRY(copy_out(ctx, off.data(), t->child_off[k], n + 1));
            for (int64_t i = 0; i < n; i++) nchild[i] = (int32_t)(off[(size_t)i + 1] - off[(size_t)i]);
        }
    }
    if (lay) {
        if (k == 0) std::fill(lay, lay + n, -1);
        else {
            std::vector<int8_t> l((size_t)n);
            PASUR_TRY(copy_out(ctx, l.data(), t->lay[k], n));
            for (int64_t i = 0; i < n; i++) lay[i] = l[(size_t)i];
        }
    }
    if (pick) {
        if (k == 0) std::fill(pick, pick + n, 0ULL);
        else PASUR_TRY(copy_out(ctx, pick, t->pick[k], n));
    }
    if (state || rus) {
        std::vector<GTState> s((size_t)n);
        PASUR_TRY(copy_out(ctx, s.data(), t->st[k], n));
        for (int64_t i = 0; i < n; i++) {
            if (state) {
                state[3 * i] = s[(size_t)i].hand[0];
                state[3 * i + 1] = s[(size_t)i].hand[1];
                state[3 * i + 2] = s[(size_t)i].pool;
            }
            if (rus)
                for (int f = 0; f < 7; f++) rus[7 * i + f] = (int8_t)rus_get(s[(size_t)i].rus, f);
        }
    }
    return PASUR_OK;
}

int pasur_leaf_values(const pasur_tree *t, float *out, int64_t cap) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (!t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_leaf_values: leaf values are fixed by the first pasur_cfr_iterate");
    if (!out || cap < t->Q[8]) return set_err(ctx, PASUR_EOVERFLOW, "pasur_leaf_values: cap too small");
    if (is_device_ptr(out)) {
        PASUR_TRY(expand_leaf_values(t, out));
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return PASUR_OK;
    }
    float *tmp = nullptr;
    const size_t b = sizeof(float) * (size_t)(t->Q[8] + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&tmp, b));
    int rc = expand_leaf_values(t, tmp);
    if (rc == PASUR_OK) rc = copy_out(ctx, out, tmp, t->Q[8]);
    dev_free(ctx, tmp, b);
    return rc;
}

int pasur_cfr_convergence(pasur_tree *t, const pasur_config *cfg, const float *next_root_util, const int64_t *checkpoints,
                          int n, double *mse_out) {
    if (check_tree(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    set_device(ctx);
    if (!cfg || !checkpoints || !mse_out || n < 1) return set_err(ctx, PASUR_EINVAL, "pasur_cfr_convergence: bad arguments");
    int64_t prev = t->iters_done;
    for (int i = 0; i < n; i++) {
        if (checkpoints[i] <= prev || checkpoints[i] - prev > INT32_MAX)
            return set_err(ctx, PASUR_EINVAL, "pasur_cfr_convergence: checkpoints must increase past the iterations done");
        prev = checkpoints[i];
    }
    std::vector<float *> snap((size_t)n, nullptr);
    double *acc = nullptr;
    size_t sb = 0;
    int rc = PASUR_OK;
    auto release = [&]() {
        for (float *p : snap)
            if (p) dev_free(ctx, p, sb);
        if (acc) dev_free(ctx, acc, sizeof(double) * (size_t)n);
    };
    for (int i = 0; i < n && rc == PASUR_OK; i++) {
        pasur_config c = *cfg;
        c.iters = (int32_t)(checkpoints[i] - t->iters_done);
        rc = pasur_cfr_iterate(t, &c, next_root_util);
        if (rc != PASUR_OK) break;
        if (!sb) {
            int64_t ce = 0;
            for (int k = 1; k < 9; k++) ce += t->cQ[k];
            sb = sizeof(float) * (size_t)(ce + 1);
        }
        rc = dev_alloc(ctx, (void **)&snap[(size_t)i], sb);
        if (rc == PASUR_OK) rc = export_sigma_solved(t, snap[(size_t)i]);
    }
    if (rc == PASUR_OK) rc = dev_alloc(ctx, (void **)&acc, sizeof(double) * (size_t)n);
    if (rc == PASUR_OK && cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)n, ctx->stream) != cudaSuccess)
        rc = set_err(ctx, PASUR_ECUDA, "pasur_cfr_convergence: memset");
    for (int i = 0; i < n && rc == PASUR_OK; i++) rc = sigma_sqdiff(t, snap[(size_t)i], snap[(size_t)(n - 1)], acc + i);
    std::vector<double> h((size_t)n, 0.0);
    if (rc == PASUR_OK && (cudaMemcpyAsync(h.data(), acc, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
                           cudaStreamSynchronize(ctx->stream) != cudaSuccess))
        rc = set_err(ctx, PASUR_ECUDA, "pasur_cfr_convergence: read back");
    release();
    if (rc != PASUR_OK) return rc;
    int64_t ne = 0;
    for (int k = 1; k < 9; k++) ne += t->Q[k];
    for (int i = 0; i < n; i++) mse_out[i] = ne > 0 ? h[(size_t)i] / (double)ne : 0.0;
    return PASUR_OK;
}

int pasur_root_paths(const pasur_tree *t, int32_t *path_out, int64_t cap) {
    if (check_tree(t)) return PASUR_EINVAL;
    if (!t->cfr_ready) return set_err(t->ctx, PASUR_EINVAL, "pasur_root_paths: no CFR run yet");
    if (!path_out || cap < t->n_roots) return set_err(t->ctx, PASUR_EOVERFLOW, "pasur_root_paths: cap < GT roots");
    for (int64_t g = 0; g < t->n_roots; g++) path_out[g] = t->croots_h[(size_t)g].cls;
    return PASUR_OK;
}

int pasur_solved_sizes(const pasur_tree *t, int64_t solved_sizes[9], int64_t *swept_edges) {
    if (check_tree(t)) return PASUR_EINVAL;
    if (!t->cfr_ready) return set_err(t->ctx, PASUR_EINVAL, "pasur_solved_sizes: no CFR run yet");
    for (int k = 0; k < 9; k++)
        if (solved_sizes) solved_sizes[k] = t->cQ[k];
    if (swept_edges) *swept_edges = t->swept_edges;
    return PASUR_OK;
}

int pasur_swept_pairs(const pasur_tree *t, int64_t *swept_pairs) {
    if (check_tree(t) || !swept_pairs) return PASUR_EINVAL;
    if (!t->cfr_ready) return set_err(t->ctx, PASUR_EINVAL, "pasur_swept_pairs: no CFR run yet");
    *swept_pairs = t->swept_pairs;
    return PASUR_OK;
}

int pasur_last_cfr_stats(const pasur_tree *t, float *ms, int64_t *edges, int32_t *launches) {
    if (check_tree(t)) return PASUR_EINVAL;
    if (ms) *ms = t->last_ms;
    if (edges) {
        int64_t ne = 0;
        for (int k = 1; k < 9; k++) ne += t->Q[k];
        *edges = ne;
    }
    if (launches) *launches = t->last_launches;
    return PASUR_OK;
}

}  // extern "C"

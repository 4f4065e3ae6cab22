// Between-hand update (section "Between-Hand Updates", CodeSnippet "BetweenHands"): the next
// round's FGT roots and the link of every FGT leaf to its next root (t_lnk).
//
// Two sorts replace the paper's chain of unique() calls: the pools of the GT leaves are sorted
// (52-bit keys) to number the distinct next pools, then every FGT leaf gets the key
// (pool number, normalised next score) and a second sort + unique numbers the next FGT roots
// in canonical order (pool ascending, then score ascending).
#include <algorithm>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

unsigned grid_for(int64_t threads, int block) {
    int64_t b = (threads + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

__global__ void k_pool_keys(const GTState *__restrict__ st, int64_t m, uint64_t *__restrict__ keys, int64_t *__restrict__ vals) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        keys[j] = st[j].pool;
        vals[j] = j;
    }
}

__global__ void k_mark_new(const uint64_t *__restrict__ keys, int64_t n, int32_t *__restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// rank[vals[i]] = number of distinct keys before sorted position i's key; uniq[rank] = key
__global__ void k_scatter_rank(const uint64_t *__restrict__ keys, const int64_t *__restrict__ vals, int64_t n,
                               const int32_t *__restrict__ flag, const int64_t *__restrict__ idx,
                               int64_t *__restrict__ rank, uint64_t *__restrict__ uniq) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = idx[i] + flag[i] - 1;
        rank[vals[i]] = r;
        if (flag[i]) uniq[r] = keys[i];
    }
}

__global__ void k_leaf_root_keys(const GTState *__restrict__ st, const int32_t *__restrict__ root, int64_t m,
                                 const int64_t *__restrict__ fgt_off, const int64_t *__restrict__ score_off,
                                 const pasur_score *__restrict__ scores, const int64_t *__restrict__ gnk,
                                 uint64_t *__restrict__ keys, int64_t *__restrict__ vals, int32_t *__restrict__ err) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        GTState s = st[j];
        int32_t g = root[j];
        int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0;
        int d = rus_diff(s.rus);
        uint64_t hi = (uint64_t)gnk[j] << kScoreKeyBits;
        for (int64_t x = 0; x < ns; x++) {
            pasur_score sc = scores[score_off[g] + x];
            int ac = sc.a_clubs + rus_get(s.rus, 0), bc = sc.b_clubs + rus_get(s.rus, 1), bonus = sc.bonus;
            int delta = sc.delta + d;
            normalize_score(ac, bc, bonus);
            if (delta < -32768 || delta > 32767 || ac > 15 || bc > 15) atomicOr(err, 4);
            keys[q0 + x] = hi | score_key(ac, bc, delta, bonus);
            vals[q0 + x] = q0 + x;
        }
    }
}

int bits_for(int64_t n) {
    int b = 0;
    while (((int64_t)1 << b) < n) b++;
    return b;
}

// sort (keys, vals) of length n, then rank[vals[i]] = distinct-key rank and uniq[] = distinct keys
int unique_rank(pasur_ctx *ctx, uint64_t *keys, int64_t *vals, int64_t n, int bits, int64_t *rank, uint64_t *uniq,
                int64_t *n_unique) {
    PASUR_TRY(radix_sort_pairs(ctx, keys, vals, n, bits));
    int32_t *flag = nullptr;
    int64_t *idx = nullptr;
    size_t fb = sizeof(int32_t) * (size_t)(n + 1), ib = sizeof(int64_t) * (size_t)(n + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&flag, fb));
    PASUR_TRY(dev_alloc(ctx, (void **)&idx, ib));
    if (n > 0) {
        k_mark_new<<<grid_for(n, 256), 256, 0, ctx->stream>>>(keys, n, flag);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    int rc = exclusive_scan_i32(ctx, flag, idx, n);
    if (rc == PASUR_OK && n > 0) {
        k_scatter_rank<<<grid_for(n, 256), 256, 0, ctx->stream>>>(keys, vals, n, flag, idx, rank, uniq);
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "k_scatter_rank");
    }
    if (rc == PASUR_OK) rc = read_i64(ctx, idx + n, n_unique);
    dev_free(ctx, flag, fb);
    dev_free(ctx, idx, ib);
    return rc;
}

}  // namespace

int next_roots(pasur_tree *t, std::vector<uint64_t> &pools, std::vector<int64_t> &score_off,
               std::vector<pasur_score> &scores) {
    pasur_ctx *ctx = t->ctx;
    int64_t m8 = t->M[8], q8 = t->Q[8];
    // 1. distinct pools of the GT leaves
    uint64_t *k1 = nullptr, *u1 = nullptr;
    int64_t *v1 = nullptr, *gnk = nullptr;
    size_t b8 = sizeof(uint64_t) * (size_t)(m8 + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&k1, b8));
    PASUR_TRY(dev_alloc(ctx, (void **)&u1, b8));
    PASUR_TRY(dev_alloc(ctx, (void **)&v1, b8));
    PASUR_TRY(dev_alloc(ctx, (void **)&gnk, b8));
    if (m8 > 0) {
        k_pool_keys<<<grid_for(m8, 256), 256, 0, ctx->stream>>>(t->st[8], m8, k1, v1);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    int64_t n_pools = 0;
    PASUR_TRY(unique_rank(ctx, k1, v1, m8, 52, gnk, u1, &n_pools));
    pools.resize((size_t)n_pools);
    if (n_pools)
        PASUR_CUDA(ctx, cudaMemcpyAsync(pools.data(), u1, sizeof(uint64_t) * (size_t)n_pools, cudaMemcpyDeviceToHost, ctx->stream));
    // 2. next FGT roots
    uint64_t *k2 = nullptr, *u2 = nullptr;
    int64_t *v2 = nullptr;
    size_t bq = sizeof(uint64_t) * (size_t)(q8 + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&k2, bq));
    PASUR_TRY(dev_alloc(ctx, (void **)&u2, bq));
    PASUR_TRY(dev_alloc(ctx, (void **)&v2, bq));
    if (!t->lnk_d) PASUR_TRY(tree_alloc(t, (void **)&t->lnk_d, bq));
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int32_t), ctx->stream));
    if (m8 > 0) {
        k_leaf_root_keys<<<grid_for(m8, 256), 256, 0, ctx->stream>>>(t->st[8], t->root[8], m8, t->fgt_off[8], t->score_off_d,
                                                                     t->scores_d, gnk, k2, v2, ctx->errflag);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    int32_t ef = 0;
    PASUR_CUDA(ctx, cudaMemcpyAsync(&ef, ctx->errflag, sizeof ef, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ef) return set_err(ctx, PASUR_EOVERFLOW, "a next-round score leaves the int16 range");
    int64_t n_roots = 0;
    PASUR_TRY(unique_rank(ctx, k2, v2, q8, kScoreKeyBits + bits_for(n_pools + 1), t->lnk_d, u2, &n_roots));
    std::vector<uint64_t> rk((size_t)n_roots);
    if (n_roots)
        PASUR_CUDA(ctx, cudaMemcpyAsync(rk.data(), u2, sizeof(uint64_t) * (size_t)n_roots, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, k1, b8);
    dev_free(ctx, u1, b8);
    dev_free(ctx, v1, b8);
    dev_free(ctx, gnk, b8);
    dev_free(ctx, k2, bq);
    dev_free(ctx, u2, bq);
    dev_free(ctx, v2, bq);
    score_off.assign((size_t)n_pools + 1, 0);
    scores.resize((size_t)n_roots);
    for (int64_t r = 0; r < n_roots; r++) {
        int64_t p = (int64_t)(rk[(size_t)r] >> kScoreKeyBits);
        int ac, bc, delta, bonus;
        score_unkey((uint32_t)(rk[(size_t)r] & ((1ULL << kScoreKeyBits) - 1)), ac, bc, delta, bonus);
        scores[(size_t)r] = pasur_score{(int16_t)ac, (int16_t)bc, (int16_t)delta, (int16_t)bonus};
        score_off[(size_t)p + 1] = r + 1;
    }
    for (int64_t p = 1; p <= n_pools; p++) score_off[(size_t)p] = std::max(score_off[(size_t)p], score_off[(size_t)p - 1]);
    t->n_next_roots = n_roots;
    t->has_next = true;
    return PASUR_OK;
}

}  // namespace pasur

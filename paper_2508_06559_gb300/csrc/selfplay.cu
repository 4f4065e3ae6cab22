// Self-play: sampled games through consecutive round trees, every move drawn from the average
// strategy of the FGT node reached (the paper's fair-value simulation, §Results and the learned-
// strategy study; one choice per parent as in §External Sampling).  One thread plays one game:
// a game touches 8 nodes per round, so the work is a chain of dependent, scattered loads and the
// kernel is latency bound; the grid keeps enough games in flight per SM to hide it.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

// Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC 2011): ten rounds of two 64x64->128-bit
// products by odd constants; high halves xored with the other counter words and the round key;
// the key advances by the two Weyl constants between rounds.  Returns word 0 of the block.
__device__ __forceinline__ uint64_t philox4x64_w0(uint64_t x0, uint64_t x1, uint64_t x2, uint64_t x3, uint64_t k0,
                                                  uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
        const uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return x0;
}

// Draw of ply `ply` of game `game`: counter (ply, game, 0, 0), key (seed, 0), the top 24 bits of
// word 0 as a float in [0, 1) (exact).
__device__ __forceinline__ float draw(uint64_t seed, uint64_t game, uint64_t ply) {
    const uint64_t w = philox4x64_w0(ply, game, 0, 0, seed, 0);
    return __fmul_rn(__uint2float_rn((unsigned)(w >> 40)), 1.0f / 16777216.0f);
}

__global__ void __launch_bounds__(128) k_selfplay(const SpRound *__restrict__ views, int n_rounds, int64_t n_deals,
                                                  int64_t n_games, const uint64_t *__restrict__ seeds,
                                                  const int64_t *__restrict__ roots, int16_t *__restrict__ out) {
    const int64_t total = n_deals * n_games;
    for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < total;
         gid += (int64_t)gridDim.x * blockDim.x) {
        const int64_t deal = gid / n_games, game = gid - deal * n_games;
        const uint64_t seed = seeds[deal];
        int64_t q = roots[deal];
        uint64_t ply = 0;
        int result = 0;
        for (int i = 0; i < n_rounds; i++) {
            const SpRound *v = views + deal * n_rounds + i;
            // GT root owning FGT root q: the last root whose first FGT node is <= q
            const int64_t *f0 = v->fgt_off[0];
            int64_t lo = 0, hi = v->n_roots - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (f0[mid] <= q) lo = mid;
                else hi = mid - 1;
            }
            int64_t j = lo;
            const int64_t s = q - f0[lo];
#pragma unroll 1
            for (int k = 0; k < 8; k++) {
                const int64_t cb = v->child_off[k][j], ce = v->child_off[k][j + 1];
                const float u = draw(seed, (uint64_t)game, ply++);
                const float *sg = v->sigma + v->sig_base[k + 1] + s;
                const int64_t *fo = v->fgt_off[k + 1];
                float tot = 0.f;
                for (int64_t c = cb; c < ce; c++) tot = __fadd_rn(tot, __ldg(sg + fo[c]));
                const float target = __fmul_rn(u, tot);
                float cum = 0.f;
                int64_t pick = -1, last = -1;
                for (int64_t c = cb; c < ce; c++) {
                    const float w = __ldg(sg + fo[c]);
                    cum = __fadd_rn(cum, w);
                    if (w > 0.f) last = c;
                    if (pick < 0 && cum > target) pick = c;
                }
                j = pick >= 0 ? pick : (last >= 0 ? last : cb);
            }
            const int64_t leaf = v->fgt_off[8][j] + s;
            if (i + 1 < n_rounds) {
                q = v->lnk[leaf];
            } else {
                // final game difference: inherited difference + this round's difference after
                // CleanUp + the 7-clubs bonus (eq. final_util)
                const GTState st = v->st8[j];
                const pasur_score sc = v->scores[v->score_off[v->root8[j]] + s];
                const uint64_t r = cleanup_rus(st.rus, st.pool);
                result = sc.delta + rus_diff(r) + bonus_points(bonus_after(sc.a_clubs, sc.b_clubs, sc.bonus, r));
            }
        }
        out[gid] = (int16_t)result;
    }
}

}  // namespace

void selfplay_view(const pasur_tree *t, const float *sigma_dev, SpRound *v) {
    memset(v, 0, sizeof *v);
    int64_t base = 0;
    for (int k = 0; k < 9; k++) {
        if (k < 8) v->child_off[k] = t->child_off[k];
        v->fgt_off[k] = t->fgt_off[k];
        if (k >= 1) {
            v->sig_base[k] = base;
            base += t->Q[k];
        }
    }
    v->sigma = sigma_dev;
    v->lnk = t->final_round ? nullptr : t->lnk_d;
    v->n_roots = t->n_roots;
    v->st8 = t->st[8];
    v->root8 = t->root[8];
    v->score_off = t->score_off_d;
    v->scores = t->scores_d;
}

int selfplay_launch(pasur_ctx *ctx, const SpRound *views_dev, int n_rounds, int64_t n_deals, int64_t n_games,
                    const uint64_t *seeds_dev, const int64_t *roots_dev, int16_t *out_dev) {
    const int64_t total = n_deals * n_games;
    ctx->selfplay_ms = 0.f;
    ctx->selfplay_games = total;
    if (total == 0) return PASUR_OK;
    const int block = 128;
    int per_sm = 0;
    PASUR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_selfplay, block, 0));
    const int64_t want = (total + block - 1) / block;
    const int64_t cap = (int64_t)std::max(1, per_sm) * ctx->num_sms;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(want, cap));
    cudaEvent_t e0, e1;
    PASUR_CUDA(ctx, cudaEventCreate(&e0));
    PASUR_CUDA(ctx, cudaEventCreate(&e1));
    PASUR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    k_selfplay<<<grid, block, 0, ctx->stream>>>(views_dev, n_rounds, n_deals, n_games, seeds_dev, roots_dev, out_dev);
    ctx->launches++;
    cudaError_t le = cudaGetLastError();
    PASUR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    PASUR_CUDA(ctx, cudaEventSynchronize(e1));
    PASUR_CUDA(ctx, cudaEventElapsedTime(&ctx->selfplay_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (le != cudaSuccess) return cuda_err(ctx, le, "k_selfplay launch");
    return PASUR_OK;
}

}  // namespace pasur

using namespace pasur;

namespace {

int64_t edges_of(const pasur_tree *t) {
    int64_t ne = 0;
    for (int k = 1; k < 9; k++) ne += t->Q[k];
    return ne;
}

}  // namespace

extern "C" {

int pasur_selfplay(pasur_ctx *ctx, pasur_tree *const *rounds, int n_rounds, const float *const *sigma, int64_t root_q,
                   int64_t n_games, uint64_t seed, int16_t *out) {
    if (!ctx) return PASUR_EINVAL;
    if (!rounds || n_rounds < 1 || n_rounds > 6) return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: need 1..6 round trees");
    if (n_games < 0 || (n_games > 0 && !out)) return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: n_games >= 0 and out required");
    for (int i = 0; i < n_rounds; i++) {
        const pasur_tree *t = rounds[i];
        if (!t || t->ctx != ctx) return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: tree missing or from another context");
        if (!t->unfolded) return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: every tree must be unfolded");
        if (!(sigma && sigma[i]) && !t->cfr_ready)
            return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: a tree without a CFR run needs its strategy passed in sigma");
        if (i + 1 < n_rounds) {
            const pasur_tree *nx = rounds[i + 1];
            if (!nx || nx->round != t->round + 1 || memcmp(nx->deck, t->deck, 52) != 0)
                return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: trees must be consecutive rounds of one deal");
            if (!t->has_next || t->n_next_roots != nx->Q[0])
                return set_err(ctx, PASUR_EINVAL,
                               "pasur_selfplay: round " + std::to_string(t->round) +
                                   " needs pasur_next_roots, and the next tree must be unfolded over exactly those roots");
        }
    }
    if (!rounds[n_rounds - 1]->final_round) return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: the last tree must be the final round");
    if (root_q < 0 || root_q >= rounds[0]->Q[0]) return set_err(ctx, PASUR_EINVAL, "pasur_selfplay: root_q out of range");
    cudaSetDevice(ctx->device);
    if (n_games == 0) {
        ctx->selfplay_ms = 0.f;
        ctx->selfplay_games = 0;
        return PASUR_OK;
    }
    std::vector<std::pair<void *, size_t>> tmp;
    auto alloc = [&](void **p, size_t b) {
        int rc = dev_alloc(ctx, p, b);
        if (rc == PASUR_OK) tmp.push_back({*p, b});
        return rc;
    };
    auto release = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (auto &x : tmp) dev_free(ctx, x.first, x.second);
    };
    int rc = PASUR_OK;
    std::vector<SpRound> views((size_t)n_rounds);
    for (int i = 0; i < n_rounds && rc == PASUR_OK; i++) {
        const pasur_tree *t = rounds[i];
        const int64_t ne = edges_of(t);
        const float *sg = sigma ? sigma[i] : nullptr;
        float *dev = nullptr;
        if (!sg || !is_device_ptr(sg)) {
            rc = alloc((void **)&dev, sizeof(float) * (size_t)(ne + 1));
            if (rc != PASUR_OK) break;
            if (sg) {
                if (ne && cudaMemcpyAsync(dev, sg, sizeof(float) * (size_t)ne, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
                    rc = set_err(ctx, PASUR_ECUDA, "pasur_selfplay: copy sigma");
            } else {
                rc = cfr_export_sigma(t, dev);
            }
            sg = dev;
        }
        selfplay_view(t, sg, &views[(size_t)i]);
    }
    SpRound *views_d = nullptr;
    uint64_t *seed_d = nullptr;
    int64_t *root_d = nullptr;
    int16_t *out_d = nullptr;
    const bool out_dev = is_device_ptr(out);
    if (rc == PASUR_OK) rc = alloc((void **)&views_d, sizeof(SpRound) * views.size());
    if (rc == PASUR_OK) rc = alloc((void **)&seed_d, sizeof(uint64_t) + sizeof(int64_t));
    if (rc == PASUR_OK) root_d = (int64_t *)(seed_d + 1);
    if (rc == PASUR_OK && !out_dev) rc = alloc((void **)&out_d, sizeof(int16_t) * (size_t)n_games);
    if (rc == PASUR_OK) {
        if (out_dev) out_d = out;
        uint64_t hb[2] = {seed, (uint64_t)root_q};
        if (cudaMemcpyAsync(views_d, views.data(), sizeof(SpRound) * views.size(), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(seed_d, hb, sizeof hb, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
            rc = set_err(ctx, PASUR_ECUDA, "pasur_selfplay: upload views");
    }
    if (rc == PASUR_OK) rc = selfplay_launch(ctx, views_d, n_rounds, 1, n_games, seed_d, root_d, out_d);
    if (rc == PASUR_OK && !out_dev &&
        cudaMemcpyAsync(out, out_d, sizeof(int16_t) * (size_t)n_games, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        rc = set_err(ctx, PASUR_ECUDA, "pasur_selfplay: copy results");
    release();
    return rc;
}

int pasur_last_selfplay_stats(const pasur_ctx *ctx, float *ms, int64_t *games) {
    if (!ctx) return PASUR_EINVAL;
    if (ms) *ms = ctx->selfplay_ms;
    if (games) *games = ctx->selfplay_games;
    return PASUR_OK;
}

}  // extern "C"

// Game values of a round under fixed or optimal play, in fp64, level by level from the leaves:
// minimax, a best response of one player to the other's strategy, or both players on a given
// strategy.  Chained over the rounds (leaf = the round's difference + the next round's value at
// the linked root, eq. passuputil) they give the best-response values whose gap is the
// exploitability of a strategy profile (section "CFR Algorithm": the average strategy converges
// to an equilibrium; exploitability measures the distance).  Sums are taken child by child in
// canonical order with explicitly rounded multiply and add.
#include <algorithm>
#include <string>
#include <vector>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

// leaf values of level 8 in FGT order (fp64)
__global__ void k_leaf_f64(const GTState *__restrict__ st, const int32_t *__restrict__ root, int64_t m,
                           const int64_t *__restrict__ fgt_off, const int64_t *__restrict__ score_off,
                           const pasur_score *__restrict__ scores, bool final_round, const int64_t *__restrict__ lnk,
                           const double *__restrict__ next, double *__restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const GTState s = st[j];
        const int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0;
        if (final_round) {
            const uint64_t r = cleanup_rus(s.rus, s.pool);
            const int d = rus_diff(r);
            for (int64_t x = 0; x < ns; x++) {
                const pasur_score sc = scores[score_off[root[j]] + x];
                out[q0 + x] = (double)(d + bonus_points(bonus_after(sc.a_clubs, sc.b_clubs, sc.bonus, r)));
            }
        } else {
            const double d = (double)rus_diff(s.rus);
            for (int64_t x = 0; x < ns; x++) out[q0 + x] = __dadd_rn(d, next[lnk[q0 + x]]);
        }
    }
}

// mode 0 minimax, 1 Alex best response (Bob follows sigma), 2 Bob best response, 3 both sigma
__global__ void k_value_level(int k, int64_t m, int mode, const int64_t *__restrict__ child_off,
                              const int64_t *__restrict__ fgt_off, const int64_t *__restrict__ fgt_off_next,
                              const float *__restrict__ sigma_next, const double *__restrict__ vnext,
                              double *__restrict__ vout) {
    const bool alex = (k & 1) == 0;
    const bool opt = mode == 0 || (mode == 1 && alex) || (mode == 2 && !alex);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cb = child_off[j], ce = child_off[j + 1];
        const int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0;
        for (int64_t s = 0; s < ns; s++) {
            double best = 0.0, ev = 0.0;
            for (int64_t c = cb; c < ce; c++) {
                const int64_t q = fgt_off_next[c] + s;
                const double v = vnext[q];
                if (c == cb || (alex ? v > best : v < best)) best = v;
                if (!opt) ev = __dadd_rn(ev, __dmul_rn((double)sigma_next[q], v));
            }
            vout[q0 + s] = opt ? best : ev;
        }
    }
}

unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1 << 20)); }

}  // namespace
}  // namespace pasur

using namespace pasur;

namespace {

// The shared part of the value and reach passes: the strategy on the device (copied, or the
// tree's own average strategy when sigma is NULL), the next-round values on the device, and the
// values of every FGT level under `mode` (v[0..8]; mode 3 = both players on sigma).  Device
// temporaries are appended to tmp.
int value_levels(pasur_tree *t, int mode, const float *sigma, const double *next_values,
                 std::vector<std::pair<void *, size_t>> &tmp, const float **sg_out, double *v[9]) {
    pasur_ctx *ctx = t->ctx;
    int rc = PASUR_OK;
    auto al = [&](void **p, size_t b) {
        if (rc != PASUR_OK) return;
        rc = dev_alloc(ctx, p, b);
        if (rc == PASUR_OK) tmp.push_back({*p, b});
    };
    int64_t ne = 0, base[9] = {0};
    for (int k = 1; k < 9; k++) {
        base[k] = ne;
        ne += t->Q[k];
    }
    const float *sg = nullptr;
    if (mode != 0) {
        if (sigma && is_device_ptr(sigma)) {
            sg = sigma;
        } else {
            float *d = nullptr;
            al((void **)&d, sizeof(float) * (size_t)(ne + 1));
            if (rc == PASUR_OK) {
                if (sigma) rc = cudaMemcpyAsync(d, sigma, sizeof(float) * (size_t)ne, cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess ? PASUR_OK : set_err(ctx, PASUR_ECUDA, "copy sigma");
                else rc = cfr_export_sigma(t, d);
            }
            sg = d;
        }
    }
    const double *nx = nullptr;
    if (!t->final_round) {
        if (is_device_ptr(next_values)) {
            nx = next_values;
        } else {
            double *d = nullptr;
            al((void **)&d, sizeof(double) * (size_t)(t->n_next_roots + 1));
            if (rc == PASUR_OK)
                rc = cudaMemcpyAsync(d, next_values, sizeof(double) * (size_t)t->n_next_roots, cudaMemcpyHostToDevice, ctx->stream) ==
                             cudaSuccess
                         ? PASUR_OK
                         : set_err(ctx, PASUR_ECUDA, "copy next values");
            nx = d;
        }
    }
    for (int k = 0; k < 9; k++) al((void **)&v[k], sizeof(double) * (size_t)(t->Q[k] + 1));
    if (rc == PASUR_OK && t->M[8] > 0) {
        k_leaf_f64<<<grid_of(t->M[8]), 256, 0, ctx->stream>>>(t->st[8], t->root[8], t->M[8], t->fgt_off[8], t->score_off_d,
                                                              t->scores_d, t->final_round, t->lnk_d, nx, v[8]);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_leaf_f64 launch");
    }
    for (int k = 7; k >= 0 && rc == PASUR_OK; k--) {
        if (t->M[k] == 0) continue;
        k_value_level<<<grid_of(t->M[k]), 256, 0, ctx->stream>>>(k, t->M[k], mode, t->child_off[k], t->fgt_off[k],
                                                                 t->fgt_off[k + 1], sg ? sg + base[k + 1] : nullptr, v[k + 1],
                                                                 v[k]);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_value_level launch");
    }
    *sg_out = sg;
    return rc;
}

}  // namespace

extern "C" int pasur_root_values(pasur_tree *t, int mode, const float *sigma, const double *next_values, double *out,
                                 int64_t cap) {
    if (!t) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    if (mode < 0 || mode > 3) return set_err(ctx, PASUR_EINVAL, "pasur_root_values: mode must be 0..3");
    if (!t->unfolded) return set_err(ctx, PASUR_EINVAL, "pasur_root_values: tree not unfolded");
    if (!t->final_round && (!next_values || !t->has_next))
        return set_err(ctx, PASUR_EINVAL, "pasur_root_values: a non-final round needs pasur_next_roots and next_values");
    if (mode != 0 && !sigma && !t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_root_values: no strategy (no CFR run, sigma NULL)");
    if (!out || cap < t->Q[0]) return set_err(ctx, PASUR_EOVERFLOW, "pasur_root_values: need " + std::to_string(t->Q[0]) + " doubles");
    cudaSetDevice(ctx->device);
    std::vector<std::pair<void *, size_t>> tmp;
    const float *sg = nullptr;
    double *v[9] = {nullptr};
    int rc = value_levels(t, mode, sigma, next_values, tmp, &sg, v);
    if (rc == PASUR_OK && t->Q[0] > 0 &&
        cudaMemcpyAsync(out, v[0], sizeof(double) * (size_t)t->Q[0], is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess)
        rc = set_err(ctx, PASUR_ECUDA, "copy root values");
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == PASUR_OK) rc = set_err(ctx, PASUR_ECUDA, "pasur_root_values: sync");
    for (auto &x : tmp) dev_free(ctx, x.first, x.second);
    return rc;
}

namespace pasur {
namespace {

// reach of the FGT nodes of level k+1 from those of level k: both players following sigma
__global__ void k_reach_level(int64_t m, const int64_t *__restrict__ child_off, const int64_t *__restrict__ fgt_off,
                              const int64_t *__restrict__ fgt_off_next, const float *__restrict__ sigma_next,
                              const double *__restrict__ rin, double *__restrict__ rout) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cb = child_off[j], ce = child_off[j + 1];
        const int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0;
        for (int64_t c = cb; c < ce; c++)
            for (int64_t s = 0; s < ns; s++) {
                const int64_t q = fgt_off_next[c] + s;
                rout[q] = __dmul_rn(rin[q0 + s], (double)sigma_next[q]);
            }
    }
}

// reach of level k+1 from level k when one player best-responds (mode 1: Alex, 2: Bob; values of
// level k+1 under that mode in vnext): at the responder's nodes the whole reach goes to the child
// its value pass chose (the first best child in canonical order), at the other player's nodes it
// follows sigma
__global__ void k_response_reach_level(int k, int64_t m, int mode, const int64_t *__restrict__ child_off,
                                       const int64_t *__restrict__ fgt_off, const int64_t *__restrict__ fgt_off_next,
                                       const float *__restrict__ sigma_next, const double *__restrict__ vnext,
                                       const double *__restrict__ rin, double *__restrict__ rout) {
    const bool alex = (k & 1) == 0;
    const bool responder = (mode == 1 && alex) || (mode == 2 && !alex);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cb = child_off[j], ce = child_off[j + 1];
        const int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0;
        for (int64_t s = 0; s < ns; s++) {
            const double r = rin[q0 + s];
            if (responder) {
                int64_t arg = cb;
                double best = 0.0;
                for (int64_t c = cb; c < ce; c++) {
                    const double v = vnext[fgt_off_next[c] + s];
                    if (c == cb || (alex ? v > best : v < best)) {
                        best = v;
                        arg = c;
                    }
                }
                for (int64_t c = cb; c < ce; c++) rout[fgt_off_next[c] + s] = c == arg ? r : 0.0;
            } else {
                for (int64_t c = cb; c < ce; c++) {
                    const int64_t q = fgt_off_next[c] + s;
                    rout[q] = __dmul_rn(r, (double)sigma_next[q]);
                }
            }
        }
    }
}

// every FGT leaf's reach added to its next-round root
__global__ void k_reach_next(int64_t n, const int64_t *__restrict__ lnk, const double *__restrict__ r, double *next) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        if (r[q] != 0.0) atomicAdd(&next[lnk[q]], r[q]);
}

}  // namespace
}  // namespace pasur

extern "C" int pasur_round_reach(pasur_tree *t, const float *sigma, const double *root_reach, double *next_reach,
                                 int64_t cap) {
    if (!t) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    if (!t->unfolded || t->final_round || !t->has_next)
        return set_err(ctx, PASUR_EINVAL, "pasur_round_reach: needs an unfolded non-final tree after pasur_next_roots");
    if (!sigma && !t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_round_reach: no strategy (no CFR run, sigma NULL)");
    if (!next_reach || cap < t->n_next_roots)
        return set_err(ctx, PASUR_EOVERFLOW, "pasur_round_reach: need " + std::to_string(t->n_next_roots) + " doubles");
    cudaSetDevice(ctx->device);
    std::vector<std::pair<void *, size_t>> tmp;
    int rc = PASUR_OK;
    auto al = [&](void **p, size_t b) {
        if (rc != PASUR_OK) return;
        rc = dev_alloc(ctx, p, b);
        if (rc == PASUR_OK) tmp.push_back({*p, b});
    };
    int64_t ne = 0, base[9] = {0};
    for (int k = 1; k < 9; k++) {
        base[k] = ne;
        ne += t->Q[k];
    }
    const float *sg = nullptr;
    if (sigma && is_device_ptr(sigma)) {
        sg = sigma;
    } else {
        float *d = nullptr;
        al((void **)&d, sizeof(float) * (size_t)(ne + 1));
        if (rc == PASUR_OK) {
            if (sigma) rc = cudaMemcpyAsync(d, sigma, sizeof(float) * (size_t)ne, cudaMemcpyHostToDevice, ctx->stream) == cudaSuccess ? PASUR_OK : set_err(ctx, PASUR_ECUDA, "copy sigma");
            else rc = cfr_export_sigma(t, d);
        }
        sg = d;
    }
    double *r[9] = {nullptr}, *nx = nullptr;
    for (int k = 0; k < 9; k++) al((void **)&r[k], sizeof(double) * (size_t)(t->Q[k] + 1));
    al((void **)&nx, sizeof(double) * (size_t)(t->n_next_roots + 1));
    if (rc == PASUR_OK) {
        std::vector<double> ones;
        const double *src = root_reach;
        if (!root_reach) {
            ones.assign((size_t)t->Q[0], 1.0);
            src = ones.data();
        }
        if (t->Q[0] > 0 && cudaMemcpyAsync(r[0], src, sizeof(double) * (size_t)t->Q[0],
                                           is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                           ctx->stream) != cudaSuccess)
            rc = set_err(ctx, PASUR_ECUDA, "copy root reach");
        if (rc == PASUR_OK && cudaMemsetAsync(nx, 0, sizeof(double) * (size_t)(t->n_next_roots + 1), ctx->stream) != cudaSuccess)
            rc = set_err(ctx, PASUR_ECUDA, "memset");
        if (rc == PASUR_OK && !root_reach) rc = cudaStreamSynchronize(ctx->stream) == cudaSuccess ? PASUR_OK : set_err(ctx, PASUR_ECUDA, "sync");
    }
    for (int k = 0; k < 8 && rc == PASUR_OK; k++) {
        if (t->M[k] == 0) continue;
        k_reach_level<<<grid_of(t->M[k]), 256, 0, ctx->stream>>>(t->M[k], t->child_off[k], t->fgt_off[k], t->fgt_off[k + 1],
                                                                 sg + base[k + 1], r[k], r[k + 1]);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_reach_level launch");
    }
    if (rc == PASUR_OK && t->Q[8] > 0) {
        k_reach_next<<<grid_of(t->Q[8]), 256, 0, ctx->stream>>>(t->Q[8], t->lnk_d, r[8], nx);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_reach_next launch");
    }
    if (rc == PASUR_OK && t->n_next_roots > 0 &&
        cudaMemcpyAsync(next_reach, nx, sizeof(double) * (size_t)t->n_next_roots,
                        is_device_ptr(next_reach) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        rc = set_err(ctx, PASUR_ECUDA, "copy next reach");
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == PASUR_OK) rc = set_err(ctx, PASUR_ECUDA, "pasur_round_reach: sync");
    for (auto &x : tmp) dev_free(ctx, x.first, x.second);
    return rc;
}

extern "C" int pasur_response_reach(pasur_tree *t, int mode, const float *sigma, const double *next_values,
                                    const double *root_reach, double *next_reach, int64_t cap) {
    if (!t) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    if (mode < 1 || mode > 3) return set_err(ctx, PASUR_EINVAL, "pasur_response_reach: mode must be 1..3");
    if (!t->unfolded || t->final_round || !t->has_next)
        return set_err(ctx, PASUR_EINVAL, "pasur_response_reach: needs an unfolded non-final tree after pasur_next_roots");
    if (!next_values) return set_err(ctx, PASUR_EINVAL, "pasur_response_reach: next_values is required");
    if (!sigma && !t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_response_reach: no strategy (no CFR run, sigma NULL)");
    if (!next_reach || cap < t->n_next_roots)
        return set_err(ctx, PASUR_EOVERFLOW, "pasur_response_reach: need " + std::to_string(t->n_next_roots) + " doubles");
    cudaSetDevice(ctx->device);
    std::vector<std::pair<void *, size_t>> tmp;
    const float *sg = nullptr;
    double *v[9] = {nullptr};
    int rc = value_levels(t, mode, sigma, next_values, tmp, &sg, v);
    auto al = [&](void **p, size_t b) {
        if (rc != PASUR_OK) return;
        rc = dev_alloc(ctx, p, b);
        if (rc == PASUR_OK) tmp.push_back({*p, b});
    };
    double *r[9] = {nullptr}, *nx = nullptr;
    for (int k = 0; k < 9; k++) al((void **)&r[k], sizeof(double) * (size_t)(t->Q[k] + 1));
    al((void **)&nx, sizeof(double) * (size_t)(t->n_next_roots + 1));
    std::vector<double> ones;
    if (rc == PASUR_OK) {
        const double *src = root_reach;
        if (!root_reach) {
            ones.assign((size_t)t->Q[0], 1.0);
            src = ones.data();
        }
        if (t->Q[0] > 0 && cudaMemcpyAsync(r[0], src, sizeof(double) * (size_t)t->Q[0],
                                           is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                           ctx->stream) != cudaSuccess)
            rc = set_err(ctx, PASUR_ECUDA, "copy root reach");
        if (rc == PASUR_OK && cudaMemsetAsync(nx, 0, sizeof(double) * (size_t)(t->n_next_roots + 1), ctx->stream) != cudaSuccess)
            rc = set_err(ctx, PASUR_ECUDA, "memset");
    }
    int64_t base[9] = {0}, ne = 0;
    for (int k = 1; k < 9; k++) {
        base[k] = ne;
        ne += t->Q[k];
    }
    for (int k = 0; k < 8 && rc == PASUR_OK; k++) {
        if (t->M[k] == 0) continue;
        k_response_reach_level<<<grid_of(t->M[k]), 256, 0, ctx->stream>>>(k, t->M[k], mode, t->child_off[k], t->fgt_off[k],
                                                                          t->fgt_off[k + 1], sg + base[k + 1], v[k + 1], r[k],
                                                                          r[k + 1]);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_response_reach_level launch");
    }
    if (rc == PASUR_OK && t->Q[8] > 0) {
        k_reach_next<<<grid_of(t->Q[8]), 256, 0, ctx->stream>>>(t->Q[8], t->lnk_d, r[8], nx);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_reach_next launch");
    }
    if (rc == PASUR_OK && t->n_next_roots > 0 &&
        cudaMemcpyAsync(next_reach, nx, sizeof(double) * (size_t)t->n_next_roots,
                        is_device_ptr(next_reach) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        rc = set_err(ctx, PASUR_ECUDA, "copy next reach");
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == PASUR_OK) rc = set_err(ctx, PASUR_ECUDA, "pasur_response_reach: sync");
    for (auto &x : tmp) dev_free(ctx, x.first, x.second);
    return rc;
}

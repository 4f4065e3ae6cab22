// Round game-tree build (legal-move enumeration, level-by-level expansion), the Unfolding
// Process and the leaf values of a round.
//
// Expansion of level k (section "Actions"): one warp per node counts its legal moves (count
// pass), a device-wide exclusive scan turns the counts into child offsets, and one warp per node
// writes its children in canonical order (emit pass).  Numeric captures come from a table of
// every set of numeric cards completing a given numeric card to 11 (the paper's t_40x2764,
// section "Numerical Actions"), sorted ascending; a warp tests 32 entries per step against the
// pool with a ballot, and in the emit pass the ballot prefix gives each found move its slot.
#include <algorithm>
#include <cstring>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

// ---- capture table (host) -------------------------------------------------------------------
// For the numeric card c (value v = rank+1), every set of other numeric cards whose values add to
// 11 - v: choose how many cards of each value 1..10 to take (value partitions of 11 - v), then
// which suits; ascending by mask.
void partitions(int value, int remaining, const int *avail, int *take, int c_excluded,
                std::vector<uint64_t> &out) {
    if (remaining == 0) {
        // expand suits: cartesian product over values of the suit combinations
        std::vector<uint64_t> acc(1, 0ULL);
        for (int v = 1; v <= 10; v++) {
            if (!take[v]) continue;
            std::vector<uint64_t> next;
            for (uint64_t base : acc) {
                for (int sm = 0; sm < 16; sm++) {
                    if (__builtin_popcount(sm) != take[v]) continue;
                    uint64_t m = 0;
                    bool ok = true;
                    for (int s = 0; s < 4; s++) {
                        if (!(sm >> s & 1)) continue;
                        int id = 4 * (v - 1) + s;
                        if (id == c_excluded) { ok = false; break; }
                        m |= 1ULL << id;
                    }
                    if (ok) next.push_back(base | m);
                }
            }
            acc.swap(next);
        }
        out.insert(out.end(), acc.begin(), acc.end());
        return;
    }
    if (value > 10 || value > remaining) return;
    for (int k = 0; k <= avail[value] && k * value <= remaining; k++) {
        take[value] = k;
        partitions(value + 1, remaining - k * value, avail, take, c_excluded, out);
    }
    take[value] = 0;
}

void capture_table(std::vector<uint64_t> &tab, std::vector<int32_t> &off) {
    tab.clear();
    off.assign(41, 0);
    for (int c = 0; c < 40; c++) {
        off[c] = (int32_t)tab.size();
        int v = c / 4 + 1;
        int avail[11], take[11] = {0};
        for (int x = 0; x <= 10; x++) avail[x] = 4;
        avail[v] = 3;
        std::vector<uint64_t> sets;
        partitions(1, 11 - v, avail, take, c, sets);
        std::sort(sets.begin(), sets.end());
        tab.insert(tab.end(), sets.begin(), sets.end());
    }
    off[40] = (int32_t)tab.size();
}

// ---- one move (CodeSnippet "ApplyActions" + the running-score update) -----------------------
__device__ __forceinline__ GTState apply_move(GTState s, int mover, int c, uint64_t pick, bool final_round) {
    uint64_t bit = 1ULL << c;
    s.hand[mover] &= ~bit;
    if (pick == 0) {
        s.pool |= bit;
    } else {
        s.pool &= ~pick;
        uint64_t cap = pick | bit;
        s.rus = rus_add(s.rus, mover, set_clubs(cap));
        s.rus = rus_add(s.rus, 3 + 2 * mover, set_points(cap));
        s.rus = rus_set(s.rus, 2, mover + 1);
        bool jack = c >= 40 && c < 44;
        if (s.pool == 0 && !jack && !final_round) s.rus = rus_add(s.rus, 4 + 2 * mover, 1);
    }
    return s;
}

struct EmitOut {
    GTState *st;
    int64_t *parent;
    int8_t *lay;
    uint64_t *pick;
    int32_t *root;
};

__device__ __forceinline__ void emit_child(const EmitOut &o, int64_t pos, const GTState &s, int mover, int c,
                                           uint64_t pick, bool final_round, int64_t node, int32_t root) {
    o.st[pos] = apply_move(s, mover, c, pick, final_round);
    o.parent[pos] = node;
    o.lay[pos] = (int8_t)c;
    o.pick[pos] = pick;
    o.root[pos] = root;
}

// first index in [b, e) with tab[i] > x (all lanes compute the same value)
__device__ __forceinline__ int upper_bound_u64(const uint64_t *tab, int b, int e, uint64_t x) {
    while (b < e) {
        int m = (b + e) >> 1;
        if (tab[m] <= x) b = m + 1;
        else e = m;
    }
    return b;
}

template <bool EMIT>
__global__ void k_expand(const GTState *__restrict__ st, int64_t m, int mover, bool final_round,
                         const uint64_t *__restrict__ tab, const int32_t *__restrict__ tab_off,
                         int32_t *__restrict__ deg_out, const int64_t *__restrict__ child_off,
                         const int32_t *__restrict__ root_in, EmitOut o) {
    int lane = threadIdx.x & 31;
    unsigned lt = (1u << lane) - 1u;
    int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t node = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; node < m; node += warps) {
        GTState s = st[node];
        uint64_t hand = s.hand[mover], pool = s.pool;
        int64_t out = EMIT ? child_off[node] : 0;
        int32_t root = EMIT ? root_in[node] : 0;
        int cnt = 0;
        while (hand) {
            int c = __ffsll((long long)hand) - 1;
            hand &= hand - 1;
            if (c < 40) {
                uint64_t pn = pool & kNumeric;
                int found = 0;
                if (pn) {
                    int b = tab_off[c];
                    int e = upper_bound_u64(tab, b, tab_off[c + 1], pn);
                    for (int base = b; base < e; base += 32) {
                        int i = base + lane;
                        uint64_t P = i < e ? tab[i] : 0;
                        bool ok = i < e && (P & ~pn) == 0;
                        unsigned bal = __ballot_sync(0xFFFFFFFFu, ok);
                        if (EMIT && ok)
                            emit_child(o, out + cnt + found + __popc(bal & lt), s, mover, c, P, final_round, node, root);
                        found += __popc(bal);
                    }
                }
                if (found == 0) {
                    if (EMIT && lane == 0) emit_child(o, out + cnt, s, mover, c, 0ULL, final_round, node, root);
                    found = 1;
                }
                cnt += found;
            } else if (c < 44) {
                if (EMIT && lane == 0)
                    emit_child(o, out + cnt, s, mover, c, pool & (kNumeric | kJacks), final_round, node, root);
                cnt += 1;
            } else {
                uint64_t same = pool & (c < 48 ? kQueens : kKings);
                int n = __popcll(same);
                if (n == 0) {
                    if (EMIT && lane == 0) emit_child(o, out + cnt, s, mover, c, 0ULL, final_round, node, root);
                    cnt += 1;
                } else {
                    if (EMIT && lane < n) {
                        uint64_t x = same;
                        for (int i = 0; i < lane; i++) x &= x - 1;
                        emit_child(o, out + cnt + lane, s, mover, c, x & (~x + 1), final_round, node, root);
                    }
                    cnt += n;
                }
            }
        }
        if (!EMIT && lane == 0) deg_out[node] = cnt;
    }
}

__global__ void k_init_roots(const uint64_t *__restrict__ pools, int64_t n, uint64_t ha, uint64_t hb,
                             GTState *__restrict__ st, int32_t *__restrict__ root) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        GTState s;
        s.hand[0] = ha;
        s.hand[1] = hb;
        s.pool = pools[i];
        s.rus = 0;
        st[i] = s;
        root[i] = (int32_t)i;
    }
}

// first GT node of every root at every level: begin(g, 0) = g, begin(g, k+1) = child_off_k[begin(g, k)]
struct OffPtrs {
    const int64_t *p[9];
};
__global__ void k_root_bounds(int64_t n_roots, OffPtrs co, int64_t *__restrict__ out) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= n_roots; g += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = g;
        out[g * 9] = b;
        for (int k = 0; k < 8; k++) {
            b = co.p[k][b];
            out[g * 9 + k + 1] = b;
        }
    }
}

__global__ void k_slots_per_node(const int32_t *__restrict__ root, int64_t m, const int64_t *__restrict__ score_off,
                                 int64_t *__restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = root[j];
        out[j] = score_off[g + 1] - score_off[g];
    }
}

// leaf values (eq. final_util and eq. passuputil) of the solved slots: solved slot x of leaf j
// (root g) takes the score and the next-round link of its representative full slot crep; out in
// solved FGT order (cfgt_off); umax receives max |value| as float bits
__global__ void k_leaf_values(const GTState *__restrict__ st, const int32_t *__restrict__ root, int64_t m,
                              const int64_t *__restrict__ fgt_off, const int64_t *__restrict__ cfgt_off,
                              const int64_t *__restrict__ csoff, const int32_t *__restrict__ crep,
                              const int64_t *__restrict__ score_off, const pasur_score *__restrict__ scores,
                              bool final_round, const int64_t *__restrict__ lnk, const float *__restrict__ next_util,
                              float *__restrict__ out, unsigned *__restrict__ umax_bits) {
    float local_max = 0.f;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        GTState s = st[j];
        int32_t g = root[j];
        const int64_t q0 = fgt_off[j], c0 = cfgt_off[j], ns = cfgt_off[j + 1] - c0;
        const int32_t *rep = crep + csoff[g];
        if (final_round) {
            uint64_t r = cleanup_rus(s.rus, s.pool);
            int d = rus_diff(r);
            for (int64_t x = 0; x < ns; x++) {
                pasur_score sc = scores[score_off[g] + rep[x]];
                float v = (float)(d + bonus_points(bonus_after(sc.a_clubs, sc.b_clubs, sc.bonus, r)));
                out[c0 + x] = v;
                local_max = fmaxf(local_max, fabsf(v));
            }
        } else {
            int d = rus_diff(s.rus);
            for (int64_t x = 0; x < ns; x++) {
                float v = (float)d + next_util[lnk[q0 + rep[x]]];
                out[c0 + x] = v;
                local_max = fmaxf(local_max, fabsf(v));
            }
        }
    }
    if (!(local_max <= 3.0e38f)) local_max = __int_as_float(0x7f800000);  // non-finite -> +inf
    if (umax_bits) atomicMax(umax_bits, __float_as_uint(local_max));
}

// Every full slot of a non-final round's leaves must see the same next-round utility as the
// representative of its solved slot; flag a leaf where it does not (bitwise comparison).
__global__ void k_check_merge(const int32_t *__restrict__ root, int64_t m, const int64_t *__restrict__ fgt_off,
                              const int64_t *__restrict__ score_off, const int64_t *__restrict__ csoff,
                              const int32_t *__restrict__ crep, const int64_t *__restrict__ cidx0,
                              const int64_t *__restrict__ lnk, const float *__restrict__ next_util, int32_t *bad) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = root[j];
        const int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0, s0 = score_off[g];
        for (int64_t s = 0; s < ns; s++) {
            const int32_t r = crep[cidx0[s0 + s]];
            if (r != s && __float_as_uint(next_util[lnk[q0 + s]]) != __float_as_uint(next_util[lnk[q0 + r]])) {
                atomicOr(bad, 1);
                break;
            }
        }
    }
}

// full leaf values from the solved ones: leaf (j, s) takes the value of its solved slot
__global__ void k_expand_leaves(const int32_t *__restrict__ root, int64_t m, const int64_t *__restrict__ fgt_off,
                                const int64_t *__restrict__ cfgt_off, const int64_t *__restrict__ score_off,
                                const int64_t *__restrict__ csoff, const int64_t *__restrict__ cidx0,
                                const float *__restrict__ in, float *__restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = root[j];
        const int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0, c0 = cfgt_off[j] - csoff[g];
        for (int64_t s = 0; s < ns; s++) out[q0 + s] = in[c0 + cidx0[score_off[g] + s]];
    }
}

unsigned grid_for(int64_t threads, int block) {
    int64_t b = (threads + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

}  // namespace

int ensure_capture_table(pasur_ctx *ctx) {
    if (ctx->tab) return PASUR_OK;
    std::vector<uint64_t> tab;
    std::vector<int32_t> off;
    capture_table(tab, off);
    PASUR_TRY(dev_alloc(ctx, (void **)&ctx->tab, tab.size() * sizeof(uint64_t)));
    PASUR_TRY(dev_alloc(ctx, (void **)&ctx->tab_off, off.size() * sizeof(int32_t)));
    PASUR_CUDA(ctx, cudaMemcpyAsync(ctx->tab, tab.data(), tab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(ctx->tab_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

int build_levels(pasur_tree *t, const uint64_t *root_pools_dev) {
    pasur_ctx *ctx = t->ctx;
    PASUR_TRY(ensure_capture_table(ctx));
    int64_t m0 = t->n_roots;
    t->M[0] = m0;
    PASUR_TRY(tree_alloc(t, (void **)&t->st[0], sizeof(GTState) * (size_t)(m0 + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->root[0], sizeof(int32_t) * (size_t)(m0 + 1)));
    if (m0 > 0) {
        k_init_roots<<<grid_for(m0, 256), 256, 0, ctx->stream>>>(root_pools_dev, m0, t->hand_a, t->hand_b, t->st[0], t->root[0]);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    for (int k = 0; k < 8; k++) {
        int64_t m = t->M[k];
        int mover = k & 1;
        int32_t *deg = nullptr;
        size_t degb = sizeof(int32_t) * (size_t)(m + 1);
        PASUR_TRY(dev_alloc(ctx, (void **)&deg, degb));
        PASUR_TRY(tree_alloc(t, (void **)&t->child_off[k], sizeof(int64_t) * (size_t)(m + 1)));
        EmitOut none{};
        if (m > 0) {
            k_expand<false><<<grid_for(m * 32, 256), 256, 0, ctx->stream>>>(t->st[k], m, mover, t->final_round, ctx->tab,
                                                                          ctx->tab_off, deg, nullptr, nullptr, none);
            ctx->launches++;
            PASUR_CUDA(ctx, cudaGetLastError());
        }
        int rc = exclusive_scan_i32(ctx, deg, t->child_off[k], m);
        dev_free(ctx, deg, degb);
        if (rc != PASUR_OK) return rc;
        int64_t m1 = 0;
        PASUR_TRY(read_i64(ctx, t->child_off[k] + m, &m1));
        t->M[k + 1] = m1;
        // the level's five arrays in one allocation, each piece 256-byte aligned
        const size_t cap = (size_t)m1 + 1;
        auto piece = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t b_st = piece(sizeof(GTState) * cap), b_par = piece(sizeof(int64_t) * cap),
                     b_lay = piece(sizeof(int8_t) * cap), b_pick = piece(sizeof(uint64_t) * cap);
        char *lv = nullptr;
        PASUR_TRY(tree_alloc(t, (void **)&lv, b_st + b_par + b_lay + b_pick + piece(sizeof(int32_t) * cap)));
        t->st[k + 1] = (GTState *)lv;
        t->parent[k + 1] = (int64_t *)(lv + b_st);
        t->lay[k + 1] = (int8_t *)(lv + b_st + b_par);
        t->pick[k + 1] = (uint64_t *)(lv + b_st + b_par + b_lay);
        t->root[k + 1] = (int32_t *)(lv + b_st + b_par + b_lay + b_pick);
        if (m > 0) {
            EmitOut o{t->st[k + 1], t->parent[k + 1], t->lay[k + 1], t->pick[k + 1], t->root[k + 1]};
            k_expand<true><<<grid_for(m * 32, 256), 256, 0, ctx->stream>>>(t->st[k], m, mover, t->final_round, ctx->tab,
                                                                         ctx->tab_off, nullptr, t->child_off[k], t->root[k], o);
            ctx->launches++;
            PASUR_CUDA(ctx, cudaGetLastError());
        }
    }
    // per-root level bounds -> RootInfo (host + device)
    int64_t nr = t->n_roots;
    size_t bb = sizeof(int64_t) * 9 * (size_t)(nr + 1);
    PASUR_TRY(tree_alloc(t, (void **)&t->bounds_d, bb));
    int64_t *bounds = t->bounds_d;
    OffPtrs co;
    for (int k = 0; k < 8; k++) co.p[k] = t->child_off[k];
    co.p[8] = nullptr;
    k_root_bounds<<<grid_for(nr + 1, 256), 256, 0, ctx->stream>>>(nr, co, bounds);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    std::vector<int64_t> hb(9 * (size_t)(nr + 1));
    PASUR_CUDA(ctx, cudaMemcpyAsync(hb.data(), bounds, bb, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    t->roots_h.assign((size_t)nr, RootInfo{});
    int64_t soff = 0;
    for (int64_t g = 0; g < nr; g++) {
        RootInfo &ri = t->roots_h[(size_t)g];
        int64_t local = 0;
        for (int k = 0; k < 9; k++) {
            ri.lvl_begin[k] = hb[(size_t)g * 9 + k];
            int64_t cnt = hb[(size_t)(g + 1) * 9 + k] - ri.lvl_begin[k];
            if (local + cnt > INT32_MAX) return set_err(ctx, PASUR_EOVERFLOW, "a root subtree exceeds 2^31 nodes");
            ri.lvl_count[k] = (int32_t)cnt;
            ri.local_start[k] = (int32_t)local;
            local += cnt;
        }
        ri.local_start[9] = (int32_t)local;
        ri.n_internal = ri.local_start[8];
        ri.struct_off = soff;
        soff += ri.n_internal;
    }
    return PASUR_OK;
}

int unfold_levels(pasur_tree *t) {
    pasur_ctx *ctx = t->ctx;
    int64_t mmax = 0;
    for (int k = 0; k < 9; k++) mmax = std::max(mmax, t->M[k]);
    // one slot-count buffer serves every level (the levels run in stream order)
    int64_t *slots = nullptr;
    const size_t sb = sizeof(int64_t) * (size_t)(mmax + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&slots, sb));
    int rc = PASUR_OK;
    for (int k = 0; k < 9 && rc == PASUR_OK; k++) {
        int64_t m = t->M[k];
        if (!t->fgt_off[k]) rc = tree_alloc(t, (void **)&t->fgt_off[k], sizeof(int64_t) * (size_t)(m + 1));
        if (rc == PASUR_OK && m > 0) {
            k_slots_per_node<<<grid_for(m, 256), 256, 0, ctx->stream>>>(t->root[k], m, t->score_off_d, slots);
            ctx->launches++;
            if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_slots_per_node launch");
        }
        if (rc == PASUR_OK) rc = exclusive_scan_i64(ctx, slots, t->fgt_off[k], m);
        if (rc == PASUR_OK) rc = read_i64(ctx, t->fgt_off[k] + m, &t->Q[k]);
    }
    dev_free(ctx, slots, sb);
    return rc;
}

// leaf values without any host synchronisation (the batch solver captures this in a CUDA graph);
// umax_bits (device, may be NULL) receives max |value| as float bits
int launch_leaf_values(pasur_tree *t, const float *next_util_dev, unsigned *umax_bits) {
    pasur_ctx *ctx = t->ctx;
    if (t->M[8] == 0) return PASUR_OK;
    k_leaf_values<<<grid_for(t->M[8], 256), 256, 0, ctx->stream>>>(t->st[8], t->root[8], t->M[8], t->fgt_off[8],
                                                                  t->cfgt_off[8], t->csoff_d, t->crep_d, t->score_off_d,
                                                                  t->scores_d, t->final_round, t->lnk_d, next_util_dev,
                                                                  t->leaf_v, umax_bits);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    return PASUR_OK;
}

int compute_leaf_values(pasur_tree *t, const float *next_util_dev) {
    pasur_ctx *ctx = t->ctx;
    int64_t q8 = t->cQ[8];
    if (!t->leaf_v) PASUR_TRY(tree_alloc(t, (void **)&t->leaf_v, sizeof(float) * (size_t)(q8 + 1)));
    unsigned *umax = nullptr;
    PASUR_TRY(dev_alloc(ctx, (void **)&umax, sizeof(unsigned)));
    PASUR_CUDA(ctx, cudaMemsetAsync(umax, 0, sizeof(unsigned), ctx->stream));
    if (t->M[8] > 0) {
        k_leaf_values<<<grid_for(t->M[8], 256), 256, 0, ctx->stream>>>(
            t->st[8], t->root[8], t->M[8], t->fgt_off[8], t->cfgt_off[8], t->csoff_d, t->crep_d, t->score_off_d,
            t->scores_d, t->final_round, t->lnk_d, next_util_dev, t->leaf_v, umax);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    unsigned hb = 0;
    PASUR_CUDA(ctx, cudaMemcpyAsync(&hb, umax, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, umax, sizeof(unsigned));
    float u;
    memcpy(&u, &hb, sizeof u);
    if (!(u <= 3.0e38f)) return set_err(ctx, PASUR_ENUMERIC, "non-finite leaf value");
    t->umax = u;
    return PASUR_OK;
}

int plan_solve_slots(pasur_tree *t, bool merge, const float *next_util_dev) {
    pasur_ctx *ctx = t->ctx;
    if (t->csoff_d) return PASUR_OK;
    const int64_t nr = t->n_roots, q0 = t->Q[0];
    // group the slots of every root by (a_clubs, b_clubs, bonus), numbered by first appearance
    std::vector<int64_t> csoff((size_t)nr + 1, 0), cidx0((size_t)q0 + 1, 0);
    std::vector<int32_t> crep;
    crep.reserve((size_t)q0 + 1);
    bool any = false;
    for (int64_t g = 0; g < nr; g++) {
        const int64_t a = t->score_off_h[(size_t)g], b = t->score_off_h[(size_t)g + 1];
        const int64_t base = (int64_t)crep.size();
        std::vector<std::pair<uint32_t, int32_t>> seen;  // key -> solved slot within the root
        for (int64_t s = a; s < b; s++) {
            const pasur_score &x = t->scores_h[(size_t)s];
            const uint32_t key = merge ? ((uint32_t)x.a_clubs << 8) | ((uint32_t)x.b_clubs << 2) | (uint32_t)x.bonus
                                       : (uint32_t)(s - a);
            int32_t c = -1;
            for (const auto &k : seen)
                if (k.first == key) c = k.second;
            if (c < 0) {
                c = (int32_t)seen.size();
                seen.push_back({key, c});
                crep.push_back((int32_t)(s - a));
            } else {
                any = true;
            }
            cidx0[(size_t)s] = base + c;
        }
        csoff[(size_t)g + 1] = (int64_t)crep.size();
    }
    const int64_t cq0 = (int64_t)crep.size();
    PASUR_TRY(tree_alloc(t, (void **)&t->csoff_d, sizeof(int64_t) * (size_t)(nr + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->crep_d, sizeof(int32_t) * (size_t)(cq0 + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->cidx0_d, sizeof(int64_t) * (size_t)(q0 + 1)));
    PASUR_CUDA(ctx, cudaMemcpyAsync(t->csoff_d, csoff.data(), sizeof(int64_t) * (size_t)(nr + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (cq0) PASUR_CUDA(ctx, cudaMemcpyAsync(t->crep_d, crep.data(), sizeof(int32_t) * (size_t)cq0, cudaMemcpyHostToDevice, ctx->stream));
    if (q0) PASUR_CUDA(ctx, cudaMemcpyAsync(t->cidx0_d, cidx0.data(), sizeof(int64_t) * (size_t)q0, cudaMemcpyHostToDevice, ctx->stream));
    // a non-final round merges only slots whose leaves see the same next-round utilities
    if (any && !t->final_round && next_util_dev && t->M[8] > 0) {
        int32_t *bad = nullptr;
        PASUR_TRY(dev_alloc(ctx, (void **)&bad, sizeof(int32_t)));
        PASUR_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int32_t), ctx->stream));
        k_check_merge<<<grid_for(t->M[8], 256), 256, 0, ctx->stream>>>(t->root[8], t->M[8], t->fgt_off[8], t->score_off_d,
                                                                      t->csoff_d, t->crep_d, t->cidx0_d, t->lnk_d,
                                                                      next_util_dev, bad);
        ctx->launches++;
        int32_t hb = 0;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        dev_free(ctx, bad, sizeof(int32_t));
        if (e != cudaSuccess) return cuda_err(ctx, e, "k_check_merge");
        if (hb) {
            // the given utilities differ between slots that differ only in delta: solve every slot
            PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            for (int64_t g = 0; g <= nr; g++) csoff[(size_t)g] = t->score_off_h[(size_t)g];
            crep.resize((size_t)q0);
            for (int64_t g = 0; g < nr; g++)
                for (int64_t s = t->score_off_h[(size_t)g]; s < t->score_off_h[(size_t)g + 1]; s++) {
                    crep[(size_t)s] = (int32_t)(s - t->score_off_h[(size_t)g]);
                    cidx0[(size_t)s] = s;
                }
            any = false;
            PASUR_TRY(tree_alloc(t, (void **)&t->crep_d, sizeof(int32_t) * (size_t)(q0 + 1)));
            PASUR_CUDA(ctx, cudaMemcpyAsync(t->csoff_d, csoff.data(), sizeof(int64_t) * (size_t)(nr + 1), cudaMemcpyHostToDevice, ctx->stream));
            if (q0) {
                PASUR_CUDA(ctx, cudaMemcpyAsync(t->crep_d, crep.data(), sizeof(int32_t) * (size_t)q0, cudaMemcpyHostToDevice, ctx->stream));
                PASUR_CUDA(ctx, cudaMemcpyAsync(t->cidx0_d, cidx0.data(), sizeof(int64_t) * (size_t)q0, cudaMemcpyHostToDevice, ctx->stream));
            }
        }
    }
    t->merged = any;
    t->csoff_h = csoff;
    {
        // full slots per solved slot (the weight of a solved slot in averages over the FGT)
        std::vector<int32_t> mult((size_t)csoff[(size_t)nr] + 1, 0);
        for (int64_t q = 0; q < q0; q++) mult[(size_t)cidx0[(size_t)q]]++;
        PASUR_TRY(tree_alloc(t, (void **)&t->cmult_d, sizeof(int32_t) * mult.size()));
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->cmult_d, mult.data(), sizeof(int32_t) * mult.size(), cudaMemcpyHostToDevice,
                                        ctx->stream));
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (!any) {
        for (int k = 0; k < 9; k++) {
            t->cfgt_off[k] = t->fgt_off[k];
            t->cQ[k] = t->Q[k];
        }
    } else {
        int64_t mmax = 0;
        for (int k = 0; k < 9; k++) mmax = std::max(mmax, t->M[k]);
        int64_t *slots = nullptr;
        const size_t sb = sizeof(int64_t) * (size_t)(mmax + 1);
        PASUR_TRY(dev_alloc(ctx, (void **)&slots, sb));
        int rc = PASUR_OK;
        for (int k = 0; k < 9 && rc == PASUR_OK; k++) {
            const int64_t m = t->M[k];
            rc = tree_alloc(t, (void **)&t->cfgt_off[k], sizeof(int64_t) * (size_t)(m + 1));
            if (rc == PASUR_OK && m > 0) {
                k_slots_per_node<<<grid_for(m, 256), 256, 0, ctx->stream>>>(t->root[k], m, t->csoff_d, slots);
                ctx->launches++;
                if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_slots_per_node launch");
            }
            if (rc == PASUR_OK) rc = exclusive_scan_i64(ctx, slots, t->cfgt_off[k], m);
            if (rc == PASUR_OK) rc = read_i64(ctx, t->cfgt_off[k] + m, &t->cQ[k]);
        }
        dev_free(ctx, slots, sb);
        if (rc != PASUR_OK) return rc;
    }
    return PASUR_OK;
}

int expand_leaf_values(const pasur_tree *t, float *out_dev) {
    pasur_ctx *ctx = t->ctx;
    if (t->M[8] == 0) return PASUR_OK;
    if (!t->merged) {
        PASUR_CUDA(ctx, cudaMemcpyAsync(out_dev, t->leaf_v, sizeof(float) * (size_t)t->Q[8], cudaMemcpyDeviceToDevice, ctx->stream));
        return PASUR_OK;
    }
    k_expand_leaves<<<grid_for(t->M[8], 256), 256, 0, ctx->stream>>>(t->root[8], t->M[8], t->fgt_off[8], t->cfgt_off[8],
                                                                    t->score_off_d, t->csoff_d, t->cidx0_d, t->leaf_v, out_dev);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    return PASUR_OK;
}

}  // namespace pasur

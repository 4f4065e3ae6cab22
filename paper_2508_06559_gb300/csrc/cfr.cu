// CFR over an unfolded round (section "CFR Algorithm"; eq. RM, eq. avsigma; DCFR eqs.
// DFCR_REG / DFCR_AVG).
//
// Round roots are independent (open hands: every FGT node is its own information set and root
// reach is 1), so the round is cut into work items: one GT root and a run of its score slots.
// A persistent grid takes items from a queue (largest first).  One thread block runs all T
// iterations of an item: per iteration a top-down pass over levels 0..6 (regret matching and
// reach) and a bottom-up pass over levels 7..0 (values, regret and strategy-sum updates), with a
// block barrier between levels; a (node, slot) pair belongs to one thread in each pass, so the
// updates of a parent's child edges need no atomics.  The item's regrets R, strategy sums S,
// values and reaches live in shared memory when they fit ("resident": no DRAM traffic per
// iteration), otherwise in device memory.  Layout of an item: local node index (level-major,
// the root's GT subtree in level order) times slots, slot-minor.
#include <algorithm>
#include <cmath>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

struct CfrParams {
    const CfrItem *items;
    int64_t n_items;
    const RootInfo *roots;
    const int32_t *lcs;
    const uint16_t *ldeg;
    const float *leaf_v;
    const int64_t *fgt_off8;
    const int64_t *fgt_off0;
    float *R, *S, *V, *P0, *P1;
    double *uacc;
    const float *dcfr;  // per iteration: regret factor if R > 0, if R <= 0, strategy-sum factor
    int iters;
    int64_t t0;
    float tau_umax;
    int32_t *counter;
    int32_t *err;
};

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ __forceinline__ size_t resident_bytes(int64_t N, int64_t Nint, int64_t W) {
    return al16((size_t)Nint * 4) + al16((size_t)Nint * 2) + 3 * al16((size_t)N * W * 4) + 2 * al16((size_t)Nint * W * 4);
}

template <int VARIANT>
__global__ void __launch_bounds__(256) k_cfr_items(CfrParams p) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int32_t s_item;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t id = s_item;
        __syncthreads();
        if (id >= p.n_items) break;
        const CfrItem it = p.items[id];
        const RootInfo &ri = p.roots[it.root];
        const int W = it.ns;
        const int N = ri.local_start[9], Nint = ri.n_internal;
        const bool resident = it.scratch_base < 0;
        const int32_t *cs;
        const uint16_t *dg;
        float *R, *S, *V, *P0, *P1;
        if (resident) {
            size_t o = 0;
            int32_t *cs_s = (int32_t *)(sm + o); o += al16((size_t)Nint * 4);
            uint16_t *dg_s = (uint16_t *)(sm + o); o += al16((size_t)Nint * 2);
            R = (float *)(sm + o); o += al16((size_t)N * W * 4);
            S = (float *)(sm + o); o += al16((size_t)N * W * 4);
            V = (float *)(sm + o); o += al16((size_t)N * W * 4);
            P0 = (float *)(sm + o); o += al16((size_t)Nint * W * 4);
            P1 = (float *)(sm + o);
            const int32_t *gcs = p.lcs + ri.struct_off;
            const uint16_t *gdg = p.ldeg + ri.struct_off;
            for (int i = tid; i < Nint; i += nth) {
                cs_s[i] = gcs[i];
                dg_s[i] = gdg[i];
            }
            const float *gR = p.R + it.data_base, *gS = p.S + it.data_base;
            for (int i = tid; i < N * W; i += nth) {
                R[i] = gR[i];
                S[i] = gS[i];
            }
            cs = cs_s;
            dg = dg_s;
        } else {
            cs = p.lcs + ri.struct_off;
            dg = p.ldeg + ri.struct_off;
            R = p.R + it.data_base;
            S = p.S + it.data_base;
            V = p.V + it.scratch_base;
            P0 = p.P0 + it.scratch_base;
            P1 = p.P1 + it.scratch_base;
        }
        // leaf values (constant over the iterations)
        {
            const int nl = ri.lvl_count[8];
            const int64_t jb = ri.lvl_begin[8];
            for (int x = tid; x < nl * W; x += nth) {
                int i = x / W, w = x - i * W;
                V[(int64_t)(Nint + i) * W + w] = p.leaf_v[p.fgt_off8[jb + i] + it.s0 + w];
            }
        }
        __syncthreads();
        double acc = 0.0;
        for (int il = 0; il < p.iters; il++) {
            const int64_t t = p.t0 + il + 1;
            const float thr = p.tau_umax * (float)t;
            float fpos = 0.f, fneg = 0.f, fs = 0.f;
            if (VARIANT == 1) {
                fpos = p.dcfr[3 * il];
                fneg = p.dcfr[3 * il + 1];
                fs = p.dcfr[3 * il + 2];
            }
            for (int w = tid; w < W; w += nth) {
                P0[w] = 1.f;
                P1[w] = 1.f;
            }
            __syncthreads();
            // top-down: reach of levels 1..7 (leaves need none)
            for (int k = 0; k < 7; k++) {
                const int nk = ri.lvl_count[k], base = ri.local_start[k];
                const bool alex = (k & 1) == 0;
                for (int x = tid; x < nk * W; x += nth) {
                    const int i = x / W, w = x - i * W, li = base + i;
                    const int c = cs[li], d = dg[li];
                    const float a0 = P0[li * W + w], a1 = P1[li * W + w];
                    if (d == 1) {
                        P0[c * W + w] = a0;
                        P1[c * W + w] = a1;
                        continue;
                    }
                    float sum = 0.f;
                    for (int a = 0; a < d; a++) {
                        float r = R[(c + a) * W + w];
                        sum += r > thr ? r : 0.f;
                    }
                    const float u = 1.f / (float)d;
                    for (int a = 0; a < d; a++) {
                        float r = R[(c + a) * W + w];
                        float sg = sum > 0.f ? (r > thr ? r / sum : 0.f) : u;
                        P0[(c + a) * W + w] = alex ? a0 * sg : a0;
                        P1[(c + a) * W + w] = alex ? a1 : a1 * sg;
                    }
                }
                __syncthreads();
            }
            // bottom-up: values, regrets, strategy sums
            for (int k = 7; k >= 0; k--) {
                const int nk = ri.lvl_count[k], base = ri.local_start[k];
                const bool alex = (k & 1) == 0;
                for (int x = tid; x < nk * W; x += nth) {
                    const int i = x / W, w = x - i * W, li = base + i;
                    const int c = cs[li], d = dg[li];
                    if (d == 1) {
                        V[li * W + w] = V[c * W + w];
                        continue;
                    }
                    const float a0 = P0[li * W + w], a1 = P1[li * W + w];
                    float sum = 0.f;
                    for (int a = 0; a < d; a++) {
                        float r = R[(c + a) * W + w];
                        sum += r > thr ? r : 0.f;
                    }
                    const float u = 1.f / (float)d;
                    const float v0 = V[c * W + w];
                    float vh = v0;
                    for (int a = 0; a < d; a++) {
                        float r = R[(c + a) * W + w];
                        float sg = sum > 0.f ? (r > thr ? r / sum : 0.f) : u;
                        vh += sg * (V[(c + a) * W + w] - v0);
                    }
                    const float pp = alex ? a0 : a1, po = alex ? a1 : a0;
                    const float spo = alex ? po : -po;
                    for (int a = 0; a < d; a++) {
                        const int q = (c + a) * W + w;
                        float r = R[q];
                        float sg = sum > 0.f ? (r > thr ? r / sum : 0.f) : u;
                        float inst = spo * (V[q] - vh);
                        if (VARIANT == 1) {
                            R[q] = r * (r > 0.f ? fpos : fneg) + inst;
                            S[q] = S[q] * fs + pp * sg;
                        } else {
                            R[q] = r + inst;
                            S[q] = S[q] + pp * sg;
                        }
                    }
                    V[li * W + w] = vh;
                }
                __syncthreads();
            }
            if (tid < W) acc += (double)V[tid];
        }
        if (tid < W) {
            if (!isfinite(acc)) atomicOr(p.err, 1);
            p.uacc[p.fgt_off0[it.root] + it.s0 + tid] += acc;
        }
        if (resident) {
            float *gR = p.R + it.data_base, *gS = p.S + it.data_base;
            for (int i = tid; i < N * W; i += nth) {
                gR[i] = R[i];
                gS[i] = S[i];
            }
        }
        __syncthreads();
    }
}

struct LevelPtrs {
    const int64_t *p[9];
    int64_t base[9];  // offset of level k in the concatenated edge output (levels 1..8)
};

// average strategy of every edge, canonical FGT order, one block per item
__global__ void k_export_sigma(const CfrItem *items, int64_t n_items, const RootInfo *roots, const int32_t *lcs,
                               const uint16_t *ldeg, const float *Sg, LevelPtrs lp, float *out) {
    for (int64_t id = blockIdx.x; id < n_items; id += gridDim.x) {
        const CfrItem it = items[id];
        const RootInfo &ri = roots[it.root];
        const int W = it.ns;
        const int32_t *cs = lcs + ri.struct_off;
        const uint16_t *dg = ldeg + ri.struct_off;
        const float *S = Sg + it.data_base;
        for (int k = 0; k < 8; k++) {
            const int nk = ri.lvl_count[k], base = ri.local_start[k];
            for (int x = threadIdx.x; x < nk * W; x += blockDim.x) {
                const int i = x / W, w = x - i * W, li = base + i;
                const int c = cs[li], d = dg[li];
                float sum = 0.f;
                for (int a = 0; a < d; a++) sum += S[(c + a) * W + w];
                for (int a = 0; a < d; a++) {
                    int64_t j = ri.lvl_begin[k + 1] + (c + a - ri.local_start[k + 1]);
                    float sb = sum > 0.f ? S[(c + a) * W + w] / sum : 1.f / (float)d;
                    out[lp.base[k + 1] + lp.p[k + 1][j] + it.s0 + w] = sb;
                }
            }
        }
    }
}

__global__ void k_export_util(const double *uacc, int64_t n, double inv_t, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(uacc[i] * inv_t);
}

// local structure of every internal GT node: first child (local index) and number of children
__global__ void k_local_structure(const int32_t *root, const int64_t *child_off, int64_t m, int k,
                                  const RootInfo *roots, int32_t *lcs, uint16_t *ldeg, int32_t *err) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const RootInfo &ri = roots[root[j]];
        int64_t li = ri.local_start[k] + (j - ri.lvl_begin[k]);
        int64_t c0 = child_off[j], d = child_off[j + 1] - c0;
        if (d < 1 || d > 65535) atomicOr(err, 2);
        lcs[ri.struct_off + li] = (int32_t)(ri.local_start[k + 1] + (c0 - ri.lvl_begin[k + 1]));
        ldeg[ri.struct_off + li] = (uint16_t)d;
    }
}

unsigned grid_for(int64_t threads, int block) {
    int64_t b = (threads + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

}  // namespace

int cfr_prepare(pasur_tree *t, const pasur_config *cfg) {
    pasur_ctx *ctx = t->ctx;
    // local structure arrays
    int64_t nint = 0;
    for (int k = 0; k < 8; k++) nint += t->M[k];
    PASUR_TRY(tree_alloc(t, (void **)&t->lcs, sizeof(int32_t) * (size_t)(nint + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->ldeg, sizeof(uint16_t) * (size_t)(nint + 1)));
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int32_t), ctx->stream));
    for (int k = 0; k < 8; k++) {
        if (t->M[k] == 0) continue;
        k_local_structure<<<grid_for(t->M[k], 256), 256, 0, ctx->stream>>>(t->root[k], t->child_off[k], t->M[k], k,
                                                                           t->roots_d, t->lcs, t->ldeg, ctx->errflag);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    int32_t ef = 0;
    PASUR_CUDA(ctx, cudaMemcpyAsync(&ef, ctx->errflag, sizeof ef, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ef) return set_err(ctx, PASUR_EOVERFLOW, "a node has more than 65535 legal moves");

    // plan the work items
    int threads = cfg->threads > 0 ? cfg->threads : 256;
    if (threads > 256 || threads % 32) return set_err(ctx, PASUR_EINVAL, "cfg.threads must be a multiple of 32 <= 256");
    size_t budget = std::min<size_t>(ctx->smem_optin, 110 * 1024);
    int wcap = cfg->slots_per_item > 0 ? cfg->slots_per_item : 64;
    t->items_h.clear();
    int64_t data = 0, scratch = 0;
    size_t smem_need = 0;
    for (int64_t g = 0; g < t->n_roots; g++) {
        const RootInfo &ri = t->roots_h[(size_t)g];
        int64_t Sg = t->score_off_h[(size_t)g + 1] - t->score_off_h[(size_t)g];
        int64_t N = ri.local_start[9], Nint = ri.n_internal;
        if (Sg == 0 || N == 0) continue;
        int64_t w = std::min<int64_t>(Sg, wcap);
        while (w > 1 && resident_bytes(N, Nint, w) > budget) w--;
        bool res = resident_bytes(N, Nint, w) <= budget;
        if (!res) w = std::min<int64_t>(Sg, 32);
        for (int64_t s0 = 0; s0 < Sg; s0 += w) {
            CfrItem it{};
            it.root = (int32_t)g;
            it.ns = (int32_t)std::min<int64_t>(w, Sg - s0);
            it.s0 = s0;
            it.data_base = data;
            data += N * it.ns;
            if (res) {
                it.scratch_base = -1;
                smem_need = std::max(smem_need, resident_bytes(N, Nint, it.ns));
            } else {
                it.scratch_base = scratch;
                scratch += N * it.ns;
            }
            it.cost = N * it.ns;
            t->items_h.push_back(it);
        }
    }
    std::stable_sort(t->items_h.begin(), t->items_h.end(), [](const CfrItem &a, const CfrItem &b) { return a.cost > b.cost; });
    t->n_items = (int64_t)t->items_h.size();
    t->data_size = data;
    t->scratch_size = scratch;
    t->cfr_smem = smem_need;
    t->cfr_threads = threads;
    if (t->n_items) {
        PASUR_TRY(tree_alloc(t, (void **)&t->items_d, sizeof(CfrItem) * (size_t)t->n_items));
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->items_d, t->items_h.data(), sizeof(CfrItem) * (size_t)t->n_items,
                                        cudaMemcpyHostToDevice, ctx->stream));
    }
    PASUR_TRY(tree_alloc(t, (void **)&t->R, sizeof(float) * (size_t)(data + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->S, sizeof(float) * (size_t)(data + 1)));
    PASUR_CUDA(ctx, cudaMemsetAsync(t->R, 0, sizeof(float) * (size_t)(data + 1), ctx->stream));
    PASUR_CUDA(ctx, cudaMemsetAsync(t->S, 0, sizeof(float) * (size_t)(data + 1), ctx->stream));
    if (scratch) {
        PASUR_TRY(tree_alloc(t, (void **)&t->V, sizeof(float) * (size_t)scratch));
        PASUR_TRY(tree_alloc(t, (void **)&t->P0, sizeof(float) * (size_t)scratch));
        PASUR_TRY(tree_alloc(t, (void **)&t->P1, sizeof(float) * (size_t)scratch));
    }
    PASUR_TRY(tree_alloc(t, (void **)&t->uacc, sizeof(double) * (size_t)(t->Q[0] + 1)));
    PASUR_CUDA(ctx, cudaMemsetAsync(t->uacc, 0, sizeof(double) * (size_t)(t->Q[0] + 1), ctx->stream));
    // persistent grid
    int per_sm = 0;
    if (t->cfr_smem > 0) {
        PASUR_CUDA(ctx, cudaFuncSetAttribute(k_cfr_items<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->cfr_smem));
        PASUR_CUDA(ctx, cudaFuncSetAttribute(k_cfr_items<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->cfr_smem));
    }
    PASUR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cfr_items<0>, threads, t->cfr_smem));
    if (per_sm < 1) return set_err(ctx, PASUR_EINVAL, "CFR kernel cannot be resident with this shared-memory plan");
    int64_t blocks = (int64_t)per_sm * ctx->num_sms;
    t->cfr_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, t->n_items));
    t->iters_done = 0;
    t->cfr_ready = true;
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

int cfr_run(pasur_tree *t, const pasur_config *cfg) {
    pasur_ctx *ctx = t->ctx;
    if (cfg->iters <= 0 || t->n_items == 0) {
        t->last_ms = 0.f;
        t->last_launches = 0;
        return PASUR_OK;
    }
    float *dcfr = nullptr;
    size_t db = 0;
    if (cfg->variant == 1) {
        std::vector<float> f(3 * (size_t)cfg->iters);
        for (int i = 0; i < cfg->iters; i++) {
            double tt = (double)(t->iters_done + i + 1), tp = tt - 1.0;
            double pa = std::pow(tp, (double)cfg->dcfr_alpha), pb = std::pow(tp, (double)cfg->dcfr_beta);
            f[3 * i] = (float)(pa / (pa + 1.0));
            f[3 * i + 1] = (float)(pb / (pb + 1.0));
            f[3 * i + 2] = (float)(tt > 1.0 ? std::pow(1.0 - 1.0 / tt, (double)cfg->dcfr_gamma) : 0.0);
        }
        db = f.size() * sizeof(float);
        PASUR_TRY(dev_alloc(ctx, (void **)&dcfr, db));
        PASUR_CUDA(ctx, cudaMemcpyAsync(dcfr, f.data(), db, cudaMemcpyHostToDevice, ctx->stream));
    }
    CfrParams p{};
    p.items = t->items_d;
    p.n_items = t->n_items;
    p.roots = t->roots_d;
    p.lcs = t->lcs;
    p.ldeg = t->ldeg;
    p.leaf_v = t->leaf_v;
    p.fgt_off8 = t->fgt_off[8];
    p.fgt_off0 = t->fgt_off[0];
    p.R = t->R;
    p.S = t->S;
    p.V = t->V;
    p.P0 = t->P0;
    p.P1 = t->P1;
    p.uacc = t->uacc;
    p.dcfr = dcfr;
    p.iters = cfg->iters;
    p.t0 = t->iters_done;
    p.tau_umax = cfg->rm_deadzone * t->umax;
    p.counter = ctx->counter;
    p.err = ctx->errflag;
    cudaEvent_t e0, e1;
    PASUR_CUDA(ctx, cudaEventCreate(&e0));
    PASUR_CUDA(ctx, cudaEventCreate(&e1));
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->counter, 0, sizeof(int32_t), ctx->stream));
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int32_t), ctx->stream));
    PASUR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    if (cfg->variant == 1)
        k_cfr_items<1><<<t->cfr_blocks, t->cfr_threads, t->cfr_smem, ctx->stream>>>(p);
    else
        k_cfr_items<0><<<t->cfr_blocks, t->cfr_threads, t->cfr_smem, ctx->stream>>>(p);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    PASUR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    int32_t ef = 0;
    PASUR_CUDA(ctx, cudaMemcpyAsync(&ef, ctx->errflag, sizeof ef, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    PASUR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (dcfr) dev_free(ctx, dcfr, db);
    t->last_ms = ms;
    t->last_launches = 1;
    t->iters_done += cfg->iters;
    if (ef) return set_err(ctx, PASUR_ENUMERIC, "non-finite root value in the CFR sweep");
    return PASUR_OK;
}

int cfr_export_sigma(const pasur_tree *t, float *out_dev) {
    pasur_ctx *ctx = t->ctx;
    LevelPtrs lp{};
    int64_t base = 0;
    for (int k = 0; k < 9; k++) {
        lp.p[k] = t->fgt_off[k];
        lp.base[k] = k >= 1 ? base : 0;
        if (k >= 1) base += t->Q[k];
    }
    if (t->n_items) {
        unsigned g = (unsigned)std::min<int64_t>(t->n_items, 65535);
        k_export_sigma<<<g, 256, 0, ctx->stream>>>(t->items_d, t->n_items, t->roots_d, t->lcs, t->ldeg, t->S, lp, out_dev);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    return PASUR_OK;
}

int cfr_export_utilities(const pasur_tree *t, float *out_dev) {
    pasur_ctx *ctx = t->ctx;
    if (t->Q[0] == 0) return PASUR_OK;
    double inv = t->iters_done > 0 ? 1.0 / (double)t->iters_done : 0.0;
    k_export_util<<<grid_for(t->Q[0], 256), 256, 0, ctx->stream>>>(t->uacc, t->Q[0], inv, out_dev);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    return PASUR_OK;
}

}  // namespace pasur

// CFR over an unfolded round (section "CFR Algorithm"; eq. RM, eq. avsigma; DCFR eqs.
// DFCR_REG / DFCR_AVG).
//
// Round roots are independent (open hands: every FGT node is its own information set and root
// reach is 1), so the round is cut into work items: one GT root and a run of W of its score
// slots.  A persistent grid takes items from a queue (largest first).  One thread block runs all
// T iterations of an item: per iteration a top-down pass over levels 0..6 (regret matching and
// reach) and a bottom-up pass over levels 7..0 (values, regret and strategy-sum updates), with a
// block barrier between levels; an (active node, slot) pair belongs to one thread in each pass,
// so the updates of a node's child edges need no atomics.
//
// Forced-move chains are resolved once: a node whose whole subtree is one path of single moves
// has sigma = 1 and zero regret on every edge below it and the value of its one leaf, so only the
// "active" nodes (a local node that is not such a chain) are swept, and state is kept only for
// local nodes (the root and the children of active nodes).  The item's regrets R, strategy sums
// S, values V and reaches live in shared memory for all T iterations (no DRAM traffic per
// iteration).  A root whose state does not fit one block is split over a thread-block cluster
// (distributed shared memory) or, beyond a cluster, swept level by level over every SM with its
// state in device memory.  Item layout: local node index times slots, slot-minor; the local nodes
// of each level are numbered in the order of their parents' entries, so the children of
// consecutive entries are consecutive.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <string>
#include <thread>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

// shared-memory classes of the resident items: budget per block (several blocks per SM), then
// the global-memory fallback.  Class 0 is sized for six 128-thread blocks per SM (228 KB per SM,
// 1 KB reserved per block, under 0.4 KB of static shared memory; six is also the register limit
// at 80 registers): on the full game it measured 2 % faster than 40 KB at five blocks per SM.
constexpr int kNumCls = 6;
constexpr size_t kClsBudget[kNumCls - 1] = {37536, 54 * 1024, 74 * 1024, 112 * 1024, 0 /* opt-in max */};
constexpr int kClsGlobal = kNumCls - 1;
constexpr int kClsCluster = 6;       // plan class of the cluster items' pseudo-items (exports only)
constexpr int kMaxClusterCtas = 16;  // CTAs of a cluster (16: non-portable size)
// default block size per class (the batch autotuner measures its own); class 3 at two 256-thread
// blocks per SM measured faster than one 512-thread block of the 512-thread instantiation; class 4
// (one block per SM) at 512 threads: more warps to cover the level steps' latency than at 256
// (seed-47 CFR 1234 -> 1175 ms) and fewer idle at the barriers than at 1024
constexpr int kClsThreads[kNumCls] = {128, 128, 256, 256, 512, 1024};

struct CfrParams {
    const CfrItem *items;
    int64_t i_begin, i_end;
    const TreeView *views;
    const float *dcfr;  // per iteration: regret factor if R > 0, if R <= 0, strategy-sum factor
    int iters;
    int64_t t0;
    float tau;  // dead zone: a regret counts as positive above tau * t * Umax(root)
    int32_t *counter;
    int32_t *err;
};

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// shared memory of a resident item: packed active entries (8 B each) and R, S, V, X per
// (local node, slot); resident items must have fewer than 65535 local nodes
__host__ __device__ __forceinline__ size_t resident_bytes(int64_t L, int64_t nA, int64_t W) {
    return L >= 65535 ? ~(size_t)0 >> 1 : 2 * al16((size_t)nA * 4) + 4 * al16((size_t)L * W * 4);
}

constexpr int kMaxSlots = 32;  // score slots per work item
// a root too large for one block is streamed (class 5) rather than split over a cluster when it
// has at least this many score slots
constexpr int64_t kStreamMinSlots = 16;

// Index of child edge a of a node whose first child is local node c, at slot w of an item of
// 2^sh slots (slot-minor layout; every item's slot count is a power of two); W1: single-slot
// items, where this is c + a.
template <bool W1>
__device__ __forceinline__ int at(int c, int a, int sh, int w) {
    return W1 ? c + a : ((c + a) << sh) + w;
}

// Pairwise sum of D values (a short dependency chain: about log2(D) additions deep).
template <int D>
__device__ __forceinline__ float tree_sum(const float *x) {
    if (D == 1) return x[0];
    if (D == 2) return x[0] + x[1];
    constexpr int H = D / 2;
    return tree_sum<H>(x) + tree_sum<D - H>(x + H);
}

// 1 / s for a positive regret sum: the fast reciprocal (at most 2 ulp; the sum is a normal
// number, since counted regrets exceed the dead zone).
__device__ __forceinline__ float rcp_pos(float s) { return __fdividef(1.f, s); }

// Regret matching over the regrets r of D > 1 child edges: the children's reaches own * sigma.
template <int D>
__device__ __forceinline__ void rm_reach(const float *r, float own, float thr, float *x) {
    float rp[D];
#pragma unroll
    for (int a = 0; a < D; a++) rp[a] = r[a] > thr ? r[a] : 0.f;
    const float sum = tree_sum<D>(rp);
    const bool pos = sum > 0.f;
    // pos: rp * scale (an fma with a zero addend rounds the product alone); otherwise every rp is
    // zero and the fma gives the uniform share: one instruction per child instead of two
    const float scale = pos ? own * rcp_pos(sum) : 0.f, u = pos ? 0.f : own * (1.f / (float)D);
#pragma unroll
    for (int a = 0; a < D; a++) x[a] = __fmaf_rn(rp[a], scale, u);
}

// Regret matching at one (active node, slot) with D children and the reach of the children.
// X[n] holds the reach of the player who moved into node n; own = the mover's reach at the node.
template <int D, bool W1>
__device__ __forceinline__ void td_node(int c, int sh, int w, float own, const float *__restrict__ R, float *__restrict__ X,
                                        float thr) {
    if constexpr (D == 1) {
        X[at<W1>(c, 0, sh, w)] = own;
        return;
    } else {
        float r[D], x[D];
#pragma unroll
        for (int a = 0; a < D; a++) r[a] = R[at<W1>(c, a, sh, w)];
        rm_reach<D>(r, own, thr, x);
#pragma unroll
        for (int a = 0; a < D; a++) X[at<W1>(c, a, sh, w)] = x[a];
    }
}

template <bool W1>
__device__ __forceinline__ void td_node_any(int c, int d, int sh, int w, float own, const float *__restrict__ R,
                                            float *__restrict__ X, float thr) {
    float sum = 0.f;
    for (int a = 0; a < d; a++) {
        const float r = R[at<W1>(c, a, sh, w)];
        sum += r > thr ? r : 0.f;
    }
    if (sum > 0.f) {
        const float inv = rcp_pos(sum);
        for (int a = 0; a < d; a++) {
            const float r = R[at<W1>(c, a, sh, w)];
            X[at<W1>(c, a, sh, w)] = r > thr ? own * (r * inv) : 0.f;
        }
    } else {
        const float u = own * (1.f / (float)d);
        for (int a = 0; a < d; a++) X[at<W1>(c, a, sh, w)] = u;
    }
}

// Value of a node from the regrets r, strategy sums s and values v of its D child edges, then
// R(h,a) += s_p pi_{-p}(h) (v(h.a) - v(h)) and S(h,a) += pi_p(h) sigma(h,a) in place in r and s.
// Returns v(h).
template <int VARIANT, int D>
__device__ __forceinline__ float bu_vals(float *r, const float *v, float *s, float pp, float spo, float thr, float fpos,
                                         float fneg, float fs) {
    float rp[D];
#pragma unroll
    for (int a = 0; a < D; a++) rp[a] = r[a] > thr ? r[a] : 0.f;
    const float sum = tree_sum<D>(rp);
    const bool pos = sum > 0.f;
    const float inv = pos ? rcp_pos(sum) : 0.f, u = pos ? 0.f : 1.f / (float)D;
    float sg[D], dv[D];
#pragma unroll
    for (int a = 0; a < D; a++) {
        sg[a] = __fmaf_rn(rp[a], inv, u);  // rp * inv, or the uniform share (as in td_node)
        dv[a] = a == 0 ? 0.f : sg[a] * (v[a] - v[0]);
    }
    const float vh = D == 1 ? v[0] : v[0] + tree_sum<D>(dv);
#pragma unroll
    for (int a = 0; a < D; a++) {
        const float inst = spo * (v[a] - vh);
        if (VARIANT == 1) {
            r[a] = r[a] * (r[a] > 0.f ? fpos : fneg) + inst;
            s[a] = s[a] * fs + pp * sg[a];
        } else {
            r[a] = r[a] + inst;
            s[a] = s[a] + pp * sg[a];
        }
    }
    return vh;
}

// Value of one (active node, slot) with D children and the updates of its child edges (bu_vals)
// in R and S.  Returns v(h).
template <int VARIANT, int D, bool W1>
__device__ __forceinline__ float bu_node(int c, int sh, int w, float pp, float spo, float *__restrict__ R,
                                         float *__restrict__ S, const float *__restrict__ V, float thr, float fpos,
                                         float fneg, float fs) {
    float r[D], v[D], s[D];
#pragma unroll
    for (int a = 0; a < D; a++) {
        const int q = at<W1>(c, a, sh, w);
        r[a] = R[q];
        v[a] = V[q];
        s[a] = S[q];
    }
    const float vh = bu_vals<VARIANT, D>(r, v, s, pp, spo, thr, fpos, fneg, fs);
#pragma unroll
    for (int a = 0; a < D; a++) {
        const int q = at<W1>(c, a, sh, w);
        R[q] = r[a];
        S[q] = s[a];
    }
    return vh;
}

template <int VARIANT, bool W1>
__device__ __forceinline__ float bu_node_any(int c, int d, int sh, int w, float pp, float spo, float *__restrict__ R,
                                             float *__restrict__ S, const float *__restrict__ V, float thr, float fpos,
                                             float fneg, float fs) {
    float sum = 0.f;
    for (int a = 0; a < d; a++) {
        const float r = R[at<W1>(c, a, sh, w)];
        sum += r > thr ? r : 0.f;
    }
    const float inv = sum > 0.f ? rcp_pos(sum) : 0.f, u = 1.f / (float)d;
    const float v0 = V[at<W1>(c, 0, sh, w)];
    float vh = v0;
    for (int a = 1; a < d; a++) {
        const float r = R[at<W1>(c, a, sh, w)];
        vh += (sum > 0.f ? (r > thr ? r * inv : 0.f) : u) * (V[at<W1>(c, a, sh, w)] - v0);
    }
    for (int a = 0; a < d; a++) {
        const int q = at<W1>(c, a, sh, w);
        const float r = R[q];
        const float sg = sum > 0.f ? (r > thr ? r * inv : 0.f) : u;
        const float inst = spo * (V[q] - vh);
        if (VARIANT == 1) {
            R[q] = r * (r > 0.f ? fpos : fneg) + inst;
            S[q] = S[q] * fs + pp * sg;
        } else {
            R[q] = r + inst;
            S[q] = S[q] + pp * sg;
        }
    }
    return vh;
}

// Active entries of an item.  Resident items keep them packed in shared memory, two 32-bit words
// per entry: (first child | moves << 16) and (local index | parent's local index << 16, 0xFFFF
// at the root); resident items have fewer than 65535 local nodes.  Items in device memory read
// the four int arrays.
template <bool PACKED>
struct Entries {
    const uint32_t *cd, *lp;
    const int32_t *li, *pl, *cs;
    const uint16_t *d;
    __device__ __forceinline__ void child(int e, int &c, int &n) const {
        if (PACKED) {
            const uint32_t u = cd[e];
            c = (int)(u & 0xFFFFu);
            n = (int)(u >> 16);
        } else {
            c = cs[e];
            n = d[e];
        }
    }
    __device__ __forceinline__ void self(int e, int &l, int &p) const {
        if (PACKED) {
            const uint32_t u = lp[e];
            l = (int)(u & 0xFFFFu);
            p = (u >> 16) == 0xFFFFu ? -1 : (int)(u >> 16);
        } else {
            l = li[e];
            p = pl[e];
        }
    }
};

// One level of the top-down pass over (active node, slot) pairs.  The active entries of a level
// are sorted by degree, so the lanes of a warp mostly take the same unrolled path.
template <int VARIANT, bool W1, bool PACKED>
__device__ __forceinline__ void td_level(int b, int n, int W, int sh, int t0x, int stride, const Entries<PACKED> &A,
                                         const float *__restrict__ R, float *__restrict__ X, const float *tu, float tf) {
    const float thr1 = tu[0] * tf;
    for (int x = t0x; x < n; x += stride) {
        const int e = W1 ? b + x : b + (x >> sh), w = W1 ? 0 : x & (W - 1);
        int c, d, li, pl;
        A.child(e, c, d);
        A.self(e, li, pl);
        const float thr = W1 ? thr1 : tu[w] * tf;
        const float own = pl < 0 ? 1.f : X[W1 ? pl : (pl << sh) + w];
        switch (d) {
            case 1: td_node<1, W1>(c, sh, w, own, R, X, thr); break;
            case 2: td_node<2, W1>(c, sh, w, own, R, X, thr); break;
            case 3: td_node<3, W1>(c, sh, w, own, R, X, thr); break;
            case 4: td_node<4, W1>(c, sh, w, own, R, X, thr); break;
            case 5: td_node<5, W1>(c, sh, w, own, R, X, thr); break;
            case 6: td_node<6, W1>(c, sh, w, own, R, X, thr); break;
            case 7: td_node<7, W1>(c, sh, w, own, R, X, thr); break;
            case 8: td_node<8, W1>(c, sh, w, own, R, X, thr); break;
            default: td_node_any<W1>(c, d, sh, w, own, R, X, thr);
        }
    }
}

// One level of the bottom-up pass over (active node, slot) pairs.
template <int VARIANT, bool W1, bool PACKED>
__device__ __forceinline__ void bu_level(bool alex, int b, int n, int W, int sh, int t0x, int stride,
                                         const Entries<PACKED> &A,
                                         float *__restrict__ R, float *__restrict__ S, float *__restrict__ V,
                                         const float *__restrict__ X, const float *tu, float tf, float fpos, float fneg,
                                         float fs) {
    const float thr1 = tu[0] * tf;
    for (int x = t0x; x < n; x += stride) {
        const int e = W1 ? b + x : b + (x >> sh), w = W1 ? 0 : x & (W - 1);
        int c, d, li, pl;
        A.child(e, c, d);
        A.self(e, li, pl);
        const float thr = W1 ? thr1 : tu[w] * tf;
        const float pp = pl < 0 ? 1.f : X[W1 ? pl : (pl << sh) + w];  // pi_p(h)
        const float po = X[W1 ? li : (li << sh) + w];                 // pi_{-p}(h)
        const float spo = alex ? po : -po;
        float vh;
        switch (d) {
            case 1: vh = bu_node<VARIANT, 1, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 2: vh = bu_node<VARIANT, 2, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 3: vh = bu_node<VARIANT, 3, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 4: vh = bu_node<VARIANT, 4, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 5: vh = bu_node<VARIANT, 5, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 6: vh = bu_node<VARIANT, 6, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 7: vh = bu_node<VARIANT, 7, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 8: vh = bu_node<VARIANT, 8, W1>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            default: vh = bu_node_any<VARIANT, W1>(c, d, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs);
        }
        V[W1 ? li : (li << sh) + w] = vh;
    }
}

// Level steps i0..i1-1 of a level schedule: sched[i] for i < 7 the top-down levels 0..6, for
// i >= 7 the bottom-up levels 7..0; each (first entry, pairs, flags: 1 = empty, 2 = at most 32
// pairs (warp 0 alone), 4 = the next non-empty level of the same pass is also small (a warp
// barrier suffices)).
template <int VARIANT, bool W1, bool PACKED>
__device__ __forceinline__ void run_passes(int i0, int i1, int W, int sh, const Entries<PACKED> &A, float *R, float *S,
                                           float *V, float *X, const int32_t *sb, const int32_t *sn, const int32_t *sf,
                                           const float *s_tu, float tf, float fpos, float fneg, float fs) {
    const int tid = threadIdx.x, nth = blockDim.x;
    const bool warp0 = tid < 32;
    for (int i = i0; i < i1; i++) {
        const int f = sf[i];
        if (f & 1) continue;
        if (i < 7) {
            if (!(f & 2)) td_level<VARIANT, W1, PACKED>(sb[i], sn[i], W, sh, tid, nth, A, R, X, s_tu, tf);
            else if (warp0) td_level<VARIANT, W1, PACKED>(sb[i], sn[i], W, sh, tid, 32, A, R, X, s_tu, tf);
        } else {
            const bool alex = ((14 - i) & 1) == 0;
            if (!(f & 2)) bu_level<VARIANT, W1, PACKED>(alex, sb[i], sn[i], W, sh, tid, nth, A, R, S, V, X, s_tu, tf, fpos, fneg, fs);
            else if (warp0) bu_level<VARIANT, W1, PACKED>(alex, sb[i], sn[i], W, sh, tid, 32, A, R, S, V, X, s_tu, tf, fpos, fneg, fs);
        }
        if (f & 4) __syncwarp();
        else __syncthreads();
    }
}

// The level schedule of an entry layout with level starts as[0..9] and W slots (thread 0).
__device__ __forceinline__ void make_schedule(const int32_t *as, int W, int32_t *sb, int32_t *sn, int32_t *sf) {
    for (int i = 0; i < 15; i++) {
        const int k = i < 7 ? i : 14 - i;
        sb[i] = as[k];
        sn[i] = (as[k + 1] - as[k]) * W;
    }
    for (int i = 0; i < 15; i++) {
        int f = sn[i] == 0 ? 1 : 0;
        const bool small = sn[i] <= 32;
        if (small) f |= 2;
        const int end = i < 7 ? 7 : 15;
        int j = i + 1;
        while (j < end && sn[j] == 0) j++;
        if (small && j < end && sn[j] <= 32) f |= 4;
        sf[i] = f;
    }
}

template <int VARIANT>
__device__ __forceinline__ void dcfr_factors(const CfrParams &p, int il, float &fpos, float &fneg, float &fs) {
    fpos = fneg = fs = 0.f;
    if (VARIANT == 1) {
        fpos = p.dcfr[3 * il];
        fneg = p.dcfr[3 * il + 1];
        fs = p.dcfr[3 * il + 2];
    }
}

// The T iterations of one item over its level schedule.
template <int VARIANT, bool W1, bool PACKED>
__device__ __forceinline__ double iterate(const CfrParams &p, int W, const Entries<PACKED> &A, float *R, float *S,
                                          float *V, float *X, const int32_t *sb, const int32_t *sn, const int32_t *sf,
                                          const float *s_tu) {
    const int tid = threadIdx.x;
    const int sh = __ffs(W) - 1;  // W is a power of two
    double acc = 0.0;
    for (int il = 0; il < p.iters; il++) {
        const float tf = (float)(p.t0 + il + 1);
        float fpos, fneg, fs;
        dcfr_factors<VARIANT>(p, il, fpos, fneg, fs);
        run_passes<VARIANT, W1, PACKED>(0, 15, W, sh, A, R, S, V, X, sb, sn, sf, s_tu, tf, fpos, fneg, fs);
        // the root values were written before the last step's block barrier and are next
        // written by the last step of the next iteration
        if (tid < W) acc += (double)V[tid];
    }
    __syncthreads();
    return acc;
}

// All T iterations of one item, its arrays in shared memory (carved from sm): the packed active
// entries, then R, S, V, X per (local node, slot).
template <int VARIANT>
__device__ __forceinline__ void run_item(const CfrParams &p, const TreeView &tv, const CfrItem &it, const CfrRoot &cr,
                                         const int32_t *s_as, float *s_tu, int32_t *sb, int32_t *sn, int32_t *sf,
                                         unsigned char *sm) {
    const int tid = threadIdx.x, nth = blockDim.x;
    const int W = it.ns;
    const int L = cr.ls[9], nA = s_as[9];
    const int32_t *gli = tv.act_li + cr.act_off, *gpl = tv.act_pl + cr.act_off, *gcs = tv.act_cs + cr.act_off;
    const uint16_t *gd = tv.act_d + cr.act_off;
    Entries<true> P{};
    size_t o = 0;
    uint32_t *scd = (uint32_t *)(sm + o); o += al16((size_t)nA * 4);
    uint32_t *slp = (uint32_t *)(sm + o); o += al16((size_t)nA * 4);
    float *R = (float *)(sm + o); o += al16((size_t)L * W * 4);
    float *S = (float *)(sm + o); o += al16((size_t)L * W * 4);
    float *V = (float *)(sm + o); o += al16((size_t)L * W * 4);
    float *X = (float *)(sm + o);
    for (int i = tid; i < nA; i += nth) {
        scd[i] = (uint32_t)gcs[i] | ((uint32_t)gd[i] << 16);
        slp[i] = (uint32_t)gli[i] | ((uint32_t)(gpl[i] < 0 ? 0xFFFF : gpl[i]) << 16);
    }
    {
        const float *gR = tv.R + it.data_base, *gS = tv.S + it.data_base;
        for (int i = tid; i < L * W; i += nth) {
            R[i] = gR[i];
            S[i] = gS[i];
        }
    }
    P.cd = scd;
    P.lp = slp;
    // values of the terminals (leaves and chain heads), constant over the iterations; root reach;
    // per slot the largest |leaf value| of the root's subtree, the scale of the dead zone
    for (int w = tid; w < W; w += nth) s_tu[w] = 0.f;
    __syncthreads();
    {
        const int64_t *tq = tv.loc_tq + cr.loc_off;
        for (int x = tid; x < L * W; x += nth) {
            const int li = x / W, w = x - li * W;
            const int64_t q = tq[li];
            if (q >= 0) {
                const float v = tv.leaf_v[q + it.s0 + w];
                V[x] = v;
                atomicMax((unsigned *)&s_tu[w], __float_as_uint(fabsf(v)));
            }
        }
        for (int w = tid; w < W; w += nth) X[w] = 1.f;
    }
    // level schedule: a level of at most 32 (node, slot) pairs runs on warp 0 alone, and only a
    // change between warp-0 and whole-block levels needs a block barrier
    if (tid == 0) make_schedule(s_as, W, sb, sn, sf);
    __syncthreads();
    for (int w = tid; w < W; w += nth) s_tu[w] = p.tau * s_tu[w];
    __syncthreads();
    const double acc = W == 1 ? iterate<VARIANT, true, true>(p, W, P, R, S, V, X, sb, sn, sf, s_tu)
                              : iterate<VARIANT, false, true>(p, W, P, R, S, V, X, sb, sn, sf, s_tu);
    if (tid < W) {
        if (!isfinite(acc)) atomicOr(p.err, 1);
        tv.uacc[tv.fgt_off0[it.root] + it.s0 + tid] += acc;
    }
    float *gR = tv.R + it.data_base, *gS = tv.S + it.data_base;
    for (int i = tid; i < L * W; i += nth) {
        gR[i] = R[i];
        gS[i] = S[i];
    }
    __syncthreads();
}

template <int VARIANT, int MAXT, int MINB = (MAXT == 256 ? 3 : 1)>
__global__ void __launch_bounds__(MAXT, MINB) k_cfr_items(CfrParams p) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int32_t s_item;
    __shared__ int32_t s_as[10];
    __shared__ int32_t s_sb[15], s_sn[15], s_sf[15];
    __shared__ float s_tu[kMaxSlots];
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t id = p.i_begin + s_item;
        if (tid < 10) s_as[tid] = id < p.i_end ? p.views[p.items[id].tree].roots[p.items[id].root].as[tid] : 0;
        __syncthreads();
        if (id >= p.i_end) break;
        const CfrItem it = p.items[id];
        const TreeView tv = p.views[it.tree];
        const CfrRoot &cr = tv.roots[it.root];
        run_item<VARIANT>(p, tv, it, cr, s_as, s_tu, s_sb, s_sn, s_sf, sm);
    }
}

// ---- class 5: a level-streaming sweep over every SM --------------------------------------------
//
// Items whose state lives in device memory are not given one block each: every level step of an
// iteration is one launch over the (entry, slot) pairs of that level of all such items of the
// plan, spread over the whole grid (the launch boundary is the level barrier).  A pair runs the
// same node code as in a block, so the results are the block sweep's bit for bit.

struct StreamPlan {
    const int64_t *pairs;  // [8][n + 1] exclusive prefix of (entry, slot) pairs per level
    const int64_t *locs;   // [n + 1] of (local node, slot) pairs
    const int64_t *slots;  // [n + 1] of slots
    uint32_t *tu;          // per slot: largest |terminal value| (float bits)
    double *acc;           // per slot: sum of the root values of the current call
    int64_t n;
    const StreamDesc *desc;  // [n] per item
};

// j with pre[j] <= x < pre[j + 1] (pre[0] = 0 <= x < pre[n])
__device__ __forceinline__ int64_t stream_item(const int64_t *pre, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (pre[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// the prefixes and descriptors of a plan's class-5 items (one thread; once per plan)
__global__ void k_stream_plan(const CfrItem *items, int64_t n, const TreeView *views, int64_t *pairs, int64_t *locs,
                              const int64_t *slots, StreamDesc *desc) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t pk[8] = {0}, pl = 0;
    for (int64_t j = 0; j < n; j++) {
        const CfrItem it = items[j];
        const TreeView &tv = views[it.tree];
        const CfrRoot &cr = tv.roots[it.root];
        for (int k = 0; k < 8; k++) {
            pairs[(int64_t)k * (n + 1) + j] = pk[k];
            pk[k] += (int64_t)(cr.as[k + 1] - cr.as[k]) * it.ns;
        }
        locs[j] = pl;
        pl += (int64_t)cr.ls[9] * it.ns;
        StreamDesc sd;
        sd.R = tv.R + it.data_base;
        sd.S = tv.S + it.data_base;
        sd.V = tv.V + it.scratch_base;
        sd.X = tv.X + it.scratch_base;
        sd.li = tv.act_li + cr.act_off;
        sd.pl = tv.act_pl + cr.act_off;
        sd.cs = tv.act_cs + cr.act_off;
        sd.d = tv.act_d + cr.act_off;
        for (int k = 0; k < 9; k++) sd.as[k] = cr.as[k];
        sd.ns = it.ns;
        sd.sh = __ffs(it.ns) - 1;
        sd.slot = slots[j];
        desc[j] = sd;
    }
    for (int k = 0; k < 8; k++) pairs[(int64_t)k * (n + 1) + n] = pk[k];
    locs[n] = pl;
}

// terminal values and the dead-zone scale per slot, root reach 1, sums cleared
__global__ void k_stream_setup(CfrParams p, StreamPlan sp) {
    const int64_t total = sp.locs[sp.n];
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = stream_item(sp.locs, sp.n, x);
        const CfrItem it = p.items[j];
        const TreeView &tv = p.views[it.tree];
        const CfrRoot &cr = tv.roots[it.root];
        const int sh = __ffs(it.ns) - 1;
        const int64_t r = x - sp.locs[j];
        const int li = (int)(r >> sh), w = (int)(r & (it.ns - 1));
        float *V = tv.V + it.scratch_base, *X = tv.X + it.scratch_base;
        const int64_t q = tv.loc_tq[cr.loc_off + li];
        if (q >= 0) {
            const float v = tv.leaf_v[q + it.s0 + w];
            V[r] = v;
            atomicMax(&sp.tu[sp.slots[j] + w], __float_as_uint(fabsf(v)));
        }
        if (li == 0) {
            X[w] = 1.f;
            sp.acc[sp.slots[j] + w] = 0.0;
        }
    }
}

// One (entry, slot) pair of level k of a streamed item: the block sweep's node code on the item's
// arrays in device memory.
template <int VARIANT, bool TD>
__device__ __forceinline__ void stream_pair(const StreamDesc &sd, int k, int64_t r, const StreamPlan &sp, float tau,
                                            float tf, bool alex, float fpos, float fneg, float fs) {
    const int sh = sd.sh;
    const int e = sd.as[k] + (int)(r >> sh), w = (int)(r & (sd.ns - 1));
    const int c = sd.cs[e], d = sd.d[e], li = sd.li[e], pl = sd.pl[e];
    float *R = sd.R, *S = sd.S, *V = sd.V, *X = sd.X;
    // the dead zone rounded as in the block sweep: (tau * Umax) * t
    const float thr = (tau * __uint_as_float(sp.tu[sd.slot + w])) * tf;
    if (TD) {
        const float own = pl < 0 ? 1.f : X[(pl << sh) + w];
        switch (d) {
            case 1: td_node<1, false>(c, sh, w, own, R, X, thr); break;
            case 2: td_node<2, false>(c, sh, w, own, R, X, thr); break;
            case 3: td_node<3, false>(c, sh, w, own, R, X, thr); break;
            case 4: td_node<4, false>(c, sh, w, own, R, X, thr); break;
            case 5: td_node<5, false>(c, sh, w, own, R, X, thr); break;
            case 6: td_node<6, false>(c, sh, w, own, R, X, thr); break;
            case 7: td_node<7, false>(c, sh, w, own, R, X, thr); break;
            case 8: td_node<8, false>(c, sh, w, own, R, X, thr); break;
            default: td_node_any<false>(c, d, sh, w, own, R, X, thr);
        }
    } else {
        const float pp = pl < 0 ? 1.f : X[(pl << sh) + w];
        const float po = X[(li << sh) + w];
        const float spo = alex ? po : -po;
        float vh;
        switch (d) {
            case 1: vh = bu_node<VARIANT, 1, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 2: vh = bu_node<VARIANT, 2, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 3: vh = bu_node<VARIANT, 3, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 4: vh = bu_node<VARIANT, 4, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 5: vh = bu_node<VARIANT, 5, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 6: vh = bu_node<VARIANT, 6, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 7: vh = bu_node<VARIANT, 7, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            case 8: vh = bu_node<VARIANT, 8, false>(c, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs); break;
            default: vh = bu_node_any<VARIANT, false>(c, d, sh, w, pp, spo, R, S, V, thr, fpos, fneg, fs);
        }
        V[(li << sh) + w] = vh;
        if (k == 0) sp.acc[sd.slot + w] += (double)vh;  // the root (one entry per item)
    }
}

constexpr int kStreamThreads = 256;

// One level step (level k; top-down or bottom-up) of iteration il of every class-5 item: a
// grid-stride loop over the level's (entry, slot) pairs of all items (consecutive threads on
// consecutive slots and entries); each pair finds its item by a binary search over the level's
// prefix (a few cached loads) and reads what it needs from the item's descriptor.
template <int VARIANT, bool TD>
__global__ void __launch_bounds__(kStreamThreads, TD ? 4 : 3) k_stream_level(CfrParams p, StreamPlan sp, int k, int il) {
    const int64_t *pre = sp.pairs + (int64_t)k * (sp.n + 1);
    const int64_t total = pre[sp.n];
    const float tf = (float)(p.t0 + il + 1);
    float fpos, fneg, fs;
    dcfr_factors<VARIANT>(p, il, fpos, fneg, fs);
    const bool alex = (k & 1) == 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = stream_item(pre, sp.n, x);
        stream_pair<VARIANT, TD>(sp.desc[j], k, x - pre[j], sp, p.tau, tf, alex, fpos, fneg, fs);
    }
}

// the call's root values into the running sums (a root without moves keeps its terminal value)
__global__ void k_stream_finalize(CfrParams p, StreamPlan sp) {
    const int64_t total = sp.slots[sp.n];
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = stream_item(sp.slots, sp.n, x);
        const CfrItem it = p.items[j];
        const TreeView &tv = p.views[it.tree];
        const CfrRoot &cr = tv.roots[it.root];
        const int w = (int)(x - sp.slots[j]);
        double acc = sp.acc[x];
        if (cr.as[1] == cr.as[0]) {
            const float v = tv.V[it.scratch_base + w];
            acc = 0.0;
            for (int il = 0; il < p.iters; il++) acc += (double)v;
        }
        if (!isfinite(acc)) atomicOr(p.err, 1);
        tv.uacc[tv.fgt_off0[it.root] + it.s0 + w] += acc;
    }
}

// The instantiation for blocks of `threads` threads of size class c: up to 256 threads at up to 80
// registers (three 256-thread blocks per SM), class 3 (two blocks per SM by its shared memory) at
// up to 128 (96 used: seed-47 CFR 1111 -> 1087 ms against 80), up to 512 at up to 128 (no spills),
// up to 1024 at 64 (the register file of one SM).
const void *cfr_kernel_for(int variant, int threads, int cls) {
    if (threads <= 256 && cls == 3) return variant == 1 ? (const void *)k_cfr_items<1, 256, 2> : (const void *)k_cfr_items<0, 256, 2>;
    if (threads <= 256) return variant == 1 ? (const void *)k_cfr_items<1, 256> : (const void *)k_cfr_items<0, 256>;
    if (threads <= 512) return variant == 1 ? (const void *)k_cfr_items<1, 512> : (const void *)k_cfr_items<0, 512>;
    return variant == 1 ? (const void *)k_cfr_items<1, 1024> : (const void *)k_cfr_items<0, 1024>;
}

// ---- a root subtree split over a thread-block cluster ------------------------------------------
//
// CTA r of the cluster holds part r (subtrees of active level-ell nodes) in its shared memory;
// CTA 0 also holds the top levels 0..ell-1.  Per iteration: CTA 0 runs the top-down pass of the
// top and pushes, for every active level-ell node, its reach and its parent's reach into the
// owning CTA's shared memory (distributed shared memory); cluster barrier; every CTA runs both
// passes over its part and pushes the node values back to CTA 0; cluster barrier; CTA 0 runs the
// bottom-up pass of the top.  Every task does the same arithmetic as in a single block.

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// all threads of all CTAs of the cluster; shared::cluster writes before it are visible after it
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// address of the same shared-memory byte in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_st(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ float cl_ld(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// byte offsets of a resident single-slot region (entries cd, lp, then R, S, V, X)
struct RegionOffsets {
    uint32_t lp, R, S, V, X, end;
};
__host__ __device__ __forceinline__ RegionOffsets region_offsets(int64_t L, int64_t nA) {
    RegionOffsets o;
    o.lp = (uint32_t)al16((size_t)nA * 4);
    o.R = o.lp + (uint32_t)al16((size_t)nA * 4);
    o.S = o.R + (uint32_t)al16((size_t)L * 4);
    o.V = o.S + (uint32_t)al16((size_t)L * 4);
    o.X = o.V + (uint32_t)al16((size_t)L * 4);
    o.end = o.X + (uint32_t)al16((size_t)L * 4);
    return o;
}

// load a single-slot region (packed entries, R, S; terminal values into V) and return the largest
// |terminal value|
__device__ __forceinline__ float load_region(const TreeView &tv, const CfrRoot &cr, int64_t data_base, int64_t slot,
                                             unsigned char *base, Entries<true> &E, float *&R, float *&S, float *&V,
                                             float *&X) {
    const int tid = threadIdx.x, nth = blockDim.x;
    const int L = cr.ls[9], nA = cr.as[9];
    const RegionOffsets o = region_offsets(L, nA);
    uint32_t *cd = (uint32_t *)base, *lp = (uint32_t *)(base + o.lp);
    R = (float *)(base + o.R);
    S = (float *)(base + o.S);
    V = (float *)(base + o.V);
    X = (float *)(base + o.X);
    const int32_t *gli = tv.act_li + cr.act_off, *gpl = tv.act_pl + cr.act_off, *gcs = tv.act_cs + cr.act_off;
    const uint16_t *gd = tv.act_d + cr.act_off;
    for (int i = tid; i < nA; i += nth) {
        cd[i] = (uint32_t)gcs[i] | ((uint32_t)gd[i] << 16);
        lp[i] = (uint32_t)gli[i] | ((uint32_t)(gpl[i] < 0 ? 0xFFFF : gpl[i]) << 16);
    }
    const float *gR = tv.R + data_base, *gS = tv.S + data_base;
    const int64_t *tq = tv.loc_tq + cr.loc_off;
    float umax = 0.f;
    for (int i = tid; i < L; i += nth) {
        R[i] = gR[i];
        S[i] = gS[i];
        const int64_t q = tq[i];
        if (q >= 0) {
            const float v = tv.leaf_v[q + slot];
            V[i] = v;
            umax = fmaxf(umax, fabsf(v));
        }
    }
    E.cd = cd;
    E.lp = lp;
    return umax;
}

__device__ __forceinline__ void store_region(const TreeView &tv, const CfrRoot &cr, int64_t data_base, const float *R,
                                             const float *S) {
    const int L = cr.ls[9];
    float *gR = tv.R + data_base, *gS = tv.S + data_base;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        gR[i] = R[i];
        gS[i] = S[i];
    }
}

template <int VARIANT, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT == 256 ? 3 : 1) k_cfr_cluster(CfrParams p, const ClusterItem *__restrict__ clu) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int32_t s_as[10], t_as[10];
    __shared__ int32_t s_sb[15], s_sn[15], s_sf[15], t_sb[15], t_sn[15], t_sf[15];
    __shared__ float s_tu[1];
    __shared__ unsigned s_umax;
    __shared__ float s_qmax[kMaxClusterCtas];
    __shared__ uint32_t s_xoff[kMaxClusterCtas];
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t q = cl_rank(), nq = cl_count();
    const ClusterItem c = clu[cl_id()];
    const TreeView tv = p.views[c.tree];
    const bool has_part = (int)q < c.nparts;
    const ClusterPart top = tv.cparts[c.part0];
    const ClusterPart part0 = tv.cparts[c.part0 + 1];
    const CfrRoot &tr = tv.roots[top.root];
    const CfrRoot &pr0 = tv.roots[part0.root];
    // CTA 0: part 0 at offset 0, the top right after it
    const uint32_t top_base = region_offsets(pr0.ls[9], pr0.as[9]).end;
    const uint32_t top_v = top_base + region_offsets(tr.ls[9], tr.as[9]).V;
    Entries<true> PE{}, TE{};
    float *PR = nullptr, *PS = nullptr, *PV = nullptr, *PX = nullptr;
    float *TR = nullptr, *TS = nullptr, *TV = nullptr, *TX = nullptr;
    if (tid == 0) s_umax = 0u;
    if (tid < (int)nq && q == 0) {
        const int r = tid;
        if (r < c.nparts) {
            const CfrRoot &prr = tv.roots[tv.cparts[c.part0 + 1 + r].root];
            s_xoff[r] = region_offsets(prr.ls[9], prr.as[9]).X;
        } else {
            s_xoff[r] = 0;
        }
    }
    __syncthreads();
    float um = 0.f;
    const ClusterPart mine = has_part ? tv.cparts[c.part0 + 1 + q] : part0;
    const CfrRoot &pr = tv.roots[mine.root];
    if (has_part) um = load_region(tv, pr, mine.data_base, c.s0, sm, PE, PR, PS, PV, PX);
    if (q == 0) um = fmaxf(um, load_region(tv, tr, top.data_base, c.s0, sm + top_base, TE, TR, TS, TV, TX));
    atomicMax(&s_umax, __float_as_uint(um));
    if (tid < 10) {
        s_as[tid] = has_part ? pr.as[tid] : 0;
        t_as[tid] = tr.as[tid];
    }
    __syncthreads();
    if (q == 0 && tid == 0) TX[0] = 1.f;  // root reach
    if (tid == 0) {
        make_schedule(s_as, 1, s_sb, s_sn, s_sf);
        make_schedule(t_as, 1, t_sb, t_sn, t_sf);
        cl_st(cl_map(&s_qmax[q], 0), __uint_as_float(s_umax));
    }
    cl_sync();
    if (tid == 0) {
        float m = 0.f;
        for (uint32_t r = 0; r < nq; r++) m = fmaxf(m, cl_ld(cl_map(&s_qmax[r], 0)));
        s_tu[0] = p.tau * m;
    }
    __syncthreads();
    const int32_t *cx = tv.cx + 5 * c.x0;
    double acc = 0.0;
    for (int il = 0; il < p.iters; il++) {
        const float tf = (float)(p.t0 + il + 1);
        float fpos, fneg, fs;
        dcfr_factors<VARIANT>(p, il, fpos, fneg, fs);
        if (q == 0) {
            run_passes<VARIANT, true, true>(0, 7, 1, 0, TE, TR, TS, TV, TX, t_sb, t_sn, t_sf, s_tu, tf, fpos, fneg, fs);
            // reaches of the active level-ell nodes and of their parents, into their owners
            for (int j = tid; j < c.nx; j += nth) {
                const int32_t *e = cx + 5 * j;
                const uint32_t r = (uint32_t)e[0];
                unsigned char *xb = sm + s_xoff[r];
                cl_st(cl_map(xb + 4 * e[3], r), TX[e[1]]);
                cl_st(cl_map(xb + 4 * e[4], r), TX[e[2]]);
            }
        }
        cl_sync();
        if (has_part) {
            run_passes<VARIANT, true, true>(0, 15, 1, 0, PE, PR, PS, PV, PX, s_sb, s_sn, s_sf, s_tu, tf, fpos, fneg, fs);
            // values of my active level-ell nodes, into the top
            for (int j = tid; j < c.nx; j += nth) {
                const int32_t *e = cx + 5 * j;
                if ((uint32_t)e[0] == q) cl_st(cl_map(sm + top_v + 4 * e[1], 0), PV[e[3]]);
            }
        }
        cl_sync();
        if (q == 0) {
            run_passes<VARIANT, true, true>(7, 15, 1, 0, TE, TR, TS, TV, TX, t_sb, t_sn, t_sf, s_tu, tf, fpos, fneg, fs);
            if (tid == 0) acc += (double)TV[0];
        }
    }
    if (has_part) store_region(tv, pr, mine.data_base, PR, PS);
    if (q == 0) {
        store_region(tv, tr, top.data_base, TR, TS);
        if (tid == 0) {
            if (!isfinite(acc)) atomicOr(p.err, 1);
            tv.uacc[tv.fgt_off0[c.root] + c.s0] += acc;
        }
    }
    cl_sync();  // no CTA leaves while another may still address its shared memory
}

// The cluster kernel for blocks of `threads` threads: up to 256 at up to 80 registers, up to 512 at
// up to 128 (no spills), beyond that at up to 64 (a 1024-thread block on one SM).
const void *const kClusterKernels[6] = {(const void *)k_cfr_cluster<0, 256>,  (const void *)k_cfr_cluster<1, 256>,
                                        (const void *)k_cfr_cluster<0, 512>,  (const void *)k_cfr_cluster<1, 512>,
                                        (const void *)k_cfr_cluster<0, 1024>, (const void *)k_cfr_cluster<1, 1024>};
const void *cluster_kernel_for(int variant, int threads) {
    return kClusterKernels[(threads > 512 ? 4 : threads > 256 ? 2 : 0) + (variant == 1)];
}

struct LevelPtrs {
    const int64_t *fgt[9];
    const int64_t *child[9];
    int64_t base[9];  // offset of level k in the concatenated edge output (levels 1..8)
};

__global__ void k_fill(float *out, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) out[i] = v;
}

// average strategy of the child edges of every active node, canonical FGT order, one block per
// item (every other edge lies below a forced move and has average strategy 1)
__global__ void k_export_sigma(const CfrItem *items, int64_t n_items, const CfrRoot *roots, const int32_t *act_cs,
                               const uint16_t *act_d, const int64_t *act_gt, const float *Sg, LevelPtrs lp, float *out) {
    for (int64_t id = blockIdx.x; id < n_items; id += gridDim.x) {
        const CfrItem it = items[id];
        const CfrRoot &cr = roots[it.root];
        const int W = it.ns;
        const float *S = Sg + it.data_base;
        for (int k = 0; k < 8; k++) {
            const int b = cr.as[k], n = (cr.as[k + 1] - b) * W;
            for (int x = threadIdx.x; x < n; x += blockDim.x) {
                const int e = b + x / W, w = x % W;
                const int c = act_cs[cr.act_off + e], d = act_d[cr.act_off + e];
                const int64_t j = act_gt[cr.act_off + e];
                float sum = 0.f;
                for (int a = 0; a < d; a++) sum += S[(c + a) * W + w];
                const int64_t c0 = lp.child[k][j];
                for (int a = 0; a < d; a++) {
                    float sb = sum > 0.f ? S[(c + a) * W + w] / sum : 1.f / (float)d;
                    out[lp.base[k + 1] + lp.fgt[k + 1][c0 + a] + it.s0 + w] = sb;
                }
            }
        }
    }
}

__global__ void k_export_util(const double *uacc, const int64_t *cidx0, int64_t n, double inv_t, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(uacc[cidx0[i]] * inv_t);
}

// One level of sum_e m_e (a_e - b_e)^2 over the solved edges e of the level (m_e: full slots that
// solved slot stands for), one warp per GT node, lanes over its solved slots; block sums in f64
// added to *acc.
__global__ void k_sigma_sqdiff(const int32_t *__restrict__ root, int64_t m, const int64_t *__restrict__ cfgt_off,
                               const int64_t *__restrict__ csoff, const int32_t *__restrict__ cmult,
                               const float *__restrict__ a, const float *__restrict__ b, double *acc) {
    __shared__ double part[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    double sum = 0.0;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < m; j += nw) {
        const int32_t g = root[j];
        const int64_t c0 = cfgt_off[j], ns = cfgt_off[j + 1] - c0, w0 = csoff[g];
        for (int64_t x = lane; x < ns; x += 32) {
            const double d = (double)a[c0 + x] - (double)b[c0 + x];
            sum += (double)cmult[w0 + x] * d * d;
        }
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
    if (lane == 0) part[wid] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += part[i];
        atomicAdd(acc, s);
    }
}

// One level of the average strategies of every full slot from those of the solved slots: one warp
// per GT node j, lanes over its full slots (consecutive output addresses); full slot s of root g
// reads solved slot cidx0[score_off[g] + s] - csoff[g] of the same node.
__global__ void k_expand_edges(const int32_t *__restrict__ root, int64_t m, const int64_t *__restrict__ fgt_off,
                               const int64_t *__restrict__ cfgt_off, const int64_t *__restrict__ score_off,
                               const int64_t *__restrict__ csoff, const int64_t *__restrict__ cidx0,
                               const float *__restrict__ in, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < m; j += nw) {
        const int32_t g = root[j];
        const int64_t q0 = fgt_off[j], ns = fgt_off[j + 1] - q0, c0 = cfgt_off[j] - csoff[g], s0 = score_off[g];
        for (int64_t s = lane; s < ns; s += 32) out[q0 + s] = in[c0 + cidx0[s0 + s]];
    }
}

// chain[j] = 1 when the subtree of j is one path of forced moves (leaves included)
__global__ void k_chain(const int64_t *child_off, int64_t m, const uint8_t *chain_next, uint8_t *chain) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t c0 = child_off[j];
        chain[j] = (child_off[j + 1] - c0 == 1 && chain_next[c0]) ? 1 : 0;
    }
}

// local and active flags of level k from level k-1 (local: the root, or the parent is active;
// active: local, not a chain, not a leaf)
__global__ void k_flags(const int64_t *parent, int64_t m, const int32_t *active_prev, const uint8_t *chain, bool leaves,
                        int32_t *local, int32_t *active) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t l = parent ? active_prev[parent[j]] : 1;
        local[j] = l;
        active[j] = (l && !leaves && !chain[j]) ? 1 : 0;
    }
}

struct RankPtrs {
    const int64_t *loc[9];
    const int64_t *act[9];
};

// per root and level: global local-rank and active-rank at the root's first node
__global__ void k_root_ranks(const int64_t *bounds, int64_t n_roots, RankPtrs rp, int64_t *out) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= n_roots; g += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 9; k++) {
            int64_t b = bounds[g * 9 + k];
            out[g * 18 + k] = rp.loc[k][b];
            out[g * 18 + 9 + k] = rp.act[k][b];
        }
}

struct ChildPtrs {
    const int64_t *p[9];
};

__global__ void k_fill_layout(int k, int64_t m, const int32_t *root, const int32_t *local, const int32_t *active,
                              const int64_t *loc_rank, const int64_t *act_rank, const int64_t *loc_rank_next,
                              const int64_t *loc_rank_prev, const int64_t *parent, ChildPtrs co, const int64_t *fgt_off8,
                              const CfrRoot *roots, int64_t *loc_tq, int32_t *act_li, int32_t *act_pl, int32_t *act_cs,
                              uint16_t *act_d, int64_t *act_gt, uint64_t *act_key, int32_t *act_rk, int32_t *err) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        if (!local[j]) continue;
        const CfrRoot &cr = roots[root[j]];
        const int64_t li = cr.ls[k] + (loc_rank[j] - cr.locbase[k]);
        if (active[j]) {
            loc_tq[cr.loc_off + li] = -1;
            const int64_t e = cr.as[k] + (act_rank[j] - cr.actbase[k]);
            const int64_t c0 = co.p[k][j], d = co.p[k][j + 1] - c0;
            if (d > 65535) atomicOr(err, 2);
            act_li[cr.act_off + e] = (int32_t)li;
            act_pl[cr.act_off + e] =
                k == 0 ? -1 : (int32_t)(cr.ls[k - 1] + (loc_rank_prev[parent[j]] - cr.locbase[k - 1]));
            act_cs[cr.act_off + e] = (int32_t)(cr.ls[k + 1] + (loc_rank_next[c0] - cr.locbase[k + 1]));
            act_d[cr.act_off + e] = (uint16_t)d;
            act_gt[cr.act_off + e] = j;
            // sort key: the (root, level) segment, then degree descending
            act_key[cr.act_off + e] = ((uint64_t)(cr.act_off + cr.as[k]) << 16) | (uint64_t)(0xFFFF - (d > 0xFFFF ? 0xFFFF : d));
            act_rk[cr.act_off + e] = (root[j] << 3) | k;
        } else {
            int64_t x = j;
            for (int kk = k; kk < 8; kk++) x = co.p[kk][x];  // follow the forced moves to the leaf
            loc_tq[cr.loc_off + li] = fgt_off8[x];
        }
    }
}

__global__ void k_widen_degrees(const uint16_t *d, int64_t n, int32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) out[i] = d[i];
}

// pos: exclusive scan of the degrees over the sorted entries.  The children of the entries of
// root g at level k, in entry order, are the local nodes of level k+1 of that root: child a of
// entry e becomes local node ls[k+1] + (pos[e] - pos[first entry of (g, k)]) + a.  lmap[old
// global local index] = new global local index.
__global__ void k_renumber_map(int64_t n, const int32_t *act_rk, const CfrRoot *roots, const int64_t *pos,
                               const int32_t *act_cs, const uint16_t *act_d, int64_t *lmap) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = act_rk[e] >> 3, k = act_rk[e] & 7;
        const CfrRoot &cr = roots[g];
        const int64_t first = cr.ls[k + 1] + (pos[e] - pos[cr.act_off + cr.as[k]]);
        const int d = act_d[e];
        for (int a = 0; a < d; a++) lmap[cr.loc_off + act_cs[e] + a] = cr.loc_off + first + a;
    }
}

__global__ void k_renumber_roots(int64_t nr, const CfrRoot *roots, int64_t *lmap) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nr; g += (int64_t)gridDim.x * blockDim.x)
        if (roots[g].ls[9] > 0) lmap[roots[g].loc_off] = roots[g].loc_off;
}

__global__ void k_renumber_apply(int64_t n, const int32_t *act_rk, const CfrRoot *roots, const int64_t *pos, const int64_t *lmap,
                                 int32_t *act_li, int32_t *act_pl, int32_t *act_cs) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = act_rk[e] >> 3, k = act_rk[e] & 7;
        const CfrRoot &cr = roots[g];
        act_li[e] = (int32_t)(lmap[cr.loc_off + act_li[e]] - cr.loc_off);
        if (act_pl[e] >= 0) act_pl[e] = (int32_t)(lmap[cr.loc_off + act_pl[e]] - cr.loc_off);
        act_cs[e] = (int32_t)(cr.ls[k + 1] + (pos[e] - pos[cr.act_off + cr.as[k]]));
    }
}

__global__ void k_renumber_tq(int64_t n, const int64_t *lmap, const int64_t *tq_old, int64_t *tq) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        tq[lmap[x]] = tq_old[x];
}

__global__ void k_iota(int64_t *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) out[i] = i;
}

template <typename T>
__global__ void k_gather(const T *in, const int64_t *perm, int64_t n, T *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) out[i] = in[perm[i]];
}

unsigned grid_for(int64_t threads, int block) {
    int64_t b = (threads + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

// Several device temporaries carved from one allocation (pieces 256-byte aligned, n + 1 elements
// each): one allocator call instead of one per array.
struct Slab {
    size_t total = 0;
    std::vector<std::pair<void **, size_t>> want;
    template <typename T>
    void add(T **p, int64_t n) {
        want.push_back({(void **)p, total});
        total += (sizeof(T) * (size_t)(n + 1) + 255) & ~(size_t)255;
    }
    int alloc(pasur_ctx *ctx, std::vector<std::pair<void *, size_t>> &tmp) {
        char *base = nullptr;
        PASUR_TRY(dev_alloc(ctx, (void **)&base, total));
        tmp.push_back({(void *)base, total});
        for (auto &w : want) *w.first = base + w.second;
        return PASUR_OK;
    }
};

int build_layout(pasur_tree *t) {
    pasur_ctx *ctx = t->ctx;
    std::vector<std::pair<void *, size_t>> tmp;
    struct Guard {
        pasur_ctx *c;
        std::vector<std::pair<void *, size_t>> *v;
        ~Guard() {
            for (auto &x : *v) dev_free(c, x.first, x.second);
        }
    } guard{ctx, &tmp};
    uint8_t *chain[9];
    int32_t *local[9], *active[9];
    int64_t *lrank[9], *arank[9];
    int64_t *ranks = nullptr;
    const int64_t nr = t->n_roots;
    {
        Slab sl;
        for (int k = 0; k < 9; k++) {
            sl.add(&chain[k], t->M[k]);
            sl.add(&local[k], t->M[k]);
            sl.add(&active[k], t->M[k]);
            sl.add(&lrank[k], t->M[k]);
            sl.add(&arank[k], t->M[k]);
        }
        sl.add(&ranks, 18 * (nr + 1));
        PASUR_TRY(sl.alloc(ctx, tmp));
    }
    PASUR_CUDA(ctx, cudaMemsetAsync(chain[8], 1, (size_t)t->M[8] + 1, ctx->stream));
    for (int k = 7; k >= 0; k--) {
        if (t->M[k] == 0) continue;
        k_chain<<<grid_for(t->M[k], 256), 256, 0, ctx->stream>>>(t->child_off[k], t->M[k], chain[k + 1], chain[k]);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    for (int k = 0; k < 9; k++) {
        if (t->M[k] > 0) {
            k_flags<<<grid_for(t->M[k], 256), 256, 0, ctx->stream>>>(k ? t->parent[k] : nullptr, t->M[k],
                                                                    k ? active[k - 1] : nullptr, chain[k], k == 8,
                                                                    local[k], active[k]);
            ctx->launches++;
            PASUR_CUDA(ctx, cudaGetLastError());
        }
        PASUR_TRY(exclusive_scan_i32(ctx, local[k], lrank[k], t->M[k]));
        PASUR_TRY(exclusive_scan_i32(ctx, active[k], arank[k], t->M[k]));
    }
    RankPtrs rp;
    for (int k = 0; k < 9; k++) {
        rp.loc[k] = lrank[k];
        rp.act[k] = arank[k];
    }
    k_root_ranks<<<grid_for(nr + 1, 256), 256, 0, ctx->stream>>>(t->bounds_d, nr, rp, ranks);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    std::vector<int64_t> hr((size_t)18 * (nr + 1));
    PASUR_CUDA(ctx, cudaMemcpyAsync(hr.data(), ranks, sizeof(int64_t) * hr.size(), cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    t->croots_h.assign((size_t)nr, CfrRoot{});
    int64_t loc_off = 0, act_off = 0;
    for (int64_t g = 0; g < nr; g++) {
        CfrRoot &cr = t->croots_h[(size_t)g];
        const int64_t *a = &hr[(size_t)g * 18], *b = &hr[(size_t)(g + 1) * 18];
        int64_t l = 0, n = 0;
        for (int k = 0; k < 9; k++) {
            cr.locbase[k] = a[k];
            cr.actbase[k] = a[9 + k];
            cr.ls[k] = (int32_t)l;
            cr.as[k] = (int32_t)n;
            l += b[k] - a[k];
            n += b[9 + k] - a[9 + k];
        }
        if (l > INT32_MAX / 64) return set_err(ctx, PASUR_EOVERFLOW, "a root's local subtree is too large");
        cr.ls[9] = (int32_t)l;
        cr.as[9] = (int32_t)n;
        cr.loc_off = loc_off;
        cr.act_off = act_off;
        loc_off += l;
        act_off += n;
    }
    t->n_local = loc_off;
    t->n_active = act_off;
    if (nr > 0) {
        PASUR_TRY(tree_alloc(t, (void **)&t->croots_d, sizeof(CfrRoot) * (size_t)nr));
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->croots_d, t->croots_h.data(), sizeof(CfrRoot) * (size_t)nr, cudaMemcpyHostToDevice,
                                        ctx->stream));
    }
    PASUR_TRY(tree_alloc(t, (void **)&t->loc_tq, sizeof(int64_t) * (size_t)(loc_off + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->act_li, sizeof(int32_t) * (size_t)(act_off + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->act_pl, sizeof(int32_t) * (size_t)(act_off + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->act_cs, sizeof(int32_t) * (size_t)(act_off + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->act_d, sizeof(uint16_t) * (size_t)(act_off + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->act_gt, sizeof(int64_t) * (size_t)(act_off + 1)));
    uint64_t *act_key = nullptr;
    int64_t *perm = nullptr, *pos = nullptr, *lmap = nullptr;
    int32_t *t32 = nullptr, *act_rk = nullptr, *deg = nullptr;
    uint16_t *t16 = nullptr;
    int64_t *t64 = nullptr;
    {
        Slab sl;
        sl.add(&act_key, act_off);
        sl.add(&perm, act_off);
        sl.add(&t32, act_off);
        sl.add(&t16, act_off);
        sl.add(&t64, act_off);
        sl.add(&act_rk, act_off);
        sl.add(&deg, act_off);
        sl.add(&pos, act_off);
        sl.add(&lmap, loc_off);
        PASUR_TRY(sl.alloc(ctx, tmp));
    }
    ChildPtrs co;
    for (int k = 0; k < 8; k++) co.p[k] = t->child_off[k];
    co.p[8] = nullptr;
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int32_t), ctx->stream));
    for (int k = 0; k < 9; k++) {
        if (t->M[k] == 0) continue;
        k_fill_layout<<<grid_for(t->M[k], 256), 256, 0, ctx->stream>>>(
            k, t->M[k], t->root[k], local[k], active[k], lrank[k], arank[k], k < 8 ? lrank[k + 1] : nullptr,
            k > 0 ? lrank[k - 1] : nullptr, k > 0 ? t->parent[k] : nullptr, co, t->cfgt_off[8], t->croots_d, t->loc_tq,
            t->act_li, t->act_pl, t->act_cs, t->act_d, t->act_gt, act_key, act_rk, ctx->errflag);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    int32_t ef = 0;
    PASUR_CUDA(ctx, cudaMemcpyAsync(&ef, ctx->errflag, sizeof ef, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ef) return set_err(ctx, PASUR_EOVERFLOW, "a node has more than 65535 legal moves");
    // order the active entries of every (root, level) by degree, largest first, so that the lanes
    // of a warp mostly run the same unrolled path
    if (act_off > 1) {
        k_iota<<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(perm, act_off);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        int bits = 16;
        while (((int64_t)1 << (bits - 16)) <= act_off) bits++;
        PASUR_TRY(radix_sort_pairs(ctx, act_key, perm, act_off, bits));
        int32_t *arr32[3] = {t->act_li, t->act_pl, t->act_cs};
        for (int i = 0; i < 3; i++) {
            k_gather<int32_t><<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(arr32[i], perm, act_off, t32);
            ctx->launches++;
            PASUR_CUDA(ctx, cudaGetLastError());
            PASUR_CUDA(ctx, cudaMemcpyAsync(arr32[i], t32, sizeof(int32_t) * (size_t)act_off, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        k_gather<uint16_t><<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(t->act_d, perm, act_off, t16);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->act_d, t16, sizeof(uint16_t) * (size_t)act_off, cudaMemcpyDeviceToDevice, ctx->stream));
        k_gather<int64_t><<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(t->act_gt, perm, act_off, t64);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->act_gt, t64, sizeof(int64_t) * (size_t)act_off, cudaMemcpyDeviceToDevice, ctx->stream));
        k_gather<int32_t><<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(act_rk, perm, act_off, t32);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        PASUR_CUDA(ctx, cudaMemcpyAsync(act_rk, t32, sizeof(int32_t) * (size_t)act_off, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    // renumber the local nodes of every level after the first in the order of their parents'
    // entries: the children of consecutive entries become consecutive nodes (a warp's child
    // accesses fall on few shared-memory banks and few device-memory sectors).  Child a of an
    // entry stays child a, so every node's arithmetic is unchanged.
    if (act_off > 0) {
        k_widen_degrees<<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(t->act_d, act_off, deg);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        PASUR_TRY(exclusive_scan_i32(ctx, deg, pos, act_off));
        k_renumber_map<<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(act_off, act_rk, t->croots_d, pos, t->act_cs, t->act_d,
                                                                        lmap);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        k_renumber_roots<<<grid_for(nr, 256), 256, 0, ctx->stream>>>(nr, t->croots_d, lmap);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        k_renumber_apply<<<grid_for(act_off, 256), 256, 0, ctx->stream>>>(act_off, act_rk, t->croots_d, pos, lmap, t->act_li,
                                                                          t->act_pl, t->act_cs);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        // terminal leaf links follow their nodes
        int64_t *tq_old = nullptr;
        PASUR_TRY(dev_alloc(ctx, (void **)&tq_old, sizeof(int64_t) * (size_t)(loc_off + 1)));
        tmp.push_back({tq_old, sizeof(int64_t) * (size_t)(loc_off + 1)});
        PASUR_CUDA(ctx, cudaMemcpyAsync(tq_old, t->loc_tq, sizeof(int64_t) * (size_t)loc_off, cudaMemcpyDeviceToDevice, ctx->stream));
        k_renumber_tq<<<grid_for(loc_off, 256), 256, 0, ctx->stream>>>(loc_off, lmap, tq_old, t->loc_tq);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

}  // namespace

// ---- roots split over thread-block clusters ----------------------------------------------------


struct SplitRoot {
    int32_t ell = 0, nparts = 0;
    int32_t top_root = 0, part_root0 = 0;   // pseudo-root ids
    int64_t x0 = 0;
    int32_t nx = 0;
    int64_t top_L = 0;
    std::vector<int64_t> part_L;            // local nodes incl. ghosts
    size_t smem = 0;                         // largest CTA need (CTA 0: part 0 + top)
};

namespace {

// Plan the split of every root that needs a cluster: subtrees of the active level-ell nodes packed
// (in GT order) into parts that each fit one block; CTA 0 also holds the top levels.  Appends the
// pseudo-roots to croots_h, their entries and local-node leaf indices to the host vectors, and
// the exchange entries to t->cx_h.
int plan_splits(pasur_tree *t, const pasur_config *cfg, size_t dyn_max, size_t part_max, const std::vector<char> &streamed,
                std::vector<SplitRoot> &splits, std::vector<int32_t> &split_of, std::vector<int32_t> &nli,
                std::vector<int32_t> &npl, std::vector<int32_t> &ncs, std::vector<uint16_t> &nd,
                std::vector<int64_t> &ngt, std::vector<int64_t> &ntq) {
    pasur_ctx *ctx = t->ctx;
    const int64_t nr = t->n_roots;
    split_of.assign((size_t)nr, -1);
    std::vector<int64_t> cand;
    for (int64_t g = 0; g < nr; g++) {
        const CfrRoot &cr = t->croots_h[(size_t)g];
        const int64_t Sg = t->csoff_h[(size_t)g + 1] - t->csoff_h[(size_t)g];
        const int64_t L = cr.ls[9], nA = cr.as[9];
        if (Sg == 0 || L == 0 || nA < 2 || streamed[(size_t)g] || !t->in_range(g)) continue;
        const size_t need = resident_bytes(L, nA, 1);
        if (need > dyn_max || (cfg->split_bytes > 0 && need > (size_t)cfg->split_bytes)) cand.push_back(g);
    }
    if (cand.empty()) return PASUR_OK;
    PhaseTimer pt(ctx->stream, "cluster splits");
    // host copies of the layout
    const int64_t NA = t->n_active, NL = t->n_local;
    std::vector<int32_t> hli((size_t)NA), hpl((size_t)NA), hcs((size_t)NA);
    std::vector<uint16_t> hd((size_t)NA);
    std::vector<int64_t> hgt((size_t)NA), htq((size_t)NL);
    PASUR_CUDA(ctx, cudaMemcpy(hli.data(), t->act_li, sizeof(int32_t) * (size_t)NA, cudaMemcpyDeviceToHost));
    PASUR_CUDA(ctx, cudaMemcpy(hpl.data(), t->act_pl, sizeof(int32_t) * (size_t)NA, cudaMemcpyDeviceToHost));
    PASUR_CUDA(ctx, cudaMemcpy(hcs.data(), t->act_cs, sizeof(int32_t) * (size_t)NA, cudaMemcpyDeviceToHost));
    PASUR_CUDA(ctx, cudaMemcpy(hd.data(), t->act_d, sizeof(uint16_t) * (size_t)NA, cudaMemcpyDeviceToHost));
    PASUR_CUDA(ctx, cudaMemcpy(hgt.data(), t->act_gt, sizeof(int64_t) * (size_t)NA, cudaMemcpyDeviceToHost));
    PASUR_CUDA(ctx, cudaMemcpy(htq.data(), t->loc_tq, sizeof(int64_t) * (size_t)NL, cudaMemcpyDeviceToHost));
    pt.mark("host copies");
    const size_t target = cfg->split_bytes > 0 ? std::min<size_t>((size_t)cfg->split_bytes, part_max) : part_max;
    const bool verbose = getenv("PASUR_VERBOSE") != nullptr;
    // the split of one root, its pseudo-roots' offsets relative to its own entries and nodes
    struct RootSplit {
        bool done = false;
        SplitRoot sr;
        CfrRoot top{};
        std::vector<CfrRoot> parts;
        std::vector<int32_t> li, pl, cs, cx;
        std::vector<uint16_t> d;
        std::vector<int64_t> gt, tq;
        std::string msg;
    };
    auto split_one = [&](int64_t g, RootSplit &o) {
        const CfrRoot cr = t->croots_h[(size_t)g];
        const int64_t L = cr.ls[9], nA = cr.as[9];
        const int32_t *li = hli.data() + cr.act_off, *pl = hpl.data() + cr.act_off, *cs = hcs.data() + cr.act_off;
        const uint16_t *dd = hd.data() + cr.act_off;
        bool done = false;
        for (int ell = 1; ell <= 6 && !done; ell++) {
            const int32_t e0 = cr.as[ell], e1 = cr.as[ell + 1];
            if (e1 - e0 < 2) continue;
            // subtree id of every local node at levels >= ell below an active level-ell node
            std::vector<int32_t> heads;  // local indices of the active level-ell nodes, GT order
            for (int32_t e = e0; e < e1; e++) heads.push_back(li[e]);
            std::sort(heads.begin(), heads.end());
            std::vector<int32_t> sub((size_t)L, -1), ent_of((size_t)L, -1);
            for (int32_t e = 0; e < nA; e++) ent_of[(size_t)li[e]] = e;
            for (size_t i = 0; i < heads.size(); i++) sub[(size_t)heads[i]] = (int32_t)i;
            const int ns = (int)heads.size();
            std::vector<int64_t> sa((size_t)ns, 0), sl((size_t)ns, 0);
            for (int k = ell; k < 8; k++)
                for (int32_t e = cr.as[k]; e < cr.as[k + 1]; e++) {
                    const int32_t sid = sub[(size_t)li[e]];
                    if (sid < 0) continue;
                    sa[(size_t)sid]++;
                    for (int a = 0; a < dd[e]; a++) sub[(size_t)(cs[e] + a)] = sid;
                }
            for (int64_t x = cr.ls[ell]; x < L; x++)
                if (sub[(size_t)x] >= 0) sl[(size_t)sub[(size_t)x]]++;
            const size_t top_bytes = resident_bytes(cr.ls[ell + 1], cr.as[ell], 1);
            if (top_bytes >= part_max) break;
            // pack the subtrees into parts (contiguous runs), balancing active entries
            int64_t tot = 0;
            for (int i = 0; i < ns; i++) tot += sa[(size_t)i];
            // parts: the target size sets the starting count (portable clusters of up to 8 CTAs
            // first), a block's shared memory is the hard limit of every part
            const size_t need = resident_bytes(L, nA, 1);
            const int q0 = (int)std::min<size_t>(cfg->split_bytes > 0 ? kMaxClusterCtas : 8,
                                                 std::max<size_t>(2, (need + target - 1) / target));
            // contiguous parts: greedy fill with an entry cap (and the byte limit); the smallest
            // cap that needs at most Q parts, by bisection
            auto greedy = [&](int64_t cap, std::vector<int> &first) -> bool {
                first.assign(1, 0);
                int64_t pa = 0, plc = 0, pg = 0;
                for (int i = 0; i < ns; i++) {
                    const size_t lim = first.size() == 1 ? part_max - top_bytes : part_max;
                    const bool fits = resident_bytes(plc + sl[(size_t)i] + pg + 1, pa + sa[(size_t)i], 1) <= lim;
                    if (pa > 0 && (!fits || pa + sa[(size_t)i] > cap)) {
                        first.push_back(i);
                        pa = plc = pg = 0;
                    }
                    const size_t lim2 = first.size() == 1 ? part_max - top_bytes : part_max;
                    pa += sa[(size_t)i];
                    plc += sl[(size_t)i];
                    pg += 1;
                    if (resident_bytes(plc + pg, pa, 1) > lim2) return false;
                }
                return true;
            };
            int64_t amax = 0;
            for (int i = 0; i < ns; i++) amax = std::max(amax, sa[(size_t)i]);
            for (int Q = q0; Q <= kMaxClusterCtas && !done; Q++) {
                std::vector<int> first;
                int64_t lo = std::max<int64_t>(amax, (tot + Q - 1) / Q), hi = tot;
                if (!greedy(hi, first) || (int)first.size() > Q) {
                    // even unlimited entries per part need more than Q parts (byte limit)
                    if (!greedy(hi, first)) break;  // a single subtree does not fit a block
                    continue;
                }
                while (lo < hi) {
                    const int64_t mid = lo + (hi - lo) / 2;
                    if (greedy(mid, first) && (int)first.size() <= Q) hi = mid;
                    else lo = mid + 1;
                }
                if (!greedy(lo, first) || (int)first.size() > Q) continue;
                first.push_back(ns);
                const int np = (int)first.size() - 1;
                // build the parts
                SplitRoot sr;
                sr.ell = ell;
                sr.nparts = np;
                sr.top_L = cr.ls[ell + 1];
                CfrRoot top = cr;
                for (int k = ell + 1; k < 10; k++) top.as[k] = cr.as[ell];
                for (int k = ell + 2; k < 10; k++) top.ls[k] = cr.ls[ell + 1];
                top.W = 1;
                top.cls = kClsCluster;
                o.top = top;
                std::vector<int32_t> part_of_sub((size_t)ns);
                for (int q = 0; q < np; q++)
                    for (int i = first[(size_t)q]; i < first[(size_t)q + 1]; i++) part_of_sub[(size_t)i] = q;
                std::vector<int32_t> newidx((size_t)L, -1), ghost((size_t)L, -1);
                size_t smax = 0;
                for (int q = 0; q < np; q++) {
                    CfrRoot pr{};
                    int64_t n = 0;
                    for (int k = 0; k <= ell; k++) pr.ls[k] = 0;
                    for (int k = ell; k <= 8; k++) {
                        pr.ls[k] = (int32_t)n;
                        for (int64_t x = cr.ls[k]; x < cr.ls[k + 1]; x++) {
                            const int32_t sid = sub[(size_t)x];
                            if (sid >= 0 && part_of_sub[(size_t)sid] == q) newidx[(size_t)x] = (int32_t)n++;
                        }
                    }
                    for (int i = first[(size_t)q]; i < first[(size_t)q + 1]; i++) ghost[(size_t)heads[(size_t)i]] = (int32_t)n++;
                    pr.ls[9] = (int32_t)n;
                    pr.loc_off = (int64_t)o.tq.size();  // relative: placed after the other roots' parts when merged
                    pr.act_off = (int64_t)o.li.size();
                    std::vector<int64_t> tq((size_t)n, -1);
                    for (int64_t x = cr.ls[ell]; x < L; x++) {
                        const int32_t sid = sub[(size_t)x];
                        if (sid >= 0 && part_of_sub[(size_t)sid] == q) tq[(size_t)newidx[(size_t)x]] = htq[(size_t)(cr.loc_off + x)];
                    }
                    o.tq.insert(o.tq.end(), tq.begin(), tq.end());
                    int32_t m = 0;
                    for (int k = 0; k <= ell; k++) pr.as[k] = 0;
                    for (int k = ell; k < 8; k++) {
                        pr.as[k] = m;
                        for (int32_t e = cr.as[k]; e < cr.as[k + 1]; e++) {
                            const int32_t sid = sub[(size_t)li[e]];
                            if (sid < 0 || part_of_sub[(size_t)sid] != q) continue;
                            o.li.push_back(newidx[(size_t)li[e]]);
                            o.pl.push_back(k == ell ? ghost[(size_t)li[e]] : newidx[(size_t)pl[e]]);
                            o.cs.push_back(newidx[(size_t)cs[e]]);
                            o.d.push_back(dd[e]);
                            o.gt.push_back(hgt[(size_t)(cr.act_off + e)]);
                            m++;
                        }
                    }
                    pr.as[8] = pr.as[9] = m;
                    pr.W = 1;
                    pr.cls = kClsCluster;
                    o.parts.push_back(pr);
                    sr.part_L.push_back(n);
                    size_t b = resident_bytes(n, m, 1);
                    if (q == 0) b += resident_bytes(sr.top_L, cr.as[ell], 1);
                    smax = std::max(smax, b);
                }
                // exchange entries: active level-ell nodes
                for (size_t i = 0; i < heads.size(); i++) {
                    const int32_t x = heads[i];
                    const int32_t e = ent_of[(size_t)x];
                    o.cx.push_back(part_of_sub[i]);
                    o.cx.push_back(x);
                    o.cx.push_back(pl[e]);
                    o.cx.push_back(newidx[(size_t)x]);
                    o.cx.push_back(ghost[(size_t)x]);
                }
                sr.nx = (int32_t)heads.size();
                sr.smem = smax;
                o.sr = std::move(sr);
                o.done = done = true;
            }
            if (!done && verbose) {
                int64_t big = 0;
                for (int i = 0; i < ns; i++) big = std::max<int64_t>(big, (int64_t)resident_bytes(sl[(size_t)i] + 1, sa[(size_t)i], 1));
                char line[256];
                snprintf(line, sizeof line, "[pasur] root %lld (L %lld, active %lld): no split at level %d: %d subtrees, top %zu B, "
                                            "largest subtree %lld B, part limit %zu B\n",
                         (long long)g, (long long)L, (long long)nA, ell, ns, top_bytes, (long long)big, part_max);
                o.msg += line;
            }
        }
    };
    // roots are independent: split them on host threads, then append the results in root order
    std::vector<RootSplit> res(cand.size());
    std::atomic<size_t> next{0};
    std::atomic<bool> failed{false};
    auto worker = [&]() {
        try {
            for (size_t i = next++; i < cand.size(); i = next++) split_one(cand[i], res[i]);
        } catch (...) {
            failed = true;
        }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nw = std::min<size_t>({(size_t)hw, (size_t)16, cand.size()});
    auto run_workers = [&](const std::function<void()> &fn) {
        std::vector<std::thread> th;
        for (size_t w = 1; w < nw; w++) th.emplace_back(fn);
        fn();
        for (auto &x : th) x.join();
    };
    run_workers(worker);
    if (failed) return set_err(ctx, PASUR_ENOMEM, "cluster split: host allocation failed");
    pt.mark("per-root splits");
    // root order: pseudo-roots, exchange entries and the offsets of every root's entries and nodes
    std::vector<size_t> a_at(cand.size() + 1, nli.size()), l_at(cand.size() + 1, ntq.size());
    for (size_t ci = 0; ci < cand.size(); ci++) {
        RootSplit &o = res[ci];
        if (!o.msg.empty()) fputs(o.msg.c_str(), stderr);
        a_at[ci + 1] = a_at[ci] + o.li.size();
        l_at[ci + 1] = l_at[ci] + o.tq.size();
        if (!o.done) continue;
        SplitRoot sr = std::move(o.sr);
        sr.top_root = (int32_t)t->croots_h.size();
        sr.part_root0 = sr.top_root + 1;
        sr.x0 = (int64_t)t->cx_h.size() / 5;
        t->croots_h.push_back(o.top);
        for (CfrRoot pr : o.parts) {
            pr.loc_off += NL + (int64_t)l_at[ci];
            pr.act_off += NA + (int64_t)a_at[ci];
            t->croots_h.push_back(pr);
        }
        t->cx_h.insert(t->cx_h.end(), o.cx.begin(), o.cx.end());
        split_of[(size_t)cand[ci]] = (int32_t)splits.size();
        splits.push_back(std::move(sr));
    }
    // the entries and node links, copied into place by the host threads
    nli.resize(a_at.back());
    npl.resize(a_at.back());
    ncs.resize(a_at.back());
    nd.resize(a_at.back());
    ngt.resize(a_at.back());
    ntq.resize(l_at.back());
    next = 0;
    run_workers([&]() {
        for (size_t ci = next++; ci < cand.size(); ci = next++) {
            const RootSplit &o = res[ci];
            std::copy(o.li.begin(), o.li.end(), nli.begin() + (ptrdiff_t)a_at[ci]);
            std::copy(o.pl.begin(), o.pl.end(), npl.begin() + (ptrdiff_t)a_at[ci]);
            std::copy(o.cs.begin(), o.cs.end(), ncs.begin() + (ptrdiff_t)a_at[ci]);
            std::copy(o.d.begin(), o.d.end(), nd.begin() + (ptrdiff_t)a_at[ci]);
            std::copy(o.gt.begin(), o.gt.end(), ngt.begin() + (ptrdiff_t)a_at[ci]);
            std::copy(o.tq.begin(), o.tq.end(), ntq.begin() + (ptrdiff_t)l_at[ci]);
        }
    });
    pt.mark("merge");
    return PASUR_OK;
}

}  // namespace

// Largest dynamic shared memory a CFR block may request: the per-block opt-in limit minus the
// kernel's own static shared memory (largest over its instantiations).
int cfr_dyn_smem_limit(pasur_ctx *ctx, size_t *limit) {
    size_t st = 0;
    cudaFuncAttributes fa;
    PASUR_CUDA(ctx, cudaFuncGetAttributes(&fa, k_cfr_items<0, 256>));
    st = std::max(st, fa.sharedSizeBytes);
    PASUR_CUDA(ctx, cudaFuncGetAttributes(&fa, k_cfr_items<1, 256>));
    st = std::max(st, fa.sharedSizeBytes);
    PASUR_CUDA(ctx, cudaFuncGetAttributes(&fa, k_cfr_items<0, 512>));
    st = std::max(st, fa.sharedSizeBytes);
    PASUR_CUDA(ctx, cudaFuncGetAttributes(&fa, k_cfr_items<1, 512>));
    st = std::max(st, fa.sharedSizeBytes);
    PASUR_CUDA(ctx, cudaFuncGetAttributes(&fa, k_cfr_items<0, 1024>));
    st = std::max(st, fa.sharedSizeBytes);
    PASUR_CUDA(ctx, cudaFuncGetAttributes(&fa, k_cfr_items<1, 1024>));
    st = std::max(st, fa.sharedSizeBytes);
    *limit = ctx->smem_optin > st ? ctx->smem_optin - st : 0;
    return PASUR_OK;
}

int cfr_cluster_smem_limit(pasur_ctx *ctx, size_t *limit);

int cfr_setup_tree(pasur_tree *t, const pasur_config *cfg, int tree, std::vector<CfrItem> *cls_items, size_t *need,
                   std::vector<ClusterItem> *clu) {
    pasur_ctx *ctx = t->ctx;
    PhaseTimer pt(ctx->stream, "cfr plan");
    PASUR_TRY(build_layout(t));
    pt.mark("layout");
    // every root goes to the smallest shared-memory class its subtree fits with one slot; its
    // items then take as many slots as that class holds
    size_t dyn_max = 0;
    PASUR_TRY(cfr_dyn_smem_limit(ctx, &dyn_max));
    size_t budget[kNumCls - 1];
    for (int c = 0; c < kNumCls - 1; c++) budget[c] = kClsBudget[c] ? std::min<size_t>(kClsBudget[c], dyn_max) : dyn_max;
    const int wcap = cfg->slots_per_item > 0 ? std::min(cfg->slots_per_item, kMaxSlots) : kMaxSlots;
    // roots too large for one block (or above cfg->split_bytes) go to thread-block clusters
    std::vector<SplitRoot> splits;
    std::vector<int32_t> split_of, nli, npl, ncs;
    std::vector<uint16_t> nd;
    std::vector<int64_t> ngt, ntq;
    t->croots_h.resize((size_t)t->n_roots);
    t->cparts_h.clear();
    t->cx_h.clear();
    // roots streamed over every SM (class 5): those above cfg->stream_bytes, and those too large
    // for one block that have enough score slots to fill the streaming sweep's warps with
    // consecutive slots; roots that fit neither a block nor a cluster reach class 5 below too
    std::vector<char> streamed((size_t)t->n_roots, 0);
    for (int64_t g = 0; g < t->n_roots; g++) {
        const CfrRoot &cr = t->croots_h[(size_t)g];
        const int64_t Sg = t->csoff_h[(size_t)g + 1] - t->csoff_h[(size_t)g];
        const int64_t L = cr.ls[9], nA = cr.as[9];
        if (Sg == 0 || L == 0 || !t->in_range(g)) continue;
        const size_t need = resident_bytes(L, nA, 1);
        streamed[(size_t)g] = (cfg->stream_bytes > 0 && need > (size_t)cfg->stream_bytes) ||
                              (need > dyn_max && Sg >= kStreamMinSlots);
    }
    size_t dyn_cl = 0;
    PASUR_TRY(cfr_cluster_smem_limit(ctx, &dyn_cl));
    PASUR_TRY(plan_splits(t, cfg, dyn_max, std::min(dyn_max, dyn_cl), streamed, splits, split_of, nli, npl, ncs, nd, ngt,
                          ntq));
    pt.mark("cluster splits");
    int64_t data = 0, scratch = 0;
    for (int64_t g = 0; g < t->n_roots; g++) {
        CfrRoot &cr = t->croots_h[(size_t)g];
        const int64_t Sg = t->csoff_h[(size_t)g + 1] - t->csoff_h[(size_t)g];
        const int64_t L = cr.ls[9], nA = cr.as[9];
        cr.W = 0;
        cr.cls = -1;
        if (Sg == 0 || L == 0 || !t->in_range(g)) continue;
        if (split_of[(size_t)g] >= 0) {
            const SplitRoot sr = splits[(size_t)split_of[(size_t)g]];
            cr.W = 1;
            cr.cls = kClsCluster;
            for (int64_t s0 = 0; s0 < Sg; s0++) {
                ClusterItem ci{};
                ci.tree = tree;
                ci.root = (int32_t)g;
                ci.s0 = s0;
                ci.part0 = (int64_t)t->cparts_h.size();
                ci.x0 = sr.x0;
                ci.nx = sr.nx;
                ci.nparts = sr.nparts;
                ci.ell = sr.ell;
                ci.smem = (int32_t)sr.smem;
                for (int q = -1; q < sr.nparts; q++) {
                    const int32_t r = q < 0 ? sr.top_root : sr.part_root0 + q;
                    const int64_t n = q < 0 ? sr.top_L : sr.part_L[(size_t)q];
                    t->cparts_h.push_back(ClusterPart{r, 0, data});
                    CfrItem it{};
                    it.root = r;
                    it.tree = tree;
                    it.ns = 1;
                    it.s0 = s0;
                    it.data_base = data;
                    it.scratch_base = -1;
                    it.cost = std::max<int64_t>(t->croots_h[(size_t)r].as[9], 1);
                    cls_items[kClsCluster].push_back(it);
                    data += n;
                }
                clu->push_back(ci);
            }
            continue;
        }
        // slots per item: a power of two (the kernel indexes slots with shifts).  Automatic: the
        // smallest class the root fits with one slot, then the largest count that class holds.
        // With cfg.slots_per_item: that many slots (at most the root's), in the smallest class
        // that holds them, fewer where no class does.
        int64_t want = 1;
        if (cfg->slots_per_item > 0)
            while (want * 2 <= std::min<int64_t>(Sg, wcap)) want *= 2;
        int cls = kClsGlobal;
        for (; want >= 1 && cls == kClsGlobal && !streamed[(size_t)g]; want /= 2)
            for (int c = 0; c < kNumCls - 1; c++)
                if (resident_bytes(L, nA, want) <= budget[c]) {
                    cls = c;
                    break;
                }
        int64_t w = 1;
        while (w * 2 <= std::min<int64_t>(Sg, wcap) && (cls == kClsGlobal || resident_bytes(L, nA, w * 2) <= budget[cls])) w *= 2;
        cr.W = (int32_t)w;
        cr.cls = cls;
        for (int64_t s0 = 0, ns = w; s0 < Sg; s0 += ns) {
            while (ns > Sg - s0) ns /= 2;
            CfrItem it{};
            it.root = (int32_t)g;
            it.tree = tree;
            it.ns = (int32_t)ns;
            it.s0 = s0;
            it.data_base = data;
            data += L * it.ns;
            if (cls == kClsGlobal) {
                it.scratch_base = scratch;
                scratch += L * it.ns;
            } else {
                it.scratch_base = -1;
                need[cls] = std::max(need[cls], resident_bytes(L, nA, it.ns));
            }
            it.cost = std::max<int64_t>(nA, 1) * it.ns;
            int32_t wmax = 0;
            for (int k = 0; k < 8; k++) wmax = std::max<int32_t>(wmax, (cr.as[k + 1] - cr.as[k]) * it.ns);
            it.width = wmax;
            cls_items[cls].push_back(it);
        }
    }
    t->data_size = data;
    t->scratch_size = scratch;
    t->swept_edges = t->swept_pairs = 0;
    for (int64_t g = 0; g < t->n_roots; g++) {
        const CfrRoot &cr = t->croots_h[(size_t)g];
        if (cr.ls[9] > 1 && t->in_range(g)) {
            const int64_t ns = t->csoff_h[(size_t)g + 1] - t->csoff_h[(size_t)g];
            t->swept_edges += (int64_t)(cr.ls[9] - 1) * ns;
            t->swept_pairs += (int64_t)cr.as[9] * ns;
        }
    }
    if (!splits.empty()) {
        // append the parts' entries and local leaf indices; pseudo-roots after the real roots
        const int64_t NA = t->n_active, NL = t->n_local, na = (int64_t)nli.size(), nl = (int64_t)ntq.size();
        int32_t *li = nullptr, *pl = nullptr, *cs = nullptr;
        uint16_t *d = nullptr;
        int64_t *gt = nullptr, *tq = nullptr;
        PASUR_TRY(tree_alloc(t, (void **)&li, sizeof(int32_t) * (size_t)(NA + na + 1)));
        PASUR_TRY(tree_alloc(t, (void **)&pl, sizeof(int32_t) * (size_t)(NA + na + 1)));
        PASUR_TRY(tree_alloc(t, (void **)&cs, sizeof(int32_t) * (size_t)(NA + na + 1)));
        PASUR_TRY(tree_alloc(t, (void **)&d, sizeof(uint16_t) * (size_t)(NA + na + 1)));
        PASUR_TRY(tree_alloc(t, (void **)&gt, sizeof(int64_t) * (size_t)(NA + na + 1)));
        PASUR_TRY(tree_alloc(t, (void **)&tq, sizeof(int64_t) * (size_t)(NL + nl + 1)));
        auto cp = [&](void *dst, const void *old_d, size_t ob, const void *new_h, size_t nb) -> int {
            PASUR_CUDA(ctx, cudaMemcpyAsync(dst, old_d, ob, cudaMemcpyDeviceToDevice, ctx->stream));
            PASUR_CUDA(ctx, cudaMemcpyAsync((char *)dst + ob, new_h, nb, cudaMemcpyHostToDevice, ctx->stream));
            return PASUR_OK;
        };
        PASUR_TRY(cp(li, t->act_li, 4 * (size_t)NA, nli.data(), 4 * (size_t)na));
        PASUR_TRY(cp(pl, t->act_pl, 4 * (size_t)NA, npl.data(), 4 * (size_t)na));
        PASUR_TRY(cp(cs, t->act_cs, 4 * (size_t)NA, ncs.data(), 4 * (size_t)na));
        PASUR_TRY(cp(d, t->act_d, 2 * (size_t)NA, nd.data(), 2 * (size_t)na));
        PASUR_TRY(cp(gt, t->act_gt, 8 * (size_t)NA, ngt.data(), 8 * (size_t)na));
        PASUR_TRY(cp(tq, t->loc_tq, 8 * (size_t)NL, ntq.data(), 8 * (size_t)nl));
        t->act_li = li;
        t->act_pl = pl;
        t->act_cs = cs;
        t->act_d = d;
        t->act_gt = gt;
        t->loc_tq = tq;
        PASUR_TRY(tree_alloc(t, (void **)&t->croots_d, sizeof(CfrRoot) * t->croots_h.size()));
        PASUR_TRY(tree_alloc(t, (void **)&t->cparts_d, sizeof(ClusterPart) * (t->cparts_h.size() + 1)));
        PASUR_TRY(tree_alloc(t, (void **)&t->cx_d, sizeof(int32_t) * (t->cx_h.size() + 1)));
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->cparts_d, t->cparts_h.data(), sizeof(ClusterPart) * t->cparts_h.size(),
                                        cudaMemcpyHostToDevice, ctx->stream));
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->cx_d, t->cx_h.data(), sizeof(int32_t) * t->cx_h.size(), cudaMemcpyHostToDevice,
                                        ctx->stream));
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (!t->croots_h.empty())
        PASUR_CUDA(ctx, cudaMemcpyAsync(t->croots_d, t->croots_h.data(), sizeof(CfrRoot) * t->croots_h.size(),
                                        cudaMemcpyHostToDevice, ctx->stream));
    PASUR_TRY(tree_alloc(t, (void **)&t->R, sizeof(float) * (size_t)(data + 1)));
    PASUR_TRY(tree_alloc(t, (void **)&t->S, sizeof(float) * (size_t)(data + 1)));
    PASUR_CUDA(ctx, cudaMemsetAsync(t->R, 0, sizeof(float) * (size_t)(data + 1), ctx->stream));
    PASUR_CUDA(ctx, cudaMemsetAsync(t->S, 0, sizeof(float) * (size_t)(data + 1), ctx->stream));
    if (scratch) {
        PASUR_TRY(tree_alloc(t, (void **)&t->V, sizeof(float) * (size_t)scratch));
        PASUR_TRY(tree_alloc(t, (void **)&t->X, sizeof(float) * (size_t)scratch));
    }
    PASUR_TRY(tree_alloc(t, (void **)&t->uacc, sizeof(double) * (size_t)(t->cQ[0] + 1)));
    PASUR_CUDA(ctx, cudaMemsetAsync(t->uacc, 0, sizeof(double) * (size_t)(t->cQ[0] + 1), ctx->stream));
    TreeView &v = t->view;
    v.roots = t->croots_d;
    v.act_li = t->act_li;
    v.act_pl = t->act_pl;
    v.act_cs = t->act_cs;
    v.act_d = t->act_d;
    v.loc_tq = t->loc_tq;
    v.leaf_v = t->leaf_v;
    v.fgt_off0 = t->cfgt_off[0];
    v.R = t->R;
    v.S = t->S;
    v.V = t->V;
    v.X = t->X;
    v.uacc = t->uacc;
    v.cparts = t->cparts_d;
    v.cx = t->cx_d;
    t->iters_done = 0;
    t->cfr_ready = true;
    pt.mark("items and state");
    return PASUR_OK;
}

int cfr_cluster_check(pasur_ctx *ctx, CfrPlan *plan, const pasur_config *cfg);

int cfr_finalize_plan(pasur_ctx *ctx, CfrPlan &plan, std::vector<CfrItem> *cls_items, const size_t *need,
                      const std::vector<TreeView> &views, const pasur_config *cfg, std::vector<std::pair<void *, size_t>> &owned,
                      const std::vector<ClusterItem> &clu) {
    if (cfg->threads < 0 || cfg->threads > 1024 || cfg->threads % 32)
        return set_err(ctx, PASUR_EINVAL, "cfg.threads must be 0 or a multiple of 32 <= 1024");
    if (cfg->split_bytes < 0) return set_err(ctx, PASUR_EINVAL, "cfg.split_bytes must be >= 0");
    if (cfg->stream_bytes < 0) return set_err(ctx, PASUR_EINVAL, "cfg.stream_bytes must be >= 0");
    plan.items_h.clear();
    // classes 0..5 are launched by k_cfr_items; class 6 holds the cluster items' pseudo-items
    for (int c = 0; c <= kClsCluster; c++) {
        std::stable_sort(cls_items[c].begin(), cls_items[c].end(),
                         [](const CfrItem &a, const CfrItem &b) { return a.cost > b.cost; });
        plan.cls_begin[c] = (int64_t)plan.items_h.size();
        plan.items_h.insert(plan.items_h.end(), cls_items[c].begin(), cls_items[c].end());
        plan.cls_end[c] = (int64_t)plan.items_h.size();
        plan.cls_smem[c] = c < kNumCls ? need[c] : 0;
    }
    plan.n_items = (int64_t)plan.items_h.size();
    plan.clu_h = clu;
    std::stable_sort(plan.clu_h.begin(), plan.clu_h.end(),
                     [](const ClusterItem &a, const ClusterItem &b) { return a.nparts < b.nparts; });
    for (int b = 0; b < kCluGroups; b++) {
        plan.clu_begin[b] = plan.clu_end[b] = 0;
        plan.clu_smem[b] = 0;
    }
    int64_t i = 0;
    for (int b = 0; b < kCluGroups; b++) {
        plan.clu_begin[b] = i;
        while (i < (int64_t)plan.clu_h.size() && plan.clu_h[(size_t)i].nparts <= plan.clu_ctas[b]) {
            plan.clu_smem[b] = std::max(plan.clu_smem[b], (size_t)plan.clu_h[(size_t)i].smem);
            i++;
        }
        plan.clu_end[b] = i;
    }
    // one block width for the cluster launches: 512 threads, one CTA per SM (seed-47 CFR with class
    // 4 at 512: 1175 -> 1110 ms; 1024 threads measured slower than 256)
    plan.clu_threads = 512;
    if (cfg->threads > 0) plan.clu_threads = cfg->threads;
    if (!plan.clu_h.empty()) {
        size_t b = sizeof(ClusterItem) * plan.clu_h.size();
        PASUR_TRY(dev_alloc(ctx, (void **)&plan.clu_d, b));
        owned.push_back({plan.clu_d, b});
        PASUR_CUDA(ctx, cudaMemcpyAsync(plan.clu_d, plan.clu_h.data(), b, cudaMemcpyHostToDevice, ctx->stream));
        PASUR_TRY(cfr_cluster_check(ctx, &plan, cfg));
    }
    if (plan.n_items) {
        size_t b = sizeof(CfrItem) * (size_t)plan.n_items;
        PASUR_TRY(dev_alloc(ctx, (void **)&plan.items_d, b));
        owned.push_back({plan.items_d, b});
        PASUR_CUDA(ctx, cudaMemcpyAsync(plan.items_d, plan.items_h.data(), b, cudaMemcpyHostToDevice, ctx->stream));
    }
    if (!views.empty()) {
        size_t b = sizeof(TreeView) * views.size();
        PASUR_TRY(dev_alloc(ctx, (void **)&plan.views_d, b));
        owned.push_back({plan.views_d, b});
        PASUR_CUDA(ctx, cudaMemcpyAsync(plan.views_d, views.data(), b, cudaMemcpyHostToDevice, ctx->stream));
    }
    // class 5 runs as the level-streaming sweep: its prefixes, per-slot scales and sums
    plan.str_n = plan.cls_end[kClsGlobal] - plan.cls_begin[kClsGlobal];
    plan.str_nslots = 0;
    if (plan.str_n > 0) {
        const int64_t n = plan.str_n, b0 = plan.cls_begin[kClsGlobal];
        std::vector<int64_t> so((size_t)n + 1, 0);
        for (int64_t j = 0; j < n; j++) so[(size_t)j + 1] = so[(size_t)j] + plan.items_h[(size_t)(b0 + j)].ns;
        plan.str_nslots = so[(size_t)n];
        auto own = [&](void **p, size_t bytes) -> int {
            PASUR_TRY(dev_alloc(ctx, p, bytes));
            owned.push_back({*p, bytes});
            return PASUR_OK;
        };
        PASUR_TRY(own((void **)&plan.str_pairs, sizeof(int64_t) * 8 * (size_t)(n + 1)));
        PASUR_TRY(own((void **)&plan.str_locs, sizeof(int64_t) * (size_t)(n + 1)));
        PASUR_TRY(own((void **)&plan.str_slots, sizeof(int64_t) * (size_t)(n + 1)));
        PASUR_TRY(own((void **)&plan.str_tu, sizeof(uint32_t) * (size_t)plan.str_nslots));
        PASUR_TRY(own((void **)&plan.str_acc, sizeof(double) * (size_t)plan.str_nslots));
        PASUR_TRY(own((void **)&plan.str_desc, sizeof(StreamDesc) * (size_t)n));
        PASUR_CUDA(ctx, cudaMemcpyAsync(plan.str_slots, so.data(), sizeof(int64_t) * so.size(), cudaMemcpyHostToDevice,
                                        ctx->stream));
        k_stream_plan<<<1, 32, 0, ctx->stream>>>(plan.items_d + b0, n, plan.views_d, plan.str_pairs, plan.str_locs,
                                                 plan.str_slots, plan.str_desc);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (!ctx->cfr_smem_raised) {
        // the attribute is global per kernel: raise it once to the largest dynamic size any plan
        // can ask for, so that plans prepared later never lower it under an earlier plan's need
        // (static plus dynamic shared memory above 48 KB needs it)
        size_t lim = 0;
        PASUR_TRY(cfr_dyn_smem_limit(ctx, &lim));
        for (int v = 0; v < 2; v++)
            for (int t : {256, 512, 1024})
                for (int c : {0, 3})
                    PASUR_CUDA(ctx, cudaFuncSetAttribute(cfr_kernel_for(v, t, c), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
        ctx->cfr_smem_raised = true;
    }
    for (int c = 0; c < kNumCls; c++) {
        plan.cls_blocks[c] = 0;
        int64_t n = plan.cls_end[c] - plan.cls_begin[c];
        int threads = cfg->threads > 0 ? cfg->threads : kClsThreads[c];
        if (cfg->threads == 0 && n > 0 && n < ctx->num_sms) {
            // fewer items than SMs: every item has an SM to itself, so widen its block towards its
            // widest level (fewer tasks per thread per level step); beyond 256 threads the block
            // barriers cost more than the shorter level steps save (measured on GB300)
            int32_t wmax = 0;
            for (int64_t i = plan.cls_begin[c]; i < plan.cls_end[c]; i++) wmax = std::max(wmax, plan.items_h[(size_t)i].width);
            int t = 128;
            while (t < wmax && t < 256) t *= 2;
            threads = std::min(std::max(threads, t), std::max(t, 256));
            // items whose state lives in device memory wait on L2/DRAM latency at every access:
            // they take a whole SM each, so give them the widest block for latency hiding
            if (c == kClsGlobal) threads = 1024;
        }
        plan.cls_threads[c] = threads;
        if (n == 0) continue;
        int per_sm = 0;
        PASUR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cfr_kernel_for(0, threads, c), threads, plan.cls_smem[c]));
        if (per_sm < 1) return set_err(ctx, PASUR_EINVAL, "CFR kernel cannot be resident with this shared-memory plan");
        plan.cls_blocks[c] = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * ctx->num_sms, n));
    }
    return PASUR_OK;
}

int cfr_occupancy(pasur_ctx *ctx, int threads, int cls, size_t smem, int64_t n_items, int *blocks) {
    int per_sm = 0;
    PASUR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cfr_kernel_for(0, threads, cls), threads, smem));
    *blocks = per_sm < 1 ? 0 : (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * ctx->num_sms, n_items));
    return PASUR_OK;
}

int cfr_dcfr_factors(pasur_ctx *ctx, const pasur_config *cfg, int64_t t0, float **out, size_t *bytes) {
    *out = nullptr;
    *bytes = 0;
    if (cfg->variant != 1 || cfg->iters <= 0) return PASUR_OK;
    std::vector<float> f(3 * (size_t)cfg->iters);
    for (int i = 0; i < cfg->iters; i++) {
        double tt = (double)(t0 + i + 1), tp = tt - 1.0;
        double pa = std::pow(tp, (double)cfg->dcfr_alpha), pb = std::pow(tp, (double)cfg->dcfr_beta);
        f[3 * i] = (float)(pa / (pa + 1.0));
        f[3 * i + 1] = (float)(pb / (pb + 1.0));
        f[3 * i + 2] = (float)(tt > 1.0 ? std::pow(1.0 - 1.0 / tt, (double)cfg->dcfr_gamma) : 0.0);
    }
    *bytes = f.size() * sizeof(float);
    PASUR_TRY(dev_alloc(ctx, (void **)out, *bytes));
    PASUR_CUDA(ctx, cudaMemcpyAsync(*out, f.data(), *bytes, cudaMemcpyHostToDevice, ctx->stream));
    return PASUR_OK;
}

int ensure_aux(pasur_ctx *ctx) {
    if (ctx->fork) return PASUR_OK;
    PASUR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming));
    int least = 0, greatest = 0;
    PASUR_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (int c = 0; c < kClsCluster + kCluGroups; c++) {
        // the level-streaming sweep is a chain of short dependent launches: its blocks go first
        // whenever an SM frees up, the persistent classes and the clusters fill the rest
        PASUR_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->aux[c], cudaStreamNonBlocking, c == kClsGlobal ? greatest : least));
        PASUR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->join[c], cudaEventDisableTiming));
        PASUR_CUDA(ctx, cudaEventCreate(&ctx->cls_t0[c]));
        PASUR_CUDA(ctx, cudaEventCreate(&ctx->cls_t1[c]));
    }
    return PASUR_OK;
}

// All iterations of the plan's class-5 items on stream st: set-up, 15 level launches per
// iteration, the root sums into the running utilities.
int stream_sweep(pasur_ctx *ctx, const CfrPlan &plan, CfrParams p, const pasur_config *cfg, cudaStream_t st) {
    p.items = plan.items_d + plan.cls_begin[kClsGlobal];
    StreamPlan sp{plan.str_pairs, plan.str_locs, plan.str_slots, plan.str_tu, plan.str_acc, plan.str_n, plan.str_desc};
    const unsigned grid = (unsigned)ctx->num_sms * 8;
    const unsigned lgrid = (unsigned)ctx->num_sms * 4;  // the level kernels: four (bottom-up: three) blocks per SM
    PASUR_CUDA(ctx, cudaMemsetAsync(plan.str_tu, 0, sizeof(uint32_t) * (size_t)plan.str_nslots, st));
    k_stream_setup<<<grid, 256, 0, st>>>(p, sp);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    for (int il = 0; il < cfg->iters; il++)
        for (int i = 0; i < 15; i++) {
            const int k = i < 7 ? i : 14 - i;
            if (cfg->variant == 1) {
                if (i < 7) k_stream_level<1, true><<<lgrid, kStreamThreads, 0, st>>>(p, sp, k, il);
                else k_stream_level<1, false><<<lgrid, kStreamThreads, 0, st>>>(p, sp, k, il);
            } else {
                if (i < 7) k_stream_level<0, true><<<lgrid, kStreamThreads, 0, st>>>(p, sp, k, il);
                else k_stream_level<0, false><<<lgrid, kStreamThreads, 0, st>>>(p, sp, k, il);
            }
            ctx->launches++;
            PASUR_CUDA(ctx, cudaGetLastError());
        }
    k_stream_finalize<<<grid, 256, 0, st>>>(p, sp);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    return PASUR_OK;
}

int cfr_launch_plan(pasur_ctx *ctx, CfrPlan &plan, const pasur_config *cfg, int64_t t0, const float *dcfr) {
    if (cfg->iters <= 0 || plan.n_items == 0) return PASUR_OK;
    PASUR_TRY(ensure_aux(ctx));
    CfrParams p{};
    p.items = plan.items_d;
    p.views = plan.views_d;
    p.dcfr = dcfr;
    p.iters = cfg->iters;
    p.t0 = t0;
    p.tau = cfg->rm_deadzone;
    p.err = ctx->errflag;
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->counter, 0, sizeof(int32_t) * kNumCls, ctx->stream));
    PASUR_CUDA(ctx, cudaEventRecord(ctx->fork, ctx->stream));
    // the classes are independent: each runs on its own forked stream, largest subtrees first; the
    // level-streaming sweep (thousands of short launches) is queued last, after every persistent
    // class and cluster launch, so that the host never waits on its queue before the others start
    for (int oi = 0; oi < kNumCls; oi++) {
        const int c = kNumCls - 1 - oi;
        if (plan.cls_end[c] == plan.cls_begin[c] || c == kClsGlobal) continue;
        cudaStream_t st = ctx->aux[c];
        PASUR_CUDA(ctx, cudaStreamWaitEvent(st, ctx->fork, 0));
        PASUR_CUDA(ctx, cudaEventRecord(ctx->cls_t0[c], st));
        p.i_begin = plan.cls_begin[c];
        p.i_end = plan.cls_end[c];
        p.counter = ctx->counter + c;
        void *args[] = {&p};
        PASUR_CUDA(ctx, cudaLaunchKernel(cfr_kernel_for(cfg->variant, plan.cls_threads[c], c), dim3((unsigned)plan.cls_blocks[c]),
                                         dim3((unsigned)plan.cls_threads[c]), args, plan.cls_smem[c], st));
        ctx->launches++;
        PASUR_CUDA(ctx, cudaEventRecord(ctx->cls_t1[c], st));
        PASUR_CUDA(ctx, cudaEventRecord(ctx->join[c], st));
        PASUR_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->join[c], 0));
    }
    // roots split over thread-block clusters: one cluster per item, a launch (and a stream) per
    // cluster size
    for (int b = 0; b < kCluGroups; b++) {
        const int64_t n = plan.clu_end[b] - plan.clu_begin[b];
        if (n == 0) continue;
        const int c = kClsCluster + b;
        cudaStream_t st = ctx->aux[c];
        PASUR_CUDA(ctx, cudaStreamWaitEvent(st, ctx->fork, 0));
        PASUR_CUDA(ctx, cudaEventRecord(ctx->cls_t0[c], st));
        cudaLaunchConfig_t lc{};
        lc.gridDim = dim3((unsigned)(n * plan.clu_ctas[b]), 1, 1);
        lc.blockDim = dim3((unsigned)plan.clu_threads, 1, 1);
        lc.dynamicSmemBytes = plan.clu_smem[b];
        lc.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)plan.clu_ctas[b];
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        const ClusterItem *ci = plan.clu_d + plan.clu_begin[b];
        void *args[] = {&p, &ci};
        PASUR_CUDA(ctx, cudaLaunchKernelExC(&lc, cluster_kernel_for(cfg->variant, plan.clu_threads), args));
        ctx->launches++;
        PASUR_CUDA(ctx, cudaEventRecord(ctx->cls_t1[c], st));
        PASUR_CUDA(ctx, cudaEventRecord(ctx->join[c], st));
        PASUR_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->join[c], 0));
    }
    if (plan.cls_end[kClsGlobal] != plan.cls_begin[kClsGlobal]) {
        cudaStream_t st = ctx->aux[kClsGlobal];
        PASUR_CUDA(ctx, cudaStreamWaitEvent(st, ctx->fork, 0));
        PASUR_CUDA(ctx, cudaEventRecord(ctx->cls_t0[kClsGlobal], st));
        PASUR_TRY(stream_sweep(ctx, plan, p, cfg, st));
        PASUR_CUDA(ctx, cudaEventRecord(ctx->cls_t1[kClsGlobal], st));
        PASUR_CUDA(ctx, cudaEventRecord(ctx->join[kClsGlobal], st));
        PASUR_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->join[kClsGlobal], 0));
    }
    return PASUR_OK;
}

// Prepare the cluster kernel for a plan's cluster items: shared-memory and cluster-size
// attributes, and a check that one cluster of this shape can be resident.
int cfr_cluster_smem_limit(pasur_ctx *ctx, size_t *limit) {
    size_t st = 0;
    cudaFuncAttributes fa;
    for (const void *k : kClusterKernels) {
        PASUR_CUDA(ctx, cudaFuncGetAttributes(&fa, k));
        st = std::max(st, fa.sharedSizeBytes);
    }
    *limit = ctx->smem_optin > st ? ctx->smem_optin - st : 0;
    return PASUR_OK;
}

int cfr_cluster_check(pasur_ctx *ctx, CfrPlan *plan, const pasur_config *cfg) {
    size_t lim = 0;
    PASUR_TRY(cfr_cluster_smem_limit(ctx, &lim));
    for (const void *k : kClusterKernels) {
        PASUR_CUDA(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
        PASUR_CUDA(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    }
    for (int b = 0; b < kCluGroups; b++) {
        if (plan->clu_end[b] == plan->clu_begin[b]) continue;
        if (plan->clu_smem[b] > lim) return set_err(ctx, PASUR_EINVAL, "cluster part exceeds the shared memory of a block");
        cudaLaunchConfig_t lc{};
        lc.gridDim = dim3((unsigned)plan->clu_ctas[b], 1, 1);
        lc.blockDim = dim3((unsigned)plan->clu_threads, 1, 1);
        lc.dynamicSmemBytes = plan->clu_smem[b];
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)plan->clu_ctas[b];
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        int nclusters = 0;
        PASUR_CUDA(ctx, cudaOccupancyMaxActiveClusters(&nclusters, cluster_kernel_for(cfg->variant, plan->clu_threads), &lc));
        if (nclusters < 1)
            return set_err(ctx, PASUR_EINVAL, "a cluster of " + std::to_string(plan->clu_ctas[b]) + " blocks of " +
                                                  std::to_string(plan->clu_smem[b]) + " B shared memory cannot be resident");
    }
    return PASUR_OK;
}

void cfr_plan_times(pasur_ctx *ctx, CfrPlan &plan) {
    for (int c = 0; c < kNumCls; c++) {
        float m = 0.f;
        if (plan.cls_end[c] != plan.cls_begin[c]) cudaEventElapsedTime(&m, ctx->cls_t0[c], ctx->cls_t1[c]);
        plan.cls_ms[c] = m;
    }
    for (int b = 0; b < kCluGroups; b++) {
        float m = 0.f;
        if (plan.clu_end[b] != plan.clu_begin[b]) cudaEventElapsedTime(&m, ctx->cls_t0[kClsCluster + b], ctx->cls_t1[kClsCluster + b]);
        plan.cls_ms[kClsCluster + b] = m;
    }
}

static void print_plan(const pasur_tree *t, const CfrPlan &plan) {
    int64_t ne = 0;
    for (int k = 1; k < 9; k++) ne += t->Q[k];
    fprintf(stderr, "[pasur] round %d: GT roots %lld, FGT edges %lld, local %lld, active %lld, items %lld\n", t->round,
            (long long)t->n_roots, (long long)ne, (long long)t->n_local, (long long)t->n_active, (long long)plan.n_items);
    for (int c = 0; c < kNumCls; c++) {
        int64_t n = plan.cls_end[c] - plan.cls_begin[c];
        if (!n) continue;
        int64_t cost = 0, maxcost = 0, swept = 0, slots = 0;
        for (int64_t i = plan.cls_begin[c]; i < plan.cls_end[c]; i++) {
            const CfrItem &it = plan.items_h[(size_t)i];
            cost += it.cost;
            maxcost = std::max(maxcost, it.cost);
            swept += (int64_t)(t->croots_h[(size_t)it.root].ls[9] - 1) * it.ns;
            slots += it.ns;
        }
        fprintf(stderr, "[pasur]   class %d: items %lld (slots %lld), smem %zu B, blocks %d x %d threads, active-node-slots "
                        "%lld (largest item %lld), swept edges %lld\n",
                c, (long long)n, (long long)slots, plan.cls_smem[c], plan.cls_blocks[c], plan.cls_threads[c], (long long)cost,
                (long long)maxcost, (long long)swept);
    }
    for (int b = 0; b < kCluGroups; b++)
        if (plan.clu_end[b] != plan.clu_begin[b]) {
            int64_t swept = 0, lmax = 0;
            for (int64_t i = plan.clu_begin[b]; i < plan.clu_end[b]; i++) {
                const int64_t L = t->croots_h[(size_t)plan.clu_h[(size_t)i].root].ls[9];
                swept += L - 1;
                lmax = std::max(lmax, L);
            }
            fprintf(stderr, "[pasur]   cluster items: %lld, %d CTAs x %d threads, smem %zu B, swept edges %lld (largest "
                            "root %lld local nodes)\n",
                    (long long)(plan.clu_end[b] - plan.clu_begin[b]), plan.clu_ctas[b], plan.clu_threads, plan.clu_smem[b],
                    (long long)swept, (long long)lmax);
        }
}

int cfr_prepare(pasur_tree *t, const pasur_config *cfg) {
    pasur_ctx *ctx = t->ctx;
    std::vector<CfrItem> cls_items[8];
    size_t need[8] = {0};
    std::vector<ClusterItem> clu;
    PASUR_TRY(cfr_setup_tree(t, cfg, 0, cls_items, need, &clu));
    std::vector<std::pair<void *, size_t>> owned;
    int rc = cfr_finalize_plan(ctx, t->plan, cls_items, need, {t->view}, cfg, owned, clu);
    for (auto &o : owned) {
        t->allocs.push_back(o.first);
        t->allocs.push_back((void *)(uintptr_t)o.second);
    }
    if (rc != PASUR_OK) return rc;
    if (getenv("PASUR_VERBOSE")) print_plan(t, t->plan);
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

int cfr_run(pasur_tree *t, const pasur_config *cfg) {
    pasur_ctx *ctx = t->ctx;
    if (cfg->iters <= 0 || t->plan.n_items == 0) {
        t->last_ms = 0.f;
        t->last_launches = 0;
        return PASUR_OK;
    }
    float *dcfr = nullptr;
    size_t db = 0;
    PASUR_TRY(cfr_dcfr_factors(ctx, cfg, t->iters_done, &dcfr, &db));
    cudaEvent_t e0, e1;
    PASUR_CUDA(ctx, cudaEventCreate(&e0));
    PASUR_CUDA(ctx, cudaEventCreate(&e1));
    PASUR_CUDA(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int32_t), ctx->stream));
    PASUR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    const int64_t before = ctx->launches;
    int rc = cfr_launch_plan(ctx, t->plan, cfg, t->iters_done, dcfr);
    if (rc != PASUR_OK) return rc;
    PASUR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    int32_t ef = 0;
    PASUR_CUDA(ctx, cudaMemcpyAsync(&ef, ctx->errflag, sizeof ef, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    PASUR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
    cfr_plan_times(ctx, t->plan);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (dcfr) dev_free(ctx, dcfr, db);
    t->last_ms = ms;
    t->last_launches = (int32_t)(ctx->launches - before);
    t->iters_done += cfg->iters;
    if (getenv("PASUR_VERBOSE")) {
        fprintf(stderr, "[pasur] round %d: %d iterations in %.3f ms (", t->round, cfg->iters, ms);
        for (int c = 0; c < kNumCls; c++) fprintf(stderr, "%s%.2f", c ? " " : "", t->plan.cls_ms[c]);
        fprintf(stderr, " ms per class; clusters");
        for (int b = 0; b < kCluGroups; b++) fprintf(stderr, " %.2f", t->plan.cls_ms[kClsCluster + b]);
        fprintf(stderr, " ms)\n");
    }
    if (ef) return set_err(ctx, PASUR_ENUMERIC, "non-finite root value in the CFR sweep");
    return PASUR_OK;
}

int sigma_sqdiff(const pasur_tree *t, const float *a_dev, const float *b_dev, double *acc_dev) {
    pasur_ctx *ctx = t->ctx;
    int64_t cb = 0;
    for (int k = 1; k < 9; k++) {
        if (t->M[k] > 0) {
            const unsigned grid = (unsigned)std::min<int64_t>((t->M[k] * 32 + 255) / 256, (int64_t)ctx->num_sms * 16);
            k_sigma_sqdiff<<<grid, 256, 0, ctx->stream>>>(t->root[k], t->M[k], t->cfgt_off[k], t->csoff_d, t->cmult_d,
                                                         a_dev + cb, b_dev + cb, acc_dev);
            ctx->launches++;
            PASUR_CUDA(ctx, cudaGetLastError());
        }
        cb += t->cQ[k];
    }
    return PASUR_OK;
}

// average strategies of the solved slots (levels 1..8 concatenated in solved FGT order)
int export_sigma_solved(const pasur_tree *t, float *out_dev) {
    pasur_ctx *ctx = t->ctx;
    LevelPtrs lp{};
    int64_t base = 0, ne = 0;
    for (int k = 0; k < 9; k++) {
        lp.fgt[k] = t->cfgt_off[k];
        lp.child[k] = k < 8 ? t->child_off[k] : nullptr;
        lp.base[k] = k >= 1 ? base : 0;
        if (k >= 1) base += t->cQ[k];
    }
    ne = base;
    if (ne > 0) {
        k_fill<<<grid_for(ne, 256), 256, 0, ctx->stream>>>(out_dev, ne, 1.0f);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    if (t->plan.n_items) {
        unsigned g = (unsigned)std::min<int64_t>(t->plan.n_items, 65535);
        k_export_sigma<<<g, 256, 0, ctx->stream>>>(t->plan.items_d, t->plan.n_items, t->croots_d, t->act_cs, t->act_d,
                                                   t->act_gt, t->S, lp, out_dev);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    return PASUR_OK;
}

int cfr_export_sigma(const pasur_tree *t, float *out_dev) {
    if (!t->merged) return export_sigma_solved(t, out_dev);
    pasur_ctx *ctx = t->ctx;
    int64_t ce = 0;
    for (int k = 1; k < 9; k++) ce += t->cQ[k];
    float *tmp = nullptr;
    const size_t tb = sizeof(float) * (size_t)(ce + 1);
    PASUR_TRY(dev_alloc(ctx, (void **)&tmp, tb));
    int rc = export_sigma_solved(t, tmp);
    // every full slot takes its solved slot's strategy, level by level
    int64_t fb = 0, cb = 0;
    for (int k = 1; k < 9 && rc == PASUR_OK; k++) {
        if (t->M[k] > 0) {
            k_expand_edges<<<grid_for(t->M[k] * 32, 256), 256, 0, ctx->stream>>>(
                t->root[k], t->M[k], t->fgt_off[k], t->cfgt_off[k], t->score_off_d, t->csoff_d, t->cidx0_d, tmp + cb,
                out_dev + fb);
            ctx->launches++;
            if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_expand_edges launch");
        }
        fb += t->Q[k];
        cb += t->cQ[k];
    }
    dev_free(ctx, tmp, tb);  // stream-ordered: freed after the expansion has read it
    return rc;
}

int cfr_export_utilities(const pasur_tree *t, float *out_dev) { return cfr_export_utilities_n(t, t->iters_done, out_dev); }

// average root utility of every full root slot, from its solved slot (no allocation: the batch
// captures this into its graph)
int cfr_export_utilities_n(const pasur_tree *t, int64_t iters, float *out_dev) {
    pasur_ctx *ctx = t->ctx;
    if (t->Q[0] == 0) return PASUR_OK;
    double inv = iters > 0 ? 1.0 / (double)iters : 0.0;
    k_export_util<<<grid_for(t->Q[0], 256), 256, 0, ctx->stream>>>(t->uacc, t->cidx0_d, t->Q[0], inv, out_dev);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    return PASUR_OK;
}

}  // namespace pasur

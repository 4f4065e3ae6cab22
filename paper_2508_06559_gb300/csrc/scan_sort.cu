// Device-wide exclusive scan and stable LSD radix sort of (key, value) pairs, used by the level
// expansion (count -> scan -> emit), the Unfolding Process (score-slot offsets) and the
// between-round deduplication.
#include "pasur_internal.cuh"

namespace pasur {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive prefix of v over the block (kScanThreads threads); *total = block sum
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int64_t ti = warp_incl_scan(t);
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;
        if (lane == kScanThreads / 32 - 1) *total = ti;
    }
    __syncthreads();
    int64_t r = warp_tot[w] + inc - v;
    __syncthreads();
    return r;
}

// sums of tiles of the sequence in[0..n) followed by one zero (length n+1)
template <typename T>
__global__ void k_tile_reduce(const T *__restrict__ in, int64_t n, int64_t *__restrict__ part) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        if (idx < n) s += (int64_t)in[idx];
    }
    __shared__ int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// out[i] = part_off[tile] + exclusive prefix inside the tile, for i in [0, n] (element n is 0)
template <typename T>
__global__ void k_tile_scan(const T *__restrict__ in, int64_t n, const int64_t *__restrict__ part_off,
                            int64_t *__restrict__ out) {
    __shared__ int64_t buf[kScanTile];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        buf[i * kScanThreads + threadIdx.x] = idx < n ? (int64_t)in[idx] : 0;
    }
    __syncthreads();
    int64_t loc[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        loc[i] = s;
        s += buf[threadIdx.x * kScanItems + i];
    }
    __shared__ int64_t tot;
    int64_t pre = block_excl_scan(s, &tot);
    int64_t off = part_off ? part_off[blockIdx.x] : 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) buf[threadIdx.x * kScanItems + i] = off + pre + loc[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i * kScanThreads + threadIdx.x;
        if (idx <= n) out[idx] = buf[i * kScanThreads + threadIdx.x];
    }
}

template <typename T>
int scan_impl(pasur_ctx *ctx, const T *in, int64_t *out, int64_t n) {
    if (n < 0) return set_err(ctx, PASUR_EINVAL, "scan: negative length");
    int64_t nb = (n + 1 + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_tile_scan<T><<<1, kScanThreads, 0, ctx->stream>>>(in, n, nullptr, out);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
        return PASUR_OK;
    }
    int64_t *part = nullptr;
    size_t bytes = sizeof(int64_t) * (size_t)(2 * nb + 2);
    PASUR_TRY(dev_alloc(ctx, (void **)&part, bytes));
    int64_t *part_off = part + nb + 1;
    k_tile_reduce<T><<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, n, part);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    int rc = e == cudaSuccess ? scan_impl<int64_t>(ctx, part, part_off, nb) : cuda_err(ctx, e, "k_tile_reduce");
    if (rc == PASUR_OK) {
        k_tile_scan<T><<<(unsigned)nb, kScanThreads, 0, ctx->stream>>>(in, n, part_off, out);
        ctx->launches++;
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "k_tile_scan");
    }
    dev_free(ctx, part, bytes);
    return rc;
}

// ---- radix sort -------------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void k_digit_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, int nblocks,
                             int32_t *__restrict__ counts) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; r++) {
        int64_t idx = base + r * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// stable scatter: elements of a tile are ranked in index order (round, warp, lane)
__global__ void k_digit_scatter(const uint64_t *__restrict__ keys, const int64_t *__restrict__ vals, int64_t n,
                                int shift, int nblocks, const int64_t *__restrict__ offs,
                                uint64_t *__restrict__ keys_out, int64_t *__restrict__ vals_out) {
    __shared__ int64_t gofs[256];
    __shared__ int32_t run[256];
    __shared__ int32_t wcnt[kSortWarps][256];
    int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    gofs[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    run[tid] = 0;
    for (int i = 0; i < kSortWarps; i++) wcnt[i][tid] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; r++) {
        int64_t idx = base + r * kSortThreads + tid;
        bool ok = idx < n;
        uint64_t k = ok ? keys[idx] : 0;
        int64_t v = ok ? vals[idx] : 0;
        int d = ok ? (int)((k >> shift) & 0xFF) : 256;
        unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        int rank = __popc(peers & lt);
        if (ok && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            int32_t before = 0;
            for (int i = 0; i < w; i++) before += wcnt[i][d];
            int64_t pos = gofs[d] + run[d] + before + rank;
            keys_out[pos] = k;
            vals_out[pos] = v;
        }
        __syncthreads();
        int32_t add = 0;
        for (int i = 0; i < kSortWarps; i++) {
            add += wcnt[i][tid];
            wcnt[i][tid] = 0;
        }
        run[tid] += add;
        __syncthreads();
    }
}

}  // namespace

int exclusive_scan_i32(pasur_ctx *ctx, const int32_t *in, int64_t *out, int64_t n) {
    return scan_impl<int32_t>(ctx, in, out, n);
}
int exclusive_scan_i64(pasur_ctx *ctx, const int64_t *in, int64_t *out, int64_t n) {
    return scan_impl<int64_t>(ctx, in, out, n);
}

int radix_sort_pairs(pasur_ctx *ctx, uint64_t *keys, int64_t *vals, int64_t n, int bits) {
    if (n <= 1 || bits <= 0) return PASUR_OK;
    int64_t nblocks = (n + kSortTile - 1) / kSortTile;
    if (nblocks * 256 >= (int64_t)1 << 31) return set_err(ctx, PASUR_EOVERFLOW, "radix sort: too many tiles");
    uint64_t *k2 = nullptr;
    int64_t *v2 = nullptr, *offs = nullptr;
    int32_t *counts = nullptr;
    size_t kb = sizeof(uint64_t) * (size_t)n, vb = sizeof(int64_t) * (size_t)n;
    size_t cb = sizeof(int32_t) * (size_t)(nblocks * 256), ob = sizeof(int64_t) * (size_t)(nblocks * 256 + 1);
    int rc = dev_alloc(ctx, (void **)&k2, kb);
    if (rc == PASUR_OK) rc = dev_alloc(ctx, (void **)&v2, vb);
    if (rc == PASUR_OK) rc = dev_alloc(ctx, (void **)&counts, cb);
    if (rc == PASUR_OK) rc = dev_alloc(ctx, (void **)&offs, ob);
    uint64_t *ka = keys, *kbuf = k2;
    int64_t *va = vals, *vbuf = v2;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes && rc == PASUR_OK; p++) {
        int shift = 8 * p;
        k_digit_hist<<<(unsigned)nblocks, kSortThreads, 0, ctx->stream>>>(ka, n, shift, (int)nblocks, counts);
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_err(ctx, e, "k_digit_hist"); break; }
        rc = exclusive_scan_i32(ctx, counts, offs, nblocks * 256);
        if (rc != PASUR_OK) break;
        k_digit_scatter<<<(unsigned)nblocks, kSortThreads, 0, ctx->stream>>>(ka, va, n, shift, (int)nblocks, offs,
                                                                            kbuf, vbuf);
        ctx->launches++;
        e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_err(ctx, e, "k_digit_scatter"); break; }
        uint64_t *tk = ka; ka = kbuf; kbuf = tk;
        int64_t *tv = va; va = vbuf; vbuf = tv;
    }
    if (rc == PASUR_OK && ka != keys) {
        cudaError_t e = cudaMemcpyAsync(keys, ka, kb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, vb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "radix sort copy-back");
    }
    if (rc == PASUR_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "radix sort");
    }
    dev_free(ctx, k2, kb);
    dev_free(ctx, v2, vb);
    dev_free(ctx, counts, cb);
    dev_free(ctx, offs, ob);
    return rc;
}

int read_i64(pasur_ctx *ctx, const int64_t *dptr, int64_t *out) {
    PASUR_CUDA(ctx, cudaMemcpyAsync(out, dptr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

}  // namespace pasur

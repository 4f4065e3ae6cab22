// pasur_move_offsets_noalloc: the count -> offsets step of the level expansion (the exclusive
// prefix sum that turns each node's number of legal moves into the CSR offsets of its children)
// for callers that cannot allocate device memory.
//
// pasur_build_round computes these offsets with a multi-level scan whose per-tile partial sums
// live in device memory it allocates (cudaMallocAsync).  Some callers cannot allocate at that
// point: an application that hands the whole GPU memory to its own arena up front and forbids any
// other allocation, a plug-in running inside a host program that owns the allocator, or real-time
// code that must not take the allocator's locks or risk an out-of-memory failure mid-run.  This
// variant keeps the partial sums in a file-scope __device__ array instead, so it allocates nothing;
// in exchange its input length is bounded (kNoAllocMaxCounts = 4,194,303 counts) and all calls
// share that one array.
//
// Set-up: the array's device address is looked up with cudaGetSymbolAddress on the first call made
// while a given device is current, and cached per device.  Make that first call outside any CUDA
// stream capture.
//
// Nothing in the array needs to start at zero: every call writes each partial sum it later reads.
// It does keep the last call's partial sums until the next call overwrites them.
#include <string>

#include "pasur_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;                       // 2048 counts per block
constexpr int64_t kNoAllocMaxTiles = kTile;                    // one block scans all tile sums
constexpr int64_t kNoAllocMaxCounts = kTile * kNoAllocMaxTiles - 1;  // 4,194,303 counts

// Partial sums of the tiles ([0, kTile)) and their exclusive prefix ([kTile, 2*kTile+1)).
// Every GPU that loads the library holds these 32 KB until the process exits.  All calls share
// them: two calls that overlap on the GPU (different streams, or the same stream from different
// threads without ordering) race on this array and produce wrong offsets.
static __device__ __align__(256) int64_t g_scan_scratch[2 * kTile + 16];

__device__ __forceinline__ int64_t warp_scan_incl(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive block prefix of v (kThreads threads); *total receives the block sum
__device__ int64_t block_scan_excl(int64_t v, int64_t *total) {
    __shared__ int64_t wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t inc = warp_scan_incl(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int64_t x = lane < kThreads / 32 ? wsum[lane] : 0;
        const int64_t xi = warp_scan_incl(x);
        if (lane < kThreads / 32) wsum[lane] = xi - x;
        if (lane == kThreads / 32 - 1) *total = xi;
    }
    __syncthreads();
    const int64_t r = wsum[w] + inc - v;
    __syncthreads();
    return r;
}

// pass 1: sum of each tile of the sequence counts[0..n) followed by one zero
__global__ void k_tile_sums(const int32_t *__restrict__ counts, int64_t n, int64_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const int64_t idx = base + i * kThreads + threadIdx.x;
        if (idx < n) s += counts[idx];
    }
    __shared__ int64_t tot;
    block_scan_excl(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// pass 2 (one block): exclusive prefix of the tile sums
__global__ void k_scan_tile_sums(const int64_t *__restrict__ sums, int64_t nb, int64_t *__restrict__ sums_off) {
    int64_t loc[kItems], s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const int64_t idx = (int64_t)threadIdx.x * kItems + i;
        loc[i] = s;
        s += idx < nb ? sums[idx] : 0;
    }
    __shared__ int64_t tot;
    const int64_t pre = block_scan_excl(s, &tot);
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const int64_t idx = (int64_t)threadIdx.x * kItems + i;
        if (idx < nb) sums_off[idx] = pre + loc[i];
    }
}

// pass 3: offsets[i] = (prefix of the tile) + (prefix inside the tile), i in [0, n]
__global__ void k_tile_offsets(const int32_t *__restrict__ counts, int64_t n, const int64_t *__restrict__ sums_off,
                               int64_t *__restrict__ offsets) {
    __shared__ int64_t buf[kTile];
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const int64_t idx = base + i * kThreads + threadIdx.x;
        buf[i * kThreads + threadIdx.x] = idx < n ? counts[idx] : 0;
    }
    __syncthreads();
    int64_t loc[kItems], s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        loc[i] = s;
        s += buf[threadIdx.x * kItems + i];
    }
    __shared__ int64_t tot;
    const int64_t pre = block_scan_excl(s, &tot);
    const int64_t off = sums_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kItems; i++) buf[threadIdx.x * kItems + i] = off + pre + loc[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const int64_t idx = base + i * kThreads + threadIdx.x;
        if (idx <= n) offsets[idx] = buf[i * kThreads + threadIdx.x];
    }
}

// device address of g_scan_scratch, looked up once per device (host code may not use the
// symbol's name as an address)
constexpr int kMaxDevices = 64;
int64_t *g_scratch_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(int64_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scan_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (int64_t *)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int pasur_move_offsets_noalloc(const int32_t *counts, int64_t n, int64_t *offsets, void *cuda_stream) {
    if (n < 0 || (n > 0 && !counts) || !offsets)
        return pasur::set_err(nullptr, PASUR_EINVAL, "pasur_move_offsets_noalloc: bad arguments");
    if (n > kNoAllocMaxCounts)
        return pasur::set_err(nullptr, PASUR_EOVERFLOW,
                              "pasur_move_offsets_noalloc: " + std::to_string(n) + " counts exceed the fixed limit of " +
                                  std::to_string(kNoAllocMaxCounts));
    int64_t *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pasur::set_err(nullptr, PASUR_ECUDA, std::string("pasur_move_offsets_noalloc: ") + cudaGetErrorString(e));
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t nb = (n + 1 + kTile - 1) / kTile;  // tiles of counts[0..n] (element n is 0)
    int64_t *sums = scratch, *sums_off = scratch + kTile;
    k_tile_sums<<<(unsigned)nb, kThreads, 0, st>>>(counts, n, sums);
    k_scan_tile_sums<<<1, kThreads, 0, st>>>(sums, nb, sums_off);
    k_tile_offsets<<<(unsigned)nb, kThreads, 0, st>>>(counts, n, sums_off, offsets);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return pasur::set_err(nullptr, PASUR_ECUDA, std::string("pasur_move_offsets_noalloc: ") + cudaGetErrorString(e));
    return PASUR_OK;
}

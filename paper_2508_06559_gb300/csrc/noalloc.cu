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
// in a given CUDA context (normally: the first call with a given device current) and cached per
// context.  Make that first call outside any CUDA stream capture.
//
// Nothing in the array needs to start at zero: every call writes each partial sum it later reads.
// It does keep the last call's partial sums until the next call overwrites them.
#include <mutex>
#include <string>
#include <utility>
#include <vector>

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

// Device address of g_scan_scratch.  Host code may not use the symbol's name as an address, so
// it is looked up with cudaGetSymbolAddress, once per CUDA context: the address belongs to the
// module loaded in the context that was current at the lookup, so a program that switches to
// another (non-primary) context, or resets the device and so loads the module again, gets a
// fresh lookup instead of a stale address.  Contexts are told apart by the driver's context id,
// which is never reused within a process; the table is guarded by a mutex, so two host threads
// making their first call at the same time look the address up once.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

struct ScratchTable {
    std::mutex mu;
    std::once_flag once;
    CtxGetCurrentFn get_current = nullptr;
    CtxGetIdFn get_id = nullptr;
    std::vector<std::pair<unsigned long long, int64_t *>> by_ctx;
};
ScratchTable g_scratch;

cudaError_t current_context_id(unsigned long long *id) {
    std::call_once(g_scratch.once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_scratch.get_current = (CtxGetCurrentFn)f;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_scratch.get_id = (CtxGetIdFn)f;
    });
    if (!g_scratch.get_current || !g_scratch.get_id) return cudaErrorNotSupported;
    void *c = nullptr;
    if (g_scratch.get_current(&c) != 0 || !c) return cudaErrorDeviceUninitialized;
    return g_scratch.get_id(c, id) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t scratch_for_current_context(int64_t **out) {
    // bind the runtime's context of the current device first (a runtime call that needs one)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    void *p = nullptr;
    unsigned long long id = 0;
    if (current_context_id(&id) != cudaSuccess) {
        e = cudaGetSymbolAddress(&p, g_scan_scratch);  // makes the device's primary context current
        if (e != cudaSuccess) return e;
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
    }
    std::lock_guard<std::mutex> lk(g_scratch.mu);
    for (const auto &x : g_scratch.by_ctx)
        if (x.first == id) {
            *out = x.second;
            return cudaSuccess;
        }
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_scan_scratch);
        if (e != cudaSuccess) return e;
    }
    g_scratch.by_ctx.push_back({id, (int64_t *)p});
    *out = (int64_t *)p;
    return cudaSuccess;
}

// true when p is an address the device can dereference (device or managed memory)
bool device_addressable(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int pasur_move_offsets_noalloc(const int32_t *counts, int64_t n, int64_t *offsets, void *cuda_stream) {
    if (n < 0 || (n > 0 && !counts) || !offsets)
        return pasur::set_err(nullptr, PASUR_EINVAL, "pasur_move_offsets_noalloc: bad arguments");
    if (n > kNoAllocMaxCounts)
        return pasur::set_err(nullptr, PASUR_EOVERFLOW,
                              "pasur_move_offsets_noalloc: " + std::to_string(n) + " counts exceed the fixed limit of " +
                                  std::to_string(kNoAllocMaxCounts));
    if (!device_addressable(offsets) || (n > 0 && !device_addressable(counts)))
        return pasur::set_err(nullptr, PASUR_EINVAL,
                              "pasur_move_offsets_noalloc: counts and offsets must be device memory");
    int64_t *scratch = nullptr;
    cudaError_t e = scratch_for_current_context(&scratch);
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

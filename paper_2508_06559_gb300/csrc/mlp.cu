// Round-start utility surrogate: a 256-256-256-256-1 GELU network trained on the GPU with Adam on
// utilities the exact solver produces, used to give a round's leaves their next-round values
// without building and solving the later rounds.  The paper's own learned part is a gradient-
// boosted model of the strategy (§Results); this surrogate of U follows the round-by-round value
// hand-off of eq. passuputil.
//
// Every dense contraction runs on the 5th-generation tensor cores: k_gemm computes
// C[M x 256] = A[M x K] . B[256 x K]^T with bf16 operands staged into shared memory by bulk async
// copies (cp.async.bulk, completion on an mbarrier), tcgen05.mma issued by one thread with the
// f32 accumulator (128 lanes x 256 columns) in tensor memory, and a fused epilogue that reads the
// accumulator back with tcgen05.ld: bias + GELU for the forward layers, the output layer, loss and
// its gradient for the last hidden layer, GELU' for the input gradients, atomics for the weight
// gradients.  Operands live in HBM in the tensor cores' canonical K-major layout without swizzle
// (8x8 core matrices of 128 contiguous bytes), ordered so that one (128-row, 64-column) tile is
// one contiguous 16 KB block: element (r, k) of an R-row matrix is at
//   ((k/64) * (R/8) + r/8) * 512 + ((k%64)/8) * 64 + (r%8) * 8 + (k%8)      (bf16 units).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

constexpr int kHid = 256;           // hidden width = input width = GEMM N
constexpr int kStages = 2;          // operand pipeline depth
constexpr uint32_t kAStage = 128 * 64 * 2, kBStage = 256 * 64 * 2;
constexpr size_t kGemmSmem = kStages * (kAStage + kBStage) + 1024 + 128;
constexpr int kParams = 3 * kHid * kHid + 3 * kHid + kHid + 1;
constexpr int64_t kTimeoutNs = 1000000000LL;  // bounded waits: one second

enum { EPI_FWD = 0, EPI_FWD_INFER = 1, EPI_LAST_TRAIN = 2, EPI_LAST_INFER = 3, EPI_DA = 4, EPI_DW = 5 };

__host__ __device__ __forceinline__ int64_t tiled(int64_t r, int64_t k, int64_t R) {
    return ((k >> 6) * (R >> 3) + (r >> 3)) * 512 + ((k >> 3) & 7) * 64 + (r & 7) * 8 + (k & 7);
}

// ---- PTX wrappers ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase with the given parity; false after one second
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const int64_t t0 = now_ns();
    while (!mbar_try(bar, parity))
        if (now_ns() - t0 > kTimeoutNs) return false;
    return true;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: canonical K-major layout, no swizzle; lbo = byte distance of
// core matrices adjacent in K, sbo = byte distance of 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}

// instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both K-major, M = 128,
// N = 256
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

// 32 consecutive f32 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 8 bf16 of row r, columns c..c+7 (c % 8 == 0) into a tiled matrix of R rows
__device__ __forceinline__ void store8_tiled(__nv_bfloat16 *M, int64_t r, int64_t c, int64_t R, const float *v) {
    __align__(16) __nv_bfloat16 b[8];
#pragma unroll
    for (int i = 0; i < 8; i++) b[i] = __float2bfloat16_rn(v[i]);
    *reinterpret_cast<uint4 *>(M + tiled(r, c, R)) = *reinterpret_cast<const uint4 *>(b);
}

struct GemmArgs {
    const __nv_bfloat16 *A;    // tiled, a_rows rows, K columns
    const __nv_bfloat16 *B;    // tiled, 256 rows, K columns
    int64_t a_rows, K;
    int64_t kcs;               // K chunks (of 64) per split
    const float *bias;         // forward: [256]
    float *z_out;              // EPI_FWD: pre-activation, f32 row-major [M x 256]
    __nv_bfloat16 *h_out;      // tiled [M x 256] (activation or pre-activation gradient)
    __nv_bfloat16 *ht_out;     // tiled [256 x M] (its transpose)
    const float *z_in;         // EPI_DA: pre-activation of the layer below, f32 row-major
    float *db;                 // column sums of the pre-activation gradient (atomics)
    float *dW;                 // EPI_DW: f32 row-major [256 x 256] (atomics)
    const float *w3, *b3, *y;  // output layer and targets
    float *yhat, *loss, *dw3, *db3;
    int64_t n_valid;
    float inv_n;
    int32_t *err;
};

template <int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm(const GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem, *sB = smem + kStages * kAStage;
    uint64_t *full = (uint64_t *)(sB + kStages * kBStage);
    uint64_t *freed = full + kStages;
    uint64_t *accd = freed + kStages;
    uint32_t *tslot = (uint32_t *)(accd + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nk = g.K >> 6;
    const int64_t c0 = (int64_t)blockIdx.y * g.kcs, c1 = min(nk, c0 + g.kcs);
    const int64_t m0 = (int64_t)blockIdx.x * 128;
    if (c1 <= c0) return;  // uniform per block: nothing to accumulate
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&freed[s], 1);
        }
        mbar_init(accd, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(256) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (threadIdx.x == 0) {
        const int64_t n = c1 - c0;
        int64_t issued = 0, landed = 0;
        bool ok = true;
        auto load = [&](int64_t i) {
            const int s = (int)(i % kStages);
            const int64_t kc = c0 + i;
            mbar_expect_tx(&full[s], kAStage + kBStage);
            bulk_load(sA + s * kAStage, g.A + (kc * (g.a_rows >> 3) + (m0 >> 3)) * 512, kAStage, &full[s]);
            bulk_load(sB + s * kBStage, g.B + kc * (kHid / 8) * 512, kBStage, &full[s]);
            issued++;
        };
        for (int64_t i = 0; i < n && i < kStages; i++) load(i);
        for (int64_t i = 0; i < n; i++) {
            const int s = (int)(i % kStages);
            const uint32_t ph = (uint32_t)((i / kStages) & 1);
            if (!mbar_wait(&full[s], ph)) { ok = false; break; }
            landed++;
            tc_fence_after();
            const uint32_t a0 = su32(sA + s * kAStage), b0 = su32(sB + s * kBStage);
#pragma unroll
            for (int kk = 0; kk < 4; kk++)
                mma_bf16(tmem, sdesc(a0 + kk * 256, 128, 1024), sdesc(b0 + kk * 256, 128, 1024), (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&freed[s]);
            if (i + kStages < n) {
                if (!mbar_wait(&freed[s], ph)) { ok = false; break; }
                load(i + kStages);
            }
        }
        mma_commit(accd);
        if (!ok) {
            atomicExch(g.err, 1);
            // let every copy still in flight land before the block's shared memory is released
            for (int64_t i = landed; i < issued; i++) mbar_wait(&full[(int)(i % kStages)], (uint32_t)((i / kStages) & 1));
        }
    }
    __syncwarp();
    const bool acc_ok = mbar_wait(accd, 0);
    tc_fence_after();
    if (!acc_ok) {
        if (lane == 0) atomicExch(g.err, 2);
    } else {
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        float v[32];
        if (EPI == EPI_DW) {
#pragma unroll 1
            for (int j = 0; j < kHid / 32; j++) {
                tmem_ld32(taddr + j * 32, v);
                float *dst = g.dW + row * kHid + j * 32;
#pragma unroll
                for (int i = 0; i < 32; i++) atomicAdd(dst + i, v[i]);
            }
        } else if (EPI == EPI_FWD || EPI == EPI_FWD_INFER) {
#pragma unroll 1
            for (int j = 0; j < kHid / 32; j++) {
                tmem_ld32(taddr + j * 32, v);
                const int c = j * 32;
#pragma unroll
                for (int i = 0; i < 32; i++) v[i] += g.bias[c + i];
                if (EPI == EPI_FWD) {
                    float4 *zo = reinterpret_cast<float4 *>(g.z_out + row * kHid + c);
#pragma unroll
                    for (int i = 0; i < 8; i++) zo[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
#pragma unroll
                for (int i = 0; i < 32; i++) v[i] = gelu(v[i]);
#pragma unroll
                for (int q = 0; q < 4; q++) store8_tiled(g.h_out, row, c + 8 * q, g.a_rows, v + 8 * q);
                if (EPI == EPI_FWD) {
#pragma unroll
                    for (int i = 0; i < 32; i++) g.ht_out[tiled(c + i, row, kHid)] = __float2bfloat16_rn(v[i]);
                }
            }
        } else if (EPI == EPI_LAST_TRAIN || EPI == EPI_LAST_INFER) {
            // output layer y = h3 . w3 + b3 with h3 = gelu(acc + b2), in f32 per row
            float yh = g.b3[0];
#pragma unroll 1
            for (int j = 0; j < kHid / 32; j++) {
                tmem_ld32(taddr + j * 32, v);
#pragma unroll
                for (int i = 0; i < 32; i++) yh += gelu(v[i] + g.bias[j * 32 + i]) * g.w3[j * 32 + i];
            }
            const bool valid = row < g.n_valid;
            if (valid) g.yhat[row] = yh;
            if (EPI == EPI_LAST_TRAIN) {
                const float err = valid ? yh - g.y[row] : 0.f;
                const float gy = 2.f * err * g.inv_n;  // d loss / d yhat
                const float l = warp_sum(err * err * g.inv_n), sg = warp_sum(gy);
                if (lane == 0) {
                    atomicAdd(g.loss, l);
                    atomicAdd(g.db3, sg);
                }
#pragma unroll 1
                for (int j = 0; j < kHid / 32; j++) {
                    tmem_ld32(taddr + j * 32, v);
                    const int c = j * 32;
#pragma unroll
                    for (int i = 0; i < 32; i++) {
                        const float z = v[i] + g.bias[c + i];
                        const float s3 = warp_sum(gy * gelu(z));
                        const float dz = gy * g.w3[c + i] * gelu_grad(z);
                        const float s2 = warp_sum(dz);
                        if (lane == 0) {
                            atomicAdd(g.dw3 + c + i, s3);
                            atomicAdd(g.db + c + i, s2);
                        }
                        v[i] = dz;
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) store8_tiled(g.h_out, row, c + 8 * q, g.a_rows, v + 8 * q);
#pragma unroll
                    for (int i = 0; i < 32; i++) g.ht_out[tiled(c + i, row, kHid)] = __float2bfloat16_rn(v[i]);
                }
            }
        } else if (EPI == EPI_DA) {
            // accumulator = gradient of the layer input; times gelu' of the layer below
#pragma unroll 1
            for (int j = 0; j < kHid / 32; j++) {
                tmem_ld32(taddr + j * 32, v);
                const int c = j * 32;
                const float *zi = g.z_in + row * kHid + c;
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const float dz = v[i] * gelu_grad(zi[i]);
                    const float s = warp_sum(dz);
                    if (lane == 0) atomicAdd(g.db + c + i, s);
                    v[i] = dz;
                }
#pragma unroll
                for (int q = 0; q < 4; q++) store8_tiled(g.h_out, row, c + 8 * q, g.a_rows, v + 8 * q);
#pragma unroll
                for (int i = 0; i < 32; i++) g.ht_out[tiled(c + i, row, kHid)] = __float2bfloat16_rn(v[i]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
}

// rows (optionally gathered through perm) of a row-major bf16 [n x 256] matrix into the tiled
// matrix [Mp x 256] and its tiled transpose [256 x Mp]; rows n..Mp-1 are zero.  Also gathers the
// targets.
__global__ void k_pack(const __nv_bfloat16 *__restrict__ X, const float *__restrict__ y, const int64_t *__restrict__ perm,
                       int64_t row0, int64_t n, int64_t Mp, __nv_bfloat16 *__restrict__ Xt, __nv_bfloat16 *__restrict__ XtT,
                       float *__restrict__ yb) {
    const int64_t total = Mp * (kHid / 8);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / (kHid / 8), c = (e % (kHid / 8)) * 8;
        uint4 w = make_uint4(0, 0, 0, 0);
        if (r < n) {
            const int64_t src = perm ? perm[row0 + r] : row0 + r;
            w = *reinterpret_cast<const uint4 *>(X + src * kHid + c);
            if (c == 0 && yb) yb[r] = y ? y[src] : 0.f;
        } else if (c == 0 && yb) {
            yb[r] = 0.f;
        }
        *reinterpret_cast<uint4 *>(Xt + tiled(r, c, Mp)) = w;
        if (XtT) {
            const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(&w);
#pragma unroll
            for (int i = 0; i < 8; i++) XtT[tiled(c + i, r, kHid)] = b[i];
        }
    }
}

// Adam (Kingma and Ba, 2015) on the flat parameters; writes the bf16 tiled weights and their
// transposes and clears the gradients.  t = step number (>= 1).
__global__ void k_adam(float *__restrict__ p, float *__restrict__ grad, float *__restrict__ m, float *__restrict__ v,
                       const int64_t *__restrict__ t_base, int64_t t_off, float lr, float b1, float b2, float eps,
                       __nv_bfloat16 *__restrict__ W, __nv_bfloat16 *__restrict__ WT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const double t = (double)(t_base[0] + t_off);
    const float c1 = (float)(1.0 / (1.0 - pow((double)b1, t))), c2 = (float)(1.0 / (1.0 - pow((double)b2, t)));
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    grad[i] = 0.f;
    // weight matrices l = 0..2 at offsets l * (256*256 + 256)
    const int per = kHid * kHid + kHid;
    const int l = i / per, o = i % per;
    if (l < 3 && o < kHid * kHid) {
        const int row = o / kHid, col = o % kHid;
        const __nv_bfloat16 b = __float2bfloat16_rn(pi);
        W[(int64_t)l * kHid * kHid + tiled(row, col, kHid)] = b;
        WT[(int64_t)l * kHid * kHid + tiled(col, row, kHid)] = b;
    }
}

__global__ void k_weights_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ W, __nv_bfloat16 *__restrict__ WT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * kHid * kHid) return;
    const int l = i / (kHid * kHid), o = i % (kHid * kHid), row = o / kHid, col = o % kHid;
    const __nv_bfloat16 b = __float2bfloat16_rn(p[(int64_t)l * (kHid * kHid + kHid) + o]);
    W[(int64_t)l * kHid * kHid + tiled(row, col, kHid)] = b;
    WT[(int64_t)l * kHid * kHid + tiled(col, row, kHid)] = b;
}

// Features of FGT roots (one thread per (GT root, slot)): card locations one-hot (Alex now or
// later, Bob now or later, pool, out), carried clubs / 8, inherited difference / 32, bonus
// one-hot, round one-hot, per-location clubs / points / Jacks / cards, zero padding; row-major
// bf16 [n x 256].
__global__ void k_features(const uint64_t *__restrict__ pools, const int64_t *__restrict__ soff,
                           const pasur_score *__restrict__ scores, int64_t n_pools, uint64_t alex, uint64_t bob, int rnd,
                           __nv_bfloat16 *__restrict__ out) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_pools; g += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t pool = pools[g];
        for (int64_t s = soff[g]; s < soff[g + 1]; s++) {
            __nv_bfloat16 *x = out + s * kHid;
            for (int c = 0; c < kHid; c++) x[c] = __float2bfloat16_rn(0.f);
            for (int c = 0; c < 52; c++) {
                const uint64_t b = 1ULL << c;
                const int loc = (pool & b) ? 2 : (alex & b) ? 0 : (bob & b) ? 1 : 3;
                x[52 * loc + c] = __float2bfloat16_rn(1.f);
            }
            const pasur_score sc = scores[s];
            x[208] = __float2bfloat16_rn(sc.a_clubs * 0.125f);
            x[209] = __float2bfloat16_rn(sc.b_clubs * 0.125f);
            x[210] = __float2bfloat16_rn(sc.delta * 0.03125f);
            x[211 + sc.bonus] = __float2bfloat16_rn(1.f);
            x[214 + rnd] = __float2bfloat16_rn(1.f);
            // per location (Alex, Bob, pool): clubs / 8, points / 8, Jacks / 4, cards / 32
            const uint64_t at[3] = {alex & ~pool, bob & ~pool, pool};
            for (int L = 0; L < 3; L++) {
                x[220 + 4 * L] = __float2bfloat16_rn(set_clubs(at[L]) * 0.125f);
                x[221 + 4 * L] = __float2bfloat16_rn(set_points(at[L]) * 0.125f);
                x[222 + 4 * L] = __float2bfloat16_rn(__popcll(at[L] & kJacks) * 0.25f);
                x[223 + 4 * L] = __float2bfloat16_rn(__popcll(at[L]) * 0.03125f);
            }
        }
    }
}

}  // namespace
}  // namespace pasur

using namespace pasur;

struct pasur_mlp {
    pasur_ctx *ctx = nullptr;
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // flat f32 [kParams]
    __nv_bfloat16 *W = nullptr, *WT = nullptr;                          // 3 tiled [256 x 256] each
    int64_t *t_d = nullptr;                                             // Adam step base
    int64_t steps = 0;
    float *loss_d = nullptr;
    int32_t *err_d = nullptr;
    // dataset (row-major bf16 features, f32 targets)
    int64_t cap = 0, n = 0;
    __nv_bfloat16 *X = nullptr;
    float *Y = nullptr;
    // work buffers for up to rows_cap rows
    int64_t rows_cap = 0;
    __nv_bfloat16 *h0 = nullptr, *h0t = nullptr, *h1 = nullptr, *h1t = nullptr, *h2 = nullptr, *h2t = nullptr;
    __nv_bfloat16 *d0 = nullptr, *d0t = nullptr, *d1 = nullptr, *d1t = nullptr, *d2 = nullptr, *d2t = nullptr;
    float *z0 = nullptr, *z1 = nullptr, *yb = nullptr, *yhat = nullptr;
    int64_t *perm_d = nullptr;
    std::vector<std::pair<void *, size_t>> owned;
    cudaGraphExec_t epoch_exec = nullptr;
    int64_t epoch_batch = 0, epoch_rows = 0;
    float last_train_ms = 0.f;
};

namespace {

int mlp_alloc(pasur_mlp *M, void **p, size_t bytes) {
    PASUR_TRY(dev_alloc(M->ctx, p, bytes));
    M->owned.push_back({*p, bytes});
    return PASUR_OK;
}

void mlp_release(pasur_mlp *M, void *p) {
    for (size_t i = 0; i < M->owned.size(); i++)
        if (M->owned[i].first == p) {
            dev_free(M->ctx, p, M->owned[i].second);
            M->owned.erase(M->owned.begin() + (long)i);
            return;
        }
}

int set_gemm_attrs(pasur_ctx *ctx) {
    static int done_dev = -1;
    if (done_dev == ctx->device) return PASUR_OK;
    PASUR_CUDA(ctx, cudaFuncSetAttribute(k_gemm<EPI_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
    PASUR_CUDA(ctx, cudaFuncSetAttribute(k_gemm<EPI_FWD_INFER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
    PASUR_CUDA(ctx, cudaFuncSetAttribute(k_gemm<EPI_LAST_TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
    PASUR_CUDA(ctx, cudaFuncSetAttribute(k_gemm<EPI_LAST_INFER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
    PASUR_CUDA(ctx, cudaFuncSetAttribute(k_gemm<EPI_DA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
    PASUR_CUDA(ctx, cudaFuncSetAttribute(k_gemm<EPI_DW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
    done_dev = ctx->device;
    return PASUR_OK;
}

int ensure_rows(pasur_mlp *M, int64_t rows) {
    if (rows <= M->rows_cap) return PASUR_OK;
    cudaStreamSynchronize(M->ctx->stream);
    void **bufs16[] = {(void **)&M->h0, (void **)&M->h0t, (void **)&M->h1, (void **)&M->h1t, (void **)&M->h2, (void **)&M->h2t,
                       (void **)&M->d0, (void **)&M->d0t, (void **)&M->d1, (void **)&M->d1t, (void **)&M->d2, (void **)&M->d2t};
    for (void **b : bufs16) {
        if (*b) mlp_release(M, *b);
        PASUR_TRY(mlp_alloc(M, b, sizeof(__nv_bfloat16) * (size_t)rows * kHid));
    }
    void **bufs32[] = {(void **)&M->z0, (void **)&M->z1};
    for (void **b : bufs32) {
        if (*b) mlp_release(M, *b);
        PASUR_TRY(mlp_alloc(M, b, sizeof(float) * (size_t)rows * kHid));
    }
    if (M->yb) mlp_release(M, M->yb);
    if (M->yhat) mlp_release(M, M->yhat);
    PASUR_TRY(mlp_alloc(M, (void **)&M->yb, sizeof(float) * (size_t)rows));
    PASUR_TRY(mlp_alloc(M, (void **)&M->yhat, sizeof(float) * (size_t)rows));
    M->rows_cap = rows;
    if (M->epoch_exec) {
        cudaGraphExecDestroy(M->epoch_exec);
        M->epoch_exec = nullptr;
    }
    return PASUR_OK;
}

GemmArgs base_args(pasur_mlp *M) {
    GemmArgs a{};
    a.err = M->err_d;
    return a;
}

template <int EPI>
int launch_gemm(pasur_mlp *M, const GemmArgs &a, int64_t m_tiles, int64_t splits) {
    pasur_ctx *ctx = M->ctx;
    dim3 grid((unsigned)m_tiles, (unsigned)splits);
    k_gemm<EPI><<<grid, 128, kGemmSmem, ctx->stream>>>(a);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    return PASUR_OK;
}

// forward (train: also the backward pass and gradients) of Mp packed rows in h0/h0t; targets in
// yb; n_valid real rows; no synchronisation (capturable)
int run_pass(pasur_mlp *M, int64_t Mp, int64_t n_valid, bool train) {
    const __nv_bfloat16 *W0 = M->W, *W1 = M->W + kHid * kHid, *W2 = M->W + 2 * kHid * kHid;
    const __nv_bfloat16 *WT1 = M->WT + kHid * kHid, *WT2 = M->WT + 2 * kHid * kHid;
    const int per = kHid * kHid + kHid;
    const float *b0 = M->p + kHid * kHid, *b1 = M->p + per + kHid * kHid, *b2 = M->p + 2 * per + kHid * kHid;
    const float *w3 = M->p + 3 * per, *b3 = w3 + kHid;
    float *g = M->grad;
    float *gW0 = g, *gb0 = g + kHid * kHid, *gW1 = g + per, *gb1 = g + per + kHid * kHid, *gW2 = g + 2 * per,
          *gb2 = g + 2 * per + kHid * kHid, *gw3 = g + 3 * per, *gb3 = gw3 + kHid;
    const int64_t mt = Mp / 128;
    GemmArgs a = base_args(M);
    a.a_rows = Mp;
    a.K = kHid;
    a.kcs = kHid / 64;
    // layer 0, 1
    a.A = M->h0; a.B = W0; a.bias = b0; a.z_out = M->z0; a.h_out = M->h1; a.ht_out = M->h1t;
    if (train) PASUR_TRY(launch_gemm<EPI_FWD>(M, a, mt, 1));
    else PASUR_TRY(launch_gemm<EPI_FWD_INFER>(M, a, mt, 1));
    a.A = M->h1; a.B = W1; a.bias = b1; a.z_out = M->z1; a.h_out = M->h2; a.ht_out = M->h2t;
    if (train) PASUR_TRY(launch_gemm<EPI_FWD>(M, a, mt, 1));
    else PASUR_TRY(launch_gemm<EPI_FWD_INFER>(M, a, mt, 1));
    // layer 2 + output layer (+ loss, output and layer-2 gradients)
    a.A = M->h2; a.B = W2; a.bias = b2; a.w3 = w3; a.b3 = b3; a.y = M->yb; a.yhat = M->yhat; a.n_valid = n_valid;
    a.inv_n = 1.f / (float)std::max<int64_t>(1, n_valid);
    if (!train) return launch_gemm<EPI_LAST_INFER>(M, a, mt, 1);
    a.loss = M->loss_d; a.dw3 = gw3; a.db3 = gb3; a.db = gb2; a.h_out = M->d2; a.ht_out = M->d2t;
    PASUR_TRY(launch_gemm<EPI_LAST_TRAIN>(M, a, mt, 1));
    // weight gradients: dW_l = dZ_l^T H_l (K = rows, split over the batch)
    const int64_t nk = Mp / 64;
    const int64_t splits = std::min<int64_t>(nk, 32), kcs = (nk + splits - 1) / splits;
    const int64_t used = (nk + kcs - 1) / kcs;
    auto dw = [&](const __nv_bfloat16 *dzt, const __nv_bfloat16 *ht, float *gW) {
        GemmArgs d = base_args(M);
        d.A = dzt; d.B = ht; d.a_rows = kHid; d.K = Mp; d.kcs = kcs; d.dW = gW;
        return launch_gemm<EPI_DW>(M, d, 2, used);
    };
    // input gradients: dH_l = dZ_l W_l, then dZ_{l-1} = dH_l * gelu'(Z_{l-1})
    auto da = [&](const __nv_bfloat16 *dz, const __nv_bfloat16 *wt, const float *zin, float *gb, __nv_bfloat16 *o,
                  __nv_bfloat16 *ot) {
        GemmArgs d = base_args(M);
        d.A = dz; d.B = wt; d.a_rows = Mp; d.K = kHid; d.kcs = kHid / 64; d.z_in = zin; d.db = gb; d.h_out = o; d.ht_out = ot;
        return launch_gemm<EPI_DA>(M, d, mt, 1);
    };
    PASUR_TRY(dw(M->d2t, M->h2t, gW2));
    PASUR_TRY(da(M->d2, WT2, M->z1, gb1, M->d1, M->d1t));
    PASUR_TRY(dw(M->d1t, M->h1t, gW1));
    PASUR_TRY(da(M->d1, WT1, M->z0, gb0, M->d0, M->d0t));
    PASUR_TRY(dw(M->d0t, M->h0t, gW0));
    return PASUR_OK;
}

int pack(pasur_mlp *M, const __nv_bfloat16 *X, const float *y, const int64_t *perm, int64_t row0, int64_t n, int64_t Mp,
         bool want_t) {
    const int64_t total = Mp * (kHid / 8);
    unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)M->ctx->num_sms * 8);
    k_pack<<<std::max(1u, grid), 256, 0, M->ctx->stream>>>(X, y, perm, row0, n, Mp, M->h0, want_t ? M->h0t : nullptr, M->yb);
    M->ctx->launches++;
    PASUR_CUDA(M->ctx, cudaGetLastError());
    return PASUR_OK;
}

int check_err(pasur_mlp *M) {
    int32_t e = 0;
    PASUR_CUDA(M->ctx, cudaMemcpyAsync(&e, M->err_d, sizeof e, cudaMemcpyDeviceToHost, M->ctx->stream));
    PASUR_CUDA(M->ctx, cudaStreamSynchronize(M->ctx->stream));
    if (e) return set_err(M->ctx, PASUR_ETIMEOUT, "surrogate GEMM: an operand copy or tensor-core wait timed out");
    return PASUR_OK;
}

int64_t pad128(int64_t n) { return std::max<int64_t>(128, (n + 127) / 128 * 128); }

// forward of n rows already in device row-major bf16 form; predictions into out_dev
int forward_rows(pasur_mlp *M, const __nv_bfloat16 *X, int64_t n, float *out_dev) {
    const int64_t chunk = 1 << 16;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t m = std::min(chunk, n - r0), Mp = pad128(m);
        PASUR_TRY(ensure_rows(M, Mp));
        PASUR_TRY(pack(M, X, nullptr, nullptr, r0, m, Mp, false));
        PASUR_TRY(run_pass(M, Mp, m, false));
        PASUR_CUDA(M->ctx, cudaMemcpyAsync(out_dev + r0, M->yhat, sizeof(float) * (size_t)m, cudaMemcpyDeviceToDevice, M->ctx->stream));
    }
    return PASUR_OK;
}

// features of (pools, score offsets, scores) host arrays of round rnd into a device buffer
int features_dev(pasur_mlp *M, const uint8_t *deck, int rnd, const uint64_t *pools, const int64_t *soff,
                 const pasur_score *scores, int64_t n_pools, __nv_bfloat16 **out, int64_t *n_rows,
                 std::vector<std::pair<void *, size_t>> &tmp) {
    pasur_ctx *ctx = M->ctx;
    const int64_t nr = soff[n_pools];
    *n_rows = nr;
    uint64_t alex = 0, bob = 0;
    for (int i = rnd; i < 6; i++)
        for (int j = 0; j < 4; j++) {
            alex |= 1ULL << deck[4 + 8 * i + j];
            bob |= 1ULL << deck[8 + 8 * i + j];
        }
    void *pp = nullptr, *so = nullptr, *sc = nullptr, *x = nullptr;
    auto al = [&](void **p, size_t b) {
        int rc = dev_alloc(ctx, p, b);
        if (rc == PASUR_OK) tmp.push_back({*p, b});
        return rc;
    };
    PASUR_TRY(al(&pp, sizeof(uint64_t) * (size_t)(n_pools + 1)));
    PASUR_TRY(al(&so, sizeof(int64_t) * (size_t)(n_pools + 1)));
    PASUR_TRY(al(&sc, sizeof(pasur_score) * (size_t)(nr + 1)));
    PASUR_TRY(al(&x, sizeof(__nv_bfloat16) * (size_t)(nr + 1) * kHid));
    PASUR_CUDA(ctx, cudaMemcpyAsync(pp, pools, sizeof(uint64_t) * (size_t)n_pools, cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(so, soff, sizeof(int64_t) * (size_t)(n_pools + 1), cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(sc, scores, sizeof(pasur_score) * (size_t)nr, cudaMemcpyHostToDevice, ctx->stream));
    if (n_pools > 0) {
        unsigned grid = (unsigned)std::min<int64_t>((n_pools + 127) / 128, 4096);
        k_features<<<grid, 128, 0, ctx->stream>>>((const uint64_t *)pp, (const int64_t *)so, (const pasur_score *)sc, n_pools,
                                                   alex, bob, rnd, (__nv_bfloat16 *)x);
        ctx->launches++;
        PASUR_CUDA(ctx, cudaGetLastError());
    }
    *out = (__nv_bfloat16 *)x;
    return PASUR_OK;
}

void free_tmp(pasur_ctx *ctx, std::vector<std::pair<void *, size_t>> &tmp) {
    cudaStreamSynchronize(ctx->stream);
    for (auto &t : tmp) dev_free(ctx, t.first, t.second);
    tmp.clear();
}

// host or device float input -> device pointer (copied into tmp when host)
int to_device(pasur_ctx *ctx, const void *src, size_t bytes, const void **dev, std::vector<std::pair<void *, size_t>> &tmp) {
    if (is_device_ptr(src)) {
        *dev = src;
        return PASUR_OK;
    }
    void *d = nullptr;
    PASUR_TRY(dev_alloc(ctx, &d, bytes + 16));
    tmp.push_back({d, bytes + 16});
    PASUR_CUDA(ctx, cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dev = d;
    return PASUR_OK;
}

int copy_to(pasur_ctx *ctx, void *dst, const void *src_dev, size_t bytes) {
    PASUR_CUDA(ctx, cudaMemcpyAsync(dst, src_dev, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

// splitmix64 uniform in [-1, 1)
double init_uniform(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

}  // namespace

extern "C" {

int pasur_mlp_create(pasur_ctx *ctx, int64_t dataset_capacity, uint64_t seed, pasur_mlp **out) {
    if (!ctx || !out) return ctx ? set_err(ctx, PASUR_EINVAL, "pasur_mlp_create: NULL argument") : PASUR_EINVAL;
    *out = nullptr;
    if (dataset_capacity < 0 || dataset_capacity > ((int64_t)1 << 31))
        return set_err(ctx, PASUR_EINVAL, "pasur_mlp_create: dataset_capacity must be 0..2^31");
    cudaSetDevice(ctx->device);
    PASUR_TRY(set_gemm_attrs(ctx));
    pasur_mlp *M = new pasur_mlp();
    M->ctx = ctx;
    int rc = PASUR_OK;
    auto A = [&](void **p, size_t b) {
        if (rc == PASUR_OK) rc = mlp_alloc(M, p, b);
    };
    A((void **)&M->p, sizeof(float) * kParams);
    A((void **)&M->grad, sizeof(float) * kParams);
    A((void **)&M->m, sizeof(float) * kParams);
    A((void **)&M->v, sizeof(float) * kParams);
    A((void **)&M->W, sizeof(__nv_bfloat16) * 3 * kHid * kHid);
    A((void **)&M->WT, sizeof(__nv_bfloat16) * 3 * kHid * kHid);
    A((void **)&M->t_d, sizeof(int64_t));
    A((void **)&M->loss_d, sizeof(float) * 4);
    A((void **)&M->err_d, sizeof(int32_t));
    M->cap = dataset_capacity;
    if (dataset_capacity > 0) {
        A((void **)&M->X, sizeof(__nv_bfloat16) * (size_t)dataset_capacity * kHid);
        A((void **)&M->Y, sizeof(float) * (size_t)dataset_capacity);
        A((void **)&M->perm_d, sizeof(int64_t) * (size_t)dataset_capacity);
    }
    if (rc == PASUR_OK) {
        // Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases
        std::vector<float> h(kParams, 0.f);
        uint64_t x = seed;
        const int per = kHid * kHid + kHid;
        for (int l = 0; l < 3; l++)
            for (int i = 0; i < kHid * kHid; i++) h[(size_t)(l * per + i)] = (float)(init_uniform(x) / 16.0);
        for (int i = 0; i < kHid; i++) h[(size_t)(3 * per + i)] = (float)(init_uniform(x) / 16.0);
        rc = pasur_mlp_set_params(M, h.data(), kParams);
    }
    if (rc != PASUR_OK) {
        pasur_mlp_free(M);
        return rc;
    }
    *out = M;
    return PASUR_OK;
}

int pasur_mlp_free(pasur_mlp *M) {
    if (!M) return PASUR_EINVAL;
    cudaSetDevice(M->ctx->device);
    cudaStreamSynchronize(M->ctx->stream);
    if (M->epoch_exec) cudaGraphExecDestroy(M->epoch_exec);
    for (auto &o : M->owned) dev_free(M->ctx, o.first, o.second);
    delete M;
    return PASUR_OK;
}

int pasur_mlp_set_params(pasur_mlp *M, const float *params, int64_t n) {
    if (!M || !params) return PASUR_EINVAL;
    pasur_ctx *ctx = M->ctx;
    if (n != kParams) return set_err(ctx, PASUR_EINVAL, "pasur_mlp_set_params: need " + std::to_string(kParams) + " floats");
    cudaSetDevice(ctx->device);
    PASUR_CUDA(ctx, cudaMemcpyAsync(M->p, params, sizeof(float) * kParams,
                                    is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaMemsetAsync(M->grad, 0, sizeof(float) * kParams, ctx->stream));
    PASUR_CUDA(ctx, cudaMemsetAsync(M->m, 0, sizeof(float) * kParams, ctx->stream));
    PASUR_CUDA(ctx, cudaMemsetAsync(M->v, 0, sizeof(float) * kParams, ctx->stream));
    PASUR_CUDA(ctx, cudaMemsetAsync(M->err_d, 0, sizeof(int32_t), ctx->stream));
    M->steps = 0;
    k_weights_bf16<<<(3 * kHid * kHid + 255) / 256, 256, 0, ctx->stream>>>(M->p, M->W, M->WT);
    ctx->launches++;
    PASUR_CUDA(ctx, cudaGetLastError());
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

int pasur_mlp_get_params(const pasur_mlp *M, float *params, int64_t cap) {
    if (!M || !params) return PASUR_EINVAL;
    if (cap < kParams) return set_err(M->ctx, PASUR_EOVERFLOW, "pasur_mlp_get_params: need " + std::to_string(kParams) + " floats");
    cudaSetDevice(M->ctx->device);
    return copy_to(M->ctx, params, M->p, sizeof(float) * kParams);
}

int pasur_mlp_forward(pasur_mlp *M, const uint16_t *x, int64_t n, float *y_out) {
    if (!M || n < 0 || (n > 0 && (!x || !y_out))) return M ? set_err(M->ctx, PASUR_EINVAL, "pasur_mlp_forward: bad arguments") : PASUR_EINVAL;
    pasur_ctx *ctx = M->ctx;
    cudaSetDevice(ctx->device);
    if (n == 0) return PASUR_OK;
    std::vector<std::pair<void *, size_t>> tmp;
    const void *xd = nullptr;
    int rc = to_device(ctx, x, sizeof(uint16_t) * (size_t)n * kHid, &xd, tmp);
    float *yd = nullptr;
    if (rc == PASUR_OK) {
        void *p = nullptr;
        rc = dev_alloc(ctx, &p, sizeof(float) * (size_t)n);
        if (rc == PASUR_OK) tmp.push_back({p, sizeof(float) * (size_t)n}), yd = (float *)p;
    }
    if (rc == PASUR_OK) rc = forward_rows(M, (const __nv_bfloat16 *)xd, n, yd);
    if (rc == PASUR_OK) rc = check_err(M);
    if (rc == PASUR_OK) rc = copy_to(ctx, y_out, yd, sizeof(float) * (size_t)n);
    free_tmp(ctx, tmp);
    return rc;
}

int pasur_mlp_gradients(pasur_mlp *M, const uint16_t *x, const float *y, int64_t n, float *loss_out, float *grads_out) {
    if (!M || n < 1 || !x || !y) return M ? set_err(M->ctx, PASUR_EINVAL, "pasur_mlp_gradients: bad arguments") : PASUR_EINVAL;
    pasur_ctx *ctx = M->ctx;
    if (n > (1 << 20)) return set_err(ctx, PASUR_EINVAL, "pasur_mlp_gradients: n must be <= 2^20");
    cudaSetDevice(ctx->device);
    std::vector<std::pair<void *, size_t>> tmp;
    const void *xd = nullptr, *yd = nullptr;
    int rc = to_device(ctx, x, sizeof(uint16_t) * (size_t)n * kHid, &xd, tmp);
    if (rc == PASUR_OK) rc = to_device(ctx, y, sizeof(float) * (size_t)n, &yd, tmp);
    const int64_t Mp = pad128(n);
    if (rc == PASUR_OK) rc = ensure_rows(M, Mp);
    if (rc == PASUR_OK) rc = cudaMemsetAsync(M->grad, 0, sizeof(float) * kParams, ctx->stream) == cudaSuccess ? PASUR_OK : PASUR_ECUDA;
    if (rc == PASUR_OK) rc = cudaMemsetAsync(M->loss_d, 0, sizeof(float), ctx->stream) == cudaSuccess ? PASUR_OK : PASUR_ECUDA;
    if (rc == PASUR_OK) rc = pack(M, (const __nv_bfloat16 *)xd, (const float *)yd, nullptr, 0, n, Mp, true);
    if (rc == PASUR_OK) rc = run_pass(M, Mp, n, true);
    if (rc == PASUR_OK) rc = check_err(M);
    if (rc == PASUR_OK && loss_out) rc = copy_to(ctx, loss_out, M->loss_d, sizeof(float));
    if (rc == PASUR_OK && grads_out) rc = copy_to(ctx, grads_out, M->grad, sizeof(float) * kParams);
    free_tmp(ctx, tmp);
    return rc;
}

int pasur_mlp_dataset_add_tree(pasur_mlp *M, const pasur_tree *t) {
    if (!M || !t) return PASUR_EINVAL;
    pasur_ctx *ctx = M->ctx;
    if (t->ctx != ctx) return set_err(ctx, PASUR_EINVAL, "pasur_mlp_dataset_add_tree: tree from another context");
    if (!t->cfr_ready || t->iters_done < 1) return set_err(ctx, PASUR_EINVAL, "pasur_mlp_dataset_add_tree: the tree has no solved utilities");
    const int64_t q0 = t->Q[0];
    if (M->n + q0 > M->cap) return set_err(ctx, PASUR_EOVERFLOW, "pasur_mlp_dataset_add_tree: dataset capacity exceeded");
    cudaSetDevice(ctx->device);
    // the tree's root pools (host) from its level-0 states
    std::vector<GTState> st((size_t)t->n_roots);
    PASUR_CUDA(ctx, cudaMemcpyAsync(st.data(), t->st[0], sizeof(GTState) * st.size(), cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<pasur_score> sc((size_t)q0);
    PASUR_CUDA(ctx, cudaMemcpyAsync(sc.data(), t->scores_d, sizeof(pasur_score) * sc.size(), cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<uint64_t> pools(st.size());
    for (size_t i = 0; i < st.size(); i++) pools[i] = st[i].pool;
    std::vector<std::pair<void *, size_t>> tmp;
    __nv_bfloat16 *x = nullptr;
    int64_t nr = 0;
    int rc = features_dev(M, t->deck, t->round, pools.data(), t->score_off_h.data(), sc.data(), t->n_roots, &x, &nr, tmp);
    if (rc == PASUR_OK && nr != q0) rc = set_err(ctx, PASUR_EINVAL, "pasur_mlp_dataset_add_tree: score slots disagree with FGT roots");
    if (rc == PASUR_OK && nr > 0) {
        if (cudaMemcpyAsync(M->X + M->n * kHid, x, sizeof(__nv_bfloat16) * (size_t)nr * kHid, cudaMemcpyDeviceToDevice, ctx->stream) !=
            cudaSuccess)
            rc = set_err(ctx, PASUR_ECUDA, "pasur_mlp_dataset_add_tree: copy");
        if (rc == PASUR_OK) rc = cfr_export_utilities(t, M->Y + M->n);
    }
    free_tmp(ctx, tmp);
    if (rc == PASUR_OK) M->n += nr;
    return rc;
}

int pasur_mlp_dataset_add_rows(pasur_mlp *M, const uint16_t *x, const float *y, int64_t n) {
    if (!M || n < 0 || (n > 0 && (!x || !y))) return M ? set_err(M->ctx, PASUR_EINVAL, "pasur_mlp_dataset_add_rows: bad arguments") : PASUR_EINVAL;
    pasur_ctx *ctx = M->ctx;
    if (M->n + n > M->cap) return set_err(ctx, PASUR_EOVERFLOW, "pasur_mlp_dataset_add_rows: dataset capacity exceeded");
    cudaSetDevice(ctx->device);
    if (n == 0) return PASUR_OK;
    PASUR_CUDA(ctx, cudaMemcpyAsync(M->X + M->n * kHid, x, sizeof(uint16_t) * (size_t)n * kHid,
                                    is_device_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(M->Y + M->n, y, sizeof(float) * (size_t)n,
                                    is_device_ptr(y) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    M->n += n;
    if (M->epoch_exec) {
        cudaGraphExecDestroy(M->epoch_exec);
        M->epoch_exec = nullptr;
    }
    return PASUR_OK;
}

int pasur_mlp_dataset_size(const pasur_mlp *M, int64_t *n) {
    if (!M || !n) return PASUR_EINVAL;
    *n = M->n;
    return PASUR_OK;
}

int pasur_mlp_dataset_export(const pasur_mlp *M, int64_t first, int64_t count, uint16_t *x_out, float *y_out) {
    if (!M || first < 0 || count < 0 || first + count > M->n) return M ? set_err(M->ctx, PASUR_EINVAL, "pasur_mlp_dataset_export: range") : PASUR_EINVAL;
    cudaSetDevice(M->ctx->device);
    if (x_out) PASUR_TRY(copy_to(M->ctx, x_out, M->X + first * kHid, sizeof(uint16_t) * (size_t)count * kHid));
    if (y_out) PASUR_TRY(copy_to(M->ctx, y_out, M->Y + first, sizeof(float) * (size_t)count));
    return PASUR_OK;
}

int pasur_mlp_dataset_clear(pasur_mlp *M) {
    if (!M) return PASUR_EINVAL;
    M->n = 0;
    if (M->epoch_exec) {
        cudaGraphExecDestroy(M->epoch_exec);
        M->epoch_exec = nullptr;
    }
    return PASUR_OK;
}

int pasur_mlp_train(pasur_mlp *M, int epochs, int64_t batch, float lr, uint64_t shuffle_seed, float *epoch_loss_out) {
    if (!M) return PASUR_EINVAL;
    pasur_ctx *ctx = M->ctx;
    if (epochs < 0 || batch < 128 || batch % 128 != 0 || batch > (1 << 16) || !(lr > 0.f))
        return set_err(ctx, PASUR_EINVAL, "pasur_mlp_train: epochs >= 0, batch a multiple of 128 in 128..65536, lr > 0");
    if (M->n < 1) return set_err(ctx, PASUR_EINVAL, "pasur_mlp_train: empty dataset");
    cudaSetDevice(ctx->device);
    PASUR_TRY(ensure_rows(M, batch));
    const int64_t n = M->n, steps = (n + batch - 1) / batch;
    // one CUDA graph per epoch: (pack batch i through the permutation, forward, backward, Adam) x steps
    if (!M->epoch_exec || M->epoch_batch != batch || M->epoch_rows != n) {
        if (M->epoch_exec) cudaGraphExecDestroy(M->epoch_exec);
        M->epoch_exec = nullptr;
        PASUR_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        int rc = PASUR_OK;
        for (int64_t s = 0; s < steps && rc == PASUR_OK; s++) {
            const int64_t r0 = s * batch, m = std::min(batch, n - r0);
            rc = pack(M, M->X, M->Y, M->perm_d, r0, m, batch, true);
            if (rc == PASUR_OK) rc = run_pass(M, batch, m, true);
            if (rc == PASUR_OK) {
                k_adam<<<(kParams + 255) / 256, 256, 0, ctx->stream>>>(M->p, M->grad, M->m, M->v, M->t_d, s + 1, lr, 0.9f, 0.999f,
                                                                     1e-8f, M->W, M->WT);
                ctx->launches++;
                if (cudaGetLastError() != cudaSuccess) rc = set_err(ctx, PASUR_ECUDA, "k_adam launch");
            }
        }
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &gr);
        if (rc != PASUR_OK) {
            if (gr) cudaGraphDestroy(gr);
            return rc;
        }
        if (e != cudaSuccess) return cuda_err(ctx, e, "pasur_mlp_train: capture");
        cudaError_t ie = cudaGraphInstantiate(&M->epoch_exec, gr, 0);
        cudaGraphDestroy(gr);
        if (ie != cudaSuccess) return cuda_err(ctx, ie, "pasur_mlp_train: instantiate");
        M->epoch_batch = batch;
        M->epoch_rows = n;
    }
    PASUR_CUDA(ctx, cudaMemsetAsync(M->grad, 0, sizeof(float) * kParams, ctx->stream));
    const int64_t launches_per_epoch = steps * 10;
    std::vector<int64_t> perm((size_t)n);
    uint64_t x = shuffle_seed;
    cudaEvent_t e0, e1;
    PASUR_CUDA(ctx, cudaEventCreate(&e0));
    PASUR_CUDA(ctx, cudaEventCreate(&e1));
    PASUR_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    for (int ep = 0; ep < epochs; ep++) {
        // Fisher-Yates shuffle of the rows (splitmix64 draws, multiply-shift bound)
        for (int64_t i = 0; i < n; i++) perm[(size_t)i] = i;
        for (int64_t i = n - 1; i > 0; i--) {
            uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
            z ^= z >> 31;
            const int64_t j = (int64_t)(((unsigned __int128)z * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
            std::swap(perm[(size_t)i], perm[(size_t)j]);
        }
        const int64_t tb = M->steps;
        PASUR_CUDA(ctx, cudaMemcpyAsync(M->perm_d, perm.data(), sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, ctx->stream));
        PASUR_CUDA(ctx, cudaMemcpyAsync(M->t_d, &tb, sizeof tb, cudaMemcpyHostToDevice, ctx->stream));
        PASUR_CUDA(ctx, cudaMemsetAsync(M->loss_d, 0, sizeof(float), ctx->stream));
        PASUR_CUDA(ctx, cudaGraphLaunch(M->epoch_exec, ctx->stream));
        ctx->launches += launches_per_epoch;
        M->steps += steps;
        float l = 0.f;
        PASUR_CUDA(ctx, cudaMemcpyAsync(&l, M->loss_d, sizeof l, cudaMemcpyDeviceToHost, ctx->stream));
        PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (epoch_loss_out) epoch_loss_out[ep] = l / (float)steps;  // mean of the batch losses
    }
    PASUR_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    PASUR_CUDA(ctx, cudaEventSynchronize(e1));
    PASUR_CUDA(ctx, cudaEventElapsedTime(&M->last_train_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return check_err(M);
}

int pasur_mlp_predict_next(pasur_mlp *M, const pasur_tree *t, float *out, int64_t cap) {
    if (!M || !t) return PASUR_EINVAL;
    pasur_ctx *ctx = M->ctx;
    if (t->ctx != ctx) return set_err(ctx, PASUR_EINVAL, "pasur_mlp_predict_next: tree from another context");
    if (t->final_round || !t->has_next) return set_err(ctx, PASUR_EINVAL, "pasur_mlp_predict_next: needs a non-final tree after pasur_next_roots");
    const int64_t nr = t->n_next_roots;
    if (!out || cap < nr) return set_err(ctx, PASUR_EOVERFLOW, "pasur_mlp_predict_next: need " + std::to_string(nr) + " floats");
    cudaSetDevice(ctx->device);
    std::vector<std::pair<void *, size_t>> tmp;
    __nv_bfloat16 *x = nullptr;
    int64_t n = 0;
    int rc = features_dev(M, t->deck, t->round + 1, t->next_pools_h.data(), t->next_soff_h.data(), t->next_scores_h.data(),
                          (int64_t)t->next_pools_h.size(), &x, &n, tmp);
    float *yd = nullptr;
    const bool dev = is_device_ptr(out);
    if (rc == PASUR_OK && !dev) {
        void *p = nullptr;
        rc = dev_alloc(ctx, &p, sizeof(float) * (size_t)(n + 1));
        if (rc == PASUR_OK) tmp.push_back({p, sizeof(float) * (size_t)(n + 1)}), yd = (float *)p;
    }
    if (rc == PASUR_OK && dev) yd = out;
    if (rc == PASUR_OK) rc = forward_rows(M, x, n, yd);
    if (rc == PASUR_OK) rc = check_err(M);
    if (rc == PASUR_OK && !dev) rc = copy_to(ctx, out, yd, sizeof(float) * (size_t)n);
    free_tmp(ctx, tmp);
    return rc;
}

int pasur_mlp_root_features(pasur_ctx *ctx, const uint8_t *deck, int round, const uint64_t *pools, const int64_t *score_offs,
                            const pasur_score *scores, int64_t n_pools, uint16_t *x_out) {
    if (!ctx || !deck || !pools || !score_offs || !scores || !x_out || n_pools < 0 || round < 0 || round > 5)
        return ctx ? set_err(ctx, PASUR_EINVAL, "pasur_mlp_root_features: bad arguments") : PASUR_EINVAL;
    cudaSetDevice(ctx->device);
    pasur_mlp tmpm;
    tmpm.ctx = ctx;
    std::vector<std::pair<void *, size_t>> tmp;
    __nv_bfloat16 *x = nullptr;
    int64_t n = 0;
    int rc = features_dev(&tmpm, deck, round, pools, score_offs, scores, n_pools, &x, &n, tmp);
    if (rc == PASUR_OK && n > 0) rc = copy_to(ctx, x_out, x, sizeof(uint16_t) * (size_t)n * kHid);
    free_tmp(ctx, tmp);
    return rc;
}

int pasur_mlp_stats(const pasur_mlp *M, float *last_train_ms, int64_t *adam_steps) {
    if (!M) return PASUR_EINVAL;
    if (last_train_ms) *last_train_ms = M->last_train_ms;
    if (adam_steps) *adam_steps = M->steps;
    return PASUR_OK;
}

}  // extern "C"

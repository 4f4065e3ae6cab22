// Checkpoint and resume of a round's CFR state.  The paper keeps every round's tensors in host
// memory between the rounds of a deal and stores the solved strategy profiles (section
// "Experimental Evaluation"); here a round can also stop and resume mid-run: its regrets R,
// strategy sums S, root-value sums and iteration count go to a host buffer and back.  A header of
// sizes and an order-independent hash of the round's leaf values make a checkpoint refuse a tree
// that was built, unfolded or given next-round utilities differently.
#include <cstring>

#include "pasur_internal.cuh"

namespace pasur {
namespace {

constexpr uint64_t kCkptMagic = 0x3154504B43525350ull;  // "PSRCKPT1", little-endian

struct CkptHeader {
    uint64_t magic;
    int32_t round, variant;
    int64_t n_roots, iters_done, data_size, n_uacc, n_leaves;
    int64_t cQ[9];
    int64_t swept_edges, swept_pairs;
    uint64_t leaf_hash;
};

// sum over i of (w[i] + 1) * (2 i + 1) mod 2^64: changes with any word or its position, and is
// independent of the order in which the terms are added
__global__ void k_word_hash(const uint32_t *__restrict__ w, int64_t n, unsigned long long *out) {
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += ((unsigned long long)w[i] + 1ull) * (2ull * (unsigned long long)i + 1ull);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

int leaf_hash(const pasur_tree *t, uint64_t *h) {
    pasur_ctx *ctx = t->ctx;
    unsigned long long *d = nullptr;
    PASUR_TRY(dev_alloc(ctx, (void **)&d, sizeof(unsigned long long)));
    int rc = PASUR_OK;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), ctx->stream);
    const int64_t n = t->cQ[8];
    if (e == cudaSuccess && n > 0) {
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
        k_word_hash<<<(unsigned)blocks, 256, 0, ctx->stream>>>((const uint32_t *)t->leaf_v, n, d);
        ctx->launches++;
        e = cudaGetLastError();
    }
    unsigned long long v = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, d, sizeof v, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = cuda_err(ctx, e, "checkpoint: leaf hash");
    dev_free(ctx, d, sizeof(unsigned long long));
    *h = v;
    return rc;
}

int make_header(const pasur_tree *t, CkptHeader *hd) {
    std::memset(hd, 0, sizeof *hd);
    hd->magic = kCkptMagic;
    hd->round = t->round;
    hd->variant = t->variant;
    hd->n_roots = t->n_roots;
    hd->iters_done = t->iters_done;
    hd->data_size = t->data_size;
    hd->n_uacc = t->cQ[0];
    hd->n_leaves = t->cQ[8];
    for (int k = 0; k < 9; k++) hd->cQ[k] = t->cQ[k];
    hd->swept_edges = t->swept_edges;
    hd->swept_pairs = t->swept_pairs;
    return leaf_hash(t, &hd->leaf_hash);
}

int tree_ok(const pasur_tree *t) { return t && t->ctx ? PASUR_OK : PASUR_EINVAL; }

size_t ckpt_bytes(const CkptHeader &hd) {
    return sizeof(CkptHeader) + 2 * sizeof(float) * (size_t)hd.data_size + sizeof(double) * (size_t)hd.n_uacc;
}

}  // namespace
}  // namespace pasur

using namespace pasur;

int pasur_save_round(const pasur_tree *t, void *buf, size_t cap, size_t *bytes) {
    if (tree_ok(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    cudaSetDevice(ctx->device);
    if (!t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_save_round: no CFR run yet");
    if (!buf && !bytes) return set_err(ctx, PASUR_EINVAL, "pasur_save_round: buf and bytes are NULL");
    CkptHeader hd;
    PASUR_TRY(make_header(t, &hd));
    const size_t need = ckpt_bytes(hd);
    if (bytes) *bytes = need;
    if (!buf) return PASUR_OK;
    if (cap < need) return set_err(ctx, PASUR_EINVAL, "pasur_save_round: cap < " + std::to_string(need) + " bytes");
    char *p = (char *)buf;
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    const size_t fb = sizeof(float) * (size_t)hd.data_size;
    PASUR_CUDA(ctx, cudaMemcpyAsync(p, t->R, fb, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(p + fb, t->S, fb, cudaMemcpyDeviceToHost, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(p + 2 * fb, t->uacc, sizeof(double) * (size_t)hd.n_uacc, cudaMemcpyDeviceToHost,
                                    ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PASUR_OK;
}

int pasur_load_round(pasur_tree *t, const void *buf, size_t bytes) {
    if (tree_ok(t)) return PASUR_EINVAL;
    pasur_ctx *ctx = t->ctx;
    cudaSetDevice(ctx->device);
    if (!t->cfr_ready) return set_err(ctx, PASUR_EINVAL, "pasur_load_round: set the tree up first (pasur_cfr_iterate, iters 0)");
    if (!buf || bytes < sizeof(CkptHeader)) return set_err(ctx, PASUR_EINVAL, "pasur_load_round: no checkpoint header");
    CkptHeader in;
    std::memcpy(&in, buf, sizeof in);
    CkptHeader mine;
    PASUR_TRY(make_header(t, &mine));
    if (in.magic != kCkptMagic) return set_err(ctx, PASUR_EINVAL, "pasur_load_round: not a round checkpoint");
    if (bytes < ckpt_bytes(in)) return set_err(ctx, PASUR_EINVAL, "pasur_load_round: checkpoint truncated");
    bool same = in.round == mine.round && in.variant == mine.variant && in.n_roots == mine.n_roots &&
                in.data_size == mine.data_size && in.n_uacc == mine.n_uacc && in.n_leaves == mine.n_leaves &&
                in.swept_edges == mine.swept_edges && in.swept_pairs == mine.swept_pairs && in.leaf_hash == mine.leaf_hash;
    for (int k = 0; k < 9; k++) same = same && in.cQ[k] == mine.cQ[k];
    if (!same)
        return set_err(ctx, PASUR_EINVAL, "pasur_load_round: the checkpoint is of another round, layout, variant or leaf values");
    if (in.iters_done < 0) return set_err(ctx, PASUR_EINVAL, "pasur_load_round: bad iteration count");
    const char *p = (const char *)buf + sizeof in;
    const size_t fb = sizeof(float) * (size_t)in.data_size;
    PASUR_CUDA(ctx, cudaMemcpyAsync(t->R, p, fb, cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(t->S, p + fb, fb, cudaMemcpyHostToDevice, ctx->stream));
    PASUR_CUDA(ctx, cudaMemcpyAsync(t->uacc, p + 2 * fb, sizeof(double) * (size_t)in.n_uacc, cudaMemcpyHostToDevice,
                                    ctx->stream));
    PASUR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    t->iters_done = in.iters_done;
    return PASUR_OK;
}

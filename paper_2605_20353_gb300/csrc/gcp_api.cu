// gcp_api.cu -- the C ABI of include/gcp.h: context set-up, argument checks,
// the stratified weights of Sec. 3.1.1, kernel launches and the GCP-Adam
// epoch loop (Algorithm 2 on one GPU).
#include <cuda_bf16.h>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "gcp_internal.h"

namespace {

thread_local std::string g_create_err;

struct DeviceGuard {  // make the context's device current for one call
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

gcp_status fail(gcp_ctx *c, gcp_status code, const std::string &msg) {
    if (c)
        c->err = msg;
    else
        g_create_err = msg;
    return code;
}

gcp_status cuda_fail(gcp_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? GCP_ERR_OOM : GCP_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define GCP_CUDA(ctx, call)                                      \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

uint64_t next_pow2(uint64_t v) {
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// status word -> first gcp_status code set
gcp_status status_code(int bits) {
    for (int c = 1; c < 31; ++c)
        if (bits & (1 << c)) return (gcp_status)c;
    return GCP_OK;
}

const char *status_text(gcp_status s) {
    switch (s) {
    case GCP_ERR_DUPLICATE: return "duplicate nonzero coordinates";
    case GCP_ERR_HASH_FULL: return "nonzero hash set is full";
    case GCP_ERR_SAMPLER_EXHAUSTED: return "a zero draw hit nonzeros max_attempts times (tensor too dense)";
    case GCP_ERR_NONFINITE: return "non-finite loss";
    case GCP_ERR_ARG: return "non-finite value in the dense tensor";
    case GCP_ERR_DOMAIN: return "value outside the loss's domain";
    default: return "device error";
    }
}

// Read and clear the device status word; synchronises the stream.
gcp_status collect(gcp_ctx *c) {
    GCP_CUDA(c, cudaMemcpyAsync(c->h_status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    GCP_CUDA(c, cudaStreamSynchronize(c->st));
    const int bits = *c->h_status;
    if (bits) {
        GCP_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
        const gcp_status s = status_code(bits);
        return fail(c, s, status_text(s));
    }
    return GCP_OK;
}

void destroy_buffers(gcp_ctx *c) {
    cudaFree(c->rec);
    cudaFree(c->hkeys);
    cudaFree(c->X);
    cudaFree(c->A);
    cudaFree(c->Abf);
    cudaFree(c->G);
    cudaFree(c->B);
    cudaFree(c->C);
    cudaFree(c->partials);
    cudaFree(c->dloss);
    cudaFree(c->status);
    cudaFree(c->det_scratch);
    if (c->det_side) cudaStreamDestroy(c->det_side);
    if (c->det_fork) cudaEventDestroy(c->det_fork);
    if (c->det_join) cudaEventDestroy(c->det_join);
    cudaFree(c->nf_coord);
    cudaFree(c->nf_val);
    cudaFree(c->hot_slot);
    cudaFree(c->hot_row);
    cudaFree(c->Grep);
    cudaFree(c->bk_A);
    cudaFree(c->bk_B);
    cudaFree(c->bk_C);
    cudaFreeHost(c->h_status);
    cudaFreeHost(c->h_loss);
    for (auto &ev : c->prof_ev) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    c->prof_ev.clear();
}

// Event pair for the next timed launch (reused across reads).
gcp_status prof_begin(gcp_ctx *c, cudaEvent_t *stop) {
    *stop = nullptr;
    if (!c->prof) return GCP_OK;
    if (c->prof_used == c->prof_ev.size()) {
        std::pair<cudaEvent_t, cudaEvent_t> ev;
        GCP_CUDA(c, cudaEventCreate(&ev.first));
        GCP_CUDA(c, cudaEventCreate(&ev.second));
        c->prof_ev.push_back(ev);
    }
    auto &ev = c->prof_ev[c->prof_used++];
    GCP_CUDA(c, cudaEventRecord(ev.first, c->st));
    *stop = ev.second;
    return GCP_OK;
}

// Shape, options and model buffers common to sparse and dense contexts.
gcp_status init_common(gcp_ctx *c, int32_t ndim, const int64_t *dims, int32_t rank, int32_t loss,
                       const gcp_options *opt) {
    if (ndim < 2 || ndim > GCP_MAX_NDIM) return fail(nullptr, GCP_ERR_ARG, "ndim must be in 2..8");
    if (!dims) return fail(nullptr, GCP_ERR_ARG, "dims is NULL");
    if (rank < 1 || rank > GCP_MAX_RANK) return fail(nullptr, GCP_ERR_ARG, "rank must be in 1..128");
    if (loss < GCP_GAUSSIAN || loss > GCP_GAMMA) return fail(nullptr, GCP_ERR_ARG, "unknown loss");
    gcp_options_default(&c->opt);
    if (opt) c->opt = *opt;
    if (c->opt.factor_dtype != GCP_FP32 && c->opt.factor_dtype != GCP_BF16)
        return fail(nullptr, GCP_ERR_ARG, "unknown factor dtype");
    if (c->opt.mttkrp != GCP_MTTKRP_ATOMIC && c->opt.mttkrp != GCP_MTTKRP_DETERMINISTIC &&
        c->opt.mttkrp != GCP_MTTKRP_NONFUSED)
        return fail(nullptr, GCP_ERR_ARG, "unknown MTTKRP variant");
    if (c->opt.max_attempts < 0) return fail(nullptr, GCP_ERR_ARG, "max_attempts < 0");
    if (c->opt.max_attempts == 0) c->opt.max_attempts = 64;
    if (c->opt.hash_max_load == 0.0) c->opt.hash_max_load = 0.3;
    if (!(c->opt.hash_max_load > 0.0 && c->opt.hash_max_load <= 0.5))
        return fail(nullptr, GCP_ERR_ARG, "hash_max_load must be in (0, 0.5]");
    c->d = ndim;
    c->R = rank;
    c->loss = loss;
    c->st = static_cast<cudaStream_t>(c->opt.stream);
    cudaGetDevice(&c->device);
    unsigned __int128 M = 1;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 1 || dims[k] > INT32_MAX) return fail(nullptr, GCP_ERR_ARG, "mode size out of range");
        c->dims[k] = dims[k];
        M *= (unsigned __int128)dims[k];
        if (M >= ((unsigned __int128)1 << 63)) return fail(nullptr, GCP_ERR_ARG, "prod(dims) must be < 2^63");
    }
    c->M = (double)(uint64_t)M;
    c->stride[ndim - 1] = 1;
    for (int k = ndim - 2; k >= 0; --k) c->stride[k] = c->stride[k + 1] * (uint64_t)dims[k + 1];
    c->total_rows = 0;
    for (int k = 0; k < ndim; ++k) {
        c->rowoff[k] = c->total_rows;
        c->total_rows += dims[k];
    }
    // Row length padded to 4 x a power of two.  A lane owns 4 columns when a
    // row is at most 32 floats (a group's reduction covers the whole
    // 128-byte row), else 8 (two half rows of >= 128 bytes).
    int Rp = 4;
    while (Rp < rank) Rp <<= 1;
    c->Rp = Rp;
    c->cols = Rp >= 64 ? 8 : 4;
    if (c->opt.lane_cols == 4 || (c->opt.lane_cols == 8 && Rp >= 8)) c->cols = c->opt.lane_cols;
    else if (c->opt.lane_cols != 0) return fail(nullptr, GCP_ERR_ARG, "lane_cols must be 0, 4 or 8");
    int L = Rp / c->cols, log2L = 0;
    while ((1 << log2L) < L) ++log2L;
    c->log2L = log2L;
    if ((double)c->total_rows * c->Rp >= 2147483647.0)
        return fail(nullptr, GCP_ERR_ARG, "sum of mode sizes x padded rank must be < 2^31");

    const size_t nparam = (size_t)c->total_rows * c->Rp;
    cudaError_t e;
    if ((e = cudaMalloc(&c->A, nparam * 4)) || (e = cudaMalloc(&c->G, nparam * 4)) ||
        (e = cudaMalloc(&c->B, nparam * 4)) || (e = cudaMalloc(&c->C, nparam * 4)) ||
        (e = cudaMalloc(&c->dloss, 4 * sizeof(double))) || (e = cudaMalloc(&c->status, sizeof(int))) ||
        (e = cudaMallocHost(&c->h_status, sizeof(int))) || (e = cudaMallocHost(&c->h_loss, 4 * sizeof(double))))
        return cuda_fail(nullptr, e, "allocating model buffers");
    if (c->opt.factor_dtype == GCP_BF16 && (e = cudaMalloc(&c->Abf, nparam * 2)))
        return cuda_fail(nullptr, e, "allocating BF16 factors");
    c->max_blocks = gcpk::fused_max_blocks(ndim, c->opt.factor_dtype == GCP_BF16, c->cols);
    if ((e = cudaMalloc(&c->partials, (size_t)c->max_blocks * 4 * sizeof(double))))
        return cuda_fail(nullptr, e, "allocating partials");
    if ((e = cudaMemsetAsync(c->A, 0, nparam * 4, c->st)) || (e = cudaMemsetAsync(c->G, 0, nparam * 4, c->st)) ||
        (e = cudaMemsetAsync(c->B, 0, nparam * 4, c->st)) || (e = cudaMemsetAsync(c->C, 0, nparam * 4, c->st)) ||
        (e = cudaMemsetAsync(c->status, 0, sizeof(int), c->st)) ||
        (c->Abf && (e = cudaMemsetAsync(c->Abf, 0, nparam * 2, c->st))))
        return cuda_fail(nullptr, e, "clearing model buffers");
    return GCP_OK;
}

gcpk::SampleSpec sample_spec(const gcp_ctx *c, uint64_t iter, int64_t p, int64_t q) {
    gcpk::SampleSpec s{};
    s.d = c->d;
    for (int k = 0; k < c->d; ++k) {
        s.dims[k] = c->dims[k];
        s.stride[k] = c->stride[k];
    }
    s.nnz = c->nnz;
    s.rec = c->rec;
    s.rec_words = c->rec_words;
    s.hkeys = c->hkeys;
    s.hbmask = c->hbmask;
    s.dense = c->X;
    s.seed = c->opt.seed;
    s.iter = iter;
    s.p = p;
    s.q = q;
    s.sampling = c->opt.sampling;
    s.max_attempts = c->opt.max_attempts;
    s.status = c->status;
    return s;
}

// Per-sample weights of Sec. 3.1.1: N/p for nonzeros, (M-N)/q for zeros;
// semi-stratified zero candidates cover all M cells (M/q); dense uniform
// sampling weighs each of the p cells M/p.
void weights(const gcp_ctx *c, int64_t p, int64_t q, double &w_nz, double &w_z) {
    if (c->opt.sampling == GCP_SAMPLING_UNIFORM) {
        w_nz = p > 0 ? c->M / (double)p : 0.0;
        w_z = 0.0;
        return;
    }
    w_nz = p > 0 ? (double)c->nnz / (double)p : 0.0;
    if (c->opt.sampling == GCP_SAMPLING_SEMI_STRATIFIED)
        w_z = q > 0 ? c->M / (double)q : 0.0;
    else
        w_z = q > 0 ? (c->M - (double)c->nnz) / (double)q : 0.0;
}

gcp_status check_counts(gcp_ctx *c, int64_t p, int64_t q) {
    if (p < 0 || q < 0) return fail(c, GCP_ERR_ARG, "negative sample count");
    if (c->dense && q != 0) return fail(c, GCP_ERR_ARG, "dense tensors take p uniform samples and q = 0");
    if (p + q >= ((int64_t)1 << 31)) return fail(c, GCP_ERR_ARG, "p + q must be below 2^31 per call");
    return GCP_OK;
}

// One fused pass: loss always, gradient into c->G when `grad`.
}  // namespace

// The fused-pass parameters of one sample set of a context (also used for
// each client of a batch).
gcpk::FusedSpec gcpk_make_spec(const gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, bool grad,
                               const float *dscale, double *w_nz_out, double *w_z_out) {
    double w_nz, w_z;
    weights(c, p, q, w_nz, w_z);
    gcpk::FusedSpec f{};
    f.s = sample_spec(c, iter, p, q);
    f.F = c->Abf ? c->Abf : (const void *)c->A;
    f.G = grad ? c->G : nullptr;
    f.Rp = c->Rp;
    f.log2L = c->log2L;
    for (int k = 0; k < c->d; ++k) f.rowoff[k] = (int)c->rowoff[k];
    f.loss = c->loss;
    f.w_nz = (float)w_nz;
    f.w_z = (float)w_z;
    f.dscale = dscale;
    f.partials = c->partials;
    for (int k = 0; k < c->d; ++k) f.small_base[k] = c->small_base[k];
    f.Grep = c->Grep;
    f.Htot = c->Htot;
    if (w_nz_out) *w_nz_out = w_nz;
    if (w_z_out) *w_z_out = w_z;
    return f;
}

gcp_status gcpk_check_counts(gcp_ctx *c, int64_t p, int64_t q) { return check_counts(c, p, q); }

namespace {

gcp_status run_fused(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, bool grad, const float *dscale) {
    gcp_status s = check_counts(c, p, q);
    if (s) return s;
    double w_nz, w_z;
    gcpk::FusedSpec f = gcpk_make_spec(c, iter, p, q, grad, dscale, &w_nz, &w_z);
    if (grad) {
        GCP_CUDA(c, cudaMemsetAsync(c->G, 0, (size_t)c->total_rows * c->Rp * 4, c->st));
        c->g_clear = false;
    }
    int blocks = 0;
    cudaEvent_t stop = nullptr;
    if ((s = prof_begin(c, &stop))) return s;
    if (grad && c->opt.mttkrp == GCP_MTTKRP_DETERMINISTIC) {
        s = gcpk_det_grad(c, f, &blocks);
        if (s) return s;
    } else if (grad && c->opt.mttkrp == GCP_MTTKRP_NONFUSED) {
        const int64_t S = p + q;
        if (S > c->nf_cap) {  // grow the gradient-tensor buffers
            cudaFree(c->nf_coord);
            cudaFree(c->nf_val);
            c->nf_coord = nullptr;
            c->nf_val = nullptr;
            c->nf_cap = 0;
            GCP_CUDA(c, cudaMalloc(&c->nf_coord, (size_t)S * c->d * 4));
            GCP_CUDA(c, cudaMalloc(&c->nf_val, (size_t)S * 4));
            c->nf_cap = S;
        }
        gcpk::FusedSpec m = f;  // pass 1: sampling, model, loss; writes the gradient tensor
        m.G = nullptr;
        m.Ycoord = c->nf_coord;
        m.Yval = c->nf_val;
        m.ystride = c->d;
        m.vstride = 1;
        GCP_CUDA(c, gcpk::launch_fused(m, c->Abf != nullptr, c->cols, c->max_blocks, c->st, &blocks));
        m.G = c->G;  // pass 2: MTTKRP of the stored gradient tensor
        GCP_CUDA(c, gcpk::launch_mttkrp_nonfused(m, c->hot_slot, c->Abf != nullptr, c->cols, c->max_blocks, c->st));
    } else {
        GCP_CUDA(c, gcpk::launch_fused(f, c->Abf != nullptr, c->cols, c->max_blocks, c->st, &blocks));
    }
    if (stop) GCP_CUDA(c, cudaEventRecord(stop, c->st));
    if (grad && c->opt.mttkrp != GCP_MTTKRP_DETERMINISTIC)
        GCP_CUDA(c, gcpk::launch_fold_replicas(c->G, c->Grep, c->hot_row, c->Htot, c->Rp, c->st));
    GCP_CUDA(c, gcpk::launch_finish_loss(c->partials, blocks, w_nz, w_z, c->dloss, c->status, c->st));
    return GCP_OK;
}

gcp_status adam_step_impl(gcp_ctx *c, const gcp_adam_params *prm, int64_t t) {
    if (t < 1) return fail(c, GCP_ERR_ARG, "Adam step t must be >= 1");
    if (!(prm->beta1 >= 0.0 && prm->beta1 < 1.0 && prm->beta2 >= 0.0 && prm->beta2 < 1.0 && prm->eps >= 0.0))
        return fail(c, GCP_ERR_ARG, "Adam parameters out of range");
    DeviceGuard g(c->device);
    const double c1 = 1.0 - std::pow(prm->beta1, (double)t), c2 = 1.0 - std::pow(prm->beta2, (double)t);
    GCP_CUDA(c, gcpk::launch_adam((int64_t)c->total_rows * c->Rp, c->Rp, c->R, c->A, c->B, c->C, c->G,
                                  (float)prm->lr, (float)prm->beta1, (float)prm->beta2, (float)(1.0 / c1),
                                  (float)(1.0 / c2), (float)prm->eps, (float)prm->lower, c->Abf, c->st));
    return GCP_OK;
}


// One training step: sampled gradient of iteration `iter` and Adam step t.
// With the atomic MTTKRP the epilogue (replica fold, loss finish, Adam, G
// cleared for the next step) is one launch after the fused pass.
gcp_status do_step(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, const gcp_adam_params *prm, int64_t t) {
    gcp_status s;
    if (c->opt.mttkrp != GCP_MTTKRP_ATOMIC) {
        if ((s = run_fused(c, iter, p, q, true, nullptr))) return s;
        return adam_step_impl(c, prm, t);
    }
    if ((s = check_counts(c, p, q))) return s;
    double w_nz, w_z;
    const gcpk::FusedSpec f = gcpk_make_spec(c, iter, p, q, true, nullptr, &w_nz, &w_z);
    if (!c->g_clear) GCP_CUDA(c, cudaMemsetAsync(c->G, 0, (size_t)c->total_rows * c->Rp * 4, c->st));
    int blocks = 0;
    cudaEvent_t stop = nullptr;
    if ((s = prof_begin(c, &stop))) return s;
    GCP_CUDA(c, gcpk::launch_fused(f, c->Abf != nullptr, c->cols, c->max_blocks, c->st, &blocks));
    if (stop) GCP_CUDA(c, cudaEventRecord(stop, c->st));
    const double c1 = 1.0 - std::pow(prm->beta1, (double)t), c2 = 1.0 - std::pow(prm->beta2, (double)t);
    gcpk::PostSpec ps{};
    ps.n = (int64_t)c->total_rows * c->Rp;
    ps.Rp = c->Rp;
    ps.R = c->R;
    ps.Htot = c->Htot;
    ps.G = c->G;
    ps.Grep = c->Grep;
    ps.A = c->A;
    ps.B = c->B;
    ps.C = c->C;
    ps.Abf = c->Abf;
    ps.hot_slot = c->hot_slot;
    ps.hot_row = c->hot_row;
    ps.lr = (float)prm->lr;
    ps.beta1 = (float)prm->beta1;
    ps.beta2 = (float)prm->beta2;
    ps.c1inv = (float)(1.0 / c1);
    ps.c2inv = (float)(1.0 / c2);
    ps.eps = (float)prm->eps;
    ps.lower = (float)prm->lower;
    ps.partials = c->partials;
    ps.nblocks = blocks;
    ps.w_nz = w_nz;
    ps.w_z = w_z;
    ps.dloss = c->dloss;
    ps.status = c->status;
    GCP_CUDA(c, gcpk::launch_post_step(ps, c->st));
    c->g_clear = true;
    return GCP_OK;
}

// Values of a dense tensor: bit GCP_ERR_ARG for a non-finite value, bit
// GCP_ERR_DOMAIN for one outside the loss's domain (the host checks of a
// sparse tensor's values, on the device).
__global__ void k_check_dense(const float *X, int64_t n, int loss, int *status) {
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = X[i];
        if (!isfinite(x))
            bad |= 1 << GCP_ERR_ARG;
        else if ((loss == GCP_POISSON && x < 0.0f) || (loss == GCP_GAMMA && x <= 0.0f) ||
                 (loss == GCP_BERNOULLI_LOGIT && x != 1.0f && x != 0.0f))
            bad |= 1 << GCP_ERR_DOMAIN;
    }
    if (bad) atomicOr(status, bad);
}

// Every mode's factor matrix (src.A[k], I_k x R row-major, device memory)
// copied into the context's padded flat layout in one launch; padding
// columns are written as zero and the BF16 copy, if any, is refreshed.
struct FactorSrc {
    const float *A[GCP_MAX_NDIM];
    int64_t rowoff[GCP_MAX_NDIM + 1];  // first row of each mode, then the total
};

__global__ void k_stage_factors(FactorSrc src, int d, int R, int log2Rp, int64_t n, float *__restrict__ A,
                                __nv_bfloat16 *__restrict__ Abf) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e >> log2Rp;
        const int col = (int)(e & ((1 << log2Rp) - 1));
        int k = 0;
        while (k + 1 < d && row >= src.rowoff[k + 1]) ++k;
        const float v = col < R ? __ldg(src.A[k] + (row - src.rowoff[k]) * R + col) : 0.0f;
        A[e] = v;
        if (Abf) Abf[e] = __float2bfloat16_rn(v);
    }
}

// y = s[0] * x elementwise (x and y may be the same array); s is FP64,
// rounded once to FP32.
__global__ void k_scale(const double *s, const float *x, float *y, int64_t n) {
    const float a = (float)__ldg(s);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

// Sum of squares of x[0..n) in FP64: block b adds its grid-stride elements
// in index order per thread, then a fixed tree; partial[b] holds the result.
__global__ void k_sumsq_blocks(const float *__restrict__ x, int64_t n, double *partial) {
    __shared__ double sh[256];
    double t = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        t += v * v;
    }
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// out[0] = sqrt(sum of the block partials), summed in block order; a
// non-finite result sets the status word.
__global__ void k_sumsq_finish(const double *__restrict__ partial, int nblocks, double *out, int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[b];
    out[0] = sqrt(t);
    if (!isfinite(t)) atomicOr(status, 1 << GCP_ERR_NONFINITE);
}

// Copy `rows` rows of `width` bytes between arrays whose rows are dpitch
// and spitch bytes apart.  With equal pitches and no padding the rows are
// one contiguous block and go as one plain copy (the strided form moves
// each row separately).
static cudaError_t copy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t rows,
                      cudaStream_t st) {
    if (dpitch == width && spitch == width)
        return cudaMemcpyAsync(dst, src, width * rows, cudaMemcpyDefault, st);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyDefault, st);
}

gcp_status copy_grad_out(gcp_ctx *c, float *G_out) {
    if (!G_out) return GCP_OK;
    GCP_CUDA(c, copy_rows(G_out, (size_t)c->R * 4, c->G, (size_t)c->Rp * 4, (size_t)c->R * 4,
                                  (size_t)c->total_rows, c->st));
    return GCP_OK;
}

gcp_status read_loss(gcp_ctx *c, double *loss_out) {
    GCP_CUDA(c, cudaMemcpyAsync(c->h_loss, c->dloss, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    gcp_status s = collect(c);
    if (loss_out) *loss_out = c->h_loss[0];
    return s;
}

gcp_status refresh_bf16(gcp_ctx *c) {
    if (!c->Abf) return GCP_OK;
    GCP_CUDA(c, gcpk::launch_to_bf16((int64_t)c->total_rows * c->Rp, c->A, c->Abf, c->st));
    return GCP_OK;
}

// Rows that receive many gradient reductions per call get replicas: every
// row of a mode with at most 512 rows (each is hit by 1/I_k of the drawn
// cells), with contiguous slots so drawn cells find theirs by arithmetic;
// then, for larger modes, rows holding at least 1/512 of the nonzeros (hit
// by that share of the nonzero samples), at most 256 per mode, hottest
// first.  A nonzero record stores the slots of its rows.
gcp_status setup_hot_rows(gcp_ctx *c, const std::vector<int64_t> &counts) {
    std::vector<int> slot((size_t)c->total_rows, -1), row;
    for (int k = 0; k < c->d; ++k) {
        c->small_base[k] = -1;
        if (c->dims[k] > 512) continue;
        c->small_base[k] = (int)row.size();
        for (int64_t i = 0; i < c->dims[k]; ++i) {
            slot[(size_t)(c->rowoff[k] + i)] = (int)row.size();
            row.push_back((int)(c->rowoff[k] + i));
        }
    }
    for (int k = 0; k < c->d && !counts.empty(); ++k) {
        if (c->dims[k] <= 512) continue;
        std::vector<std::pair<int64_t, int>> hot;
        for (int64_t i = 0; i < c->dims[k]; ++i) {
            const int64_t n = counts[(size_t)(c->rowoff[k] + i)];
            if ((double)n * 512.0 >= (double)c->nnz) hot.push_back({n, (int)(c->rowoff[k] + i)});
        }
        std::stable_sort(hot.begin(), hot.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
        if (hot.size() > 256) hot.resize(256);
        for (const auto &h : hot) {
            slot[(size_t)h.second] = (int)row.size();
            row.push_back(h.second);
        }
    }
    c->Htot = (int)row.size();
    if (c->Htot == 0) return GCP_OK;
    const size_t rep_bytes = (size_t)gcpk::kReplicas * c->Htot * c->Rp * 4;
    cudaError_t e;
    if ((e = cudaMalloc(&c->hot_slot, slot.size() * 4)) || (e = cudaMalloc(&c->hot_row, row.size() * 4)) ||
        (e = cudaMalloc(&c->Grep, rep_bytes)) ||
        (e = cudaMemcpy(c->hot_slot, slot.data(), slot.size() * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(c->hot_row, row.data(), row.size() * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemsetAsync(c->Grep, 0, rep_bytes, c->st)))
        return cuda_fail(nullptr, e, "allocating hot-row replicas");
    return GCP_OK;
}

}  // namespace

void gcpk_set_noctx_error(const char *msg) { g_create_err = msg; }

// =================================================================== ABI
extern "C" {

void gcp_options_default(gcp_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->factor_dtype = GCP_FP32;
    opt->mttkrp = GCP_MTTKRP_ATOMIC;
    opt->sampling = GCP_SAMPLING_STRATIFIED;
    opt->max_attempts = 64;
    opt->hash_max_load = 0.3;
}

gcp_status gcp_create(int32_t ndim, const int64_t *dims, int64_t nnz, const int32_t *coords, const float *vals,
                      int32_t rank, int32_t loss, const gcp_options *opt, gcp_ctx **out) {
    if (!out) return fail(nullptr, GCP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nnz < 1 || !coords || !vals) return fail(nullptr, GCP_ERR_ARG, "need nnz >= 1, coords and vals");
    if (opt && opt->sampling == GCP_SAMPLING_UNIFORM)
        return fail(nullptr, GCP_ERR_ARG, "uniform sampling is for dense tensors (gcp_create_dense)");
    // host checks of the nonzeros
    if (ndim >= 2 && ndim <= GCP_MAX_NDIM && dims) {
        for (int64_t e = 0; e < nnz; ++e) {
            for (int k = 0; k < ndim; ++k) {
                const int32_t v = coords[e * ndim + k];
                if (v < 0 || v >= dims[k]) return fail(nullptr, GCP_ERR_ARG, "coordinate out of range");
            }
            const float x = vals[e];
            if (!std::isfinite(x)) return fail(nullptr, GCP_ERR_ARG, "non-finite value");
            if ((loss == GCP_POISSON && x < 0.0f) || (loss == GCP_GAMMA && x <= 0.0f) ||
                (loss == GCP_BERNOULLI_LOGIT && x != 1.0f && x != 0.0f))
                return fail(nullptr, GCP_ERR_DOMAIN, "value outside the loss's domain");
        }
    }
    gcp_ctx *c = new (std::nothrow) gcp_ctx();
    if (!c) return fail(nullptr, GCP_ERR_OOM, "host allocation");
    gcp_status s = init_common(c, ndim, dims, rank, loss, opt);
    if (s) {
        destroy_buffers(c);
        delete c;
        return s;
    }
    if ((double)nnz > c->M) {
        destroy_buffers(c);
        delete c;
        return fail(nullptr, GCP_ERR_ARG, "more nonzeros than cells");
    }
    c->nnz = nnz;
    {
        std::vector<int64_t> counts((size_t)c->total_rows, 0);
        for (int64_t e = 0; e < nnz; ++e)
            for (int k = 0; k < ndim; ++k) ++counts[(size_t)(c->rowoff[k] + coords[e * ndim + k])];
        s = setup_hot_rows(c, counts);
        if (s) {
            destroy_buffers(c);
            delete c;
            return s;
        }
    }
    c->rec_words = gcpk::rec_words_for(ndim);
    const uint64_t cap = next_pow2((uint64_t)std::ceil((double)nnz / c->opt.hash_max_load)) < 4
                             ? 4
                             : next_pow2((uint64_t)std::ceil((double)nnz / c->opt.hash_max_load));
    c->hbmask = cap / 4 - 1;
    int32_t *dcoords = nullptr;
    float *dvals = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&c->rec, (size_t)nnz * c->rec_words * 4)) || (e = cudaMalloc(&c->hkeys, cap * 8)) ||
        (e = cudaMalloc(&dcoords, (size_t)nnz * ndim * 4)) || (e = cudaMalloc(&dvals, (size_t)nnz * 4))) {
        cudaFree(dcoords);
        cudaFree(dvals);
        destroy_buffers(c);
        delete c;
        return cuda_fail(nullptr, e, "allocating nonzero storage");
    }
    if ((e = cudaMemsetAsync(c->hkeys, 0xFF, cap * 8, c->st)) ||
        (e = cudaMemcpyAsync(dcoords, coords, (size_t)nnz * ndim * 4, cudaMemcpyHostToDevice, c->st)) ||
        (e = cudaMemcpyAsync(dvals, vals, (size_t)nnz * 4, cudaMemcpyHostToDevice, c->st)) ||
        (e = gcpk::launch_build_records(dcoords, dvals, nnz, ndim, c->stride, c->rowoff, c->hot_slot,
                                        c->rec_words, c->rec, c->hkeys, c->hbmask, c->status, c->st)) ||
        (e = cudaStreamSynchronize(c->st))) {
        cudaFree(dcoords);
        cudaFree(dvals);
        destroy_buffers(c);
        delete c;
        return cuda_fail(nullptr, e, "building nonzero records");
    }
    cudaFree(dcoords);
    cudaFree(dvals);
    s = collect(c);
    if (s) {
        g_create_err = c->err;
        destroy_buffers(c);
        delete c;
        return s;
    }
    *out = c;
    return GCP_OK;
}

gcp_status gcp_create_dense(int32_t ndim, const int64_t *dims, const float *X, int32_t rank, int32_t loss,
                            const gcp_options *opt, gcp_ctx **out) {
    if (!out) return fail(nullptr, GCP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!X) return fail(nullptr, GCP_ERR_ARG, "X is NULL");
    gcp_ctx *c = new (std::nothrow) gcp_ctx();
    if (!c) return fail(nullptr, GCP_ERR_OOM, "host allocation");
    gcp_options o;
    gcp_options_default(&o);
    if (opt) o = *opt;
    o.sampling = GCP_SAMPLING_UNIFORM;
    gcp_status s = init_common(c, ndim, dims, rank, loss, &o);
    if (s) {
        destroy_buffers(c);
        delete c;
        return s;
    }
    c->dense = true;
    c->nnz = (int64_t)c->M;
    s = setup_hot_rows(c, std::vector<int64_t>());
    if (s) {
        destroy_buffers(c);
        delete c;
        return s;
    }
    const size_t bytes = (size_t)c->M * 4;
    cudaError_t e;
    if ((e = cudaMalloc(&c->X, bytes)) ||
        (e = cudaMemcpyAsync(c->X, X, bytes, cudaMemcpyDefault, c->st))) {
        destroy_buffers(c);
        delete c;
        return cuda_fail(nullptr, e, "copying the dense tensor");
    }
    k_check_dense<<<4096, 256, 0, c->st>>>(c->X, (int64_t)c->M, c->loss, c->status);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        destroy_buffers(c);
        delete c;
        return cuda_fail(nullptr, e, "checking the dense tensor");
    }
    s = collect(c);  // synchronises
    if (s) {
        g_create_err = c->err;
        destroy_buffers(c);
        delete c;
        return s;
    }
    *out = c;
    return GCP_OK;
}

void gcp_destroy(gcp_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->st);
    destroy_buffers(c);
    delete c;
}

const char *gcp_last_error(const gcp_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int32_t gcp_ndim(const gcp_ctx *c) { return c ? c->d : 0; }
int32_t gcp_rank(const gcp_ctx *c) { return c ? c->R : 0; }
int64_t gcp_nnz(const gcp_ctx *c) { return c ? c->nnz : 0; }
int64_t gcp_num_params(const gcp_ctx *c) { return c ? c->total_rows * c->R : 0; }

gcp_status gcp_set_factors(gcp_ctx *c, const float *A) {
    if (!c || !A) return fail(c, GCP_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    GCP_CUDA(c, copy_rows(c->A, (size_t)c->Rp * 4, A, (size_t)c->R * 4, (size_t)c->R * 4,
                                  (size_t)c->total_rows, c->st));
    return refresh_bf16(c);
}

gcp_status gcp_set_factor(gcp_ctx *c, int32_t mode, const float *A_mode) {
    if (!c || !A_mode) return fail(c, GCP_ERR_ARG, "NULL argument");
    if (mode < 0 || mode >= c->d) return fail(c, GCP_ERR_ARG, "mode out of range");
    DeviceGuard g(c->device);
    GCP_CUDA(c, copy_rows(c->A + c->rowoff[mode] * c->Rp, (size_t)c->Rp * 4, A_mode, (size_t)c->R * 4,
                                  (size_t)c->R * 4, (size_t)c->dims[mode], c->st));
    return refresh_bf16(c);
}

gcp_status gcp_set_factor_list(gcp_ctx *c, const float *const *A_modes) {
    if (!c || !A_modes) return fail(c, GCP_ERR_ARG, "NULL argument");
    for (int k = 0; k < c->d; ++k)
        if (!A_modes[k]) return fail(c, GCP_ERR_ARG, "NULL factor pointer");
    DeviceGuard g(c->device);
    for (int k = 0; k < c->d; ++k)
        GCP_CUDA(c, copy_rows(c->A + c->rowoff[k] * c->Rp, (size_t)c->Rp * 4, A_modes[k], (size_t)c->R * 4,
                                      (size_t)c->R * 4, (size_t)c->dims[k], c->st));
    return refresh_bf16(c);
}

gcp_status gcp_get_factors(gcp_ctx *c, float *A_out) {
    if (!c || !A_out) return fail(c, GCP_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    GCP_CUDA(c, copy_rows(A_out, (size_t)c->R * 4, c->A, (size_t)c->Rp * 4, (size_t)c->R * 4,
                                  (size_t)c->total_rows, c->st));
    return collect(c);
}

gcp_status gcp_reset_adam(gcp_ctx *c) {
    if (!c) return fail(c, GCP_ERR_ARG, "NULL context");
    DeviceGuard g(c->device);
    const size_t bytes = (size_t)c->total_rows * c->Rp * 4;
    GCP_CUDA(c, cudaMemsetAsync(c->B, 0, bytes, c->st));
    GCP_CUDA(c, cudaMemsetAsync(c->C, 0, bytes, c->st));
    return GCP_OK;
}

gcp_status gcp_sample(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, int32_t *idx_out, float *x_out,
                      float *w_out) {
    if (!c) return fail(c, GCP_ERR_ARG, "NULL context");
    DeviceGuard g(c->device);
    gcp_status s = check_counts(c, p, q);
    if (s) return s;
    double w_nz, w_z;
    weights(c, p, q, w_nz, w_z);
    GCP_CUDA(c, gcpk::launch_sample(sample_spec(c, iter, p, q), idx_out, x_out, w_out, (float)w_nz, (float)w_z,
                                    c->st));
    return GCP_OK;
}

gcp_status gcp_loss(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, double *loss_out) {
    if (!c || !loss_out) return fail(c, GCP_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    gcp_status s = run_fused(c, iter, p, q, false, nullptr);
    if (s) return s;
    return read_loss(c, loss_out);
}

gcp_status gcp_loss_async(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, double *dloss_out) {
    if (!c || !dloss_out) return fail(c, GCP_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    gcp_status s = run_fused(c, iter, p, q, false, nullptr);
    if (s) return s;
    GCP_CUDA(c, cudaMemcpyAsync(dloss_out, c->dloss, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return GCP_OK;
}

gcp_status gcp_grad(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, float *G_out, double *loss_out) {
    if (!c) return fail(c, GCP_ERR_ARG, "NULL context");
    DeviceGuard g(c->device);
    gcp_status s = run_fused(c, iter, p, q, true, nullptr);
    if (s) return s;
    s = copy_grad_out(c, G_out);
    if (s) return s;
    return loss_out ? read_loss(c, loss_out) : GCP_OK;
}

gcp_status gcp_grad_async(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, const float *dscale, float *G_out,
                          double *dloss_out) {
    if (!c) return fail(c, GCP_ERR_ARG, "NULL context");
    DeviceGuard g(c->device);
    gcp_status s = run_fused(c, iter, p, q, true, dscale);
    if (s) return s;
    s = copy_grad_out(c, G_out);
    if (s) return s;
    if (dloss_out)
        GCP_CUDA(c, cudaMemcpyAsync(dloss_out, c->dloss, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return GCP_OK;
}

gcp_status gcp_grad_factors_async(gcp_ctx *c, const float *const *A_modes, uint64_t iter, int64_t p, int64_t q,
                                  float *G_out, double *dloss_out) {
    if (!c || !A_modes) return fail(c, GCP_ERR_ARG, "NULL argument");
    FactorSrc src{};
    for (int k = 0; k < c->d; ++k) {
        if (!A_modes[k]) return fail(c, GCP_ERR_ARG, "NULL factor pointer");
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, A_modes[k]) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
            (at.type == cudaMemoryTypeDevice && at.device != c->device)) {
            cudaGetLastError();  // a host pointer is an argument error, not a sticky CUDA error
            return fail(c, GCP_ERR_ARG, "factor matrices must be device or managed memory of the context's device");
        }
        src.A[k] = A_modes[k];
        src.rowoff[k] = c->rowoff[k];
    }
    src.rowoff[c->d] = c->total_rows;
    DeviceGuard g(c->device);
    gcp_status s = check_counts(c, p, q);
    if (s) return s;
    const int64_t n = c->total_rows * c->Rp;
    int log2Rp = 0;
    while ((1 << log2Rp) < c->Rp) ++log2Rp;
    const int64_t want = (n + 255) / 256;
    k_stage_factors<<<(unsigned)(want < 8192 ? want : 8192), 256, 0, c->st>>>(
        src, c->d, c->R, log2Rp, n, c->A, static_cast<__nv_bfloat16 *>(c->Abf));
    GCP_CUDA(c, cudaGetLastError());
    if ((s = run_fused(c, iter, p, q, G_out != nullptr, nullptr))) return s;
    if ((s = copy_grad_out(c, G_out))) return s;
    if (dloss_out)
        GCP_CUDA(c, cudaMemcpyAsync(dloss_out, c->dloss, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return GCP_OK;
}

gcp_status gcp_scale_async(gcp_ctx *c, const double *dscale, const float *x, float *y, int64_t n) {
    if (!c) return fail(c, GCP_ERR_ARG, "NULL context");
    if (!dscale || !x || !y || n < 0) return fail(c, GCP_ERR_ARG, "NULL array or negative length");
    if (n == 0) return GCP_OK;
    DeviceGuard g(c->device);
    const int64_t want = (n + 255) / 256;
    k_scale<<<(unsigned)(want < 8192 ? want : 8192), 256, 0, c->st>>>(dscale, x, y, n);
    GCP_CUDA(c, cudaGetLastError());
    return GCP_OK;
}

gcp_status gcp_adam_step(gcp_ctx *c, const gcp_adam_params *prm, int64_t t) {
    if (!c || !prm) return fail(c, GCP_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    return adam_step_impl(c, prm, t);
}

gcp_status gcp_step(gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, const gcp_adam_params *prm, int64_t t,
                    double *dloss_out) {
    if (!c || !prm) return fail(c, GCP_ERR_ARG, "NULL argument");
    if (t < 1) return fail(c, GCP_ERR_ARG, "Adam step t must be >= 1");
    if (!(prm->beta1 >= 0.0 && prm->beta1 < 1.0 && prm->beta2 >= 0.0 && prm->beta2 < 1.0 && prm->eps >= 0.0))
        return fail(c, GCP_ERR_ARG, "Adam parameters out of range");
    DeviceGuard g(c->device);
    gcp_status s = do_step(c, iter, p, q, prm, t);
    if (s) return s;
    if (dloss_out)
        GCP_CUDA(c, cudaMemcpyAsync(dloss_out, c->dloss, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    return GCP_OK;
}

gcp_status gcp_grad_norm(gcp_ctx *c, double *norm_out) {
    if (!c || !norm_out) return fail(c, GCP_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    const int64_t n = (int64_t)c->total_rows * c->Rp;  // padding columns hold zeros
    const int64_t want = (n + 255) / 256;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(want, 4 * (int64_t)c->max_blocks));
    // the loss partials are free once the gradient's loss is finished (stream order)
    k_sumsq_blocks<<<nb, 256, 0, c->st>>>(c->G, n, c->partials);
    k_sumsq_finish<<<1, 32, 0, c->st>>>(c->partials, nb, c->dloss + 2, c->status);
    GCP_CUDA(c, cudaGetLastError());
    GCP_CUDA(c, cudaMemcpyAsync(c->h_loss + 2, c->dloss + 2, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    const gcp_status s = collect(c);  // synchronises
    *norm_out = c->h_loss[2];
    return s;
}

gcp_status gcp_sync(gcp_ctx *c) {
    if (!c) return fail(c, GCP_ERR_ARG, "NULL context");
    DeviceGuard g(c->device);
    return collect(c);
}

gcp_status gcp_fit(gcp_ctx *c, const gcp_fit_params *prm, gcp_fit_report *rep) {
    if (!c || !prm) return fail(c, GCP_ERR_ARG, "NULL argument");
    if (prm->iters < 1 || prm->max_epochs < 0 || prm->max_fails < 1 || !(prm->decay > 0.0))
        return fail(c, GCP_ERR_ARG, "bad fit parameters");
    DeviceGuard g(c->device);
    const size_t bytes = (size_t)c->total_rows * c->Rp * 4;
    if (!c->bk_A) {
        cudaError_t e;
        if ((e = cudaMalloc(&c->bk_A, bytes)) || (e = cudaMalloc(&c->bk_B, bytes)) ||
            (e = cudaMalloc(&c->bk_C, bytes)))
            return cuda_fail(c, e, "allocating fit backups");
    }
    gcp_fit_report r;
    std::memset(&r, 0, sizeof(r));
    const auto t0 = std::chrono::steady_clock::now();
    auto objective = [&](double &F) -> gcp_status {
        gcp_status s = run_fused(c, GCP_ITER_OBJECTIVE, prm->p_obj, prm->q_obj, false, nullptr);
        if (s) return s;
        s = read_loss(c, &F);
        r.attempts_per_zero = prm->q_obj > 0 ? c->h_loss[1] / (double)prm->q_obj : 0.0;
        return s;
    };
    auto backup = [&](bool save) -> gcp_status {
        float *src[3] = {c->A, c->B, c->C}, *dst[3] = {c->bk_A, c->bk_B, c->bk_C};
        for (int i = 0; i < 3; ++i)
            GCP_CUDA(c, cudaMemcpyAsync(save ? dst[i] : src[i], save ? src[i] : dst[i], bytes,
                                        cudaMemcpyDeviceToDevice, c->st));
        return save ? GCP_OK : refresh_bf16(c);
    };
    double F = 0.0;
    gcp_status s = objective(F);
    if (s) return s;
    r.objective0 = F;
    double Fbest = F;
    int64_t t = 0, t_saved = 0, steps_run = 0;
    gcp_adam_params adam = prm->adam;
    uint64_t iter = prm->iter0;
    if ((s = backup(true))) return s;
    for (int epoch = 0; epoch < prm->max_epochs; ++epoch) {
        for (int it = 0; it < prm->iters; ++it) {
            if ((s = do_step(c, iter++, prm->p, prm->q, &adam, t + 1))) return s;
            ++t;
            ++steps_run;
        }
        if ((s = objective(F))) return s;
        if (epoch < GCP_FIT_TRACE) r.trace[epoch] = F;
        r.epochs = epoch + 1;
        if (!(F < Fbest)) {  // failed epoch: restore and decay the rate
            if ((s = backup(false))) return s;
            t = t_saved;
            adam.lr *= prm->decay;
            if (++r.fails >= prm->max_fails) break;
        } else {
            Fbest = F;
            t_saved = t;
            if ((s = backup(true))) return s;
        }
    }
    GCP_CUDA(c, cudaStreamSynchronize(c->st));
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    r.iterations = t;
    r.objective = Fbest;
    r.lr = adam.lr;
    r.grad_samples_per_s = r.seconds > 0 ? (double)(prm->p + prm->q) * (double)steps_run / r.seconds : 0.0;
    if (rep) *rep = r;
    return GCP_OK;
}

gcp_status gcp_profile(gcp_ctx *c, int32_t enable) {
    if (!c) return fail(c, GCP_ERR_ARG, "NULL context");
    c->prof = enable != 0;
    return GCP_OK;
}

gcp_status gcp_profile_read(gcp_ctx *c, double *kernel_ms, int64_t *launches) {
    if (!c || !kernel_ms || !launches) return fail(c, GCP_ERR_ARG, "NULL argument");
    DeviceGuard g(c->device);
    GCP_CUDA(c, cudaStreamSynchronize(c->st));
    double total = 0.0;
    for (size_t i = 0; i < c->prof_used; ++i) {
        float ms = 0.0f;
        GCP_CUDA(c, cudaEventElapsedTime(&ms, c->prof_ev[i].first, c->prof_ev[i].second));
        total += ms;
    }
    *kernel_ms = total;
    *launches = (int64_t)c->prof_used;
    c->prof_used = 0;
    return GCP_OK;
}

}  // extern "C"

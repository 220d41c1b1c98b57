// gcp_batch.cu -- many independent GCP subproblems advanced together.
//
// The federated schemes of the paper (LocalSGD, Alg. 3; GCP-FedAdam, Alg. 4)
// run many local GCP-Adam steps on independent shards.  Here the shards
// ("clients") live on one GPU, each with its own tensor, model and Adam
// state (a gcp_ctx).  One local step of every client is one launch of each
// of: zero the gradients, the multi-client fused sampled gradient
// (sampling, model, loss, all-mode MTTKRP; Sec. 3.1.1-3.1.2), fold the hot-row
// replicas, finish the per-client losses, the multi-client Adam update
// (Alg. 1), advance the step counters.  tau local steps are captured once in
// a CUDA graph and replayed; the iteration number and Adam step live in
// device memory so every replay continues where the last one stopped.
//
// The fused kernel is persistent: warps walk a global list of 32-sample
// tiles; client c owns tiles tile_start[c] .. tile_start[c+1]-1, so a tile
// never mixes clients, and a warp stages the client's parameters in shared
// memory next to the tile's samples (double-buffered like them).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gcp_batch_fused.cuh"
#include "gcp_device.cuh"
#include "gcp_epilogue.cuh"
#include "gcp_internal.h"

using namespace gcpdev;

namespace gcpb {

// the fused kernel's tile sizes live in their own translation units
extern template cudaError_t batch_fused_launch<16>(int, bool, int, int, const int4 *, const int *, int, int, int,
                                                   int, const uint64_t *, float2 *, cudaStream_t);
extern template cudaError_t batch_fused_launch<32>(int, bool, int, int, const int4 *, const int *, int, int, int,
                                                   int, const uint64_t *, float2 *, cudaStream_t);
extern template cudaError_t batch_fused_launch<64>(int, bool, int, int, const int4 *, const int *, int, int, int,
                                                   int, const uint64_t *, float2 *, cudaStream_t);
extern template cudaError_t batch_fused_allow<16>(int, bool, int);
extern template cudaError_t batch_fused_allow<32>(int, bool, int);
extern template cudaError_t batch_fused_allow<64>(int, bool, int);
extern template int batch_fused_occupancy<16>(int, bool, int);
extern template int batch_fused_occupancy<32>(int, bool, int);
extern template int batch_fused_occupancy<64>(int, bool, int);

// Per-client state used by the zero / fold / finish / Adam kernels.
struct ClientAux {
    float *A, *B, *C, *G, *Grep;
    void *Abf;
    const int *hot_row;   // replica slot -> row
    const int *hot_slot;  // row -> replica slot, or -1
    int Htot;
    int64_t nparam;  // total_rows * Rp
    int R, Rp;
    double w_nz, w_z;
    int tile0[3], ntiles[3];  // first tile and tile count at 16, 32 and 64 samples per tile
};

// Samples per warp tile: 16, 32 or 64 (index 0, 1, 2 of the per-size arrays).
constexpr int kTileSizes[3] = {16, 32, 64};
__host__ __device__ constexpr int tile_index(int ts) { return ts == 16 ? 0 : (ts == 32 ? 1 : 2); }

// ------------------------------------------------- per-client small kernels
// grid.y = client; blocks of grid.x stride over that client's elements.
// G = 0, one 16-byte quad per thread and step (nparam is a multiple of 4).
// Adam constants in device memory: adam[0..4] = lr, beta1, beta2, eps, lower
// (Alg. 1); adam[5..6] = the bias corrections 1/(1 - beta1^t) and
// 1/(1 - beta2^t) of the step t = step[1] + 1 about to run; adam[7..8] =
// beta1^t and beta2^t, advanced by one multiplication per step.
__device__ __forceinline__ void set_bias_corrections(double *adam, double p1, double p2) {
    adam[7] = p1;
    adam[8] = p2;
    adam[5] = 1.0 / (1.0 - p1);
    adam[6] = 1.0 / (1.0 - p2);
}

// Counters and hyperparameters of one gcp_batch_local_steps call, passed as
// kernel arguments so that back-to-back calls cannot see each other's values.
__global__ void k_batch_set(uint64_t *step, double *adam, uint64_t iter0, uint64_t t0, double lr, double beta1,
                            double beta2, double eps, double lower) {
    step[0] = iter0;
    step[1] = t0;
    adam[0] = lr;
    adam[1] = beta1;
    adam[2] = beta2;
    adam[3] = eps;
    adam[4] = lower;
    set_bias_corrections(adam, pow(beta1, (double)(t0 + 1)), pow(beta2, (double)(t0 + 1)));
}

// Block-wide, fixed-order sum of client a's per-tile loss partials, weighted
// (FP64).  Each thread adds its tiles t, t + kThreads, ... in that order; eight
// loads are issued before their adds so the chain does not wait on each one.
__device__ __forceinline__ void finish_client_loss(const ClientAux &a, int ti, const float2 *__restrict__ tile_loss,
                                                   double *out) {
    __shared__ double sh[2][kThreads];
    double nz = 0.0, z = 0.0;
    const float2 *tl = tile_loss + a.tile0[ti];
    const int ntiles = a.ntiles[ti];
    int t = threadIdx.x;
    for (; t + 7 * kThreads < ntiles; t += 8 * kThreads) {
        float2 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = tl[t + r * kThreads];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            nz += v[r].x;
            z += v[r].y;
        }
    }
    for (; t < ntiles; t += kThreads) {
        const float2 v = tl[t];
        nz += v.x;
        z += v.y;
    }
    sh[0][threadIdx.x] = nz;
    sh[1][threadIdx.x] = z;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + h];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = a.w_nz * sh[0][0] + a.w_z * sh[1][0];
}

// Algorithm 1 on one 16-byte quad (4 entries of one row, columns col..col+3)
// with its gradient g4; entries in padded columns stay zero.
struct AdamConsts {
    float lr, beta1, beta2, eps, lower, c1inv, c2inv;
};

__device__ __forceinline__ void adam_quad(const ClientAux &a, int64_t qi, int col, float4 g4, float4 b4, float4 c4,
                                          float4 x4, const AdamConsts &k) {
    const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
    float bv[4] = {b4.x, b4.y, b4.z, b4.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w}, xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (col + j >= a.R) continue;  // padded columns stay zero
        const float g = gv[j];
        bv[j] = k.beta1 * bv[j] + (1.0f - k.beta1) * g;
        cv[j] = k.beta2 * cv[j] + (1.0f - k.beta2) * g * g;
        xv[j] = fmaxf(xv[j] - k.lr * ((bv[j] * k.c1inv) / sqrtf(cv[j] * k.c2inv + k.eps)), k.lower);
    }
    reinterpret_cast<float4 *>(a.B)[qi] = make_float4(bv[0], bv[1], bv[2], bv[3]);
    reinterpret_cast<float4 *>(a.C)[qi] = make_float4(cv[0], cv[1], cv[2], cv[3]);
    reinterpret_cast<float4 *>(a.A)[qi] = make_float4(xv[0], xv[1], xv[2], xv[3]);
    if (a.Abf) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(xv[0], xv[1]), hi = __floats2bfloat162_rn(xv[2], xv[3]);
        static_cast<uint2 *>(a.Abf)[qi] =
            make_uint2(*reinterpret_cast<const unsigned *>(&lo), *reinterpret_cast<const unsigned *>(&hi));
    }
}

// The epilogue of one local step of every client, one launch over a chunk
// list built at batch creation.  A chunk {client, code} is
//  - code == -1: finish that client's loss;
//  - code >= 0: the client's parameter quads code .. code + kThreads - 1,
//    one per thread, all loads (gradient, moments, factor, replica slot)
//    issued before any is used, then Algorithm 1; quads of hot rows are
//    left to the hot chunks;
//  - code <= -2: the client's hot quads h .. h + kThreads / kHotLanes - 1
//    (h = -2 - code; hot quad h is column quad h % (Rp/4) of replica slot
//    h / (Rp/4)), one per group of kHotLanes lanes: the group loads all
//    replica quads at once (gcpe::hot_quad_sum, which clears them), its
//    first lane adds them to the gradient quad and applies Algorithm 1.
// G itself is cleared at the start of the next step, just before the fused
// pass, so that its lines are still in L2 when the reductions arrive.
// Quads per thread of a streaming chunk, all loads issued together, with
// the kernel held to three blocks per SM (78 registers): 0.3725 ms per
// local step of the 64-client batch, against 0.381 ms with four quads per
// thread at two blocks per SM, 0.395 ms with two at four blocks and
// 0.379-0.383 ms with three at two or five and six at two.
constexpr int kPostUnroll = 3;
constexpr int kPostMinBlocks = 3;
constexpr int kPostQuads = kThreads * kPostUnroll;              // quads of a streaming chunk
constexpr int kHotQuadsPerChunk = kThreads / gcpe::kHotLanes;   // hot quads of a hot chunk
static_assert(gcpk::kReplicas % gcpe::kHotLanes == 0, "hot-quad replicas split evenly over the folding lanes");

__global__ void __launch_bounds__(kThreads, kPostMinBlocks) k_batch_post(const ClientAux *__restrict__ aux,
                                                         const int2 *__restrict__ chunks,
                                                         const float2 *__restrict__ tile_loss, double *client_loss,
                                                         const double *__restrict__ adam, int ti) {
    const int2 ch = chunks[blockIdx.x];
    const ClientAux &a = aux[ch.x];
    if (ch.y == -1) {
        finish_client_loss(a, ti, tile_loss, client_loss + ch.x);
        return;
    }
    const AdamConsts k{(float)adam[0], (float)adam[1], (float)adam[2], (float)adam[3],
                       (float)adam[4], (float)adam[5], (float)adam[6]};
    const int log2Rp = __ffs(a.Rp) - 1;  // Rp is a power of two and a multiple of 4
    const float4 *__restrict__ G4 = reinterpret_cast<const float4 *>(a.G);
    const float4 *__restrict__ A4 = reinterpret_cast<const float4 *>(a.A);
    const float4 *__restrict__ B4 = reinterpret_cast<const float4 *>(a.B);
    const float4 *__restrict__ C4 = reinterpret_cast<const float4 *>(a.C);
    if (ch.y <= -2) {  // hot quads, one per group of kHotLanes lanes
        const int log2Q = log2Rp - 2;
        const int64_t hq = (int64_t)(-2 - ch.y) + threadIdx.x / gcpe::kHotLanes;
        if (hq >= ((int64_t)a.Htot << log2Q)) return;  // the whole group leaves together
        const int slot = (int)(hq >> log2Q), cq = (int)(hq & ((1 << log2Q) - 1));
        const int64_t q = ((int64_t)__ldg(a.hot_row + slot) << log2Q) + cq;
        const bool lead = (threadIdx.x & (gcpe::kHotLanes - 1)) == 0;
        float4 g4, b4, c4, x4;
        if (lead) {
            g4 = G4[q];
            b4 = B4[q];
            c4 = C4[q];
            x4 = A4[q];
        }
        const float4 t = gcpe::hot_quad_sum<gcpk::kReplicas>(reinterpret_cast<float4 *>(a.Grep),
                                                             ((int64_t)a.Htot * a.Rp) >> 2, hq,
                                                             gcpe::hot_group_mask());
        const int col = cq << 2;
        if (!lead || col >= a.R) return;
        g4.x += t.x;
        g4.y += t.y;
        g4.z += t.z;
        g4.w += t.w;
        adam_quad(a, q, col, g4, b4, c4, x4, k);
        return;
    }
    const int64_t nq = a.nparam >> 2;
    float4 g4[kPostUnroll], b4[kPostUnroll], c4[kPostUnroll], x4[kPostUnroll];
    int hs[kPostUnroll];
#pragma unroll
    for (int u = 0; u < kPostUnroll; ++u) {
        const int64_t q = (int64_t)ch.y + threadIdx.x + u * kThreads;
        hs[u] = 0;
        if (q < nq) {
            g4[u] = G4[q];
            b4[u] = B4[q];
            c4[u] = C4[q];
            x4[u] = A4[q];
            hs[u] = a.hot_slot ? __ldg(a.hot_slot + ((q << 2) >> log2Rp)) : -1;
        }
    }
#pragma unroll
    for (int u = 0; u < kPostUnroll; ++u) {
        const int64_t q = (int64_t)ch.y + threadIdx.x + u * kThreads;
        const int col = (int)((q << 2) & (a.Rp - 1));
        if (hs[u] >= 0 || col >= a.R) continue;  // beyond the client, or a hot quad (the hot chunks take it)
        adam_quad(a, q, col, g4[u], b4[u], c4[u], x4[u], k);
    }
}

// Gradients cleared before the fused pass (grid.y = client).
__global__ void k_batch_zero(const ClientAux *__restrict__ aux) {
    const ClientAux &a = aux[blockIdx.y];
    float4 *G = reinterpret_cast<float4 *>(a.G);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (a.nparam >> 2);
         e += (int64_t)gridDim.x * blockDim.x)
        G[e] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__global__ void k_batch_advance(uint64_t *step, double *adam) {
    step[0] += 1;
    step[1] += 1;
    set_bias_corrections(adam, adam[7] * adam[1], adam[8] * adam[2]);
}

// ------------------------------------------------------ GCP-FedAdam server
// Clients of one model (identical shapes): U is the server model with Adam
// moments Bs, Cs.  Init: U = client 0's factors, moments cleared, every
// client set to U.
__global__ void k_fed_init(const ClientAux *__restrict__ aux, int n, float *U, float *Bs, float *Cs) {
    const ClientAux &a0 = aux[0];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a0.nparam; e += (int64_t)gridDim.x * blockDim.x) {
        const float u = a0.A[e];
        U[e] = u;
        Bs[e] = 0.0f;
        Cs[e] = 0.0f;
        for (int c = 1; c < n; ++c) {
            aux[c].A[e] = u;
            if (aux[c].Abf) static_cast<__nv_bfloat16 *>(aux[c].Abf)[e] = __float2bfloat16_rn(u);
        }
    }
}

// Reconciliation of Algorithm 4: D = U - mean_c M_c (clients summed in
// order), Adam (Algorithm 1) on U with the server hyperparameters
// c = {lr, beta1, beta2, 1/(1-beta1^t), 1/(1-beta2^t), eps, lower}, then
// M_c = U for every client.  Padded columns stay zero.
__global__ void k_fed_server(const ClientAux *__restrict__ aux, int n, float *U, float *Bs, float *Cs,
                             const float *__restrict__ c7) {
    const ClientAux &a0 = aux[0];
    const float lr = c7[0], b1 = c7[1], b2 = c7[2], c1 = c7[3], c2 = c7[4], eps = c7[5], lower = c7[6];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a0.nparam; e += (int64_t)gridDim.x * blockDim.x) {
        if ((int)(e % a0.Rp) >= a0.R) continue;
        float sum = 0.0f;
        for (int c = 0; c < n; ++c) sum += aux[c].A[e];
        const float d = U[e] - sum / (float)n;
        const float b = b1 * Bs[e] + (1.0f - b1) * d;
        const float cc = b2 * Cs[e] + (1.0f - b2) * d * d;
        Bs[e] = b;
        Cs[e] = cc;
        const float u = fmaxf(U[e] - lr * ((b * c1) / sqrtf(cc * c2 + eps)), lower);
        U[e] = u;
        for (int c = 0; c < n; ++c) {
            aux[c].A[e] = u;
            if (aux[c].Abf) static_cast<__nv_bfloat16 *>(aux[c].Abf)[e] = __float2bfloat16_rn(u);
        }
    }
}

}  // namespace gcpb

// ======================================================================= host
struct gcp_batch {
    int n = 0, d = 0, R = 0, Rp = 0, loss = 0, device = 0;
    bool bf16 = false;
    std::vector<gcp_ctx *> clients;
    std::vector<int64_t> p, q;
    int total_tiles[3] = {0, 0, 0};  // tiles of 16, 32 and 64 samples
    int cols = 4, blocks = 0;        // tuning knobs: columns per lane, fused-kernel grid,
    int ts = 32;                     //   samples per warp tile
    int4 *specs = nullptr;           // n x kSpecWords
    int *tile_start = nullptr;       // 3 x (n + 1): first tile of each client, per tile size
    int2 *chunks = nullptr;          // epilogue work list: {client, -1} loss, {client, first quad} Adam
    int nchunks = 0;
    gcpb::ClientAux *aux = nullptr;  // n
    float2 *tile_loss = nullptr;     // total_tiles of the smallest tile size
    double *client_loss = nullptr;   // n
    uint64_t *step = nullptr;        // [0] iteration of the next gradient, [1] Adam steps done
    double *adam = nullptr;          // lr, beta1, beta2, eps, lower, bias corrections, beta powers
    double *h_loss = nullptr;
    int64_t max_param = 0, max_rep = 0;
    cudaStream_t st = nullptr, user_st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_tau = 0, graph_cols = 0, graph_blocks = 0, graph_ts = 0;
    float *U = nullptr, *Bs = nullptr, *Cs = nullptr;  // FedAdam server model and moments
    float *fed_c = nullptr, *h_fed_c = nullptr;        // server Adam constants (device, pinned)
    std::string err;
};

namespace {

thread_local std::string g_batch_create_err;

gcp_status bfail(gcp_batch *b, gcp_status s, const std::string &m) {
    if (b)
        b->err = m;
    else
        g_batch_create_err = m;
    return s;
}

#define BCUDA(b, call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? GCP_ERR_OOM : GCP_ERR_CUDA,        \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

void batch_free(gcp_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->specs);
    cudaFree(b->tile_start);
    cudaFree(b->chunks);
    cudaFree(b->aux);
    cudaFree(b->tile_loss);
    cudaFree(b->client_loss);
    cudaFree(b->step);
    cudaFree(b->adam);
    cudaFreeHost(b->h_loss);
    cudaFree(b->U);
    cudaFree(b->Bs);
    cudaFree(b->Cs);
    cudaFree(b->fed_c);
    cudaFreeHost(b->h_fed_c);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->st) cudaStreamDestroy(b->st);
}

int default_blocks(const gcp_batch *b, int cols, int ts) {
    const int per_sm = ts == 16 ? gcpb::batch_fused_occupancy<16>(b->d, b->bf16, cols)
                                : (ts == 64 ? gcpb::batch_fused_occupancy<64>(b->d, b->bf16, cols)
                                            : gcpb::batch_fused_occupancy<32>(b->d, b->bf16, cols));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    return per_sm * sms;
}

cudaError_t allow_batch_fused(const gcp_batch *b) {
    return b->ts == 16 ? gcpb::batch_fused_allow<16>(b->d, b->bf16, b->cols)
                       : (b->ts == 64 ? gcpb::batch_fused_allow<64>(b->d, b->bf16, b->cols)
                                      : gcpb::batch_fused_allow<32>(b->d, b->bf16, b->cols));
}

cudaError_t launch_batch_fused(const gcp_batch *b) {
    int log2L = 0;
    while ((1 << log2L) * b->cols < b->Rp) ++log2L;
    const int ti = gcpb::tile_index(b->ts);
    const int *tstart = b->tile_start + ti * (b->n + 1);
    auto go = [&](auto launch) {
        return launch(b->d, b->bf16, b->cols, b->blocks, b->specs, tstart, b->n, b->total_tiles[ti], log2L, b->Rp,
                      b->step, b->tile_loss, b->st);
    };
    if (b->ts == 16) return go(gcpb::batch_fused_launch<16>);
    if (b->ts == 64) return go(gcpb::batch_fused_launch<64>);
    return go(gcpb::batch_fused_launch<32>);
}

// One local step of every client, enqueued on b->st (also used for capture):
// gradients cleared, the multi-client fused pass, one epilogue launch, the
// counter advance.
gcp_status enqueue_step(gcp_batch *b) {
    const int nb = gcpb::kThreads;
    const dim3 gp((unsigned)std::min<int64_t>(64, (b->max_param / 4 + nb - 1) / nb), (unsigned)b->n);
    gcpb::k_batch_zero<<<gp, nb, 0, b->st>>>(b->aux);
    BCUDA(b, launch_batch_fused(b));
    gcpb::k_batch_post<<<b->nchunks, nb, 0, b->st>>>(b->aux, b->chunks, b->tile_loss, b->client_loss, b->adam,
                                                     gcpb::tile_index(b->ts));
    gcpb::k_batch_advance<<<1, 1, 0, b->st>>>(b->step, b->adam);
    BCUDA(b, cudaGetLastError());
    return GCP_OK;
}

}  // namespace

extern "C" {

gcp_status gcp_batch_create(int32_t nclients, gcp_ctx *const *clients, const int64_t *p, const int64_t *q,
                            gcp_batch **out) {
    if (!out) return bfail(nullptr, GCP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nclients < 1 || !clients || !p || !q) return bfail(nullptr, GCP_ERR_ARG, "need nclients >= 1, clients, p, q");
    const gcp_ctx *c0 = clients[0];
    if (!c0) return bfail(nullptr, GCP_ERR_ARG, "NULL client");
    int64_t tiles = 0;
    for (int i = 0; i < nclients; ++i) {
        const gcp_ctx *c = clients[i];
        if (!c) return bfail(nullptr, GCP_ERR_ARG, "NULL client");
        if (c->dense || c->opt.sampling == GCP_SAMPLING_UNIFORM)
            return bfail(nullptr, GCP_ERR_ARG, "batched clients must be sparse tensors");
        if (c->opt.mttkrp != GCP_MTTKRP_ATOMIC) return bfail(nullptr, GCP_ERR_ARG, "batched clients use the atomic MTTKRP");
        if (c->d != c0->d || c->R != c0->R || c->Rp != c0->Rp || c->loss != c0->loss ||
            (c->Abf != nullptr) != (c0->Abf != nullptr) || c->device != c0->device || c->st != c0->st)
            return bfail(nullptr, GCP_ERR_ARG,
                         "clients must share order, rank, loss, factor dtype, device and stream");
        if (p[i] < 0 || q[i] < 0 || p[i] + q[i] >= ((int64_t)1 << 31))
            return bfail(nullptr, GCP_ERR_ARG, "per-client sample counts must be >= 0 and sum below 2^31");
        tiles += (p[i] + q[i] + 15) / 16;  // the smallest tiles give the most
    }
    if (tiles >= ((int64_t)1 << 31)) return bfail(nullptr, GCP_ERR_ARG, "too many samples in the batch");
    gcp_batch *b = new (std::nothrow) gcp_batch();
    if (!b) return bfail(nullptr, GCP_ERR_OOM, "host allocation");
    b->n = nclients;
    b->d = c0->d;
    b->R = c0->R;
    b->Rp = c0->Rp;
    b->loss = c0->loss;
    b->bf16 = c0->Abf != nullptr;
    b->device = c0->device;
    b->user_st = c0->st;
    b->clients.assign(clients, clients + nclients);
    b->p.assign(p, p + nclients);
    b->q.assign(q, q + nclients);
    b->cols = c0->cols;
    std::vector<int4> specs((size_t)nclients * gcpb::kSpecWords);
    std::vector<int> tstart(3 * (nclients + 1), 0);  // per tile size: first tile of each client, then the total
    std::vector<gcpb::ClientAux> aux(nclients);
    for (int i = 0; i < nclients; ++i) {
        gcp_ctx *c = clients[i];
        double w_nz, w_z;
        const gcpk::FusedSpec f = gcpk_make_spec(c, 0, p[i], q[i], true, nullptr, &w_nz, &w_z);
        std::memcpy(&specs[(size_t)i * gcpb::kSpecWords], &f, sizeof(f));
        for (int t = 0; t < 3; ++t) {
            const int ts = gcpb::kTileSizes[t], *row = &tstart[(size_t)t * (nclients + 1)];
            const int nt = (int)((p[i] + q[i] + ts - 1) / ts);
            tstart[(size_t)t * (nclients + 1) + i + 1] = row[i] + nt;
        }
        gcpb::ClientAux &a = aux[i];
        a.A = c->A;
        a.B = c->B;
        a.C = c->C;
        a.G = c->G;
        a.Grep = c->Grep;
        a.Abf = c->Abf;
        a.hot_row = c->hot_row;
        a.hot_slot = c->hot_slot;
        a.Htot = c->Htot;
        a.nparam = c->total_rows * c->Rp;
        a.R = c->R;
        a.Rp = c->Rp;
        a.w_nz = w_nz;
        a.w_z = w_z;
        for (int t = 0; t < 3; ++t) {
            a.tile0[t] = tstart[(size_t)t * (nclients + 1) + i];
            a.ntiles[t] = tstart[(size_t)t * (nclients + 1) + i + 1] - a.tile0[t];
            b->total_tiles[t] = tstart[(size_t)t * (nclients + 1) + i + 1];
        }
        b->max_param = std::max<int64_t>(b->max_param, a.nparam);
        b->max_rep = std::max<int64_t>(b->max_rep, (int64_t)a.Htot * a.Rp);
    }
    std::vector<int2> chunks;  // loss chunks first, so they start with the first wave
    for (int i = 0; i < nclients; ++i) chunks.push_back(make_int2(i, -1));
    for (int i = 0; i < nclients; ++i)
        for (int64_t q0 = 0; q0 < aux[i].nparam / 4; q0 += gcpb::kPostQuads) chunks.push_back(make_int2(i, (int)q0));
    for (int i = 0; i < nclients; ++i)  // hot chunks: code -2 - (first hot quad)
        for (int64_t h = 0; h < (int64_t)aux[i].Htot * (aux[i].Rp / 4); h += gcpb::kHotQuadsPerChunk)
            chunks.push_back(make_int2(i, (int)(-2 - h)));
    b->nchunks = (int)chunks.size();
    cudaError_t e;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if ((e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking)) ||
        (e = cudaMalloc(&b->chunks, chunks.size() * sizeof(int2))) ||
        (e = cudaMemcpy(b->chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice)) ||
        (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) ||
        (e = cudaMalloc(&b->specs, specs.size() * sizeof(int4))) ||
        (e = cudaMalloc(&b->tile_start, tstart.size() * sizeof(int))) ||
        (e = cudaMalloc(&b->aux, aux.size() * sizeof(gcpb::ClientAux))) ||
        (e = cudaMalloc(&b->tile_loss, (size_t)std::max(1, b->total_tiles[0]) * sizeof(float2))) ||
        (e = cudaMalloc(&b->client_loss, (size_t)nclients * sizeof(double))) ||
        (e = cudaMalloc(&b->step, 2 * sizeof(uint64_t))) || (e = cudaMalloc(&b->adam, 9 * sizeof(double))) ||
        (e = cudaMallocHost(&b->h_loss, (size_t)nclients * sizeof(double))) ||
        (e = cudaMemcpy(b->specs, specs.data(), specs.size() * sizeof(int4), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->tile_start, tstart.data(), tstart.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->aux, aux.data(), aux.size() * sizeof(gcpb::ClientAux), cudaMemcpyHostToDevice))) {
        batch_free(b);
        delete b;
        if (prev >= 0) cudaSetDevice(prev);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? GCP_ERR_OOM : GCP_ERR_CUDA,
                     std::string("creating the batch: ") + cudaGetErrorString(e));
    }
    b->blocks = default_blocks(b, b->cols, b->ts);
    if (prev >= 0) cudaSetDevice(prev);
    *out = b;
    return GCP_OK;
}

void gcp_batch_destroy(gcp_batch *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->st);
    batch_free(b);
    delete b;
}

const char *gcp_batch_last_error(const gcp_batch *b) { return b ? b->err.c_str() : g_batch_create_err.c_str(); }

gcp_status gcp_batch_tune(gcp_batch *b, int32_t lane_cols, int32_t blocks) {
    if (!b) return bfail(b, GCP_ERR_ARG, "NULL batch");
    const int cols = lane_cols == 0 ? b->clients[0]->cols : lane_cols;
    if (cols != 4 && !(cols == 8 && b->Rp >= 8)) return bfail(b, GCP_ERR_ARG, "lane_cols must be 0, 4 or 8 (8 needs rank > 4)");
    if (blocks < 0) return bfail(b, GCP_ERR_ARG, "blocks must be >= 0");
    b->cols = cols;
    b->blocks = blocks == 0 ? default_blocks(b, cols, b->ts) : blocks;
    return GCP_OK;
}

gcp_status gcp_batch_tune_tile(gcp_batch *b, int32_t samples_per_warp) {
    if (!b) return bfail(b, GCP_ERR_ARG, "NULL batch");
    const int ts = samples_per_warp == 0 ? 32 : samples_per_warp;
    if (ts != 16 && ts != 32 && ts != 64) return bfail(b, GCP_ERR_ARG, "samples_per_warp must be 0, 16, 32 or 64");
    const bool auto_blocks = b->blocks == default_blocks(b, b->cols, b->ts);
    b->ts = ts;
    if (auto_blocks) b->blocks = default_blocks(b, b->cols, ts);
    return GCP_OK;
}

gcp_status gcp_batch_local_steps(gcp_batch *b, int32_t tau, const gcp_adam_params *prm, uint64_t iter0, int64_t t0) {
    if (!b || !prm) return bfail(b, GCP_ERR_ARG, "NULL argument");
    if (tau < 1 || tau > 4096) return bfail(b, GCP_ERR_ARG, "tau must be in 1..4096");
    if (t0 < 0) return bfail(b, GCP_ERR_ARG, "t0 must be >= 0");
    if (!(prm->beta1 >= 0.0 && prm->beta1 < 1.0 && prm->beta2 >= 0.0 && prm->beta2 < 1.0 && prm->eps >= 0.0))
        return bfail(b, GCP_ERR_ARG, "Adam parameters out of range");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    if (!b->graph || b->graph_tau != tau || b->graph_cols != b->cols || b->graph_blocks != b->blocks ||
        b->graph_ts != b->ts) {
        if (b->graph) {
            BCUDA(b, cudaStreamSynchronize(b->st));
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        BCUDA(b, allow_batch_fused(b));  // before the capture: a host call on the kernel
        BCUDA(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
        gcp_status s = GCP_OK;
        for (int k = 0; k < tau && !s; ++k) s = enqueue_step(b);
        cudaError_t e = cudaStreamEndCapture(b->st, &g);
        if (s) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        BCUDA(b, e);
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCUDA(b, e);
        b->graph_tau = tau;
        b->graph_cols = b->cols;
        b->graph_blocks = b->blocks;
        b->graph_ts = b->ts;
    }
    BCUDA(b, cudaEventRecord(b->ev_in, b->user_st));  // after the clients' earlier work
    BCUDA(b, cudaStreamWaitEvent(b->st, b->ev_in, 0));
    gcpb::k_batch_set<<<1, 1, 0, b->st>>>(b->step, b->adam, iter0, (uint64_t)t0, prm->lr, prm->beta1, prm->beta2,
                                          prm->eps, prm->lower);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaGraphLaunch(b->graph, b->st));
    for (gcp_ctx *c : b->clients) c->g_clear = false;  // G holds the last local step's gradient
    BCUDA(b, cudaEventRecord(b->ev_out, b->st));  // the clients' later work waits for the steps
    BCUDA(b, cudaStreamWaitEvent(b->user_st, b->ev_out, 0));
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return GCP_OK;
}

gcp_status gcp_batch_losses(gcp_batch *b, double *loss_out) {
    if (!b || !loss_out) return bfail(b, GCP_ERR_ARG, "NULL argument");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    BCUDA(b, cudaMemcpyAsync(b->h_loss, b->client_loss, (size_t)b->n * sizeof(double), cudaMemcpyDeviceToHost,
                             b->st));
    BCUDA(b, cudaStreamSynchronize(b->st));
    std::memcpy(loss_out, b->h_loss, (size_t)b->n * sizeof(double));
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    for (gcp_ctx *c : b->clients) {  // device errors of any client (sampler exhausted, ...)
        gcp_status s = gcp_sync(c);
        if (s) return bfail(b, s, std::string("client error: ") + gcp_last_error(c));
    }
    return GCP_OK;
}

gcp_status gcp_batch_server_init(gcp_batch *b) {
    if (!b) return bfail(b, GCP_ERR_ARG, "NULL batch");
    const gcp_ctx *c0 = b->clients[0];
    for (const gcp_ctx *c : b->clients)
        for (int k = 0; k < b->d; ++k)
            if (c->dims[k] != c0->dims[k])
                return bfail(b, GCP_ERR_ARG, "the FedAdam server needs clients of one model shape");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    const size_t bytes = (size_t)b->max_param * sizeof(float);
    if (!b->U) {
        BCUDA(b, cudaMalloc(&b->U, bytes));
        BCUDA(b, cudaMalloc(&b->Bs, bytes));
        BCUDA(b, cudaMalloc(&b->Cs, bytes));
        BCUDA(b, cudaMalloc(&b->fed_c, 8 * sizeof(float)));
        BCUDA(b, cudaMallocHost(&b->h_fed_c, 8 * sizeof(float)));
    }
    BCUDA(b, cudaEventRecord(b->ev_in, b->user_st));
    BCUDA(b, cudaStreamWaitEvent(b->st, b->ev_in, 0));
    const int blocks = (int)std::min<int64_t>(1024, (b->max_param + gcpb::kThreads - 1) / gcpb::kThreads);
    gcpb::k_fed_init<<<blocks, gcpb::kThreads, 0, b->st>>>(b->aux, b->n, b->U, b->Bs, b->Cs);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaEventRecord(b->ev_out, b->st));
    BCUDA(b, cudaStreamWaitEvent(b->user_st, b->ev_out, 0));
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return GCP_OK;
}

gcp_status gcp_batch_server_step(gcp_batch *b, const gcp_adam_params *prm, int64_t t) {
    if (!b || !prm) return bfail(b, GCP_ERR_ARG, "NULL argument");
    if (!b->U) return bfail(b, GCP_ERR_STATE, "call gcp_batch_server_init first");
    if (t < 1) return bfail(b, GCP_ERR_ARG, "server step t must be >= 1");
    if (!(prm->beta1 >= 0.0 && prm->beta1 < 1.0 && prm->beta2 >= 0.0 && prm->beta2 < 1.0 && prm->eps >= 0.0))
        return bfail(b, GCP_ERR_ARG, "Adam parameters out of range");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    BCUDA(b, cudaStreamSynchronize(b->st));  // the pinned constants are reused
    b->h_fed_c[0] = (float)prm->lr;
    b->h_fed_c[1] = (float)prm->beta1;
    b->h_fed_c[2] = (float)prm->beta2;
    b->h_fed_c[3] = (float)(1.0 / (1.0 - std::pow(prm->beta1, (double)t)));
    b->h_fed_c[4] = (float)(1.0 / (1.0 - std::pow(prm->beta2, (double)t)));
    b->h_fed_c[5] = (float)prm->eps;
    b->h_fed_c[6] = (float)prm->lower;
    BCUDA(b, cudaEventRecord(b->ev_in, b->user_st));
    BCUDA(b, cudaStreamWaitEvent(b->st, b->ev_in, 0));
    BCUDA(b, cudaMemcpyAsync(b->fed_c, b->h_fed_c, 8 * sizeof(float), cudaMemcpyHostToDevice, b->st));
    const int blocks = (int)std::min<int64_t>(1024, (b->max_param + gcpb::kThreads - 1) / gcpb::kThreads);
    gcpb::k_fed_server<<<blocks, gcpb::kThreads, 0, b->st>>>(b->aux, b->n, b->U, b->Bs, b->Cs, b->fed_c);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaEventRecord(b->ev_out, b->st));
    BCUDA(b, cudaStreamWaitEvent(b->user_st, b->ev_out, 0));
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return GCP_OK;
}

}  // extern "C"

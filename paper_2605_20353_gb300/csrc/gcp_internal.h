// gcp_internal.h -- state and kernel-launch interface shared by the C ABI
// (gcp_api.cu) and the kernels (gcp_kernels.cu, gcp_mttkrp_det.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/gcp.h"

namespace gcpk {

// Where the samples of one call come from (Sec. 3.1.1).
struct SampleSpec {
    int d;
    int64_t dims[GCP_MAX_NDIM];
    uint64_t stride[GCP_MAX_NDIM];  // linear-index strides, last mode fastest
    int64_t nnz;
    const int32_t *rec;             // nonzero records: d int32 coords + float bits, padded
    int rec_words;                  // 4, 8 or 16 words per record
    const uint64_t *hkeys;          // hash set of nonzero linear indices
    uint64_t hbmask;                // number of 4-slot buckets - 1
    const float *dense;             // dense tensor values (uniform sampling) or null
    uint64_t seed, iter;
    int64_t p, q;                   // nonzero / zero (or p uniform) samples
    int sampling;                   // gcp_sampling_t
    int max_attempts;
    int *status;                    // device status word (bit = gcp_status code)
};

// The fused model / loss / MTTKRP pass over one sample set.
struct FusedSpec {
    SampleSpec s;
    const void *F;                  // factors the kernels read (FP32 or BF16), row stride Rp
    float *G;                       // gradient, row stride Rp; null = loss only
    int Rp;                         // padded row length: cols x lanes per sample (power of 2)
    int log2L;                      // log2(lanes per sample); each lane owns cols = 4 or 8 columns
    int rowoff[GCP_MAX_NDIM];       // first row of each mode in F and G
    int loss;
    float w_nz, w_z;                // per-sample weights (FP32 copies)
    const float *dscale;            // gradient scale (device) or null
    double *partials;               // per block: sum f over nonzero / zero samples, attempts, -
    int small_base[GCP_MAX_NDIM];   // replica slot of row 0 of a mode whose rows all have
                                    // slots (contiguous), else -1; used for drawn cells
    float *Grep;                    // kReplicas x Htot x Rp replica rows (zero between calls)
    int Htot;                       // replicated rows
    int32_t *Ycoord;                // materialize mode (G null): per-sample coordinates
    float *Yval;                    //   and gradient-tensor values w f' scale (0 if no sample):
    int ystride, vstride;           //   sample s at Ycoord[s * ystride + k], Yval[s * vstride]
};

// Rows that many samples hit (Zipf heads, rows of small modes) are
// accumulated in this many global replicas, then folded into G.
constexpr int kReplicas = 64;

// The epilogue of one training step (gcp_step): loss finish, replica fold,
// Adam and gradient clearing in one launch.
struct PostSpec {
    int64_t n;                      // total_rows * Rp
    int Rp, R, Htot;
    float *G, *Grep, *A, *B, *C;
    void *Abf;
    const int *hot_slot;            // row -> replica slot, or -1
    const int *hot_row;             // replica slot -> row
    float lr, beta1, beta2, c1inv, c2inv, eps, lower;
    const double *partials;
    int nblocks;
    double w_nz, w_z;
    double *dloss;
    int *status;
};

struct LaunchCfg {
    int blocks;
    int threads;
};

// ---------------------------------------------------------------- kernels
// All launches are asynchronous on `st`; device errors go to the status word.
cudaError_t launch_build_records(const int32_t *coords, const float *vals, int64_t nnz, int d,
                                 const uint64_t *stride, const int64_t *rowoff, const int *hot_slot,
                                 int rec_words, int32_t *rec, uint64_t *hkeys, uint64_t hbmask, int *status,
                                 cudaStream_t st);
cudaError_t launch_sample(const SampleSpec &s, int32_t *idx_out, float *x_out, float *w_out, float w_nz,
                          float w_z, cudaStream_t st);
cudaError_t launch_fused(const FusedSpec &f, bool bf16, int cols, int max_blocks, cudaStream_t st,
                         int *blocks_used);
cudaError_t launch_fold_replicas(float *G, float *Grep, const int *hot_row, int Htot, int Rp, cudaStream_t st);
cudaError_t launch_mttkrp_nonfused(const FusedSpec &f, const int *hot_slot, bool bf16, int cols, int max_blocks,
                                   cudaStream_t st);
cudaError_t launch_finish_loss(const double *partials, int nblocks, double w_nz, double w_z, double *dloss,
                               int *status, cudaStream_t st);
cudaError_t launch_adam(int64_t n, int Rp, int R, float *A, float *B, float *C, const float *G, float lr,
                        float beta1, float beta2, float c1inv, float c2inv, float eps, float lower,
                        void *Abf, cudaStream_t st);
cudaError_t launch_to_bf16(int64_t n, const float *A, void *Abf, cudaStream_t st);
cudaError_t launch_post_step(const PostSpec &p, cudaStream_t st);
int fused_max_blocks(int d, bool bf16, int cols);

}  // namespace gcpk

// --------------------------------------------------------------- context
struct gcp_ctx {
    int d = 0;
    int64_t dims[GCP_MAX_NDIM] = {0};
    uint64_t stride[GCP_MAX_NDIM] = {0};
    int64_t rowoff[GCP_MAX_NDIM] = {0};
    int64_t total_rows = 0;
    int R = 0, Rp = 0, log2L = 0, cols = 4;
    int loss = 0;
    int64_t nnz = 0;
    double M = 0;  // number of cells (exact below 2^53, used for weights)
    bool dense = false;
    gcp_options opt{};
    cudaStream_t st = nullptr;
    int device = 0;

    // device buffers (owned)
    int32_t *rec = nullptr;
    int rec_words = 0;
    uint64_t *hkeys = nullptr;
    uint64_t hbmask = 0;
    float *X = nullptr;           // dense values
    float *A = nullptr;           // FP32 master factors [total_rows x Rp]
    void *Abf = nullptr;          // BF16 copy read by the kernels (BF16 storage)
    float *G = nullptr;           // gradient
    float *B = nullptr, *C = nullptr;  // Adam moments
    double *partials = nullptr;   // per-block reduction partials
    int max_blocks = 0;
    double *dloss = nullptr;      // [0] loss, [1] zero attempts, [2] gradient norm
    int *status = nullptr;        // device status word
    int *h_status = nullptr;      // pinned mirror
    double *h_loss = nullptr;     // pinned mirror of dloss

    // hot-row replicas of the gradient
    bool g_clear = true;          // G is all zero (gcp_step leaves it so)
    int *hot_slot = nullptr;      // [total_rows] row -> replica slot or -1
    int *hot_row = nullptr;       // [Htot] slot -> row
    int small_base[GCP_MAX_NDIM] = {0};
    float *Grep = nullptr;        // [kReplicas x Htot x Rp]
    int Htot = 0;

    // deterministic MTTKRP scratch
    void *det_scratch = nullptr;
    size_t det_scratch_bytes = 0;
    cudaStream_t det_side = nullptr;             // second stream of the sort (its wide passes)
    cudaEvent_t det_fork = nullptr, det_join = nullptr;

    // non-fused MTTKRP: the materialised gradient tensor
    int32_t *nf_coord = nullptr;
    float *nf_val = nullptr;
    int64_t nf_cap = 0;

    // gcp_fit: last accepted factors and moments
    float *bk_A = nullptr, *bk_B = nullptr, *bk_C = nullptr;

    // kernel timing (gcp_profile)
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
    size_t prof_used = 0;

    std::string err;
};

namespace gcpk {
// Words per packed nonzero record: d int32 coordinates, the value's bits,
// then the d 16-bit gradient replica slots of its rows (0xFFFF = none),
// padded to 16, 32 or 64 bytes so a record sits in whole 32-byte sectors
// and loads as 16-byte vectors.
__host__ __device__ constexpr int rec_words_for(int d) {
    return d + 1 + (d + 1) / 2 <= 4 ? 4 : (d + 1 + (d + 1) / 2 <= 8 ? 8 : 16);
}
constexpr unsigned kNoSlot = 0xFFFFu;
}  // namespace gcpk

// Deterministic MTTKRP gradient of one sample set (gcp_mttkrp_det.cu): fills
// f.G and the loss partials; *blocks = number of partials written.
gcp_status gcpk_det_grad(gcp_ctx *c, const gcpk::FusedSpec &f, int *blocks);

// Record the message of a failed call that has no context; gcp_last_error(NULL)
// returns it.
void gcpk_set_noctx_error(const char *msg);

// Fused-pass parameters of one sample set of a context (weights returned in
// FP64), and the sample-count checks of the sampling calls.
gcpk::FusedSpec gcpk_make_spec(const gcp_ctx *c, uint64_t iter, int64_t p, int64_t q, bool grad,
                               const float *dscale, double *w_nz_out, double *w_z_out);
gcp_status gcpk_check_counts(gcp_ctx *c, int64_t p, int64_t q);

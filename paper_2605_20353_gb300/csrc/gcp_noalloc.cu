// gcp_noalloc.cu -- sampled GCP loss and gradient of a caller-supplied
// sample list, without any device allocation.
//
// Some callers cannot allocate device memory: code that runs under a device
// memory budget fixed when it starts (a host framework that owns every
// allocation through its own pool, or a long-running service that must not
// grow its footprint after start-up).  This entry point takes all of its
// inputs and outputs from the caller and keeps its only scratch -- one loss
// partial per block -- in the file-scope device array below.  That array is
// part of the library image: every GPU that loads the library holds it
// (GCP_NOALLOC_MAX_SAMPLES / 2048 blocks x 16 bytes = 128 KB) until the
// process exits.
#include <mutex>

#include "../../include/gcp.h"
#include "gcp_device.cuh"
#include "gcp_internal.h"

using namespace gcpdev;

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaSamplesPerBlock = 2048;
constexpr int kNaMaxBlocks = (int)(GCP_NOALLOC_MAX_SAMPLES / kNaSamplesPerBlock);
constexpr int kNaMaxDevices = 64;

// Per-block (loss partial, skipped-sample count), shared by every call on a
// device.  Each call writes the slots of the blocks it launches before it
// reads them, so nothing has to start at zero; calls that overlap on the
// GPU race on these slots.
__device__ __align__(256) double2 g_na_partials[kNaMaxBlocks];

struct NaShape {
    int d, R;
    int64_t dims[GCP_MAX_NDIM];
    int64_t rowoff[GCP_MAX_NDIM];
};

// One warp per sample; lane l owns columns l, l+32, ... of the rows.
__global__ void __launch_bounds__(kNaThreads) k_na_grad(const NaShape sh, int loss, int64_t n,
                                                        const int32_t *__restrict__ idx, const float *__restrict__ x,
                                                        const float *__restrict__ w, const float *__restrict__ A,
                                                        float *__restrict__ G, double2 *partials) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t first = (int64_t)blockIdx.x * kNaSamplesPerBlock;
    const int64_t last = first + kNaSamplesPerBlock < n ? first + kNaSamplesPerBlock : n;
    double acc = 0.0, skipped = 0.0;
    for (int64_t s = first + warp; s < last; s += kNaThreads / 32) {
        int32_t ii[GCP_MAX_NDIM];
        bool ok = true;
        for (int k = 0; k < sh.d; ++k) {
            ii[k] = idx[s * sh.d + k];
            ok = ok && ii[k] >= 0 && ii[k] < sh.dims[k];
        }
        if (!ok) {  // out-of-range coordinates: the sample is skipped and counted
            skipped += 1.0;
            continue;
        }
        float m = 0.0f;
        for (int r = lane; r < sh.R; r += 32) {
            float prod = 1.0f;
            for (int k = 0; k < sh.d; ++k) prod *= __ldg(A + (sh.rowoff[k] + ii[k]) * sh.R + r);
            m += prod;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xFFFFFFFFu, m, o);
        float f, df;
        loss_eval(loss, __ldg(x + s), m, f, df);
        const float ws = __ldg(w + s);
        acc += (double)ws * (double)f;
        const float y = ws * df;
        for (int r = lane; r < sh.R; r += 32) {
            for (int nmode = 0; nmode < sh.d; ++nmode) {
                float prod = y;
                for (int k = 0; k < sh.d; ++k)
                    if (k != nmode) prod *= __ldg(A + (sh.rowoff[k] + ii[k]) * sh.R + r);
                atomicAdd(G + (sh.rowoff[nmode] + ii[nmode]) * sh.R + r, prod);
            }
        }
    }
    // block partial: lane 0 of each warp holds the warp's sums
    __shared__ double2 red[kNaThreads / 32];
    if (lane == 0) red[warp] = make_double2(acc, skipped);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int i = 0; i < kNaThreads / 32; ++i) {
            t.x += red[i].x;
            t.y += red[i].y;
        }
        partials[blockIdx.x] = t;
    }
}

// Fixed-order sum of the block partials: loss_out[0] = loss,
// loss_out[1] = samples skipped for out-of-range coordinates.
__global__ void __launch_bounds__(kNaThreads) k_na_sum(const double2 *partials, int nblocks, double *loss_out) {
    __shared__ double2 sh[kNaThreads];
    double2 t = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nblocks; b += kNaThreads) {
        t.x += partials[b].x;
        t.y += partials[b].y;
    }
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int h = kNaThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sh[threadIdx.x].x += sh[threadIdx.x + h].x;
            sh[threadIdx.x].y += sh[threadIdx.x + h].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        loss_out[0] = sh[0].x;
        loss_out[1] = sh[0].y;
    }
}

// Device address of g_na_partials, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so the kernel must be
// given the address that cudaGetSymbolAddress returns for the current
// device.
std::mutex g_na_mutex;
double2 *g_na_addr[kNaMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = static_cast<double2 *>(p);
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}

gcp_status na_fail(gcp_status s, const char *msg) {
    gcpk_set_noctx_error(msg);  // read back with gcp_last_error(NULL)
    return s;
}

}  // namespace

extern "C" gcp_status gcp_grad_samples_noalloc(int32_t ndim, const int64_t *dims, int32_t rank, int32_t loss,
                                               int64_t nsamples, const int32_t *idx, const float *x, const float *w,
                                               const float *A, float *G, double *loss_out, void *stream) {
    if (ndim < 2 || ndim > GCP_MAX_NDIM || !dims) return na_fail(GCP_ERR_ARG, "ndim must be in 2..8");
    if (rank < 1 || rank > GCP_MAX_RANK) return na_fail(GCP_ERR_ARG, "rank must be in 1..128");
    if (loss < GCP_GAUSSIAN || loss > GCP_GAMMA) return na_fail(GCP_ERR_ARG, "unknown loss");
    if (nsamples < 0) return na_fail(GCP_ERR_ARG, "nsamples < 0");
    if (nsamples > GCP_NOALLOC_MAX_SAMPLES)
        return na_fail(GCP_ERR_ARG, "nsamples exceeds GCP_NOALLOC_MAX_SAMPLES (16777216), the capacity of this "
                                    "entry point's fixed scratch; split the samples over several calls");
    if (!A || !G || !loss_out || (nsamples > 0 && (!idx || !x || !w)))
        return na_fail(GCP_ERR_ARG, "NULL device pointer");
    NaShape sh{};
    sh.d = ndim;
    sh.R = rank;
    int64_t rows = 0;
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 1 || dims[k] > INT32_MAX) return na_fail(GCP_ERR_ARG, "mode size out of range");
        sh.dims[k] = dims[k];
        sh.rowoff[k] = rows;
        rows += dims[k];
    }
    double2 *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return na_fail(GCP_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((e = cudaMemsetAsync(G, 0, (size_t)rows * rank * sizeof(float), st)) != cudaSuccess)
        return na_fail(GCP_ERR_CUDA, cudaGetErrorString(e));
    const int nblocks = (int)((nsamples + kNaSamplesPerBlock - 1) / kNaSamplesPerBlock);
    if (nblocks > 0) k_na_grad<<<nblocks, kNaThreads, 0, st>>>(sh, loss, nsamples, idx, x, w, A, G, scratch);
    k_na_sum<<<1, kNaThreads, 0, st>>>(scratch, nblocks, loss_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(GCP_ERR_CUDA, cudaGetErrorString(e));
    return GCP_OK;
}

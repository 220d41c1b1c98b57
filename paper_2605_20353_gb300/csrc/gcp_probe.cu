// gcp_probe.cu -- measured ceilings of the L2-resident model traffic.
//
// The fused pass gathers factor rows and adds gradient rows that stay in
// L2, so its binding limit is the SM -> L2 path, not HBM.  These probes move
// whole rows of an L2-resident buffer in the fused pass's own access
// pattern and nothing else (no sampling, no loss), so that the pass's row
// traffic can be set against what the hardware sustains for that pattern:
//   GCP_PROBE_RED : per op, one group of Rp/4 lanes adds a 16-byte slice per
//                   lane (red.global.add.v4.f32) to each of `rows_per_op`
//                   random rows -- the scatter of the atomic MTTKRP;
//   GCP_PROBE_LOAD: the same rows read with 16-byte vector loads -- the
//                   factor gathers;
//   GCP_PROBE_BOTH: per op, `rows_per_op` rows read, then `rows_per_op`
//                   other rows added -- one sample's model traffic.
// Rows are drawn by a splitmix64 hash of the op index, uniformly.  The lanes
// of a group cover a row as the fused pass's do: one 16-byte quad per lane
// for rows of up to 32 floats, two (columns 4g.. and Rp/2 + 4g..) above.
#include "../../include/gcp.h"
#include "gcp_device.cuh"
#include "gcp_internal.h"

using namespace gcpdev;

namespace {

constexpr int kProbeThreads = 256;

template <int KIND, int NQ>
__global__ void __launch_bounds__(kProbeThreads) k_probe(float *__restrict__ buf, int64_t rows, int log2L,
                                                         int rows_per_op, int64_t ops, float *sink) {
    const int L = 1 << log2L, Rp = 4 * NQ * L;
    const int lane = threadIdx.x & 31, glane = lane & (L - 1);
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) >> log2L;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> log2L;
    float acc = 0.0f;
    for (int64_t op = g0; op < ops; op += ngroups) {
        uint64_t h = mix64((uint64_t)op * 0x9E3779B97F4A7C15ull + 1);
        if (KIND != 0) {
            for (int k = 0; k < rows_per_op; ++k) {
                const int64_t r = (int64_t)__umul64hi(h, (uint64_t)rows);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 v =
                        __ldg(reinterpret_cast<const float4 *>(buf + r * Rp + q * (Rp >> 1) + 4 * glane));
                    acc += v.x + v.y + v.z + v.w;
                }
                h = mix64(h);
            }
        }
        if (KIND != 1) {
            const float y = 1e-30f * (float)(op & 7);
            for (int k = 0; k < rows_per_op; ++k) {
                const int64_t r = (int64_t)__umul64hi(h, (uint64_t)rows);
#pragma unroll
                for (int q = 0; q < NQ; ++q) red_add_v4(buf + r * Rp + q * (Rp >> 1) + 4 * glane, y + acc, y, y, y);
                h = mix64(h);
            }
        }
    }
    if (KIND == 1 && isnan(acc)) sink[0] = acc;  // keeps the loads; never true for a buffer of finite values
}

}  // namespace

extern "C" gcp_status gcp_probe_l2(int32_t kind, int32_t row_floats, int32_t rows_per_op, float *buf, int64_t rows,
                                   int64_t ops, void *stream) {
    if (kind < GCP_PROBE_RED || kind > GCP_PROBE_BOTH) {
        gcpk_set_noctx_error("gcp_probe_l2: unknown kind");
        return GCP_ERR_ARG;
    }
    if (row_floats < 4 || row_floats > 128 || (row_floats & (row_floats - 1))) {
        gcpk_set_noctx_error("gcp_probe_l2: row_floats must be a power of two in 4..128");
        return GCP_ERR_ARG;
    }
    if (rows_per_op < 1 || rows_per_op > GCP_MAX_NDIM || rows < 1 || ops < 0 || !buf ||
        (reinterpret_cast<uintptr_t>(buf) & 15)) {
        gcpk_set_noctx_error("gcp_probe_l2: rows_per_op in 1..8, rows >= 1, ops >= 0, 16-byte aligned buffer");
        return GCP_ERR_ARG;
    }
    const int nq = row_floats > 32 ? 2 : 1;  // quads per lane, as in the fused pass
    const int L = row_floats / (4 * nq);
    int log2L = 0;
    while ((1 << log2L) < L) ++log2L;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups_per_block = kProbeThreads / L;
    int64_t blocks = (ops + groups_per_block - 1) / groups_per_block;
    const int64_t cap = (int64_t)sms * 8;  // full residency, then a persistent loop
    if (blocks > cap) blocks = cap;
    if (blocks < 1) return GCP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // rows x row_floats floats; the load probe's sink is the buffer's first float
#define GCP_PROBE_LAUNCH(K)                                                                             \
    (nq == 2 ? k_probe<K, 2><<<(int)blocks, kProbeThreads, 0, st>>>(buf, rows, log2L, rows_per_op, ops, buf) \
             : k_probe<K, 1><<<(int)blocks, kProbeThreads, 0, st>>>(buf, rows, log2L, rows_per_op, ops, buf))
    if (kind == GCP_PROBE_RED)
        GCP_PROBE_LAUNCH(0);
    else if (kind == GCP_PROBE_LOAD)
        GCP_PROBE_LAUNCH(1);
    else
        GCP_PROBE_LAUNCH(2);
#undef GCP_PROBE_LAUNCH
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gcpk_set_noctx_error(cudaGetErrorString(e));
        return GCP_ERR_CUDA;
    }
    return GCP_OK;
}

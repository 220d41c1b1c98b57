// gcp_batch_fused.cuh -- the multi-client fused sampled-gradient kernel of
// the batched clients (gcp_batch.cu), templated on the order D, the factor
// storage TF, the columns per lane COLS and the samples per warp tile TS.
// Each tile size is instantiated in its own translation unit
// (gcp_batch_fused_t16.cu, _t32.cu, _t64.cu) so that they compile in
// parallel; gcp_batch.cu reaches them through batch_fused_launch<TS>,
// batch_fused_allow<TS> and batch_fused_occupancy<TS>.
#pragma once

#include <cuda_bf16.h>

#include "gcp_device.cuh"
#include "gcp_internal.h"

namespace gcpb {

using namespace gcpdev;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSpecWords = (int)((sizeof(gcpk::FusedSpec) + 15) / 16);  // 16-byte words of a FusedSpec

template <int D>
__device__ __forceinline__ void draw_tuple_b(const gcpk::SampleSpec &S, uint64_t stream, uint64_t j, uint64_t sub0,
                                             int32_t (&idx)[D]) {
#pragma unroll
    for (int b = 0; 4 * b < D; ++b) {
        const U64x4 w = philox4x64_10(j, sub0 + (uint64_t)b, S.iter, 0, S.seed, stream);
#pragma unroll
        for (int k = 4 * b; k < D && k < 4 * b + 4; ++k)
            idx[k] = (int32_t)map_range(w.v[k - 4 * b], (uint64_t)S.dims[k]);
    }
}

template <int D>
__device__ __forceinline__ uint64_t linear_b(const gcpk::SampleSpec &S, const int32_t (&idx)[D]) {
    uint64_t L = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) L += (uint64_t)idx[k] * S.stride[k];
    return L;
}

__device__ __forceinline__ int client_of(const int *__restrict__ tile_start, int nclients, int tile) {
    int lo = 0, hi = nclients;  // last c with tile_start[c] <= tile
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(tile_start + mid) <= tile)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Multi-client fused sampled gradient.  Each client's FusedSpec (stored as
// kSpecWords 16-byte words) gives its tensor, model, gradient and weights;
// the iteration number is step[0].  A tile holds TS consecutive samples of
// one client (TS = 16, 32 or 64 samples per warp, a tuning knob): in phase
// A, lane l stages the samples at positions l, l + 32, ... of the tile
// (for TS = 16 lanes 16..31 stage nothing); in phase B the warp's groups
// take the tile's samples in turn.  Per tile, the FP32 loss sums (nonzero,
// zero) go to tile_loss[tile].
template <int D, typename TF, int COLS, int TS>
__global__ void __launch_bounds__(kThreads, (D <= 4 ? (COLS == 4 ? 4 : 3) : 1)) k_batch_fused(const int4 *__restrict__ specs,
                                                         const int *__restrict__ tile_start, int nclients,
                                                         int total_tiles, int log2L, int Rp,
                                                         const uint64_t *__restrict__ step, float2 *tile_loss) {
    constexpr int SW = gcpk::rec_words_for(D);
    constexpr int NQ = COLS / 4;
    constexpr int SPL = TS >= 32 ? TS / 32 : 1;  // tile positions a lane stages
    static_assert(TS == 16 || TS == 32 || TS == 64, "16, 32 or 64 samples per warp");
    // staging in dynamic shared memory (batch_fused_smem bytes; 64-sample
    // tiles need more than the 48 KB a kernel may declare statically)
    extern __shared__ __align__(16) unsigned char smem[];
    auto &s_slot = *reinterpret_cast<int32_t(*)[2][kWarps][TS][SW]>(smem);
    auto &s_bkt = *reinterpret_cast<uint64_t(*)[2][kWarps][TS][4]>(smem + sizeof(int32_t) * 2 * kWarps * TS * SW);
    auto &s_spec = *reinterpret_cast<int4(*)[2][kWarps][kSpecWords]>(
        smem + sizeof(int32_t) * 2 * kWarps * TS * SW + sizeof(uint64_t) * 2 * kWarps * TS * 4);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int L = 1 << log2L;
    const int glane = lane & (L - 1);
    const int grp = lane >> log2L;
    const int ngrp = 32 >> log2L;
    const unsigned gmask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (grp * L));
    int col[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) col[q] = q * (Rp >> 1) + 4 * glane;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t iter = __ldg(step);
    int cur_client[2] = {-1, -1};

    auto spec_of = [&](int st) -> const gcpk::FusedSpec & {
        return *reinterpret_cast<const gcpk::FusedSpec *>(&s_spec[st][warp][0]);
    };
    // Stage the parameters of the client owning `tile` (whole warp).
    auto stage_spec = [&](int tile, int st) -> int {
        const int c = client_of(tile_start, nclients, tile);
        if (c != cur_client[st]) {
            const int4 *src = specs + (size_t)c * kSpecWords;  // specs padded to kSpecWords words
            for (int i = lane; i < kSpecWords; i += 32) s_spec[st][warp][i] = __ldg(src + i);
            __syncwarp();
            if (lane == 0) reinterpret_cast<gcpk::FusedSpec *>(&s_spec[st][warp][0])->s.iter = iter;
            __syncwarp();
            cur_client[st] = c;
        }
        return c;
    };

    // A1: start the draws of this lane's positions of `tile` into stage st;
    // key[j] = the stratified zero candidate of position lane + 32 j, else kEmpty.
    auto issue = [&](int tile, int st, uint64_t (&key)[SPL]) {
#pragma unroll
        for (int j = 0; j < SPL; ++j) key[j] = kEmpty;
        if (tile >= total_tiles) return;
        const int c = stage_spec(tile, st);
        const gcpk::FusedSpec &P = spec_of(st);
        const int p = (int)P.s.p, S = (int)(P.s.p + P.s.q);
        const int base = (tile - __ldg(tile_start + c)) * TS;
        const bool semi = P.s.sampling == GCP_SAMPLING_SEMI_STRATIFIED;
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const int pos = lane + 32 * j;
            const int s = base + pos;
            if (pos >= TS || s >= S) continue;
            int32_t *slot = s_slot[st][warp][pos];
            if (s < p) {
                const U64x4 w = philox4x64_10((uint64_t)s, 0, P.s.iter, 0, P.s.seed, kStreamNonzero);
                const int32_t *rec = P.s.rec + map_range(w.v[0], (uint64_t)P.s.nnz) * SW;
#pragma unroll
                for (int v = 0; v < SW / 4; ++v) cp_async16(slot + 4 * v, rec + 4 * v);
                continue;
            }
            int32_t idx[D];
            draw_tuple_b<D>(P.s, semi ? kStreamSemiZero : kStreamZero, (uint64_t)(s - p), 0, idx);
#pragma unroll
            for (int k = 0; k < D; ++k) slot[k] = idx[k];
            slot[D] = 0;
            if (semi) continue;
            key[j] = linear_b<D>(P.s, idx);
            const uint64_t *b = P.s.hkeys + 4 * (mix64(key[j]) & P.s.hbmask);
            cp_async16(&s_bkt[st][warp][pos][0], b);
            cp_async16(&s_bkt[st][warp][pos][2], b + 2);
        }
    };

    // A2: finish the draw of position pos of stage st; whether the sample exists.
    auto finish = [&](int tile, int st, uint64_t key, int pos) -> bool {
        const gcpk::FusedSpec &P = spec_of(st);
        const int p = (int)P.s.p, S = (int)(P.s.p + P.s.q);
        const int s = (tile - __ldg(tile_start + cur_client[st])) * TS + pos;
        if (pos >= TS || s >= S) return false;
        if (key == kEmpty) return true;
        const ulonglong2 lo = *reinterpret_cast<const ulonglong2 *>(&s_bkt[st][warp][pos][0]);
        const ulonglong2 hi = *reinterpret_cast<const ulonglong2 *>(&s_bkt[st][warp][pos][2]);
        int h = bucket_decide(lo, hi, key);
        if (h == 2)
            h = hash_contains_from(P.s.hkeys, P.s.hbmask, key, ((mix64(key) & P.s.hbmask) + 1) & P.s.hbmask, 1);
        if (h == 0) return true;
        int32_t *slot = s_slot[st][warp][pos];
        const uint64_t j = (uint64_t)(s - p);
        for (int a = 1; h == 1 && a < P.s.max_attempts; ++a) {
            int32_t idx[D];
            draw_tuple_b<D>(P.s, kStreamZero, j, 4 * (uint64_t)a, idx);
            h = hash_contains(P.s.hkeys, P.s.hbmask, linear_b<D>(P.s, idx));
            if (h == 0) {
#pragma unroll
                for (int k = 0; k < D; ++k) slot[k] = idx[k];
                return true;
            }
        }
        atomicOr(P.s.status, h < 0 ? kErrHashFull : kErrExhausted);
        return false;
    };

    int tile = warp0;
    uint64_t key_next[SPL];
    issue(tile, 0, key_next);
    cp_async_commit();
    for (int st = 0; tile < total_tiles; tile += nwarps, st ^= 1) {
        uint64_t key[SPL];
#pragma unroll
        for (int j = 0; j < SPL; ++j) key[j] = key_next[j];
        __syncwarp();
        issue(tile + nwarps, st ^ 1, key_next);
        cp_async_commit();
        cp_async_wait<1>();
        uint64_t okmask = 0;  // bit pos: the sample at tile position pos exists
#pragma unroll
        for (int j = 0; j < SPL; ++j)
            okmask |= (uint64_t)__ballot_sync(0xFFFFFFFFu, finish(tile, st, key[j], lane + 32 * j)) << (32 * j);
        __syncwarp();

        const gcpk::FusedSpec &P = spec_of(st);
        const TF *__restrict__ F = static_cast<const TF *>(P.F);
        const int p = (int)P.s.p;
        const int tbase = (tile - __ldg(tile_start + cur_client[st])) * TS;
        const bool semi = P.s.sampling == GCP_SAMPLING_SEMI_STRATIFIED;
        float *const grep = P.Grep ? P.Grep + (size_t)(warp0 & (gcpk::kReplicas - 1)) * P.Htot * Rp : nullptr;
        float tf_nz = 0.0f, tf_z = 0.0f;
        for (int it = 0; it * ngrp < TS; ++it) {
            const int src = it * ngrp + grp;
            if (src >= TS || !((okmask >> src) & 1ull)) continue;  // uniform within the group
            const int32_t *slot = s_slot[st][warp][src];
            int32_t ii[D];
#pragma unroll
            for (int k = 0; k < D; ++k) ii[k] = slot[k];
            const float xs = __int_as_float(slot[D]);
            const bool is_nz = (tbase + src) < p;
            int off[D];
            float a[D][COLS];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                off[k] = (P.rowoff[k] + ii[k]) * Rp;
#pragma unroll
                for (int q = 0; q < NQ; ++q) Quad<TF>::load(F + off[k] + col[q], a[k] + 4 * q);
            }
            float suf[D][COLS];
#pragma unroll
            for (int v = 0; v < COLS; ++v) suf[D - 1][v] = 1.0f;
#pragma unroll
            for (int k = D - 2; k >= 0; --k)
#pragma unroll
                for (int v = 0; v < COLS; ++v) suf[k][v] = suf[k + 1][v] * a[k + 1][v];
            float m = 0.0f;
#pragma unroll
            for (int v = 0; v < COLS; ++v) m = fmaf(a[0][v], suf[0][v], m);
            for (int o = L >> 1; o > 0; o >>= 1) m += __shfl_xor_sync(gmask, m, o);
            float f, df;
            loss_eval(P.loss, xs, m, f, df);
            if (semi && is_nz) {
                float f0, df0;
                loss_eval(P.loss, 0.0f, m, f0, df0);
                f -= f0;
                df -= df0;
            }
            if (is_nz)
                tf_nz += f;
            else
                tf_z += f;
            const float y = (is_nz ? P.w_nz : P.w_z) * df;
            float pre[COLS];
#pragma unroll
            for (int v = 0; v < COLS; ++v) pre[v] = y;
#pragma unroll
            for (int n = 0; n < D; ++n) {
                unsigned hs;
                if (is_nz)
                    hs = ((unsigned)slot[D + 1 + n / 2] >> (16 * (n & 1))) & 0xFFFFu;
                else
                    hs = P.small_base[n] >= 0 ? (unsigned)(P.small_base[n] + ii[n]) : gcpk::kNoSlot;
                float *g = hs != gcpk::kNoSlot ? grep + (int)hs * Rp : P.G + off[n];
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    red_add_v4(g + col[q], pre[4 * q] * suf[n][4 * q], pre[4 * q + 1] * suf[n][4 * q + 1],
                               pre[4 * q + 2] * suf[n][4 * q + 2], pre[4 * q + 3] * suf[n][4 * q + 3]);
#pragma unroll
                for (int v = 0; v < COLS; ++v) pre[v] *= a[n][v];
            }
        }
        // tile loss sums: one value per group leader, reduced over the warp
        if (glane != 0) tf_nz = tf_z = 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tf_nz += __shfl_xor_sync(0xFFFFFFFFu, tf_nz, o);
            tf_z += __shfl_xor_sync(0xFFFFFFFFu, tf_z, o);
        }
        if (lane == 0) tile_loss[tile] = make_float2(tf_nz, tf_z);
    }
    cp_async_wait<0>();
}

// Dynamic shared memory of k_batch_fused<D, *, *, TS>: the double-buffered
// sample slots and hash buckets of every warp, and the staged client specs.
constexpr size_t batch_fused_smem(int d, int ts) {
    return (size_t)2 * kWarps * ts * (gcpk::rec_words_for(d) * sizeof(int32_t) + 4 * sizeof(uint64_t)) +
           (size_t)2 * kWarps * kSpecWords * sizeof(int4);
}

using FusedKernel = void (*)(const int4 *, const int *, int, int, int, int, const uint64_t *, float2 *);

// The instantiation for (dtype, cols); with `allow`, its dynamic shared
// memory limit is raised to what it needs (a host call made before any
// launch or stream capture that uses it, on the batch's device).
template <int D, typename TF, int COLS, int TS>
cudaError_t fused_kernel_of(FusedKernel *k, bool allow) {
    *k = k_batch_fused<D, TF, COLS, TS>;
    if (!allow) return cudaSuccess;
    return cudaFuncSetAttribute(k_batch_fused<D, TF, COLS, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batch_fused_smem(D, TS));
}

template <int D, int TS>
cudaError_t fused_kernel_ts(bool bf16, int cols, FusedKernel *k, bool allow) {
    if (bf16)
        return cols == 8 ? fused_kernel_of<D, __nv_bfloat16, 8, TS>(k, allow)
                         : fused_kernel_of<D, __nv_bfloat16, 4, TS>(k, allow);
    return cols == 8 ? fused_kernel_of<D, float, 8, TS>(k, allow) : fused_kernel_of<D, float, 4, TS>(k, allow);
}

template <int D, int TS>
cudaError_t launch_fused_ts(bool bf16, int cols, int blocks, const int4 *specs, const int *tile_start, int n,
                            int total_tiles, int log2L, int Rp, const uint64_t *step, float2 *tile_loss,
                            cudaStream_t st) {
    FusedKernel k = nullptr;
    cudaError_t e = fused_kernel_ts<D, TS>(bf16, cols, &k, false);
    if (e != cudaSuccess) return e;
    k<<<blocks, kThreads, batch_fused_smem(D, TS), st>>>(specs, tile_start, n, total_tiles, log2L, Rp, step,
                                                          tile_loss);
    return cudaGetLastError();
}

template <int D, int TS>
int occupancy_ts(bool bf16, int cols) {
    FusedKernel k = nullptr;
    int per_sm = 0;
    if (fused_kernel_ts<D, TS>(bf16, cols, &k, true) == cudaSuccess)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, batch_fused_smem(D, TS));
    return per_sm < 1 ? 1 : per_sm;
}

// Per tile size: the launch, the raised shared-memory limit (a host call
// before any launch or capture that uses the kernel) and the resident
// blocks per SM, for an order d in 2..8.
#define GCPB_FOR_D(d, EXPR)  \
    switch (d) {               \
    case 2: { constexpr int D = 2; EXPR; } \
    case 3: { constexpr int D = 3; EXPR; } \
    case 4: { constexpr int D = 4; EXPR; } \
    case 5: { constexpr int D = 5; EXPR; } \
    case 6: { constexpr int D = 6; EXPR; } \
    case 7: { constexpr int D = 7; EXPR; } \
    case 8: { constexpr int D = 8; EXPR; } \
    default: break;            \
    }

template <int TS>
cudaError_t batch_fused_launch(int d, bool bf16, int cols, int blocks, const int4 *specs, const int *tile_start,
                               int n, int total_tiles, int log2L, int Rp, const uint64_t *step, float2 *tile_loss,
                               cudaStream_t st) {
    GCPB_FOR_D(d, return (launch_fused_ts<D, TS>(bf16, cols, blocks, specs, tile_start, n, total_tiles, log2L, Rp,
                                                 step, tile_loss, st)))
    return cudaErrorInvalidValue;
}

template <int TS>
cudaError_t batch_fused_allow(int d, bool bf16, int cols) {
    FusedKernel k = nullptr;
    GCPB_FOR_D(d, return (fused_kernel_ts<D, TS>(bf16, cols, &k, true)))
    return cudaErrorInvalidValue;
}

template <int TS>
int batch_fused_occupancy(int d, bool bf16, int cols) {
    GCPB_FOR_D(d, return (occupancy_ts<D, TS>(bf16, cols)))
    return 1;
}

#undef GCPB_FOR_D

}  // namespace gcpb

// gcp_kernels.cu -- the fused stochastic GCP gradient on sm_103a.
//
// One pass per sample set (the fused Sampling-MTTKRP of Sec. 3.1.2, here with
// stratified sampling and hash rejection):
//   phase A, one sample per lane: Philox4x64-10 counters -> nonzero record
//            load, or zero candidates probed against the nonzero hash set
//            until one is absent (Sec. 3.1.1);
//   phase B, one sample per group of L = Rp / (16 B / elt) lanes: each lane
//            gathers a 16-byte slice of the d factor rows, forms the CP model
//            entry m (Eq. cp) with a shuffle reduction over the group,
//            evaluates f and f', and scatters w f' prod_{k!=n} A_k(i_k,:)
//            into every mode's gradient row with FP32 vector reductions
//            (Eq. gcp-gradient, atomic MTTKRP of Sec. 3.1.2).
// The sampled loss is accumulated in FP64 per lane, reduced per block into
// a partials array and finished by a single-block kernel in fixed order.
#include <cuda_bf16.h>

#include "gcp_device.cuh"
#include "gcp_epilogue.cuh"
#include "gcp_internal.h"

using namespace gcpdev;

namespace gcpk {

constexpr int kThreads = 256;

static int elementwise_blocks(int64_t n);
static int num_sms();

struct RowOffsets {
    int64_t off[GCP_MAX_NDIM];
};

template <int D>
__device__ __forceinline__ void draw_tuple(const SampleSpec &S, uint64_t stream, uint64_t j, uint64_t sub0,
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
__device__ __forceinline__ uint64_t linear_of(const SampleSpec &S, const int32_t (&idx)[D]) {
    uint64_t L = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) L += (uint64_t)idx[k] * S.stride[k];
    return L;
}

template <int D>
__device__ __forceinline__ void load_record(const int32_t *__restrict__ rec, uint64_t e, int32_t (&idx)[D],
                                            float &x) {
    constexpr int NV = (D + 4) / 4;  // 16-byte vectors holding D coordinates + value
    constexpr int RW = rec_words_for(D);
    const int4 *r = reinterpret_cast<const int4 *>(rec + e * RW);
    int w[4 * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const int4 t = __ldg(r + v);
        w[4 * v] = t.x;
        w[4 * v + 1] = t.y;
        w[4 * v + 2] = t.z;
        w[4 * v + 3] = t.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) idx[k] = w[k];
    x = __int_as_float(w[D]);
}

// Draw sample s of the set.  Returns false when the sample does not exist
// (exhausted zero draw); idx then holds the last candidate.
template <int D>
__device__ __forceinline__ bool draw_sample(const SampleSpec &S, int64_t s, int32_t (&idx)[D], float &x,
                                            int &attempts) {
    if (S.sampling == GCP_SAMPLING_UNIFORM) {
        draw_tuple<D>(S, kStreamUniform, (uint64_t)s, 0, idx);
        x = __ldg(S.dense + linear_of<D>(S, idx));
        return true;
    }
    if (s < S.p) {
        const U64x4 w = philox4x64_10((uint64_t)s, 0, S.iter, 0, S.seed, kStreamNonzero);
        load_record<D>(S.rec, map_range(w.v[0], (uint64_t)S.nnz), idx, x);
        return true;
    }
    const uint64_t j = (uint64_t)(s - S.p);
    x = 0.0f;
    if (S.sampling == GCP_SAMPLING_SEMI_STRATIFIED) {
        draw_tuple<D>(S, kStreamSemiZero, j, 0, idx);
        return true;
    }
    for (int a = 0; a < S.max_attempts; ++a) {
        draw_tuple<D>(S, kStreamZero, j, 4 * (uint64_t)a, idx);
        const int h = hash_contains(S.hkeys, S.hbmask, linear_of<D>(S, idx));
        if (h == 0) {
            attempts += a + 1;
            return true;
        }
        if (h < 0) {
            atomicOr(S.status, kErrHashFull);
            return false;
        }
    }
    attempts += S.max_attempts;
    atomicOr(S.status, kErrExhausted);
    return false;
}

// ------------------------------------------------------------ fused pass
// Per warp and per tile of 32 consecutive samples:
//   A1 (tile t+1, one sample per lane): Philox draw; the nonzero record, the
//      dense value or the first hash bucket of the zero candidate is copied
//      into shared memory with cp.async while tile t is processed;
//   A2 (tile t): finish the draw -- a zero candidate found in its bucket is
//      rejected and redrawn with direct probes (rare: 1/(1-N/M) attempts);
//   B  (tile t, one sample per group of L = Rp/COLS lanes): lane g owns
//      COLS columns as COLS/4 quads (4g..4g+3, and Rp/2+4g.. when COLS = 8),
//      so a group's loads and vector reductions cover whole 32-byte sectors
//      and, for rows up to 128 bytes, one whole row per instruction.
// Gradient rows that many samples hit go to one of kReplicas replicas
// (chosen by warp), folded into G afterwards, so that the reductions of hot
// rows do not serialise on one address.
constexpr int kWarps = kThreads / 32;

template <int D, typename TF, int COLS>
__global__ void __launch_bounds__(kThreads, (D <= 4 ? (COLS == 4 ? 4 : 3) : 1)) k_fused(const FusedSpec P) {
    constexpr int SW = rec_words_for(D);  // words per staged sample: coordinates, value, replica slots
    constexpr int NQ = COLS / 4;          // quads of columns per lane
    __shared__ __align__(16) int32_t s_slot[2][kWarps][32][SW];
    __shared__ __align__(16) uint64_t s_bkt[2][kWarps][32][4];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int log2L = P.log2L;
    const int L = 1 << log2L;
    const int glane = lane & (L - 1);
    const int grp = lane >> log2L;
    const int ngrp = 32 >> log2L;
    const unsigned gmask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (grp * L));
    int col[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) col[q] = q * (P.Rp >> 1) + 4 * glane;
    const int p = (int)P.s.p;  // sample counts of one call are below 2^31
    const int S = (int)(P.s.p + P.s.q);
    const int ntiles = (int)(((int64_t)S + 31) >> 5);  // S may be 2^31 - 1
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const TF *__restrict__ F = static_cast<const TF *>(P.F);
    const float scale = P.dscale ? __ldg(P.dscale) : 1.0f;
    const bool semi = P.s.sampling == GCP_SAMPLING_SEMI_STRATIFIED;
    const bool uniform = P.s.sampling == GCP_SAMPLING_UNIFORM;
    float *const grep = P.Grep ? P.Grep + (size_t)(warp0 & (kReplicas - 1)) * P.Htot * P.Rp : nullptr;

    double acc_nz = 0.0, acc_z = 0.0;
    int attempts = 0;

    // A1: start the draw of this lane's sample of `tile` into stage `st`;
    // returns the key of a stratified zero candidate (kEmpty otherwise).
    auto issue = [&](int tile, int st) -> uint64_t {
        if (tile >= ntiles) return kEmpty;
        const int s = (tile << 5) + lane;
        int32_t *slot = s_slot[st][warp][lane];
        if (s >= S) return kEmpty;
        if (uniform) {
            int32_t idx[D];
            draw_tuple<D>(P.s, kStreamUniform, (uint64_t)s, 0, idx);
#pragma unroll
            for (int k = 0; k < D; ++k) slot[k] = idx[k];
            cp_async4(slot + D, P.s.dense + linear_of<D>(P.s, idx));
            return kEmpty;
        }
        if (s < p) {
            const U64x4 w = philox4x64_10((uint64_t)s, 0, P.s.iter, 0, P.s.seed, kStreamNonzero);
            const int32_t *rec = P.s.rec + map_range(w.v[0], (uint64_t)P.s.nnz) * SW;
#pragma unroll
            for (int v = 0; v < SW / 4; ++v) cp_async16(slot + 4 * v, rec + 4 * v);
            return kEmpty;
        }
        int32_t idx[D];
        draw_tuple<D>(P.s, semi ? kStreamSemiZero : kStreamZero, (uint64_t)(s - p), 0, idx);
#pragma unroll
        for (int k = 0; k < D; ++k) slot[k] = idx[k];
        slot[D] = 0;  // x = 0.0f
        if (semi) return kEmpty;
        const uint64_t key = linear_of<D>(P.s, idx);
        const uint64_t *b = P.s.hkeys + 4 * (mix64(key) & P.s.hbmask);
        cp_async16(&s_bkt[st][warp][lane][0], b);
        cp_async16(&s_bkt[st][warp][lane][2], b + 2);
        return key;
    };

    // A2: finish the draw of stage `st`; returns whether the sample exists.
    auto finish = [&](int tile, int st, uint64_t key) -> bool {
        const int s = (tile << 5) + lane;
        if (s >= S) return false;
        if (key == kEmpty) return true;  // nonzero, semi-stratified or dense draw
        const ulonglong2 lo = *reinterpret_cast<const ulonglong2 *>(&s_bkt[st][warp][lane][0]);
        const ulonglong2 hi = *reinterpret_cast<const ulonglong2 *>(&s_bkt[st][warp][lane][2]);
        int h = bucket_decide(lo, hi, key);
        if (h == 2)
            h = hash_contains_from(P.s.hkeys, P.s.hbmask, key, ((mix64(key) & P.s.hbmask) + 1) & P.s.hbmask, 1);
        if (h == 0) {
            attempts += 1;
            return true;
        }
        // rejected: redraw until a candidate is absent (Sec. 3.1.1)
        int32_t *slot = s_slot[st][warp][lane];
        const uint64_t j = (uint64_t)(s - p);
        for (int a = 1; h == 1 && a < P.s.max_attempts; ++a) {
            int32_t idx[D];
            draw_tuple<D>(P.s, kStreamZero, j, 4 * (uint64_t)a, idx);
            h = hash_contains(P.s.hkeys, P.s.hbmask, linear_of<D>(P.s, idx));
            if (h == 0) {
#pragma unroll
                for (int k = 0; k < D; ++k) slot[k] = idx[k];
                attempts += a + 1;
                return true;
            }
        }
        if (h < 0) {
            atomicOr(P.s.status, kErrHashFull);
        } else {
            attempts += P.s.max_attempts;
            atomicOr(P.s.status, kErrExhausted);
        }
        return false;
    };

    int tile = warp0;
    uint64_t key_next = issue(tile, 0);
    cp_async_commit();
    for (int st = 0; tile < ntiles; tile += nwarps, st ^= 1) {
        const uint64_t key = key_next;
        __syncwarp();  // stage st^1 is free: the previous tile's phase B is done
        key_next = issue(tile + nwarps, st ^ 1);
        cp_async_commit();
        cp_async_wait<1>();  // this lane's copies into stage st have landed
        const bool ok = finish(tile, st, key);
        const unsigned okmask = __ballot_sync(0xFFFFFFFFu, ok);
        __syncwarp();  // every lane's staged sample is visible to the warp

        // phase B: one sample per group; the group leader keeps FP32 loss
        // sums of the tile, added to the FP64 totals once per tile
        float tf_nz = 0.0f, tf_z = 0.0f;
        for (int it = 0; it < L; ++it) {
            const int src = it * ngrp + grp;
            if (!((okmask >> src) & 1u)) {  // uniform within the group
                const int sm = (tile << 5) + src;
                if (P.Yval && glane == 0 && sm < S) {  // no sample: a zero entry at a valid cell
#pragma unroll
                    for (int k = 0; k < D; ++k) P.Ycoord[(int64_t)sm * P.ystride + k] = s_slot[st][warp][src][k];
                    P.Yval[(int64_t)sm * P.vstride] = 0.0f;
                }
                continue;
            }
            const int32_t *slot = s_slot[st][warp][src];
            int32_t ii[D];
#pragma unroll
            for (int k = 0; k < D; ++k) ii[k] = slot[k];
            const float xs = __int_as_float(slot[D]);
            const bool is_nz = !uniform && ((tile << 5) + src) < p;

            int off[D];
            float a[D][COLS];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                off[k] = (P.rowoff[k] + ii[k]) * P.Rp;
#pragma unroll
                for (int q = 0; q < NQ; ++q) Quad<TF>::load(F + off[k] + col[q], a[k] + 4 * q);
            }
            float suf[D][COLS];  // suf[k] = prod_{j>k} a_j
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
            if (is_nz || uniform)
                tf_nz += f;
            else
                tf_z += f;
            if (P.Yval) {  // materialize the gradient tensor entry (non-fused MTTKRP input)
                if (glane == 0) {
                    const int sm = (tile << 5) + src;
#pragma unroll
                    for (int k = 0; k < D; ++k) P.Ycoord[(int64_t)sm * P.ystride + k] = ii[k];
                    P.Yval[(int64_t)sm * P.vstride] = ((is_nz || uniform) ? P.w_nz : P.w_z) * df * scale;
                }
            } else if (P.G) {
                const float y = ((is_nz || uniform) ? P.w_nz : P.w_z) * df * scale;
                float pre[COLS];
#pragma unroll
                for (int v = 0; v < COLS; ++v) pre[v] = y;
#pragma unroll
                for (int n = 0; n < D; ++n) {
                    // replica slot: stored in a nonzero's record; for drawn
                    // cells, rows of fully replicated modes only
                    unsigned hs;
                    if (is_nz)
                        hs = ((unsigned)slot[D + 1 + n / 2] >> (16 * (n & 1))) & 0xFFFFu;
                    else
                        hs = P.small_base[n] >= 0 ? (unsigned)(P.small_base[n] + ii[n]) : kNoSlot;
                    float *g = hs != kNoSlot ? grep + (int)hs * P.Rp : P.G + off[n];
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        red_add_v4(g + col[q], pre[4 * q] * suf[n][4 * q], pre[4 * q + 1] * suf[n][4 * q + 1],
                                   pre[4 * q + 2] * suf[n][4 * q + 2], pre[4 * q + 3] * suf[n][4 * q + 3]);
#pragma unroll
                    for (int v = 0; v < COLS; ++v) pre[v] *= a[n][v];
                }
            }
        }
        if (glane == 0) {
            acc_nz += (double)tf_nz;
            acc_z += (double)tf_z;
        }
    }
    cp_async_wait<0>();

    // block reduction of the FP64 loss sums and attempt counts
    double att = (double)attempts;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_nz += __shfl_xor_sync(0xFFFFFFFFu, acc_nz, o);
        acc_z += __shfl_xor_sync(0xFFFFFFFFu, acc_z, o);
        att += __shfl_xor_sync(0xFFFFFFFFu, att, o);
    }
    double(*red)[kWarps] = reinterpret_cast<double(*)[kWarps]>(&s_bkt[0][0][0][0]);  // staging is free now
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = acc_nz;
        red[1][warp] = acc_z;
        red[2][warp] = att;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += red[threadIdx.x][w];
        P.partials[4 * blockIdx.x + threadIdx.x] = t;
    }
}

// G(hot row) += sum over replicas, then the replicas are cleared for the
// next call (fixed replica order).  G may already hold contributions of
// drawn cells to a replicated row of a large mode.  All kReplicas loads of
// an element are issued before any add: there are few hot elements, so one
// round trip per element beats the occupancy that fewer registers would
// give (16 loads at a time measured 8 µs against 5 µs per launch).
__device__ __forceinline__ void fold_range(float *__restrict__ G, float *__restrict__ Grep,
                                           const int *__restrict__ hot_row, int Htot, int Rp, int64_t first,
                                           int64_t stride) {
    const int64_t n = (int64_t)Htot * Rp, plane = (int64_t)Htot * Rp;
    for (int64_t e = first; e < n; e += stride) {
        float v[kReplicas];
#pragma unroll
        for (int r = 0; r < kReplicas; ++r) v[r] = Grep[r * plane + e];
        float t = 0.0f;
#pragma unroll
        for (int r = 0; r < kReplicas; ++r) t += v[r];
#pragma unroll
        for (int r = 0; r < kReplicas; ++r) Grep[r * plane + e] = 0.0f;
        const int log2Rp = __ffs(Rp) - 1;  // Rp is a power of two
        const int slot = (int)(e >> log2Rp), col = (int)(e & (Rp - 1));
        G[(int64_t)hot_row[slot] * Rp + col] += t;
    }
}

__global__ void k_fold_replicas(float *__restrict__ G, float *__restrict__ Grep, const int *__restrict__ hot_row,
                                int Htot, int Rp) {
    fold_range(G, Grep, hot_row, Htot, Rp, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
               (int64_t)gridDim.x * blockDim.x);
}

// Fixed-order reduction of the block partials (one block).
__global__ void __launch_bounds__(kThreads) k_finish_loss(const double *__restrict__ partials, int nblocks,
                                                         double w_nz, double w_z, double *dloss, int *status) {
    __shared__ double sh[3][kThreads];
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int c = 0; c < 3; ++c) t[c] += partials[4 * b + c];
    for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = t[c];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double loss = w_nz * sh[0][0] + w_z * sh[1][0];
        dloss[0] = loss;
        dloss[1] = sh[2][0];
        if (!isfinite(loss)) atomicOr(status, kErrNonfinite);
    }
}

// ------------------------------------------------------------- sampling
template <int D>
__global__ void __launch_bounds__(kThreads) k_sample(const SampleSpec S, int32_t *idx_out, float *x_out,
                                                    float *w_out, float w_nz, float w_z) {
    const int64_t n = S.p + S.q;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        int32_t idx[D];
        float x = 0.0f;
        int att = 0;
        draw_sample<D>(S, s, idx, x, att);
        if (idx_out)
#pragma unroll
            for (int k = 0; k < D; ++k) idx_out[s * D + k] = idx[k];
        if (x_out) x_out[s] = x;
        if (w_out) w_out[s] = s < S.p ? w_nz : w_z;
    }
}

// ------------------------------------------------------ nonzero records
__global__ void k_build_records(const int32_t *__restrict__ coords, const float *__restrict__ vals, int64_t nnz,
                                int d, SampleSpec S, RowOffsets ro, const int *__restrict__ hot_slot, int rec_words,
                                int32_t *rec, uint64_t *hkeys, uint64_t hbmask, int *status) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t L = 0;
        int32_t *r = rec + e * rec_words;
        for (int k = d + 1; k < rec_words; ++k) r[k] = 0;
        for (int k = 0; k < d; ++k) {
            const int32_t c = coords[e * d + k];
            r[k] = c;
            L += (uint64_t)c * S.stride[k];
            const int hs = hot_slot ? hot_slot[ro.off[k] + c] : -1;
            const unsigned code = hs >= 0 ? (unsigned)hs : kNoSlot;
            r[d + 1 + k / 2] |= (int32_t)(code << (16 * (k & 1)));
        }
        r[d] = __float_as_int(vals[e]);
        const int rc = hash_insert(hkeys, hbmask, L);
        if (rc) atomicOr(status, rc);
    }
}

// ------------------------------------------------------------------ Adam
// Algorithm 1 on the flat parameter vector (Sec. 3.1.3); padded columns
// (col >= R) stay zero.  With BF16 storage the kernel-read copy is refreshed.
// Algorithm 1 on one 16-byte quad of parameters (columns col..col+3 of one
// row); padded columns (>= R) stay as they are (zero).  Abf, if not NULL,
// receives the BF16 copy of the quad.
__device__ __forceinline__ void adam_quad(float4 &a4, float4 &b4, float4 &c4, const float4 g4, int col, int R,
                                          float lr, float beta1, float beta2, float c1inv, float c2inv, float eps,
                                          float lower, uint2 *Abf) {
    float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w}, cv[4] = {c4.x, c4.y, c4.z, c4.w};
    const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (col + j >= R) continue;
        const float g = gv[j];
        bv[j] = beta1 * bv[j] + (1.0f - beta1) * g;
        cv[j] = beta2 * cv[j] + (1.0f - beta2) * g * g;
        av[j] = fmaxf(av[j] - lr * ((bv[j] * c1inv) / sqrtf(cv[j] * c2inv + eps)), lower);
    }
    a4 = make_float4(av[0], av[1], av[2], av[3]);
    b4 = make_float4(bv[0], bv[1], bv[2], bv[3]);
    c4 = make_float4(cv[0], cv[1], cv[2], cv[3]);
    if (Abf) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(av[0], av[1]), hi = __floats2bfloat162_rn(av[2], av[3]);
        *Abf = make_uint2(*reinterpret_cast<const unsigned *>(&lo), *reinterpret_cast<const unsigned *>(&hi));
    }
}

// Algorithm 1 over the flat parameter vector, one quad per thread and step
// (n and Rp are multiples of 4, Rp a power of two, so a quad is in one row).
__global__ void k_adam(int64_t n, int Rp, int R, float *__restrict__ A, float *__restrict__ B,
                       float *__restrict__ C, const float *__restrict__ G, float lr, float beta1, float beta2,
                       float c1inv, float c2inv, float eps, float lower, __nv_bfloat16 *Abf) {
    for (int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; qi < (n >> 2);
         qi += (int64_t)gridDim.x * blockDim.x) {
        const int col = (int)((qi << 2) & (Rp - 1));
        if (col >= R) continue;
        float4 a4 = reinterpret_cast<const float4 *>(A)[qi], b4 = reinterpret_cast<const float4 *>(B)[qi],
               c4 = reinterpret_cast<const float4 *>(C)[qi];
        adam_quad(a4, b4, c4, reinterpret_cast<const float4 *>(G)[qi], col, R, lr, beta1, beta2, c1inv, c2inv, eps,
                  lower, Abf ? reinterpret_cast<uint2 *>(Abf) + qi : nullptr);
        reinterpret_cast<float4 *>(A)[qi] = a4;
        reinterpret_cast<float4 *>(B)[qi] = b4;
        reinterpret_cast<float4 *>(C)[qi] = c4;
    }
}

// One training step's epilogue after the fused pass, in one launch, on
// 16-byte quads of the flat parameter vector (Rp is a power of two and a
// multiple of 4, so a quad lies in one row):
//  - the last block finishes the FP64 loss from the block partials (fixed
//    order);
//  - the first `ncold` blocks stream the quads of rows without replicas:
//    each thread takes kPostUnroll quads per iteration and issues all of
//    their loads (gradient, moments, factor, replica slot) before using any,
//    then applies Algorithm 1 and clears G for the next step;
//  - the blocks between take the quads of hot rows, one per group of
//    kHotLanes lanes: the group loads the quad's kReplicas replica quads at
//    once (gcpe::hot_quad_sum, which also clears them), and its first lane
//    adds them to the gradient quad and applies Algorithm 1.
// The streaming blocks run at the copy rate on models larger than L2; the
// hot quads cost one memory round trip each instead of one per group of
// replica loads.
// Quads per streaming thread and iteration.  One quad per thread at full
// occupancy streamed the HBM-resident epilogue (121.6M parameters) at
// 6.0 TB/s; two or four per thread, with fewer resident warps, at 3.6 and
// 4.1 TB/s.
constexpr int kPostUnroll = 1;
static_assert(kReplicas % gcpe::kHotLanes == 0, "hot-quad replicas split evenly over the folding lanes");

__global__ void __launch_bounds__(kThreads) k_post_step(PostSpec P, int ncold) {
    if (blockIdx.x == gridDim.x - 1) {  // the last block only finishes the loss
        __shared__ double sh[3][kThreads];
        double t[3] = {0.0, 0.0, 0.0};
        for (int b = threadIdx.x; b < P.nblocks; b += kThreads)
            for (int c = 0; c < 3; ++c) t[c] += P.partials[4 * b + c];
        for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = t[c];
        __syncthreads();
        for (int w = kThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w)
                for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double loss = P.w_nz * sh[0][0] + P.w_z * sh[1][0];
            P.dloss[0] = loss;
            P.dloss[1] = sh[2][0];
            if (!isfinite(loss)) atomicOr(P.status, kErrNonfinite);
        }
        return;
    }
    float4 *__restrict__ G4 = reinterpret_cast<float4 *>(P.G);
    float4 *__restrict__ A4 = reinterpret_cast<float4 *>(P.A);
    float4 *__restrict__ B4 = reinterpret_cast<float4 *>(P.B);
    float4 *__restrict__ C4 = reinterpret_cast<float4 *>(P.C);
    uint2 *__restrict__ Abf = static_cast<uint2 *>(P.Abf);
    const int log2Rp = __ffs(P.Rp) - 1;
    if ((int)blockIdx.x >= ncold) {  // hot quads, one per group of kHotLanes lanes
        const int log2Q = log2Rp - 2;  // quads per row = Rp / 4
        const int64_t hq = (int64_t)(blockIdx.x - ncold) * (kThreads / gcpe::kHotLanes) +
                           (threadIdx.x / gcpe::kHotLanes);
        if (hq >= ((int64_t)P.Htot << log2Q)) return;  // the whole group leaves together
        const int slot = (int)(hq >> log2Q), cq = (int)(hq & ((1 << log2Q) - 1));
        const int64_t q = ((int64_t)__ldg(P.hot_row + slot) << log2Q) + cq;
        const bool lead = (threadIdx.x & (gcpe::kHotLanes - 1)) == 0;
        float4 g, a, b, c;
        if (lead) {
            g = G4[q];
            a = A4[q];
            b = B4[q];
            c = C4[q];
        }
        const float4 t = gcpe::hot_quad_sum<kReplicas>(reinterpret_cast<float4 *>(P.Grep),
                                                       ((int64_t)P.Htot * P.Rp) >> 2, hq, gcpe::hot_group_mask());
        if (!lead) return;
        g.x += t.x;
        g.y += t.y;
        g.z += t.z;
        g.w += t.w;
        G4[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const int col = cq << 2;
        if (col >= P.R) return;  // a quad of padding columns
        adam_quad(a, b, c, g, col, P.R, P.lr, P.beta1, P.beta2, P.c1inv, P.c2inv, P.eps, P.lower,
                  Abf ? Abf + q : nullptr);
        A4[q] = a;
        B4[q] = b;
        C4[q] = c;
        return;
    }
    // block tiles of kThreads * kPostUnroll consecutive quads; thread t takes
    // quads t, t + kThreads, ... of its block's tile
    const int64_t nq = P.n >> 2;
    constexpr int64_t kTile = (int64_t)kThreads * kPostUnroll;
    for (int64_t q0 = (int64_t)blockIdx.x * kTile + threadIdx.x; q0 < nq; q0 += (int64_t)ncold * kTile) {
        float4 g[kPostUnroll], a[kPostUnroll], b[kPostUnroll], c[kPostUnroll];
        int hs[kPostUnroll];
#pragma unroll
        for (int u = 0; u < kPostUnroll; ++u) {
            const int64_t q = q0 + u * kThreads;
            hs[u] = -1;
            if (q < nq) {
                g[u] = G4[q];
                a[u] = A4[q];
                b[u] = B4[q];
                c[u] = C4[q];
                if (P.hot_slot) hs[u] = __ldg(P.hot_slot + ((q << 2) >> log2Rp));
            }
        }
#pragma unroll
        for (int u = 0; u < kPostUnroll; ++u) {
            const int64_t q = q0 + u * kThreads;
            if (q >= nq || hs[u] >= 0) continue;  // hot quads belong to the hot blocks
            G4[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const int col = (int)((q << 2) & (P.Rp - 1));
            if (col >= P.R) continue;  // a quad of padding columns: nothing to update
            adam_quad(a[u], b[u], c[u], g[u], col, P.R, P.lr, P.beta1, P.beta2, P.c1inv, P.c2inv, P.eps, P.lower,
                      Abf ? Abf + q : nullptr);
            A4[q] = a[u];
            B4[q] = b[u];
            C4[q] = c[u];
        }
    }
}

cudaError_t launch_post_step(const PostSpec &p, cudaStream_t st) {
    static int resident = 0;  // streaming blocks that fit on the GPU at once
    if (!resident) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_post_step, kThreads, 0);
        resident = (per_sm < 1 ? 1 : per_sm) * num_sms();
    }
    const int64_t want = ((p.n >> 2) + (int64_t)kThreads * kPostUnroll - 1) / ((int64_t)kThreads * kPostUnroll);
    const int ncold = (int)(want < 1 ? 1 : (want > resident ? resident : want));
    const int64_t hot_quads = (int64_t)p.Htot * (p.Rp >> 2);
    const int nhot = (int)((hot_quads + kThreads / gcpe::kHotLanes - 1) / (kThreads / gcpe::kHotLanes));
    k_post_step<<<ncold + nhot + 1, kThreads, 0, st>>>(p, ncold);  // + the loss block
    return cudaGetLastError();
}

__global__ void k_to_bf16(int64_t n, const float *__restrict__ A, __nv_bfloat16 *Abf) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        Abf[e] = __float2bfloat16_rn(A[e]);
}

// --------------------------------------------------------------- launches
static int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms;
}

static int elementwise_blocks(int64_t n) {
    const int64_t want = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

cudaError_t launch_build_records(const int32_t *coords, const float *vals, int64_t nnz, int d,
                                 const uint64_t *stride, const int64_t *rowoff, const int *hot_slot,
                                 int rec_words, int32_t *rec, uint64_t *hkeys, uint64_t hbmask, int *status,
                                 cudaStream_t st) {
    SampleSpec S{};
    S.d = d;
    RowOffsets ro{};
    for (int k = 0; k < d; ++k) {
        S.stride[k] = stride[k];
        ro.off[k] = rowoff[k];
    }
    k_build_records<<<elementwise_blocks(nnz), kThreads, 0, st>>>(coords, vals, nnz, d, S, ro, hot_slot, rec_words,
                                                                   rec, hkeys, hbmask, status);
    return cudaGetLastError();
}

#define GCP_DISPATCH_D(d, MACRO) \
    switch (d) {                 \
    case 2: MACRO(2); break;     \
    case 3: MACRO(3); break;     \
    case 4: MACRO(4); break;     \
    case 5: MACRO(5); break;     \
    case 6: MACRO(6); break;     \
    case 7: MACRO(7); break;     \
    case 8: MACRO(8); break;     \
    default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_sample(const SampleSpec &s, int32_t *idx_out, float *x_out, float *w_out, float w_nz,
                          float w_z, cudaStream_t st) {
    const int64_t n = s.p + s.q;
    if (n == 0) return cudaSuccess;
    const int blocks = elementwise_blocks(n);
#define GCP_LAUNCH_SAMPLE(D) k_sample<D><<<blocks, kThreads, 0, st>>>(s, idx_out, x_out, w_out, w_nz, w_z)
    GCP_DISPATCH_D(s.d, GCP_LAUNCH_SAMPLE)
#undef GCP_LAUNCH_SAMPLE
    return cudaGetLastError();
}

template <int D, typename TF, int COLS>
static int occupancy_blocks() {
    static int nb = -1;
    if (nb < 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<D, TF, COLS>, kThreads, 0);
        nb = (per_sm < 1 ? 1 : per_sm) * num_sms();
    }
    return nb;
}

template <int D>
static int occupancy_of(bool bf16, int cols) {
    if (bf16) return cols == 8 ? occupancy_blocks<D, __nv_bfloat16, 8>() : occupancy_blocks<D, __nv_bfloat16, 4>();
    return cols == 8 ? occupancy_blocks<D, float, 8>() : occupancy_blocks<D, float, 4>();
}

int fused_max_blocks(int d, bool bf16, int cols) {
    switch (d) {
    case 2: return occupancy_of<2>(bf16, cols);
    case 3: return occupancy_of<3>(bf16, cols);
    case 4: return occupancy_of<4>(bf16, cols);
    case 5: return occupancy_of<5>(bf16, cols);
    case 6: return occupancy_of<6>(bf16, cols);
    case 7: return occupancy_of<7>(bf16, cols);
    case 8: return occupancy_of<8>(bf16, cols);
    default: return num_sms();
    }
}

template <int D>
static void launch_fused_d(const FusedSpec &f, bool bf16, int cols, int blocks, cudaStream_t st) {
    if (bf16) {
        if (cols == 8)
            k_fused<D, __nv_bfloat16, 8><<<blocks, kThreads, 0, st>>>(f);
        else
            k_fused<D, __nv_bfloat16, 4><<<blocks, kThreads, 0, st>>>(f);
    } else {
        if (cols == 8)
            k_fused<D, float, 8><<<blocks, kThreads, 0, st>>>(f);
        else
            k_fused<D, float, 4><<<blocks, kThreads, 0, st>>>(f);
    }
}

cudaError_t launch_fused(const FusedSpec &f, bool bf16, int cols, int max_blocks, cudaStream_t st,
                         int *blocks_used) {
    const int64_t S = f.s.p + f.s.q;
    const int64_t ntiles = (S + 31) / 32;
    int64_t want = (ntiles + kWarps - 1) / kWarps;
    if (want < 1) want = 1;
    const int blocks = (int)(want < max_blocks ? want : max_blocks);
    *blocks_used = blocks;
    switch (f.s.d) {
    case 2: launch_fused_d<2>(f, bf16, cols, blocks, st); break;
    case 3: launch_fused_d<3>(f, bf16, cols, blocks, st); break;
    case 4: launch_fused_d<4>(f, bf16, cols, blocks, st); break;
    case 5: launch_fused_d<5>(f, bf16, cols, blocks, st); break;
    case 6: launch_fused_d<6>(f, bf16, cols, blocks, st); break;
    case 7: launch_fused_d<7>(f, bf16, cols, blocks, st); break;
    case 8: launch_fused_d<8>(f, bf16, cols, blocks, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Non-fused MTTKRP (Sec. 3.1.2 before fusion): reads the gradient tensor the
// sampling pass wrote (cells Ycoord, values Yval), gathers the factor rows
// again and adds y prod_{k!=n} A_k(i_k,:) to every mode's rows, with the
// same hot-row replicas as the fused pass (slots looked up by row).
template <int D, typename TF, int COLS>
__global__ void __launch_bounds__(kThreads) k_mttkrp_nonfused(const FusedSpec P, const int *__restrict__ hot_slot,
                                                             int S) {
    constexpr int NQ = COLS / 4;
    const int lane = threadIdx.x & 31;
    const int L = 1 << P.log2L;
    const int glane = lane & (L - 1);
    const int group = (blockIdx.x * blockDim.x + threadIdx.x) >> P.log2L;
    const int ngroups = (gridDim.x * blockDim.x) >> P.log2L;
    const int warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const TF *__restrict__ F = static_cast<const TF *>(P.F);
    float *const grep = P.Grep ? P.Grep + (size_t)(warp0 & (kReplicas - 1)) * P.Htot * P.Rp : nullptr;
    int col[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) col[q] = q * (P.Rp >> 1) + 4 * glane;
    for (int s = group; s < S; s += ngroups) {
        const float y = __ldg(P.Yval + (int64_t)s * P.vstride);
        int ii[D], off[D];
        float a[D][COLS];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            ii[k] = __ldg(P.Ycoord + (int64_t)s * P.ystride + k);
            off[k] = (P.rowoff[k] + ii[k]) * P.Rp;
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
        float pre[COLS];
#pragma unroll
        for (int v = 0; v < COLS; ++v) pre[v] = y;
#pragma unroll
        for (int n = 0; n < D; ++n) {
            const int hs = hot_slot ? __ldg(hot_slot + P.rowoff[n] + ii[n]) : -1;
            float *g = hs >= 0 ? grep + hs * P.Rp : P.G + off[n];
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                red_add_v4(g + col[q], pre[4 * q] * suf[n][4 * q], pre[4 * q + 1] * suf[n][4 * q + 1],
                           pre[4 * q + 2] * suf[n][4 * q + 2], pre[4 * q + 3] * suf[n][4 * q + 3]);
#pragma unroll
            for (int v = 0; v < COLS; ++v) pre[v] *= a[n][v];
        }
    }
}

template <int D>
static void launch_nonfused_d(const FusedSpec &f, const int *hot_slot, int S, bool bf16, int cols, int blocks,
                              cudaStream_t st) {
    if (bf16) {
        if (cols == 8)
            k_mttkrp_nonfused<D, __nv_bfloat16, 8><<<blocks, kThreads, 0, st>>>(f, hot_slot, S);
        else
            k_mttkrp_nonfused<D, __nv_bfloat16, 4><<<blocks, kThreads, 0, st>>>(f, hot_slot, S);
    } else {
        if (cols == 8)
            k_mttkrp_nonfused<D, float, 8><<<blocks, kThreads, 0, st>>>(f, hot_slot, S);
        else
            k_mttkrp_nonfused<D, float, 4><<<blocks, kThreads, 0, st>>>(f, hot_slot, S);
    }
}

cudaError_t launch_mttkrp_nonfused(const FusedSpec &f, const int *hot_slot, bool bf16, int cols, int max_blocks,
                                   cudaStream_t st) {
    const int S = (int)(f.s.p + f.s.q);
    if (S == 0) return cudaSuccess;
    const int64_t lanes = (int64_t)S << f.log2L;
    int64_t want = (lanes + kThreads - 1) / kThreads;
    const int blocks = (int)(want < max_blocks ? (want < 1 ? 1 : want) : max_blocks);
    switch (f.s.d) {
    case 2: launch_nonfused_d<2>(f, hot_slot, S, bf16, cols, blocks, st); break;
    case 3: launch_nonfused_d<3>(f, hot_slot, S, bf16, cols, blocks, st); break;
    case 4: launch_nonfused_d<4>(f, hot_slot, S, bf16, cols, blocks, st); break;
    case 5: launch_nonfused_d<5>(f, hot_slot, S, bf16, cols, blocks, st); break;
    case 6: launch_nonfused_d<6>(f, hot_slot, S, bf16, cols, blocks, st); break;
    case 7: launch_nonfused_d<7>(f, hot_slot, S, bf16, cols, blocks, st); break;
    case 8: launch_nonfused_d<8>(f, hot_slot, S, bf16, cols, blocks, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fold_replicas(float *G, float *Grep, const int *hot_row, int Htot, int Rp, cudaStream_t st) {
    if (Htot == 0) return cudaSuccess;
    k_fold_replicas<<<elementwise_blocks((int64_t)Htot * Rp), kThreads, 0, st>>>(G, Grep, hot_row, Htot, Rp);
    return cudaGetLastError();
}

cudaError_t launch_finish_loss(const double *partials, int nblocks, double w_nz, double w_z, double *dloss,
                               int *status, cudaStream_t st) {
    k_finish_loss<<<1, kThreads, 0, st>>>(partials, nblocks, w_nz, w_z, dloss, status);
    return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, int Rp, int R, float *A, float *B, float *C, const float *G, float lr,
                        float beta1, float beta2, float c1inv, float c2inv, float eps, float lower, void *Abf,
                        cudaStream_t st) {
    k_adam<<<elementwise_blocks(n), kThreads, 0, st>>>(n, Rp, R, A, B, C, G, lr, beta1, beta2, c1inv, c2inv, eps,
                                                        lower, static_cast<__nv_bfloat16 *>(Abf));
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(int64_t n, const float *A, void *Abf, cudaStream_t st) {
    k_to_bf16<<<elementwise_blocks(n), kThreads, 0, st>>>(n, A, static_cast<__nv_bfloat16 *>(Abf));
    return cudaGetLastError();
}

}  // namespace gcpk

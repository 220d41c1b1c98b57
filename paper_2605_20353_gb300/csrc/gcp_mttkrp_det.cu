// gcp_mttkrp_det.cu -- deterministic all-mode sampled MTTKRP.
//
// The gradient of a sample set is G_n(i_n,:) = sum_s y_s prod_{k!=n}
// A_k(i_k,:) (Eq. gcp-gradient on the sampled gradient tensor).  The atomic
// variant adds these terms in whatever order the hardware applies the
// reductions.  This variant fixes the order, so G is bit-identical from run
// to run, in the spirit of the permutation-based MTTKRP of Sec. 3.1.2:
//   1. the fused kernel in materialize mode writes every sample's cell and
//      value y_s = w f'(x_s, m_s) (the non-fused gradient tensor) as one
//      record of RW words (i_0 .. i_{d-1}, y_s, zeros), so that a later
//      lookup of a sample reads one 16-byte vector (d <= 3);
//   2. per mode n, a stable LSD radix sort (8-bit digits, or one 10-bit
//      pass) orders the sample ids by row i_n, ties in sample order.  The
//      first pass of every mode is counted and scanned once for all modes,
//      and the modes are sorted side by side: pass p of every mode that has
//      one is a single launch over all their tiles, so that it fills whole
//      waves of resident blocks;
//   3. a chunked segmented reduction walks the sorted list in chunks of kChunk
//      (64) positions, one chunk per group of lanes, recomputing the Khatri-Rao row
//      products.  A run of equal rows that lies inside one chunk is stored to
//      G directly; a run that crosses a chunk edge leaves one partial vector
//      per chunk it touches (in fixed slots: the right slot of its first
//      chunk, the left slots of the others);
//   4. a finishing pass sums each crossing run's partials in a fixed order
//      and stores the row.
// Every step has a fixed shape and order, so the result depends only on the
// inputs.
#include <cuda_bf16.h>

#include <utility>

#include "gcp_device.cuh"
#include "gcp_internal.h"

using namespace gcpdev;

namespace {

constexpr int kT = 256;            // threads per block
constexpr int kTile = 4096;        // keys per radix-sort block
constexpr int kChunk = 64;         // sorted positions per segmented-reduction chunk
constexpr int kScanBlock = 2048;   // elements per block of the multi-block scan
constexpr int kAhead = 4;          // partial vectors fetched ahead per lane group in the finishing pass

// --------------------------------------------------------------- radix sort
// One sort pass can sort several modes side by side (so that its blocks
// fill the GPU's waves): segment q sorts one mode's keys (kin, kstride words
// apart) with their values (vin, or the sample ids when null) into kout /
// vout.  Its digit counts start at obase in the count matrix, and `sub` is
// taken off its scanned offsets (k_radix_scatter).  Blocks [q * per, (q +
// 1) * per) of a launch work on segment q.
struct SortSeg {
    const int32_t *kin, *vin;
    int32_t *kout, *vout;
    int64_t obase;
    uint32_t sub;
    int kstride;
};
struct SortSegs {
    int nseg;
    SortSeg s[GCP_MAX_NDIM];
};

// Segment q, read with constant indices only: a runtime index into a kernel
// parameter array would copy the whole array to local memory per thread.
__device__ __forceinline__ SortSeg pick_seg(const SortSegs &S, int q) {
    SortSeg r = S.s[0];
#pragma unroll
    for (int i = 1; i < GCP_MAX_NDIM; ++i)
        if (q == i) r = S.s[i];
    return r;
}

// Digits of NB = 256 (8 bits) or 1024 (10 bits) values: keys of up to 10
// bits sort in one pass, longer ones in 8-bit passes.  Segment q's count of
// digit d in tile t goes to hist[obase_q + d * ntiles + t].  A block counts
// kHistTiles consecutive tiles, so that it writes kHistTiles consecutive
// counts of each digit together.
constexpr int kHistTiles = 4;

template <int NB>
__global__ void k_radix_hist(const SortSegs SG, int64_t n, int shift, int32_t *__restrict__ hist, int ntiles) {
    __shared__ int h[kHistTiles][NB];
    for (int i = threadIdx.x; i < kHistTiles * NB; i += kT) (&h[0][0])[i] = 0;
    __syncthreads();
    const int per = (ntiles + kHistTiles - 1) / kHistTiles;
    const SortSeg sg = pick_seg(SG, blockIdx.x / per);
    const int32_t *__restrict__ keys = sg.kin;
    const int key_stride = sg.kstride;
    const int t0 = (blockIdx.x % per) * kHistTiles;
    const int64_t first = (int64_t)t0 * kTile;
    constexpr int kB = 4;  // keys per tile loaded together, for every tile of the block
    for (int i0 = threadIdx.x; i0 < kTile; i0 += kB * kT) {
        int k[kHistTiles][kB];
#pragma unroll
        for (int g = 0; g < kHistTiles; ++g)
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int64_t i = first + (int64_t)g * kTile + i0 + u * kT;
                k[g][u] = i < n ? keys[i * key_stride] : -1;
            }
#pragma unroll
        for (int g = 0; g < kHistTiles; ++g)
#pragma unroll
            for (int u = 0; u < kB; ++u)
                if (k[g][u] >= 0) atomicAdd(&h[g][(k[g][u] >> shift) & (NB - 1)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHistTiles * NB; i += kT) {
        const int d = i / kHistTiles, g = i % kHistTiles;
        if (t0 + g < ntiles) hist[sg.obase + (int64_t)d * ntiles + t0 + g] = h[g][d];
    }
}

// Words of a sample record: d coordinates and y, padded to 4, 8 or 16.
__host__ __device__ constexpr int rec_words(int d) { return d + 1 <= 4 ? 4 : (d + 1 <= 8 ? 8 : 16); }

// The first pass of every mode (shift 0) counted in one pass over the
// records: mode k's pass has nb[k] digits and its counts go to
// hist[base[k] + d * ntiles + t], the modes' count matrices side by side,
// so that one scan serves them all.  Shared counters of mode k start at
// soff[k].
struct FirstPlan {
    int d, rw;
    int nb[GCP_MAX_NDIM], soff[GCP_MAX_NDIM];
    int64_t base[GCP_MAX_NDIM];
};

__global__ void __launch_bounds__(kT) k_radix_hist_first(const int32_t *__restrict__ recs, int64_t n,
                                                          const FirstPlan F, int32_t *__restrict__ hist,
                                                          int ntiles, int G) {
    extern __shared__ int h[];  // [G][used]
    const int d = F.d;
    const int used = F.soff[d - 1] + F.nb[d - 1];
    for (int i = threadIdx.x; i < G * used; i += kT) h[i] = 0;
    __syncthreads();
    const int t0 = blockIdx.x * G;
    // kB records per thread at a time, their 16-byte vectors loaded together
    constexpr int kB = 4;
    const int nv = F.rw / 4;
    for (int g = 0; g < G; ++g) {
        const int64_t first = (int64_t)(t0 + g) * kTile;
        const int tile_n = first >= n ? 0 : (n - first < kTile ? (int)(n - first) : kTile);
        const int4 *__restrict__ r = reinterpret_cast<const int4 *>(recs + first * F.rw);
        int *hg = h + g * used;
        for (int i0 = threadIdx.x; i0 < tile_n; i0 += kB * kT)
            for (int v = 0; v < nv && 4 * v < d; ++v) {
                int4 q[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u)
                    q[u] = i0 + u * kT < tile_n ? __ldg(r + (int64_t)(i0 + u * kT) * nv + v) : make_int4(0, 0, 0, 0);
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    if (i0 + u * kT >= tile_n) break;
                    const int c[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int k = 4 * v + j;
                        if (k < d) atomicAdd(&hg[F.soff[k] + (c[j] & (F.nb[k] - 1))], 1);
                    }
                }
            }
    }
    __syncthreads();
    // G consecutive counts of a digit are written together
    for (int k = 0; k < d; ++k)
        for (int i = threadIdx.x; i < F.nb[k] * G; i += kT) {
            const int dg = i / G, g = i % G;
            if (t0 + g < ntiles) hist[F.base[k] + (int64_t)dg * ntiles + t0 + g] = h[g * used + F.soff[k] + dg];
        }
}

// Exclusive prefix sum of n ints of `in` (in = out scans in place), left in
// two parts: out[i] holds the scan within its block of kScanBlock elements
// and block_sums[i / kScanBlock] the scan of the block totals, so the full
// value is their sum (consumers add the two).  Each block scans its
// elements and records its total; the last block to finish (a ticket on
// `done`, which it clears again for the next scan) then scans the totals.
// Sums are taken modulo 2^32 (see k_radix_scatter).
__global__ void k_scan_blocks(const int32_t *in, int32_t *out, int64_t n, int32_t *block_sums, unsigned *done) {
    __shared__ int32_t warp_tot[kT / 32];
    __shared__ bool last;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * (kScanBlock / kT);
    int32_t v[kScanBlock / kT];
    int32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanBlock / kT; ++j) {
        v[j] = base + j < n ? in[base + j] : 0;
        sum += v[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = sum;  // inclusive scan of the thread sums within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int32_t before = 0, block_total = 0;
    for (int w = 0; w < kT / 32; ++w) {
        if (w < warp) before += warp_tot[w];
        block_total += warp_tot[w];
    }
    int32_t run = before + incl - sum;
#pragma unroll
    for (int j = 0; j < kScanBlock / kT; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 0) {
        block_sums[blockIdx.x] = block_total;
        __threadfence();  // the total is visible before the ticket is taken
        last = atomicAdd(done, 1u) == gridDim.x - 1;
        if (last) __threadfence();  // and the other blocks' totals are seen after it
    }
    __syncthreads();
    if (!last) return;
    // the last block: exclusive scan of the gridDim.x totals, in place
    __shared__ int64_t part[kT];
    const int64_t nb = gridDim.x;
    const int64_t per = (nb + kT - 1) / kT;
    const int64_t lo = (int64_t)threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += __ldcg(block_sums + i);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t r = 0;
        for (int t = 0; t < kT; ++t) {
            const int64_t x = part[t];
            part[t] = r;
            r += x;
        }
        *done = 0u;
    }
    __syncthreads();
    int64_t r = part[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        const int32_t x = __ldcg(block_sums + i);
        block_sums[i] = static_cast<int32_t>(static_cast<uint32_t>(r));
        r += x;
    }
}

void scan_two_part(const int32_t *in, int32_t *a, int64_t n, int32_t *block_sums, unsigned *done, cudaStream_t st) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_blocks<<<(unsigned)nb, kT, 0, st>>>(in, a, n, block_sums, done);
}

// Stable scatter of one digit pass (NB digit values).  The tile's keys are
// first ranked into shared memory in index order (rounds of kT keys, warps
// in order, lanes in order), which leaves the tile sorted by digit; the
// sorted tile is then written out in order, so consecutive threads store
// consecutive positions of a digit's run and the global writes are
// coalesced.  Thread t looks after digits t, t + kT, ... (NB / kT of them).
// Block b sorts tile b % ntiles of segment b / ntiles.  The offset of digit
// d in this tile is offsets[obase + d * ntiles + tile] plus its block's
// sum, minus `sub`: the counts of the segments (modes) whose count matrices
// come first in a shared scan (each sums to n).  The sums are
// taken modulo 2^32, so the difference is exact even where the running
// total passes 2^31.
// Shared memory (dynamic): keys and values of the tile, then per digit the
// next local position, the global shift and one count per warp.
constexpr int kKeysPerThread = kTile / kT;

template <int NB>
constexpr size_t scatter_smem_bytes() {
    return (size_t)(2 * kTile + 2 * NB + (kT / 32) * NB + kT / 32) * sizeof(int32_t);
}

template <int NB>
__global__ void __launch_bounds__(kT, NB == 256 ? 5 : 3) k_radix_scatter(const SortSegs SG, int64_t n, int shift,
                                                      const int32_t *__restrict__ offsets,
                                                      const int32_t *__restrict__ offset_blocks, int ntiles) {
    const SortSeg sg = pick_seg(SG, blockIdx.x / ntiles);
    const int tile = blockIdx.x % ntiles;
    const int32_t *__restrict__ keys = sg.kin;
    const int32_t *__restrict__ vals = sg.vin;
    int32_t *__restrict__ keys_out = sg.kout;
    int32_t *__restrict__ vals_out = sg.vout;
    const int key_stride = sg.kstride;
    constexpr int DPT = NB / kT;  // digits per thread
    extern __shared__ __align__(16) int32_t smem[];
    int32_t *s_key = smem, *s_val = smem + kTile;
    int *running = smem + 2 * kTile;          // [NB]
    int *gshift = running + NB;               // [NB]
    int *wcount = gshift + NB;                // [kT / 32][NB]
    int *wsum = wcount + (kT / 32) * NB;      // [kT / 32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t first = (int64_t)tile * kTile;
    const int tile_n = n - first < kTile ? (int)(n - first) : kTile;
    int32_t key[kKeysPerThread], val[kKeysPerThread];
    for (int d = threadIdx.x; d < NB; d += kT) {
        running[d] = 0;
        for (int w = 0; w < kT / 32; ++w) wcount[w * NB + d] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kKeysPerThread; ++r) {
        const int i = r * kT + threadIdx.x;
        key[r] = 0;
        val[r] = 0;
        if (i < tile_n) {
            key[r] = keys[(first + i) * key_stride];
            val[r] = vals ? vals[first + i] : (int32_t)(first + i);
            atomicAdd(&running[(key[r] >> shift) & (NB - 1)], 1);  // the tile's digit counts
        }
    }
    __syncthreads();
    // exclusive scan of the NB digit counts: thread t sums digits DPT t ..
    // DPT t + DPT - 1, then a block scan of the thread sums
    int cnt[DPT], tsum = 0;
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        cnt[j] = running[DPT * threadIdx.x + j];
        tsum += cnt[j];
    }
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int start = incl - tsum;
    for (int w = 0; w < warp; ++w) start += wsum[w];
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        const int d = DPT * threadIdx.x + j;
        const int64_t oi = sg.obase + (int64_t)d * ntiles + tile;
        const uint32_t off = (uint32_t)offsets[oi] + (uint32_t)offset_blocks[oi / kScanBlock] - sg.sub;
        gshift[d] = (int)off - start;
        running[d] = start;
        start += cnt[j];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kKeysPerThread; ++r) {
        const bool valid = r * kT + (int)threadIdx.x < tile_n;
        const int digit = valid ? (key[r] >> shift) & (NB - 1) : NB;  // NB never matches a real digit
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, digit);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcount[warp * NB + digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = running[digit] + rank;
            for (int w = 0; w < warp; ++w) pos += wcount[w * NB + digit];
            s_key[pos] = key[r];
            s_val[pos] = val[r];
        }
        __syncthreads();
        for (int d = threadIdx.x; d < NB; d += kT) {
            int add = 0;
            for (int w = 0; w < kT / 32; ++w) {
                add += wcount[w * NB + d];
                wcount[w * NB + d] = 0;
            }
            running[d] += add;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < tile_n; i += kT) {
        const int32_t k = s_key[i];
        const int pos = gshift[(k >> shift) & (NB - 1)] + i;
        keys_out[pos] = k;
        vals_out[pos] = s_val[i];
    }
}

// ------------------------------------------------------ segmented reduction
struct SegSpec {
    int n_mode;        // mode whose gradient rows are reduced
    int rown;          // its first row in G
    int d, Rp, cols, log2L;
    int rowoff[GCP_MAX_NDIM];
    const void *F;     // factors read by the kernels (FP32 or BF16)
    const int32_t *recs;  // sample records: d coordinates, y, padding (rec_words(d) words)
    float *G;
};

template <typename TF, int NQ>
__device__ __forceinline__ void load_cols(const TF *F, int off, const int (&col)[NQ], float (&o)[4 * NQ]) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) Quad<TF>::load(F + off + col[q], o + 4 * q);
}

// Emit one run of equal keys: a run inside the chunk is final (stored to G),
// a run touching a chunk edge leaves the chunk's partial in its left slot
// (the run started earlier; also when it continues later) or its right slot
// (the run starts here and continues later).
template <int NQ>
__device__ __forceinline__ void emit_run(float *G, int Rp, int row_base, int key, const float (&acc)[4 * NQ],
                                         const int (&col)[NQ], bool before, bool after, int64_t chunk, float *cvec) {
    float *dst;
    if (!before && !after)
        dst = G + (int64_t)(row_base + key) * Rp;
    else
        dst = cvec + (2 * chunk + (before ? 0 : 1)) * Rp;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        *reinterpret_cast<float4 *>(dst + col[q]) = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
}

// Level 1: sorted sample ids of one mode -> G rows and edge carries.
// The group walks its chunk in batches of L positions.  Each lane first
// fetches one position's metadata (row key, then the sample's record: y_s
// and the coordinates that give the factor-row offsets), so the dependent
// id -> record lookups of a batch overlap; the positions are then taken in order, their metadata broadcast
// by shuffles and the factor rows of U positions gathered before any of
// them is accumulated.  Products and sums keep the sequential order.
template <typename TF, int COLS, int D>
__global__ void __launch_bounds__(kT, COLS == 8 && D >= 5 ? 2 : 3) k_seg_samples(const SegSpec P, const int32_t *__restrict__ keys,
                                                    const int32_t *__restrict__ ids, int64_t n, float *cvec,
                                                    int32_t *rowstart) {
    constexpr int NQ = COLS / 4;
    constexpr int U0 = 32 / ((D - 1) * COLS);
    constexpr int U = U0 < 1 ? 1 : (U0 > 4 ? 4 : U0);  // positions gathered ahead
    const int lane = threadIdx.x & 31;
    const int L = 1 << P.log2L;
    const int glane = lane & (L - 1);
    const unsigned gmask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (lane & ~(L - 1)));
    const int64_t group = ((int64_t)blockIdx.x * kT + threadIdx.x) >> P.log2L;
    const int64_t ngroups = ((int64_t)gridDim.x * kT) >> P.log2L;
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    const int nm = P.n_mode;
    const TF *__restrict__ F = static_cast<const TF *>(P.F);
    constexpr int RW = rec_words(D);
    const int4 *__restrict__ recs = reinterpret_cast<const int4 *>(P.recs);
    int col[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) col[q] = q * (P.Rp >> 1) + 4 * glane;
    int roff[D - 1];  // first rows of the other modes (constant indices only)
#pragma unroll
    for (int j = 0; j < D - 1; ++j) roff[j] = j < nm ? P.rowoff[j] : P.rowoff[j + 1];
    const int rown = P.rown;
    for (int64_t c = group; c < nchunks; c += ngroups) {
        const int64_t lo = c * kChunk, hi = lo + kChunk < n ? lo + kChunk : n;
        const int len = (int)(hi - lo);
        float acc[COLS];
#pragma unroll
        for (int v = 0; v < COLS; ++v) acc[v] = 0.0f;
        int cur = keys[lo];
        bool before = lo > 0 && keys[lo - 1] == cur;
        if (!before && glane == 0) rowstart[cur] = (int32_t)lo;  // a run starts at the chunk's start
        // the first batch's metadata: key and id, then the record
        int nkey = 0;
        int64_t nid = 0;
        int4 nrec[RW / 4];
        if (lo + glane < hi) {
            nkey = keys[lo + glane];
            nid = ids[lo + glane];
        }
#pragma unroll
        for (int v = 0; v < RW / 4; ++v)
            nrec[v] = lo + glane < hi ? __ldg(recs + nid * (RW / 4) + v) : make_int4(0, 0, 0, 0);
        for (int b = 0; b < len; b += L) {
            // this lane's position of the batch (its metadata was fetched
            // during the previous batch): key, y and the D-1 row offsets of
            // the other modes (mode k < n at j = k, k > n at k-1)
            const int mkey = nkey;
            int w[RW];
#pragma unroll
            for (int v = 0; v < RW / 4; ++v) {
                w[4 * v] = nrec[v].x;
                w[4 * v + 1] = nrec[v].y;
                w[4 * v + 2] = nrec[v].z;
                w[4 * v + 3] = nrec[v].w;
            }
            const float my = __int_as_float(w[D]);
            int moff[D - 1];
#pragma unroll
            for (int j = 0; j < D - 1; ++j) moff[j] = (roff[j] + (j < nm ? w[j] : w[j + 1])) * P.Rp;
            // the next batch's key and id now; its record once the first
            // rows of this batch are on their way
            const int64_t pn = lo + b + L + glane;
            const bool has_next = pn < hi;
            if (has_next) {
                nkey = keys[pn];
                nid = ids[pn];
            }
            const int nb = len - b < L ? len - b : L;
            for (int t0 = 0; t0 < nb; t0 += U) {
                int key[U];
                float y[U], a[U][D - 1][COLS];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + u < nb ? t0 + u : nb - 1;  // group-uniform
                    key[u] = __shfl_sync(gmask, mkey, t, L);
                    y[u] = __shfl_sync(gmask, my, t, L);
#pragma unroll
                    for (int j = 0; j < D - 1; ++j)
                        load_cols<TF, NQ>(F, __shfl_sync(gmask, moff[j], t, L), col, a[u][j]);
                }
                if (t0 == 0)
#pragma unroll
                    for (int v = 0; v < RW / 4; ++v)
                        nrec[v] = has_next ? __ldg(recs + nid * (RW / 4) + v) : make_int4(0, 0, 0, 0);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (t0 + u >= nb) break;
                    if (key[u] != cur) {
                        emit_run<NQ>(P.G, P.Rp, rown, cur, acc, col, before, false, c, cvec);
#pragma unroll
                        for (int v = 0; v < COLS; ++v) acc[v] = 0.0f;
                        cur = key[u];
                        before = false;
                        if (glane == 0) rowstart[cur] = (int32_t)(lo + b + t0 + u);  // a run starts here
                    }
                    float prod[COLS];
#pragma unroll
                    for (int v = 0; v < COLS; ++v) prod[v] = y[u];
#pragma unroll
                    for (int j = 0; j < D - 1; ++j)
#pragma unroll
                        for (int v = 0; v < COLS; ++v) prod[v] *= a[u][j][v];
#pragma unroll
                    for (int v = 0; v < COLS; ++v) acc[v] += prod[v];
                }
            }
        }
        const bool after = hi < n && keys[hi] == cur;
        emit_run<NQ>(P.G, P.Rp, rown, cur, acc, col, before, after, c, cvec);
    }
}

// Finishing pass: the runs that cross chunk edges.  Lane l of warp w
// checks chunk c = 32 w + l: it owns a run if the chunk's first run began
// in an earlier chunk and ends in this one.  The warp then takes its owned
// chunks one by one.  The run's first chunk c0 comes from the run's start
// position, which level 1 recorded per row (rowstart); its partials are
// the right slot of c0 and the left slots of c0 + 1 .. c (a chunk the run
// covers entirely uses its left slot), 1 + c - c0 vectors in all.  The
// warp's 32 / L lane groups each add every (32 / L)-th of them in order,
// kAhead at a time; the group sums are then combined by a butterfly over
// the groups; the order is fixed by (c0, c) alone, so the row is the same
// from run to run.
template <int COLS>
__global__ void __launch_bounds__(kT) k_seg_finish(const SegSpec P, const int32_t *__restrict__ keys, int64_t n,
                                                   const float *__restrict__ cvec,
                                                   const int32_t *__restrict__ rowstart) {
    constexpr int NQ = COLS / 4;
    const int lane = threadIdx.x & 31;
    const int L = 1 << P.log2L;
    const int glane = lane & (L - 1);
    const int grp = lane >> P.log2L, ngrp = 32 >> P.log2L;
    const int64_t nchunks = (n + kChunk - 1) / kChunk;
    const int64_t warp = ((int64_t)blockIdx.x * kT + threadIdx.x) >> 5;
    const int64_t cl = warp * 32 + lane;  // the chunk this lane checks
    bool own = false;
    int mykey = 0;
    if (cl < nchunks) {
        const int64_t lo = cl * kChunk, hi = lo + kChunk < n ? lo + kChunk : n;
        mykey = keys[lo];
        own = lo > 0 && keys[lo - 1] == mykey &&            // the first run began earlier
              !(keys[hi - 1] == mykey && hi < n && keys[hi] == mykey);  // and ends in this chunk
    }
    int col[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) col[q] = q * (P.Rp >> 1) + 4 * glane;
    for (unsigned owners = __ballot_sync(0xFFFFFFFFu, own); owners; owners &= owners - 1) {
        const int j = __ffs(owners) - 1;
        const int64_t c = warp * 32 + j;
        const int key = __shfl_sync(0xFFFFFFFFu, mykey, j);
        const int64_t c0 = __ldg(rowstart + key) / kChunk;
        const int64_t np = 1 + c - c0;  // partials: right slot of c0, left slots of c0 + 1 .. c
        float acc[COLS];
#pragma unroll
        for (int v = 0; v < COLS; ++v) acc[v] = 0.0f;
        for (int64_t k0 = grp; k0 < np; k0 += (int64_t)kAhead * ngrp) {
            float4 t[kAhead][NQ];
#pragma unroll
            for (int u = 0; u < kAhead; ++u) {
                const int64_t k = k0 + (int64_t)u * ngrp;
                const int64_t slot = k < np ? (k == 0 ? 2 * c0 + 1 : 2 * (c0 + k)) : 2 * c;
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    t[u][q] = *reinterpret_cast<const float4 *>(cvec + slot * P.Rp + col[q]);
            }
#pragma unroll
            for (int u = 0; u < kAhead; ++u) {
                if (k0 + (int64_t)u * ngrp >= np) break;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    acc[4 * q] += t[u][q].x;
                    acc[4 * q + 1] += t[u][q].y;
                    acc[4 * q + 2] += t[u][q].z;
                    acc[4 * q + 3] += t[u][q].w;
                }
            }
        }
        for (int o = L; o < 32; o <<= 1)  // butterfly over the groups, fixed order
#pragma unroll
            for (int v = 0; v < COLS; ++v) acc[v] += __shfl_xor_sync(0xFFFFFFFFu, acc[v], o);
        if (grp == 0) {
            float *dst = P.G + (int64_t)(P.rown + key) * P.Rp;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                *reinterpret_cast<float4 *>(dst + col[q]) =
                    make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
    }
}

int grid_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 65535) b = 65535;
    return (int)b;
}

}  // namespace

// Modes sorted side by side: as many as fit sort buffers of 1 GiB (each
// mode needs two key/id pairs of S ints), at least one.
static int det_group(const gcp_ctx *c, int64_t S) {
    const int64_t per_mode = 16 * (S > 0 ? S : 1);
    const int64_t g = ((int64_t)1 << 30) / per_mode;
    return (int)(g < 1 ? 1 : (g > c->d ? c->d : g));
}

// Scratch for the deterministic variant, grown on demand.  The scans'
// ticket comes first, so that it keeps its place (and its zero) whatever
// the sample count.
static gcp_status det_scratch(gcp_ctx *c, int64_t S, size_t *offs) {
    const int64_t ntiles = (S + kTile - 1) / kTile;
    const int64_t nchunk = (S + kChunk - 1) / kChunk + 1;
    const int64_t nfirst = (int64_t)1024 * c->d * ntiles;  // first-pass counts of all modes (at most)
    const int g = det_group(c, S);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    offs[0] = take(4);                              // the scans' finishing ticket (zero between scans)
    offs[1] = take((size_t)S * rec_words(c->d) * 4);  // sample records
    offs[2] = take((size_t)g * 4 * S * 4);          // per mode of a group: keys and ids, two of each
    offs[3] = take((size_t)nfirst * 4);             // first-pass digit counts / offsets of every mode
    offs[4] = take((size_t)((nfirst + kScanBlock - 1) / kScanBlock + 1) * 4);  // their scan block sums
    offs[5] = take((size_t)g * 256 * ntiles * 4);   // later-pass digit counts / offsets of a group
    offs[6] = take((size_t)((g * 256 * ntiles + kScanBlock - 1) / kScanBlock + 1) * 4);  // their block sums
    offs[7] = take((size_t)2 * nchunk * c->Rp * 4); // partial vectors: a left and a right slot per chunk
    int64_t maxdim = 1;
    for (int k = 0; k < c->d; ++k) maxdim = c->dims[k] > maxdim ? c->dims[k] : maxdim;
    offs[8] = take((size_t)maxdim * 4);             // start position of each row's run (one mode at a time)
    if (o > c->det_scratch_bytes) {
        cudaFree(c->det_scratch);
        c->det_scratch = nullptr;
        c->det_scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&c->det_scratch, o);
        if (e != cudaSuccess) {
            c->err = std::string("allocating deterministic MTTKRP scratch: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? GCP_ERR_OOM : GCP_ERR_CUDA;
        }
        c->det_scratch_bytes = o;
        e = cudaMemsetAsync(c->det_scratch, 0, 4, c->st);
        if (e != cudaSuccess) {
            c->err = std::string("clearing deterministic MTTKRP scratch: ") + cudaGetErrorString(e);
            return GCP_ERR_CUDA;
        }
    }
    return GCP_OK;
}

#define DET_CUDA(call)                                                           \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            c->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return GCP_ERR_CUDA;                                                 \
        }                                                                        \
    } while (0)

template <typename TF, int D>
static void launch_seg_samples_d(const SegSpec &P, int cols, int grid, const int32_t *keys, const int32_t *ids,
                                 int64_t n, float *cvec, int32_t *rowstart, cudaStream_t st) {
    if (cols == 8)
        k_seg_samples<TF, 8, D><<<grid, kT, 0, st>>>(P, keys, ids, n, cvec, rowstart);
    else
        k_seg_samples<TF, 4, D><<<grid, kT, 0, st>>>(P, keys, ids, n, cvec, rowstart);
}

template <typename TF>
static void launch_seg_samples(const SegSpec &P, int cols, int grid, const int32_t *keys, const int32_t *ids,
                               int64_t n, float *cvec, int32_t *rowstart, cudaStream_t st) {
    switch (P.d) {
        case 2: launch_seg_samples_d<TF, 2>(P, cols, grid, keys, ids, n, cvec, rowstart, st); break;
        case 3: launch_seg_samples_d<TF, 3>(P, cols, grid, keys, ids, n, cvec, rowstart, st); break;
        case 4: launch_seg_samples_d<TF, 4>(P, cols, grid, keys, ids, n, cvec, rowstart, st); break;
        case 5: launch_seg_samples_d<TF, 5>(P, cols, grid, keys, ids, n, cvec, rowstart, st); break;
        case 6: launch_seg_samples_d<TF, 6>(P, cols, grid, keys, ids, n, cvec, rowstart, st); break;
        case 7: launch_seg_samples_d<TF, 7>(P, cols, grid, keys, ids, n, cvec, rowstart, st); break;
        default: launch_seg_samples_d<TF, 8>(P, cols, grid, keys, ids, n, cvec, rowstart, st); break;
    }
}

// The 1024-digit scatter needs more than the default 48 KB of dynamic
// shared memory; raised once per device.
static cudaError_t allow_wide_scatter() {
    static int done_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || done_dev == dev) return e;
    e = cudaFuncSetAttribute(k_radix_scatter<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem_bytes<1024>());
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

gcp_status gcpk_det_grad(gcp_ctx *c, const gcpk::FusedSpec &f0, int *blocks) {
    const int64_t S = f0.s.p + f0.s.q;
    size_t offs[9];
    gcp_status s = det_scratch(c, S > 0 ? S : 1, offs);
    if (s) return s;
    char *base = static_cast<char *>(c->det_scratch);
    const int rw = rec_words(c->d);
    unsigned *ticket = reinterpret_cast<unsigned *>(base + offs[0]);
    int32_t *recs = reinterpret_cast<int32_t *>(base + offs[1]);
    int32_t *sortbuf = reinterpret_cast<int32_t *>(base + offs[2]);
    int32_t *histF = reinterpret_cast<int32_t *>(base + offs[3]);
    int32_t *bsumF = reinterpret_cast<int32_t *>(base + offs[4]);
    int32_t *histL = reinterpret_cast<int32_t *>(base + offs[5]);
    int32_t *bsumL = reinterpret_cast<int32_t *>(base + offs[6]);
    float *cvec = reinterpret_cast<float *>(base + offs[7]);
    int32_t *rowstart = reinterpret_cast<int32_t *>(base + offs[8]);
    cudaStream_t st = c->st;
    DET_CUDA(allow_wide_scatter());

    // 1. loss partials and the materialised gradient tensor, as records
    gcpk::FusedSpec f = f0;
    f.G = nullptr;
    f.Ycoord = recs;
    f.Yval = reinterpret_cast<float *>(recs + c->d);
    f.ystride = rw;
    f.vstride = rw;
    DET_CUDA(gcpk::launch_fused(f, c->Abf != nullptr, c->cols, c->max_blocks, st, blocks));
    if (S == 0) return GCP_OK;

    // 2a. the first pass of every mode: counted and scanned once
    const int64_t ntiles = (S + kTile - 1) / kTile;
    int bits[GCP_MAX_NDIM], npass[GCP_MAX_NDIM];
    FirstPlan FP{};
    FP.d = c->d;
    FP.rw = rw;
    int64_t nfirst = 0;
    for (int k = 0; k < c->d; ++k) {
        bits[k] = 1;
        while ((1ll << bits[k]) < c->dims[k]) ++bits[k];
        const bool wide = bits[k] > 8 && bits[k] <= 10;  // one 10-bit pass instead of 8 + 2
        FP.nb[k] = wide ? 1024 : 256;
        npass[k] = wide ? 1 : (bits[k] + 7) / 8;
        FP.soff[k] = k ? FP.soff[k - 1] + FP.nb[k - 1] : 0;
        FP.base[k] = nfirst;
        nfirst += (int64_t)FP.nb[k] * ntiles;
    }
    const int used = FP.soff[c->d - 1] + FP.nb[c->d - 1];
    const int G = used <= 3072 ? kHistTiles : 1;  // at most 48 KB of counters
    k_radix_hist_first<<<(int)((ntiles + G - 1) / G), kT, (size_t)G * used * 4, st>>>(recs, S, FP, histF,
                                                                                     (int)ntiles, G);
    scan_two_part(histF, histF, nfirst, bsumF, ticket, st);
    DET_CUDA(cudaGetLastError());

    SegSpec P{};
    P.d = c->d;
    P.Rp = c->Rp;
    P.cols = c->cols;
    P.log2L = c->log2L;
    for (int k = 0; k < c->d; ++k) P.rowoff[k] = (int)c->rowoff[k];
    P.F = f0.F;
    P.recs = recs;
    P.G = c->G;
    const int lanes = 1 << c->log2L;
    const int group = det_group(c, S);
    // sort buffers of mode n (the j-th of its group): keys and ids, pass p
    // writing pair p % 2
    auto keys_of = [&](int j, int p) { return sortbuf + ((int64_t)j * 4 + 2 * (p & 1)) * S; };
    auto ids_of = [&](int j, int p) { return sortbuf + ((int64_t)j * 4 + 2 * (p & 1) + 1) * S; };
    bool joined = true;  // no side-stream work outstanding
    for (int m0 = 0; m0 < c->d; m0 += group) {
        const int m1 = m0 + group < c->d ? m0 + group : c->d;
        // 2b. stable LSD radix sort of sample ids by row, the modes of the
        // group side by side: pass p of every mode in one launch (the
        // first passes by digit width)
        for (int p = 0;; ++p) {
            SortSegs segs[2] = {};  // 256-digit and 1024-digit passes
            for (int n = m0; n < m1; ++n) {
                if (p >= npass[n]) continue;
                SortSegs &sg = segs[FP.nb[n] == 1024 ? 1 : 0];
                SortSeg &q = sg.s[sg.nseg];
                q.kin = p == 0 ? recs + n : keys_of(n - m0, p - 1);
                q.kstride = p == 0 ? rw : 1;
                q.vin = p == 0 ? nullptr : ids_of(n - m0, p - 1);
                q.kout = keys_of(n - m0, p);
                q.vout = ids_of(n - m0, p);
                if (p == 0) {  // offsets from the shared first-pass scan
                    q.obase = FP.base[n];
                    q.sub = (uint32_t)((uint64_t)n * (uint64_t)S);
                } else {       // offsets from this pass's own count
                    q.obase = (int64_t)sg.nseg * 256 * ntiles;
                    q.sub = (uint32_t)((uint64_t)sg.nseg * (uint64_t)S);
                }
                ++sg.nseg;
            }
            if (segs[0].nseg + segs[1].nseg == 0) break;
            const int shift = 8 * p;
            if (p > 0) {  // later passes: counted over the previous pass's order
                const int per = (int)((ntiles + kHistTiles - 1) / kHistTiles);
                k_radix_hist<256><<<segs[0].nseg * per, kT, 0, st>>>(segs[0], S, shift, histL, (int)ntiles);
                scan_two_part(histL, histL, (int64_t)segs[0].nseg * 256 * ntiles, bsumL, ticket, st);
            }
            const int32_t *offsets = p == 0 ? histF : histL, *blks = p == 0 ? bsumF : bsumL;
            // both widths in one pass: the 1024-digit launch runs on the side
            // stream beside the 256-digit one, so that each fills the other's
            // partial waves (both read only the records and the first-pass
            // offsets, and write their own modes' buffers)
            cudaStream_t wst = st;
            if (segs[0].nseg && segs[1].nseg) {
                if (!c->det_side) {
                    DET_CUDA(cudaStreamCreateWithFlags(&c->det_side, cudaStreamNonBlocking));
                    DET_CUDA(cudaEventCreateWithFlags(&c->det_fork, cudaEventDisableTiming));
                    DET_CUDA(cudaEventCreateWithFlags(&c->det_join, cudaEventDisableTiming));
                }
                DET_CUDA(cudaEventRecord(c->det_fork, st));
                DET_CUDA(cudaStreamWaitEvent(c->det_side, c->det_fork, 0));
                wst = c->det_side;
            }
            if (segs[1].nseg)
                k_radix_scatter<1024><<<(int)(segs[1].nseg * ntiles), kT, scatter_smem_bytes<1024>(), wst>>>(
                    segs[1], S, shift, offsets, blks, (int)ntiles);
            if (segs[0].nseg)
                k_radix_scatter<256><<<(int)(segs[0].nseg * ntiles), kT, scatter_smem_bytes<256>(), st>>>(
                    segs[0], S, shift, offsets, blks, (int)ntiles);
            DET_CUDA(cudaGetLastError());
            if (wst != st) {
                DET_CUDA(cudaEventRecord(c->det_join, wst));
                joined = false;
            }
        }
        if (!joined) {  // the wide modes' sort is done before their reduction
            DET_CUDA(cudaStreamWaitEvent(st, c->det_join, 0));
            joined = true;
        }
        for (int n = m0; n < m1; ++n) {
            P.n_mode = n;
            P.rown = (int)c->rowoff[n];
            const int32_t *kin = keys_of(n - m0, npass[n] - 1), *vin = ids_of(n - m0, npass[n] - 1);
            // 3. chunked segmented reduction over the sorted samples
            const int64_t nch = (S + kChunk - 1) / kChunk;
            const int grid = grid_for(nch * lanes, kT);
            if (c->Abf)
                launch_seg_samples<__nv_bfloat16>(P, c->cols, grid, kin, vin, S, cvec, rowstart, st);
            else
                launch_seg_samples<float>(P, c->cols, grid, kin, vin, S, cvec, rowstart, st);
            DET_CUDA(cudaGetLastError());
            // 4. the runs that cross chunk edges: a lane per chunk decides, a warp sums
            const int fgrid = grid_for(((nch + 31) / 32) * 32, kT);  // a lane per chunk
            if (c->cols == 8)
                k_seg_finish<8><<<fgrid, kT, 0, st>>>(P, kin, S, cvec, rowstart);
            else
                k_seg_finish<4><<<fgrid, kT, 0, st>>>(P, kin, S, cvec, rowstart);
            DET_CUDA(cudaGetLastError());
        }
    }
    return GCP_OK;
}

/*
 * gcp_oracle.c -- plain, slow, FP64 CPU oracle of the stochastic GCP gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The GPU library never links,
 * includes or calls it, and this file includes nothing from the GPU library.
 *
 * Every function restates a definition from Myers & Phipps, "Synchronous and
 * Asynchronous Parallelism Approaches for GCP Tensor Decomposition with GenTen":
 *   - CP model entry            m_i = sum_r prod_k A_k(i_k, r)        (Eq. cp, Sec. 3.1.1)
 *   - GCP objective             F = sum_i f(x_i, m_i)                 (Eq. gcp-model)
 *   - GCP gradient as MTTKRP    G_k = Y_(k) Z_k^T, y_i = df/dm        (Eq. gcp-gradient)
 *   - stratified sampling       p nonzeros (weight N/p), q zeros drawn by
 *                               rejection (weight (M-N)/q)            (Sec. 3.1.1)
 *   - serial MTTKRP             one sample at a time, no races        (Sec. 3.1.2)
 *   - Adam update               Algorithm 1
 * The four losses are not written out in the paper; they follow the GCP
 * source it cites (Hong & Kolda 2020): Gaussian, Poisson (identity link),
 * Bernoulli-logit and Gamma, with eps = 1e-10.
 *
 * Random numbers: Philox4x64-10, written from Salmon, Moraes, Dror & Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): 10 rounds of the
 * 4x64 S-box with their published multipliers and Weyl key increments.
 * Counter layout (a choice of this library, fixed on both sides):
 *   key = (seed, stream), counter = (j, sub, t, 0)
 *   stream 0: nonzero draw j of iteration t, sub = 0, word 0
 *   stream 1: zero draw j, attempt a, words for modes 4b..4b+3 at sub = 4a+b
 *   stream 2: uniform (dense) draw j, words for modes 4b..4b+3 at sub = b
 *   stream 3: semi-stratified zero draw j (no rejection), sub = b
 * An integer u in [0, 2^64) maps to [0, n) as floor(u * n / 2^64).
 * Linear index of (i_0..i_{d-1}): row-major, last mode fastest, uint64.
 *
 * All sums run in plain sample order, in double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GAUSSIAN 0
#define ORC_POISSON 1
#define ORC_BERNOULLI_LOGIT 2
#define ORC_GAMMA 3
#define ORC_EPS 1e-10
#define ORC_MAX_NDIM 16

/* ---------------------------------------------------------------- Philox */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t mult0 = 0xD2E7470EE14C6C93ULL, mult1 = 0xCA5A826395121157ULL;
    const uint64_t weyl0 = 0x9E3779B97F4A7C15ULL, weyl1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        unsigned __int128 prod0 = (unsigned __int128)mult0 * x0;
        unsigned __int128 prod1 = (unsigned __int128)mult1 * x2;
        uint64_t hi0 = (uint64_t)(prod0 >> 64), lo0 = (uint64_t)prod0;
        uint64_t hi1 = (uint64_t)(prod1 >> 64), lo1 = (uint64_t)prod1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* floor(u * n / 2^64): an exact integer map of a 64-bit word onto [0, n). */
uint64_t orc_map64(uint64_t u, uint64_t n)
{
    return (uint64_t)(((unsigned __int128)u * n) >> 64);
}

static uint64_t linear_index(int d, const int64_t *dims, const int64_t *idx)
{
    uint64_t L = 0;
    for (int k = 0; k < d; ++k)
        L = L * (uint64_t)dims[k] + (uint64_t)idx[k];
    return L;
}

/* Sorted-list membership test (Sec. 3.1.1: lexicographically sorted
 * coordinates searched in O(log N)). */
static int is_nonzero(uint64_t L, const uint64_t *sorted_keys, int64_t nnz)
{
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (sorted_keys[mid] < L)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < nnz && sorted_keys[lo] == L;
}

/* ---------------------------------------------------------- sample draws */
int64_t orc_draw_nonzero(uint64_t seed, uint64_t t, uint64_t j, int64_t nnz)
{
    uint64_t ctr[4] = {j, 0, t, 0}, key[2] = {seed, 0}, w[4];
    orc_philox4x64_10(ctr, key, w);
    return (int64_t)orc_map64(w[0], (uint64_t)nnz);
}

/* One candidate coordinate tuple from `stream` with sub-counter base `sub0`. */
static void draw_tuple(uint64_t seed, uint64_t stream, uint64_t t, uint64_t j, uint64_t sub0,
                       int d, const int64_t *dims, int64_t *idx)
{
    for (int b = 0; 4 * b < d; ++b) {
        uint64_t ctr[4] = {j, sub0 + (uint64_t)b, t, 0}, key[2] = {seed, stream}, w[4];
        orc_philox4x64_10(ctr, key, w);
        for (int k = 4 * b; k < d && k < 4 * b + 4; ++k)
            idx[k] = (int64_t)orc_map64(w[k - 4 * b], (uint64_t)dims[k]);
    }
}

/* Zero draw j: repeat candidate draws until the tuple is not a nonzero
 * (Sec. 3.1.1); the first accepted attempt in counter order wins.  Returns
 * the number of attempts used, or -1 when `cap` attempts all hit nonzeros. */
int orc_draw_zero(uint64_t seed, uint64_t t, uint64_t j, int d, const int64_t *dims,
                  const uint64_t *sorted_keys, int64_t nnz, int cap, int64_t *idx)
{
    for (int a = 0; a < cap; ++a) {
        draw_tuple(seed, 1, t, j, 4 * (uint64_t)a, d, dims, idx);
        if (!is_nonzero(linear_index(d, dims, idx), sorted_keys, nnz))
            return a + 1;
    }
    return -1;
}

void orc_draw_uniform(uint64_t seed, uint64_t t, uint64_t j, int d, const int64_t *dims,
                      int64_t *idx)
{
    draw_tuple(seed, 2, t, j, 0, d, dims, idx);
}

void orc_draw_semi_zero(uint64_t seed, uint64_t t, uint64_t j, int d, const int64_t *dims,
                        int64_t *idx)
{
    draw_tuple(seed, 3, t, j, 0, d, dims, idx);
}

/* Stratified sample set of iteration t: samples 0..p-1 are nonzeros with
 * weight N/p, samples p..p+q-1 are zeros with weight (M-N)/q (Sec. 3.1.1).
 * Writes (p+q) x d coordinates, values and weights.  Returns 0, or -(1 + j)
 * when zero draw j exhausted `cap` attempts.  *attempts_out = total zero
 * attempts. */
int64_t orc_stratified_samples(uint64_t seed, uint64_t t, int64_t p, int64_t q, int d,
                               const int64_t *dims, int64_t nnz, const int32_t *coords,
                               const float *vals, const uint64_t *sorted_keys, int cap,
                               int32_t *idx_out, double *x_out, double *w_out,
                               int64_t *attempts_out)
{
    double M = 1.0;
    for (int k = 0; k < d; ++k)
        M *= (double)dims[k];
    double w_nz = p > 0 ? (double)nnz / (double)p : 0.0;
    double w_z = q > 0 ? (M - (double)nnz) / (double)q : 0.0;
    int64_t attempts = 0;
    for (int64_t j = 0; j < p; ++j) {
        int64_t e = orc_draw_nonzero(seed, t, (uint64_t)j, nnz);
        for (int k = 0; k < d; ++k)
            idx_out[j * d + k] = coords[e * d + k];
        x_out[j] = (double)vals[e];
        w_out[j] = w_nz;
    }
    for (int64_t j = 0; j < q; ++j) {
        int64_t idx[ORC_MAX_NDIM];
        int a = orc_draw_zero(seed, t, (uint64_t)j, d, dims, sorted_keys, nnz, cap, idx);
        if (a < 0) {
            *attempts_out = attempts;
            return -(1 + j);
        }
        attempts += a;
        for (int k = 0; k < d; ++k)
            idx_out[(p + j) * d + k] = (int32_t)idx[k];
        x_out[p + j] = 0.0;
        w_out[p + j] = w_z;
    }
    *attempts_out = attempts;
    return 0;
}

/* Uniform sample set of a dense tensor X (row-major, last mode fastest):
 * s entries, weight M/s.  X may be NULL (values then 0). */
void orc_uniform_samples(uint64_t seed, uint64_t t, int64_t s, int d, const int64_t *dims,
                         const float *X, int32_t *idx_out, double *x_out, double *w_out)
{
    double M = 1.0;
    for (int k = 0; k < d; ++k)
        M *= (double)dims[k];
    for (int64_t j = 0; j < s; ++j) {
        int64_t idx[ORC_MAX_NDIM];
        orc_draw_uniform(seed, t, (uint64_t)j, d, dims, idx);
        for (int k = 0; k < d; ++k)
            idx_out[j * d + k] = (int32_t)idx[k];
        x_out[j] = X ? (double)X[linear_index(d, dims, idx)] : 0.0;
        w_out[j] = M / (double)s;
    }
}

/* Semi-stratified sample set (Sec. 3.1.1): p nonzeros as above and q zero
 * candidates drawn uniformly over all M cells with no search.  The zero
 * weight is M/q (every cell is a candidate); flag_out[j] = 1 marks the
 * nonzero samples, whose value later enters as f'(x,m) - f'(0,m). */
void orc_semi_stratified_samples(uint64_t seed, uint64_t t, int64_t p, int64_t q, int d,
                                 const int64_t *dims, int64_t nnz, const int32_t *coords,
                                 const float *vals, int32_t *idx_out, double *x_out,
                                 double *w_out)
{
    double M = 1.0;
    for (int k = 0; k < d; ++k)
        M *= (double)dims[k];
    for (int64_t j = 0; j < p; ++j) {
        int64_t e = orc_draw_nonzero(seed, t, (uint64_t)j, nnz);
        for (int k = 0; k < d; ++k)
            idx_out[j * d + k] = coords[e * d + k];
        x_out[j] = (double)vals[e];
        w_out[j] = (double)nnz / (double)p;
    }
    for (int64_t j = 0; j < q; ++j) {
        int64_t idx[ORC_MAX_NDIM];
        orc_draw_semi_zero(seed, t, (uint64_t)j, d, dims, idx);
        for (int k = 0; k < d; ++k)
            idx_out[(p + j) * d + k] = (int32_t)idx[k];
        x_out[p + j] = 0.0;
        w_out[p + j] = M / (double)q;
    }
}

/* ------------------------------------------------------------ the losses */
void orc_loss(int loss, double x, double m, double *f, double *df)
{
    switch (loss) {
    case ORC_GAUSSIAN:
        *f = (x - m) * (x - m);
        *df = 2.0 * (m - x);
        break;
    case ORC_POISSON:
        *f = m - x * log(m + ORC_EPS);
        *df = 1.0 - x / (m + ORC_EPS);
        break;
    case ORC_BERNOULLI_LOGIT:
        /* log(1 + e^m) - x m, and d/dm = e^m / (1 + e^m) - x */
        *f = (m > 0.0 ? m + log1p(exp(-m)) : log1p(exp(m))) - x * m;
        *df = (m >= 0.0 ? 1.0 / (1.0 + exp(-m)) : exp(m) / (1.0 + exp(m))) - x;
        break;
    case ORC_GAMMA:
        *f = x / (m + ORC_EPS) + log(m + ORC_EPS);
        *df = 1.0 / (m + ORC_EPS) - x / ((m + ORC_EPS) * (m + ORC_EPS));
        break;
    default:
        *f = NAN;
        *df = NAN;
    }
}

void orc_loss_vec(int loss, int64_t n, const double *x, const double *m, double *f, double *df)
{
    for (int64_t i = 0; i < n; ++i)
        orc_loss(loss, x[i], m[i], &f[i], &df[i]);
}

/* ------------------------------------------------- model, loss, gradient */
static void mode_offsets(int d, const int64_t *dims, int R, int64_t *off)
{
    off[0] = 0;
    for (int k = 1; k < d; ++k)
        off[k] = off[k - 1] + dims[k - 1] * (int64_t)R;
}

/* m_i = sum_r prod_k A_k(i_k, r); A is all factors concatenated, mode by
 * mode, each I_k x R row-major (Sec. 3.1.3: one contiguous array). */
double orc_model(int d, const int64_t *dims, int R, const double *A, const int32_t *idx)
{
    int64_t off[ORC_MAX_NDIM];
    mode_offsets(d, dims, R, off);
    double m = 0.0;
    for (int r = 0; r < R; ++r) {
        double prod = 1.0;
        for (int k = 0; k < d; ++k)
            prod *= A[off[k] + (int64_t)idx[k] * R + r];
        m += prod;
    }
    return m;
}

/* One sample's loss term w f(x, m) and, if G != NULL, its MTTKRP
 * contribution G_n(i_n, :) += w f'(x, m) prod_{k != n} A_k(i_k, :) for every
 * mode n (Eq. gcp-gradient, one nonzero of the gradient tensor).  With
 * semi != 0 the derivative is f'(x,m) - f'(0,m), the semi-stratified
 * nonzero value of Sec. 3.1.1, and the loss term f(x,m) - f(0,m) (the
 * zero candidates already counted f(0,m) for every cell). */
static double add_sample(int d, const int64_t *dims, const int64_t *off, int R, const double *A,
                         int loss, const int32_t *i, double x, double w, int semi, double *G)
{
    double m = orc_model(d, dims, R, A, i);
    double f, df;
    orc_loss(loss, x, m, &f, &df);
    if (semi) { /* the same correction keeps the loss estimate unbiased too */
        double f0, df0;
        orc_loss(loss, 0.0, m, &f0, &df0);
        f -= f0;
        df -= df0;
    }
    if (G) {
        double y = w * df;
        for (int n = 0; n < d; ++n) {
            for (int r = 0; r < R; ++r) {
                double prod = 1.0;
                for (int k = 0; k < d; ++k)
                    if (k != n)
                        prod *= A[off[k] + (int64_t)i[k] * R + r];
                G[off[n] + (int64_t)i[n] * R + r] += y * prod;
            }
        }
    }
    return w * f;
}

static int64_t total_rows_of(int d, const int64_t *dims)
{
    int64_t rows = 0;
    for (int k = 0; k < d; ++k)
        rows += dims[k];
    return rows;
}

/* Sampled loss sum_s w_s f(x_s, m_s) and, if G != NULL, the sampled gradient
 * (the serial MTTKRP of Sec. 3.1.2 applied to the sampled gradient tensor),
 * one sample at a time in sample order.  G is zeroed first.  semi may be
 * NULL; semi[s] = 1 marks a semi-stratified nonzero sample. */
double orc_sampled_loss_grad(int d, const int64_t *dims, int R, const double *A, int loss,
                             int64_t S, const int32_t *idx, const double *x, const double *w,
                             const uint8_t *semi, double *G)
{
    int64_t off[ORC_MAX_NDIM];
    mode_offsets(d, dims, R, off);
    if (G)
        memset(G, 0, sizeof(double) * (size_t)(total_rows_of(d, dims) * R));
    double F = 0.0;
    for (int64_t s = 0; s < S; ++s)
        F += add_sample(d, dims, off, R, A, loss, idx + s * d, x[s], w[s], semi ? semi[s] : 0, G);
    return F;
}

/* Full (unsampled) GCP loss and gradient of a dense tensor X by enumerating
 * all M cells with weight 1 (Eq. gcp-model and Eq. gcp-gradient).  Tiny
 * tensors only. */
double orc_full_loss_grad(int d, const int64_t *dims, int R, const double *A, int loss,
                          const double *X, double *G)
{
    int64_t off[ORC_MAX_NDIM];
    mode_offsets(d, dims, R, off);
    if (G)
        memset(G, 0, sizeof(double) * (size_t)(total_rows_of(d, dims) * R));
    int64_t M = 1;
    for (int k = 0; k < d; ++k)
        M *= dims[k];
    double F = 0.0;
    for (int64_t L = 0; L < M; ++L) {
        int32_t idx[ORC_MAX_NDIM];
        int64_t rem = L; /* multi-index of L, last mode fastest */
        for (int k = d - 1; k >= 0; --k) {
            idx[k] = (int32_t)(rem % dims[k]);
            rem /= dims[k];
        }
        F += add_sample(d, dims, off, R, A, loss, idx, X[L], 1.0, 0, G);
    }
    return F;
}

/* ------------------------------------------------------------------ Adam */
/* Algorithm 1 applied to one flat parameter vector (Sec. 3.1.3), step t >= 1. */
void orc_adam_step(int64_t n, double *A, double *B, double *C, const double *G, double lr,
                   double beta1, double beta2, double eps, double lower, int64_t t)
{
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t e = 0; e < n; ++e) {
        B[e] = beta1 * B[e] + (1.0 - beta1) * G[e];
        C[e] = beta2 * C[e] + (1.0 - beta2) * G[e] * G[e];
        double Bh = B[e] / c1;
        double Ch = C[e] / c2;
        A[e] = A[e] - lr * (Bh / sqrt(Ch + eps));
        if (A[e] < lower)
            A[e] = lower;
    }
}

/* ------------------------------------------------------- GCP-FedAdam server */
/* Reconciliation of Algorithm 4 for n clients of one model: the
 * pseudo-gradient D = U - M_c, all-reduced as the mean over clients, updates
 * the server model U with Adam (Algorithm 1, server moments B, C, step t);
 * the caller then sets every client model to U.  M holds the n client models
 * one after another (n x len). */
void orc_fedadam_server(int64_t n, int64_t len, const double *M, double *U, double *B, double *C, double lr,
                        double beta1, double beta2, double eps, double lower, int64_t t)
{
    double *D = (double *)malloc(sizeof(double) * (size_t)len);
    for (int64_t e = 0; e < len; ++e) {
        double mean = 0.0;
        for (int64_t c = 0; c < n; ++c)
            mean += M[c * len + e];
        mean /= (double)n;
        D[e] = U[e] - mean;
    }
    orc_adam_step(len, U, B, C, D, lr, beta1, beta2, eps, lower, t);
    free(D);
}

// gcp_device.cuh -- device building blocks of the stochastic GCP gradient:
// counter-based random numbers, the nonzero hash set, the four losses and
// the vector reduction into the gradient.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gcpdev {

constexpr uint64_t kEmpty = ~0ull;  // empty hash slot (no linear index reaches 2^64-1)

// Status bits set by kernels (bit = gcp_status code).
constexpr int kErrHashFull = 1 << 5;
constexpr int kErrExhausted = 1 << 6;
constexpr int kErrNonfinite = 1 << 7;
constexpr int kErrDuplicate = 1 << 4;

// Philox stream ids (key word 1).
constexpr uint64_t kStreamNonzero = 0, kStreamZero = 1, kStreamUniform = 2, kStreamSemiZero = 3;

// ---------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon et al., SC'11): ten rounds of two 64x64->128
// multiplies; the key advances by the two Weyl constants between rounds.
struct U64x4 {
    uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B97F4A7C15ull;
            k1 += 0xBB67AE8584CAA73Bull;
        }
        const uint64_t a = 0xD2E7470EE14C6C93ull * c0, ah = __umul64hi(0xD2E7470EE14C6C93ull, c0);
        const uint64_t b = 0xCA5A826395121157ull * c2, bh = __umul64hi(0xCA5A826395121157ull, c2);
        const uint64_t n0 = bh ^ c1 ^ k0, n2 = ah ^ c3 ^ k1;
        c0 = n0;
        c1 = b;
        c2 = n2;
        c3 = a;
    }
    U64x4 r;
    r.v[0] = c0;
    r.v[1] = c1;
    r.v[2] = c2;
    r.v[3] = c3;
    return r;
}

// floor(u * n / 2^64): exact map of a 64-bit word onto [0, n).
__device__ __forceinline__ uint64_t map_range(uint64_t u, uint64_t n) { return __umul64hi(u, n); }

// --------------------------------------------------------------- hash set
// Open addressing over buckets of four uint64 keys (one 32-byte sector),
// linear probing bucket by bucket; slots of a bucket fill in order and are
// never removed, so an empty slot ends a search.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 finalizer
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

// Lookup continuing at bucket b after `done` buckets were searched:
// 1 = present, 0 = absent, -1 = probed every bucket without an answer.
__device__ __forceinline__ int hash_contains_from(const uint64_t *__restrict__ keys, uint64_t bmask,
                                                  uint64_t key, uint64_t b, uint64_t done) {
    for (uint64_t probe = done; probe <= bmask; ++probe) {
        const ulonglong2 *slot = reinterpret_cast<const ulonglong2 *>(keys + 4 * b);
        const ulonglong2 lo = __ldg(slot), hi = __ldg(slot + 1);
        if (lo.x == key || lo.y == key || hi.x == key || hi.y == key) return 1;
        if (lo.x == kEmpty || lo.y == kEmpty || hi.x == kEmpty || hi.y == kEmpty) return 0;
        b = (b + 1) & bmask;
    }
    return -1;
}

__device__ __forceinline__ int hash_contains(const uint64_t *__restrict__ keys, uint64_t bmask, uint64_t key) {
    return hash_contains_from(keys, bmask, key, mix64(key) & bmask, 0);
}

// Decide a lookup from one bucket already in registers: 1 / 0 as above,
// 2 = bucket full without the key (continue at the next bucket).
__device__ __forceinline__ int bucket_decide(ulonglong2 lo, ulonglong2 hi, uint64_t key) {
    if (lo.x == key || lo.y == key || hi.x == key || hi.y == key) return 1;
    if (lo.x == kEmpty || lo.y == kEmpty || hi.x == kEmpty || hi.y == kEmpty) return 0;
    return 2;
}

// 0 = inserted, kErrDuplicate, or kErrHashFull.
__device__ __forceinline__ int hash_insert(uint64_t *keys, uint64_t bmask, uint64_t key) {
    uint64_t b = mix64(key) & bmask;
    for (uint64_t probe = 0; probe <= bmask; ++probe) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long *>(keys + 4 * b + s),
                                                (unsigned long long)kEmpty, (unsigned long long)key);
            if (prev == kEmpty) return 0;
            if (prev == key) return kErrDuplicate;
        }
        b = (b + 1) & bmask;
    }
    return kErrHashFull;
}

// ----------------------------------------------------------------- losses
constexpr float kLossEps = 1e-10f;

// FP32 losses with the fast hardware log, exp and division (__logf,
// __expf, __fdividef: a few ulp, or 2^-21 absolute for log outside
// [0.5, 2]); the sampled loss and gradient stay within 1e-5 relative of the
// FP64 definitions.
__device__ __forceinline__ void loss_eval(int loss, float x, float m, float &f, float &df) {
    switch (loss) {
    case 0: {  // Gaussian
        const float r = x - m;
        f = r * r;
        df = -2.0f * r;
        break;
    }
    case 1: {  // Poisson, identity link
        const float me = m + kLossEps;
        f = m - x * __logf(me);
        df = 1.0f - __fdividef(x, me);
        break;
    }
    case 2: {  // Bernoulli, logit link
        const float e = __expf(-fabsf(m));
        const float inv = __fdividef(1.0f, 1.0f + e);
        f = fmaxf(m, 0.0f) + log1pf(e) - x * m;
        df = (m >= 0.0f ? inv : e * inv) - x;
        break;
    }
    default: {  // Gamma
        const float me = m + kLossEps;
        const float inv = __fdividef(1.0f, me);
        f = x * inv + __logf(me);
        df = inv - x * inv * inv;
        break;
    }
    }
}

// ------------------------------------------------------------ vector I/O
// Four consecutive factor entries widened to FP32 (16 B of FP32 or 8 B of
// BF16), read through the non-coherent path: factors do not change while a
// kernel runs.
template <typename TF>
struct Quad;

template <>
struct Quad<float> {
    __device__ __forceinline__ static void load(const float *p, float *o) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
};

template <>
struct Quad<__nv_bfloat16> {
    __device__ __forceinline__ static void load(const __nv_bfloat16 *p, float *o) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        o[0] = __uint_as_float(v.x << 16);
        o[1] = __uint_as_float(v.x & 0xFFFF0000u);
        o[2] = __uint_as_float(v.y << 16);
        o[3] = __uint_as_float(v.y & 0xFFFF0000u);
    }
};

// Asynchronous global -> shared copies (LDGSTS), grouped per thread.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Fire-and-forget FP32 vector reduction into global memory (sm_90+).
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

}  // namespace gcpdev

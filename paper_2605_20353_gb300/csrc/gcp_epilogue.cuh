// gcp_epilogue.cuh -- the hot-row replica fold shared by the step epilogues
// (k_post_step for one context, k_batch_post for a batch of clients).
//
// The fused pass sends the gradient reductions of rows that many samples hit
// to kReplicas replicas (gcpk::kReplicas planes of Htot x Rp floats); the
// epilogue adds them into the row's gradient before Adam.  A hot quad (four
// columns of a hot row) has kReplicas replica quads; loaded one after
// another they cost a memory round trip per group, so instead a group of
// kHotLanes lanes takes one hot quad and every replica load is in flight at
// once.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gcpe {

constexpr int kHotLanes = 16;  // lanes that fold one hot quad together

// Sum of the nrep replica quads R4[r * plane4 + o], r = 0..nrep-1, over a
// group of kHotLanes lanes: lane l of the group (l = lane & 15) loads
// replicas l, l + 16, l + 32, ..., adds them in that order, then the group
// sums its lanes with a butterfly (offsets 8, 4, 2, 1).  The order is fixed,
// so the result does not vary from run to run.  Every lane returns the
// total; each lane clears the replicas it loaded.  All lanes of the group
// must call it together (gmask = the group's lanes).
template <int nrep>
__device__ __forceinline__ float4 hot_quad_sum(float4 *__restrict__ R4, int64_t plane4, int64_t o, unsigned gmask) {
    static_assert(nrep % kHotLanes == 0, "replicas split evenly over the group's lanes");
    constexpr int kPer = nrep / kHotLanes;
    const int l = threadIdx.x & (kHotLanes - 1);
    float4 v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) v[i] = R4[(int64_t)(l + kHotLanes * i) * plane4 + o];
    float4 t = v[0];
#pragma unroll
    for (int i = 1; i < kPer; ++i) {
        t.x += v[i].x;
        t.y += v[i].y;
        t.z += v[i].z;
        t.w += v[i].w;
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) R4[(int64_t)(l + kHotLanes * i) * plane4 + o] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int off = kHotLanes / 2; off > 0; off >>= 1) {
        t.x += __shfl_xor_sync(gmask, t.x, off);
        t.y += __shfl_xor_sync(gmask, t.y, off);
        t.z += __shfl_xor_sync(gmask, t.z, off);
        t.w += __shfl_xor_sync(gmask, t.w, off);
    }
    return t;
}

// Mask of the kHotLanes-lane group of the calling lane.
__device__ __forceinline__ unsigned hot_group_mask() {
    return ((1u << kHotLanes) - 1u) << ((threadIdx.x & 31) & ~(kHotLanes - 1));
}

}  // namespace gcpe

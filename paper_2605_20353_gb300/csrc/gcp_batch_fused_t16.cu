// gcp_batch_fused_t16.cu -- the multi-client fused kernel with 16 samples
// per warp tile, every order, factor storage and lane-column count.
#include "gcp_batch_fused.cuh"

namespace gcpb {

template cudaError_t batch_fused_launch<16>(int, bool, int, int, const int4 *, const int *, int, int, int, int,
                                            const uint64_t *, float2 *, cudaStream_t);
template cudaError_t batch_fused_allow<16>(int, bool, int);
template int batch_fused_occupancy<16>(int, bool, int);

}  // namespace gcpb

// Instantiation of the leaf kernels for float TRSM.
#include "leaf_block256.cuh"
#include "leaf_blocked.cuh"
#include "leaf_impl.cuh"

namespace trx {
template cudaError_t leaf_dispatch<float, true>(const LeafArgs<float>&, int64_t, int, int64_t, cudaStream_t);
template cudaError_t leaf_configure<float, true>();
template cudaError_t leaf_blocked_configure<float>();
template cudaError_t leaf_blocked_launch<float>(const LeafArgs<float>&, int64_t, cudaStream_t);
template cudaError_t leaf_b256_configure<float>();
template cudaError_t leaf_b256_launch<float>(const LeafArgs<float>&, cudaStream_t);
}  // namespace trx

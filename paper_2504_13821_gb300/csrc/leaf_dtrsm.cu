// Instantiation of the leaf kernels for double TRSM.
#include "leaf_block256.cuh"
#include "leaf_blocked.cuh"
#include "leaf_impl.cuh"

namespace trx {
template cudaError_t leaf_dispatch<double, true>(const LeafArgs<double>&, int64_t, int, int64_t, cudaStream_t);
template cudaError_t leaf_configure<double, true>();
template cudaError_t leaf_blocked_configure<double>();
template cudaError_t leaf_blocked_launch<double>(const LeafArgs<double>&, int64_t, cudaStream_t);
template cudaError_t leaf_b256_configure<double>();
template cudaError_t leaf_b256_launch<double>(const LeafArgs<double>&, cudaStream_t);
}  // namespace trx

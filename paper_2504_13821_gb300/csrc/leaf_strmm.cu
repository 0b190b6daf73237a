// Instantiation of the leaf kernels for float TRMM.
#include "leaf_impl.cuh"

namespace trx {
template cudaError_t leaf_dispatch<float, false>(const LeafArgs<float>&, int64_t, int, int64_t, cudaStream_t);
template cudaError_t leaf_configure<float, false>();
}  // namespace trx

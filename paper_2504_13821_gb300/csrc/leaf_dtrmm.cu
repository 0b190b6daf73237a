// Instantiation of the leaf kernels for double TRMM.
#include "leaf_impl.cuh"

namespace trx {
template cudaError_t leaf_dispatch<double, false>(const LeafArgs<double>&, int64_t, int, int64_t, cudaStream_t);
template cudaError_t leaf_configure<double, false>();
}  // namespace trx

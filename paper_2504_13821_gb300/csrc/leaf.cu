// Leaf kernels: lane-count choice and dispatch. The kernels themselves are in
// leaf_impl.cuh.
#include <cstdlib>
#include <type_traits>

#include "leaf_impl.cuh"

namespace trx {

// One translation unit per (type, operation) keeps the unrolled sweeps'
// compile time in parallel; leaf_*.cu instantiate these.
template <typename T, bool TRSM>
cudaError_t leaf_dispatch(const LeafArgs<T>& a, int64_t nleaves, int G, int64_t max_ctas,
                          cudaStream_t s);
extern template cudaError_t leaf_dispatch<float, true>(const LeafArgs<float>&, int64_t, int, int64_t, cudaStream_t);
extern template cudaError_t leaf_dispatch<float, false>(const LeafArgs<float>&, int64_t, int, int64_t, cudaStream_t);
extern template cudaError_t leaf_dispatch<double, true>(const LeafArgs<double>&, int64_t, int, int64_t, cudaStream_t);
extern template cudaError_t leaf_dispatch<double, false>(const LeafArgs<double>&, int64_t, int, int64_t, cudaStream_t);

template <typename T, bool TRSM>
cudaError_t leaf_configure();
extern template cudaError_t leaf_configure<float, true>();
extern template cudaError_t leaf_configure<float, false>();
extern template cudaError_t leaf_configure<double, true>();
extern template cudaError_t leaf_configure<double, false>();

cudaError_t tc_configure();

template <typename T>
cudaError_t leaf_blocked_configure();
template <typename T>
cudaError_t leaf_blocked_launch(const LeafArgs<T>& a, int64_t max_ctas, cudaStream_t s);
extern template cudaError_t leaf_blocked_configure<float>();
extern template cudaError_t leaf_blocked_configure<double>();
extern template cudaError_t leaf_blocked_launch<float>(const LeafArgs<float>&, int64_t, cudaStream_t);
extern template cudaError_t leaf_blocked_launch<double>(const LeafArgs<double>&, int64_t, cudaStream_t);

template <typename T>
cudaError_t leaf_b256_configure();
template <typename T>
cudaError_t leaf_b256_launch(const LeafArgs<T>& a, cudaStream_t s);
extern template cudaError_t leaf_b256_configure<float>();
extern template cudaError_t leaf_b256_configure<double>();
extern template cudaError_t leaf_b256_launch<float>(const LeafArgs<float>&, cudaStream_t);
extern template cudaError_t leaf_b256_launch<double>(const LeafArgs<double>&, cudaStream_t);

cudaError_t leaf_wide_configure();
cudaError_t leaf_wide_launch(const LeafArgs<float>& a, int num_sms, cudaStream_t s);
cudaError_t convert_configure();
cudaError_t refine_configure();
cudaError_t dag_configure();
cudaError_t thin_configure();

// Kernel attributes (dynamic shared-memory limits) for the current device:
// run once per device by every handle's and the allocation-free entry's
// set-up, since an attribute set on one device does not carry to another.
cudaError_t leaf_configure_all() {
    cudaError_t e;
    if ((e = leaf_configure<float, true>()) != cudaSuccess) return e;
    if ((e = leaf_configure<float, false>()) != cudaSuccess) return e;
    if ((e = leaf_configure<double, true>()) != cudaSuccess) return e;
    if ((e = leaf_configure<double, false>()) != cudaSuccess) return e;
    if ((e = leaf_blocked_configure<float>()) != cudaSuccess) return e;
    if ((e = leaf_blocked_configure<double>()) != cudaSuccess) return e;
    if ((e = leaf_b256_configure<float>()) != cudaSuccess) return e;
    if ((e = leaf_b256_configure<double>()) != cudaSuccess) return e;
    if ((e = leaf_wide_configure()) != cudaSuccess) return e;
    if ((e = convert_configure()) != cudaSuccess) return e;
    if ((e = refine_configure()) != cudaSuccess) return e;
    if ((e = dag_configure()) != cudaSuccess) return e;
    if ((e = thin_configure()) != cudaSuccess) return e;
    return tc_configure();
}

template <typename T>
cudaError_t launch_leaf(bool trsm, const Canon<T>& p, int64_t r0, int b,
                        int64_t nleaves, T alpha, const Planes* planes,
                        int num_sms, cudaStream_t s) {
    if (b < 1 || nleaves < 1 || nleaves > 65535) return cudaErrorInvalidValue;
    if (b > kMaxLeaf && !(trsm && nleaves == 1 && b <= kMaxBlockLeaf)) return cudaErrorInvalidValue;
    if (p.nrhs <= 0) return cudaSuccess;
    LeafArgs<T> a;
    a.p = p;
    a.r0 = r0;
    a.b = b;
    a.alpha = alpha;
    a.planes = planes != nullptr;
    if (planes) a.pl = *planes;
    // A single TRSM leaf with at least 1024 right-hand sides takes a blocked
    // kernel: FP32 leaves of 65..128 rows the wide kernel, other leaves of
    // 33..128 rows the blocked kernel (16-row substitutions + rank-16
    // updates); the lane-split sweep below covers the rest.
    // TRX_LEAF_BLOCKED=0 turns both off.
    static const bool blocked_on = [] {
        const char* e = std::getenv("TRX_LEAF_BLOCKED");
        return !(e && e[0] == '0');
    }();
    if (trsm && b > kMaxLeaf) return leaf_b256_launch<T>(a, s);   // block leaf, 129..256 rows
    // FP32, one leaf of 65..128 rows, many right-hand sides: the wide kernel
    // (register-resident tiles, four column groups per CTA).
    if constexpr (std::is_same<T, float>::value) {
        if (blocked_on && trsm && nleaves == 1 && b > 64 && p.nrhs >= 1024)
            return leaf_wide_launch(a, num_sms, s);
    }
    if (blocked_on && trsm && nleaves == 1 && b > 32 && p.nrhs >= 1024)
        return leaf_blocked_launch<T>(a, (int64_t)(num_sms > 0 ? num_sms : 1) * 2, s);

    // Lanes per right-hand side, from the right-hand sides per SM: one lane
    // per column when there are many (no shuffles, widest vector reuse),
    // more lanes when there are few, to keep enough warps in flight.
    const int64_t cols_per_sm = p.nrhs * nleaves / (num_sms > 0 ? num_sms : 1);
    // (Measured at b = 64, 16384 right-hand sides: 4 lanes beat 8 and 16;
    // one lane per column is used where its registers allow, b <= 32.)
    int G = 16;
    if (cols_per_sm >= 2048 && b <= 32) G = 1;
    else if (cols_per_sm >= 64) G = 4;
    else if (cols_per_sm >= 16) G = 8;
    // TRX_LEAF_LANES (1, 4, 8 or 16) overrides the choice, for tuning runs.
    static const int forced = [] {
        const char* e = std::getenv("TRX_LEAF_LANES");
        return e ? std::atoi(e) : 0;
    }();
    if (forced == 1 || forced == 4 || forced == 8 || forced == 16) G = forced;
    // One leaf: a few CTAs per SM walk its panels. Many leaves at once (the
    // level-batched TRMM): enough CTAs that panel latencies overlap across
    // CTAs instead of queueing inside each.
    const int64_t max_ctas = (int64_t)(num_sms > 0 ? num_sms : 1) * (nleaves > 1 ? 32 : 4);
    return trsm ? leaf_dispatch<T, true>(a, nleaves, G, max_ctas, s)
                : leaf_dispatch<T, false>(a, nleaves, G, max_ctas, s);
}

template cudaError_t launch_leaf<float>(bool, const Canon<float>&, int64_t, int, int64_t, float,
                                        const Planes*, int, cudaStream_t);
template cudaError_t launch_leaf<double>(bool, const Canon<double>&, int64_t, int, int64_t, double,
                                         const Planes*, int, cudaStream_t);

}  // namespace trx

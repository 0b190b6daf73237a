// Leaf ("base case") TRSM and TRMM kernels, Section 3.3 of the paper.
//
// Below the recursion cutoff a diagonal block of M (b x b, lower, canonical
// form of common.cuh) is applied to all right-hand sides of its row block:
//   TRSM: solve M_blk X = alpha C_blk by forward substitution, X -> C_blk
//   TRMM: C_blk := alpha M_blk C_blk
//
// Layout on the device. One CTA takes one b-row block and a panel of NCOL
// right-hand sides. The triangle (zero above the diagonal and beyond a
// ragged edge) and its reciprocal diagonal sit in shared memory; the panel
// is staged through shared memory with coalesced loads (rows or columns
// fastest, whichever is contiguous in global memory) and then held in
// registers. G lanes share one right-hand side: lane g owns rows g, g+G,
// g+2G, ... (interleaved, so the shrinking active set stays balanced).
//
// The sweep: step j broadcasts x_j from its owner lane with a warp shuffle
// (G > 1) and every lane updates its own rows below j with one FMA each,
// reading M(i, j) from shared memory (a broadcast across the panel's
// columns). There is no block-level barrier inside the sweep: the
// dependency between rows that the paper resolves with one synchronisation
// per row is carried by the shuffle inside the G-lane group, and columns are
// independent (Section 3.3, "Reformulation of algorithm for parallelism").
// With G = 1 a thread owns a whole column and the sweep needs no
// communication at all.
//
// TRMM runs the columns of M in descending order, so every x_j is read
// before any update writes row j (in place, no copy).
#pragma once
#include <type_traits>

#include "common.cuh"

namespace trx {

template <typename T>
struct LeafArgs {
    Canon<T> p;
    int64_t r0;     // start row of leaf 0 of this launch
    int b;          // leaf size (row stride between batched leaves)
    T alpha;
    Planes pl;
    int planes;     // TRSM on the tensor-core path: also write the Y planes
};

namespace {

template <typename T, int B, int G>
struct LeafShape {
    static constexpr int NT = (sizeof(T) == 8 && B == 128) ? 64 : 128;
    static constexpr int NCOL = NT / G;
    static constexpr int PAD = (G == 1) ? 1 : G;   // bank-conflict-free panel
    static constexpr int LDS = B + PAD;
    static constexpr int RPL = B / G;               // rows per lane
    static constexpr size_t smem = sizeof(T) * (size_t)(B * B + B + NCOL * LDS);
    static_assert((B * B) % NT == 0 && (B * NCOL) % NT == 0, "staging loops assume whole passes");
};

template <typename T, int B, int G, bool TRSM>
__global__ void __launch_bounds__(LeafShape<T, B, G>::NT)
leaf_kernel(LeafArgs<T> a) {
    using S = LeafShape<T, B, G>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sT = reinterpret_cast<T*>(smem_raw);   // sT[l*B + i] = M(r0+i, r0+l), i > l
    T* sD = sT + B * B;                        // 1/M(i,i) (TRSM) or M(i,i) (TRMM)
    T* sC = sD + B;                            // sC[c*LDS + i] = C(r0+i, j0+c)

    const int tid = threadIdx.x;
    const Canon<T>& p = a.p;
    const int64_t r0 = a.r0 + (int64_t)blockIdx.y * a.b;
    const int64_t rem = p.k - r0;
    if (rem <= 0) return;
    const int bs = rem < a.b ? (int)rem : a.b;
    const int64_t j0 = (int64_t)blockIdx.x * S::NCOL;

    // Diagonal block of M: strictly-lower part and diagonal.
    // Every staging loop is unrolled (compile-time trip counts) so all of
    // its global loads are in flight together.
    const bool a_row_fast = (p.a_rs == 1 || p.a_rs == -1);
#pragma unroll
    for (int u = 0; u < B * B / S::NT; ++u) {
        const int idx = tid + u * S::NT;
        int i, l;
        if (a_row_fast) { i = idx % B; l = idx / B; } else { l = idx % B; i = idx / B; }
        T v = T(0);
        if (i < bs && l < i) v = p.A[(r0 + i) * p.a_rs + (r0 + l) * p.a_cs];
        sT[l * B + i] = v;
    }
    for (int i = tid; i < B; i += S::NT) {
        T d = T(1);
        if (i < bs && !p.unit) d = p.A[(r0 + i) * (p.a_rs + p.a_cs)];
        if (TRSM) sD[i] = (i < bs && !p.unit) ? T(1) / d : T(1);
        else      sD[i] = (i < bs) ? d : T(0);
    }
    // Right-hand-side panel.
    const bool c_row_fast = (p.c_rs == 1 || p.c_rs == -1);
#pragma unroll
    for (int u = 0; u < B * S::NCOL / S::NT; ++u) {
        const int idx = tid + u * S::NT;
        int i, c;
        if (c_row_fast) { i = idx % B; c = idx / B; } else { c = idx % S::NCOL; i = idx / S::NCOL; }
        const int64_t j = j0 + c;
        T v = T(0);
        if (i < bs && j < p.nrhs) v = p.C[(r0 + i) * p.c_rs + j * p.c_cs];
        sC[c * S::LDS + i] = v;
    }
    __syncthreads();

    const int c = tid / G, g = tid % G;
    T r[S::RPL];
#pragma unroll
    for (int q = 0; q < S::RPL; ++q) r[q] = sC[c * S::LDS + q * G + g];

    if (TRSM) {
#pragma unroll
        for (int q = 0; q < S::RPL; ++q) r[q] *= a.alpha;
#pragma unroll
        for (int jj = 0; jj < B; ++jj) {
            const int qj = jj / G, gj = jj % G;
            const T v = r[qj] * sD[jj];
            T xj;
            if (G == 1) {
                r[qj] = v;
                xj = v;
            } else {
                xj = __shfl_sync(0xffffffffu, v, gj, G);
                if (g == gj) r[qj] = v;
            }
#pragma unroll
            for (int q = qj; q < S::RPL; ++q) {
                if (q == qj && g <= gj) continue;
                r[q] = fma(-sT[jj * B + q * G + g], xj, r[q]);
            }
        }
    } else {
#pragma unroll
        for (int jj = B - 1; jj >= 0; --jj) {
            const int qj = jj / G, gj = jj % G;
            const T xj = (G == 1) ? r[qj] : __shfl_sync(0xffffffffu, r[qj], gj, G);
#pragma unroll
            for (int q = qj; q < S::RPL; ++q) {
                if (q == qj && g <= gj) continue;
                r[q] = fma(sT[jj * B + q * G + g], xj, r[q]);
            }
            if (g == gj) r[qj] = sD[jj] * xj;
        }
#pragma unroll
        for (int q = 0; q < S::RPL; ++q) r[q] *= a.alpha;
    }

#pragma unroll
    for (int q = 0; q < S::RPL; ++q) sC[c * S::LDS + q * G + g] = r[q];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < B * S::NCOL / S::NT; ++u) {
        const int idx = tid + u * S::NT;
        int i, cc;
        if (c_row_fast) { i = idx % B; cc = idx / B; } else { cc = idx % S::NCOL; i = idx / S::NCOL; }
        const int64_t j = j0 + cc;
        if (i < bs && j < p.nrhs) p.C[(r0 + i) * p.c_rs + j * p.c_cs] = sC[cc * S::LDS + i];
    }
    if constexpr (std::is_same<T, float>::value) {
        if (TRSM && a.planes) {
            // Y planes, element (l, j) at j*ldy + l: rows fastest.
#pragma unroll
            for (int u = 0; u < B * S::NCOL / S::NT; ++u) {
                const int idx = tid + u * S::NT;
                const int i = idx % B, cc = idx / B;
                const int64_t j = j0 + cc;
                if (i < bs && j < p.nrhs) {
                    const float x = sC[cc * S::LDS + i];
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                    const int64_t o = j * a.pl.ldy + r0 + i;
                    a.pl.y_hi[o] = hi;
                    a.pl.y_lo[o] = lo;
                }
            }
        }
    }
}

template <typename T, int B, int G, bool TRSM>
cudaError_t configure_one() {
    using S = LeafShape<T, B, G>;
    return cudaFuncSetAttribute(leaf_kernel<T, B, G, TRSM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
}

template <typename T, int B, int G, bool TRSM>
cudaError_t launch_one(const LeafArgs<T>& a, int64_t nleaves, cudaStream_t s) {
    using S = LeafShape<T, B, G>;
    const int64_t nx = (a.p.nrhs + S::NCOL - 1) / S::NCOL;
    dim3 grid((unsigned)nx, (unsigned)nleaves);
    leaf_kernel<T, B, G, TRSM><<<grid, S::NT, S::smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int B, bool TRSM>
cudaError_t launch_b(const LeafArgs<T>& a, int64_t nleaves, int G, cudaStream_t s) {
    // A thread owns B/G rows in registers; B/G is kept at 64 or below so the
    // fully unrolled sweep keeps them in registers.
    if constexpr (B <= 64) {
        if (G == 1) return launch_one<T, B, 1, TRSM>(a, nleaves, s);
    }
    if (G <= 4) return launch_one<T, B, 4, TRSM>(a, nleaves, s);
    return launch_one<T, B, 16, TRSM>(a, nleaves, s);
}

}  // namespace

// Shared-memory limits of every instantiation, once per device (the
// handle calls this at creation, before any launch can be captured).
template <typename T, bool TRSM>
cudaError_t leaf_configure() {
    cudaError_t e;
#define TRX_CFG(B, G) \
    if ((e = configure_one<T, B, G, TRSM>()) != cudaSuccess) return e;
    TRX_CFG(16, 1) TRX_CFG(16, 4) TRX_CFG(16, 16)
    TRX_CFG(32, 1) TRX_CFG(32, 4) TRX_CFG(32, 16)
    TRX_CFG(64, 1) TRX_CFG(64, 4) TRX_CFG(64, 16)
    TRX_CFG(128, 4) TRX_CFG(128, 16)
#undef TRX_CFG
    return cudaSuccess;
}

template <typename T, bool TRSM>
cudaError_t leaf_dispatch(const LeafArgs<T>& a, int64_t nleaves, int G, cudaStream_t s) {
    if (a.b <= 16) return launch_b<T, 16, TRSM>(a, nleaves, G, s);
    if (a.b <= 32) return launch_b<T, 32, TRSM>(a, nleaves, G, s);
    if (a.b <= 64) return launch_b<T, 64, TRSM>(a, nleaves, G, s);
    return launch_b<T, 128, TRSM>(a, nleaves, G, s);
}


}  // namespace trx

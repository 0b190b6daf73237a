// Batched uneven TRSM / TRMM: thousands of small independent problems
// (order k <= 512) in one persistent launch.
//
// Each problem is first mapped on the host to the canonical lower form of
// common.cuh (any side/uplo/trans/diag, TRSM or TRMM). The descriptors are
// sorted by cost (k^2 * nrhs, largest first) and the CTAs of one persistent
// grid take them from an atomic counter, so big problems start first and
// the tail is filled with small ones.
//
// Inside a CTA a problem runs on its right-hand side staged in shared
// memory in chunks of NC columns (k rows x NC, row-major):
//   TRSM (forward): rows taken sb at a time (sb = 4, 8 or 16, per problem
//     from the tuning table): substitution on the sb-row diagonal block (one
//     thread per column, the block's tile of M staged in shared memory during
//     the previous block's update), then a rank-sb update of every row below
//     it, each thread a register tile of 4 rows x 4 columns;
//   TRMM: out of place, every row's alpha * sum_{l <= i} M(i,l) C(l,:)
//     formed from the staged original columns and written straight back to
//     global memory, again in 4 x 4 register tiles.
// M is read through the read-only cache (its rows are reused across the
// column groups of a CTA). Problems with k > 512 belong to the plain
// recursive entry points.
#include <algorithm>

#include "common.cuh"

namespace trx {

struct BatchDesc {
    int64_t k, nrhs;
    const void* A;
    int64_t a_rs, a_cs;
    void* C;
    int64_t c_rs, c_cs;
    double alpha;
    int unit, trsm, sb, pad;
};

constexpr int kBatchMaxK = 512;

namespace {

template <typename T>
struct BShape {
    static constexpr int NT = 256;
    static constexpr int NC = sizeof(T) == 4 ? 32 : 16;    // columns per chunk
    static constexpr int LDC = NC + 1;                     // odd stride: three CTAs per SM
    static constexpr int CG = NC / 4;                      // column groups of 4
    static constexpr int RG = NT / CG;                     // row groups
    static constexpr int SBMAX = 16;                       // largest substitution block
    // panel, diagonal, two staged diagonal tiles of the substitution blocks
    static constexpr size_t smem =
        sizeof(T) * ((size_t)kBatchMaxK * LDC + kBatchMaxK + 2 * SBMAX * SBMAX);
};

template <typename T>
__device__ __forceinline__ T ldA(const T* A, int64_t i, int64_t l, int64_t rs, int64_t cs) {
    return __ldg(A + i * rs + l * cs);
}

template <typename T, int SB>
__device__ __forceinline__ void trsm_chunk(const BatchDesc& d, T* sC, const T* sD, T* sTile,
                                           int k) {
    using S = BShape<T>;
    static_assert(SB <= S::SBMAX, "substitution block above the staged tile size");
    const int tid = threadIdx.x;
    const T* A = static_cast<const T*>(d.A);
    const int cg = tid % S::CG, rg = tid / S::CG;
    // The SB x SB diagonal tile of block s (strictly lower, zeros elsewhere)
    // is staged in shared memory during block s-1's update, so the serial
    // substitution reads it without waiting on global memory.
    const bool row_fast = (d.a_rs == 1 || d.a_rs == -1);
    auto stage_tile = [&](int s1, T* dst) {
        for (int e = tid; e < SB * SB; e += S::NT) {
            const int q = row_fast ? e % SB : e / SB, jj = row_fast ? e / SB : e % SB;
            dst[q * SB + jj] = (q > jj && s1 + q < k) ? ldA(A, s1 + q, s1 + jj, d.a_rs, d.a_cs)
                                                      : T(0);
        }
    };
    stage_tile(0, sTile);
    __syncthreads();
    int buf = 0;
    for (int s0 = 0; s0 < k; s0 += SB) {
        const int sbn = min(SB, k - s0);
        const T* tile = sTile + buf * S::SBMAX * S::SBMAX;
        if (tid < S::NC) {
            T x[SB];
#pragma unroll
            for (int q = 0; q < SB; ++q) x[q] = q < sbn ? sC[(s0 + q) * S::LDC + tid] : T(0);
            // Rows past k (a ragged last block) stay zero: their diagonal
            // factor is 1 and their tile entries are zero.
#pragma unroll
            for (int jj = 0; jj < SB; ++jj) {
                x[jj] *= (jj < sbn) ? sD[s0 + jj] : T(1);
#pragma unroll
                for (int q = jj + 1; q < SB; ++q) x[q] = fma(-tile[q * SB + jj], x[jj], x[q]);
            }
#pragma unroll
            for (int q = 0; q < SB; ++q)
                if (q < sbn) sC[(s0 + q) * S::LDC + tid] = x[q];
        }
        __syncthreads();
        if (s0 + SB < k) stage_tile(s0 + SB, sTile + (buf ^ 1) * S::SBMAX * S::SBMAX);
        // Rank-SB update of the rows below the block: each thread a tile of
        // 4 rows x 4 columns (4 loads of M feed 16 multiply-adds).
        for (int i0 = s0 + SB + 4 * rg; i0 < k; i0 += 4 * S::RG) {
            T acc[4][4] = {};
            // M(i0+r, s0+kk) by pointers walking along the block's columns
            const T* ap[4];
            bool ok[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                ok[r] = i0 + r < k;
                ap[r] = A + (int64_t)(ok[r] ? i0 + r : 0) * d.a_rs + (int64_t)s0 * d.a_cs;
            }
#pragma unroll 4
            for (int kk = 0; kk < SB; ++kk) {
                const int l = s0 + kk;
                T t[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    t[r] = ok[r] ? __ldg(ap[r]) : T(0);
                    ap[r] += d.a_cs;
                }
                T xv[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) xv[v] = sC[l * S::LDC + 4 * cg + v];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[r][v] = fma(t[r], xv[v], acc[r][v]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (i0 + r < k) {
#pragma unroll
                    for (int v = 0; v < 4; ++v) sC[(i0 + r) * S::LDC + 4 * cg + v] -= acc[r][v];
                }
        }
        __syncthreads();
        buf ^= 1;
    }
}

// TRMM out of place: the chunk's original columns stay in shared memory and
// every row's new value alpha * sum_{l <= i} M(i,l) C(l,:) goes straight to
// global memory, each thread a tile of 4 rows x 4 columns.
template <typename T>
__device__ __forceinline__ void trmm_chunk(const BatchDesc& d, const T* sC, const T* sD, int k, T alpha,
                           T* C, int64_t c0, int ncols) {
    using S = BShape<T>;
    const int tid = threadIdx.x;
    const T* A = static_cast<const T*>(d.A);
    const int cg = tid % S::CG, rg = tid / S::CG;
    for (int i0 = 4 * rg; i0 < k; i0 += 4 * S::RG) {
        T acc[4][4] = {};
        const int lend = min(i0 + 3, k - 1);          // strictly-lower columns l < i
        const T* ap[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) ap[r] = A + (int64_t)(i0 + r < k ? i0 + r : 0) * d.a_rs;
#pragma unroll 2
        for (int l = 0; l < lend; ++l) {
            T t[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                t[r] = (l < i0 + r && i0 + r < k) ? __ldg(ap[r]) : T(0);
                ap[r] += d.a_cs;
            }
            T xv[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) xv[v] = sC[l * S::LDC + 4 * cg + v];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[r][v] = fma(t[r], xv[v], acc[r][v]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + r;
            if (i >= k) break;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int c = 4 * cg + v;
                if (c < ncols)
                    C[i * d.c_rs + (c0 + c) * d.c_cs] =
                        alpha * fma(sD[i], sC[i * S::LDC + c], acc[r][v]);
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 3) batched_kernel(const BatchDesc* descs, int64_t count,
                                                      int* counter) {
    using S = BShape<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sC = reinterpret_cast<T*>(smem_raw);         // panel: row i, column c at i*LDC + c
    T* sD = sC + (size_t)kBatchMaxK * S::LDC;         // reciprocal (TRSM) or plain (TRMM) diagonal
    T* sTile = sD + kBatchMaxK;                        // two staged diagonal tiles
    __shared__ int s_next;
    pdl_trigger();
    pdl_wait();
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t idx = s_next;
        __syncthreads();
        if (idx >= count) break;
        const BatchDesc d = descs[idx];
        const int k = (int)d.k;
        const T* A = static_cast<const T*>(d.A);
        T* C = static_cast<T*>(d.C);
        if (d.trsm == 2) {   // alpha == 0: B := 0, A is not read
            for (int64_t e = tid; e < d.k * d.nrhs; e += S::NT)
                C[(e % d.k) * d.c_rs + (e / d.k) * d.c_cs] = T(0);
            continue;
        }
        // Pull the problem's triangle toward L2 in 128-byte lines along A's
        // contiguous index, so the blocks' first reads of M do not each wait
        // on DRAM.
        {
            constexpr int LINE = 128 / (int)sizeof(T);
            const bool rf = (d.a_rs == 1 || d.a_rs == -1);
            const int per = (k + LINE - 1) / LINE;
            for (int e = tid; e < k * per; e += S::NT) {
                const int fixed = e / per, w = (e % per) * LINE;   // fixed: column (rf) or row
                const int i = rf ? w : fixed, l = rf ? fixed : w;
                if (i < k && l < k) {
                    const T* ptr = A + (int64_t)i * d.a_rs + (int64_t)l * d.a_cs;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
                }
            }
        }
        for (int i = tid; i < k; i += S::NT) {
            T dg = T(1);
            if (!d.unit) dg = A[(int64_t)i * (d.a_rs + d.a_cs)];
            sD[i] = d.trsm ? T(1) / dg : dg;
        }
        for (int64_t c0 = 0; c0 < d.nrhs; c0 += S::NC) {
            const int ncols = (int)min((int64_t)S::NC, d.nrhs - c0);
            // stage the chunk; rows fastest when C's rows are contiguous
            const bool row_fast = (d.c_rs == 1 || d.c_rs == -1);
            for (int e = tid; e < k * S::NC; e += S::NT) {
                const int i = row_fast ? e % k : e / S::NC, c = row_fast ? e / k : e % S::NC;
                T v = T(0);
                if (c < ncols) v = C[i * d.c_rs + (c0 + c) * d.c_cs];
                sC[i * S::LDC + c] = d.trsm ? (T)d.alpha * v : v;
            }
            __syncthreads();
            if (d.trsm) {
                if (d.sb == 4) trsm_chunk<T, 4>(d, sC, sD, sTile, k);
                else if (d.sb == 8) trsm_chunk<T, 8>(d, sC, sD, sTile, k);
                else trsm_chunk<T, 16>(d, sC, sD, sTile, k);
                for (int e = tid; e < k * S::NC; e += S::NT) {
                    const int i = row_fast ? e % k : e / S::NC, c = row_fast ? e / k : e % S::NC;
                    if (c < ncols) C[i * d.c_rs + (c0 + c) * d.c_cs] = sC[i * S::LDC + c];
                }
            } else {
                trmm_chunk<T>(d, sC, sD, k, (T)d.alpha, C, c0, ncols);
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t batched_configure() {
    cudaError_t e = cudaFuncSetAttribute(batched_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BShape<float>::smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batched_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)BShape<double>::smem);
}

// Resident CTAs per SM of the batched kernel (occupancy query, at least 1).
int batched_ctas_per_sm(int elem_bytes) {
    int n = 0;
    const cudaError_t e = elem_bytes == 4
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_kernel<float>, BShape<float>::NT,
                                                        BShape<float>::smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_kernel<double>, BShape<double>::NT,
                                                        BShape<double>::smem);
    return (e == cudaSuccess && n > 0) ? n : 1;
}

// descs: device array of `count` descriptors sorted largest first; counter:
// device int, zeroed here before the launch. grid_ctas persistent CTAs.
cudaError_t launch_batched(int elem_bytes, const BatchDesc* descs, int64_t count, int* counter,
                           int grid_ctas, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(grid_ctas, count);
    if (elem_bytes == 4)
        return launch_kernel(batched_kernel<float>, dim3(grid), dim3(256), BShape<float>::smem, s,
                             descs, count, counter);
    return launch_kernel(batched_kernel<double>, dim3(grid), dim3(256), BShape<double>::smem, s,
                         descs, count, counter);
}

}  // namespace trx

// Block leaf TRSM: one leaf of up to 256 rows (Section 3.1's base case with a
// larger cutoff) over many right-hand sides, in one launch.
//
// The recursion's bottom levels are many short dependent launches (64-row
// leaves and 64..256-row GEMM updates), each bounded by launch and memory
// latency rather than work. A 256-row leaf replaces three of those levels: a
// CTA takes 32 right-hand sides, stages their 256 rows in shared memory once
// and runs the forward substitution there in 16-row bands:
//   1. warp 0 solves the band's 16x16 diagonal block, one lane per column
//      (16 values in registers, no communication);
//   2. all eight warps update the rows below the band with it, a rank-16
//      update: lane = column, warp w takes every 8th row; the band's 16
//      solved values sit in each lane's registers and the 16 entries of M for
//      a row come from shared memory as four 16-byte broadcasts.
// The band of M (rows below it x 16 columns) is staged row-major in shared
// memory, the next band's global loads in flight during the current update.
// The solved panel is written back (and, on the tensor-core path, split into
// the BF16 Y planes the later GEMM updates read).
#pragma once
#include <type_traits>

#include "common.cuh"
#include "leaf_impl.cuh"

namespace trx {
namespace {

template <typename T>
struct B256 {
    static constexpr int KB = 256;          // largest leaf
    static constexpr int NT = 256;          // 8 warps
    static constexpr int NC = 32;           // right-hand sides per CTA (one per lane)
    static constexpr int SB = 16;           // band height
    static constexpr int LDP = NC + 1;      // panel row stride (column = lane: conflict-free)
    static constexpr int LDB = SB + 4;      // band row stride (16-byte aligned rows)
    static constexpr size_t smem = sizeof(T) * ((size_t)KB * LDP + 2 * (size_t)KB * LDB + KB);
};

template <typename T>
__global__ void __launch_bounds__(256) leaf_trsm_b256_kernel(LeafArgs<T> a) {
    using S = B256<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sB = reinterpret_cast<T*>(smem_raw);               // 2 bands: M(r0+i, r0+s0+kk) at i*LDB + kk
    T* sP = sB + 2 * S::KB * S::LDB;                        // panel: C(r0+i, j0+c) at i*LDP + c
    T* sD = sP + S::KB * S::LDP;                            // reciprocal diagonal
    pdl_trigger();
    pdl_wait();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Canon<T>& p = a.p;
    const int64_t r0 = a.r0;
    const int kb = (int)(p.k - r0 < a.b ? p.k - r0 : a.b);
    if (kb <= 0) return;
    const int64_t j0 = (int64_t)blockIdx.x * S::NC;
    const bool col_ok = j0 + lane < p.nrhs;

    // Band loader: rows [s0, kb) x columns [s0, s0+16) of the leaf's M into
    // band buffer `buf`, coalesced along A's contiguous index.
    const bool a_row_fast = (p.a_rs == 1 || p.a_rs == -1);
    auto load_band = [&](int s0, int buf) {
        T* dst = sB + buf * S::KB * S::LDB;
        const int rows = kb - s0;
        if (a_row_fast) {                    // 16 columns of contiguous rows
#pragma unroll 4
            for (int e = tid; e < rows * S::SB; e += S::NT) {
                const int i = e % rows, kk = e / rows;
                const int gi = s0 + i, gl = s0 + kk;
                dst[i * S::LDB + kk] = (gl < gi && gl < kb)
                    ? p.A[(r0 + gi) * p.a_rs + (r0 + gl) * p.a_cs] : T(0);
            }
        } else {                             // rows of 16 contiguous entries
#pragma unroll 4
            for (int e = tid; e < rows * S::SB; e += S::NT) {
                const int kk = e % S::SB, i = e / S::SB;
                const int gi = s0 + i, gl = s0 + kk;
                dst[i * S::LDB + kk] = (gl < gi && gl < kb)
                    ? p.A[(r0 + gi) * p.a_rs + (r0 + gl) * p.a_cs] : T(0);
            }
        }
    };

    // Stage the panel (alpha applied) and the reciprocal diagonal.
    {
        const bool c_row_fast = (p.c_rs == 1 || p.c_rs == -1);
        if (c_row_fast) {
#pragma unroll 8
            for (int e = tid; e < kb * S::NC; e += S::NT) {
                const int i = e % kb, c = e / kb;
                T v = T(0);
                if (j0 + c < p.nrhs) v = a.alpha * p.C[(r0 + i) * p.c_rs + (j0 + c) * p.c_cs];
                sP[i * S::LDP + c] = v;
            }
        } else {
#pragma unroll 8
            for (int e = tid; e < kb * S::NC; e += S::NT) {
                const int c = e % S::NC, i = e / S::NC;
                T v = T(0);
                if (j0 + c < p.nrhs) v = a.alpha * p.C[(r0 + i) * p.c_rs + (j0 + c) * p.c_cs];
                sP[i * S::LDP + c] = v;
            }
        }
        for (int i = tid; i < kb; i += S::NT)
            sD[i] = p.unit ? T(1) : T(1) / p.A[(r0 + i) * (p.a_rs + p.a_cs)];
    }
    load_band(0, 0);
    __syncthreads();

    const int nb = (kb + S::SB - 1) / S::SB;
#pragma unroll 1
    for (int bi = 0; bi < nb; ++bi) {
        const int s0 = bi * S::SB;
        const int sbn = kb - s0 < S::SB ? kb - s0 : S::SB;
        const T* band = sB + (bi & 1) * S::KB * S::LDB;   // row i (relative to s0) at i*LDB
        // 1. warp 0: substitution on the band's diagonal block
        if (warp == 0) {
            T x[S::SB];
#pragma unroll
            for (int q = 0; q < S::SB; ++q) x[q] = q < sbn ? sP[(s0 + q) * S::LDP + lane] : T(0);
#pragma unroll
            for (int jj = 0; jj < S::SB; ++jj) {
                x[jj] *= (jj < sbn) ? sD[s0 + jj] : T(1);
#pragma unroll
                for (int q = jj + 1; q < S::SB; ++q) x[q] = fma(-band[q * S::LDB + jj], x[jj], x[q]);
            }
#pragma unroll
            for (int q = 0; q < S::SB; ++q)
                if (q < sbn) sP[(s0 + q) * S::LDP + lane] = x[q];
        } else if (bi + 1 < nb) {
            // warps 1..7 fetch the next band meanwhile
            const int s1 = s0 + S::SB;
            T* dst = sB + ((bi + 1) & 1) * S::KB * S::LDB;
            const int rows = kb - s1;
            const int t7 = tid - 32;
#pragma unroll 4
            for (int e = t7; e < rows * S::SB; e += S::NT - 32) {
                int i, kk;
                if (a_row_fast) { i = e % rows; kk = e / rows; } else { kk = e % S::SB; i = e / S::SB; }
                const int gi = s1 + i, gl = s1 + kk;
                dst[i * S::LDB + kk] = (gl < gi && gl < kb)
                    ? p.A[(r0 + gi) * p.a_rs + (r0 + gl) * p.a_cs] : T(0);
            }
        }
        __syncthreads();
        // 2. rank-16 update of the rows below the band: lane = column
        if (s0 + S::SB < kb) {
            T xb[S::SB];
#pragma unroll
            for (int kk = 0; kk < S::SB; ++kk) xb[kk] = sP[(s0 + kk) * S::LDP + lane];
            for (int i = s0 + S::SB + warp; i < kb; i += 8) {
                const T* trow = band + (i - s0) * S::LDB;
                T acc0 = T(0), acc1 = T(0);
#pragma unroll
                for (int kk = 0; kk < S::SB; kk += Vec<T>::n) {
                    T t[Vec<T>::n];
                    vload(trow + kk, t);
#pragma unroll
                    for (int e = 0; e < Vec<T>::n; e += 2) {
                        acc0 = fma(t[e], xb[kk + e], acc0);
                        acc1 = fma(t[e + 1], xb[kk + e + 1], acc1);
                    }
                }
                sP[i * S::LDP + lane] -= acc0 + acc1;
            }
        }
        __syncthreads();
    }

    // Write back, and the Y planes on the tensor-core path.
    {
        const bool c_row_fast = (p.c_rs == 1 || p.c_rs == -1);
        if (c_row_fast) {
            for (int e = tid; e < kb * S::NC; e += S::NT) {
                const int i = e % kb, c = e / kb;
                if (j0 + c < p.nrhs) p.C[(r0 + i) * p.c_rs + (j0 + c) * p.c_cs] = sP[i * S::LDP + c];
            }
        } else {
            for (int e = tid; e < kb * S::NC; e += S::NT) {
                const int c = e % S::NC, i = e / S::NC;
                if (j0 + c < p.nrhs) p.C[(r0 + i) * p.c_rs + (j0 + c) * p.c_cs] = sP[i * S::LDP + c];
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (a.planes) {
                for (int e = tid; e < kb * S::NC; e += S::NT) {
                    const int i = e % kb, c = e / kb;
                    if (j0 + c < p.nrhs) {
                        put_y(a.pl, (j0 + c) * a.pl.ldy + r0 + i, sP[i * S::LDP + c]);
                    }
                }
            }
        }
    }
    (void)col_ok;
}

}  // namespace

template <typename T>
cudaError_t leaf_b256_configure() {
    return cudaFuncSetAttribute(leaf_trsm_b256_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)B256<T>::smem);
}

template <typename T>
cudaError_t leaf_b256_launch(const LeafArgs<T>& a, cudaStream_t s) {
    const int64_t nx = (a.p.nrhs + B256<T>::NC - 1) / B256<T>::NC;
    return launch_kernel(leaf_trsm_b256_kernel<T>, dim3((unsigned)nx), dim3(256), B256<T>::smem, s,
                         a);
}

}  // namespace trx

// Blocked leaf TRSM (Section 3.3 base kernel), for leaves of 64 or 128 rows
// with many right-hand sides.
//
// The plain substitution sweep of leaf_impl.cuh carries a serial chain of b
// steps per column with one shared-memory load per FMA; at b = 64 it is
// latency-bound. Here the leaf's rows are taken 16 at a time:
//   1. substitution on the 16-row diagonal block: one thread per column,
//      16 rows in registers, no communication (the triangle and the
//      reciprocal diagonal are broadcast from shared memory);
//   2. rank-16 update of every row below the block,
//        C[below, :] -= M[below, block] * X[block, :],
//      as a register-tiled outer product: each thread owns a few rows x four
//      columns and reads the solved rows as 16-byte vectors.
// About three quarters of the leaf's multiply-adds land in step 2, which runs
// at the FMA pipe's rate; step 1's chain is 16 steps, not b. The result is the
// forward substitution of the leaf with its sum split in 16-row blocks.
//
// A CTA holds the triangle once and walks NCOL-column panels of the
// right-hand side (persistent); each panel is staged row-major in shared
// memory with coalesced global loads.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "leaf_impl.cuh"

namespace trx {
namespace {

template <typename T, int B>
struct BlkShape {
    static constexpr int NT = 256;
    static constexpr int SB = 16;              // sub-block rows
    static constexpr int NCOL = 64;            // right-hand sides per panel
    static constexpr int LDC = NCOL + 4;       // row stride of the panel in smem
    static constexpr int CG = NCOL / 4;        // column groups of four (16)
    static constexpr int RG = NT / CG;         // row groups (16)
    static constexpr size_t smem = sizeof(T) * (size_t)(B * B + B + B * LDC);
    static_assert(NCOL <= NT, "one thread per column in the substitution");
};

template <typename T, int B>
__global__ void __launch_bounds__(256, B == 64 ? 2 : 1) leaf_trsm_blocked_kernel(LeafArgs<T> a) {
    using S = BlkShape<T, B>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sT = reinterpret_cast<T*>(smem_raw);   // M(r0+i, r0+l) at l*B + i (i > l, else 0)
    T* sD = sT + B * B;                        // reciprocal diagonal (1 if unit / ragged)
    T* sC = sD + B;                            // panel: C(r0+i, j0+c) at i*LDC + c
    pdl_trigger();
    pdl_wait();
    const int tid = threadIdx.x;
    const Canon<T>& p = a.p;
    const int64_t r0 = a.r0;
    const int64_t rem = p.k - r0;
    if (rem <= 0) return;
    const int bs = rem < a.b ? (int)rem : a.b;

    // Panel staging map: each thread keeps the index that is contiguous in C
    // (`fi`) and walks the other (`w = wi + u*adv`, u < PL) with a pointer.
    const bool c_row_fast = (p.c_rs == 1 || p.c_rs == -1);
    constexpr int PL = B * S::NCOL / S::NT;
    const int fmod = c_row_fast ? B : S::NCOL;
    const int fi = tid % fmod, wi = tid / fmod, adv = S::NT / fmod;
    const int64_t st_walk = c_row_fast ? p.c_cs : p.c_rs;
    const int64_t npanels = (p.nrhs + S::NCOL - 1) / S::NCOL;
    auto panel_base = [&](int64_t j0) {
        return p.C + (c_row_fast ? (r0 + fi) * p.c_rs + (j0 + wi) * p.c_cs
                                 : (r0 + wi) * p.c_rs + (j0 + fi) * p.c_cs);
    };
    auto load_panel = [&](int64_t j0, T (&v)[PL]) {
        const T* src = panel_base(j0);
#pragma unroll
        for (int u = 0; u < PL; ++u) {
            const int w = wi + u * adv;
            const int i = c_row_fast ? fi : w, c = c_row_fast ? w : fi;
            v[u] = (i < bs && j0 + c < p.nrhs) ? a.alpha * *src : T(0);
            src += adv * st_walk;
        }
    };
    // The first panel's loads go out before the triangle's, so the two
    // global-memory latencies overlap.
    T pre[PL];
    int64_t panel = blockIdx.x;
    if (panel < npanels) load_panel(panel * S::NCOL, pre);

    // Triangle, read along A's contiguous index (one fixed index per thread).
    {
        const bool a_row_fast = (p.a_rs == 1 || p.a_rs == -1);
        constexpr int ADV = S::NT / B;
        constexpr int TP = B / ADV;
        const int fixed = tid % B, first = tid / B;
        const int64_t st_fixed = a_row_fast ? p.a_rs : p.a_cs;
        const int64_t st_walk_a = a_row_fast ? p.a_cs : p.a_rs;
        const T* src = p.A + (r0 + fixed) * st_fixed + (r0 + first) * st_walk_a;
#pragma unroll 8
        for (int u = 0; u < TP; ++u) {
            const int w = first + u * ADV;
            const int i = a_row_fast ? fixed : w, l = a_row_fast ? w : fixed;
            sT[l * B + i] = (i < bs && l < i) ? *src : T(0);
            src += ADV * st_walk_a;
        }
        for (int i = tid; i < B; i += S::NT) {
            T d = T(1);
            if (i < bs && !p.unit) d = T(1) / p.A[(r0 + i) * (p.a_rs + p.a_cs)];
            sD[i] = d;
        }
    }

    // update-phase tile: row group rg (rows rg, rg+RG, ...), columns 4*cg..4*cg+3
    const int cg = tid % S::CG, rg = tid / S::CG;
#pragma unroll 1
    for (; panel < npanels; panel += gridDim.x) {
        const int64_t j0 = panel * S::NCOL;
#pragma unroll
        for (int u = 0; u < PL; ++u) {
            const int w = wi + u * adv;
            const int i = c_row_fast ? fi : w, c = c_row_fast ? w : fi;
            sC[i * S::LDC + c] = pre[u];
        }
        __syncthreads();
        // next panel's loads in flight during this panel's sweep
        if (panel + gridDim.x < npanels) load_panel((panel + gridDim.x) * S::NCOL, pre);
#pragma unroll
        for (int s0 = 0; s0 < B; s0 += S::SB) {
            // 1. substitution on rows s0 .. s0+15, one thread per column
            if (tid < S::NCOL) {
                T x[S::SB];
#pragma unroll
                for (int q = 0; q < S::SB; ++q) x[q] = sC[(s0 + q) * S::LDC + tid];
#pragma unroll
                for (int jj = 0; jj < S::SB; ++jj) {
                    x[jj] *= sD[s0 + jj];
#pragma unroll
                    for (int q = jj + 1; q < S::SB; ++q)
                        x[q] = fma(-sT[(s0 + jj) * B + s0 + q], x[jj], x[q]);
                }
#pragma unroll
                for (int q = 0; q < S::SB; ++q) sC[(s0 + q) * S::LDC + tid] = x[q];
            }
            __syncthreads();
            // 2. rank-16 update of rows below the block
            constexpr int ROWS = B - 16;             // upper bound over s0
            if (s0 + S::SB < B) {
                constexpr int TRMAX = (ROWS + S::RG - 1) / S::RG;
                T acc[TRMAX][4];
#pragma unroll
                for (int u = 0; u < TRMAX; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
#pragma unroll
                for (int kk = 0; kk < S::SB; ++kk) {
                    const int l = s0 + kk;
                    T xv[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) xv[v] = sC[l * S::LDC + 4 * cg + v];
#pragma unroll
                    for (int u = 0; u < TRMAX; ++u) {
                        const int i = s0 + S::SB + rg + u * S::RG;
                        if (i < B) {
                            const T t = sT[l * B + i];
#pragma unroll
                            for (int v = 0; v < 4; ++v) acc[u][v] = fma(t, xv[v], acc[u][v]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < TRMAX; ++u) {
                    const int i = s0 + S::SB + rg + u * S::RG;
                    if (i < B) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) sC[i * S::LDC + 4 * cg + v] -= acc[u][v];
                    }
                }
            }
            __syncthreads();
        }
        // write back (and the Y planes on the tensor-core path)
        {
            T* dst = panel_base(j0);
#pragma unroll
            for (int u = 0; u < PL; ++u) {
                const int w = wi + u * adv;
                const int i = c_row_fast ? fi : w, c = c_row_fast ? w : fi;
                if (i < bs && j0 + c < p.nrhs) *dst = sC[i * S::LDC + c];
                dst += adv * st_walk;
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (a.planes) {
                const int pi = tid % B, pc = tid / B;
                constexpr int PADV = S::NT / B;
#pragma unroll
                for (int c = pc; c < S::NCOL; c += PADV) {
                    if (pi < bs && j0 + c < p.nrhs) {
                        put_y(a.pl, (j0 + c) * a.pl.ldy + r0 + pi, sC[pi * S::LDC + c]);
                    }
                }
            }
        }
        __syncthreads();   // sC is refilled by the next panel
    }
}

}  // namespace

template <typename T>
cudaError_t leaf_blocked_configure() {
    cudaError_t e = cudaFuncSetAttribute(leaf_trsm_blocked_kernel<T, 64>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BlkShape<T, 64>::smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(leaf_trsm_blocked_kernel<T, 128>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)BlkShape<T, 128>::smem);
}

// One leaf (a.r0, a.b rows, a.b <= 128), persistent CTAs over the panels.
template <typename T>
cudaError_t leaf_blocked_launch(const LeafArgs<T>& a, int64_t max_ctas, cudaStream_t s) {
    const int64_t npanels = (a.p.nrhs + 63) / 64;
    const int64_t nx = npanels < max_ctas ? npanels : max_ctas;
    if (a.b <= 64)
        return launch_kernel(leaf_trsm_blocked_kernel<T, 64>, dim3((unsigned)nx), dim3(256),
                             BlkShape<T, 64>::smem, s, a);
    return launch_kernel(leaf_trsm_blocked_kernel<T, 128>, dim3((unsigned)nx), dim3(256),
                         BlkShape<T, 128>::smem, s, a);
}

}  // namespace trx

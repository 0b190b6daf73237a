// Wide TRSM leaf (Section 3.1's base case at a 128-row cutoff), FP32, for
// leaves with many right-hand sides.
//
// At the bottom of the recursion each 128-row node is two 64-row leaves and
// one 64x64 GEMM update between them: three dependent launches, each bounded
// by launch and memory latency rather than work. This kernel solves the whole
// 128-row leaf in one launch, by forward substitution in 16-row blocks:
//   1. the 16 rows of block s are solved by one warp, lane = column, the
//      16 values of each column in registers (no communication);
//   2. every row below the block takes the rank-16 update
//        C[i, :] -= sum_{l in block s} M(i, l) X(l, :).
// The sum for a row is split in 16-row pieces and accumulated in that order;
// the result is the substitution of the leaf.
//
// Layout: a CTA holds the leaf's triangle once in shared memory (column l
// of M contiguous over i) and runs four independent groups of 128 threads.
// A group solves one 32-column panel at a time: thread (rg, cg) owns rows
// 8rg..8rg+7 x columns 4cg..4cg+3 of the panel and keeps that tile in
// registers across all eight blocks, so the rank-16 updates never touch
// shared memory for C; a row block's owners publish it to the group's panel
// buffer just before its substitution, and the solved rows stay there for
// the updates and the write-back. Groups synchronise with their own named
// barriers, so one group's substitution overlaps the others' updates.
//
// A warp owns a 32-row chunk; the bottom chunk updates in seven of the eight
// blocks, the top one in one. The chunk-to-warp map is rotated by the group
// index, so each of the SM's four warp schedulers (warp w runs on w % 4)
// holds one warp of every chunk, and the top chunk's warp, idle after the
// second block, runs the substitutions.
#include <type_traits>

#include "common.cuh"
#include "leaf_impl.cuh"

namespace trx {
namespace {

struct Wide {
    static constexpr int B = 128;                 // leaf rows
    static constexpr int SB = 16;                 // substitution block
    static constexpr int GROUPS = 4;              // independent column groups per CTA
    static constexpr int GT = 128;                // threads per group
    static constexpr int NT = GROUPS * GT;
    static constexpr int NC = 32;                 // columns per panel
    static constexpr int LDC = NC + 4;            // panel row stride (16-byte rows)
    static constexpr size_t smem = sizeof(float) * ((size_t)B * B + B + (size_t)GROUPS * B * LDC);
};

// Packed FP32 pairs (Blackwell's f32x2 FMA: two independent
// round-to-nearest FMAs per instruction).
__device__ __forceinline__ uint64_t pack2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(uint64_t r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(Wide::GT) : "memory");
}

// ROWS: C's rows are contiguous (side L); one layout per instance keeps the
// kernel's code small (instruction fetch was its largest stall).
template <bool ROWS>
__global__ void __launch_bounds__(Wide::NT, 1) leaf_trsm_wide_kernel(LeafArgs<float> a,
                                                                   int64_t npanels) {
    using S = Wide;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sT = reinterpret_cast<float*>(smem_raw);   // M(r0+i, r0+l) at l*B + i (i > l, else 0)
    float* sD = sT + S::B * S::B;                       // reciprocal diagonal (1: unit / ragged)
    const int tid = threadIdx.x, g = tid / S::GT, gt = tid % S::GT;
    float* sC = sD + S::B + (size_t)g * S::B * S::LDC;  // this group's panel: row i at i*LDC
    pdl_trigger();
    pdl_wait();
    const Canon<float>& p = a.p;
    const int64_t r0 = a.r0;
    const int64_t rem = p.k - r0;
    if (rem <= 0) return;
    const int bs = rem < a.b ? (int)rem : a.b;
    const int nblk = (bs + S::SB - 1) / S::SB;

    // Panel staging (alpha * C, zeros outside the leaf): thread = row when
    // C's rows are contiguous, else thread = column.
    constexpr bool c_row_fast = ROWS;
    auto load_panel = [&](int64_t j0, float (&v)[S::NC]) {
        const int ncols = (int)(p.nrhs - j0 < S::NC ? p.nrhs - j0 : S::NC);
        if constexpr (c_row_fast) {
            const int i = gt;
            const float* src = p.C + (r0 + i) * p.c_rs + j0 * p.c_cs;
#pragma unroll
            for (int c = 0; c < S::NC; ++c)
                v[c] = (i < bs && c < ncols) ? a.alpha * src[(int64_t)c * p.c_cs] : 0.f;
        } else {
            const int c = gt & 31, i0 = gt >> 5;
#pragma unroll
            for (int u = 0; u < S::NC; ++u) {
                const int i = i0 + 4 * u;
                v[u] = (i < bs && c < ncols) ? a.alpha * p.C[(r0 + i) * p.c_rs + (j0 + c) * p.c_cs]
                                             : 0.f;
            }
        }
    };
    auto store_panel = [&](const float (&v)[S::NC]) {
        if constexpr (c_row_fast) {
#pragma unroll
            for (int c4 = 0; c4 < S::NC / 4; ++c4)
                *reinterpret_cast<float4*>(sC + gt * S::LDC + 4 * c4) =
                    make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
        } else {
            const int c = gt & 31, i0 = gt >> 5;
#pragma unroll
            for (int u = 0; u < S::NC; ++u) sC[(i0 + 4 * u) * S::LDC + c] = v[u];
        }
    };
    // The first panel's loads go out before the triangle's, so the two
    // memory latencies overlap.
    float pre[S::NC];
    int64_t panel = blockIdx.x + (int64_t)gridDim.x * g;
    const int64_t pstride = (int64_t)gridDim.x * S::GROUPS;
    if (panel < npanels) load_panel(panel * S::NC, pre);

    // Triangle, read along A's contiguous index.
    {
        const bool a_row_fast = (p.a_rs == 1 || p.a_rs == -1);
        constexpr int ADV = S::NT / S::B;          // 4
        constexpr int TP = S::B / ADV;             // 32
        const int fixed = tid % S::B, first = tid / S::B;
        const int64_t st_fixed = a_row_fast ? p.a_rs : p.a_cs;
        const int64_t st_walk = a_row_fast ? p.a_cs : p.a_rs;
        const float* src = p.A + (r0 + fixed) * st_fixed + (r0 + first) * st_walk;
#pragma unroll 8
        for (int u = 0; u < TP; ++u) {
            const int w = first + u * ADV;
            const int i = a_row_fast ? fixed : w, l = a_row_fast ? w : fixed;
            sT[l * S::B + i] = (i < bs && l < i) ? *src : 0.f;
            src += ADV * st_walk;
        }
        for (int i = tid; i < S::B; i += S::NT)
            sD[i] = (i < bs && !p.unit) ? 1.f / p.A[(r0 + i) * (p.a_rs + p.a_cs)] : 1.f;
    }
    __syncthreads();

    const int lane = gt & 31;
    const int chunk = ((gt >> 5) + g) & 3;           // rows 32*chunk .. of the panel
    const int rg = 4 * chunk + (lane >> 3), cg = lane & 7;   // tile rows 8rg.., columns 4cg..
    const bool subst_warp = chunk == 0;
#pragma unroll 1
    for (bool first = true; panel < npanels; panel += pstride, first = false) {
        const int64_t j0 = panel * S::NC;
        const int ncols = (int)(p.nrhs - j0 < S::NC ? p.nrhs - j0 : S::NC);
        if (!first) load_panel(j0, pre);
        store_panel(pre);
        group_sync(g);
        // The tile is kept negated, as pairs of rows (2u, 2u+1) per column v:
        // y = -x, so each update y += M(i,l) X(l,:) is a plain packed FMA
        // (and rounds exactly as x - M(i,l) X(l,:) would).
        uint64_t y[4][4];
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
            const float4 w0 = *reinterpret_cast<const float4*>(sC + (8 * rg + 2 * u2) * S::LDC + 4 * cg);
            const float4 w1 = *reinterpret_cast<const float4*>(sC + (8 * rg + 2 * u2 + 1) * S::LDC + 4 * cg);
            y[u2][0] = pack2(-w0.x, -w1.x);
            y[u2][1] = pack2(-w0.y, -w1.y);
            y[u2][2] = pack2(-w0.z, -w1.z);
            y[u2][3] = pack2(-w0.w, -w1.w);
        }

#pragma unroll 1
        for (int s = 0; s < nblk; ++s) {
            const int s0 = s * S::SB;
            // 1. the block's owners publish their (fully updated) rows
            if ((rg >> 1) == s) {
#pragma unroll
                for (int u2 = 0; u2 < 4; ++u2) {
                    float a[4], b[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) unpack2(y[u2][v], a[v], b[v]);
                    *reinterpret_cast<float4*>(sC + (8 * rg + 2 * u2) * S::LDC + 4 * cg) =
                        make_float4(-a[0], -a[1], -a[2], -a[3]);
                    *reinterpret_cast<float4*>(sC + (8 * rg + 2 * u2 + 1) * S::LDC + 4 * cg) =
                        make_float4(-b[0], -b[1], -b[2], -b[3]);
                }
            }
            group_sync(g);
            // 2. substitution on the 16x16 diagonal block, lane = column;
            //    column jj+1 of the block's M is loaded (four 16-byte
            //    broadcasts) while column jj is applied
            if (subst_warp) {
                float y[S::SB];
#pragma unroll
                for (int q = 0; q < S::SB; ++q) y[q] = sC[(s0 + q) * S::LDC + lane];
                const float* mcol = sT + s0 * S::B + s0;      // M(s0+q, s0+jj) at jj*B + q
                float4 cur[4], nxt[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) cur[v] = *reinterpret_cast<const float4*>(mcol + 4 * v);
#pragma unroll
                for (int jj = 0; jj < S::SB; ++jj) {
                    if (jj + 1 < S::SB) {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            nxt[v] = *reinterpret_cast<const float4*>(mcol + (jj + 1) * S::B + 4 * v);
                    }
                    const float m[16] = {cur[0].x, cur[0].y, cur[0].z, cur[0].w,
                                         cur[1].x, cur[1].y, cur[1].z, cur[1].w,
                                         cur[2].x, cur[2].y, cur[2].z, cur[2].w,
                                         cur[3].x, cur[3].y, cur[3].z, cur[3].w};
                    y[jj] *= sD[s0 + jj];
#pragma unroll
                    for (int q = jj + 1; q < S::SB; ++q) y[q] = fmaf(-m[q], y[jj], y[q]);
#pragma unroll
                    for (int v = 0; v < 4; ++v) cur[v] = nxt[v];
                }
#pragma unroll
                for (int q = 0; q < S::SB; ++q) sC[(s0 + q) * S::LDC + lane] = y[q];
            }
            group_sync(g);
            // 3. rank-16 update of the owned rows below the block
            if (rg >= 2 * s + 2) {
#pragma unroll 4
                for (int kk = 0; kk < S::SB; ++kk) {
                    const int l = s0 + kk;
                    const float4 xv = *reinterpret_cast<const float4*>(sC + l * S::LDC + 4 * cg);
                    const float4 t0 = *reinterpret_cast<const float4*>(sT + l * S::B + 8 * rg);
                    const float4 t1 = *reinterpret_cast<const float4*>(sT + l * S::B + 8 * rg + 4);
                    const uint64_t tp[4] = {pack2(t0.x, t0.y), pack2(t0.z, t0.w),
                                            pack2(t1.x, t1.y), pack2(t1.z, t1.w)};
                    const uint64_t xb[4] = {pack2(xv.x, xv.x), pack2(xv.y, xv.y),
                                            pack2(xv.z, xv.z), pack2(xv.w, xv.w)};
#pragma unroll
                    for (int u2 = 0; u2 < 4; ++u2)
#pragma unroll
                        for (int v = 0; v < 4; ++v) y[u2][v] = ffma2(tp[u2], xb[v], y[u2][v]);
                }
            }
        }

        // Write back (and the Y planes on the tensor-core path). The last
        // barrier above follows the last substitution, so every row is final.
        if constexpr (c_row_fast) {
            const int i = gt;
            if (i < bs) {
                float* dst = p.C + (r0 + i) * p.c_rs + j0 * p.c_cs;
#pragma unroll
                for (int c4 = 0; c4 < S::NC / 4; ++c4) {
                    const float4 w = *reinterpret_cast<const float4*>(sC + i * S::LDC + 4 * c4);
                    const float v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 4 * c4 + e;
                        if (c < ncols) {
                            dst[(int64_t)c * p.c_cs] = v[e];
                            if (a.planes) put_y(a.pl, (j0 + c) * a.pl.ldy + r0 + i, v[e]);
                        }
                    }
                }
            }
        } else {
            const int c = gt & 31, i0 = gt >> 5;
            if (c < ncols) {
#pragma unroll 4
                for (int u = 0; u < S::B / 4; ++u) {
                    const int i = i0 + 4 * u;
                    if (i < bs) p.C[(r0 + i) * p.c_rs + (j0 + c) * p.c_cs] = sC[i * S::LDC + c];
                }
            }
            if (a.planes) {
                const int i = gt;
                if (i < bs) {
                    for (int c2 = 0; c2 < ncols; ++c2) {
                        put_y(a.pl, (j0 + c2) * a.pl.ldy + r0 + i, sC[i * S::LDC + c2]);
                    }
                }
            }
        }
        group_sync(g);   // the panel buffer is refilled by the next panel
    }
}

}  // namespace

cudaError_t leaf_wide_configure() {
    const cudaError_t e = cudaFuncSetAttribute(leaf_trsm_wide_kernel<true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)Wide::smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(leaf_trsm_wide_kernel<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Wide::smem);
}

// One FP32 TRSM leaf of up to 128 rows (a.r0, a.b), one CTA per SM at most,
// 32-column panels dealt round-robin over the CTAs' four groups.
cudaError_t leaf_wide_launch(const LeafArgs<float>& a, int num_sms, cudaStream_t s) {
    if (a.b < 1 || a.b > Wide::B) return cudaErrorInvalidValue;
    const int64_t npanels = (a.p.nrhs + Wide::NC - 1) / Wide::NC;
    const int64_t sms = num_sms > 0 ? num_sms : 1;
    const int64_t grid = npanels < sms ? npanels : sms;
    const bool rows = a.p.c_rs == 1 || a.p.c_rs == -1;
    return launch_kernel(rows ? leaf_trsm_wide_kernel<true> : leaf_trsm_wide_kernel<false>,
                         dim3((unsigned)grid), dim3(Wide::NT), Wide::smem, s,
                         a, npanels);
}

}  // namespace trx

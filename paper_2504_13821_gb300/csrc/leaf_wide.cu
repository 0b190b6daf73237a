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
// registers across the blocks, so the rank-16 updates never touch shared
// memory for C. Groups synchronise with their own named barriers.
//
// Schedule of a panel: one group barrier per block step. After the barrier
// that makes X_s visible, the substitution warp (the one owning rows 0..31,
// which has no update of its own after the first block) takes block s+1's
// rows from the panel buffer, applies their last update (by X_s) itself and
// solves them, while the other warps apply X_s to the rows further down;
// the owners of block s+2 then publish their rows, which lack only the
// update by X_s+1. So the substitution overlaps the updates instead of
// following them. Every row still takes its updates in block order with the
// same FMAs (the owners keep their tile negated, y = -x, so y += M X rounds
// exactly as x - M X), and the result is bitwise that of solving block after
// block.
//
// Staging: the triangle and the panel arrive by cp.async (one memory round
// trip, no registers held); alpha is applied where the panel is first read.
// Write-back: a lane stores 8 rows x 4 columns of the panel, each column's
// 8 rows as 16-byte vectors of C and of every Y plane (packed BF16
// conversions), where the addresses line up; else one element per lane.
//
// The chunk-to-warp map is rotated by the group index, so each of the SM's
// four warp schedulers (warp w runs on w % 4) holds one warp of every chunk,
// and the four groups' substitution warps sit on different schedulers.
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

// One float global -> shared without registers; invalid: the word is zeroed
// (src-size 0, nothing read).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}
// Two floats to BF16 (round to nearest even, as __float2bfloat16_rn), a in
// the high half; and the halves back to float (exact).
__device__ __forceinline__ uint32_t bf16x2(float a, float b) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }

// The slices (put_split's) of 8 consecutive rows of one Y-plane column,
// stored as one 16-byte vector per plane at element offset o.
__device__ __forceinline__ void put_y8(const Planes& pl, int64_t o, const float (&v)[8]) {
    uint32_t h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = bf16x2(v[2 * e + 1], v[2 * e]);
    *reinterpret_cast<uint4*>(pl.y_hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
    if (pl.slices < 2) return;
    float r[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        r[2 * e] = v[2 * e] - bf_lo(h[e]);
        r[2 * e + 1] = v[2 * e + 1] - bf_hi(h[e]);
    }
    uint32_t l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) l[e] = bf16x2(r[2 * e + 1], r[2 * e]);
    *reinterpret_cast<uint4*>(pl.y_lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
    if (pl.slices < 3) return;
#pragma unroll
    for (int e = 0; e < 4; ++e) l[e] = bf16x2(r[2 * e + 1] - bf_hi(l[e]), r[2 * e] - bf_lo(l[e]));
    *reinterpret_cast<uint4*>(pl.y_lo2 + o) = make_uint4(l[0], l[1], l[2], l[3]);
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
    const float alpha = a.alpha;

    // Panel staging: C itself (alpha is applied where it is first read),
    // zeros outside the leaf; thread = row when C's rows are contiguous,
    // else thread = column.
    auto fetch_panel = [&](int64_t j0) {
        const int ncols = (int)(p.nrhs - j0 < S::NC ? p.nrhs - j0 : S::NC);
        if constexpr (ROWS) {
            const int i = gt;
            const float* src = p.C + (r0 + i) * p.c_rs + j0 * p.c_cs;
#pragma unroll
            for (int c = 0; c < S::NC; ++c) {
                const bool in = i < bs && c < ncols;
                cp_async4(sC + i * S::LDC + c, in ? src + (int64_t)c * p.c_cs : p.C, in);
            }
        } else {
            const int c = gt & 31, i0 = gt >> 5;
#pragma unroll
            for (int u = 0; u < S::NC; ++u) {
                const int i = i0 + 4 * u;
                const bool in = i < bs && c < ncols;
                cp_async4(sC + i * S::LDC + c,
                          in ? p.C + (r0 + i) * p.c_rs + (j0 + c) * p.c_cs : p.C, in);
            }
        }
    };
    int64_t panel = blockIdx.x + (int64_t)gridDim.x * g;
    const int64_t pstride = (int64_t)gridDim.x * S::GROUPS;
    if (panel < npanels) fetch_panel(panel * S::NC);

    // Triangle, read along A's contiguous index; its copies are in flight
    // together with the first panel's.
    {
        const bool a_row_fast = (p.a_rs == 1 || p.a_rs == -1);
        constexpr int ADV = S::NT / S::B;          // 4
        constexpr int TP = S::B / ADV;             // 32
        const int fixed = tid % S::B, first = tid / S::B;
        const int64_t st_fixed = a_row_fast ? p.a_rs : p.a_cs;
        const int64_t st_walk = a_row_fast ? p.a_cs : p.a_rs;
        const float* src = p.A + (r0 + fixed) * st_fixed + (r0 + first) * st_walk;
#pragma unroll
        for (int u = 0; u < TP; ++u) {
            const int w = first + u * ADV;
            const int i = a_row_fast ? fixed : w, l = a_row_fast ? w : fixed;
            const bool in = i < bs && l < i;
            cp_async4(sT + l * S::B + i, in ? src + (int64_t)u * ADV * st_walk : p.A, in);
        }
        if (tid < S::B)
            sD[tid] = (tid < bs && !p.unit) ? 1.f / p.A[(r0 + tid) * (p.a_rs + p.a_cs)] : 1.f;
        cp_async_wait_all();
    }
    __syncthreads();

    const int lane = gt & 31;
    const int chunk = ((gt >> 5) + g) & 3;           // rows 32*chunk .. of the panel
    const int rg = 4 * chunk + (lane >> 3), cg = lane & 7;   // tile rows 8rg.., columns 4cg..
    const bool subst_warp = chunk == 0;

    // Substitution on the 16x16 diagonal block at s0 for this lane's column,
    // in place; column jj+1 of the block's M is loaded (four 16-byte
    // broadcasts) while column jj is applied.
    auto solve_block = [&](float (&v)[S::SB], int s0) {
        const float* mcol = sT + s0 * S::B + s0;      // M(s0+q, s0+jj) at jj*B + q
        float4 cur[4], nxt[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) cur[w] = *reinterpret_cast<const float4*>(mcol + 4 * w);
#pragma unroll
        for (int jj = 0; jj < S::SB; ++jj) {
            if (jj + 1 < S::SB) {
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    nxt[w] = *reinterpret_cast<const float4*>(mcol + (jj + 1) * S::B + 4 * w);
            }
            const float m[16] = {cur[0].x, cur[0].y, cur[0].z, cur[0].w,
                                 cur[1].x, cur[1].y, cur[1].z, cur[1].w,
                                 cur[2].x, cur[2].y, cur[2].z, cur[2].w,
                                 cur[3].x, cur[3].y, cur[3].z, cur[3].w};
            v[jj] *= sD[s0 + jj];
#pragma unroll
            for (int q = jj + 1; q < S::SB; ++q) v[q] = fmaf(-m[q], v[jj], v[q]);
#pragma unroll
            for (int w = 0; w < 4; ++w) cur[w] = nxt[w];
        }
    };

    // Write-back form: 16-byte vectors when the addresses line up.
    const bool y_vec = a.planes && (reinterpret_cast<uintptr_t>(a.pl.y_hi) & 15) == 0 &&
                       (reinterpret_cast<uintptr_t>(a.pl.y_lo) & 15) == 0 &&
                       (reinterpret_cast<uintptr_t>(a.pl.y_lo2) & 15) == 0 &&
                       (a.pl.ldy & 7) == 0 && (r0 & 7) == 0;
    const bool c_vec = !ROWS || (p.c_rs == 1 && (reinterpret_cast<uintptr_t>(p.C) & 15) == 0 &&
                                 (p.c_cs & 3) == 0 && (r0 & 3) == 0);
    const bool vec_wb = y_vec && c_vec;

#pragma unroll 1
    for (bool first = true; panel < npanels; panel += pstride, first = false) {
        const int64_t j0 = panel * S::NC;
        const int ncols = (int)(p.nrhs - j0 < S::NC ? p.nrhs - j0 : S::NC);
        if (!first) {
            fetch_panel(j0);
            cp_async_wait_all();
            group_sync(g);
        }
        // The owners' tiles are kept negated, as pairs of rows (2u, 2u+1)
        // per column v: y = -x, so each update y += M(i,l) X(l,:) is a plain
        // packed FMA (and rounds exactly as x - M(i,l) X(l,:) would). The
        // substitution warp keeps the block it solved last, xs (its column).
        uint64_t y[4][4];
        float xs[S::SB];
        if (subst_warp) {
#pragma unroll
            for (int q = 0; q < S::SB; ++q) xs[q] = alpha * sC[q * S::LDC + lane];
            solve_block(xs, 0);
#pragma unroll
            for (int q = 0; q < S::SB; ++q) sC[q * S::LDC + lane] = xs[q];
        } else {
#pragma unroll
            for (int u2 = 0; u2 < 4; ++u2) {
                const float4 w0 = *reinterpret_cast<const float4*>(sC + (8 * rg + 2 * u2) * S::LDC + 4 * cg);
                const float4 w1 = *reinterpret_cast<const float4*>(sC + (8 * rg + 2 * u2 + 1) * S::LDC + 4 * cg);
                y[u2][0] = pack2(-(alpha * w0.x), -(alpha * w1.x));
                y[u2][1] = pack2(-(alpha * w0.y), -(alpha * w1.y));
                y[u2][2] = pack2(-(alpha * w0.z), -(alpha * w1.z));
                y[u2][3] = pack2(-(alpha * w0.w), -(alpha * w1.w));
            }
        }

#pragma unroll 1
        for (int s = 0; s + 1 < nblk; ++s) {
            // X_s is in the buffer; so are block s+1's rows, with every
            // update but the one by X_s.
            group_sync(g);
            const int s0 = s * S::SB;
            if (subst_warp) {
                const int t0 = s0 + S::SB;
                const float sc = s == 0 ? alpha : 1.f;   // block 1 still holds C itself
                uint64_t v2[S::SB / 2];                  // rows t0 + 2h, t0 + 2h + 1
#pragma unroll
                for (int h = 0; h < S::SB / 2; ++h)
                    v2[h] = pack2(sc * sC[(t0 + 2 * h) * S::LDC + lane],
                                  sc * sC[(t0 + 2 * h + 1) * S::LDC + lane]);
                const float* mb = sT + s0 * S::B + t0;   // M(t0+q, s0+kk) at kk*B + q
#pragma unroll
                for (int kk = 0; kk < S::SB; ++kk) {
                    const float4 m0 = *reinterpret_cast<const float4*>(mb + kk * S::B);
                    const float4 m1 = *reinterpret_cast<const float4*>(mb + kk * S::B + 4);
                    const float4 m2 = *reinterpret_cast<const float4*>(mb + kk * S::B + 8);
                    const float4 m3 = *reinterpret_cast<const float4*>(mb + kk * S::B + 12);
                    const uint64_t xn = pack2(-xs[kk], -xs[kk]);
                    v2[0] = ffma2(pack2(m0.x, m0.y), xn, v2[0]);
                    v2[1] = ffma2(pack2(m0.z, m0.w), xn, v2[1]);
                    v2[2] = ffma2(pack2(m1.x, m1.y), xn, v2[2]);
                    v2[3] = ffma2(pack2(m1.z, m1.w), xn, v2[3]);
                    v2[4] = ffma2(pack2(m2.x, m2.y), xn, v2[4]);
                    v2[5] = ffma2(pack2(m2.z, m2.w), xn, v2[5]);
                    v2[6] = ffma2(pack2(m3.x, m3.y), xn, v2[6]);
                    v2[7] = ffma2(pack2(m3.z, m3.w), xn, v2[7]);
                }
#pragma unroll
                for (int h = 0; h < S::SB / 2; ++h) unpack2(v2[h], xs[2 * h], xs[2 * h + 1]);
                solve_block(xs, t0);
#pragma unroll
                for (int q = 0; q < S::SB; ++q) sC[(t0 + q) * S::LDC + lane] = xs[q];
            } else if (rg >= 2 * s + 4) {
                // rank-16 update of the owned rows below block s+1
#pragma unroll 4
                for (int kk = 0; kk < S::SB; ++kk) {
                    const int l = s0 + kk;
                    const float4 xv = *reinterpret_cast<const float4*>(sC + l * S::LDC + 4 * cg);
                    const float4 t0v = *reinterpret_cast<const float4*>(sT + l * S::B + 8 * rg);
                    const float4 t1v = *reinterpret_cast<const float4*>(sT + l * S::B + 8 * rg + 4);
                    const uint64_t tp[4] = {pack2(t0v.x, t0v.y), pack2(t0v.z, t0v.w),
                                            pack2(t1v.x, t1v.y), pack2(t1v.z, t1v.w)};
                    const uint64_t xb[4] = {pack2(xv.x, xv.x), pack2(xv.y, xv.y),
                                            pack2(xv.z, xv.z), pack2(xv.w, xv.w)};
#pragma unroll
                    for (int u2 = 0; u2 < 4; ++u2)
#pragma unroll
                        for (int v = 0; v < 4; ++v) y[u2][v] = ffma2(tp[u2], xb[v], y[u2][v]);
                }
                // block s+2's owners publish their rows for its substitution
                if ((rg >> 1) == s + 2 && s + 2 < nblk) {
#pragma unroll
                    for (int u2 = 0; u2 < 4; ++u2) {
                        float a0[4], b0[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) unpack2(y[u2][v], a0[v], b0[v]);
                        *reinterpret_cast<float4*>(sC + (8 * rg + 2 * u2) * S::LDC + 4 * cg) =
                            make_float4(-a0[0], -a0[1], -a0[2], -a0[3]);
                        *reinterpret_cast<float4*>(sC + (8 * rg + 2 * u2 + 1) * S::LDC + 4 * cg) =
                            make_float4(-b0[0], -b0[1], -b0[2], -b0[3]);
                    }
                }
            }
        }
        group_sync(g);   // the last block solved is visible: every row is final

        // Write back (and the Y planes on the tensor-core path).
        if (vec_wb) {
            // lane: rows 8ro..8ro+7 x columns 4c4..4c4+3 (a warp: 32 rows)
            const int ro = 4 * (gt >> 5) + (lane >> 3), c4 = lane & 7;
            const int i0 = 8 * ro;
            if (i0 < bs && 4 * c4 < ncols) {
                float4 w[8];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    w[e] = *reinterpret_cast<const float4*>(sC + (i0 + e) * S::LDC + 4 * c4);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int c = 4 * c4 + cc;
                    if (c >= ncols) break;
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        v[e] = cc == 0 ? w[e].x : cc == 1 ? w[e].y : cc == 2 ? w[e].z : w[e].w;
                    if (i0 + 8 <= bs) {
                        put_y8(a.pl, (j0 + c) * a.pl.ldy + r0 + i0, v);
                        if constexpr (ROWS) {
                            float* dst = p.C + (r0 + i0) + (j0 + c) * p.c_cs;
                            *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
                            *reinterpret_cast<float4*>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
                        }
                    } else {
#pragma unroll 1
                        for (int e = 0; e < 8 && i0 + e < bs; ++e) {
                            put_y(a.pl, (j0 + c) * a.pl.ldy + r0 + i0 + e, v[e]);
                            if constexpr (ROWS) p.C[(r0 + i0 + e) + (j0 + c) * p.c_cs] = v[e];
                        }
                    }
                }
            }
            if constexpr (!ROWS) {
                const int c = gt & 31, ii = gt >> 5;
                if (c < ncols) {
#pragma unroll 4
                    for (int u = 0; u < S::B / 4; ++u) {
                        const int i = ii + 4 * u;
                        if (i < bs) p.C[(r0 + i) * p.c_rs + (j0 + c) * p.c_cs] = sC[i * S::LDC + c];
                    }
                }
            }
        } else if constexpr (ROWS) {
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

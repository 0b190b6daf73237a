// CUDA-core GEMM update (FP32 FMA / FP64 DFMA) on the canonical matrices:
//
//   C[rc+i, j] = beta * C[rc+i, j] + gamma * sum_l M(rc+i, rk+l) * Y[rk+l, j]
//
// with Y = C (a different row block of the same buffer) inside the recursion.
// This is the off-diagonal step of the recursion (Section 3.1): for TRSM
// B2 := beta*B2 - M21 X1 (gamma = -1), for TRMM B2 += alpha M21 B1. Rows
// [rc, rc+mlen) and [rk, rk+klen) are disjoint row blocks of one buffer.
//
// It is the GEMM engine of the FP64 path (tcgen05 has no FP64 kind), the
// FP32 path's engine for small updates whose K is not a multiple of the
// tensor-core K tile, and the FP32 engine when the tensor cores are switched
// off. Tile 64x64x16, 256 threads, 4x4 outputs per thread, operands staged
// through shared memory with the global loop order chosen so the contiguous
// index runs fastest (the matrices arrive with arbitrary signed strides).
// An update with fewer 64x64 tiles than twice the SMs takes 32x32 (2x2
// outputs per thread) or 16x16 tiles (one output), four or sixteen times the
// CTAs: the FP64 pipe is about 1/64 of the FP32 one per SM on this part, so
// a small FP64 update on a few SMs was the FP64 path's bottleneck at small
// orders.
#include "common.cuh"

namespace trx {
namespace {

constexpr int BK = 16, NT = 256;

template <typename T>
struct GemmArgs {
    Canon<T> p;
    const T* Y;            // K operand, Y(l, j) = Y[l*y_rs + j*y_cs] (C in the recursion)
    int64_t y_rs, y_cs;
    int64_t rc, mlen, rk, klen;
    T beta, gamma;
};

// TM x TM outputs per thread; tile BM = BN = 16 TM.
template <typename T, int TM>
__global__ void __launch_bounds__(NT) gemm_simt_kernel(GemmArgs<T> g) {
    constexpr int BM = 16 * TM, BN = 16 * TM, LE = BM * BK / NT;   // loads per thread
    __shared__ T sA[2][BK][BM + 4];   // sA[l][i] = M(rc+i0+i, rk+l0+l)
    __shared__ T sB[2][BK][BN + 4];   // sB[l][j] = C(rk+l0+l, j0+j)
    pdl_trigger();
    pdl_wait();
    const Canon<T>& p = g.p;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t i0 = (int64_t)blockIdx.y * BM;
    const int64_t j0 = (int64_t)blockIdx.x * BN;
    const bool a_row_fast = (p.a_rs == 1 || p.a_rs == -1);
    const bool y_row_fast = (g.y_rs == 1 || g.y_rs == -1);

    T ra[LE], rb[LE];
    auto load = [&](int64_t l0) {
#pragma unroll
        for (int u = 0; u < LE; ++u) {
            const int e = tid + u * NT;
            int i, l;
            if (a_row_fast) { i = e % BM; l = e / BM; } else { l = e % BK; i = e / BK; }
            const int64_t gi = i0 + i, gl = l0 + l;
            ra[u] = (gi < g.mlen && gl < g.klen) ? p.A[(g.rc + gi) * p.a_rs + (g.rk + gl) * p.a_cs] : T(0);
            int lb, jb;
            if (y_row_fast) { lb = e % BK; jb = e / BK; } else { jb = e % BN; lb = e / BN; }
            const int64_t gl2 = l0 + lb, gj = j0 + jb;
            rb[u] = (gl2 < g.klen && gj < p.nrhs) ? g.Y[(g.rk + gl2) * g.y_rs + gj * g.y_cs] : T(0);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < LE; ++u) {
            const int e = tid + u * NT;
            int i, l;
            if (a_row_fast) { i = e % BM; l = e / BM; } else { l = e % BK; i = e / BK; }
            sA[buf][l][i] = ra[u];
            int lb, jb;
            if (y_row_fast) { lb = e % BK; jb = e / BK; } else { jb = e % BN; lb = e / BN; }
            sB[buf][lb][jb] = rb[u];
        }
    };

    T acc[TM][TM];
#pragma unroll
    for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TM; ++v) acc[u][v] = T(0);

    int buf = 0;
    load(0);
    store(0);
    __syncthreads();
    for (int64_t l0 = 0; l0 < g.klen; l0 += BK) {
        const bool more = l0 + BK < g.klen;
        if (more) load(l0 + BK);   // next tile in flight during the FMAs
#pragma unroll
        for (int l = 0; l < BK; ++l) {
            T a[TM], b[TM];
#pragma unroll
            for (int u = 0; u < TM; ++u) a[u] = sA[buf][l][tx + 16 * u];
#pragma unroll
            for (int v = 0; v < TM; ++v) b[v] = sB[buf][l][ty + 16 * v];
#pragma unroll
            for (int u = 0; u < TM; ++u)
#pragma unroll
                for (int v = 0; v < TM; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        if (more) {
            store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int u = 0; u < TM; ++u) {
        const int64_t gi = i0 + tx + 16 * u;
        if (gi >= g.mlen) continue;
#pragma unroll
        for (int v = 0; v < TM; ++v) {
            const int64_t gj = j0 + ty + 16 * v;
            if (gj >= p.nrhs) continue;
            T* c = p.C + (g.rc + gi) * p.c_rs + gj * p.c_cs;
            *c = g.beta * *c + g.gamma * acc[u][v];
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_gemm_simt(const Canon<T>& p, const T* Y, int64_t y_rs, int64_t y_cs,
                             int64_t rc, int64_t mlen, int64_t rk, int64_t klen, T beta,
                             T gamma, cudaStream_t s, int num_sms) {
    if (mlen <= 0 || p.nrhs <= 0) return cudaSuccess;
    GemmArgs<T> g;
    g.p = p;
    g.Y = Y;
    g.y_rs = y_rs;
    g.y_cs = y_cs;
    g.rc = rc;
    g.mlen = mlen;
    g.rk = rk;
    g.klen = klen;
    g.beta = beta;
    g.gamma = gamma;
    // the largest tile (64, 32, 16 rows) that still gives every SM two CTAs
    auto tiles = [&](int tm) {
        return ((mlen + 16 * tm - 1) / (16 * tm)) * ((p.nrhs + 16 * tm - 1) / (16 * tm));
    };
    const int64_t want = 2 * (int64_t)(num_sms > 0 ? num_sms : 1);
    const int tm = tiles(4) >= want ? 4 : tiles(2) >= want ? 2 : 1;
    const int64_t gy = (mlen + 16 * tm - 1) / (16 * tm), gx = (p.nrhs + 16 * tm - 1) / (16 * tm);
    if (gy > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    if (tm == 1) return launch_kernel(gemm_simt_kernel<T, 1>, grid, dim3(NT), 0, s, g);
    if (tm == 2) return launch_kernel(gemm_simt_kernel<T, 2>, grid, dim3(NT), 0, s, g);
    return launch_kernel(gemm_simt_kernel<T, 4>, grid, dim3(NT), 0, s, g);
}

template cudaError_t launch_gemm_simt<float>(const Canon<float>&, const float*, int64_t, int64_t,
                                             int64_t, int64_t, int64_t, int64_t, float, float,
                                             cudaStream_t, int);
template cudaError_t launch_gemm_simt<double>(const Canon<double>&, const double*, int64_t,
                                              int64_t, int64_t, int64_t, int64_t, int64_t,
                                              double, double, cudaStream_t, int);

}  // namespace trx

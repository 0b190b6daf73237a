// Operand preparation for the tensor-core FP32 path, and the alpha == 0
// quick return.
//
// The tcgen05 GEMM update multiplies BF16 operands. An FP32 value x is carried
// as one, two or three BF16 slices (x0 = bf16(x), x1 = bf16(x - x0), x2 =
// bf16(x - x0 - x1); Planes in common.cuh) and a product as the slice
// products above FP32's rounding level, with FP32 accumulation. These
// kernels write the planes in the canonical K-major order the GEMM's TMA
// loads expect:
//   M planes: strictly-lower part of M, (i, l) at i*ldm + l; with diagonal
//             blocks requested, also explicit zeros on and above the
//             diagonal inside each block, so a block can be used as a dense
//             GEMM operand
//   Y planes: C (TRMM's original right-hand side), (l, j) at j*ldy + l
// 32x32 tiles go through shared memory, so reads are coalesced along
// whichever index is contiguous in the caller's storage and writes along the
// planes' contiguous index.
#include "common.cuh"

namespace trx {
namespace {

// Planes of slice q (0, 1, 2) of an M or Y plane set.
__device__ __forceinline__ __nv_bfloat16* m_plane(const Planes& pl, int q) {
    return q == 0 ? pl.m_hi : q == 1 ? pl.m_lo : pl.m_lo2;
}
__device__ __forceinline__ __nv_bfloat16* y_plane(const Planes& pl, int q) {
    return q == 0 ? pl.y_hi : q == 1 ? pl.y_lo : pl.y_lo2;
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

// M planes: 64x64 tiles of the lower triangle (tiles above it exit at once,
// except inside a diagonal block of zdb tiles when zdb > 0), read along A's
// contiguous index (every load of a thread issued before its first shared
// store), written four l values at a time: 8-byte stores of packed slices.
__global__ void __launch_bounds__(256) convert_m_kernel(Canon<float> p, Planes pl, int zdb) {
    pdl_trigger();
    pdl_wait();
    __shared__ float tile[64][65];
    const int64_t ti = blockIdx.y, tl = blockIdx.x;
    if (tl > ti && (zdb == 0 || tl / zdb != ti / zdb)) return;
    const int64_t i0 = ti * 64, l0 = tl * 64;
    const int tid = threadIdx.x;
    const bool row_fast = (p.a_rs == 1 || p.a_rs == -1);
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * u;
        const int ii = row_fast ? (e & 63) : (e >> 6), ll = row_fast ? (e >> 6) : (e & 63);
        const int64_t i = i0 + ii, l = l0 + ll;
        v[u] = (i < p.k && l < i) ? p.A[i * p.a_rs + l * p.a_cs] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * u;
        const int ii = row_fast ? (e & 63) : (e >> 6), ll = row_fast ? (e >> 6) : (e & 63);
        tile[ii][ll] = v[u];
    }
    __syncthreads();
    const bool vec = (pl.ldm & 3) == 0 && (reinterpret_cast<uintptr_t>(pl.m_hi) & 7) == 0 &&
                     (reinterpret_cast<uintptr_t>(pl.m_lo) & 7) == 0 &&
                     (reinterpret_cast<uintptr_t>(pl.m_lo2) & 7) == 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int e = tid + 256 * u;
        const int ii = e >> 4, lq = (e & 15) * 4;
        const int64_t i = i0 + ii, l = l0 + lq;
        if (i >= p.k || l >= p.k) continue;
        const int64_t off = i * pl.ldm + l;
        const float x[4] = {tile[ii][lq], tile[ii][lq + 1], tile[ii][lq + 2], tile[ii][lq + 3]};
        if (vec && l + 3 < p.k) {
            uint32_t h[2];
            h[0] = bf16x2(x[1], x[0]);
            h[1] = bf16x2(x[3], x[2]);
            *reinterpret_cast<uint2*>(pl.m_hi + off) = make_uint2(h[0], h[1]);
            if (pl.slices < 2) continue;
            const float r[4] = {x[0] - bf_lo(h[0]), x[1] - bf_hi(h[0]), x[2] - bf_lo(h[1]),
                                x[3] - bf_hi(h[1])};
            uint32_t q[2];
            q[0] = bf16x2(r[1], r[0]);
            q[1] = bf16x2(r[3], r[2]);
            *reinterpret_cast<uint2*>(pl.m_lo + off) = make_uint2(q[0], q[1]);
            if (pl.slices < 3) continue;
            q[0] = bf16x2(r[1] - bf_hi(q[0]), r[0] - bf_lo(q[0]));
            q[1] = bf16x2(r[3] - bf_hi(q[1]), r[2] - bf_lo(q[1]));
            *reinterpret_cast<uint2*>(pl.m_lo2 + off) = make_uint2(q[0], q[1]);
        } else {
            for (int c = 0; c < 4 && l + c < p.k; ++c) {
                __nv_bfloat16 sl[3];
                split_slices(x[c], pl.slices, sl);
                for (int s = 0; s < pl.slices; ++s) m_plane(pl, s)[off + c] = sl[s];
            }
        }
    }
}

// Y planes when C's rows are contiguous (side L): no transpose, four
// consecutive rows per thread, 8-byte stores.
__global__ void __launch_bounds__(256) convert_y_contig_kernel(Canon<float> p, Planes pl) {
    pdl_trigger();
    pdl_wait();
    const int64_t l = ((int64_t)blockIdx.x * 256 + threadIdx.x) * 4;
    if (l >= p.k) return;
    for (int64_t j = blockIdx.y; j < p.nrhs; j += gridDim.y) {
        const float* src = p.C + j * p.c_cs;
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = (l + q < p.k) ? src[(l + q) * p.c_rs] : 0.f;
        __nv_bfloat16 sl[4][3];
#pragma unroll
        for (int q = 0; q < 4; ++q) split_slices(v[q], pl.slices, sl[q]);
        const int64_t off = j * pl.ldy + l;
        if (l + 3 < p.k) {
            for (int s = 0; s < pl.slices; ++s) {
                __nv_bfloat162 hv[2] = {__halves2bfloat162(sl[0][s], sl[1][s]),
                                        __halves2bfloat162(sl[2][s], sl[3][s])};
                *reinterpret_cast<uint2*>(y_plane(pl, s) + off) = *reinterpret_cast<uint2*>(hv);
            }
        } else {
            for (int q = 0; l + q < p.k; ++q)
                for (int s = 0; s < pl.slices; ++s) y_plane(pl, s)[off + q] = sl[q][s];
        }
    }
}

// Y planes when C's columns are contiguous (side R): 32x32 transpose tiles.
__global__ void __launch_bounds__(256) convert_y_kernel(Canon<float> p, Planes pl) {
    pdl_trigger();
    pdl_wait();
    __shared__ float tile[32][33];              // tile[jj][ll]
    const int64_t l0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const bool row_fast = (p.c_rs == 1 || p.c_rs == -1);
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int x = threadIdx.x;
        const int ll = row_fast ? x : r, jj = row_fast ? r : x;
        const int64_t l = l0 + ll, j = j0 + jj;
        float v = 0.f;
        if (l < p.k && j < p.nrhs) v = p.C[l * p.c_rs + j * p.c_cs];
        tile[jj][ll] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t j = j0 + r, l = l0 + threadIdx.x;
        if (l < p.k && j < p.nrhs) put_y(pl, j * pl.ldy + l, tile[r][threadIdx.x]);
    }
}

// Generic block: tile[rr][cc] staged so that both sides are coalesced.
__global__ void __launch_bounds__(256) convert_rect_kernel(const float* src, int64_t rs,
                                                           int64_t cs, int64_t rows, int64_t cols,
                                                           __nv_bfloat16* hi, __nv_bfloat16* lo,
                                                           __nv_bfloat16* lo2, int slices,
                                                           int64_t ld, int row_major) {
    pdl_trigger();
    pdl_wait();
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const bool src_row_fast = (rs == 1 || rs == -1);
    for (int t = threadIdx.y; t < 32; t += 8) {
        const int rr = src_row_fast ? threadIdx.x : t, cc = src_row_fast ? t : threadIdx.x;
        const int64_t r = r0 + rr, c = c0 + cc;
        tile[rr][cc] = (r < rows && c < cols) ? src[r * rs + c * cs] : 0.f;
    }
    __syncthreads();
    for (int t = threadIdx.y; t < 32; t += 8) {
        // destination contiguous index runs along threadIdx.x
        const int rr = row_major ? t : threadIdx.x, cc = row_major ? threadIdx.x : t;
        const int64_t r = r0 + rr, c = c0 + cc;
        if (r < rows && c < cols)
            put_split(hi, lo, lo2, slices, row_major ? r * ld + c : c * ld + r, tile[rr][cc]);
    }
}

// Inverse of each full b x b diagonal block of the canonical lower M,
// W = inv(M_ii) (lower triangular), as split planes over rows and columns
// [r0, r0 + b) of a row-major plane pair (element (i, l) at i * ld + l,
// zeros above the diagonal), or, compact, at rows [r0, r0 + b) and columns
// [0, b) of a k x ld plane. One CTA per block: the block is staged in
// shared memory and thread j solves M_ii w_j = e_j by forward substitution
// for column j of W.
__global__ void __launch_bounds__(128) invert_diag_kernel(Canon<float> p, int b,
                                                          __nv_bfloat16* w_hi,
                                                          __nv_bfloat16* w_lo,
                                                          __nv_bfloat16* w_lo2, int slices,
                                                          int64_t ld, int compact) {
    pdl_trigger();
    pdl_wait();
    extern __shared__ float inv_sm[];
    float* Ls = inv_sm;                      // b x (b + 1), M_ii row by row
    float* Ws = inv_sm + b * (b + 1);        // b x b, W row by row
    const int64_t r0 = (int64_t)blockIdx.x * b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int i = e / b, l = e % b;
        float v = 0.f;
        if (l < i)
            v = p.A[(r0 + i) * p.a_rs + (r0 + l) * p.a_cs];
        else if (l == i)
            v = p.unit ? 1.f : p.A[(r0 + i) * (p.a_rs + p.a_cs)];
        Ls[i * (b + 1) + l] = v;
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < b) {
        for (int i = 0; i < b; ++i) {
            float w = 0.f;
            if (i >= j) {
                float acc = (i == j) ? 1.f : 0.f;
                for (int l = j; l < i; ++l) acc -= Ls[i * (b + 1) + l] * Ws[l * b + j];
                w = acc / Ls[i * (b + 1) + i];
            }
            Ws[i * b + j] = w;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int i = e / b, l = e % b;
        put_split(w_hi, w_lo, w_lo2, slices, (r0 + i) * ld + (compact ? 0 : r0) + l,
                  Ws[i * b + l]);
    }
}

template <typename T>
__global__ void zero_kernel(T* B, int64_t m, int64_t n, int64_t ldb) {
    pdl_trigger();
    pdl_wait();
    const int64_t total = m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % m, j = e / m;
        B[i + j * ldb] = T(0);
    }
}

}  // namespace

cudaError_t launch_convert_m(const Canon<float>& p, const Planes& pl, int diag_block,
                             cudaStream_t s) {
    if (p.k <= 0 || (p.k <= 1 && diag_block == 0)) return cudaSuccess;
    const int64_t t = (p.k + 63) / 64;
    if (t > 65535 || diag_block % 64 != 0) return cudaErrorInvalidValue;
    return launch_kernel(convert_m_kernel, dim3((unsigned)t, (unsigned)t), dim3(256), 0, s, p, pl,
                         diag_block / 64);
}

cudaError_t launch_convert_y(const Canon<float>& p, const Planes& pl, cudaStream_t s) {
    if (p.k <= 0 || p.nrhs <= 0) return cudaSuccess;
    if (p.c_rs == 1 || p.c_rs == -1) {
        const int64_t gx = (p.k + 1023) / 1024;
        const int64_t gy = p.nrhs < 65535 ? p.nrhs : 65535;
        return launch_kernel(convert_y_contig_kernel, dim3((unsigned)gx, (unsigned)gy), dim3(256),
                             0, s, p, pl);
    }
    const int64_t tl = (p.k + 31) / 32, tj = (p.nrhs + 31) / 32;
    if (tj > 65535) return cudaErrorInvalidValue;
    return launch_kernel(convert_y_kernel, dim3((unsigned)tl, (unsigned)tj), dim3(32, 8), 0, s, p,
                         pl);
}

cudaError_t launch_invert_diag(const Canon<float>& p, int b, __nv_bfloat16* w_hi,
                               __nv_bfloat16* w_lo, __nv_bfloat16* w_lo2, int slices, int64_t ld,
                               cudaStream_t s, bool compact) {
    if (b < 1 || b > 128 || (compact && ld < b)) return cudaErrorInvalidValue;
    const int64_t blocks = p.k / b;          // full blocks only
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    const int smem = (int)((size_t)b * (2 * b + 1) * sizeof(float));
    return launch_kernel(invert_diag_kernel, dim3((unsigned)blocks), dim3(128), smem, s, p, b,
                         w_hi, w_lo, w_lo2, slices, ld, compact ? 1 : 0);
}

// Shared-memory limit of the inversion kernel; like every kernel attribute
// it applies to the current device only, so it runs once per device (from
// the per-device set-up of handles and of the allocation-free entry).
cudaError_t convert_configure() {
    return cudaFuncSetAttribute(invert_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                128 * (2 * 128 + 1) * (int)sizeof(float));
}

// Y planes of C's rows [r0, r0 + rows) only (the rows of one TRSM leaf).
cudaError_t launch_convert_y_rows(const Canon<float>& p, const Planes& pl, int64_t r0,
                                  int64_t rows, cudaStream_t s) {
    if (r0 < 0 || rows < 0 || r0 + rows > p.k || r0 % 4 != 0) return cudaErrorInvalidValue;
    Canon<float> v = p;
    v.C = p.C + r0 * p.c_rs;
    v.k = rows;
    Planes w = pl;
    w.y_hi = pl.y_hi + r0;
    w.y_lo = pl.y_lo ? pl.y_lo + r0 : nullptr;
    w.y_lo2 = pl.y_lo2 ? pl.y_lo2 + r0 : nullptr;
    return launch_convert_y(v, w, s);
}

cudaError_t launch_convert_rect(const float* src, int64_t rs, int64_t cs, int64_t rows,
                                int64_t cols, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                __nv_bfloat16* lo2, int slices, int64_t ld, bool row_major,
                                cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int64_t gy = (rows + 31) / 32, gx = (cols + 31) / 32;
    if (gy > 65535) return cudaErrorInvalidValue;
    return launch_kernel(convert_rect_kernel, dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, s,
                         src, rs, cs, rows, cols, hi, lo, lo2, slices, ld, row_major ? 1 : 0);
}

template <typename T>
cudaError_t launch_zero(T* B, int64_t m, int64_t n, int64_t ldb, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int64_t total = m * n;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    return launch_kernel(zero_kernel<T>, dim3((unsigned)blocks), dim3(256), 0, s, B, m, n, ldb);
}

template cudaError_t launch_zero<float>(float*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_zero<double>(double*, int64_t, int64_t, int64_t, cudaStream_t);

}  // namespace trx

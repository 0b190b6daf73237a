// Element-wise and reduction kernels of the refined FP32 TRSM (iterative
// refinement in FP64 around the FP32 solve): precision casts, the residual
// R = alpha B - op(A) X, the correction X += D, and the infinity norms that
// decide when to stop. All column-major, leading dimensions in elements.
#include "common.cuh"

namespace trx {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) cast_f32_f64_kernel(const float* src, int64_t lds,
                                                                double* dst, int64_t ldd,
                                                                int64_t m, int64_t n,
                                                                double scale) {
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < m * n;
         e += (int64_t)gridDim.x * kThreads) {
        const int64_t i = e % m, j = e / m;
        dst[i + j * ldd] = scale * (double)src[i + j * lds];
    }
}

__global__ void __launch_bounds__(kThreads) cast_f64_f32_kernel(const double* src, int64_t lds,
                                                                float* dst, int64_t ldd,
                                                                int64_t m, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < m * n;
         e += (int64_t)gridDim.x * kThreads) {
        const int64_t i = e % m, j = e / m;
        dst[i + j * ldd] = (float)src[i + j * lds];
    }
}

// r := b - r (b already holds alpha B in FP64)
__global__ void __launch_bounds__(kThreads) residual_kernel(const double* b, int64_t ldb,
                                                            double* r, int64_t ldr, int64_t m,
                                                            int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < m * n;
         e += (int64_t)gridDim.x * kThreads) {
        const int64_t i = e % m, j = e / m;
        r[i + j * ldr] = b[i + j * ldb] - r[i + j * ldr];
    }
}

// x := x + d
__global__ void __launch_bounds__(kThreads) add_f32_kernel(double* x, int64_t ldx,
                                                           const float* d, int64_t ldd,
                                                           int64_t m, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < m * n;
         e += (int64_t)gridDim.x * kThreads) {
        const int64_t i = e % m, j = e / m;
        x[i + j * ldx] += (double)d[i + j * ldd];
    }
}

// Row sums of |M| (m x n, column-major), one thread per row.
__global__ void __launch_bounds__(kThreads) row_abs_sum_kernel(const double* a, int64_t lda,
                                                               int64_t m, int64_t n,
                                                               double* sums) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += fabs(a[i + j * lda]);
    sums[i] = s;
}

// Row sums of |op(A)| over A's referenced triangle (the unit diagonal counts
// 1), A k x k column-major: row i of op(A) is row i of A ('N') or column i.
__global__ void __launch_bounds__(kThreads) op_row_abs_sum_kernel(const double* a, int64_t lda,
                                                                  int64_t k, int lower, int trans,
                                                                  int unit, double* sums) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= k) return;
    // entries of row i of op(A): op(A)(i, l) = A(i, l) or A(l, i)
    const bool eff_lower = (lower != 0) != (trans != 0);   // op(A) lower triangular
    const int64_t l0 = eff_lower ? 0 : i, l1 = eff_lower ? i + 1 : k;
    double s = 0.0;
    for (int64_t l = l0; l < l1; ++l) {
        if (l == i) {
            s += unit ? 1.0 : fabs(a[i + i * lda]);
            continue;
        }
        s += fabs(trans ? a[l + i * lda] : a[i + l * lda]);
    }
    sums[i] = s;
}

// out[0] := max(v[0..n-1]) (one block).
__global__ void __launch_bounds__(kThreads) max_kernel(const double* v, int64_t n, double* out) {
    __shared__ double red[kThreads];
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kThreads) mx = fmax(mx, v[i]);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

int grid_for(int64_t count) {
    const int64_t g = (count + kThreads - 1) / kThreads;
    return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

cudaError_t refine_cast_f32_f64(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t m,
                                int64_t n, double scale, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    cast_f32_f64_kernel<<<grid_for(m * n), kThreads, 0, s>>>(src, lds, dst, ldd, m, n, scale);
    return cudaGetLastError();
}
cudaError_t refine_cast_f64_f32(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t m,
                                int64_t n, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    cast_f64_f32_kernel<<<grid_for(m * n), kThreads, 0, s>>>(src, lds, dst, ldd, m, n);
    return cudaGetLastError();
}
cudaError_t refine_residual(const double* b, int64_t ldb, double* r, int64_t ldr, int64_t m,
                            int64_t n, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    residual_kernel<<<grid_for(m * n), kThreads, 0, s>>>(b, ldb, r, ldr, m, n);
    return cudaGetLastError();
}
cudaError_t refine_add(double* x, int64_t ldx, const float* d, int64_t ldd, int64_t m, int64_t n,
                       cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    add_f32_kernel<<<grid_for(m * n), kThreads, 0, s>>>(x, ldx, d, ldd, m, n);
    return cudaGetLastError();
}
// out[0] := ||M||_inf; sums: m doubles of scratch.
cudaError_t refine_norm_inf(const double* a, int64_t lda, int64_t m, int64_t n, double* sums,
                            double* out, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    row_abs_sum_kernel<<<(unsigned)((m + kThreads - 1) / kThreads), kThreads, 0, s>>>(a, lda, m, n,
                                                                                     sums);
    max_kernel<<<1, kThreads, 0, s>>>(sums, m, out);
    return cudaGetLastError();
}
// out[0] := ||op(A)||_inf over the referenced triangle; sums: k doubles.
cudaError_t refine_op_norm_inf(const double* a, int64_t lda, int64_t k, bool lower, bool trans,
                               bool unit, double* sums, double* out, cudaStream_t s) {
    if (k <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    op_row_abs_sum_kernel<<<(unsigned)((k + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        a, lda, k, lower, trans, unit, sums);
    max_kernel<<<1, kThreads, 0, s>>>(sums, k, out);
    return cudaGetLastError();
}

}  // namespace trx

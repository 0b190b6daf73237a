// Element-wise and reduction kernels of the refined FP32 TRSM (iterative
// refinement in FP64 around the FP32 solve): precision casts, the residual
// R = alpha B - op(A) X, the correction X += D, and the infinity norms that
// decide when to stop. All column-major, leading dimensions in elements.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "trx.h"

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
__global__ void __launch_bounds__(kThreads) scale_f64_kernel(const double* src, int64_t lds,
                                                             double* dst, int64_t ldd, int64_t m,
                                                             int64_t n, double scale) {
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < m * n;
         e += (int64_t)gridDim.x * kThreads) {
        const int64_t i = e % m, j = e / m;
        dst[i + j * ldd] = scale * src[i + j * lds];
    }
}
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

constexpr int kNormSlices = 32;   // column slices of the row-sum partials

// Row sums of |M| (m x n, column-major) in kNormSlices column slices: the
// partial of slice blockIdx.y for row i goes to part[blockIdx.y * m + i]
// (neighbouring threads read neighbouring rows); part_sum_kernel adds the
// slices in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kThreads) row_abs_part_kernel(const T* a, int64_t lda,
                                                                int64_t m, int64_t n,
                                                                double* part) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= m) return;
    const int64_t slice = (n + kNormSlices - 1) / kNormSlices;
    const int64_t j0 = blockIdx.y * slice, j1 = j0 + slice < n ? j0 + slice : n;
    double s = 0.0;
    for (int64_t j = j0; j < j1; ++j) s += fabs((double)a[i + j * lda]);
    part[blockIdx.y * m + i] = s;
}

// Row sums of |op(A)| over A's referenced triangle (the unit diagonal counts
// 1), A k x k FP32 column-major. Row i of op(A) is row i of A ('N': one
// thread per row, neighbouring threads read neighbouring rows) or column i
// (transposed: one warp per column, reading down it).
__global__ void __launch_bounds__(kThreads) op_row_abs_part_kernel(const float* a, int64_t lda,
                                                                   int64_t k, int lower, int unit,
                                                                   double* part) {
    // block: 64 rows x 4 phases of l; blockIdx.y: one of kNormSlices l-slices
    __shared__ double red[4][64];
    const int tx = threadIdx.x & 63, ph = threadIdx.x >> 6;
    const int64_t i = (int64_t)blockIdx.x * 64 + tx;
    const int64_t slice = (k + kNormSlices - 1) / kNormSlices;
    const int64_t s0 = blockIdx.y * slice, s1 = s0 + slice < k ? s0 + slice : k;
    double s = 0.0;
    if (i < k) {
        const int64_t l0 = lower ? s0 : (s0 > i ? s0 : i);
        const int64_t l1 = lower ? (s1 < i + 1 ? s1 : i + 1) : s1;
        for (int64_t l = l0 + ph; l < l1; l += 4)
            s += (l == i) ? (unit ? 1.0 : fabs((double)a[i + i * lda]))
                          : fabs((double)a[i + l * lda]);
    }
    red[ph][tx] = s;
    __syncthreads();
    if (ph == 0 && i < k)
        part[blockIdx.y * k + i] = red[0][tx] + red[1][tx] + red[2][tx] + red[3][tx];
}
__global__ void __launch_bounds__(kThreads) part_sum_kernel(const double* part, int64_t k,
                                                            double* sums) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= k) return;
    double s = 0.0;
    for (int q = 0; q < kNormSlices; ++q) s += part[q * k + i];
    sums[i] = s;
}
__global__ void __launch_bounds__(kThreads) op_col_abs_sum_kernel(const float* a, int64_t lda,
                                                                  int64_t k, int lower, int unit,
                                                                  double* sums) {
    const int64_t i = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= k) return;
    // column i of A holds rows i..k-1 (lower) or 0..i (upper)
    const int64_t l0 = lower ? i : 0, l1 = lower ? k : i + 1;
    double s = 0.0;
    for (int64_t l = l0 + lane; l < l1; l += 32)
        s += (l == i) ? (unit ? 1.0 : fabs((double)a[i + i * lda])) : fabs((double)a[l + i * lda]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sums[i] = s;
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

// dst(j, i) := scale * src(i, j) for src rows x cols (32 x 32 tiles through
// shared memory, both sides coalesced).
template <typename S, typename D>
__global__ void __launch_bounds__(256) transpose_kernel(const S* src, int64_t lds, D* dst,
                                                        int64_t ldd, int64_t rows, int64_t cols,
                                                        double scale) {
    __shared__ D tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + tx, j = j0 + r;
        if (i < rows && j < cols) tile[r][tx] = (D)(scale * (double)src[i + j * lds]);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + tx, i = i0 + r;
        if (i < rows && j < cols) dst[j + i * ldd] = tile[tx][r];
    }
}

// Column sums of |M| (m x n): one warp per column.
__global__ void __launch_bounds__(kThreads) col_abs_sum_kernel(const double* a, int64_t lda,
                                                               int64_t m, int64_t n,
                                                               double* sums) {
    const int64_t j = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    double s = 0.0;
    for (int64_t i = lane; i < m; i += 32) s += fabs(a[i + j * lda]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sums[j] = s;
}

// ---- residual in float-float on the FP32 pipes ------------------------------
// R := B - op(A) X for op(A) k x k triangular (FP32) and X k x n, B and R
// FP64 (R may be B).
//
// Each product a xh is split exactly into p + e with one FMA
// (e = a xh - p); p joins the running sum hi through the error-free
// two-sum (hi + p = t + err exactly, Knuth), and err + e + a xl go to a
// float lo. Every kFold stages lo is moved into a second float pair
// (mid, lo2) by another two-sum, so no step of the loop touches GB300's
// slow FP64 pipe; the four floats are added in FP64 once, at the end. The
// result keeps about 2^-46 of sum |a x| per output on random data (2^-44
// with cancelling terms spread over many binades), against 2^-24 for an
// FP32 dot product, at about six FP32 operations per term on the packed
// f32x2 path.
//
// Three modes: kFull (X = xh + xl, the residual from X), kSingle (X one
// float plane, e.g. a correction D: the update R - op(A) D keeps the same
// error-free accumulation without the xl products) and kPlain (one float
// plane, plain FP32 FMA accumulation: for an update whose D is so small
// against X that FP32 rounding of op(A) D is below the target).
//
// Operands are packed once into the order the kernel reads them, so every
// pipeline stage is two contiguous bulk copies (cp.async.bulk, completion
// counted on an mbarrier) into a three-stage ring:
//  - op(A) (once per refined solve): per 64-row tile, its 16-column chunks
//    that meet the triangle, each 16 x 64 float4 (a, a, -a, -a), masked to
//    the triangle, the unit diagonal written as 1: both packed operands of
//    a row in one 16-byte load;
//  - X (once per step): per 64-column tile, rows in 16-row chunks, each row
//    32 float4 (xh_a, xh_b, xl_a, xl_b) for the thread's column pair
//    (tx + 32 c, tx + 32 c + 16), zero beyond k and n.
// Tiles of 64 rows x 64 columns, 16 terms per stage, 256 threads; a thread
// owns rows ty + 16 r and column pairs (tx + 32 c, tx + 32 c + 16).
constexpr int kRM = 64, kRN = 64, kRK = 16, kFold = 2;   // fold every 32 terms
constexpr int kStages = 3;
constexpr uint32_t kABytes = kRK * kRM * 16, kXBytes = kRK * 32 * 16;
constexpr uint32_t kStageBytes = kABytes + kXBytes;
constexpr int kPipeSmem = kStages * (int)kStageBytes + 2 * kStages * 8 + 16;
enum { kFull = 0, kSingle = 1, kPlain = 2, kPair = 3 };
// kPair: FP64 data. op(A) is packed as float pairs (ah, ah, al, al) with
// ah = fl32(a), al = fl32(a - ah), X = xh + xl as in kFull; the term
// ah xh is split exactly (FMA) and two-summed into hi, and ah xl + al xh go
// to lo (al xl, below 2^-48 of a x, is left out).
constexpr uint64_t kSign2 = 0x8000000080000000ull;

__device__ __forceinline__ uint64_t pk(float a, float b) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ void upk(uint64_t v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// s + b = t + err exactly (two-sum, both lanes); returns err, s := t
__device__ __forceinline__ uint64_t two_sum2(uint64_t& s, uint64_t b) {
    const uint64_t t = add2(s, b);
    const uint64_t bp = sub2(t, s);
    const uint64_t err = add2(sub2(s, sub2(t, bp)), sub2(b, bp));
    s = t;
    return err;
}

// mbarrier and bulk-copy wrappers
__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// Bounded wait for phase `parity`: false once the CTA has aborted or
// `limit` ns have passed (then it aborts the CTA and sets the error word).
__device__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int* abort, int* err,
                         uint64_t limit, bool honour_abort) {
    if (bar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    while (true) {
        if (bar_try(bar, parity)) return true;
        if (honour_abort && *abort) return false;
        if (now_ns() - t0 > limit) {
            *abort = 1;
            atomicExch(err, TRX_ERR_TIMEOUT);
            return false;
        }
    }
}

// Chunks of row tile rt (16 columns of op(A) each) and the first one's
// column index / 16, for K16 = ceil(k / 16) column chunks.
__host__ __device__ __forceinline__ void tile_chunks(int64_t rt, int64_t K16, bool lower,
                                                     int64_t& first, int64_t& count,
                                                     int64_t& offset) {
    if (lower) {
        first = 0;
        count = 4 * (rt + 1) < K16 ? 4 * (rt + 1) : K16;
        offset = 2 * rt * (rt + 1);                      // sum of 4 (r + 1), r < rt
    } else {
        first = 4 * rt;
        count = K16 - 4 * rt;
        offset = rt * K16 - 2 * rt * (rt - 1);           // sum of K16 - 4 r, r < rt
    }
}

// op(A) packed: block (chunk q of row tile blockIdx.y, quarter blockIdx.x % 4).
// op(A) of FP64 data packed as (ah, ah, al, al), same layout as above.
template <bool TRANS>
__global__ void __launch_bounds__(256) pack_a64_kernel(const double* A, int64_t lda, int64_t k,
                                                       int lower, int unit, float4* Ap) {
    const int64_t K16 = (k + 15) / 16, rt = blockIdx.y, q = blockIdx.x >> 2;
    int64_t first, count, offset;
    tile_chunks(rt, K16, lower != 0, first, count, offset);
    if (q >= count) return;
    const int e = (int)(blockIdx.x & 3) * 256 + threadIdx.x;
    const int l = TRANS ? (e & 15) : (e >> 6), i = TRANS ? (e >> 4) : (e & 63);
    const int64_t gi = rt * kRM + i, gl = (first + q) * kRK + l;
    double v = 0.0;
    if (gi < k && gl < k && (lower ? gl <= gi : gl >= gi)) {
        if (gl == gi && unit) v = 1.0;
        else v = TRANS ? A[gl + gi * lda] : A[gi + gl * lda];
    }
    const float h = (float)v, lo = (float)(v - (double)h);
    Ap[(offset + q) * (kRK * kRM) + l * kRM + i] = make_float4(h, h, lo, lo);
}

template <bool TRANS>
__global__ void __launch_bounds__(256) pack_a_kernel(const float* A, int64_t lda, int64_t k,
                                                     int lower, int unit, float4* Ap) {
    const int64_t K16 = (k + 15) / 16, rt = blockIdx.y, q = blockIdx.x >> 2;
    int64_t first, count, offset;
    tile_chunks(rt, K16, lower != 0, first, count, offset);
    if (q >= count) return;
    const int e = (int)(blockIdx.x & 3) * 256 + threadIdx.x;      // element of the chunk
    // read order: along rows (i) for A[i + l lda], along columns (l) otherwise
    const int l = TRANS ? (e & 15) : (e >> 6), i = TRANS ? (e >> 4) : (e & 63);
    const int64_t gi = rt * kRM + i, gl = (first + q) * kRK + l;
    float v = 0.0f;
    if (gi < k && gl < k && (lower ? gl <= gi : gl >= gi)) {
        if (gl == gi && unit) v = 1.0f;
        else v = TRANS ? A[gl + gi * lda] : A[gi + gl * lda];
    }
    Ap[(offset + q) * (kRK * kRM) + l * kRM + i] = make_float4(v, v, -v, -v);
}

// X packed: rows 8 blockIdx.x .. + 7 of column tile blockIdx.y, one row per
// warp; lane t = (pair pc, lane jj).
template <bool SPLIT>
__global__ void __launch_bounds__(256) pack_x_kernel(const double* X64, const float* X32,
                                                     int64_t ldx, int64_t k, int64_t n,
                                                     int64_t rows, double scale, float4* Xp) {
    const int64_t l = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), ct = blockIdx.y;
    const int t = threadIdx.x & 31, pc = t >> 4, jj = t & 15;
    const int64_t ja = ct * kRN + jj + 32 * pc, jb = ja + 16;
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (l < k) {
        if (SPLIT) {
            const double xa = ja < n ? scale * X64[l + ja * ldx] : 0.0;
            const double xb = jb < n ? scale * X64[l + jb * ldx] : 0.0;
            v.x = (float)xa;
            v.y = (float)xb;
            v.z = (float)(xa - (double)v.x);
            v.w = (float)(xb - (double)v.y);
        } else {
            v.x = ja < n ? X32[l + ja * ldx] : 0.0f;
            v.y = jb < n ? X32[l + jb * ldx] : 0.0f;
        }
    }
    Xp[(ct * rows + l) * 32 + t] = v;
}

// Work units: a row tile's chunks are cut into pieces of at most
// kUnitChunks, so no CTA carries much more than its share of the triangle
// (the last row tile alone is k / 16 chunks). Unit = (row tile, first
// chunk, end chunk, partial slot): slot -1 writes R directly, otherwise the
// piece's sum goes to partial slot `slot` and refine_combine adds the
// pieces of a row tile in a fixed order (bitwise repeatable).
constexpr int kUnitChunks = 128;

template <int MODE>
__global__ void __launch_bounds__(256) residual_pipe_kernel(const float4* __restrict__ Ap,
                                                            const float4* __restrict__ Xp,
                                                            const int4* __restrict__ units,
                                                            double* part, int64_t rows, int64_t k,
                                                            int lower, const double* B,
                                                            int64_t ldb, double* R, int64_t ldr,
                                                            int64_t n, int* err,
                                                            long long wait_ns) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    volatile int* abort = reinterpret_cast<volatile int*>(empty + kStages);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31;
    const int64_t nct = (n + kRN - 1) / kRN, K16 = (k + 15) / 16;
    const int4 u = units[blockIdx.x / nct];      // units are sorted heaviest first
    const int64_t ct = blockIdx.x % nct, rt = u.x;
    const int64_t i0 = rt * kRM, j0 = ct * kRN;
    int64_t first, count, offset;
    tile_chunks(rt, K16, lower != 0, first, count, offset);
    // this unit: chunks u.y .. u.z - 1 of the row tile
    const float4* a_src = Ap + (offset + u.y) * (kRK * kRM);
    const float4* x_src = Xp + (ct * rows + (first + u.y) * kRK) * 32;
    count = u.z - u.y;
    const uint64_t limit = (uint64_t)wait_ns;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(saddr(&full[s]), 1);
            bar_init(saddr(&empty[s]), 8);       // one arrival per warp
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int64_t issued = 0;                          // thread 0: stages whose copies were issued
    auto issue = [&](int64_t q) {
        const int s = (int)(q % kStages);
        unsigned char* dst = smem + s * kStageBytes;
        bar_expect(saddr(&full[s]), kStageBytes);
        bulk_load(saddr(dst), a_src + q * (kRK * kRM), kABytes, saddr(&full[s]));
        bulk_load(saddr(dst + kABytes), x_src + q * (kRK * 32), kXBytes, saddr(&full[s]));
    };
    if (tid == 0)
        for (; issued < count && issued < kStages; ++issued) issue(issued);

    uint64_t hi[4][2], lo[4][2], mid[4][2], lo2[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) hi[r][c] = lo[r][c] = mid[r][c] = lo2[r][c] = 0ull;
    int stage = 0;
    bool ok = true;
    for (int64_t q = 0; q < count; ++q) {
        const int s = (int)(q % kStages);
        const uint32_t parity = (uint32_t)((q / kStages) & 1);
        if (!bar_wait(saddr(&full[s]), parity, abort, err, limit, true)) {
            ok = false;
            break;
        }
        const float4* As = reinterpret_cast<const float4*>(smem + s * kStageBytes);
        const float4* Xs = reinterpret_cast<const float4*>(smem + s * kStageBytes + kABytes);
#pragma unroll 4
        for (int l = 0; l < kRK; ++l) {
            const float4 x0 = Xs[l * 32 + tx], x1 = Xs[l * 32 + 16 + tx];
            const uint64_t xh[2] = {pk(x0.x, x0.y), pk(x1.x, x1.y)};
            const uint64_t xl[2] = {pk(x0.z, x0.w), pk(x1.z, x1.w)};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float4 av = As[l * kRM + ty + 16 * r];
                const uint64_t a2 = pk(av.x, av.y), na2 = pk(av.z, av.w);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (MODE == kPair) {                           // na2 holds (al, al)
                        const uint64_t p = mul2(a2, xh[c]);
                        const uint64_t e = fma2(a2, xh[c], p ^ kSign2);   // ah xh - p, exact
                        const uint64_t t = add2(hi[r][c], p);
                        const uint64_t bp = sub2(t, hi[r][c]);
                        const uint64_t er = add2(sub2(hi[r][c], sub2(t, bp)), sub2(p, bp));
                        hi[r][c] = t;
                        lo[r][c] = fma2(na2, xh[c], fma2(a2, xl[c], add2(lo[r][c], add2(er, e))));
                        continue;
                    }
                    if (MODE == kPlain) {
                        hi[r][c] = fma2(a2, xh[c], hi[r][c]);
                        continue;
                    }
                    const uint64_t np = mul2(na2, xh[c]);         // -p, p = fl(a xh)
                    const uint64_t e = fma2(a2, xh[c], np);        // a xh - p, exact
                    const uint64_t t = sub2(hi[r][c], np);         // hi + p
                    const uint64_t bp = sub2(t, hi[r][c]);
                    const uint64_t qq = add2(np, bp);              // -(p - bp)
                    const uint64_t er = sub2(sub2(hi[r][c], sub2(t, bp)), qq);
                    hi[r][c] = t;
                    if (MODE == kFull)
                        lo[r][c] = fma2(a2, xl[c], add2(lo[r][c], add2(er, e)));
                    else
                        lo[r][c] = add2(lo[r][c], add2(er, e));
                }
            }
        }
        __syncwarp();
        if (lane == 0) bar_arrive(saddr(&empty[s]));
        // refill this slot with stage q + kStages once every warp is done
        if (tid == 0 && issued < count) {
            if (!bar_wait(saddr(&empty[s]), parity, abort, err, limit, true)) {
                ok = false;
                break;
            }
            issue(issued++);
        }
        if (MODE != kPlain && ++stage == kFold) {
            stage = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    lo2[r][c] = add2(lo2[r][c], two_sum2(mid[r][c], lo[r][c]));
                    lo[r][c] = 0ull;
                }
        }
    }
    if (!ok || *abort) {
        // copies still in flight land before the CTA exits (waits of at
        // least 1 s, whatever the budget)
        if (tid == 0) {
            const uint64_t drain = limit > 1000000000ull ? limit : 1000000000ull;
            for (int64_t q = issued - kStages < 0 ? 0 : issued - kStages; q < issued; ++q)
                bar_wait(saddr(&full[q % kStages]), (uint32_t)((q / kStages) & 1), abort, err,
                         drain, false);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gi = i0 + ty + 16 * r;
        if (gi >= k) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float h[2], m[2], sm[2], t[2];
            upk(hi[r][c], h[0], h[1]);
            upk(mid[r][c], m[0], m[1]);
            upk(lo[r][c], sm[0], sm[1]);
            upk(lo2[r][c], t[0], t[1]);
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const int64_t j = j0 + tx + 32 * c + 16 * w;
                if (j >= n) continue;
                const double sum = (double)h[w] + ((double)m[w] + ((double)sm[w] + (double)t[w]));
                if (u.w < 0)
                    R[gi + j * ldr] = (B ? B[gi + j * ldb] : 0.0) - sum;
                else
                    part[((int64_t)u.w * n + j) * kRM + (ty + 16 * r)] = sum;
            }
        }
    }
}

// R := B - (sum of a row tile's pieces), for the row tiles cut into more
// than one piece: tiles[y] = (row tile, first partial slot, pieces).
__global__ void __launch_bounds__(256) combine_kernel(const int4* tiles, const double* part,
                                                      int64_t k, int64_t n, const double* B,
                                                      int64_t ldb, double* R, int64_t ldr) {
    const int4 t = tiles[blockIdx.y];
    const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (int64_t)kRM * n) return;
    const int64_t il = e % kRM, j = e / kRM, gi = (int64_t)t.x * kRM + il;
    if (gi >= k) return;
    double sum = 0.0;
    for (int p = 0; p < t.z; ++p) sum += part[((int64_t)(t.y + p) * n + j) * kRM + il];
    R[gi + j * ldr] = (B ? B[gi + j * ldb] : 0.0) - sum;
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
template <typename S, typename D>
cudaError_t launch_transpose(const S* src, int64_t lds, D* dst, int64_t ldd, int64_t rows,
                             int64_t cols, double scale, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    transpose_kernel<S, D><<<grid, 256, 0, s>>>(src, lds, dst, ldd, rows, cols, scale);
    return cudaGetLastError();
}
cudaError_t refine_transpose_f32(const float* src, int64_t lds, float* dst, int64_t ldd,
                                 int64_t rows, int64_t cols, cudaStream_t s) {
    return launch_transpose<float, float>(src, lds, dst, ldd, rows, cols, 1.0, s);
}
cudaError_t refine_transpose_f32_f64(const float* src, int64_t lds, double* dst, int64_t ldd,
                                     int64_t rows, int64_t cols, double scale, cudaStream_t s) {
    return launch_transpose<float, double>(src, lds, dst, ldd, rows, cols, scale, s);
}
cudaError_t refine_transpose_f64(const double* src, int64_t lds, double* dst, int64_t ldd,
                                 int64_t rows, int64_t cols, cudaStream_t s) {
    return launch_transpose<double, double>(src, lds, dst, ldd, rows, cols, 1.0, s);
}
cudaError_t refine_transpose_f64_scaled(const double* src, int64_t lds, double* dst, int64_t ldd,
                                        int64_t rows, int64_t cols, double scale,
                                        cudaStream_t s) {
    return launch_transpose<double, double>(src, lds, dst, ldd, rows, cols, scale, s);
}
cudaError_t refine_transpose_f64_f32(const double* src, int64_t lds, float* dst, int64_t ldd,
                                     int64_t rows, int64_t cols, cudaStream_t s) {
    return launch_transpose<double, float>(src, lds, dst, ldd, rows, cols, 1.0, s);
}
cudaError_t refine_scale_f64(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t m,
                             int64_t n, double scale, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    scale_f64_kernel<<<grid_for(m * n), kThreads, 0, s>>>(src, lds, dst, ldd, m, n, scale);
    return cudaGetLastError();
}
size_t refine_pack_a_bytes(int64_t k, bool lower) {
    if (k <= 0) return 0;
    const int64_t nrt = (k + kRM - 1) / kRM, K16 = (k + 15) / 16;
    int64_t first, count, offset;
    tile_chunks(nrt - 1, K16, lower, first, count, offset);
    return (size_t)(offset + count) * kABytes;
}
size_t refine_pack_x_bytes(int64_t k, int64_t n) {
    if (k <= 0 || n <= 0) return 0;
    return (size_t)((n + kRN - 1) / kRN) * (size_t)((k + 15) / 16 * 16) * 32 * 16;
}
cudaError_t refine_pack_a(const float* A, int64_t lda, int64_t k, bool lower, bool trans,
                          bool unit, void* Ap, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const int64_t nrt = (k + kRM - 1) / kRM, K16 = (k + 15) / 16;
    if (nrt > 65535 || 4 * K16 > 0x7fffffff) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(4 * K16), (unsigned)nrt);
    if (trans)
        pack_a_kernel<true><<<grid, 256, 0, s>>>(A, lda, k, lower, unit,
                                                 static_cast<float4*>(Ap));
    else
        pack_a_kernel<false><<<grid, 256, 0, s>>>(A, lda, k, lower, unit,
                                                  static_cast<float4*>(Ap));
    return cudaGetLastError();
}
cudaError_t refine_pack_a64(const double* A, int64_t lda, int64_t k, bool lower, bool trans,
                            bool unit, void* Ap, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const int64_t nrt = (k + kRM - 1) / kRM, K16 = (k + 15) / 16;
    if (nrt > 65535 || 4 * K16 > 0x7fffffff) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(4 * K16), (unsigned)nrt);
    if (trans)
        pack_a64_kernel<true><<<grid, 256, 0, s>>>(A, lda, k, lower, unit,
                                                   static_cast<float4*>(Ap));
    else
        pack_a64_kernel<false><<<grid, 256, 0, s>>>(A, lda, k, lower, unit,
                                                    static_cast<float4*>(Ap));
    return cudaGetLastError();
}
cudaError_t refine_pack_x(const double* X64, const float* X32, int64_t ldx, int64_t k,
                          int64_t n, void* Xp, cudaStream_t s, double scale) {
    if (k <= 0 || n <= 0) return cudaSuccess;
    const int64_t rows = (k + 15) / 16 * 16, nct = (n + kRN - 1) / kRN;
    if (nct > 65535 || rows > 0x7fffffff) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(rows / 8), (unsigned)nct);      // rows: a multiple of 16
    if (X64)
        pack_x_kernel<true><<<grid, 256, 0, s>>>(X64, nullptr, ldx, k, n, rows, scale,
                                                 static_cast<float4*>(Xp));
    else
        pack_x_kernel<false><<<grid, 256, 0, s>>>(nullptr, X32, ldx, k, n, rows, 1.0,
                                                  static_cast<float4*>(Xp));
    return cudaGetLastError();
}
void refine_plan_units(int64_t k, bool lower, std::vector<int4>& units,
                       std::vector<int4>& tiles, int64_t& slots) {
    units.clear();
    tiles.clear();
    slots = 0;
    if (k <= 0) return;
    const int64_t nrt = (k + kRM - 1) / kRM, K16 = (k + 15) / 16;
    for (int64_t rt = 0; rt < nrt; ++rt) {
        int64_t first, count, offset;
        tile_chunks(rt, K16, lower, first, count, offset);
        const int64_t pieces = (count + kUnitChunks - 1) / kUnitChunks;
        if (pieces == 1) {
            units.push_back(make_int4((int)rt, 0, (int)count, -1));
            continue;
        }
        tiles.push_back(make_int4((int)rt, (int)slots, (int)pieces, 0));
        for (int64_t p = 0; p < pieces; ++p) {
            const int64_t q0 = count * p / pieces, q1 = count * (p + 1) / pieces;
            units.push_back(make_int4((int)rt, (int)q0, (int)q1, (int)(slots + p)));
        }
        slots += pieces;
    }
    // heaviest first, ties by row tile, so the grid drains evenly
    std::stable_sort(units.begin(), units.end(), [](const int4& a, const int4& b) {
        return (a.z - a.y) > (b.z - b.y);
    });
}
template <int MODE>
cudaError_t launch_pipe(unsigned blocks, const void* Ap, const void* Xp, const int4* units,
                        double* part, int64_t rows, int64_t k, bool lower, const double* B,
                        int64_t ldb, double* R, int64_t ldr, int64_t n, int* err,
                        long long wait_ns, cudaStream_t s) {
    residual_pipe_kernel<MODE><<<blocks, 256, kPipeSmem, s>>>(
        static_cast<const float4*>(Ap), static_cast<const float4*>(Xp), units, part, rows, k,
        lower, B, ldb, R, ldr, n, err, wait_ns);
    return cudaGetLastError();
}
// Shared-memory limits of the residual kernels, for the current device
// (kernel attributes are per device; called from each device's set-up).
cudaError_t refine_configure() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(residual_pipe_kernel<kFull>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(residual_pipe_kernel<kSingle>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(residual_pipe_kernel<kPlain>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmem)) !=
        cudaSuccess)
        return e;
    return cudaFuncSetAttribute(residual_pipe_kernel<kPair>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmem);
}

cudaError_t refine_residual_packed(int mode, const void* Ap, const void* Xp, const void* units,
                                   int64_t nunits, const void* tiles, int64_t ntiles,
                                   double* part, int64_t k, bool lower, const double* B,
                                   int64_t ldb, double* R, int64_t ldr, int64_t n, int* err,
                                   long long wait_ns, cudaStream_t s) {
    if (k <= 0 || n <= 0) return cudaSuccess;
    if (mode < kFull || mode > kPair) return cudaErrorInvalidValue;
    const int64_t nct = (n + kRN - 1) / kRN, blocks = nunits * nct;
    if (blocks > 0x7fffffff || ntiles > 65535) return cudaErrorInvalidValue;
    const int64_t rows = (k + 15) / 16 * 16;
    const int4* u = static_cast<const int4*>(units);
    cudaError_t e;
    if (mode == kFull)
        e = launch_pipe<kFull>((unsigned)blocks, Ap, Xp, u, part, rows, k, lower, B, ldb, R, ldr,
                               n, err, wait_ns, s);
    else if (mode == kSingle)
        e = launch_pipe<kSingle>((unsigned)blocks, Ap, Xp, u, part, rows, k, lower, B, ldb, R,
                                 ldr, n, err, wait_ns, s);
    else if (mode == kPair)
        e = launch_pipe<kPair>((unsigned)blocks, Ap, Xp, u, part, rows, k, lower, B, ldb, R, ldr,
                               n, err, wait_ns, s);
    else
        e = launch_pipe<kPlain>((unsigned)blocks, Ap, Xp, u, part, rows, k, lower, B, ldb, R, ldr,
                                n, err, wait_ns, s);
    if (e != cudaSuccess || ntiles == 0) return e;
    const int64_t gx = (kRM * n + 255) / 256;
    if (gx > 0x7fffffff) return cudaErrorInvalidValue;
    combine_kernel<<<dim3((unsigned)gx, (unsigned)ntiles), 256, 0, s>>>(
        static_cast<const int4*>(tiles), part, k, n, B, ldb, R, ldr);
    return cudaGetLastError();
}
// The work-unit table of refine_plan_units built on the device (one thread:
// at most a few thousand entries), so an asynchronous caller needs no host
// copy. Row tiles are taken heaviest first (the triangle's long rows) rather
// than sorted by piece size; the order only balances the grid, the pieces
// and their partial slots (numbered in row-tile order) are the host plan's,
// so the residual is bitwise the same.
__global__ void plan_units_kernel(int64_t k, int lower, int4* units, int4* tiles) {
    const int64_t nrt = (k + kRM - 1) / kRM, K16 = (k + 15) / 16;
    int64_t nu = 0, nt = 0, slot = 0;
    // the split row tiles and their first slots, in row-tile order
    for (int64_t rt = 0; rt < nrt; ++rt) {
        int64_t first, count, offset;
        tile_chunks(rt, K16, lower != 0, first, count, offset);
        const int64_t pieces = (count + kUnitChunks - 1) / kUnitChunks;
        if (pieces > 1) {
            tiles[nt++] = make_int4((int)rt, (int)slot, (int)pieces, 0);
            slot += pieces;
        }
    }
    // units, long rows first (descending row tiles for a lower triangle):
    // the split tiles are then met in the reverse of the order above
    int64_t ti = lower ? nt - 1 : 0;
    for (int64_t v = 0; v < nrt; ++v) {
        const int64_t rt = lower ? nrt - 1 - v : v;
        int64_t first, count, offset;
        tile_chunks(rt, K16, lower != 0, first, count, offset);
        const int64_t pieces = (count + kUnitChunks - 1) / kUnitChunks;
        if (pieces == 1) {
            units[nu++] = make_int4((int)rt, 0, (int)count, -1);
            continue;
        }
        const int64_t s0 = tiles[ti].y;
        ti += lower ? -1 : 1;
        for (int64_t q = 0; q < pieces; ++q) {
            const int64_t q0 = count * q / pieces, q1 = count * (q + 1) / pieces;
            units[nu++] = make_int4((int)rt, (int)q0, (int)q1, (int)(s0 + q));
        }
    }
}

cudaError_t refine_plan_units_device(int64_t k, bool lower, void* units, void* tiles,
                                     cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    plan_units_kernel<<<1, 1, 0, s>>>(k, lower ? 1 : 0, static_cast<int4*>(units),
                                      static_cast<int4*>(tiles));
    return cudaGetLastError();
}
// sums[i] := row i's sum of |M| through kNormSlices partials at sums + m.
template <typename T>
void row_sums(const T* a, int64_t lda, int64_t m, int64_t n, double* sums, cudaStream_t s) {
    double* part = sums + m;
    row_abs_part_kernel<T><<<dim3((unsigned)((m + kThreads - 1) / kThreads), kNormSlices),
                             kThreads, 0, s>>>(a, lda, m, n, part);
    part_sum_kernel<<<(unsigned)((m + kThreads - 1) / kThreads), kThreads, 0, s>>>(part, m, sums);
}
// out[0] := ||D||_inf (rows) or max column sum (by_cols) of an FP32 array.
__global__ void __launch_bounds__(kThreads) col_abs_sum_f32_kernel(const float* a, int64_t lda,
                                                                   int64_t m, int64_t n,
                                                                   double* sums) {
    const int64_t j = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    double s = 0.0;
    for (int64_t i = lane; i < m; i += 32) s += fabs((double)a[i + j * lda]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sums[j] = s;
}
cudaError_t refine_norm_f32(const float* a, int64_t lda, int64_t m, int64_t n, bool by_cols,
                            double* sums, double* out, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    if (by_cols)
        col_abs_sum_f32_kernel<<<(unsigned)((n * 32 + kThreads - 1) / kThreads), kThreads, 0,
                                 s>>>(a, lda, m, n, sums);
    else
        row_sums<float>(a, lda, m, n, sums, s);
    max_kernel<<<1, kThreads, 0, s>>>(sums, by_cols ? n : m, out);
    return cudaGetLastError();
}
// out[0] := max column sum of |M| (m x n); sums: n doubles of scratch.
cudaError_t refine_norm_one(const double* a, int64_t lda, int64_t m, int64_t n, double* sums,
                            double* out, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    col_abs_sum_kernel<<<(unsigned)((n * 32 + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        a, lda, m, n, sums);
    max_kernel<<<1, kThreads, 0, s>>>(sums, n, out);
    return cudaGetLastError();
}
// out[0] := ||M||_inf; sums: (kNormSlices + 1) m doubles of scratch.
cudaError_t refine_norm_inf(const double* a, int64_t lda, int64_t m, int64_t n, double* sums,
                            double* out, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    row_sums<double>(a, lda, m, n, sums, s);
    max_kernel<<<1, kThreads, 0, s>>>(sums, m, out);
    return cudaGetLastError();
}
// out[0] := ||op(A)||_inf over the referenced triangle; sums: (kNormSlices +
// 1) k doubles of scratch.
cudaError_t refine_op_norm_inf(const float* a, int64_t lda, int64_t k, bool lower, bool trans,
                               bool unit, double* sums, double* out, cudaStream_t s) {
    if (k <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    if (trans) {
        op_col_abs_sum_kernel<<<(unsigned)((k * 32 + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            a, lda, k, lower, unit, sums);
    } else {
        double* part = sums + k;
        op_row_abs_part_kernel<<<dim3((unsigned)((k + 63) / 64), kNormSlices), kThreads, 0, s>>>(
            a, lda, k, lower, unit, part);
        part_sum_kernel<<<(unsigned)((k + kThreads - 1) / kThreads), kThreads, 0, s>>>(part, k,
                                                                                      sums);
    }
    max_kernel<<<1, kThreads, 0, s>>>(sums, k, out);
    return cudaGetLastError();
}
size_t refine_norm_scratch(int64_t k) { return (size_t)(kNormSlices + 1) * (size_t)k * 8; }

}  // namespace trx

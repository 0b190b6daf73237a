// Internal declarations shared by the trx CUDA sources.
//
// Every kernel works on one canonical form of the problem. The C-ABI layer
// (api.cu) maps each of the 16 side/uplo/trans/diag variants of Eq. 1-4
// (Section 2.1) onto it:
//
//   * M is a k x k LOWER triangular matrix read through signed strides,
//     M(i,l) = A[i*a_rs + l*a_cs]. op(A) is used directly for side 'L'
//     (op(A) X = alpha B) and op(A)^T for side 'R' (X op(A) = alpha B is
//     op(A)^T X^T = alpha B^T); an effectively-upper matrix is turned into a
//     lower one by reversing the index order (i -> k-1-i), which makes the
//     back substitution a forward one.
//   * C is the k x nrhs right-hand side / result, C(i,j) = C[i*c_rs + j*c_cs]
//     (B itself for side 'L', B^T for side 'R', row-reversed with M).
//
// So the recursion of Section 3.1 is written once, for the lower case:
// TRSM solves M11 X1 = C1, updates C2 -= M21 X1 (GEMM), solves M22 X2 = C2;
// TRMM forms C2 := M22 C2 + M21 C1 and C1 := M11 C1.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>
#include <vector>

namespace trx {

// ---- programmatic dependent launch ------------------------------------------
// Every kernel of a call's chain is launched with programmatic stream
// serialisation: it may start (and run its prologue) while the previous
// kernel finishes, and it waits for that kernel's results with
// pdl_wait() before its first read of data the chain produced. Launched
// without the attribute, both device calls are no-ops.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Whether launches on this host thread carry the attribute (the handle's
// TRX_OPT_PDL, set around each call).
bool& pdl_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename T>
struct Canon {
    int64_t k = 0;       // order of M
    int64_t nrhs = 0;    // right-hand sides (columns of C)
    const T* A = nullptr;
    int64_t a_rs = 0, a_cs = 0;
    T* C = nullptr;
    int64_t c_rs = 0, c_cs = 0;
    int unit = 0;        // diag == 'U': M(i,i) taken as 1, never read
};

// Split-BF16 operand planes of the tensor-core FP32 path (canonical order).
//   M planes: strictly-lower part of M, element (i, l) at i*ldm + l
//             (K-major A operand of the GEMM update).
//   Y planes: the GEMM's B operand, element (l, j) at j*ldy + l
//             (K-major): the solved X rows for TRSM, the original C for TRMM.
// An FP32 value x is carried as `slices` BF16 values:
//   x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)
// (each difference is exact in FP32). One slice keeps 8 significant bits
// (2^-9 relative), two about 17 (2^-17), three all 24 of FP32 (x0 + x1 + x2
// = x for normal x). The GEMM forms a product from the slice products whose
// weight is above FP32's unit roundoff: 1 term (x0 y0), 3 terms (+ x0 y1 +
// x1 y0) or 6 terms (+ x0 y2 + x1 y1 + x2 y0), FP32 accumulation.
struct Planes {
    __nv_bfloat16* m_hi = nullptr;
    __nv_bfloat16* m_lo = nullptr;
    __nv_bfloat16* m_lo2 = nullptr;
    int64_t ldm = 0;
    __nv_bfloat16* y_hi = nullptr;
    __nv_bfloat16* y_lo = nullptr;
    __nv_bfloat16* y_lo2 = nullptr;
    int64_t ldy = 0;
    int slices = 2;
};

// Product terms of a split (1, 3, 6) <-> slices per operand (1, 2, 3).
inline int slices_of_terms(int terms) { return terms == 1 ? 1 : terms == 6 ? 3 : 2; }
inline int terms_of_slices(int slices) { return slices == 1 ? 1 : slices == 3 ? 6 : 3; }

// The slices of x (above) into s0[o], s1[o], s2[o] for the first `slices`.
__device__ __forceinline__ void put_split(__nv_bfloat16* s0, __nv_bfloat16* s1,
                                          __nv_bfloat16* s2, int slices, int64_t o, float x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    s0[o] = h;
    if (slices > 1) {
        const float r = x - __bfloat162float(h);
        const __nv_bfloat16 l = __float2bfloat16_rn(r);
        s1[o] = l;
        if (slices > 2) s2[o] = __float2bfloat16_rn(r - __bfloat162float(l));
    }
}
// The slices of x as three values (unused ones zero).
__device__ __forceinline__ void split_slices(float x, int slices, __nv_bfloat16 (&v)[3]) {
    v[0] = __float2bfloat16_rn(x);
    const float r = x - __bfloat162float(v[0]);
    v[1] = slices > 1 ? __float2bfloat16_rn(r) : __float2bfloat16_rn(0.f);
    v[2] = slices > 2 ? __float2bfloat16_rn(r - __bfloat162float(v[1])) : __float2bfloat16_rn(0.f);
}
// Y-plane element o of the result x (solved rows, TRMM originals).
__device__ __forceinline__ void put_y(const Planes& pl, int64_t o, float x) {
    put_split(pl.y_hi, pl.y_lo, pl.y_lo2, pl.slices, o, x);
}

// ---- launchers (host) --------------------------------------------------------

// Leaf TRSM / TRMM (Section 3.3) on rows [r0 + t*b, r0 + t*b + b) for
// t = 0 .. nleaves-1 (clipped to k), all right-hand sides. alpha scales the
// right-hand side (TRSM) or the product (TRMM). With planes != nullptr the
// TRSM leaf also writes its solved rows into the Y planes.
template <typename T>
cudaError_t launch_leaf(bool trsm, const Canon<T>& p, int64_t r0, int b,
                        int64_t nleaves, T alpha, const Planes* planes,
                        int num_sms, cudaStream_t s);

// Largest leaf the kernels support; single TRSM leaves go up to
// kMaxBlockLeaf rows (the block-leaf kernel).
constexpr int kMaxLeaf = 128;
constexpr int kMaxBlockLeaf = 256;

// CUDA-core GEMM update on the canonical matrices:
//   C[rc+i, j] = beta*C[rc+i, j] + gamma * sum_l M(rc+i, rk+l) * Y[rk+l, j]
// for i < mlen, l < klen, j < nrhs, Y(l, j) = Y[l*y_rs + j*y_cs]. In the
// recursion Y is C itself and rows [rc, rc+mlen), [rk, rk+klen) are disjoint.
template <typename T>
cudaError_t launch_gemm_simt(const Canon<T>& p, const T* Y, int64_t y_rs, int64_t y_cs,
                             int64_t rc, int64_t mlen, int64_t rk, int64_t klen, T beta,
                             T gamma, cudaStream_t s, int num_sms = 152);

// B := 0 over an m x n column-major block (alpha == 0 quick return).
template <typename T>
cudaError_t launch_zero(T* B, int64_t m, int64_t n, int64_t ldb, cudaStream_t s);

// Split-BF16 planes of the strictly-lower part of M (rows/cols [0,k)).
// diag_block > 0 (a multiple of 64): the planes also carry zeros on and
// above the diagonal within each diag_block x diag_block diagonal block.
cudaError_t launch_convert_m(const Canon<float>& p, const Planes& pl, int diag_block,
                             cudaStream_t s);
// Split-BF16 planes of C rows [0,k), all columns (TRMM's original values).
cudaError_t launch_convert_y(const Canon<float>& p, const Planes& pl, cudaStream_t s);
// Y planes of C's rows [r0, r0 + rows) (r0 a multiple of 4).
cudaError_t launch_convert_y_rows(const Canon<float>& p, const Planes& pl, int64_t r0,
                                  int64_t rows, cudaStream_t s);
// Inverses of the full b x b diagonal blocks of M (b <= 128) as split
// planes at rows and columns [r0, r0 + b) of a row-major pair (leading
// dimension ld), zeros above each block's diagonal.
cudaError_t launch_invert_diag(const Canon<float>& p, int b, __nv_bfloat16* w_hi,
                               __nv_bfloat16* w_lo, __nv_bfloat16* w_lo2, int slices, int64_t ld,
                               cudaStream_t s, bool compact = false);
// Split-BF16 planes of a rows x cols block, src(r, c) = src[r*rs + c*cs];
// dst(r, c) at dst[r*ld + c] (row_major) or dst[c*ld + r] (otherwise).
cudaError_t launch_convert_rect(const float* src, int64_t rs, int64_t cs, int64_t rows,
                                int64_t cols, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                __nv_bfloat16* lo2, int slices, int64_t ld, bool row_major,
                                cudaStream_t s);

// Tensor-core GEMM update, one launch for a group of updates that write
// disjoint row ranges (FP32 in/out, split BF16 products of pl.slices slices
// per operand, FP32 accumulation in TMEM):
//   C[rc+i, j] = beta*C[rc+i, j] + gamma * sum_l M(rc+i, rk+l) Y(rk+l, j)
struct TcGemm {
    int64_t rc, mlen, rk, klen;
};
struct TcMaps;   // opaque: tensor maps over the planes (gemm_tc.cu)
int tc_maps_size();
cudaError_t tc_make_maps(const Planes& pl, int64_t k, int64_t nrhs, void* maps_out);
// Optional second output of a tensor-core GEMM: the split BF16 planes (as
// many slices as the operand planes) of result rows [row0, row1) (canonical rows), element (i, j) at
// j * ld + i, as the Y planes are laid out.
struct TcYOut {
    __nv_bfloat16* hi = nullptr;
    __nv_bfloat16* lo = nullptr;
    __nv_bfloat16* lo2 = nullptr;
    int64_t ld = 0, row0 = 0, row1 = 0;
};
cudaError_t launch_gemm_tc(const Canon<float>& p, const void* maps, int slices,
                           const TcGemm* gemms, int ngemms, float beta,
                           float gamma, int* err_word, long long wait_limit,
                           int num_sms, cudaStream_t s, bool diag_beta = false,
                           const TcYOut* yout = nullptr);
// Refined TRSM helpers (refine.cu): casts, residual, correction, norms.
cudaError_t refine_cast_f32_f64(const float* src, int64_t lds, double* dst, int64_t ldd, int64_t m,
                                int64_t n, double scale, cudaStream_t s);
cudaError_t refine_cast_f64_f32(const double* src, int64_t lds, float* dst, int64_t ldd, int64_t m,
                                int64_t n, cudaStream_t s);
cudaError_t refine_residual(const double* b, int64_t ldb, double* r, int64_t ldr, int64_t m,
                            int64_t n, cudaStream_t s);
cudaError_t refine_add(double* x, int64_t ldx, const float* d, int64_t ldd, int64_t m, int64_t n,
                       cudaStream_t s);
cudaError_t refine_norm_inf(const double* a, int64_t lda, int64_t m, int64_t n, double* sums,
                            double* out, cudaStream_t s);
cudaError_t refine_transpose_f32(const float* src, int64_t lds, float* dst, int64_t ldd,
                                 int64_t rows, int64_t cols, cudaStream_t s);
cudaError_t refine_transpose_f32_f64(const float* src, int64_t lds, double* dst, int64_t ldd,
                                     int64_t rows, int64_t cols, double scale, cudaStream_t s);
cudaError_t refine_transpose_f64(const double* src, int64_t lds, double* dst, int64_t ldd,
                                 int64_t rows, int64_t cols, cudaStream_t s);
cudaError_t refine_transpose_f64_scaled(const double* src, int64_t lds, double* dst, int64_t ldd,
                                        int64_t rows, int64_t cols, double scale,
                                        cudaStream_t s);
cudaError_t refine_transpose_f64_f32(const double* src, int64_t lds, float* dst, int64_t ldd,
                                     int64_t rows, int64_t cols, cudaStream_t s);
// dst := scale * src (m x n FP64, leading dimensions lds, ldd)
cudaError_t refine_scale_f64(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t m,
                             int64_t n, double scale, cudaStream_t s);
// The float-float residual: op(A) packed once (refine_pack_a_bytes),
// X packed per step (refine_pack_x_bytes; from FP64 X split into two
// floats, or from one FP32 plane), then R := B - op(A) X with mode 0
// (X = xh + xl) or 1 (one plane), error-free accumulation, 2 (one
// plane, plain FP32 accumulation) or 3 (A packed from FP64 as pairs by
// refine_pack_a64, X = xh + xl). R may be B; B null reads as zero
// (R := -op(A) X: the float-float TRMM). Waits bounded by wait_ns; on
// timeout *err := TRX_ERR_TIMEOUT and R is not written.
size_t refine_pack_a_bytes(int64_t k, bool lower);
size_t refine_pack_x_bytes(int64_t k, int64_t n);
cudaError_t refine_pack_a(const float* A, int64_t lda, int64_t k, bool lower, bool trans,
                          bool unit, void* Ap, cudaStream_t s);
// op(A) of FP64 data as float pairs (ah, al), for mode 3 (A and X both
// pairs: the residual of FP64 data).
cudaError_t refine_pack_a64(const double* A, int64_t lda, int64_t k, bool lower, bool trans,
                            bool unit, void* Ap, cudaStream_t s);
// X64 (times `scale`, in FP64, before the split) or X32 packed.
cudaError_t refine_pack_x(const double* X64, const float* X32, int64_t ldx, int64_t k,
                          int64_t n, void* Xp, cudaStream_t s, double scale = 1.0);
// Work units of the residual (row-tile pieces, heaviest first) and the row
// tiles whose pieces refine_residual_packed combines; slots = partial
// blocks of 64 x n doubles the pieces write.
void refine_plan_units(int64_t k, bool lower, std::vector<int4>& units, std::vector<int4>& tiles,
                       int64_t& slots);
// The same table built on the device (units, then tiles; the counts and
// slots are refine_plan_units's): no host copy on the asynchronous path.
cudaError_t refine_plan_units_device(int64_t k, bool lower, void* units, void* tiles,
                                     cudaStream_t s);
cudaError_t refine_residual_packed(int mode, const void* Ap, const void* Xp, const void* units,
                                   int64_t nunits, const void* tiles, int64_t ntiles,
                                   double* part, int64_t k, bool lower, const double* B,
                                   int64_t ldb, double* R, int64_t ldr, int64_t n, int* err,
                                   long long wait_ns, cudaStream_t s);
cudaError_t refine_norm_f32(const float* a, int64_t lda, int64_t m, int64_t n, bool by_cols,
                            double* sums, double* out, cudaStream_t s);
cudaError_t refine_norm_one(const double* a, int64_t lda, int64_t m, int64_t n, double* sums,
                            double* out, cudaStream_t s);
size_t refine_norm_scratch(int64_t k);   // bytes refine_op_norm_inf needs at `sums`
cudaError_t refine_op_norm_inf(const float* a, int64_t lda, int64_t k, bool lower, bool trans,
                               bool unit, double* sums, double* out, cudaStream_t s);

// A BF16 plane (inner index contiguous, leading dimension ld elements) as a
// 2-D tensor map with boxes of 32 x box_outer and the 64-byte swizzle (map:
// a CUtensorMap, 64-byte aligned).
bool tc_encode_bf16_2d(void* map, void* base, uint64_t inner, uint64_t outer, uint64_t ld,
                       uint32_t box_outer);

// Device-scheduled TRSM for few right-hand sides (trsm_dag.cu): applies to
// the canonical lower solve when the order is a multiple of kDagBlock.
// w: the inverted diagonal blocks as compact planes (row r of the k x 128
// plane holds row r of its block's inverse); flags: blocks * panels ints
// and a task counter after them (zeroed by the launch).
constexpr int kDagBlock = 128, kDagPanel = 64;
size_t dag_flag_bytes(int64_t k, int64_t nrhs);
cudaError_t launch_trsm_dag(const Canon<float>& p, const Planes& pl, __nv_bfloat16* const w[3],
                            float alpha, int* flags, int* err, long long wait_ns, int num_sms,
                            cudaStream_t s);

// FP32 TRSM with few right-hand sides as one persistent CUDA-core launch
// (thin.cu): 64-row blocks x 16-column panels, left-looking, flags between
// tasks. scratch: thin_scratch_bytes ints, zeroed by the launch itself.
constexpr int kThinBlock = 64, kThinPanel = 16;
size_t thin_scratch_bytes(int64_t k, int64_t nrhs);
// withhold: test hook, block row 0 is never published, so the bounded waits
// of the blocks after it run out (TRX_ERR_TIMEOUT).
cudaError_t launch_thin_trsm(const Canon<float>& c, float alpha, int* scratch, int* err,
                             long long wait_ns, int num_sms, cudaStream_t s,
                             bool withhold = false);
// The thin TRMM (thin.cu): C := alpha M C in one launch after a packing
// pass of C's original rows (no waits); scratch: thin_trmm_scratch_bytes.
size_t thin_trmm_scratch_bytes(int64_t k, int64_t nrhs);
cudaError_t launch_thin_trmm(const Canon<float>& c, float alpha, int* scratch, int num_sms,
                             cudaStream_t s);

// K granularity the tensor-core GEMM needs (klen and rk multiples of this).
constexpr int kTcKQuantum = 64;

}  // namespace trx

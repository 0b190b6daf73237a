/*
 * trx — recursive triangular matrix multiply (TRMM) and triangular solve
 * (TRSM) for NVIDIA GB300 (sm_103a). C ABI.
 *
 * The operations are those of Section 2.1 of "Toward Portable GPU Performance:
 * Julia Recursive Implementation of TRMM and TRSM" (arXiv 2504.13821):
 *
 *   TRMM   B := alpha * op(A) * B      side = 'L'   (Eq. 1)
 *          B := alpha * B * op(A)      side = 'R'   (Eq. 2)
 *   TRSM   op(A) * X = alpha * B       side = 'L'   (Eq. 3)
 *          X * op(A) = alpha * B       side = 'R'   (Eq. 4), X overwrites B
 *
 * computed by the recursive scheme of Section 3.1: A is split into A11, A21,
 * A22, the recursion descends on the diagonal blocks down to a leaf tile
 * solved/multiplied in shared memory (Section 3.3) and the off-diagonal
 * blocks become in-place GEMM updates (e.g. B2 -= A21 * X1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Storage is BLAS column-major: element (i,j) of A is A[i + j*lda], of B is
 *   B[i + j*ldb]. B is m x n; A is k x k with k = m (side 'L') or k = n
 *   (side 'R'). Both pointers are DEVICE pointers on the handle's device,
 *   owned by the caller. A is read only; only its uplo triangle is read and,
 *   with diag = 'U', not its diagonal (taken as 1). B is overwritten.
 *   A must not overlap B (undefined result, as in BLAS).
 * - side in {'L','R'}, uplo in {'L','U'}, transa in {'N','T','C'} ('C' means
 *   'T' for real data), diag in {'N','U'}; case-insensitive.
 * - The call is asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *   default stream) and returns once the work is enqueued. It allocates no
 *   device memory: the tensor-core FP32 path uses the handle's workspace.
 * - Return codes: 0 on success; -i if the i-th BLAS argument is illegal
 *   (side=1, uplo=2, transa=3, diag=4, m=5, n=6, alpha=7, A=8, lda=9, B=10,
 *   ldb=11), checked before anything else and before the handle is used;
 *   a positive TRX_ERR_* code otherwise. On any error nothing is enqueued.
 * - m == 0 or n == 0 returns at once. alpha == 0 sets B to zero and does not
 *   read A (the BLAS quick return). A zero on a non-unit diagonal is not
 *   checked; Inf/NaN propagate.
 * - A handle is not thread-safe: calls sharing one handle must be issued from
 *   one host thread, and calls on different streams that share one handle
 *   must not overlap on the device (they share its workspace).
 *
 * Entry points
 * ------------
 *   handle and workspace   trx_create, trx_destroy, trx_set_workspace,
 *                          trx_workspace_size
 *   the four operations    trx_strsm, trx_dtrsm, trx_strmm, trx_dtrmm
 *   the GEMM update alone  trx_sgemm_update
 *   batched problems       trx_batched, trx_{s,d}{trsm,trmm}_batched,
 *                          trx_batch_create / run / destroy,
 *                          trx_batched_autotune, trx_batched_get_tuning /
 *                          set_tuning
 *   refined FP32 TRSM      trx_strsm_refined (FP64-accurate result),
 *                          trx_strsm_refined_async (fixed corrections)
 *   prepared factors       trx_sfactor_create / update, trx_factor_destroy,
 *                          trx_strsm_factor, trx_strmm_factor
 *   host triangle upload   trx_copy_triangle_h2d
 *   request server         trx_server_create / register_factor /
 *                          release_factor / submit / submit_refined / poll /
 *                          pending / wait / destroy
 *   allocation-free TRSM   trx_strsm_noalloc, trx_noalloc_check_error
 *   options, diagnostics   trx_set_option, trx_get_option, trx_get_profile,
 *                          trx_check_device_error, trx_error_string,
 *                          trx_last_error_detail, trx_debug_plan, trx_version
 *   peak-rate probes       trx_peak_probe
 */
#ifndef TRX_H_
#define TRX_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct trx_handle_s* trx_handle_t;

/* Positive error codes (negative codes are BLAS argument positions). */
enum {
    TRX_SUCCESS = 0,
    TRX_ERR_HANDLE = 1,        /* null or destroyed handle                  */
    TRX_ERR_CUDA = 2,          /* a CUDA runtime/driver call failed         */
    TRX_ERR_WORKSPACE = 3,     /* workspace missing or smaller than needed  */
    TRX_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up        */
    TRX_ERR_DEVICE = 5,        /* device is not sm_103 (GB300)              */
    TRX_ERR_ALLOC = 6,         /* host or device allocation failed          */
    TRX_ERR_INVALID_VALUE = 7  /* bad option or option value                */
};

/* Options for trx_set_option(). */
enum {
    TRX_OPT_LEAF = 1,      /* leaf cutoff b (Section 3.1 "chosen threshold"):
                              16, 32, 64, 128 or 256 (256: TRSM block
                              leaves; TRMM stops at 128); 0 = automatic
                              (default: 128 for FP32 TRSM, else 64)        */
    TRX_OPT_GEMM = 2,      /* FP32 GEMM-update engine: 0 automatic, 1 CUDA
                              cores (FP32 FMA), 2 tensor cores (tcgen05,
                              split BF16 products of TRX_OPT_SPLIT terms,
                              FP32 accumulation)                            */
    TRX_OPT_GRAPH = 3,     /* 1 (default): replay the launch chain as a
                              cached CUDA graph; 0: launch directly         */
    TRX_OPT_PROFILE = 4,   /* 1: time every launch with CUDA events and
                              accumulate into trx_profile_t (launches
                              directly, no graph); 0 (default): off        */
    TRX_OPT_WAIT_LIMIT = 5,/* nanoseconds a device-side wait may spin
                              before it gives up and the launch reports
                              TRX_ERR_TIMEOUT (default 2e9, minimum 1000) */
    TRX_OPT_PANELS = 7,    /* TRSM column-panel branches (right-hand sides
                              are independent; each panel runs its own
                              recursion chain on its own stream, all in one
                              graph): 1..4; 0 = automatic (default: 1)    */
    TRX_OPT_PDL = 6,       /* 1: launch the chain's kernels with
                              programmatic dependent launch, so each one's
                              prologue overlaps the previous one's tail;
                              0 (default): plain stream order              */
    TRX_OPT_TRMM_DENSE = 8,/* FP32 TRMM on the tensor-core path: leaves of
                              this many rows (64 .. 2048, a power of two)
                              formed in one grouped GEMM launch over the
                              diagonal blocks (the block's strictly-lower
                              part on the tensor cores in 128-row tiles,
                              each tile's K range ending at its last row;
                              the diagonal term in FP32 in the epilogue),
                              replacing the leaf kernel and the recursion
                              levels below that size;
                              -1 off; 0 = automatic (default: 1024 rows when
                              the order is at least 1024 and TRX_OPT_LEAF
                              is automatic, else off)                     */
    TRX_OPT_RESIDUAL = 9,  /* residual of trx_strsm_refined: 0 (automatic)
                              or 2: float-float on the FP32 pipes (pairs of
                              floats, exact product split and two-sum,
                              about 2^-46 relative, 2^-44 for adversarial
                              rows); 1: the library's FP64
                              TRMM on an FP64 copy of A (FP64 pipe);
                              3: FP32-grade on the tensor cores, op(A) times
                              X rounded to FP32 by the library's FP32 TRMM
                              with the 6-term split, then alpha B minus it in
                              FP64 (a few units of 2^-24 of |op(A)||X|: for
                              targets down to about 1e-7; the handle's
                              workspace must hold the 6-term planes)       */
    TRX_OPT_TRSM_TC_LEAF = 10,/* FP32 TRSM on the tensor-core path, leaves of
                              64 or 128 rows: 1 = each leaf as one GEMM,
                              X = alpha inv(A_ii) B_i, with the diagonal
                              blocks inverted in FP32 (substitution) once
                              per call (per update of a prepared factor) and
                              the leaf's input planes written by the
                              preceding update's epilogue; -1 or 0
                              (default): the substitution leaf kernels      */
    TRX_OPT_SPLIT = 11,    /* FP32 on the tensor cores: product terms of the
                              BF16 split, each FP32 operand carried as 1, 2
                              or 3 BF16 slices (x0 = bf16(x), x1 =
                              bf16(x - x0), x2 = bf16(x - x0 - x1)):
                              6 = three slices, products x0y0 + x0y1 +
                              x1y0 + x0y2 + x1y1 + x2y0 (every slice
                              product above 2^-24: FP32-grade);
                              3 = two slices, x0y0 + x0y1 + x1y0 (about
                              2^-16 relative per product);
                              1 = one slice, x0y0 (about 2^-8);
                              FP32 accumulation in every case; 0 =
                              automatic (default: 6). trx_get_option
                              reads back the terms in use. A prepared
                              factor keeps the split it was created with. */
    TRX_OPT_FP64_TRSM = 12,/* trx_dtrsm's engine: 0 (default) the recursive
                              FP64 solve (CUDA-core DFMA updates); n in
                              1..16: for orders of at least 64 (below, the
                              recursive solve) the mixed form, the FP32 solve on
                              fl32(A) then n corrections with the residual
                              alpha B - op(A) X in float-float arithmetic on
                              the FP32 pipes (A and X as float pairs, about
                              2^-44 of |op(A)||X|) and FP32 correction solves,
                              X accumulated in FP64 (asynchronous, as
                              trx_strsm_refined_async; uses the handle's
                              refinement scratch). The pairs assume entries
                              inside FP32's exponent range (about 1e-30 ..
                              1e38 in magnitude); outside it use 0         */
    TRX_OPT_CHECKED = 13,  /* 1: check every call's launch plan before
                              enqueueing it (every leaf block, GEMM row and K
                              range inside the order of A, each update's K
                              range before its rows, tensor-core K ranges on
                              whole K steps); a violation returns
                              TRX_ERR_INVALID_VALUE with the reason in
                              trx_last_error_detail and enqueues nothing.
                              trx_debug_plan always checks. 0 (default) off */
    TRX_OPT_NVTX = 14,     /* 1: an NVTX range around each launch step
                              ("trx leaf ...", "trx gemm ...": kind and row
                              ranges) for an attached profiler; with graph
                              replay (TRX_OPT_GRAPH 1) they mark the capture
                              only, so pair it with TRX_OPT_GRAPH 0 or
                              TRX_OPT_PROFILE 1. 0 (default) off          */
    TRX_OPT_TRSM_DAG = 15, /* FP32 TRSM on the tensor-core path with the
                              order a multiple of 128 (at least 256): 1 =
                              one persistent device-scheduled launch in place
                              of the recursion's launch chain (128-row blocks
                              x 64-column panels taken in order from a
                              counter; a block's off-diagonal products start
                              as soon as the blocks it needs are published,
                              its diagonal solve is a product with the
                              block's inverse, made once per call; bounded
                              waits); -1 = the recursive chain; 0 =
                              automatic (default: the device-scheduled solve
                              with at most 1024 right-hand sides). Needs the
                              workspace trx_workspace_size reports (planes
                              + inverses + flags)                         */
    TRX_OPT_FP64_TRMM = 16,/* trx_dtrmm's engine: 0 (default) the recursive
                              FP64 product (CUDA-core DFMA updates); 1 = for
                              orders of at least 64, the whole product
                              alpha op(A) B in one float-float pass on the
                              FP32 pipes (A and B as float pairs, about
                              2^-44 of |op(A)||B|, inside 8 k u of FP64 for
                              k >= 64; the refinement residual's kernel with
                              a zero B). Entries must lie inside FP32's
                              exponent range (as for TRX_OPT_FP64_TRSM).
                              Uses the handle's refinement scratch        */
    TRX_OPT_THIN = 17,     /* FP32 TRSM and TRMM with few right-hand sides:
                              1 = one persistent CUDA-core launch in place of
                              the recursion (64-row blocks x 16-column
                              panels; TRSM left-looking: each block row adds
                              its products with the published blocks before
                              it, then multiplies by its diagonal block's
                              inverse, made by substitution in FP32, blocks
                              published as tagged words, bounded waits;
                              TRMM: every block row's sum from a packed copy
                              of B, long rows in pieces added in a fixed
                              order, no waits; FP32 FMA, no operand split);
                              -1 = the recursion; 0 = automatic (default:
                              order above 256; TRSM with at most 64
                              right-hand sides, or at most 256 while order
                              x right-hand sides <= 2^21 and the thin
                              leaves of TRX_OPT_THIN_LEAF do not apply;
                              TRMM with at most 32). Its scratch lives in a
                              handle buffer grown on first use (cached
                              graphs are dropped when it grows)           */
    TRX_OPT_TEST_WITHHOLD = 18, /* test hook for the bounded waits: 1 = the
                              thin TRSM (TRX_OPT_THIN) never publishes its
                              first block row, so the waits of the blocks
                              after it run out and the call leaves
                              TRX_ERR_TIMEOUT for trx_check_device_error
                              (B is then not the solution). 0 (default)  */
    TRX_OPT_THIN_LEAF = 19 /* FP32 TRSM on the tensor-core path: the
                              recursion stops at leaves of this many rows
                              (256 .. 8192, a multiple of 128) and each
                              leaf runs as the thin solve of TRX_OPT_THIN
                              (one persistent CUDA-core launch) on its own
                              rows, its result converted to the GEMM
                              operand planes for the updates after it;
                              -1 = off; 0 = automatic (default: from
                              order 4096, leaves of 2048 rows for 65 .. 256
                              right-hand sides (129 .. 256 below order
                              8192), of 1024 rows for 257 .. 1024; off
                              when TRX_OPT_LEAF sets the cutoff). Where
                              this and an automatic whole-call
                              thin solve (TRX_OPT_THIN 0) both apply, the
                              leaves are taken; a forced one (TRX_OPT_THIN
                              1) wins over them. Shares TRX_OPT_THIN's
                              scratch buffer                              */
};

/* Kernel classes reported by trx_get_profile(). */
enum {
    TRX_KERNEL_LEAF_TRSM = 0,
    TRX_KERNEL_LEAF_TRMM = 1,
    TRX_KERNEL_GEMM_TC = 2,    /* tcgen05 GEMM update                     */
    TRX_KERNEL_GEMM_SIMT = 3,  /* CUDA-core GEMM update                   */
    TRX_KERNEL_CONVERT = 4,    /* FP32 -> split BF16 operand planes       */
    TRX_KERNEL_OTHER = 5,      /* scale / zero                            */
    TRX_KERNEL_CLASSES = 6
};

/* Per-class accumulated device time (CUDA events around each launch on the
 * call's stream), launch count and algorithmic work: flops = 2*M*N*K for a
 * GEMM update and the exact multiply-add count for a leaf; bytes = the
 * minimum bytes a launch must move (operands read once, outputs written
 * once). Only filled while TRX_OPT_PROFILE is 1. */
typedef struct {
    double ms[TRX_KERNEL_CLASSES];
    double flops[TRX_KERNEL_CLASSES];
    double bytes[TRX_KERNEL_CLASSES];
    int64_t launches[TRX_KERNEL_CLASSES];
} trx_profile_t;

/* Create a handle on CUDA device `device` (that device becomes current for
 * the calling thread). workspace_bytes > 0 makes the handle allocate and own
 * a workspace of that size; 0 allocates none (see trx_set_workspace).
 * Returns TRX_ERR_DEVICE if the device is not compute capability 10.3. */
int trx_create(trx_handle_t* handle, int device, size_t workspace_bytes);

/* Destroy a handle: synchronises the device, frees what the handle owns
 * (its workspace, cached graphs, events). NULL is accepted. */
int trx_destroy(trx_handle_t handle);

/* Give the handle a caller-owned device workspace (replaces, and frees, any
 * workspace the handle owned). The memory must stay valid until it is
 * replaced or the handle destroyed. ptr must be 256-byte aligned. */
int trx_set_workspace(trx_handle_t handle, void* ptr, size_t bytes);

/* Bytes of workspace a call needs. elem_bytes is 4 (FP32) or 8 (FP64);
 * op is 'S' (TRSM) or 'M' (TRMM), for which side/m/n are the call's; 'Y' for
 * a call on a prepared factor (TRSM or TRMM, same side/m/n); or 'G' for a
 * tensor-core trx_sgemm_update, with m = M + K and n = N (side 'L').
 * Depends on the handle's options (the CUDA-core and FP64 paths need none,
 * except FP64 TRSM on the mixed engine, TRX_OPT_FP64_TRSM, which needs the
 * FP32 solve's).
 * Returns 0 and sets *bytes, or an argument code as for the compute calls. */
int trx_workspace_size(trx_handle_t handle, char op, char side, int64_t m,
                       int64_t n, int elem_bytes, size_t* bytes);

/* TRSM (Eq. 3-4), FP32 and FP64. B (m x n) is overwritten by X. */
int trx_strsm(trx_handle_t handle, char side, char uplo, char transa,
              char diag, int64_t m, int64_t n, float alpha, const float* A,
              int64_t lda, float* B, int64_t ldb, void* stream);
int trx_dtrsm(trx_handle_t handle, char side, char uplo, char transa,
              char diag, int64_t m, int64_t n, double alpha, const double* A,
              int64_t lda, double* B, int64_t ldb, void* stream);

/* TRMM (Eq. 1-2), FP32 and FP64. B (m x n) is overwritten by the product. */
int trx_strmm(trx_handle_t handle, char side, char uplo, char transa,
              char diag, int64_t m, int64_t n, float alpha, const float* A,
              int64_t lda, float* B, int64_t ldb, void* stream);
int trx_dtrmm(trx_handle_t handle, char side, char uplo, char transa,
              char diag, int64_t m, int64_t n, double alpha, const double* A,
              int64_t lda, double* B, int64_t ldb, void* stream);

/* The recursion's off-diagonal step on its own (Section 3.1, e.g.
 * B2 := B2 - A21 * X1), FP32, column-major device arrays:
 *   C := beta * C + gamma * A * Y,  A M x K, Y K x N, C M x N (C must not
 *   overlap A or Y).
 * engine 1: CUDA cores (FP32 FMA); engine 2: tensor cores (3-term split
 * BF16 products, FP32 accumulation; K must be a multiple of 64 and the
 * handle's workspace at least trx_workspace_size('G', 'L', M + K, N)).
 * Returns 0, -i for an illegal i-th argument (handle = 1, M = 2, N = 3,
 * K = 4, beta = 5, gamma = 6, A = 7, lda = 8, Y = 9, ldy = 10, C = 11,
 * ldc = 12, engine = 13), or a TRX_ERR_* code. Asynchronous on stream. */
int trx_sgemm_update(trx_handle_t handle, int64_t M, int64_t N, int64_t K,
                     float beta, float gamma, const float* A, int64_t lda,
                     const float* Y, int64_t ldy, float* C, int64_t ldc,
                     int engine, void* stream);

/* ---- batched uneven problems (one persistent launch) --------------------
 * One TRSM or TRMM of the kind above per entry; all entries of a call share
 * the element type. Pointers are device pointers; problems must not overlap
 * each other's B. Orders k (m for side 'L', n for side 'R') up to
 * TRX_BATCH_MAX_K; larger problems belong to trx_?trsm / trx_?trmm. */
#define TRX_BATCH_MAX_K 512

typedef struct {
    char op;                 /* 'S' TRSM, 'M' TRMM                         */
    char side, uplo, transa, diag;
    int64_t m, n;
    double alpha;            /* converted to the element type              */
    const void* A;
    int64_t lda;
    void* B;
    int64_t ldb;
} trx_problem_t;

/* Run `count` problems (host array) in one persistent launch: problems are
 * mapped to the library's canonical form, sorted largest first and taken by
 * the CTAs from a shared counter; the launch is replayed from a cached CUDA
 * graph. elem_bytes is 4 (FP32) or 8 (FP64). Returns 0, or
 * TRX_ERR_INVALID_VALUE if a problem is malformed or too large (the detail
 * string names it), or another TRX_ERR_* code; nothing is enqueued then.
 * The handle keeps (and grows on demand) a device descriptor array and a
 * pinned host staging buffer for the batch; a call waits for the previous
 * batched call's descriptor upload before reusing the staging buffer. */
int trx_batched(trx_handle_t handle, int elem_bytes, int64_t count,
                const trx_problem_t* problems, void* stream);

/* The same with one operation and element type per call: every problem's
 * op must be 'S' (the trsm entry points) or 'M' (the trmm ones), else
 * TRX_ERR_INVALID_VALUE and nothing is enqueued; s = FP32, d = FP64. */
int trx_strsm_batched(trx_handle_t handle, int64_t count, const trx_problem_t* problems,
                      void* stream);
int trx_dtrsm_batched(trx_handle_t handle, int64_t count, const trx_problem_t* problems,
                      void* stream);
int trx_strmm_batched(trx_handle_t handle, int64_t count, const trx_problem_t* problems,
                      void* stream);
int trx_dtrmm_batched(trx_handle_t handle, int64_t count, const trx_problem_t* problems,
                      void* stream);

/* Refined FP32 TRSM (the precision form): the FP32 solve of trx_strsm, then
 * iterative refinement towards an FP64-accurate X: the residual
 * R = alpha B - op(A) X with more than FP32 precision (TRX_OPT_RESIDUAL:
 * float-float on the FP32 pipes by default, or FP64 arithmetic), a
 * correction op(A) D = R (or D op(A) = R) solved in FP32 on the same
 * recursive path, X += D in FP64 (float-float: R is then updated as
 * R - op(A) D, with plain FP32 accumulation once sqrt(k) 2^-24 ||D|| /
 * ||X|| is below tol / 8; FP64: recomputed from X), until the normwise
 * backward error
 * ||R|| / (||op(A)|| ||X||) (infinity norms) is at most tol, max_iter
 * corrections were made, or a correction did not lower it. A (k x k) and
 * B (m x n) are FP32 device arrays as in trx_strsm, B is not modified;
 * X (m x n, FP64, leading dimension ldx) is the result. Synchronous: it
 * reads the residual norm back after every step. Needs the workspace of
 * trx_strsm (trx_workspace_size 'S') and allocates its own scratch on the
 * handle (about 36 m n bytes, plus 8 k^2 for the FP64 residual; kept for later
 * calls). info (may be NULL): corrections made, the final residual norm
 * and backward error (of the updated residual on the float-float path: it
 * leaves out the first residual's own rounding, about 2^-46 relative), and
 * the backward error of the plain FP32 solve.
 * Returns -i for an illegal i-th argument of this call (side 2, uplo 3,
 * transa 4, diag 5, m 6, n 7, alpha 8, A 9, lda 10, B 11, ldb 12, X 13,
 * ldx 14, max_iter < 0: 15, tol < 0 or NaN: 16), or a TRX_ERR_* code. (The
 * paper's base solve and GEMM updates are the FP32 steps; the refinement
 * loop around them is this library's.) */
typedef struct {
    int iterations;                 /* corrections applied                  */
    double residual_norm;           /* ||alpha B - op(A) X||_inf at the end  */
    double backward_error;          /* ||R|| / (||op(A)|| ||X||) at the end  */
    double initial_backward_error;  /* the same for the plain FP32 solve     */
} trx_refine_info_t;
int trx_strsm_refined(trx_handle_t handle, char side, char uplo, char transa, char diag,
                      int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
                      const float* B, int64_t ldb, double* X, int64_t ldx, int max_iter,
                      double tol, trx_refine_info_t* info, void* stream);

/* Refined FP32 TRSM with a fixed number of corrections and no host
 * read-back (for callers that must not synchronise, e.g. a request server):
 * the FP32 solve, then `corrections` (0..16) steps of the float-float
 * residual R = alpha B - op(A) X (from X each time), the FP32 correction
 * solve op(A) D = R and X += D in FP64, all enqueued on `stream`. Arguments
 * as trx_strsm_refined without max_iter/tol/info (corrections is argument
 * 15). Nothing is read back: a timed-out device wait shows in
 * trx_check_device_error. The refinement scratch (as trx_strsm_refined's)
 * is grown on the handle when a call needs more than any call before it;
 * that growth synchronises the stream, so a caller that must never block
 * makes one call of its largest size first. Needs the workspace of
 * trx_strsm. Two corrections reach an FP64-level backward error for
 * condition numbers up to about 1e4 (each one gains about
 * log2(1 / (kappa 2^-24)) bits). */
int trx_strsm_refined_async(trx_handle_t handle, char side, char uplo, char transa, char diag,
                            int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
                            const float* B, int64_t ldb, double* X, int64_t ldx,
                            int corrections, void* stream);

/* Prepared FP32 factor (no counterpart in the paper: an interface for
 * callers that solve with or multiply by one triangle many times). The
 * tensor-core path multiplies split-BF16 planes of the canonical triangle
 * (Section 3.1's off-diagonal blocks of op(A), or of op(A)^T for side 'R');
 * a factor makes them once and every trx_s{trsm,trmm}_factor call on it skips
 * the conversion. The factor keeps A (device pointer, lda) and reads it in
 * every call (base kernels, TRMM's diagonal): A must stay valid, and after
 * A's contents change trx_sfactor_update must run before the next call.
 *
 * trx_sfactor_create: side/uplo/transa/diag/A/lda as in trx_strsm with k the
 * order of A; enqueues the conversion on stream and returns; the planes are
 * owned by the factor (device memory, 4 k^2 bytes when k > 128, none
 * otherwise). Returns -i for an illegal i-th argument of this call (side 2,
 * uplo 3, transa 4, diag 5, k 6, A 7, lda 8), TRX_ERR_HANDLE,
 * TRX_ERR_ALLOC, TRX_ERR_CUDA. trx_sfactor_update re-converts from A (the
 * same layout; the pointer may change; -3 if A is NULL with k > 0) on
 * stream. trx_strsm_factor / trx_strmm_factor: B := X or alpha op(A) B as
 * trx_strsm / trx_strmm with the factor's side/uplo/transa/diag/A; nrhs is
 * the number of right-hand sides (n for side 'L', m for side 'R'); B is
 * k x nrhs (side 'L') or nrhs x k (side 'R'), column-major, leading
 * dimension ldb; -3 for nrhs < 0, -5 for a NULL B, -6 for a bad ldb; the
 * workspace needs only the Y planes (trx_workspace_size with op 'Y').
 * trx_factor_destroy synchronises the device and frees the factor (NULL is
 * accepted). A factor belongs to the device of the handle that made it. */
typedef struct trx_factor_s* trx_factor_t;
int trx_sfactor_create(trx_handle_t handle, char side, char uplo, char transa, char diag,
                       int64_t k, const float* A, int64_t lda, void* stream,
                       trx_factor_t* factor);
int trx_sfactor_update(trx_handle_t handle, trx_factor_t factor, const float* A, void* stream);
int trx_strsm_factor(trx_handle_t handle, trx_factor_t factor, int64_t nrhs, float alpha,
                     float* B, int64_t ldb, void* stream);
int trx_strmm_factor(trx_handle_t handle, trx_factor_t factor, int64_t nrhs, float alpha,
                     float* B, int64_t ldb, void* stream);
int trx_factor_destroy(trx_factor_t factor);

/* Upload of the triangle the four operations read (no counterpart in the
 * paper, whose operands are on the device: Eq. 1-4 reference one triangle of
 * A, so a caller whose A is in host memory need not send the other one).
 * Copies the k x k triangle uplo of the column-major host array A_host
 * (leading dimension lda_host, elements of elem = 4 or 8 bytes), diagonal
 * included ('L': rows j..k-1 of column j; 'U': rows 0..j), into the
 * column-major device array A_dev (leading dimension lda_dev). It runs as one
 * rectangular cudaMemcpy2DAsync per block of 256 columns, so inside the
 * 256 x 256 diagonal blocks the other triangle's host values are copied too;
 * everything else of the other triangle in A_dev is left as it was. About
 * k^2 / 2 + 128 k elements move instead of k^2. Enqueued on stream (a
 * cudaStream_t, NULL for the legacy stream); with pinned host memory it is
 * asynchronous, otherwise CUDA stages it. The caller owns both arrays.
 * Returns 0, -i for an illegal i-th argument (uplo 1, k 2, elem 3, A_host 4,
 * lda_host 5, A_dev 6, lda_dev 7), TRX_ERR_CUDA. */
int trx_copy_triangle_h2d(char uplo, int64_t k, int elem, const void* A_host, int64_t lda_host,
                          void* A_dev, int64_t lda_dev, void* stream);

/* Prepared batch: the same problems run many times (fixed pointers; the
 * contents of A and B may change between runs). trx_batch_create checks,
 * canonicalises and cost-sorts the problems once (with the handle's current
 * tuning table) and keeps the descriptors on the handle's device, so a run
 * is one counter reset and one persistent launch (replayed from a cached
 * graph), with no host work per run. (No counterpart in the paper: the
 * batched workload is this library's.) Argument errors as trx_batched;
 * TRX_ERR_ALLOC if the device copy cannot be made. trx_batch_run enqueues
 * on stream (asynchronous); runs of one batch must not overlap (its work
 * counter is shared), different batches may run concurrently on different
 * streams. trx_batch_destroy synchronises the device and frees the batch;
 * NULL is accepted. A batch belongs to the handle it was created with. */
typedef struct trx_batch_s* trx_batch_t;
int trx_batch_create(trx_handle_t handle, int elem_bytes, int64_t count,
                     const trx_problem_t* problems, trx_batch_t* batch);
int trx_batch_run(trx_handle_t handle, trx_batch_t batch, void* stream);
int trx_batch_destroy(trx_batch_t batch);

/* Tuning table of the batched kernel: the substitution block height (4, 8
 * or 16 rows) per order bucket (k <= 64, 128, 256, 512) and right-hand-side
 * bucket (nrhs <= 8, 24, more), for each element type; 8 everywhere on a new
 * handle. */
#define TRX_TUNE_K_BUCKETS 4
#define TRX_TUNE_N_BUCKETS 3

/* Time the batch with each block height per (order, right-hand-side) bucket,
 * keep the fastest per bucket in the handle for later batched calls and
 * prepared batches, and write the table as JSON into json (if not NULL):
 * {"dtype", "buckets": [{"kmax", "nrhs_max", "problems", "sb", "ms": {"4",
 * "8", "16"}}, ...]} in order-major bucket order. The problems' B arrays are
 * overwritten (the batch runs several times): tune on representative
 * scratch data. Synchronises the stream. */
int trx_batched_autotune(trx_handle_t handle, int elem_bytes, int64_t count,
                         const trx_problem_t* problems, void* stream,
                         char* json, size_t json_len);

/* Read / replace the handle's tuning table for one element type (count =
 * TRX_TUNE_K_BUCKETS * TRX_TUNE_N_BUCKETS entries, order-major), e.g. to
 * persist a tuned table and restore it in a later process. set rejects
 * entries other than 4, 8, 16 (TRX_ERR_INVALID_VALUE). */
int trx_batched_get_tuning(trx_handle_t handle, int elem_bytes, int* table, int count);
int trx_batched_set_tuning(trx_handle_t handle, int elem_bytes, const int* table, int count);

/* ---- serving: continuous batching over resident factors ----------------
 * (The paper has no serving layer; this drives the entry points above.)
 * Factors are registered once and stay resident (the caller keeps A alive
 * until the factor is released and its requests have completed); requests
 * name a factor, an operation, a side, alpha and a right-hand side B
 * (device, overwritten by the result, kept alive by the caller until its
 * request completes). trx_server_submit only queues. Each trx_server_poll
 * is one scheduling tick: retire launch groups whose completion event has
 * fired, admit queued requests oldest first while the in-flight request
 * count and the device-memory budget allow (B's bytes, plus 4 k (k + nrhs)
 * for an FP32 call on the tensor-core path; a request larger than the
 * budget is admitted alone on an idle server), launch the admitted ones —
 * orders up to small_k as one persistent trx_batched launch per element
 * type on the server's batch stream, the rest one trx_?trsm / trx_?trmm
 * each, on whichever of the `streams` streams has the least estimated cost
 * in flight (k^2 n plus a fixed latency term per request), one handle and
 * workspace per stream — and report up to `capacity` completed requests with their
 * status (0 or a TRX_ERR_* code). A request's launch waits for an event
 * recorded on input_stream at submission, so B may still be in flight
 * there. The plan a request gets depends only on its own problem, so its
 * result is bitwise the same alone and in a mix. One thread at a time. */
typedef struct trx_server_s* trx_server_t;
typedef struct {
    int streams;            /* streams (and handles) for large requests, 1..16 (4)  */
    int small_k;            /* orders up to this go to trx_batched, 0..512 (512);
                               FP64 problems only while k^2 n <= 2^20 (one CTA
                               each there, on the FP64 pipe)                     */
    int64_t max_inflight;   /* requests admitted and not yet completed (4096)       */
    size_t budget_bytes;    /* device bytes admitted requests may hold (150 GiB)    */
    size_t workspace_bytes; /* per-stream workspace made at creation (0); a larger
                               need grows it (stream-ordered: that stream waits
                               for its own earlier work, the others run on)     */
    int graphs;             /* 1: large requests replay cached CUDA graphs (one
                               capture per new problem shape); 0: direct
                               launches (1)                                      */
    int refine_corrections; /* corrections of a refined request, 0..16 (2)       */
    int fp64_corrections;   /* FP64 TRSM requests: 0 the recursive DFMA solve;
                               n in 1..16 the FP32 solve plus n float-float
                               corrections (TRX_OPT_FP64_TRSM) (0)             */
    int fp64_trmm;          /* FP64 TRMM requests: 0 the recursive DFMA product;
                               1 one float-float pass (TRX_OPT_FP64_TRMM) (0)   */
} trx_server_config_t;
/* config NULL: the defaults in brackets above. */
int trx_server_create(int device, const trx_server_config_t* config, trx_server_t* server);
/* Synchronises the server's streams, then frees it (queued requests are
 * dropped unlaunched). */
int trx_server_destroy(trx_server_t server);
/* -i for an illegal i-th argument (uplo 2, transa 3, diag 4, k 5,
 * elem_bytes 6, A 7, lda 8, factor_id 9). */
int trx_server_register_factor(trx_server_t server, char uplo, char transa, char diag, int64_t k,
                               int elem_bytes, const void* A, int64_t lda, int* factor_id);
/* No new requests for the factor; it is dropped once its last request has
 * completed. */
int trx_server_release_factor(trx_server_t server, int factor_id);
/* op 'S' (TRSM) or 'M' (TRMM); B is m x n with k = m (side 'L') or n ('R').
 * -i for an illegal i-th argument (factor_id 2, op 3, side 4, B 6, m 7,
 * n 8, ldb 9, request_id 11). */
int trx_server_submit(trx_server_t server, int factor_id, char op, char side, double alpha,
                      void* B, int64_t m, int64_t n, int64_t ldb, void* input_stream,
                      int64_t* request_id);
/* A refined FP32 TRSM request: op(A) X = alpha B (side 'L') or
 * X op(A) = alpha B ('R') on an FP32 factor, B (FP32, m x n, not modified)
 * and X (FP64, m x n, leading dimension ldx, the result) device buffers
 * kept alive by the caller until the request completes; the FP32 solve plus
 * refine_corrections float-float corrections (trx_strsm_refined_async), on
 * the streams of the large requests whatever the order. -i for an illegal
 * i-th argument (factor_id 2, also an FP64 factor; side 3, B 5, m 7, n 8,
 * ldb 9, X 10, ldx 11, request_id 13). */
int trx_server_submit_refined(trx_server_t server, int factor_id, char side, double alpha,
                              const void* B, int64_t m, int64_t n, int64_t ldb, double* X,
                              int64_t ldx, void* input_stream, int64_t* request_id);
/* One tick (above). Returns 0, or the first error of this tick (the
 * requests it concerns complete with that status). */
int trx_server_poll(trx_server_t server, int64_t* request_ids, int* status, int capacity,
                    int* count);
/* Requests queued, in flight, and completed but not yet reported. */
int trx_server_pending(trx_server_t server, int64_t* waiting, int64_t* inflight,
                       int64_t* unreported);
/* Block until the oldest launch group in flight has finished. */
int trx_server_wait(trx_server_t server);

/* Set / read an option (TRX_OPT_*). Unknown options or values return
 * TRX_ERR_INVALID_VALUE. */
int trx_set_option(trx_handle_t handle, int option, int64_t value);
int trx_get_option(trx_handle_t handle, int option, int64_t* value);

/* Read (and with reset != 0 clear) the accumulated profile. Blocks until
 * the profiled launches have finished. */
int trx_get_profile(trx_handle_t handle, trx_profile_t* out, int reset);

/* Read and clear the handle's device error word: returns TRX_SUCCESS or
 * TRX_ERR_TIMEOUT if a bounded wait in an earlier launch gave up (that
 * launch's output is then invalid). Synchronises the handle's device. */
int trx_check_device_error(trx_handle_t handle);

/* Static description of an error code. Never NULL. */
const char* trx_error_string(int code);

/* Detail of the last positive error returned on the calling thread (the
 * failing CUDA call and its message, or the workspace size needed). Never
 * NULL; empty if there was none. */
const char* trx_last_error_detail(void);

/* Diagnostic, host only (no device work, no handle): write into buf the
 * launch sequence a call would enqueue for the given problem, one step per
 * line ("conv_m", "conv_y", "leaf ...", "thin ...", "gemm ..." with their row
 * ranges in the canonical lower-triangular order), for alpha = 2. elem_bytes
 * 4 or 8, leaf as TRX_OPT_LEAF, gemm_mode as TRX_OPT_GEMM, trmm_dense as
 * TRX_OPT_TRMM_DENSE, trsm_tc_leaf as TRX_OPT_TRSM_TC_LEAF, thin_leaf as
 * TRX_OPT_THIN_LEAF (the recursion's plan: the whole-call thin solve of
 * TRX_OPT_THIN is not shown), op 'S' (TRSM) or 'M' (TRMM). Returns an
 * argument code, TRX_ERR_INVALID_VALUE if buf is too small, or 0. */
int trx_debug_plan(char op, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                   int elem_bytes, int leaf, int gemm_mode, int trmm_dense, int trsm_tc_leaf,
                   int thin_leaf, char* buf, size_t buflen);

/* Size of the static device scratch behind trx_strsm_noalloc (64 MiB). */
#define TRX_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* FP32 TRSM (same arguments and result as trx_strsm with a default handle)
 * for callers that cannot allocate device memory where they solve: a solve
 * issued while the stream is being captured into a CUDA graph (cudaMalloc
 * cannot be captured), code inside a framework that hands out device memory
 * only from its own pool, or a latency-bound loop that must not pay
 * cudaMalloc's implicit synchronisation or risk its out-of-memory failure.
 * The paper has no counterpart; it is a packaging of the same kernels.
 *
 * No handle: it runs on the calling thread's current device, launches
 * directly onto `stream` and calls no cudaMalloc/cudaFree. The tensor-core
 * path's scratch is one file-scope __device__ array of
 * TRX_NOALLOC_SCRATCH_BYTES that every device using this library holds
 * until the process exits; problems needing more (the split operand planes:
 * 2 * s * k * (k + nrhs) bytes with s BF16 slices per operand, 6 k (k + nrhs)
 * with the default 6-term split; k the order of A, nrhs the other dimension
 * of B, both rounded up to 64) return TRX_ERR_WORKSPACE before anything is
 * enqueued.
 * The first call on a device sets that device up (looks up the array's
 * device address, sets kernel attributes): make that first call outside any
 * stream capture. All calls share the one array, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race: serialise
 * them on one stream. A device-side wait that runs out of time (2 s; the
 * environment variable TRX_NOALLOC_WAIT_NS, read at a device's set-up,
 * overrides it) leaves B invalid and sets the device's error word, which
 * trx_noalloc_check_error reads. Returns 0, -i for an illegal i-th argument
 * (BLAS numbering as trx_strsm without the handle), or a TRX_ERR_* code. */
int trx_strsm_noalloc(char side, char uplo, char transa, char diag, int64_t m,
                      int64_t n, float alpha, const float* A, int64_t lda,
                      float* B, int64_t ldb, void* stream);

/* Read and clear the error word of trx_strsm_noalloc on the calling thread's
 * current device: TRX_SUCCESS, or TRX_ERR_TIMEOUT if a bounded wait of an
 * earlier call gave up (that call's B is invalid). Call it after the solves'
 * stream has been synchronised; it copies one int from the device (no
 * allocation). TRX_SUCCESS if no call has run on the device yet. */
int trx_noalloc_check_error(void);

/* Peak-rate probes (no counterpart in the paper): the arithmetic rates the
 * library's rooflines are quoted against, measured by its own kernels.
 * kind: TRX_PEAK_FFMA (FP32 FMA, CUDA cores), TRX_PEAK_DFMA (FP64 FMA),
 * TRX_PEAK_DMMA (FP64 mma.sync m8n8k4), TRX_PEAK_TC_TF32 (tcgen05.mma
 * kind::tf32, 128x256x8), TRX_PEAK_TC_BF16 (tcgen05.mma kind::f16, BF16,
 * 128x256x16). One launch (one CTA per SM for the tensor-core kinds, eight
 * of 256 threads per SM otherwise) of `iters` loop steps on `device`,
 * timed with CUDA events: *tflops = dense TFLOP/s (2 flop per
 * multiply-add), *ms (may be NULL) = the launch's time. Synchronous;
 * allocates and frees 64 KiB. Returns 0, TRX_ERR_INVALID_VALUE,
 * TRX_ERR_DEVICE, TRX_ERR_CUDA, or TRX_ERR_TIMEOUT if the tensor-core
 * probe's bounded wait (2 s) gave up. */
enum {
    TRX_PEAK_FFMA = 0,
    TRX_PEAK_DFMA = 1,
    TRX_PEAK_DMMA = 2,
    TRX_PEAK_TC_TF32 = 3,
    TRX_PEAK_TC_BF16 = 4
};
int trx_peak_probe(int device, int kind, int64_t iters, double* tflops, double* ms);

/* Library version as major*10000 + minor*100 + patch. */
int trx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TRX_H_ */

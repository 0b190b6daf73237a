// C-ABI of the trx library: argument checking, canonical form, recursion
// planner and launch-chain execution (direct or as a cached CUDA graph).
//
// The recursion is the one of Section 3.1 (split the triangle at about half,
// recurse on the diagonal blocks, GEMM-update the off-diagonal block, base
// kernels below a cutoff), written once for the canonical lower form of
// common.cuh. Each of the 16 variants of Eq. 1-4 reaches it by a stride
// mapping (side 'R' solves with op(A)^T on B^T; an effectively-upper triangle
// is index-reversed), so no variant needs its own kernels.
#include <algorithm>
#include <cctype>
#include <cmath>
#include <type_traits>
#include <cstdio>
#include <cstring>
#include <string>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "plan.cuh"
#include "trx.h"

namespace trx {
// Leaf kernels set their shared-memory limits once per device (leaf.cu).
cudaError_t leaf_configure_all();

struct BatchDesc {
    int64_t k, nrhs;
    const void* A;
    int64_t a_rs, a_cs;
    void* C;
    int64_t c_rs, c_cs;
    double alpha;
    int unit, trsm, sb, pad;
};
cudaError_t batched_configure();
cudaError_t launch_batched(int elem_bytes, const BatchDesc* descs, int64_t count, int* counter,
                           int grid_ctas, cudaStream_t s);
int batched_ctas_per_sm(int elem_bytes);
}  // namespace trx

using namespace trx;

namespace {

constexpr int kMagic = 0x54525831;  // "TRX1"
constexpr long long kDefaultWaitNs = 2000000000LL;   // 2 s
constexpr size_t kGraphCacheSize = 16;
constexpr int64_t kBatchMaxK = TRX_BATCH_MAX_K;
constexpr int kMaxPanels = 4;
constexpr int kBatchSlots = 4;     // batched descriptor staging slots per handle
// Auto stays at one chain: measured at m = n = 16384, 2 and 4 branches were
// slower (the persistent GEMM update takes every SM, so branches serialise).

thread_local char g_detail[256] = "";

}  // namespace

namespace trx {
bool& pdl_enabled() {
    static thread_local bool on = false;
    return on;
}

const char* set_detail(const char* msg) {
    snprintf(g_detail, sizeof(g_detail), "%s", msg);
    return g_detail;
}
}  // namespace trx

namespace {

int fail_cuda(cudaError_t e, const char* what) {
    snprintf(g_detail, sizeof(g_detail), "%s: %s", what, cudaGetErrorString(e));
    return TRX_ERR_CUDA;
}

int upc(char c) { return (c >= 'a' && c <= 'z') ? c - 'a' + 'A' : c; }

int check_args(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
               const void* A, int64_t lda, const void* B, int64_t ldb) {
    const int s = upc(side), u = upc(uplo), t = upc(transa), d = upc(diag);
    if (s != 'L' && s != 'R') return -1;
    if (u != 'L' && u != 'U') return -2;
    if (t != 'N' && t != 'T' && t != 'C') return -3;
    if (d != 'N' && d != 'U') return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    const int64_t k = (s == 'L') ? m : n;
    if (m > 0 && n > 0 && A == nullptr) return -8;
    if (lda < std::max<int64_t>(1, k)) return -9;
    if (m > 0 && n > 0 && B == nullptr) return -10;
    if (ldb < std::max<int64_t>(1, m)) return -11;
    return 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
Canon<T> canonicalize(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                      const T* A, int64_t lda, T* B, int64_t ldb) {
    const bool left = upc(side) == 'L', lower = upc(uplo) == 'L';
    const bool trans = upc(transa) != 'N', unit = upc(diag) == 'U';
    Canon<T> c;
    c.k = left ? m : n;
    c.nrhs = left ? n : m;
    c.unit = unit;
    int64_t rs, cs;
    bool eff_lower;
    if (left) {                  // M = op(A), C = B
        rs = trans ? lda : 1;
        cs = trans ? 1 : lda;
        eff_lower = lower != trans;
        c.c_rs = 1;
        c.c_cs = ldb;
    } else {                     // M = op(A)^T, C = B^T
        rs = trans ? 1 : lda;
        cs = trans ? lda : 1;
        eff_lower = lower == trans;
        c.c_rs = ldb;
        c.c_cs = 1;
    }
    c.A = A;
    c.a_rs = rs;
    c.a_cs = cs;
    c.C = B;
    if (!eff_lower) {            // reverse the index order: upper -> lower
        c.A = A + (c.k - 1) * (rs + cs);
        c.a_rs = -rs;
        c.a_cs = -cs;
        c.C = B + (c.k - 1) * c.c_rs;
        c.c_rs = -c.c_rs;
    }
    return c;
}

// Workspace of the tensor-core path: `slices` M planes then `slices` Y
// planes (m_bytes and y_bytes each).
struct WsLayout {
    int64_t ldm = 0, ldy = 0;
    int slices = 2;
    size_t m_bytes = 0, y_bytes = 0, total = 0;
};

WsLayout ws_layout(int64_t k, int64_t nrhs, int slices) {
    WsLayout w;
    w.ldm = round_up(std::max<int64_t>(k, 1), 64);
    w.ldy = w.ldm;
    w.slices = slices;
    w.m_bytes = align256((size_t)k * w.ldm * 2);
    w.y_bytes = align256((size_t)nrhs * w.ldy * 2);
    w.total = (size_t)slices * (w.m_bytes + w.y_bytes);
    return w;
}

// Extra workspace of the device-scheduled TRSM after the planes: the
// diagonal blocks' inverses as `slices` compact k x 128 planes, then the
// block flags and the task counter.
size_t dag_extra_bytes(int64_t k, int64_t nrhs, int slices) {
    return (size_t)slices * align256((size_t)k * kDagBlock * 2) +
           align256(dag_flag_bytes(k, nrhs));
}

// Plane pointers of a workspace laid out as above (M planes from m_base
// unless the caller supplies them, Y planes from y_base).
void set_m_planes(Planes& pl, char* m_base, size_t m_bytes, int slices) {
    pl.m_hi = reinterpret_cast<__nv_bfloat16*>(m_base);
    pl.m_lo = slices > 1 ? reinterpret_cast<__nv_bfloat16*>(m_base + m_bytes) : nullptr;
    pl.m_lo2 = slices > 2 ? reinterpret_cast<__nv_bfloat16*>(m_base + 2 * m_bytes) : nullptr;
}
void set_y_planes(Planes& pl, char* y_base, size_t y_bytes, int slices) {
    pl.y_hi = reinterpret_cast<__nv_bfloat16*>(y_base);
    pl.y_lo = slices > 1 ? reinterpret_cast<__nv_bfloat16*>(y_base + y_bytes) : nullptr;
    pl.y_lo2 = slices > 2 ? reinterpret_cast<__nv_bfloat16*>(y_base + 2 * y_bytes) : nullptr;
}

}  // namespace

struct trx_handle_s {
    int magic = kMagic;
    int device = 0, num_sms = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    int64_t opt_leaf = 0, opt_gemm = 0, opt_graph = 1, opt_profile = 0, opt_pdl = 0;
    int64_t opt_split = 0;   // product terms of the tensor-core split (0: automatic)
    int64_t opt_fp64_trsm = 0;   // FP64 TRSM: 0 DFMA; n > 0 FP32 solve + n corrections
    int64_t opt_checked = 0;     // validate every plan before enqueueing it
    int64_t opt_trsm_dag = 0;    // device-scheduled TRSM: -1 off, 0 automatic, 1 on
    int64_t opt_nvtx = 0;        // an NVTX range around every launch step
    int64_t opt_fp64_trmm = 0;   // FP64 TRMM: 0 DFMA; 1 one float-float pass (order >= 64)
    long long wait_ns = kDefaultWaitNs;
    int* d_err = nullptr;
    cudaStream_t cap_stream = nullptr;
    trx_profile_t prof{};
    struct Pending {
        int cls;
        double flops, bytes;
        cudaEvent_t e0, e1;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    struct GraphEntry {
        std::string key;
        cudaGraphExec_t exec;
        uint64_t used;
    };
    std::vector<GraphEntry> graphs;
    uint64_t tick = 0;
    std::vector<unsigned char> maps;
    // batched path: device descriptors + counter, pinned staging, tuning
    // batched descriptors: a ring of staging slots (pinned host + device
    // copy + upload event), so an upload waits only for the launch kBatchSlots
    // back, not for the one before it
    BatchDesc* b_dev_ring[kBatchSlots] = {};
    BatchDesc* b_host_ring[kBatchSlots] = {};
    cudaEvent_t b_uploaded_ring[kBatchSlots] = {};
    int b_slot = 0;
    int* b_counter = nullptr;
    int64_t b_cap = 0;
    // batched substitution block height per [element type][order bucket]
    // [right-hand-side bucket] (trx_batched_autotune); 8 until tuned
    int tune_sb[2][TRX_TUNE_K_BUCKETS][TRX_TUNE_N_BUCKETS] = {};
    // column-panel branches of a TRSM: streams and fork/join events
    int64_t opt_panels = 0;
    int64_t opt_trmm_dense = 0;
    int64_t opt_residual = 0;
    int64_t opt_trsm_tc_leaf = 0;
    // refined TRSM scratch (grown on demand)
    void* rf_buf = nullptr;
    size_t rf_bytes = 0;
    // thin-right-hand-side TRSM: task counter and block flags (grown on demand)
    int64_t opt_thin = 0;
    int64_t opt_thin_leaf = 0;       // TRSM leaves as thin solves (TRX_OPT_THIN_LEAF)
    int64_t opt_test_withhold = 0;   // test hook (TRX_OPT_TEST_WITHHOLD)
    int* thin_buf = nullptr;
    size_t thin_bytes = 0;
    cudaStream_t aux[kMaxPanels] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kMaxPanels] = {};
};

namespace {

bool valid(trx_handle_t h) { return h != nullptr && h->magic == kMagic; }

// Slices per operand of the handle's tensor-core split.
int slices_for(const trx_handle_s* h) { return slices_of_terms(split_terms(h->opt_split)); }

cudaEvent_t get_event(trx_handle_t h) {
    if (!h->free_events.empty()) {
        cudaEvent_t e = h->free_events.back();
        h->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}


template <typename T>
bool use_tc(trx_handle_t h, int64_t k, bool trsm, int64_t nrhs) {
    return use_tc_mode((int)sizeof(T), h->opt_gemm, k,
                       leaf_for(h->opt_leaf, k, trsm, (int)sizeof(T), nrhs));
}

template <typename T>
struct Exec {
    trx_handle_t h;
    Canon<T> c;
    Planes pl;
    const void* maps = nullptr;
    // inverted diagonal blocks (TRSM leaves on the tensor cores): their
    // planes and the tensor maps over them and the Y planes
    const void* maps_w = nullptr;
    __nv_bfloat16* w_hi = nullptr;
    __nv_bfloat16* w_lo = nullptr;
    __nv_bfloat16* w_lo2 = nullptr;
    int* dag_flags = nullptr;      // device-scheduled TRSM: block flags + task counter
    int* thin_scratch = nullptr;   // thin TRSM: task counter, stop word, block flags
    cudaStream_t s;
    bool profile;

    // NVTX range name of a step (TRX_OPT_NVTX): kind and its row ranges
    static void nvtx_push(const Step& st) {
        char name[128];
        switch (st.kind) {
            case kLeaf:
                snprintf(name, sizeof(name), "trx leaf %s rows %lld+%dx%lld",
                         st.trsm ? "trsm" : "trmm", (long long)st.r0, st.b,
                         (long long)st.nleaves);
                break;
            case kGemm:
                snprintf(name, sizeof(name), "trx gemm%s x%zu rows %lld+%lld K %lld",
                         st.tc ? " tc" : "", st.gemms.size(),
                         (long long)(st.gemms.empty() ? 0 : st.gemms[0].rc),
                         (long long)(st.gemms.empty() ? 0 : st.gemms[0].mlen),
                         (long long)(st.gemms.empty() ? 0 : st.gemms[0].klen));
                break;
            default:
                snprintf(name, sizeof(name), "trx planes");
                break;
        }
        nvtxRangePushA(name);
    }

    int run(const Plan& plan) {
        for (const Step& st : plan.steps) {
            int cls = TRX_KERNEL_OTHER;
            double flops = 0, bytes = 0;
            const double w = sizeof(T);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (h->opt_nvtx) nvtx_push(st);
            if (profile) {
                e0 = get_event(h);
                e1 = get_event(h);
                cudaEventRecord(e0, s);
            }
            cudaError_t e = cudaSuccess;
            switch (st.kind) {
                case kLeaf: {
                    e = launch_leaf<T>(st.trsm, c, st.r0, st.b, st.nleaves, (T)st.alpha,
                                       st.planes ? &pl : nullptr, h->num_sms, s);
                    cls = st.trsm ? TRX_KERNEL_LEAF_TRSM : TRX_KERNEL_LEAF_TRMM;
                    const int64_t rows = std::min<int64_t>(st.b * st.nleaves, c.k - st.r0);
                    const double bb = st.b;
                    flops = (double)rows * bb * c.nrhs;                   // ~b^2 n per leaf
                    bytes = w * (2.0 * rows * c.nrhs + rows * (bb + 1) / 2);
                    break;
                }
                case kGemm: {
                    if (st.tc) {
                        TcYOut yo;
                        yo.hi = pl.y_hi;
                        yo.lo = pl.y_lo;
                        yo.lo2 = pl.y_lo2;
                        yo.ld = pl.ldy;
                        yo.row0 = st.y0;
                        yo.row1 = st.y1;
                        e = launch_gemm_tc(*reinterpret_cast<const Canon<float>*>(&c),
                                           st.inv ? maps_w : maps, pl.slices, st.gemms.data(),
                                           (int)st.gemms.size(), (float)st.beta, (float)st.gamma,
                                           h->d_err, h->wait_ns, h->num_sms, s, st.dense,
                                           st.y1 > st.y0 ? &yo : nullptr);
                        cls = st.inv ? TRX_KERNEL_LEAF_TRSM : TRX_KERNEL_GEMM_TC;
                    } else {
                        for (const TcGemm& g : st.gemms) {
                            e = launch_gemm_simt<T>(c, c.C, c.c_rs, c.c_cs, g.rc, g.mlen, g.rk,
                                                    g.klen, (T)st.beta, (T)st.gamma, s,
                                                    h->num_sms);
                            if (e != cudaSuccess) break;
                        }
                        cls = TRX_KERNEL_GEMM_SIMT;
                    }
                    for (const TcGemm& g : st.gemms) {
                        if (st.dense) {      // rows of a triangular block: (i+1) 2n each
                            const double i0 = (double)(g.rc - g.rk);
                            flops += (double)c.nrhs * g.mlen * (2.0 * i0 + g.mlen + 1);
                            bytes += w * ((double)g.mlen * (i0 + (g.mlen + 1) / 2.0) +
                                          3.0 * g.mlen * c.nrhs);
                        } else {
                            flops += 2.0 * g.mlen * g.klen * c.nrhs;
                            bytes += w * ((double)g.mlen * g.klen + 2.0 * g.mlen * c.nrhs +
                                          (double)g.klen * c.nrhs);
                        }
                    }
                    break;
                }
                case kConvM:
                    e = launch_convert_m(*reinterpret_cast<const Canon<float>*>(&c), pl, st.b, s);
                    cls = TRX_KERNEL_CONVERT;
                    bytes = 8.0 * c.k * (c.k - 1) / 2;
                    break;
                case kConvY:
                    e = launch_convert_y(*reinterpret_cast<const Canon<float>*>(&c), pl, s);
                    cls = TRX_KERNEL_CONVERT;
                    bytes = 8.0 * c.k * c.nrhs;
                    break;
                case kConvYRows:
                    e = launch_convert_y_rows(*reinterpret_cast<const Canon<float>*>(&c), pl,
                                              st.r0, st.b, s);
                    cls = TRX_KERNEL_CONVERT;
                    bytes = 8.0 * st.b * c.nrhs;
                    break;
                case kInvDiag:
                    e = launch_invert_diag(*reinterpret_cast<const Canon<float>*>(&c), st.b, w_hi,
                                           w_lo, w_lo2, pl.slices, pl.ldm, s);
                    cls = TRX_KERNEL_CONVERT;
                    bytes = 4.0 * c.k * st.b * 1.5;
                    break;
                case kInvCompact:
                    e = launch_invert_diag(*reinterpret_cast<const Canon<float>*>(&c), st.b, w_hi,
                                           w_lo, w_lo2, pl.slices, st.b, s, true);
                    cls = TRX_KERNEL_CONVERT;
                    bytes = 4.0 * c.k * st.b * 1.5;
                    break;
                case kThin: {
                    // b == 0: the whole problem; else the leaf on rows
                    // [r0, r0 + b): the same canonical problem restricted
                    // to those rows and columns of M and rows of C
                    Canon<float> tc = *reinterpret_cast<const Canon<float>*>(&c);
                    if (st.b > 0) {
                        tc.A += st.r0 * (tc.a_rs + tc.a_cs);
                        tc.C += st.r0 * tc.c_rs;
                        tc.k = st.b;
                    }
                    if (st.trsm)
                        e = launch_thin_trsm(tc, (float)st.alpha, thin_scratch, h->d_err,
                                             h->wait_ns, h->num_sms, s,
                                             h->opt_test_withhold != 0);
                    else
                        e = launch_thin_trmm(tc, (float)st.alpha, thin_scratch, h->num_sms, s);
                    if (e == cudaSuccess && st.b > 0 && st.planes && st.r0 + st.b < c.k)
                        e = launch_convert_y_rows(*reinterpret_cast<const Canon<float>*>(&c), pl,
                                                  st.r0, st.b, s);
                    cls = st.trsm ? TRX_KERNEL_LEAF_TRSM : TRX_KERNEL_LEAF_TRMM;
                    flops = (double)tc.k * tc.k * tc.nrhs;
                    bytes = 4.0 * ((double)tc.k * (tc.k + 1) / 2 + 2.0 * tc.k * tc.nrhs);
                    break;
                }
                case kDag: {
                    __nv_bfloat16* const w3[3] = {w_hi, w_lo, w_lo2};
                    e = launch_trsm_dag(*reinterpret_cast<const Canon<float>*>(&c), pl, w3,
                                        (float)st.alpha, dag_flags, h->d_err, h->wait_ns,
                                        h->num_sms, s);
                    cls = TRX_KERNEL_GEMM_TC;
                    flops = (double)c.k * c.k * c.nrhs;
                    bytes = 4.0 * ((double)c.k * (c.k + 1) / 2 + 2.0 * c.k * c.nrhs);
                    break;
                }
            }
            if (h->opt_nvtx) nvtxRangePop();
            if (e != cudaSuccess) return fail_cuda(e, "kernel launch");
            if (profile) {
                cudaEventRecord(e1, s);
                h->pending.push_back({cls, flops, bytes, e0, e1});
            }
        }
        return TRX_SUCCESS;
    }
};

struct GraphKey {
    int op, elem, tc, b, slices, dag, thin;
    int64_t k, nrhs, a_rs, a_cs, c_rs, c_cs, unit;
    const void* A;
    const void* C;
    const void* ws;
    const void* planes;
    double alpha;
    long long wait_ns;
    int pdl, panels, dense, tc_leaf;
};

}  // namespace

// A prepared FP32 factor: its canonical triangle's split-BF16 planes, made
// once and reused by every call on it (the conversion step is skipped).
struct trx_factor_s {
    int magic = 0;
    int device = 0;
    char side = 'L', uplo = 'L', transa = 'N', diag = 'N';
    int64_t k = 0, lda = 1;
    const float* A = nullptr;
    __nv_bfloat16* m_hi = nullptr;   // null when k is too small for the tensor-core path
    __nv_bfloat16* m_lo = nullptr;
    __nv_bfloat16* m_lo2 = nullptr;
    int64_t ldm = 0;
    int slices = 2;                  // of the planes (the handle's split at creation)
    // inverted diagonal blocks of w_block rows (TRSM leaves on the tensor
    // cores), made by updates while the handle's TRX_OPT_TRSM_TC_LEAF is on
    __nv_bfloat16* w_hi = nullptr;
    __nv_bfloat16* w_lo = nullptr;
    __nv_bfloat16* w_lo2 = nullptr;
    int w_block = 0;
};

namespace {
void drop_graphs(trx_handle_t h);   // defined below

constexpr int kFactorMagic = 0x54524631;   // "TRF1"
// Diagonal blocks zeroed above the diagonal in a factor's planes: every
// TRMM diagonal-block size up to this one reads them as dense tiles.
constexpr int kFactorDenseRows = 2048;

int refine_fixed(trx_handle_t h, bool fp64_data, char side, char uplo, char transa, char diag,
                 int64_t m, int64_t n, double alpha, const void* A, int64_t lda, const void* B,
                 int64_t ldb, double* X, int64_t ldx, int corrections, void* stream);
int refine_scratch(trx_handle_t h, size_t need, cudaStream_t s);
int pair_trmm(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
              double alpha, const double* A, int64_t lda, double* B, int64_t ldb,
              cudaStream_t s);
// Smallest order the float-float FP64 engines take (the TRMM pass, the
// mixed TRSM's residual): their error, a few 2^-48 of |op(A)||B| per
// element, is inside 8 k u of FP64 from here on.
constexpr int64_t kPairMinK = 64;

template <typename T>
int execute(trx_handle_t h, bool trsm, char side, char uplo, char transa, char diag, int64_t m,
            int64_t n, T alpha, const T* A, int64_t lda, T* B, int64_t ldb, void* stream,
            const trx_factor_s* f = nullptr, int terms_override = 0) {
    const int info = check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    if (info) return info;
    if (!valid(h)) return TRX_ERR_HANDLE;
    if (m == 0 || n == 0) return TRX_SUCCESS;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    pdl_enabled() = h->opt_pdl != 0;
    if (alpha == T(0)) {
        e = launch_zero<T>(B, m, n, ldb, s);
        return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "zero");
    }
    if (std::is_same<T, double>::value && trsm && h->opt_fp64_trsm > 0 &&
        (upc(side) == 'L' ? m : n) >= kPairMinK)
        return refine_fixed(h, true, side, uplo, transa, diag, m, n, (double)alpha, A, lda, B,
                            ldb, reinterpret_cast<double*>(B), ldb, (int)h->opt_fp64_trsm,
                            stream);
    if (std::is_same<T, double>::value && !trsm && h->opt_fp64_trmm > 0 &&
        (upc(side) == 'L' ? m : n) >= kPairMinK)
        return pair_trmm(h, side, uplo, transa, diag, m, n, (double)alpha,
                         reinterpret_cast<const double*>(A), lda, reinterpret_cast<double*>(B),
                         ldb, s);
    Exec<T> ex;
    ex.h = h;
    ex.c = canonicalize<T>(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    ex.s = s;
    ex.profile = h->opt_profile != 0;
    const int64_t k = ex.c.k;
    int b = leaf_for(h->opt_leaf, k, trsm, (int)sizeof(T), ex.c.nrhs);

    // Thin right-hand sides: one persistent CUDA-core launch (thin.cu), no
    // planes, for the whole call; or, on the tensor-core path, the same
    // solve for each leaf of thin_leaf rows. Its task counter and flags live
    // in a handle buffer, grown here (never inside a stream capture: a
    // capture keeps the recursive chain with the ordinary leaves).
    const bool tc_ok = use_tc<T>(h, k, trsm, ex.c.nrhs);
    bool thin = std::is_same<T, float>::value &&
                use_thin_mode(h->opt_thin, trsm, (int)sizeof(T), k, ex.c.nrhs);
    // (an explicit leaf size turns the automatic thin leaves off)
    const int64_t tl_opt = (h->opt_leaf != 0 && h->opt_thin_leaf == 0) ? -1 : h->opt_thin_leaf;
    int thin_leaf = std::is_same<T, float>::value
                        ? thin_leaf_rows(tl_opt, tc_ok, trsm, (int)sizeof(T), k, ex.c.nrhs)
                        : 0;
    // both apply: a forced whole-call solve wins, else the thin leaves
    if (thin && thin_leaf > 0) {
        if (h->opt_thin > 0) thin_leaf = 0;
        else thin = false;
    }
    Plan plan;
    plan.tc = !thin && tc_ok;
    const size_t thin_need = thin ? (trsm ? thin_scratch_bytes(k, ex.c.nrhs)
                                          : thin_trmm_scratch_bytes(k, ex.c.nrhs))
                             : thin_leaf > 0 ? thin_scratch_bytes(thin_leaf, ex.c.nrhs)
                                             : 0;
    if (thin_need > 0 && h->thin_bytes < thin_need) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(s, &cs);
        if (e != cudaSuccess) return fail_cuda(e, "cudaStreamIsCapturing");
        if (cs != cudaStreamCaptureStatusNone) {
            thin = false;
            thin_leaf = 0;
            plan.tc = tc_ok;
        } else {
            const size_t want = std::max<size_t>(2 * thin_need, 1 << 16);
            // cached graphs hold the old buffer's address: dropped with it
            drop_graphs(h);
            if (h->thin_buf) cudaFree(h->thin_buf);        // waits for its last use
            h->thin_buf = nullptr;
            h->thin_bytes = 0;
            if ((e = cudaMalloc(&h->thin_buf, want)) != cudaSuccess) {
                snprintf(g_detail, sizeof(g_detail), "thin TRSM flags: %s", cudaGetErrorString(e));
                return TRX_ERR_ALLOC;
            }
            h->thin_bytes = want;
        }
    }
    ex.thin_scratch = (thin || thin_leaf > 0) ? h->thin_buf : nullptr;
    if (thin_leaf > 0) b = thin_leaf;
    plan.thin_leaf = thin_leaf > 0;
    // A prepared factor supplies the M planes (and its split): the workspace
    // holds Y only.
    const bool factor_planes = plan.tc && f != nullptr && f->m_hi != nullptr;
    const int slices = factor_planes ? f->slices
                       : terms_override ? slices_of_terms(terms_override) : slices_for(h);
    const bool dag = std::is_same<T, float>::value &&
                     use_dag_mode(h->opt_trsm_dag, plan.tc, trsm, (int)sizeof(T), k, ex.c.nrhs);
    if (plan.tc) {
        const WsLayout w = ws_layout(k, ex.c.nrhs, slices);
        const size_t planes = factor_planes ? (size_t)slices * w.y_bytes : w.total;
        const size_t need = planes + (dag ? dag_extra_bytes(k, ex.c.nrhs, slices) : 0);
        if (h->ws == nullptr || h->ws_bytes < need) {
            snprintf(g_detail, sizeof(g_detail), "workspace of %zu bytes needed, %zu set",
                     need, h->ws_bytes);
            return TRX_ERR_WORKSPACE;
        }
        char* base = static_cast<char*>(h->ws);
        ex.pl.ldm = w.ldm;
        ex.pl.ldy = w.ldy;
        ex.pl.slices = slices;
        if (factor_planes) {
            ex.pl.m_hi = f->m_hi;
            ex.pl.m_lo = f->m_lo;
            ex.pl.m_lo2 = f->m_lo2;
            set_y_planes(ex.pl, base, w.y_bytes, slices);
        } else {
            set_m_planes(ex.pl, base, w.m_bytes, slices);
            set_y_planes(ex.pl, base + (size_t)slices * w.m_bytes, w.y_bytes, slices);
        }
        if (dag) {
            // compact inverses and the flags after the planes
            char* d = base + planes;
            const size_t wb = align256((size_t)k * kDagBlock * 2);
            ex.w_hi = reinterpret_cast<__nv_bfloat16*>(d);
            ex.w_lo = slices > 1 ? reinterpret_cast<__nv_bfloat16*>(d + wb) : nullptr;
            ex.w_lo2 = slices > 2 ? reinterpret_cast<__nv_bfloat16*>(d + 2 * wb) : nullptr;
            ex.dag_flags = reinterpret_cast<int*>(d + (size_t)slices * wb);
        }
    }
    // TRSM leaves on the tensor cores: the inverted diagonal blocks sit in
    // the M planes' own diagonal blocks (no TRSM update reads inside a leaf
    // block) or, for a prepared factor, in the factor's W planes made for
    // this leaf size (its M planes serve TRMM's diagonal blocks too).
    plan.tc_leaf = std::is_same<T, float>::value && trsm && !dag && !plan.thin_leaf &&
                   tc_leaf_mode(h->opt_trsm_tc_leaf, plan.tc, b) &&
                   (!factor_planes || (f->w_hi != nullptr && f->w_block == b));
    if (plan.tc_leaf) {
        ex.w_hi = factor_planes ? f->w_hi : ex.pl.m_hi;
        ex.w_lo = factor_planes ? f->w_lo : ex.pl.m_lo;
        ex.w_lo2 = factor_planes ? f->w_lo2 : ex.pl.m_lo2;
    }
    // TRSM right-hand sides are independent: with many of them the chain runs
    // as P column-panel branches (forked streams, one graph), so the
    // latency-bound bottom of the recursion of one panel overlaps the others'.
    int P = 1;
    if (trsm && !dag && !thin && !plan.thin_leaf) {
        if (h->opt_panels > 0) P = (int)h->opt_panels;
        const int64_t step = round_up((ex.c.nrhs + P - 1) / P, 256);
        P = (int)std::max<int64_t>(1, (ex.c.nrhs + step - 1) / step);
    }
    std::vector<Exec<T>> parts((size_t)P, ex);
    std::vector<std::vector<unsigned char>> maps((size_t)P);
    {
        const int64_t step = P > 1 ? round_up((ex.c.nrhs + P - 1) / P, 256) : ex.c.nrhs;
        for (int i = 0; i < P; ++i) {
            const int64_t j0 = step * i;
            Exec<T>& x = parts[i];
            x.c.C = ex.c.C + j0 * ex.c.c_cs;
            x.c.nrhs = std::min<int64_t>(step, ex.c.nrhs - j0);
            if (plan.tc) {
                x.pl.y_hi = ex.pl.y_hi + j0 * ex.pl.ldy;
                if (ex.pl.y_lo) x.pl.y_lo = ex.pl.y_lo + j0 * ex.pl.ldy;
                if (ex.pl.y_lo2) x.pl.y_lo2 = ex.pl.y_lo2 + j0 * ex.pl.ldy;
                maps[i].resize(2 * tc_maps_size());
                e = tc_make_maps(x.pl, k, x.c.nrhs, maps[i].data());
                if (e != cudaSuccess) return fail_cuda(e, "tensor map encode");
                x.maps = maps[i].data();
                x.maps_w = x.maps;
                if (plan.tc_leaf && ex.w_hi != ex.pl.m_hi) {
                    Planes wp = x.pl;
                    wp.m_hi = ex.w_hi;
                    wp.m_lo = ex.w_lo;
                    wp.m_lo2 = ex.w_lo2;
                    e = tc_make_maps(wp, k, x.c.nrhs, maps[i].data() + tc_maps_size());
                    if (e != cudaSuccess) return fail_cuda(e, "tensor map encode");
                    x.maps_w = maps[i].data() + tc_maps_size();
                }
            }
        }
    }
    const int dense = trsm ? 0 : trmm_dense_mode(h->opt_trmm_dense, h->opt_leaf, plan.tc, k);
    Plan pre, body;
    pre.tc = body.tc = plan.tc;
    body.tc_leaf = plan.tc_leaf;
    body.thin_leaf = plan.thin_leaf;
    if (plan.tc && !factor_planes) {
        Step cm{kConvM};
        cm.b = dense;
        pre.steps.push_back(cm);
        if (plan.tc_leaf) {
            Step iv{kInvDiag};
            iv.b = b;
            pre.steps.push_back(iv);
        }
    }
    if (dag) {
        // the device-scheduled solve in place of the recursion's chain: the
        // diagonal blocks' inverses, then one persistent launch
        Step iv{kInvCompact};
        iv.b = kDagBlock;
        body.steps.push_back(iv);
        Step dg{kDag};
        dg.alpha = (double)alpha;
        body.steps.push_back(dg);
    } else if (thin) {
        Step th{kThin};
        th.trsm = trsm;
        th.alpha = (double)alpha;
        body.steps.push_back(th);
    } else {
        make_plan(body, trsm, k, b, (double)alpha, /*conv_m=*/false, dense);
    }
    if (h->opt_checked) {
        if (const char* why = validate_plan(body, k)) {
            snprintf(g_detail, sizeof(g_detail), "checked plan: %s", why);
            return TRX_ERR_INVALID_VALUE;
        }
    }

    // The whole call on stream st: prelude, then the panels (forked when P > 1).
    auto run_all = [&](cudaStream_t st) -> int {
        ex.s = st;
        int rc = ex.run(pre);
        if (rc != TRX_SUCCESS) return rc;
        if (P == 1) {
            parts[0].s = st;
            return parts[0].run(body);
        }
        cudaError_t ee = cudaEventRecord(h->fork_ev, st);
        if (ee != cudaSuccess) return fail_cuda(ee, "fork");
        for (int i = 0; i < P; ++i) {
            if ((ee = cudaStreamWaitEvent(h->aux[i], h->fork_ev, 0)) != cudaSuccess)
                return fail_cuda(ee, "fork wait");
            parts[i].s = h->aux[i];
            if ((rc = parts[i].run(body)) != TRX_SUCCESS) return rc;
            if ((ee = cudaEventRecord(h->join_ev[i], h->aux[i])) != cudaSuccess ||
                (ee = cudaStreamWaitEvent(st, h->join_ev[i], 0)) != cudaSuccess)
                return fail_cuda(ee, "join");
        }
        return TRX_SUCCESS;
    };

    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamIsCapturing");
    if (ex.profile || !h->opt_graph || cap != cudaStreamCaptureStatusNone) return run_all(s);

    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.op = trsm;
    key.elem = sizeof(T);
    key.tc = plan.tc;
    key.b = b;
    key.slices = plan.tc ? slices : 0;
    key.dag = dag;
    key.thin = thin ? 1 + (int)h->opt_test_withhold
               : plan.thin_leaf ? 3 + (int)h->opt_test_withhold : 0;
    key.k = k;
    key.nrhs = ex.c.nrhs;
    key.a_rs = ex.c.a_rs;
    key.a_cs = ex.c.a_cs;
    key.c_rs = ex.c.c_rs;
    key.c_cs = ex.c.c_cs;
    key.unit = ex.c.unit;
    key.A = ex.c.A;
    key.C = ex.c.C;
    key.ws = plan.tc ? h->ws : nullptr;
    key.planes = factor_planes ? f->m_hi : nullptr;
    key.alpha = (double)alpha;
    key.wait_ns = h->wait_ns;
    key.pdl = (int)h->opt_pdl;
    key.tc_leaf = (int)plan.tc_leaf;
    key.panels = P;
    key.dense = dense;
    const std::string ks(reinterpret_cast<const char*>(&key), sizeof(key));
    ++h->tick;
    for (auto& g : h->graphs) {
        if (g.key == ks) {
            g.used = h->tick;
            e = cudaGraphLaunch(g.exec, s);
            return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "cudaGraphLaunch");
        }
    }
    e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamBeginCapture");
    const int rc = run_all(h->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (rc != TRX_SUCCESS) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
    if (h->graphs.size() >= kGraphCacheSize) {
        auto old = std::min_element(h->graphs.begin(), h->graphs.end(),
                                    [](const auto& a, const auto& b) { return a.used < b.used; });
        cudaGraphExecDestroy(old->exec);
        h->graphs.erase(old);
    }
    h->graphs.push_back({ks, exec, h->tick});
    e = cudaGraphLaunch(exec, s);
    return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "cudaGraphLaunch");
}

}  // namespace

namespace {
void drop_graphs(trx_handle_t h);
void free_owned_ws(trx_handle_t h);
}  // namespace

namespace trx {

// The request server's workspace growth: swap without a device-wide
// synchronisation (the server has waited for the handle's stream, the only
// one its work runs on). Cached graphs point into the old buffer: dropped.
int handle_swap_workspace(trx_handle_t h, void* ptr, size_t bytes) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if ((reinterpret_cast<uintptr_t>(ptr) & 255) != 0) return TRX_ERR_INVALID_VALUE;
    drop_graphs(h);
    free_owned_ws(h);
    h->ws = ptr;
    h->ws_bytes = ptr ? bytes : 0;
    return TRX_SUCCESS;
}

// For trx_strsm_noalloc (noalloc.cu): BLAS argument check, the scratch a
// call needs on the tensor-core path, and the call itself with a caller-
// supplied scratch and error word, on a handle that lives on the stack
// (no device allocation, no graph: launches go straight onto the stream).
int noalloc_check_args(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                       const void* A, int64_t lda, const void* B, int64_t ldb) {
    return check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
}

size_t noalloc_scratch_bytes(char side, int64_t m, int64_t n) {
    const int64_t k = upc(side) == 'L' ? m : n, nrhs = upc(side) == 'L' ? n : m;
    if (k <= 0 || nrhs <= 0) return 0;
    const int b = leaf_for(0, k, true, 4, nrhs);
    return use_tc_mode(4, 0, k, b) ? ws_layout(k, nrhs, slices_of_terms(split_terms(0))).total
                                   : 0;
}

int noalloc_strsm(int device, int num_sms, void* scratch, size_t scratch_bytes, int* err_word,
                  long long wait_ns, char side, char uplo, char transa, char diag, int64_t m,
                  int64_t n, float alpha, const float* A, int64_t lda, float* B, int64_t ldb,
                  void* stream) {
    trx_handle_s hs;
    hs.device = device;
    hs.num_sms = num_sms;
    hs.ws = scratch;
    hs.ws_bytes = scratch_bytes;
    hs.d_err = err_word;
    hs.wait_ns = wait_ns;
    hs.opt_graph = 0;
    hs.opt_panels = 1;   // no handle streams here: one chain on the caller's stream
    hs.opt_trsm_dag = -1;   // the recursive chain only: its scratch is the planes
    hs.opt_thin = -1;       // (the thin solve's flags would need an allocation)
    hs.opt_thin_leaf = -1;
    return execute<float>(&hs, true, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb,
                          stream);
}

}  // namespace trx

namespace {

void free_owned_ws(trx_handle_t h) {
    if (h->ws_owned && h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    h->ws_owned = false;
}

void drop_graphs(trx_handle_t h) {
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

int bucket_of(int64_t k) { return k <= 64 ? 0 : k <= 128 ? 1 : k <= 256 ? 2 : 3; }
int nbucket_of(int64_t nrhs) { return nrhs <= 8 ? 0 : nrhs <= 24 ? 1 : 2; }
int tune_index(int64_t k, int64_t nrhs) { return bucket_of(k) * TRX_TUNE_N_BUCKETS + nbucket_of(nrhs); }

// Validate and map the problems to sorted canonical descriptors (host).
int batch_descs(trx_handle_t h, int elem_bytes, int64_t count, const trx_problem_t* probs,
                std::vector<BatchDesc>& out, const int* sb_override) {
    out.clear();
    out.reserve((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const trx_problem_t& q = probs[i];
        const int op = upc(q.op);
        int info = (op == 'S' || op == 'M') ? 0 : -100;
        if (!info)
            info = check_args(q.side, q.uplo, q.transa, q.diag, q.m, q.n, q.A, q.lda, q.B, q.ldb);
        const int64_t k = upc(q.side) == 'L' ? q.m : q.n;
        if (!info && k > kBatchMaxK) info = -200;
        if (info) {
            snprintf(g_detail, sizeof(g_detail),
                     "batched problem %lld: %s", (long long)i,
                     info == -100 ? "op must be 'S' or 'M'"
                     : info == -200 ? "order above TRX_BATCH_MAX_K"
                                    : trx_error_string(info));
            return TRX_ERR_INVALID_VALUE;
        }
        if (q.m == 0 || q.n == 0) continue;
        BatchDesc d;
        std::memset(&d, 0, sizeof(d));
        if (elem_bytes == 4) {
            const Canon<float> c = canonicalize<float>(q.side, q.uplo, q.transa, q.diag, q.m, q.n,
                                                       static_cast<const float*>(q.A), q.lda,
                                                       static_cast<float*>(q.B), q.ldb);
            d.k = c.k; d.nrhs = c.nrhs; d.A = c.A; d.a_rs = c.a_rs; d.a_cs = c.a_cs;
            d.C = c.C; d.c_rs = c.c_rs; d.c_cs = c.c_cs; d.unit = c.unit;
        } else {
            const Canon<double> c = canonicalize<double>(q.side, q.uplo, q.transa, q.diag, q.m,
                                                         q.n, static_cast<const double*>(q.A),
                                                         q.lda, static_cast<double*>(q.B), q.ldb);
            d.k = c.k; d.nrhs = c.nrhs; d.A = c.A; d.a_rs = c.a_rs; d.a_cs = c.a_cs;
            d.C = c.C; d.c_rs = c.c_rs; d.c_cs = c.c_cs; d.unit = c.unit;
        }
        d.alpha = q.alpha;
        d.trsm = q.alpha == 0.0 ? 2 : (op == 'S' ? 1 : 0);   // 2: B := 0, A not read
        const int b = tune_index(d.k, d.nrhs);
        d.sb = sb_override ? sb_override[b]
                           : (&h->tune_sb[elem_bytes == 4 ? 0 : 1][0][0])[b];
        out.push_back(d);
    }
    std::stable_sort(out.begin(), out.end(), [](const BatchDesc& x, const BatchDesc& y) {
        return (double)x.k * x.k * x.nrhs > (double)y.k * y.k * y.nrhs;
    });
    return TRX_SUCCESS;
}

// Upload descriptors through the pinned staging buffer and launch; with
// use_graph the launch (counter reset + kernel) replays from a cached graph.
int batch_run(trx_handle_t h, int elem_bytes, const std::vector<BatchDesc>& d, cudaStream_t s,
              bool use_graph) {
    const int64_t n = (int64_t)d.size();
    if (n == 0) return TRX_SUCCESS;
    cudaError_t e;
    if (n > h->b_cap) {
        for (int i = 0; i < kBatchSlots; ++i) {
            if (h->b_uploaded_ring[i]) cudaEventSynchronize(h->b_uploaded_ring[i]);
            if (h->b_dev_ring[i]) cudaFree(h->b_dev_ring[i]);
            if (h->b_host_ring[i]) cudaFreeHost(h->b_host_ring[i]);
            h->b_dev_ring[i] = nullptr;
            h->b_host_ring[i] = nullptr;
        }
        h->b_cap = 0;
        const int64_t cap = std::max<int64_t>(n, 1024);
        for (int i = 0; i < kBatchSlots; ++i)
            if ((e = cudaMalloc(&h->b_dev_ring[i], cap * sizeof(BatchDesc))) != cudaSuccess ||
                (e = cudaMallocHost(&h->b_host_ring[i], cap * sizeof(BatchDesc))) != cudaSuccess)
                return fail_cuda(e, "batch buffers");
        h->b_cap = cap;
        drop_graphs(h);
    }
    if (!h->b_counter && (e = cudaMalloc(&h->b_counter, 256)) != cudaSuccess)
        return fail_cuda(e, "batch counter");
    const int slot = h->b_slot;
    h->b_slot = (slot + 1) % kBatchSlots;
    cudaEvent_t& up = h->b_uploaded_ring[slot];
    if (!up && (e = cudaEventCreateWithFlags(&up, cudaEventDisableTiming)) != cudaSuccess)
        return fail_cuda(e, "batch event");
    if ((e = cudaEventSynchronize(up)) != cudaSuccess) return fail_cuda(e, "batch staging wait");
    BatchDesc* const b_dev = h->b_dev_ring[slot];
    std::memcpy(h->b_host_ring[slot], d.data(), n * sizeof(BatchDesc));
    if ((e = cudaMemcpyAsync(b_dev, h->b_host_ring[slot], n * sizeof(BatchDesc),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaEventRecord(up, s)) != cudaSuccess)
        return fail_cuda(e, "batch upload");
    // persistent CTAs: as many per SM as fit (shared memory bound)
    const int grid = h->num_sms * batched_ctas_per_sm(elem_bytes);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (!use_graph || cap != cudaStreamCaptureStatusNone) {
        e = launch_batched(elem_bytes, b_dev, n, h->b_counter, grid, s);
        return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "batched launch");
    }
    char kbuf[64];
    snprintf(kbuf, sizeof(kbuf), "batched:%d:%lld:%p", elem_bytes, (long long)n, (void*)b_dev);
    const std::string ks(kbuf);
    ++h->tick;
    for (auto& g : h->graphs) {
        if (g.key == ks) {
            g.used = h->tick;
            e = cudaGraphLaunch(g.exec, s);
            return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "cudaGraphLaunch");
        }
    }
    if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return fail_cuda(e, "cudaStreamBeginCapture");
    const cudaError_t le = launch_batched(elem_bytes, b_dev, n, h->b_counter, grid, h->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail_cuda(le != cudaSuccess ? le : e, "batched capture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
    if (h->graphs.size() >= kGraphCacheSize) {
        auto old = std::min_element(h->graphs.begin(), h->graphs.end(),
                                    [](const auto& a, const auto& b) { return a.used < b.used; });
        cudaGraphExecDestroy(old->exec);
        h->graphs.erase(old);
    }
    h->graphs.push_back({ks, exec, h->tick});
    e = cudaGraphLaunch(exec, s);
    return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "cudaGraphLaunch");
}

}  // namespace

struct trx_batch_s {
    int magic = 0;
    int device = 0, elem = 4, grid = 0;
    int64_t n = 0;
    BatchDesc* d = nullptr;      // device descriptors, cost-sorted
    int* counter = nullptr;      // device work counter
    cudaGraphExec_t exec = nullptr;
};

namespace {
constexpr int kBatchMagic = 0x54524231;  // "TRB1"
}

extern "C" {

int trx_batch_create(trx_handle_t h, int elem_bytes, int64_t count, const trx_problem_t* problems,
                     trx_batch_t* out) {
    if (!out) return TRX_ERR_INVALID_VALUE;
    *out = nullptr;
    if (!valid(h)) return TRX_ERR_HANDLE;
    if ((elem_bytes != 4 && elem_bytes != 8) || count < 0 || (count > 0 && !problems))
        return TRX_ERR_INVALID_VALUE;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    std::vector<BatchDesc> d;
    const int rc = batch_descs(h, elem_bytes, count, problems, d, nullptr);
    if (rc != TRX_SUCCESS) return rc;
    auto* b = new (std::nothrow) trx_batch_s;
    if (!b) return TRX_ERR_ALLOC;
    b->device = h->device;
    b->elem = elem_bytes;
    b->n = (int64_t)d.size();
    b->grid = h->num_sms * batched_ctas_per_sm(elem_bytes);
    if ((e = cudaMalloc(&b->counter, 256)) != cudaSuccess ||
        (b->n > 0 && (e = cudaMalloc(&b->d, b->n * sizeof(BatchDesc))) != cudaSuccess) ||
        (b->n > 0 &&
         (e = cudaMemcpy(b->d, d.data(), b->n * sizeof(BatchDesc), cudaMemcpyHostToDevice)) !=
             cudaSuccess)) {
        if (b->d) cudaFree(b->d);
        if (b->counter) cudaFree(b->counter);
        delete b;
        snprintf(g_detail, sizeof(g_detail), "batch descriptors: %s", cudaGetErrorString(e));
        return TRX_ERR_ALLOC;
    }
    b->magic = kBatchMagic;
    *out = b;
    return TRX_SUCCESS;
}

int trx_batch_run(trx_handle_t h, trx_batch_t b, void* stream) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if (!b || b->magic != kBatchMagic || b->device != h->device) return TRX_ERR_INVALID_VALUE;
    if (b->n == 0) return TRX_SUCCESS;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    pdl_enabled() = h->opt_pdl != 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess)
        return fail_cuda(e, "cudaStreamIsCapturing");
    if (!h->opt_graph || cap != cudaStreamCaptureStatusNone) {
        e = launch_batched(b->elem, b->d, b->n, b->counter, b->grid, s);
        return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "batched launch");
    }
    if (!b->exec) {
        if ((e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            return fail_cuda(e, "cudaStreamBeginCapture");
        const cudaError_t le = launch_batched(b->elem, b->d, b->n, b->counter, b->grid,
                                              h->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail_cuda(le != cudaSuccess ? le : e, "batched capture");
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return fail_cuda(e, "cudaGraphInstantiate");
        }
    }
    e = cudaGraphLaunch(b->exec, s);
    return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "cudaGraphLaunch");
}

int trx_batch_destroy(trx_batch_t b) {
    if (b == nullptr) return TRX_SUCCESS;
    if (b->magic != kBatchMagic) return TRX_ERR_INVALID_VALUE;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d) cudaFree(b->d);
    if (b->counter) cudaFree(b->counter);
    b->magic = 0;
    delete b;
    return TRX_SUCCESS;
}

int trx_batched(trx_handle_t h, int elem_bytes, int64_t count, const trx_problem_t* problems,
                void* stream) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if ((elem_bytes != 4 && elem_bytes != 8) || count < 0 || (count > 0 && !problems))
        return TRX_ERR_INVALID_VALUE;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    pdl_enabled() = h->opt_pdl != 0;
    std::vector<BatchDesc> d;
    const int rc = batch_descs(h, elem_bytes, count, problems, d, nullptr);
    if (rc != TRX_SUCCESS) return rc;
    return batch_run(h, elem_bytes, d, reinterpret_cast<cudaStream_t>(stream), h->opt_graph != 0);
}

// One operation and element type per call: the problems' op must be the
// entry point's ('S' for TRSM, 'M' for TRMM); then as trx_batched.
static int batched_typed(trx_handle_t h, char op, int elem_bytes, int64_t count,
                         const trx_problem_t* problems, void* stream) {
    if (count < 0 || (count > 0 && !problems)) return TRX_ERR_INVALID_VALUE;
    for (int64_t i = 0; i < count; ++i)
        if (upc(problems[i].op) != op) {
            snprintf(g_detail, sizeof(g_detail), "problem %lld: op '%c' in a %s batch",
                     (long long)i, problems[i].op, op == 'S' ? "TRSM" : "TRMM");
            return TRX_ERR_INVALID_VALUE;
        }
    return trx_batched(h, elem_bytes, count, problems, stream);
}
int trx_strsm_batched(trx_handle_t h, int64_t count, const trx_problem_t* problems, void* stream) {
    return batched_typed(h, 'S', 4, count, problems, stream);
}
int trx_dtrsm_batched(trx_handle_t h, int64_t count, const trx_problem_t* problems, void* stream) {
    return batched_typed(h, 'S', 8, count, problems, stream);
}
int trx_strmm_batched(trx_handle_t h, int64_t count, const trx_problem_t* problems, void* stream) {
    return batched_typed(h, 'M', 4, count, problems, stream);
}
int trx_dtrmm_batched(trx_handle_t h, int64_t count, const trx_problem_t* problems, void* stream) {
    return batched_typed(h, 'M', 8, count, problems, stream);
}

int trx_batched_autotune(trx_handle_t h, int elem_bytes, int64_t count,
                         const trx_problem_t* problems, void* stream, char* json,
                         size_t json_len) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if ((elem_bytes != 4 && elem_bytes != 8) || count < 0 || (count > 0 && !problems))
        return TRX_ERR_INVALID_VALUE;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    constexpr int NB = TRX_TUNE_K_BUCKETS * TRX_TUNE_N_BUCKETS;
    const int sbs[3] = {4, 8, 16};
    double best_ms[NB], all_ms[NB][3];
    int best[NB], count_b[NB];
    const int t = elem_bytes == 4 ? 0 : 1;
    for (int b = 0; b < NB; ++b) {
        best_ms[b] = 1e30;
        best[b] = (&h->tune_sb[t][0][0])[b];
        count_b[b] = 0;
    }
    cudaEvent_t e0 = get_event(h), e1 = get_event(h);
    for (int bkt = 0; bkt < NB; ++bkt) {
        for (int v = 0; v < 3; ++v) {
            int ov[NB];
            for (int b = 0; b < NB; ++b) ov[b] = sbs[v];
            std::vector<BatchDesc> all, mine;
            int rc = batch_descs(h, elem_bytes, count, problems, all, ov);
            if (rc != TRX_SUCCESS) return rc;
            for (auto& x : all)
                if (tune_index(x.k, x.nrhs) == bkt) mine.push_back(x);
            all_ms[bkt][v] = 0.0;
            count_b[bkt] = (int)mine.size();
            if (mine.empty()) continue;
            double ms_sum = 0.0;
            for (int rep = 0; rep < 4; ++rep) {
                cudaEventRecord(e0, s);
                rc = batch_run(h, elem_bytes, mine, s, false);
                if (rc != TRX_SUCCESS) return rc;
                cudaEventRecord(e1, s);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return fail_cuda(e, "autotune");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_sum += ms;   // first run warms up
            }
            all_ms[bkt][v] = ms_sum / 3.0;
            if (all_ms[bkt][v] < best_ms[bkt]) {
                best_ms[bkt] = all_ms[bkt][v];
                best[bkt] = sbs[v];
            }
        }
    }
    h->free_events.push_back(e0);
    h->free_events.push_back(e1);
    for (int b = 0; b < NB; ++b) (&h->tune_sb[t][0][0])[b] = best[b];
    drop_graphs(h);
    if (json && json_len) {
        std::string out = std::string("{\"dtype\": \"") + (t ? "f64" : "f32") + "\", \"buckets\": [";
        const int kmax[4] = {64, 128, 256, 512};
        const int nmax[3] = {8, 24, 64};
        char buf[320];
        for (int b = 0; b < NB; ++b) {
            snprintf(buf, sizeof(buf),
                     "%s{\"kmax\": %d, \"nrhs_max\": %d, \"problems\": %d, \"sb\": %d, "
                     "\"ms\": {\"4\": %.5f, \"8\": %.5f, \"16\": %.5f}}",
                     b ? ", " : "", kmax[b / TRX_TUNE_N_BUCKETS],
                     nmax[b % TRX_TUNE_N_BUCKETS], count_b[b], best[b], all_ms[b][0],
                     all_ms[b][1], all_ms[b][2]);
            out += buf;
        }
        out += "]}";
        if (out.size() + 1 > json_len) return TRX_ERR_INVALID_VALUE;
        std::memcpy(json, out.c_str(), out.size() + 1);
    }
    return TRX_SUCCESS;
}

int trx_batched_get_tuning(trx_handle_t h, int elem_bytes, int* table, int count) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if ((elem_bytes != 4 && elem_bytes != 8) || !table ||
        count != TRX_TUNE_K_BUCKETS * TRX_TUNE_N_BUCKETS)
        return TRX_ERR_INVALID_VALUE;
    std::memcpy(table, &h->tune_sb[elem_bytes == 4 ? 0 : 1][0][0], sizeof(int) * count);
    return TRX_SUCCESS;
}

int trx_batched_set_tuning(trx_handle_t h, int elem_bytes, const int* table, int count) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if ((elem_bytes != 4 && elem_bytes != 8) || !table ||
        count != TRX_TUNE_K_BUCKETS * TRX_TUNE_N_BUCKETS)
        return TRX_ERR_INVALID_VALUE;
    for (int i = 0; i < count; ++i)
        if (table[i] != 4 && table[i] != 8 && table[i] != 16) return TRX_ERR_INVALID_VALUE;
    std::memcpy(&h->tune_sb[elem_bytes == 4 ? 0 : 1][0][0], table, sizeof(int) * count);
    drop_graphs(h);
    return TRX_SUCCESS;
}

int trx_create(trx_handle_t* handle, int device, size_t workspace_bytes) {
    if (!handle) return TRX_ERR_HANDLE;
    *handle = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return TRX_ERR_DEVICE;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3) {
        snprintf(g_detail, sizeof(g_detail), "device %d is sm_%d%d, the kernels are sm_103a",
                 device, prop.major, prop.minor);
        return TRX_ERR_DEVICE;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    trx_handle_t h = new (std::nothrow) trx_handle_s;
    if (!h) return TRX_ERR_ALLOC;
    h->device = device;
    h->num_sms = prop.multiProcessorCount;
    for (int t = 0; t < 2; ++t)
        for (int b = 0; b < TRX_TUNE_K_BUCKETS; ++b)
            for (int c = 0; c < TRX_TUNE_N_BUCKETS; ++c) h->tune_sb[t][b][c] = 8;
    if ((e = cudaMalloc(&h->d_err, 256)) != cudaSuccess ||
        (e = cudaMemset(h->d_err, 0, 256)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = leaf_configure_all()) != cudaSuccess || (e = batched_configure()) != cudaSuccess) {
        trx_destroy(h);
        return fail_cuda(e, "handle setup");
    }
    for (int i = 0; i < kMaxPanels; ++i) {
        if ((e = cudaStreamCreateWithFlags(&h->aux[i], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->join_ev[i], cudaEventDisableTiming)) != cudaSuccess) {
            trx_destroy(h);
            return fail_cuda(e, "handle streams");
        }
    }
    if (workspace_bytes > 0) {
        e = cudaMalloc(&h->ws, workspace_bytes);
        if (e != cudaSuccess) {
            h->ws = nullptr;
            trx_destroy(h);
            snprintf(g_detail, sizeof(g_detail), "workspace cudaMalloc: %s", cudaGetErrorString(e));
            return TRX_ERR_ALLOC;
        }
        h->ws_bytes = workspace_bytes;
        h->ws_owned = true;
    }
    *handle = h;
    return TRX_SUCCESS;
}

int trx_destroy(trx_handle_t h) {
    if (h == nullptr) return TRX_SUCCESS;
    if (!valid(h)) return TRX_ERR_HANDLE;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    drop_graphs(h);
    for (auto& p : h->pending) {
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    for (auto ev : h->free_events) cudaEventDestroy(ev);
    for (int i = 0; i < kBatchSlots; ++i) {
        if (h->b_dev_ring[i]) cudaFree(h->b_dev_ring[i]);
        if (h->b_host_ring[i]) cudaFreeHost(h->b_host_ring[i]);
        if (h->b_uploaded_ring[i]) cudaEventDestroy(h->b_uploaded_ring[i]);
    }
    if (h->b_counter) cudaFree(h->b_counter);
    if (h->rf_buf) {
        cudaFreeAsync(h->rf_buf, 0);        // stream-ordered allocation
        cudaDeviceSynchronize();
    }
    if (h->thin_buf) cudaFree(h->thin_buf);
    free_owned_ws(h);
    if (h->d_err) cudaFree(h->d_err);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int i = 0; i < kMaxPanels; ++i) {
        if (h->aux[i]) cudaStreamDestroy(h->aux[i]);
        if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    h->magic = 0;
    delete h;
    return TRX_SUCCESS;
}

int trx_set_workspace(trx_handle_t h, void* ptr, size_t bytes) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if ((reinterpret_cast<uintptr_t>(ptr) & 255) != 0) return TRX_ERR_INVALID_VALUE;
    if (ptr == h->ws && bytes == h->ws_bytes) return TRX_SUCCESS;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    drop_graphs(h);   // cached graphs point into the old workspace
    free_owned_ws(h);
    h->ws = ptr;
    h->ws_bytes = ptr ? bytes : 0;
    return TRX_SUCCESS;
}

int trx_workspace_size(trx_handle_t h, char op, char side, int64_t m, int64_t n, int elem_bytes,
                       size_t* bytes) {
    if (upc(side) != 'L' && upc(side) != 'R') return -1;
    if (m < 0) return -5;
    if (n < 0) return -6;
    if (!valid(h)) return TRX_ERR_HANDLE;
    const int o = upc(op);
    if ((elem_bytes != 4 && elem_bytes != 8) || (o != 'S' && o != 'M' && o != 'G' && o != 'Y') ||
        !bytes)
        return TRX_ERR_INVALID_VALUE;
    int64_t k = upc(side) == 'L' ? m : n, nrhs = upc(side) == 'L' ? n : m;
    if (o == 'Y') {         // factor calls (TRSM or TRMM): the Y planes only
        const bool tc_s = elem_bytes == 4 && use_tc<float>(h, k, true, nrhs);
        const bool tc = tc_s || (elem_bytes == 4 && use_tc<float>(h, k, false, nrhs));
        const int sl = slices_for(h);
        *bytes = (tc && k > 0 && nrhs > 0) ? (size_t)sl * ws_layout(k, nrhs, sl).y_bytes : 0;
        if (tc_s && k > 0 && nrhs > 0 && use_dag_mode(h->opt_trsm_dag, true, true, 4, k, nrhs))
            *bytes += dag_extra_bytes(k, nrhs, sl);
        return TRX_SUCCESS;
    }
    // FP64 TRSM on the mixed engine solves in FP32: that call's planes
    const bool mixed64 = elem_bytes == 8 && o == 'S' && h->opt_fp64_trsm > 0;
    bool tc = (elem_bytes == 4 || mixed64) ? use_tc<float>(h, k, o == 'S', nrhs) : false;
    if (upc(op) == 'G') {   // tensor-core trx_sgemm_update: m = M + K rows, n = N
        k = m;
        nrhs = n;
        tc = true;
    }
    *bytes = (tc && k > 0 && nrhs > 0) ? ws_layout(k, nrhs, slices_for(h)).total : 0;
    if (*bytes && o == 'S' && use_dag_mode(h->opt_trsm_dag, true, true, 4, k, nrhs))
        *bytes += dag_extra_bytes(k, nrhs, slices_for(h));
    return TRX_SUCCESS;
}

int trx_strsm(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
              float alpha, const float* A, int64_t lda, float* B, int64_t ldb, void* stream) {
    return execute<float>(h, true, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, stream);
}
int trx_dtrsm(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
              double alpha, const double* A, int64_t lda, double* B, int64_t ldb, void* stream) {
    return execute<double>(h, true, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, stream);
}
int trx_strmm(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
              float alpha, const float* A, int64_t lda, float* B, int64_t ldb, void* stream) {
    return execute<float>(h, false, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb, stream);
}
int trx_dtrmm(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
              double alpha, const double* A, int64_t lda, double* B, int64_t ldb, void* stream) {
    return execute<double>(h, false, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb,
                           stream);
}

int trx_strsm_refined(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t m,
                      int64_t n, float alpha, const float* A, int64_t lda, const float* B,
                      int64_t ldb, double* X, int64_t ldx, int max_iter, double tol,
                      trx_refine_info_t* info, void* stream) {
    // argument positions of this call: side 2 .. ldb 12 (the BLAS ones + 1),
    // X 13, ldx 14, max_iter 15, tol 16
    const int ia = check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    if (ia) return ia - 1;
    if (m > 0 && n > 0 && X == nullptr) return -13;
    if (ldx < std::max<int64_t>(1, m)) return -14;
    if (max_iter < 0) return -15;
    if (!(tol >= 0.0)) return -16;
    if (!valid(h)) return TRX_ERR_HANDLE;
    if (info) *info = trx_refine_info_t{0, 0.0, 0.0, 0.0};
    if (m == 0 || n == 0) return TRX_SUCCESS;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Internally always side L: X op(A) = alpha B is op(A)^T X^T = alpha B^T,
    // so side R works on the transposes with the transpose flag flipped.
    const bool left = upc(side) == 'L';
    const int64_t k = left ? m : n, nr = left ? n : m;
    const bool trans = upc(transa) != 'N';
    const char transI = (left ? trans : !trans) ? 'T' : 'N';
    const bool lower = upc(uplo) == 'L', unit = upc(diag) == 'U';
    const bool fp64_residual = h->opt_residual == 1;
    // FP32-grade residual on the tensor cores: op(A) fl32(X) by the library's
    // own FP32 TRMM with the 6-term split (accurate to a few units of 2^-24
    // of |op(A)| |X|: enough for backward errors down to about 1e-7)
    const bool tc_residual = h->opt_residual == 3;
    const bool ff_residual = !fp64_residual && !tc_residual;
    const bool lowerI = lower != (transI == 'T');
    // scratch: Xi, B64, R64 (k x nr FP64), D32 (k x nr FP32), row/column
    // sums, norms, and either the packed op(A) and X of the float-float
    // residual or an FP64 copy of A
    const size_t mn64 = align256((size_t)k * nr * 8), mn32 = align256((size_t)k * nr * 4);
    const size_t sums = align256(std::max((size_t)std::max(k, nr) * 8, refine_norm_scratch(k)));
    const size_t a64 = fp64_residual ? align256((size_t)k * k * 8) : 0;
    const size_t ap = ff_residual ? align256(refine_pack_a_bytes(k, lowerI)) : 0;
    const size_t xp = ff_residual ? align256(refine_pack_x_bytes(k, nr)) : 0;
    std::vector<int4> units, tiles;
    int64_t slots = 0;
    if (ff_residual) refine_plan_units(k, lowerI, units, tiles, slots);
    const size_t ub = align256((units.size() + tiles.size()) * sizeof(int4));
    const size_t pb = align256((size_t)slots * 64 * (size_t)nr * 8);
    const size_t need = 3 * mn64 + mn32 + sums + 256 + a64 + ap + xp + ub + pb;
    int rc0 = refine_scratch(h, need, s);
    if (rc0 != TRX_SUCCESS) return rc0;
    char* base = static_cast<char*>(h->rf_buf);
    double* Xi = reinterpret_cast<double*>(base);
    double* B64 = reinterpret_cast<double*>(base + mn64);
    double* R64 = reinterpret_cast<double*>(base + 2 * mn64);
    float* D32 = reinterpret_cast<float*>(base + 3 * mn64);
    double* sm = reinterpret_cast<double*>(base + 3 * mn64 + mn32);
    double* norms = reinterpret_cast<double*>(base + 3 * mn64 + mn32 + sums);
    char* tail = base + 3 * mn64 + mn32 + sums + 256;
    double* A64 = fp64_residual ? reinterpret_cast<double*>(tail) : nullptr;
    void* Ap = ff_residual ? tail : nullptr;
    void* Xp = ff_residual ? tail + ap : nullptr;
    int4* Ud = ff_residual ? reinterpret_cast<int4*>(tail + ap + xp) : nullptr;
    int4* Td = Ud ? Ud + units.size() : nullptr;
    double* part = ff_residual ? reinterpret_cast<double*>(tail + ap + xp + ub) : nullptr;
    // infinity norms of the caller's m x n arrays: row sums of the internal
    // k x nr array for side L, column sums for side R
    auto norm = [&](const double* a, double* out) {
        return left ? refine_norm_inf(a, k, k, nr, sm, out, s)
                    : refine_norm_one(a, k, k, nr, sm, out, s);
    };
    int rc;
    // 1. the FP32 solve (the plain recursive path), Xi := its result in FP64
    e = left ? cudaMemcpy2DAsync(D32, k * 4, B, ldb * 4, k * 4, nr, cudaMemcpyDeviceToDevice, s)
             : refine_transpose_f32(B, ldb, D32, k, m, n, s);
    if (e != cudaSuccess) return fail_cuda(e, "refine copy");
    if ((rc = execute<float>(h, true, 'L', uplo, transI, diag, k, nr, alpha, A, lda, D32, k,
                             stream)) != TRX_SUCCESS)
        return rc;
    if ((e = refine_cast_f32_f64(D32, k, Xi, k, k, nr, 1.0, s)) != cudaSuccess ||
        (e = left ? refine_cast_f32_f64(B, ldb, B64, k, k, nr, (double)alpha, s)
                  : refine_transpose_f32_f64(B, ldb, B64, k, m, n, (double)alpha, s)) !=
            cudaSuccess ||
        (fp64_residual && (e = refine_cast_f32_f64(A, lda, A64, k, k, k, 1.0, s)) != cudaSuccess) ||
        (ff_residual &&
         (e = refine_pack_a(A, lda, k, lowerI, transI == 'T', unit, Ap, s)) != cudaSuccess))
        return fail_cuda(e, "refine setup");
    if (ff_residual) {
        // the work-unit table (pageable source: staged before the call returns)
        std::vector<int4> table(units);
        table.insert(table.end(), tiles.begin(), tiles.end());
        if ((e = cudaMemcpyAsync(Ud, table.data(), table.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return fail_cuda(e, "refine setup");
    }
    // ||op(A)||_inf of the caller's op(A): row sums of op(A) with its own flag
    e = refine_op_norm_inf(A, lda, k, lower, trans, unit, sm, norms, s);
    if (e != cudaSuccess) return fail_cuda(e, "refine norm");
    double host[4] = {0, 0, 0, 0};
    int dev_err = 0;
    double eta0 = 0.0, eta = 0.0, eta_prev = 0.0, rnorm = 0.0;
    int it = 0;
    for (;; ++it) {
        // 2. the residual R = alpha B - op(A) X, products of FP32 data exact
        if (tc_residual) {
            // D32 := fl32(X), D32 := op(A) D32 (6-term split TRMM),
            // R := alpha B - D32 in FP64
            if ((e = refine_cast_f64_f32(Xi, k, D32, k, k, nr, s)) != cudaSuccess)
                return fail_cuda(e, "refine cast");
            if ((rc = execute<float>(h, false, 'L', uplo, transI, diag, k, nr, 1.0f, A, lda, D32,
                                     k, stream, nullptr, 6)) != TRX_SUCCESS)
                return rc;
            e = refine_cast_f32_f64(D32, k, R64, k, k, nr, 1.0, s);
            if (e == cudaSuccess) e = refine_residual(B64, k, R64, k, k, nr, s);
        } else if (fp64_residual) {
            // from X each time, on the FP64 pipe
            if ((e = cudaMemcpyAsync(R64, Xi, (size_t)k * nr * 8, cudaMemcpyDeviceToDevice, s)) !=
                cudaSuccess)
                return fail_cuda(e, "refine copy");
            if ((rc = execute<double>(h, false, 'L', uplo, transI, diag, k, nr, 1.0, A64, k, R64,
                                      k, stream)) != TRX_SUCCESS)
                return rc;
            e = refine_residual(B64, k, R64, k, k, nr, s);
        } else if (it == 0) {
            // from X = xh + xl, float-float
            e = refine_pack_x(Xi, nullptr, k, k, nr, Xp, s);
            if (e == cudaSuccess)
                e = refine_residual_packed(0, Ap, Xp, Ud, (int64_t)units.size(), Td,
                                           (int64_t)tiles.size(), part, k, lowerI, B64, k, R64, k,
                                           nr, h->d_err, h->wait_ns, s);
        } else {
            // updated by the last correction D (one float plane, D32):
            // R := R - op(A) D. The update's rounding is relative to
            // ||op(A)|| ||D||; plain FP32 accumulation (typical error
            // sqrt(k) 2^-24 of it, the same sqrt(k) reading as the default
            // tolerance) once that is below tol / 8 of ||op(A)|| ||X||,
            // float-float otherwise.
            const double rho = host[2] > 0 ? host[3] / host[2] : 0.0;
            const int mode = (std::sqrt((double)k) * 0x1p-24 * rho <= tol / 8) ? 2 : 1;
            e = refine_pack_x(nullptr, D32, k, k, nr, Xp, s);
            if (e == cudaSuccess)
                e = refine_residual_packed(mode, Ap, Xp, Ud, (int64_t)units.size(), Td,
                                           (int64_t)tiles.size(), part, k, lowerI, R64, k, R64, k,
                                           nr, h->d_err, h->wait_ns, s);
        }
        if (e != cudaSuccess || (e = norm(R64, norms + 1)) != cudaSuccess ||
            (it == 0 && (e = norm(Xi, norms + 2)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(host, norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(&dev_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail_cuda(e, "refine residual");
        if (dev_err != 0) {
            // a bounded wait in the residual kernel gave up: clear the word
            cudaMemsetAsync(h->d_err, 0, sizeof(int), s);
            cudaStreamSynchronize(s);
            snprintf(g_detail, sizeof(g_detail), "refine residual: device wait timed out");
            return TRX_ERR_TIMEOUT;
        }
        rnorm = host[1];
        const double den = host[0] * host[2];
        eta = den > 0 ? rnorm / den : rnorm;
        if (it == 0) eta0 = eta;
        // stop: converged, out of corrections, NaN, or no progress
        if (eta <= tol || it >= max_iter || !(eta == eta) || (it > 0 && eta >= eta_prev)) break;
        eta_prev = eta;
        // 3. correction: op(A) D = R solved in FP32, X += D; ||X||, ||D||
        if ((e = refine_cast_f64_f32(R64, k, D32, k, k, nr, s)) != cudaSuccess)
            return fail_cuda(e, "refine cast");
        if ((rc = execute<float>(h, true, 'L', uplo, transI, diag, k, nr, 1.0f, A, lda, D32, k,
                                 stream)) != TRX_SUCCESS)
            return rc;
        if ((e = refine_add(Xi, k, D32, k, k, nr, s)) != cudaSuccess ||
            (e = norm(Xi, norms + 2)) != cudaSuccess)
            return fail_cuda(e, "refine update");
        if (ff_residual &&
            ((e = refine_norm_f32(D32, k, k, nr, !left, sm, norms + 3, s)) != cudaSuccess ||
             (e = cudaMemcpyAsync(host + 2, norms + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                  s)) != cudaSuccess ||
             (e = cudaStreamSynchronize(s)) != cudaSuccess))
            return fail_cuda(e, "refine update");
    }
    // 4. the caller's X
    e = left ? cudaMemcpy2DAsync(X, ldx * 8, Xi, k * 8, k * 8, nr, cudaMemcpyDeviceToDevice, s)
             : refine_transpose_f64(Xi, k, X, ldx, k, nr, s);
    if (e != cudaSuccess) return fail_cuda(e, "refine result");
    if (info) *info = trx_refine_info_t{it, rnorm, eta, eta0};
    return TRX_SUCCESS;
}

}  // extern "C"

namespace {

// Grow the handle's refinement scratch to `need` bytes (a call that needs
// more than any before it). Stream-ordered: the old buffer is released after
// the stream's earlier work and the new one allocated in stream order, so
// neither the host nor the device waits.
int refine_scratch(trx_handle_t h, size_t need, cudaStream_t s) {
    if (h->rf_bytes >= need) return TRX_SUCCESS;
    if (h->rf_buf) cudaFreeAsync(h->rf_buf, s);
    h->rf_buf = nullptr;
    h->rf_bytes = 0;
    cudaError_t e = cudaMallocAsync(&h->rf_buf, need, s);
    if (e != cudaSuccess) {
        snprintf(g_detail, sizeof(g_detail), "refine scratch: %s", cudaGetErrorString(e));
        return TRX_ERR_ALLOC;
    }
    h->rf_bytes = need;
    return TRX_SUCCESS;
}

// Refinement with a fixed number of corrections and no host read-back:
// every step is enqueued on the stream. Data FP32 (A, B float) or FP64 (A,
// B double: the solves run on fl32(A) in FP32, the residual takes A as float
// pairs). X (FP64, leading dimension ldx) may be B for FP64 data (in place).
// Steps (side L internally; side R on the transposes, as trx_strsm_refined):
//   X := the FP32 solve of op(A) X = alpha B
//   repeat `corrections` times:
//     R := alpha B - op(A) X   (float-float on the FP32 pipes, from X)
//     D := the FP32 solve of op(A) D = fl32(R);  X := X + D (FP64)
int refine_fixed(trx_handle_t h, bool fp64_data, char side, char uplo, char transa, char diag,
                 int64_t m, int64_t n, double alpha, const void* A, int64_t lda, const void* B,
                 int64_t ldb, double* X, int64_t ldx, int corrections, void* stream) {
    if (m == 0 || n == 0) return TRX_SUCCESS;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool left = upc(side) == 'L';
    const int64_t k = left ? m : n, nr = left ? n : m;
    const bool trans = upc(transa) != 'N';
    const char transI = (left ? trans : !trans) ? 'T' : 'N';
    const bool lower = upc(uplo) == 'L', unit = upc(diag) == 'U';
    const bool lowerI = lower != (transI == 'T');
    const size_t mn64 = align256((size_t)k * nr * 8), mn32 = align256((size_t)k * nr * 4);
    const size_t a32 = fp64_data ? align256((size_t)k * k * 4) : 0;
    const size_t ap = align256(refine_pack_a_bytes(k, lowerI));
    const size_t xp = align256(refine_pack_x_bytes(k, nr));
    std::vector<int4> units, tiles;
    int64_t slots = 0;
    refine_plan_units(k, lowerI, units, tiles, slots);     // counts (the table: on the device)
    const size_t ub = align256((units.size() + tiles.size()) * sizeof(int4));
    const size_t pb = align256((size_t)slots * 64 * (size_t)nr * 8);
    // Orders up to the batched kernel's limit: every FP32 solve is one
    // persistent launch over 64-column panels of D (one problem per panel,
    // descriptors uploaded once per call: the first solve's with alpha, the
    // corrections' with 1), in place of the recursion's chain of launches.
    const bool small = k <= kBatchMaxK;
    const int64_t npan = small ? (nr + 63) / 64 : 0;
    const size_t db = small ? align256((size_t)2 * npan * sizeof(BatchDesc)) + 256 : 0;
    const size_t need = 3 * mn64 + mn32 + a32 + ap + xp + ub + pb + db;
    int rc = refine_scratch(h, need, s);
    if (rc != TRX_SUCCESS) return rc;
    // The solves launch directly: their graph key would hold this call's
    // right-hand-side count, so a server's stream of differently shaped
    // requests would capture and instantiate a new graph every time.
    struct GraphOff {
        trx_handle_t h;
        int64_t saved;
        ~GraphOff() { h->opt_graph = saved; }
    } graph_off{h, h->opt_graph};
    h->opt_graph = 0;
    char* base = static_cast<char*>(h->rf_buf);
    double* Xi = reinterpret_cast<double*>(base);
    double* B64 = reinterpret_cast<double*>(base + mn64);
    double* R64 = reinterpret_cast<double*>(base + 2 * mn64);
    float* D32 = reinterpret_cast<float*>(base + 3 * mn64);
    char* tail = base + 3 * mn64 + mn32;
    float* A32 = fp64_data ? reinterpret_cast<float*>(tail) : nullptr;
    void* Ap = tail + a32;
    void* Xp = tail + a32 + ap;
    int4* Ud = reinterpret_cast<int4*>(tail + a32 + ap + xp);
    int4* Td = Ud + units.size();
    double* part = reinterpret_cast<double*>(tail + a32 + ap + xp + ub);
    BatchDesc* Dd = small ? reinterpret_cast<BatchDesc*>(tail + a32 + ap + xp + ub + pb) : nullptr;
    int* dcount = small ? reinterpret_cast<int*>(reinterpret_cast<char*>(Dd) + db - 256) : nullptr;
    const float* As = fp64_data ? A32 : static_cast<const float*>(A);
    const int64_t ldas = fp64_data ? k : lda;
    const double* Bd = static_cast<const double*>(B);
    const float* Bf = static_cast<const float*>(B);
    // operands: fl32(A), D32 := B (for the first solve), B64 := alpha B, packed op(A)
    if (fp64_data &&
        (e = refine_cast_f64_f32(static_cast<const double*>(A), lda, A32, k, k, k, s)) !=
            cudaSuccess)
        return fail_cuda(e, "refine setup");
    if (fp64_data)
        e = left ? refine_cast_f64_f32(Bd, ldb, D32, k, k, nr, s)
                 : refine_transpose_f64_f32(Bd, ldb, D32, k, m, n, s);
    else
        e = left ? cudaMemcpy2DAsync(D32, k * 4, Bf, ldb * 4, k * 4, nr, cudaMemcpyDeviceToDevice,
                                     s)
                 : refine_transpose_f32(Bf, ldb, D32, k, m, n, s);
    if (e == cudaSuccess) {
        if (fp64_data)
            e = left ? refine_scale_f64(Bd, ldb, B64, k, k, nr, alpha, s)
                     : refine_transpose_f64_scaled(Bd, ldb, B64, k, m, n, alpha, s);
        else
            e = left ? refine_cast_f32_f64(Bf, ldb, B64, k, k, nr, alpha, s)
                     : refine_transpose_f32_f64(Bf, ldb, B64, k, m, n, alpha, s);
    }
    if (e == cudaSuccess)
        e = fp64_data ? refine_pack_a64(static_cast<const double*>(A), lda, k, lowerI,
                                        transI == 'T', unit, Ap, s)
                      : refine_pack_a(static_cast<const float*>(A), lda, k, lowerI, transI == 'T',
                                      unit, Ap, s);
    if (e == cudaSuccess) e = refine_plan_units_device(k, lowerI, Ud, Td, s);
    if (e == cudaSuccess && small) {
        std::vector<BatchDesc> dv((size_t)(2 * npan));
        for (int64_t q = 0; q < 2 * npan; ++q) {
            const int64_t j0 = (q % npan) * 64, nc = std::min<int64_t>(64, nr - j0);
            const Canon<float> c = canonicalize<float>('L', uplo, transI, diag, k, nc, As, ldas,
                                                       D32 + j0 * k, k);
            BatchDesc& d = dv[(size_t)q];
            std::memset(&d, 0, sizeof(d));
            d.k = c.k; d.nrhs = c.nrhs; d.A = c.A; d.a_rs = c.a_rs; d.a_cs = c.a_cs;
            d.C = c.C; d.c_rs = c.c_rs; d.c_cs = c.c_cs; d.unit = c.unit;
            d.alpha = q < npan ? alpha : 1.0;
            d.trsm = 1;
            d.sb = (&h->tune_sb[0][0][0])[tune_index(k, nc)];
        }
        // pageable source: staged before the call returns
        e = cudaMemcpyAsync(Dd, dv.data(), dv.size() * sizeof(BatchDesc), cudaMemcpyHostToDevice,
                            s);
    }
    if (e != cudaSuccess) return fail_cuda(e, "refine setup");
    const int bgrid = h->num_sms * batched_ctas_per_sm(4);
    // one FP32 solve of op(A) D = alpha D in place (first: alpha, else 1)
    auto solve32 = [&](bool first) -> int {
        if (small) {
            const cudaError_t le = launch_batched(4, Dd + (first ? 0 : npan), npan, dcount, bgrid,
                                                  s);
            return le == cudaSuccess ? TRX_SUCCESS : fail_cuda(le, "refine solve");
        }
        return execute<float>(h, true, 'L', uplo, transI, diag, k, nr,
                              first ? (float)alpha : 1.0f, As, ldas, D32, k, stream);
    };
    // the FP32 solve, Xi := its result
    if ((rc = solve32(true)) != TRX_SUCCESS) return rc;
    if ((e = refine_cast_f32_f64(D32, k, Xi, k, k, nr, 1.0, s)) != cudaSuccess)
        return fail_cuda(e, "refine cast");
    for (int it = 0; it < corrections; ++it) {
        e = refine_pack_x(Xi, nullptr, k, k, nr, Xp, s);
        if (e == cudaSuccess)
            e = refine_residual_packed(fp64_data ? 3 : 0, Ap, Xp, Ud, (int64_t)units.size(), Td,
                                       (int64_t)tiles.size(), part, k, lowerI, B64, k, R64, k, nr,
                                       h->d_err, h->wait_ns, s);
        if (e == cudaSuccess) e = refine_cast_f64_f32(R64, k, D32, k, k, nr, s);
        if (e != cudaSuccess) return fail_cuda(e, "refine residual");
        if ((rc = solve32(false)) != TRX_SUCCESS) return rc;
        if ((e = refine_add(Xi, k, D32, k, k, nr, s)) != cudaSuccess)
            return fail_cuda(e, "refine update");
    }
    e = left ? cudaMemcpy2DAsync(X, ldx * 8, Xi, k * 8, k * 8, nr, cudaMemcpyDeviceToDevice, s)
             : refine_transpose_f64(Xi, k, X, ldx, k, nr, s);
    return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "refine result");
}

// FP64 TRMM in one float-float pass on the FP32 pipes: B := alpha op(A) B
// as R := 0 - op(A) (-alpha B) by the refinement residual's kernel (mode 3:
// op(A) packed as float pairs, B scaled in FP64 and split into pairs; the
// sums kept in two float pairs and added in FP64 at the end). Side R on
// the transpose, B^T := alpha op(A)^T B^T, through a k x m copy.
int pair_trmm(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
              double alpha, const double* A, int64_t lda, double* B, int64_t ldb,
              cudaStream_t s) {
    const bool left = upc(side) == 'L';
    const int64_t k = left ? m : n, nr = left ? n : m;
    const bool trans = upc(transa) != 'N';
    const bool transI = left ? trans : !trans;
    const bool lowerI = (upc(uplo) == 'L') != transI, unit = upc(diag) == 'U';
    const size_t ap = align256(refine_pack_a_bytes(k, lowerI));
    const size_t xp = align256(refine_pack_x_bytes(k, nr));
    std::vector<int4> units, tiles;
    int64_t slots = 0;
    refine_plan_units(k, lowerI, units, tiles, slots);
    const size_t ub = align256((units.size() + tiles.size()) * sizeof(int4));
    const size_t pb = align256((size_t)slots * 64 * (size_t)nr * 8);
    const size_t bt = left ? 0 : align256((size_t)k * nr * 8);
    const int rc = refine_scratch(h, ap + xp + ub + pb + bt, s);
    if (rc != TRX_SUCCESS) return rc;
    char* base = static_cast<char*>(h->rf_buf);
    void* Ap = base;
    void* Xp = base + ap;
    int4* Ud = reinterpret_cast<int4*>(base + ap + xp);
    int4* Td = Ud + units.size();
    double* part = reinterpret_cast<double*>(base + ap + xp + ub);
    double* Bt = left ? B : reinterpret_cast<double*>(base + ap + xp + ub + pb);
    const int64_t ldt = left ? ldb : k;
    cudaError_t e = refine_pack_a64(A, lda, k, lowerI, transI, unit, Ap, s);
    if (e == cudaSuccess) e = refine_plan_units_device(k, lowerI, Ud, Td, s);
    if (e == cudaSuccess && !left) e = refine_transpose_f64(B, ldb, Bt, k, m, n, s);
    if (e == cudaSuccess) e = refine_pack_x(Bt, nullptr, ldt, k, nr, Xp, s, -alpha);
    if (e == cudaSuccess)
        e = refine_residual_packed(3, Ap, Xp, Ud, (int64_t)units.size(), Td,
                                   (int64_t)tiles.size(), part, k, lowerI, nullptr, 0, Bt, ldt,
                                   nr, h->d_err, h->wait_ns, s);
    if (e == cudaSuccess && !left) e = refine_transpose_f64(Bt, k, B, ldb, k, m, s);
    return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "float-float TRMM");
}

}  // namespace

extern "C" {

int trx_strsm_refined_async(trx_handle_t h, char side, char uplo, char transa, char diag,
                            int64_t m, int64_t n, float alpha, const float* A, int64_t lda,
                            const float* B, int64_t ldb, double* X, int64_t ldx, int corrections,
                            void* stream) {
    // argument positions as trx_strsm_refined; corrections 15
    const int ia = check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    if (ia) return ia - 1;
    if (m > 0 && n > 0 && X == nullptr) return -13;
    if (ldx < std::max<int64_t>(1, m)) return -14;
    if (corrections < 0 || corrections > 16) return -15;
    if (!valid(h)) return TRX_ERR_HANDLE;
    if (m == 0 || n == 0) return TRX_SUCCESS;
    return refine_fixed(h, false, side, uplo, transa, diag, m, n, (double)alpha, A, lda, B, ldb, X,
                        ldx, corrections, stream);
}

int trx_sfactor_create(trx_handle_t h, char side, char uplo, char transa, char diag, int64_t k,
                       const float* A, int64_t lda, void* stream, trx_factor_t* out) {
    if (!out) return TRX_ERR_INVALID_VALUE;
    *out = nullptr;
    // argument positions of this call: side 2, uplo 3, transa 4, diag 5,
    // k 6, A 7, lda 8
    const int info = check_args(side, uplo, transa, diag, k, k, A, lda, A, std::max<int64_t>(1, k));
    if (info >= -4 && info <= -1) return info - 1;
    if (info == -5 || info == -6) return -6;
    if (info == -8) return -7;
    if (info == -9) return -8;
    if (!valid(h)) return TRX_ERR_HANDLE;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    auto* f = new (std::nothrow) trx_factor_s;
    if (!f) return TRX_ERR_ALLOC;
    f->device = h->device;
    f->side = (char)upc(side);
    f->uplo = (char)upc(uplo);
    f->transa = (char)upc(transa);
    f->diag = (char)upc(diag);
    f->k = k;
    f->lda = lda;
    f->A = A;
    f->slices = slices_for(h);
    if (k > kMaxLeaf) {                 // some call on it may take the tensor-core path
        const WsLayout w = ws_layout(k, 0, f->slices);
        f->ldm = w.ldm;
        if ((e = cudaMalloc(&f->m_hi, w.m_bytes)) != cudaSuccess ||
            (f->slices > 1 && (e = cudaMalloc(&f->m_lo, w.m_bytes)) != cudaSuccess) ||
            (f->slices > 2 && (e = cudaMalloc(&f->m_lo2, w.m_bytes)) != cudaSuccess)) {
            if (f->m_hi) cudaFree(f->m_hi);
            if (f->m_lo) cudaFree(f->m_lo);
            delete f;
            snprintf(g_detail, sizeof(g_detail), "factor planes: %s", cudaGetErrorString(e));
            return TRX_ERR_ALLOC;
        }
    }
    f->magic = kFactorMagic;
    const int rc = trx_sfactor_update(h, f, A, stream);
    if (rc != TRX_SUCCESS) {
        trx_factor_destroy(f);
        return rc;
    }
    *out = f;
    return TRX_SUCCESS;
}

int trx_sfactor_update(trx_handle_t h, trx_factor_t f, const float* A, void* stream) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if (!f || f->magic != kFactorMagic || f->device != h->device) return TRX_ERR_INVALID_VALUE;
    if (A == nullptr && f->k > 0) return -3;           // A is argument 3 of this call
    f->A = A;
    if (!f->m_hi || f->k == 0) return TRX_SUCCESS;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    pdl_enabled() = h->opt_pdl != 0;
    const bool left = f->side == 'L';
    const Canon<float> c = canonicalize<float>(f->side, f->uplo, f->transa, f->diag,
                                               left ? f->k : 1, left ? 1 : f->k, A, f->lda,
                                               nullptr, f->k);
    Planes pl;
    pl.ldm = f->ldm;
    pl.ldy = f->ldm;
    pl.slices = f->slices;
    pl.m_hi = f->m_hi;
    pl.m_lo = f->m_lo;
    pl.m_lo2 = f->m_lo2;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->opt_profile) {
        e0 = get_event(h);
        e1 = get_event(h);
        cudaEventRecord(e0, s);
    }
    e = launch_convert_m(c, pl, kFactorDenseRows, s);
    if (e != cudaSuccess) return fail_cuda(e, "factor planes");
    // inverted diagonal blocks for TRSM leaves on the tensor cores, at the
    // leaf size FP32 TRSM calls on this factor take
    const int wb = leaf_for(h->opt_leaf, f->k, true, 4, 0);
    if (tc_leaf_mode(h->opt_trsm_tc_leaf, true, wb)) {
        if (!f->w_hi) {
            const WsLayout w = ws_layout(f->k, 0, f->slices);
            if ((e = cudaMalloc(&f->w_hi, w.m_bytes)) != cudaSuccess ||
                (f->slices > 1 && (e = cudaMalloc(&f->w_lo, w.m_bytes)) != cudaSuccess) ||
                (f->slices > 2 && (e = cudaMalloc(&f->w_lo2, w.m_bytes)) != cudaSuccess)) {
                if (f->w_hi) cudaFree(f->w_hi);
                if (f->w_lo) cudaFree(f->w_lo);
                f->w_hi = f->w_lo = f->w_lo2 = nullptr;
                snprintf(g_detail, sizeof(g_detail), "factor inverse planes: %s",
                         cudaGetErrorString(e));
                return TRX_ERR_ALLOC;
            }
        }
        if ((e = launch_invert_diag(c, wb, f->w_hi, f->w_lo, f->w_lo2, f->slices, f->ldm, s)) !=
            cudaSuccess)
            return fail_cuda(e, "factor inverse planes");
        f->w_block = wb;
    } else {
        f->w_block = 0;               // stale inverses are not used
    }
    if (h->opt_profile) {
        cudaEventRecord(e1, s);
        h->pending.push_back({TRX_KERNEL_CONVERT, 0.0, 8.0 * f->k * (f->k - 1) / 2, e0, e1});
    }
    return TRX_SUCCESS;
}

int trx_factor_destroy(trx_factor_t f) {
    if (f == nullptr) return TRX_SUCCESS;
    if (f->magic != kFactorMagic) return TRX_ERR_INVALID_VALUE;
    cudaSetDevice(f->device);
    cudaDeviceSynchronize();
    if (f->m_hi) cudaFree(f->m_hi);
    if (f->m_lo) cudaFree(f->m_lo);
    if (f->m_lo2) cudaFree(f->m_lo2);
    if (f->w_hi) cudaFree(f->w_hi);
    if (f->w_lo) cudaFree(f->w_lo);
    if (f->w_lo2) cudaFree(f->w_lo2);
    f->magic = 0;
    delete f;
    return TRX_SUCCESS;
}

static int factor_call(trx_handle_t h, trx_factor_t f, bool trsm, int64_t nrhs, float alpha,
                       float* B, int64_t ldb, void* stream) {
    if (!f || f->magic != kFactorMagic) return TRX_ERR_INVALID_VALUE;
    if (valid(h) && f->device != h->device) return TRX_ERR_INVALID_VALUE;
    const bool left = f->side == 'L';
    const int64_t m = left ? f->k : nrhs, n = left ? nrhs : f->k;
    // argument positions of the factor calls: nrhs 3, B 5, ldb 6
    const int info = check_args(f->side, f->uplo, f->transa, f->diag, m, n, f->A, f->lda, B, ldb);
    if (info == -5 || info == -6) return -3;
    if (info == -10) return -5;
    if (info == -11) return -6;
    if (info) return info;
    return execute<float>(h, trsm, f->side, f->uplo, f->transa, f->diag, m, n, alpha, f->A,
                          f->lda, B, ldb, stream, f);
}

int trx_strsm_factor(trx_handle_t h, trx_factor_t f, int64_t nrhs, float alpha, float* B,
                     int64_t ldb, void* stream) {
    return factor_call(h, f, true, nrhs, alpha, B, ldb, stream);
}

int trx_strmm_factor(trx_handle_t h, trx_factor_t f, int64_t nrhs, float alpha, float* B,
                     int64_t ldb, void* stream) {
    return factor_call(h, f, false, nrhs, alpha, B, ldb, stream);
}

int trx_sgemm_update(trx_handle_t h, int64_t M, int64_t N, int64_t K, float beta, float gamma,
                     const float* A, int64_t lda, const float* Y, int64_t ldy, float* C,
                     int64_t ldc, int engine, void* stream) {
    if (M < 0) return -2;
    if (N < 0) return -3;
    if (K < 0) return -4;
    if (M > 0 && K > 0 && A == nullptr) return -7;
    if (lda < std::max<int64_t>(1, M)) return -8;
    if (K > 0 && N > 0 && Y == nullptr) return -9;
    if (ldy < std::max<int64_t>(1, K)) return -10;
    if (M > 0 && N > 0 && C == nullptr) return -11;
    if (ldc < std::max<int64_t>(1, M)) return -12;
    if (engine != 1 && engine != 2) return -13;
    if (!valid(h)) return TRX_ERR_HANDLE;
    if (M == 0 || N == 0) return TRX_SUCCESS;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    // Canonical frame: rows [0, K) hold Y, rows [K, K+M) hold C, and
    // M(K+i, l) = A(i, l); the update is rc = K, rk = 0.
    Canon<float> c;
    c.k = K + M;
    c.nrhs = N;
    c.A = A - K;
    c.a_rs = 1;
    c.a_cs = lda;
    c.C = C - K;
    c.c_rs = 1;
    c.c_cs = ldc;
    if (engine == 1 || K == 0) {
        e = launch_gemm_simt<float>(c, Y, 1, ldy, K, M, 0, K, beta, K == 0 ? 0.f : gamma, s,
                                    h->num_sms);
        return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "gemm_simt");
    }
    if (K % kTcKQuantum != 0) return -4;
    const int slices = slices_for(h);
    const WsLayout w = ws_layout(K + M, N, slices);
    if (h->ws == nullptr || h->ws_bytes < w.total) {
        snprintf(g_detail, sizeof(g_detail), "workspace of %zu bytes needed, %zu set", w.total,
                 h->ws_bytes);
        return TRX_ERR_WORKSPACE;
    }
    char* base = static_cast<char*>(h->ws);
    Planes pl;
    pl.ldm = w.ldm;
    pl.ldy = w.ldy;
    pl.slices = slices;
    set_m_planes(pl, base, w.m_bytes, slices);
    set_y_planes(pl, base + (size_t)slices * w.m_bytes, w.y_bytes, slices);
    auto rowk = [&](__nv_bfloat16* q) { return q ? q + K * pl.ldm : nullptr; };
    if ((e = launch_convert_rect(A, 1, lda, M, K, rowk(pl.m_hi), rowk(pl.m_lo), rowk(pl.m_lo2),
                                 slices, pl.ldm, true, s)) != cudaSuccess ||
        (e = launch_convert_rect(Y, 1, ldy, K, N, pl.y_hi, pl.y_lo, pl.y_lo2, slices, pl.ldy,
                                 false, s)) != cudaSuccess)
        return fail_cuda(e, "convert");
    h->maps.resize(tc_maps_size());
    if ((e = tc_make_maps(pl, K + M, N, h->maps.data())) != cudaSuccess)
        return fail_cuda(e, "tensor map encode");
    const TcGemm g{K, M, 0, K};
    e = launch_gemm_tc(c, h->maps.data(), slices, &g, 1, beta, gamma, h->d_err, h->wait_ns,
                       h->num_sms, s);
    return e == cudaSuccess ? TRX_SUCCESS : fail_cuda(e, "gemm_tc");
}

int trx_set_option(trx_handle_t h, int option, int64_t value) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    switch (option) {
        case TRX_OPT_LEAF:
            if (value != 0 && value != 16 && value != 32 && value != 64 && value != 128 &&
                value != 256)
                return TRX_ERR_INVALID_VALUE;
            h->opt_leaf = value;
            break;
        case TRX_OPT_GEMM:
            if (value < 0 || value > 2) return TRX_ERR_INVALID_VALUE;
            h->opt_gemm = value;
            break;
        case TRX_OPT_GRAPH:
            if (value != 0 && value != 1) return TRX_ERR_INVALID_VALUE;
            h->opt_graph = value;
            break;
        case TRX_OPT_PROFILE:
            if (value != 0 && value != 1) return TRX_ERR_INVALID_VALUE;
            h->opt_profile = value;
            break;
        case TRX_OPT_WAIT_LIMIT:
            if (value < 1000) return TRX_ERR_INVALID_VALUE;
            h->wait_ns = value;
            break;
        case TRX_OPT_PDL:
            if (value != 0 && value != 1) return TRX_ERR_INVALID_VALUE;
            h->opt_pdl = value;
            break;
        case TRX_OPT_PANELS:
            if (value < 0 || value > kMaxPanels) return TRX_ERR_INVALID_VALUE;
            h->opt_panels = value;
            break;
        case TRX_OPT_TRMM_DENSE:
            if (value != -1 && value != 0 && value != 64 && value != 128 && value != 256 &&
                value != 512 && value != 1024 && value != 2048)
                return TRX_ERR_INVALID_VALUE;
            h->opt_trmm_dense = value;
            break;
        case TRX_OPT_RESIDUAL:
            if (value < 0 || value > 3) return TRX_ERR_INVALID_VALUE;
            h->opt_residual = value;
            break;
        case TRX_OPT_TRSM_TC_LEAF:
            if (value < -1 || value > 1) return TRX_ERR_INVALID_VALUE;
            h->opt_trsm_tc_leaf = value;
            break;
        case TRX_OPT_SPLIT:
            if (value != 0 && value != 1 && value != 3 && value != 6) return TRX_ERR_INVALID_VALUE;
            h->opt_split = value;
            break;
        case TRX_OPT_FP64_TRSM:
            if (value < 0 || value > 16) return TRX_ERR_INVALID_VALUE;
            h->opt_fp64_trsm = value;
            break;
        case TRX_OPT_CHECKED:
            if (value != 0 && value != 1) return TRX_ERR_INVALID_VALUE;
            h->opt_checked = value;
            break;
        case TRX_OPT_NVTX:
            if (value != 0 && value != 1) return TRX_ERR_INVALID_VALUE;
            h->opt_nvtx = value;
            break;
        case TRX_OPT_TRSM_DAG:
            if (value < -1 || value > 1) return TRX_ERR_INVALID_VALUE;
            h->opt_trsm_dag = value;
            break;
        case TRX_OPT_FP64_TRMM:
            if (value != 0 && value != 1) return TRX_ERR_INVALID_VALUE;
            h->opt_fp64_trmm = value;
            break;
        case TRX_OPT_THIN:
            if (value < -1 || value > 1) return TRX_ERR_INVALID_VALUE;
            h->opt_thin = value;
            break;
        case TRX_OPT_TEST_WITHHOLD:
            if (value != 0 && value != 1) return TRX_ERR_INVALID_VALUE;
            h->opt_test_withhold = value;
            break;
        case TRX_OPT_THIN_LEAF:
            if (!(value == -1 || value == 0 || (value >= 256 && value <= 8192 && value % 128 == 0)))
                return TRX_ERR_INVALID_VALUE;
            h->opt_thin_leaf = value;
            break;
        default:
            return TRX_ERR_INVALID_VALUE;
    }
    return TRX_SUCCESS;
}

int trx_get_option(trx_handle_t h, int option, int64_t* value) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    if (!value) return TRX_ERR_INVALID_VALUE;
    switch (option) {
        case TRX_OPT_LEAF: *value = h->opt_leaf; break;
        case TRX_OPT_GEMM: *value = h->opt_gemm; break;
        case TRX_OPT_GRAPH: *value = h->opt_graph; break;
        case TRX_OPT_PROFILE: *value = h->opt_profile; break;
        case TRX_OPT_WAIT_LIMIT: *value = h->wait_ns; break;
        case TRX_OPT_PDL: *value = h->opt_pdl; break;
        case TRX_OPT_PANELS: *value = h->opt_panels; break;
        case TRX_OPT_TRMM_DENSE: *value = h->opt_trmm_dense; break;
        case TRX_OPT_RESIDUAL: *value = h->opt_residual; break;
        case TRX_OPT_TRSM_TC_LEAF: *value = h->opt_trsm_tc_leaf; break;
        case TRX_OPT_SPLIT: *value = split_terms(h->opt_split); break;
        case TRX_OPT_FP64_TRSM: *value = h->opt_fp64_trsm; break;
        case TRX_OPT_CHECKED: *value = h->opt_checked; break;
        case TRX_OPT_NVTX: *value = h->opt_nvtx; break;
        case TRX_OPT_TRSM_DAG: *value = h->opt_trsm_dag; break;
        case TRX_OPT_FP64_TRMM: *value = h->opt_fp64_trmm; break;
        case TRX_OPT_THIN: *value = h->opt_thin; break;
        case TRX_OPT_TEST_WITHHOLD: *value = h->opt_test_withhold; break;
        case TRX_OPT_THIN_LEAF: *value = h->opt_thin_leaf; break;
        default: return TRX_ERR_INVALID_VALUE;
    }
    return TRX_SUCCESS;
}

int trx_get_profile(trx_handle_t h, trx_profile_t* out, int reset) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    cudaSetDevice(h->device);
    for (auto& p : h->pending) {
        cudaError_t e = cudaEventSynchronize(p.e1);
        if (e != cudaSuccess) return fail_cuda(e, "cudaEventSynchronize");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.e0, p.e1);
        h->prof.ms[p.cls] += ms;
        h->prof.flops[p.cls] += p.flops;
        h->prof.bytes[p.cls] += p.bytes;
        h->prof.launches[p.cls] += 1;
        h->free_events.push_back(p.e0);
        h->free_events.push_back(p.e1);
    }
    h->pending.clear();
    if (out) *out = h->prof;
    if (reset) std::memset(&h->prof, 0, sizeof(h->prof));
    return TRX_SUCCESS;
}

int trx_check_device_error(trx_handle_t h) {
    if (!valid(h)) return TRX_ERR_HANDLE;
    cudaSetDevice(h->device);
    int v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "cudaDeviceSynchronize");
    e = cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(e, "read error word");
    if (v != 0) {
        cudaMemset(h->d_err, 0, sizeof(int));
        return v;
    }
    return TRX_SUCCESS;
}

const char* trx_error_string(int code) {
    if (code < 0 && code >= -11) {
        static const char* names[] = {"side", "uplo", "transa", "diag", "m", "n",
                                      "alpha", "A", "lda", "B", "ldb"};
        static thread_local char buf[64];
        snprintf(buf, sizeof(buf), "illegal argument %d (%s)", -code, names[-code - 1]);
        return buf;
    }
    switch (code) {
        case TRX_SUCCESS: return "success";
        case TRX_ERR_HANDLE: return "invalid handle";
        case TRX_ERR_CUDA: return "CUDA error";
        case TRX_ERR_WORKSPACE: return "workspace missing or too small";
        case TRX_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case TRX_ERR_DEVICE: return "device is not sm_103 (GB300)";
        case TRX_ERR_ALLOC: return "allocation failed";
        case TRX_ERR_INVALID_VALUE: return "invalid option or value";
        default: return "unknown error";
    }
}

const char* trx_last_error_detail(void) { return g_detail; }

int trx_debug_plan(char op, char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                   int elem_bytes, int leaf, int gemm_mode, int trmm_dense, int trsm_tc_leaf,
                   int thin_leaf, char* buf, size_t buflen) {
    const int info = check_args(side, uplo, transa, diag, m, n, "", std::max<int64_t>(1, upc(side) == 'L' ? m : n),
                                "", std::max<int64_t>(1, m));
    if (info) return info;
    if ((upc(op) != 'S' && upc(op) != 'M') || (elem_bytes != 4 && elem_bytes != 8) ||
        (leaf != 0 && leaf != 16 && leaf != 32 && leaf != 64 && leaf != 128 && leaf != 256) ||
        gemm_mode < 0 ||
        gemm_mode > 2 || !buf || buflen == 0 ||
        (trmm_dense != -1 && trmm_dense != 0 && trmm_dense != 64 && trmm_dense != 128 &&
         trmm_dense != 256 && trmm_dense != 512 && trmm_dense != 1024 && trmm_dense != 2048) ||
        trsm_tc_leaf < -1 || trsm_tc_leaf > 1 ||
        !(thin_leaf == -1 || thin_leaf == 0 ||
          (thin_leaf >= 256 && thin_leaf <= 8192 && thin_leaf % 128 == 0)))
        return TRX_ERR_INVALID_VALUE;
    buf[0] = 0;
    const int64_t k = upc(side) == 'L' ? m : n;
    if (m == 0 || n == 0) return TRX_SUCCESS;
    const bool is_trsm = upc(op) == 'S';
    const int64_t nrhs = upc(side) == 'L' ? n : m;
    int b = leaf_for(leaf, k, is_trsm, elem_bytes, nrhs);
    Plan plan;
    plan.tc = use_tc_mode(elem_bytes, gemm_mode, k, b);
    const int tl = thin_leaf_rows((leaf != 0 && thin_leaf == 0) ? -1 : thin_leaf, plan.tc,
                                  is_trsm, elem_bytes, k, nrhs);
    if (tl > 0) b = tl;
    plan.thin_leaf = tl > 0;
    plan.tc_leaf = is_trsm && elem_bytes == 4 && !plan.thin_leaf &&
                   tc_leaf_mode(trsm_tc_leaf, plan.tc, b);
    const int dense = is_trsm ? 0 : trmm_dense_mode(trmm_dense, leaf, plan.tc, k);
    make_plan(plan, is_trsm, k, b, 2.0, true, dense);
    if (const char* why = validate_plan(plan, k)) {
        snprintf(g_detail, sizeof(g_detail), "plan check: %s", why);
        return TRX_ERR_INVALID_VALUE;
    }
    std::string out;
    char line[256];
    for (const Step& st : plan.steps) {
        switch (st.kind) {
            case kConvM:
                snprintf(line, sizeof(line), "conv_m diag_block=%d\n", st.b);
                out += line;
                break;
            case kConvY: out += "conv_y\n"; break;
            case kConvYRows:
                snprintf(line, sizeof(line), "conv_y_rows r0=%lld b=%d\n", (long long)st.r0, st.b);
                out += line;
                break;
            case kInvDiag:
                snprintf(line, sizeof(line), "inv_diag b=%d\n", st.b);
                out += line;
                break;
            case kThin:
                snprintf(line, sizeof(line), "thin trsm=%d r0=%lld b=%d alpha=%.17g planes=%d\n",
                         (int)st.trsm, (long long)st.r0, st.b, st.alpha, (int)st.planes);
                out += line;
                break;
            case kLeaf:
                snprintf(line, sizeof(line), "leaf trsm=%d r0=%lld b=%d nleaves=%lld alpha=%.17g planes=%d\n",
                         (int)st.trsm, (long long)st.r0, st.b, (long long)st.nleaves, st.alpha,
                         (int)st.planes);
                out += line;
                break;
            case kGemm:
                for (size_t i = 0; i < st.gemms.size(); ++i) {
                    const TcGemm& g = st.gemms[i];
                    snprintf(line, sizeof(line),
                             "gemm tc=%d member=%zu rc=%lld mlen=%lld rk=%lld klen=%lld beta=%.17g "
                             "gamma=%.17g dense=%d inv=%d y0=%lld y1=%lld\n",
                             (int)st.tc, i, (long long)g.rc, (long long)g.mlen, (long long)g.rk,
                             (long long)g.klen, st.beta, st.gamma, (int)st.dense, (int)st.inv,
                             (long long)st.y0, (long long)st.y1);
                    out += line;
                }
                break;
        }
    }
    if (out.size() + 1 > buflen) return TRX_ERR_INVALID_VALUE;
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return TRX_SUCCESS;
}

int trx_version(void) { return 100; }

// Upload of the triangle a call reads: one rectangular copy per block of
// 256 columns (rows j0..k-1 of the block for 'L', 0..j1-1 for 'U'), so the
// other triangle's bytes, all but the parts inside the 256 x 256 diagonal
// blocks, stay on the host.
int trx_copy_triangle_h2d(char uplo, int64_t k, int elem, const void* A_host, int64_t lda_host,
                          void* A_dev, int64_t lda_dev, void* stream) {
    const char u = (char)std::toupper((unsigned char)uplo);
    if (u != 'L' && u != 'U') return -1;
    if (k < 0) return -2;
    if (elem != 4 && elem != 8) return -3;
    if (k > 0 && A_host == nullptr) return -4;
    if (lda_host < std::max<int64_t>(1, k)) return -5;
    if (k > 0 && A_dev == nullptr) return -6;
    if (lda_dev < std::max<int64_t>(1, k)) return -7;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    constexpr int64_t kBlock = 256;
    for (int64_t j0 = 0; j0 < k; j0 += kBlock) {
        const int64_t j1 = std::min(k, j0 + kBlock);
        const int64_t r0 = u == 'L' ? j0 : 0, r1 = u == 'L' ? k : j1;
        const char* src = static_cast<const char*>(A_host) + (r0 + j0 * lda_host) * elem;
        char* dst = static_cast<char*>(A_dev) + (r0 + j0 * lda_dev) * elem;
        const cudaError_t e =
            cudaMemcpy2DAsync(dst, (size_t)(lda_dev * elem), src, (size_t)(lda_host * elem),
                              (size_t)((r1 - r0) * elem), (size_t)(j1 - j0),
                              cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail_cuda(e, "triangle upload");
    }
    return TRX_SUCCESS;
}

}  // extern "C"

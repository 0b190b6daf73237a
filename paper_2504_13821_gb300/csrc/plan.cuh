// Launch planning for one call: the recursion tree of Section 3.1 as an
// ordered list of steps (operand-plane conversions, leaves, GEMM updates),
// and the automatic choices that shape it (leaf cutoff, tensor-core engine,
// TRMM diagonal blocks). Host code only, no device work.
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace trx {

constexpr int kDefaultLeaf = 64;
// Automatic cutoff for FP32 TRSM: 128-row leaves (one leaf launch in place of
// two 64-row leaves and the update between them; measured faster at 256 ..
// 16384 right-hand sides, with the wide leaf kernel from 1024). Block leaves
// (256) are never chosen automatically (measured slower); TRX_OPT_LEAF = 256
// asks.
constexpr int kF32TrsmLeaf = 128;
constexpr int64_t kTcMinOrder = 256;                 // auto: tensor cores from this order
constexpr int64_t kTrmmDenseMinOrder = 1024;         // auto: dense TRMM diagonal blocks from here
constexpr int kTrmmDenseRows = 1024;                 // auto: their size

inline int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

// Section 3.1 splits at n = N/2. For orders that are not powers of two the
// split is rounded up to a multiple of max(b, 64) (so every tensor-core GEMM
// update has K a multiple of its K tile, and every node starts on a multiple
// of b), or of b where that would leave the second half empty.
inline int64_t split_point(int64_t s, int b) {
    const int64_t half = (s + 1) / 2;
    const int64_t q = std::max<int64_t>(b, kTcKQuantum);
    int64_t s1 = round_up(half, q);
    if (s1 >= s) s1 = round_up(half, b);
    return s1;
}

enum StepKind { kLeaf, kGemm, kConvM, kConvY, kConvYRows, kInvDiag, kInvCompact, kDag, kThin };

struct Step {
    StepKind kind;
    bool trsm = true;        // leaf: TRSM or TRMM
    int64_t r0 = 0;          // leaf: first row
    int b = 0;               // leaf: size (and stride of batched leaves); conv_m: diagonal
                             // block carried densely in the planes (0: none)
    int64_t nleaves = 1;
    double alpha = 1.0;      // leaf scale
    bool planes = false;     // TRSM leaf writes Y planes
    bool tc = false;         // GEMM on tensor cores
    std::vector<TcGemm> gemms;
    double beta = 1.0, gamma = 1.0;
    bool dense = false;      // GEMM over dense lower-triangular diagonal blocks (TRMM leaves):
                             // row i's beta is beta * M(i, i)
    bool inv = false;        // GEMM whose M operand is the inverted b x b diagonal blocks:
                             // a TRSM leaf on the tensor cores, X = gamma inv(M_ii) Y
    int64_t y0 = 0, y1 = 0;  // GEMM: also write the split Y planes of result rows [y0, y1)
    bool tc_leaf = false;    // leaf (while planning): to become an inverse GEMM
};

struct Plan {
    std::vector<Step> steps;
    bool tc = false;
    bool tc_leaf = false;    // TRSM leaves of the full size b as inverse GEMMs
    bool thin_leaf = false;  // TRSM leaves as thin solves on their rows (kThin, b > 0)
};

inline void plan_trsm(Plan& pl, int64_t r0, int64_t s, bool first, int b, double alpha) {
    if (s <= b && pl.thin_leaf) {
        // the leaf as the thin solve on rows [r0, r0 + s); its result goes
        // to the Y planes for the updates after it
        Step st{kThin};
        st.trsm = true;
        st.r0 = r0;
        st.b = (int)s;
        st.alpha = first ? alpha : 1.0;
        st.planes = pl.tc;
        pl.steps.push_back(st);
        return;
    }
    if (s <= b) {
        Step st{kLeaf};
        st.trsm = true;
        st.r0 = r0;
        st.b = (int)s;
        st.alpha = first ? alpha : 1.0;
        st.planes = pl.tc;
        // only full b-row leaves (they start on multiples of b, where the
        // inverted diagonal blocks are)
        st.tc_leaf = pl.tc && pl.tc_leaf && s == b && r0 % b == 0;
        pl.steps.push_back(st);
        return;
    }
    const int64_t s1 = split_point(s, b);
    plan_trsm(pl, r0, s1, first, b, alpha);
    Step g{kGemm};
    g.tc = pl.tc && (s1 % kTcKQuantum == 0);
    g.gemms.push_back(TcGemm{r0 + s1, s - s1, r0, s1});
    g.beta = first ? alpha : 1.0;
    g.gamma = -1.0;
    pl.steps.push_back(g);
    plan_trsm(pl, r0 + s1, s - s1, false, b, alpha);
}

// Paper order for TRMM (lower): C2 := M22 C2, C2 += M21 C1, C1 := M11 C1, so
// every GEMM reads C1 before it is overwritten.
inline void plan_trmm_seq(Plan& pl, int64_t r0, int64_t s, int b, double alpha) {
    if (s <= b) {
        Step st{kLeaf};
        st.trsm = false;
        st.r0 = r0;
        st.b = (int)s;
        st.alpha = alpha;
        pl.steps.push_back(st);
        return;
    }
    const int64_t s1 = split_point(s, b);
    plan_trmm_seq(pl, r0 + s1, s - s1, b, alpha);
    Step g{kGemm};
    g.tc = pl.tc && (s1 % kTcKQuantum == 0);
    g.gemms.push_back(TcGemm{r0 + s1, s - s1, r0, s1});
    g.beta = 1.0;
    g.gamma = alpha;
    pl.steps.push_back(g);
    plan_trmm_seq(pl, r0, s1, b, alpha);
}

// TRMM with the original right-hand side kept in the Y planes: no GEMM update
// reads a row another step writes, so the same recursion tree runs as one
// launch for all leaves followed by one grouped launch per recursion level
// (the updates of one level write disjoint rows).
//
// With dense = true the leaves (b a multiple of 64) run on the tensor cores
// too: the operand planes carry each b x b diagonal block's strictly-lower
// part with zeros on and above the diagonal, and one grouped launch forms
// every leaf product at once,
//   C[i] = alpha * M(i,i) * C[i] + alpha * sum_{r <= l < i} M(i,l) * Y[l],
// the diagonal term in FP32 from C's original value (a per-row beta in the
// GEMM epilogue) and the rest on the tensor cores. Each 128-row tile of a
// block is its own group member whose K range ends at the tile's last row,
// so no tile multiplies the zeros above the diagonal beyond its own 128
// columns.
inline void plan_trmm_levels(Plan& pl, int64_t k, int b, double alpha, bool dense = false) {
    if (dense) {
        Step d{kGemm};
        d.tc = true;
        d.dense = true;
        d.beta = alpha;
        d.gamma = alpha;
        for (int64_t r = 0; r < k; r += b) {
            const int64_t len = std::min<int64_t>(b, k - r);
            for (int64_t t = 0; t < len; t += 128) {
                const int64_t mlen = std::min<int64_t>(128, len - t);
                d.gemms.push_back(TcGemm{r + t, mlen, r, round_up(t + mlen, 32)});
            }
        }
        pl.steps.push_back(d);
    } else {
        Step lf{kLeaf};
        lf.trsm = false;
        lf.r0 = 0;
        lf.b = b;
        lf.nleaves = (k + b - 1) / b;
        lf.alpha = alpha;
        pl.steps.push_back(lf);
    }
    std::vector<std::pair<int64_t, int64_t>> level{{0, k}}, next;
    while (!level.empty()) {
        Step g{kGemm};
        g.tc = true;
        g.beta = 1.0;
        g.gamma = alpha;
        next.clear();
        for (auto& nd : level) {
            const int64_t r0 = nd.first, s = nd.second;
            if (s <= b) continue;
            const int64_t s1 = split_point(s, b);
            g.gemms.push_back(TcGemm{r0 + s1, s - s1, r0, s1});
            next.push_back({r0, s1});
            next.push_back({r0 + s1, s - s1});
        }
        if (!g.gemms.empty()) pl.steps.push_back(g);
        level.swap(next);
    }
}

// The whole launch sequence of one call: operand planes (tensor-core path),
// then the recursion of Section 3.1.
// dense > 0 (TRMM on the tensor-core path only): leaves of that many rows as
// dense diagonal-block GEMMs, in place of the leaf kernel and of the levels
// below that size.
// TRSM leaves on the tensor cores: each marked leaf becomes one GEMM
// X = gamma inv(M_ii) Y with beta = 0, reading the leaf rows' Y planes and
// writing X and X's planes. Those input planes come from the epilogue of
// the tensor-core update right before the leaf (the last step to write the
// rows: the recursion descends into a second half right after updating
// it), or, for the first leaf, from a conversion of its rows.
inline void apply_tc_leaves(Plan& pl) {
    std::vector<Step> out;
    out.reserve(pl.steps.size() + 1);
    for (const Step& st : pl.steps) {
        if (!(st.kind == kLeaf && st.tc_leaf)) {
            out.push_back(st);
            continue;
        }
        const bool fed = !out.empty() && out.back().kind == kGemm && out.back().tc &&
                         !out.back().inv && out.back().gemms.size() == 1 &&
                         out.back().gemms[0].rc == st.r0;
        if (fed) {
            out.back().y0 = st.r0;
            out.back().y1 = st.r0 + st.b;
        } else {
            Step cy{kConvYRows};
            cy.r0 = st.r0;
            cy.b = st.b;
            out.push_back(cy);
        }
        Step g{kGemm};
        g.tc = true;
        g.inv = true;
        g.gemms.push_back(TcGemm{st.r0, st.b, st.r0, st.b});
        g.beta = 0.0;
        g.gamma = st.alpha;
        g.y0 = st.r0;
        g.y1 = st.r0 + st.b;
        out.push_back(g);
    }
    pl.steps.swap(out);
}

inline void make_plan(Plan& plan, bool trsm, int64_t k, int b, double alpha, bool conv_m = true,
               int dense = 0) {
    if (plan.tc && conv_m) {
        Step cm{kConvM};
        cm.b = trsm ? 0 : dense;
        plan.steps.push_back(cm);
        if (trsm && plan.tc_leaf) {
            Step iv{kInvDiag};       // the inverted diagonal blocks, over M's own
            iv.b = b;
            plan.steps.push_back(iv);
        }
    }
    if (trsm) {
        plan_trsm(plan, 0, k, true, b, alpha);
        if (plan.tc && plan.tc_leaf) apply_tc_leaves(plan);
    } else {
        if (plan.tc) plan.steps.push_back(Step{kConvY});
        if (plan.tc && dense > 0) plan_trmm_levels(plan, k, dense, alpha, true);
        else if (plan.tc && b % kTcKQuantum == 0) plan_trmm_levels(plan, k, b, alpha);
        else plan_trmm_seq(plan, 0, k, b, alpha);
    }
}

// Structural check of a plan against the problem (the checked mode,
// TRX_OPT_CHECKED, and every host plan dump): every leaf block and every
// GEMM row and K range lies inside [0, k) (a tensor-core K range may run
// into the zero-filled rest of its last K step); an off-diagonal update reads a
// K range that ends at or before its rows (the recursion's disjoint blocks),
// a dense diagonal-block tile reads from its block's first row up to its own
// rows; tensor-core updates have K a multiple of the 32-element K step and
// start on an 8-element boundary; plane windows lie inside [0, k). Returns
// nullptr, or a description of the first violation.
inline const char* validate_plan(const Plan& plan, int64_t k) {
    for (const Step& st : plan.steps) {
        switch (st.kind) {
            case kLeaf:
                if (st.b < 1 || st.nleaves < 1 || st.r0 < 0 || st.r0 >= k ||
                    st.r0 + (int64_t)st.b * (st.nleaves - 1) >= k)
                    return "leaf block outside the triangle";
                break;
            case kConvYRows:
                if (st.r0 < 0 || st.b < 1 || st.r0 + st.b > k) return "plane rows outside [0, k)";
                break;
            case kThin:
                // b == 0: the whole problem; else a leaf on rows [r0, r0 + b)
                if (st.b < 0 || st.r0 < 0 || (st.b > 0 && st.r0 + st.b > k))
                    return "thin leaf outside the triangle";
                break;
            case kGemm:
                if (st.y0 < 0 || st.y1 < st.y0 || st.y1 > k) return "plane window outside [0, k)";
                for (const TcGemm& g : st.gemms) {
                    // a tensor-core K range may end past k inside its last
                    // 32-element step: the operand loads fill zeros there
                    const int64_t kend = st.tc ? round_up(k, 32) : k;
                    if (g.rc < 0 || g.mlen < 1 || g.rc + g.mlen > k || g.rk < 0 || g.klen < 1 ||
                        g.rk + g.klen > kend)
                        return "GEMM block outside the triangle";
                    if (st.dense) {
                        if (g.rk > g.rc || g.rc + g.mlen > g.rk + g.klen + 31)
                            return "dense diagonal tile reads outside its block";
                    } else if (st.inv) {
                        if (g.rk != g.rc || g.klen != g.mlen)
                            return "inverse leaf GEMM not square on its rows";
                    } else if (g.rk + g.klen > g.rc) {
                        return "update reads rows it writes";
                    }
                    if (st.tc && (g.klen % 32 != 0 || g.rk % 8 != 0))
                        return "tensor-core K range not a multiple of the K step";
                }
                break;
            default:
                break;
        }
    }
    return nullptr;
}

// Rows of the dense TRMM diagonal blocks: the handle's TRX_OPT_TRMM_DENSE
// (-1 off, else the size), or automatically 1024 once the order reaches 1024
// and the leaf size was left automatic. Tensor-core path only.
inline int trmm_dense_mode(int64_t opt, int64_t opt_leaf, bool tc, int64_t k) {
    if (!tc || opt < 0) return 0;
    if (opt > 0) return (int)opt;
    return (opt_leaf == 0 && k >= kTrmmDenseMinOrder) ? kTrmmDenseRows : 0;
}

// Recursion cutoff: TRX_OPT_LEAF when set, else 128 for FP32 TRSM and 64
// otherwise. With 256 a TRSM's leaves run as block leaves (one launch per 256
// rows); TRMM leaves stop at 128 rows.
inline int leaf_for(int64_t opt_leaf, int64_t k, bool trsm, int elem, int64_t nrhs) {
    int b = kDefaultLeaf;
    if (opt_leaf > 0) b = (int)opt_leaf;
    else if (trsm && elem == 4) b = kF32TrsmLeaf;
    if (!trsm && b > kMaxLeaf) b = kMaxLeaf;
    (void)nrhs;
    return (int)std::min<int64_t>(b, std::max<int64_t>(k, 1));
}

// TRSM leaves on the tensor cores (TRX_OPT_TRSM_TC_LEAF: -1 off, 1 on,
// 0 automatic = off): tensor-core path, leaves of 64 or 128 rows. Off by
// default: measured at m = n = 16384 the step took 18.78 ms against 18.90
// (the updates before each leaf pay for the planes they now write), and at
// 256 right-hand sides 1.38 ms against 1.21.
inline bool tc_leaf_mode(int64_t opt, bool tc, int b) {
    if (!tc || opt <= 0) return false;
    return b == 64 || b == 128;
}

// Product terms of the tensor-core split (TRX_OPT_SPLIT: 1, 3 or 6; 0 =
// automatic, 6: three BF16 slices per operand, the FP32-grade form).
constexpr int kDefaultSplitTerms = 6;
inline int split_terms(int64_t opt) {
    return (opt == 1 || opt == 3 || opt == 6) ? (int)opt : kDefaultSplitTerms;
}

// The device-scheduled TRSM (trsm_dag.cu) in place of the recursion's launch
// chain (TRX_OPT_TRSM_DAG: -1 off, 1 on where it applies, 0 automatic): FP32
// TRSM on the tensor-core path with the order a multiple of 128 (at least
// 256); automatically with at most kDagMaxNrhs right-hand sides, where the
// chain's launch and leaf latency bound the recursive path.
constexpr int64_t kDagMaxNrhs = 1024;
constexpr bool kDagAuto = false;
inline bool use_dag_mode(int64_t opt, bool tc, bool trsm, int elem, int64_t k, int64_t nrhs) {
    if (opt < 0 || !tc || !trsm || elem != 4 || k < 256 || k % kDagBlock != 0) return false;
    return opt > 0 || (kDagAuto && nrhs <= kDagMaxNrhs);
}

// The persistent CUDA-core TRSM for thin right-hand sides (thin.cu) in place
// of the recursion (TRX_OPT_THIN: -1 off, 1 on for FP32 TRSM of any order,
// 0 automatic): automatically for FP32 TRSM of order above kThinMinK with
// at most kThinMaxNrhs right-hand sides, or up to kThinWideNrhs of them
// while order x right-hand sides stays within kThinMaxWork, where the
// chain's launch and leaf latency bound the recursive path (measured on
// GB300: 1.04-4.2x faster there; at order 16384 with 256 right-hand sides
// the chain's tensor-core updates win). Where the thin leaves below also
// apply automatically, the call takes those instead (execute in api.cu).
constexpr int64_t kThinMaxNrhs = 64, kThinWideNrhs = 256;
constexpr int64_t kThinMaxWork = (int64_t)1 << 21;
constexpr int64_t kThinMinK = 256;
// TRMM (thin.cu's one-launch product): automatically with at most
// kThinTrmmMaxNrhs right-hand sides above order kThinMinK (measured on
// GB300: 1.1-2.9x the recursion's grouped product up to 32 right-hand
// sides; from 64 on the tensor-core product is as fast or faster).
constexpr int64_t kThinTrmmMaxNrhs = 32;
inline bool use_thin_mode(int64_t opt, bool trsm, int elem, int64_t k, int64_t nrhs) {
    if (opt < 0 || elem != 4 || k <= 0 || nrhs <= 0) return false;
    if (opt > 0) return true;
    if (!trsm) return k > kThinMinK && nrhs <= kThinTrmmMaxNrhs;
    return k > kThinMinK &&
           (nrhs <= kThinMaxNrhs || (nrhs <= kThinWideNrhs && k * nrhs <= kThinMaxWork));
}

// Leaves of the recursion as thin solves (TRX_OPT_THIN_LEAF: -1 off, a row
// count 256 .. 8192 (multiple of 128) on, 0 automatic): FP32 TRSM on the
// tensor-core path whose order exceeds the leaf. Automatically from order
// kThinLeafMinK: leaves of 2048 rows for 65 .. 256 right-hand sides (from
// order 8192 when there are at most 128: below it the whole-call thin solve
// is faster), of 1024 rows for 257 .. 1024 (measured on GB300 against the
// chain of 128-row leaves and the whole-call thin solve: 1.57x the chain at
// order 16384 with 256 right-hand sides, 1.56x the whole-call thin solve
// with 128, 1.13-1.3x the chain at 512 and 1024). Returns the leaf rows, or
// 0.
constexpr int64_t kThinLeafMinK = 4096;
inline int thin_leaf_rows(int64_t opt, bool tc, bool trsm, int elem, int64_t k, int64_t nrhs) {
    if (opt < 0 || !tc || !trsm || elem != 4) return 0;
    if (opt > 0) return k > opt ? (int)opt : 0;
    if (k < kThinLeafMinK || nrhs <= kThinMaxNrhs || nrhs > 1024) return 0;
    if (nrhs <= 128 && k < 2 * kThinLeafMinK) return 0;
    return nrhs <= kThinWideNrhs ? 2048 : 1024;
}

inline bool use_tc_mode(int elem, int64_t gemm_mode, int64_t k, int b) {
    if (elem != 4 || gemm_mode == 1 || k <= b) return false;   // k <= b: one leaf, no update
    if (gemm_mode == 2) return k > b;
    return k >= kTcMinOrder;
}

}  // namespace trx

// Tensor-core GEMM update for the FP32 path (tcgen05 + TMEM + TMA, sm_103a).
//
//   C[rc+i, j] = beta * C[rc+i, j] + gamma * sum_l M(rc+i, rk+l) * Y(rk+l, j)
//
// (with beta == 0, C is not read: C[rc+i, j] = gamma * sum ...; with a
// per-row beta, beta * M(rc+i, rc+i) multiplies row i's old value)
//
// This is the off-diagonal step of the recursion of Section 3.1 (TRSM:
// B2 := beta*B2 - M21 X1; TRMM: B2 += alpha M21 B1), where the paper's
// speed comes from (Section 3.3: the base kernels must stay small next to the
// GEMMs). FP32 operands are carried as S split BF16 planes (convert.cu, leaf
// kernels; S = 1, 2 or 3 slices per operand) and every product is formed
// from the slice products above FP32's rounding level with FP32
// accumulation in tensor memory:
//   S = 1: x0 y0                                (1 term, about 2^-8 relative)
//   S = 2: + x0 y1 + x1 y0                      (3 terms, about 2^-16)
//   S = 3: + x0 y2 + x1 y1 + x2 y0              (6 terms, a few units of
//                                                FP32's 2^-24: FP32-grade)
//
// One launch handles a group of updates whose output rows are disjoint (one
// recursion node for TRSM, one whole recursion level for TRMM); the tiles of
// all of them form one persistent tile sequence.
//
// Structure (one CTA per SM, 192 threads, warp-specialised), for an output
// tile of 128 rows x BN right-hand sides (BN = 256, or 128 / 64 when the
// group has too few tiles to cover the SMs):
//   warp 0     TMA producer: 2S tiles per K step (A slices 128x32, Y slices
//              BNx32, 64-byte swizzle) into a shared-memory ring of 3-4
//              stages
//   warp 1     TMEM allocator and MMA issuer: per K step 2 x terms
//              tcgen05.mma (M=128, N=BN, K=16, BF16 in, FP32 accumulate),
//              tcgen05.commit frees the ring slot
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//              lanes 32*(w%4) ..), read-modify-write of C in global memory
// Two BN-column accumulators (2*BN TMEM columns) let the epilogue of one
// tile overlap the main loop of the next.
//
// Every wait on an mbarrier is bounded by a wall-clock budget: past it the
// kernel writes TRX_ERR_TIMEOUT to the error word, stops issuing work, drains
// the copies and MMAs it has in flight (again with a bound), frees its TMEM
// and returns.
#include <cuda.h>
#include <stdint.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace trx {
namespace tc {

constexpr int BM = 128, BK = 32;                    // BK in BF16 elements (64 B)
constexpr int MAX_STAGES = 4;
constexpr int A_TILE = BM * BK * 2;                 // 8 KiB
constexpr int MAXG = 256;
constexpr int NTHREADS = 192;
// Precise accumulation (the 6-term split, S = 3): K is taken in chunks of
// CH K steps; in each chunk the dominant slice product x0 y0 accumulates in
// TMEM columns [0, BN) and the five smaller ones in [BN, 2 BN), both from
// zero, and eight epilogue warps add the two into FP32 register sums
// (round-to-nearest) before the next chunk. The tensor core's own
// accumulation thus runs over at most CH * BK = 256 terms per value, and
// the small products never round against the large running sum: measured
// against the FP32 FMA engine, accumulating whole K ranges in TMEM made
// long updates about ten times less accurate, whatever the split.
constexpr int NTHREADS_P = 320;
constexpr int CH = 8;
template <int S>
struct Precise {
    static constexpr bool value = S == 3;
};
constexpr int kTimeout = 4;                          // TRX_ERR_TIMEOUT

// Per N tile (256, 128 or 64 columns of the right-hand side) and slice
// count S: ring-stage size and depth (4 stages, 3 when four do not fit in
// shared memory), tensor memory (two accumulators of BN FP32 columns) and
// the kind::f16 instruction descriptor (FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = BN).
template <int BN, int S>
struct Cfg {
    static constexpr int B_TILE = BN * BK * 2;
    static constexpr int STAGE_BYTES = S * A_TILE + S * B_TILE;
    static constexpr int STAGES =
        (1024 + MAX_STAGES * STAGE_BYTES + 256 <= 227 * 1024) ? MAX_STAGES : 3;
    static constexpr int TMEM_COLS = 2 * BN;
    static constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 256;
    static_assert(SMEM_BYTES <= 227 * 1024, "ring does not fit in shared memory");
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                      ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(BM >> 4) << 24);
    static constexpr int MAP = BN == 256 ? 0 : BN == 128 ? 1 : 2;
};

struct Maps {
    CUtensorMap a[3];               // A slices 0..2
    CUtensorMap b[3][3];            // [slice][box of 256, 128, 64 rows]
};

struct Params {
    Maps maps;
    float* C;
    int64_t c_rs, c_cs, nrhs;
    float beta, gamma;
    int read_c;                     // 0 when beta == 0: C is written, never read
    // diag_beta: row i's beta is beta * d_i, d_i = M's diagonal entry
    // dA[i * d_step] (1 for a unit diagonal): TRMM's diagonal term taken in
    // FP32 from C's original value while the strictly-lower part of a
    // diagonal block goes through the tensor cores
    int diag_beta, unit;
    const float* dA;
    int64_t d_step;
    // optional second output: the split BF16 planes of result rows
    // [y_row0, y_row1) (canonical rows), element (i, j) at y[j * ldy + i]
    __nv_bfloat16* y_hi;
    __nv_bfloat16* y_lo;
    __nv_bfloat16* y_lo2;
    int64_t ldy, y_row0, y_row1;
    int ngemms, n_tiles_n, total_tiles;
    int* err;
    long long wait_ns;
};

// The launch's update list. Launches of at most MAXG_SMALL updates (every
// TRSM step, most TRMM levels) take the short form: a parameter block of
// about 1 KB instead of about 11 KB, which the host copies on every launch.
constexpr int MAXG_SMALL = 4;
template <int MG>
struct ParamsT : Params {
    int tile_start[MG + 1];
    TcGemm g[MG];
};

struct Smem {
    uint64_t full[MAX_STAGES], empty[MAX_STAGES], acc_full[2], acc_empty[2], drain;
    uint32_t tmem_base;
    int abort;
};

// Wait for phase `parity` of an mbarrier, bounded: false on timeout (the
// error word and the CTA's abort flag are set) or when another role of the
// CTA has already aborted.
// Drains (honour_abort == false) wait at least 1 s whatever the configured
// budget, so in-flight copies and MMAs land before the CTA exits.
__device__ bool wait_bounded(uint32_t bar, uint32_t parity, const Params& p, volatile int* abort,
                             bool honour_abort = true) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    const uint64_t limit = honour_abort ? (uint64_t)p.wait_ns
                                        : max((uint64_t)p.wait_ns, (uint64_t)1000000000ull);
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (honour_abort && *abort) return false;
        if (gtimer() - t0 > limit) {
            *abort = 1;
            atomicExch(p.err, kTimeout);
            return false;
        }
    }
}

struct Tile {
    int g, m, n;
};

// Tile t of the group: find its update (prefix sums), then raster the
// update's (m, n) tiles in bands of 8 M-tiles so that the CTAs running at one
// time share operand rows and columns in L2.
template <class PP>
__device__ __forceinline__ Tile map_tile(const PP& p, int t) {
    int lo = 0, hi = p.ngemms - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.tile_start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int local = t - p.tile_start[lo];
    const int mt = (int)((p.g[lo].mlen + BM - 1) / BM);
    // Tiles run in bands of GM tile rows, column by column inside a band, so
    // the CTAs of one wave share A row panels and Y column panels in L2
    // (measured at 16384: 16 above 8 above 4).
    constexpr int GM = 16;
    const int band = local / (GM * p.n_tiles_n);
    const int first = band * GM;
    const int gm = min(GM, mt - first);
    const int idx = local - band * GM * p.n_tiles_n;
    Tile r;
    r.g = lo;
    r.m = first + idx % gm;
    r.n = idx / gm;
    return r;
}

template <int BN, int S, int MG>
__global__ void __launch_bounds__(Precise<S>::value ? NTHREADS_P : NTHREADS, 1)
    gemm_tc_kernel(const __grid_constant__ ParamsT<MG> p) {
    using C = Cfg<BN, S>;
    constexpr bool P = Precise<S>::value;
    constexpr int STAGES = C::STAGES;
    constexpr int STAGE_BYTES = C::STAGE_BYTES;
    constexpr int B_TILE = C::B_TILE;
    constexpr int TMEM_COLS = C::TMEM_COLS;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // Stage buffers must sit on a 1024-byte boundary (swizzle atom repeat).
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t ring = (raw + 1023u) & ~1023u;
    Smem* sm = reinterpret_cast<Smem*>(smem_raw + (ring - raw) + STAGES * STAGE_BYTES);
    volatile int* abort = &sm->abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&sm->full[s]), 1);
            mbar_init(smem_u32(&sm->empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&sm->acc_full[a]), 1);
            mbar_init(smem_u32(&sm->acc_empty[a]), P ? 8 : 4);   // epilogue warps
        }
        mbar_init(smem_u32(&sm->drain), 1);
        sm->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    // Prologue done (barriers, TMEM); from here on the previous kernel's
    // results (planes, C) are read.
    pdl_trigger();
    pdl_wait();

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int stage = 0, issued = 0;
        uint32_t phase = 0;
        for (int t = blockIdx.x; t < p.total_tiles && !*abort; t += gridDim.x) {
            const Tile ti = map_tile(p, t);
            const TcGemm& G = p.g[ti.g];
            const int nkb = (int)(G.klen / BK);
            const int ya = (int)(G.rc + (int64_t)ti.m * BM);
            const int yb = ti.n * BN;
            for (int kb = 0; kb < nkb; ++kb) {
                const uint32_t fb = smem_u32(&sm->full[stage]);
                if (!wait_bounded(smem_u32(&sm->empty[stage]), phase ^ 1u, p, abort)) break;
                mbar_expect_tx(fb, STAGE_BYTES);
                const int x = (int)(G.rk + (int64_t)kb * BK);
                const uint32_t base = ring + stage * STAGE_BYTES;
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    tma_load_2d(base + q * A_TILE, &p.maps.a[q], fb, x, ya);
                    tma_load_2d(base + S * A_TILE + q * B_TILE, &p.maps.b[q][C::MAP], fb, x, yb);
                }
                ++issued;
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        }
        // Copies still in flight must land before the CTA exits.
        for (int i = 0; i < STAGES && i < issued; ++i) {
            if (--stage < 0) { stage = STAGES - 1; phase ^= 1u; }
            wait_bounded(smem_u32(&sm->full[stage]), phase, p, abort, false);
        }
    } else if (P && warp == 1 && lane == 0) {
        // ---------------- MMA issuer, precise accumulation ----------------
        int stage = 0;
        uint32_t phase = 0, acc_phase = 0;
        const uint32_t dbig = tmem, dsmall = tmem + BN;
        for (int t = blockIdx.x; t < p.total_tiles && !*abort; t += gridDim.x) {
            const Tile ti = map_tile(p, t);
            const int nkb = (int)(p.g[ti.g].klen / BK);
            bool ok = true;
            for (int kb0 = 0; kb0 < nkb && ok; kb0 += CH) {
                if (!wait_bounded(smem_u32(&sm->acc_empty[0]), acc_phase ^ 1u, p, abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int kb1 = min(nkb, kb0 + CH);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!wait_bounded(smem_u32(&sm->full[stage]), phase, p, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = ring + stage * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t acc_on = (kb == kb0 && kk == 0) ? 0u : 1u;
                        const uint64_t a0 = sdesc(base + kk * 32);
                        const uint64_t b0 = sdesc(base + S * A_TILE + kk * 32);
                        umma(dbig, a0, b0, C::IDESC, acc_on);
                        if constexpr (S >= 2) {
                            const uint64_t a1 = sdesc(base + A_TILE + kk * 32);
                            const uint64_t b1 = sdesc(base + S * A_TILE + B_TILE + kk * 32);
                            umma(dsmall, a0, b1, C::IDESC, acc_on);
                            umma(dsmall, a1, b0, C::IDESC, 1u);
                            if constexpr (S >= 3) {
                                const uint64_t a2 = sdesc(base + 2 * A_TILE + kk * 32);
                                const uint64_t b2 =
                                    sdesc(base + S * A_TILE + 2 * B_TILE + kk * 32);
                                umma(dsmall, a0, b2, C::IDESC, 1u);
                                umma(dsmall, a1, b1, C::IDESC, 1u);
                                umma(dsmall, a2, b0, C::IDESC, 1u);
                            }
                        }
                    }
                    umma_commit(smem_u32(&sm->empty[stage]));
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                umma_commit(smem_u32(&sm->acc_full[0]));
                acc_phase ^= 1u;
            }
            if (!ok) break;
        }
        umma_commit(smem_u32(&sm->drain));
        wait_bounded(smem_u32(&sm->drain), 0, p, abort, false);
    } else if (P && warp >= 2) {
        // ---------------- epilogue, precise accumulation ----------------
        // warp w: TMEM lanes 32 (w % 4) .., columns [half * HC, half * HC + HC)
        constexpr int HC = BN / 2;
        const int q = warp & 3, half = (warp - 2) >> 2;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
            const Tile ti = map_tile(p, t);
            const TcGemm& G = p.g[ti.g];
            const int nkb = (int)(G.klen / BK);
            const int64_t row = (int64_t)ti.m * BM + q * 32 + lane;
            const bool row_ok = row < G.mlen;
            const int64_t grow = G.rc + row;
            const bool yrow = p.y_hi != nullptr && row_ok && grow >= p.y_row0 && grow < p.y_row1;
            float beta = p.beta;
            if (p.diag_beta && row_ok && !p.unit) beta *= __ldg(p.dA + grow * p.d_step);
            float* wrow = p.C + grow * p.c_rs;
            const int64_t jbase = (int64_t)ti.n * BN + half * HC;
            float sum[HC];
#pragma unroll
            for (int c = 0; c < HC; ++c) sum[c] = 0.f;
            bool ok = true;
            for (int kb0 = 0; kb0 < nkb; kb0 += CH) {
                int w = 1;
                if (lane == 0) w = wait_bounded(smem_u32(&sm->acc_full[0]), acc_phase, p, abort);
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int cc = 0; cc < HC / 16; ++cc) {
                    float v[16];
                    const uint32_t ta = tmem + (uint32_t)(half * HC + cc * 16) +
                                        ((uint32_t)(q * 32) << 16);
                    tmem_ld16(ta, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) sum[cc * 16 + i] += v[i];
                    if constexpr (S >= 2) {
                        tmem_ld16(ta + BN, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) sum[cc * 16 + i] += v[i];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sm->acc_empty[0]));
                acc_phase ^= 1u;
            }
            if (!ok) break;
            // C := beta C + gamma sum over this thread's row and columns
#pragma unroll
            for (int cc = 0; cc < HC / 16; ++cc) {
                const int64_t j0 = jbase + cc * 16;
                float* dst = wrow + j0 * p.c_cs;
                float cv[16];
                if (!p.read_c || !row_ok) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) cv[c] = 0.f;
                } else if (j0 + 16 <= p.nrhs) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) cv[c] = __ldcg(dst + c * p.c_cs);
                } else {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        cv[c] = (j0 + c < p.nrhs) ? __ldcg(dst + c * p.c_cs) : 0.f;
                }
                if (!row_ok) continue;
                const int64_t yo = j0 * p.ldy + grow;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (j0 + c < p.nrhs) {
                        const float o = fmaf(beta, cv[c], p.gamma * sum[cc * 16 + c]);
                        dst[c * p.c_cs] = o;
                        if (yrow) put_split(p.y_hi, p.y_lo, p.y_lo2, S, yo + c * p.ldy, o);
                    }
                }
            }
        }
    } else if (!P && warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        int stage = 0, acc = 0;
        uint32_t phase = 0, acc_phase = 0;
        for (int t = blockIdx.x; t < p.total_tiles && !*abort; t += gridDim.x) {
            const Tile ti = map_tile(p, t);
            const int nkb = (int)(p.g[ti.g].klen / BK);
            if (!wait_bounded(smem_u32(&sm->acc_empty[acc]), acc_phase ^ 1u, p, abort)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(acc * BN);
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                if (!wait_bounded(smem_u32(&sm->full[stage]), phase, p, abort)) { ok = false; break; }
                tc_fence_after();
                const uint32_t base = ring + stage * STAGE_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    // slice products of weight 1, 2^-8 and 2^-16 (S = 1, 2, 3)
                    const uint64_t a0 = sdesc(base + kk * 32);
                    const uint64_t b0 = sdesc(base + S * A_TILE + kk * 32);
                    umma(d, a0, b0, C::IDESC, (kb | kk) != 0 ? 1u : 0u);
                    if constexpr (S >= 2) {
                        const uint64_t a1 = sdesc(base + A_TILE + kk * 32);
                        const uint64_t b1 = sdesc(base + S * A_TILE + B_TILE + kk * 32);
                        umma(d, a0, b1, C::IDESC, 1u);
                        umma(d, a1, b0, C::IDESC, 1u);
                        if constexpr (S >= 3) {
                            const uint64_t a2 = sdesc(base + 2 * A_TILE + kk * 32);
                            const uint64_t b2 = sdesc(base + S * A_TILE + 2 * B_TILE + kk * 32);
                            umma(d, a0, b2, C::IDESC, 1u);
                            umma(d, a1, b1, C::IDESC, 1u);
                            umma(d, a2, b0, C::IDESC, 1u);
                        }
                    }
                }
                umma_commit(smem_u32(&sm->empty[stage]));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            umma_commit(smem_u32(&sm->acc_full[acc]));
            if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
        }
        // All MMAs issued by this CTA complete before TMEM is released.
        umma_commit(smem_u32(&sm->drain));
        wait_bounded(smem_u32(&sm->drain), 0, p, abort, false);
    } else if (!P && warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;                 // TMEM lanes 32q .. 32q+31
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
            const Tile ti = map_tile(p, t);
            const TcGemm& G = p.g[ti.g];
            const int64_t row = (int64_t)ti.m * BM + q * 32 + lane;
            const bool row_ok = row < G.mlen;
            const int64_t grow = G.rc + row;
            const bool yrow = p.y_hi != nullptr && row_ok && grow >= p.y_row0 && grow < p.y_row1;
            float beta = p.beta;
            if (p.diag_beta && row_ok && !p.unit) beta *= __ldg(p.dA + (G.rc + row) * p.d_step);
            const float* crow = p.C + (G.rc + row) * p.c_rs;
            float* wrow = p.C + (G.rc + row) * p.c_rs;
            const int64_t jbase = (int64_t)ti.n * BN;
            // C is read ahead of use, two 32-column chunks deep, the first
            // two before the accumulator is even ready: the loads of a chunk
            // are all in flight together instead of one load-store pair at a
            // time (a store to C could alias any later load as far as the
            // compiler knows).
            auto load_chunk = [&](int ch, float (&dst)[32]) {
                const int64_t j0 = jbase + ch * 32;
                const float* src = crow + j0 * p.c_cs;
                if (!p.read_c) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) dst[c] = 0.f;
                } else if (row_ok && j0 + 32 <= p.nrhs) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) dst[c] = __ldcg(src + c * p.c_cs);
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        dst[c] = (row_ok && j0 + c < p.nrhs) ? __ldcg(src + c * p.c_cs) : 0.f;
                }
            };
            float c0[32], c1[32];
            load_chunk(0, c0);
            load_chunk(1, c1);
            // One lane waits and the warp follows its verdict, so the
            // warp-collective TMEM loads below never run on a partial warp.
            int ok = 1;
            if (lane == 0) ok = wait_bounded(smem_u32(&sm->acc_full[acc]), acc_phase, p, abort);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
#pragma unroll 1
            for (int ch = 0; ch < BN / 32; ++ch) {
                float c2[32];
                if (ch + 2 < BN / 32) load_chunk(ch + 2, c2);
                float v[32];
                tmem_ld32(tmem + (uint32_t)(acc * BN + ch * 32) + ((uint32_t)(q * 32) << 16), v);
                if (ch == BN / 32 - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&sm->acc_empty[acc]));
                }
                const int64_t j0 = jbase + ch * 32;
                float* dst = wrow + j0 * p.c_cs;
                if (yrow) {
                    // the result and its planes (same split as the conversions)
                    const int64_t yo = j0 * p.ldy + grow;
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        if (j0 + c < p.nrhs) {
                            const float o = fmaf(beta, c0[c], p.gamma * v[c]);
                            dst[c * p.c_cs] = o;
                            put_split(p.y_hi, p.y_lo, p.y_lo2, S, yo + c * p.ldy, o);
                        }
                    }
                } else if (row_ok && j0 + 32 <= p.nrhs) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) dst[c * p.c_cs] = fmaf(beta, c0[c], p.gamma * v[c]);
                } else if (row_ok) {
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        if (j0 + c < p.nrhs) dst[c * p.c_cs] = fmaf(beta, c0[c], p.gamma * v[c]);
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    c0[c] = c1[c];
                    c1[c] = c2[c];
                }
            }
            if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---- host ------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

static bool encode(CUtensorMap* m, void* base, uint64_t inner, uint64_t outer, uint64_t ld,
                   uint32_t box_outer) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

int tc_maps_size() { return (int)sizeof(tc::Maps); }

// A BF16 plane as a 2-D tensor map (inner index contiguous, leading dimension
// ld elements), boxes of 32 inner x box_outer, 64-byte swizzle: the operand
// layout of every tensor-core kernel here.
bool tc_encode_bf16_2d(void* map, void* base, uint64_t inner, uint64_t outer, uint64_t ld,
                       uint32_t box_outer) {
    return tc::encode(reinterpret_cast<CUtensorMap*>(map), base, inner, outer, ld, box_outer);
}

template <int S, int MG>
static cudaError_t tc_configure_sg() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(tc::gemm_tc_kernel<256, S, MG>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::Cfg<256, S>::SMEM_BYTES)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(tc::gemm_tc_kernel<128, S, MG>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tc::Cfg<128, S>::SMEM_BYTES)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(tc::gemm_tc_kernel<64, S, MG>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tc::Cfg<64, S>::SMEM_BYTES);
}

template <int S>
static cudaError_t tc_configure_s() {
    cudaError_t e = tc_configure_sg<S, tc::MAXG>();
    return e != cudaSuccess ? e : tc_configure_sg<S, tc::MAXG_SMALL>();
}

cudaError_t tc_configure() {
    cudaError_t e;
    if ((e = tc_configure_s<1>()) != cudaSuccess) return e;
    if ((e = tc_configure_s<2>()) != cudaSuccess) return e;
    return tc_configure_s<3>();
}

cudaError_t tc_make_maps(const Planes& pl, int64_t k, int64_t nrhs, void* out) {
    tc::Maps* m = reinterpret_cast<tc::Maps*>(out);
    if (k <= 0 || nrhs <= 0 || pl.slices < 1 || pl.slices > 3) return cudaErrorInvalidValue;
    __nv_bfloat16* const ma[3] = {pl.m_hi, pl.m_lo, pl.m_lo2};
    __nv_bfloat16* const yb[3] = {pl.y_hi, pl.y_lo, pl.y_lo2};
    const uint32_t boxes[3] = {256, 128, 64};
    for (int q = 0; q < pl.slices; ++q) {
        if (!ma[q] || !yb[q] || !tc::encode(&m->a[q], ma[q], k, k, pl.ldm, tc::BM))
            return cudaErrorInvalidValue;
        for (int b = 0; b < 3; ++b)
            if (!tc::encode(&m->b[q][b], yb[q], k, nrhs, pl.ldy, boxes[b]))
                return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t launch_gemm_tc(const Canon<float>& p, const void* maps, int slices,
                           const TcGemm* gemms, int ngemms, float beta, float gamma,
                           int* err_word, long long wait_ns, int num_sms, cudaStream_t s,
                           bool diag_beta, const TcYOut* yout) {
    if (slices < 1 || slices > 3) return cudaErrorInvalidValue;
    using namespace tc;
    for (int g0 = 0; g0 < ngemms; g0 += MAXG) {
        const int ng = (ngemms - g0) < MAXG ? (ngemms - g0) : MAXG;
        // N tile: the widest whose tile count still covers every SM (wide
        // tiles feed the tensor pipe best; small updates are epilogue-bound
        // and want all SMs on them).
        int64_t mtiles = 0;
        for (int i = 0; i < ng; ++i) mtiles += (gemms[g0 + i].mlen + BM - 1) / BM;
        int bn = 64;
        if (mtiles * ((p.nrhs + 255) / 256) >= num_sms) bn = 256;
        else if (mtiles * ((p.nrhs + 127) / 128) >= num_sms) bn = 128;
        static thread_local ParamsT<MAXG> prm;
        prm.maps = *reinterpret_cast<const Maps*>(maps);
        prm.C = p.C;
        prm.c_rs = p.c_rs;
        prm.c_cs = p.c_cs;
        prm.nrhs = p.nrhs;
        prm.beta = beta;
        prm.gamma = gamma;
        prm.read_c = beta != 0.f;
        prm.diag_beta = diag_beta;
        prm.unit = p.unit;
        prm.dA = p.A;
        prm.d_step = p.a_rs + p.a_cs;
        prm.y_hi = yout ? yout->hi : nullptr;
        prm.y_lo = yout ? yout->lo : nullptr;
        prm.y_lo2 = yout ? yout->lo2 : nullptr;
        prm.ldy = yout ? yout->ld : 0;
        prm.y_row0 = yout ? yout->row0 : 0;
        prm.y_row1 = yout ? yout->row1 : 0;
        prm.ngemms = ng;
        prm.n_tiles_n = (int)((p.nrhs + bn - 1) / bn);
        prm.err = err_word;
        prm.wait_ns = wait_ns;
        int64_t tiles = 0;
        for (int i = 0; i < ng; ++i) {
            const TcGemm& G = gemms[g0 + i];
            if (G.klen <= 0 || G.klen % BK != 0 || G.rk % 8 != 0) return cudaErrorInvalidValue;
            prm.g[i] = G;
            prm.tile_start[i] = (int)tiles;
            tiles += ((G.mlen + BM - 1) / BM) * (int64_t)prm.n_tiles_n;
        }
        prm.tile_start[ng] = (int)tiles;
        if (tiles <= 0) continue;
        if (tiles > (int64_t)1 << 30) return cudaErrorInvalidValue;
        prm.total_tiles = (int)tiles;
        const int grid = (int)(tiles < num_sms ? tiles : num_sms);
        cudaError_t e;
        static thread_local ParamsT<MAXG_SMALL> prm_small;
        const bool small = ng <= MAXG_SMALL;
        if (small) {
            static_cast<Params&>(prm_small) = static_cast<const Params&>(prm);
            for (int i = 0; i <= ng; ++i) prm_small.tile_start[i] = prm.tile_start[i];
            for (int i = 0; i < ng; ++i) prm_small.g[i] = prm.g[i];
        }
#define TRX_TC_LAUNCH(BNV, SV)                                                             \
    (small ? launch_kernel(gemm_tc_kernel<BNV, SV, MAXG_SMALL>, dim3(grid),                 \
                           dim3(Precise<SV>::value ? NTHREADS_P : NTHREADS),               \
                           Cfg<BNV, SV>::SMEM_BYTES, s, prm_small)                         \
           : launch_kernel(gemm_tc_kernel<BNV, SV, MAXG>, dim3(grid),                       \
                           dim3(Precise<SV>::value ? NTHREADS_P : NTHREADS),               \
                           Cfg<BNV, SV>::SMEM_BYTES, s, prm))
        if (slices == 1)
            e = bn == 256 ? TRX_TC_LAUNCH(256, 1) : bn == 128 ? TRX_TC_LAUNCH(128, 1)
                                                              : TRX_TC_LAUNCH(64, 1);
        else if (slices == 2)
            e = bn == 256 ? TRX_TC_LAUNCH(256, 2) : bn == 128 ? TRX_TC_LAUNCH(128, 2)
                                                              : TRX_TC_LAUNCH(64, 2);
        else
            e = bn == 256 ? TRX_TC_LAUNCH(256, 3) : bn == 128 ? TRX_TC_LAUNCH(128, 3)
                                                              : TRX_TC_LAUNCH(64, 3);
#undef TRX_TC_LAUNCH
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace trx

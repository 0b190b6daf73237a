// Device-scheduled TRSM for few right-hand sides (tcgen05 + TMEM + TMA,
// sm_103a): the whole solve in one persistent launch.
//
// The recursion of Section 3.1 turns a TRSM into a dependent chain of leaf
// solves and GEMM updates. With few right-hand sides every link of that
// chain is a short launch, and the solve is bound by launch and leaf
// latency, not by arithmetic (the recursive path reaches about 21 TFLOP/s at
// order 16384 with 256 right-hand sides). Here the same blocks run as a
// dependency graph on the device instead:
//
//   the canonical lower M is cut into 128-row blocks, the right-hand side
//   into 64-column panels; task (i, p) computes
//       S = sum_{j < i} M_ij X_jp                (tensor cores, block by block)
//       R = alpha B_ip - S
//       X_ip = inv(M_ii) R                        (tensor cores)
//   and publishes X_ip (FP32 into C and its split BF16 planes) with a flag.
//
// Tasks are taken in order from an atomic counter, so a task only waits for
// tasks taken before it, which are running or done: the solve progresses
// whatever the number of resident CTAs. A task starts multiplying block j as
// soon as X_jp is published, so the off-diagonal products of later blocks
// overlap the chain; the chain itself is one 128 x 64 x 128 product, one
// residual and one 128 x 64 x 128 product per block. The leaf solve of
// Section 3.3 becomes a product with the diagonal block's inverse (computed
// once per call by substitution in FP32, convert.cu), rounding as the
// inverse-GEMM leaves do.
//
// Every product is formed from the BF16 slice planes like the GEMM update
// (gemm_tc.cu): slice products above FP32's rounding level, the dominant
// one and the small ones in separate TMEM accumulators, added in FP32 in
// registers every 256 K elements.
//
// CTA: 192 threads. Warp 0 is the TMA producer (it also waits on the flags),
// warp 1 allocates TMEM and issues the MMAs, warps 2-5 are the epilogue
// (thread = row of the block, 64 columns of the panel). Two CTAs per SM.
// Every wait (mbarrier or flag) is bounded: past the budget the CTA writes
// TRX_ERR_TIMEOUT to the error word, stops, drains what it has in flight and
// frees its tensor memory; tasks waiting on it then time out too.
#include <cuda.h>
#include <stdint.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace trx {
namespace dag {
using namespace tc;

constexpr int R = kDagBlock;         // block rows = MMA M
constexpr int W = kDagPanel;         // panel columns = MMA N
constexpr int BK = 32;               // K per stage (64-byte rows of BF16)
constexpr int KB_BLOCK = R / BK;     // stages per block of K
constexpr int CH = 8;                // stages per accumulation chunk
constexpr int STAGES = 3;
constexpr int NTHREADS = 192;
constexpr int A_TILE = R * BK * 2;   // 8 KiB
constexpr int B_TILE = W * BK * 2;   // 4 KiB
constexpr int TMEM_COLS = 256;       // [0,64) S big, [64,128) S small, [128,192) X big, [192,256) X small
constexpr int kTimeout = 4;          // TRX_ERR_TIMEOUT

template <int S>
struct Cfg {
    static constexpr int STAGE_BYTES = S * (A_TILE + B_TILE);
    static constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + 256;
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                      ((uint32_t)(W >> 3) << 17) | ((uint32_t)(R >> 4) << 24);
};

struct Maps {
    CUtensorMap m[3];    // M planes (k x k, row-major), boxes 32 x 128
    CUtensorMap y[3];    // Y planes (element (l, j) at j ldy + l), boxes 32 x 64
    CUtensorMap w[3];    // compact inverses (k x 128, row-major), boxes 32 x 128
};

struct Params {
    Maps maps;
    float* C;
    int64_t c_rs, c_cs, k, nrhs;
    int np, ntasks;
    float alpha;
    __nv_bfloat16* y[3];
    int64_t ldy;
    int* flags;          // nb * np, then the task counter
    int* err;
    long long wait_ns;
};

struct Smem {
    uint64_t full[STAGES], empty[STAGES];
    uint64_t s_full, s_empty, x_full, x_empty, r_ready, drain;
    uint32_t tmem_base;
    int task;
    int abort;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded mbarrier wait (as the GEMM update's): false on timeout or once the
// CTA has aborted; drains (honour_abort false) wait at least 1 s.
__device__ bool wait_bar(uint32_t bar, uint32_t parity, const Params& p, volatile int* abort,
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

// Bounded wait for block (j, panel) to be published.
__device__ bool wait_flag(const int* f, const Params& p, volatile int* abort) {
    if (ld_acquire(f)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (ld_acquire(f)) return true;
        if (*abort) return false;
        if (gtimer() - t0 > (uint64_t)p.wait_ns) {
            *abort = 1;
            atomicExch(p.err, kTimeout);
            return false;
        }
        __nanosleep(64);
    }
}

template <int S>
__global__ void __launch_bounds__(NTHREADS, 2) trsm_dag_kernel(const __grid_constant__ Params p) {
    using Cf = Cfg<S>;
    constexpr int STAGE_BYTES = Cf::STAGE_BYTES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
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
        mbar_init(smem_u32(&sm->s_full), 1);
        mbar_init(smem_u32(&sm->s_empty), 4);
        mbar_init(smem_u32(&sm->x_full), 1);
        mbar_init(smem_u32(&sm->x_empty), 4);
        mbar_init(smem_u32(&sm->r_ready), 4);
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
    pdl_trigger();
    pdl_wait();

    int* counter = p.flags + (int64_t)(p.k / R) * p.np;
    // per-role ring and barrier phases, carried across tasks
    int stage = 0, issued = 0;
    uint32_t phase = 0, s_phase = 0, x_phase = 0, r_phase = 0;
    float acc[W];   // epilogue: this thread's row of the running sum, then of X

    while (true) {
        if (threadIdx.x == 0) sm->task = *abort ? p.ntasks : atomicAdd(counter, 1);
        __syncthreads();
        const int t = sm->task;
        if (t >= p.ntasks) break;
        const int i = t / p.np, pn = t - i * p.np;
        const int nkb = i * KB_BLOCK;          // stages of the off-diagonal sum
        if (warp == 0 && lane == 0) {
            // ---------------- TMA producer ----------------
            bool ok = true;
            for (int kb = 0; kb < nkb + KB_BLOCK && ok; ++kb) {
                const bool diag = kb >= nkb;
                if (!diag && kb % KB_BLOCK == 0) {
                    // X of block j published: its planes may be loaded
                    ok = wait_flag(p.flags + (int64_t)(kb / KB_BLOCK) * p.np + pn, p, abort);
                    if (!ok) break;
                    fence_proxy_async_global();
                }
                if (kb == nkb) {
                    // the residual's planes written by this CTA's epilogue
                    ok = wait_bar(smem_u32(&sm->r_ready), r_phase, p, abort);
                    r_phase ^= 1u;
                    if (!ok) break;
                    fence_proxy_async_global();
                }
                const uint32_t fb = smem_u32(&sm->full[stage]);
                if (!wait_bar(smem_u32(&sm->empty[stage]), phase ^ 1u, p, abort)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(fb, STAGE_BYTES);
                const uint32_t base = ring + stage * STAGE_BYTES;
                const int xk = diag ? (kb - nkb) * BK : kb * BK;
                const int yrow = diag ? i * R + (kb - nkb) * BK : kb * BK;
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    tma_load_2d(base + q * A_TILE, diag ? &p.maps.w[q] : &p.maps.m[q], fb, xk,
                                i * R);
                    tma_load_2d(base + S * A_TILE + q * B_TILE, &p.maps.y[q], fb, yrow, pn * W);
                }
                ++issued;
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        } else if (warp == 1 && lane == 0) {
            // ---------------- MMA issuer ----------------
            // one accumulation chunk: stages [kb0, kb1) into the sum's
            // accumulator pair (diag false) or the diagonal block's (true)
            auto chunk = [&](int kb0, int kb1, bool diag) {
                uint64_t* empty_bar = diag ? &sm->x_empty : &sm->s_empty;
                uint32_t& ph = diag ? x_phase : s_phase;
                if (!wait_bar(smem_u32(empty_bar), ph ^ 1u, p, abort)) return false;
                tc_fence_after();
                const uint32_t dbig = tmem + (diag ? 2 * W : 0), dsmall = dbig + W;
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!wait_bar(smem_u32(&sm->full[stage]), phase, p, abort)) return false;
                    tc_fence_after();
                    const uint32_t base = ring + stage * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t on = (kb == kb0 && kk == 0) ? 0u : 1u;
                        const uint64_t a0 = sdesc(base + kk * 32);
                        const uint64_t b0 = sdesc(base + S * A_TILE + kk * 32);
                        umma(dbig, a0, b0, Cf::IDESC, on);
                        if constexpr (S >= 2) {
                            const uint64_t a1 = sdesc(base + A_TILE + kk * 32);
                            const uint64_t b1 = sdesc(base + S * A_TILE + B_TILE + kk * 32);
                            umma(dsmall, a0, b1, Cf::IDESC, on);
                            umma(dsmall, a1, b0, Cf::IDESC, 1u);
                            if constexpr (S >= 3) {
                                const uint64_t a2 = sdesc(base + 2 * A_TILE + kk * 32);
                                const uint64_t b2 = sdesc(base + S * A_TILE + 2 * B_TILE + kk * 32);
                                umma(dsmall, a0, b2, Cf::IDESC, 1u);
                                umma(dsmall, a1, b1, Cf::IDESC, 1u);
                                umma(dsmall, a2, b0, Cf::IDESC, 1u);
                            }
                        }
                    }
                    umma_commit(smem_u32(&sm->empty[stage]));
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                umma_commit(smem_u32(diag ? &sm->x_full : &sm->s_full));
                ph ^= 1u;
                return true;
            };
            bool ok = true;
            for (int kb0 = 0; kb0 < nkb && ok; kb0 += CH) ok = chunk(kb0, min(nkb, kb0 + CH), false);
            if (ok) chunk(nkb, nkb + KB_BLOCK, true);
        } else if (warp >= 2) {
            // ---------------- epilogue: thread = row of the block ----------------
            const int q = warp & 3;
            const int64_t row = (int64_t)i * R + q * 32 + lane;     // k % R == 0: always < k
            const uint32_t lane_off = (uint32_t)(q * 32) << 16;
            bool ok = true;
#pragma unroll
            for (int c = 0; c < W; ++c) acc[c] = 0.f;
            auto take = [&](uint64_t* full_bar, uint64_t* empty_bar, uint32_t& ph, uint32_t col0) {
                int w = 1;
                if (lane == 0) w = wait_bar(smem_u32(full_bar), ph, p, abort);
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) return false;
                tc_fence_after();
#pragma unroll
                for (int cc = 0; cc < W / 16; ++cc) {
                    float v[16];
                    tmem_ld16(tmem + col0 + cc * 16 + lane_off, v);
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[cc * 16 + e] += v[e];
                    if constexpr (S >= 2) {
                        tmem_ld16(tmem + col0 + W + cc * 16 + lane_off, v);
#pragma unroll
                        for (int e = 0; e < 16; ++e) acc[cc * 16 + e] += v[e];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(empty_bar));
                ph ^= 1u;
                return true;
            };
            for (int kb0 = 0; kb0 < nkb && ok; kb0 += CH) ok = take(&sm->s_full, &sm->s_empty, s_phase, 0);
            if (ok) {
                // R = alpha B - S (C's block is untouched until this task
                // writes X), as split planes into the block's Y rows
                const int64_t j0 = (int64_t)pn * W;
                const float* crow = p.C + row * p.c_rs;
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    const int64_t j = j0 + c;
                    if (j < p.nrhs) {
                        const float r = fmaf(p.alpha, __ldcg(crow + j * p.c_cs), -acc[c]);
                        put_split(p.y[0], p.y[1], p.y[2], S, j * p.ldy + row, r);
                    }
                }
                fence_proxy_async_global();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sm->r_ready));
#pragma unroll
                for (int c = 0; c < W; ++c) acc[c] = 0.f;
                ok = take(&sm->x_full, &sm->x_empty, x_phase, 2 * W);
            }
            if (ok) {
                // X into C and its planes, then publish the block
                const int64_t j0 = (int64_t)pn * W;
                float* crow = p.C + row * p.c_rs;
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    const int64_t j = j0 + c;
                    if (j < p.nrhs) {
                        crow[j * p.c_cs] = acc[c];
                        put_split(p.y[0], p.y[1], p.y[2], S, j * p.ldy + row, acc[c]);
                    }
                }
                __threadfence();
                fence_proxy_async_global();
            }
            // the four epilogue warps: every row written before the flag
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (ok && !*abort && warp == 2 && lane == 0)
                st_release(p.flags + (int64_t)i * p.np + pn, 1);
        }
        __syncthreads();
    }
    // Copies and MMAs still in flight land before TMEM is released.
    if (warp == 0 && lane == 0) {
        // stages issued but perhaps not consumed: wait for their arrival
        int st = stage;
        uint32_t ph = phase;
        for (int n = 0; n < STAGES && n < issued; ++n) {
            if (--st < 0) { st = STAGES - 1; ph ^= 1u; }
            wait_bar(smem_u32(&sm->full[st]), ph, p, abort, false);
        }
    } else if (warp == 1 && lane == 0) {
        umma_commit(smem_u32(&sm->drain));
        wait_bar(smem_u32(&sm->drain), 0, p, abort, false);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
}

}  // namespace dag

size_t dag_flag_bytes(int64_t k, int64_t nrhs) {
    const int64_t nb = k / kDagBlock, np = (nrhs + kDagPanel - 1) / kDagPanel;
    return (size_t)(nb * np + 1) * sizeof(int);
}

cudaError_t dag_configure() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(dag::trsm_dag_kernel<1>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  dag::Cfg<1>::SMEM)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(dag::trsm_dag_kernel<2>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  dag::Cfg<2>::SMEM)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(dag::trsm_dag_kernel<3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, dag::Cfg<3>::SMEM);
}

cudaError_t launch_trsm_dag(const Canon<float>& c, const Planes& pl, __nv_bfloat16* const w[3],
                            float alpha, int* flags, int* err, long long wait_ns, int num_sms,
                            cudaStream_t s) {
    using namespace dag;
    if (c.k <= 0 || c.nrhs <= 0) return cudaSuccess;
    if (c.k % R != 0 || pl.slices < 1 || pl.slices > 3) return cudaErrorInvalidValue;
    static thread_local Params prm;
    __nv_bfloat16* const ms[3] = {pl.m_hi, pl.m_lo, pl.m_lo2};
    __nv_bfloat16* const ys[3] = {pl.y_hi, pl.y_lo, pl.y_lo2};
    for (int q = 0; q < pl.slices; ++q) {
        if (!tc_encode_bf16_2d(&prm.maps.m[q], ms[q], c.k, c.k, pl.ldm, R) ||
            !tc_encode_bf16_2d(&prm.maps.y[q], ys[q], c.k, c.nrhs, pl.ldy, W) ||
            !tc_encode_bf16_2d(&prm.maps.w[q], w[q], R, c.k, R, R))
            return cudaErrorInvalidValue;
        prm.y[q] = ys[q];
    }
    for (int q = pl.slices; q < 3; ++q) prm.y[q] = nullptr;
    prm.C = c.C;
    prm.c_rs = c.c_rs;
    prm.c_cs = c.c_cs;
    prm.k = c.k;
    prm.nrhs = c.nrhs;
    prm.np = (int)((c.nrhs + W - 1) / W);
    const int64_t ntasks = (c.k / R) * (int64_t)prm.np;
    if (ntasks > 0x7fffffff) return cudaErrorInvalidValue;
    prm.ntasks = (int)ntasks;
    prm.alpha = alpha;
    prm.ldy = pl.ldy;
    prm.flags = flags;
    prm.err = err;
    prm.wait_ns = wait_ns;
    cudaError_t e = cudaMemsetAsync(flags, 0, dag_flag_bytes(c.k, c.nrhs), s);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(ntasks, 2 * (int64_t)num_sms);
    if (pl.slices == 1)
        return launch_kernel(trsm_dag_kernel<1>, dim3(grid), dim3(NTHREADS), Cfg<1>::SMEM, s, prm);
    if (pl.slices == 2)
        return launch_kernel(trsm_dag_kernel<2>, dim3(grid), dim3(NTHREADS), Cfg<2>::SMEM, s, prm);
    return launch_kernel(trsm_dag_kernel<3>, dim3(grid), dim3(NTHREADS), Cfg<3>::SMEM, s, prm);
}

}  // namespace trx

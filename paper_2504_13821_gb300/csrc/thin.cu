// FP32 TRSM with few right-hand sides as one persistent launch on the CUDA
// cores.
//
// With a thin right-hand side the recursion of Section 3.1 is a long chain
// of small launches (a leaf and a GEMM update per 128 rows), each bound by
// latency: at order 8192 with 16 right-hand sides the chain takes about
// 1.4 ms to read a 128 MB triangle. Here the canonical lower M is cut into
// 64-row blocks and the right-hand side into 16-column panels, and task
// (i, p) runs the blocked forward substitution of block row i, left-looking:
//
//     S'   = sum_{j < i-1} M_ij X_jp        (64 x 64 x 16 products, FP32 FMA)
//     P    = inv(M_ii) (alpha B_ip - S')
//     X_ip = P - Z X_i-1,p,   Z = inv(M_ii) M_i,i-1
//
// then writes X_ip into C and publishes it. inv(M_ii) (substitution against
// the identity, FP32, one reciprocal of each diagonal entry: the leaf solve
// of Section 3.3 as a product with the inverted block) and Z are made by
// the task before its first wait when the right-hand side is one panel,
// and by a preparatory pass (thin_prep_kernel, one CTA per block row, the
// same code) when it is several, so the panels' tasks of a block row do not
// each repeat them; the products of a task start as soon as the blocks X_jp
// they need are published, so the reads of M (every element once per
// panel, the dominant traffic) overlap the chain of diagonal blocks; the
// chain itself is one 64 x 64 x 16 product per block.
//
// The same launch also serves as the recursion's leaf for 65 .. 1024
// right-hand sides (the thin leaves): on a leaf's rows, its columns of M
// and its rows of C, with the tensor-core updates between leaves.
//
// A block is published as 1024 tagged 64-bit words (FP32 bits in the low
// half, 1 in the high half; a 64-bit access is single-copy atomic, so value
// and tag arrive together): a consumer polls the words themselves, one L2
// round trip, with no flag and no fence between data and signal. The words
// are zeroed by a memset before each launch.
//
// Tasks are taken in order from an atomic counter (block row major), so a
// task only waits for tasks taken before it, which are running or done: the
// solve progresses whatever the number of resident CTAs. Every wait is
// bounded: past the budget the CTA writes TRX_ERR_TIMEOUT to the error word
// and the launch's stop word, and every waiting CTA then stops.
//
// Arithmetic: FP32 FMA throughout (no operand split), partial sums in a
// fixed order, so results are bitwise repeatable.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace trx {
namespace thin {

constexpr int BR = kThinBlock;       // rows of a block
constexpr int NP = kThinPanel;       // columns of a panel
constexpr int NT = 256;
constexpr int LD = BR + 4;           // shared row stride (floats): 16-byte aligned rows
constexpr int LDT = BR + 1;          // inverse work tile: conflict-free column reads
constexpr int kTimeout = 4;          // TRX_ERR_TIMEOUT

struct Params {
    int64_t k, nrhs;
    const float* A;
    int64_t a_rs, a_cs;
    float* C;
    int64_t c_rs, c_cs;
    float alpha;
    int unit;
    int nbr, npan;
    int64_t ntask;
    int* ticket;     // next task
    int* stop;       // set by a CTA whose wait ran out: the others stop waiting
    // published blocks: X_ip as 64 x 16 tagged words (FP32 bits, tag 1 in
    // the high half), tile (p, i) at words [(p nbr + i) 1024, + 1024),
    // row-major; zeroed by the launch's memset, so a tag of 1 means "this
    // element of this launch"
    unsigned long long* xt;
    int* err;
    long long wait_ns;
    int withhold;    // test hook: block row 0 is never published (waits run out)
    // inv(M_ii) and Z_i for every block row, made once by thin_prep_kernel
    // when the launch has several panels (block row i at [2 i, 2 i + 2)
    // tiles of BR x LD floats: inv, then Z); nullptr: each task makes its own
    const float* invz;
};

// Ring stages: STAGES - 1 tiles in flight (cp.async); four stages measured
// the same as three.
constexpr int STAGES = 3;

struct Smem {
    // M_ij tiles, k-major: m[s][kk * LD + r] = M[i0 + r][j0 + kk]; tile j of
    // a task's sum sits in stage (j + 1) % STAGES (stage 0 also serves as the
    // work tile of the inverse and of Z before the ring reaches it)
    float m[STAGES][BR * LD];
    float inv[BR * LD];      // inv(M_ii), k-major: inv[kk * LD + r] = Inv[r][kk]
    float z[BR * LD];        // Z = inv(M_ii) M_i,i-1, k-major
    float x[BR * NP];        // X_jp tile / right-hand side: x[kk * NP + c]
    float dinv[BR];
    int task;
    int abort;
};
constexpr unsigned long long kTag = 1ull << 32;

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr int Q = (BR * NP) / NT;    // tagged words of a block per thread

// Issue the loads of this thread's four words of X_jp (all in flight; the
// values are checked by finish_x, so they can be issued a step ahead).
__device__ __forceinline__ void issue_x(const Params& p, int pn, int j,
                                        unsigned long long (&w)[Q]) {
    const unsigned long long* src = p.xt + ((int64_t)pn * p.nbr + j) * (BR * NP);
#pragma unroll
    for (int q = 0; q < Q; ++q) w[q] = ld_relaxed64(src + threadIdx.x + NT * q);
}

// X_jp into sm.x from its tagged words: a word loaded before it was
// published (tag 0) is polled again (single-copy atomic 64-bit loads: value
// and tag arrive together), at most wait_ns. False on timeout (the error
// word and the launch's stop word are set) or once another CTA has stopped
// the launch.
__device__ bool finish_x(const Params& p, Smem& sm, int pn, int j,
                         const unsigned long long (&w)[Q]) {
    const unsigned long long* src = p.xt + ((int64_t)pn * p.nbr + j) * (BR * NP);
    const int t = threadIdx.x;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int idx = t + NT * q;
        unsigned long long v = w[q];
        if (v < kTag) {
            const uint64_t t0 = gtimer();
            while ((v = ld_relaxed64(src + idx)) < kTag) {
                if (*(volatile int*)p.stop) { ok = false; break; }
                if (gtimer() - t0 > (uint64_t)p.wait_ns) {
                    atomicExch(p.err, kTimeout);
                    atomicExch(p.stop, 1);
                    ok = false;
                    break;
                }
            }
            if (!ok) break;
        }
        sm.x[idx] = __uint_as_float((unsigned)v);
    }
    return ok;
}

// Tile (i0.., j0..) of M into registers, 16 elements a thread, along M's
// contiguous direction; zero outside the strict lower triangle of the order
// (off-diagonal tiles lie below the diagonal: only the order bounds rows).
__device__ __forceinline__ void load_m(const Params& p, int64_t i0, int64_t j0, bool colmajor,
                                       float (&r)[16]) {
    const int t = threadIdx.x;
    const int rr = colmajor ? (t & 63) : (t >> 6), cc = colmajor ? (t >> 6) : (t & 63);
    const float* src = p.A + (i0 + rr) * p.a_rs + (j0 + cc) * p.a_cs;
    const int64_t step = 4 * (colmajor ? p.a_cs : p.a_rs);
    const int64_t rows_left = p.k - (i0 + rr);      // rows of this thread inside the order
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const bool in = colmajor ? rows_left > 0 : rows_left > 4 * q;
        r[q] = in ? __ldg(src + q * step) : 0.0f;
    }
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// all but the newest STAGES - 2 groups complete: the oldest tile in flight has landed
__device__ __forceinline__ void cp_wait_ring() {
    asm volatile("cp.async.wait_group %0;" ::"n"(STAGES - 2) : "memory");
}

// Tile (i0.., j0..) of M into ring stage `dst` by cp.async (element by
// element along M's contiguous direction, into the k-major layout); rows
// past the order are zero-filled (no read). Commits one group.
__device__ __forceinline__ void issue_m(const Params& p, float* dst, int64_t i0, int64_t j0,
                                        bool colmajor) {
    const int t = threadIdx.x;
    const int rr0 = colmajor ? (t & 63) : (t >> 6), cc0 = colmajor ? (t >> 6) : (t & 63);
    const float* src = p.A + (i0 + rr0) * p.a_rs + (j0 + cc0) * p.a_cs;
    const int64_t step = 4 * (colmajor ? p.a_cs : p.a_rs);
    const int64_t rows_left = p.k - (i0 + rr0);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int rr = colmajor ? rr0 : rr0 + 4 * q, cc = colmajor ? cc0 + 4 * q : cc0;
        const bool in = colmajor ? rows_left > 0 : rows_left > 4 * q;
        cp_async4(dst + cc * LD + rr, in ? src + q * step : p.A, in);
    }
    cp_commit();
}

// Packed FP32 pairs: fma.rn.f32x2 does two independent round-to-nearest
// FMAs in one instruction (the same results as two fmaf).
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// acc[e] += sum_kk a[kk][4 ty + e] * x[kk][tx] over kk < kend (rows in
// packed pairs (4 ty, 4 ty + 1), (4 ty + 2, 4 ty + 3): two FMA
// instructions per kk instead of four).
__device__ __forceinline__ void mma_tile(const float* a, const float* x, int kend,
                                         float (&acc)[4]) {
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    uint64_t s01 = pk2(acc[0], acc[1]), s23 = pk2(acc[2], acc[3]);
#pragma unroll 8
    for (int kk = 0; kk < kend; ++kk) {
        const float4 m = *reinterpret_cast<const float4*>(a + kk * LD + 4 * ty);
        const float xv = x[kk * NP + tx];
        const uint64_t xx = pk2(xv, xv);
        s01 = fma2(pk2(m.x, m.y), xx, s01);
        s23 = fma2(pk2(m.z, m.w), xx, s23);
    }
    upk2(s01, acc[0], acc[1]);
    upk2(s23, acc[2], acc[3]);
}

// inv(M_ii) into sm.inv. M_ii's lower triangle goes to a work tile (aliasing
// sm.m) with rows past the order as identity rows; warp w then solves
// M y = e_c for columns c = 8w .. 8w + 7, lane l holding rows l and l + 32:
// at step r the lane owning row r finishes y_r = (delta_rc - s_r) / m_rr
// (reciprocal of m_rr made once), broadcasts it, and every lane adds
// m_row,r y_r into the partial sums of its later rows.
__device__ void invert_diag(const Params& p, Smem& sm, int64_t i0) {
    float* T = sm.m[0];
    const int t = threadIdx.x, w = t >> 5, l = t & 31;
    const bool colmajor = p.a_rs == 1 || p.a_rs == -1;
    for (int e = t; e < BR * BR; e += NT) {
        const int rr = colmajor ? e % BR : e / BR;
        const int cc = colmajor ? e / BR : e % BR;
        const int64_t gi = i0 + rr, gj = i0 + cc;
        float v = 0.0f;
        if (gi >= p.k) v = rr == cc ? 1.0f : 0.0f;
        else if (cc < rr) v = __ldg(p.A + gi * p.a_rs + gj * p.a_cs);
        else if (cc == rr) v = p.unit ? 1.0f : __ldg(p.A + gi * p.a_rs + gj * p.a_cs);
        T[rr * LDT + cc] = v;
    }
    __syncthreads();
    if (t < BR) sm.dinv[t] = 1.0f / T[t * LDT + t];
    __syncthreads();
    float y0[8], y1[8];          // rows l and l + 32, columns 8 w + u
#pragma unroll
    for (int u = 0; u < 8; ++u) y0[u] = y1[u] = 0.0f;
    for (int r = 0; r < BR; ++r) {
        const float dr = sm.dinv[r];
        const int owner = r & 31;
        const bool hi = r >= 32;
        const float m0 = T[l * LDT + r], m1 = T[(l + 32) * LDT + r];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float s = hi ? y1[u] : y0[u];
            const float v = ((r == 8 * w + u) ? 1.0f : 0.0f) - s;
            const float yr = __shfl_sync(0xffffffffu, v * dr, owner);
            if (l == owner) {
                if (hi) y1[u] = yr; else y0[u] = yr;
            }
            if (l > r) y0[u] = fmaf(m0, yr, y0[u]);
            if (l + 32 > r) y1[u] = fmaf(m1, yr, y1[u]);
        }
    }
    // s_r accumulated with +: the recurrence above keeps s = sum m y and
    // y_r = (delta - s) / m_rr
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        sm.inv[(8 * w + u) * LD + l] = y0[u];
        sm.inv[(8 * w + u) * LD + l + 32] = y1[u];
    }
    __syncthreads();
}

// Z = inv(M_ii) M_i,i-1 into sm.z (k-major), M_i,i-1 staged row-major in
// sm.m; thread (ty, tx) forms rows 4 ty .. 4 ty + 3, columns tx + 16 u
// (inv is lower: terms q < 8 (warp + 1) only).
__device__ void make_z(const Params& p, Smem& sm, int64_t i0, bool colmajor) {
    float r[16];
    load_m(p, i0, i0 - BR, colmajor, r);
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int rr = colmajor ? (t & 63) : (t >> 6) + 4 * q;
        const int cc = colmajor ? (t >> 6) + 4 * q : (t & 63);
        sm.m[0][rr * LD + cc] = r[q];
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[e][u] = 0.0f;
    const int qend = 8 * ((t >> 5) + 1);
    for (int q = 0; q < qend; ++q) {
        const float4 iv = *reinterpret_cast<const float4*>(sm.inv + q * LD + 4 * ty);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float mv = sm.m[0][q * LD + tx + 16 * u];
            acc[0][u] = fmaf(iv.x, mv, acc[0][u]);
            acc[1][u] = fmaf(iv.y, mv, acc[1][u]);
            acc[2][u] = fmaf(iv.z, mv, acc[2][u]);
            acc[3][u] = fmaf(iv.w, mv, acc[3][u]);
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int u = 0; u < 4; ++u) sm.z[(tx + 16 * u) * LD + 4 * ty + e] = acc[e][u];
    __syncthreads();
}

// inv(M_ii) and Z_i = inv(M_ii) M_i,i-1 of block row blockIdx.x into
// p.invz, by the same code (so the same values) as a task of the solve
// makes them; with several panels every task of a block row would repeat it.
__global__ void __launch_bounds__(NT) thin_prep_kernel(const Params p, float* invz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int i = blockIdx.x;
    const int64_t i0 = (int64_t)i * BR;
    invert_diag(p, sm, i0);
    if (i > 0) make_z(p, sm, i0, p.a_rs == 1 || p.a_rs == -1);
    float4* dst = reinterpret_cast<float4*>(invz + (size_t)i * 2 * BR * LD);
    for (int e = threadIdx.x; e < BR * LD / 4; e += NT) {
        dst[e] = reinterpret_cast<const float4*>(sm.inv)[e];
        if (i > 0) dst[BR * LD / 4 + e] = reinterpret_cast<const float4*>(sm.z)[e];
    }
}

__global__ void __launch_bounds__(NT, 2) thin_trsm_kernel(const Params p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const bool colmajor = p.a_rs == 1 || p.a_rs == -1;
    if (t == 0) sm.abort = 0;
    while (true) {
        __syncthreads();
        if (t == 0) sm.task = atomicAdd(p.ticket, 1);
        __syncthreads();
        const int64_t task = sm.task;
        if (task >= p.ntask || sm.abort) break;
        const int i = (int)(task / p.npan), pn = (int)(task % p.npan);
        const int64_t i0 = (int64_t)i * BR, c0 = (int64_t)pn * NP;
        // this task's right-hand side rows, read before anything is written
        float b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t gi = i0 + 4 * ty + e, gj = c0 + tx;
            b[e] = (gi < p.k && gj < p.nrhs) ? __ldcg(p.C + gi * p.c_rs + gj * p.c_cs) : 0.0f;
        }
        // S' = sum_{j < i-1} M_ij X_jp (X_i-1,p enters through Z): tile j of M
        // arrives through the cp.async ring (STAGES - 1 tiles ahead), X_jp's words
        // are loaded one step ahead
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        unsigned long long w[Q];
        const int jz = i - 1;
        if (p.invz) {
            // inv(M_ii) and Z_i made by thin_prep_kernel: the oldest copy
            // group, complete by the ring's first wait or the wait below
            const float* src = p.invz + (size_t)i * 2 * BR * LD;
            for (int e = t; e < BR * LD / 4; e += NT) {
                cp_async16(sm.inv + 4 * e, src + 4 * e);
                if (i > 0) cp_async16(sm.z + 4 * e, src + BR * LD + 4 * e);
            }
            cp_commit();
        }
#pragma unroll
        for (int q = 0; q < STAGES - 1; ++q) {      // tiles 0 .. STAGES - 2
            if (q < jz) issue_m(p, sm.m[(q + 1) % STAGES], i0, (int64_t)q * BR, colmajor);
            else cp_commit();
        }
        if (!p.invz) {
            invert_diag(p, sm, i0);
            if (i > 0) make_z(p, sm, i0, colmajor);
        }
        if (jz > 0) issue_x(p, pn, 0, w);
        for (int j = 0; j < jz; ++j) {
            cp_wait_ring();                               // this thread's copies of tile j
            if (!finish_x(p, sm, pn, j, w)) sm.abort = 1;
            __syncthreads();
            if (sm.abort) break;
            // tile j - 1's stage is free: tile j + STAGES - 1 goes there
            if (j + STAGES - 1 < jz)
                issue_m(p, sm.m[j % STAGES], i0, (int64_t)(j + STAGES - 1) * BR, colmajor);
            else cp_commit();
            if (j + 1 < jz) issue_x(p, pn, j + 1, w);
            mma_tile(sm.m[(j + 1) % STAGES], sm.x, BR, acc);
            __syncthreads();
        }
        if (sm.abort) break;
        if (i > 0) issue_x(p, pn, i - 1, w);
        // P = inv(M_ii) (alpha B - S'), then X = P - Z X_i-1,p
#pragma unroll
        for (int e = 0; e < 4; ++e) sm.x[(4 * ty + e) * NP + tx] = fmaf(p.alpha, b[e], -acc[e]);
        if (p.invz) asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        float xo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        mma_tile(sm.inv, sm.x, 8 * ((t >> 5) + 1), xo);   // inv is lower: kk <= row
        if (i > 0) {
            __syncthreads();
            if (!finish_x(p, sm, pn, i - 1, w)) sm.abort = 1;
            __syncthreads();
            if (sm.abort) break;
            float zx[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            mma_tile(sm.z, sm.x, BR, zx);
#pragma unroll
            for (int e = 0; e < 4; ++e) xo[e] -= zx[e];
        }
        // publish the block (tagged words: the chain), then the result in C
        unsigned long long* dst = p.xt + ((int64_t)pn * p.nbr + i) * (BR * NP);
        if (!(p.withhold && i == 0)) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                st_relaxed64(dst + (4 * ty + e) * NP + tx, kTag | __float_as_uint(xo[e]));
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t gi = i0 + 4 * ty + e, gj = c0 + tx;
            if (gi < p.k && gj < p.nrhs) p.C[gi * p.c_rs + gj * p.c_cs] = xo[e];
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // nothing in flight at exit
}

// ---- TRMM with few right-hand sides ---------------------------------------
// C := alpha M C (canonical lower), one persistent launch after a packing
// pass: task (i, p) forms the 64 x 16 block
//     alpha (sum_{j < i} M_ij B_jp + tril(M_ii) B_ip)
// from a packed copy of C's original rows (so no task reads a block another
// task has overwritten) and writes it into C. The tasks need nothing from
// one another; they are taken longest first (block rows from the bottom),
// M tiles and packed B tiles through a cp.async ring.

struct SmemM {
    float m[STAGES][BR * LD];        // M_ij, k-major (as the TRSM's)
    float x[STAGES][BR * NP];        // packed B_jp tiles, row-major
    float d[BR * LD];                // M_ii's lower triangle (unit: diagonal 1), k-major
    int task;
    int last;                        // this CTA's piece arrived last in its row
};

// C's original rows as tiles: tile (p, j) at Bp[(p nbr + j) * BR * NP],
// element (kk, c) at kk * NP + c; zero past the order and the columns.
__global__ void __launch_bounds__(256) thin_pack_kernel(const Params p, float* Bp) {
    const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t total = (int64_t)p.npan * p.nbr * (BR * NP);
    if (e >= total) return;
    const int c = (int)(e % NP), kk = (int)((e / NP) % BR);
    const int64_t tile = e / (BR * NP), j = tile % p.nbr, pn = tile / p.nbr;
    const int64_t gi = j * BR + kk, gj = pn * NP + c;
    Bp[e] = (gi < p.k && gj < p.nrhs) ? p.C[gi * p.c_rs + gj * p.c_cs] : 0.0f;
}

// M_ij and B_jp into ring stage s (one commit group).
__device__ __forceinline__ void issue_mb(const Params& p, SmemM& sm, int s, int64_t i0, int j,
                                         const float* btiles, bool colmajor) {
    const int t = threadIdx.x;
    const int rr0 = colmajor ? (t & 63) : (t >> 6), cc0 = colmajor ? (t >> 6) : (t & 63);
    const float* src = p.A + (i0 + rr0) * p.a_rs + ((int64_t)j * BR + cc0) * p.a_cs;
    const int64_t step = 4 * (colmajor ? p.a_cs : p.a_rs);
    const int64_t rows_left = p.k - (i0 + rr0);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int rr = colmajor ? rr0 : rr0 + 4 * q, cc = colmajor ? cc0 + 4 * q : cc0;
        const bool in = colmajor ? rows_left > 0 : rows_left > 4 * q;
        cp_async4(sm.m[s] + cc * LD + rr, in ? src + q * step : p.A, in);
    }
    cp_async16(sm.x[s] + 4 * t, btiles + (int64_t)j * (BR * NP) + 4 * t);   // 256 x 16 B
    cp_commit();
}

// Long block rows are cut into pieces of at most kPiece off-diagonal tiles
// (the last piece also takes the diagonal block), so no task streams more
// than kPiece + 1 tiles; a row of several pieces writes their partial sums
// to slots, and the piece that arrives last (an atomic count per row)
// adds them in piece order, so the result does not depend on which CTA
// finishes when. Pieces of row i: P_i = max(1, ceil(i / kPiece)).
constexpr int kPiece = 32;
__host__ __device__ __forceinline__ int64_t pieces_of(int64_t i) {
    return i == 0 ? 1 : (i + kPiece - 1) / kPiece;
}
// pieces of rows 0 .. r (r >= -1)
__host__ __device__ __forceinline__ int64_t pieces_upto(int64_t r) {
    if (r < 0) return 0;
    const int64_t a = r / kPiece, b = r % kPiece;
    return 1 + (int64_t)kPiece / 2 * a * (a + 1) + b * (a + 1);
}

__global__ void __launch_bounds__(NT, 2) thin_trmm_kernel(const Params p, const float* Bp,
                                                          float* part, int* count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemM& sm = *reinterpret_cast<SmemM*>(smem_raw);
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const bool colmajor = p.a_rs == 1 || p.a_rs == -1;
    const int64_t total = pieces_upto(p.nbr - 1);
    while (true) {
        __syncthreads();
        if (t == 0) sm.task = atomicAdd(p.ticket, 1);
        __syncthreads();
        const int64_t task = sm.task;
        if (task >= p.ntask) break;
        // pieces are taken from the bottom row up: piece index tp counts
        // down from the last row's pieces
        const int64_t tp = task / p.npan;
        const int pn = (int)(task % p.npan);
        int lo = 0, hi = p.nbr - 1;                  // largest i with pieces of rows >= i > tp
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (total - pieces_upto(mid - 1) > tp) lo = mid; else hi = mid - 1;
        }
        const int i = lo;
        const int64_t np_i = pieces_of(i);
        const int q = (int)(tp - (total - pieces_upto(i)));
        const bool last_piece = q == np_i - 1;
        const int jb = q * kPiece, je = (int)((q + 1) * kPiece < i ? (q + 1) * kPiece : i);
        const int64_t i0 = (int64_t)i * BR, c0 = (int64_t)pn * NP;
        const float* btiles = Bp + (int64_t)pn * p.nbr * (BR * NP);
#pragma unroll
        for (int q = 0; q < STAGES - 1; ++q) {      // tiles jb .. jb + STAGES - 2
            if (jb + q < je) issue_mb(p, sm, (jb + q) % STAGES, i0, jb + q, btiles, colmajor);
            else cp_commit();
        }
        if (last_piece) {
            // M_ii's lower triangle, k-major: d[kk][r] = M(r, kk) for kk <= r
            for (int e = t; e < BR * BR; e += NT) {
                const int rr = colmajor ? e % BR : e / BR, cc = colmajor ? e / BR : e % BR;
                const int64_t gi = i0 + rr, gj = i0 + cc;
                float v = 0.0f;
                if (gi < p.k) {
                    if (cc < rr) v = __ldg(p.A + gi * p.a_rs + gj * p.a_cs);
                    else if (cc == rr) v = p.unit ? 1.0f : __ldg(p.A + gi * p.a_rs + gj * p.a_cs);
                }
                sm.d[cc * LD + rr] = v;
            }
        }
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int j = jb; j < je; ++j) {
            cp_wait_ring();                          // this thread's copies of tile j
            __syncthreads();
            // tile j - 1's stage is free: tile j + STAGES - 1 goes there
            if (j + STAGES - 1 < je)
                issue_mb(p, sm, (j + STAGES - 1) % STAGES, i0, j + STAGES - 1, btiles, colmajor);
            else cp_commit();
            mma_tile(sm.m[j % STAGES], sm.x[j % STAGES], BR, acc);
            __syncthreads();
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (last_piece) {
            // the diagonal block with B_ip (plain loads into stage 0's x)
            *reinterpret_cast<float4*>(sm.x[0] + 4 * t) =
                *reinterpret_cast<const float4*>(btiles + (int64_t)i * (BR * NP) + 4 * t);
            __syncthreads();
            mma_tile(sm.d, sm.x[0], 8 * ((t >> 5) + 1), acc);   // lower: kk <= row
        }
        if (np_i > 1) {
            // partial sums to this piece's slot; the last to arrive combines
            float* slots = part + ((int64_t)pn * total + pieces_upto(i - 1)) * (BR * NP);
#pragma unroll
            for (int e = 0; e < 4; ++e) __stcg(slots + q * (BR * NP) + (4 * ty + e) * NP + tx, acc[e]);
            __threadfence();
            __syncthreads();
            if (t == 0) sm.last = atomicAdd(count + (int64_t)pn * p.nbr + i, 1) == np_i - 1;
            __syncthreads();
            if (!sm.last) continue;
            __threadfence();
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float sum = 0.0f;
                for (int64_t r = 0; r < np_i; ++r)
                    sum += __ldcg(slots + r * (BR * NP) + (4 * ty + e) * NP + tx);
                acc[e] = sum;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t gi = i0 + 4 * ty + e, gj = c0 + tx;
            if (gi < p.k && gj < p.nrhs) p.C[gi * p.c_rs + gj * p.c_cs] = p.alpha * acc[e];
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

}  // namespace thin

// The thin TRSM's scratch: ticket and stop word (16 bytes), the tagged
// words of every (block, panel), and with several panels the block rows'
// inv / Z tiles.
static size_t thin_words_bytes(int64_t nbr, int64_t npan) {
    return 16 + (size_t)(nbr * npan) * kThinBlock * kThinPanel * 8;
}
size_t thin_scratch_bytes(int64_t k, int64_t nrhs) {
    const int64_t nbr = (k + kThinBlock - 1) / kThinBlock;
    const int64_t npan = (nrhs + kThinPanel - 1) / kThinPanel;
    return thin_words_bytes(nbr, npan) +
           (npan > 1 ? (size_t)nbr * 2 * thin::BR * thin::LD * sizeof(float) : 0);
}

static int g_thin_ctas_per_sm = 0, g_thin_trmm_ctas_per_sm = 0;

cudaError_t thin_configure() {
    cudaError_t e0 = cudaFuncSetAttribute(thin::thin_trmm_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(thin::SmemM));
    if (e0 != cudaSuccess) return e0;
    int nm = 0;
    e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nm, thin::thin_trmm_kernel, thin::NT,
                                                       sizeof(thin::SmemM));
    if (e0 != cudaSuccess) return e0;
    g_thin_trmm_ctas_per_sm = nm > 0 ? nm : 1;
    cudaError_t e = cudaFuncSetAttribute(thin::thin_trsm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(thin::Smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(thin::thin_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(thin::Smem));
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, thin::thin_trsm_kernel, thin::NT,
                                                      sizeof(thin::Smem));
    if (e != cudaSuccess) return e;
    g_thin_ctas_per_sm = n > 0 ? n : 1;
    return cudaSuccess;
}

cudaError_t launch_thin_trsm(const Canon<float>& c, float alpha, int* scratch, int* err,
                             long long wait_ns, int num_sms, cudaStream_t s, bool withhold) {
    if (c.k <= 0 || c.nrhs <= 0) return cudaSuccess;
    thin::Params p;
    p.k = c.k;
    p.nrhs = c.nrhs;
    p.A = c.A;
    p.a_rs = c.a_rs;
    p.a_cs = c.a_cs;
    p.C = c.C;
    p.c_rs = c.c_rs;
    p.c_cs = c.c_cs;
    p.alpha = alpha;
    p.unit = c.unit ? 1 : 0;
    const int64_t nbr = (c.k + kThinBlock - 1) / kThinBlock;
    const int64_t npan = (c.nrhs + kThinPanel - 1) / kThinPanel;
    if (nbr * npan > (int64_t)1 << 30) return cudaErrorInvalidValue;
    p.nbr = (int)nbr;
    p.npan = (int)npan;
    p.ntask = nbr * npan;
    p.ticket = scratch;
    p.stop = scratch + 1;
    p.xt = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(scratch) + 16);
    p.err = err;
    p.wait_ns = wait_ns;
    p.withhold = withhold ? 1 : 0;
    p.invz = nullptr;
    // the words (and ticket) are zeroed every launch; inv / Z are written
    cudaError_t e = cudaMemsetAsync(scratch, 0, thin_words_bytes(nbr, npan), s);
    if (e != cudaSuccess) return e;
    if (npan > 1) {
        float* invz = reinterpret_cast<float*>(reinterpret_cast<char*>(scratch) +
                                               thin_words_bytes(nbr, npan));
        thin::thin_prep_kernel<<<(unsigned)nbr, thin::NT, sizeof(thin::Smem), s>>>(p, invz);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        p.invz = invz;
    }
    const int per_sm = g_thin_ctas_per_sm > 0 ? g_thin_ctas_per_sm : 1;
    const int64_t cap = (int64_t)num_sms * per_sm;
    const int grid = (int)(p.ntask < cap ? p.ntask : cap);
    thin::thin_trsm_kernel<<<grid, thin::NT, sizeof(thin::Smem), s>>>(p);
    return cudaGetLastError();
}

// The thin TRMM's scratch: ticket (16 bytes), per-row piece counts, C's
// rows packed by tiles, the pieces' partial sums; zeroed / written by the
// launch itself.
static int64_t align_words(int64_t n) { return (n + 3) / 4 * 4; }   // 16-byte steps (4-byte words)

size_t thin_trmm_scratch_bytes(int64_t k, int64_t nrhs) {
    const int64_t nbr = (k + kThinBlock - 1) / kThinBlock;
    const int64_t npan = (nrhs + kThinPanel - 1) / kThinPanel;
    const int64_t tile = (int64_t)kThinBlock * kThinPanel;
    return 4 * (size_t)(4 + align_words(nbr * npan) + nbr * npan * tile +
                        thin::pieces_upto(nbr - 1) * npan * tile);
}

cudaError_t launch_thin_trmm(const Canon<float>& c, float alpha, int* scratch, int num_sms,
                             cudaStream_t s) {
    if (c.k <= 0 || c.nrhs <= 0) return cudaSuccess;
    thin::Params p{};
    p.k = c.k;
    p.nrhs = c.nrhs;
    p.A = c.A;
    p.a_rs = c.a_rs;
    p.a_cs = c.a_cs;
    p.C = c.C;
    p.c_rs = c.c_rs;
    p.c_cs = c.c_cs;
    p.alpha = alpha;
    p.unit = c.unit ? 1 : 0;
    const int64_t nbr = (c.k + kThinBlock - 1) / kThinBlock;
    const int64_t npan = (c.nrhs + kThinPanel - 1) / kThinPanel;
    const int64_t total = thin::pieces_upto(nbr - 1);
    if (total * npan > (int64_t)1 << 30) return cudaErrorInvalidValue;
    p.nbr = (int)nbr;
    p.npan = (int)npan;
    p.ntask = total * npan;
    p.ticket = scratch;
    int* count = scratch + 4;
    float* Bp = reinterpret_cast<float*>(scratch + 4 + align_words(nbr * npan));
    float* part = Bp + nbr * npan * (int64_t)(kThinBlock * kThinPanel);
    cudaError_t e = cudaMemsetAsync(scratch, 0, 4 * (size_t)(4 + align_words(nbr * npan)), s);
    if (e != cudaSuccess) return e;
    const int64_t packed = nbr * npan * (kThinBlock * kThinPanel);
    thin::thin_pack_kernel<<<(unsigned)((packed + 255) / 256), 256, 0, s>>>(p, Bp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int per_sm = g_thin_trmm_ctas_per_sm > 0 ? g_thin_trmm_ctas_per_sm : 1;
    const int64_t cap = (int64_t)num_sms * per_sm;
    const int grid = (int)(p.ntask < cap ? p.ntask : cap);
    thin::thin_trmm_kernel<<<grid, thin::NT, sizeof(thin::SmemM), s>>>(p, Bp, part, count);
    return cudaGetLastError();
}

}  // namespace trx

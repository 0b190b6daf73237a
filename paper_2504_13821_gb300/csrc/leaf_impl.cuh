// Leaf ("base case") TRSM and TRMM kernels, Section 3.3 of the paper.
//
// Below the recursion cutoff a diagonal block of M (b x b, lower, canonical
// form of common.cuh) is applied to all right-hand sides of its row block:
//   TRSM: solve M_blk X = alpha C_blk by forward substitution, X -> C_blk
//   TRMM: C_blk := alpha M_blk C_blk
//
// Work split. G lanes of one warp share a right-hand side; lane g owns the
// rows g, g+G, g+2G, ... of its column (interleaved, so the shrinking active
// set of a forward sweep stays balanced across the lanes) and holds them in
// registers. A CTA of 128 threads covers NCOL = 128/G right-hand sides at a
// time and is persistent: it stages the triangle once and then walks panels
// of NCOL columns (each staged through shared memory with coalesced loads
// along whichever index is contiguous in C), so the triangle is read from L2
// once per CTA, not once per panel. G is picked per launch from the number of right-hand sides per SM
// (G = 1 when there are many: a thread owns a whole column and the sweep
// needs no communication; larger G to keep enough warps in flight when
// there are few).
//
// The sweep. Step j takes x_j from its owner lane by a warp shuffle (G > 1)
// and every lane updates its own rows below j with one FMA each. There is no
// block-level barrier inside the sweep: the row dependency that the paper
// resolves with one synchronisation per row (Section 3.3, "Reformulation of
// algorithm for parallelism") is carried by the shuffle inside the G-lane
// group, and columns are independent.
//
// Shared-memory layout of the triangle: column l of M holds its rows in
// lane-major order, row i at (i % G) * RPLP + i / G, so the RPL rows one lane
// owns are contiguous and come in 16-byte vector loads; RPLP = RPL + 4 pads
// the lanes of a column group onto different banks. All lanes working on one
// column group read the same addresses for every other column group of the
// warp (a broadcast).
//
// TRMM runs the columns of M in descending order, so every x_j is read
// before any update writes row j (in place, no copy).
#pragma once
#include <type_traits>

#include "common.cuh"

namespace trx {

template <typename T>
struct LeafArgs {
    Canon<T> p;
    int64_t r0;     // start row of leaf 0 of this launch
    int b;          // leaf size (row stride between batched leaves)
    T alpha;
    Planes pl;
    int planes;     // TRSM on the tensor-core path: also write the Y planes
};

namespace {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int n = 2;
};

template <typename T, int B, int G>
struct LeafShape {
    static constexpr int NT = 128;
    static constexpr int NCOL = NT / G;
    static constexpr int RPL = B / G;                        // rows per lane
    static constexpr int VN = Vec<T>::n;
    static constexpr int RPLP = (G == 1) ? RPL : RPL + 4;    // padded lane stride
    static constexpr int LDT = G * RPLP;                     // column stride of sT
    static constexpr int PAD = (G == 1) ? 1 : G;              // conflict-free panel reads
    static constexpr int LDS = B + PAD;                       // column stride of sC
    static constexpr size_t smem = sizeof(T) * (size_t)(B * LDT + B + NCOL * LDS);
    static_assert((B * NCOL) % NT == 0, "panel staging in whole passes");
    static_assert(RPL % VN == 0 && RPLP % VN == 0, "vector loads need aligned lane blocks");
};

template <typename T>
__device__ __forceinline__ void vload(const T* p, T (&v)[Vec<T>::n]) {
    const typename Vec<T>::type w = *reinterpret_cast<const typename Vec<T>::type*>(p);
    if constexpr (Vec<T>::n == 4) {
        v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else {
        v[0] = w.x; v[1] = w.y;
    }
}

// The vector groups of column l that a sweep step needs (rows at or below
// the step's own row block), into v[q] for this lane's rows q.
template <typename T, typename S>
__device__ __forceinline__ void load_col(const T* my, int l, T (&v)[S::RPL]) {
    const int first = ((l / (S::NT / S::NCOL)) / S::VN) * S::VN;   // l / G, rounded to a group
#pragma unroll
    for (int q0 = 0; q0 < S::RPL; q0 += S::VN) {
        if (q0 < first) continue;
        T t[S::VN];
        vload(my + l * S::LDT + q0, t);
#pragma unroll
        for (int e = 0; e < S::VN; ++e) v[q0 + e] = t[e];
    }
}

template <typename T, int B, int G, bool TRSM>
__global__ void __launch_bounds__(128)
leaf_kernel(LeafArgs<T> a) {
    using S = LeafShape<T, B, G>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sT = reinterpret_cast<T*>(smem_raw);   // M(r0+i, r0+l) at l*LDT + (i%G)*RPLP + i/G
    T* sD = sT + B * S::LDT;                   // 1/M(i,i) (TRSM) or M(i,i) (TRMM)
    T* sC = sD + B;                            // panel: C(r0+i, j0+c) at c*LDS + i

    pdl_trigger();
    pdl_wait();
    const int tid = threadIdx.x;
    const Canon<T>& p = a.p;
    const int64_t r0 = a.r0 + (int64_t)blockIdx.y * a.b;
    const int64_t rem = p.k - r0;
    if (rem <= 0) return;
    const int bs = rem < a.b ? (int)rem : a.b;

    // Triangle (strictly lower part; zero elsewhere and past a ragged edge),
    // read along A's contiguous index; all loads of a thread in flight.
    // Each thread keeps one fixed index (the contiguous one) and walks the
    // other with a pointer, so unrolled loads need no per-element address.
    const bool a_row_fast = (p.a_rs == 1 || p.a_rs == -1);
    {
        constexpr int TPASS = (B * B + S::NT - 1) / S::NT;
        constexpr int ADV = S::NT / B;          // other-index advance per pass
        const int fixed = tid % B, first = tid / B;
        const int64_t st_fixed = a_row_fast ? p.a_rs : p.a_cs;
        const int64_t st_walk = a_row_fast ? p.a_cs : p.a_rs;
        const T* src = p.A + (r0 + fixed) * st_fixed + (r0 + first) * st_walk;
#pragma unroll
        for (int u = 0; u < TPASS; ++u) {
            const int w = first + u * ADV;
            if (w < B) {
                const int i = a_row_fast ? fixed : w, l = a_row_fast ? w : fixed;
                T v = T(0);
                if (i < bs && l < i) v = *src;
                sT[l * S::LDT + (i % G) * S::RPLP + i / G] = v;
            }
            src += ADV * st_walk;
        }
    }
    for (int i = tid; i < B; i += S::NT) {
        T d = T(1);
        if (i < bs && !p.unit) d = p.A[(r0 + i) * (p.a_rs + p.a_cs)];
        if (TRSM) sD[i] = (i < bs && !p.unit) ? T(1) / d : T(1);
        else      sD[i] = (i < bs) ? d : T(0);
    }
    __syncthreads();

    const int c = tid / G, g = tid % G;
    const T* my = sT + g * S::RPLP;            // this lane's rows of column l: my[l*LDT + q]
    const bool c_row_fast = (p.c_rs == 1 || p.c_rs == -1);
    const int64_t npanels = (p.nrhs + S::NCOL - 1) / S::NCOL;
#pragma unroll 1
    for (int64_t panel = blockIdx.x; panel < npanels; panel += gridDim.x) {
        const int64_t j0 = panel * S::NCOL;
        // Panel through shared memory: coalesced along whichever index is
        // contiguous in C, all of a thread's loads in flight.
        // Thread keeps row `fi` (rows contiguous in C) or column `fi`
        // (columns contiguous) and walks the other index by a pointer.
        const int np = B * S::NCOL / S::NT;
        const int fmod = c_row_fast ? B : S::NCOL;
        const int fi = tid % fmod, wi = tid / fmod, adv = S::NT / fmod;
        const int64_t st_fixed = c_row_fast ? p.c_rs : p.c_cs;
        const int64_t st_walk = c_row_fast ? p.c_cs : p.c_rs;
        {
            const T* src = p.C + (c_row_fast ? (r0 + fi) * p.c_rs + (j0 + wi) * p.c_cs
                                             : (r0 + wi) * p.c_rs + (j0 + fi) * p.c_cs);
#pragma unroll
            for (int u = 0; u < np; ++u) {
                const int w = wi + u * adv;
                const int i = c_row_fast ? fi : w, cc = c_row_fast ? w : fi;
                T v = T(0);
                if (i < bs && j0 + cc < p.nrhs) v = *src;
                sC[cc * S::LDS + i] = v;
                src += adv * st_walk;
            }
        }
        __syncthreads();
        T r[S::RPL];
#pragma unroll
        for (int q = 0; q < S::RPL; ++q) r[q] = sC[c * S::LDS + q * G + g];

        // Column jj of the triangle is consumed from registers loaded one
        // step earlier (cur), while the next column's loads (nxt) are in
        // flight: the shared-memory latency hides behind a step of FMAs.
        // The compiler barrier at the end of a step stops it from hoisting
        // more columns than that into registers.
        T cur[S::RPL], nxt[S::RPL];
        if (TRSM) {
#pragma unroll
            for (int q = 0; q < S::RPL; ++q) r[q] *= a.alpha;
            load_col<T, S>(my, 0, cur);
#pragma unroll
            for (int jj = 0; jj < B; ++jj) {
                const int qj = jj / G, gj = jj % G;
                if (jj + 1 < B) load_col<T, S>(my, jj + 1, nxt);
                const T v = r[qj] * sD[jj];
                T xj;
                if (G == 1) {
                    r[qj] = v;
                    xj = v;
                } else {
                    xj = __shfl_sync(0xffffffffu, v, gj, G);
                    if (g == gj) r[qj] = v;
                }
#pragma unroll
                for (int q = qj; q < S::RPL; ++q) {
                    if (q == qj && g <= gj) continue;
                    r[q] = fma(-cur[q], xj, r[q]);
                }
#pragma unroll
                for (int q = 0; q < S::RPL; ++q) cur[q] = nxt[q];
                asm volatile("" ::: "memory");
            }
        } else {
            load_col<T, S>(my, B - 1, cur);
#pragma unroll
            for (int jj = B - 1; jj >= 0; --jj) {
                const int qj = jj / G, gj = jj % G;
                if (jj > 0) load_col<T, S>(my, jj - 1, nxt);
                const T xj = (G == 1) ? r[qj] : __shfl_sync(0xffffffffu, r[qj], gj, G);
#pragma unroll
                for (int q = qj; q < S::RPL; ++q) {
                    if (q == qj && g <= gj) continue;
                    r[q] = fma(cur[q], xj, r[q]);
                }
                if (g == gj) r[qj] = sD[jj] * xj;
#pragma unroll
                for (int q = 0; q < S::RPL; ++q) cur[q] = nxt[q];
                asm volatile("" ::: "memory");
            }
#pragma unroll
            for (int q = 0; q < S::RPL; ++q) r[q] *= a.alpha;
        }

#pragma unroll
        for (int q = 0; q < S::RPL; ++q) sC[c * S::LDS + q * G + g] = r[q];
        __syncthreads();
        {
            T* dst = p.C + (c_row_fast ? (r0 + fi) * p.c_rs + (j0 + wi) * p.c_cs
                                       : (r0 + wi) * p.c_rs + (j0 + fi) * p.c_cs);
#pragma unroll
            for (int u = 0; u < np; ++u) {
                const int w = wi + u * adv;
                const int i = c_row_fast ? fi : w, cc = c_row_fast ? w : fi;
                if (i < bs && j0 + cc < p.nrhs) *dst = sC[cc * S::LDS + i];
                dst += adv * st_walk;
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (TRSM && a.planes) {
                // Y planes, element (l, j) at j*ldy + l: rows fastest.
                const int pi = tid % B, pc = tid / B;
                int64_t yo = (j0 + pc) * a.pl.ldy + r0 + pi;
                const int64_t ystep = (int64_t)(S::NT / B) * a.pl.ldy;
#pragma unroll
                for (int u = 0; u < np; ++u) {
                    const int cc = pc + u * (S::NT / B);
                    if (pi < bs && j0 + cc < p.nrhs) put_y(a.pl, yo, sC[cc * S::LDS + pi]);
                    yo += ystep;
                }
            }
        }
        __syncthreads();   // sC is refilled by the next panel
    }
}

template <typename T, int B, int G, bool TRSM>
cudaError_t configure_one() {
    using S = LeafShape<T, B, G>;
    return cudaFuncSetAttribute(leaf_kernel<T, B, G, TRSM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
}

// grid.x: persistent CTAs per leaf (at most one per panel), grid.y: leaves.
template <typename T, int B, int G, bool TRSM>
cudaError_t launch_one(const LeafArgs<T>& a, int64_t nleaves, int64_t max_ctas, cudaStream_t s) {
    using S = LeafShape<T, B, G>;
    const int64_t npanels = (a.p.nrhs + S::NCOL - 1) / S::NCOL;
    int64_t per_leaf = (max_ctas + nleaves - 1) / nleaves;
    if (per_leaf < 1) per_leaf = 1;
    const int64_t nx = npanels < per_leaf ? npanels : per_leaf;
    dim3 grid((unsigned)nx, (unsigned)nleaves);
    return launch_kernel(leaf_kernel<T, B, G, TRSM>, grid, dim3(S::NT), S::smem, s, a);
}

template <typename T, int B, bool TRSM>
cudaError_t launch_b(const LeafArgs<T>& a, int64_t nleaves, int G, int64_t max_ctas,
                     cudaStream_t s) {
    // A thread owns B/G rows in registers: at most 32 (64 for FP32 with
    // G = 4) so the fully unrolled sweep stays in registers, and at least 4
    // so a lane's rows fill a vector load.
    if constexpr (B <= 32) {
        if (G == 1) return launch_one<T, B, 1, TRSM>(a, nleaves, max_ctas, s);
    }
    if constexpr (B == 128 && sizeof(T) == 8) {
        if (G <= 8) return launch_one<T, B, 8, TRSM>(a, nleaves, max_ctas, s);
    }
    if constexpr (B >= 64) {
        if (G >= 16) return launch_one<T, B, 16, TRSM>(a, nleaves, max_ctas, s);
    }
    if constexpr (B >= 32) {
        if (G >= 8) return launch_one<T, B, 8, TRSM>(a, nleaves, max_ctas, s);
    }
    return launch_one<T, B, 4, TRSM>(a, nleaves, max_ctas, s);
}

}  // namespace

// Shared-memory limits of every instantiation, once per device (the
// handle calls this at creation, before any launch can be captured).
template <typename T, bool TRSM>
cudaError_t leaf_configure() {
    cudaError_t e;
#define TRX_CFG(B, G) \
    if ((e = configure_one<T, B, G, TRSM>()) != cudaSuccess) return e;
    TRX_CFG(16, 1) TRX_CFG(16, 4)
    TRX_CFG(32, 1) TRX_CFG(32, 4) TRX_CFG(32, 8)
    TRX_CFG(64, 4) TRX_CFG(64, 8) TRX_CFG(64, 16)
    TRX_CFG(128, 8) TRX_CFG(128, 16)
    if constexpr (sizeof(T) == 4) {
        TRX_CFG(128, 4)
    }
#undef TRX_CFG
    return cudaSuccess;
}

template <typename T, bool TRSM>
cudaError_t leaf_dispatch(const LeafArgs<T>& a, int64_t nleaves, int G, int64_t max_ctas,
                          cudaStream_t s) {
    if (a.b <= 16) return launch_b<T, 16, TRSM>(a, nleaves, G, max_ctas, s);
    if (a.b <= 32) return launch_b<T, 32, TRSM>(a, nleaves, G, max_ctas, s);
    if (a.b <= 64) return launch_b<T, 64, TRSM>(a, nleaves, G, max_ctas, s);
    return launch_b<T, 128, TRSM>(a, nleaves, G, max_ctas, s);
}

}  // namespace trx

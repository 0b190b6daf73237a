// Peak-rate probes: the arithmetic rates the rooflines of this library are
// quoted against, measured with its own kernels on the device it runs on
// (the BF16 tensor and HBM copy peaks come from outside measurements; the
// others have no source but these).
//
//   TRX_PEAK_FFMA      FP32 FMA on the CUDA cores (the CUDA-core update
//                      engine and the leaf kernels' arithmetic)
//   TRX_PEAK_DFMA      FP64 FMA on the CUDA cores (the FP64 update engine)
//   TRX_PEAK_DMMA      FP64 warp-level MMA, mma.sync m8n8k4 (the alternative
//                      FP64 update engine)
//   TRX_PEAK_TC_TF32   tcgen05.mma kind::tf32, M = 128, N = 256, K = 8
//   TRX_PEAK_TC_BF16   tcgen05.mma kind::f16 with BF16 operands, M = 128,
//                      N = 256, K = 16 (cross-check of the outside BF16 peak)
//
// Each probe is one launch of one CTA per SM (several for the CUDA-core
// probes) whose loop keeps the unit busy with independent work; the rate is
// the work of the launch over its CUDA-event time. The tensor-core probes
// issue MMAs back to back on operands resident in shared memory (filled
// with small finite values), with the accumulator in tensor memory, and
// wait for them on an mbarrier with a bounded wait (the error word gets
// TRX_ERR_TIMEOUT past 2 s and the CTA still frees its tensor memory).
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "trx.h"

namespace trx {
namespace {

constexpr int kFmaThreads = 256;
constexpr int kChains = 8;                // independent FMA chains per thread

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) fma_probe_kernel(int64_t iters, T seed, T* sink) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T b = (T)0.999999, d = (T)1e-7;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-1.2345) sink[threadIdx.x] = s;     // keeps the loop, never taken
}

// mma.sync m8n8k4 FP64: D(8x8) += A(8x4) B(4x8), one per warp per step.
__global__ void __launch_bounds__(kFmaThreads) dmma_probe_kernel(int64_t iters, double seed,
                                                                 double* sink) {
    double acc[kChains][2];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double a = seed + threadIdx.x * 1e-3, b = seed - threadIdx.x * 1e-3;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            asm volatile(
                "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                : "+d"(acc[c][0]), "+d"(acc[c][1])
                : "d"(a), "d"(b));
        }
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c][0] + acc[c][1];
    if (s == -1.2345) sink[threadIdx.x] = s;
}

// ---- tcgen05 probes -----------------------------------------------------------
constexpr int kTcN = 256, kTcM = 128;
constexpr int kTcATile = kTcM * 64;              // bytes: 128 rows x 64 B (one K step)
constexpr int kTcBTile = kTcN * 64;
constexpr int kTcSmem = 1024 + kTcATile + kTcBTile + 64;

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// K-major operand, 64-byte swizzle, 8-row groups 512 B apart (as the GEMM
// update's operands).
__device__ __forceinline__ uint64_t probe_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// kind::f16 with BF16 operands: K = 16 per MMA (32 B of each 64-B operand
// row), two MMAs per step over the two halves of the rows.
__global__ void __launch_bounds__(128, 1) tc_probe_bf16_kernel(int64_t iters, int* err,
                                                              long long wait_ns) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const uint32_t raw = su32(sm_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = sm_raw + (base - raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(gbase + kTcATile + kTcBTile);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    // small finite operands: 1 + (i mod 7) / 8
    for (int i = threadIdx.x; i < (kTcATile + kTcBTile) / 4; i += blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(1.0f + (float)(i % 7) * 0.125f);
        const uint16_t hb = *reinterpret_cast<const uint16_t*>(&h);
        reinterpret_cast<uint32_t*>(gbase)[i] = (uint32_t)hb | ((uint32_t)hb << 16);
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tmem_slot)),
                     "r"(kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        // D = F32, A and B BF16, both K-major
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
        const uint64_t a0 = probe_desc(base), b0 = probe_desc(base + kTcATile);
        const uint64_t a1 = probe_desc(base + 32), b1 = probe_desc(base + kTcATile + 32);
        for (int64_t it = 0; it < iters; ++it) {
            const uint32_t acc0 = it > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                "l"(a0), "l"(b0), "r"(idesc), "r"(acc0));
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                "l"(a1), "l"(b1), "r"(idesc), "r"(1u));
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(bar))
            : "memory");
        // bounded wait for the MMAs
        uint64_t t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        while (true) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(ok)
                : "r"(su32(bar))
                : "memory");
            if (ok) break;
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > (uint64_t)wait_ns) {
                atomicExch(err, TRX_ERR_TIMEOUT);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcN)
                     : "memory");
}

}  // namespace
}  // namespace trx

// kind::tf32: K = 8 per MMA (32 B of each 64-B operand row of FP32 values),
// two MMAs per step; D = F32, A and B TF32 (format 2), both K-major.
namespace trx {
namespace {
__global__ void __launch_bounds__(128, 1) tc_probe_tf32_kernel(int64_t iters, int* err,
                                                              long long wait_ns) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const uint32_t raw = su32(sm_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = sm_raw + (base - raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(gbase + kTcATile + kTcBTile);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    for (int i = threadIdx.x; i < (kTcATile + kTcBTile) / 4; i += blockDim.x)
        reinterpret_cast<float*>(gbase)[i] = 1.0f + (float)(i % 7) * 0.125f;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tmem_slot)),
                     "r"(kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                               ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
        const uint64_t a0 = probe_desc(base), b0 = probe_desc(base + kTcATile);
        const uint64_t a1 = probe_desc(base + 32), b1 = probe_desc(base + kTcATile + 32);
        for (int64_t it = 0; it < iters; ++it) {
            const uint32_t acc0 = it > 0 ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                "l"(a0), "l"(b0), "r"(idesc), "r"(acc0));
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                "l"(a1), "l"(b1), "r"(idesc), "r"(1u));
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                su32(bar))
            : "memory");
        uint64_t t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        while (true) {
            uint32_t ok;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(ok)
                : "r"(su32(bar))
                : "memory");
            if (ok) break;
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > (uint64_t)wait_ns) {
                atomicExch(err, TRX_ERR_TIMEOUT);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcN)
                     : "memory");
}
}  // namespace
}  // namespace trx

extern "C" int trx_peak_probe(int device, int kind, int64_t iters, double* tflops, double* ms) {
    using namespace trx;
    if (kind < TRX_PEAK_FFMA || kind > TRX_PEAK_TC_BF16) return TRX_ERR_INVALID_VALUE;
    if (iters <= 0 || !tflops) return TRX_ERR_INVALID_VALUE;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return TRX_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return TRX_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return TRX_ERR_DEVICE;
    const int sms = prop.multiProcessorCount;
    void* scratch = nullptr;
    if (cudaMalloc(&scratch, 64 * 1024) != cudaSuccess) return TRX_ERR_ALLOC;
    int* err = static_cast<int*>(scratch);
    cudaMemset(err, 0, sizeof(int));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double flop = 0.0;
    const int ctas_cc = sms * 8;              // CUDA-core probes: 8 CTAs of 256 per SM
    cudaEventRecord(e0);
    switch (kind) {
        case TRX_PEAK_FFMA:
            fma_probe_kernel<float><<<ctas_cc, kFmaThreads>>>(iters, 1.0f,
                                                              static_cast<float*>(scratch) + 64);
            flop = 2.0 * ctas_cc * kFmaThreads * (double)iters * 16 * kChains;
            break;
        case TRX_PEAK_DFMA:
            fma_probe_kernel<double><<<ctas_cc, kFmaThreads>>>(iters, 1.0,
                                                               static_cast<double*>(scratch) + 32);
            flop = 2.0 * ctas_cc * kFmaThreads * (double)iters * 16 * kChains;
            break;
        case TRX_PEAK_DMMA:
            dmma_probe_kernel<<<ctas_cc, kFmaThreads>>>(iters, 1.0,
                                                        static_cast<double*>(scratch) + 32);
            // per warp per step: 8 x 8 x 4 multiply-adds
            flop = 2.0 * 8 * 8 * 4 * (double)ctas_cc * (kFmaThreads / 32) * iters * kChains;
            break;
        case TRX_PEAK_TC_TF32:
            cudaFuncSetAttribute(tc_probe_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kTcSmem);
            tc_probe_tf32_kernel<<<sms, 128, kTcSmem>>>(iters, err, 2000000000LL);
            flop = 2.0 * kTcM * kTcN * 8 * 2.0 * (double)iters * sms;
            break;
        case TRX_PEAK_TC_BF16:
            cudaFuncSetAttribute(tc_probe_bf16_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
            tc_probe_bf16_kernel<<<sms, 128, kTcSmem>>>(iters, err, 2000000000LL);
            flop = 2.0 * kTcM * kTcN * 16 * 2.0 * (double)iters * sms;
            break;
    }
    e = cudaGetLastError();
    cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    int dev_err = 0;
    if (e == cudaSuccess) {
        cudaEventElapsedTime(&t, e0, e1);
        e = cudaMemcpy(&dev_err, err, sizeof(int), cudaMemcpyDeviceToHost);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    if (e != cudaSuccess) return TRX_ERR_CUDA;
    if (dev_err) return TRX_ERR_TIMEOUT;
    *tflops = t > 0 ? flop / (t * 1e-3) / 1e12 : 0.0;
    if (ms) *ms = t;
    return TRX_SUCCESS;
}

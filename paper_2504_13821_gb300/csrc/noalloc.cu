// trx_strsm_noalloc: FP32 TRSM that allocates no device memory.
//
// Who needs this: code that may not call cudaMalloc at the point where it
// solves, for example a solve issued while a stream is being captured into a
// CUDA graph (cudaMalloc is not capturable), inside a framework that hands
// out device memory only from its own fixed pool, or in a latency-bound
// loop that must not pay cudaMalloc's implicit synchronisation or risk its
// out-of-memory failure halfway through. Such callers cannot create a
// handle (trx_create allocates the handle's error word) nor supply a
// workspace.
//
// The tensor-core path's scratch (the split-BF16 operand planes) lives
// instead in one file-scope __device__ array of TRX_NOALLOC_SCRATCH_BYTES,
// reserved on every device that loads this library until the process
// exits. In host code the array's name is only a host-side stand-in, never a
// device address: the set-up below asks the runtime for the real address
// (cudaGetSymbolAddress, once per device, with that device current) and the
// kernels are given that pointer.
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "trx.h"

namespace trx {
cudaError_t leaf_configure_all();
int noalloc_check_args(char side, char uplo, char transa, char diag, int64_t m, int64_t n,
                       const void* A, int64_t lda, const void* B, int64_t ldb);
size_t noalloc_scratch_bytes(char side, int64_t m, int64_t n);
int noalloc_strsm(int device, int num_sms, void* scratch, size_t scratch_bytes, int* err_word,
                  long long wait_ns, char side, char uplo, char transa, char diag, int64_t m,
                  int64_t n, float alpha, const float* A, int64_t lda, float* B, int64_t ldb,
                  void* stream);
const char* set_detail(const char* msg);
}  // namespace trx

static __device__ __align__(256) unsigned char trx_noalloc_scratch[TRX_NOALLOC_SCRATCH_BYTES];
// Error word of the bounded device-side waits: cleared by every call, read
// and cleared by trx_noalloc_check_error.
static __device__ __align__(256) int trx_noalloc_err_word[64];

namespace {

struct DeviceSetup {
    bool ready = false;
    void* scratch = nullptr;
    int* err = nullptr;
    int num_sms = 0;
    long long wait_ns = 2000000000LL;
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: device addresses of the two
// arrays, the SM count and the kernels' shared-memory limits.
int setup_device(int dev, DeviceSetup** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return TRX_ERR_CUDA;
        if (prop.major != 10 || prop.minor != 3) return TRX_ERR_DEVICE;
        void* scratch = nullptr;
        void* err = nullptr;
        if (cudaGetSymbolAddress(&scratch, trx_noalloc_scratch) != cudaSuccess ||
            cudaGetSymbolAddress(&err, trx_noalloc_err_word) != cudaSuccess)
            return TRX_ERR_CUDA;
        if (trx::leaf_configure_all() != cudaSuccess) return TRX_ERR_CUDA;
        s.scratch = scratch;
        s.err = static_cast<int*>(err);
        s.num_sms = prop.multiProcessorCount;
        // budget of each bounded device-side wait (2 s; TRX_NOALLOC_WAIT_NS
        // overrides it, at least 1000 ns, read once per device here)
        if (const char* v = std::getenv("TRX_NOALLOC_WAIT_NS")) {
            const long long w = std::atoll(v);
            if (w >= 1000) s.wait_ns = w;
        }
        s.ready = true;
    }
    *out = &s;
    return TRX_SUCCESS;
}

}  // namespace

extern "C" int trx_strsm_noalloc(char side, char uplo, char transa, char diag, int64_t m,
                                 int64_t n, float alpha, const float* A, int64_t lda, float* B,
                                 int64_t ldb, void* stream) {
    const int info = trx::noalloc_check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    if (info) return info;
    if (m == 0 || n == 0) return TRX_SUCCESS;
    const size_t need = trx::noalloc_scratch_bytes(side, m, n);
    if (need > TRX_NOALLOC_SCRATCH_BYTES) {
        trx::set_detail("trx_strsm_noalloc: problem needs more scratch than the static "
                        "TRX_NOALLOC_SCRATCH_BYTES array holds");
        return TRX_ERR_WORKSPACE;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TRX_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TRX_ERR_DEVICE;
    DeviceSetup* s = nullptr;
    const int rc = setup_device(dev, &s);
    if (rc != TRX_SUCCESS) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(s->err, 0, sizeof(int), st) != cudaSuccess) return TRX_ERR_CUDA;
    return trx::noalloc_strsm(dev, s->num_sms, s->scratch, TRX_NOALLOC_SCRATCH_BYTES, s->err,
                              s->wait_ns, side, uplo, transa, diag, m, n, alpha, A, lda, B, ldb,
                              stream);
}

// Read and clear the error word of the current device (a plain copy from the
// symbol: nothing is allocated). 0 if no call has run on this device yet.
extern "C" int trx_noalloc_check_error(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TRX_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TRX_ERR_DEVICE;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_setup[dev].ready) return TRX_SUCCESS;
    }
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, trx_noalloc_err_word, sizeof(int)) != cudaSuccess)
        return TRX_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(trx_noalloc_err_word, &zero, sizeof(int)) != cudaSuccess)
            return TRX_ERR_CUDA;
    }
    return v;
}

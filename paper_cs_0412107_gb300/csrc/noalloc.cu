// noalloc.cu -- the tensor-core block accumulation for callers that cannot
// allocate device memory.
//
// mcinv_block_accumulate_noalloc runs the same two steps as one batch of the
// block estimate -- the BF16 tensor-core contraction D = A B^T into an FP32
// product, then the FP64 fold sum += D, sq += D^2 * scale_sq -- but the FP32
// product lives in a fixed array compiled into the library instead of memory
// the library allocates.  Callers that budget all device memory up front (a
// serving process holding a fixed arena), or that cannot afford the implicit
// device-wide synchronisation of cudaMalloc/cudaFree in the middle of their
// work, pass their own operands and FP64 accumulators and the library
// allocates nothing, on the device or the host.
#include <mutex>

#include "../../include/mcinv.h"
#include "internal.h"
#include "tc_gemm.h"

namespace {

constexpr long long kMaxProduct = 1LL << 21;  // FP32 elements of D: 8 MiB
constexpr long long kStatusOffset = kMaxProduct * 4;

// D (kMaxProduct floats), then one status word.  Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kStatusOffset + 256];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (in host code the symbol is only a host-side stand-in).  The address
// is kept for the life of the process: after a cudaDeviceReset the module is
// loaded again and the kept address may no longer be the array's, so the
// entry point must not be used across a device reset.
cudaError_t scratch_on_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = (unsigned char *)p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

// sum += D, sq += D^2 * scale_sq over the M*N product, unless the contraction
// reported a failure in *status: then the caller's accumulators are left as
// they were (tiles abandoned after an expired wait were never written, so D
// still holds an earlier call's product there).  One element a thread per
// step, explicit round-to-nearest double operations as in the handle's fold.
__global__ void guarded_fold_kernel(long long elems, double scale_sq, const float *__restrict__ D,
                                    double *__restrict__ sum, double *__restrict__ sq,
                                    const int *__restrict__ status)
{
    if (*(const volatile int *)status != 0) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < elems; e += stride) {
        const double x = D[e];
        sum[e] = __dadd_rn(sum[e], x);
        sq[e] = __fma_rn(__dmul_rn(x, x), scale_sq, sq[e]);
    }
}

}  // namespace

extern "C" mcinv_status mcinv_block_accumulate_noalloc(int64_t M, int64_t N, int64_t inner, const uint16_t *A,
                                                       int64_t lda, const uint16_t *B, int64_t ldb,
                                                       double scale_sq, double *sum, double *sq, void *stream,
                                                       const char **error)
{
    // messages are string literals: reporting an error allocates nothing either
    const char *dummy = nullptr;
    const char *&msg = error ? *error : dummy;
    if (M <= 0 || N <= 0 || inner <= 0 || !A || !B || !sum || !sq || lda < inner || ldb < inner) {
        msg = "bad arguments (need M, N, inner > 0, lda, ldb >= inner, non-NULL pointers)";
        return MCINV_E_ARG;
    }
    if (M * N > kMaxProduct) {
        msg = "M * N exceeds the fixed product buffer of 2^21 FP32 elements (8 MiB)";
        return MCINV_E_ARG;
    }
    if (M > (1LL << 31) || N > (1LL << 31) || (lda % 8) || (ldb % 8) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) {
        msg = "operands must start on 16-byte boundaries with lda, ldb multiples of 8";
        return MCINV_E_ARG;
    }
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess || major != 10 || minor != 3) {
        msg = "the tensor-core contraction is built for sm_103a only";
        return MCINV_E_UNSUPPORTED;
    }
    unsigned char *scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) {
        msg = "cudaGetSymbolAddress of the fixed product buffer failed";
        return MCINV_E_CUDA;
    }
    float *D = (float *)scratch;
    int *status = (int *)(scratch + kStatusOffset);
    cudaStream_t s = (cudaStream_t)stream;
    // the product is overwritten whole by the contraction; only the status word
    // must start at zero
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
        msg = "cudaMemsetAsync of the status word failed";
        return MCINV_E_CUDA;
    }
    const char *why = "";
    e = mcinv::tc_gemm_run_direct(A, lda, B, ldb, M, N, inner, D, status, s, &why);
    if (e != cudaSuccess) {
        msg = (why && *why) ? why : "tensor-core contraction launch failed";
        return e == cudaErrorNotSupported ? MCINV_E_UNSUPPORTED : MCINV_E_CUDA;
    }
    long long blocks = (M * N + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    guarded_fold_kernel<<<(unsigned)blocks, 256, 0, s>>>(M * N, scale_sq, D, sum, sq, status);
    if (cudaGetLastError() != cudaSuccess) {
        msg = "fold launch failed";
        return MCINV_E_CUDA;
    }
    int st = 0;
    if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        msg = "CUDA error while running the contraction";
        return MCINV_E_CUDA;
    }
    if (st) {
        msg = "a bounded wait in the tensor-core contraction expired (sum and sq were left unchanged)";
        return MCINV_E_TIMEOUT;
    }
    msg = "";
    return MCINV_OK;
}

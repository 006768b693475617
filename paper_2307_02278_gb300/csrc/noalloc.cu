// Tridiagonal Gauss quadrature that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc/cudaFree: their device
// memory is owned by another allocator (a framework's caching allocator, a
// pool registered with a communication library), or they cannot afford the
// device-wide synchronisation that cudaMalloc/cudaFree imply.  This entry
// point gives them the quadrature of mbd_tridiag_quadrature with caller-owned
// device inputs and outputs; the little scratch it needs (the coefficients in
// probe-innermost order, the Krylov lengths, a status word and the flags of
// probes handed to QL) lives in one
// file-scope device array that every GPU loading the library holds until the
// process exits.
#include "mbd_internal.cuh"

#include <mutex>

namespace mbd {
namespace {

constexpr int kNoAllocMaxProbes = MBD_NOALLOC_MAX_PROBES;
constexpr size_t kCoefBytes = sizeof(double) * (size_t)kMaxSteps * kNoAllocMaxProbes;   // 1 MiB
constexpr size_t kScratchBytes = 2 * kCoefBytes + 2 * sizeof(int) * kNoAllocMaxProbes + 256;

// [a^T: m x R doubles][b^T: m x R doubles][length: R ints][status: int, padded][fallback: R ints]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// [R][m] -> [m][R], the Krylov length of each probe (the first zero coupling
// ends the tridiagonal), and the status word reset for this call.
__global__ void k_noalloc_prepare(const double *__restrict__ a, const double *__restrict__ b, int R, int m,
                                  double *__restrict__ at, double *__restrict__ bt, int *__restrict__ length,
                                  int *__restrict__ status) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) *status = 0;
    if (r >= R) return;
    int n = m;
    for (int k = 0; k < m; ++k) {
        at[(size_t)k * R + r] = a[(size_t)r * m + k];
        const double bv = b[(size_t)r * m + k];
        bt[(size_t)k * R + r] = bv;
        if (n == m && k < m - 1 && bv == 0.0) n = k + 1;
    }
    length[r] = n;
}

// The device address of the scratch array on the current device, looked up
// once per device (cudaGetSymbolAddress) and cached.
mbd_status scratch_address(void **out) {
    int dev = 0;
    MBD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MBD_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        MBD_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return MBD_OK;
}

}  // namespace
}  // namespace mbd

extern "C" mbd_status mbd_tridiag_quadrature_noalloc(int32_t n_probes, int32_t n_steps, const double *a_dev,
                                                     const double *b_dev, double *q_dev, void *cuda_stream) {
    using namespace mbd;
    if (!a_dev || !b_dev || !q_dev) return MBD_ERR_INVALID_ARG;
    if (n_probes < 1 || n_probes > kNoAllocMaxProbes || n_steps < 1 || n_steps > kMaxSteps)
        return MBD_ERR_INVALID_ARG;
    void *base = nullptr;
    MBD_TRY(scratch_address(&base));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *p = static_cast<unsigned char *>(base);
    double *at = reinterpret_cast<double *>(p);
    double *bt = reinterpret_cast<double *>(p + kCoefBytes);
    int *length = reinterpret_cast<int *>(p + 2 * kCoefBytes);
    int *status = reinterpret_cast<int *>(p + 2 * kCoefBytes + sizeof(int) * kNoAllocMaxProbes);
    int *fallback = reinterpret_cast<int *>(p + 2 * kCoefBytes + sizeof(int) * kNoAllocMaxProbes + 256);
    k_noalloc_prepare<<<(n_probes + 127) / 128, 128, 0, st>>>(a_dev, b_dev, n_probes, n_steps, at, bt, length,
                                                             status);
    MBD_LAUNCH_CHECK();
    MBD_TRY(launch_quadrature(at, bt, length, n_probes, n_probes, n_steps, q_dev, nullptr, status, fallback, st,
                              MBD_QUAD_CHEBYSHEV));
    int bits = 0;
    MBD_CUDA_TRY(cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    MBD_CUDA_TRY(cudaStreamSynchronize(st));
    if (bits & 1) return MBD_ERR_NOT_POSITIVE_DEFINITE;
    if (bits & 6) return MBD_ERR_NONFINITE;
    return MBD_OK;
}

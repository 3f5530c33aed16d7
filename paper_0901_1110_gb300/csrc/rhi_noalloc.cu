// Allocation-free RMS norm: the block-partial reduction of the residual norm with its scratch
// in a file-scope device array instead of memory from cudaMalloc.
//
// Callers that may not allocate device memory (code running while a CUDA stream is being
// captured into a graph, where cudaMalloc is not allowed, or a host application that owns all
// device memory through its own pool) can still evaluate the convergence measure of a
// residual they hold.  The scratch below is reserved on every GPU that loads the library, for
// the life of the process.
#include <mutex>

#include "rhi_internal.cuh"

namespace {

constexpr int NA_BLOCK = 256;
constexpr long long NA_MAX_PARTIALS = RHI_NOALLOC_MAX_COUNT / NA_BLOCK;

// one partial sum per block of the first kernel (the result goes to the caller's `out`)
static __device__ __align__(256) double na_scratch[NA_MAX_PARTIALS];

__global__ void __launch_bounds__(NA_BLOCK) k_na_partials(const double* __restrict__ v, long long n,
                                                          double* __restrict__ part) {
    const long long i = blockIdx.x * (long long)NA_BLOCK + threadIdx.x;
    double x = (i < n) ? v[i] : 0.0;
    const double s = rhi::block_sum<NA_BLOCK>(x * x);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

constexpr int NA_RED = 1024;
__global__ void __launch_bounds__(NA_RED) k_na_finish(const double* __restrict__ part, int np,
                                                      double inv_count, double* __restrict__ out) {
    double acc = 0.0;
    for (int q = threadIdx.x; q < np; q += NA_RED) acc += part[q];
    const double s = rhi::block_sum<NA_RED>(acc);
    if (threadIdx.x == 0) out[0] = sqrt(s * inv_count);
}

// device address of the scratch, looked up once per device with that device current
constexpr int NA_MAX_DEVICES = 64;
double* na_addr[NA_MAX_DEVICES] = {nullptr};
std::mutex na_mutex;

}  // namespace

extern "C" int rhi_rms_norm_noalloc(const double* v, long long n, long long count,
                                    double* out, void* stream) {
    if (!v || !out || n < 1 || count < 1) return RHI_ERR_ARG;
    if (n > RHI_NOALLOC_MAX_COUNT) return RHI_ERR_ARG;       // scratch holds n / 256 partials
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return RHI_ERR_CUDA;
    double* part = nullptr;
    {
        std::lock_guard<std::mutex> lock(na_mutex);
        if (!na_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) return RHI_ERR_CUDA;
            na_addr[dev] = (double*)p;
        }
        part = na_addr[dev];
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const long long nb = (n + NA_BLOCK - 1) / NA_BLOCK;      // <= NA_MAX_PARTIALS
    // a launch error left pending by earlier work of this host thread is cleared here, so that
    // each launch below is judged on its own status
    (void)cudaGetLastError();
    k_na_partials<<<(unsigned)nb, NA_BLOCK, 0, st>>>(v, n, part);
    if (cudaGetLastError() != cudaSuccess) return RHI_ERR_CUDA;
    k_na_finish<<<1, NA_RED, 0, st>>>(part, (int)nb, 1.0 / (double)count, out);
    if (cudaGetLastError() != cudaSuccess) return RHI_ERR_CUDA;
    return RHI_OK;
}

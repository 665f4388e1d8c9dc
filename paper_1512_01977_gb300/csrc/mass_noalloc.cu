// Allocation-free variant of the FP64 mass reduction (kernel (c)).
//
// Some callers cannot let a library allocate device memory on their behalf:
// a serving loop that runs out of a fixed, pre-reserved arena, or a framework
// whose caching allocator must see every device byte.  For them this file
// keeps the reduction's per-block partial sums in a file-scope static device
// array (64 KB, held by every GPU that loads the library until the process
// exits) instead of memory the library would allocate; the caller passes the
// density field and the output buffer.
#include <mutex>

#include "lbm_axi.h"
#include "lbm_kernels.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 8;
constexpr int kNodesPerBlock = kThreads * kNodesPerThread;
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_NODES / kNodesPerBlock;
static_assert(LBM_NOALLOC_MAX_NODES % kNodesPerBlock == 0, "whole blocks");

// Per-block partials (sum (j + 1/2) rho, sum rho); every call overwrites the
// slots of the blocks it launches and reads only those.
static __device__ __align__(256) double g_mass_partials[2 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_partials_addr[kMaxDevices] = {};

// Device address of the static array on the current device (the host-side
// name of the array is only a stand-in and must not be passed to a kernel).
int partials_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        g_partials_addr[dev] = p;
    }
    *out = static_cast<double*>(g_partials_addr[dev]);
    return LBM_OK;
}

// One partial pair per block of kNodesPerBlock consecutive nodes (index j*nz + k).
__global__ void __launch_bounds__(kThreads) k_mass_partials(const double* __restrict__ rho, int nz, long long n,
                                                            double* __restrict__ partial) {
    double v[2] = {0.0, 0.0};
    const long long base = (long long)blockIdx.x * kNodesPerBlock;
#pragma unroll
    for (int q = 0; q < kNodesPerThread; q++) {
        const long long c = base + (long long)q * kThreads + threadIdx.x;
        if (c < n) {
            const int j = (int)(c / nz);
            const double r = rho[c];
            v[0] += (j + 0.5) * r;
            v[1] += r;
        }
    }
    lbm::block_sum<2>(v, partial + 2 * blockIdx.x);
}

}  // namespace

extern "C" int lbm_axi_mass_field_noalloc(const double* d_rho, int nz, int nr, double* d_out, void* stream) {
    if (!d_rho || !d_out || nz < 1 || nr < 1) return LBM_ERR_INVALID_ARG;
    const long long n = (long long)nz * nr;
    if (n > LBM_NOALLOC_MAX_NODES) return LBM_ERR_INVALID_ARG;
    double* partial = nullptr;
    const int rc = partials_address(&partial);
    if (rc != LBM_OK) return rc;
    const int blocks = (int)((n + kNodesPerBlock - 1) / kNodesPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_mass_partials<<<blocks, kThreads, 0, s>>>(d_rho, nz, n, partial);
    lbm::k_reduce_final<2><<<1, 32, 0, s>>>(partial, blocks, d_out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

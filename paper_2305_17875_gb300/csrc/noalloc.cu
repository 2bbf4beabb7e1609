// noalloc.cu - the right-hand-side projection without any allocation.
//
// Some callers cannot allocate device memory at the moment they need this
// step: time-step loops that must not stall on the allocator (cudaMalloc can
// synchronise the device and takes driver locks), and host programs whose
// device memory is owned by another pool (a simulation that reserved most of
// the GPU for its own fields up front, or a framework's caching allocator
// that must see every byte).  For them this file computes b = J (f - mean_J f)
// with its reduction scratch in a fixed static device array instead of
// allocated memory.
//
// The array is file-scope and every GPU that loads the library holds it until
// the process exits.  All calls share it and it keeps the last call's
// partial sums; each call overwrites every entry it reads before reading it,
// so nothing has to start at zero.  Calls that overlap on the GPU (different
// streams, or host threads without ordering) race on the array.
//
// Host code cannot hand the array's name to a kernel (in host code it is a
// stand-in, not a device address): its device address is looked up with
// cudaGetSymbolAddress on the first call on each device, with that device
// current, and kept per device index.  The cache is keyed by the device
// index, not by the context: a caller that drives a device through a context
// other than its primary one gets the primary context's address, and after a
// cudaDeviceReset the cached address is stale (restart the process).
#include <atomic>
#include <cstdio>
#include <string>

#include "engine.h"

namespace mgs {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 16384;                                  // one partial pair per block
constexpr long long kNaMaxCells = (long long)kNaMaxBlocks * kNaThreads;  // 4,194,304 cells
constexpr int kNaSlots = 2 * kNaMaxBlocks + 8;                        // partials + result slots

// Scratch: [2 b] = sum J f, [2 b + 1] = sum J over block b; the last 8 slots
// hold the finished sums and the mean.  128 KB per GPU.
static __device__ __align__(256) double g_noalloc_scratch[kNaSlots];

__global__ void __launch_bounds__(kNaThreads) k_na_partials(const double* __restrict__ J, const double* __restrict__ f,
                                                            int n, double* scratch) {
    __shared__ double sh[8];
    const int c = blockIdx.x * kNaThreads + threadIdx.x;
    double jf = 0.0, jj = 0.0;
    if (c < n) {
        jf = J[c] * f[c];
        jj = J[c];
    }
    const double s1 = block_sum_256(jf, sh);
    const double s2 = block_sum_256(jj, sh);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = s1;
        scratch[2 * blockIdx.x + 1] = s2;
    }
}

// One block: the partials in a fixed order, then mean = sum J f / sum J.
__global__ void __launch_bounds__(kNaThreads) k_na_mean(int nblocks, double* scratch, double* mean_out) {
    __shared__ double sh[8];
    double a = 0.0, b = 0.0;
    for (int p = threadIdx.x; p < nblocks; p += kNaThreads) {
        a += scratch[2 * p];
        b += scratch[2 * p + 1];
    }
    const double sa = block_sum_256(a, sh);
    const double sb = block_sum_256(b, sh);
    if (threadIdx.x == 0) {
        const double mean = sa / sb;
        scratch[2 * kNaMaxBlocks + 0] = sa;
        scratch[2 * kNaMaxBlocks + 1] = sb;
        scratch[2 * kNaMaxBlocks + 2] = mean;
        if (mean_out) *mean_out = mean;
    }
}

__global__ void __launch_bounds__(kNaThreads) k_na_project(const double* __restrict__ J, const double* __restrict__ f,
                                                           double* __restrict__ b, int n, const double* scratch) {
    const double mean = scratch[2 * kNaMaxBlocks + 2];
    const int c = blockIdx.x * kNaThreads + threadIdx.x;
    if (c < n) b[c] = J[c] * (f[c] - mean);
}

// Device address of the scratch array, looked up once per device (host
// threads may race on the first lookup: both find the same address).
constexpr int kNaMaxDevices = 64;
std::atomic<double*> g_scratch_ptr[kNaMaxDevices] = {};

mg_status scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("device index out of range for the static scratch table");
        return MG_EINVAL;
    }
    double* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void* q = nullptr;
        e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return MG_ECUDA;
        }
        p = (double*)q;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return MG_OK;
}

// A caller array must be device memory of the current device: the kernels
// run there (cudaPointerGetAttributes allocates nothing).
mg_status check_on_device(const void* ptr, int dev, const char* name) {
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("mg_project_rhs_noalloc: ") + name + " is not a CUDA pointer");
        return MG_EINVAL;
    }
    const bool device_mem = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    if (!device_mem || (a.type == cudaMemoryTypeDevice && a.device != dev)) {
        set_error(std::string("mg_project_rhs_noalloc: ") + name + " is not memory of the current device " +
                  std::to_string(dev));
        return MG_EINVAL;
    }
    return MG_OK;
}

}  // namespace
}  // namespace mgs

extern "C" mg_status mg_project_rhs_noalloc(const double* J_dev, const double* f_dev, double* b_dev,
                                            long long n, void* cuda_stream, double* mean_dev) {
    using namespace mgs;
    if (!J_dev || !f_dev || !b_dev || n < 1) {
        set_error("mg_project_rhs_noalloc: null pointer or empty grid");
        return MG_EINVAL;
    }
    if (n > kNaMaxCells) {
        set_error("mg_project_rhs_noalloc: " + std::to_string(n) + " cells exceed the static scratch limit of " +
                  std::to_string(kNaMaxCells) + " cells");
        return MG_EINVAL;
    }
    double* scratch = nullptr;
    mg_status st = scratch_for_current_device(&scratch);
    if (st != MG_OK) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    if ((st = check_on_device(J_dev, dev, "J")) != MG_OK || (st = check_on_device(f_dev, dev, "f")) != MG_OK ||
        (st = check_on_device(b_dev, dev, "b")) != MG_OK ||
        (mean_dev && (st = check_on_device(mean_dev, dev, "mean")) != MG_OK))
        return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (int)((n + kNaThreads - 1) / kNaThreads);
    k_na_partials<<<nb, kNaThreads, 0, s>>>(J_dev, f_dev, (int)n, scratch);
    k_na_mean<<<1, kNaThreads, 0, s>>>(nb, scratch, mean_dev);
    k_na_project<<<nb, kNaThreads, 0, s>>>(J_dev, f_dev, b_dev, (int)n, scratch);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("mg_project_rhs_noalloc: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    return MG_OK;
}

// outer.cu - deterministic FP64 reductions used at set-up and by the
// component entry points: sums (J-weighted means, Eq. volumeavg), maxima and
// the fixed-order finalisation of block partials.  The outer-iteration steps
// themselves run as batched operations (batch.cu).
#include "mg_kernels.h"

namespace mgs {

namespace {

constexpr int kT = 256;

#define GRID_STRIDE(var, n) \
    for (i64 var = blockIdx.x * (i64)blockDim.x + threadIdx.x; var < (n); var += (i64)gridDim.x * blockDim.x)

__global__ void __launch_bounds__(kT) k_sum(const double* __restrict__ a, const double* __restrict__ w, i64 n,
                                             double* __restrict__ partials) {
    __shared__ double sh[8];
    double acc = 0.0;
    GRID_STRIDE(c, n) acc += w ? a[c] * w[c] : a[c];
    const double s = block_sum_256(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kT) k_absmax(const double* __restrict__ a, i64 n, double* __restrict__ partials) {
    __shared__ double sh[8];
    double m = 0.0;
    GRID_STRIDE(c, n) m = fmax(m, fabs(a[c]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < kT / 32; ++w) r = fmax(r, sh[w]);
        partials[blockIdx.x] = r;
    }
}

// 2^-round(log2(rms)) for rms = sqrt(sum / n): exact power of two.
__device__ double unit_scale(double sum, i64 n) {
    const double rms = sqrt(sum / (double)n);
    if (!(rms > 0.0) || !isfinite(rms)) return 1.0;
    return ldexp(1.0, -(int)lround(log2(rms)));
}

// FIN_SUM / FIN_SCALE: sum, FIN_MAX: max.  One block; fixed order.
__global__ void k_finalize(const double* __restrict__ partials, int np, int op, double* __restrict__ out,
                           double* __restrict__ scal, i64 n) {
    __shared__ double sh[8];
    double v = 0.0;
    const bool mx = op == FIN_MAX;
    for (int p = threadIdx.x; p < np; p += blockDim.x) v = mx ? fmax(v, partials[p]) : v + partials[p];
    if (mx) {
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double r = 0.0;
            for (int w = 0; w < kT / 32; ++w) r = fmax(r, sh[w]);
            out[0] = r;
        }
    } else {
        const double s = block_sum_256(v, sh);
        if (threadIdx.x == 0) {
            out[0] = s;
            if (op == FIN_SCALE) scal[SC_SCUR] = unit_scale(s, n);
        }
    }
}

}  // namespace

int red_blocks(i64 n) {
    i64 b = (n + kT - 1) / kT;
    if (b > kRedBlocks) b = kRedBlocks;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_sum(const double* a, const double* w, i64 n, double* partials, cudaStream_t s) {
    k_sum<<<red_blocks(n), kT, 0, s>>>(a, w, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const double* a, i64 n, double* partials, cudaStream_t s) {
    k_absmax<<<red_blocks(n), kT, 0, s>>>(a, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nparts, int op, double* out, cudaStream_t s,
                            double* scal, i64 n) {
    k_finalize<<<1, kT, 0, s>>>(partials, nparts, op, out, scal, n);
    return cudaGetLastError();
}

}  // namespace mgs

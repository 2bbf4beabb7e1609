// outer.cu - FP64 outer-iteration kernels and deterministic reductions:
// the right side b = |J^{-1}| (f - mean_J f) of Eq. PC_6, the outer residual
// r = b - A x with its norm and FP32 cast, the solution update and the
// J-weighted gauge (discrete volume average, Eq. volumeavg).
#include "mg_kernels.h"

namespace mgs {

namespace {

constexpr int kT = 256;

#define GRID_STRIDE(var, n) \
    for (i64 var = blockIdx.x * (i64)blockDim.x + threadIdx.x; var < (n); var += (i64)gridDim.x * blockDim.x)

template <int S>
__global__ void __launch_bounds__(kT) k_outer_residual(CoefF64 cf, Dims D, const double* __restrict__ x,
                                                        const double* __restrict__ b, float* __restrict__ r32,
                                                        double* scal, double* __restrict__ partials) {
    __shared__ double sh[8];
    XRead<double> X{x, D};
    const double scale = r32 ? scal[SC_SCUR] : 1.0;
    if (r32 && blockIdx.x == 0 && threadIdx.x == 0) scal[SC_SUSED] = scale;
    double acc = 0.0;
    GRID_STRIDE(c, D.n()) {
        const double r = b[c] - apply_cell<S, double>(cf, X, D, decode(D, c));
        if (r32) r32[c] = (float)(r * scale);
        acc = fma(r, r, acc);
    }
    const double s = block_sum_256(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

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

__global__ void __launch_bounds__(kT) k_update(double* __restrict__ x, const float* __restrict__ e,
                                                const double* __restrict__ scal, i64 n) {
    const double inv = 1.0 / scal[SC_SUSED];   // exact: a power of two
    GRID_STRIDE(c, n) x[c] = fma((double)e[c], inv, x[c]);
}

__global__ void __launch_bounds__(kT) k_rhs(const double* __restrict__ J, const double* __restrict__ f,
                                             const double* __restrict__ num, double den, double* __restrict__ b,
                                             i64 n, double* __restrict__ partials) {
    __shared__ double sh[8];
    const double mean = num[0] / den;
    double acc = 0.0;
    GRID_STRIDE(c, n) {
        const double v = J[c] * (f[c] - mean);
        b[c] = v;
        acc = fma(v, v, acc);
    }
    const double s = block_sum_256(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kT) k_shift(double* __restrict__ x, const double* __restrict__ num, double den, i64 n) {
    const double m = num[0] / den;
    GRID_STRIDE(c, n) x[c] -= m;
}

}  // namespace

int red_blocks(i64 n) {
    i64 b = (n + kT - 1) / kT;
    if (b > kRedBlocks) b = kRedBlocks;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_outer_residual(const LevelView& lv, const double* x, const double* b, float* r32,
                                  double* scal, double* partials, cudaStream_t s) {
    const int nb = red_blocks(lv.D.n());
    if (lv.stencil == 19)
        k_outer_residual<19><<<nb, kT, 0, s>>>(lv.c64, lv.D, x, b, r32, scal, partials);
    else
        k_outer_residual<7><<<nb, kT, 0, s>>>(lv.c64, lv.D, x, b, r32, scal, partials);
    return cudaGetLastError();
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

cudaError_t launch_update(double* x, const float* e, const double* scal, i64 n, cudaStream_t s) {
    i64 nb = (n + kT - 1) / kT;
    if (nb > 152 * 16) nb = 152 * 16;
    k_update<<<(int)nb, kT, 0, s>>>(x, e, scal, n);
    return cudaGetLastError();
}

cudaError_t launch_rhs(const double* J, const double* f, const double* num, double den, double* b,
                       i64 n, double* partials, cudaStream_t s) {
    k_rhs<<<red_blocks(n), kT, 0, s>>>(J, f, num, den, b, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_shift(double* x, const double* num, double den, i64 n, cudaStream_t s) {
    i64 nb = (n + kT - 1) / kT;
    if (nb > 152 * 16) nb = 152 * 16;
    k_shift<<<(int)nb, kT, 0, s>>>(x, num, den, n);
    return cudaGetLastError();
}

}  // namespace mgs

// stencil.cu - multigrid level operations on the conservative shell operator
// (Section 3.3, Eqs. PC_term1-3): apply, multicolour Gauss-Seidel, weighted
// Jacobi, fused residual + restriction, trilinear prolongation + correction,
// and the coarsest-level dense solve.
#include "mg_kernels.h"

namespace mgs {

namespace {

constexpr int kThreads = 256;

int blocks_for(i64 work) {
    i64 b = (work + kThreads - 1) / kThreads;
    const i64 cap = 152 * 16;   // grid-stride beyond 16 resident blocks per SM
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ C3 decode(const Dims& D, i64 c) {
    C3 r;
    r.k = (int)(c % D.nph);
    const i64 ji = c / D.nph;
    r.i = (int)(ji % D.nth);
    r.j = (int)(ji / D.nth);
    return r;
}

#define GRID_STRIDE(var, n) \
    for (i64 var = blockIdx.x * (i64)blockDim.x + threadIdx.x; var < (n); var += (i64)gridDim.x * blockDim.x)

template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_apply(CF cf, Dims D, const T* __restrict__ x, T* __restrict__ y) {
    XRead<T> X{x, D};
    GRID_STRIDE(c, D.n()) { y[c] = apply_cell<S, T>(cf, X, D, decode(D, c)); }
}

// One colour of multicolour Gauss-Seidel, in place: x_c += (b_c - (A x)_c) / A_cc
// for every cell of the colour.  Cells of one colour share no stencil entry, so
// the pass equals the sequential sweep over that colour.
// 7-point: colour (i + j + k) mod 2.  19-point: ((i + j) mod 2) + 2 ((j + k) mod 2).
template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_gs(CF cf, Dims D, T* x, const T* __restrict__ b, int colour) {
    XRead<T> X{x, D};
    const int hk = D.nph >> 1;
    const i64 work = (i64)D.nr * D.nth * hk;
    GRID_STRIDE(t, work) {
        const int kk = (int)(t % hk);
        const i64 row = t / hk;
        const int i = (int)(row % D.nth);
        const int j = (int)(row / D.nth);
        int k;
        if (S == 7) {
            k = 2 * kk + ((colour + i + j) & 1);
        } else {
            if (((i + j) & 1) != (colour & 1)) continue;
            k = 2 * kk + (((colour >> 1) + j) & 1);
        }
        const C3 c{j, i, k};
        const i64 id = cidx(D, c);
        const T r = b[id] - apply_cell<S, T>(cf, X, D, c);
        x[id] += r / diag_cell<S, T>(cf, D, c);
    }
}

// Weighted Jacobi, out of place: xo = x + omega (b - A x) / diag(A).
template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_jacobi(CF cf, Dims D, const T* __restrict__ x, T* __restrict__ xo,
                                                      const T* __restrict__ b, T omega) {
    XRead<T> X{x, D};
    GRID_STRIDE(c, D.n()) {
        const C3 cc = decode(D, c);
        const T r = b[c] - apply_cell<S, T>(cf, X, D, cc);
        xo[c] = x[c] + omega * r / diag_cell<S, T>(cf, D, cc);
    }
}

// rc(C) = sum over the children c of C of (b - A x)_c; optionally zero ec.
template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_restrict(CF cf, Dims D, const T* __restrict__ x, const T* __restrict__ b,
                                                        Dims Dc, int cz, int ce, int cx, T* __restrict__ rc,
                                                        T* __restrict__ ec_zero) {
    XRead<T> X{x, D};
    GRID_STRIDE(t, Dc.n()) {
        const C3 C = decode(Dc, t);
        T s = 0;
        for (int dj = 0; dj < ce; ++dj)
            for (int di = 0; di < cz; ++di)
                for (int dk = 0; dk < cx; ++dk) {
                    const C3 c{ce * C.j + dj, cz * C.i + di, cx * C.k + dk};
                    s += b[cidx(D, c)] - apply_cell<S, T>(cf, X, D, c);
                }
        rc[t] = s;
        if (ec_zero) ec_zero[t] = 0;
    }
}

// 1-D cell-centred linear weights of fine cell f from a grid halved by c:
// child s of coarse cell C sits at C + (2s - 1)/4, so it takes 3/4 of C and
// 1/4 of C -/+ 1 (the mirror C itself at a wall, wrapped when periodic).
__device__ __forceinline__ void lin1d(int f, int c, int nc, bool periodic, int idx[2], float w[2]) {
    if (c == 1) {
        idx[0] = idx[1] = f;
        w[0] = 1.0f;
        w[1] = 0.0f;
        return;
    }
    const int C = f >> 1;
    int nb = (f & 1) ? C + 1 : C - 1;
    if (periodic) nb = nb < 0 ? nb + nc : (nb >= nc ? nb - nc : nb);
    else if (nb < 0 || nb >= nc) nb = C;
    idx[0] = C;
    idx[1] = nb;
    w[0] = 0.75f;
    w[1] = 0.25f;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_prolong(Dims D, Dims Dc, int cz, int ce, int cx, const T* __restrict__ ec,
                                                       T* __restrict__ x) {
    GRID_STRIDE(c, D.n()) {
        const C3 f = decode(D, c);
        int ij[2], ii[2], ik[2];
        float wj[2], wi[2], wk[2];
        lin1d(f.j, ce, Dc.nr, false, ij, wj);
        lin1d(f.i, cz, Dc.nth, false, ii, wi);
        lin1d(f.k, cx, Dc.nph, true, ik, wk);
        T s = 0;
        for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb)
                for (int e = 0; e < 2; ++e) {
                    const T w = (T)wj[a] * (T)wi[bb] * (T)wk[e];
                    if (w != (T)0) s += w * ec[cidx(Dc, ij[a], ii[bb], ik[e])];
                }
        x[c] += s;
    }
}

// e = Binv r (FP64 accumulate), one warp per row.
template <typename T>
__global__ void k_coarse(const double* __restrict__ binv, int n, const T* __restrict__ r, T* __restrict__ e) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += warps) {
        double s = 0.0;
        for (int m = lane; m < n; m += 32) s += binv[(i64)row * n + m] * (double)r[m];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) e[row] = (T)s;
    }
}

}  // namespace

// Dispatch on (precision, stencil): T = value type, cf = coefficient reader.
#define MG_DISPATCH(lv, prec, ...)                                           \
    do {                                                                     \
        if ((prec) == PREC64) {                                              \
            typedef double T;                                                \
            const CoefF64& cf = (lv).c64;                                    \
            if ((lv).stencil == 19) { constexpr int S = 19; __VA_ARGS__; }   \
            else { constexpr int S = 7; __VA_ARGS__; }                       \
        } else if ((prec) == PREC32) {                                       \
            typedef float T;                                                 \
            const CoefF32& cf = (lv).c32;                                    \
            if ((lv).stencil == 19) { constexpr int S = 19; __VA_ARGS__; }   \
            else { constexpr int S = 7; __VA_ARGS__; }                       \
        } else {                                                             \
            typedef float T;                                                 \
            const CoefF16& cf = (lv).c16;                                    \
            if ((lv).stencil == 19) { constexpr int S = 19; __VA_ARGS__; }   \
            else { constexpr int S = 7; __VA_ARGS__; }                       \
        }                                                                    \
    } while (0)

cudaError_t launch_apply(const LevelView& lv, int prec, const void* x, void* y, cudaStream_t s) {
    const int nb = blocks_for(lv.D.n());
    MG_DISPATCH(lv, prec, (k_apply<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (const T*)x, (T*)y)));
    return cudaGetLastError();
}

cudaError_t launch_gs_colour(const LevelView& lv, int prec, void* x, const void* b, int colour,
                             cudaStream_t s) {
    const int nb = blocks_for((i64)lv.D.nr * lv.D.nth * (lv.D.nph / 2));
    MG_DISPATCH(lv, prec, (k_gs<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (T*)x, (const T*)b, colour)));
    return cudaGetLastError();
}

cudaError_t launch_jacobi(const LevelView& lv, int prec, const void* x, void* xo, const void* b,
                          cudaStream_t s) {
    const int nb = blocks_for(lv.D.n());
    const double omega = lv.stencil == 7 ? 6.0 / 7.0 : 4.0 / 5.0;
    MG_DISPATCH(lv, prec, (k_jacobi<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (const T*)x, (T*)xo,
                                                                  (const T*)b, (T)omega)));
    return cudaGetLastError();
}

cudaError_t launch_restrict_residual(const LevelView& lv, Dims Dc, int prec, const void* x,
                                     const void* b, void* rc, void* ec_zero, cudaStream_t s) {
    const int nb = blocks_for(Dc.n());
    MG_DISPATCH(lv, prec, (k_restrict<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (const T*)x, (const T*)b, Dc,
                                                                    lv.cz, lv.ce, lv.cx, (T*)rc, (T*)ec_zero)));
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const LevelView& lv, Dims Dc, int prec, const void* ec, void* x,
                               cudaStream_t s) {
    const int nb = blocks_for(lv.D.n());
    if (prec == PREC64)
        k_prolong<double><<<nb, kThreads, 0, s>>>(lv.D, Dc, lv.cz, lv.ce, lv.cx, (const double*)ec, (double*)x);
    else
        k_prolong<float><<<nb, kThreads, 0, s>>>(lv.D, Dc, lv.cz, lv.ce, lv.cx, (const float*)ec, (float*)x);
    return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const double* binv, int n, int prec, const void* r, void* e,
                                cudaStream_t s) {
    const int rows_per_block = kThreads / 32;
    int nb = (n + rows_per_block - 1) / rows_per_block;
    if (nb > 152 * 4) nb = 152 * 4;
    if (prec == PREC64)
        k_coarse<double><<<nb, kThreads, 0, s>>>(binv, n, (const double*)r, (double*)e);
    else
        k_coarse<float><<<nb, kThreads, 0, s>>>(binv, n, (const float*)r, (float*)e);
    return cudaGetLastError();
}

}  // namespace mgs

// line_smooth.cuh - radial-line Gauss-Seidel colour pass (internal).
//
// Every radial line (fixed colatitude index i and longitude index k) is one
// block of a block Gauss-Seidel sweep: x_L += A_LL^{-1} (b - A x)_L, with
// A_LL the tridiagonal part of the level operator on the line, solved by the
// Thomas algorithm of Section 3.5.  Lines are coloured so that no two lines
// of a colour are coupled: 7 points (i + k) mod 2, 19 points (i mod 2) +
// 2 (k mod 2) (the 19-point operator couples a line with its eight
// neighbours in the (i, k) plane); a sweep runs the colours in order.
//
// A_LL is fixed per level, so its factorisation is made once at set-up and
// stored per cell as the coefficients of two first-order recurrences:
//   forward   d_j = beta_j r_j + alpha_j d_{j-1}   (beta = 1/b'_j, alpha = -a_j/b'_j)
//   backward  e_j = d_j + gamma_j e_{j+1}          (gamma = -c_j/b'_j)
// with b'_j the pivots of the elimination; x_j += e_j.
//
// One line is split into W chunks of at most kC rows, one thread per chunk
// (warps hold the same chunk of consecutive lines, so loads coalesce across
// lines).  Each thread runs both recurrences on its chunk from a zero start
// in registers and publishes the chunk's affine map (value leaving = P * value
// entering + Q); the value entering each chunk is the composition of the
// maps before it (at most W - 1 steps through shared memory), and a last pass
// over the registers adds P_j times it.  Same recurrences as the sequential
// sweep, regrouped, so the results agree up to rounding.
#pragma once

#include "mg_internal.cuh"

namespace mgs {

template <typename T>
struct LineRows {
    static constexpr int kC = 16;   // rows of a chunk held in registers
};

// Chunks per line: the smallest power of two W with W * kC >= nr (W <= 16
// keeps at least 16 lines in a block of 256 threads).
__host__ __device__ inline int line_chunks(int nr, int kC) {
    int w = 1;
    while (w * kC < nr) w <<= 1;
    return w;
}

// Radial lines of colour `colour` on a level.
__host__ __device__ inline i64 line_count(const Dims& D, int stencil, int colour) {
    const i64 hk = D.nph >> 1;
    if (stencil == 7) return (i64)D.nth * hk;
    return (i64)((D.nth + 1 - (colour & 1)) >> 1) * hk;
}

template <int S, typename T, typename CF>
__device__ __forceinline__ T line_residual(const CF& cf, const Dims& D, const T* x, const T* b, int j, int i,
                                           int k) {
    if constexpr (S == 7) {
        Cell7<T> q;
        q.load(cf, D, j, i, k, XLin<T>{x});
        return q.resid(b[q.c]);
    } else {
        const C3 p{j, i, k};
        const int c = cidx(D, p);
        Nbr19<T> X;
        X.load(XLin<T>{x}, D, c, p, !cf.has(2));
        return b[c] - apply19<T>(cf, X, D, c, p);
    }
}

// One colour pass on the lines of virtual blocks lb, lb + nblocks, ...
// (blockDim.x = 256; every thread of the block takes part).  fac holds alpha,
// beta, gamma as three arrays of n cells.
template <int S, typename T, typename CF>
__device__ __forceinline__ void line_pass(const CF& cf, const Dims& D, T* x, const T* b, const T* fac,
                                          int colour, int lb, int nblocks) {
    constexpr int kC = LineRows<T>::kC;
    __shared__ T sP[256], sQ[256];
    const int W = line_chunks(D.nr, kC);
    const int LB = 256 / W;
    const int w = threadIdx.x / LB, l = threadIdx.x - w * LB;
    const int rows = (D.nr + W - 1) / W;
    const int j0 = min(w * rows, D.nr), nj = min(j0 + rows, D.nr) - j0;
    const int hk = D.nph >> 1;
    const i64 lines = line_count(D, S, colour);
    const i64 groups = (lines + LB - 1) / LB;
    const i64 N = D.n();
    const int plane = D.nth * D.nph;
    const T* alpha = fac;
    const T* beta = fac + N;
    const T* gamma = fac + 2 * N;
    for (i64 g = lb; g < groups; g += nblocks) {
        const i64 t = g * LB + l;
        const int n = t < lines ? nj : 0;   // rows this thread works on
        int i = 0, k = 0;
        if (n > 0) {
            const unsigned row = D.dhk.div((unsigned)t);
            const int kk = (int)((unsigned)t - row * (unsigned)hk);
            if (S == 7) {
                i = (int)row;
                k = 2 * kk + ((colour + i) & 1);
            } else {
                i = 2 * (int)row + (colour & 1);
                k = 2 * kk + (colour >> 1);
            }
        }
        const int c0 = (j0 * D.nth + i) * D.nph + k;
        T d[kC], P[kC];
        // forward recurrence on the chunk from d = 0
        T q = 0, p = 1;
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            if (u < n) {
                const int c = c0 + u * plane;
                const T r = line_residual<S, T>(cf, D, x, b, j0 + u, i, k);
                const T a = alpha[c];
                q = fma(a, q, beta[c] * r);
                p = p * a;
                d[u] = q;
                P[u] = p;
            }
        }
        sP[threadIdx.x] = p;
        sQ[threadIdx.x] = q;
        __syncthreads();
        T in = 0;
        for (int v = 0; v < w; ++v) in = fma(sP[v * LB + l], in, sQ[v * LB + l]);
        __syncthreads();
        // backward recurrence on the chunk from e = 0, on the corrected d
        q = 0;
        p = 1;
#pragma unroll
        for (int u = kC - 1; u >= 0; --u) {
            if (u < n) {
                const T gm = gamma[c0 + u * plane];
                q = fma(gm, q, fma(P[u], in, d[u]));
                p = p * gm;
                d[u] = q;
                P[u] = p;
            }
        }
        sP[threadIdx.x] = p;
        sQ[threadIdx.x] = q;
        __syncthreads();
        in = 0;
        for (int v = W - 1; v > w; --v) in = fma(sP[v * LB + l], in, sQ[v * LB + l]);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            if (u < n) {
                const int c = c0 + u * plane;
                x[c] = x[c] + fma(P[u], in, d[u]);
            }
        }
    }
}

}  // namespace mgs

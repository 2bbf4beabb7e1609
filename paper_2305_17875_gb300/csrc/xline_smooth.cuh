// xline_smooth.cuh - longitude-line Gauss-Seidel colour pass (internal).
//
// Every longitude line (fixed radius index j and colatitude index i, periodic
// in k) is one block of a block Gauss-Seidel sweep: x_L += T_L^{-1} (b - A x)_L
// with T_L the cyclic tridiagonal part of the level operator on the line,
// solved by the periodic Thomas algorithm of Section 3.5: with T_c the
// leading (n-1) x (n-1) block,
//   psi1 = T_c^{-1} r[0 .. n-2],   psi2 = T_c^{-1} (-a_0, 0, .., 0, -c_{n-2}),
//   d_{n-1} = (r_{n-1} - c_{n-1} psi1_0 - a_{n-1} psi1_{n-2})
//             / (b_{n-1} + c_{n-1} psi2_0 + a_{n-1} psi2_{n-2}),
//   d_k = psi1_k + psi2_k d_{n-1}   (k < n-1).
// Lines are coloured so that no two lines of a colour are coupled: 7 points
// (i + j) mod 2, 19 points (i mod 2) + 2 (j mod 2).
//
// T_L is fixed per level, so everything but psi1 is made at set-up
// (k_xline_factors): four arrays of n cells, alpha, beta, gamma (the
// normalised elimination of T_c: forward q_k = beta_k r_k + alpha_k q_{k-1},
// backward e_k = q_k + gamma_k e_{k+1}) and psi2; in the slot of the last
// cell of each line alpha holds c_{n-1}, gamma holds a_{n-1}, beta holds
// 1 / (b_{n-1} + c_{n-1} psi2_0 + a_{n-1} psi2_{n-2}).
//
// One thread per line, the line's residual evaluated on the fly in the
// forward recurrence (the line's own x is rewritten only at the end), the
// recurrence values kept in the level's scratch array.  Levels need at least
// four longitudes (the caller smooths narrower levels pointwise).
#pragma once

#include "line_smooth.cuh"

namespace mgs {

// Longitude lines of colour `colour` on a level (upper bound of the work
// items: rows of the colour that fall outside the grid are skipped).
__host__ __device__ inline i64 xline_items(const Dims& D, int stencil) {
    if (stencil == 7) return (i64)D.nr * ((D.nth + 1) >> 1);
    return (i64)((D.nr + 1) >> 1) * ((D.nth + 1) >> 1);
}

// Work item t of colour `colour` -> (j, i), or false when it lies outside.
__device__ __forceinline__ bool xline_of(const Dims& D, int stencil, int colour, i64 t, int& j, int& i) {
    const int h = (D.nth + 1) >> 1;
    const int row = (int)(t / h), u = (int)(t - (i64)row * h);
    if (stencil == 7) {
        j = row;
        i = 2 * u + ((colour + j) & 1);
    } else {
        j = 2 * row + (colour >> 1);
        i = 2 * u + (colour & 1);
    }
    return j < D.nr && i < D.nth;
}

template <int S, typename T, typename CF>
__device__ __forceinline__ void xline_pass(const CF& cf, const Dims& D, T* x, const T* b, const T* fac, T* work,
                                           int colour, i64 first, i64 stride) {
    const i64 N = D.n();
    const T* alpha = fac;
    const T* beta = fac + N;
    const T* gamma = fac + 2 * N;
    const T* psi2 = fac + 3 * N;
    const int n = D.nph;
    const i64 items = xline_items(D, S);
    for (i64 t = first; t < items; t += stride) {
        int j, i;
        if (!xline_of(D, S, colour, t, j, i)) continue;
        const int c0 = (j * D.nth + i) * D.nph, cl = c0 + n - 1;
        // forward recurrence of T_c on the residual
        T q = 0;
        for (int k = 0; k < n - 1; ++k) {
            const T r = line_residual<S, T>(cf, D, x, b, j, i, k);
            q = fma(alpha[c0 + k], q, beta[c0 + k] * r);
            work[c0 + k] = q;
        }
        const T rl = line_residual<S, T>(cf, D, x, b, j, i, n - 1);
        // backward recurrence: psi1
        T e = 0;
        for (int k = n - 2; k >= 0; --k) {
            e = fma(gamma[c0 + k], e, work[c0 + k]);
            work[c0 + k] = e;
        }
        // the last unknown, then the correction of the line
        const T dl = (rl - alpha[cl] * work[c0] - gamma[cl] * work[c0 + n - 2]) * beta[cl];
        for (int k = 0; k < n - 1; ++k) x[c0 + k] = x[c0 + k] + fma(psi2[c0 + k], dl, work[c0 + k]);
        x[cl] = x[cl] + dl;
    }
}

// Chunks of the leading block's rows per line for the chunked pass: W threads
// per line (a power of two, at most 16), each holding at most kC rows in
// registers; 0 when the lines are too long for it.
__host__ __device__ inline int xline_chunks(int nph, int kC) {
    const int w = line_chunks(nph - 1, kC);
    return w <= 16 ? w : 0;
}

// The same colour pass with W threads per line (blockDim.x = 256, every
// thread of the block takes part; virtual blocks lb, lb + nblocks, ...): each
// thread runs the recurrences of T_c on its chunk of rows from a zero start,
// the chunks' affine maps are composed through shared memory as in the
// radial-line pass, then the periodic closure (psi1_0 and psi1_{n-2} through
// shared memory, d_{n-1} by the line's last thread) and the correction.
template <int S, typename T, typename CF>
__device__ __forceinline__ void xline_pass_chunked(const CF& cf, const Dims& D, T* x, const T* b, const T* fac,
                                                   int colour, int lb, int nblocks) {
    constexpr int kC = LineRows<T>::kC;
    __shared__ T sP[256], sQ[256], s0[256], s1[256], sD[256];
    const i64 N = D.n();
    const T* alpha = fac;
    const T* beta = fac + N;
    const T* gamma = fac + 2 * N;
    const T* psi2 = fac + 3 * N;
    const int n = D.nph, m = n - 1;                 // rows of the leading block
    const int W = line_chunks(m, kC);
    const int LB = 256 / W;
    const int w = threadIdx.x / LB, l = threadIdx.x - w * LB;
    const int rows = (m + W - 1) / W;
    const int k0 = min(w * rows, m), nk = min(k0 + rows, m) - k0;
    const i64 lines = xline_items(D, S);
    const i64 groups = (lines + LB - 1) / LB;
    for (i64 g = lb; g < groups; g += nblocks) {
        const i64 t = g * LB + l;
        int j = 0, i = 0;
        const bool valid = t < lines && xline_of(D, S, colour, t, j, i);
        const int cnt = valid ? nk : 0;             // rows this thread works on
        const int c0 = (j * D.nth + i) * D.nph;
        const int cl = c0 + n - 1;
        T d[kC], P[kC];
        T q = 0, p = 1;
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            if (u < cnt) {
                const int k = k0 + u;
                const T r = line_residual<S, T>(cf, D, x, b, j, i, k);
                const T a = alpha[c0 + k];
                q = fma(a, q, beta[c0 + k] * r);
                p = p * a;
                d[u] = q;
                P[u] = p;
            }
        }
        T rl = 0;
        if (valid && w == W - 1) rl = line_residual<S, T>(cf, D, x, b, j, i, n - 1);
        sP[threadIdx.x] = p;
        sQ[threadIdx.x] = q;
        __syncthreads();
        T in = 0;
        for (int v = 0; v < w; ++v) in = fma(sP[v * LB + l], in, sQ[v * LB + l]);
        __syncthreads();
        q = 0;
        p = 1;
        T last = 0;   // the backward value of the chunk's last row
#pragma unroll
        for (int u = kC - 1; u >= 0; --u) {
            if (u < cnt) {
                const T gm = gamma[c0 + k0 + u];
                q = fma(gm, q, fma(P[u], in, d[u]));
                p = p * gm;
                d[u] = q;
                P[u] = p;
                if (u == cnt - 1) last = q;
            }
        }
        sP[threadIdx.x] = p;
        sQ[threadIdx.x] = q;
        __syncthreads();
        in = 0;
        for (int v = W - 1; v > w; --v) in = fma(sP[v * LB + l], in, sQ[v * LB + l]);
        // psi1 of the first and the last row of the leading block; the chunk
        // holding the last row has only empty chunks after it (in = 0), so
        // its backward value there is final
        if (cnt > 0 && k0 == 0) s0[l] = fma(P[0], in, d[0]);
        if (cnt > 0 && k0 + cnt == m) s1[l] = last;
        __syncthreads();
        if (valid && w == W - 1) {
            const T dl = (rl - alpha[cl] * s0[l] - gamma[cl] * s1[l]) * beta[cl];
            sD[l] = dl;
            x[cl] = x[cl] + dl;
        }
        __syncthreads();
        const T dl = sD[l];
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            if (u < cnt) {
                const int c = c0 + k0 + u;
                x[c] = x[c] + fma(psi2[c], dl, fma(P[u], in, d[u]));
            }
        }
    }
}

}  // namespace mgs

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

}  // namespace mgs

// plane_smooth.cuh - zebra plane relaxation of the semi-coarsening multigrid
// (device side; internal).
//
// The solver class of Section 3.6 is a semi-coarsening multigrid.  This
// library's GPU form for the 7-point operator: the 3-D hierarchy halves the
// colatitude only; the smoother relaxes every (radius, longitude) plane of
// fixed colatitude row i as one block of a block Gauss-Seidel sweep, planes
// with i even first, then odd (the 7-point operator couples a plane to its
// two neighbours only, so the planes of one parity are independent):
//   x_P += A_PP^{-1} (b - A x)_P,
// A_PP approximated by `plane_cycles` V(1,1) cycles of a 2-D multigrid on the
// plane block, started from zero:
//   * 2-D levels m = 0, 1, ..: the radius halved at each (nr a power of two, down
//     to one row), coarse plane operator R B P with R the sum of the two radius
//     children and P the linear prolongation along the radius (3/4, 1/4,
//     mirrored at the walls), a 9-point stencil in (radius, longitude);
//   * relaxation: zebra longitude lines (rows of fixed j, even first), each
//     line x_L += T_L^{-1} (r - B x)_L with T_L the cyclic tridiagonal part of
//     B on the line, solved by the periodic Thomas algorithm of Section 3.5
//     from factors made at set-up (the layout of xline_smooth.cuh);
//   * the coarsest level (one row) is one line: its relaxation from zero is
//     the exact solve.
//
// Every array of a 2-D level uses the 3-D layout (j * nth + i) * nph + k with
// nr >> m rows, so a plane is the cells of one i.  The nine plane operator
// entries of a cell are stored as nine arrays, offsets (dj, dk) in the order
// of kPlaneOff.  A launch works on the planes of one parity `p` of a level;
// relaxation also on the rows of one parity `q` (colour = p + 2 q).
#pragma once

#include "mg_internal.cuh"

namespace mgs {

// (dj, dk) of the nine plane operator entries: centre, radius -/+, longitude
// -/+, then the four corners (-,-), (-,+), (+,-), (+,+).
__host__ __device__ constexpr int plane_dj(int o) {
    return o == 1 ? -1 : o == 2 ? 1 : (o == 5 || o == 6) ? -1 : (o == 7 || o == 8) ? 1 : 0;
}
__host__ __device__ constexpr int plane_dk(int o) {
    return o == 3 ? -1 : o == 4 ? 1 : (o == 5 || o == 7) ? -1 : (o == 6 || o == 8) ? 1 : 0;
}

// Cells of the planes of parity p: (nth + 1 - p) / 2 planes.
__host__ __device__ inline i64 plane_cells(const Dims& D, int p) {
    return (i64)D.nr * ((D.nth + 1 - p) >> 1) * D.nph;
}

// work item t of the planes of parity p -> cell (j, i, k)
__device__ __forceinline__ C3 plane_cell(const Dims& D, int p, i64 t) {
    const int np = (D.nth + 1 - p) >> 1;
    const int k = (int)(t % D.nph);
    const i64 q = t / D.nph;
    C3 c;
    c.k = k;
    c.i = 2 * (int)(q % np) + p;
    c.j = (int)(q / np);
    return c;
}

// (B e)_c of the 9-point plane operator: entries beyond the radius walls are
// zero; the longitude wraps.
template <typename T>
__device__ __forceinline__ T plane_apply(const T* const* c, const T* e, const Dims& D, int j, int i, int k) {
    const int row = (j * D.nth + i) * D.nph;
    const int cell = row + k;
    T s = 0;
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        const int jj = j + plane_dj(o);
        if (jj < 0 || jj >= D.nr) continue;
        int kk = k + plane_dk(o);
        kk = kk < 0 ? kk + D.nph : (kk >= D.nph ? kk - D.nph : kk);
        s = fma(c[o][cell], e[(jj * D.nth + i) * D.nph + kk], s);
    }
    return s;
}

// r = b - A x on the planes of parity p (7-point operator of the 3-D level),
// and the 2-D correction e zeroed.
template <typename T, typename CF>
__device__ __forceinline__ void plane_res3d(const CF& cf, const Dims& D, const T* x, const T* b, T* r, T* e, int p,
                                            i64 first, i64 stride) {
    const i64 n = plane_cells(D, p);
    for (i64 t = first; t < n; t += stride) {
        const C3 c = plane_cell(D, p, t);
        Cell7<T> q;
        q.load(cf, D, c.j, c.i, c.k, XLin<T>{x});
        r[q.c] = q.resid(b[q.c]);
        e[q.c] = (T)0;
    }
}

// One zebra half-sweep of longitude lines: the lines of rows j = q mod 2 of
// the planes of parity p, each x_L += T_L^{-1} (r - B x)_L by the periodic
// elimination of xline_smooth.cuh (factors from set-up).  One warp per line
// (work items = lines x 32): every lane takes a chunk of at most kPlaneChunk consecutive cells of the
// line's leading block [0, n - 1), evaluates their residuals, runs both
// recurrences on its chunk from zero and publishes the chunk's affine map
// (value leaving = P * value entering + Q); an inclusive warp scan of the maps
// (shuffles) gives every chunk its entering value, as the chunked radial- and
// longitude-line passes do through shared memory.  The recurrences of the
// sequential elimination, regrouped (equal up to rounding).  n - 1 <= 32 *
// kPlaneChunk.
constexpr int kPlaneChunk = 16;

template <typename T>
__device__ __forceinline__ void warp_scan_maps(T& P, T& Q, int lane, bool reverse) {
    // inclusive composition over the lanes in order (reverse: from lane 31 down)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T pp = reverse ? __shfl_down_sync(0xffffffffu, P, o) : __shfl_up_sync(0xffffffffu, P, o);
        const T qq = reverse ? __shfl_down_sync(0xffffffffu, Q, o) : __shfl_up_sync(0xffffffffu, Q, o);
        const bool has = reverse ? lane + o < 32 : lane >= o;
        if (has) {   // (P, Q) after (pp, qq): x -> P (pp x + qq) + Q
            Q = fma(P, qq, Q);
            P = P * pp;
        }
    }
}

template <typename T>
__device__ __forceinline__ void plane_relax_warp(const T* const* c, const Dims& D, T* e, const T* r, const T* fac,
                                                 int p, int q, i64 first, i64 stride) {
    const i64 N = D.n();
    const T* alpha = fac;
    const T* beta = fac + N;
    const T* gamma = fac + 2 * N;
    const T* psi2 = fac + 3 * N;
    const int n = D.nph, m = n - 1;                       // the leading block: cells 0 .. n - 2
    const int lane = threadIdx.x & 31;
    const int rows = (m + 31) / 32;                        // cells per chunk (<= kPlaneChunk)
    const int k0 = min(lane * rows, m), nk = min(k0 + rows, m) - k0;
    const int np = (D.nth + 1 - p) >> 1, nq = (D.nr + 1 - q) >> 1;
    const i64 lines = (i64)np * nq;
    for (i64 t = first >> 5; t < lines; t += stride >> 5) {   // uniform per warp
        const int i = 2 * (int)(t % np) + p, j = 2 * (int)(t / np) + q;
        const int c0 = (j * D.nth + i) * D.nph, cl = c0 + n - 1;
        T d[kPlaneChunk], P[kPlaneChunk];
        // residuals and the forward recurrence on the chunk from zero
        T fq = 0, fp = 1;
#pragma unroll
        for (int u = 0; u < kPlaneChunk; ++u) {
            if (u < nk) {
                const int k = k0 + u;
                const T res = r[c0 + k] - plane_apply<T>(c, e, D, j, i, k);
                const T a = alpha[c0 + k];
                fq = fma(a, fq, beta[c0 + k] * res);
                fp = fp * a;
                d[u] = fq;
                P[u] = fp;
            }
        }
        const T rl = lane == 31 ? r[cl] - plane_apply<T>(c, e, D, j, i, n - 1) : (T)0;
        // entering value of each chunk: the composed maps of the chunks before it
        T sp = fp, sq = fq;
        warp_scan_maps<T>(sp, sq, lane, false);
        T in = __shfl_up_sync(0xffffffffu, sq, 1);
        if (lane == 0) in = 0;
        // backward recurrence on the corrected forward values, from zero
        T bq = 0, bp = 1, last = 0;
#pragma unroll
        for (int u = kPlaneChunk - 1; u >= 0; --u) {
            if (u < nk) {
                const T gm = gamma[c0 + k0 + u];
                bq = fma(gm, bq, fma(P[u], in, d[u]));
                bp = bp * gm;
                d[u] = bq;
                P[u] = bp;
                if (u == nk - 1) last = bq;
            }
        }
        sp = bp;
        sq = bq;
        warp_scan_maps<T>(sp, sq, lane, true);
        T bin = __shfl_down_sync(0xffffffffu, sq, 1);
        if (lane == 31) bin = 0;
        // psi1 at the first and the last cell of the leading block
        const int first_lane = 0, last_lane = (m - 1) / rows;
        const T w0 = __shfl_sync(0xffffffffu, nk > 0 ? fma(P[0], bin, d[0]) : (T)0, first_lane);
        const T wl = __shfl_sync(0xffffffffu, last, last_lane);   // the chunk with the last cell has bin = 0
        const T rl_all = __shfl_sync(0xffffffffu, rl, 31);
        const T dl = (rl_all - alpha[cl] * w0 - gamma[cl] * wl) * beta[cl];
#pragma unroll
        for (int u = 0; u < kPlaneChunk; ++u) {
            if (u < nk) {
                const int cc = c0 + k0 + u;
                e[cc] = e[cc] + fma(psi2[cc], dl, fma(P[u], bin, d[u]));
            }
        }
        if (lane == 31) e[cl] = e[cl] + dl;
        __syncwarp();
    }
}

// rc = R (r - B e): the two radius children of every coarse cell of the
// planes of parity p; ec zeroed.
template <typename T>
__device__ __forceinline__ void plane_restrict(const T* const* c, const Dims& D, const T* e, const T* r,
                                               const Dims& Dc, T* rc, T* ec, int p, i64 first, i64 stride) {
    const i64 n = plane_cells(Dc, p);
    for (i64 t = first; t < n; t += stride) {
        const C3 C = plane_cell(Dc, p, t);
        T s = 0;
        for (int dj = 0; dj < 2; ++dj) {
            const int j = 2 * C.j + dj;
            const int f = (j * D.nth + C.i) * D.nph + C.k;
            s += r[f] - plane_apply<T>(c, e, D, j, C.i, C.k);
        }
        const int cc = (C.j * Dc.nth + C.i) * Dc.nph + C.k;
        rc[cc] = s;
        ec[cc] = (T)0;
    }
}

// Weight of coarse row J in the prolongation of fine row j (nc coarse rows):
// 3/4 on J = j / 2, 1/4 on its neighbour towards j, which is J itself at a
// wall (weight 1).
__host__ __device__ inline double plane_pw(int j, int J, int nc) {
    const int C = j >> 1;
    int nb = (j & 1) ? C + 1 : C - 1;
    if (nb < 0 || nb >= nc) nb = C;
    return (J == C ? 0.75 : 0.0) + (J == nb ? 0.25 : 0.0);
}

// e += P ec on the planes of parity p.
template <typename T>
__device__ __forceinline__ void plane_prolong(const Dims& D, T* e, const Dims& Dc, const T* ec, int p, i64 first,
                                              i64 stride) {
    const i64 n = plane_cells(D, p);
    for (i64 t = first; t < n; t += stride) {
        const C3 f = plane_cell(D, p, t);
        const int C = f.j >> 1;
        int nb = (f.j & 1) ? C + 1 : C - 1;
        if (nb < 0 || nb >= Dc.nr) nb = C;
        const T a = ec[(C * Dc.nth + f.i) * Dc.nph + f.k];
        const T b = ec[(nb * Dc.nth + f.i) * Dc.nph + f.k];
        const int fc = (f.j * D.nth + f.i) * D.nph + f.k;
        e[fc] = e[fc] + fma((T)0.25, b, (T)0.75 * a);
    }
}

// x += e on the planes of parity p.
template <typename T>
__device__ __forceinline__ void plane_update(const Dims& D, T* x, const T* e, int p, i64 first, i64 stride) {
    const i64 n = plane_cells(D, p);
    for (i64 t = first; t < n; t += stride) {
        const C3 c = plane_cell(D, p, t);
        const int cc = cidx(D, c);
        x[cc] = x[cc] + e[cc];
    }
}

}  // namespace mgs

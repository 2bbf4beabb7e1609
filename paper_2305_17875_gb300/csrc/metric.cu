// metric.cu - set-up kernels: face metric of Section 3.2, coarse-level
// aggregation, precision casts and the dense coarsest operator.  FP64 throughout.
#include "mg_kernels.h"
#include "pc.h"

namespace mgs {

namespace {

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Cartesian position of vertex (i, j, k) in the paper's (zeta, eta, xi) order.
__device__ __forceinline__ V3 vert(const MetricTables& t, int i, int j, int k) {
    const double r = t.rho[j + 1], ct = t.cth[i + 1], st = t.sth[i + 1];
    const double cp = t.cph[k + 1], sp = t.sph[k + 1];
    return {t.ax1 * r * ct, t.ax2 * r * st * cp, r * st * sp};
}

// Section 3.2, step 1: the three columns dx/dzeta_p of J^{-1} at the d-normal
// face whose lowest corner is vertex v (paper order).  Normal column: 0.125 x
// (the four face-corner vertices one plane up - the four one plane down);
// tangential columns: 0.5 x (sum over the face's two edges of the edge vector).
__device__ void face_columns(const MetricTables& t, int d, const int v[3], V3 col[3]) {
    const int t1 = d == 0 ? 1 : 0;
    const int t2 = d == 2 ? 1 : 2;
    auto P = [&](int od, int o1, int o2) {
        int w[3] = {v[0], v[1], v[2]};
        w[d] += od;
        w[t1] += o1;
        w[t2] += o2;
        return vert(t, w[0], w[1], w[2]);
    };
    const V3 c00 = P(0, 0, 0), c10 = P(0, 1, 0), c01 = P(0, 0, 1), c11 = P(0, 1, 1);
    V3 up = P(1, 0, 0) + P(1, 1, 0) + P(1, 0, 1) + P(1, 1, 1);
    V3 dn = P(-1, 0, 0) + P(-1, 1, 0) + P(-1, 0, 1) + P(-1, 1, 1);
    col[d] = 0.125 * (up - dn);
    col[t1] = 0.5 * ((c10 - c00) + (c11 - c01));
    col[t2] = 0.5 * ((c01 - c00) + (c11 - c10));
}

// Steps 2, 4, 5: with a_p = col_{p+1} x col_{p+2} the columns of cof(J^{-1}),
// det = col_0 . a_0 and J = cof^T / det, so
//   G_pq = |det| sum_a J_pa J_qa = (a_p . a_q) / |det|.
// Returns |det| and writes row d of G.
__device__ double g_from_columns(const V3 col[3], int d, double row[3]) {
    const V3 a0 = cross(col[1], col[2]);
    const V3 a1 = cross(col[2], col[0]);
    const V3 a2 = cross(col[0], col[1]);
    const double adet = fabs(dot(col[0], a0));
    const V3 ad = d == 0 ? a0 : (d == 1 ? a1 : a2);
    row[0] = dot(ad, a0) / adet;
    row[1] = dot(ad, a1) / adet;
    row[2] = dot(ad, a2) / adet;
    return adet;
}

__device__ double face_metric(const MetricTables& t, int d, const int v[3], double row[3]) {
    V3 col[3];
    face_columns(t, d, v, col);
    return g_from_columns(col, d, row);
}

// The analytic option: the columns dx/dzeta_p exactly at the face centre
// from the mapping (x1 = ax1 r cos th, x2 = ax2 r sin th cos ph,
// x3 = r sin th sin ph) and the derivatives of r(eta), th(zeta), ph(xi);
// steps 2 to 5 as above.  Tables at half-index resolution: entry t is the
// value at index t / 2 (faces at even t, cell centres at odd t).
__device__ double face_metric_analytic(const AnalyticTables& t, int d, int i, int j, int k, double row[3]) {
    const int tr = 2 * j + (d == 1 ? 0 : 1), tt = 2 * i + (d == 0 ? 0 : 1), tp = 2 * k + (d == 2 ? 0 : 1);
    const double r = t.rho[tr], dr = t.drho[tr];
    const double ct = t.cth[tt], st = t.sth[tt], cp = t.cph[tp], sp = t.sph[tp];
    V3 col[3];
    col[0] = {-t.ax1 * r * st * t.dth, t.ax2 * r * ct * cp * t.dth, r * ct * sp * t.dth};
    col[1] = {t.ax1 * ct * dr, t.ax2 * st * cp * dr, st * sp * dr};
    col[2] = {0.0, -t.ax2 * r * st * sp * t.dph, r * st * cp * t.dph};
    return g_from_columns(col, d, row);
}

__global__ void k_face_metric(MetricTables t, Dims D, int stencil, double* g0,
                              double* g1, double* g2, double* g3, double* g4, double* g5,
                              double* g6, double* g7, double* g8, double* J) {
    const i64 n = D.n();
    double* g[9] = {g0, g1, g2, g3, g4, g5, g6, g7, g8};
    for (i64 c = blockIdx.x * (i64)blockDim.x + threadIdx.x; c < n; c += (i64)gridDim.x * blockDim.x) {
        const C3 cc = decode(D, c);
        const int k = cc.k, i = cc.i, j = cc.j;
        double row[3], det_sum = 0.0;
        // lower faces: rows stored (zero on the lower walls), determinants kept
        for (int d = 0; d < 3; ++d) {
            const int v[3] = {i, j, k};
            det_sum += face_metric(t, d, v, row);
            const bool wall = (d == 0 && i == 0) || (d == 1 && j == 0);
            for (int q = 0; q < 3; ++q) {
                double* dst = g[3 * d + q];
                if (dst && (stencil == 19 || q == d)) dst[c] = wall ? 0.0 : row[q];
            }
        }
        // upper faces: determinants only (step 3 averages all six faces)
        {
            const int vz[3] = {i + 1, j, k};
            const int ve[3] = {i, j + 1, k};
            const int vx[3] = {i, j, k + 1};
            det_sum += face_metric(t, 0, vz, row);
            det_sum += face_metric(t, 1, ve, row);
            det_sum += face_metric(t, 2, vx, row);
        }
        J[c] = det_sum / 6.0;
    }
}

// G_dd on the four wall planes (Section 3.2 steps 1-5 at the wall faces):
// radius walls j = 0 and j = nr ([nth][nph] each), colatitude walls i = 0 and
// i = nth ([nr][nph] each).
__global__ void k_wall_G(MetricTables t, Dims D, double* r_lo, double* r_hi, double* th_lo, double* th_hi) {
    const i64 nr_w = (i64)D.nth * D.nph, nt_w = (i64)D.nr * D.nph;
    double row[3];
    for (i64 q = blockIdx.x * (i64)blockDim.x + threadIdx.x; q < nr_w + nt_w; q += (i64)gridDim.x * blockDim.x) {
        if (q < nr_w) {
            const int i = (int)(q / D.nph), k = (int)(q % D.nph);
            const int vl[3] = {i, 0, k}, vh[3] = {i, D.nr, k};
            face_metric(t, 1, vl, row);
            r_lo[q] = row[1];
            face_metric(t, 1, vh, row);
            r_hi[q] = row[1];
        } else {
            const i64 p = q - nr_w;
            const int j = (int)(p / D.nph), k = (int)(p % D.nph);
            const int vl[3] = {0, j, k}, vh[3] = {D.nth, j, k};
            // on the full sphere these faces lie on the polar axis: zero area, no flux
            face_metric(t, 0, vl, row);
            th_lo[p] = D.cut ? 0.0 : row[0];
            face_metric(t, 0, vh, row);
            th_hi[p] = D.cut ? 0.0 : row[0];
        }
    }
}

// The face metric of the analytic option, stored like k_face_metric's.
__global__ void k_face_metric_analytic(AnalyticTables t, Dims D, int stencil, double* g0, double* g1, double* g2,
                                       double* g3, double* g4, double* g5, double* g6, double* g7, double* g8,
                                       double* J) {
    const i64 n = D.n();
    double* g[9] = {g0, g1, g2, g3, g4, g5, g6, g7, g8};
    for (i64 c = blockIdx.x * (i64)blockDim.x + threadIdx.x; c < n; c += (i64)gridDim.x * blockDim.x) {
        const C3 cc = decode(D, c);
        const int k = cc.k, i = cc.i, j = cc.j;
        double row[3], det_sum = 0.0;
        for (int d = 0; d < 3; ++d) {
            det_sum += face_metric_analytic(t, d, i, j, k, row);
            const bool wall = (d == 0 && i == 0) || (d == 1 && j == 0);
            for (int q = 0; q < 3; ++q) {
                double* dst = g[3 * d + q];
                if (dst && (stencil == 19 || q == d)) dst[c] = wall ? 0.0 : row[q];
            }
        }
        det_sum += face_metric_analytic(t, 0, i + 1, j, k, row);
        det_sum += face_metric_analytic(t, 1, i, j + 1, k, row);
        det_sum += face_metric_analytic(t, 2, i, j, k + 1, row);
        J[c] = det_sum / 6.0;
    }
}

// C and 1/|J^{-1}| of every cell's three lower faces: with a_p = col_{p+1} x
// col_{p+2} (the cofactor columns of J^{-1}) and det = col_0 . a_0, the
// inverse has rows a_p / det, so C row p = |det| a_p / det = sign(det) a_p.
struct CArrays {
    double* C[27];
    double* inv[3];
};
__global__ void k_face_C(MetricTables t, Dims D, CArrays out) {
    const i64 n = D.n();
    for (i64 c = blockIdx.x * (i64)blockDim.x + threadIdx.x; c < n; c += (i64)gridDim.x * blockDim.x) {
        const C3 cc = decode(D, c);
        for (int d = 0; d < 3; ++d) {
            const int v[3] = {cc.i, cc.j, cc.k};
            V3 col[3];
            face_columns(t, d, v, col);
            const V3 a[3] = {cross(col[1], col[2]), cross(col[2], col[0]), cross(col[0], col[1])};
            const double det = dot(col[0], a[0]);
            const double sg = det < 0.0 ? -1.0 : 1.0;
            for (int p = 0; p < 3; ++p) {
                out.C[9 * d + 3 * p + 0][c] = sg * a[p].x;
                out.C[9 * d + 3 * p + 1][c] = sg * a[p].y;
                out.C[9 * d + 3 * p + 2][c] = sg * a[p].z;
            }
            out.inv[d][c] = 1.0 / fabs(det);
        }
    }
}

// A coarse face is tiled by the fine faces of the children next to it:
// G^c_dq = (sum of those fine G_dq) / c_q.
__global__ void k_coarsen(CoefF64 f, Dims Df, int cz, int ce, int cx, int stencil, Dims Dc,
                          double* g0, double* g1, double* g2, double* g3, double* g4,
                          double* g5, double* g6, double* g7, double* g8) {
    double* g[9] = {g0, g1, g2, g3, g4, g5, g6, g7, g8};
    const int cfac[3] = {cz, ce, cx};
    const i64 n = Dc.n();
    for (i64 c = blockIdx.x * (i64)blockDim.x + threadIdx.x; c < n; c += (i64)gridDim.x * blockDim.x) {
        const C3 cc = decode(Dc, c);
        const int K = cc.k, I = cc.i, Jr = cc.j;
        for (int d = 0; d < 3; ++d) {
            // fine plane of the face along d; children along the other two axes
            const int j0 = ce * Jr, i0 = cz * I, k0 = cx * K;
            const int nj = d == 1 ? 1 : ce, ni = d == 0 ? 1 : cz, nk = d == 2 ? 1 : cx;
            for (int q = 0; q < 3; ++q) {
                const int a = 3 * d + q;
                if (!g[a]) continue;
                double s = 0.0;
                for (int dj = 0; dj < nj; ++dj)
                    for (int di = 0; di < ni; ++di)
                        for (int dk = 0; dk < nk; ++dk)
                            s += f.g[a][cidx(Df, j0 + dj, i0 + di, k0 + dk)];
                g[a][c] = s / cfac[q];
            }
        }
    }
}

__global__ void k_cast32(const double* src, float* dst, i64 n) {
    for (i64 c = blockIdx.x * (i64)blockDim.x + threadIdx.x; c < n; c += (i64)gridDim.x * blockDim.x)
        dst[c] = (float)src[c];
}
__global__ void k_cast16(const double* src, __half* dst, i64 n, float inv_scale) {
    for (i64 c = blockIdx.x * (i64)blockDim.x + threadIdx.x; c < n; c += (i64)gridDim.x * blockDim.x)
        dst[c] = __float2half_rn((float)src[c] * inv_scale);
}

// Column m of A: apply the operator to the unit vector e_m (row c per thread).
struct UnitX {
    i64 m;
    Dims D;
    __device__ __forceinline__ double operator()(C3 c) const { return cidx(D, c) == m ? 1.0 : 0.0; }
};
template <int S>
__global__ void k_dense(CoefF64 cf, Dims D, double* A) {
    const i64 n = D.n();
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n * n; t += (i64)gridDim.x * blockDim.x) {
        const i64 row = t / n, m = t % n;
        const int k = (int)(row % D.nph);
        const i64 ji = row / D.nph;
        C3 c{(int)(ji / D.nth), (int)(ji % D.nth), k};
        UnitX X{m, D};
        A[t] = apply_cell<S, double>(cf, X, D, c);
    }
}

// Assembled operator rows of a level (row_off order): coefficient n of cell c is
// the operator applied to the unit vector of neighbour n, evaluated at c.  A
// neighbour that coincides with an earlier one (a longitude ring of two cells,
// or a cell across the pole that is also a longitude neighbour) keeps its
// coefficient on the earlier entry and stores 0.
template <int S>
__global__ void k_assemble(CoefF64 cf, Dims D, double* a, int nrows) {
    const i64 N = D.n();
    for (i64 cl = blockIdx.x * (i64)blockDim.x + threadIdx.x; cl < N; cl += (i64)gridDim.x * blockDim.x) {
        const C3 p = decode(D, cl);
        if (S == 7) {
            a[cl] = diag_cell<7, double>(cf, D, p);
            continue;
        }
        i64 t[19];
        for (int n = 0; n < nrows; ++n) {
            const int j = p.j + row_off(n, 0), i = p.i + row_off(n, 1);
            int k = p.k + row_off(n, 2);
            k = k < 0 ? k + D.nph : (k >= D.nph ? k - D.nph : k);
            int cell, pole;
            if (j >= 0 && j < D.nr && across_pole(D, p, row_off(n, 0), row_off(n, 1), row_off(n, 2), &cell, &pole))
                t[n] = cell;   // the cell across the pole
            else
                t[n] = (j < 0 || j >= D.nr || i < 0 || i >= D.nth) ? -1 : (i64)cidx(D, j, i, k);
            bool dup = false;
            for (int m = 0; m < n; ++m) dup = dup || (t[n] >= 0 && t[m] == t[n]);
            a[n * N + cl] = (t[n] < 0 || dup) ? 0.0 : apply_cell<19, double>(cf, UnitX{t[n], D}, D, p);
        }
    }
}

// Factorisation of the radial-line blocks A_LL (tridiagonal: the operator's
// couplings at radial offsets -1, 0, +1, found by applying the operator to
// unit vectors) for the radial-line smoother: Thomas elimination in FP64
// along every line, stored as alpha = -a_j / b'_j, beta = 1 / b'_j,
// gamma = -c_j / b'_j (three arrays of n cells, value type T).  A zero or
// non-finite pivot counts in *bad.
template <int S, typename T>
__global__ void k_line_factors(CoefF64 cf, Dims D, T* fac, unsigned* bad) {
    const i64 N = D.n();
    const i64 lines = (i64)D.nth * D.nph;
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < lines; t += (i64)gridDim.x * blockDim.x) {
        const int i = (int)(t / D.nph), k = (int)(t % D.nph);
        double cprev = 0.0;
        for (int j = 0; j < D.nr; ++j) {
            const C3 p{j, i, k};
            const i64 c = cidx(D, p);
            const double lo = j > 0 ? apply_cell<S, double>(cf, UnitX{c - D.nth * D.nph, D}, D, p) : 0.0;
            const double dd = apply_cell<S, double>(cf, UnitX{c, D}, D, p);
            const double up = j + 1 < D.nr ? apply_cell<S, double>(cf, UnitX{c + D.nth * D.nph, D}, D, p) : 0.0;
            const double ib = 1.0 / (dd - lo * cprev);
            cprev = up * ib;
            const double al = -lo * ib;
            if (!isfinite(ib) || !isfinite(al) || !isfinite(cprev)) atomicAdd(bad, 1u);
            fac[c] = (T)al;
            fac[N + c] = (T)ib;
            fac[2 * N + c] = (T)(-cprev);
        }
    }
}

// Factors of the longitude-line blocks (the cyclic tridiagonal part of the
// operator on every line of fixed j and i: couplings at longitude offsets
// -1, 0, +1, found by applying the operator to unit vectors) for the
// longitude-line smoother, in the layout of xline_smooth.cuh: the normalised
// Thomas elimination of the leading block T_c (alpha, beta, gamma), psi2 =
// T_c^{-1} (-a_0, 0, .., 0, -c_{n-2}), and in the last cell's slot c_{n-1},
// 1 / (b_{n-1} + c_{n-1} psi2_0 + a_{n-1} psi2_{n-2}) and a_{n-1}.  FP64
// elimination; the backward pass of psi2 reads the stored (type T) factors,
// as the smoother does.  Needs nph >= 4.  A zero or non-finite pivot counts
// in *bad.
template <int S, typename T>
__global__ void k_xline_factors(CoefF64 cf, Dims D, T* fac, unsigned* bad) {
    const i64 N = D.n();
    const i64 lines = (i64)D.nr * D.nth;
    const int n = D.nph;
    T* alpha = fac;
    T* beta = fac + N;
    T* gamma = fac + 2 * N;
    T* psi2 = fac + 3 * N;
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < lines; t += (i64)gridDim.x * blockDim.x) {
        const int j = (int)(t / D.nth), i = (int)(t % D.nth);
        const i64 c0 = (i64)(j * D.nth + i) * n;
        auto coupling = [&](int k, int m) {   // A(c_k, c_m)
            const C3 p{j, i, k};
            return apply_cell<S, double>(cf, UnitX{c0 + m, D}, D, p);
        };
        bool ok = true;
        // forward elimination of T_c; psi2's forward recurrence alongside
        double cprev = 0.0, q = 0.0;
        for (int k = 0; k < n - 1; ++k) {
            const double lo = k > 0 ? coupling(k, k - 1) : 0.0;
            const double dd = coupling(k, k);
            const double up = k < n - 2 ? coupling(k, k + 1) : 0.0;
            const double ib = 1.0 / (dd - lo * cprev);
            const double a = -lo * ib;
            cprev = up * ib;
            double e = 0.0;                               // right side of psi2
            if (k == 0) e -= coupling(0, n - 1);
            if (k == n - 2) e -= coupling(n - 2, n - 1);
            q = fma(a, q, ib * e);
            ok = ok && isfinite(ib) && isfinite(a) && isfinite(cprev);
            alpha[c0 + k] = (T)a;
            beta[c0 + k] = (T)ib;
            gamma[c0 + k] = (T)(-cprev);
            psi2[c0 + k] = (T)q;                          // forward value, finished below
        }
        double e = 0.0, p2_first = 0.0, p2_last = 0.0;
        for (int k = n - 2; k >= 0; --k) {
            e = fma((double)gamma[c0 + k], e, (double)psi2[c0 + k]);
            psi2[c0 + k] = (T)e;
            if (k == n - 2) p2_last = e;
            if (k == 0) p2_first = e;
        }
        const double an = coupling(n - 1, n - 2), cn = coupling(n - 1, 0), bn = coupling(n - 1, n - 1);
        const double inv = 1.0 / (bn + cn * p2_first + an * p2_last);
        ok = ok && isfinite(inv);
        alpha[c0 + n - 1] = (T)cn;
        beta[c0 + n - 1] = (T)inv;
        gamma[c0 + n - 1] = (T)an;
        psi2[c0 + n - 1] = (T)0;
        if (!ok) atomicAdd(bad, 1u);
    }
}

// ---- in-place Gauss-Jordan inversion with partial pivoting (FP64), for the
// bordered coarsest matrix [A 1; 1^T 0] of order m.  A zero pivot (singular
// matrix) sets *bad.
__global__ void k_bordered(const double* __restrict__ A, int n, double* __restrict__ M) {
    const int m = n + 1;
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < (i64)m * m; t += (i64)gridDim.x * blockDim.x) {
        const int r = (int)(t / m), c = (int)(t % m);
        M[t] = r < n && c < n ? A[(i64)r * n + c] : (r == n && c == n ? 0.0 : 1.0);
    }
}

// One launch for the whole inversion: a cooperative grid (every CTA
// co-resident) in which CTA b owns rows b, b + G, ...; pivot rows are never
// moved (implicit partial pivoting), so the in-place result M satisfies
// inverse[i][j] = M[piv[i]][ipiv[j]] with ipiv the inverse permutation.
// Step k: every CTA reduces the candidates (|M[r][k]|, r) the CTAs published
// for column k (the largest |.| over unused rows, ties to the lower row) to
// the pivot row p, copies row p, scales it by 1 / M[p][k] (M[p][k] becomes
// 1 / M[p][k]) and eliminates column k from its own rows r != p
// (M[r][c] -= M[r][k] * row_p[c], M[r][k] = -M[r][k] / M[p][k]), publishing
// its candidates for column k + 1 on the way; the owner of p writes the scaled
// row after the step's barrier (the other CTAs read the unscaled one during
// the step).  One grid barrier per column.  Barrier waits are bounded: a wait
// that gives up sets *bad = 2 and the CTA leaves.
struct GjShared {
    double row[kMaxGj];     // the pivot row (scaled)
    double f[kMaxGj];       // multipliers M[r][k] of this CTA's rows
    double cv[32];          // block reductions
    int ci[32];
    int piv[kMaxGj];
    unsigned char used[kMaxGj];
};

__device__ bool gj_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks, int* bad) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd((unsigned*)gen, 1u);
        } else {
            for (int it = 0; it < (1 << 22) && *gen == g; ++it)
                if (it > 64) __nanosleep(64);
            if (*gen == g) {
                ok = 0;
                atomicExch(bad, 2);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Largest (|v|, row) over the block's threads, ties to the lower row; the
// result in thread 0.
__device__ void gj_reduce(double& v, int& r, GjShared& sh) {
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const int orr = __shfl_down_sync(0xffffffffu, r, o);
        if (ov > v || (ov == v && orr < r)) v = ov, r = orr;
    }
    if ((threadIdx.x & 31) == 0) sh.cv[threadIdx.x >> 5] = v, sh.ci[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sh.cv[w] > v || (sh.cv[w] == v && sh.ci[w] < r)) v = sh.cv[w], r = sh.ci[w];
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_gj_coop(double* __restrict__ M, int m, double* cand_v, int* cand_r,
                                                  unsigned* bar, int* piv_out, int* ipiv_out, int* bad) {
    __shared__ GjShared sh;
    const int G = gridDim.x, b = blockIdx.x;
    for (int r = threadIdx.x; r < m; r += blockDim.x) sh.used[r] = 0;
    {   // candidates for column 0
        double v = -1.0;
        int rr = m;
        for (int r = b + (int)threadIdx.x * G; r < m; r += (int)blockDim.x * G) {
            const double a = fabs(M[(i64)r * m]);
            if (a > v || (a == v && r < rr)) v = a, rr = r;
        }
        gj_reduce(v, rr, sh);
        if (threadIdx.x == 0) {
            cand_v[b] = v;
            cand_r[b] = rr;
        }
    }
    if (!gj_barrier(bar, bar + 1, G, bad)) return;
    int pending = -1;   // a scaled pivot row of this CTA not yet written
    for (int k = 0; k < m; ++k) {
        const int buf = (k & 1) * G;
        if (pending >= 0) {   // the previous step's pivot row, scaled
            for (int c = threadIdx.x; c < m; c += blockDim.x) M[(i64)pending * m + c] = sh.row[c];
            pending = -1;
            __syncthreads();
        }
        // the pivot: every CTA reduces the same candidates the same way
        double v = -1.0;
        int p = m;
        for (int q = threadIdx.x; q < G; q += blockDim.x) {
            const double cv = __ldcg(cand_v + buf + q);
            const int cr = __ldcg(cand_r + buf + q);
            if (cv > v || (cv == v && cr < p)) v = cv, p = cr;
        }
        gj_reduce(v, p, sh);
        if (threadIdx.x == 0) {
            sh.ci[0] = p;
            if (!(v > 0.0) || p >= m) atomicExch(bad, 1);
        }
        __syncthreads();
        p = sh.ci[0];
        if (p >= m) return;   // singular (flagged): every CTA leaves here
        // the pivot row, scaled
        const double inv = 1.0 / __ldcg(M + (i64)p * m + k);
        for (int c = threadIdx.x; c < m; c += blockDim.x)
            sh.row[c] = c == k ? inv : __ldcg(M + (i64)p * m + c) * inv;
        if (threadIdx.x == 0) {
            sh.used[p] = 1;
            sh.piv[k] = p;
        }
        __syncthreads();
        // the multipliers first: column k is overwritten below
        for (int r = b + (int)threadIdx.x * G; r < m; r += (int)blockDim.x * G) sh.f[(r - b) / G] = M[(i64)r * m + k];
        __syncthreads();
        // eliminate column k from this CTA's rows; candidates for column k + 1
        double bv = -1.0;
        int br = m;
        for (int r = b; r < m; r += G) {
            if (r == p) continue;
            const double f = sh.f[(r - b) / G];
            for (int c = threadIdx.x; c < m; c += blockDim.x) {
                const double nv = c == k ? -f * inv : fma(-f, sh.row[c], M[(i64)r * m + c]);
                M[(i64)r * m + c] = nv;
                if (c == k + 1 && !sh.used[r]) {
                    const double a = fabs(nv);
                    if (a > bv || (a == bv && r < br)) bv = a, br = r;
                }
            }
        }
        if (p % G == b) pending = p;
        gj_reduce(bv, br, sh);
        if (threadIdx.x == 0) {
            cand_v[((k + 1) & 1) * G + b] = bv;
            cand_r[((k + 1) & 1) * G + b] = br;
        }
        if (!gj_barrier(bar, bar + 1, G, bad)) return;
    }
    if (pending >= 0)
        for (int c = threadIdx.x; c < m; c += blockDim.x) M[(i64)pending * m + c] = sh.row[c];
    if (b == 0)
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            piv_out[k] = sh.piv[k];
            ipiv_out[sh.piv[k]] = k;
        }
}

// binv = leading n x n block of the inverse: binv[i][j] = M[piv[i]][ipiv[j]].
__global__ void k_gj_finish(const double* __restrict__ M, int m, const int* __restrict__ piv,
                            const int* __restrict__ ipiv, double* __restrict__ binv) {
    const int n = m - 1;
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < (i64)n * n; t += (i64)gridDim.x * blockDim.x) {
        const int r = (int)(t / n), c = (int)(t % n);
        binv[t] = M[(i64)piv[r] * m + ipiv[c]];
    }
}

int grid_for(i64 n, int threads) {
    i64 b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_face_metric(const MetricTables& t, Dims D, int stencil, double* const g[9],
                               double* J, cudaStream_t s) {
    k_face_metric<<<grid_for(D.n(), 128), 128, 0, s>>>(t, D, stencil, g[0], g[1], g[2], g[3],
                                                       g[4], g[5], g[6], g[7], g[8], J);
    return cudaGetLastError();
}

cudaError_t launch_bordered_inverse(const double* A, int n, double* work, double* col, int* piv, int* perm,
                                   int* bad, double* binv, cudaStream_t s) {
    const int m = n + 1;
    if (m > kMaxGj) return cudaErrorInvalidValue;
    const i64 mm = (i64)m * m;
    k_bordered<<<grid_for(mm, 256), 256, 0, s>>>(A, n, work);
    // a cooperative grid of one CTA per SM (at most one per row); col holds
    // the barrier words and the double-buffered candidates
    int dev = 0, sms = 0, per = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gj_coop, 256, 0);
    if (e != cudaSuccess) return e;
    if (!coop || per < 1) return cudaErrorNotSupported;
    int G = std::min(std::min(sms, m), kGjMaxCtas);
    unsigned* bar = reinterpret_cast<unsigned*>(col);                 // count, generation
    double* cand_v = col + 1;                                          // 2 G values
    int* cand_r = reinterpret_cast<int*>(col + 1 + 2 * G);             // 2 G rows
    e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    int mv = m;
    void* args[] = {&work, &mv, &cand_v, &cand_r, &bar, &piv, &perm, &bad};
    e = cudaLaunchCooperativeKernel((const void*)k_gj_coop, dim3(G), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    k_gj_finish<<<grid_for((i64)n * n, 256), 256, 0, s>>>(work, m, piv, perm, binv);
    return cudaGetLastError();
}

cudaError_t launch_assemble_rows(const LevelView& lv, double* a, cudaStream_t s) {
    if (lv.stencil == 19)
        k_assemble<19><<<grid_for(lv.D.n(), 128), 128, 0, s>>>(lv.c64, lv.D, a, assembled_rows(lv));
    else k_assemble<7><<<grid_for(lv.D.n(), 256), 256, 0, s>>>(lv.c64, lv.D, a, 1);
    return cudaGetLastError();
}

cudaError_t launch_line_factors(const LevelView& lv, int prec, void* fac, unsigned* bad, cudaStream_t s) {
    const i64 lines = (i64)lv.D.nth * lv.D.nph;
    const int nb = grid_for(lines, 128);
    if (prec == PREC64) {
        if (lv.stencil == 19) k_line_factors<19, double><<<nb, 128, 0, s>>>(lv.c64, lv.D, (double*)fac, bad);
        else k_line_factors<7, double><<<nb, 128, 0, s>>>(lv.c64, lv.D, (double*)fac, bad);
    } else {
        if (lv.stencil == 19) k_line_factors<19, float><<<nb, 128, 0, s>>>(lv.c64, lv.D, (float*)fac, bad);
        else k_line_factors<7, float><<<nb, 128, 0, s>>>(lv.c64, lv.D, (float*)fac, bad);
    }
    return cudaGetLastError();
}

cudaError_t launch_xline_factors(const LevelView& lv, int prec, void* fac, unsigned* bad, cudaStream_t s) {
    const i64 lines = (i64)lv.D.nr * lv.D.nth;
    const int nb = grid_for(lines, 128);
    if (prec == PREC64) {
        if (lv.stencil == 19) k_xline_factors<19, double><<<nb, 128, 0, s>>>(lv.c64, lv.D, (double*)fac, bad);
        else k_xline_factors<7, double><<<nb, 128, 0, s>>>(lv.c64, lv.D, (double*)fac, bad);
    } else {
        if (lv.stencil == 19) k_xline_factors<19, float><<<nb, 128, 0, s>>>(lv.c64, lv.D, (float*)fac, bad);
        else k_xline_factors<7, float><<<nb, 128, 0, s>>>(lv.c64, lv.D, (float*)fac, bad);
    }
    return cudaGetLastError();
}

cudaError_t launch_face_metric_analytic(const AnalyticTables& t, Dims D, int stencil, double* const g[9],
                                        double* J, cudaStream_t s) {
    k_face_metric_analytic<<<grid_for(D.n(), 128), 128, 0, s>>>(t, D, stencil, g[0], g[1], g[2], g[3], g[4],
                                                                 g[5], g[6], g[7], g[8], J);
    return cudaGetLastError();
}

cudaError_t launch_wall_G(const MetricTables& t, Dims D, double* const g[4], cudaStream_t s) {
    const i64 n = (i64)D.nth * D.nph + (i64)D.nr * D.nph;
    k_wall_G<<<grid_for(n, 128), 128, 0, s>>>(t, D, g[0], g[1], g[2], g[3]);
    return cudaGetLastError();
}

cudaError_t launch_face_C(const MetricTables& t, Dims D, double* const C[27], double* const inv_det[3],
                          cudaStream_t s) {
    CArrays a;
    for (int q = 0; q < 27; ++q) a.C[q] = C[q];
    for (int d = 0; d < 3; ++d) a.inv[d] = inv_det[d];
    k_face_C<<<grid_for(D.n(), 128), 128, 0, s>>>(t, D, a);
    return cudaGetLastError();
}

cudaError_t launch_coarsen_faces(const LevelView& f, Dims Dc, double* const gc[9], cudaStream_t s) {
    k_coarsen<<<grid_for(Dc.n(), 128), 128, 0, s>>>(f.c64, f.D, f.cz, f.ce, f.cx, f.stencil, Dc, gc[0],
                                                    gc[1], gc[2], gc[3], gc[4], gc[5], gc[6], gc[7], gc[8]);
    return cudaGetLastError();
}

cudaError_t launch_cast32(const double* src, float* dst, i64 n, cudaStream_t s) {
    k_cast32<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_cast16(const double* src, __half* dst, i64 n, float inv_scale, cudaStream_t s) {
    k_cast16<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n, inv_scale);
    return cudaGetLastError();
}

cudaError_t launch_dense_operator(const LevelView& lv, double* A, cudaStream_t s) {
    const i64 nn = lv.D.n() * lv.D.n();
    if (lv.stencil == 19)
        k_dense<19><<<grid_for(nn, 256), 256, 0, s>>>(lv.c64, lv.D, A);
    else
        k_dense<7><<<grid_for(nn, 256), 256, 0, s>>>(lv.c64, lv.D, A);
    return cudaGetLastError();
}

}  // namespace mgs

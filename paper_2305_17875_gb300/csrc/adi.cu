// adi.cu - the ADI-CN implicit viscous sweeps of Section 3.4 (Eqs. solve_2 to
// solve_4) for one cell-centred field on a handle's fine grid, FP64.
//
// With kappa = (h / 2) sqrt(Pr / Ra) and L_p the diagonal viscous term of
// direction p (Eq. PC_term1 in flux form; zeta = colatitude i, eta = radius
// j, xi = longitude k):
//   sweep zeta:  (J - kappa L_zeta) u*   = J u^n + s + kappa L_zeta u^n + 2 kappa (L_eta + L_xi) u^n
//   sweep eta:   (J - kappa L_eta)  u**  = J u* - kappa L_eta u^n
//   sweep xi:    (J - kappa L_xi)   u*** = J u** - kappa L_xi u^n     (periodic)
// One launch per sweep, two threads per grid line (adjacent lanes): each
// forms the rows of its half of the line's tridiagonal system from the face
// metric (G_pp of the row's two faces, J) and the stencil of u^n, and
// eliminates towards the middle row as it goes (a twisted factorisation:
// normalised Thomas from both ends, pivot ratios in a work array laid out
// [row][line]); the lanes swap their last pivots by a shuffle, solve the
// middle row and substitute outwards into u.  Periodic longitude lines carry
// the corner column as an extra right side (Eqs. TAP2-TAP8).  Up to four
// fields with the same kappa and wall kinds (the three velocity components)
// share the matrix: one division per row serves all of them, and their
// independent recurrences fill a thread's FP64 pipeline.  Colatitude and
// radius lines are adjacent in memory along longitude, so their loads
// coalesce; longitude lines are contiguous (a thread walks a run of
// consecutive cells).  Right sides read only the line's own cell of the
// previous sweep's result, so every sweep works in place on u.
//
// Walls: zero flux, or a value held on the wall face half a cell from the
// centre, whose face flux is 2 G_pp(wall face) (u_w - u_c) outward; G_pp of
// the wall faces comes from the face metric (k_wall_G).
#include <algorithm>
#include <cmath>
#include <string>

#include "engine.h"
#include "pc.h"

namespace mgs {
namespace {

constexpr int kAT = 128;
constexpr int kMaxF = 4;    // fields per launch (the three velocity components share one matrix)

unsigned adi_blocks(i64 lines) { return (unsigned)((lines + kAT - 1) / kAT); }

struct AdiArgs {
    Dims D;
    const double* G[3];     // G_pp on the lower p-face of every cell (0 on lower walls)
    const double* J;
    const double* un[kMaxF];
    const double* src[kMaxF];   // may be null
    double* u[kMaxF];           // result; input of the eta and xi sweeps
    double* w;              // 2 N doubles of line-solve work
    double kappa;
    int wall[2];            // per direction 0 (colatitude), 1 (radius): 1 = value, 0 = zero flux
    double wv[kMaxF][2][2]; // wall values [field][direction][lower, upper]
    const double* wg[2][2]; // wall-face G_pp [direction][lower, upper]: colatitude [nr][nph], radius [nth][nph]
};

// Fluxes of direction p through the lower and upper faces of cell (j, i, k)
// for field f of u^n: interior faces G (x_up - x_down); value walls
// 2 G_w (x_c - x_w) (lower) and 2 G_w (x_w - x_c) (upper); zero-flux walls 0.
template <int P>
__device__ __forceinline__ double diag_term(const AdiArgs& A, int f, i64 c, int j, int i, int k) {
    const Dims& D = A.D;
    const double* x = A.un[f];
    const double xc = __ldg(x + c);
    double flo, fhi;
    if constexpr (P == 2) {
        const i64 km = k == 0 ? c + D.nph - 1 : c - 1;
        const i64 kp = k == D.nph - 1 ? c - D.nph + 1 : c + 1;
        flo = __ldg(A.G[2] + c) * (xc - __ldg(x + km));
        fhi = __ldg(A.G[2] + kp) * (__ldg(x + kp) - xc);
    } else {
        const int m = P == 0 ? i : j;
        const int n = P == 0 ? D.nth : D.nr;
        const i64 st = P == 0 ? (i64)D.nph : (i64)D.nth * D.nph;
        const i64 wi = P == 0 ? (i64)j * D.nph + k : (i64)i * D.nph + k;
        if (m > 0) flo = __ldg(A.G[P] + c) * (xc - __ldg(x + c - st));
        else flo = A.wall[P] ? 2.0 * __ldg(A.wg[P][0] + wi) * (xc - A.wv[f][P][0]) : 0.0;
        if (m < n - 1) fhi = __ldg(A.G[P] + c + st) * (__ldg(x + c + st) - xc);
        else fhi = A.wall[P] ? 2.0 * __ldg(A.wg[P][1] + wi) * (A.wv[f][P][1] - xc) : 0.0;
    }
    return fhi - flo;
}

// Row of the sweep along direction P at cell (j, i, k): the matrix entries a
// (lower neighbour), b, cc (upper neighbour), shared by the fields, and the
// right side g[f] of each field.
template <int P, int NF>
__device__ __forceinline__ void adi_row(const AdiArgs& A, i64 c, int j, int i, int k, double& a, double& b,
                                        double& cc, double g[NF]) {
    const Dims& D = A.D;
    const double kap = A.kappa;
    double glo, ghi;          // face coefficients of the implicit part
    double gwl = 0.0, gwh = 0.0;   // wall-face coefficients of value walls
    if constexpr (P == 2) {
        const i64 kp = k == D.nph - 1 ? c - D.nph + 1 : c + 1;
        glo = __ldg(A.G[2] + c);
        ghi = __ldg(A.G[2] + kp);
        a = -kap * glo;
        cc = -kap * ghi;
    } else {
        const int m = P == 0 ? i : j;
        const int n = P == 0 ? D.nth : D.nr;
        const i64 st = P == 0 ? (i64)D.nph : (i64)D.nth * D.nph;
        const i64 wi = P == 0 ? (i64)j * D.nph + k : (i64)i * D.nph + k;
        if (m > 0) {
            glo = __ldg(A.G[P] + c);
            a = -kap * glo;
        } else {
            a = 0.0;
            glo = A.wall[P] ? 2.0 * __ldg(A.wg[P][0] + wi) : 0.0;
            gwl = glo;
        }
        if (m < n - 1) {
            ghi = __ldg(A.G[P] + c + st);
            cc = -kap * ghi;
        } else {
            cc = 0.0;
            ghi = A.wall[P] ? 2.0 * __ldg(A.wg[P][1] + wi) : 0.0;
            gwh = ghi;
        }
    }
    const double Jc = __ldg(A.J + c);
    b = __fma_rn(kap, glo + ghi, Jc);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        double gw = 0.0;   // right-side term of the wall values
        if constexpr (P < 2) gw = __fma_rn(gwh, A.wv[f][P][1], gwl * A.wv[f][P][0]);
        if constexpr (P == 0) {
            double r = Jc * __ldg(A.un[f] + c);
            if (A.src[f]) r += __ldg(A.src[f] + c);
            const double l0 = diag_term<0>(A, f, c, j, i, k);
            const double l12 = diag_term<1>(A, f, c, j, i, k) + diag_term<2>(A, f, c, j, i, k);
            r = __fma_rn(kap, l0, r);
            r = __fma_rn(2.0 * kap, l12, r);
            g[f] = __fma_rn(kap, gw, r);
        } else {
            const double l = diag_term<P>(A, f, c, j, i, k);
            g[f] = __fma_rn(kap, gw, __fma_rn(-kap, l, Jc * A.u[f][c]));
        }
    }
}

// Colatitude and radius sweeps: two threads per line (adjacent lanes) eliminate
// from both ends towards the middle row p = n / 2 (a twisted factorisation:
// top-down x_m = dp_m - cp_m x_{m+1} above, bottom-up x_m = ep_m - ap_m x_{m-1}
// below), exchange their last pivots by a lane shuffle, both solve row p, and
// substitute outwards; the sequential chain is half the line, the thread
// count twice the line count.
template <int P, int NF>
__global__ void __launch_bounds__(kAT) k_adi2(AdiArgs A) {
    static_assert(P < 2, "two-way sweeps are for the walled directions");
    const Dims& D = A.D;
    const i64 nl = P == 0 ? (i64)D.nr * D.nph : (i64)D.nth * D.nph;
    const i64 line = (blockIdx.x * (i64)kAT + threadIdx.x) >> 1;
    const int side = threadIdx.x & 1;   // 0: rows 0 .. p-1 downwards; 1: rows n-1 .. p+1 upwards
    const bool live = line < nl;        // both lanes of a pair share it; every lane reaches the shuffles
    const int n = P == 0 ? D.nth : D.nr;
    const int p = n >> 1;
    const i64 sm = P == 0 ? (i64)D.nph : (i64)D.nth * D.nph;
    int j = 0, i = 0, k = 0;
    i64 base = 0;
    if (live) {
        if (P == 0) {
            j = (int)(line / D.nph);
            k = (int)(line - (i64)j * D.nph);
            base = (i64)j * D.nth * D.nph + k;
        } else {
            i = (int)(line / D.nph);
            k = (int)(line - (i64)i * D.nph);
            base = (i64)i * D.nph + k;
        }
    }
    auto at = [&](int m, int& jj, int& ii, int& kk) {
        jj = P == 1 ? m : j;
        ii = P == 0 ? m : i;
        kk = k;
        return base + (i64)m * sm;
    };
    // elimination towards row p: q = cp (top) or ap (bottom), d[f] = dp or ep
    double q = 0.0, d[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) d[f] = 0.0;
    const int cnt = live ? (side == 0 ? p : n - 1 - p) : 0;
#pragma unroll 2
    for (int t = 0; t < cnt; ++t) {
        const int m = side == 0 ? t : n - 1 - t;
        int jj, ii, kk;
        const i64 c = at(m, jj, ii, kk);
        double a, b, cc, g[NF];
        adi_row<P, NF>(A, c, jj, ii, kk, a, b, cc, g);
        const double toward = side == 0 ? a : cc;   // coupling to the row already eliminated
        const double away = side == 0 ? cc : a;     // coupling to the next row
        const double r = 1.0 / __fma_rn(-toward, q, b);
        q = away * r;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            d[f] = __dmul_rn(__fma_rn(-toward, d[f], g[f]), r);
            A.u[f][c] = d[f];
        }
        A.w[(i64)m * nl + line] = q;
    }
    // row p, read by both lanes before either writes it (__syncwarp below
    // orders those reads before the write)
    int jj, ii, kk;
    const i64 cpv = at(p, jj, ii, kk);
    double a = 0.0, b = 1.0, cc = 0.0, g[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) g[f] = 0.0;
    if (live) adi_row<P, NF>(A, cpv, jj, ii, kk, a, b, cc, g);
    // the partner's last pivot
    const double qo = __shfl_xor_sync(0xffffffffu, q, 1);
    double dother[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) dother[f] = __shfl_xor_sync(0xffffffffu, d[f], 1);
    __syncwarp();
    if (!live) return;
    const double qt = side == 0 ? q : qo, qb = side == 0 ? qo : q;   // cp_{p-1}, ap_{p+1}
    const double r = 1.0 / __fma_rn(-cc, qb, __fma_rn(-a, qt, b));
    double x[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const double dt = side == 0 ? d[f] : dother[f], db = side == 0 ? dother[f] : d[f];
        x[f] = __dmul_rn(__fma_rn(-cc, db, __fma_rn(-a, dt, g[f])), r);
        if (side == 0) A.u[f][cpv] = x[f];
    }
    // substitute outwards from row p
    for (int t = cnt - 1; t >= 0; --t) {
        const int m = side == 0 ? t : n - 1 - t;
        const i64 c = base + (i64)m * sm;
        const double qm = A.w[(i64)m * nl + line];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            x[f] = __fma_rn(-qm, x[f], A.u[f][c]);
            A.u[f][c] = x[f];
        }
    }
}

// Longitude sweep (periodic, Eqs. TAP2-TAP8), two threads per line: the
// leading block A_c (rows 0 .. n-2, corners taken out) is solved by the
// twisted elimination for every field's right side and for the corner column
// (-a_0, 0, .., 0, -c_{n-2}) together (psi1 per field, psi2 shared); the lanes
// swap their end values psi_0 and psi_{n-2}, form psi_{n-1} (Eq. TAP8) and
// add psi2 psi_{n-1} to their own rows (Eq. TAP4).
template <int NF>
__global__ void __launch_bounds__(kAT) k_adi2p(AdiArgs A) {
    const Dims& D = A.D;
    const i64 nl = (i64)D.nr * D.nth;
    const i64 line = (blockIdx.x * (i64)kAT + threadIdx.x) >> 1;
    const int side = threadIdx.x & 1;   // 0: rows 0 .. p-1 downwards; 1: rows n-2 .. p+1 upwards
    const bool live = line < nl;
    const int n = D.nph, nc = n - 1, p = nc >> 1;
    int j = 0, i = 0;
    i64 base = 0;
    if (live) {
        j = (int)(line / D.nth);
        i = (int)(line - (i64)j * D.nth);
        base = line * D.nph;
    }
    double* wq = A.w;                    // pivot ratios of A_c
    double* w2 = A.w + (i64)nc * nl;     // corner column: eliminated, then psi2
    // row m of A_c (corner entries out) and the corner column's entry
    auto row = [&](int m, double& am, double& b, double& cm, double& em, double g[NF]) {
        double a, cc;
        adi_row<2, NF>(A, base + m, j, i, m, a, b, cc, g);
        am = m > 0 ? a : 0.0;
        cm = m < nc - 1 ? cc : 0.0;
        em = (m == 0 ? -a : 0.0) + (m == nc - 1 ? -cc : 0.0);
    };
    double q = 0.0, d2 = 0.0, d[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) d[f] = 0.0;
    const int cnt = live ? (side == 0 ? p : nc - 1 - p) : 0;
#pragma unroll 2
    for (int t = 0; t < cnt; ++t) {
        const int m = side == 0 ? t : nc - 1 - t;
        double am, b, cm, em, g[NF];
        row(m, am, b, cm, em, g);
        const double toward = side == 0 ? am : cm, away = side == 0 ? cm : am;
        const double r = 1.0 / __fma_rn(-toward, q, b);
        q = away * r;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            d[f] = __dmul_rn(__fma_rn(-toward, d[f], g[f]), r);
            A.u[f][base + m] = d[f];
        }
        d2 = __dmul_rn(__fma_rn(-toward, d2, em), r);
        wq[(i64)m * nl + line] = q;
        w2[(i64)m * nl + line] = d2;
    }
    // rows p and n-1, read by both lanes before either writes them
    double ap = 0.0, bp = 1.0, cp = 0.0, ep = 0.0, gp[NF], al = 0.0, bl = 1.0, cl = 0.0, gl[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) gp[f] = gl[f] = 0.0;
    if (live) {
        row(p, ap, bp, cp, ep, gp);
        adi_row<2, NF>(A, base + nc, j, i, nc, al, bl, cl, gl);
    }
    const double qo = __shfl_xor_sync(0xffffffffu, q, 1);
    const double d2o = __shfl_xor_sync(0xffffffffu, d2, 1);
    double dother[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) dother[f] = __shfl_xor_sync(0xffffffffu, d[f], 1);
    __syncwarp();
    const double qt = side == 0 ? q : qo, qb = side == 0 ? qo : q;
    const double rp = 1.0 / __fma_rn(-cp, qb, __fma_rn(-ap, qt, bp));
    double x[NF], x2;
    x2 = __dmul_rn(__fma_rn(-cp, side == 0 ? d2o : d2, __fma_rn(-ap, side == 0 ? d2 : d2o, ep)), rp);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const double dt = side == 0 ? d[f] : dother[f], db = side == 0 ? dother[f] : d[f];
        x[f] = __dmul_rn(__fma_rn(-cp, db, __fma_rn(-ap, dt, gp[f])), rp);
        if (live && side == 0) A.u[f][base + p] = x[f];
    }
    if (live && side == 0) w2[(i64)p * nl + line] = x2;
    // substitute outwards: psi1 into u, psi2 into w2
    for (int t = cnt - 1; t >= 0; --t) {
        const int m = side == 0 ? t : nc - 1 - t;
        const i64 c = base + m;
        const double qm = wq[(i64)m * nl + line];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            x[f] = __fma_rn(-qm, x[f], A.u[f][c]);
            A.u[f][c] = x[f];
        }
        x2 = __fma_rn(-qm, x2, w2[(i64)m * nl + line]);
        w2[(i64)m * nl + line] = x2;
    }
    // the lanes end at psi_0 (top) and psi_{n-2} (bottom; psi_p when it has no rows)
    const double x2o = __shfl_xor_sync(0xffffffffu, x2, 1);
    double xo[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) xo[f] = __shfl_xor_sync(0xffffffffu, x[f], 1);
    if (!live) return;
    const double s20 = side == 0 ? x2 : x2o, s2e = side == 0 ? x2o : x2;
    const double rden = 1.0 / __fma_rn(al, s2e, __fma_rn(cl, s20, bl));
    double last[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const double s10 = side == 0 ? x[f] : xo[f], s1e = side == 0 ? xo[f] : x[f];
        last[f] = __dmul_rn(__fma_rn(-al, s1e, __fma_rn(-cl, s10, gl[f])), rden);
    }
    // Eq. TAP4 on the lane's rows: top 0 .. p, bottom p+1 .. n-2; row n-1 = psi_{n-1}
    const int m0 = side == 0 ? 0 : p + 1, m1 = side == 0 ? p : nc - 1;
    for (int m = m0; m <= m1; ++m) {
        const i64 c = base + m;
        const double s2 = w2[(i64)m * nl + line];
#pragma unroll
        for (int f = 0; f < NF; ++f) A.u[f][c] = __fma_rn(s2, last[f], A.u[f][c]);
    }
    if (side == 0) {
#pragma unroll
        for (int f = 0; f < NF; ++f) A.u[f][base + nc] = last[f];
    }
}

template <int NF>
void launch_sweeps(const AdiArgs& A, cudaStream_t s) {
    const Dims& D = A.D;
    k_adi2<0, NF><<<adi_blocks(2 * (i64)D.nr * D.nph), kAT, 0, s>>>(A);
    k_adi2<1, NF><<<adi_blocks(2 * (i64)D.nth * D.nph), kAT, 0, s>>>(A);
    k_adi2p<NF><<<adi_blocks(2 * (i64)D.nr * D.nth), kAT, 0, s>>>(A);
}

mg_status ensure_adi(mg_handle* h) {
    if (h->adi_w) return MG_OK;
    const Dims& D = h->L[0].D;
    const i64 sz[4] = {(i64)D.nth * D.nph, (i64)D.nth * D.nph, (i64)D.nr * D.nph, (i64)D.nr * D.nph};
    double* g[4];
    for (int q = 0; q < 4; ++q)
        if (!(g[q] = (double*)handle_alloc(h, sizeof(double) * sz[q]))) return MG_ENOMEM;
    double* w = (double*)handle_alloc(h, sizeof(double) * 2 * D.n());
    if (!w) return MG_ENOMEM;
    const cudaError_t e = launch_wall_G(h->mtab, D, g, h->stream);
    if (e != cudaSuccess) {
        set_error(std::string("wall metric: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    for (int q = 0; q < 4; ++q) h->wallG[q] = g[q];
    h->adi_w = w;
    return MG_OK;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mg_status mg_adi_substep(mg_handle* h, double kappa, int nfields, const mg_walls* walls,
                                    const double* const* un, const double* const* src, double* const* u) {
    if (!h || nfields < 1 || !un || !u || !(kappa >= 0.0) || !std::isfinite(kappa)) {
        set_error("mg_adi_substep: null handle or arrays, nfields < 1, or kappa not finite and >= 0");
        return MG_EINVAL;
    }
    for (int f = 0; f < nfields; ++f) {
        bool bad = !un[f] || !u[f];
        for (int e = 0; e < nfields && !bad; ++e) bad = u[f] == un[e] || (src && u[f] == src[e]) || (e != f && u[f] == u[e]);
        const mg_walls* w = walls ? &walls[f] : nullptr;
        if (w) {
            bad = bad || !(w->radius == MG_WALL_FLUX0 || w->radius == MG_WALL_VALUE) ||
                  !(w->colatitude == MG_WALL_FLUX0 || w->colatitude == MG_WALL_VALUE) ||
                  !std::isfinite(w->v_r_in) || !std::isfinite(w->v_r_out) || !std::isfinite(w->v_th0) ||
                  !std::isfinite(w->v_th1) || w->radius != walls[0].radius || w->colatitude != walls[0].colatitude;
        }
        if (bad) {
            set_error("mg_adi_substep: field " + std::to_string(f) +
                      ": null or aliased array, or a bad wall kind or value (kinds must agree across fields)");
            return MG_EINVAL;
        }
    }
    if (h->opts.metric != MG_METRIC_DISCRETE) {
        set_error("mg_adi_substep: the implicit sweeps need the discrete metric of Section 3.2");
        return MG_EINVAL;
    }
    if (cudaEventRecord(h->ev_in, h->user_stream) != cudaSuccess ||
        cudaStreamWaitEvent(h->stream, h->ev_in, 0) != cudaSuccess) {
        set_error("stream join failed");
        return MG_ECUDA;
    }
    mg_status st = ensure_adi(h);
    if (st != MG_OK) return st;
    const Level& L0 = h->L[0];
    AdiArgs A{};
    A.D = L0.D;
    A.G[0] = L0.g64[0];
    A.G[1] = L0.g64[4];
    A.G[2] = L0.g64[8];
    A.J = h->J64;
    A.w = h->adi_w;
    A.kappa = kappa;
    A.wall[0] = walls ? walls[0].colatitude : MG_WALL_VALUE;   // no-slip (value 0) by default
    A.wall[1] = walls ? walls[0].radius : MG_WALL_VALUE;
    A.wg[0][0] = h->wallG[2];
    A.wg[0][1] = h->wallG[3];
    A.wg[1][0] = h->wallG[0];
    A.wg[1][1] = h->wallG[1];
    cudaError_t e = cudaSuccess;
    for (int f0 = 0; f0 < nfields && e == cudaSuccess; f0 += kMaxF) {
        const int nf = std::min(kMaxF, nfields - f0);
        for (int q = 0; q < nf; ++q) {
            const int f = f0 + q;
            A.un[q] = un[f];
            A.src[q] = src ? src[f] : nullptr;
            A.u[q] = u[f];
            if (walls) {
                A.wv[q][0][0] = walls[f].v_th0;
                A.wv[q][0][1] = walls[f].v_th1;
                A.wv[q][1][0] = walls[f].v_r_in;
                A.wv[q][1][1] = walls[f].v_r_out;
            } else {
                A.wv[q][0][0] = A.wv[q][0][1] = A.wv[q][1][0] = A.wv[q][1][1] = 0.0;
            }
        }
        if (nf == 1) launch_sweeps<1>(A, h->stream);
        else if (nf == 2) launch_sweeps<2>(A, h->stream);
        else if (nf == 3) launch_sweeps<3>(A, h->stream);
        else launch_sweeps<4>(A, h->stream);
        e = cudaGetLastError();
        h->launches += 3;
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->user_stream, h->ev_out, 0);
    if (e != cudaSuccess) {
        set_error(std::string("mg_adi_substep: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    return MG_OK;
}

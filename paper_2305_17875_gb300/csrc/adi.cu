// adi.cu - the ADI-CN implicit viscous sweeps of Section 3.4 (Eqs. solve_2 to
// solve_4) for one cell-centred field on a handle's fine grid, FP64.
//
// With kappa = (h / 2) sqrt(Pr / Ra) and L_p the diagonal viscous term of
// direction p (Eq. PC_term1 in flux form; zeta = colatitude i, eta = radius
// j, xi = longitude k):
//   sweep zeta:  (J - kappa L_zeta) u*   = J u^n + s + kappa L_zeta u^n + 2 kappa (L_eta + L_xi) u^n
//   sweep eta:   (J - kappa L_eta)  u**  = J u* - kappa L_eta u^n
//   sweep xi:    (J - kappa L_xi)   u*** = J u** - kappa L_xi u^n     (periodic)
// One launch per sweep, one thread per grid line: the thread forms each row
// of its tridiagonal system from the face metric (G_pp of the row's two faces,
// J) and the stencil of u^n, then eliminates as it goes (normalised Thomas,
// cp kept in a work array laid out [row][line]) and back-substitutes into u.
// Colatitude and radius lines are adjacent in memory along longitude, so
// their loads coalesce; longitude lines are contiguous (one thread walks a
// run of consecutive cells).  Right sides read only the line's own cell of
// the previous sweep's result, so every sweep works in place on u.
//
// Walls: zero flux, or a value held on the wall face half a cell from the
// centre, whose face flux is 2 G_pp(wall face) (u_w - u_c) outward; G_pp of
// the wall faces comes from the face metric (k_wall_G).
#include <cmath>
#include <string>

#include "engine.h"
#include "pc.h"

namespace mgs {
namespace {

constexpr int kAT = 128;

struct AdiArgs {
    Dims D;
    const double* G[3];     // G_pp on the lower p-face of every cell (0 on lower walls)
    const double* J;
    const double* un;
    const double* src;      // may be null
    double* u;              // result; input of the eta and xi sweeps
    double* w;              // 2 N doubles of line-solve work
    double kappa;
    int wall[2];            // per direction 0 (colatitude), 1 (radius): 1 = value, 0 = zero flux
    double wv[2][2];        // wall values [direction][lower, upper]
    const double* wg[2][2]; // wall-face G_pp [direction][lower, upper]: colatitude [nr][nph], radius [nth][nph]
};

// Fluxes of direction p through the lower and upper faces of cell (j, i, k)
// for the field x: interior faces G (x_up - x_down); value walls
// 2 G_w (x_c - x_w) (lower) and 2 G_w (x_w - x_c) (upper); zero-flux walls 0.
template <int P>
__device__ __forceinline__ void face_fluxes(const AdiArgs& A, const double* x, i64 c, int j, int i, int k,
                                            double& flo, double& fhi) {
    const Dims& D = A.D;
    const double xc = __ldg(x + c);
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
        else flo = A.wall[P] ? 2.0 * __ldg(A.wg[P][0] + wi) * (xc - A.wv[P][0]) : 0.0;
        if (m < n - 1) fhi = __ldg(A.G[P] + c + st) * (__ldg(x + c + st) - xc);
        else fhi = A.wall[P] ? 2.0 * __ldg(A.wg[P][1] + wi) * (A.wv[P][1] - xc) : 0.0;
    }
}

template <int P>
__device__ __forceinline__ double diag_term(const AdiArgs& A, const double* x, i64 c, int j, int i, int k) {
    double flo, fhi;
    face_fluxes<P>(A, x, c, j, i, k, flo, fhi);
    return fhi - flo;
}

// Row of the sweep along direction P at cell (j, i, k): a (lower neighbour),
// b, cc (upper neighbour), g (right side).
template <int P>
__device__ __forceinline__ void adi_row(const AdiArgs& A, i64 c, int j, int i, int k, double& a, double& b,
                                        double& cc, double& g) {
    const Dims& D = A.D;
    const double kap = A.kappa;
    double glo, ghi;   // face coefficients of the implicit part
    double gw = 0.0;   // right-side term of the wall values
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
            gw = __fma_rn(glo, A.wv[P][0], gw);
        }
        if (m < n - 1) {
            ghi = __ldg(A.G[P] + c + st);
            cc = -kap * ghi;
        } else {
            cc = 0.0;
            ghi = A.wall[P] ? 2.0 * __ldg(A.wg[P][1] + wi) : 0.0;
            gw = __fma_rn(ghi, A.wv[P][1], gw);
        }
    }
    const double Jc = __ldg(A.J + c);
    b = __fma_rn(kap, glo + ghi, Jc);
    if constexpr (P == 0) {
        double r = Jc * __ldg(A.un + c);
        if (A.src) r += __ldg(A.src + c);
        const double l0 = diag_term<0>(A, A.un, c, j, i, k);
        const double l12 = diag_term<1>(A, A.un, c, j, i, k) + diag_term<2>(A, A.un, c, j, i, k);
        r = __fma_rn(kap, l0, r);
        r = __fma_rn(2.0 * kap, l12, r);
        g = __fma_rn(kap, gw, r);
    } else {
        const double l = diag_term<P>(A, A.un, c, j, i, k);
        g = __fma_rn(kap, gw, __fma_rn(-kap, l, Jc * A.u[c]));
    }
}

template <int P>
__global__ void __launch_bounds__(kAT) k_adi(AdiArgs A) {
    const Dims& D = A.D;
    const i64 line = blockIdx.x * (i64)kAT + threadIdx.x;
    // lines: colatitude (j, k), radius (i, k), longitude (j, i)
    const i64 nl = P == 0 ? (i64)D.nr * D.nph : (P == 1 ? (i64)D.nth * D.nph : (i64)D.nr * D.nth);
    if (line >= nl) return;
    const int n = P == 0 ? D.nth : (P == 1 ? D.nr : D.nph);
    const i64 sm = P == 0 ? (i64)D.nph : (P == 1 ? (i64)D.nth * D.nph : 1);
    int j = 0, i = 0, k = 0;
    i64 base;
    if (P == 0) {
        j = (int)(line / D.nph);
        k = (int)(line - (i64)j * D.nph);
        base = (i64)j * D.nth * D.nph + k;
    } else if (P == 1) {
        i = (int)(line / D.nph);
        k = (int)(line - (i64)i * D.nph);
        base = (i64)i * D.nph + k;
    } else {
        j = (int)(line / D.nth);
        i = (int)(line - (i64)j * D.nth);
        base = line * D.nph;
    }
    double* u = A.u;
    auto at = [&](int m, int& jj, int& ii, int& kk) {
        jj = P == 1 ? m : j;
        ii = P == 0 ? m : i;
        kk = P == 2 ? m : k;
        return base + (i64)m * sm;
    };
    if constexpr (P < 2) {
        double cp = 0.0, dp = 0.0;
#pragma unroll 4
        for (int m = 0; m < n; ++m) {
            int jj, ii, kk;
            const i64 c = at(m, jj, ii, kk);
            double a, b, cc, g;
            adi_row<P>(A, c, jj, ii, kk, a, b, cc, g);
            const double r = 1.0 / __fma_rn(-a, cp, b);
            cp = cc * r;
            dp = __dmul_rn(__fma_rn(-a, dp, g), r);
            u[c] = dp;
            if (m < n - 1) A.w[(i64)m * nl + line] = cp;
        }
        double psi = dp;
        for (int m = n - 2; m >= 0; --m) {
            const i64 c = base + (i64)m * sm;
            psi = __fma_rn(-A.w[(i64)m * nl + line], psi, u[c]);
            u[c] = psi;
        }
    } else {
        // periodic (Eqs. TAP2-TAP8): psi1, psi2 on the leading block share cp;
        // psi1_0, psi2_0 summed during the sweep (see lines.cu)
        const int nc = n - 1;
        double* wcp = A.w;
        double* wd2 = A.w + (i64)nc * nl;
        double cp = 0.0, d1 = 0.0, d2 = 0.0, prod = 1.0, s1 = 0.0, s2 = 0.0;
#pragma unroll 4
        for (int m = 0; m < nc; ++m) {
            int jj, ii, kk;
            const i64 c = at(m, jj, ii, kk);
            double a, b, cc, g;
            adi_row<2>(A, c, jj, ii, kk, a, b, cc, g);
            const double am = m > 0 ? a : 0.0;
            const double em = (m == 0 ? -a : 0.0) + (m == nc - 1 ? -cc : 0.0);
            const double r = 1.0 / __fma_rn(-am, cp, b);
            cp = m < nc - 1 ? cc * r : 0.0;
            d1 = __dmul_rn(__fma_rn(-am, d1, g), r);
            d2 = __dmul_rn(__fma_rn(-am, d2, em), r);
            s1 = __fma_rn(prod, d1, s1);
            s2 = __fma_rn(prod, d2, s2);
            prod = -prod * cp;
            u[c] = d1;
            wd2[(i64)m * nl + line] = d2;
            if (m < nc - 1) wcp[(i64)m * nl + line] = cp;
        }
        int jj, ii, kk;
        const i64 cl = at(nc, jj, ii, kk);
        double al, bl, cl_, gl;
        adi_row<2>(A, cl, jj, ii, kk, al, bl, cl_, gl);
        const double last = __fma_rn(-al, d1, __fma_rn(-cl_, s1, gl)) / __fma_rn(al, d2, __fma_rn(cl_, s2, bl));
        u[cl] = last;
        double psi = __fma_rn(d2, last, d1);
        u[base + (i64)(nc - 1) * sm] = psi;
        for (int m = nc - 2; m >= 0; --m) {
            const i64 c = base + (i64)m * sm;
            const double dm = __fma_rn(wd2[(i64)m * nl + line], last, u[c]);
            psi = __fma_rn(-wcp[(i64)m * nl + line], psi, dm);
            u[c] = psi;
        }
    }
}

unsigned adi_blocks(i64 lines) { return (unsigned)((lines + kAT - 1) / kAT); }

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

extern "C" mg_status mg_adi_substep(mg_handle* h, double kappa, const mg_walls* walls, const double* un,
                                    const double* src, double* u) {
    if (!h || !un || !u || un == u || src == u || !(kappa >= 0.0) || !std::isfinite(kappa)) {
        set_error("mg_adi_substep: null or aliased array, or kappa not finite and >= 0");
        return MG_EINVAL;
    }
    mg_walls wl{};
    wl.radius = wl.colatitude = MG_WALL_VALUE;   // no-slip (u = 0) by default
    if (walls) wl = *walls;
    const bool ok_kind = (wl.radius == MG_WALL_FLUX0 || wl.radius == MG_WALL_VALUE) &&
                         (wl.colatitude == MG_WALL_FLUX0 || wl.colatitude == MG_WALL_VALUE);
    if (!ok_kind || !std::isfinite(wl.v_r_in) || !std::isfinite(wl.v_r_out) || !std::isfinite(wl.v_th0) ||
        !std::isfinite(wl.v_th1)) {
        set_error("mg_adi_substep: bad wall kind or value");
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
    const Dims& D = L0.D;
    AdiArgs A{};
    A.D = D;
    A.G[0] = L0.g64[0];
    A.G[1] = L0.g64[4];
    A.G[2] = L0.g64[8];
    A.J = h->J64;
    A.un = un;
    A.src = src;
    A.u = u;
    A.w = h->adi_w;
    A.kappa = kappa;
    A.wall[0] = wl.colatitude;
    A.wall[1] = wl.radius;
    A.wv[0][0] = wl.v_th0;
    A.wv[0][1] = wl.v_th1;
    A.wv[1][0] = wl.v_r_in;
    A.wv[1][1] = wl.v_r_out;
    A.wg[0][0] = h->wallG[2];
    A.wg[0][1] = h->wallG[3];
    A.wg[1][0] = h->wallG[0];
    A.wg[1][1] = h->wallG[1];
    k_adi<0><<<adi_blocks((i64)D.nr * D.nph), kAT, 0, h->stream>>>(A);
    k_adi<1><<<adi_blocks((i64)D.nth * D.nph), kAT, 0, h->stream>>>(A);
    k_adi<2><<<adi_blocks((i64)D.nr * D.nth), kAT, 0, h->stream>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->user_stream, h->ev_out, 0);
    if (e != cudaSuccess) {
        set_error(std::string("mg_adi_substep: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    h->launches += 3;
    return MG_OK;
}

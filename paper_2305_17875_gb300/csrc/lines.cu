// lines.cu - batched tridiagonal line solves (Section 3.5): the Thomas
// algorithm (Eqs. FIBRE_TA1, FIBRE_TA2) and its periodic variant (Eqs.
// FIBRE_TAP1 to FIBRE_TAP8).
//
// Row m of a line reads a_m psi_{m-1} + b_m psi_m + c_m psi_{m+1} = g_m; a
// periodic line closes the ring (a_0 couples psi_{n-1}, c_{n-1} couples
// psi_0).  Element m of line (l1, l2) sits at l1 s1 + l2 s2 + m sm in every
// array, so the radial, colatitude and longitude lines of an [nr][nth][nph]
// field are all solved in place of the field.  Consecutive threads take
// consecutive l2: lines adjacent in memory (s2 = 1) give coalesced loads;
// for contiguous lines (sm = 1) each thread reads its line in runs of kU
// elements, one or two sectors per array at a time.
//
// Lines take two threads each (a twisted factorisation, k_thomas2 and
// k_thomas2p), except many contiguous ones (one thread each).  The sweep is the normalised form of the
// paper's forward elimination: cp_m = c_m / (b_m - a_m cp_{m-1}),
// dp_m = (g_m - a_m dp_{m-1}) / (same), so back substitution
// psi_m = dp_m - cp_m psi_{m+1} needs only cp and dp (dp is kept in x, cp in
// the work array, laid out [m][line] so that its accesses are coalesced
// whatever the line layout).  Same elimination, same pivots as the paper's
// b'_m = b_m - a_m c_{m-1} / b'_{m-1}.
//
// Periodic lines (Eqs. TAP2 to TAP8): psi1 and psi2 solve the leading
// (n-1)-block with right sides g and (-a_0, 0, .., 0, -c_{n-2}); both share
// cp.  The paper finds psi1_0 and psi2_0 by back substitution before Eq. TAP8
// gives psi_{n-1}; here they are summed during the forward sweep instead
// (back substitution from the top gives psi_0 = sum_m dp_m prod_{k<m} (-cp_k)),
// so psi_{n-1} is known when the sweep ends and a single back substitution
// of dp1 + dp2 psi_{n-1} gives psi = psi1 + psi2 psi_{n-1} (Eq. TAP4).
//
// One IEEE division per row (the hardware's double-precision reciprocal
// approximation plus refinement; a hand-rolled Newton reciprocal from the
// single-precision one measured slower).
#include <algorithm>
#include <string>

#include "engine.h"

namespace mgs {
namespace {

constexpr int kLT = 128;   // threads per block
constexpr int kU = 8;      // rows loaded ahead per thread

struct LineGeom {
    int n;
    i64 n1, n2, nl;
    i64 sm, s1, s2;
};

__device__ __forceinline__ i64 line_base(const LineGeom& L, i64 line) {
    const i64 l1 = line / L.n2;
    return l1 * L.s1 + (line - l1 * L.n2) * L.s2;
}

// Plain lines, one thread per line.  x may alias g (g_m is read before x_m is
// written).
__global__ void __launch_bounds__(kLT) k_thomas(LineGeom L, const double* __restrict__ a,
                                                 const double* __restrict__ b,
                                                 const double* __restrict__ c, const double* g,
                                                 double* x, double* __restrict__ w) {
    const i64 line = blockIdx.x * (i64)kLT + threadIdx.x;
    if (line >= L.nl) return;
    const i64 base = line_base(L, line);
    const int n = L.n;
    double cp = 0.0, dp = 0.0;
    for (int m0 = 0; m0 < n; m0 += kU) {
        const int cnt = min(kU, n - m0);
        double ra[kU], rb[kU], rc[kU], rg[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (u < cnt) {
                const i64 o = base + (i64)(m0 + u) * L.sm;
                const int m = m0 + u;
                ra[u] = m > 0 ? a[o] : 0.0;
                rb[u] = b[o];
                rc[u] = m < n - 1 ? c[o] : 0.0;
                rg[u] = g[o];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (u < cnt) {
                const int m = m0 + u;
                const double r = 1.0 / __fma_rn(-ra[u], cp, rb[u]);
                cp = rc[u] * r;
                dp = __dmul_rn(__fma_rn(-ra[u], dp, rg[u]), r);
                x[base + (i64)m * L.sm] = dp;
                if (m < n - 1) w[(i64)m * L.nl + line] = cp;
            }
        }
    }
    // back substitution; x_{n-1} = dp_{n-1} is already in place
    double psi = dp;
    for (int m = n - 2; m >= 0; --m) {
        const i64 o = base + (i64)m * L.sm;
        psi = __fma_rn(-w[(i64)m * L.nl + line], psi, x[o]);
        x[o] = psi;
    }
}

// Plain lines, two threads per line (adjacent lanes): the top lane eliminates
// rows 0 .. p-1 downwards (x_m = dp_m - cp_m x_{m+1}), the bottom lane rows
// n-1 .. p+1 upwards (x_m = ep_m - ap_m x_{m-1}), p = n / 2; they swap their
// last pivots by a lane shuffle, both solve row p, and substitute outwards (a
// twisted factorisation: half the sequential chain, twice the threads).  The
// work array holds cp at rows 0 .. p-1 and ap at rows p .. n-2 (row m - 1
// for m > p).  x may alias g: every row is read before it is written, row p
// by both lanes before the barrier and written after it.
__global__ void __launch_bounds__(kLT) k_thomas2(LineGeom L, const double* __restrict__ a,
                                                  const double* __restrict__ b,
                                                  const double* __restrict__ c, const double* g,
                                                  double* x, double* __restrict__ w) {
    const i64 line = (blockIdx.x * (i64)kLT + threadIdx.x) >> 1;
    const int side = threadIdx.x & 1;
    const bool live = line < L.nl;
    const i64 base = live ? line_base(L, line) : 0;
    const int n = L.n, p = n >> 1;
    const int cnt = live ? (side == 0 ? p : n - 1 - p) : 0;
    auto wrow = [&](int m) { return (i64)(m > p ? m - 1 : m) * L.nl + line; };
    double q = 0.0, d = 0.0;
    for (int t0 = 0; t0 < cnt; t0 += kU) {
        const int k = min(kU, cnt - t0);
        double rt[kU], rb[kU], ra[kU], rg[kU];   // toward, diagonal, away, right side
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (u < k) {
                const int m = side == 0 ? t0 + u : n - 1 - t0 - u;
                const i64 o = base + (i64)m * L.sm;
                const double am = m > 0 ? a[o] : 0.0, cm = m < n - 1 ? c[o] : 0.0;
                rt[u] = side == 0 ? am : cm;
                ra[u] = side == 0 ? cm : am;
                rb[u] = b[o];
                rg[u] = g[o];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (u < k) {
                const int m = side == 0 ? t0 + u : n - 1 - t0 - u;
                const double r = 1.0 / __fma_rn(-rt[u], q, rb[u]);
                q = ra[u] * r;
                d = __dmul_rn(__fma_rn(-rt[u], d, rg[u]), r);
                x[base + (i64)m * L.sm] = d;
                w[wrow(m)] = q;
            }
        }
    }
    double ap = 0.0, bp = 1.0, cp = 0.0, gp = 0.0;
    const i64 op = base + (i64)p * L.sm;
    if (live) {
        ap = p > 0 ? a[op] : 0.0;
        cp = p < n - 1 ? c[op] : 0.0;
        bp = b[op];
        gp = g[op];
    }
    const double qo = __shfl_xor_sync(0xffffffffu, q, 1);
    const double dother = __shfl_xor_sync(0xffffffffu, d, 1);
    __syncwarp();
    if (!live) return;
    const double qt = side == 0 ? q : qo, qb = side == 0 ? qo : q;
    const double dt = side == 0 ? d : dother, db = side == 0 ? dother : d;
    double xv = __fma_rn(-cp, db, __fma_rn(-ap, dt, gp)) / __fma_rn(-cp, qb, __fma_rn(-ap, qt, bp));
    if (side == 0) x[op] = xv;
    for (int t = cnt - 1; t >= 0; --t) {
        const int m = side == 0 ? t : n - 1 - t;
        const i64 o = base + (i64)m * L.sm;
        xv = __fma_rn(-w[wrow(m)], xv, x[o]);
        x[o] = xv;
    }
}

// Periodic lines (n >= 3).  w holds cp in [0, n-2) and dp2 in [n-1, 2n-2)
// blocks of nl entries.  x may alias g.
__global__ void __launch_bounds__(kLT) k_thomas_periodic(LineGeom L, const double* __restrict__ a,
                                                          const double* __restrict__ b,
                                                          const double* __restrict__ c,
                                                          const double* g, double* x,
                                                          double* __restrict__ w) {
    const i64 line = blockIdx.x * (i64)kLT + threadIdx.x;
    if (line >= L.nl) return;
    const i64 base = line_base(L, line);
    const int n = L.n, nc = n - 1;      // nc rows in the leading block A_c
    double* wcp = w;
    double* wd2 = w + (i64)nc * L.nl;
    double cp = 0.0, d1 = 0.0, d2 = 0.0;
    double prod = 1.0, s1 = 0.0, s2 = 0.0;   // prod_{k<m} (-cp_k); sums giving psi1_0, psi2_0
    for (int m0 = 0; m0 < nc; m0 += kU) {
        const int cnt = min(kU, nc - m0);
        double ra[kU], rb[kU], rc[kU], rg[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (u < cnt) {
                const i64 o = base + (i64)(m0 + u) * L.sm;
                ra[u] = a[o];
                rb[u] = b[o];
                rc[u] = c[o];
                rg[u] = g[o];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (u < cnt) {
                const int m = m0 + u;
                const double am = m > 0 ? ra[u] : 0.0;            // a_0 is a corner, not in A_c
                const double em = (m == 0 ? -ra[u] : 0.0) + (m == nc - 1 ? -rc[u] : 0.0);
                const double r = 1.0 / __fma_rn(-am, cp, rb[u]);
                cp = m < nc - 1 ? rc[u] * r : 0.0;
                d1 = __dmul_rn(__fma_rn(-am, d1, rg[u]), r);
                d2 = __dmul_rn(__fma_rn(-am, d2, em), r);
                s1 = __fma_rn(prod, d1, s1);
                s2 = __fma_rn(prod, d2, s2);
                prod = -prod * cp;
                x[base + (i64)m * L.sm] = d1;
                wd2[(i64)m * L.nl + line] = d2;
                if (m < nc - 1) wcp[(i64)m * L.nl + line] = cp;
            }
        }
    }
    // Eq. TAP8 with psi1_{n-2} = dp1_{n-2}, psi2_{n-2} = dp2_{n-2}
    const i64 ol = base + (i64)nc * L.sm;
    const double al = a[ol], bl = b[ol], cl = c[ol], gl = g[ol];
    const double num = __fma_rn(-al, d1, __fma_rn(-cl, s1, gl));
    const double den = __fma_rn(al, d2, __fma_rn(cl, s2, bl));
    const double last = num / den;
    x[ol] = last;
    // one back substitution of dp1 + dp2 last
    double psi = __fma_rn(d2, last, d1);
    x[base + (i64)(nc - 1) * L.sm] = psi;
    for (int m = nc - 2; m >= 0; --m) {
        const i64 o = base + (i64)m * L.sm;
        const double dm = __fma_rn(wd2[(i64)m * L.nl + line], last, x[o]);
        psi = __fma_rn(-wcp[(i64)m * L.nl + line], psi, dm);
        x[o] = psi;
    }
}

// Periodic lines, two threads per line: the leading block A_c (rows 0 .. n-2,
// corners out) is solved by the twisted elimination for g and for the corner
// column (-a_0, 0, .., 0, -c_{n-2}) together (psi1, psi2); the lanes swap
// their end values psi_0 and psi_{n-2}, form psi_{n-1} (Eq. TAP8) and add
// psi2 psi_{n-1} to their own rows (Eq. TAP4).  w: pivot ratios in rows
// [0, n-1) (row p unused), psi2 in rows [n-1, 2n-2).  x may alias g.
__global__ void __launch_bounds__(kLT) k_thomas2p(LineGeom L, const double* __restrict__ a,
                                                   const double* __restrict__ b,
                                                   const double* __restrict__ c, const double* g,
                                                   double* x, double* __restrict__ w) {
    const i64 line = (blockIdx.x * (i64)kLT + threadIdx.x) >> 1;
    const int side = threadIdx.x & 1;
    const bool live = line < L.nl;
    const i64 base = live ? line_base(L, line) : 0;
    const int n = L.n, nc = n - 1, p = nc >> 1;
    double* wq = w;
    double* w2 = w + (i64)nc * L.nl;
    auto row = [&](int m, double& am, double& bm, double& cm, double& em, double& gm) {
        const i64 o = base + (i64)m * L.sm;
        const double aa = a[o], cc = c[o];
        am = m > 0 ? aa : 0.0;
        cm = m < nc - 1 ? cc : 0.0;
        em = (m == 0 ? -aa : 0.0) + (m == nc - 1 ? -cc : 0.0);
        bm = b[o];
        gm = g[o];
    };
    double q = 0.0, d = 0.0, d2 = 0.0;
    const int cnt = live ? (side == 0 ? p : nc - 1 - p) : 0;
    for (int t = 0; t < cnt; ++t) {
        const int m = side == 0 ? t : nc - 1 - t;
        double am, bm, cm, em, gm;
        row(m, am, bm, cm, em, gm);
        const double toward = side == 0 ? am : cm, away = side == 0 ? cm : am;
        const double r = 1.0 / __fma_rn(-toward, q, bm);
        q = away * r;
        d = __dmul_rn(__fma_rn(-toward, d, gm), r);
        d2 = __dmul_rn(__fma_rn(-toward, d2, em), r);
        x[base + (i64)m * L.sm] = d;
        wq[(i64)m * L.nl + line] = q;
        w2[(i64)m * L.nl + line] = d2;
    }
    // rows p and n-1, read by both lanes before either writes them
    double ap = 0.0, bp = 1.0, cp = 0.0, ep = 0.0, gp = 0.0, al = 0.0, bl = 1.0, cl = 0.0, gl = 0.0;
    const i64 ol = base + (i64)nc * L.sm;
    if (live) {
        row(p, ap, bp, cp, ep, gp);
        al = a[ol];
        bl = b[ol];
        cl = c[ol];
        gl = g[ol];
    }
    const double qo = __shfl_xor_sync(0xffffffffu, q, 1);
    const double dO = __shfl_xor_sync(0xffffffffu, d, 1);
    const double d2o = __shfl_xor_sync(0xffffffffu, d2, 1);
    __syncwarp();
    const double qt = side == 0 ? q : qo, qb = side == 0 ? qo : q;
    const double rp = 1.0 / __fma_rn(-cp, qb, __fma_rn(-ap, qt, bp));
    double xv = __dmul_rn(__fma_rn(-cp, side == 0 ? dO : d, __fma_rn(-ap, side == 0 ? d : dO, gp)), rp);
    double x2 = __dmul_rn(__fma_rn(-cp, side == 0 ? d2o : d2, __fma_rn(-ap, side == 0 ? d2 : d2o, ep)), rp);
    if (live && side == 0) {
        x[base + (i64)p * L.sm] = xv;
        w2[(i64)p * L.nl + line] = x2;
    }
    for (int t = cnt - 1; t >= 0; --t) {
        const int m = side == 0 ? t : nc - 1 - t;
        const i64 o = base + (i64)m * L.sm;
        const double qm = wq[(i64)m * L.nl + line];
        xv = __fma_rn(-qm, xv, x[o]);
        x[o] = xv;
        x2 = __fma_rn(-qm, x2, w2[(i64)m * L.nl + line]);
        w2[(i64)m * L.nl + line] = x2;
    }
    const double xo = __shfl_xor_sync(0xffffffffu, xv, 1);
    const double x2o = __shfl_xor_sync(0xffffffffu, x2, 1);
    if (!live) return;
    const double s10 = side == 0 ? xv : xo, s1e = side == 0 ? xo : xv;
    const double s20 = side == 0 ? x2 : x2o, s2e = side == 0 ? x2o : x2;
    const double last = __fma_rn(-al, s1e, __fma_rn(-cl, s10, gl)) / __fma_rn(al, s2e, __fma_rn(cl, s20, bl));
    const int m0 = side == 0 ? 0 : p + 1, m1 = side == 0 ? p : nc - 1;
    for (int m = m0; m <= m1; ++m) {
        const i64 o = base + (i64)m * L.sm;
        x[o] = __fma_rn(w2[(i64)m * L.nl + line], last, x[o]);
    }
    if (side == 0) x[ol] = last;
}

bool geom_of(const mg_lines* in, int periodic, LineGeom* L) {
    if (!in || in->n < 1 || (periodic && in->n < 3) || in->n1 < 0 || in->n2 < 0) return false;
    L->n = in->n;
    L->n1 = in->n1;
    L->n2 = in->n2;
    L->nl = (i64)in->n1 * in->n2;
    L->sm = in->sm;
    L->s1 = in->s1;
    L->s2 = in->s2;
    return true;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" size_t mg_thomas_work_bytes(const mg_lines* lines, int periodic) {
    LineGeom L;
    if (!geom_of(lines, periodic, &L)) return 0;
    const i64 rows = periodic ? 2 * (i64)(L.n - 1) : (i64)std::max(L.n - 1, 1);
    return (size_t)(rows * L.nl) * sizeof(double);
}

extern "C" mg_status mg_thomas(const mg_lines* lines, const double* a, const double* b, const double* c,
                               const double* g, double* x, double* work, int periodic, void* stream) {
    LineGeom L;
    if (!geom_of(lines, periodic, &L)) {
        set_error(periodic ? "mg_thomas: periodic lines need n >= 3 and n1, n2 >= 0"
                           : "mg_thomas: lines need n >= 1 and n1, n2 >= 0");
        return MG_EINVAL;
    }
    if (L.nl == 0) return MG_OK;
    if (!a || !b || !c || !g || !x || !work) {
        set_error("mg_thomas: null array");
        return MG_EINVAL;
    }
    if (x == a || x == b || x == c || work == x || work == g || work == a || work == b || work == c) {
        set_error("mg_thomas: x and work may not alias the coefficients (x may alias g)");
        return MG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((L.nl + kLT - 1) / kLT);
    // two threads per line where the shorter chain pays (measured): plain
    // lines unless contiguous and numerous; periodic lines (whose twisted form
    // adds a pass) only when contiguous and few
    const bool two = L.sm != 1 || L.nl < 32768;
    if (periodic && L.sm == 1 && L.nl < 32768)
        k_thomas2p<<<(unsigned)((2 * L.nl + kLT - 1) / kLT), kLT, 0, s>>>(L, a, b, c, g, x, work);
    else if (periodic) k_thomas_periodic<<<blocks, kLT, 0, s>>>(L, a, b, c, g, x, work);
    // two threads per line unless the lines are contiguous and numerous (then
    // two lanes streaming far-apart runs of one line cost more than the
    // shorter chain gains: 1.34 vs 1.10 ms for 65536 lines of 512)
    else if (two)
        k_thomas2<<<(unsigned)((2 * L.nl + kLT - 1) / kLT), kLT, 0, s>>>(L, a, b, c, g, x, work);
    else k_thomas<<<blocks, kLT, 0, s>>>(L, a, b, c, g, x, work);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("mg_thomas: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    return MG_OK;
}

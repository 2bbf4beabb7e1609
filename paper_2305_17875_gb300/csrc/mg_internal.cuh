// mg_internal.cuh - device-side building blocks shared by the kernels.
//
// Grid layout: cell (j, i, k) = (radius eta, colatitude zeta, longitude xi) at
// linear index (j * nth + i) * nph + k.  Coefficients are stored per cell as
// the metric rows of its three LOWER faces (structure of arrays):
//   component a = 3 d + q, d = face normal, q = column, both in (zeta, eta, xi)
//   order; e.g. a = 4 is G_eta,eta on the face between (j-1, i, k) and (j, i, k).
// Lower wall faces (i = 0 for zeta, j = 0 for eta) hold zero; upper wall faces
// are not stored and carry no flux either.  Longitude wraps.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mgs {

typedef long long i64;

// Division of 32-bit unsigned n by a fixed d with one high multiply:
// s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1, n / d = (hi32(n m) + n) >> s
// (the round-up method of Granlund and Montgomery, exact for all n < 2^32).
struct FastDiv {
    unsigned d = 1, m = 1, s = 0;
    __host__ __device__ FastDiv() {}
    __host__ __device__ explicit FastDiv(unsigned dd) : d(dd ? dd : 1) {
        s = 0;
        while ((1ull << s) < d) ++s;
        m = (unsigned)((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    }
    __host__ __device__ __forceinline__ unsigned div(unsigned n) const {
#ifdef __CUDA_ARCH__
        const unsigned t = __umulhi(n, m);
#else
        const unsigned t = (unsigned)(((unsigned long long)n * m) >> 32);
#endif
        return (unsigned)(((unsigned long long)t + n) >> s);
    }
};

// Cells per direction, with the divisors the kernels decode indices by.
// Grids hold fewer than 2^31 cells, so linear indices are 32-bit.
struct Dims {
    int nr = 0, nth = 0, nph = 0;
    FastDiv dph, dth, dhk, dq, dth2;   // by nph, nth, nph / 2, nph / 4, (nth + 1) / 2
    int cut = 0;                       // full sphere: colatitude lines joined through the poles
    __host__ __device__ Dims() {}
    __host__ __device__ Dims(int r, int t, int p)
        : nr(r), nth(t), nph(p), dph((unsigned)p), dth((unsigned)t), dhk((unsigned)(p >= 2 ? p / 2 : 1)),
          dq((unsigned)(p >= 4 ? p / 4 : 1)), dth2((unsigned)((t + 1) / 2)) {}
    __host__ __device__ i64 n() const { return (i64)nr * nth * nph; }
};

// Launch clock (profiling): stamp[0] = the earliest start of the launch's
// CTAs (after their grid-dependency wait), stamp[1] = the latest end, on the
// global nanosecond timer; a null stamp records nothing.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void stamp_start(unsigned long long* stamp) {
    if (stamp && threadIdx.x == 0) atomicMin(stamp, global_ns());
}
__device__ __forceinline__ void stamp_end(unsigned long long* stamp) {
    if (stamp && threadIdx.x == 0) atomicMax(stamp + 1, global_ns());
}

// Rows of a level split into groups of four longitude cells (aligned 16-byte
// vectors of FP32) when nph is a multiple of 4; the batched level operations
// then work on whole groups.
__host__ __device__ __forceinline__ bool vec4(const Dims& D) { return (D.nph & 3) == 0; }
// The 19-point colour passes work on groups of four longitudes on walled grids
// of vec4 rows (the full sphere's pole rows take the scalar pass).
__host__ __device__ __forceinline__ bool gs19_groups(const Dims& D) { return vec4(D) && !D.cut; }

struct C3 {
    int j, i, k;
};

__host__ __device__ __forceinline__ int cidx(const Dims& D, int j, int i, int k) {
    return (j * D.nth + i) * D.nph + k;
}
__host__ __device__ __forceinline__ int cidx(const Dims& D, C3 c) { return cidx(D, c.j, c.i, c.k); }

// linear cell index -> (j, i, k)
__host__ __device__ __forceinline__ C3 decode(const Dims& D, i64 cl) {
    const unsigned c = (unsigned)cl;
    const unsigned q = D.dph.div(c);
    const unsigned j = D.dth.div(q);
    C3 r;
    r.k = (int)(c - q * (unsigned)D.nph);
    r.i = (int)(q - j * (unsigned)D.nth);
    r.j = (int)j;
    return r;
}

// work item t of a colour pass (rows of nph / 2 items) -> (kk, i, j)
__host__ __device__ __forceinline__ void decode_half(const Dims& D, i64 tl, int& kk, int& i, int& j) {
    const unsigned t = (unsigned)tl;
    const unsigned row = D.dhk.div(t);
    const unsigned jj = D.dth.div(row);
    kk = (int)(t - row * (unsigned)(D.nph >> 1));
    i = (int)(row - jj * (unsigned)D.nth);
    j = (int)jj;
}

// Neighbour along paper direction q (0 zeta -> i, 1 eta -> j, 2 xi -> k):
// mirror-clamp at the colatitude and radial walls, wrap in longitude.
template <int q>
__device__ __forceinline__ C3 shift(C3 c, int s, const Dims& D) {
    if (q == 0) {
        int v = c.i + s;
        if (D.cut && (v < 0 || v >= D.nth)) {   // across a pole: same row, longitude + nph/2
            const int k = c.k + (D.nph >> 1);
            c.k = k >= D.nph ? k - D.nph : k;
        }
        c.i = v < 0 ? 0 : (v >= D.nth ? D.nth - 1 : v);
    } else if (q == 1) {
        int v = c.j + s;
        c.j = v < 0 ? 0 : (v >= D.nr ? D.nr - 1 : v);
    } else {
        int v = c.k + s;
        c.k = v < 0 ? v + D.nph : (v >= D.nph ? v - D.nph : v);
    }
    return c;
}

// Prolongation of one fine cell on the full sphere (shell cut): cell-centred
// trilinear weights (3/4, 1/4 per halved direction; mirror at the radius
// walls, wrap in longitude) where the colatitude partner of a fine cell in the
// first or last coarse row lies across the pole: the coarse cell of the same
// row at longitude K + nph_c / 2.  Returns the weighted sum of ec, read
// through ld (a functor taking the element's address).
template <typename T, typename LD>
__device__ __forceinline__ T prolong_cut_cell(const Dims& Dc, int cz, int ce, int cx, const T* ec, C3 f, LD ld) {
    int ij[2], ii[2], ik[2];
    float wj[2], wi[2], wk[2];
    bool turn = false;   // the second colatitude partner is across the pole
    auto lin = [](int v, int c, int nc, int mode, int idx[2], float w[2], bool* across) {
        // mode 0 mirror, 1 periodic, 2 cut
        if (c == 1) {
            idx[0] = idx[1] = v;
            w[0] = 1.0f;
            w[1] = 0.0f;
            return;
        }
        const int C = v >> 1;
        int nb = (v & 1) ? C + 1 : C - 1;
        if (mode == 1) {
            nb = nb < 0 ? nb + nc : (nb >= nc ? nb - nc : nb);
        } else if (nb < 0 || nb >= nc) {
            if (mode == 2) *across = true;
            nb = C;
        }
        idx[0] = C;
        idx[1] = nb;
        w[0] = 0.75f;
        w[1] = 0.25f;
    };
    bool dummy = false;
    lin(f.j, ce, Dc.nr, 0, ij, wj, &dummy);
    lin(f.i, cz, Dc.nth, 2, ii, wi, &turn);
    lin(f.k, cx, Dc.nph, 1, ik, wk, &dummy);
    const int half = Dc.nph >> 1;
    T s = 0;
    for (int a = 0; a < ce; ++a)
        for (int bb = 0; bb < cz; ++bb)
            for (int e = 0; e < cx; ++e) {
                int k = ik[e];
                if (turn && bb == 1) k = k + half >= Dc.nph ? k + half - Dc.nph : k + half;
                s = fma((T)wj[a] * (T)wi[bb] * (T)wk[e], ld(ec + cidx(Dc, ij[a], ii[bb], k)), s);
            }
    return s;
}

// ---------------------------------------------------------------- coefficients
// A metric component whose array is absent (null) is zero: the cross terms
// of the 7-point operator, and on an axisymmetric mapping the longitude cross
// terms of the 19-point one (zero to rounding there).
struct CoefF64 {
    const double* g[9];
    __device__ __forceinline__ bool has(int a) const { return g[a] != nullptr; }
    __device__ __forceinline__ double operator()(int a, i64 idx) const { return __ldg(g[a] + idx); }
    // four consecutive cells from idx (a multiple of 4)
    __device__ __forceinline__ void load4(int a, int idx, double v[4]) const {
        const double2 p = __ldg(reinterpret_cast<const double2*>(g[a] + idx));
        const double2 q = __ldg(reinterpret_cast<const double2*>(g[a] + idx) + 1);
        v[0] = p.x, v[1] = p.y, v[2] = q.x, v[3] = q.y;
    }
};
struct CoefF32 {
    const float* g[9];
    __device__ __forceinline__ bool has(int a) const { return g[a] != nullptr; }
    __device__ __forceinline__ float operator()(int a, i64 idx) const { return __ldg(g[a] + idx); }
    __device__ __forceinline__ void load4(int a, int idx, float v[4]) const {
        const float4 p = __ldg(reinterpret_cast<const float4*>(g[a] + idx));
        v[0] = p.x, v[1] = p.y, v[2] = p.z, v[3] = p.w;
    }
};
// FP16 storage, FP32 arithmetic: value = half * s[a] (s a power of two per level
// and component, chosen so the largest magnitude lands in [2^13, 2^14)).
struct CoefF16 {
    const __half* g[9];
    float s[9];
    __device__ __forceinline__ bool has(int a) const { return g[a] != nullptr; }
    __device__ __forceinline__ float operator()(int a, i64 idx) const {
        return __half2float(__ldg(g[a] + idx)) * s[a];
    }
    __device__ __forceinline__ void load4(int a, int idx, float v[4]) const {
        const uint2 p = __ldg(reinterpret_cast<const uint2*>(g[a] + idx));
        const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&p.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&p.y));
        v[0] = lo.x * s[a], v[1] = lo.y * s[a], v[2] = hi.x * s[a], v[3] = hi.y * s[a];
    }
};

template <typename T>
struct XRead {
    const T* x;
    Dims D;
    __device__ __forceinline__ T operator()(C3 c) const { return x[cidx(D, c)]; }
};

// ---------------------------------------------------------------- Eqs. PC_term1-3
// Flux through the face between L and U = L + e_d, with the metric row of U's
// lower d-face:  F = G_dd (x_U - x_L)
//                  + sum_{q != d} G_dq / 4 [ (x_{L+q} + x_{U+q}) - (x_{L-q} + x_{U-q}) ].
// The per-cell arithmetic is written as explicit multiply-add chains, so every
// kernel that evaluates a cell (whatever the compiler would contract) rounds
// identically and all schedules of a solve give the same bits.
template <int d, int q, typename T, typename XA>
__device__ __forceinline__ T cross_diff(const XA& X, const Dims& D, C3 L, C3 U) {
    const T plus = X(shift<q>(L, +1, D)) + X(shift<q>(U, +1, D));
    const T minus = X(shift<q>(L, -1, D)) + X(shift<q>(U, -1, D));
    return plus - minus;
}

// acc + sgn F for the face (L, U)
template <int S, int d, typename T, typename CF, typename XA>
__device__ __forceinline__ T add_flux(T acc, T sgn, const CF& cf, const XA& X, const Dims& D, C3 L, C3 U) {
    const i64 u = cidx(D, U);
    acc = fma(sgn * (T)cf(4 * d, u), X(U) - X(L), acc);   // 4 d = 3 d + d
    if (S == 19) {
        if (d != 0 && cf.has(3 * d + 0)) acc = fma(sgn * (T)0.25 * (T)cf(3 * d + 0, u), cross_diff<d, 0, T>(X, D, L, U), acc);
        if (d != 1 && cf.has(3 * d + 1)) acc = fma(sgn * (T)0.25 * (T)cf(3 * d + 1, u), cross_diff<d, 1, T>(X, D, L, U), acc);
        if (d != 2 && cf.has(3 * d + 2)) acc = fma(sgn * (T)0.25 * (T)cf(3 * d + 2, u), cross_diff<d, 2, T>(X, D, L, U), acc);
    }
    return acc;
}

// (A x)_c = sum_d F_d(c + 1/2 e_d) - F_d(c - 1/2 e_d); wall faces carry no flux.
template <int S, typename T, typename CF, typename XA>
__device__ __forceinline__ T apply_cell(const CF& cf, const XA& X, const Dims& D, C3 c) {
    T acc = 0;
    if (c.j > 0) acc = add_flux<S, 1>(acc, (T)-1, cf, X, D, shift<1>(c, -1, D), c);
    if (c.j < D.nr - 1) acc = add_flux<S, 1>(acc, (T)1, cf, X, D, c, shift<1>(c, +1, D));
    if (c.i > 0) acc = add_flux<S, 0>(acc, (T)-1, cf, X, D, shift<0>(c, -1, D), c);
    if (c.i < D.nth - 1) acc = add_flux<S, 0>(acc, (T)1, cf, X, D, c, shift<0>(c, +1, D));
    acc = add_flux<S, 2>(acc, (T)-1, cf, X, D, shift<2>(c, -1, D), c);
    acc = add_flux<S, 2>(acc, (T)1, cf, X, D, c, shift<2>(c, +1, D));
    return acc;
}

// The coefficient rows of one cell's six faces as the formulas below read
// them: face 0 = the cell's own (lower-face) rows, 1 / 2 / 3 = the rows of the
// next cell along radius / colatitude / longitude (the cell's upper faces).
// CellRows reads them from the coefficient arrays; the one-pass sweeps hand
// over rows already loaded into registers through the same interface, so the
// arithmetic is one piece of code.
template <typename CF>
struct CellRows {
    const CF& cf;
    i64 self, eu, zu, xu;
    __device__ __forceinline__ bool has(int a) const { return cf.has(a); }
    template <int F>
    __device__ __forceinline__ auto at(int a) const {
        return cf(a, F == 0 ? self : (F == 1 ? eu : (F == 2 ? zu : xu)));
    }
};
template <typename CF>
__device__ __forceinline__ CellRows<CF> cell_rows(const CF& cf, const Dims& D, C3 c) {
    const i64 self = cidx(D, c);
    return CellRows<CF>{cf, self, c.j < D.nr - 1 ? cidx(D, c.j + 1, c.i, c.k) : self,
                        c.i < D.nth - 1 ? cidx(D, c.j, c.i + 1, c.k) : self,
                        cidx(D, c.j, c.i, c.k + 1 == D.nph ? 0 : c.k + 1)};
}

// Face rows of one cell held in registers: v[1 + a] = component a of the
// cell's own rows, v[10 + q] = component 3 + q of the radius-upper row,
// v[13 + q] = component q of the colatitude-upper row, v[16 + q] = component
// 6 + q of the longitude-upper row (v[0] is free: the callers keep b there),
// read by the formulas below through CellRows' interface.  AXI: the
// longitude cross components 2, 5, 6, 7 are not stored.
template <typename T, bool AXI>
struct RegRows {
    const T* v;
    __device__ __forceinline__ static constexpr bool stored(int a) {
        return !AXI || (a != 2 && a != 5 && a != 6 && a != 7);
    }
    __device__ __forceinline__ bool has(int a) const { return stored(a); }
    template <int F>
    __device__ __forceinline__ T at(int a) const {
        return F == 0 ? v[1 + a] : (F == 1 ? v[10 + a - 3] : (F == 2 ? v[13 + a] : v[16 + a - 6]));
    }
};

template <int S, typename T, typename R>
__device__ __forceinline__ T diag_cell_r(const R& cr, const Dims& D, C3 c) {
    T dg = 0;
    // lower/upper coefficient rows of the six faces (upper = neighbour's lower row)
    const bool hasEl = c.j > 0, hasEu = c.j < D.nr - 1;
    const bool hasZl = c.i > 0, hasZu = c.i < D.nth - 1;
    if (hasEl) dg -= (T)cr.template at<0>(4);
    if (hasEu) dg -= (T)cr.template at<1>(4);
    if (hasZl) dg -= (T)cr.template at<0>(0);
    if (hasZu) dg -= (T)cr.template at<2>(0);
    dg -= (T)cr.template at<0>(8);
    dg -= (T)cr.template at<3>(8);
    if (S == 19) {
        // mirrored-onto-self weight along q: +1 at the top wall, -1 at the
        // bottom (none in colatitude on the full sphere: the neighbour beyond
        // a pole row is the cell across the pole)
        const T sz = D.cut ? (T)0 : (T)((c.i == D.nth - 1) - (c.i == 0));   // q = zeta
        const T se = (T)((c.j == D.nr - 1) - (c.j == 0));    // q = eta
        if (sz != (T)0) {
            T w = 0;
            if (hasEu) w += (T)cr.template at<1>(3);     // eta faces, column zeta
            if (hasEl) w -= (T)cr.template at<0>(3);
            if (cr.has(6)) {
                w += (T)cr.template at<3>(6);             // xi faces, column zeta
                w -= (T)cr.template at<0>(6);
            }
            dg = fma((T)0.25 * sz, w, dg);
        }
        if (se != (T)0) {
            T w = 0;
            if (hasZu) w += (T)cr.template at<2>(1);     // zeta faces, column eta
            if (hasZl) w -= (T)cr.template at<0>(1);
            if (cr.has(7)) {
                w += (T)cr.template at<3>(7);             // xi faces, column eta
                w -= (T)cr.template at<0>(7);
            }
            dg = fma((T)0.25 * se, w, dg);
        }
    }
    return dg;
}

// Exact diagonal A_cc of the operator above.  Besides -sum of the six G_dd, a
// cross term reaches x_c itself when a tangential neighbour is mirrored onto c
// at a wall: +G_dq/4 at an upper face and -G_dq/4 at a lower face when c is
// on the top wall in q, with opposite signs on the bottom wall.
template <int S, typename T, typename CF>
__device__ __forceinline__ T diag_cell(const CF& cf, const Dims& D, C3 c) {
    return diag_cell_r<S, T>(cell_rows(cf, D, c), D, c);
}

// ---------------------------------------------------------------- 7-point fast path
// The 7-point operator at cell c = (j, i, k) from one base index: neighbours
// at c -/+ 1 (longitude, wrapped), c -/+ nph (colatitude), c -/+ nth*nph
// (radius).  Lower wall faces store G = 0 and upper wall faces are not read;
// a neighbour across a wall is replaced by x_c, which meets a zero
// coefficient.  Same operator as apply_cell with S = 7 (Eq. PC_term1 in each
// direction); each coefficient is loaded once for A x and the diagonal.
// (A x)_c of the 7-point operator from the six neighbour values and face
// coefficients, as one explicit multiply-add chain (see apply_cell).
template <typename T>
__device__ __forceinline__ T ax7(T xc, T xjm, T xjp, T xim, T xip, T xkm, T xkp, T el, T eu, T zl, T zu, T xl,
                                 T xu) {
    T a = eu * (xjp - xc);
    a = fma(-el, xc - xjm, a);
    a = fma(zu, xip - xc, a);
    a = fma(-zl, xc - xim, a);
    a = fma(xu, xkp - xc, a);
    a = fma(-xl, xc - xkm, a);
    return a;
}

template <typename T>
struct Cell7 {
    int c;
    T xc, xjm, xjp, xim, xip, xkm, xkp;   // x at c and its six neighbours
    T el, eu, zl, zu, xl, xu;            // G of the six faces
    template <typename CF, typename XL>
    __device__ __forceinline__ void load(const CF& cf, const Dims& D, int j, int i, int k, const XL& X) {
        const int plane = D.nth * D.nph;
        c = (j * D.nth + i) * D.nph + k;
        const int km = k == 0 ? c + D.nph - 1 : c - 1;
        const int kp = k == D.nph - 1 ? c - D.nph + 1 : c + 1;
        const bool jl = j > 0, ju = j + 1 < D.nr, il = i > 0, iu = i + 1 < D.nth;
        xc = X(c);
        el = (T)cf(4, c);
        eu = ju ? (T)cf(4, c + plane) : (T)0;
        zl = (T)cf(0, c);
        zu = iu ? (T)cf(0, c + D.nph) : (T)0;
        xl = (T)cf(8, c);
        xu = (T)cf(8, kp);
        xjm = jl ? X(c - plane) : xc;
        xjp = ju ? X(c + plane) : xc;
        xim = il ? X(c - D.nph) : xc;
        xip = iu ? X(c + D.nph) : xc;
        xkm = X(km);
        xkp = X(kp);
    }
    __device__ __forceinline__ T ax() const {
        return ax7(xc, xjm, xjp, xim, xip, xkm, xkp, el, eu, zl, zu, xl, xu);
    }
    __device__ __forceinline__ T diag() const { return -(el + eu + zl + zu + xl + xu); }
    // Gauss-Seidel / Jacobi step x_c + (b - A x)_c / A_cc
    __device__ __forceinline__ T gs(T b) const { return xc + (b - ax()) / diag(); }
    // b - A x with the centre coefficient a0 = A_cc stored: seven multiply-adds
    __device__ __forceinline__ T resid_rows(T b, T a0) const {
        T r = fma(-a0, xc, b);
        r = fma(-el, xjm, r);
        r = fma(-eu, xjp, r);
        r = fma(-zl, xim, r);
        r = fma(-zu, xip, r);
        r = fma(-xl, xkm, r);
        r = fma(-xu, xkp, r);
        return r;
    }
    // b - A x with every face term fused into one multiply-add
    __device__ __forceinline__ T resid(T b) const {
        T r = b;
        r = fma(el, xc - xjm, r);
        r = fma(eu, xc - xjp, r);
        r = fma(zl, xc - xim, r);
        r = fma(zu, xc - xip, r);
        r = fma(xl, xc - xkm, r);
        r = fma(xu, xc - xkp, r);
        return r;
    }
};

// ---------------------------------------------------------------- assembled rows
// The operator row of a cell as explicit coefficients on its neighbour cells,
// for the FP64 outer residual, which is FP64-issue bound: 19 multiply-adds per
// cell instead of about 80 FP64 instructions of the face form.  Order of the
// 19 neighbours (dj, di, dk): centre, -/+ radius, -/+ colatitude, -/+
// longitude, then the radius-colatitude, radius-longitude and
// colatitude-longitude edges, each as (-,-), (-,+), (+,-), (+,+).  A neighbour
// beyond a wall has coefficient 0 (its mirrored contributions sit on the cell
// it is mirrored onto); on the full sphere a neighbour beyond a pole row is
// the cell across the pole (across_pole) and keeps its own coefficient.  The 7-point row stores only the centre; its six face
// coefficients are the G arrays themselves.
__host__ __device__ constexpr int row_off(int n, int axis) {   // axis 0 radius, 1 colatitude, 2 longitude
    if (n == 0) return 0;
    if (n <= 6) return (n - 1) / 2 == axis ? (((n - 1) & 1) ? 1 : -1) : 0;
    const int g = (n - 7) / 4, m = (n - 7) & 3;
    const int a0 = g == 2 ? 1 : 0, a1 = g == 0 ? 1 : 2;
    if (axis == a0) return (m >> 1) ? 1 : -1;
    if (axis == a1) return (m & 1) ? 1 : -1;
    return 0;
}

// Entry of the 19-point neighbourhood at offset (dj, di, dk), in row_off order.
__host__ __device__ constexpr int row_index(int dj, int di, int dk) {
    return (dj == 0 && di == 0 && dk == 0) ? 0
           : (di == 0 && dk == 0)          ? (dj < 0 ? 1 : 2)
           : (dj == 0 && dk == 0)          ? (di < 0 ? 3 : 4)
           : (dj == 0 && di == 0)          ? (dk < 0 ? 5 : 6)
           : dk == 0                        ? 7 + 2 * (dj > 0) + (di > 0)
           : di == 0                        ? 11 + 2 * (dj > 0) + (dk > 0)
                                            : 15 + 2 * (di > 0) + (dk > 0);
}

// The cell across a pole of the shell cut for the 19-point neighbour at
// colatitude offset di of a cell in the first or last row: the same row,
// radius j + dj (mirrored at the radial walls), longitude k + dk + nph/2.
// Its place in a pole-row copy laid out [side][j][k] (side 0: row 0, 1: row
// nth - 1) is returned in *pole.
__device__ __forceinline__ bool across_pole(const Dims& D, C3 p, int dj, int di, int dk, int* cell, int* pole) {
    if (!D.cut || di == 0 || (di < 0 && p.i > 0) || (di > 0 && p.i + 1 < D.nth)) return false;
    const int j = (p.j + dj < 0 || p.j + dj >= D.nr) ? p.j : p.j + dj;
    int k = p.k + dk + (D.nph >> 1);
    k = k < 0 ? k + D.nph : (k >= D.nph ? k - D.nph : k);
    *cell = (j * D.nth + p.i) * D.nph + k;
    *pole = ((di < 0 ? 0 : 1) * D.nr + j) * D.nph + k;
    return true;
}

// x on the 19-point neighbourhood of cell c, with the operator's neighbour
// rules: mirror (clamp) at the radial and colatitude walls, wrap in longitude,
// and on the full sphere the cell across the pole beyond the first and last
// colatitude rows.
template <typename T>
struct Nbr19 {
    T v[19];
    // axi: the longitude cross terms are absent, so the eight edges with a
    // longitude offset and a radial or colatitude offset are not read (zero).
    // poles: a copy of the first and last rows of x taken before a colour pass
    // (the values every cell of the pass must see across the pole), or null.
    template <typename XL>
    __device__ __forceinline__ void load(const XL& X, const Dims& D, int c, C3 p, bool axi,
                                         const T* poles = nullptr) {
        const int plane = D.nth * D.nph;
        const int oj[3] = {p.j > 0 ? -plane : 0, 0, p.j + 1 < D.nr ? plane : 0};
        const int oi[3] = {p.i > 0 ? -D.nph : 0, 0, p.i + 1 < D.nth ? D.nph : 0};
        const int ok[3] = {p.k > 0 ? -1 : D.nph - 1, 0, p.k + 1 < D.nph ? 1 : 1 - D.nph};
#pragma unroll
        for (int n = 0; n < 19; ++n) {
            const bool phi_edge = row_off(n, 2) != 0 && (row_off(n, 0) != 0 || row_off(n, 1) != 0);
            v[n] = (axi && phi_edge) ? (T)0
                                     : X(c + oj[row_off(n, 0) + 1] + oi[row_off(n, 1) + 1] + ok[row_off(n, 2) + 1]);
        }
        if (D.cut && (p.i == 0 || p.i + 1 == D.nth)) pole_row(X, D, p, axi, poles);
    }
    // the entries across the pole of a first or last row (full sphere), kept
    // apart from the common path
    template <typename XL>
    __device__ __forceinline__ void pole_row(const XL& X, const Dims& D, C3 p, bool axi, const T* poles) {
#pragma unroll
        for (int n = 3; n < 19; ++n) {   // (unrolled: v stays in registers)
            const bool phi_edge = row_off(n, 2) != 0 && (row_off(n, 0) != 0 || row_off(n, 1) != 0);
            int cell, pole;
            if (!(axi && phi_edge) && across_pole(D, p, row_off(n, 0), row_off(n, 1), row_off(n, 2), &cell, &pole))
                v[n] = poles ? poles[pole] : X(cell);
        }
    }
    // value at offset a along paper direction da and b along direction db
    // (directions 0 zeta -> i, 1 eta -> j, 2 xi -> k)
    template <int da, int a, int db, int b>
    __device__ __forceinline__ T at() const {
        constexpr int dj = (da == 1 ? a : 0) + (db == 1 ? b : 0);
        constexpr int di = (da == 0 ? a : 0) + (db == 0 ? b : 0);
        constexpr int dk = (da == 2 ? a : 0) + (db == 2 ? b : 0);
        return v[row_index(dj, di, dk)];
    }
};

// acc + sgn F for the lower (side -1) or upper (side +1) d-face of the cell,
// from registers: the arithmetic of add_flux step by step (same bits).  F is
// the face's row in the cell's rows (0 for a lower face).
template <int d, int side, int F, typename T, typename R>
__device__ __forceinline__ T add_flux19(T acc, const R& cr, const Nbr19<T>& X) {
    constexpr int sL = side < 0 ? -1 : 0, sU = side < 0 ? 0 : 1;
    const T sgn = (T)side;
    acc = fma(sgn * (T)cr.template at<F>(4 * d), X.template at<d, sU, d, 0>() - X.template at<d, sL, d, 0>(), acc);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q == d || !cr.has(3 * d + q)) continue;
        T plus, minus;
        if (q == 0) {
            plus = X.template at<d, sL, 0, 1>() + X.template at<d, sU, 0, 1>();
            minus = X.template at<d, sL, 0, -1>() + X.template at<d, sU, 0, -1>();
        } else if (q == 1) {
            plus = X.template at<d, sL, 1, 1>() + X.template at<d, sU, 1, 1>();
            minus = X.template at<d, sL, 1, -1>() + X.template at<d, sU, 1, -1>();
        } else {
            plus = X.template at<d, sL, 2, 1>() + X.template at<d, sU, 2, 1>();
            minus = X.template at<d, sL, 2, -1>() + X.template at<d, sU, 2, -1>();
        }
        acc = fma(sgn * (T)0.25 * (T)cr.template at<F>(3 * d + q), plus - minus, acc);
    }
    return acc;
}

// (A x)_c of the 19-point operator from the loaded neighbourhood and the
// cell's face rows; equal bit for bit to apply_cell<19>.
template <typename T, typename R>
__device__ __forceinline__ T apply19_r(const R& cr, const Nbr19<T>& X, const Dims& D, C3 p) {
    T acc = 0;
    if (p.j > 0) acc = add_flux19<1, -1, 0>(acc, cr, X);
    if (p.j < D.nr - 1) acc = add_flux19<1, 1, 1>(acc, cr, X);
    if (p.i > 0) acc = add_flux19<0, -1, 0>(acc, cr, X);
    if (p.i < D.nth - 1) acc = add_flux19<0, 1, 2>(acc, cr, X);
    acc = add_flux19<2, -1, 0>(acc, cr, X);
    acc = add_flux19<2, 1, 3>(acc, cr, X);
    return acc;
}

template <typename T, typename CF>
__device__ __forceinline__ T apply19(const CF& cf, const Nbr19<T>& X, const Dims& D, int c, C3 p) {
    const int plane = D.nth * D.nph;
    const CellRows<CF> cr{cf, c, c + plane, c + D.nph, p.k + 1 < D.nph ? c + 1 : c + 1 - D.nph};
    return apply19_r<T>(cr, X, D, p);
}

// resid_rows19 for a first or last row of the full sphere: the entries
// beyond the row are the cells across the pole (same multiply-add order).
static __device__ __noinline__ double resid_rows19_pole(const double* __restrict__ a, i64 N, const double* __restrict__ x,
                                                        const Dims& D, int c, C3 p, double b, int nrows) {
    const int plane = D.nth * D.nph;
    const int oj[3] = {p.j > 0 ? -plane : 0, 0, p.j + 1 < D.nr ? plane : 0};
    const int oi[3] = {p.i > 0 ? -D.nph : 0, 0, p.i + 1 < D.nth ? D.nph : 0};
    const int ok[3] = {p.k > 0 ? -1 : D.nph - 1, 0, p.k + 1 < D.nph ? 1 : 1 - D.nph};
    double r = b;
    for (int n = 0; n < nrows; ++n) {
        int o = oj[row_off(n, 0) + 1] + oi[row_off(n, 1) + 1] + ok[row_off(n, 2) + 1];
        int cell, pole;
        if (across_pole(D, p, row_off(n, 0), row_off(n, 1), row_off(n, 2), &cell, &pole)) o = cell - c;
        r = fma(-__ldcs(a + n * N + c), __ldg(x + c + o), r);
    }
    return r;
}

// b_c - (A x)_c from the assembled coefficients a[n * N + c] (row_off order;
// nrows = 19, or 11 when the longitude edges 11..18 are absent).
__device__ __forceinline__ double resid_rows19(const double* __restrict__ a, i64 N, const double* __restrict__ x,
                                               const Dims& D, int c, C3 p, double b, int nrows) {
    const int plane = D.nth * D.nph;
    const int oj[3] = {p.j > 0 ? -plane : 0, 0, p.j + 1 < D.nr ? plane : 0};
    const int oi[3] = {p.i > 0 ? -D.nph : 0, 0, p.i + 1 < D.nth ? D.nph : 0};
    const int ok[3] = {p.k > 0 ? -1 : D.nph - 1, 0, p.k + 1 < D.nph ? 1 : 1 - D.nph};
    if (D.cut && (p.i == 0 || p.i + 1 == D.nth)) return resid_rows19_pole(a, N, x, D, c, p, b, nrows);
    double r = b;
#pragma unroll
    for (int n = 0; n < 19; ++n) {
        if (n >= nrows) break;
        const int o = oj[row_off(n, 0) + 1] + oi[row_off(n, 1) + 1] + ok[row_off(n, 2) + 1];
        r = fma(-__ldcs(a + n * N + c), __ldg(x + c + o), r);
    }
    return r;
}

// ---------------------------------------------------------------- IEEE-754 conversions
// Conversions by exponent arithmetic.  FP64 instructions issue at a small
// fraction of the FP32 rate on this GPU, so the FP64 <-> FP32
// conversions of the outer loop are done on the integer pipes: exact
// re-biasing of the exponent, and round-to-nearest-even of the 29 dropped
// mantissa bits.  Zero, subnormal, infinite and NaN inputs, and results
// outside the normal range, take the hardware conversion.

// k with s = 2^k, for s a normal power of two (the residual scales).
__device__ __forceinline__ int pow2_exponent(double s) {
    return (int)((__double_as_longlong(s) >> 52) & 0x7ff) - 1023;
}

// The rare cases, kept out of line so the common path is not predicated
// through them.
static __device__ __noinline__ double widen_slow(float f, int k) { return ldexp((double)f, k); }
static __device__ __noinline__ float narrow_slow(double d) { return __double2float_rn(d); }

// (double)f * 2^k, exact.
__device__ __forceinline__ double scaled_widen(float f, int k) {
    const unsigned u = __float_as_uint(f);
    const int ef = (int)((u >> 23) & 0xff);
    const int ed = ef + (1023 - 127) + k;
    if (ef == 0 || ef == 0xff || ed <= 0 || ed >= 0x7ff) return widen_slow(f, k);
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)ed << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// (float)d, round to nearest even.
__device__ __forceinline__ float narrow_rn(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((u >> 52) & 0x7ff);
    const int ef = e - (1023 - 127);
    if (ef <= 0 || ef >= 0xff) return narrow_slow(d);
    const unsigned long long m = u & 0xfffffffffffffull;
    const unsigned rest = (unsigned)(m & 0x1fffffffu);   // the 29 dropped bits
    unsigned bits = ((unsigned)(u >> 63) << 31) | ((unsigned)ef << 23) | (unsigned)(m >> 29);
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ? 1u : 0u;   // carries into the exponent
    return __uint_as_float(bits);
}

template <typename T>
struct XLin {   // x by linear index
    const T* x;
    __device__ __forceinline__ T operator()(int c) const { return x[c]; }
};

// ---------------------------------------------------------------- reductions
// Fixed-shape block sum (blockDim.x = 256); deterministic for a given launch.
template <typename T>
__device__ __forceinline__ T block_sum_256(T v, T* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < 8 ? sh[threadIdx.x] : (T)0;
        for (int o = 4; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;   // valid in thread 0
}

}  // namespace mgs

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
    FastDiv dph, dth, dhk;   // by nph, by nth, by nph / 2
    __host__ __device__ Dims() {}
    __host__ __device__ Dims(int r, int t, int p)
        : nr(r), nth(t), nph(p), dph((unsigned)p), dth((unsigned)t), dhk((unsigned)(p >= 2 ? p / 2 : 1)) {}
    __host__ __device__ i64 n() const { return (i64)nr * nth * nph; }
};

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

// ---------------------------------------------------------------- coefficients
struct CoefF64 {
    const double* g[9];
    __device__ __forceinline__ double operator()(int a, i64 idx) const { return __ldg(g[a] + idx); }
};
struct CoefF32 {
    const float* g[9];
    __device__ __forceinline__ float operator()(int a, i64 idx) const { return __ldg(g[a] + idx); }
};
// FP16 storage, FP32 arithmetic: value = half * s[a] (s a power of two per level
// and component, chosen so the largest magnitude lands in [2^13, 2^14)).
struct CoefF16 {
    const __half* g[9];
    float s[9];
    __device__ __forceinline__ float operator()(int a, i64 idx) const {
        return __half2float(__ldg(g[a] + idx)) * s[a];
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
template <int S, int d, int q, typename T, typename CF, typename XA>
__device__ __forceinline__ T cross_term(const CF& cf, const XA& X, const Dims& D, C3 L, C3 U, i64 u) {
    T w = (T)0.25 * (T)cf(3 * d + q, u);
    T plus = X(shift<q>(L, +1, D)) + X(shift<q>(U, +1, D));
    T minus = X(shift<q>(L, -1, D)) + X(shift<q>(U, -1, D));
    return w * (plus - minus);
}

template <int S, int d, typename T, typename CF, typename XA>
__device__ __forceinline__ T face_flux(const CF& cf, const XA& X, const Dims& D, C3 L, C3 U) {
    const i64 u = cidx(D, U);
    T F = (T)cf(4 * d, u) * (X(U) - X(L));           // 4 d = 3 d + d
    if (S == 19) {
        if (d != 0) F += cross_term<S, d, 0, T>(cf, X, D, L, U, u);
        if (d != 1) F += cross_term<S, d, 1, T>(cf, X, D, L, U, u);
        if (d != 2) F += cross_term<S, d, 2, T>(cf, X, D, L, U, u);
    }
    return F;
}

// (A x)_c = sum_d F_d(c + 1/2 e_d) - F_d(c - 1/2 e_d); wall faces carry no flux.
template <int S, typename T, typename CF, typename XA>
__device__ __forceinline__ T apply_cell(const CF& cf, const XA& X, const Dims& D, C3 c) {
    T acc = 0;
    if (c.j > 0) acc -= face_flux<S, 1, T>(cf, X, D, shift<1>(c, -1, D), c);
    if (c.j < D.nr - 1) acc += face_flux<S, 1, T>(cf, X, D, c, shift<1>(c, +1, D));
    if (c.i > 0) acc -= face_flux<S, 0, T>(cf, X, D, shift<0>(c, -1, D), c);
    if (c.i < D.nth - 1) acc += face_flux<S, 0, T>(cf, X, D, c, shift<0>(c, +1, D));
    acc -= face_flux<S, 2, T>(cf, X, D, shift<2>(c, -1, D), c);
    acc += face_flux<S, 2, T>(cf, X, D, c, shift<2>(c, +1, D));
    return acc;
}

// r_c = b_c - (A x)_c with every face term fused into one multiply-add on r:
// r = b - sum_d [F_d(upper) - F_d(lower)], each F expanded term by term.
// Same operator as apply_cell; fewer FP64 instructions (FP64 issues at about
// 1/64 of the FP32 rate on GB300, so the outer residual is instruction bound).
template <int S, int d, typename XA>
__device__ __forceinline__ double face_into(double r, double sgn, const CoefF64& cf, const XA& X, const Dims& D,
                                            C3 L, C3 U) {
    const i64 u = cidx(D, U);
    r = fma(sgn * cf(4 * d, u), X(U) - X(L), r);
    if (S == 19) {
        if (d != 0) {
            const double w = sgn * 0.25 * cf(3 * d + 0, u);
            r = fma(w, (X(shift<0>(L, +1, D)) + X(shift<0>(U, +1, D))) - (X(shift<0>(L, -1, D)) + X(shift<0>(U, -1, D))), r);
        }
        if (d != 1) {
            const double w = sgn * 0.25 * cf(3 * d + 1, u);
            r = fma(w, (X(shift<1>(L, +1, D)) + X(shift<1>(U, +1, D))) - (X(shift<1>(L, -1, D)) + X(shift<1>(U, -1, D))), r);
        }
        if (d != 2) {
            const double w = sgn * 0.25 * cf(3 * d + 2, u);
            r = fma(w, (X(shift<2>(L, +1, D)) + X(shift<2>(U, +1, D))) - (X(shift<2>(L, -1, D)) + X(shift<2>(U, -1, D))), r);
        }
    }
    return r;
}

template <int S, typename XA>
__device__ __forceinline__ double residual_cell(const CoefF64& cf, const XA& X, const Dims& D, C3 c, double b) {
    double r = b;
    if (c.j > 0) r = face_into<S, 1>(r, +1.0, cf, X, D, shift<1>(c, -1, D), c);
    if (c.j < D.nr - 1) r = face_into<S, 1>(r, -1.0, cf, X, D, c, shift<1>(c, +1, D));
    if (c.i > 0) r = face_into<S, 0>(r, +1.0, cf, X, D, shift<0>(c, -1, D), c);
    if (c.i < D.nth - 1) r = face_into<S, 0>(r, -1.0, cf, X, D, c, shift<0>(c, +1, D));
    r = face_into<S, 2>(r, +1.0, cf, X, D, shift<2>(c, -1, D), c);
    r = face_into<S, 2>(r, -1.0, cf, X, D, c, shift<2>(c, +1, D));
    return r;
}

// Exact diagonal A_cc of the operator above.  Besides -sum of the six G_dd, a
// cross term reaches x_c itself when a tangential neighbour is mirrored onto c
// at a wall: +G_dq/4 at an upper face and -G_dq/4 at a lower face when c is
// on the top wall in q, with opposite signs on the bottom wall.
template <int S, typename T, typename CF>
__device__ __forceinline__ T diag_cell(const CF& cf, const Dims& D, C3 c) {
    const i64 self = cidx(D, c);
    T dg = 0;
    // lower/upper coefficient rows of the six faces (upper = neighbour's lower row)
    const bool hasEl = c.j > 0, hasEu = c.j < D.nr - 1;
    const bool hasZl = c.i > 0, hasZu = c.i < D.nth - 1;
    const i64 eu = hasEu ? cidx(D, c.j + 1, c.i, c.k) : self;
    const i64 zu = hasZu ? cidx(D, c.j, c.i + 1, c.k) : self;
    const i64 xu = cidx(D, c.j, c.i, c.k + 1 == D.nph ? 0 : c.k + 1);
    if (hasEl) dg -= (T)cf(4, self);
    if (hasEu) dg -= (T)cf(4, eu);
    if (hasZl) dg -= (T)cf(0, self);
    if (hasZu) dg -= (T)cf(0, zu);
    dg -= (T)cf(8, self);
    dg -= (T)cf(8, xu);
    if (S == 19) {
        // mirrored-onto-self weight along q: +1 at the top wall, -1 at the bottom
        const T sz = (T)((c.i == D.nth - 1) - (c.i == 0));   // q = zeta
        const T se = (T)((c.j == D.nr - 1) - (c.j == 0));    // q = eta
        if (sz != (T)0) {
            T w = 0;
            if (hasEu) w += (T)cf(3, eu);     // eta faces, column zeta
            if (hasEl) w -= (T)cf(3, self);
            w += (T)cf(6, xu);                 // xi faces, column zeta
            w -= (T)cf(6, self);
            dg += (T)0.25 * sz * w;
        }
        if (se != (T)0) {
            T w = 0;
            if (hasZu) w += (T)cf(1, zu);     // zeta faces, column eta
            if (hasZl) w -= (T)cf(1, self);
            w += (T)cf(7, xu);                 // xi faces, column eta
            w -= (T)cf(7, self);
            dg += (T)0.25 * se * w;
        }
    }
    return dg;
}

// ---------------------------------------------------------------- 7-point fast path
// The 7-point operator at cell c = (j, i, k) from one base index: neighbours
// at c -/+ 1 (longitude, wrapped), c -/+ nph (colatitude), c -/+ nth*nph
// (radius).  Lower wall faces store G = 0 and upper wall faces are not read;
// a neighbour across a wall is replaced by x_c, which meets a zero
// coefficient.  Same operator as apply_cell with S = 7 (Eq. PC_term1 in each
// direction); each coefficient is loaded once for A x and the diagonal.
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
        return eu * (xjp - xc) - el * (xc - xjm) + zu * (xip - xc) - zl * (xc - xim) + xu * (xkp - xc) -
               xl * (xc - xkm);
    }
    __device__ __forceinline__ T diag() const { return -(el + eu + zl + zu + xl + xu); }
    // Gauss-Seidel / Jacobi step x_c + (b - A x)_c / A_cc
    __device__ __forceinline__ T gs(T b) const { return xc + (b - ax()) / diag(); }
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

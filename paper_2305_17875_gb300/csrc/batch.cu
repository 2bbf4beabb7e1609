// batch.cu - one launch per level operation over a joint work list of many
// shells (the solve of one shell is the batch of one).
//
// A launch covers a list of tasks, each a (shell, level) piece with its own
// virtual grid of `nblocks` blocks; the CTAs of the launch walk the virtual
// blocks of all tasks.  Inside a task the work items are mapped exactly as
// in a stand-alone launch of `nblocks` blocks, so per-cell arithmetic and the
// layout of every reduction's partial sums are those of a single solve.
// Shells whose active flag is 0 skip their tasks.
#include <cooperative_groups.h>
#include <cstdlib>
#include <type_traits>

#include "mg_kernels.h"
#include "line_smooth.cuh"
#include "xline_smooth.cuh"
#include "plane_smooth.cuh"

namespace mgs {

namespace {

constexpr int kBT = 256;

template <int P>
struct Prec;
template <>
struct Prec<PREC64> {
    typedef double T;
    typedef CoefF64 CF;
    __device__ static const CF& cf(const LevelView& v) { return v.c64; }
};
template <>
struct Prec<PREC32> {
    typedef float T;
    typedef CoefF32 CF;
    __device__ static const CF& cf(const LevelView& v) { return v.c32; }
};
template <>
struct Prec<PREC16> {
    typedef float T;
    typedef CoefF16 CF;
    __device__ static const CF& cf(const LevelView& v) { return v.c16; }
};

// multicolour Gauss-Seidel colour pass (same cells and arithmetic as stencil.cu)
// poles (19 points on the full sphere): the first and last rows of x as they
// were before the pass (BOP_POLES), read for the cells across the pole: cells
// of one colour couple across the pole, and a colour is updated as one step.
template <int S, typename T, typename CF>
__device__ __forceinline__ void gs_pass(const CF& cf, const Dims& D, T* x, const T* b, int colour, i64 first,
                                        i64 stride, const T* poles = nullptr) {
    const int hk = D.nph >> 1;
    if constexpr (S == 7) {
        const i64 work = (i64)D.nr * D.nth * hk;
        for (i64 t = first; t < work; t += stride) {
            int kk, i, j;
            decode_half(D, t, kk, i, j);
            Cell7<T> q;
            q.load(cf, D, j, i, 2 * kk + ((colour + i + j) & 1), XLin<T>{x});
            x[q.c] = q.gs(b[q.c]);
        }
    } else {
        // 19 points: only rows with (i + j) = colour mod 2 hold cells of the colour
        const int nth2 = (D.nth + 1) >> 1;
        const i64 work = (i64)D.nr * nth2 * hk;
        for (i64 t = first; t < work; t += stride) {
            const unsigned row = D.dhk.div((unsigned)t);
            const unsigned jj = D.dth2.div(row);
            const int kk = (int)((unsigned)t - row * (unsigned)hk);
            const int j = (int)jj, i = 2 * (int)(row - jj * (unsigned)nth2) + ((colour ^ j) & 1);
            if (i >= D.nth) continue;
            const C3 p{j, i, 2 * kk + (((colour >> 1) + j) & 1)};
            const int c = cidx(D, p);
            Nbr19<T> X;
            X.load(XLin<T>{x}, D, c, p, !cf.has(2), poles);
            const T r = b[c] - apply19<T>(cf, X, D, c, p);
            x[c] = X.v[0] + r / diag_cell<S, T>(cf, D, p);
        }
    }
}

// ---- four-cell groups (vec4 levels): the same per-cell arithmetic as the
// scalar forms, with the longitude rows moved as 16-byte vectors.
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
    const double2 q0 = *reinterpret_cast<const double2*>(p);
    const double2 q1 = *(reinterpret_cast<const double2*>(p) + 1);
    v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
}
__device__ __forceinline__ void ldg4(const float* p, float v[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
__device__ __forceinline__ void ldg4(const double* p, double v[4]) {
    const double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
    const double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *(reinterpret_cast<double2*>(p) + 1) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(double* p, double a, double b) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// ---- L2 residency of a level's lines.  A level small enough to stay in L2
// across its passes (its x, b and coefficients; the coarse levels of a
// V-cycle are visited by ten launches an iteration) keeps its lines
// (evict_last); the fine level, which streams through L2 every pass, marks
// its read-only b and coefficients evict_first so that they do not push the
// coarse levels out (its x keeps the normal priority: the next pass reads
// it again).  Hints change where lines live, never values.
constexpr long long kL2KeepBytes = 48ll << 20;
constexpr long long kL2KeepXBytes = 24ll << 20;
__device__ __forceinline__ unsigned long long l2_policy(int kind) {   // 0 first, 1 normal, 2 last
    unsigned long long p;
    if (kind == 2) asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else if (kind == 1) asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    else asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Plain accesses (FP64 cycles)
struct PlainMem {
    template <typename T>
    __device__ __forceinline__ void ld4x(const T* p, T v[4]) const { ld4(p, v); }
    template <typename T>
    __device__ __forceinline__ void ld4r(const T* p, T v[4]) const { ldg4(p, v); }
    template <typename T>
    __device__ __forceinline__ T ldx(const T* p) const { return *p; }
    template <typename T>
    __device__ __forceinline__ void st4x(T* p, const T v[4]) const { st4(p, v); }
    template <typename T>
    __device__ __forceinline__ void st2x(T* p, T a, T b) const { st2(p, a, b); }
    template <typename CF, typename T>
    __device__ __forceinline__ void cf4(const CF& cf, int a, int idx, T v[4]) const { cf.load4(a, idx, v); }
    template <typename CF>
    __device__ __forceinline__ auto cf1(const CF& cf, int a, int idx) const { return cf(a, idx); }
};
// FP32 values with L2 priorities: xp for x, rp for b and the coefficients
struct HintMem {
    unsigned long long xp, rp;
    __device__ __forceinline__ void ld4x(const float* p, float v[4]) const {
        asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p), "l"(xp));
    }
    __device__ __forceinline__ void ld4r(const float* p, float v[4]) const {
        asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p), "l"(rp));
    }
    __device__ __forceinline__ float ldx(const float* p) const {
        float v;
        asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(xp));
        return v;
    }
    __device__ __forceinline__ void st4x(float* p, const float v[4]) const {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v[0]), "f"(v[1]),
                     "f"(v[2]), "f"(v[3]), "l"(xp)
                     : "memory");
    }
    __device__ __forceinline__ void st2x(float* p, float a, float b) const {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(a), "f"(b), "l"(xp)
                     : "memory");
    }
    __device__ __forceinline__ void cf4(const CoefF32& cf, int a, int idx, float v[4]) const {
        ld4r(cf.g[a] + idx, v);
    }
    __device__ __forceinline__ float cf1(const CoefF32& cf, int a, int idx) const {
        float v;
        asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(cf.g[a] + idx), "l"(rp));
        return v;
    }
    // FP16 storage: the same conversion as CoefF16's readers
    __device__ __forceinline__ void cf4(const CoefF16& cf, int a, int idx, float v[4]) const {
        unsigned u0, u1;
        asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(u0), "=r"(u1) : "l"(cf.g[a] + idx), "l"(rp));
        const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u0));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u1));
        v[0] = lo.x * cf.s[a], v[1] = lo.y * cf.s[a], v[2] = hi.x * cf.s[a], v[3] = hi.y * cf.s[a];
    }
    __device__ __forceinline__ float cf1(const CoefF16& cf, int a, int idx) const { return cf(a, idx); }
};
// The accesses of a level of n cells at vb / cb bytes per value / coefficient.
__device__ __forceinline__ HintMem level_mem(long long n, int vb, int cb, int ncomp) {
    const bool keep = n * (2ll * vb + (long long)ncomp * cb) <= kL2KeepBytes;
    const bool keep_x = keep || n * vb <= kL2KeepXBytes;   // a fine level whose x alone fits
    return HintMem{l2_policy(keep_x ? 2 : 1), l2_policy(keep ? 2 : 0)};
}

// x, b and the six face coefficients of the four cells (j, i, k0 .. k0 + 3)
// of a 7-point level; cell(m) gives the Cell7 of cell k0 + m.
template <typename T>
struct Group7 {
    int c0;
    T X0[4], Jm[4], Jp[4], Im[4], Ip[4], EL[4], EU[4], ZL[4], ZU[4], XL[4];
    T xkm, xkp, xu3;
    template <typename CF, typename M = PlainMem>
    __device__ __forceinline__ void load(const CF& cf, const Dims& D, const T* x, int j, int i, int k0,
                                         const M& mem = M()) {
        const int plane = D.nth * D.nph;
        c0 = (j * D.nth + i) * D.nph + k0;
        const int rb = c0 - k0;
        const bool jl = j > 0, ju = j + 1 < D.nr, il = i > 0, iu = i + 1 < D.nth;
        mem.ld4x(x + c0, X0);
        if (jl) mem.ld4x(x + c0 - plane, Jm);
        else for (int m = 0; m < 4; ++m) Jm[m] = X0[m];
        if (ju) mem.ld4x(x + c0 + plane, Jp);
        else for (int m = 0; m < 4; ++m) Jp[m] = X0[m];
        if (il) mem.ld4x(x + c0 - D.nph, Im);
        else for (int m = 0; m < 4; ++m) Im[m] = X0[m];
        if (iu) mem.ld4x(x + c0 + D.nph, Ip);
        else for (int m = 0; m < 4; ++m) Ip[m] = X0[m];
        const int kw = k0 + 4 == D.nph ? rb : c0 + 4;
        xkm = mem.ldx(x + (k0 == 0 ? rb + D.nph - 1 : c0 - 1));
        xkp = mem.ldx(x + kw);
        mem.cf4(cf, 4, c0, EL);
        if (ju) mem.cf4(cf, 4, c0 + plane, EU);
        else for (int m = 0; m < 4; ++m) EU[m] = (T)0;
        mem.cf4(cf, 0, c0, ZL);
        if (iu) mem.cf4(cf, 0, c0 + D.nph, ZU);
        else for (int m = 0; m < 4; ++m) ZU[m] = (T)0;
        mem.cf4(cf, 8, c0, XL);
        xu3 = (T)mem.cf1(cf, 8, kw);
    }
    __device__ __forceinline__ Cell7<T> cell(int m) const {   // m a compile-time constant after unrolling
        Cell7<T> q;
        q.c = c0 + m;
        q.xc = X0[m], q.xjm = Jm[m], q.xjp = Jp[m], q.xim = Im[m], q.xip = Ip[m];
        q.xkm = m == 0 ? xkm : X0[m == 0 ? 0 : m - 1];
        q.xkp = m == 3 ? xkp : X0[m == 3 ? 3 : m + 1];
        q.el = EL[m], q.eu = EU[m], q.zl = ZL[m], q.zu = ZU[m], q.xl = XL[m];
        q.xu = m == 3 ? xu3 : XL[m == 3 ? 3 : m + 1];
        return q;
    }
};

// One colour of the 7-point red-black pass over groups: in a group the cells
// of the colour are k0 + p and k0 + p + 2, p = (colour + i + j) & 1.
template <typename T, typename CF>
__device__ __forceinline__ void gs_pass7v(const CF& cf, const Dims& D, T* x, const T* b, int colour, i64 first,
                                          i64 stride) {
    const int nq = D.nph >> 2;
    const i64 work = (i64)D.nr * D.nth * nq;
    // FP32 values: the level's L2 priorities; FP64 plain
    typedef typename std::conditional<sizeof(T) == 4, HintMem, PlainMem>::type M;
    M mem{};
    if constexpr (sizeof(T) == 4) mem = level_mem(D.n(), 4, sizeof(cf.g[0][0]), 3);
    for (i64 t = first; t < work; t += stride) {
        const unsigned row = D.dq.div((unsigned)t);
        const unsigned jj = D.dth.div(row);
        const int k0 = 4 * (int)((unsigned)t - row * (unsigned)nq);
        const int i = (int)(row - jj * (unsigned)D.nth), j = (int)jj;
        Group7<T> g;
        g.load(cf, D, x, j, i, k0, mem);
        T B[4];
        mem.ld4r(b + g.c0, B);
        // the group is written back whole (16-byte store, full sectors); the two
        // cells of the other colour keep the values every reader sees this pass
        T out[4] = {g.X0[0], g.X0[1], g.X0[2], g.X0[3]};
        if (((colour + i + j) & 1) == 0) {
            out[0] = g.cell(0).gs(B[0]);
            out[2] = g.cell(2).gs(B[2]);
        } else {
            out[1] = g.cell(1).gs(B[1]);
            out[3] = g.cell(3).gs(B[3]);
        }
        mem.st4x(x + g.c0, out);
    }
}

// 19-point colour pass over groups of four longitudes (nph a multiple of 4,
// walled grids): a work item is a group of a row of the colour and updates
// its two cells of the colour (positions P, P + 2, P the colour's longitude
// parity) from 16-byte loads of the nine (radius, colatitude) rows around it,
// the two longitudes either side, and the face rows; each cell's neighbourhood
// and rows are then picked out of those registers and go through the scalar
// pass's arithmetic (apply19_r, diag_cell_r), so the bits are those of
// gs_pass.  The group is written back whole (the other two cells unchanged).
template <typename T, typename CF, bool AXI, int P>
__device__ __forceinline__ void group19(const CF& cf, const Dims& D, T* x, const T* b, int j, int i, int q) {
    const int plane = D.nth * D.nph;
    const int k0 = 4 * q;
    const int c0 = (j * D.nth + i) * D.nph + k0;
    const int oj[3] = {j > 0 ? -plane : 0, 0, j + 1 < D.nr ? plane : 0};
    const int oi[3] = {i > 0 ? -D.nph : 0, 0, i + 1 < D.nth ? D.nph : 0};
    const int km = k0 == 0 ? c0 + D.nph - 1 : c0 - 1;   // longitude k0 - 1 of the row (wrapped)
    const int kp = k0 + 4 == D.nph ? c0 - k0 : c0 + 4;   // longitude k0 + 4
    // x on the nine rows; the longitudes either side where a longitude offset is read
    T X[3][3][4], E[3][3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int o = oj[a] + oi[e];
            ld4(x + c0 + o, X[a][e]);
            const bool edge = (a == 1 && e == 1) || (!AXI && (a == 1 || e == 1));
            E[a][e][0] = edge ? x[km + o] : (T)0;
            E[a][e][1] = edge ? x[kp + o] : (T)0;
        }
    // face rows: own components, radius-upper 3..5, colatitude-upper 0..2,
    // longitude-upper 6..8 (the next group's first cell for the last one)
    T C[9][4], EU[3][4], ZU[3][4], XN[3];
    const bool ju = j + 1 < D.nr, iu = i + 1 < D.nth;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        if (RegRows<T, AXI>::stored(a)) cf.load4(a, c0, C[a]);
        else C[a][0] = C[a][1] = C[a][2] = C[a][3] = (T)0;
    }
#pragma unroll
    for (int qq = 0; qq < 3; ++qq) {
        if (ju && RegRows<T, AXI>::stored(3 + qq)) cf.load4(3 + qq, c0 + plane, EU[qq]);
        else EU[qq][0] = EU[qq][1] = EU[qq][2] = EU[qq][3] = (T)0;
        if (iu && RegRows<T, AXI>::stored(qq)) cf.load4(qq, c0 + D.nph, ZU[qq]);
        else ZU[qq][0] = ZU[qq][1] = ZU[qq][2] = ZU[qq][3] = (T)0;
        XN[qq] = RegRows<T, AXI>::stored(6 + qq) ? (T)cf(6 + qq, kp) : (T)0;
    }
    T B[4];
    ldg4(b + c0, B);
    T out[4] = {X[1][1][0], X[1][1][1], X[1][1][2], X[1][1][3]};
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
        const int m = P + 2 * e2;
        Nbr19<T> N;
#pragma unroll
        for (int n = 0; n < 19; ++n) {
            const int dj = row_off(n, 0), di = row_off(n, 1), dk = row_off(n, 2);
            const bool phi_edge = dk != 0 && (dj != 0 || di != 0);
            const int kk = m + dk;
            N.v[n] = (AXI && phi_edge) ? (T)0
                     : (kk < 0 ? E[dj + 1][di + 1][0] : (kk > 3 ? E[dj + 1][di + 1][1] : X[dj + 1][di + 1][kk < 0 ? 0 : (kk > 3 ? 3 : kk)]));
        }
        T v[19];
        v[0] = B[m];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[1 + a] = C[a][m];
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) {
            v[10 + qq] = EU[qq][m];
            v[13 + qq] = ZU[qq][m];
            v[16 + qq] = m < 3 ? C[6 + qq][m < 3 ? m + 1 : 3] : XN[qq];
        }
        const RegRows<T, AXI> cr{v};
        const C3 p3{j, i, k0 + m};
        const T r = v[0] - apply19_r<T>(cr, N, D, p3);
        out[m] = N.v[0] + r / diag_cell_r<19, T>(cr, D, p3);
    }
    st4(x + c0, out);
}

template <typename T, typename CF, bool AXI>
__device__ __forceinline__ void gs_pass19v(const CF& cf, const Dims& D, T* x, const T* b, int colour, i64 first,
                                           i64 stride) {
    const int nq = D.nph >> 2, nth2 = (D.nth + 1) >> 1;
    const i64 work = (i64)D.nr * nth2 * nq;
    for (i64 t = first; t < work; t += stride) {
        const unsigned row = D.dq.div((unsigned)t);
        const unsigned jj = D.dth2.div(row);
        const int q = (int)((unsigned)t - row * (unsigned)nq);
        const int j = (int)jj, i = 2 * (int)(row - jj * (unsigned)nth2) + ((colour ^ j) & 1);
        if (i >= D.nth) continue;
        if ((((colour >> 1) + j) & 1) == 0) group19<T, CF, AXI, 0>(cf, D, x, b, j, i, q);
        else group19<T, CF, AXI, 1>(cf, D, x, b, j, i, q);
    }
}

// 7-point residual + children-sum restriction over groups of four fine
// longitude cells in every child row: four coarse cells when longitude is
// not halved, two when it is.  Sums in the order of the scalar form.
template <typename T, typename CF>
__device__ __forceinline__ void restrict_pass7v(const CF& cf, const Dims& D, const T* x, const T* b, const Dims& Dc,
                                                int cz, int ce, int cx, T* rc, T* ec_zero, i64 first, i64 stride) {
    const int nq = D.nph >> 2;
    const i64 work = (i64)Dc.nr * Dc.nth * nq;
    // FP32 values: the fine level's L2 priorities for its reads, the coarse
    // level's for the coarse right side and correction written
    typedef typename std::conditional<sizeof(T) == 4, HintMem, PlainMem>::type M;
    M fm{}, cm{};
    if constexpr (sizeof(T) == 4) {
        fm = level_mem(D.n(), 4, sizeof(cf.g[0][0]), 3);
        cm = level_mem(Dc.n(), 4, sizeof(cf.g[0][0]), 3);
    }
    for (i64 t = first; t < work; t += stride) {
        const unsigned row = D.dq.div((unsigned)t);
        const unsigned J = Dc.dth.div(row);
        const int q = (int)((unsigned)t - row * (unsigned)nq);
        const int I = (int)(row - J * (unsigned)Dc.nth);
        T s[4] = {(T)0, (T)0, (T)0, (T)0};
        for (int dj = 0; dj < ce; ++dj)
            for (int di = 0; di < cz; ++di) {
                Group7<T> g;
                g.load(cf, D, x, ce * (int)J + dj, cz * I + di, 4 * q, fm);
                T B[4];
                fm.ld4r(b + g.c0, B);
                const T r0 = g.cell(0).resid(B[0]), r1 = g.cell(1).resid(B[1]);
                const T r2 = g.cell(2).resid(B[2]), r3 = g.cell(3).resid(B[3]);
                if (cx == 1) {
                    s[0] += r0, s[1] += r1, s[2] += r2, s[3] += r3;
                } else {
                    s[0] += r0;
                    s[0] += r1;
                    s[1] += r2;
                    s[1] += r3;
                }
            }
        const int cb = ((int)J * Dc.nth + I) * Dc.nph;
        if (cx == 1) {
            cm.st4x(rc + cb + 4 * q, s);
            if (ec_zero) {
                const T z[4] = {(T)0, (T)0, (T)0, (T)0};
                cm.st4x(ec_zero + cb + 4 * q, z);
            }
        } else {
            cm.st2x(rc + cb + 2 * q, s[0], s[1]);
            if (ec_zero) cm.st2x(ec_zero + cb + 2 * q, (T)0, (T)0);
        }
    }
}

// ---- 19-point four-cell groups (residual + restriction).  x on the nine (j, i) rows around the group
// (radius and colatitude clamped at the walls: mirror ghosts) as 16-byte
// vectors, with the longitude halo of the five rows the stencil reaches
// along k; coefficients streamed face by face as vectors.  Each cell's
// arithmetic is apply19's chain (same bits).
template <typename T>
struct Group19 {
    int c0, rb, kw;      // first cell, its row start, the longitude index after the group (wrapped)
    T R[9][4];           // row (dj, di) at (dj + 1) * 3 + (di + 1)
    T lo[9], hi[9];      // longitude k0 - 1 and k0 + 4 of the rows with dj == 0 or di == 0
    bool ju, iu;
    int plane;
    // axi: no longitude cross terms, so the off-centre rows need no cells
    // beyond the group in longitude
    __device__ __forceinline__ void load(const T* x, const Dims& D, int j, int i, int k0, bool axi) {
        plane = D.nth * D.nph;
        c0 = (j * D.nth + i) * D.nph + k0;
        rb = c0 - k0;
        kw = k0 + 4 == D.nph ? 0 : k0 + 4;
        ju = j + 1 < D.nr;
        iu = i + 1 < D.nth;
        const int oj[3] = {j > 0 ? -plane : 0, 0, ju ? plane : 0};
        const int oi[3] = {i > 0 ? -D.nph : 0, 0, iu ? D.nph : 0};
        const int km = k0 == 0 ? D.nph - 1 : k0 - 1;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int r = a * 3 + b, o = oj[a] + oi[b];
                ld4(x + c0 + o, R[r]);
                if ((a == 1 && b == 1) || (!axi && (a == 1 || b == 1))) {
                    lo[r] = x[rb + o + km];
                    hi[r] = x[rb + o + kw];
                } else {
                    lo[r] = hi[r] = (T)0;
                }
            }
    }
    // x at offset (dj, di, dk) from cell m of the group
    template <int m, int dj, int di, int dk>
    __device__ __forceinline__ T at() const {
        constexpr int r = (dj + 1) * 3 + (di + 1), pos = m + dk;
        return pos < 0 ? lo[r] : (pos > 3 ? hi[r] : R[r][pos < 0 ? 0 : (pos > 3 ? 3 : pos)]);
    }
    // x at offset a along paper direction da and b along db (0 zeta -> i, 1 eta -> j, 2 xi -> k)
    template <int m, int da, int a, int db, int b>
    __device__ __forceinline__ T atd() const {
        return at<m, (da == 1 ? a : 0) + (db == 1 ? b : 0), (da == 0 ? a : 0) + (db == 0 ? b : 0),
                  (da == 2 ? a : 0) + (db == 2 ? b : 0)>();
    }
};

// acc + sgn F for the d-face of cell m of the group; G[q][m] is component
// 3d + q of the face's metric row.
template <int d, int side, int m, typename T>
__device__ __forceinline__ T face19g(T acc, const Group19<T>& g, const T G[3][4], bool axi) {
    constexpr int sL = side < 0 ? -1 : 0, sU = side < 0 ? 0 : 1;
    const T sgn = (T)side;
    acc = fma(sgn * G[d][m], g.template atd<m, d, sU, d, 0>() - g.template atd<m, d, sL, d, 0>(), acc);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (q == d || (axi && (q == 2 || d == 2))) continue;   // absent longitude cross terms
        T plus, minus;
        if (q == 0) {
            plus = g.template atd<m, d, sL, 0, 1>() + g.template atd<m, d, sU, 0, 1>();
            minus = g.template atd<m, d, sL, 0, -1>() + g.template atd<m, d, sU, 0, -1>();
        } else if (q == 1) {
            plus = g.template atd<m, d, sL, 1, 1>() + g.template atd<m, d, sU, 1, 1>();
            minus = g.template atd<m, d, sL, 1, -1>() + g.template atd<m, d, sU, 1, -1>();
        } else {
            plus = g.template atd<m, d, sL, 2, 1>() + g.template atd<m, d, sU, 2, 1>();
            minus = g.template atd<m, d, sL, 2, -1>() + g.template atd<m, d, sU, 2, -1>();
        }
        acc = fma(sgn * (T)0.25 * G[q][m], plus - minus, acc);
    }
    return acc;
}

template <int d, int side, int MASK, typename T>
__device__ __forceinline__ void face19g_all(T acc[4], const Group19<T>& g, const T G[3][4], bool axi) {
    if (MASK & 1) acc[0] = face19g<d, side, 0>(acc[0], g, G, axi);
    if (MASK & 2) acc[1] = face19g<d, side, 1>(acc[1], g, G, axi);
    if (MASK & 4) acc[2] = face19g<d, side, 2>(acc[2], g, G, axi);
    if (MASK & 8) acc[3] = face19g<d, side, 3>(acc[3], g, G, axi);
}

// component a of four consecutive cells, zero when the component is absent
template <typename T, typename CF>
__device__ __forceinline__ void load4_or0(const CF& cf, int a, int idx, T v[4]) {
    if (cf.has(a)) cf.load4(a, idx, v);
    else v[0] = v[1] = v[2] = v[3] = (T)0;
}

// (A x) of the group's cells in MASK (bit m), in apply19's face order.  Lower
// faces read the cells' own metric rows, upper faces those of the next cell
// along the direction; wall faces carry no flux and are skipped.
template <int MASK, typename T, typename CF>
__device__ __forceinline__ void apply19_group(const CF& cf, const Dims& D, const Group19<T>& g, int j, int i,
                                              T acc[4]) {
    T G[3][4];
    const bool axi = !cf.has(2);
    for (int m = 0; m < 4; ++m) acc[m] = (T)0;
    if (j > 0) {
        for (int q = 0; q < 3; ++q) load4_or0<T>(cf, 3 + q, g.c0, G[q]);
        face19g_all<1, -1, MASK>(acc, g, G, axi);
    }
    if (g.ju) {
        for (int q = 0; q < 3; ++q) load4_or0<T>(cf, 3 + q, g.c0 + g.plane, G[q]);
        face19g_all<1, 1, MASK>(acc, g, G, axi);
    }
    if (i > 0) {
        for (int q = 0; q < 3; ++q) load4_or0<T>(cf, q, g.c0, G[q]);
        face19g_all<0, -1, MASK>(acc, g, G, axi);
    }
    if (g.iu) {
        for (int q = 0; q < 3; ++q) load4_or0<T>(cf, q, g.c0 + D.nph, G[q]);
        face19g_all<0, 1, MASK>(acc, g, G, axi);
    }
    for (int q = 0; q < 3; ++q) load4_or0<T>(cf, 6 + q, g.c0, G[q]);
    face19g_all<2, -1, MASK>(acc, g, G, axi);
    // upper longitude faces: the next cell's lower face
    for (int q = 0; q < 3; ++q) {
        const T nxt = cf.has(6 + q) ? (T)cf(6 + q, g.rb + g.kw) : (T)0;
        G[q][0] = G[q][1], G[q][1] = G[q][2], G[q][2] = G[q][3], G[q][3] = nxt;
    }
    face19g_all<2, 1, MASK>(acc, g, G, axi);
}

// 19-point residual + children-sum restriction over groups (as restrict_pass7v).
template <typename T, typename CF>
__device__ __forceinline__ void restrict_pass19v(const CF& cf, const Dims& D, const T* x, const T* b, const Dims& Dc,
                                                 int cz, int ce, int cx, T* rc, T* ec_zero, i64 first, i64 stride) {
    const int nq = D.nph >> 2;
    const i64 work = (i64)Dc.nr * Dc.nth * nq;
    for (i64 t = first; t < work; t += stride) {
        const unsigned row = D.dq.div((unsigned)t);
        const unsigned J = Dc.dth.div(row);
        const int q = (int)((unsigned)t - row * (unsigned)nq);
        const int I = (int)(row - J * (unsigned)Dc.nth);
        T s[4] = {(T)0, (T)0, (T)0, (T)0};
        for (int dj = 0; dj < ce; ++dj)
            for (int di = 0; di < cz; ++di) {
                const int j = ce * (int)J + dj, i = cz * I + di;
                Group19<T> g;
                g.load(x, D, j, i, 4 * q, !cf.has(2));
                T B[4], ax[4];
                ldg4(b + g.c0, B);
                apply19_group<15>(cf, D, g, j, i, ax);
                const T r0 = B[0] - ax[0], r1 = B[1] - ax[1], r2 = B[2] - ax[2], r3 = B[3] - ax[3];
                if (cx == 1) {
                    s[0] += r0, s[1] += r1, s[2] += r2, s[3] += r3;
                } else {
                    s[0] += r0;
                    s[0] += r1;
                    s[1] += r2;
                    s[1] += r3;
                }
            }
        const int cb = ((int)J * Dc.nth + I) * Dc.nph;
        if (cx == 1) {
            st4(rc + cb + 4 * q, s);
            if (ec_zero) {
                const T z[4] = {(T)0, (T)0, (T)0, (T)0};
                st4(ec_zero + cb + 4 * q, z);
            }
        } else {
            st2(rc + cb + 2 * q, s[0], s[1]);
            if (ec_zero) st2(ec_zero + cb + 2 * q, (T)0, (T)0);
        }
    }
}

template <int S, typename T, typename CF>
__device__ __forceinline__ void jacobi_pass(const CF& cf, const Dims& D, const T* x, T* xo, const T* b, i64 first,
                                            i64 stride) {
    XRead<T> X{x, D};
    const T omega = S == 7 ? (T)(6.0 / 7.0) : (T)(4.0 / 5.0);
    for (i64 c = first; c < D.n(); c += stride) {
        const C3 cc = decode(D, c);
        const T r = b[c] - apply_cell<S, T>(cf, X, D, cc);
        xo[c] = x[c] + omega * r / diag_cell<S, T>(cf, D, cc);
    }
}

template <int S, typename T, typename CF>
__device__ __forceinline__ void restrict_pass(const CF& cf, const Dims& D, const T* x, const T* b, const Dims& Dc,
                                              int cz, int ce, int cx, T* rc, T* ec_zero, i64 first, i64 stride) {
    for (i64 t = first; t < Dc.n(); t += stride) {
        const C3 C = decode(Dc, t);
        T s = 0;
        for (int dj = 0; dj < ce; ++dj)
            for (int di = 0; di < cz; ++di)
                for (int dk = 0; dk < cx; ++dk) {
                    const C3 c{ce * C.j + dj, cz * C.i + di, cx * C.k + dk};
                    if constexpr (S == 7) {
                        Cell7<T> q;
                        q.load(cf, D, c.j, c.i, c.k, XLin<T>{x});
                        s += q.resid(b[q.c]);
                    } else {
                        const int id = cidx(D, c);
                        Nbr19<T> X;
                        X.load(XLin<T>{x}, D, id, c, !cf.has(2));
                        s += b[id] - apply19<T>(cf, X, D, id, c);
                    }
                }
        rc[t] = s;
        if (ec_zero) ec_zero[t] = 0;
    }
}

__device__ __forceinline__ void lin1d(int f, int c, int nc, bool periodic, int idx[2], float w[2]) {
    if (c == 1) {
        idx[0] = idx[1] = f;
        w[0] = 1.0f;
        w[1] = 0.0f;
        return;
    }
    const int C = f >> 1;
    int nb = (f & 1) ? C + 1 : C - 1;
    if (periodic) nb = nb < 0 ? nb + nc : (nb >= nc ? nb - nc : nb);
    else if (nb < 0 || nb >= nc) nb = C;
    idx[0] = C;
    idx[1] = nb;
    w[0] = 0.75f;
    w[1] = 0.25f;
}

template <typename T>
__device__ __forceinline__ void prolong_pass(const Dims& D, const Dims& Dc, int cz, int ce, int cx, const T* ec, T* x,
                                             i64 first, i64 stride) {
    for (i64 c = first; c < D.n(); c += stride) {
        const C3 f = decode(D, c);
        int ij[2], ii[2], ik[2];
        float wj[2], wi[2], wk[2];
        lin1d(f.j, ce, Dc.nr, false, ij, wj);
        lin1d(f.i, cz, Dc.nth, false, ii, wi);
        lin1d(f.k, cx, Dc.nph, true, ik, wk);
        T s = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a >= ce) break;   // only the entries with nonzero weight
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                if (bb >= cz) break;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (e >= cx) break;
                    s = fma((T)wj[a] * (T)wi[bb] * (T)wk[e], ec[cidx(Dc, ij[a], ii[bb], ik[e])], s);
                }
            }
        }
        x[c] = x[c] + s;
    }
}

// Prolongation over groups of four fine longitude cells: the coarse rows and
// weights along radius and colatitude are shared by the group.  Same weights
// and summation order as prolong_pass.
template <typename T>
__device__ __forceinline__ void prolong_pass_v(const Dims& D, const Dims& Dc, int cz, int ce, int cx, const T* ec,
                                               T* x, i64 first, i64 stride, int cb = 4) {
    const int nq = D.nph >> 2;
    const i64 work = (i64)D.nr * D.nth * nq;
    // FP32 values: the fine and coarse levels' L2 priorities (cb: bytes of a
    // stored coefficient, which size the levels as the colour passes do)
    typedef typename std::conditional<sizeof(T) == 4, HintMem, PlainMem>::type M;
    M fm{}, cm{};
    if constexpr (sizeof(T) == 4) {
        fm = level_mem(D.n(), 4, cb, 3);
        cm = level_mem(Dc.n(), 4, cb, 3);
    }
    for (i64 t = first; t < work; t += stride) {
        const unsigned row = D.dq.div((unsigned)t);
        const unsigned jj = D.dth.div(row);
        const int k0 = 4 * (int)((unsigned)t - row * (unsigned)nq);
        const int i = (int)(row - jj * (unsigned)D.nth), j = (int)jj;
        int ij[2], ii[2];
        float wj[2], wi[2];
        lin1d(j, ce, Dc.nr, false, ij, wj);
        lin1d(i, cz, Dc.nth, false, ii, wi);
        const int c0 = (j * D.nth + i) * D.nph + k0;
        T X[4];
        fm.ld4x(x + c0, X);
        if (cx == 1) {   // longitude not halved: coarse groups of four, weight 1 along k
            T s[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (a >= ce) break;
#pragma unroll
                for (int bb = 0; bb < 2; ++bb) {
                    if (bb >= cz) break;
                    const T wab = (T)wj[a] * (T)wi[bb];
                    T E[4];
                    cm.ld4r(ec + (ij[a] * Dc.nth + ii[bb]) * Dc.nph + k0, E);
                    for (int m = 0; m < 4; ++m) s[m] = fma(wab * (T)1.0f, E[m], s[m]);
                }
            }
            for (int m = 0; m < 4; ++m) X[m] = X[m] + s[m];
            fm.st4x(x + c0, X);
            continue;
        }
        if (cx == 2) {   // halved: fine k0..k0+3 from coarse K0-1 .. K0+2, K0 = k0 / 2
            const int K0 = k0 >> 1;
            const int Km = K0 == 0 ? Dc.nph - 1 : K0 - 1, Kp = K0 + 2 == Dc.nph ? 0 : K0 + 2;
            T s[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (a >= ce) break;
#pragma unroll
                for (int bb = 0; bb < 2; ++bb) {
                    if (bb >= cz) break;
                    const T wab = (T)wj[a] * (T)wi[bb];
                    const T* er = ec + (ij[a] * Dc.nth + ii[bb]) * Dc.nph;
                    const T e0 = cm.ldx(er + K0), e1 = cm.ldx(er + K0 + 1), em = cm.ldx(er + Km), ep = cm.ldx(er + Kp);
                    // weights 3/4 on the coarse cell, 1/4 on its neighbour (e = 0, 1)
                    s[0] = fma(wab * (T)0.75f, e0, s[0]);
                    s[0] = fma(wab * (T)0.25f, em, s[0]);
                    s[1] = fma(wab * (T)0.75f, e0, s[1]);
                    s[1] = fma(wab * (T)0.25f, e1, s[1]);
                    s[2] = fma(wab * (T)0.75f, e1, s[2]);
                    s[2] = fma(wab * (T)0.25f, e0, s[2]);
                    s[3] = fma(wab * (T)0.75f, e1, s[3]);
                    s[3] = fma(wab * (T)0.25f, ep, s[3]);
                }
            }
            for (int m = 0; m < 4; ++m) X[m] = X[m] + s[m];
            fm.st4x(x + c0, X);
            continue;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            int ik[2];
            float wk[2];
            lin1d(k0 + m, cx, Dc.nph, true, ik, wk);
            T s = 0;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (a >= ce) break;   // only the entries with nonzero weight
#pragma unroll
                for (int bb = 0; bb < 2; ++bb) {
                    if (bb >= cz) break;
                    const int rowc = (ij[a] * Dc.nth + ii[bb]) * Dc.nph;
                    const T wab = (T)wj[a] * (T)wi[bb];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (e >= cx) break;
                        s = fma(wab * (T)wk[e], ec[rowc + ik[e]], s);
                    }
                }
            }
            X[m] = X[m] + s;
        }
        st4(x + c0, X);
    }
}

__device__ double unit_scale_b(double sum, i64 n) {
    const double rms = sqrt(sum / (double)n);
    if (!(rms > 0.0) || !isfinite(rms)) return 1.0;
    return ldexp(1.0, -(int)lround(log2(rms)));
}

// Stencil operations of one virtual block.
template <int S, int P, int OP>
__device__ __forceinline__ void run_block(const BTask& tk, int colour, i64 first, i64 stride, int lb, double* sh) {
    typedef typename Prec<P>::T T;
    const auto& cf = Prec<P>::cf(tk.v);
    if constexpr (OP == BOP_GS) {
        // 19 points: the scalar form (a group would load four cells to update two
        // with twice the registers); 7 points: groups when nph is a multiple of 4
        if (S == 7 && vec4(tk.v.D)) gs_pass7v<T>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, colour, first, stride);
        else if (S == 19 && gs19_groups(tk.v.D)) {
            if (cf.has(2)) gs_pass19v<T, typename Prec<P>::CF, false>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, colour, first, stride);
            else gs_pass19v<T, typename Prec<P>::CF, true>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, colour, first, stride);
        } else gs_pass<S, T>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, colour, first, stride, (const T*)tk.z);
    } else if constexpr (OP == BOP_LINE) {
        line_pass<S, T>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, (const T*)tk.z, colour, lb, tk.nblocks);
    } else if constexpr (OP == BOP_XLINE) {
        if (tk.n)   // chunked: W threads per line (uniform per task, so per block)
            xline_pass_chunked<S, T>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, (const T*)tk.z, colour, lb, tk.nblocks);
        else
            xline_pass<S, T>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, (const T*)tk.z, (T*)tk.y, colour, first, stride);
    } else if constexpr (OP == BOP_PRES) {
        plane_res3d<T>(cf, tk.v.D, (const T*)tk.x, (const T*)tk.b, (T*)tk.y, (T*)tk.z, colour, first, stride);
    } else if constexpr (OP == BOP_PRELAX || OP == BOP_PRESTRICT) {
        // the plane operator of a 2-D level: FP64 arrays for the FP64 cycle, FP32 copies otherwise
        const T* const* pc = (const T* const*)(P == PREC64 ? (const void* const*)tk.v.c64.g
                                                           : (const void* const*)tk.v.c32.g);
        if constexpr (OP == BOP_PRELAX)
            plane_relax_warp<T>(pc, tk.v.D, (T*)tk.x, (const T*)tk.b, (const T*)tk.z, colour & 1, colour >> 1, first,
                                stride);
        else
            plane_restrict<T>(pc, tk.v.D, (const T*)tk.x, (const T*)tk.b, tk.Dc, (T*)tk.y, (T*)tk.z, colour, first,
                              stride);
    } else if constexpr (OP == BOP_PPROLONG) {
        plane_prolong<T>(tk.v.D, (T*)tk.x, tk.Dc, (const T*)tk.b, colour, first, stride);
    } else if constexpr (OP == BOP_PUPDATE) {
        plane_update<T>(tk.v.D, (T*)tk.x, (const T*)tk.b, colour, first, stride);
    } else if constexpr (OP == BOP_JACOBI) {
        jacobi_pass<S, T>(cf, tk.v.D, (const T*)tk.x, (T*)tk.y, (const T*)tk.b, first, stride);
    } else if constexpr (OP == BOP_RESTRICT) {
        if (S == 7 && vec4(tk.v.D))
            restrict_pass7v<T>(cf, tk.v.D, (const T*)tk.x, (const T*)tk.b, tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx,
                               (T*)tk.y, (T*)tk.z, first, stride);
        else if (S == 19 && vec4(tk.v.D) && !tk.v.D.cut)   // (the groups know no pole partners)
            restrict_pass19v<T>(cf, tk.v.D, (const T*)tk.x, (const T*)tk.b, tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx,
                                (T*)tk.y, (T*)tk.z, first, stride);
        else
            restrict_pass<S, T>(cf, tk.v.D, (const T*)tk.x, (const T*)tk.b, tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx,
                                (T*)tk.y, (T*)tk.z, first, stride);
    } else if constexpr (OP == BOP_PROLONG) {
        if (tk.v.D.cut)
            for (i64 c = first; c < tk.v.D.n(); c += stride) {
                T* x = (T*)tk.x;
                x[c] = x[c] + prolong_cut_cell<T>(tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx, (const T*)tk.b,
                                                  decode(tk.v.D, c), [](const T* p) { return *p; });
            }
        else if (vec4(tk.v.D))
            prolong_pass_v<T>(tk.v.D, tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx, (const T*)tk.b, (T*)tk.x, first, stride,
                              P == PREC16 ? 2 : 4);
        else
            prolong_pass<T>(tk.v.D, tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx, (const T*)tk.b, (T*)tk.x, first, stride);
    } else if constexpr (OP == BOP_RESID) {   // FP64 outer residual on the fine level (+ FP32 cast)
        const double* b = (const double*)tk.b;
        float* r32 = (float*)tk.y;
        double* scal = tk.scal;
        const double scale = r32 ? scal[SC_SCUR] : 1.0;
        if (r32 && lb == 0 && threadIdx.x == 0) scal[SC_SUSED] = scale;
        double acc = 0.0;
        const float scale32 = (float)scale;   // a power of two: exact in FP32
        const i64 N = tk.v.D.n();
        for (i64 c = first; c < N; c += stride) {
            const C3 cc = decode(tk.v.D, c);
            double r;
            if constexpr (S == 7) {
                Cell7<double> q;
                q.load(tk.v.c64, tk.v.D, cc.j, cc.i, cc.k, XLin<double>{(const double*)tk.x});
                r = q.resid_rows(__ldcs(b + c), __ldcs(tk.a64 + c));
            } else {
                r = resid_rows19(tk.a64, N, (const double*)tk.x, tk.v.D, (int)c, cc, __ldcs(b + c),
                                 tk.v.c64.has(2) ? 19 : 11);
            }
            if (r32) r32[c] = narrow_rn(r) * scale32;
            if (tk.e0) ((float*)tk.e0)[c] = 0.0f;   // the next cycle starts from e = 0
            acc = fma(r, r, acc);
        }
        const double s = block_sum_256(acc, sh);
        if (threadIdx.x == 0) ((double*)tk.z)[lb] = s;
    }
}

// Stencil passes are latency bound: cap their registers for four resident
// CTAs per SM.
template <int P, int OP, int S>
constexpr int min_ctas() {
    if (OP == BOP_LINE) return 2;          // two chunks of 16 rows per thread: fits 128 registers
    if (P == PREC64 || (OP != BOP_GS && OP != BOP_RESTRICT)) return 1;
    if (OP == BOP_GS) return S == 19 ? 2 : 4;   // the 19-point groups hold ~100 values per thread
    if (S == 19) return 2;                 // the 19-point restriction groups hold ~100 values per thread
    return P == PREC32 ? 3 : 1;
}

template <int P, int OP, int S>
__global__ void __launch_bounds__(kBT, min_ctas<P, OP, S>()) k_batch(const BTask* __restrict__ tasks, int ntasks, int total,
                                                const int* __restrict__ active, int colour, int early_trigger,
                                                unsigned long long* stamp) {
    __shared__ double sh[8];
    __shared__ __align__(16) unsigned char tk_raw[sizeof(BTask)];
    __shared__ int tk_index;
    const BTask& tk = *reinterpret_cast<const BTask*>(tk_raw);
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    stamp_start(stamp);
    if (early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        // the block's task descriptor is staged once in shared memory
        if (threadIdx.x == 0) {
            int lo = 0, hi = ntasks - 1;
            while (lo < hi) {                   // last task with block0 <= vb
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&tasks[mid].block0) <= vb) lo = mid;
                else hi = mid - 1;
            }
            tk_index = lo;
        }
        __syncthreads();
        {
            const unsigned* src = reinterpret_cast<const unsigned*>(tasks + tk_index);
            unsigned* dst = reinterpret_cast<unsigned*>(tk_raw);
            for (int w = threadIdx.x; w < (int)(sizeof(BTask) / 4); w += kBT) dst[w] = __ldg(src + w);
        }
        __syncthreads();
        if (active && !active[tk.shell]) {
            __syncthreads();
            continue;
        }
        const int lb = vb - tk.block0;
        const i64 first = (i64)lb * kBT + threadIdx.x;
        const i64 stride = (i64)tk.nblocks * kBT;
        // vector operations: groups of four elements (16-byte aligned arrays),
        // then the remainder
        const bool al = ((reinterpret_cast<uintptr_t>(tk.x) | reinterpret_cast<uintptr_t>(tk.b)) & 15) == 0;
        const i64 n4 = al ? tk.n >> 2 : 0;
        if constexpr (OP == BOP_UPDATE) {
            double* x = (double*)tk.x;
            const float* e = (const float*)tk.b;
            const int k = -pow2_exponent(tk.scal[SC_SUSED]);   // e / s = e * 2^k exactly
            for (i64 g = first; g < n4; g += stride) {
                float E[4];
                double X[4];
                ldg4(e + 4 * g, E);
                ld4(x + 4 * g, X);
                for (int m = 0; m < 4; ++m) X[m] += scaled_widen(E[m], k);
                st4(x + 4 * g, X);
            }
            for (i64 c = 4 * n4 + first; c < tk.n; c += stride) x[c] += scaled_widen(e[c], k);
        } else if constexpr (OP == BOP_POLES) {   // rows 0 and nth - 1 of x -> z [side][j][k]
            typedef typename Prec<P>::T T;
            const Dims& D = tk.v.D;
            const T* x = (const T*)tk.x;
            T* z = (T*)tk.z;
            const i64 per = (i64)D.nr * D.nph;
            for (i64 e = first; e < 2 * per; e += stride) {
                const int side = e >= per ? 1 : 0;
                const i64 r = e - side * per;
                const int j = (int)(r / D.nph), k = (int)(r - (i64)j * D.nph);
                z[e] = x[((i64)j * D.nth + (side ? D.nth - 1 : 0)) * D.nph + k];
            }
        } else if constexpr (OP == BOP_ZERO) {
            unsigned* x = (unsigned*)tk.x;
            for (i64 g = first; g < n4; g += stride) reinterpret_cast<uint4*>(x)[g] = make_uint4(0u, 0u, 0u, 0u);
            for (i64 c = 4 * n4 + first; c < tk.n; c += stride) x[c] = 0u;
        } else if constexpr (OP == BOP_COPY) {
            unsigned* x = (unsigned*)tk.x;
            const unsigned* b = (const unsigned*)tk.b;
            for (i64 g = first; g < n4; g += stride)
                reinterpret_cast<uint4*>(x)[g] = __ldg(reinterpret_cast<const uint4*>(b) + g);
            for (i64 c = 4 * n4 + first; c < tk.n; c += stride) x[c] = b[c];
        } else if constexpr (OP == BOP_SUM) {
            const double* a = (const double*)tk.b;
            const double* w = (const double*)tk.y;
            double acc = 0.0;
            for (i64 c = first; c < tk.n; c += stride) acc += w ? a[c] * w[c] : a[c];
            const double s = block_sum_256(acc, sh);
            if (threadIdx.x == 0) ((double*)tk.z)[lb] = s;
        } else if constexpr (OP == BOP_RHS) {
            double* out = (double*)tk.x;
            const double* f = (const double*)tk.b;
            const double* J = (const double*)tk.y;
            const double mean = tk.scal[SC_SUMJF] / tk.aux;
            double acc = 0.0;
            for (i64 c = first; c < tk.n; c += stride) {
                const double v = J[c] * (f[c] - mean);
                out[c] = v;
                acc = fma(v, v, acc);
            }
            const double s = block_sum_256(acc, sh);
            if (threadIdx.x == 0) ((double*)tk.z)[lb] = s;
        } else if constexpr (OP == BOP_SHIFT) {
            double* x = (double*)tk.x;
            const double m = tk.scal[SC_SUMJX] / tk.aux;
            for (i64 c = first; c < tk.n; c += stride) x[c] -= m;
        } else if constexpr (OP == BOP_FINALIZE) {
            const double* part = (const double*)tk.z;
            double v = 0.0;
            for (int p = threadIdx.x; p < (int)tk.n; p += kBT) v += part[p];
            const double s = block_sum_256(v, sh);
            if (threadIdx.x == 0) {
                tk.scal[tk.slot] = s;
                if (tk.fin_scale) tk.scal[SC_SCUR] = unit_scale_b(s, tk.ncells);
                if (tk.y) ((double*)tk.y)[0] = s;
            }
        } else if constexpr (OP == BOP_COARSE) {
            typedef typename Prec<P>::T T;
            const int lane = threadIdx.x & 31;
            const int n = (int)tk.n;
            const T* r = (const T*)tk.b;
            T* e = (T*)tk.x;
            for (int row = (int)(first >> 5); row < n; row += (int)(stride >> 5)) {
                double s = 0.0;
                for (int m = lane; m < n; m += 32) s += __ldg(tk.binv + (i64)row * n + m) * (double)r[m];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                if (lane == 0) e[row] = (T)s;
            }
        } else {
            run_block<S, P, OP>(tk, colour, first, stride, lb, sh);
        }
        __syncthreads();   // the descriptor is rewritten for the next virtual block
    }
    stamp_end(stamp);
    if (!early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}


// Self-check of narrow_rn and scaled_widen against the hardware conversions on
// a million bit patterns: splitmix64 draws with exponents around the FP32
// range (normal, subnormal and overflowing results), rounding ties of both
// parities, zeros, infinities and NaNs.  Counts mismatches into *bad.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_convert_check(int n, unsigned* bad) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const unsigned long long h = splitmix64((unsigned long long)t);
        // FP64 -> FP32
        unsigned long long e = 1023 - 160 + (h >> 40) % 321;          // 2^-160 .. 2^160
        unsigned long long m = splitmix64(h) & 0xfffffffffffffull;
        if ((t & 7) == 1) m = (m & ~0x1fffffffull) | 0x10000000ull;     // exact tie
        if ((t & 7) == 2) m = (m & ~0x1fffffffull) | 0x0fffffffull;     // just below a tie
        if (t == 3) e = 0, m = 0;                                       // zero
        if (t == 4) e = 0x7ff, m = 0;                                   // infinity
        if (t == 5) e = 0x7ff, m = 1;                                   // NaN
        if (t == 6) e = 1023 + 127, m = 0xfffffffffffffull;             // rounds to infinity
        const double d = __longlong_as_double((long long)(((h & 1) << 63) | (e << 52) | m));
        const float a = narrow_rn(d), b = __double2float_rn(d);
        const bool same = (__float_as_uint(a) == __float_as_uint(b)) || (a != a && b != b);
        // FP32 -> FP64 times 2^k
        const unsigned fb = (unsigned)(splitmix64(h + 1) >> 32);
        const float f = __uint_as_float((t & 15) == 9 ? (fb & 0x807fffffu) : fb);   // some subnormals
        const int k = (int)((h >> 8) % 241) - 120;
        const double w = scaled_widen(f, k), v = ldexp((double)f, k);
        const bool same_w = (__double_as_longlong(w) == __double_as_longlong(v)) || (w != w && v != v);
        if (!same || !same_w) atomicAdd(bad, 1u);
    }
}

bool use_pdl() {
    static const bool on = std::getenv("MG_NO_PDL") == nullptr;
    return on;
}

}  // namespace

template <int P, int OP, int S>
static cudaError_t batch_launch(const BTask* tasks, int ntasks, int total, const int* active, int colour,
                                cudaStream_t s, unsigned long long* stamp) {
    const int early = total <= 152 * 8 ? 1 : 0;   // fits one wave at 8 CTAs per SM
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total, 1, 1);              // one CTA per virtual block
    cfg.blockDim = dim3(kBT, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = use_pdl() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch<P, OP, S>, tasks, ntasks, total, active, colour, early, stamp);
}

template <int P>
static cudaError_t batch_dispatch(const BTask* tasks, int ntasks, int total, const int* active, int op, int colour,
                                  int stencil, cudaStream_t s, unsigned long long* stamp) {
#define STENCIL_OP(OPV)                                                                         \
    case OPV:                                                                                   \
        return stencil == 19 ? batch_launch<P, OPV, 19>(tasks, ntasks, total, active, colour, s, stamp) \
                             : batch_launch<P, OPV, 7>(tasks, ntasks, total, active, colour, s, stamp);
#define PLAIN_OP(OPV) \
    case OPV:         \
        return batch_launch<P, OPV, 0>(tasks, ntasks, total, active, colour, s, stamp);
    switch (op) {
        STENCIL_OP(BOP_GS)
        STENCIL_OP(BOP_JACOBI)
        STENCIL_OP(BOP_LINE)
        STENCIL_OP(BOP_XLINE)
        STENCIL_OP(BOP_RESTRICT)
        STENCIL_OP(BOP_RESID)
        PLAIN_OP(BOP_PROLONG)
        PLAIN_OP(BOP_UPDATE)
        PLAIN_OP(BOP_ZERO)
        PLAIN_OP(BOP_COPY)
        PLAIN_OP(BOP_SUM)
        PLAIN_OP(BOP_RHS)
        PLAIN_OP(BOP_SHIFT)
        PLAIN_OP(BOP_FINALIZE)
        PLAIN_OP(BOP_COARSE)
        PLAIN_OP(BOP_PRES)
        PLAIN_OP(BOP_PRELAX)
        PLAIN_OP(BOP_PRESTRICT)
        PLAIN_OP(BOP_PPROLONG)
        PLAIN_OP(BOP_PUPDATE)
        PLAIN_OP(BOP_POLES)
        default:
            return cudaErrorInvalidValue;
    }
#undef STENCIL_OP
#undef PLAIN_OP
}

namespace {
__global__ void k_stamp_reset(unsigned long long* st, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        st[2 * i] = ~0ull;
        st[2 * i + 1] = 0ull;
    }
}
}  // namespace

cudaError_t launch_stamp_reset(unsigned long long* stamps, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_stamp_reset<<<(n + 255) / 256, 256, 0, s>>>(stamps, n);
    return cudaGetLastError();
}

namespace {
__global__ void __launch_bounds__(256) k_stamp_accum(unsigned long long* st, int n, unsigned long long* acc) {
    __shared__ unsigned long long lo, hi;
    if (threadIdx.x == 0) {
        lo = ~0ull;
        hi = 0ull;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long a = st[2 * i], b = st[2 * i + 1];
        if (a != ~0ull && b >= a) {
            acc[2 * i] += b - a;
            acc[2 * i + 1] += 1;
            atomicMin(&lo, a);
            atomicMax(&hi, b);
        }
        st[2 * i] = ~0ull;
        st[2 * i + 1] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0 && lo != ~0ull) {
        acc[2 * n] += hi - lo;
        acc[2 * n + 1] += 1;
    }
}

__global__ void __launch_bounds__(256) k_loop_check(LoopShell* S, int n, const double* __restrict__ fin,
                                                    int* active, int* passes, cudaGraphConditionalHandle cond) {
    int running = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        LoopShell& q = S[i];
        if (active[i]) {
            q.it += 1;
            q.rr = fin[4 * i + 2];
        }
        if (!q.done) {
            const double rel = sqrt(q.rr) / q.bnorm;
            if (q.it < kLoopHist) q.hist[q.it] = rel;
            q.rel = rel;
            if (!isfinite(rel)) {
                q.why = LOOP_NAN;
                q.done = 1;
            } else if (rel <= q.tol) {
                q.done = 1;
            } else {
                q.best = fmin(q.best, rel);
                if (rel > 1e3 * q.best) {
                    q.why = LOOP_DIVERGED;
                    q.done = 1;
                } else if (q.it >= q.max_iters) {
                    q.why = LOOP_NOCONV;
                    q.done = 1;
                }
            }
        }
        active[i] = q.done ? 0 : 1;
        running |= q.done ? 0 : 1;
    }
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) {
        const int p = passes[0] + 1;
        passes[0] = p;
        cudaGraphSetConditional(cond, (running && p < passes[1]) ? 1u : 0u);
    }
}
}  // namespace

cudaError_t launch_stamp_accum(unsigned long long* stamps, int n, unsigned long long* acc, cudaStream_t s) {
    k_stamp_accum<<<1, 256, 0, s>>>(stamps, n, acc);
    return cudaGetLastError();
}

cudaError_t launch_loop_check(LoopShell* S, int n, const double* fin, int* active, int* passes,
                              cudaGraphConditionalHandle cond, cudaStream_t s) {
    k_loop_check<<<1, 256, 0, s>>>(S, n, fin, active, passes, cond);
    return cudaGetLastError();
}

cudaError_t launch_convert_check(unsigned* bad, cudaStream_t s) {
    k_convert_check<<<512, 256, 0, s>>>(1 << 20, bad);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BTask* tasks, int ntasks, int total_blocks, const int* active, int op, int colour,
                         int stencil, int prec, cudaStream_t s, unsigned long long* stamp) {
    if (ntasks <= 0 || total_blocks <= 0) return cudaSuccess;
    cudaError_t e;
    if (prec == PREC64) e = batch_dispatch<PREC64>(tasks, ntasks, total_blocks, active, op, colour, stencil, s, stamp);
    else if (prec == PREC32)
        e = batch_dispatch<PREC32>(tasks, ntasks, total_blocks, active, op, colour, stencil, s, stamp);
    else e = batch_dispatch<PREC16>(tasks, ntasks, total_blocks, active, op, colour, stencil, s, stamp);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mgs

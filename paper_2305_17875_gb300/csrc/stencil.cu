// stencil.cu - multigrid level operations on the conservative shell operator
// (Section 3.3, Eqs. PC_term1-3): apply, multicolour Gauss-Seidel, weighted
// Jacobi, fused residual + restriction, trilinear prolongation + correction,
// and the coarsest-level dense solve.
#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <type_traits>

#include "mg_kernels.h"
#include "line_smooth.cuh"
#include "xline_smooth.cuh"

namespace mgs {

namespace {

constexpr int kThreads = 256;

int blocks_for(i64 work) {
    i64 b = (work + kThreads - 1) / kThreads;
    const i64 cap = 152 * 16;   // grid-stride beyond 16 resident blocks per SM
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

#define GRID_STRIDE(var, n) \
    for (i64 var = blockIdx.x * (i64)blockDim.x + threadIdx.x; var < (n); var += (i64)gridDim.x * blockDim.x)

// Loads of values that other CTAs of a cluster may have written earlier in the
// same launch go through L2 (CG = true); otherwise plain loads.
template <typename T, bool CG>
__device__ __forceinline__ T ldv(const T* p) {
    if (CG) return __ldcg(p);
    return *p;
}
template <typename T, bool CG>
struct XAcc {
    const T* x;
    Dims D;
    __device__ __forceinline__ T operator()(C3 c) const { return ldv<T, CG>(x + cidx(D, c)); }
};
template <typename T, bool CG>
struct XLinAcc {   // by linear index (Cell7)
    const T* x;
    __device__ __forceinline__ T operator()(int c) const { return ldv<T, CG>(x + c); }
};

// ---- range forms: work items first, first + stride, ... (one launch or one cluster)

// One colour of multicolour Gauss-Seidel, in place: x_c += (b_c - (A x)_c) / A_cc
// for every cell of the colour.  Cells of one colour share no stencil entry, so
// the pass equals the sequential sweep over that colour.
// 7-point: colour (i + j + k) mod 2.  19-point: ((i + j) mod 2) + 2 ((j + k) mod 2).
// On the full sphere the 19-point cells of a colour couple across the pole;
// poles (the first and last rows as the pass starts) gives them the values
// of the colour's simultaneous update.
template <int S, typename T, typename CF, bool CG>
__device__ __forceinline__ void gs_colour_range(const CF& cf, const Dims& D, T* x, const T* b, int colour,
                                                i64 first, i64 stride, const T* poles = nullptr) {
    const int hk = D.nph >> 1;
    if constexpr (S == 7) {   // the 7-point fast form (same arithmetic as the batched passes)
        const i64 work = (i64)D.nr * D.nth * hk;
        for (i64 t = first; t < work; t += stride) {
            int kk, i, j;
            decode_half(D, t, kk, i, j);
            Cell7<T> q;
            q.load(cf, D, j, i, 2 * kk + ((colour + i + j) & 1), XLinAcc<T, CG>{x});
            x[q.c] = q.gs(ldv<T, CG>(b + q.c));
        }
    } else {   // rows with (i + j) = colour mod 2 only; the neighbourhood in registers
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
            X.load(XLinAcc<T, CG>{x}, D, c, p, !cf.has(2), poles);
            const T r = ldv<T, CG>(b + c) - apply19<T>(cf, X, D, c, p);
            x[c] = X.v[0] + r / diag_cell<S, T>(cf, D, p);
        }
    }
}

// rc(C) = sum over the children c of C of (b - A x)_c; optionally zero ec.
template <int S, typename T, typename CF, bool CG>
__device__ __forceinline__ void restrict_range(const CF& cf, const Dims& D, const T* x, const T* b, const Dims& Dc,
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
                        q.load(cf, D, c.j, c.i, c.k, XLinAcc<T, CG>{x});
                        s += q.resid(ldv<T, CG>(b + q.c));
                    } else {
                        const int id = cidx(D, c);
                        Nbr19<T> X;
                        X.load(XLinAcc<T, CG>{x}, D, id, c, !cf.has(2));
                        s += ldv<T, CG>(b + id) - apply19<T>(cf, X, D, id, c);
                    }
                }
        rc[t] = s;
        if (ec_zero) ec_zero[t] = 0;
    }
}

// 1-D cell-centred linear weights of fine cell f from a grid halved by c:
// child s of coarse cell C sits at C + (2s - 1)/4, so it takes 3/4 of C and
// 1/4 of C -/+ 1 (the mirror C itself at a wall, wrapped when periodic).
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

// x += P ec (cell-centred trilinear).
template <typename T, bool CG>
__device__ __forceinline__ void prolong_range(const Dims& D, const Dims& Dc, int cz, int ce, int cx, const T* ec,
                                              T* x, i64 first, i64 stride) {
    if (D.cut) {   // full sphere: colatitude partners across the poles
        for (i64 c = first; c < D.n(); c += stride)
            x[c] = ldv<T, CG>(x + c) +
                   prolong_cut_cell<T>(Dc, cz, ce, cx, ec, decode(D, c), [](const T* p) { return ldv<T, CG>(p); });
        return;
    }
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
                    s = fma((T)wj[a] * (T)wi[bb] * (T)wk[e], ldv<T, CG>(ec + cidx(Dc, ij[a], ii[bb], ik[e])), s);
                }
            }
        }
        x[c] = ldv<T, CG>(x + c) + s;
    }
}

// e = Binv r (FP64 accumulate), one warp per row.
template <typename T, bool CG>
__device__ __forceinline__ void coarse_range(const double* binv, int n, const T* r, T* e, int warp_first,
                                             int warp_stride) {
    const int lane = threadIdx.x & 31;
    for (int row = warp_first; row < n; row += warp_stride) {
        double s = 0.0;
        for (int m = lane; m < n; m += 32) s += __ldg(binv + (i64)row * n + m) * (double)ldv<T, CG>(r + m);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) e[row] = (T)s;
    }
}

// ---- one-launch kernels
template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_apply(CF cf, Dims D, const T* __restrict__ x, T* __restrict__ y) {
    XRead<T> X{x, D};
    GRID_STRIDE(c, D.n()) { y[c] = apply_cell<S, T>(cf, X, D, decode(D, c)); }
}

template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_gs(CF cf, Dims D, T* x, const T* __restrict__ b, int colour,
                                                 const T* __restrict__ poles) {
    gs_colour_range<S, T, CF, false>(cf, D, x, b, colour, blockIdx.x * (i64)blockDim.x + threadIdx.x,
                                     (i64)gridDim.x * blockDim.x, poles);
}

// Rows 0 and nth - 1 of x into poles [side][j][k] (before a 19-point colour
// pass on the full sphere).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_poles(Dims D, const T* __restrict__ x, T* __restrict__ poles) {
    const i64 per = (i64)D.nr * D.nph;
    GRID_STRIDE(e, 2 * per) {
        const int side = e >= per ? 1 : 0;
        const i64 r = e - side * per;
        const int j = (int)(r / D.nph), k = (int)(r - (i64)j * D.nph);
        poles[e] = x[((i64)j * D.nth + (side ? D.nth - 1 : 0)) * D.nph + k];
    }
}

// One colour of the radial-line Gauss-Seidel sweep (line_smooth.cuh).
template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads, 2) k_line(CF cf, Dims D, T* x, const T* __restrict__ b,
                                                    const T* __restrict__ fac, int colour) {
    line_pass<S, T>(cf, D, x, b, fac, colour, blockIdx.x, gridDim.x);
}

template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_xline(CF cf, Dims D, T* x, const T* __restrict__ b,
                                                     const T* __restrict__ fac, T* work, int colour) {
    xline_pass<S, T>(cf, D, x, b, fac, work, colour, blockIdx.x * (i64)blockDim.x + threadIdx.x,
                     (i64)gridDim.x * blockDim.x);
}

// Weighted Jacobi, out of place: xo = x + omega (b - A x) / diag(A).
template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_jacobi(CF cf, Dims D, const T* __restrict__ x, T* __restrict__ xo,
                                                      const T* __restrict__ b, T omega) {
    XRead<T> X{x, D};
    GRID_STRIDE(c, D.n()) {
        const C3 cc = decode(D, c);
        const T r = b[c] - apply_cell<S, T>(cf, X, D, cc);
        xo[c] = x[c] + omega * r / diag_cell<S, T>(cf, D, cc);
    }
}

template <int S, typename T, typename CF>
__global__ void __launch_bounds__(kThreads) k_restrict(CF cf, Dims D, const T* __restrict__ x, const T* __restrict__ b,
                                                        Dims Dc, int cz, int ce, int cx, T* __restrict__ rc,
                                                        T* __restrict__ ec_zero) {
    restrict_range<S, T, CF, false>(cf, D, x, b, Dc, cz, ce, cx, rc, ec_zero,
                                    blockIdx.x * (i64)blockDim.x + threadIdx.x, (i64)gridDim.x * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_prolong(Dims D, Dims Dc, int cz, int ce, int cx, const T* __restrict__ ec,
                                                       T* __restrict__ x) {
    prolong_range<T, false>(D, Dc, cz, ce, cx, ec, x, blockIdx.x * (i64)blockDim.x + threadIdx.x,
                            (i64)gridDim.x * blockDim.x);
}

template <typename T>
__global__ void k_coarse(const double* __restrict__ binv, int n, const T* __restrict__ r, T* __restrict__ e) {
    coarse_range<T, false>(binv, n, r, e, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                           (gridDim.x * blockDim.x) >> 5);
}

// ---- the coarse tail: every level from the tail's top to the coarsest in one
// launch, one thread-block cluster per task, a cluster barrier between phases.
template <int P>
struct CoefOf;
template <>
struct CoefOf<PREC64> {
    typedef CoefF64 type;
    __device__ static const CoefF64& get(const LevelView& v) { return v.c64; }
};
template <>
struct CoefOf<PREC32> {
    typedef CoefF32 type;
    __device__ static const CoefF32& get(const LevelView& v) { return v.c32; }
};
template <>
struct CoefOf<PREC16> {
    typedef CoefF16 type;
    __device__ static const CoefF16& get(const LevelView& v) { return v.c16; }
};

template <int S, typename T, int P>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const TailTask* __restrict__ tasks, int csize,
                                                          unsigned long long* stamp) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const TailTask& tk = tasks[blockIdx.x / csize];
    stamp_start(stamp);
    if (tk.active && !tk.active[tk.shell]) {           // uniform over the cluster
        stamp_end(stamp);
        return;
    }
    const i64 first = (i64)cl.block_rank() * blockDim.x + threadIdx.x;
    const i64 stride = (i64)csize * blockDim.x;
    const int ncol = S == 7 ? 2 : 4;
    const int nl = tk.nlev;
    for (int l = 0; l < nl - 1; ++l) {
        const TailLevel& L = tk.lev[l];
        const TailLevel& C = tk.lev[l + 1];
        const auto& cf = CoefOf<P>::get(L.v);
        for (int sw = 0; sw < tk.nu1; ++sw)
            for (int c = 0; c < ncol; ++c) {
                gs_colour_range<S, T, typename CoefOf<P>::type, true>(cf, L.v.D, (T*)L.e, (const T*)L.r, c, first,
                                                                      stride);
                cl.sync();
            }
        restrict_range<S, T, typename CoefOf<P>::type, true>(cf, L.v.D, (const T*)L.e, (const T*)L.r, C.v.D,
                                                             L.v.cz, L.v.ce, L.v.cx, (T*)C.r, (T*)C.e, first,
                                                             stride);
        cl.sync();
    }
    coarse_range<T, true>(tk.binv, tk.ncoarse, (const T*)tk.lev[nl - 1].r, (T*)tk.lev[nl - 1].e, (int)(first >> 5),
                          (int)(stride >> 5));
    cl.sync();
    for (int l = nl - 2; l >= 0; --l) {
        const TailLevel& L = tk.lev[l];
        const TailLevel& C = tk.lev[l + 1];
        const auto& cf = CoefOf<P>::get(L.v);
        prolong_range<T, true>(L.v.D, C.v.D, L.v.cz, L.v.ce, L.v.cx, (const T*)C.e, (T*)L.e, first, stride);
        cl.sync();
        for (int sw = 0; sw < tk.nu2; ++sw)
            for (int c = 0; c < ncol; ++c) {
                gs_colour_range<S, T, typename CoefOf<P>::type, true>(cf, L.v.D, (T*)L.e, (const T*)L.r, c, first,
                                                                      stride);
                cl.sync();
            }
    }
    stamp_end(stamp);
}

// ---- the coarse tail in the cluster's shared memory (layout in
// tail_sm_layout).  Each CTA works on the cells it holds; a neighbour held by
// another CTA is read through the cluster's shared-memory window.  Per cell
// the arithmetic is that of k_tail (Cell7 or Nbr19 + apply19 + diag_cell,
// the same restriction, prolongation and coarse rows), so both forms give
// the same bits.  Not for the full sphere's 19-point cells (no pole copy).

// One level array spread over the cluster, read through the cluster's
// shared-memory window (32-bit addresses) and written by the CTA that holds
// the cell through its own shared memory.
template <typename T>
struct SmArr {
    T* p;             // this CTA's chunk
    unsigned base;    // the same as a shared-memory address
    int sh;
    int me;           // this CTA's rank
    __device__ __forceinline__ unsigned off(int c) const {
        return base + (unsigned)(c & ((1 << sh) - 1)) * (unsigned)sizeof(T);
    }
    // any cell (a CTA's own cells map to its own shared memory)
    __device__ __forceinline__ T operator()(int c) const {
        unsigned a;
        asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(off(c)), "r"((unsigned)(c >> sh)));
        T v;
        if constexpr (sizeof(T) == 4)
            asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
        else
            asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
        return v;
    }
    // a cell this CTA holds
    __device__ __forceinline__ void st(int c, T v) const {
        if constexpr (sizeof(T) == 4) asm volatile("st.shared.f32 [%0], %1;" ::"r"(off(c)), "f"(v) : "memory");
        else asm volatile("st.shared.f64 [%0], %1;" ::"r"(off(c)), "d"(v) : "memory");
    }
};
// The three 7-point components of a level, as the global readers give them.
template <typename T>
struct SmCoef7 {
    SmArr<T> g0, g4, g8;
    __device__ __forceinline__ T operator()(int a, i64 idx) const {
        return a == 0 ? g0((int)idx) : (a == 4 ? g4((int)idx) : g8((int)idx));
    }
};
// The nine 19-point components (consecutive arrays; an absent one, as on an
// axisymmetric mapping, is never read: has() says so as the global readers do).
template <typename T>
struct SmCoef19 {
    SmArr<T> g0;        // component a at g0 + a arrays
    unsigned astride;   // bytes between components
    int n;              // values per array
    unsigned mask;      // bit a: component a stored
    __device__ __forceinline__ bool has(int a) const { return (mask >> a) & 1u; }
    __device__ __forceinline__ T operator()(int a, i64 idx) const {
        SmArr<T> q = g0;
        q.base += (unsigned)a * astride;
        return q((int)idx);
    }
    __device__ __forceinline__ T* chunk(int a) const { return g0.p + a * n; }
};
template <int S, typename T>
struct SmLevel {
    SmArr<T> e, r;
    typename std::conditional<S == 7, SmCoef7<T>, SmCoef19<T>>::type cf;
    int lo, hi;   // the cells this CTA holds
};
template <int S, typename T>
__device__ __forceinline__ SmLevel<S, T> sm_level(unsigned char* dyn, const TailSmLayout& L, const Dims& D, int l,
                                                  int rank, unsigned mask = 0) {
    const int s = L.sh[l];
    T* b = reinterpret_cast<T*>(dyn + L.off[l]);
    const int n = 1 << s;
    const unsigned a = (unsigned)__cvta_generic_to_shared(b);
    const unsigned w = (unsigned)(n * sizeof(T));
    SmLevel<S, T> v;
    v.e = SmArr<T>{b, a, s, rank};
    v.r = SmArr<T>{b + n, a + w, s, rank};
    if constexpr (S == 7)
        v.cf = SmCoef7<T>{{b + 2 * n, a + 2 * w, s, rank}, {b + 3 * n, a + 3 * w, s, rank},
                          {b + 4 * n, a + 4 * w, s, rank}};
    else
        v.cf = SmCoef19<T>{{b + 2 * n, a + 2 * w, s, rank}, w, n, mask};
    v.lo = rank << s;
    v.hi = min((rank + 1) << s, (int)D.n());
    return v;
}

// One colour of the pass (gs_colour_range).  7 points: item t is cell 2t or
// 2t + 1, so the items of the cells a CTA holds are t in [lo / 2, hi / 2).
// 19 points: the CTA's cells of the colour ((i + j) mod 2 + 2 ((j + k) mod 2)).
template <int S, typename T>
__device__ __forceinline__ void sm_gs(const SmLevel<S, T>& V, const Dims D, int colour) {
    if constexpr (S == 7) {
        const int work = D.nr * D.nth * (D.nph >> 1);
        const int t1 = min(V.hi >> 1, work);
        for (int t = (V.lo >> 1) + threadIdx.x; t < t1; t += blockDim.x) {
            int kk, i, j;
            decode_half(D, t, kk, i, j);
            Cell7<T> q;
            q.load(V.cf, D, j, i, 2 * kk + ((colour + i + j) & 1), V.e);
            V.e.st(q.c, q.gs(V.r(q.c)));
        }
    } else {
        for (int c = V.lo + threadIdx.x; c < V.hi; c += blockDim.x) {
            const C3 p = decode(D, c);
            if (((p.i + p.j) & 1) + 2 * ((p.j + p.k) & 1) != colour) continue;
            Nbr19<T> X;
            X.load(V.e, D, c, p, !V.cf.has(2));
            const T r = V.r(c) - apply19<T>(V.cf, X, D, c, p);
            V.e.st(c, X.v[0] + r / diag_cell<S, T>(V.cf, D, p));
        }
    }
}

// Residual restricted into the coarse cells this CTA holds (restrict_range),
// their correction zeroed.
template <int S, typename T>
__device__ __forceinline__ void sm_restrict(const SmLevel<S, T>& F, const Dims D, const SmLevel<S, T>& C,
                                            const Dims Dc, int cz, int ce, int cx) {
    for (int t = C.lo + threadIdx.x; t < C.hi; t += blockDim.x) {
        const C3 P = decode(Dc, t);
        T s = 0;
        for (int dj = 0; dj < ce; ++dj)
            for (int di = 0; di < cz; ++di)
                for (int dk = 0; dk < cx; ++dk) {
                    if constexpr (S == 7) {
                        Cell7<T> q;
                        q.load(F.cf, D, ce * P.j + dj, cz * P.i + di, cx * P.k + dk, F.e);
                        s += q.resid(F.r(q.c));
                    } else {
                        const C3 c{ce * P.j + dj, cz * P.i + di, cx * P.k + dk};
                        const int id = cidx(D, c);
                        Nbr19<T> X;
                        X.load(F.e, D, id, c, !F.cf.has(2));
                        s += F.r(id) - apply19<T>(F.cf, X, D, id, c);
                    }
                }
        C.r.st(t, s);
        C.e.st(t, (T)0);
    }
}

// x += P ec on the fine cells this CTA holds (prolong_range).
template <int S, typename T>
__device__ __forceinline__ void sm_prolong(const SmLevel<S, T>& F, const Dims D, const SmLevel<S, T>& C,
                                           const Dims Dc, int cz, int ce, int cx) {
    for (int c = F.lo + threadIdx.x; c < F.hi; c += blockDim.x) {
        T* xc = F.e.p + (c - F.lo);   // this CTA's own cell
        if (D.cut) {
            // prolong_cut_cell reads through addresses: offsets from a base
            const T* base = C.e.p;
            *xc = *xc + prolong_cut_cell<T>(Dc, cz, ce, cx, base, decode(D, c),
                                            [&](const T* p) { return C.e((int)(p - base)); });
            continue;
        }
        const C3 f = decode(D, c);
        int ij[2], ii[2], ik[2];
        float wj[2], wi[2], wk[2];
        lin1d(f.j, ce, Dc.nr, false, ij, wj);
        lin1d(f.i, cz, Dc.nth, false, ii, wi);
        lin1d(f.k, cx, Dc.nph, true, ik, wk);
        T s = 0;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a >= ce) break;
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                if (bb >= cz) break;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (e >= cx) break;
                    s = fma((T)wj[a] * (T)wi[bb] * (T)wk[e], C.e(cidx(Dc, ij[a], ii[bb], ik[e])), s);
                }
            }
        }
        *xc = *xc + s;
    }
}

// e = Binv r on the coarsest rows this CTA holds, one warp per row
// (coarse_range).
// e = Binv r on the coarsest rows this CTA holds, one warp per row
// (coarse_range's sums: each lane over m = lane, lane + 32, ..., then the
// shuffle tree).  rd: the coarsest r converted to FP64 once, in this CTA's
// shared memory; the lane's loads of a block of eight terms go out together.
template <int S, typename T>
__device__ __forceinline__ void sm_coarse(const double* binv, const double* rd, int n, const SmLevel<S, T>& V) {
    const int lane = threadIdx.x & 31;
    const int hi = min(V.hi, n);
    for (int row = V.lo + (int)(threadIdx.x >> 5); row < hi; row += (int)(blockDim.x >> 5)) {
        const double* brow = binv + (i64)row * n;
        double s = 0.0;
        for (int m0 = lane; m0 < n; m0 += 32 * 8) {
            double bv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) bv[u] = m0 + 32 * u < n ? __ldg(brow + m0 + 32 * u) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (m0 + 32 * u < n) s += bv[u] * rd[m0 + 32 * u];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) V.e.st(row, (T)s);
    }
}

// Threads of a shared-memory tail CTA (FP64 and 19 points halve them for
// registers).
template <int S, typename T>
constexpr int tail_sm_threads() {
    return (sizeof(T) == 8 || S == 19) ? kTailSmThreads / 2 : kTailSmThreads;
}

// Asynchronous 4- or 8-byte copy global -> this CTA's shared memory.
template <typename T>
__device__ __forceinline__ void cp_async_val(T* sdst, const T* gsrc) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte values");
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    if constexpr (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// count values from global to this CTA's shared memory, spread over the
// CTA's threads: 16-byte copies when both ends are 16-byte aligned, the rest
// one value at a time.
template <typename T>
__device__ __forceinline__ void stage_span(T* sdst, const T* gsrc, int count) {
    constexpr int V = 16 / (int)sizeof(T);
    int done = 0;
    if (((reinterpret_cast<uintptr_t>(gsrc) | reinterpret_cast<uintptr_t>(sdst)) & 15) == 0) {
        const int nv = count / V;
        for (int q = threadIdx.x; q < nv; q += blockDim.x) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(sdst + q * V);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc + q * V) : "memory");
        }
        done = nv * V;
    }
    for (int q = done + (int)threadIdx.x; q < count; q += blockDim.x) cp_async_val<T>(sdst + q, gsrc + q);
}

template <int S, typename T, int P>
__global__ void __launch_bounds__(tail_sm_threads<S, T>(), 1) k_tail_sm(const TailTask* __restrict__ tasks, int csize,
                                                                     unsigned long long* stamp) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ TailSmLayout lay;
    __shared__ unsigned comp[kMaxTail];   // per level: the stored components (19 points)
    cg::cluster_group cl = cg::this_cluster();
    const TailTask& tk = tasks[blockIdx.x / csize];
    stamp_start(stamp);
    if (tk.active && !tk.active[tk.shell]) {   // uniform over the cluster
        stamp_end(stamp);
        return;
    }
    const int rank = (int)cl.block_rank();
    const int nl = tk.nlev;
    if (threadIdx.x == 0) {
        tail_sm_layout(tk, csize, (int)sizeof(T), lay);
        for (int l = 0; l < nl; ++l) {
            unsigned m = 0;
            for (int a = 0; a < 9; ++a) m |= CoefOf<P>::get(tk.lev[l].v).has(a) ? 1u << a : 0u;
            comp[l] = m;
        }
    }
    __syncthreads();
    auto level = [&](int l) { return sm_level<S, T>(dyn, lay, tk.lev[l].v.D, l, rank, comp[l]); };
    // stage (copies all in flight at once): the components of every level, e
    // and r of the first, this CTA's rows of Binv toward L2
    for (int l = 0; l < nl; ++l) {
        const auto& cf = CoefOf<P>::get(tk.lev[l].v);
        const SmLevel<S, T> V = level(l);
        const int cnt = V.hi - V.lo;
        if (cnt <= 0) continue;
        if constexpr (S == 7) {
            if constexpr (P == PREC16) {   // FP16 storage: converted as the global readers do
                for (int c = V.lo + threadIdx.x; c < V.hi; c += blockDim.x) {
                    const int o = c - V.lo;
                    V.cf.g0.p[o] = (T)cf(0, c);
                    V.cf.g4.p[o] = (T)cf(4, c);
                    V.cf.g8.p[o] = (T)cf(8, c);
                }
            } else {
                stage_span<T>(V.cf.g0.p, cf.g[0] + V.lo, cnt);
                stage_span<T>(V.cf.g4.p, cf.g[4] + V.lo, cnt);
                stage_span<T>(V.cf.g8.p, cf.g[8] + V.lo, cnt);
            }
        } else {
            for (int a = 0; a < 9; ++a) {
                if (!cf.has(a)) continue;
                T* dst = V.cf.chunk(a);
                if constexpr (P == PREC16) {
                    for (int c = V.lo + threadIdx.x; c < V.hi; c += blockDim.x) dst[c - V.lo] = (T)cf(a, c);
                } else {
                    stage_span<T>(dst, cf.g[a] + V.lo, cnt);
                }
            }
        }
        if (l == 0) {
            stage_span<T>(V.e.p, (const T*)tk.lev[0].e + V.lo, cnt);
            stage_span<T>(V.r.p, (const T*)tk.lev[0].r + V.lo, cnt);
        }
    }
    {
        const SmLevel<S, T> V = level(nl - 1);
        const int n = tk.ncoarse;
        const i64 b0 = (i64)V.lo * n, b1 = (i64)min(V.hi, n) * n;
        for (i64 q = b0 + 16 * (i64)threadIdx.x; q < b1; q += 16 * (i64)blockDim.x)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(tk.binv + q));
    }
    cp_async_wait_all();
    cl.sync();
    constexpr int ncol = S == 7 ? 2 : 4;
    for (int l = 0; l < nl - 1; ++l) {
        const LevelView& A = tk.lev[l].v;
        const SmLevel<S, T> F = level(l);
        for (int sw = 0; sw < tk.nu1; ++sw)
            for (int c = 0; c < ncol; ++c) {
                sm_gs<S, T>(F, A.D, c);
                cl.sync();
            }
        const SmLevel<S, T> C = level(l + 1);
        sm_restrict<S, T>(F, A.D, C, tk.lev[l + 1].v.D, A.cz, A.ce, A.cx);
        cl.sync();
    }
    {
        const SmLevel<S, T> V = level(nl - 1);
        double* rd = reinterpret_cast<double*>(dyn + lay.rd_off);
        for (int m = threadIdx.x; m < tk.ncoarse; m += blockDim.x) rd[m] = (double)V.r(m);
        __syncthreads();
        sm_coarse<S, T>(tk.binv, rd, tk.ncoarse, V);
    }
    cl.sync();
    for (int l = nl - 2; l >= 0; --l) {
        const LevelView& A = tk.lev[l].v;
        const SmLevel<S, T> F = level(l);
        const SmLevel<S, T> C = level(l + 1);
        sm_prolong<S, T>(F, A.D, C, tk.lev[l + 1].v.D, A.cz, A.ce, A.cx);
        cl.sync();
        for (int sw = 0; sw < tk.nu2; ++sw)
            for (int c = 0; c < ncol; ++c) {
                sm_gs<S, T>(F, A.D, c);
                cl.sync();
            }
    }
    // the top level's correction back to global memory
    const SmLevel<S, T> V = level(0);
    for (int c = V.lo + threadIdx.x; c < V.hi; c += blockDim.x) ((T*)tk.lev[0].e)[c] = V.e.p[c - V.lo];
    stamp_end(stamp);
}

}  // namespace

// Dispatch on (precision, stencil): T = value type, cf = coefficient reader.
#define MG_DISPATCH(lv, prec, ...)                                           \
    do {                                                                     \
        if ((prec) == PREC64) {                                              \
            typedef double T;                                                \
            const CoefF64& cf = (lv).c64;                                    \
            if ((lv).stencil == 19) { constexpr int S = 19; __VA_ARGS__; }   \
            else { constexpr int S = 7; __VA_ARGS__; }                       \
        } else if ((prec) == PREC32) {                                       \
            typedef float T;                                                 \
            const CoefF32& cf = (lv).c32;                                    \
            if ((lv).stencil == 19) { constexpr int S = 19; __VA_ARGS__; }   \
            else { constexpr int S = 7; __VA_ARGS__; }                       \
        } else {                                                             \
            typedef float T;                                                 \
            const CoefF16& cf = (lv).c16;                                    \
            if ((lv).stencil == 19) { constexpr int S = 19; __VA_ARGS__; }   \
            else { constexpr int S = 7; __VA_ARGS__; }                       \
        }                                                                    \
    } while (0)

cudaError_t launch_apply(const LevelView& lv, int prec, const void* x, void* y, cudaStream_t s) {
    const int nb = blocks_for(lv.D.n());
    MG_DISPATCH(lv, prec, (k_apply<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (const T*)x, (T*)y)));
    return cudaGetLastError();
}

cudaError_t launch_gs_colour(const LevelView& lv, int prec, void* x, const void* b, int colour,
                             cudaStream_t s, const void* poles) {
    const int nb = blocks_for((i64)lv.D.nr * lv.D.nth * (lv.D.nph / 2));
    MG_DISPATCH(lv, prec, (k_gs<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (T*)x, (const T*)b, colour,
                                                              (const T*)poles)));
    return cudaGetLastError();
}

cudaError_t launch_poles(const LevelView& lv, int prec, const void* x, void* poles, cudaStream_t s) {
    const int nb = blocks_for(2LL * lv.D.nr * lv.D.nph);
    if (prec == PREC64) k_poles<double><<<nb, kThreads, 0, s>>>(lv.D, (const double*)x, (double*)poles);
    else k_poles<float><<<nb, kThreads, 0, s>>>(lv.D, (const float*)x, (float*)poles);
    return cudaGetLastError();
}

cudaError_t launch_line_colour(const LevelView& lv, int prec, void* x, const void* b, const void* fac,
                               int colour, cudaStream_t s) {
    const int kc = prec == PREC64 ? LineRows<double>::kC : LineRows<float>::kC;
    const i64 lines = line_count(lv.D, lv.stencil, colour);
    const int nb = blocks_for(lines * line_chunks(lv.D.nr, kc));
    MG_DISPATCH(lv, prec, (k_line<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (T*)x, (const T*)b, (const T*)fac,
                                                                colour)));
    return cudaGetLastError();
}

cudaError_t launch_xline_colour(const LevelView& lv, int prec, void* x, const void* b, const void* fac,
                                void* work, int colour, cudaStream_t s) {
    const int nb = blocks_for(xline_items(lv.D, lv.stencil));
    MG_DISPATCH(lv, prec, (k_xline<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (T*)x, (const T*)b, (const T*)fac,
                                                                 (T*)work, colour)));
    return cudaGetLastError();
}

cudaError_t launch_jacobi(const LevelView& lv, int prec, const void* x, void* xo, const void* b,
                          cudaStream_t s) {
    const int nb = blocks_for(lv.D.n());
    const double omega = lv.stencil == 7 ? 6.0 / 7.0 : 4.0 / 5.0;
    MG_DISPATCH(lv, prec, (k_jacobi<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (const T*)x, (T*)xo,
                                                                  (const T*)b, (T)omega)));
    return cudaGetLastError();
}

cudaError_t launch_restrict_residual(const LevelView& lv, Dims Dc, int prec, const void* x,
                                     const void* b, void* rc, void* ec_zero, cudaStream_t s) {
    const int nb = blocks_for(Dc.n());
    MG_DISPATCH(lv, prec, (k_restrict<S, T><<<nb, kThreads, 0, s>>>(cf, lv.D, (const T*)x, (const T*)b, Dc,
                                                                    lv.cz, lv.ce, lv.cx, (T*)rc, (T*)ec_zero)));
    return cudaGetLastError();
}

cudaError_t launch_prolong_add(const LevelView& lv, Dims Dc, int prec, const void* ec, void* x,
                               cudaStream_t s) {
    const int nb = blocks_for(lv.D.n());
    if (prec == PREC64)
        k_prolong<double><<<nb, kThreads, 0, s>>>(lv.D, Dc, lv.cz, lv.ce, lv.cx, (const double*)ec, (double*)x);
    else
        k_prolong<float><<<nb, kThreads, 0, s>>>(lv.D, Dc, lv.cz, lv.ce, lv.cx, (const float*)ec, (float*)x);
    return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const double* binv, int n, int prec, const void* r, void* e,
                                cudaStream_t s) {
    const int rows_per_block = kThreads / 32;
    int nb = (n + rows_per_block - 1) / rows_per_block;
    if (nb > 152 * 4) nb = 152 * 4;
    if (prec == PREC64)
        k_coarse<double><<<nb, kThreads, 0, s>>>(binv, n, (const double*)r, (double*)e);
    else
        k_coarse<float><<<nb, kThreads, 0, s>>>(binv, n, (const float*)r, (float*)e);
    return cudaGetLastError();
}

// The tail kernel of (stencil, precision); the shared-memory form when smem > 0.
template <int S, typename T, int P>
static void* tail_kernel(size_t smem) {
    if (smem > 0) return reinterpret_cast<void*>(k_tail_sm<S, T, P>);
    return reinterpret_cast<void*>(k_tail<S, T, P>);
}

static void tail_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int ntasks, int csize, size_t smem,
                        int sm_threads, cudaStream_t s) {
    cfg = {};
    cfg.gridDim = dim3(ntasks * csize, 1, 1);
    cfg.blockDim = dim3(smem > 0 ? sm_threads : kTailThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

// Kernel attributes, set once per kernel: the shared-memory form's dynamic
// shared memory limit; clusters above the portable 8 CTAs.
static cudaError_t tail_attrs(const void* k, size_t smem, int csize) {
    static std::mutex mu;
    static std::map<const void*, size_t> smem_done;
    static std::map<const void*, bool> wide_done;
    std::lock_guard<std::mutex> lk(mu);
    if (smem > smem_done[k]) {
        const cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmMaxBytes);
        if (e != cudaSuccess) return e;
        smem_done[k] = kTailSmMaxBytes;
    }
    if (csize > 8 && !wide_done[k]) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        wide_done[k] = true;
    }
    return cudaSuccess;
}

template <int S, typename T, int P>
static cudaError_t tail_launch(const TailTask* tasks, int ntasks, int csize, cudaStream_t s,
                               unsigned long long* stamp, size_t smem) {
    if (smem > kTailSmMaxBytes) return cudaErrorInvalidValue;
    if (csize < 1 || csize > kTailMaxCluster) return cudaErrorInvalidValue;
    const void* k = tail_kernel<S, T, P>(smem);
    const cudaError_t ea = tail_attrs(k, smem, csize);
    if (ea != cudaSuccess) return ea;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    tail_config(cfg, attr, ntasks, csize, smem, tail_sm_threads<S, T>(), s);
    void* args[] = {(void*)&tasks, (void*)&csize, (void*)&stamp};
    return cudaLaunchKernelExC(&cfg, k, args);
}

template <int S, typename T, int P>
static int tail_clusters(int csize, size_t smem) {
    if (smem > kTailSmMaxBytes) return 0;
    if (csize < 1 || csize > kTailMaxCluster) return 0;
    const void* k = tail_kernel<S, T, P>(smem);
    if (tail_attrs(k, smem, csize) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    tail_config(cfg, attr, 1, csize, smem, tail_sm_threads<S, T>(), nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int tail_max_clusters(int csize, int stencil, int prec, size_t smem) {
    if (prec == PREC64)
        return stencil == 19 ? tail_clusters<19, double, PREC64>(csize, smem)
                             : tail_clusters<7, double, PREC64>(csize, smem);
    if (prec == PREC32)
        return stencil == 19 ? tail_clusters<19, float, PREC32>(csize, smem)
                             : tail_clusters<7, float, PREC32>(csize, smem);
    return stencil == 19 ? tail_clusters<19, float, PREC16>(csize, smem) : tail_clusters<7, float, PREC16>(csize, smem);
}

cudaError_t launch_tail(const TailTask* tasks, int ntasks, int csize, int stencil, int prec, cudaStream_t s,
                        unsigned long long* stamp, size_t smem) {
    cudaError_t e;
    if (prec == PREC64)
        e = stencil == 19 ? tail_launch<19, double, PREC64>(tasks, ntasks, csize, s, stamp, smem)
                          : tail_launch<7, double, PREC64>(tasks, ntasks, csize, s, stamp, smem);
    else if (prec == PREC32)
        e = stencil == 19 ? tail_launch<19, float, PREC32>(tasks, ntasks, csize, s, stamp, smem)
                          : tail_launch<7, float, PREC32>(tasks, ntasks, csize, s, stamp, smem);
    else
        e = stencil == 19 ? tail_launch<19, float, PREC16>(tasks, ntasks, csize, s, stamp, smem)
                          : tail_launch<7, float, PREC16>(tasks, ntasks, csize, s, stamp, smem);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mgs

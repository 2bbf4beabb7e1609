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

#include "mg_kernels.h"

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

// multicolour Gauss-Seidel colour pass (same cell mapping as stencil.cu)
template <int S, typename T, typename CF>
__device__ __forceinline__ void gs_pass(const CF& cf, const Dims& D, T* x, const T* b, int colour, i64 first,
                                        i64 stride) {
    XRead<T> X{x, D};
    const int hk = D.nph >> 1;
    const i64 work = (i64)D.nr * D.nth * hk;
    for (i64 t = first; t < work; t += stride) {
        int kk, i, j;
        decode_half(D, t, kk, i, j);
        int k;
        if (S == 7) {
            k = 2 * kk + ((colour + i + j) & 1);
        } else {
            if (((i + j) & 1) != (colour & 1)) continue;
            k = 2 * kk + (((colour >> 1) + j) & 1);
        }
        if constexpr (S == 7) {
            Cell7<T> q;
            q.load(cf, D, j, i, k, XLin<T>{x});
            x[q.c] = q.gs(b[q.c]);
        } else {
            const C3 c{j, i, k};
            const i64 id = cidx(D, c);
            const T r = b[id] - apply_cell<S, T>(cf, X, D, c);
            x[id] = x[id] + r / diag_cell<S, T>(cf, D, c);
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
    XRead<T> X{x, D};
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
                        s += b[cidx(D, c)] - apply_cell<S, T>(cf, X, D, c);
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
        for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb)
                for (int e = 0; e < 2; ++e) {
                    const T w = (T)wj[a] * (T)wi[bb] * (T)wk[e];
                    if (w != (T)0) s += w * ec[cidx(Dc, ij[a], ii[bb], ik[e])];
                }
        x[c] = x[c] + s;
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
        gs_pass<S, T>(cf, tk.v.D, (T*)tk.x, (const T*)tk.b, colour, first, stride);
    } else if constexpr (OP == BOP_JACOBI) {
        jacobi_pass<S, T>(cf, tk.v.D, (const T*)tk.x, (T*)tk.y, (const T*)tk.b, first, stride);
    } else if constexpr (OP == BOP_RESTRICT) {
        restrict_pass<S, T>(cf, tk.v.D, (const T*)tk.x, (const T*)tk.b, tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx,
                            (T*)tk.y, (T*)tk.z, first, stride);
    } else if constexpr (OP == BOP_PROLONG) {
        prolong_pass<T>(tk.v.D, tk.Dc, tk.v.cz, tk.v.ce, tk.v.cx, (const T*)tk.b, (T*)tk.x, first, stride);
    } else if constexpr (OP == BOP_RESID) {   // FP64 outer residual on the fine level (+ FP32 cast)
        XRead<double> X{(const double*)tk.x, tk.v.D};
        const double* b = (const double*)tk.b;
        float* r32 = (float*)tk.y;
        double* scal = tk.scal;
        const double scale = r32 ? scal[SC_SCUR] : 1.0;
        if (r32 && lb == 0 && threadIdx.x == 0) scal[SC_SUSED] = scale;
        double acc = 0.0;
        for (i64 c = first; c < tk.v.D.n(); c += stride) {
            double r;
            if constexpr (S == 7) {
                const C3 cc = decode(tk.v.D, c);
                Cell7<double> q;
                q.load(tk.v.c64, tk.v.D, cc.j, cc.i, cc.k, XLin<double>{(const double*)tk.x});
                r = q.resid(b[c]);
            } else {
                r = residual_cell<S>(tk.v.c64, X, tk.v.D, decode(tk.v.D, c), b[c]);
            }
            if (r32) r32[c] = (float)(r * scale);
            acc = fma(r, r, acc);
        }
        const double s = block_sum_256(acc, sh);
        if (threadIdx.x == 0) ((double*)tk.z)[lb] = s;
    }
}

template <int P, int OP, int S>
__global__ void __launch_bounds__(kBT) k_batch(const BTask* __restrict__ tasks, int ntasks, int total,
                                                const int* __restrict__ active, int colour, int early_trigger) {
    __shared__ double sh[8];
    __shared__ __align__(16) unsigned char tk_raw[sizeof(BTask)];
    __shared__ int tk_index;
    const BTask& tk = *reinterpret_cast<const BTask*>(tk_raw);
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
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
        if constexpr (OP == BOP_UPDATE) {
            double* x = (double*)tk.x;
            const float* e = (const float*)tk.b;
            const double inv = 1.0 / tk.scal[SC_SUSED];
            for (i64 c = first; c < tk.n; c += stride) x[c] = fma((double)e[c], inv, x[c]);
        } else if constexpr (OP == BOP_ZERO) {
            unsigned* x = (unsigned*)tk.x;
            for (i64 c = first; c < tk.n; c += stride) x[c] = 0u;
        } else if constexpr (OP == BOP_COPY) {
            unsigned* x = (unsigned*)tk.x;
            const unsigned* b = (const unsigned*)tk.b;
            for (i64 c = first; c < tk.n; c += stride) x[c] = b[c];
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
    if (!early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}


// ---- one red-black sweep of the 7-point operator per launch (overlapped tiles)
//
// A CTA owns a tile of kRbJ x kRbI x kRbK cells.  It stages the old iterate on
// the tile plus a 2-cell ring in shared memory, updates the red cells of the
// tile plus a 1-cell ring in place (red cells read only black neighbours),
// then the black cells of the tile in place (they read only red neighbours,
// now new), and writes the tile to the output array.  The ring work is
// repeated by the neighbouring tiles; the input array is never written, so
// the result is the sequential sweep "all red, then all black".
// Ring entries outside the radial / colatitude walls are clamped copies that
// only ever meet zero wall coefficients; longitude wraps.
constexpr int kRgJ = kRbJ + 4, kRgI = kRbI + 4, kRgK = kRbK + 4;
constexpr int kRB7 = 512;   // threads per tile

template <typename T, typename CF>
struct Faces7b {
    T el, eu, zl, zu, xl, xu;
    __device__ __forceinline__ void load(const CF& cf, const Dims& D, int j, int i, int k) {
        const int c = cidx(D, j, i, k);
        const int plane = D.nth * D.nph;
        el = (T)cf(4, c);
        eu = j + 1 < D.nr ? (T)cf(4, c + plane) : (T)0;
        zl = (T)cf(0, c);
        zu = i + 1 < D.nth ? (T)cf(0, c + D.nph) : (T)0;
        xl = (T)cf(8, c);
        xu = (T)cf(8, c - k + (k + 1 == D.nph ? 0 : k + 1));
    }
    // x_c + (b - A x)_c / A_cc from the six neighbour values
    __device__ __forceinline__ T update(T b, T xc, T xel, T xeu, T xzl, T xzu, T xxl, T xxu) const {
        const T ax = eu * (xeu - xc) - el * (xc - xel) + zu * (xzu - xc) - zl * (xc - xzl) +
                     xu * (xxu - xc) - xl * (xc - xxl);
        const T dg = -(el + eu + zl + zu + xl + xu);
        return xc + (b - ax) / dg;
    }
};

__device__ __forceinline__ int wrap_k(const Dims& D, int k) {   // k >= -nph
    const int kp = k + D.nph;
    return kp - D.nph * (int)D.dph.div((unsigned)kp);
}
__device__ __forceinline__ int clamp_to(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

template <typename T, typename CF>
__device__ void rb7_tile(const BTask& tk, const CF& cf, int lb, T* sx) {
    const Dims& D = tk.v.D;
    const int ntk = (D.nph + kRbK - 1) / kRbK, nti = (D.nth + kRbI - 1) / kRbI;
    const int tkk = lb % ntk, tii = (lb / ntk) % nti, tjj = lb / (ntk * nti);
    const int j0 = tjj * kRbJ, i0 = tii * kRbI, k0 = tkk * kRbK;
    const T* __restrict__ x = (const T*)tk.x;
    const T* __restrict__ b = (const T*)tk.b;
    T* __restrict__ out = (T*)tk.y;
    auto S = [&](int jj, int ii, int kk) -> T& { return sx[(jj * kRgI + ii) * kRgK + kk]; };

    // 1. old iterate on tile + 2-cell ring, copied asynchronously (all issued, then one wait)
    for (int w = threadIdx.x; w < kRgJ * kRgI * kRgK; w += kRB7) {
        const int jj = w / (kRgI * kRgK), rem = w - jj * (kRgI * kRgK);
        const int ii = rem / kRgK, kk = rem - ii * kRgK;
        const int j = clamp_to(j0 - 2 + jj, D.nr), i = clamp_to(i0 - 2 + ii, D.nth);
        const int k = wrap_k(D, k0 - 2 + kk);
        const unsigned sa = (unsigned)__cvta_generic_to_shared(sx + w);
        const T* g = x + cidx(D, j, i, k);
        if (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g));
        else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g));
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();

    // 2. red cells ((i + j + k) even) of tile + 1-cell ring, in place
    constexpr int NJ = kRbJ + 2, NI = kRbI + 2, NK2 = (kRbK + 2) / 2;
#pragma unroll 2
    for (int w = threadIdx.x; w < NJ * NI * NK2; w += kRB7) {
        const int jj = w / (NI * NK2), rem = w - jj * (NI * NK2);
        const int ii = rem / NK2, m = rem - ii * NK2;
        const int j = j0 - 1 + jj, i = i0 - 1 + ii;
        if (j < 0 || j >= D.nr || i < 0 || i >= D.nth) continue;
        const int kk = 2 * m + ((j + i + k0 - 1) & 1);        // first red in the row
        const int kw = wrap_k(D, k0 - 1 + kk);
        Faces7b<T, CF> F;
        F.load(cf, D, j, i, kw);
        const int a = jj + 1, c = ii + 1, e = kk + 1;         // region coordinates
        S(a, c, e) = F.update(b[cidx(D, j, i, kw)], S(a, c, e), S(a - 1, c, e), S(a + 1, c, e), S(a, c - 1, e),
                              S(a, c + 1, e), S(a, c, e - 1), S(a, c, e + 1));
    }
    __syncthreads();

    // 3. black cells of the tile, in place
    constexpr int BK2 = kRbK / 2;
#pragma unroll 2
    for (int w = threadIdx.x; w < kRbJ * kRbI * BK2; w += kRB7) {
        const int jj = w / (kRbI * BK2), rem = w - jj * (kRbI * BK2);
        const int ii = rem / BK2, m = rem - ii * BK2;
        const int j = j0 + jj, i = i0 + ii;
        const int kk = 2 * m + (((j + i + k0) & 1) ^ 1);      // first black in the row
        const int k = k0 + kk;
        if (j >= D.nr || i >= D.nth || k >= D.nph) continue;
        Faces7b<T, CF> F;
        F.load(cf, D, j, i, k);
        const int a = jj + 2, c = ii + 2, e = kk + 2;
        S(a, c, e) = F.update(b[cidx(D, j, i, k)], S(a, c, e), S(a - 1, c, e), S(a + 1, c, e), S(a, c - 1, e),
                              S(a, c + 1, e), S(a, c, e - 1), S(a, c, e + 1));
    }
    __syncthreads();

    // 4. the tile out, coalesced along longitude
#pragma unroll 4
    for (int w = threadIdx.x; w < kRbJ * kRbI * kRbK; w += kRB7) {
        const int jj = w / (kRbI * kRbK), rem = w - jj * (kRbI * kRbK);
        const int ii = rem / kRbK, kk = rem - ii * kRbK;
        const int j = j0 + jj, i = i0 + ii, k = k0 + kk;
        if (j >= D.nr || i >= D.nth || k >= D.nph) continue;
        out[cidx(D, j, i, k)] = S(jj + 2, ii + 2, kk + 2);
    }
}

template <int P>
__global__ void __launch_bounds__(kRB7) k_rb7(const BTask* __restrict__ tasks, int ntasks, int total,
                                              const int* __restrict__ active, int early_trigger) {
    typedef typename Prec<P>::T T;
    extern __shared__ __align__(16) unsigned char dyn[];
    T* sx = reinterpret_cast<T*>(dyn);
    __shared__ __align__(16) unsigned char tk_raw[sizeof(BTask)];
    __shared__ int tk_index;
    const BTask& tk = *reinterpret_cast<const BTask*>(tk_raw);
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = ntasks - 1;
            while (lo < hi) {
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
            for (int w = threadIdx.x; w < (int)(sizeof(BTask) / 4); w += kRB7) dst[w] = __ldg(src + w);
        }
        __syncthreads();
        if (!active || active[tk.shell]) rb7_tile<T>(tk, Prec<P>::cf(tk.v), vb - tk.block0, sx);
        __syncthreads();
    }
    if (!early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

bool use_pdl() {
    static const bool on = std::getenv("MG_NO_PDL") == nullptr;
    return on;
}

}  // namespace

template <int P, int OP, int S>
static cudaError_t batch_launch(const BTask* tasks, int ntasks, int total, const int* active, int colour,
                                cudaStream_t s) {
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
    return cudaLaunchKernelEx(&cfg, k_batch<P, OP, S>, tasks, ntasks, total, active, colour, early);
}

template <int P>
static cudaError_t batch_dispatch(const BTask* tasks, int ntasks, int total, const int* active, int op, int colour,
                                  int stencil, cudaStream_t s) {
#define STENCIL_OP(OPV)                                                                         \
    case OPV:                                                                                   \
        return stencil == 19 ? batch_launch<P, OPV, 19>(tasks, ntasks, total, active, colour, s) \
                             : batch_launch<P, OPV, 7>(tasks, ntasks, total, active, colour, s);
#define PLAIN_OP(OPV) \
    case OPV:         \
        return batch_launch<P, OPV, 0>(tasks, ntasks, total, active, colour, s);
    switch (op) {
        STENCIL_OP(BOP_GS)
        STENCIL_OP(BOP_JACOBI)
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
        default:
            return cudaErrorInvalidValue;
    }
#undef STENCIL_OP
#undef PLAIN_OP
}

template <int P>
static cudaError_t rb7_launch(const BTask* tasks, int ntasks, int total, const int* active, cudaStream_t s) {
    typedef typename Prec<P>::T T;
    const size_t smem = sizeof(T) * kRgJ * kRgI * kRgK;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_rb7<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int early = total <= 152 * 2 ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total, 1, 1);
    cfg.blockDim = dim3(kRB7, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = use_pdl() ? 1 : 0;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_rb7<P>, tasks, ntasks, total, active, early);
}

cudaError_t launch_batch(const BTask* tasks, int ntasks, int total_blocks, const int* active, int op, int colour,
                         int stencil, int prec, cudaStream_t s) {
    if (ntasks <= 0 || total_blocks <= 0) return cudaSuccess;
    cudaError_t e;
    if (op == BOP_RB7) {
        if (prec == PREC64) e = rb7_launch<PREC64>(tasks, ntasks, total_blocks, active, s);
        else if (prec == PREC32) e = rb7_launch<PREC32>(tasks, ntasks, total_blocks, active, s);
        else e = rb7_launch<PREC16>(tasks, ntasks, total_blocks, active, s);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (prec == PREC64) e = batch_dispatch<PREC64>(tasks, ntasks, total_blocks, active, op, colour, stencil, s);
    else if (prec == PREC32) e = batch_dispatch<PREC32>(tasks, ntasks, total_blocks, active, op, colour, stencil, s);
    else e = batch_dispatch<PREC16>(tasks, ntasks, total_blocks, active, op, colour, stencil, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mgs

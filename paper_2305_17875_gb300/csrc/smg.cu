// smg.cu - set-up of the plane hierarchies of the semi-coarsening multigrid
// (plane_smooth.cuh): the plane operator of every 3-D level, its radius
// coarsening R B P, and the periodic line factors of every 2-D level.  FP64.
#include "mg_kernels.h"
#include "plane_smooth.cuh"

namespace mgs {

namespace {

int sgrid(i64 n, int threads) {
    i64 b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

struct Nine {
    double* c[9];
};
struct NineC {
    const double* c[9];
};

// The plane block of the 7-point operator: centre A_cc (all six faces, the
// colatitude ones included), radius and longitude neighbours from the face
// coefficients; the corners are zero.  Faces on the radius walls carry no
// flux (lower wall rows store zero; upper ones are not read).
__global__ void k_plane_op0(CoefF64 cf, Dims D, Nine out) {
    const int plane = D.nth * D.nph;
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < D.n(); t += (i64)gridDim.x * blockDim.x) {
        const C3 p = decode(D, t);
        const int c = (int)t;
        const int kp = p.k == D.nph - 1 ? c - D.nph + 1 : c + 1;
        // the six face coefficients of Cell7 (lower wall rows store zero)
        const double el = cf(4, c);
        const double eu = p.j + 1 < D.nr ? cf(4, c + plane) : 0.0;
        const double zl = cf(0, c);
        const double zu = p.i + 1 < D.nth ? cf(0, c + D.nph) : 0.0;
        const double xl = cf(8, c);
        const double xu = cf(8, kp);
        out.c[0][t] = -(el + eu + zl + zu + xl + xu);
        out.c[1][t] = el;
        out.c[2][t] = eu;
        out.c[3][t] = xl;
        out.c[4][t] = xu;
        for (int o = 5; o < 9; ++o) out.c[o][t] = 0.0;
    }
}

// Coarse plane operator R B P (radius halved): entry (dJ, dk) of coarse cell
// (J, i, k) = sum over the children j = 2J, 2J+1 and the fine entries
// (dj, dk) of B(j) times the prolongation weight of fine row j + dj on coarse
// row J + dJ.
__global__ void k_plane_coarsen(NineC f, Dims D, Dims Dc, Nine out) {
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < Dc.n(); t += (i64)gridDim.x * blockDim.x) {
        const C3 C = decode(Dc, t);
        double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int dj2 = 0; dj2 < 2; ++dj2) {
            const int j = 2 * C.j + dj2;
            const int fc = (j * D.nth + C.i) * D.nph + C.k;
            for (int o = 0; o < 9; ++o) {
                const int j2 = j + plane_dj(o);
                if (j2 < 0 || j2 >= D.nr) continue;
                const double b = f.c[o][fc];
                if (b == 0.0) continue;
                for (int dJ = -1; dJ <= 1; ++dJ) {
                    const int J2 = C.j + dJ;
                    if (J2 < 0 || J2 >= Dc.nr) continue;
                    const double wgt = plane_pw(j2, J2, Dc.nr);
                    if (wgt == 0.0) continue;
                    // the coarse entry with offsets (dJ, dk of o)
                    const int dk = plane_dk(o);
                    const int oc = dJ == 0 ? (dk == 0 ? 0 : (dk < 0 ? 3 : 4))
                                           : (dk == 0 ? (dJ < 0 ? 1 : 2)
                                                      : (dJ < 0 ? (dk < 0 ? 5 : 6) : (dk < 0 ? 7 : 8)));
                    v[oc] = fma(b, wgt, v[oc]);
                }
            }
        }
        for (int o = 0; o < 9; ++o) out.c[o][t] = v[o];
    }
}

// Factors of every longitude line (fixed j, i) of a 2-D level, the
// cyclic tridiagonal part of the plane operator on the line: a_k = entry
// (0, -1), b_k = centre, c_k = entry (0, +1); the layout of xline_smooth.cuh
// (normalised elimination of the leading block, psi2 = T_c^{-1} (-a_0, 0, ..,
// -c_{n-2}), and in the last cell's slot c_{n-1}, the closure's reciprocal,
// a_{n-1}).  FP64 elimination; psi2's backward pass reads the stored factors.
template <typename T>
__global__ void k_plane_factors(NineC f, Dims D, T* fac, unsigned* bad) {
    const i64 N = D.n();
    const i64 lines = (i64)D.nr * D.nth;
    const int n = D.nph;
    T* alpha = fac;
    T* beta = fac + N;
    T* gamma = fac + 2 * N;
    T* psi2 = fac + 3 * N;
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < lines; t += (i64)gridDim.x * blockDim.x) {
        const i64 c0 = t * n;
        auto A = [&](int k, int m) {   // entry (row k, column m) of the line block
            const int d = m - k;
            const int dk = d == 0 ? 0 : ((d == 1 || d == 1 - n) ? 1 : -1);
            return f.c[dk == 0 ? 0 : (dk < 0 ? 3 : 4)][c0 + k];
        };
        bool ok = true;
        double cprev = 0.0, q = 0.0;
        for (int k = 0; k < n - 1; ++k) {
            const double lo = k > 0 ? A(k, k - 1) : 0.0;
            const double dd = A(k, k);
            const double up = k < n - 2 ? A(k, k + 1) : 0.0;
            const double ib = 1.0 / (dd - lo * cprev);
            const double a = -lo * ib;
            cprev = up * ib;
            double e = 0.0;
            if (k == 0) e -= A(0, n - 1);
            if (k == n - 2) e -= A(n - 2, n - 1);
            q = fma(a, q, ib * e);
            ok = ok && isfinite(ib) && isfinite(a) && isfinite(cprev);
            alpha[c0 + k] = (T)a;
            beta[c0 + k] = (T)ib;
            gamma[c0 + k] = (T)(-cprev);
            psi2[c0 + k] = (T)q;
        }
        double e = 0.0, p2_first = 0.0, p2_last = 0.0;
        for (int k = n - 2; k >= 0; --k) {
            e = fma((double)gamma[c0 + k], e, (double)psi2[c0 + k]);
            psi2[c0 + k] = (T)e;
            if (k == n - 2) p2_last = e;
            if (k == 0) p2_first = e;
        }
        const double an = A(n - 1, n - 2), cn = A(n - 1, 0), bn = A(n - 1, n - 1);
        const double inv = 1.0 / (bn + cn * p2_first + an * p2_last);
        ok = ok && isfinite(inv);
        alpha[c0 + n - 1] = (T)cn;
        beta[c0 + n - 1] = (T)inv;
        gamma[c0 + n - 1] = (T)an;
        psi2[c0 + n - 1] = (T)0;
        if (!ok) atomicAdd(bad, 1u);
    }
}

}  // namespace

cudaError_t launch_plane_op0(const LevelView& lv, double* const out[9], cudaStream_t s) {
    Nine o;
    for (int a = 0; a < 9; ++a) o.c[a] = out[a];
    k_plane_op0<<<sgrid(lv.D.n(), 128), 128, 0, s>>>(lv.c64, lv.D, o);
    return cudaGetLastError();
}

cudaError_t launch_plane_coarsen(const double* const fine[9], const Dims& D, const Dims& Dc, double* const out[9],
                                 cudaStream_t s) {
    NineC f;
    Nine o;
    for (int a = 0; a < 9; ++a) {
        f.c[a] = fine[a];
        o.c[a] = out[a];
    }
    k_plane_coarsen<<<sgrid(Dc.n(), 128), 128, 0, s>>>(f, D, Dc, o);
    return cudaGetLastError();
}

cudaError_t launch_plane_factors(const double* const c[9], const Dims& D, int prec, void* fac, unsigned* bad,
                                 cudaStream_t s) {
    NineC f;
    for (int a = 0; a < 9; ++a) f.c[a] = c[a];
    const i64 lines = (i64)D.nr * D.nth;
    if (prec == PREC64) k_plane_factors<double><<<sgrid(lines, 128), 128, 0, s>>>(f, D, (double*)fac, bad);
    else k_plane_factors<float><<<sgrid(lines, 128), 128, 0, s>>>(f, D, (float*)fac, bad);
    return cudaGetLastError();
}

}  // namespace mgs

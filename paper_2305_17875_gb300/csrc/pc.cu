// pc.cu - the steps either side of the pressure solve (Section 3.6) on a
// staggered velocity: the right side of Eq. PC_6 and the correction of
// Eq. PC_7.
//
// The intermediate velocity u*** is given by its Cartesian components at the
// centre of every cell's three lower faces (the layout of the face metric):
// 9 arrays of N doubles, component 3 d + a = Cartesian a (x1, x2, x3) on the
// face normal to d (zeta, eta, xi).  Wall faces carry no flux: the lower wall
// faces' entries are not read, upper wall faces are not stored.
//
// Right side: the contravariant flux through a d-face is U_d = sum_a C_da u_a
// with the face's own C (Eq. skewness); the cell's flux balance D(U) is the
// discrete d_j(C_ji u_i) of Eq. PC_6 with unit computational spacing, and
// f = D(U) / |J^{-1}| is the pointwise right side mg_solve takes (its answer
// is x = h dP).
// Correction: at every interior face u_a -= (1/|J^{-1}|_face) sum_p C_pa g_p,
// g the gradient of the operator's face flux (Eqs. PC_term1-3: the normal
// difference; for 19 points the averaged tangential differences with mirror
// ghosts and longitude wrap).  Since C C^T / |J^{-1}| = G at the face, the
// corrected contravariant flux is U_d - F_d(x) with F_d the operator's face
// flux, so D(corrected U) = D(U) - A x: the solver's residual.
#include <cstdio>
#include <string>

#include "engine.h"
#include "pc.h"

namespace mgs {
namespace {

constexpr int kPT = 256;

struct FaceC {
    const double* C[27];
    const double* inv[3];
};
struct FaceU {
    const double* u[9];
};
struct FaceUw {
    double* u[9];
};

__device__ __forceinline__ double flux(const FaceC& F, const FaceU& U, int d, int c) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) s = fma(__ldg(F.C[9 * d + 3 * d + a] + c), __ldg(U.u[3 * d + a] + c), s);
    return s;
}

__global__ void __launch_bounds__(kPT) k_pc_rhs(FaceC F, FaceU U, const double* __restrict__ J, Dims D,
                                               double* __restrict__ f) {
    const int plane = D.nth * D.nph;
    for (i64 cl = blockIdx.x * (i64)blockDim.x + threadIdx.x; cl < D.n(); cl += (i64)gridDim.x * blockDim.x) {
        const int c = (int)cl;
        const C3 p = decode(D, cl);
        double s = 0.0;
        if (p.i + 1 < D.nth) s += flux(F, U, 0, c + D.nph);     // upper zeta face
        if (p.i > 0) s -= flux(F, U, 0, c);                     // lower zeta face
        if (p.j + 1 < D.nr) s += flux(F, U, 1, c + plane);
        if (p.j > 0) s -= flux(F, U, 1, c);
        s += flux(F, U, 2, p.k + 1 < D.nph ? c + 1 : c + 1 - D.nph);
        s -= flux(F, U, 2, c);
        f[c] = s / __ldg(J + c);
    }
}

// gradient of the operator's flux at the lower d-face of cell p (interior face)
template <int S>
__device__ __forceinline__ void face_grad(const double* __restrict__ x, const Dims& D, int d, C3 p, double g[3]) {
    const C3 U = p;
    const C3 L = d == 0 ? shift<0>(p, -1, D) : (d == 1 ? shift<1>(p, -1, D) : shift<2>(p, -1, D));
    auto X = [&](C3 c) { return __ldg(x + cidx(D, c)); };
    g[0] = g[1] = g[2] = 0.0;
    g[d] = X(U) - X(L);
    if (S == 19) {
        if (d != 0)
            g[0] = ((X(shift<0>(L, 1, D)) + X(shift<0>(U, 1, D))) - (X(shift<0>(L, -1, D)) + X(shift<0>(U, -1, D)))) * 0.25;
        if (d != 1)
            g[1] = ((X(shift<1>(L, 1, D)) + X(shift<1>(U, 1, D))) - (X(shift<1>(L, -1, D)) + X(shift<1>(U, -1, D)))) * 0.25;
        if (d != 2)
            g[2] = ((X(shift<2>(L, 1, D)) + X(shift<2>(U, 1, D))) - (X(shift<2>(L, -1, D)) + X(shift<2>(U, -1, D)))) * 0.25;
    }
}

template <int S>
__global__ void __launch_bounds__(kPT) k_pc_correct(FaceC F, FaceUw U, const double* __restrict__ x, Dims D) {
    for (i64 cl = blockIdx.x * (i64)blockDim.x + threadIdx.x; cl < D.n(); cl += (i64)gridDim.x * blockDim.x) {
        const int c = (int)cl;
        const C3 p = decode(D, cl);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if ((d == 0 && p.i == 0) || (d == 1 && p.j == 0)) continue;   // wall face: unchanged
            double g[3];
            face_grad<S>(x, D, d, p, g);
            const double inv = __ldg(F.inv[d] + c);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < 3; ++q) s = fma(__ldg(F.C[9 * d + 3 * q + a] + c), g[q], s);
                U.u[3 * d + a][c] -= inv * s;
            }
        }
    }
}

int pc_blocks(i64 n) {
    i64 b = (n + kPT - 1) / kPT;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

// Face C and 1/|J^{-1}| on first use (30 arrays of N doubles, owned by the handle).
mg_status ensure_face_C(mg_handle* h) {
    if (h->pcC[0]) return MG_OK;
    const i64 N = h->L[0].D.n();
    double* C[27];
    double* inv[3];
    for (int q = 0; q < 27; ++q)
        if (!(C[q] = (double*)handle_alloc(h, sizeof(double) * N))) return MG_ENOMEM;
    for (int d = 0; d < 3; ++d)
        if (!(inv[d] = (double*)handle_alloc(h, sizeof(double) * N))) return MG_ENOMEM;
    const cudaError_t e = launch_face_C(h->mtab, h->L[0].D, C, inv, h->stream);
    if (e != cudaSuccess) {
        set_error(std::string("face C: ") + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    for (int q = 0; q < 27; ++q) h->pcC[q] = C[q];
    for (int d = 0; d < 3; ++d) h->pcInv[d] = inv[d];
    return MG_OK;
}

FaceC face_C(const mg_handle* h) {
    FaceC F;
    for (int q = 0; q < 27; ++q) F.C[q] = h->pcC[q];
    for (int d = 0; d < 3; ++d) F.inv[d] = h->pcInv[d];
    return F;
}

mg_status finish(mg_handle* h, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_out, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->user_stream, h->ev_out, 0);
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return MG_ECUDA;
    }
    return MG_OK;
}

mg_status start(mg_handle* h) {
    if (h->opts.metric != MG_METRIC_DISCRETE) {
        set_error("the pressure-correction steps need the discrete metric of Section 3.2");
        return MG_EINVAL;
    }
    if (cudaEventRecord(h->ev_in, h->user_stream) != cudaSuccess ||
        cudaStreamWaitEvent(h->stream, h->ev_in, 0) != cudaSuccess) {
        set_error("stream join failed");
        return MG_ECUDA;
    }
    return MG_OK;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mg_status mg_pc_rhs(mg_handle* h, const double* u_face, double* f) {
    if (!h || !u_face || !f) {
        set_error("mg_pc_rhs: null argument");
        return MG_EINVAL;
    }
    mg_status st = start(h);
    if (st == MG_OK) st = ensure_face_C(h);
    if (st != MG_OK) return st;
    const Dims& D = h->L[0].D;
    const i64 N = D.n();
    FaceU U;
    for (int q = 0; q < 9; ++q) U.u[q] = u_face + q * N;
    k_pc_rhs<<<pc_blocks(N), kPT, 0, h->stream>>>(face_C(h), U, h->J64, D, f);
    return finish(h, "mg_pc_rhs");
}

extern "C" mg_status mg_pc_correct(mg_handle* h, const double* x, double* u_face) {
    if (!h || !x || !u_face) {
        set_error("mg_pc_correct: null argument");
        return MG_EINVAL;
    }
    mg_status st = start(h);
    if (st == MG_OK) st = ensure_face_C(h);
    if (st != MG_OK) return st;
    const Dims& D = h->L[0].D;
    const i64 N = D.n();
    FaceUw U;
    for (int q = 0; q < 9; ++q) U.u[q] = u_face + q * N;
    if (h->stencil == 19) k_pc_correct<19><<<pc_blocks(N), kPT, 0, h->stream>>>(face_C(h), U, x, D);
    else k_pc_correct<7><<<pc_blocks(N), kPT, 0, h->stream>>>(face_C(h), U, x, D);
    return finish(h, "mg_pc_correct");
}

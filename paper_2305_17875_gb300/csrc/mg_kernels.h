// mg_kernels.h - host-side launchers of the device kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include "mg_internal.cuh"

namespace mgs {

// One multigrid level as the kernels see it.
struct LevelView {
    Dims D;
    int cz, ce, cx;          // halving factors to the next level (0 = coarsest)
    int stencil;             // 7 or 19
    CoefF64 c64;
    CoefF32 c32;
    CoefF16 c16;
};

enum { PREC64 = 0, PREC32 = 1, PREC16 = 2 };

// ---- setup (metric.cu)
struct MetricTables {
    const double* rho;   // radius of vertex planes j = -1 .. nr + 1   (index j + 1)
    const double* cth;   // cos/sin colatitude of planes i = -1 .. nth + 1
    const double* sth;
    const double* cph;   // cos/sin longitude of planes k = -1 .. nph + 1 (wrapped)
    const double* sph;
    double ax1, ax2;     // x1 scale (1 - flattening), x2 scale (1 + e2)
};
cudaError_t launch_face_metric(const MetricTables& t, Dims D, int stencil, double* const g[9],
                               double* J, cudaStream_t s);
cudaError_t launch_coarsen_faces(const LevelView& fine, Dims Dc, double* const gc[9], cudaStream_t s);
cudaError_t launch_cast32(const double* src, float* dst, i64 n, cudaStream_t s);
cudaError_t launch_cast16(const double* src, __half* dst, i64 n, float inv_scale, cudaStream_t s);
cudaError_t launch_dense_operator(const LevelView& lv, double* A, cudaStream_t s);

// ---- reductions (solve.cu); partials has room for kRedBlocks doubles
constexpr int kRedBlocks = 1216;   // 8 x 152 SMs; fixed so results are reproducible
int red_blocks(i64 n);
cudaError_t launch_sum(const double* a, const double* w, i64 n, double* partials, cudaStream_t s);
cudaError_t launch_absmax(const double* a, i64 n, double* partials, cudaStream_t s);
cudaError_t launch_finalize(const double* partials, int nparts, int op, double* out, cudaStream_t s);

// ---- level operations (stencil.cu); x/b/y are double* for PREC64, float* otherwise
cudaError_t launch_apply(const LevelView& lv, int prec, const void* x, void* y, cudaStream_t s);
cudaError_t launch_gs_colour(const LevelView& lv, int prec, void* x, const void* b, int colour,
                             cudaStream_t s);
cudaError_t launch_jacobi(const LevelView& lv, int prec, const void* x, void* xo, const void* b,
                          cudaStream_t s);
cudaError_t launch_restrict_residual(const LevelView& lv, Dims Dc, int prec, const void* x,
                                     const void* b, void* rc, void* ec_zero, cudaStream_t s);
cudaError_t launch_prolong_add(const LevelView& lv, Dims Dc, int prec, const void* ec, void* x,
                               cudaStream_t s);
cudaError_t launch_coarse_solve(const double* binv, int n, int prec, const void* r, void* e,
                                cudaStream_t s);

// ---- outer FP64 pieces (solve.cu)
// r = b - A64 x; writes r32 = float(r * scale) when r32 != nullptr and
// partials of ||r||^2 (red_blocks(n) doubles).
cudaError_t launch_outer_residual(const LevelView& lv, const double* x, const double* b, float* r32,
                                  double scale, double* partials, cudaStream_t s);
// x += e * inv_scale
cudaError_t launch_update(double* x, const float* e, double inv_scale, i64 n, cudaStream_t s);
// b = J (f - num[0] / den), partials of ||b||^2
cudaError_t launch_rhs(const double* J, const double* f, const double* num, double den, double* b,
                       i64 n, double* partials, cudaStream_t s);
// x -= num[0] / den
cudaError_t launch_shift(double* x, const double* num, double den, i64 n, cudaStream_t s);

}  // namespace mgs

// pc.h - the steps either side of the pressure solve (Section 3.6) and the
// implicit viscous sweeps (Section 3.4): internal interface between set-up
// (metric.cu) and the step kernels (pc.cu, adi.cu).
#pragma once

#include "mg_kernels.h"

namespace mgs {

// C of every cell's three lower faces (Section 3.2, Eq. skewness: C_pa =
// |J^{-1}| dzeta_p/dx_a of the face), 27 arrays at index 9 d + 3 p + a (face
// normal d and row p in zeta, eta, xi order, Cartesian column a), and
// 1 / |J^{-1}| of the face, 3 arrays.
cudaError_t launch_face_C(const MetricTables& t, Dims D, double* const C[27], double* const inv_det[3],
                          cudaStream_t s);

// Tables of the analytic metric option at half-index resolution (entry t at
// index t / 2): radius and d radius / d eta (2 nr + 1 entries), cos / sin of
// the colatitude (2 nth + 1) and of the longitude (2 nph + 1).
struct AnalyticTables {
    const double* rho;
    const double* drho;
    const double* cth;
    const double* sth;
    const double* cph;
    const double* sph;
    double dth, dph;     // d th / d zeta, d ph / d xi
    double ax1, ax2;     // x1 scale (1 - flattening), x2 scale (1 + e2)
};
cudaError_t launch_face_metric_analytic(const AnalyticTables& t, Dims D, int stencil, double* const g[9],
                                        double* J, cudaStream_t s);

// G_dd on the wall planes: g[0], g[1] the radius walls j = 0 and j = nr
// ([nth][nph]), g[2], g[3] the colatitude walls i = 0 and i = nth ([nr][nph]).
cudaError_t launch_wall_G(const MetricTables& t, Dims D, double* const g[4], cudaStream_t s);

}  // namespace mgs

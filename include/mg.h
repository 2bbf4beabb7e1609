/*
 * mg.h - C ABI of the GB300 shell pressure-correction Poisson solver.
 *
 * The library solves the pressure-correction Poisson equation of the
 * generalized-curvilinear shell solver (Section 3.6, Eq. PC_6),
 *
 *     (1/|J^{-1}|) d_p ( G_pq d_q p ) = f,
 *
 * discretised conservatively on the Jacobi-transformed grid (Section 3.3,
 * Eqs. PC_8 and PC_term1-3) with face metrics G_pq and cell volumes |J^{-1}|
 * built by the five-step procedure of Section 3.2 (Eqs. jacobi, skewness) on
 * a spherical, oblate or triaxial shell with tanh radial clustering
 * (Section 3.7, Eq. stretching).  Walls in radius and colatitude carry zero
 * flux; longitude is periodic (Section 3.7).
 *
 * Conventions shared by every entry point
 *  - Grids are cell-centred, stored C-contiguous as [nr][nth][nph]
 *    (radius slowest, longitude fastest).  The paper's index triple is
 *    (i, j, k) = (colatitude zeta, radius eta, longitude xi).
 *  - Pointers named *_dev are device pointers on the handle's current device;
 *    *_host are host pointers.  The caller owns every buffer it passes; the
 *    library never frees or retains caller memory beyond the call.
 *  - All work of a handle is issued on the handle's stream (mg_setup's
 *    `cuda_stream`, a cudaStream_t; NULL = the legacy default stream).  Calls
 *    that return results in host memory (reports, norms) synchronise that
 *    stream before returning.
 *  - Every call returns an mg_status.  No C++ exception crosses the ABI.  A
 *    CUDA error is returned as MG_ECUDA and also recorded for mg_last_error().
 *  - Handles are not thread safe: serialise calls on one handle.  Distinct
 *    handles may be used from distinct threads.
 */
#ifndef MG_SHELL_H
#define MG_SHELL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_EINVAL = 1,     /* bad argument (grid, options, pointer, size) */
    MG_ENOMEM = 2,     /* device or host allocation failed */
    MG_ENOCONV = 3,    /* max_iters reached; x holds the last iterate */
    MG_ENAN = 4,       /* NaN or Inf in the right-hand side or the residual */
    MG_EDIVERGED = 5,  /* residual grew by more than 1e3 over its minimum */
    MG_ETIMEOUT = 6,   /* a bounded device wait ran out */
    MG_EAGAIN = 7,     /* serve loop: request not finished yet */
    MG_ECUDA = 8       /* CUDA runtime error (see mg_last_error) */
} mg_status;

enum { MG_MAP_SPHERE = 0, MG_MAP_OBLATE = 1, MG_MAP_TRIAXIAL = 2 };
enum { MG_PREC_FP64 = 0,        /* plain FP64 multigrid */
       MG_PREC_FP32_IR = 1,     /* FP32 V-cycles inside FP64 iterative refinement */
       MG_PREC_FP16C_IR = 2 };  /* FP16 coefficients, FP32 arithmetic, inside FP64 IR */
enum { MG_SMOOTH_GS = 0, MG_SMOOTH_JACOBI = 1, MG_SMOOTH_LINE = 2, MG_SMOOTH_XLINE = 3, MG_SMOOTH_ALT = 4,
       MG_SMOOTH_PLANE = 5 };
enum { MG_METRIC_DISCRETE = 0, MG_METRIC_ANALYTIC = 1 };
enum { MG_COARSEN_SEMI = 0, MG_COARSEN_FULL = 1 };

/* Grid and mapping (Section 2 mapping; Section 3.7 Eq. stretching).
 * Vertex (i, j, k) sits at radius r_in + (r_out - r_in)(s(j) + 1/2), s the
 * tanh clustering of Eq. stretching with factor `stretch` (0 = uniform),
 * colatitude th0 + (th1 - th0) i / nth and longitude 2 pi k / nph, mapped to
 * x1 = (1 - flattening) r cos th, x2 = (1 + e2) r sin th cos ph,
 * x3 = r sin th sin ph.  Requirements: nr, nth >= 1; nph >= 4 and even;
 * 0 < r_in < r_out; 0 < th0 < th1 < pi between zero-flux colatitude walls,
 * or, with cut = 1, the full sphere th0 = 0, th1 = pi (the shell cut of
 * Sections 3.5 and 3.7: a colatitude line continues through either pole into
 * the line at longitude k + nph/2; the zeta faces on the polar axis have zero
 * area and carry no flux).  The shell cut is built for the 7-point operator
 * (the sphere mapping); other stencils return MG_EINVAL with it. */
typedef struct {
    int nr, nth, nph;
    double r_in, r_out;
    double th0, th1;
    int mapping;              /* MG_MAP_* */
    double flattening, e2;
    double stretch;
    int cut;                  /* 0: colatitude walls; 1: full sphere with the shell cut */
} mg_grid_desc;

/* Solver options; mg_default_opts fills the defaults noted here. */
typedef struct {
    int precision;      /* MG_PREC_*, default MG_PREC_FP32_IR */
    int smoother;       /* MG_SMOOTH_*, default GS (multicolour Gauss-Seidel); LINE =
                           radial-line Gauss-Seidel (every radial line solved exactly by
                           the Thomas algorithm of Section 3.5; lines coloured (i+k) mod 2
                           for 7 points, (i mod 2) + 2 (k mod 2) for 19 points; at most
                           256 radial cells; the coarse tail and the one-pass red-black
                           tiles apply to GS only); XLINE = longitude-line Gauss-Seidel
                           (every longitude line solved by the periodic Thomas algorithm
                           of Section 3.5 on the cyclic tridiagonal part of the operator
                           on it; lines coloured (i+j) mod 2 for 7 points, (i mod 2) +
                           2 (j mod 2) for 19 points; a level with fewer than four
                           longitudes takes a point sweep instead); ALT = one LINE sweep
                           then one XLINE sweep per smoothing step; PLANE = the
                           semi-coarsening multigrid of Section 3.6: the hierarchy halves
                           the colatitude only (down to one plane, which the dense
                           bordered solve takes, so it must hold at most 2048 cells),
                           and the smoother is zebra plane relaxation (every (radius,
                           longitude) plane of fixed colatitude row one block, even rows
                           first), each plane solved by plane_cycles V(1,1) cycles of a
                           2-D multigrid (radius halved down to one row, coarse plane
                           operators R B P, zebra longitude lines by the periodic
                           Thomas algorithm of Section 3.5).  7-point operator only,
                           nr a power of two; the coarse-level and coarsening options
                           (max_levels, coarsen, coarse_max) are not used */
    int nu1, nu2;       /* pre/post sweeps, default 2, 2 */
    int max_levels;     /* default 16 */
    int coarsen;        /* MG_COARSEN_*, default SEMI */
    int coarse_max;     /* stop coarsening at <= this many cells, default 512 */
    int max_iters;      /* outer iterations (V-cycles), default 100 */
    int stencil;        /* 0 auto (7 for the sphere, 19 otherwise), 7 or 19 */
    int autotune;       /* 1 (default): at set-up, time a few launch schedules of one outer
                           iteration (blocks per SM of the level kernels, the single-launch
                           coarse tail, one-pass sweeps and their tile shapes) once per
                           hierarchy shape in the process and keep the fastest; every
                           schedule gives the same bits.  2: take the schedule tuned earlier
                           in this process for the same hierarchy shape, else the default;
                           never times (what the serve loop uses).  0: the default schedule. */
    int metric;         /* MG_METRIC_DISCRETE (default): the face metric of Section 3.2 from
                           vertex differences (step 1); MG_METRIC_ANALYTIC: exact derivatives of
                           the mapping at the face centres, steps 2-5 unchanged (an O(h^2)
                           different operator).  The pressure-correction steps and the ADI
                           sweeps need the discrete metric (MG_EINVAL otherwise). */
    int plane_cycles;   /* PLANE smoother: 2-D cycles per plane solve, default 1 */
} mg_opts;

#define MG_HIST 64
typedef struct {
    int iters;                 /* V-cycles performed */
    int levels;                /* multigrid levels */
    int stencil;               /* 7 or 19 */
    int status;                /* mg_status of the solve */
    double rel_res;            /* ||b - A x||_2 / ||b||_2 at exit (FP64) */
    double res_hist[MG_HIST];  /* rel_res before each V-cycle, then at exit */
    double seconds;            /* device time of the solve (CUDA events) */
    double removed_mean;       /* J-weighted mean removed from f */
    double model_bytes;        /* algorithmic HBM bytes of the solve */
    long long launches;        /* kernels the solve launched */
} mg_report;

typedef struct mg_handle mg_handle;

/* Version string of the library build. */
const char* mg_version(void);
/* Text of the last error recorded on the calling thread ("" if none). */
const char* mg_last_error(void);
mg_status mg_default_opts(mg_opts* opts);

/* Device memory a handle for this grid and these options would hold after
 * mg_setup (bytes; an upper estimate), or 0 if the description is invalid.
 * Arrays made on first use are not included: the face C of the
 * pressure-correction steps (30 nr*nth*nph doubles), the ADI line work and
 * wall metric (about 2 nr*nth*nph doubles), radial-line factors requested by
 * mg_smooth on a handle set up with another smoother. */
size_t mg_footprint_bytes(const mg_grid_desc* grid, const mg_opts* opts);

/* Build a handle: face metrics of Section 3.2 on the device (FP64), the
 * multigrid hierarchy by face-metric aggregation, FP32/FP16 coefficient
 * copies and the coarsest-level bordered inverse.  `cuda_stream` is a
 * cudaStream_t (NULL = default stream).  On success *out owns all device
 * memory of the solve; free it with mg_destroy.  Errors: MG_EINVAL (grid or
 * options), MG_ENOMEM, MG_ECUDA. */
mg_status mg_setup(const mg_grid_desc* grid, const mg_opts* opts, void* cuda_stream,
                   mg_handle** out);
void mg_destroy(mg_handle* h);
/* Re-target a handle's work to another stream of the same device. */
mg_status mg_set_stream(mg_handle* h, void* cuda_stream);

/* Solve (1/J) d_p(G_pq d_q x) = f (Eq. PC_6 with the pointwise right side f):
 * b = |J^{-1}| (f - mean_J f), iterate until ||b - A x||_2 <= tol ||b||_2,
 * then remove the J-weighted mean of x.  f_dev: nr*nth*nph doubles (read
 * only).  x_dev: same size; initial guess on entry (zeros = cold start),
 * solution on exit (best iterate on MG_ENOCONV).  `rep` may be NULL.
 * Errors: MG_EINVAL, MG_ENAN, MG_ENOCONV, MG_EDIVERGED, MG_ECUDA. */
mg_status mg_solve(mg_handle* h, const double* f_dev, double* x_dev, double tol, mg_report* rep);

/* The same solve from host buffers: f_host is copied to the device, x_host
 * is both the initial guess and the result.  Copies run on the handle's
 * stream through pinned staging buffers owned by the handle. */
mg_status mg_solve_host(mg_handle* h, const double* f_host, double* x_host, double tol,
                        mg_report* rep);

/* Solve n independent problems together: every level operation of all the
 * shells still iterating is one launch over a joint work list, and one outer
 * iteration of the whole batch is a captured CUDA graph.  hs[s], f_dev[s],
 * x_dev[s], tol[s] as in mg_solve; reps may be NULL.  All handles must live
 * on the same device and use the same precision; work runs on hs[0]'s
 * stream.  Each shell's result is bitwise the one mg_solve gives it. */
mg_status mg_solve_batch(mg_handle* const* hs, int n, const double* const* f_dev,
                         double* const* x_dev, const double* tol, mg_report* reps);

/* ---------------------------------------------------------------------------
 * Component entry points (one multigrid level operation each), for parity
 * tests against an independent implementation and for users who assemble
 * their own cycles.  `level` 0 is the fine grid; `prec` is 0 (double buffers,
 * FP64 coefficients), 1 (float buffers, FP32 coefficients) or 2 (float
 * buffers, FP16 coefficients); the handle must have been set up with a
 * precision that holds the requested copy (FP64 copies always exist).
 * Buffers are C-contiguous [nr_l][nth_l][nph_l] of the level's shape.
 * ------------------------------------------------------------------------- */
typedef struct {
    int nr, nth, nph;        /* cells on this level */
    int cz, ce, cx;          /* halving factors (colatitude, radius, longitude)
                                to the next level; 0 on the coarsest */
    int stencil;             /* 7 or 19 */
    int levels;              /* number of levels of the hierarchy */
} mg_level_info;
mg_status mg_get_level_info(mg_handle* h, int level, mg_level_info* info);

/* Copy the FP64 face metric of a level to caller memory (dst_dev, device).
 * component 0..8 = row d, column q of G at the lower d-normal face of every
 * cell, index 3 d + q with d, q in (zeta, eta, xi) order (Section 3.2 step 5;
 * wall faces hold 0); component 9 = cell |J^{-1}| (step 3, fine level only).
 * On coarse levels G is the aggregate of the fine faces tiling each face. */
mg_status mg_get_metric(mg_handle* h, int level, int component, double* dst_dev);

/* y = A_l x on one level (Eqs. PC_term1-3 summed over the nine terms). */
mg_status mg_apply(mg_handle* h, int level, int prec, const void* x_dev, void* y_dev);

/* `sweeps` smoothing sweeps on A_l x = b in place: multicolour Gauss-Seidel
 * (kind 0; 7-point: red then black by (i+j+k) mod 2; 19-point: colours
 * ((i+j) mod 2) + 2((j+k) mod 2) in order 0..3), weighted Jacobi (kind 1,
 * omega 6/7 for 7-point, 4/5 for 19-point; the diagonal is that of A_l) or
 * radial-line Gauss-Seidel (kind 2: x_L += A_LL^{-1} (b - A_l x)_L line by
 * line, A_LL the tridiagonal part of A_l on the line; line colours as for
 * MG_SMOOTH_LINE, in order), longitude-line Gauss-Seidel (kind 3, as
 * MG_SMOOTH_XLINE; uses the level's scratch array) or both (kind 4, radial
 * then longitude lines per sweep).  Kinds 2 to 4 on a handle set up with
 * another smoother first factor the line blocks of every level (allocates). */
mg_status mg_smooth(mg_handle* h, int level, int prec, void* x_dev, const void* b_dev,
                    int sweeps, int kind);

/* rc = R (b - A_l x): residual on level l summed over the children of every
 * cell of level l+1. */
mg_status mg_restrict_residual(mg_handle* h, int level, int prec, const void* x_dev,
                               const void* b_dev, void* rc_dev);

/* x += P ec: cell-centred trilinear interpolation from level l+1 (weights
 * 3/4, 1/4 per halved direction, mirror at walls, wrap in longitude). */
mg_status mg_prolong_add(mg_handle* h, int level, int prec, const void* ec_dev, void* x_dev);

/* Coarsest level: e = first block of [A 1; 1^T 0]^{-1} [r; 0] in FP64. */
mg_status mg_coarse_solve(mg_handle* h, int prec, const void* r_dev, void* e_dev);

/* One V(nu1, nu2) cycle on A_0 x = b (prec as above; level arrays of the
 * coarse levels are the handle's). */
mg_status mg_vcycle(mg_handle* h, int prec, void* x_dev, const void* b_dev);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of independent solve requests (a library
 * pattern; the paper, which solves one pressure correction per time
 * substep, has no counterpart).  Requests are admitted while the device
 * memory reserved for admitted requests (mg_footprint_bytes + their f and x)
 * stays within max_bytes and fewer than max_slots iterate; worker threads
 * build each request's hierarchy (or reuse an idle one of the same grid and
 * options, kept up to cache_bytes) and upload its right side; every step of
 * the server is one outer iteration of all admitted requests as one batch.
 * Requests that become ready join at the next step and converged ones retire
 * at once, so their work overlaps on the device.  Each result is bitwise the
 * one mg_solve gives for the same grid, options, f and a zero initial guess.
 * ------------------------------------------------------------------------- */
typedef struct mg_server mg_server;
typedef struct {
    size_t max_bytes;     /* device bytes for admitted requests; 0 = 80% of free memory */
    int max_slots;        /* requests iterating at once (default 64) */
    int setup_threads;    /* host threads building hierarchies (default 4) */
    size_t cache_bytes;   /* idle hierarchies kept for reuse; 0 = max_bytes / 4 */
    int device;           /* CUDA device; -1 = the calling thread's current device */
} mg_serve_opts;
typedef struct {
    long long queued;               /* submitted, not yet admitted */
    long long active;               /* admitted, not yet retired */
    long long steps;                /* batched outer iterations run */
    long long retired;              /* requests finished */
    long long cache_hits;           /* hierarchies reused */
    long long cached_hierarchies;   /* idle hierarchies held */
    size_t bytes_reserved;          /* device bytes reserved for admitted requests */
    /* host seconds the stepping thread spent, by phase */
    double t_start;                 /* prologues of newly admitted requests */
    double t_plan;                  /* rebuilding the batched step after arrivals / retirements */
    double t_step;                  /* batched outer iterations (launch, device time, stop test) */
    double t_retire;                /* epilogues and result copies of finished requests */
    long long plan_rebuilds;        /* times the batched step was rebuilt */
} mg_serve_stats_t;
mg_status mg_serve_default_opts(mg_serve_opts* opts);
/* Start a server (threads and a stream on `device`).  Free with mg_serve_destroy. */
mg_status mg_serve_create(const mg_serve_opts* opts, mg_server** out);
/* Queue one solve: grid and options as in mg_setup (opts may be NULL), f_host
 * the pointwise right side (nr*nth*nph doubles, copied before the call
 * returns), tolerance as in mg_solve.  *ticket identifies the request.  The
 * server never times schedules (timings taken while other requests run would
 * measure the load): a hierarchy takes the schedule tuned earlier in the
 * process for its shape (mg_setup with autotune = 1, e.g. of representative
 * shapes before the server starts), else the default (opts->autotune is
 * read as 2); results are the same bits either way. */
mg_status mg_serve_submit(mg_server* sv, const mg_grid_desc* grid, const mg_opts* opts, const double* f_host,
                          double tol, uint64_t* ticket);
/* MG_EAGAIN while the request is queued or iterating; otherwise its final
 * status, with the solution copied to x_host (nr*nth*nph doubles, may be
 * NULL) and the report (seconds = latency from submit to result) to rep.
 * A finished ticket is released by the poll that returns it. */
mg_status mg_serve_poll(mg_server* sv, uint64_t ticket, double* x_host, mg_report* rep);
mg_status mg_serve_stats(mg_server* sv, mg_serve_stats_t* out);
/* Stop the threads, wait for the device, free everything; unfinished
 * requests are dropped. */
void mg_serve_destroy(mg_server* sv);

/* The launch schedule a handle runs (see mg_opts.autotune).  No counterpart in
 * the paper: it changes speed, never results. */
typedef struct {
    int blocks_per_sm;      /* cap of the level kernels' virtual grids, in blocks of 256 per SM */
    int tail_level;         /* first level of the single-launch coarse tail, 0 = none */
    int tail_cluster;       /* CTAs per tail cluster */
    int one_pass_tiles;     /* 1: Gauss-Seidel sweeps as one launch per sweep (all colours,
                               shared-memory plane tiles) on every level a tile fits */
    int source;             /* 0 default, 1 tuned at this set-up, 2 from the process cache,
                               3 forced by MG_TAIL / MG_FUSED_RB / MG_VB_CAP / MG_TILE in the
                               environment (MG_VB_CAP = blocks per SM; MG_TILE = "cells,planes,kmax[,min_cells]";
                               MG_FUSED_RB alone sweeps every level a tile fits in one pass) */
    int candidates;         /* schedules timed (source 1) */
    double ms_per_iteration;/* device time of one outer iteration under the chosen schedule
                               (source 1 and 2; 0 otherwise) */
    int tile_cells;         /* one-pass tiles: target cells per plane (colatitude rows x longitudes) */
    int tile_planes;        /* one-pass tiles: radius planes per chunk (0: chosen per level) */
    int tile_kmax;          /* one-pass tiles: widest tile in longitudes (whole rows up to it) */
    long long tile_min_cells; /* one-pass tiles: levels with fewer cells keep the colour passes */
    int tile0[3];           /* the fine level's tile (colatitude rows, radius planes, longitudes);
                               zeros when the fine level is swept by colour passes */
    int tail_smem_bytes;    /* > 0: the 7-point tail keeps its levels in the cluster's shared
                               memory, this many bytes per CTA (MG_TAIL_GLOBAL=1: global memory) */
} mg_schedule;
mg_status mg_get_schedule(const mg_handle* h, mg_schedule* out);

/* ---------------------------------------------------------------------------
 * The steps either side of the solve in the pressure correction (Section 3.6)
 * for a staggered intermediate velocity.
 *
 * u_face: device array of 9 * nr*nth*nph doubles (owned by the caller): the
 * Cartesian components (x1, x2, x3) of u*** at the centre of every cell's
 * three LOWER faces, block 3 d + a = component a on the face normal to d
 * (d in zeta = colatitude, eta = radius, xi = longitude order), each block
 * [nr][nth][nph] like the face metric.  Wall faces carry no flux: the entries
 * of the lower wall faces (zeta faces at i = 0, eta faces at j = 0) are not
 * read and are left unchanged; upper wall faces are not stored.
 * The face C of Section 3.2 (Eq. skewness) is computed on the first call of
 * either function on a handle (30 extra arrays of nr*nth*nph doubles, freed
 * with the handle).  Work is queued on the handle's stream order (the
 * caller's stream of mg_setup / mg_set_stream); neither call synchronises.
 * ------------------------------------------------------------------------- */
/* Right side of Eq. PC_6: f = D(U) / |J^{-1}| per cell, where U_d = sum_a C_da
 * u_a is the contravariant flux through a d-face and D(U) the cell's flux
 * balance.  mg_solve(h, f, x) then returns x = h dP of Eq. PC_6.  f: device,
 * nr*nth*nph doubles. */
mg_status mg_pc_rhs(mg_handle* h, const double* u_face, double* f);
/* Correction of Eq. PC_7 on the faces: at every interior face
 * u_a -= (1/|J^{-1}|_face) sum_p C_pa g_p, with g the gradient of the
 * operator's face flux (Eqs. PC_term1-3; the face-normal difference only for
 * the 7-point operator) of x = h dP from mg_solve.  The corrected field's
 * flux balance equals the solver's residual b - A x. */
mg_status mg_pc_correct(mg_handle* h, const double* x, double* u_face);

/* ---------------------------------------------------------------------------
 * Batched tridiagonal line solves: the Thomas algorithm of Section 3.5
 * (Eqs. FIBRE_TA1, FIBRE_TA2: forward elimination, back substitution) and its
 * periodic variant (Eqs. FIBRE_TAP1 to FIBRE_TAP8), in FP64, one GPU thread
 * per line, for the implicit sweeps along one grid direction.
 *
 * Row m of a line is a_m psi_{m-1} + b_m psi_m + c_m psi_{m+1} = g_m.  A plain
 * line ignores a_0 and c_{n-1}; a periodic line (the longitude direction)
 * uses them as the corners (a_0 multiplies psi_{n-1}, c_{n-1} multiplies
 * psi_0).  No pivoting: the forward sweep must meet no zero pivot (the
 * diagonally dominant systems of the implicit sweeps do not); a zero pivot
 * gives inf / NaN in x and no error status.
 * ------------------------------------------------------------------------- */
typedef struct {
    int n;                 /* unknowns per line: >= 1, >= 3 for periodic lines */
    int n1, n2;            /* the lines are (l1, l2), 0 <= l1 < n1, 0 <= l2 < n2 */
    long long sm, s1, s2;  /* strides in elements: entry m of line (l1, l2) sits at
                              l1*s1 + l2*s2 + m*sm of a, b, c, g and x.  Lines along
                              axis 0, 1, 2 of a C-contiguous [d0][d1][d2] array:
                              (n,n1,n2,sm,s1,s2) = (d0,d1,d2,d1*d2,d2,1),
                              (d1,d0,d2,d2,d1*d2,1), (d2,d0,d1,1,d1*d2,d2).  Lines
                              adjacent in memory (s2 = 1) give coalesced access. */
} mg_lines;
/* Bytes of the device work array mg_thomas needs: (n - 1) * n1 * n2 doubles
 * for plain lines (at least one row), 2 (n - 1) n1 n2 for periodic ones; 0 for
 * an invalid geometry. */
size_t mg_thomas_work_bytes(const mg_lines* lines, int periodic);
/* Solve every line.  a, b, c, g, x, work: device arrays owned by the caller
 * (work of mg_thomas_work_bytes bytes, contents on return unspecified); x may
 * be the same array as g (solved in place), otherwise no array may overlap
 * another.  Queued on `stream` (a cudaStream_t; NULL = the legacy default
 * stream), not synchronised.  MG_EINVAL for a bad geometry, a null array
 * (unless n1 * n2 = 0) or x / work aliasing a coefficient; MG_ECUDA if the
 * launch fails. */
mg_status mg_thomas(const mg_lines* lines, const double* a, const double* b, const double* c,
                    const double* g, double* x, double* work, int periodic, void* stream);

/* ---------------------------------------------------------------------------
 * The ADI-CN implicit viscous sweeps of Section 3.4 (Eqs. solve_2, solve_3,
 * solve_4) for one cell-centred field (a velocity component or the
 * temperature) on the handle's fine grid, FP64.  With kappa = (h/2)
 * sqrt(Pr/Ra) (h the RKW3 sub-step) and L_p the diagonal viscous term of
 * direction p (Eq. PC_term1 in flux form, the operator's G_pp faces):
 *   (J - kappa L_zeta) u*   = J u^n + src + kappa L_zeta u^n + 2 kappa (L_eta + L_xi) u^n
 *   (J - kappa L_eta)  u**  = J u*  - kappa L_eta u^n
 *   (J - kappa L_xi)   u*** = J u** - kappa L_xi u^n          (periodic longitude)
 * J = |J^{-1}| of the cell; src the caller's explicit terms (beta h times
 * advection, cross diffusion, pressure and buoyancy), volume integrated like
 * J u.  Each sweep is one tridiagonal system per grid line (Thomas; periodic
 * Thomas in longitude), formed on the fly from the face metric.
 * ------------------------------------------------------------------------- */
enum { MG_WALL_FLUX0 = 0, MG_WALL_VALUE = 1 };
typedef struct {
    int radius;              /* MG_WALL_FLUX0 (zero flux) or MG_WALL_VALUE at the walls j = 0, j = nr */
    int colatitude;          /* the same at the walls i = 0, i = nth */
    double v_r_in, v_r_out;  /* MG_WALL_VALUE: the value on the wall face (half a cell from the
                                centre; face flux 2 G_pp (u_w - u_c) outward) */
    double v_th0, v_th1;
} mg_walls;
/* One sub-step of `nfields` fields with the same kappa: u[f] = u*** from
 * un[f].  un[f], src[f] and u[f] are device arrays of nr*nth*nph doubles,
 * [nr][nth][nph], owned by the caller; src may be NULL (no explicit terms), as
 * may any src[f]; no u[f] may alias another array.  walls: NULL = no-slip
 * (value 0 on all four walls), else nfields entries whose kinds agree (the
 * fields share the matrices: one division per row serves up to four fields,
 * as the three velocity components of a sub-step); values may differ.
 * The first call on a handle computes G_pp of the wall faces and allocates
 * 2 nr*nth*nph doubles of line work (freed with the handle).  Queued on the
 * handle's stream order, not synchronised.  MG_EINVAL for null or aliased
 * arrays, nfields < 1, kappa < 0 or not finite, a bad wall kind or value. */
mg_status mg_adi_substep(mg_handle* h, double kappa, int nfields, const mg_walls* walls,
                         const double* const* un, const double* const* src, double* const* u);

/* Bytes the library's device memory pool has handed out and not taken back
 * on `device` (hierarchies, request buffers, work arrays of live handles and
 * servers); freed blocks kept for reuse are not counted.  Test hook: with
 * MG_TEST_FAIL_ALLOC_AFTER=n in the environment, every set-up fails its
 * (n+1)-th device allocation with MG_ENOMEM (releasing what it took). */
size_t mg_device_bytes_in_use(int device);

/* ---------------------------------------------------------------------------
 * Kernel timing.  With mg_profile_enable(h, 1) every kernel a solve launches
 * records its own clock on the GPU's global nanosecond timer: the earliest
 * start of its thread blocks (after they wait for the previous launch) and
 * the latest end.  Each launch's span is added to its slot, so the slots hold
 * device time of the kernels proper; the launches run as in an untimed solve
 * (the clocks add a reset, and per outer iteration an accumulation or a
 * read-back).  With mode 2 every launch is bracketed by CUDA events instead,
 * the launches run eagerly and the outer loop on the host (a slower solve:
 * event records between launches; a cross-check of the clocks).  Slots:
 * 0 = fine-level smoothing launches, 1 = outer FP64 residual, 2 = fine-level
 * residual + restriction, 3 = fine-level prolongation + correction, 4 = outer
 * update, 5 = the single-launch coarse tail of the V-cycle, 6 = everything
 * else (zeroing, reductions, the coarsest solve, copies; the device loop's
 * stop tests and the clock bookkeeping are in no slot), 7 = with clocks, the
 * time inside each program
 * run (prologue, outer iteration, epilogue) between its first start and last
 * end that no launch covers (launch gaps), MG_PROF_LEVEL_BASE + l = the
 * smoothing, restriction and prolongation launches of level l (1 <= l < 16;
 * deeper levels share the last slot).  Stand-alone component calls
 * (mg_smooth, mg_vcycle) time slots 0, 2, 3 and 5 only, with CUDA events
 * around their launches in either mode.
 * ------------------------------------------------------------------------- */
enum { MG_PROF_SMOOTH0 = 0, MG_PROF_RESIDUAL = 1, MG_PROF_RESTRICT0 = 2, MG_PROF_PROLONG0 = 3,
       MG_PROF_UPDATE = 4, MG_PROF_TAIL = 5, MG_PROF_OTHER = 6, MG_PROF_GAPS = 7, MG_PROF_LEVEL_BASE = 8,
       MG_PROF_SLOTS = 24 };
/* Enable (on = 1 clocks, 2 events) or disable (0) timing; either way the
 * accumulators reset. */
mg_status mg_profile_enable(mg_handle* h, int on);
/* Accumulated device milliseconds and launch count of one slot. */
mg_status mg_profile_read(mg_handle* h, int slot, double* ms, long long* launches);

/* ---------------------------------------------------------------------------
 * Right-hand-side projection without allocation.  The paper has no
 * counterpart: this is a library convenience for callers that cannot
 * allocate device memory when they need it (a time-step loop that must not
 * stall on the allocator, or a program whose GPU memory is owned by another
 * pool or a framework's caching allocator).  Computes mean = sum J f / sum J
 * and b = J (f - mean) for caller device arrays J (cell volumes, e.g. from
 * mg_get_metric component 9), f and b of n doubles on the current device, and
 * writes the mean to the caller's device double mean_dev (may be NULL).  Work
 * is queued on cuda_stream (a cudaStream_t; NULL = the legacy default
 * stream); the call does not synchronise.
 * No allocation: the reduction scratch is a 128 KB static device array in
 * the library, present on every GPU that loads it until the process exits.
 * n must not exceed 4,194,304 cells (MG_EINVAL otherwise, with the limit in
 * mg_last_error()); arrays that are not memory of the current device are
 * refused with MG_EINVAL.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it for that device index
 * (not per context; a device reset needs a new process); make that first
 * call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU race.
 * ------------------------------------------------------------------------- */
mg_status mg_project_rhs_noalloc(const double* J_dev, const double* f_dev, double* b_dev, long long n,
                                 void* cuda_stream, double* mean_dev);

#ifdef __cplusplus
}
#endif
#endif /* MG_SHELL_H */

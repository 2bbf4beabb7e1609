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
// Assembled FP64 rows of a level (row_off order): 19 x n doubles for the
// 19-point operator (11 x n without the longitude cross terms: the entries
// 11..18 are the longitude edges), n (the centre coefficient) for the
// 7-point one.
inline int assembled_rows(const LevelView& lv) {
    return lv.stencil == 7 ? 1 : (lv.c64.g[2] ? 19 : 11);
}
cudaError_t launch_assemble_rows(const LevelView& lv, double* a, cudaStream_t s);
cudaError_t launch_cast32(const double* src, float* dst, i64 n, cudaStream_t s);
cudaError_t launch_cast16(const double* src, __half* dst, i64 n, float inv_scale, cudaStream_t s);
cudaError_t launch_dense_operator(const LevelView& lv, double* A, cudaStream_t s);
// Factors of the radial-line blocks of a level for the radial-line smoother:
// 3 x n values of the cycle's type (double for PREC64, float otherwise);
// *bad (zeroed by the caller) counts zero or non-finite pivots.
cudaError_t launch_line_factors(const LevelView& lv, int prec, void* fac, unsigned* bad, cudaStream_t s);
// Longitude-line factors (4 n values of the precision class of prec; layout of
// xline_smooth.cuh); the level needs nph >= 4.
cudaError_t launch_xline_factors(const LevelView& lv, int prec, void* fac, unsigned* bad, cudaStream_t s);
// Leading n x n block of [A 1; 1^T 0]^{-1} (A: n x n row-major) by Gauss-Jordan
// elimination on the device, one cooperative launch (n + 1 <= kMaxGj).
// work: (n+1)^2 doubles, col: kGjScratch doubles (barrier words and pivot
// candidates), piv and perm: n+1 ints each, *bad (zeroed by the caller) set
// on a zero pivot (1) or a grid barrier that gave up waiting (2).
constexpr int kMaxGj = 2049;
constexpr int kGjMaxCtas = 256;
constexpr int kGjScratch = 1 + 3 * kGjMaxCtas;
cudaError_t launch_bordered_inverse(const double* A, int n, double* work, double* col, int* piv, int* perm,
                                   int* bad, double* binv, cudaStream_t s);

// Device scalar slots of a solve (mg_handle::scal).
enum {
    SC_SUMJF = 0,   // sum J f
    SC_BB = 1,      // ||b||^2
    SC_RR = 2,      // ||r||^2 of the latest outer residual
    SC_SUMJX = 3,   // sum J x (gauge)
    SC_SCUR = 8,    // power-of-two scale for the next FP32 residual
    SC_SUSED = 9,   // scale the latest FP32 residual was written with
    SC_COUNT = 16
};
enum { FIN_SUM = 0, FIN_MAX = 1, FIN_SCALE = 2 };

// ---- reductions (outer.cu); partials has room for kRedBlocks doubles
constexpr int kRedBlocks = 1216;   // 8 x 152 SMs; fixed so results are reproducible
int red_blocks(i64 n);
cudaError_t launch_sum(const double* a, const double* w, i64 n, double* partials, cudaStream_t s);
cudaError_t launch_absmax(const double* a, i64 n, double* partials, cudaStream_t s);
// op FIN_SUM / FIN_MAX: out[0] = sum / max of the partials.  FIN_SCALE: out[0]
// = sum, and scal[SC_SCUR] = 2^-round(log2(sqrt(sum / n))) (the scale that
// brings the next FP32 residual to unit RMS).
cudaError_t launch_finalize(const double* partials, int nparts, int op, double* out, cudaStream_t s,
                            double* scal = nullptr, i64 n = 1);

// ---- level operations (stencil.cu); x/b/y are double* for PREC64, float* otherwise
cudaError_t launch_apply(const LevelView& lv, int prec, const void* x, void* y, cudaStream_t s);
// poles: for 19 points on the full sphere, the first and last rows of x as the
// pass starts (launch_poles), else null.
cudaError_t launch_gs_colour(const LevelView& lv, int prec, void* x, const void* b, int colour,
                             cudaStream_t s, const void* poles = nullptr);
// Rows 0 and nth - 1 of x into poles, laid out [side][j][k] (2 nr nph values).
cudaError_t launch_poles(const LevelView& lv, int prec, const void* x, void* poles, cudaStream_t s);
cudaError_t launch_jacobi(const LevelView& lv, int prec, const void* x, void* xo, const void* b,
                          cudaStream_t s);
// One colour of the longitude-line Gauss-Seidel sweep (fac from
// launch_xline_factors; work: n values of scratch).
cudaError_t launch_xline_colour(const LevelView& lv, int prec, void* x, const void* b, const void* fac,
                                void* work, int colour, cudaStream_t s);
// One colour of the radial-line Gauss-Seidel sweep (fac from launch_line_factors).
cudaError_t launch_line_colour(const LevelView& lv, int prec, void* x, const void* b, const void* fac,
                               int colour, cudaStream_t s);
cudaError_t launch_restrict_residual(const LevelView& lv, Dims Dc, int prec, const void* x,
                                     const void* b, void* rc, void* ec_zero, cudaStream_t s);
cudaError_t launch_prolong_add(const LevelView& lv, Dims Dc, int prec, const void* ec, void* x,
                               cudaStream_t s);
cudaError_t launch_coarse_solve(const double* binv, int n, int prec, const void* r, void* e,
                                cudaStream_t s);

// ---- coarse tail (stencil.cu): the V-cycle from a level down to the coarsest
// and back in one launch; one thread-block cluster of csize CTAs per task.
constexpr int kMaxTail = 16;
constexpr int kTailThreads = 512;
constexpr int kTailMaxCluster = 16;   // above 8: a non-portable cluster size
struct TailLevel {
    LevelView v;       // dims, factors to the next level, coefficients
    void* e;           // iterate / correction of the level
    void* r;           // right side of the level
};
struct TailTask {
    TailLevel lev[kMaxTail];
    int nlev;          // levels in the tail (the last one is the coarsest)
    int nu1, nu2;
    const double* binv;
    int ncoarse;
    const int* active; // per-shell flags of a batch (null: always run)
    int shell;
};
// The tail can keep every level in the cluster's shared memory: cell c of
// level l on CTA c >> sh[l] at offset c & (2^sh[l] - 1), arrays of 2^sh[l]
// values per level (e, r, then the lower-face components: 0, 4, 8 for 7
// points, all nine for 19), level l's first array at byte off[l].
constexpr int kTailSmThreads = 1024;
constexpr unsigned kTailSmMaxBytes = 200u * 1024u;
struct TailSmLayout {
    int sh[kMaxTail];
    unsigned off[kMaxTail];
    unsigned rd_off;     // the coarsest level's r in FP64 (ncoarse values), every CTA a copy
    unsigned bytes;
};
__host__ __device__ inline int tail_sm_arrays(const TailTask& tk) { return tk.lev[0].v.stencil == 19 ? 11 : 5; }
__host__ __device__ inline void tail_sm_layout(const TailTask& tk, int csize, int vbytes, TailSmLayout& L) {
    const unsigned arrays = (unsigned)tail_sm_arrays(tk);
    unsigned at = 0;
    for (int l = 0; l < tk.nlev; ++l) {
        const long long n = (long long)tk.lev[l].v.D.nr * tk.lev[l].v.D.nth * tk.lev[l].v.D.nph;
        const long long per = (n + csize - 1) / csize;
        int s = 5;   // at least 32 cells (an even chunk: a colour pass's items split on it)
        while ((1LL << s) < per) ++s;
        L.sh[l] = s;
        L.off[l] = at;
        at += (arrays * (unsigned)vbytes) << s;
    }
    L.rd_off = at;
    at += 8u * (unsigned)tk.ncoarse;
    L.bytes = at;
}
// smem > 0: the shared-memory form with that much dynamic shared memory
// (7-point only); 0: levels in global memory.
cudaError_t launch_tail(const TailTask* tasks, int ntasks, int csize, int stencil, int prec, cudaStream_t s,
                        unsigned long long* stamp = nullptr, size_t smem = 0);
// Clusters of csize tail CTAs that can be co-resident (0: cluster launch unavailable).
int tail_max_clusters(int csize, int stencil, int prec, size_t smem = 0);

// ---- batched level operations (batch.cu)
enum {
    BOP_GS = 0,       // colour pass: x, b
    BOP_JACOBI,       // x -> y with b
    BOP_RESTRICT,     // x, b -> y = rc, z = ec zeroed
    BOP_PROLONG,      // x += P b   (b = coarse e)
    BOP_RESID,        // FP64: x, b -> y = r32 (or null), z = partials, scal
    BOP_UPDATE,       // x (double) += b (float) / scal[SC_SUSED]; n cells
    BOP_ZERO,         // n 32-bit words of x
    BOP_COPY,         // n 32-bit words b -> x
    BOP_SUM,          // partials z of sum b * y (y may be null); n cells
    BOP_RHS,          // x = y (J) * (b (f) - scal[SC_SUMJF] / aux), partials z of ||x||^2
    BOP_SHIFT,        // x -= scal[SC_SUMJX] / aux
    BOP_FINALIZE,     // scal[slot] = sum of n partials z; y (if set) gets a copy
    BOP_COARSE,       // x = binv b, n rows
    BOP_SWEEP,        // one whole multicolour sweep, x -> y (sweep.cu; launched by launch_sweep)
    BOP_LINE,         // radial-line Gauss-Seidel colour pass: x, b, z = line factors
    BOP_XLINE,        // longitude-line Gauss-Seidel colour pass: x, b, z = factors, y = scratch
    // plane relaxation of the semi-coarsening multigrid (plane_smooth.cuh);
    // colour = plane parity p (+ 2 q for the row parity q of BOP_PRELAX)
    BOP_PRES,         // y = b - A x (7-point, 3-D level) on the planes, z (2-D e) zeroed
    BOP_PRELAX,       // zebra longitude lines of a 2-D level: x = e, b = r, z = factors, y = scratch
    BOP_PRESTRICT,    // y = R (b - B x) on the next 2-D level (dims Dc), z = its e zeroed
    BOP_PPROLONG,     // x += P b (b = the next 2-D level's e, dims Dc)
    BOP_PUPDATE,      // x += b on the planes (3-D level)
    BOP_POLES         // z [side][j][k] = rows 0 and nth - 1 of x (19 points on the full sphere, before a colour pass)
};
struct BTask {
    LevelView v;       // level of the task (dims, factors, coefficients, stencil)
    Dims Dc;           // next-coarser level (restriction / prolongation)
    void* x;
    const void* b;
    void* y;
    void* z;
    double* scal;      // the shell's device scalars
    const double* binv;
    const double* a64; // assembled FP64 rows of the level (outer residual)
    i64 n;             // element / row / partial count of vector operations
    i64 ncells;        // fine cells (scale of the next FP32 residual)
    double aux;        // sum J
    int slot;          // FINALIZE destination
    int fin_scale;     // FINALIZE also sets scal[SC_SCUR]
    int block0;        // first virtual block of the task in its launch
    int nblocks;       // virtual blocks (work mapping of a stand-alone launch)
    int shell;         // index of the active flag
    int tile[3];       // one-pass sweep: colatitude rows, radius planes, longitudes of a tile
    const void* tmap;  // one-pass sweep: its tensor maps (device, 64-byte aligned, 128 bytes each)
    void* e0;          // outer residual of an FP32 / FP16 cycle: the fine correction, zeroed for the next cycle
};
static_assert(sizeof(BTask) % 4 == 0, "BTask is staged in shared memory word by word");
// ---- one-pass multicolour sweeps (sweep.cu).  A tile is tile[0] colatitude
// rows x tile[2] longitudes (tile[2] == nph: whole rows) x a chunk of tile[1]
// radius planes.  A task's arrays are staged through sweep_map_count tensor
// maps (128 bytes each, 64-byte aligned, at tmap) made by encode_sweep_maps
// from the task's x, b, level view and tile: for the 7-point FP32 / FP16
// sweep x, b and three coefficient arrays, otherwise x alone.
// Most compute threads of a 7-point FP32 / FP16 sweep CTA (one per quad of TI
// + 2 rows; with the copy warp, 19 warps: five per SM sub-partition leave 96
// registers a thread).
constexpr int kRB7MaxThreads = 576;
bool sweep_tile_ok(const Dims& D, int stencil, int prec, const int tile[3]);
size_t sweep_smem_bytes(int stencil, int prec, const Dims& D, const int tile[3]);
int sweep_threads(int stencil, int prec, const Dims& D, const int tile[3]);
int sweep_units(const Dims& D, const int tile[3]);
int sweep_map_count(int stencil, int prec);
cudaError_t encode_sweep_maps(void* maps, const BTask& t, int stencil, int prec);
// All tasks of one launch share stencil, precision and axi; smem and
// threads = the largest sweep_smem_bytes and sweep_threads of its tasks.
// axi: 19 points without the longitude cross terms (the handle's stored
// components); every task of the launch shares it.
cudaError_t launch_sweep(const BTask* tasks, int ntasks, int total, const int* active, int stencil, bool axi,
                         int prec, size_t smem, int threads, cudaStream_t s, unsigned long long* stamp = nullptr);
// The fault word of the sweeps (a plane copy that did not land in time);
// clear resets it.
cudaError_t sweep_fault_read(unsigned* out, bool clear);

// ---- plane hierarchies of the semi-coarsening multigrid (smg.cu).  A 2-D
// level uses the 3-D layout with nr >> m rows; its plane operator is nine
// arrays in the order of plane_smooth.cuh's offsets.
cudaError_t launch_plane_op0(const LevelView& lv, double* const out[9], cudaStream_t s);
cudaError_t launch_plane_coarsen(const double* const fine[9], const Dims& D, const Dims& Dc, double* const out[9],
                                 cudaStream_t s);
// Periodic longitude-line factors (4 n values of the cycle's type of prec);
// *bad (zeroed by the caller) counts zero or non-finite pivots.
cudaError_t launch_plane_factors(const double* const c[9], const Dims& D, int prec, void* fac, unsigned* bad,
                                 cudaStream_t s);

// Checks the integer-pipe FP64 <-> FP32 conversions (narrow_rn, scaled_widen)
// against the hardware ones; *bad (zeroed by the caller) counts mismatches.
cudaError_t launch_convert_check(unsigned* bad, cudaStream_t s);
// All tasks of one launch share `stencil` (7 or 19) for the stencil ops.
// stamp (profiling, may be null): the launch clock of stamp_start / stamp_end.
cudaError_t launch_batch(const BTask* tasks, int ntasks, int total_blocks, const int* active, int op, int colour,
                         int stencil, int prec, cudaStream_t s, unsigned long long* stamp = nullptr);
// n launch clocks to (never started, never ended).
cudaError_t launch_stamp_reset(unsigned long long* stamps, int n, cudaStream_t s);
// Adds n launch clocks into acc (per launch: nanoseconds, count; then the
// span from the first start to the last end, and the number of spans) and
// resets the clocks.  One CTA.
cudaError_t launch_stamp_accum(unsigned long long* stamps, int n, unsigned long long* acc, cudaStream_t s);

// One shell's stop test of the outer iteration, kept on the device while the
// iteration loops there (the test a solve makes between V-cycles, same
// arithmetic: relative residual sqrt(rr) / ||b||, history, tolerance, growth
// above 1e3 x the best so far, iteration limit).
constexpr int kLoopHist = 64;
enum { LOOP_RUN = 0, LOOP_NAN = 1, LOOP_DIVERGED = 2, LOOP_NOCONV = 3 };
struct LoopShell {
    double bnorm, best, tol, rr, rel;
    int it, max_iters, done, why;   // why: LOOP_* (set with done)
    double hist[kLoopHist];
};
// After an outer iteration: the active shells' iteration count and residual
// (fin[4 i + 2]), their stop tests, the new active flags; passes[0] counts
// the calls.  Sets the while node's condition to "some shell still active
// and fewer than passes[1] calls".  One CTA.
cudaError_t launch_loop_check(LoopShell* S, int n, const double* fin, int* active, int* passes,
                              cudaGraphConditionalHandle cond, cudaStream_t s);

}  // namespace mgs

// engine.h - the solver handle and the host-side multigrid driver (internal).
#pragma once

#include <cmath>
#include <string>
#include <vector>

#include "mg.h"
#include "mg_kernels.h"

namespace mgs {

struct Plan;

// One 2-D level of the plane hierarchy of a 3-D level (all its planes at
// once): nr >> m rows in the 3-D layout.
struct PlaneLevel {
    Dims D{};
    double* c64[9] = {};   // plane operator (set-up, plain FP64 cycles)
    float* c32[9] = {};    // FP32 copy (FP32 and FP16-coefficient cycles)
    void* fac = nullptr;   // longitude-line factors, 4 n values of the cycle's type
    void* e = nullptr;     // correction, right side, line scratch (cycle's type)
    void* r = nullptr;
    void* w = nullptr;
};

struct Level {
    Dims D{};
    int cz = 0, ce = 0, cx = 0;       // halving factors to the next level
    double* g64[9] = {};
    float* g32[9] = {};
    __half* g16[9] = {};
    float s16[9] = {};
    double* a64 = nullptr;            // assembled FP64 rows (fine level only; outer residual)
    // work arrays in the cycle's value type (double for PREC64, float otherwise)
    void* e = nullptr;   // correction / iterate
    void* r = nullptr;   // right side on this level
    void* t = nullptr;   // scratch (Jacobi)
    void* poles = nullptr;   // 19 points on the full sphere: rows 0 and nth - 1 before a colour pass (2 nr nph values)
    void* lf[2] = {};    // radial-line factors, double / float (3 n values), made on first use
    void* xf[2] = {};    // longitude-line factors, double / float (4 n values), made on first use
    std::vector<PlaneLevel> planes;   // plane hierarchy (semi-coarsening multigrid), made at set-up
    LevelView view(int stencil) const;
};

void set_error(const std::string& m);

// The library's device memory pool (one per device, stream-ordered, freed
// blocks kept for reuse): hierarchies and request buffers come from it, so
// building and dropping hierarchies does not synchronise the device.
cudaMemPool_t lib_pool(int device);

}  // namespace mgs

struct mg_handle {
    mg_grid_desc grid{};
    mg_opts opts{};
    int stencil = 7;
    bool axi = false;                 // 19 points on an axisymmetric mapping: longitude cross terms dropped
    int prec = 1;                     // PREC64 / PREC32 / PREC16
    cudaStream_t stream = nullptr;        // private work stream of the handle
    cudaStream_t user_stream = nullptr;   // caller's stream; joined by events
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int device = 0;
    std::vector<mgs::Level> L;
    std::vector<void*> dev_allocs;
    double* J64 = nullptr;            // cell |J^{-1}| (fine)
    double* x64 = nullptr;            // the iterate (fine); copied from / to the caller's x
    double* b64 = nullptr;            // volume-integrated right side (fine)
    double* part = nullptr;           // reduction partials (kRedBlocks)
    double* scal = nullptr;           // device scalars
    double hscal[mgs::SC_COUNT] = {}; // host copy of scal (set-up reductions)
    double* binv = nullptr;           // coarsest bordered inverse block (n x n)
    int ncoarse = 0;
    double sumJ = 0.0;
    size_t bytes = 0;
    long long fail_alloc_after = -1;  // test hook (MG_TEST_FAIL_ALLOC_AFTER): fail set-up allocations from this one on
    long long allocs_done = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    long long launches = 0;           // kernels launched by the current solve
    // kernel timing (mg_profile_enable): events around stand-alone component
    // calls; a solve's launches record their own clocks (solver.cu)
    struct Pending {
        int slot;
        cudaEvent_t a, b;
        int n;
    };
    mgs::MetricTables mtab{};         // vertex tables of the fine grid (device)
    double* pcC[27] = {};             // face C of the pressure-correction steps (on first use)
    double* pcInv[3] = {};            // 1 / |J^{-1}| of the faces
    double* wallG[4] = {};            // G_dd on the wall planes (implicit sweeps, on first use)
    double* adi_w = nullptr;          // line-solve work of the implicit sweeps (2 N doubles)
    bool prof_on = false;
    bool prof_events = false;         // mode 2: CUDA events around eager launches
    double prof_ms[MG_PROF_SLOTS] = {};
    long long prof_n[MG_PROF_SLOTS] = {};
    cudaEvent_t prof_open[MG_PROF_SLOTS] = {};
    std::vector<Pending> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    // outer iterations run as captured graphs (solver.cu)
    bool use_graph = true;
    int plane_levels = 0;             // PLANE smoother: leading levels relaxed by planes (the rest: GS)
    bool one_pass = false;            // one-pass multicolour sweeps where a tile fits (schedule choice)
    int sweep_cells = 2048;           // one-pass tiles: target cells per plane (rows x longitudes)
    int sweep_tj = 0;                 // one-pass tiles: radius planes per chunk (0: per level)
    int sweep_kmax = 256;             // one-pass tiles: widest tile in longitudes (whole rows up to it)
    long long sweep_min_cells = 1 << 20;   // one-pass tiles: only on levels of at least this many cells
    bool sweep_tile_env = false;      // MG_TILE given: its plane area also fixes the 7-point sweep's rows
    int vb_cap = 16;                  // blocks per SM of the level kernels' virtual grids
    int sched_source = 0;             // mg_schedule.source
    int sched_candidates = 0;
    double sched_ms = 0.0;
    mgs::BTask* one_task = nullptr;   // task table of stand-alone one-pass sweeps
    void* one_map = nullptr;          // tensor maps of a stand-alone one-pass sweep (up to 5 x 128 bytes)
    mgs::BTask* plane_tasks = nullptr;    // task table of stand-alone plane relaxations
    size_t plane_tasks_cap = 0;
    int tail_level = 0;               // first level of the single-launch coarse tail (0: none)
    int tail_cluster = 8;             // CTAs per tail cluster
    size_t tail_smem = 0;             // >0: the tail's levels in shared memory (bytes per CTA)
    mgs::TailTask* tail_dev = nullptr;
    mgs::TailTask tail_host{};
    mgs::Plan* solo = nullptr;             // the batch-of-one plan of mg_solve
    mgs::Plan* batch = nullptr;            // last mg_solve_batch plan led by this handle
    std::vector<unsigned long long> batch_key;   // serials of the batch plan's handles
    unsigned long long serial = 0;                // unique per handle in the process
    // mg_solve_host staging
    double* hf = nullptr;
    double* hx = nullptr;
    double* df = nullptr;
    double* dx = nullptr;
};

namespace mgs {

mg_status vcycle(mg_handle* h, int prec, void* x0, const void* b0);
void prof_begin(mg_handle* h, int slot);
void prof_end(mg_handle* h, int slot, int nlaunch);
void prof_collect(mg_handle* h);   // after a stream synchronisation
// batch plans (solver.cu)
struct SolveState {             // one shell's outer-iteration bookkeeping
    double bnorm = 1.0, best = INFINITY, tol = 0.0, rr = 0.0;
    int it = 0;
    mg_status st = MG_OK;
    bool done = false;
    mg_report R{};
};
// A plan launches on its lead handle's private stream, or on ``stream`` for
// its whole life when one is given (callers whose handles come and go).
// ``iteration`` = false skips the outer-iteration program (plans used only
// for prologues / epilogues).
mg_status plan_create(mg_handle* const* hs, int n, Plan** out, cudaStream_t stream = nullptr, bool iteration = true);
mg_status plan_reset(Plan* pl, mg_handle* const* hs, int n, bool iteration = true);
void plan_destroy(Plan* pl);
mg_status plan_solve(Plan* pl, const double* const* f, double* const* x, const double* tol, mg_report* reps);

// Device memory owned by the handle (freed with it); null when out of memory.
void* handle_alloc(mg_handle* h, size_t bytes);

// Free a handle whose last device work was queued on `last` (or on its own
// stream when null) without waiting for it: the frees are stream-ordered.
void destroy_handle_after(mg_handle* h, cudaStream_t last);
mg_status plan_start(Plan* pl, const double* const* f, double* const* x, const double* tol, SolveState* S);
int plan_check(Plan* pl, SolveState* S);
mg_status plan_iterate(Plan* pl, SolveState* S, bool use_graph);
// Device time of one outer iteration of every shell of the plan (graph
// launched, all shells active): `warm` untimed iterations, then the mean of
// `reps`.  The iterates are not meaningful afterwards.
mg_status plan_time(Plan* pl, int warm, int reps, double* ms);
mg_status plan_finish(Plan* pl, double* const* x);
mg_status smooth(mg_handle* h, int level, int prec, void* x, const void* b, int sweeps, int kind);
double model_bytes_per_iteration(const mg_handle* h);
// The one-pass sweep tile of a level under the handle's schedule (colatitude
// rows, radius planes per chunk, longitudes); false when the level is
// smoothed by colour passes.
bool sweep_tile_for(const mg_handle* h, int level, int tile[3]);
// smoothers that sweep radial lines / longitude lines (the alternating one both)
inline bool radial_lines(int smoother) { return smoother == MG_SMOOTH_LINE || smoother == MG_SMOOTH_ALT; }
// The smoother of a level: the handle's, except that a PLANE handle relaxes
// by planes only its leading levels of two or more planes above the
// coarsest (the colatitude-only part of its hierarchy); the levels below a
// coarsest plane too large for the dense solve take point Gauss-Seidel.
inline int level_smoother(const mg_handle* h, int level) {
    if (h->opts.smoother != MG_SMOOTH_PLANE) return h->opts.smoother;
    return level < h->plane_levels ? MG_SMOOTH_PLANE : MG_SMOOTH_GS;
}
// One sweep of zebra plane relaxation of level `level` (x, b in the cycle's
// type): the launches in order, each one task over the planes of one parity.
struct PlaneStep {
    int op, colour;
    BTask t;
    int nblocks;
};
void plane_sweep_steps(const mg_handle* h, int level, void* x, const void* b, std::vector<PlaneStep>& out);
inline bool longitude_lines(int smoother) { return smoother == MG_SMOOTH_XLINE || smoother == MG_SMOOTH_ALT; }
}  // namespace mgs

// solver.cu - the solve driver: FP64 iterative refinement (or plain FP64
// multigrid) over a batch of shells, one launch per level operation for all
// shells, the outer iteration captured as one CUDA graph.  A single solve is
// the batch of one.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "xline_smooth.cuh"

static_assert(mgs::kLoopHist == MG_HIST, "device stop-test history length");

namespace mgs {

namespace {

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                 \
            return MG_ECUDA;                                                               \
        }                                                                                  \
    } while (0)
#define CKS(call)                   \
    do {                            \
        mg_status s_ = (call);      \
        if (s_ != MG_OK) return s_; \
    } while (0)

// Virtual grid of a task: one thread per work item up to the handle's cap of
// blocks per SM (a schedule choice), grid-stride beyond.
int vblocks(const mg_handle* h, i64 work) {
    i64 b = (work + 255) / 256;
    const i64 cap = 152LL * (h ? h->vb_cap : 16);
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// Work items (threads) of the batched level operations; 7-point colour passes,
// restrictions and prolongations work on groups of four longitude cells when
// nph is a multiple of 4, vector operations on groups of four elements.
i64 gs_items(const Dims& D, int stencil) {
    if (stencil == 19)   // rows of the colour only; groups of four longitudes or cells of the colour
        return (i64)D.nr * ((D.nth + 1) / 2) * (gs19_groups(D) ? D.nph / 4 : D.nph / 2);
    return (i64)D.nr * D.nth * (vec4(D) ? D.nph / 4 : D.nph / 2);
}
i64 restrict_items(const Dims& D, const Dims& Dc) { return vec4(D) ? (i64)Dc.nr * Dc.nth * (D.nph / 4) : Dc.n(); }
i64 prolong_items(const Dims& D) { return vec4(D) ? D.n() / 4 : D.n(); }
i64 vector_items(i64 n) { return (n + 3) / 4; }
// radial-line colour passes: W threads per line (one per chunk of rows)
i64 line_items(const Dims& D, int stencil, int prec) {
    const int kc = prec == PREC64 ? LineRows<double>::kC : LineRows<float>::kC;
    return line_count(D, stencil, 0) * line_chunks(D.nr, kc);
}

// one launch of a level operation over some tasks
struct Launch {
    int op = 0, colour = 0;
    int stencil = 0;               // stencil shared by the tasks of stencil operations
    int t0 = 0, nt = 0, total = 0;
    int prof = -1, prof_n = 0;     // profiling slot around this launch
    int level = -1;                // level of a level operation (timing attribution)
    int tail_stencil = 0;          // >0: a coarse-tail launch of this stencil
    size_t smem = 0;               // one-pass sweep launches: dynamic shared memory
    int threads = 0;               // one-pass sweep launches: threads per CTA
    bool axi = false;              // one-pass sweep launches: 19 points without longitude cross terms
};

// Tensor maps of a one-pass sweep task (made from the task when the plan's
// tables are uploaded).
struct MapReq {
    int task;
    int stencil, prec;
};

struct Program {
    std::vector<BTask> tasks;
    std::vector<Launch> launches;
    std::vector<TailTask> tails;   // tail tasks (7-point first, then 19-point)
    std::vector<MapReq> maps;      // tensor maps of the one-pass sweep tasks

    Launch& begin(int op, int colour = 0, int stencil = 0) {
        Launch L;
        L.op = op;
        L.colour = colour;
        L.stencil = stencil;
        L.t0 = (int)tasks.size();
        launches.push_back(L);
        return launches.back();
    }
    void add(BTask t, int nblocks) {
        Launch& L = launches.back();
        t.block0 = L.total;
        t.nblocks = nblocks;
        L.total += nblocks;
        L.nt += 1;
        tasks.push_back(t);
    }
    void drop_empty() {
        launches.erase(std::remove_if(launches.begin(), launches.end(),
                                      [](const Launch& L) { return L.nt == 0 && L.tail_stencil == 0; }),
                       launches.end());
    }
};

size_t vbytes(int prec) { return prec == PREC64 ? 8 : 4; }

}  // namespace

struct Plan {
    std::vector<mg_handle*> hs;
    int prec = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t fixed = nullptr; // when set, the plan launches here instead of on its lead handle's stream
    Program iter;                 // one outer iteration (graph)
    // device buffers, grown on demand and reused when the plan is re-targeted
    BTask* d_iter = nullptr;
    size_t iter_cap = 0;
    TailTask* d_tails = nullptr;
    size_t tails_cap = 0;
    unsigned char* d_maps = nullptr;   // tensor maps of the iteration's sweep tasks (128 bytes each)
    size_t maps_cap = 0;
    int* d_active = nullptr;      // per-shell flags
    int* h_active = nullptr;      // pinned
    double* d_fin = nullptr;      // per shell: [sum J f, ||b||^2, ||r||^2, sum J x]
    double* h_fin = nullptr;      // pinned
    size_t dact_cap = 0, hact_cap = 0, dfin_cap = 0, hfin_cap = 0;
    BTask* d_call = nullptr;      // prologue / epilogue tasks of the current call
    size_t call_cap = 0;
    cudaGraphExec_t gexec = nullptr;
    bool graph_prof = false;
    long long graph_launches = 0;
    // launch clocks while profiling (two words a launch: first start, last
    // end): the iteration's own (captured in its graph) and a prologue's or
    // epilogue's; the host copies are pinned
    unsigned long long *d_stamp_it = nullptr, *h_stamp_it = nullptr;
    unsigned long long *d_stamp_call = nullptr, *h_stamp_call = nullptr;
    size_t stamp_it_cap = 0, stamp_call_cap = 0;
    // the device-side outer loop: a graph whose while node repeats the
    // iteration and the stop test of every shell until none is active
    cudaGraphExec_t lexec = nullptr;
    bool loop_prof = false;       // built with clocks
    bool loop_failed = false;     // the runtime refused the graph: host loop
    long long loop_launches = 0;  // kernels per pass
    LoopShell* d_loop = nullptr;  // per-shell stop tests
    LoopShell* h_loop = nullptr;  // pinned
    int* d_ctl = nullptr;         // [passes made, pass limit]
    int* h_ctl = nullptr;         // pinned
    size_t dloop_cap = 0, hloop_cap = 0, dctl_cap = 0, hctl_cap = 0;
    unsigned long long *d_acc = nullptr, *h_acc = nullptr;   // clocks summed over the passes
    size_t acc_cap = 0;
};

namespace {

mg_handle* lead(Plan* p) { return p->hs[0]; }
// Kernel timing by launch clocks (mg_profile_enable 1); mode 2 brackets every
// launch with CUDA events instead, run eagerly.
bool clocks(const mg_handle* h) { return h->prof_on && !h->prof_events; }

BTask task_of(const mg_handle* h, int level) {
    BTask t{};
    t.v = h->L[level].view(h->stencil);
    if (level + 1 < (int)h->L.size()) t.Dc = h->L[level + 1].D;
    t.scal = h->scal;
    return t;
}

// Level-ell iterate / right side of shell s inside the cycle.
void level_bufs(const mg_handle* h, int prec, int level, void** x, const void** b) {
    if (level == 0) {
        *x = prec == PREC64 ? (void*)h->x64 : h->L[0].e;
        *b = prec == PREC64 ? (const void*)h->b64 : (const void*)h->L[0].r;
    } else {
        *x = h->L[level].e;
        *b = h->L[level].r;
    }
}

int top_of(const mg_handle* h) { return h->tail_level > 0 ? h->tail_level : (int)h->L.size() - 1; }

// Levels smoothed by one-pass sweeps (the schedule's choice, where the tile
// fits the level).
bool fused_level(const mg_handle* h, int level) {
    int tile[3];
    return sweep_tile_for(h, level, tile);
}

void add_smooth_launches(Program& P, Plan* pl, int level, int sweeps) {
    const int prec = pl->prec;
    int maxc = 0, maxl = 0, maxx = 0;
    bool any_jacobi = false, any_fused = false;
    for (mg_handle* h : pl->hs) {
        if (level >= top_of(h)) continue;
        const int nc = h->stencil == 7 ? 2 : 4;
        if (level_smoother(h, level) == MG_SMOOTH_JACOBI) any_jacobi = true;
        else if (radial_lines(level_smoother(h, level)) || longitude_lines(level_smoother(h, level))) {
            if (radial_lines(level_smoother(h, level))) maxl = std::max(maxl, nc);
            if (longitude_lines(level_smoother(h, level))) maxx = std::max(maxx, nc);
        } else if (fused_level(h, level)) any_fused = true;
        else maxc = std::max(maxc, nc);
    }
    for (int sw = 0; sw < sweeps; ++sw) {
        if (any_fused)   // ping-pong between the level iterate and its scratch
            for (int kind = 0; kind < 3; ++kind) {   // 7 points; 19 axisymmetric; 19 full
                const int st = kind == 0 ? 7 : 19;
                const bool axi = kind == 1;
                Launch& L = P.begin(BOP_SWEEP, 0, st);
                L.axi = axi;
                if (level == 0) {
                    L.prof = MG_PROF_SMOOTH0;
                    L.prof_n = 1;
                }
                for (size_t s = 0; s < pl->hs.size(); ++s) {
                    mg_handle* h = pl->hs[s];
                    int tile[3];
                    if (level >= top_of(h) || h->stencil != st || (st == 19 && h->axi != axi) ||
                        !sweep_tile_for(h, level, tile))
                        continue;
                    const Dims& D = h->L[level].D;
                    BTask t = task_of(h, level);
                    void* xb;
                    const void* bb;
                    level_bufs(h, prec, level, &xb, &bb);
                    t.x = (sw & 1) ? h->L[level].t : xb;
                    t.y = (sw & 1) ? xb : h->L[level].t;
                    t.b = bb;
                    t.shell = (int)s;
                    for (int a = 0; a < 3; ++a) t.tile[a] = tile[a];
                    P.maps.push_back(MapReq{(int)P.tasks.size(), st, prec});
                    L.smem = std::max(L.smem, sweep_smem_bytes(st, prec, D, tile));
                    L.threads = std::max(L.threads, sweep_threads(st, prec, D, tile));
                    P.add(t, sweep_units(D, tile));
                }
            }
        for (int c = 0; c < maxc; ++c)
            for (int st : {7, 19}) {
            auto colour_pass = [&](const mg_handle* h) {
                return level < top_of(h) && level_smoother(h, level) == MG_SMOOTH_GS && h->stencil == st &&
                       !fused_level(h, level) && c < (h->stencil == 7 ? 2 : 4);
            };
            if (st == 19) {   // full-sphere levels: their pole rows as the pass starts
                P.begin(BOP_POLES);
                for (size_t s = 0; s < pl->hs.size(); ++s) {
                    mg_handle* h = pl->hs[s];
                    if (!colour_pass(h) || !h->L[level].D.cut) continue;
                    BTask t = task_of(h, level);
                    level_bufs(h, prec, level, &t.x, &t.b);
                    t.z = h->L[level].poles;
                    t.shell = (int)s;
                    P.add(t, vblocks(h, 2LL * h->L[level].D.nr * h->L[level].D.nph));
                }
            }
            Launch& L = P.begin(BOP_GS, c, st);
            if (level == 0) {
                L.prof = MG_PROF_SMOOTH0;
                L.prof_n = 1;
            }
            for (size_t s = 0; s < pl->hs.size(); ++s) {
                mg_handle* h = pl->hs[s];
                if (!colour_pass(h)) continue;
                BTask t = task_of(h, level);
                level_bufs(h, prec, level, &t.x, &t.b);
                if (st == 19 && h->L[level].D.cut) t.z = h->L[level].poles;
                t.shell = (int)s;
                P.add(t, vblocks(h, gs_items(h->L[level].D, h->stencil)));
            }
        }
        for (int c = 0; c < maxl; ++c)
            for (int st : {7, 19}) {
            Launch& L = P.begin(BOP_LINE, c, st);
            if (level == 0) {
                L.prof = MG_PROF_SMOOTH0;
                L.prof_n = 1;
            }
            for (size_t s = 0; s < pl->hs.size(); ++s) {
                mg_handle* h = pl->hs[s];
                if (level >= top_of(h) || !radial_lines(level_smoother(h, level)) || h->stencil != st) continue;
                if (c >= (h->stencil == 7 ? 2 : 4)) continue;
                BTask t = task_of(h, level);
                level_bufs(h, prec, level, &t.x, &t.b);
                t.z = h->L[level].lf[prec == PREC64 ? 0 : 1];
                t.shell = (int)s;
                P.add(t, vblocks(h, line_items(h->L[level].D, h->stencil, prec)));
            }
        }
        // longitude lines after the radial ones (the alternating smoother);
        // levels narrower than four longitudes take a point colour instead
        for (int c = 0; c < maxx; ++c)
            for (int st : {7, 19})
                for (int narrow = 0; narrow < 2; ++narrow) {
                    Launch& L = P.begin(narrow ? BOP_GS : BOP_XLINE, c, st);
                    if (level == 0) {
                        L.prof = MG_PROF_SMOOTH0;
                        L.prof_n = 1;
                    }
                    for (size_t s = 0; s < pl->hs.size(); ++s) {
                        mg_handle* h = pl->hs[s];
                        if (level >= top_of(h) || !longitude_lines(level_smoother(h, level)) || h->stencil != st) continue;
                        if (c >= (h->stencil == 7 ? 2 : 4) || (h->L[level].D.nph < 4) != (narrow == 1)) continue;
                        BTask t = task_of(h, level);
                        level_bufs(h, prec, level, &t.x, &t.b);
                        t.shell = (int)s;
                        if (narrow) {
                            P.add(t, vblocks(h, gs_items(h->L[level].D, h->stencil)));
                        } else {
                            // MG_XLINE_CHUNKS=1: W threads per line where the lines fit
                            const Dims& D = h->L[level].D;
                            const int kc = prec == PREC64 ? LineRows<double>::kC : LineRows<float>::kC;
                            const int W = std::getenv("MG_XLINE_CHUNKS") ? xline_chunks(D.nph, kc) : 0;
                            t.z = h->L[level].xf[prec == PREC64 ? 0 : 1];
                            t.y = h->L[level].t;
                            t.n = W > 0 ? 1 : 0;
                            P.add(t, vblocks(h, xline_items(D, h->stencil) * (W > 0 ? W : 1)));
                        }
                    }
                }
        if (any_jacobi) {
            for (int st : {7, 19}) {
            Launch& L = P.begin(BOP_JACOBI, 0, st);
            if (level == 0) {
                L.prof = MG_PROF_SMOOTH0;
                L.prof_n = 1;
            }
            for (size_t s = 0; s < pl->hs.size(); ++s) {
                mg_handle* h = pl->hs[s];
                if (level >= top_of(h) || level_smoother(h, level) != MG_SMOOTH_JACOBI || h->stencil != st) continue;
                BTask t = task_of(h, level);
                level_bufs(h, prec, level, &t.x, &t.b);
                t.y = h->L[level].t;
                t.shell = (int)s;
                P.add(t, vblocks(h, h->L[level].D.n()));
            }
            }
            P.begin(BOP_COPY);
            for (size_t s = 0; s < pl->hs.size(); ++s) {
                mg_handle* h = pl->hs[s];
                if (level >= top_of(h) || level_smoother(h, level) != MG_SMOOTH_JACOBI) continue;
                BTask t{};
                void* x;
                const void* b;
                level_bufs(h, prec, level, &x, &b);
                t.x = x;
                t.b = h->L[level].t;
                t.n = h->L[level].D.n() * (i64)(vbytes(prec) / 4);
                t.shell = (int)s;
                P.add(t, vblocks(h, vector_items(t.n)));
            }
        }
        // zebra plane relaxation (semi-coarsening multigrid): each handle's
        // launches in order (plane hierarchies differ from handle to handle)
        for (size_t s = 0; s < pl->hs.size(); ++s) {
            mg_handle* h = pl->hs[s];
            if (level >= top_of(h) || level_smoother(h, level) != MG_SMOOTH_PLANE) continue;
            void* xb;
            const void* bb;
            level_bufs(h, prec, level, &xb, &bb);
            std::vector<PlaneStep> st;
            plane_sweep_steps(h, level, xb, bb, st);
            for (const PlaneStep& q : st) {
                Launch& L = P.begin(q.op, q.colour, 7);
                if (level == 0) {
                    L.prof = MG_PROF_SMOOTH0;
                    L.prof_n = 1;
                }
                BTask t = q.t;
                t.shell = (int)s;
                P.add(t, q.nblocks);
            }
        }
    }
    if (any_fused && (sweeps & 1)) {   // an odd count ends in the scratch: copy back
        P.begin(BOP_COPY);
        for (size_t s = 0; s < pl->hs.size(); ++s) {
            mg_handle* h = pl->hs[s];
            if (level >= top_of(h) || !fused_level(h, level)) continue;
            BTask t{};
            void* xb;
            const void* bb;
            level_bufs(h, prec, level, &xb, &bb);
            t.x = xb;
            t.b = h->L[level].t;
            t.n = h->L[level].D.n() * (i64)(vbytes(prec) / 4);
            t.shell = (int)s;
            P.add(t, vblocks(h, vector_items(t.n)));
        }
    }
}

void add_smooth(Program& P, Plan* pl, int level, int sweeps) {
    const size_t first_launch = P.launches.size();
    add_smooth_launches(P, pl, level, sweeps);
    for (size_t i = first_launch; i < P.launches.size(); ++i) P.launches[i].level = level;
}

// Outer FP64 residual and its norm for every shell.
void add_residual(Program& P, Plan* pl) {
    for (int st : {7, 19}) {
    Launch& L = P.begin(BOP_RESID, 0, st);
    L.prof = MG_PROF_RESIDUAL;
    L.prof_n = 1;
    for (size_t s = 0; s < pl->hs.size(); ++s) {
        mg_handle* h = pl->hs[s];
        if (h->stencil != st) continue;
        BTask t = task_of(h, 0);
        t.x = h->x64;
        t.b = h->b64;
        t.a64 = h->L[0].a64;
        t.y = pl->prec == PREC64 ? nullptr : h->L[0].r;
        t.e0 = pl->prec == PREC64 ? nullptr : h->L[0].e;   // (the cycle's ZERO, fused here)
        t.z = h->part;
        t.shell = (int)s;
        P.add(t, red_blocks(h->L[0].D.n()));
    }
    }
    P.begin(BOP_FINALIZE);
    for (size_t s = 0; s < pl->hs.size(); ++s) {
        mg_handle* h = pl->hs[s];
        BTask t{};
        t.scal = h->scal;
        t.z = h->part;
        t.n = red_blocks(h->L[0].D.n());
        t.slot = SC_RR;
        t.fin_scale = 1;
        t.ncells = h->L[0].D.n();
        t.y = pl->d_fin + 4 * s + 2;
        t.shell = (int)s;
        P.add(t, 1);
    }
}

void build_iteration(Plan* pl) {
    Program& P = pl->iter;
    const int prec = pl->prec;
    int depth = 0;
    for (mg_handle* h : pl->hs) depth = std::max(depth, top_of(h));
    // the fine correction starts at zero: the outer residual that ends the
    // prologue and every iteration clears it (FP32 / FP16 cycles)
    // down leg
    for (int l = 0; l < depth; ++l) {
        add_smooth(P, pl, l, pl->hs[0]->opts.nu1);
        for (int st : {7, 19}) {
        Launch& L = P.begin(BOP_RESTRICT, 0, st);
        L.level = l;
        if (l == 0) {
            L.prof = MG_PROF_RESTRICT0;
            L.prof_n = 1;
        }
        for (size_t s = 0; s < pl->hs.size(); ++s) {
            mg_handle* h = pl->hs[s];
            if (l >= top_of(h) || h->stencil != st) continue;
            BTask t = task_of(h, l);
            level_bufs(h, prec, l, &t.x, &t.b);
            t.y = h->L[l + 1].r;
            t.z = h->L[l + 1].e;
            t.shell = (int)s;
            P.add(t, vblocks(h, restrict_items(h->L[l].D, h->L[l + 1].D)));
        }
        }
    }
    // bottom: coarse tails (one launch per stencil) and dense coarse solves
    for (int st : {7, 19}) {
        bool any = false;
        size_t smem = 0;
        for (size_t s = 0; s < pl->hs.size(); ++s) {
            mg_handle* h = pl->hs[s];
            if (h->tail_level <= 0 || h->stencil != st) continue;
            TailTask tt = h->tail_host;
            tt.active = pl->d_active;
            tt.shell = (int)s;
            P.tails.push_back(tt);
            // the shared-memory form when every shell's tail has it (the two
            // forms give the same bits)
            const size_t own = h->tail_cluster == lead(pl)->tail_cluster ? h->tail_smem : 0;
            smem = !any ? own : (own && smem ? std::max(smem, own) : 0);
            any = true;
        }
        if (any) {
            Launch& L = P.begin(-1);
            L.tail_stencil = st;
            L.prof = MG_PROF_TAIL;
            L.prof_n = 1;
            L.smem = smem;
        }
    }
    P.begin(BOP_COARSE);
    for (size_t s = 0; s < pl->hs.size(); ++s) {
        mg_handle* h = pl->hs[s];
        if (h->tail_level > 0) continue;
        BTask t{};
        const int nl = (int)h->L.size();
        t.binv = h->binv;
        t.n = h->ncoarse;
        void* x;
        const void* b;
        level_bufs(h, prec, nl - 1, &x, &b);
        t.x = x;
        t.b = b;
        t.shell = (int)s;
        P.add(t, std::min((h->ncoarse + 7) / 8, 152 * 4));
    }
    // up leg
    for (int l = depth - 1; l >= 0; --l) {
        Launch& L = P.begin(BOP_PROLONG);
        L.level = l;
        if (l == 0) {
            L.prof = MG_PROF_PROLONG0;
            L.prof_n = 1;
        }
        for (size_t s = 0; s < pl->hs.size(); ++s) {
            mg_handle* h = pl->hs[s];
            if (l >= top_of(h)) continue;
            BTask t = task_of(h, l);
            level_bufs(h, prec, l, &t.x, &t.b);
            t.b = h->L[l + 1].e;
            t.shell = (int)s;
            P.add(t, vblocks(h, prolong_items(h->L[l].D)));
        }
        add_smooth(P, pl, l, pl->hs[0]->opts.nu2);
    }
    if (prec != PREC64) {
        Launch& L = P.begin(BOP_UPDATE);
        L.prof = MG_PROF_UPDATE;
        L.prof_n = 1;
        for (size_t s = 0; s < pl->hs.size(); ++s) {
            mg_handle* h = pl->hs[s];
            BTask t{};
            t.x = h->x64;
            t.b = h->L[0].e;
            t.scal = h->scal;
            t.n = h->L[0].D.n();
            t.shell = (int)s;
            P.add(t, vblocks(h, vector_items(t.n)));
        }
    }
    add_residual(P, pl);
    P.drop_empty();
}

// The timing slot of a launch: the named fine-level ones, the coarser
// levels' operations by level, the rest together.
int slot_of(const Launch& L) {
    return L.prof >= 0   ? L.prof
           : L.level > 0 ? MG_PROF_LEVEL_BASE + std::min(L.level, MG_PROF_SLOTS - 1 - MG_PROF_LEVEL_BASE)
                         : MG_PROF_OTHER;
}

// Launch-clock buffers for n launches (device and pinned host), grown on
// demand; a grown iteration buffer needs a new graph (the old one holds the
// old address).
mg_status stamp_buffers(size_t n, unsigned long long** d, unsigned long long** hbuf, size_t* cap) {
    if (n <= *cap && *d) return MG_OK;
    if (*d) cudaFree(*d);
    if (*hbuf) cudaFreeHost(*hbuf);
    *d = *hbuf = nullptr;
    *cap = 0;
    // two words a launch, and two more for the accumulated spans
    CK(cudaMalloc((void**)d, 2 * sizeof(unsigned long long) * (n + 1)));
    CK(cudaMallocHost((void**)hbuf, 2 * sizeof(unsigned long long) * (n + 1)));
    *cap = n;
    return MG_OK;
}

// Launches P's kernels in order.  With d_st (profiling), every launch also
// records its clock (its CTAs' first start after the grid-dependency wait and
// last end) in d_st + 2 i.  Unlike events between launches, the clocks leave
// the launches' programmatic overlap as it is.
mg_status run_program(Plan* pl, const Program& P, const BTask* d_tasks, const int* active,
                      unsigned long long* d_st = nullptr) {
    mg_handle* h0 = lead(pl);
    const int nl = (int)P.launches.size();
    for (int i = 0; i < nl; ++i) {
        const Launch& L = P.launches[i];
        if (!L.tail_stencil && L.total == 0) continue;   // launches nothing
        unsigned long long* st = d_st ? d_st + 2 * i : nullptr;
        const int slot = slot_of(L);
        if (h0->prof_events) prof_begin(h0, slot);
        if (L.tail_stencil) {
            int first = 0, n = 0;
            for (size_t k = 0; k < P.tails.size(); ++k) {
                const int sten = P.tails[k].lev[0].v.stencil;
                if (sten != L.tail_stencil) continue;
                if (n == 0) first = (int)k;
                ++n;
            }
            CK(launch_tail(pl->d_tails + first, n, h0->tail_cluster, L.tail_stencil, pl->prec, pl->stream, st,
                           L.smem));
        } else if (L.op == BOP_SWEEP) {
            CK(launch_sweep(d_tasks + L.t0, L.nt, L.total, active, L.stencil, L.axi, pl->prec, L.smem, L.threads,
                            pl->stream, st));
        } else {
            CK(launch_batch(d_tasks + L.t0, L.nt, L.total, active, L.op, L.colour, L.stencil, pl->prec,
                            pl->stream, st));
        }
        if (h0->prof_events) prof_end(h0, slot, L.prof >= 0 ? L.prof_n : 1);
        h0->launches += 1;
    }
    return MG_OK;
}

// run_program with clocks: reset, the launches, the clocks copied to h_st;
// stamps_collect reads them once the stream has passed that copy.
mg_status run_clocked(Plan* pl, const Program& P, const BTask* d_tasks, const int* active,
                      unsigned long long* d_st, unsigned long long* h_st) {
    const int nl = (int)P.launches.size();
    CK(launch_stamp_reset(d_st, nl, pl->stream));
    lead(pl)->launches += 1;
    CKS(run_program(pl, P, d_tasks, active, d_st));
    if (nl > 0)
        CK(cudaMemcpyAsync(h_st, d_st, 2 * sizeof(unsigned long long) * nl, cudaMemcpyDeviceToHost, pl->stream));
    return MG_OK;
}

// Adds the launch clocks of one run of P (read back into h_st) to the slots;
// the time between its first start and last end that no launch covers goes
// to the gap slot.
void stamps_collect(mg_handle* h0, const Program& P, const unsigned long long* h_st) {
    unsigned long long lo = ~0ull, hi = 0, busy = 0;
    for (size_t i = 0; i < P.launches.size(); ++i) {
        const unsigned long long a = h_st[2 * i], b = h_st[2 * i + 1];
        if (a == ~0ull || b < a) continue;   // the launch ran no CTA
        const Launch& L = P.launches[i];
        const int slot = slot_of(L);
        h0->prof_ms[slot] += (double)(b - a) * 1e-6;
        h0->prof_n[slot] += L.prof >= 0 ? L.prof_n : 1;
        busy += b - a;
        lo = std::min(lo, a);
        hi = std::max(hi, b);
    }
    if (lo != ~0ull && hi - lo >= busy) {
        h0->prof_ms[MG_PROF_GAPS] += (double)(hi - lo - busy) * 1e-6;
        h0->prof_n[MG_PROF_GAPS] += 1;
    }
}

// The same from clocks accumulated on the device (launch_stamp_accum) over
// the passes of the device-side loop.
void acc_collect(mg_handle* h0, const Program& P, const unsigned long long* acc) {
    const size_t nl = P.launches.size();
    unsigned long long busy = 0;
    for (size_t i = 0; i < nl; ++i) {
        if (!acc[2 * i + 1]) continue;
        const Launch& L = P.launches[i];
        const int slot = slot_of(L);
        h0->prof_ms[slot] += (double)acc[2 * i] * 1e-6;
        h0->prof_n[slot] += (long long)acc[2 * i + 1] * (L.prof >= 0 ? L.prof_n : 1);
        busy += acc[2 * i];
    }
    if (acc[2 * nl + 1] && acc[2 * nl] >= busy) {
        h0->prof_ms[MG_PROF_GAPS] += (double)(acc[2 * nl] - busy) * 1e-6;
        h0->prof_n[MG_PROF_GAPS] += (long long)acc[2 * nl + 1];
    }
}

mg_status upload_call(Plan* pl, const Program& P) {
    const size_t need = P.tasks.size() * sizeof(BTask);
    if (need > pl->call_cap) {
        if (pl->d_call) cudaFree(pl->d_call);
        pl->d_call = nullptr;
        const size_t cap = std::max(need, (size_t)64 * sizeof(BTask));
        CK(cudaMalloc(&pl->d_call, cap));
        pl->call_cap = cap;
    }
    if (need) CK(cudaMemcpyAsync(pl->d_call, P.tasks.data(), need, cudaMemcpyHostToDevice, pl->stream));
    return MG_OK;
}

// The iteration's clock buffer; a new one retires the graphs that hold the
// old address.
mg_status iter_stamps(Plan* pl) {
    if (pl->iter.launches.size() > pl->stamp_it_cap && (pl->gexec || pl->lexec)) {
        CK(cudaStreamSynchronize(pl->stream));   // no graph in flight uses the old buffer
        if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
        if (pl->lexec) cudaGraphExecDestroy(pl->lexec);
        pl->gexec = nullptr;
        pl->lexec = nullptr;
    }
    CKS(stamp_buffers(pl->iter.launches.size(), &pl->d_stamp_it, &pl->h_stamp_it, &pl->stamp_it_cap));
    return MG_OK;
}

// A prologue or epilogue (not captured), clocked while profiling.
mg_status run_call(Plan* pl, const Program& P) {
    if (!clocks(lead(pl))) return run_program(pl, P, pl->d_call, nullptr);
    CKS(stamp_buffers(P.launches.size(), &pl->d_stamp_call, &pl->h_stamp_call, &pl->stamp_call_cap));
    return run_clocked(pl, P, pl->d_call, nullptr, pl->d_stamp_call, pl->h_stamp_call);
}

mg_status build_graph(Plan* pl) {
    mg_handle* h0 = lead(pl);
    if (pl->gexec) {
        cudaGraphExecDestroy(pl->gexec);
        pl->gexec = nullptr;
    }
    const bool prof = clocks(h0);
    if (prof) CKS(iter_stamps(pl));
    const long long before = h0->launches;
    CK(cudaStreamBeginCapture(pl->stream, cudaStreamCaptureModeThreadLocal));
    const mg_status st = prof ? run_clocked(pl, pl->iter, pl->d_iter, pl->d_active, pl->d_stamp_it, pl->h_stamp_it)
                              : run_program(pl, pl->iter, pl->d_iter, pl->d_active);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(pl->stream, &g);
    if (st != MG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    CK(e);
    pl->graph_launches = h0->launches - before;
    h0->launches = before;
    const cudaError_t ei = cudaGraphInstantiate(&pl->gexec, g, 0);
    cudaGraphDestroy(g);
    CK(ei);
    pl->graph_prof = prof;
    return MG_OK;
}

mg_status read_fin(Plan* pl) {
    CK(cudaMemcpyAsync(pl->h_fin, pl->d_fin, sizeof(double) * 4 * pl->hs.size(), cudaMemcpyDeviceToHost,
                       pl->stream));
    CK(cudaStreamSynchronize(pl->stream));
    prof_collect(lead(pl));
    return MG_OK;
}

}  // namespace

void plan_destroy(Plan* pl) {
    if (!pl) return;
    if (pl->stream) cudaStreamSynchronize(pl->stream);
    if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
    if (pl->d_iter) cudaFree(pl->d_iter);
    if (pl->d_tails) cudaFree(pl->d_tails);
    if (pl->d_maps) cudaFree(pl->d_maps);
    if (pl->d_active) cudaFree(pl->d_active);
    if (pl->d_fin) cudaFree(pl->d_fin);
    if (pl->d_call) cudaFree(pl->d_call);
    if (pl->h_active) cudaFreeHost(pl->h_active);
    if (pl->h_fin) cudaFreeHost(pl->h_fin);
    if (pl->d_stamp_it) cudaFree(pl->d_stamp_it);
    if (pl->h_stamp_it) cudaFreeHost(pl->h_stamp_it);
    if (pl->d_stamp_call) cudaFree(pl->d_stamp_call);
    if (pl->h_stamp_call) cudaFreeHost(pl->h_stamp_call);
    if (pl->lexec) cudaGraphExecDestroy(pl->lexec);
    if (pl->d_loop) cudaFree(pl->d_loop);
    if (pl->h_loop) cudaFreeHost(pl->h_loop);
    if (pl->d_ctl) cudaFree(pl->d_ctl);
    if (pl->h_ctl) cudaFreeHost(pl->h_ctl);
    if (pl->d_acc) cudaFree(pl->d_acc);
    if (pl->h_acc) cudaFreeHost(pl->h_acc);
    delete pl;
}

namespace {

template <typename P>
cudaError_t grow(P** ptr, size_t* cap, size_t need, bool pinned) {
    if (need <= *cap && *ptr) return cudaSuccess;
    const size_t c = std::max(need, *cap * 2 + 1);
    if (*ptr) {
        if (pinned) cudaFreeHost(*ptr);
        else cudaFree(*ptr);
        *ptr = nullptr;
    }
    cudaError_t e = pinned ? cudaMallocHost((void**)ptr, sizeof(P) * c) : cudaMalloc((void**)ptr, sizeof(P) * c);
    if (e == cudaSuccess) *cap = c;
    return e;
}

}  // namespace

// Point a plan at a (new) set of handles: rebuild the iteration tables and
// upload them into the plan's buffers (grown only when too small).
mg_status plan_reset(Plan* pl, mg_handle* const* hs, int n, bool iteration) {
    if (n <= 0) return MG_EINVAL;
    for (int s = 0; s < n; ++s)
        if (!hs[s] || hs[s]->prec != hs[0]->prec || hs[s]->device != hs[0]->device) {
            set_error("batch handles must share device and precision");
            return MG_EINVAL;
        }
    // a plan pinned to one stream is only ever used in that stream's order;
    // otherwise wait until the previous handles' work is done
    if (pl->stream && !pl->fixed) CK(cudaStreamSynchronize(pl->stream));
    pl->hs.assign(hs, hs + n);
    pl->prec = hs[0]->prec;
    pl->stream = pl->fixed ? pl->fixed : hs[0]->stream;
    if (pl->gexec) {
        cudaGraphExecDestroy(pl->gexec);
        pl->gexec = nullptr;
    }
    if (pl->lexec) {
        cudaGraphExecDestroy(pl->lexec);
        pl->lexec = nullptr;
    }
    CK(grow(&pl->d_active, &pl->dact_cap, (size_t)n, false));
    CK(grow(&pl->d_loop, &pl->dloop_cap, (size_t)n, false));
    CK(grow(&pl->h_loop, &pl->hloop_cap, (size_t)n, true));
    CK(grow(&pl->d_ctl, &pl->dctl_cap, (size_t)2, false));
    CK(grow(&pl->h_ctl, &pl->hctl_cap, (size_t)2, true));
    CK(grow(&pl->h_active, &pl->hact_cap, (size_t)n, true));
    CK(grow(&pl->d_fin, &pl->dfin_cap, (size_t)4 * n, false));
    CK(grow(&pl->h_fin, &pl->hfin_cap, (size_t)4 * n, true));
    pl->iter = Program();
    if (!iteration) return MG_OK;
    build_iteration(pl);
    std::stable_sort(pl->iter.tails.begin(), pl->iter.tails.end(),
                     [](const TailTask& a, const TailTask& b) { return a.lev[0].v.stencil < b.lev[0].v.stencil; });
    if (!pl->iter.maps.empty()) {
        size_t count = 0;
        for (const MapReq& q : pl->iter.maps) count += sweep_map_count(q.stencil, q.prec);
        const size_t nb = 128 * count;
        CK(grow(&pl->d_maps, &pl->maps_cap, nb, false));
        // host images of the maps (CUtensorMap is 128 bytes, 64-byte aligned)
        std::vector<unsigned long long> img(nb / 8);
        size_t at = 0;
        for (const MapReq& q : pl->iter.maps) {
            BTask& t = pl->iter.tasks[q.task];
            CK(encode_sweep_maps(&img[16 * at], t, q.stencil, q.prec));
            t.tmap = pl->d_maps + 128 * at;
            at += sweep_map_count(q.stencil, q.prec);
        }
        CK(cudaMemcpyAsync(pl->d_maps, img.data(), nb, cudaMemcpyHostToDevice, pl->stream));
        CK(cudaStreamSynchronize(pl->stream));   // img is pageable and local
    }
    CK(grow(&pl->d_iter, &pl->iter_cap, pl->iter.tasks.size() + 1, false));
    if (!pl->iter.tasks.empty())
        CK(cudaMemcpyAsync(pl->d_iter, pl->iter.tasks.data(), sizeof(BTask) * pl->iter.tasks.size(),
                           cudaMemcpyHostToDevice, pl->stream));
    if (!pl->iter.tails.empty()) {
        CK(grow(&pl->d_tails, &pl->tails_cap, pl->iter.tails.size(), false));
        CK(cudaMemcpyAsync(pl->d_tails, pl->iter.tails.data(), sizeof(TailTask) * pl->iter.tails.size(),
                           cudaMemcpyHostToDevice, pl->stream));
    }
    if (!pl->fixed) CK(cudaStreamSynchronize(pl->stream));
    return MG_OK;
}

mg_status plan_create(mg_handle* const* hs, int n, Plan** out, cudaStream_t stream, bool iteration) {
    *out = nullptr;
    if (n <= 0) return MG_EINVAL;
    Plan* pl = new Plan();
    pl->fixed = stream;
    const mg_status st = plan_reset(pl, hs, n, iteration);
    if (st != MG_OK) {
        plan_destroy(pl);
        return st;
    }
    *out = pl;
    return MG_OK;
}

// Prologue for every shell of the plan: x in, b = J (f - mean_J f), first
// residual and its norm; initialises the per-shell states.
mg_status plan_start(Plan* pl, const double* const* f, double* const* x, const double* tol, SolveState* S) {
    const int n = (int)pl->hs.size();
    Program pro;
    pro.begin(BOP_COPY);
    for (int i = 0; i < n; ++i) {
        BTask t{};
        t.x = pl->hs[i]->x64;
        t.b = x[i];
        t.n = 2 * pl->hs[i]->L[0].D.n();
        t.shell = i;
        pro.add(t, vblocks(pl->hs[i], vector_items(t.n)));
    }
    pro.begin(BOP_SUM);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        BTask t{};
        t.b = h->J64;
        t.y = (void*)f[i];
        t.z = h->part;
        t.n = h->L[0].D.n();
        t.shell = i;
        pro.add(t, red_blocks(t.n));
    }
    pro.begin(BOP_FINALIZE);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        BTask t{};
        t.scal = h->scal;
        t.z = h->part;
        t.n = red_blocks(h->L[0].D.n());
        t.slot = SC_SUMJF;
        t.y = pl->d_fin + 4 * i + 0;
        t.shell = i;
        pro.add(t, 1);
    }
    pro.begin(BOP_RHS);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        BTask t{};
        t.x = h->b64;
        t.b = f[i];
        t.y = h->J64;
        t.z = h->part;
        t.scal = h->scal;
        t.aux = h->sumJ;
        t.n = h->L[0].D.n();
        t.shell = i;
        pro.add(t, red_blocks(t.n));
    }
    pro.begin(BOP_FINALIZE);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        BTask t{};
        t.scal = h->scal;
        t.z = h->part;
        t.n = red_blocks(h->L[0].D.n());
        t.slot = SC_BB;
        t.fin_scale = 1;
        t.ncells = h->L[0].D.n();
        t.y = pl->d_fin + 4 * i + 1;
        t.shell = i;
        pro.add(t, 1);
    }
    add_residual(pro, pl);
    pro.drop_empty();   // the residual launch of the stencil no shell has
    CKS(upload_call(pl, pro));
    CKS(run_call(pl, pro));
    CKS(read_fin(pl));
    if (clocks(pl->hs[0])) stamps_collect(pl->hs[0], pro, pl->h_stamp_call);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        SolveState& q = S[i];
        q = SolveState();
        q.tol = tol[i];
        std::memset(&q.R, 0, sizeof(mg_report));
        q.R.levels = (int)h->L.size();
        q.R.stencil = h->stencil;
        q.R.removed_mean = pl->h_fin[4 * i] / h->sumJ;
        const double bn = std::sqrt(pl->h_fin[4 * i + 1]);
        if (!std::isfinite(bn)) {
            q.st = MG_ENAN;
            q.done = true;
            set_error("non-finite right-hand side");
        }
        q.bnorm = bn > 0 ? bn : 1.0;
        q.rr = pl->h_fin[4 * i + 2];
    }
    return MG_OK;
}

// The stop test of every shell (the same rule as a lone solve); returns the
// number still iterating and sets the active flags (host side).
int plan_check(Plan* pl, SolveState* S) {
    const int n = (int)pl->hs.size();
    int nactive = 0;
    for (int i = 0; i < n; ++i) {
        SolveState& q = S[i];
        if (!q.done) {
            const double rel = std::sqrt(q.rr) / q.bnorm;
            if (q.it < MG_HIST) q.R.res_hist[q.it] = rel;
            q.R.rel_res = rel;
            if (!std::isfinite(rel)) {
                q.st = MG_ENAN;
                set_error("non-finite residual");
                q.done = true;
            } else if (rel <= q.tol) {
                q.done = true;
            } else {
                q.best = std::min(q.best, rel);
                if (rel > 1e3 * q.best) {
                    q.st = MG_EDIVERGED;
                    set_error("residual diverged");
                    q.done = true;
                } else if (q.it >= pl->hs[i]->opts.max_iters) {
                    q.st = MG_ENOCONV;
                    set_error("max_iters reached");
                    q.done = true;
                }
            }
        }
        pl->h_active[i] = q.done ? 0 : 1;
        nactive += q.done ? 0 : 1;
    }
    return nactive;
}

// One outer iteration for the shells whose flag plan_check set, then the new
// residual norms into the states.
mg_status plan_iterate(Plan* pl, SolveState* S, bool use_graph) {
    const int n = (int)pl->hs.size();
    mg_handle* h0 = lead(pl);
    CK(cudaMemcpyAsync(pl->d_active, pl->h_active, sizeof(int) * n, cudaMemcpyHostToDevice, pl->stream));
    const bool prof = clocks(h0);
    if (use_graph) {
        if (!pl->gexec || pl->graph_prof != prof) CKS(build_graph(pl));
        CK(cudaGraphLaunch(pl->gexec, pl->stream));
        h0->launches += pl->graph_launches;
    } else {
        if (prof) {
            CKS(iter_stamps(pl));
            CKS(run_clocked(pl, pl->iter, pl->d_iter, pl->d_active, pl->d_stamp_it, pl->h_stamp_it));
        } else {
            CKS(run_program(pl, pl->iter, pl->d_iter, pl->d_active));
        }
    }
    CKS(read_fin(pl));
    if (prof) stamps_collect(h0, pl->iter, pl->h_stamp_it);
    for (int i = 0; i < n; ++i)
        if (pl->h_active[i]) {
            S[i].it += 1;
            S[i].rr = pl->h_fin[4 * i + 2];
        }
    return MG_OK;
}

mg_status plan_time(Plan* pl, int warm, int reps, double* ms) {
    const int n = (int)pl->hs.size();
    std::vector<SolveState> S(n);
    for (int i = 0; i < n; ++i) pl->h_active[i] = 1;
    mg_handle* h0 = lead(pl);
    for (int r = 0; r < warm; ++r) CKS(plan_iterate(pl, S.data(), true));
    CK(cudaEventRecord(h0->ev0, pl->stream));
    for (int r = 0; r < reps; ++r) {
        for (int i = 0; i < n; ++i) pl->h_active[i] = 1;
        CKS(plan_iterate(pl, S.data(), true));
    }
    CK(cudaEventRecord(h0->ev1, pl->stream));
    CK(cudaEventSynchronize(h0->ev1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h0->ev0, h0->ev1));
    *ms = (double)t / (reps > 0 ? reps : 1);
    return MG_OK;
}

// Epilogue for every shell of the plan: remove the J-weighted mean, x out.
mg_status plan_finish(Plan* pl, double* const* x) {
    const int n = (int)pl->hs.size();
    Program epi;
    epi.begin(BOP_SUM);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        BTask t{};
        t.b = h->J64;
        t.y = h->x64;
        t.z = h->part;
        t.n = h->L[0].D.n();
        t.shell = i;
        epi.add(t, red_blocks(t.n));
    }
    epi.begin(BOP_FINALIZE);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        BTask t{};
        t.scal = h->scal;
        t.z = h->part;
        t.n = red_blocks(h->L[0].D.n());
        t.slot = SC_SUMJX;
        t.y = pl->d_fin + 4 * i + 3;
        t.shell = i;
        epi.add(t, 1);
    }
    epi.begin(BOP_SHIFT);
    for (int i = 0; i < n; ++i) {
        mg_handle* h = pl->hs[i];
        BTask t{};
        t.x = h->x64;
        t.scal = h->scal;
        t.aux = h->sumJ;
        t.n = h->L[0].D.n();
        t.shell = i;
        epi.add(t, vblocks(pl->hs[i], t.n));
    }
    epi.begin(BOP_COPY);
    for (int i = 0; i < n; ++i) {
        BTask t{};
        t.x = x[i];
        t.b = pl->hs[i]->x64;
        t.n = 2 * pl->hs[i]->L[0].D.n();
        t.shell = i;
        epi.add(t, vblocks(pl->hs[i], vector_items(t.n)));
    }
    CKS(upload_call(pl, epi));
    CKS(run_call(pl, epi));
    if (clocks(lead(pl))) {
        CK(cudaStreamSynchronize(pl->stream));
        stamps_collect(lead(pl), epi, pl->h_stamp_call);
    }
    return MG_OK;
}

namespace {

// The while-node graph of the device-side loop: one pass = the iteration,
// the stop tests (which set the node's condition), and with clocks their
// accumulation.  False with the runtime's error cleared when the graph
// cannot be made (the caller then loops on the host).
bool build_loop(Plan* pl) {
    mg_handle* h0 = lead(pl);
    if (pl->lexec) {
        cudaGraphExecDestroy(pl->lexec);
        pl->lexec = nullptr;
    }
    const bool prof = clocks(h0);
    const int nl = (int)pl->iter.launches.size();
    if (prof && (iter_stamps(pl) != MG_OK ||
                 stamp_buffers((size_t)nl, &pl->d_acc, &pl->h_acc, &pl->acc_cap) != MG_OK)) {
        cudaGetLastError();
        return false;
    }
    cudaGraph_t top = nullptr;
    if (cudaGraphCreate(&top, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bool ok = false;
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node = nullptr;
    if (cudaGraphConditionalHandleCreate(&cond, top, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = cudaGraphAddNode(&node, top, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const long long before = h0->launches;
        ok = cudaStreamBeginCaptureToGraph(pl->stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            bool run = run_program(pl, pl->iter, pl->d_iter, pl->d_active, prof ? pl->d_stamp_it : nullptr) == MG_OK;
            run = run && launch_loop_check(pl->d_loop, (int)pl->hs.size(), pl->d_fin, pl->d_active, pl->d_ctl, cond,
                                           pl->stream) == cudaSuccess;
            h0->launches += 1;
            if (prof) {
                run = run && launch_stamp_accum(pl->d_stamp_it, nl, pl->d_acc, pl->stream) == cudaSuccess;
                h0->launches += 1;
            }
            cudaGraph_t got = nullptr;
            ok = cudaStreamEndCapture(pl->stream, &got) == cudaSuccess && run;
        }
        pl->loop_launches = h0->launches - before;
        h0->launches = before;
    }
    if (ok) ok = cudaGraphInstantiate(&pl->lexec, top, 0) == cudaSuccess;
    cudaGraphDestroy(top);
    if (!ok) {
        if (pl->lexec) cudaGraphExecDestroy(pl->lexec);
        pl->lexec = nullptr;
        cudaGetLastError();
        return false;
    }
    pl->loop_prof = prof;
    return true;
}

// Runs the outer iterations of every still-active shell on the device (the
// loop graph), then takes the stop tests' results back into S: the same
// iterates, counts, histories and statuses as the host loop gives.  Sets
// *unavailable (and returns MG_OK) when the graph cannot be made.
mg_status plan_loop(Plan* pl, SolveState* S, bool* unavailable) {
    const int n = (int)pl->hs.size();
    mg_handle* h0 = lead(pl);
    const bool prof = clocks(h0);
    *unavailable = false;
    if (!pl->lexec || pl->loop_prof != prof) {
        if (!build_loop(pl)) {
            pl->loop_failed = true;
            *unavailable = true;
            return MG_OK;
        }
    }
    long long most = 0;
    for (int i = 0; i < n; ++i) {
        const SolveState& q = S[i];
        LoopShell& L = pl->h_loop[i];
        L.bnorm = q.bnorm;
        L.best = q.best;
        L.tol = q.tol;
        L.rr = q.rr;
        L.rel = q.R.rel_res;
        L.it = q.it;
        L.max_iters = pl->hs[i]->opts.max_iters;
        L.done = q.done ? 1 : 0;
        L.why = LOOP_RUN;
        if (!q.done) most = std::max(most, (long long)L.max_iters - q.it);
    }
    // never binds: every pass moves each active shell one iteration toward
    // its limit
    pl->h_ctl[0] = 0;
    pl->h_ctl[1] = (int)std::min<long long>(most + 1, INT_MAX);
    cudaStream_t s = pl->stream;
    CK(cudaMemcpyAsync(pl->d_loop, pl->h_loop, sizeof(LoopShell) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pl->d_ctl, pl->h_ctl, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pl->d_active, pl->h_active, sizeof(int) * n, cudaMemcpyHostToDevice, s));
    const size_t nl = pl->iter.launches.size();
    if (prof) {
        CK(cudaMemsetAsync(pl->d_acc, 0, 2 * sizeof(unsigned long long) * (nl + 1), s));
        CK(launch_stamp_reset(pl->d_stamp_it, (int)nl, s));
        h0->launches += 1;
    }
    CK(cudaGraphLaunch(pl->lexec, s));
    CK(cudaMemcpyAsync(pl->h_loop, pl->d_loop, sizeof(LoopShell) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pl->h_ctl, pl->d_ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (prof)
        CK(cudaMemcpyAsync(pl->h_acc, pl->d_acc, 2 * sizeof(unsigned long long) * (nl + 1), cudaMemcpyDeviceToHost,
                           s));
    CK(cudaStreamSynchronize(s));
    h0->launches += (long long)pl->h_ctl[0] * pl->loop_launches;
    if (prof) acc_collect(h0, pl->iter, pl->h_acc);
    for (int i = 0; i < n; ++i) {
        SolveState& q = S[i];
        if (q.done) continue;
        const LoopShell& L = pl->h_loop[i];
        for (int k = q.it + 1; k <= L.it && k < MG_HIST; ++k) q.R.res_hist[k] = L.hist[k];
        q.it = L.it;
        q.rr = L.rr;
        q.best = L.best;
        q.R.rel_res = L.rel;
        q.done = true;
        if (L.why == LOOP_NAN) {
            q.st = MG_ENAN;
            set_error("non-finite residual");
        } else if (L.why == LOOP_DIVERGED) {
            q.st = MG_EDIVERGED;
            set_error("residual diverged");
        } else if (L.why == LOOP_NOCONV) {
            q.st = MG_ENOCONV;
            set_error("max_iters reached");
        } else if (!L.done) {
            q.st = MG_ENOCONV;
            set_error("outer loop stopped at its pass limit");
        }
    }
    return MG_OK;
}

bool host_loop_forced() { return std::getenv("MG_HOST_LOOP") != nullptr; }

}  // namespace

// Solve every shell of the plan; the stop logic per shell is the one of a
// lone solve, so a shell's iterates do not depend on its batch companions.
mg_status plan_solve(Plan* pl, const double* const* f, double* const* x, const double* tol, mg_report* reps) {
    const int n = (int)pl->hs.size();
    mg_handle* h0 = lead(pl);
    cudaStream_t s = pl->stream;
    h0->launches = 0;
    CK(cudaEventRecord(h0->ev0, s));
    std::vector<SolveState> S(n);
    CKS(plan_start(pl, f, x, tol, S.data()));
    int active = plan_check(pl, S.data());
    const bool graphs = h0->use_graph && !h0->prof_events;
    if (active > 0 && graphs && !pl->loop_failed && !host_loop_forced()) {
        bool unavailable = false;
        CKS(plan_loop(pl, S.data(), &unavailable));
        if (!unavailable) active = 0;
    }
    while (active > 0) {
        CKS(plan_iterate(pl, S.data(), graphs));
        active = plan_check(pl, S.data());
    }
    CKS(plan_finish(pl, x));
    CK(cudaEventRecord(h0->ev1, s));
    CK(cudaEventSynchronize(h0->ev1));
    prof_collect(h0);
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h0->ev0, h0->ev1));
    mg_status worst = MG_OK;
    for (int i = 0; i < n; ++i) {
        SolveState& q = S[i];
        q.R.iters = q.it;
        q.R.seconds = ms * 1e-3;
        q.R.model_bytes = model_bytes_per_iteration(pl->hs[i]) * q.it;
        q.R.status = q.st;
        q.R.launches = h0->launches;
        if (reps) reps[i] = q.R;
        if (q.st != MG_OK && worst == MG_OK) worst = q.st;
    }
    return worst;
}

}  // namespace mgs

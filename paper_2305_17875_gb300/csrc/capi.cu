// capi.cu - handle lifecycle, multigrid hierarchy, V-cycle schedule, the
// FP64 iterative-refinement loop and the C ABI of include/mg.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "pc.h"
#include "line_smooth.cuh"
#include "plane_smooth.cuh"

using namespace mgs;

namespace mgs {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }

LevelView Level::view(int stencil) const {
    LevelView v{};
    v.D = D;
    v.cz = cz;
    v.ce = ce;
    v.cx = cx;
    v.stencil = stencil;
    for (int a = 0; a < 9; ++a) {
        v.c64.g[a] = g64[a];
        v.c32.g[a] = g32[a];
        v.c16.g[a] = g16[a];
        v.c16.s[a] = s16[a];
    }
    return v;
}

cudaMemPool_t lib_pool(int device) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64) device = 0;
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            cudaDeviceGetDefaultMemPool(&p, device);
        } else {
            unsigned long long keep = ~0ull;   // keep freed blocks for the next hierarchy
            cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pools[device] = p;
    }
    return pools[device];
}

}  // namespace mgs

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                 \
            return MG_ECUDA;                                                               \
        }                                                                                  \
    } while (0)

#define CKS(call)                           \
    do {                                    \
        mg_status s_ = (call);              \
        if (s_ != MG_OK) return s_;         \
    } while (0)

namespace {

constexpr int kMaxCoarse = 2048;   // largest coarsest level (dense bordered inverse)
// Semi-coarsening: a direction halves only if its mean diagonal coefficient is
// at least this fraction of the strongest coarsenable direction's.
constexpr double kSemiRatio = 0.7;
// Coarse-tail threshold when MG_TAIL=1 forces the tail without a cell count
// (MG_TAIL_CELLS); the tuner tries 16384.
constexpr i64 kTailCells = 65536;

bool finite(double v) { return std::isfinite(v); }

std::string check_grid(const mg_grid_desc* g) {
    if (!g) return "grid is NULL";
    if (g->nr < 1 || g->nth < 1) return "nr and nth must be >= 1";
    if (g->nph < 4 || (g->nph & 1)) return "nph must be even and >= 4";   // two cells degenerate the face metric
    if ((long long)g->nr * g->nth * g->nph > (1LL << 31)) return "grid too large";
    if (!(finite(g->r_in) && finite(g->r_out) && g->r_in > 0 && g->r_out > g->r_in))
        return "need 0 < r_in < r_out";
    if (g->cut != 0 && g->cut != 1) return "cut must be 0 or 1";
    if (g->cut) {
        if (!(g->th0 == 0.0 && g->th1 == M_PI)) return "the shell cut needs th0 = 0 and th1 = pi";
    } else if (!(finite(g->th0) && finite(g->th1) && g->th0 > 0 && g->th1 > g->th0 && g->th1 < M_PI)) {
        return "need 0 < th0 < th1 < pi";
    }
    if (g->mapping < 0 || g->mapping > 2) return "mapping must be 0, 1 or 2";
    if (!(finite(g->flattening) && g->flattening > -1 && g->flattening < 1)) return "need |flattening| < 1";
    if (!(finite(g->e2) && g->e2 > -1)) return "need e2 > -1";
    if (!(finite(g->stretch) && g->stretch >= 0)) return "need stretch >= 0";
    return "";
}

std::string check_opts(const mg_opts* o) {
    if (!o) return "opts is NULL";
    if (o->precision < 0 || o->precision > 2) return "precision must be 0, 1 or 2";
    if (o->smoother < 0 || o->smoother > 5) return "smoother must be 0 .. 5";
    if (o->smoother == MG_SMOOTH_PLANE && (o->plane_cycles < 1 || o->plane_cycles > 64))
        return "plane_cycles must be in 1..64";
    if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 > 64) return "bad nu1/nu2";
    if (o->max_levels < 1 || o->max_levels > 32) return "max_levels must be in 1..32";
    if (o->coarsen < 0 || o->coarsen > 1) return "coarsen must be 0 or 1";
    if (o->coarse_max < 1) return "coarse_max must be >= 1";
    if (o->max_iters < 0) return "max_iters must be >= 0";
    if (o->stencil != 0 && o->stencil != 7 && o->stencil != 19) return "stencil must be 0, 7 or 19";
    if (o->autotune < 0 || o->autotune > 2) return "autotune must be 0, 1 or 2";
    if (o->metric != MG_METRIC_DISCRETE && o->metric != MG_METRIC_ANALYTIC) return "metric must be 0 or 1";
    return "";
}

int stencil_of(const mg_grid_desc* g, const mg_opts* o) {
    if (o->stencil) return o->stencil;
    return g->mapping == MG_MAP_SPHERE ? 7 : 19;
}

// Combinations of a valid grid and valid options that are not built.
std::string check_pair(const mg_grid_desc* g, const mg_opts* o) {
    if (g->cut && stencil_of(g, o) == 19) {
        if (g->mapping == MG_MAP_TRIAXIAL)
            return "the shell cut with 19 points is built for axisymmetric mappings (sphere, oblate) only";
        if (o->smoother != MG_SMOOTH_GS && o->smoother != MG_SMOOTH_JACOBI)
            return "the shell cut with 19 points is built for the point smoothers (Gauss-Seidel, Jacobi) only";
    }
    if (o->smoother == MG_SMOOTH_PLANE) {
        if (stencil_of(g, o) != 7) return "plane relaxation is built for the 7-point operator only";
        if (g->nr & (g->nr - 1)) return "plane relaxation needs nr a power of two (the plane cycles end on one row)";
        if (g->nph > 512) return "plane relaxation: at most 512 longitudes (a warp solves a line in chunks of 16)";
    }
    return "";
}

void* dalloc(mg_handle* h, size_t bytes) {
    void* p = nullptr;
    if (h->fail_alloc_after >= 0 && h->allocs_done++ >= h->fail_alloc_after) return nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, lib_pool(h->device), h->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    h->dev_allocs.push_back(p);
    h->bytes += bytes;
    return p;
}

// Set-up scratch on the handle's stream, freed (stream-ordered) when the
// guard leaves scope.
struct TmpDev {
    void* p = nullptr;
    cudaStream_t s;
    TmpDev(size_t bytes, cudaStream_t st, int device) : s(st) {
        if (cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, lib_pool(device), s) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    ~TmpDev() {
        if (p) cudaFreeAsync(p, s);
    }
    TmpDev(const TmpDev&) = delete;
    TmpDev& operator=(const TmpDev&) = delete;
};

// Eq. stretching on a 0-based (possibly fractional / ghost) vertex index.
double stretch_unit(double jv, int n, double rx) {
    const double t = jv / n - 0.5;
    return rx == 0.0 ? t : std::tanh(rx * t) / (2.0 * std::tanh(rx / 2.0));
}

// Its derivative with respect to the index (the analytic metric option).
double d_stretch_unit(double jv, int n, double rx) {
    if (rx == 0.0) return 1.0 / n;
    const double c = std::cosh(rx * (jv / n - 0.5));
    return rx / (n * c * c * 2.0 * std::tanh(rx / 2.0));
}

int ncomp(int stencil) { return stencil == 19 ? 9 : 3; }
// Metric components kept per level: the diagonal for 7 points; all nine for
// 19 points, except on an axisymmetric mapping, whose longitude cross
// components (zeta-xi, eta-xi, xi-zeta, xi-eta) vanish to rounding face by face
// and are dropped (the operator is then the 11-point one they leave).
bool stored(const mg_handle* h, int a) {
    if (h->stencil == 7) return a == 0 || a == 4 || a == 8;
    return !h->axi || (a != 2 && a != 5 && a != 6 && a != 7);
}

mg_status read_scalars(mg_handle* h, int count) {
    CK(cudaMemcpyAsync(h->hscal, h->scal, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    prof_collect(h);
    return MG_OK;
}

// sum of a (optionally weighted by w) into scal[slot]
mg_status device_sum(mg_handle* h, const double* a, const double* w, i64 n, int slot) {
    CK(launch_sum(a, w, n, h->part, h->stream));
    CK(launch_finalize(h->part, red_blocks(n), 0, h->scal + slot, h->stream));
    h->launches += 2;
    return MG_OK;
}

// In-place LU with partial pivoting, then the first n columns / rows of the
// inverse of the bordered matrix [A 1; 1^T 0].
void free_handle(mg_handle* h) {
    if (!h) return;
    for (void* p : h->dev_allocs) cudaFreeAsync(p, h->stream);
    if (h->hf) cudaFreeHost(h->hf);
    if (h->hx) cudaFreeHost(h->hx);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (auto& p : h->prof_pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (int s = 0; s < MG_PROF_SLOTS; ++s)
        if (h->prof_open[s]) cudaEventDestroy(h->prof_open[s]);
    for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
    plan_destroy(h->solo);
    plan_destroy(h->batch);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// The index decoders divide by magic numbers; check them against true
// division on boundary and sampled dividends up to the level's cell count.
bool fastdiv_ok(const Dims& D) {
    const FastDiv* fd[5] = {&D.dph, &D.dth, &D.dhk, &D.dq, &D.dth2};
    const unsigned long long top = (unsigned long long)D.n() + 2;
    for (const FastDiv* f : fd) {
        unsigned long long n = 0;
        for (int it = 0; it < 4096 && n < top; ++it) {
            const unsigned v = (unsigned)n;
            if (f->div(v) != v / f->d) return false;
            n = n < 64 ? n + 1 : n + n / 7 + 1;
        }
        for (unsigned long long v : {(unsigned long long)f->d - 1, (unsigned long long)f->d,
                                     (unsigned long long)f->d + 1, top - 1, 0x7fffffffull}) {
            if (f->div((unsigned)v) != (unsigned)v / f->d) return false;
        }
    }
    return true;
}

// Radial-line factors of every level in the value type of `prec`, made on
// first use (set-up of a radial-line handle, or mg_smooth with kind 2).
mg_status ensure_line_factors(mg_handle* h, int prec) {
    const int cls = prec == PREC64 ? 0 : 1;
    const int kc = cls == 0 ? LineRows<double>::kC : LineRows<float>::kC;
    if (line_chunks(h->L[0].D.nr, kc) > 16) {
        set_error("radial-line smoother: at most " + std::to_string(16 * kc) + " radial cells in this precision");
        return MG_EINVAL;
    }
    bool missing = false;
    for (const Level& lv : h->L) missing = missing || !lv.lf[cls];
    if (!missing) return MG_OK;
    TmpDev tb(sizeof(unsigned), h->stream, h->device);
    if (!tb.p) return MG_ENOMEM;
    CK(cudaMemsetAsync(tb.p, 0, sizeof(unsigned), h->stream));
    for (Level& lv : h->L) {
        if (lv.lf[cls]) continue;
        if (!(lv.lf[cls] = dalloc(h, 3 * (size_t)(cls == 0 ? 8 : 4) * lv.D.n()))) return MG_ENOMEM;
        CK(launch_line_factors(lv.view(h->stencil), prec, lv.lf[cls], (unsigned*)tb.p, h->stream));
    }
    unsigned hb = 0;
    CK(cudaMemcpyAsync(&hb, tb.p, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hb) {
        set_error("a radial-line block of the operator has a zero pivot");
        return MG_EINVAL;
    }
    return MG_OK;
}

// Longitude-line factors of every level with at least four longitudes, in
// the value type of `prec`, made on first use.
mg_status ensure_xline_factors(mg_handle* h, int prec) {
    const int cls = prec == PREC64 ? 0 : 1;
    bool missing = false;
    for (const Level& lv : h->L) missing = missing || (lv.D.nph >= 4 && !lv.xf[cls]);
    if (!missing) return MG_OK;
    TmpDev tb(sizeof(unsigned), h->stream, h->device);
    if (!tb.p) return MG_ENOMEM;
    CK(cudaMemsetAsync(tb.p, 0, sizeof(unsigned), h->stream));
    for (Level& lv : h->L) {
        if (lv.xf[cls] || lv.D.nph < 4) continue;
        if (!(lv.xf[cls] = dalloc(h, 4 * (size_t)(cls == 0 ? 8 : 4) * lv.D.n()))) return MG_ENOMEM;
        CK(launch_xline_factors(lv.view(h->stencil), prec, lv.xf[cls], (unsigned*)tb.p, h->stream));
    }
    unsigned hb = 0;
    CK(cudaMemcpyAsync(&hb, tb.p, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hb) {
        set_error("a longitude-line block of the operator has a zero pivot");
        return MG_EINVAL;
    }
    return MG_OK;
}

// Plane hierarchies of every level above the coarsest (the semi-coarsening
// multigrid's smoother): the plane operator of the level (FP64), its radius
// coarsening R B P down to one row, the cycle-precision copies, the
// longitude-line factors and the work arrays of every 2-D level.
mg_status build_planes(mg_handle* h) {
    const bool f32 = h->prec != PREC64;
    const size_t vb = f32 ? sizeof(float) : sizeof(double);
    TmpDev tb(sizeof(unsigned), h->stream, h->device);
    if (!tb.p) return MG_ENOMEM;
    CK(cudaMemsetAsync(tb.p, 0, sizeof(unsigned), h->stream));
    for (size_t l = 0; l < (size_t)h->plane_levels; ++l) {
        Level& lv = h->L[l];
        lv.planes.clear();
        Dims D = lv.D;
        for (int m = 0;; ++m) {
            PlaneLevel P;
            P.D = D;
            const i64 n = D.n();
            for (int o = 0; o < 9; ++o) {
                if (!(P.c64[o] = (double*)dalloc(h, sizeof(double) * n))) return MG_ENOMEM;
                if (f32 && !(P.c32[o] = (float*)dalloc(h, sizeof(float) * n))) return MG_ENOMEM;
            }
            if (!(P.fac = dalloc(h, 4 * vb * n)) || !(P.e = dalloc(h, vb * n)) || !(P.r = dalloc(h, vb * n)) ||
                !(P.w = dalloc(h, vb * n)))
                return MG_ENOMEM;
            if (m == 0) {
                CK(launch_plane_op0(lv.view(h->stencil), P.c64, h->stream));
            } else {
                const PlaneLevel& F = lv.planes.back();
                CK(launch_plane_coarsen(F.c64, F.D, D, P.c64, h->stream));
            }
            if (f32)
                for (int o = 0; o < 9; ++o) CK(launch_cast32(P.c64[o], P.c32[o], n, h->stream));
            CK(launch_plane_factors(P.c64, D, h->prec, P.fac, (unsigned*)tb.p, h->stream));
            lv.planes.push_back(P);
            if (D.nr % 2 || D.nr < 2) break;   // one row: the plane cycles end here
            D = Dims{D.nr / 2, D.nth, D.nph};
            D.cut = lv.D.cut;
        }
    }
    unsigned hb = 0;
    CK(cudaMemcpyAsync(&hb, tb.p, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hb) {
        set_error("a longitude line of a plane operator has a zero pivot");
        return MG_EINVAL;
    }
    return MG_OK;
}

// The outer loop converts between FP64 and FP32 on the integer pipes; check
// those conversions against the hardware ones once per device and process.
mg_status conversion_check(mg_handle* h) {
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (h->device >= 0 && h->device < 64 && done[h->device]) return MG_OK;
    unsigned* bad = (unsigned*)h->part;
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned), h->stream));
    CK(launch_convert_check(bad, h->stream));
    unsigned hb = 0;
    CK(cudaMemcpyAsync(&hb, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hb != 0) {
        set_error("FP64/FP32 conversion self-check failed on " + std::to_string(hb) + " values");
        return MG_EINVAL;
    }
    if (h->device >= 0 && h->device < 64) done[h->device] = true;
    return MG_OK;
}

// Longest-first plan of the next level: which directions halve.
mg_status plan_next(mg_handle* h, const Level& lv, int f[3], bool* ok) {
    if (h->opts.smoother == MG_SMOOTH_PLANE && h->plane_levels == 0) {
        // semi-coarsening: the colatitude only, down to one plane (or an odd
        // row count), which the dense bordered solve takes when it fits; a
        // larger one hands over to the policy below (plane_levels set)
        if (lv.D.nth % 2 == 0 && lv.D.nth > 1) {
            *ok = true;
            f[0] = 2;
            f[1] = f[2] = 1;
            return MG_OK;
        }
        f[0] = f[1] = f[2] = 1;
        *ok = false;
        if (lv.D.n() <= kMaxCoarse) return MG_OK;
        h->plane_levels = (int)h->L.size() - 1 + (lv.D.nth >= 2 ? 1 : 0);
    }
    if (h->opts.smoother == MG_SMOOTH_PLANE && lv.D.n() <= h->opts.coarse_max) {
        *ok = false;
        f[0] = f[1] = f[2] = 1;
        return MG_OK;
    }
    const int n[3] = {lv.D.nth, lv.D.nr, lv.D.nph};
    bool can[3];
    for (int d = 0; d < 3; ++d) can[d] = n[d] % 2 == 0 && n[d] >= 4 && (d != 2 || n[d] % 4 == 0);
    *ok = can[0] || can[1] || can[2];
    f[0] = f[1] = f[2] = 1;
    if (!*ok) return MG_OK;
    if (h->opts.coarsen == MG_COARSEN_FULL) {
        for (int d = 0; d < 3; ++d) f[d] = can[d] ? 2 : 1;
        return MG_OK;
    }
    // mean diagonal coefficient over the faces that carry flux, per direction
    const i64 N = lv.D.n();
    CKS(device_sum(h, lv.g64[0], nullptr, N, 4));
    CKS(device_sum(h, lv.g64[4], nullptr, N, 5));
    CKS(device_sum(h, lv.g64[8], nullptr, N, 6));
    CKS(read_scalars(h, 7));
    const double cnt[3] = {(double)lv.D.nr * (lv.D.nth - 1) * lv.D.nph,
                           (double)(lv.D.nr - 1) * lv.D.nth * lv.D.nph, (double)N};
    double m[3];
    for (int d = 0; d < 3; ++d) m[d] = cnt[d] > 0 ? h->hscal[4 + d] / cnt[d] : 0.0;
    double top = 0.0;
    for (int d = 0; d < 3; ++d)
        if (can[d]) top = std::max(top, m[d]);
    for (int d = 0; d < 3; ++d) f[d] = (can[d] && m[d] >= kSemiRatio * top) ? 2 : 1;
    return MG_OK;
}

// Coarse tail over the deepest run of levels of at most `cells` cells, one
// thread-block cluster of `cluster` CTAs per shell; none when the run is
// shorter than two levels or clusters cannot be co-resident.
mg_status configure_tail(mg_handle* h, i64 cells, int cluster) {
    h->tail_level = 0;
    h->tail_smem = 0;
    if (cells <= 0 || h->opts.smoother != MG_SMOOTH_GS) return MG_OK;
    if (h->grid.cut && h->stencil == 19) return MG_OK;   // the tail's passes know no pole copy
    const int nl = (int)h->L.size();
    int t = nl;
    while (t - 1 >= 1 && h->L[t - 1].D.n() <= cells) --t;
    if (nl - t < 2 || nl - t > kMaxTail || tail_max_clusters(cluster, h->stencil, h->prec) <= 0) return MG_OK;
    h->tail_smem = 0;
    TailTask task{};
    task.nlev = nl - t;
    task.nu1 = h->opts.nu1;
    task.nu2 = h->opts.nu2;
    task.binv = h->binv;
    task.ncoarse = h->ncoarse;
    for (int l = t; l < nl; ++l) task.lev[l - t] = TailLevel{h->L[l].view(h->stencil), h->L[l].e, h->L[l].r};
    if (!h->tail_dev && !(h->tail_dev = (TailTask*)dalloc(h, sizeof(TailTask)))) return MG_ENOMEM;
    CK(cudaMemcpyAsync(h->tail_dev, &task, sizeof(TailTask), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->tail_host = task;
    h->tail_level = t;
    h->tail_cluster = cluster;
    // every level in the cluster's shared memory when it fits
    // (MG_TAIL_GLOBAL keeps the global-memory form)
    if (!std::getenv("MG_TAIL_GLOBAL")) {
        TailSmLayout lay;
        tail_sm_layout(task, cluster, h->prec == PREC64 ? 8 : 4, lay);
        if (lay.bytes <= kTailSmMaxBytes && tail_max_clusters(cluster, h->stencil, h->prec, lay.bytes) > 0)
            h->tail_smem = lay.bytes;
    }
    return MG_OK;
}

// ---- schedule tuner.  Candidates: blocks per SM of the level kernels (8, 16,
// 32), the coarse tail below 16384 cells, one-pass red-black tiles; chosen by
// coordinate descent on the device time of one outer iteration of this
// handle, and remembered per hierarchy shape for the rest of the process.
struct Schedule {
    int vb_cap = 16;
    i64 tail_cells = 0;
    int tail_cluster = 8;     // CTAs per tail cluster
    bool fused = false;       // one-pass sweeps
    int tile_cells = 2048;    // one-pass tiles: target cells per plane
    int tile_tj = 0;          // one-pass tiles: planes per chunk (0: per level)
    int tile_kmax = 256;      // one-pass tiles: widest tile in longitudes
    i64 tile_min = 1 << 20;   // one-pass tiles: smallest level (cells) swept in one pass
};

std::string shape_key(const mg_handle* h) {
    std::string k = std::to_string(h->prec) + "/" + std::to_string(h->stencil) + "/" +
                    std::to_string(h->opts.smoother) + "/" + std::to_string(h->opts.nu1) + "/" +
                    std::to_string(h->opts.nu2);
    for (const Level& lv : h->L)
        k += "|" + std::to_string(lv.D.nr) + "x" + std::to_string(lv.D.nth) + "x" + std::to_string(lv.D.nph);
    return k;
}

void set_tiles(mg_handle* h, bool on, int cells, int tj, int kmax, i64 min_cells) {
    h->one_pass = on;
    h->sweep_cells = cells;
    h->sweep_tj = tj;
    h->sweep_kmax = kmax;
    h->sweep_min_cells = min_cells;
}

// One-pass sweeps apply to Gauss-Seidel handles with a level a tile fits.
bool can_fuse(mg_handle* h, const Schedule& sc) {
    if (h->opts.smoother != MG_SMOOTH_GS) return false;
    const bool was = h->one_pass;
    const int c = h->sweep_cells, tj = h->sweep_tj, km = h->sweep_kmax;
    const i64 mc = h->sweep_min_cells;
    set_tiles(h, true, sc.tile_cells, sc.tile_tj, sc.tile_kmax, sc.tile_min);
    bool any = false;
    int tile[3];
    for (int l = 0; l < (int)h->L.size() && !any; ++l) any = sweep_tile_for(h, l, tile);
    set_tiles(h, was, c, tj, km, mc);
    return any;
}

mg_status apply_schedule(mg_handle* h, const Schedule& sc) {
    h->vb_cap = sc.vb_cap;
    set_tiles(h, sc.fused && can_fuse(h, sc), sc.tile_cells, sc.tile_tj, sc.tile_kmax, sc.tile_min);
    return configure_tail(h, sc.tail_cells, sc.tail_cluster);
}

mg_status time_schedule(mg_handle* h, const Schedule& sc, double* ms) {
    CKS(apply_schedule(h, sc));
    Plan* pl = nullptr;
    CKS(plan_create(&h, 1, &pl));
    // the least of three short runs: clock ramps and other tenants of the
    // GPU only ever slow a run down
    mg_status st = MG_OK;
    *ms = 0.0;
    for (int r = 0; r < 3 && st == MG_OK; ++r) {
        double t = 0.0;
        st = plan_time(pl, r == 0 ? 2 : 1, 4, &t);
        if (st == MG_OK && (r == 0 || t < *ms)) *ms = t;
    }
    plan_destroy(pl);
    return st;
}

// Schedules tuned in this process, per hierarchy shape.
std::mutex g_sched_mu;
std::unordered_map<std::string, std::pair<Schedule, double>> g_sched_cache;

// The cached schedule of the handle's shape, if any (source 2).
mg_status cached_schedule(mg_handle* h, bool* found) {
    std::pair<Schedule, double> hit;
    {
        std::lock_guard<std::mutex> lk(g_sched_mu);
        auto it = g_sched_cache.find(shape_key(h));
        *found = it != g_sched_cache.end();
        if (!*found) return MG_OK;
        hit = it->second;
    }
    CKS(apply_schedule(h, hit.first));
    h->sched_source = 2;
    h->sched_ms = hit.second;
    return MG_OK;
}

mg_status autotune(mg_handle* h) {
    bool found = false;
    CKS(cached_schedule(h, &found));
    if (found) return MG_OK;
    const std::string key = shape_key(h);
    // finite data for the timing runs (the iterates are discarded)
    const i64 N = h->L[0].D.n();
    CK(cudaMemsetAsync(h->x64, 0, sizeof(double) * N, h->stream));
    CK(cudaMemsetAsync(h->b64, 0, sizeof(double) * N, h->stream));
    if (h->prec != PREC64) {
        CK(cudaMemsetAsync(h->L[0].r, 0, sizeof(float) * N, h->stream));
        CK(cudaMemsetAsync(h->L[0].e, 0, sizeof(float) * N, h->stream));
    }
    Schedule best;
    double best_ms = 0.0;
    int tried = 1;
    CKS(time_schedule(h, best, &best_ms));
    auto consider = [&](const Schedule& sc) -> mg_status {
        double ms = 0.0, again = 0.0;
        CKS(time_schedule(h, sc, &ms));
        CKS(time_schedule(h, best, &again));   // the incumbent timed beside it
        best_ms = std::min(best_ms, again);
        ++tried;
        if (ms < 0.98 * best_ms) {   // a clear win only: timings carry noise
            best = sc;
            best_ms = ms;
        }
        return MG_OK;
    };
    for (int cap : {4, 8, 32}) {   // 4: one wave of the level kernels at four resident CTAs per SM
        Schedule sc = best;
        sc.vb_cap = cap;
        CKS(consider(sc));
    }
    if (h->opts.smoother == MG_SMOOTH_GS) {
        // the tail keeps its levels in shared memory, where 16 CTAs halve
        // each phase's work
        Schedule sc = best;
        sc.tail_cells = 16384;
        sc.tail_cluster = 16;
        CKS(consider(sc));
        if (best.tail_cells) {
            Schedule w = best;   // the other cluster size, then one level more
            w.tail_cluster = best.tail_cluster == 16 ? 8 : 16;
            CKS(consider(w));
            Schedule d = best;
            d.tail_cells = 65536;
            CKS(consider(d));
        }
    }
    {   // one-pass sweeps on the large levels: two plane areas, then the
        // chunk depth, the smallest level swept in one pass and the tile width
        // (the 7-point sweep of the FP32 / FP16 cycles takes whole rows and
        // sizes its tiles itself: only the chunk depth and the smallest level
        // are candidates there)
        const bool rb7 = h->stencil == 7 && h->prec != PREC64;
        for (int cells : {2048, 3072}) {
            if (rb7 && cells != 2048) continue;
            Schedule sc = best;
            sc.fused = true;
            sc.tile_cells = cells;
            if (can_fuse(h, sc)) CKS(consider(sc));
        }
        if (best.fused) {
            for (int tj : {8, 32}) {
                Schedule t = best;
                t.tile_tj = tj;
                CKS(consider(t));
            }
            for (i64 mc : {(i64)1 << 18, (i64)1 << 22}) {
                Schedule t = best;
                t.tile_min = mc;
                if (can_fuse(h, t)) CKS(consider(t));
            }
            if (h->stencil == 7 && !rb7) {
                Schedule t = best;
                t.tile_kmax = 128;
                CKS(consider(t));
            }
        }
    }
    CKS(apply_schedule(h, best));
    h->sched_source = 1;
    h->sched_candidates = tried;
    h->sched_ms = best_ms;
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched_cache[key] = {best, best_ms};
    return MG_OK;
}

mg_status setup_impl(const mg_grid_desc* g, const mg_opts* o, cudaStream_t stream, mg_handle* h) {
    h->grid = *g;
    h->opts = *o;
    if (const char* v = std::getenv("MG_TEST_FAIL_ALLOC_AFTER")) h->fail_alloc_after = std::atoll(v);
    h->stencil = stencil_of(g, o);
    h->axi = h->stencil == 19 && g->mapping != MG_MAP_TRIAXIAL && std::getenv("MG_FULL19") == nullptr;
    if (g->cut && h->stencil == 19 && !h->axi) {
        // the longitude cross terms would couple a cell with itself across the
        // pole on a two-longitude level, which the cell-wise diagonal ignores
        set_error("the shell cut with 19 points needs the axisymmetric operator (no longitude cross terms)");
        return MG_EINVAL;
    }
    h->prec = o->precision;
    h->user_stream = stream;
    h->use_graph = std::getenv("MG_NO_GRAPH") == nullptr;
    h->one_pass = std::getenv("MG_FUSED_RB") != nullptr;   // one-pass sweeps: forced
    if (h->one_pass) h->sweep_min_cells = 0;   // forced: every level a tile fits
    if (const char* v = std::getenv("MG_TILE")) {   // "cells,planes,kmax[,min_cells]"
        int c = 2048, tj = 0, km = 256;
        long long mc = h->sweep_min_cells;
        std::sscanf(v, "%d,%d,%d,%lld", &c, &tj, &km, &mc);
        h->sweep_cells = std::max(0, c);
        h->sweep_tj = std::max(0, tj);
        h->sweep_kmax = std::max(4, km);
        h->sweep_min_cells = std::max(0LL, mc);
        h->sweep_tile_env = true;
    }
    CK(cudaGetDevice(&h->device));
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    CK(cudaEventRecord(h->ev_in, h->user_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
    stream = h->stream;
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));

    // --- fine level: 1-D vertex tables (host), face metric (device)
    const int nr = g->nr, nth = g->nth, nph = g->nph;
    std::vector<double> rho(nr + 3), cth(nth + 3), sth(nth + 3), cph(nph + 3), sph(nph + 3);
    for (int j = -1; j <= nr + 1; ++j)
        rho[j + 1] = g->r_in + (g->r_out - g->r_in) * (stretch_unit(j, nr, g->stretch) + 0.5);
    for (int i = -1; i <= nth + 1; ++i) {
        const double th = g->th0 + (g->th1 - g->th0) * i / nth;
        cth[i + 1] = std::cos(th);
        sth[i + 1] = std::sin(th);
    }
    for (int k = -1; k <= nph + 1; ++k) {
        const int kw = ((k % nph) + nph) % nph;   // longitude planes are periodic
        const double ph = 2.0 * M_PI * kw / nph;
        cph[k + 1] = std::cos(ph);
        sph[k + 1] = std::sin(ph);
    }
    const size_t tb = sizeof(double) * (rho.size() + cth.size() * 2 + cph.size() * 2);
    double* tables = (double*)dalloc(h, tb);
    if (!tables) return MG_ENOMEM;
    double* p = tables;
    MetricTables T{};
    auto up = [&](const std::vector<double>& v, const double** dst) -> cudaError_t {
        *dst = p;
        cudaError_t e = cudaMemcpyAsync(p, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, stream);
        p += v.size();
        return e;
    };
    CK(up(rho, &T.rho));
    CK(up(cth, &T.cth));
    CK(up(sth, &T.sth));
    CK(up(cph, &T.cph));
    CK(up(sph, &T.sph));
    T.ax1 = g->mapping >= MG_MAP_OBLATE ? 1.0 - g->flattening : 1.0;
    T.ax2 = g->mapping == MG_MAP_TRIAXIAL ? 1.0 + g->e2 : 1.0;
    h->mtab = T;

    Level L0;
    L0.D = Dims{nr, nth, nph};
    L0.D.cut = g->cut;
    const i64 N = L0.D.n();
    for (int a = 0; a < 9; ++a)
        if (stored(h, a) && !(L0.g64[a] = (double*)dalloc(h, sizeof(double) * N))) return MG_ENOMEM;
    if (!(h->J64 = (double*)dalloc(h, sizeof(double) * N))) return MG_ENOMEM;
    if (!(h->b64 = (double*)dalloc(h, sizeof(double) * N))) return MG_ENOMEM;
    if (!(h->x64 = (double*)dalloc(h, sizeof(double) * N))) return MG_ENOMEM;
    if (!(h->part = (double*)dalloc(h, sizeof(double) * kRedBlocks))) return MG_ENOMEM;
    if (!(h->scal = (double*)dalloc(h, sizeof(double) * SC_COUNT))) return MG_ENOMEM;
    if (!(h->one_task = (BTask*)dalloc(h, sizeof(BTask)))) return MG_ENOMEM;
    if (!(h->one_map = dalloc(h, 128 * 5))) return MG_ENOMEM;
    if (o->metric == MG_METRIC_ANALYTIC) {
        // exact derivatives at the face centres: tables at half-index resolution
        std::vector<double> ar(2 * nr + 1), adr(2 * nr + 1), act(2 * nth + 1), ast(2 * nth + 1),
            acp(2 * nph + 1), asp(2 * nph + 1);
        for (int t = 0; t <= 2 * nr; ++t) {
            ar[t] = g->r_in + (g->r_out - g->r_in) * (stretch_unit(0.5 * t, nr, g->stretch) + 0.5);
            adr[t] = (g->r_out - g->r_in) * d_stretch_unit(0.5 * t, nr, g->stretch);
        }
        for (int t = 0; t <= 2 * nth; ++t) {
            const double th = g->th0 + (g->th1 - g->th0) * (0.5 * t) / nth;
            act[t] = std::cos(th);
            ast[t] = std::sin(th);
        }
        for (int t = 0; t <= 2 * nph; ++t) {
            const double ph = 2.0 * M_PI * (0.5 * t) / nph;
            acp[t] = std::cos(ph);
            asp[t] = std::sin(ph);
        }
        const size_t ab = sizeof(double) * (2 * ar.size() + 2 * act.size() + 2 * acp.size());
        double* at = (double*)dalloc(h, ab);
        if (!at) return MG_ENOMEM;
        p = at;
        AnalyticTables AT{};
        CK(up(ar, &AT.rho));
        CK(up(adr, &AT.drho));
        CK(up(act, &AT.cth));
        CK(up(ast, &AT.sth));
        CK(up(acp, &AT.cph));
        CK(up(asp, &AT.sph));
        AT.dth = (g->th1 - g->th0) / nth;
        AT.dph = 2.0 * M_PI / nph;
        AT.ax1 = T.ax1;
        AT.ax2 = T.ax2;
        CK(launch_face_metric_analytic(AT, L0.D, h->stencil, L0.g64, h->J64, stream));
        CK(cudaStreamSynchronize(stream));   // the host tables leave scope
    } else {
        CK(launch_face_metric(T, L0.D, h->stencil, L0.g64, h->J64, stream));
    }
    {
        const i64 rows = assembled_rows(L0.view(h->stencil));
        if (!(L0.a64 = (double*)dalloc(h, sizeof(double) * rows * N))) return MG_ENOMEM;
        CK(launch_assemble_rows(L0.view(h->stencil), L0.a64, stream));
    }
    CKS(device_sum(h, h->J64, nullptr, N, 0));
    CKS(read_scalars(h, 1));
    h->sumJ = h->hscal[0];
    h->L.push_back(L0);

    // --- hierarchy by face-metric aggregation
    const bool plane = o->smoother == MG_SMOOTH_PLANE;   // coarsens to one plane whatever the size
    while ((plane && h->plane_levels == 0) ||
           ((int)h->L.size() < o->max_levels && h->L.back().D.n() > o->coarse_max)) {
        int f[3];
        bool ok;
        CKS(plan_next(h, h->L.back(), f, &ok));
        if (!ok) break;
        Level& fine = h->L.back();
        fine.cz = f[0];
        fine.ce = f[1];
        fine.cx = f[2];
        Level c;
        c.D = Dims{fine.D.nr / fine.ce, fine.D.nth / fine.cz, fine.D.nph / fine.cx};
        c.D.cut = fine.D.cut;
        for (int a = 0; a < 9; ++a)
            if (stored(h, a) && !(c.g64[a] = (double*)dalloc(h, sizeof(double) * c.D.n())))
                return MG_ENOMEM;
        CK(launch_coarsen_faces(fine.view(h->stencil), c.D, c.g64, stream));
        h->L.push_back(c);
    }
    if (plane && h->plane_levels == 0) h->plane_levels = (int)h->L.size() - 1;   // every level above the coarsest
    for (const Level& lv : h->L)
        if (!fastdiv_ok(lv.D)) {
            set_error("index divisor self-check failed");
            return MG_EINVAL;
        }
    CKS(conversion_check(h));
    Level& last = h->L.back();
    last.cz = last.ce = last.cx = 0;
    h->ncoarse = (int)last.D.n();
    if (h->ncoarse > kMaxCoarse) {
        set_error("coarsest level has " + std::to_string(h->ncoarse) + " cells (> " +
                  std::to_string(kMaxCoarse) + "); use dimensions with more factors of two");
        return MG_EINVAL;
    }

    // --- coefficient copies of the cycle precision
    for (Level& lv : h->L) {
        const i64 n = lv.D.n();
        for (int a = 0; a < 9; ++a) {
            if (!stored(h, a)) continue;
            if (h->prec == PREC32) {
                if (!(lv.g32[a] = (float*)dalloc(h, sizeof(float) * n))) return MG_ENOMEM;
                CK(launch_cast32(lv.g64[a], lv.g32[a], n, stream));
            } else if (h->prec == PREC16) {
                CK(launch_absmax(lv.g64[a], n, h->part, stream));
                CK(launch_finalize(h->part, red_blocks(n), 1, h->scal + 7, stream));
                CKS(read_scalars(h, 8));
                const double mx = h->hscal[7];
                float s = 1.0f;
                if (mx > 0) s = std::ldexp(1.0f, (int)std::ceil(std::log2(mx)) - 14);
                lv.s16[a] = s;
                if (!(lv.g16[a] = (__half*)dalloc(h, sizeof(__half) * n))) return MG_ENOMEM;
                CK(launch_cast16(lv.g64[a], lv.g16[a], n, 1.0f / s, stream));
            }
        }
    }

    // --- work arrays: level 0 holds the FP32 correction cycle's e, r; every
    // level has a scratch of 8 bytes per cell; coarse levels hold e, r wide
    // enough for either precision.
    for (size_t l = 0; l < h->L.size(); ++l) {
        Level& lv = h->L[l];
        const i64 n = lv.D.n();
        if (!(lv.t = dalloc(h, sizeof(double) * n))) return MG_ENOMEM;
        if (lv.D.cut && h->stencil == 19 && !(lv.poles = dalloc(h, sizeof(double) * 2 * lv.D.nr * lv.D.nph)))
            return MG_ENOMEM;
        if (l == 0) {
            if (h->prec != PREC64) {
                if (!(lv.e = dalloc(h, sizeof(float) * n))) return MG_ENOMEM;
                if (!(lv.r = dalloc(h, sizeof(float) * n))) return MG_ENOMEM;
            }
        } else {
            if (!(lv.e = dalloc(h, sizeof(double) * n))) return MG_ENOMEM;
            if (!(lv.r = dalloc(h, sizeof(double) * n))) return MG_ENOMEM;
        }
    }

    if (radial_lines(o->smoother)) CKS(ensure_line_factors(h, h->prec));
    if (longitude_lines(o->smoother)) CKS(ensure_xline_factors(h, h->prec));
    if (o->smoother == MG_SMOOTH_PLANE) CKS(build_planes(h));

    // --- coarsest level: dense operator -> bordered inverse (device, FP64)
    const int nc = h->ncoarse;
    if (!(h->binv = (double*)dalloc(h, sizeof(double) * nc * nc))) return MG_ENOMEM;
    {
        const size_t m = (size_t)nc + 1;
        TmpDev tA(sizeof(double) * nc * nc, stream, h->device);
        TmpDev tw(sizeof(double) * (m * m + kGjScratch) + sizeof(int) * (2 * m + 1), stream, h->device);
        if (!tA.p || !tw.p) return MG_ENOMEM;
        double* dA = (double*)tA.p;
        double* work = (double*)tw.p;
        double* col = work + m * m;
        int* piv = (int*)(col + kGjScratch);
        int* perm = piv + m;
        int* bad = perm + m;
        CK(cudaMemsetAsync(bad, 0, sizeof(int), stream));
        CK(launch_dense_operator(last.view(h->stencil), dA, stream));
        CK(launch_bordered_inverse(dA, nc, work, col, piv, perm, bad, h->binv, stream));
        int hbad = 0;
        CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        if (hbad) {
            set_error(hbad == 2 ? "coarsest inverse: a grid barrier gave up waiting"
                                : "coarsest bordered operator is singular");
            return MG_EINVAL;
        }
    }

    CK(cudaStreamSynchronize(stream));
    CK(cudaGetLastError());

    // --- launch schedule: forced by the environment, tuned, or the default
    const bool env_sched =
        std::getenv("MG_TAIL") || std::getenv("MG_FUSED_RB") || std::getenv("MG_VB_CAP") || std::getenv("MG_TILE");
    if (env_sched) {
        h->sched_source = 3;
        if (const char* v = std::getenv("MG_VB_CAP")) h->vb_cap = std::max(1, std::min(64, std::atoi(v)));
        if (std::getenv("MG_TAIL")) {
            i64 cells = kTailCells;
            int cluster = 8;
            if (const char* v = std::getenv("MG_TAIL_CELLS")) cells = std::atoll(v);
            if (const char* v = std::getenv("MG_TAIL_CLUSTER"))
                cluster = std::max(1, std::min(kTailMaxCluster, std::atoi(v)));
            CKS(configure_tail(h, cells, cluster));
        }
    } else if (o->autotune == 1) {
        CKS(autotune(h));
    } else if (o->autotune == 2) {
        bool found = false;
        CKS(cached_schedule(h, &found));
    }
    return MG_OK;
}

size_t value_bytes(int prec) { return prec == PREC64 ? 8 : 4; }
size_t coef_bytes(int prec) { return prec == PREC64 ? 8 : (prec == PREC32 ? 4 : 2); }

bool has_prec(const mg_handle* h, int prec) {
    if (prec == PREC64) return true;
    return prec == h->prec;
}

}  // namespace

namespace mgs {

void* handle_alloc(mg_handle* h, size_t bytes) { return dalloc(h, bytes); }

void destroy_handle_after(mg_handle* h, cudaStream_t last) {
    if (!h) return;
    if (last && last != h->stream) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(e, last);
            cudaStreamWaitEvent(h->stream, e, 0);
            cudaEventDestroy(e);
        } else {
            cudaGetLastError();
            cudaStreamSynchronize(last);
        }
    }
    free_handle(h);
}

}  // namespace mgs

namespace mgs {

static cudaEvent_t prof_event(mg_handle* h) {
    if (!h->prof_pool.empty()) {
        cudaEvent_t e = h->prof_pool.back();
        h->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(mg_handle* h, int slot) {
    if (!h->prof_on) return;
    cudaEvent_t e = prof_event(h);
    cudaEventRecord(e, h->stream);
    h->prof_open[slot] = e;
}

void prof_end(mg_handle* h, int slot, int nlaunch) {
    if (!h->prof_on || !h->prof_open[slot]) return;
    cudaEvent_t e = prof_event(h);
    cudaEventRecord(e, h->stream);
    h->prof_pending.push_back({slot, h->prof_open[slot], e, nlaunch});
    h->prof_open[slot] = nullptr;
}

void prof_collect(mg_handle* h) {
    for (auto& p : h->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            h->prof_ms[p.slot] += ms;
            h->prof_n[p.slot] += p.n;
        }
        cudaGetLastError();
        h->prof_pool.push_back(p.a);
        h->prof_pool.push_back(p.b);
    }
    h->prof_pending.clear();
}

void plane_sweep_steps(const mg_handle* h, int level, void* x, const void* b, std::vector<PlaneStep>& out) {
    const Level& lv = h->L[level];
    const std::vector<PlaneLevel>& P = lv.planes;
    const int M = (int)P.size() - 1;
    auto vb = [](i64 work) {
        i64 n = (work + 255) / 256;
        return (int)std::max<i64>(1, std::min<i64>(n, 152 * 16));
    };
    auto two_d = [&](int m) {   // a task over 2-D level m
        BTask t{};
        t.v.D = P[m].D;
        t.v.stencil = 7;
        for (int o = 0; o < 9; ++o) {
            t.v.c64.g[o] = P[m].c64[o];
            t.v.c32.g[o] = P[m].c32[o];
        }
        t.x = P[m].e;
        t.b = P[m].r;
        t.z = P[m].fac;
        t.y = P[m].w;
        return t;
    };
    auto relax = [&](int m, int p, int q) {
        const Dims& D = P[m].D;
        const i64 lines = (i64)((D.nth + 1 - p) >> 1) * ((D.nr + 1 - q) >> 1);
        if (lines > 0) out.push_back(PlaneStep{BOP_PRELAX, p + 2 * q, two_d(m), vb(32 * lines)});   // a warp per line
    };
    for (int p = 0; p < 2; ++p) {
        if (plane_cells(lv.D, p) == 0) continue;
        {   // the 3-D residual on the planes of parity p, e of 2-D level 0 zeroed
            BTask t{};
            t.v = lv.view(h->stencil);
            t.x = x;
            t.b = b;
            t.y = P[0].r;
            t.z = P[0].e;
            out.push_back(PlaneStep{BOP_PRES, p, t, vb(plane_cells(lv.D, p))});
        }
        for (int c = 0; c < h->opts.plane_cycles; ++c) {
            for (int m = 0; m < M; ++m) {
                relax(m, p, 0);
                relax(m, p, 1);
                BTask t = two_d(m);
                t.Dc = P[m + 1].D;
                t.y = P[m + 1].r;
                t.z = P[m + 1].e;
                out.push_back(PlaneStep{BOP_PRESTRICT, p, t, vb(plane_cells(P[m + 1].D, p))});
            }
            relax(M, p, 0);   // one row from zero: the exact solve
            relax(M, p, 1);   // (no rows of odd index on one row)
            for (int m = M - 1; m >= 0; --m) {
                BTask t = two_d(m);
                t.Dc = P[m + 1].D;
                t.b = P[m + 1].e;
                out.push_back(PlaneStep{BOP_PPROLONG, p, t, vb(plane_cells(P[m].D, p))});
                relax(m, p, 0);
                relax(m, p, 1);
            }
        }
        BTask t{};
        t.v.D = lv.D;
        t.x = x;
        t.b = P[0].e;
        out.push_back(PlaneStep{BOP_PUPDATE, p, t, vb(plane_cells(lv.D, p))});
    }
}

// The 7-point sweep of the FP32 and FP16-coefficient cycles: whole rows, one
// thread per quad of TI + 2 rows.  The rows and chunk depth minimise the
// estimate ceil(tiles / 152) (TJ + 3) (TI + 3): one wave of tiles on the SMs,
// a tile takes TJ + 2 steps and a step costs about its rows plus a fixed
// part.  MG_TILE fixes the rows (its cells / nph, at least one; cells 0 or
// rows that do not fit: automatic), a schedule's chunk depth fixes TJ.
bool rb7_tile_for(const mg_handle* h, const Dims& D, int tile[3]) {
    const int NQ = D.nph / 4;
    if (D.nph % 4 != 0 || NQ < 1) return false;
    const int ti_max = std::min(D.nth, kRB7MaxThreads / NQ - 2);
    if (ti_max < 1) return false;
    int lo = 1, hi = ti_max;
    if (h->sweep_tile_env && h->sweep_cells > 0) lo = hi = std::max(1, std::min(ti_max, h->sweep_cells / D.nph));
    bool found = false;
    double best = 0.0;
    for (int pass = 0; pass < 2 && !found; ++pass, lo = 1, hi = ti_max)   // forced rows that do not fit: automatic
    for (int ti = lo; ti <= hi; ++ti)
        for (int tj = 1; tj <= D.nr; ++tj) {
            if (h->sweep_tj > 0 && tj != std::min(h->sweep_tj, D.nr)) continue;
            const int t3[3] = {ti, tj, D.nph};
            if (!sweep_tile_ok(D, 7, h->prec, t3)) continue;
            const double cost = std::ceil(sweep_units(D, t3) / 152.0) * (tj + 3) * (ti + 3);
            if (!found || cost < best) {
                found = true;
                best = cost;
                tile[0] = ti, tile[1] = tj, tile[2] = D.nph;
            }
        }
    return found;
}

bool sweep_tile_for(const mg_handle* h, int level, int tile[3]) {
    if (!h->one_pass || h->opts.smoother != MG_SMOOTH_GS || level < 0 || level >= (int)h->L.size()) return false;
    const Dims& D = h->L[level].D;
    if (D.n() < h->sweep_min_cells) return false;
    if (h->stencil == 7 && h->prec != PREC64) return !D.cut && rb7_tile_for(h, D, tile);
    // longitudes: whole rows up to the widest tile, else the largest
    // power-of-two divisor of nph up to 128
    // (19 points: at most 128, the buffers hold four halo rows either side)
    const int kmax = h->stencil == 19 ? std::min(h->sweep_kmax, 128) : h->sweep_kmax;
    int tk = D.nph;
    if (tk > kmax) {
        tk = 0;
        for (int c = 128; c >= 8 && !tk; c >>= 1)
            if (D.nph % c == 0 && c <= kmax) tk = c;
        if (!tk) return false;
    }
    // rows: the plane area, at least four rows (the halo is 2 or 4 rows)
    const int ti = std::max(4, std::min(D.nth, h->sweep_cells / tk));
    int tj = h->sweep_tj;
    if (tj <= 0) {   // deep chunks, while the level still has two tiles per SM
        tj = 32;
        for (;;) {
            const int t3[3] = {ti, tj, tk};
            if (tj <= 4 || sweep_units(D, t3) >= 2 * 152) break;
            tj >>= 1;
        }
    }
    tile[0] = ti;
    tile[1] = tj;
    tile[2] = tk;
    return sweep_tile_ok(D, h->stencil, h->prec, tile);
}

mg_status smooth(mg_handle* h, int level, int prec, void* x, const void* b, int sweeps, int kind) {
    Level& lv = h->L[level];
    const LevelView v = lv.view(h->stencil);
    if (sweeps == 0) return MG_OK;
    if (level == 0) prof_begin(h, MG_PROF_SMOOTH0);
    int n = 0;
    int tile[3];
    if (kind == MG_SMOOTH_GS && prec == h->prec && sweep_tile_for(h, level, tile)) {
        // one-pass sweeps ping-pong between x and the level's scratch
        void* bufs[2] = {x, lv.t};
        for (int s = 0; s < sweeps; ++s, ++n) {
            BTask t{};
            t.v = v;
            t.x = bufs[s & 1];
            t.y = bufs[(s + 1) & 1];
            t.b = b;
            t.block0 = 0;
            t.nblocks = sweep_units(lv.D, tile);
            for (int a = 0; a < 3; ++a) t.tile[a] = tile[a];
            t.tmap = h->one_map;
            alignas(64) unsigned char map[128 * 5];
            CK(encode_sweep_maps(map, t, h->stencil, prec));
            // pageable sources: both copies are staged before the calls return
            CK(cudaMemcpyAsync(h->one_map, map, 128 * (size_t)sweep_map_count(h->stencil, prec),
                               cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(h->one_task, &t, sizeof(BTask), cudaMemcpyHostToDevice, h->stream));
            CK(launch_sweep(h->one_task, 1, t.nblocks, nullptr, h->stencil, h->axi, prec,
                            sweep_smem_bytes(h->stencil, prec, lv.D, tile),
                            sweep_threads(h->stencil, prec, lv.D, tile), h->stream));
        }
        if (sweeps & 1) {
            CK(cudaMemcpyAsync(x, lv.t, value_bytes(prec) * lv.D.n(), cudaMemcpyDeviceToDevice, h->stream));
        }
    } else if (kind == MG_SMOOTH_PLANE) {
        std::vector<PlaneStep> st;
        plane_sweep_steps(h, level, x, b, st);
        if (st.size() > h->plane_tasks_cap) {
            if (!(h->plane_tasks = (BTask*)dalloc(h, sizeof(BTask) * st.size()))) return MG_ENOMEM;
            h->plane_tasks_cap = st.size();
        }
        std::vector<BTask> tasks(st.size());
        for (size_t i = 0; i < st.size(); ++i) {
            tasks[i] = st[i].t;
            tasks[i].block0 = 0;
            tasks[i].nblocks = st[i].nblocks;
        }
        CK(cudaMemcpyAsync(h->plane_tasks, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice,
                           h->stream));
        for (int sw = 0; sw < sweeps; ++sw)
            for (size_t i = 0; i < st.size(); ++i, ++n)
                CK(launch_batch(h->plane_tasks + i, 1, st[i].nblocks, nullptr, st[i].op, st[i].colour, 7, prec,
                                h->stream));
    } else if (kind == MG_SMOOTH_GS) {
        const int ncol = h->stencil == 7 ? 2 : 4;
        const bool poles = h->stencil == 19 && lv.D.cut;   // cells of a colour couple across the pole
        for (int s = 0; s < sweeps; ++s)
            for (int c = 0; c < ncol; ++c, ++n) {
                if (poles) {
                    CK(launch_poles(v, prec, x, lv.poles, h->stream));
                    ++n;
                }
                CK(launch_gs_colour(v, prec, x, b, c, h->stream, poles ? lv.poles : nullptr));
            }
    } else if (kind == MG_SMOOTH_LINE || kind == MG_SMOOTH_XLINE || kind == MG_SMOOTH_ALT) {
        // radial lines, longitude lines, or both in that order per sweep; a
        // level narrower than four longitudes takes a point sweep for the
        // longitude lines
        const int ncol = h->stencil == 7 ? 2 : 4;
        const int cls = prec == PREC64 ? 0 : 1;
        if (radial_lines(kind)) CKS(ensure_line_factors(h, prec));
        if (longitude_lines(kind)) CKS(ensure_xline_factors(h, prec));
        for (int s = 0; s < sweeps; ++s) {
            if (radial_lines(kind))
                for (int c = 0; c < ncol; ++c, ++n) CK(launch_line_colour(v, prec, x, b, lv.lf[cls], c, h->stream));
            if (!longitude_lines(kind)) continue;
            if (lv.D.nph < 4) {
                for (int c = 0; c < ncol; ++c, ++n) CK(launch_gs_colour(v, prec, x, b, c, h->stream));
                continue;
            }
            for (int c = 0; c < ncol; ++c, ++n)
                CK(launch_xline_colour(v, prec, x, b, lv.xf[cls], lv.t, c, h->stream));
        }
    } else {
        const size_t bytes = value_bytes(prec) * lv.D.n();
        for (int s = 0; s < sweeps; ++s, ++n) {
            CK(launch_jacobi(v, prec, x, lv.t, b, h->stream));
            CK(cudaMemcpyAsync(x, lv.t, bytes, cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    if (level == 0) prof_end(h, MG_PROF_SMOOTH0, n);
    h->launches += n;
    return MG_OK;
}

// V(nu1, nu2) on A_0 x0 = b0; coarse levels use the handle's e / r arrays.
mg_status vcycle(mg_handle* h, int prec, void* x0, const void* b0) {
    const int nl = (int)h->L.size();
    (void)0;
    h->launches += 1;
    if (nl == 1) {
        CK(launch_coarse_solve(h->binv, h->ncoarse, prec, b0, x0, h->stream));
        return MG_OK;
    }
    // levels [0, top) run launch by launch; level top starts the tail, or is the coarsest
    const int top = h->tail_level > 0 ? h->tail_level : nl - 1;
    for (int l = 0; l < top; ++l) {
        void* x = l == 0 ? x0 : h->L[l].e;
        const void* b = l == 0 ? b0 : h->L[l].r;
        CKS(smooth(h, l, prec, x, b, h->opts.nu1, level_smoother(h, l)));
        if (l == 0) prof_begin(h, MG_PROF_RESTRICT0);
        CK(launch_restrict_residual(h->L[l].view(h->stencil), h->L[l + 1].D, prec, x, b, h->L[l + 1].r,
                                    h->L[l + 1].e, h->stream));
        if (l == 0) prof_end(h, MG_PROF_RESTRICT0, 1);
        h->launches += 1;
    }
    if (h->tail_level > 0) {
        prof_begin(h, MG_PROF_TAIL);
        CK(launch_tail(h->tail_dev, 1, h->tail_cluster, h->stencil, prec, h->stream, nullptr, h->tail_smem));
        prof_end(h, MG_PROF_TAIL, 1);
    } else {
        CK(launch_coarse_solve(h->binv, h->ncoarse, prec, h->L[nl - 1].r, h->L[nl - 1].e, h->stream));
    }
    for (int l = top - 1; l >= 0; --l) {
        void* x = l == 0 ? x0 : h->L[l].e;
        const void* b = l == 0 ? b0 : h->L[l].r;
        if (l == 0) prof_begin(h, MG_PROF_PROLONG0);
        CK(launch_prolong_add(h->L[l].view(h->stencil), h->L[l + 1].D, prec, h->L[l + 1].e, x, h->stream));
        if (l == 0) prof_end(h, MG_PROF_PROLONG0, 1);
        h->launches += 1;
        CKS(smooth(h, l, prec, x, b, h->opts.nu2, level_smoother(h, l)));
    }
    return MG_OK;
}

// Algorithmic HBM bytes of one outer iteration: each array a kernel touches
// is counted once per launch (neighbour re-reads are assumed to hit cache).
double model_bytes_per_iteration(const mg_handle* h) {
    const int nc = h->stencil == 19 ? 9 : 3;
    const double vb = (double)value_bytes(h->prec), cb = (double)coef_bytes(h->prec);
    const int ncol = h->opts.smoother != MG_SMOOTH_JACOBI ? (h->stencil == 7 ? 2 : 4) : 1;
    // line factors (radial 3, longitude 4 values per cell; the longitude pass
    // also writes and reads its scratch)
    const double fac_bytes = (radial_lines(h->opts.smoother) ? 3 * vb : 0.0) +
                             (longitude_lines(h->opts.smoother) ? 6 * vb : 0.0);
    double total = 0.0;
    for (size_t l = 0; l < h->L.size(); ++l) {
        const double n = (double)h->L[l].D.n();
        if (l + 1 == h->L.size()) {
            total += 8.0 * n * n + 2.0 * vb * n;
            break;
        }
        const double nc_cells = (double)h->L[l + 1].D.n();
        const double sweep = n * (2 * vb + vb + nc * cb + fac_bytes) * ncol;   // each colour pass reads the arrays
        total += (h->opts.nu1 + h->opts.nu2) * sweep;
        total += n * (vb + vb + nc * cb) + 2.0 * nc_cells * vb;     // residual + restriction
        total += n * 2 * vb + nc_cells * vb;                         // prolongation + correction
    }
    const double N = (double)h->L[0].D.n();
    if (h->prec == PREC64) total += N * (8 + 8 + nc * 8);           // outer residual
    else total += N * (8 + 8 + nc * 8 + 4) + N * (4 + 16) + N * 4;  // residual, update, zero e
    return total;
}

// Orders a call's work after the caller's stream and the caller's stream
// after the call's work (the handle computes on a private stream).
struct StreamJoin {
    mg_handle* h;
    explicit StreamJoin(mg_handle* hh) : h(hh) {
        cudaEventRecord(h->ev_in, h->user_stream);
        cudaStreamWaitEvent(h->stream, h->ev_in, 0);
    }
    ~StreamJoin() {
        cudaEventRecord(h->ev_out, h->stream);
        cudaStreamWaitEvent(h->user_stream, h->ev_out, 0);
    }
};

}  // namespace mgs

// ============================================================ C ABI
extern "C" {

const char* mg_version(void) { return "mgshell 0.1 (sm_103a)"; }

const char* mg_last_error(void) { return g_err.c_str(); }

mg_status mg_default_opts(mg_opts* o) {
    if (!o) return MG_EINVAL;
    o->precision = MG_PREC_FP32_IR;
    o->smoother = MG_SMOOTH_GS;
    o->nu1 = 2;
    o->nu2 = 2;
    o->max_levels = 16;
    o->coarsen = MG_COARSEN_SEMI;
    o->coarse_max = 512;
    o->max_iters = 100;
    o->stencil = 0;
    o->autotune = 1;
    o->metric = MG_METRIC_DISCRETE;
    o->plane_cycles = 1;
    return MG_OK;
}

size_t mg_device_bytes_in_use(int device) {
    size_t used = 0;
    cudaMemPool_t p = lib_pool(device);
    unsigned long long v = 0;   // the attribute is a 64-bit count
    if (p && cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &v) == cudaSuccess) used = (size_t)v;
    else cudaGetLastError();
    return used;
}

mg_status mg_get_schedule(const mg_handle* h, mg_schedule* out) {
    if (!h || !out) return MG_EINVAL;
    out->blocks_per_sm = h->vb_cap;
    out->tail_level = h->tail_level;
    out->tail_cluster = h->tail_cluster;
    out->tail_smem_bytes = h->tail_level > 0 ? (int)h->tail_smem : 0;
    out->one_pass_tiles = h->one_pass ? 1 : 0;
    out->tile_cells = h->sweep_cells;
    out->tile_planes = h->sweep_tj;
    out->tile_kmax = h->sweep_kmax;
    out->tile_min_cells = h->sweep_min_cells;
    int tile[3] = {0, 0, 0};
    if (!sweep_tile_for(h, 0, tile)) tile[0] = tile[1] = tile[2] = 0;
    for (int a = 0; a < 3; ++a) out->tile0[a] = tile[a];
    out->source = h->sched_source;
    out->candidates = h->sched_candidates;
    out->ms_per_iteration = h->sched_ms;
    return MG_OK;
}

size_t mg_footprint_bytes(const mg_grid_desc* g, const mg_opts* o) {
    mg_opts d;
    if (!o) {
        mg_default_opts(&d);
        o = &d;
    }
    if (!check_grid(g).empty() || !check_opts(o).empty() || !check_pair(g, o).empty()) return 0;
    const double n = (double)g->nr * g->nth * g->nph;
    const int nc = stencil_of(g, o) == 19 ? 9 : 3;
    const double cb = (double)coef_bytes(o->precision);
    // fine level + coarse levels (at most the fine size again under semi-coarsening)
    const double fine = n * (nc * (8 + (o->precision == PREC64 ? 0 : cb)) + 8 /*t*/ +
                             (o->precision == PREC64 ? 0 : 8) /*e,r*/);
    const double coarse = n * (nc * (8 + (o->precision == PREC64 ? 0 : cb)) + 24);
    const double rows = n * 8 * (nc == 9 ? 19 : 1);   // assembled fine rows
    const double fixed = n * 16 /*J, b*/ + rows + 8.0 * kMaxCoarse * kMaxCoarse + (1 << 20);
    const double lines = (radial_lines(o->smoother) ? 2 * n * 3 * value_bytes(o->precision) : 0.0) +
                         (longitude_lines(o->smoother) ? 2 * n * 4 * value_bytes(o->precision) : 0.0);
    return (size_t)(fine + coarse + fixed + lines);
}

mg_status mg_setup(const mg_grid_desc* g, const mg_opts* o, void* stream, mg_handle** out) {
    if (!out) return MG_EINVAL;
    *out = nullptr;
    cudaGetLastError();   // an earlier failed call of this thread is not set-up's to report
    mg_opts d;
    if (!o) {
        mg_default_opts(&d);
        o = &d;
    }
    std::string why = check_grid(g);
    if (why.empty()) why = check_opts(o);
    if (why.empty()) why = check_pair(g, o);
    if (!why.empty()) {
        set_error(why);
        return MG_EINVAL;
    }
    mg_handle* h = new (std::nothrow) mg_handle();
    if (!h) return MG_ENOMEM;
    static std::atomic<unsigned long long> next_serial{1};
    h->serial = next_serial++;
    mg_status st;
    try {
        st = setup_impl(g, o, (cudaStream_t)stream, h);
    } catch (const std::bad_alloc&) {
        st = MG_ENOMEM;
    } catch (...) {
        st = MG_EINVAL;
    }
    if (st != MG_OK) {
        if (st == MG_ENOMEM) set_error("out of memory during setup");
        cudaStreamSynchronize((cudaStream_t)stream);
        free_handle(h);
        return st;
    }
    *out = h;
    return MG_OK;
}

void mg_destroy(mg_handle* h) {
    if (!h) return;
    // the handle's buffers may have been used on other streams (batches, the
    // caller's stream): wait for the device, then free
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_handle(h);
}

mg_status mg_set_stream(mg_handle* h, void* stream) {
    if (!h) return MG_EINVAL;
    h->user_stream = (cudaStream_t)stream;
    return MG_OK;
}

mg_status mg_get_level_info(mg_handle* h, int level, mg_level_info* info) {
    if (!h || !info || level < 0 || level >= (int)h->L.size()) return MG_EINVAL;
    const Level& lv = h->L[level];
    info->nr = lv.D.nr;
    info->nth = lv.D.nth;
    info->nph = lv.D.nph;
    info->cz = lv.cz;
    info->ce = lv.ce;
    info->cx = lv.cx;
    info->stencil = h->stencil;
    info->levels = (int)h->L.size();
    return MG_OK;
}

mg_status mg_get_metric(mg_handle* h, int level, int component, double* dst) {
    if (!h || !dst || level < 0 || level >= (int)h->L.size() || component < 0 || component > 9)
        return MG_EINVAL;
    const Level& lv = h->L[level];
    const size_t bytes = sizeof(double) * lv.D.n();
    StreamJoin join(h);
    if (component == 9) {
        if (level != 0) return MG_EINVAL;
        CK(cudaMemcpyAsync(dst, h->J64, bytes, cudaMemcpyDeviceToDevice, h->stream));
    } else if (lv.g64[component]) {
        CK(cudaMemcpyAsync(dst, lv.g64[component], bytes, cudaMemcpyDeviceToDevice, h->stream));
    } else {
        CK(cudaMemsetAsync(dst, 0, bytes, h->stream));   // 7-point grids keep no cross terms
    }
    return MG_OK;
}

#define LEVEL_CHECK(h, level, prec)                                                           \
    do {                                                                                      \
        if (!(h) || (level) < 0 || (level) >= (int)(h)->L.size()) return MG_EINVAL;          \
        if ((prec) < 0 || (prec) > 2 || !has_prec((h), (prec))) {                             \
            set_error("the handle holds no coefficient copy of that precision");              \
            return MG_EINVAL;                                                                 \
        }                                                                                     \
    } while (0)

mg_status mg_apply(mg_handle* h, int level, int prec, const void* x, void* y) {
    LEVEL_CHECK(h, level, prec);
    if (!x || !y) return MG_EINVAL;
    StreamJoin join(h);
    CK(launch_apply(h->L[level].view(h->stencil), prec, x, y, h->stream));
    return MG_OK;
}

mg_status mg_smooth(mg_handle* h, int level, int prec, void* x, const void* b, int sweeps, int kind) {
    LEVEL_CHECK(h, level, prec);
    if (!x || !b || sweeps < 0 || kind < 0 || kind > 5) return MG_EINVAL;
    if (kind == MG_SMOOTH_PLANE && (h->opts.smoother != MG_SMOOTH_PLANE || prec != h->prec ||
                                    level >= h->plane_levels)) {
        set_error("plane relaxation: a handle set up with the PLANE smoother, its own precision, a level relaxed by planes");
        return MG_EINVAL;
    }
    StreamJoin join(h);
    return smooth(h, level, prec, x, b, sweeps, kind);
}

mg_status mg_restrict_residual(mg_handle* h, int level, int prec, const void* x, const void* b, void* rc) {
    LEVEL_CHECK(h, level, prec);
    if (!x || !b || !rc || level + 1 >= (int)h->L.size()) return MG_EINVAL;
    StreamJoin join(h);
    CK(launch_restrict_residual(h->L[level].view(h->stencil), h->L[level + 1].D, prec, x, b, rc, nullptr,
                                h->stream));
    return MG_OK;
}

mg_status mg_prolong_add(mg_handle* h, int level, int prec, const void* ec, void* x) {
    LEVEL_CHECK(h, level, prec);
    if (!x || !ec || level + 1 >= (int)h->L.size()) return MG_EINVAL;
    StreamJoin join(h);
    CK(launch_prolong_add(h->L[level].view(h->stencil), h->L[level + 1].D, prec, ec, x, h->stream));
    return MG_OK;
}

mg_status mg_coarse_solve(mg_handle* h, int prec, const void* r, void* e) {
    if (!h || !r || !e || prec < 0 || prec > 2) return MG_EINVAL;
    StreamJoin join(h);
    CK(launch_coarse_solve(h->binv, h->ncoarse, prec, r, e, h->stream));
    return MG_OK;
}

mg_status mg_vcycle(mg_handle* h, int prec, void* x, const void* b) {
    LEVEL_CHECK(h, 0, prec);
    if (!x || !b) return MG_EINVAL;
    StreamJoin join(h);
    return vcycle(h, prec, x, b);
}

mg_status mg_solve(mg_handle* h, const double* f, double* x, double tol, mg_report* rep) {
    if (!h || !f || !x || !(tol >= 0) || !std::isfinite(tol)) return MG_EINVAL;
    StreamJoin join(h);
    if (!h->solo) CKS(plan_create(&h, 1, &h->solo));
    return plan_solve(h->solo, &f, &x, &tol, rep);
}

mg_status mg_solve_host(mg_handle* h, const double* f_host, double* x_host, double tol, mg_report* rep) {
    if (!h || !f_host || !x_host) return MG_EINVAL;
    const i64 N = h->L[0].D.n();
    const size_t bytes = sizeof(double) * N;
    if (!h->df) {
        if (!(h->df = (double*)dalloc(h, bytes)) || !(h->dx = (double*)dalloc(h, bytes))) return MG_ENOMEM;
        CK(cudaMallocHost((void**)&h->hf, bytes));
        CK(cudaMallocHost((void**)&h->hx, bytes));
    }
    // caller memory that is already page-locked is copied directly
    cudaPointerAttributes af{}, ax{};
    const bool pinned_f = cudaPointerGetAttributes(&af, f_host) == cudaSuccess && af.type == cudaMemoryTypeHost;
    const bool pinned_x = cudaPointerGetAttributes(&ax, x_host) == cudaSuccess && ax.type == cudaMemoryTypeHost;
    cudaGetLastError();
    const double* srcf = f_host;
    if (!pinned_f) {
        std::memcpy(h->hf, f_host, bytes);
        srcf = h->hf;
    }
    double* xs = pinned_x ? x_host : h->hx;
    if (!pinned_x) std::memcpy(h->hx, x_host, bytes);
    CK(cudaMemcpyAsync(h->df, srcf, bytes, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->dx, xs, bytes, cudaMemcpyHostToDevice, h->stream));
    const mg_status st = mg_solve(h, h->df, h->dx, tol, rep);
    if (st != MG_OK && st != MG_ENOCONV) return st;
    CK(cudaMemcpyAsync(xs, h->dx, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (!pinned_x) std::memcpy(x_host, h->hx, bytes);
    return st;
}

mg_status mg_profile_enable(mg_handle* h, int on) {
    if (!h || on < 0 || on > 2) return MG_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    prof_collect(h);
    h->prof_on = on != 0;
    h->prof_events = on == 2;
    for (int s = 0; s < MG_PROF_SLOTS; ++s) {
        h->prof_ms[s] = 0.0;
        h->prof_n[s] = 0;
    }
    return MG_OK;
}

mg_status mg_profile_read(mg_handle* h, int slot, double* ms, long long* launches) {
    if (!h || slot < 0 || slot >= MG_PROF_SLOTS) return MG_EINVAL;
    CK(cudaStreamSynchronize(h->stream));
    prof_collect(h);
    if (ms) *ms = h->prof_ms[slot];
    if (launches) *launches = h->prof_n[slot];
    return MG_OK;
}

mg_status mg_solve_batch(mg_handle* const* hs, int n, const double* const* f, double* const* x,
                         const double* tol, mg_report* reps) {
    if (!hs || n < 0 || (n > 0 && (!f || !x || !tol))) return MG_EINVAL;
    if (n == 0) return MG_OK;
    for (int s = 0; s < n; ++s) {
        if (!hs[s] || !f[s] || !x[s] || !(tol[s] >= 0) || !std::isfinite(tol[s])) return MG_EINVAL;
        for (int q = 0; q < s; ++q)
            if (hs[q] == hs[s]) {
                set_error("a handle appears twice in the batch");
                return MG_EINVAL;
            }
    }
    mg_handle* h0 = hs[0];
    StreamJoin join(h0);
    std::vector<unsigned long long> key;
    for (int s = 0; s < n; ++s) key.push_back(hs[s]->serial);
    if (!h0->batch || h0->batch_key != key) {
        plan_destroy(h0->batch);
        h0->batch = nullptr;
        h0->batch_key.clear();
        CKS(plan_create(hs, n, &h0->batch));
        h0->batch_key = key;
    }
    // the other handles' caller streams are ordered before the batch as well
    for (int s = 1; s < n; ++s) {
        CK(cudaEventRecord(hs[s]->ev_in, hs[s]->user_stream));
        CK(cudaStreamWaitEvent(h0->stream, hs[s]->ev_in, 0));
    }
    const mg_status st = plan_solve(h0->batch, f, x, tol, reps);
    for (int s = 1; s < n; ++s) {
        CK(cudaEventRecord(hs[s]->ev_out, h0->stream));
        CK(cudaStreamWaitEvent(hs[s]->user_stream, hs[s]->ev_out, 0));
    }
    return st;
}

}  // extern "C"

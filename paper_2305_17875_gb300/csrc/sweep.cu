// sweep.cu - one whole multicolour Gauss-Seidel sweep per launch.
//
// The colour passes of the smoother (batch.cu) each read every x, b and
// coefficient sector of a level while updating 1/2 (7 points) or 1/4 (19
// points) of its cells.  Here one launch does the whole sweep: a CTA owns a
// tile of TI colatitude rows x TK longitudes (TK = nph: whole rows) and
// marches along the radius through a chunk of TJ planes.  The old iterate
// arrives plane by plane in a ring of shared-memory buffers, each plane one
// three-dimensional bulk tensor copy (tile plus halo; rows or longitudes
// outside the grid read as zero and are never used, see below) completing on
// the slot's mbarrier.  In step s the colours are updated plane by plane with
// a lag of one plane per colour, in place in the ring:
//   7 points (red = (i + j + k) even, black = odd): red on plane s, then
//   black on plane s - 1;
//   19 points (colour ((i + j) & 1) + 2 ((j + k) & 1), order 0, 1, 2, 3):
//   colour c on plane s - c.
// A cell of colour c reads colours below c already updated and colours above
// c not yet updated on the planes either side of it, exactly as in the
// sequential sweep; to update the tile, colour c is also updated on a ring
// of (C - 1 - c) cells around it (and as many planes beyond the chunk), from
// the old iterate: neighbouring tiles repeat that work, so no tile waits for
// another.  The sweep is out of place (x -> y), so a tile's halo is never
// changed under it.  A finished plane leaves as 16-byte stores of the tile.
//
// Per cell the arithmetic is that of the colour passes (Cell7::gs, apply19 and
// diag_cell with the same neighbour values: the mirror at the radius and
// colatitude walls, the longitude wrap), so a sweep gives the same bits as
// its C colour passes.  b and the coefficients are read from global memory
// (each cell's own entries once; the upper faces' entries a second time from
// L1/L2).
//
// Waits are bounded: a copy that has not landed after about a tenth of a
// second makes the CTA set the fault word, wait (bounded again) for its
// copies in flight, write NaN over its output tile and return, so the solve
// ends with MG_ENAN instead of hanging.
#include <cuda.h>

#include <map>
#include <mutex>
#include <utility>

#include "mg_kernels.h"

namespace mgs {

__device__ unsigned g_sweep_fault;   // set when a plane copy did not complete in time

namespace {

constexpr int kSW = 256;   // threads per CTA

template <int P>
struct SPrec;
template <>
struct SPrec<PREC64> {
    typedef double T;
    __device__ static const CoefF64& cf(const LevelView& v) { return v.c64; }
};
template <>
struct SPrec<PREC32> {
    typedef float T;
    __device__ static const CoefF32& cf(const LevelView& v) { return v.c32; }
};
template <>
struct SPrec<PREC16> {
    typedef float T;
    __device__ static const CoefF16& cf(const LevelView& v) { return v.c16; }
};

// ---- mbarrier and bulk tensor copy (inline PTX)
__device__ __forceinline__ unsigned sptr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sptr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(sptr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sptr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sptr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sptr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on phase `parity` of a slot's barrier: false after about 0.1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (int it = 0; it < (1 << 20); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it >= 32) __nanosleep(100);
    }
    return false;
}
// Orders this thread's earlier shared-memory accesses (generic proxy) before
// its later bulk copies (async proxy) into the same buffers.
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// The tensor map is written by a host copy before the launch; acquire it for
// the tensor-map proxy once per tile.
__device__ __forceinline__ void tmap_acquire(const void* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(map) : "memory");
}
// Box of the 3-D map (longitude, colatitude, radius) at (c0, c1, c2) into dst.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(sptr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(sptr(bar))
        : "memory");
}

// ---- geometry of one tile's sweep (all quantities in cells)
template <typename T>
struct SweepGeom {
    int TI, TJ, TK;        // tile rows, planes per chunk, longitudes (TK == nph: whole rows)
    bool full;             // whole longitude rows: the wrap is taken inside the buffer
    int H, HK;             // halo rows / longitudes of the plane buffers
    int rows, cols;        // plane buffer shape
    int i0, j0, k0, jend;  // tile origin, end of the chunk's planes
    int plo, phi;          // planes staged: [plo, phi]
    int ring;              // plane buffers
    unsigned pbytes;       // bytes of one buffer (multiple of 128)
    unsigned box_bytes;    // bytes of one copy
    unsigned char* base;   // the ring of plane buffers
    // the buffer holding plane p (plo <= p <= phi)
    __device__ __forceinline__ T* buf(int p) const {
        return reinterpret_cast<T*>(base + (size_t)((p - plo) % ring) * pbytes);
    }
};

__host__ __device__ inline int halo_rows(int stencil) { return stencil == 7 ? 2 : 4; }
// Longitude halo of a tile narrower than the grid: at least the stencil's
// reach, and a multiple of 16 bytes (the copy's inner coordinate).
__host__ __device__ inline int halo_cols(int stencil, int vbytes) {
    const int a = 16 / vbytes, h = halo_rows(stencil);
    return h > a ? h : a;
}
__host__ __device__ inline int ring_planes(int stencil) { return stencil == 7 ? 6 : 8; }

// Longitude k (global, maybe a few cells beyond the tile) -> buffer column.
template <typename T>
__device__ __forceinline__ int col_of(const SweepGeom<T>& g, int k) {
    return g.full ? k : k - g.k0 + g.HK;
}

// ---- colour stages.  Stage (s, c): the cells of colour c on plane s - c over
// the tile widened by the colour's ring.  A stage's cells are numbered row by
// row; thread t takes cells t, t + kSW, ... (at most StageSize<S>::kCells of them,
// checked on the host), so the loads of a stage are spread evenly and issued
// together.
template <int S>
struct StageSize;
template <>
struct StageSize<7> {
    static constexpr int kCells = 8;   // cells per thread and stage
    static constexpr int kVals = 7;    // b and the six face coefficients of Cell7
};
template <>
struct StageSize<19> {
    static constexpr int kCells = 4;
    static constexpr int kVals = 19;   // b, the cell's nine rows, three upper rows of three
};

struct Stage {
    int p, colour;   // plane, colour
    int ia, rstep;   // first row of the colour, row step (1, or 2 for 19 points)
    int ka, half;    // first longitude of the widened tile, cells of the colour per row
    int ncell;       // cells of the stage (0: plane outside the colour's range)
    float inv_half;  // 1 / half: row of cell u = floor((u + 1/2) / half), exact for u, half < 2^12
};

template <int S, typename T>
__device__ __forceinline__ Stage make_stage(const SweepGeom<T>& g, const Dims& D, int s, int c) {
    constexpr int C = S == 7 ? 2 : 4;
    Stage st;
    st.p = s - c;
    st.colour = c;
    const int ring = C - 1 - c;   // cells beyond the tile this colour must cover
    const bool on = st.p >= max(g.j0 - ring, 0) && st.p <= min(g.jend - 1 + ring, D.nr - 1);
    int ia = max(g.i0 - ring, 0);
    const int ib = min(g.i0 + g.TI + ring, D.nth);
    st.ka = g.full ? 0 : g.k0 - ring;
    const int kb = g.full ? D.nph : g.k0 + g.TK + ring;
    st.half = (kb - st.ka) >> 1;   // the widened width is even
    int rows;
    if (S == 19) {                 // rows with (i + p) = colour mod 2 only
        ia += ((ia + st.p) & 1) != (c & 1) ? 1 : 0;
        rows = ib > ia ? (ib - ia + 1) >> 1 : 0;
        st.rstep = 2;
    } else {
        rows = ib > ia ? ib - ia : 0;
        st.rstep = 1;
    }
    st.ia = ia;
    st.ncell = on ? rows * st.half : 0;
    st.inv_half = 1.0f / (float)(st.half > 0 ? st.half : 1);
    return st;
}

// cell u of a stage -> colatitude i and longitude k (k beyond [0, nph) on
// tiles narrower than the grid: the caller wraps it)
template <int S>
__device__ __forceinline__ void stage_cell(const Stage& st, int u, int& i, int& k) {
    // (u + 1/2) / half is at least 1 / (2 half) away from an integer, far more
    // than the rounding of the product for u, half < 2^12
    const int r = (int)(((float)u + 0.5f) * st.inv_half), m = u - r * st.half;
    i = st.ia + st.rstep * r;
    const int par = S == 7 ? ((st.colour + st.p + i) & 1) : (((st.colour >> 1) + st.p) & 1);
    k = st.ka + ((par - st.ka) & 1) + 2 * m;
}

__device__ __forceinline__ int wrap_k(const Dims& D, int k) { return k < 0 ? k + D.nph : (k >= D.nph ? k - D.nph : k); }

// Loads of one stage into registers.
template <int S, bool AXI, typename T, typename CF>
__device__ __forceinline__ void stage_load(const CF& cf, const Dims& D, const T* __restrict__ b, const Stage& st,
                                           T (&v)[StageSize<S>::kCells][StageSize<S>::kVals]) {
    const int plane = D.nth * D.nph;
    if (st.ncell == 0) return;
    // every slot runs the same straight-line code (an idle slot repeats the
    // stage's last cell), so the slots' loads issue back to back
#pragma unroll
    for (int m = 0; m < StageSize<S>::kCells; ++m) {
        const int u = min((int)threadIdx.x + m * kSW, st.ncell - 1);
        int i, k;
        stage_cell<S>(st, u, i, k);
        k = wrap_k(D, k);
        const int c = (st.p * D.nth + i) * D.nph + k;
        const int kp = k == D.nph - 1 ? c - D.nph + 1 : c + 1;
        const bool ju = st.p + 1 < D.nr, iu = i + 1 < D.nth;
        v[m][0] = __ldg(b + c);
        if (S == 7) {   // Cell7: el, eu, zl, zu, xl, xu
            v[m][1] = (T)cf(4, c);
            v[m][2] = ju ? (T)cf(4, c + plane) : (T)0;
            v[m][3] = (T)cf(0, c);
            v[m][4] = iu ? (T)cf(0, c + D.nph) : (T)0;
            v[m][5] = (T)cf(8, c);
            v[m][6] = (T)cf(8, kp);
        } else {
#pragma unroll
            for (int a = 0; a < 9; ++a) v[m][1 + a] = RegRows<T, AXI>::stored(a) ? (T)cf(a, c) : (T)0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                v[m][10 + q] = ju && RegRows<T, AXI>::stored(3 + q) ? (T)cf(3 + q, c + plane) : (T)0;
                v[m][13 + q] = iu && RegRows<T, AXI>::stored(q) ? (T)cf(q, c + D.nph) : (T)0;
                v[m][16 + q] = RegRows<T, AXI>::stored(6 + q) ? (T)cf(6 + q, kp) : (T)0;
            }
        }
    }
}

// One stage: every cell x_c + (b - A x)_c / A_cc with the neighbours from the
// plane buffers (the colour passes' neighbour rules: mirror at the radius and
// colatitude walls, longitude wrap), the new values written in place.
template <int S, bool AXI, typename T>
__device__ __forceinline__ void stage_run(const Dims& D, const SweepGeom<T>& g, const Stage& st,
                                          const T (&v)[StageSize<S>::kCells][StageSize<S>::kVals]) {
    if (st.ncell == 0) return;
    const int p = st.p;
    T* p0 = g.buf(p);
    const T* pm = p > g.plo ? g.buf(p - 1) : p0;
    const T* pp = p < g.phi ? g.buf(p + 1) : p0;
    const int cols = g.cols;
    // every cell of the stage first, the stores after: no cell of a colour
    // reads another of the same colour, and the separate stores let the cells'
    // loads and arithmetic interleave
    T res[StageSize<S>::kCells];
    int at[StageSize<S>::kCells];
#pragma unroll
    for (int m = 0; m < StageSize<S>::kCells; ++m) {
        const int u0 = (int)threadIdx.x + m * kSW;
        const int u = min(u0, st.ncell - 1);   // idle slots repeat the last cell, not stored
        int i, k;
        stage_cell<S>(st, u, i, k);
        const int lr = i - g.i0 + g.H, lc = col_of(g, k);
        const int o = lr * cols + lc;
        const bool jl = p > 0, ju = p + 1 < D.nr, il = i > 0, iu = i + 1 < D.nth;
        const int om = g.full && lc == 0 ? o + cols - 1 : o - 1;
        const int op = g.full && lc == cols - 1 ? o - cols + 1 : o + 1;
        T out;
        if (S == 7) {
            Cell7<T> q;
            q.xc = p0[o];
            q.el = v[m][1], q.eu = v[m][2], q.zl = v[m][3], q.zu = v[m][4], q.xl = v[m][5], q.xu = v[m][6];
            q.xjm = jl ? pm[o] : q.xc;
            q.xjp = ju ? pp[o] : q.xc;
            q.xim = il ? p0[o - cols] : q.xc;
            q.xip = iu ? p0[o + cols] : q.xc;
            q.xkm = p0[om];
            q.xkp = p0[op];
            out = q.gs(v[m][0]);
        } else {
            // the neighbourhood of Nbr19::load
            const T* pl[3] = {jl ? pm : p0, p0, ju ? pp : p0};
            const int orow[3] = {il ? -cols : 0, 0, iu ? cols : 0};
            const int ocol[3] = {om - o, 0, op - o};
            Nbr19<T> X;
#pragma unroll
            for (int n = 0; n < 19; ++n) {
                const bool phi_edge = row_off(n, 2) != 0 && (row_off(n, 0) != 0 || row_off(n, 1) != 0);
                X.v[n] = (AXI && phi_edge) ? (T)0 : pl[row_off(n, 0) + 1][o + orow[row_off(n, 1) + 1] + ocol[row_off(n, 2) + 1]];
            }
            const C3 c3{p, i, wrap_k(D, k)};
            const RegRows<T, AXI> cr{v[m]};
            const T r = v[m][0] - apply19_r<T>(cr, X, D, c3);
            out = X.v[0] + r / diag_cell_r<19, T>(cr, D, c3);
        }
        res[m] = out;
        at[m] = u0 < st.ncell ? o : -1;
    }
#pragma unroll
    for (int m = 0; m < StageSize<S>::kCells; ++m)
        if (at[m] >= 0) p0[at[m]] = res[m];
}

// The tile's cells of plane p from its buffer to the output, 16 bytes per store
// where the row allows.
template <typename T>
__device__ __forceinline__ void store_plane(const Dims& D, const SweepGeom<T>& g, T* out, int p) {
    const T* src = g.buf(p);
    const int ib = min(g.i0 + g.TI, D.nth);
    constexpr int V = 16 / sizeof(T);
    const int nv = g.TK / V;   // TK is a multiple of V
    const int items = (ib - g.i0) * nv;
    for (int t = threadIdx.x; t < items; t += kSW) {
        const int r = t / nv, v = t - r * nv;
        const int i = g.i0 + r, k = g.k0 + v * V;
        const T* s = src + (i - g.i0 + g.H) * g.cols + col_of(g, k);
        T* d = out + (p * D.nth + i) * D.nph + k;
        if (sizeof(T) == 4) {
            *reinterpret_cast<float4*>(d) = make_float4(s[0], s[1], s[2], s[3]);
        } else {
            *reinterpret_cast<double2*>(d) = make_double2(s[0], s[1]);
        }
    }
}

// NaN over the tile's output (a plane copy timed out).
template <typename T>
__device__ void poison_tile(const Dims& D, const SweepGeom<T>& g, T* out) {
    const int ib = min(g.i0 + g.TI, D.nth);
    const int per = (ib - g.i0) * g.TK;
    const T nan = (T)__int_as_float(0x7fc00000);
    for (int p = g.j0; p < g.jend; ++p)
        for (int t = threadIdx.x; t < per; t += kSW) {
            const int r = t / g.TK, kk = t - r * g.TK;
            out[(p * D.nth + g.i0 + r) * D.nph + g.k0 + kk] = nan;
        }
}

template <int S, bool AXI, typename T, typename CF>
__device__ void sweep_tile(const BTask& tk, const CF& cf_shared, int lb, unsigned char* smem) {
    // the task descriptor lives in shared memory, which the stages write:
    // registers copies, so its fields are not reloaded after every store
    const Dims D = tk.v.D;
    const CF cf = cf_shared;
    SweepGeom<T> g;
    g.TI = tk.tile[0];
    g.TJ = tk.tile[1];
    g.TK = tk.tile[2];
    g.full = g.TK == D.nph;
    g.H = halo_rows(S);
    g.HK = g.full ? 0 : halo_cols(S, (int)sizeof(T));
    g.rows = g.TI + 2 * g.H;
    g.cols = g.full ? D.nph : g.TK + 2 * g.HK;
    g.ring = ring_planes(S);
    g.box_bytes = (unsigned)(g.rows * g.cols * sizeof(T));
    g.pbytes = (g.box_bytes + 127u) & ~127u;
    const int nK = D.nph / g.TK, nI = (D.nth + g.TI - 1) / g.TI;
    const int kt = lb % nK, it = (lb / nK) % nI, jc = lb / (nK * nI);
    g.i0 = it * g.TI;
    g.k0 = kt * g.TK;
    g.j0 = jc * g.TJ;
    g.jend = min(g.j0 + g.TJ, D.nr);
    constexpr int C = S == 7 ? 2 : 4;          // colours
    const int reach = C;                        // planes staged beyond the chunk
    g.plo = max(g.j0 - reach, 0);
    g.phi = min(g.jend - 1 + reach, D.nr - 1);
    const void* map = tk.tmap;
    const T* b = (const T*)tk.b;
    T* out = (T*)tk.y;
    const T* xin = (const T*)tk.x;

    g.base = smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)g.ring * g.pbytes);

    if (threadIdx.x == 0) {
        tmap_acquire(map);
        for (int r = 0; r < g.ring; ++r) mbar_init(&bars[r], 1);
        fence_barrier_init();
    }
    __syncthreads();

    int nxt = g.plo;   // next plane to copy (thread 0)
    auto issue = [&](int upto) {
        for (; nxt <= g.phi && nxt <= upto; ++nxt) {
            const int slot = (nxt - g.plo) % g.ring;
            mbar_expect_tx(&bars[slot], g.box_bytes);
            tma_load_3d(g.buf(nxt), map, g.full ? 0 : g.k0 - g.HK, g.i0 - g.H, nxt, &bars[slot]);
        }
    };
    if (threadIdx.x == 0) issue(g.plo + g.ring - 1);

    // Tiles narrower than the grid at the longitude seam: the copy reads zeros
    // beyond the grid; the halo columns there take the wrapped values.
    const bool seam = !g.full && (kt == 0 || kt == nK - 1);
    auto fix_seam = [&](int p) {
        T* dst = g.buf(p);
        const int n = g.rows * 2 * g.HK;
        for (int t = threadIdx.x; t < n; t += kSW) {
            const int r = t / (2 * g.HK), h = t - r * (2 * g.HK);
            const int i = g.i0 - g.H + r;
            if (i < 0 || i >= D.nth) continue;
            const int lc = h < g.HK ? h : g.TK + h;               // left halo, then right
            const int k = g.k0 - g.HK + lc;
            if (k >= 0 && k < D.nph) continue;                      // inside the grid: copied
            const int kw = k < 0 ? k + D.nph : k - D.nph;
            dst[r * g.cols + lc] = xin[(p * D.nth + i) * D.nph + kw];
        }
    };

    int waited = g.plo - 1;
    bool fault = false;
    // The planes the stage of step s reads, the last stored plane, the ring
    // slots freed: colour c works on plane s - c and reads planes s - c - 1 ..
    // s - c + 1; plane q is final after step q + C - 1 and stored in step
    // q + C; so in step s the planes up to s - C - 1 are free.
    const int s_first = max(g.j0 - (C - 1), 0);
    const int s_last = g.jend - 1 + (C - 1);
    // b and coefficients of each stage are loaded one stage ahead (they do not
    // depend on the iterate), so their latency overlaps the barrier and the
    // plane copies
    T v[StageSize<S>::kCells][StageSize<S>::kVals];
    Stage st = make_stage<S, T>(g, D, s_first, 0);
    stage_load<S, AXI, T>(cf, D, b, st, v);
    for (int s = s_first; s <= s_last && !fault; ++s) {
        if (threadIdx.x == 0) issue(s - C - 1 + g.ring);
        const int need = min(s + 1, g.phi);
        bool ok = true;
        while (waited < need && ok) {
            const int q = waited + 1;
            ok = mbar_wait(&bars[(q - g.plo) % g.ring], (unsigned)(((q - g.plo) / g.ring) & 1));
            if (ok) {
                waited = q;
                if (seam) fix_seam(q);
            }
        }
        if (__syncthreads_or(!ok)) {
            fault = true;
            break;
        }
        // the plane finished in the previous step leaves
        if (s - C >= g.j0 && s - C < g.jend) store_plane(D, g, out, s - C);
        for (int c = 0; c < C; ++c) {
            stage_run<S, AXI, T>(D, g, st, v);
            st = c + 1 < C ? make_stage<S, T>(g, D, s, c + 1) : make_stage<S, T>(g, D, s + 1, 0);
            if (c + 1 < C || s < s_last) stage_load<S, AXI, T>(cf, D, b, st, v);
            // the step's shared-memory writes precede the next copies into
            // these buffers (issued after the barrier)
            if (c == C - 1) fence_async_shared();
            __syncthreads();
        }
    }
    if (!fault && s_last - C + 1 >= g.j0) {
        // planes finished in the last step(s) without a following store
        for (int q = max(s_last - C + 1, g.j0); q < g.jend; ++q) store_plane(D, g, out, q);
    }
    if (fault) {
        if (threadIdx.x == 0) atomicOr(&g_sweep_fault, 1u);
        // copies in flight still write into the buffers: wait for them (bounded)
        for (int q = waited + 1; q < nxt; ++q) {
            const int slot = (q - g.plo) % g.ring;
            mbar_wait(&bars[slot], (unsigned)(((q - g.plo) / g.ring) & 1));
        }
        poison_tile(D, g, out);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int r = 0; r < g.ring; ++r) mbar_inval(&bars[r]);
    __syncthreads();
}

template <int S, int P, bool AXI>
__global__ void __launch_bounds__(kSW) k_sweep(const BTask* __restrict__ tasks, int ntasks, int total,
                                               const int* __restrict__ active, int early_trigger,
        unsigned long long* stamp) {
    typedef typename SPrec<P>::T T;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(16) unsigned char tk_raw[sizeof(BTask)];
    __shared__ int tk_index;
    const BTask& tk = *reinterpret_cast<const BTask*>(tk_raw);
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    stamp_start(stamp);
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
            for (int w = threadIdx.x; w < (int)(sizeof(BTask) / 4); w += kSW) dst[w] = __ldg(src + w);
        }
        __syncthreads();
        if (!active || active[tk.shell]) sweep_tile<S, AXI, T>(tk, SPrec<P>::cf(tk.v), vb - tk.block0, dyn);
        __syncthreads();
    }
    stamp_end(stamp);
    if (!early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

bool sweep_pdl() {
    static const bool on = std::getenv("MG_NO_PDL") == nullptr;
    return on;
}

// Resident CTAs per SM of a sweep kernel at (threads, dynamic shared memory):
// the kernel's shared-memory limit is raised and the runtime asked once per
// configuration (the query costs host time on every eager launch otherwise).
// Serialised: launches come from several host threads.
template <typename K>
cudaError_t sweep_per_sm(K kernel, int threads, size_t smem, int* per_sm) {
    static std::mutex mu;
    static std::map<std::pair<const void*, std::pair<int, size_t>>, int> known;
    static std::map<const void*, size_t> smem_attr;
    const void* key = reinterpret_cast<const void*>(kernel);
    std::lock_guard<std::mutex> lk(mu);
    auto it = known.find({key, {threads, smem}});
    if (it != known.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    if (smem > smem_attr[key]) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_attr[key] = smem;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, threads, smem);
    if (e == cudaSuccess) known[{key, {threads, smem}}] = *per_sm;
    return e;
}

template <int S, int P, bool AXI>
cudaError_t sweep_launch(const BTask* tasks, int ntasks, int total, const int* active, size_t smem, cudaStream_t s,
                         unsigned long long* stamp) {
    int per_sm = 0;
    cudaError_t e = sweep_per_sm(k_sweep<S, P, AXI>, kSW, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(total, 152 * per_sm);   // persistent beyond one wave
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kSW, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = sweep_pdl() ? 1 : 0;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep<S, P, AXI>, tasks, ntasks, total, active, grid >= total ? 1 : 0, stamp);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return (EncodeTiledFn)p;
    }();
    return fn;
}


// ---- the 7-point red-black sweep on whole longitude rows (FP32 iterate;
// FP32 or FP16 coefficients).
//
// A CTA owns TI colatitude rows i0 .. i0 + TI - 1 and a chunk of TJ radius
// planes, one thread per quad (four consecutive longitudes) of the rows
// i0 - 1 .. i0 + TI: the two rows outside the tile carry red updates only,
// which the black cells of the tile's edge rows read.  Every plane of x (rows
// i0 - 2 .. i0 + TI + 1), of b and of the three lower-face coefficient arrays
// (rows i0 - 1 .. i0 + TI + 1) arrives as five bulk tensor copies on one
// mbarrier, in a ring of four slots that a copy warp keeps filled: it reuses a
// slot once every compute warp has released the plane in it (a second
// mbarrier per slot), so copies never wait on the compute warps' steps and the
// compute warps meet only among themselves (a named barrier) once per step.
//
// Step s updates the red cells of plane s and the black cells of plane s - 1;
// in a quad both are the positions P, P + 2 with P = (i + s) mod 2.  A thread
// holds its quad on planes s - 2 .. s + 1 in registers (the radius
// neighbours never pass through shared memory), reads the colatitude and
// longitude neighbours of its red cells from the copied plane (old values:
// black cells of plane s are updated only in step s + 1) and those of its
// black cells from a small double-buffered array where every thread leaves
// its two new red values of the plane (written in step s - 1), and stores the
// finished quad of plane s - 1 with one 16-byte store.  The red ring rows and
// the red planes j0 - 1 and jend repeat work of the neighbouring tiles from
// the old iterate, so no tile waits for another; the sweep is out of place.
//
// The arithmetic is Cell7::gs with the colour passes' neighbour values
// (mirror at the radius and colatitude walls, longitude wrap), so a sweep
// gives the bits of its two colour passes.
constexpr int kRB7Max = kRB7MaxThreads + 32;   // threads: up to nine rows of 64 quads, and the copy warp
constexpr int kRB7Slots = 4;   // plane slots of the copy ring

struct RB7Layout {
    unsigned xoff, boff, eoff, zoff, loff;   // the five arrays within a slot
    unsigned slot;                           // bytes of one slot (multiple of 128)
    unsigned tx;                             // bytes the five copies of a plane deliver
    unsigned roff, boff_bars, total;         // red-value array, mbarriers, whole layout
};

__host__ __device__ inline unsigned rb7_up128(unsigned v) { return (v + 127u) & ~127u; }

__host__ __device__ inline RB7Layout rb7_layout(int TI, int nph, int cbytes) {
    RB7Layout L;
    const unsigned xb = (unsigned)((TI + 4) * nph * 4), bb = (unsigned)((TI + 3) * nph * 4);
    const unsigned cb = (unsigned)((TI + 3) * nph * cbytes);
    L.xoff = 0;
    L.boff = rb7_up128(xb);
    L.eoff = L.boff + rb7_up128(bb);
    L.zoff = L.eoff + rb7_up128(cb);
    L.loff = L.zoff + rb7_up128(cb);
    L.slot = L.loff + rb7_up128(cb);
    L.tx = xb + bb + 3 * cb;
    L.roff = kRB7Slots * L.slot;
    L.boff_bars = L.roff + rb7_up128((unsigned)(2 * (TI + 2) * (nph / 4) * 8));
    L.total = L.boff_bars + 16 * kRB7Slots + 16;   // full and empty barriers, the abort flag
    return L;
}

template <typename CT>
struct RB7Coef;
template <>
struct RB7Coef<float> {
    static constexpr int kBytes = 4;
    __device__ static float scale(const LevelView& v, int a) { return 1.0f; }
    __device__ static const void* array(const LevelView& v, int a) { return v.c32.g[a]; }
    __device__ static void quad(const float* row, int k0, float, float (&v)[4]) {
        const float4 p = *reinterpret_cast<const float4*>(row + k0);
        v[0] = p.x, v[1] = p.y, v[2] = p.z, v[3] = p.w;
    }
    __device__ static float one(const float* row, int k, float) { return row[k]; }
};
// FP16 storage: the value is the half times the component's power-of-two
// scale, as CoefF16 reads it
template <>
struct RB7Coef<__half> {
    static constexpr int kBytes = 2;
    __device__ static float scale(const LevelView& v, int a) { return v.c16.s[a]; }
    __device__ static const void* array(const LevelView& v, int a) { return v.c16.g[a]; }
    __device__ static void quad(const __half* row, int k0, float s, float (&v)[4]) {
        const uint2 p = *reinterpret_cast<const uint2*>(row + k0);
        const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&p.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&p.y));
        v[0] = lo.x * s, v[1] = lo.y * s, v[2] = hi.x * s, v[3] = hi.y * s;
    }
    __device__ static float one(const __half* row, int k, float s) { return __half2float(row[k]) * s; }
};

__device__ __forceinline__ void lds4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}

// Coefficients of the quad's cells on one plane, as Cell7::load reads them:
// b, the lower radius / colatitude / longitude faces, the upper colatitude
// face (the next row's lower one, zero on the wall row) and the upper
// longitude face of the last cell (the next quad's first lower one).
struct RB7Plane {
    float B[4], EL[4], ZL[4], ZU[4], XL[4];
    float XLn;
};

// Red cells P, P + 2 of plane s.  X0 = the quad on plane s, XM1 = on plane
// s - 1 (black there: old), X1 = on plane s + 1 (old); XIM / XIP = the rows
// i -/+ 1 of plane s (old); xadj = the longitude neighbour outside the quad
// (k0 - 1 for P = 0, k0 + 4 for P = 1); EU = the lower radius faces of plane
// s + 1 (zero above the last plane).
template <int P>
__device__ __forceinline__ void rb7_red(const RB7Plane& c, const float (&EU)[4], const float (&X0)[4],
                                        const float (&XM1)[4], const float (&X1)[4], const float (&XIM)[4],
                                        const float (&XIP)[4], float xadj, bool jl, bool ju, bool il, bool iu,
                                        float (&rn)[2]) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int m = P + 2 * e;
        Cell7<float> q;
        q.xc = X0[m];
        q.xjm = jl ? XM1[m] : q.xc;
        q.xjp = ju ? X1[m] : q.xc;
        q.xim = il ? XIM[m] : q.xc;
        q.xip = iu ? XIP[m] : q.xc;
        q.xkm = m == 0 ? xadj : X0[m == 0 ? 0 : m - 1];
        q.xkp = m == 3 ? xadj : X0[m == 3 ? 3 : m + 1];
        q.el = c.EL[m], q.eu = EU[m], q.zl = c.ZL[m], q.zu = c.ZU[m], q.xl = c.XL[m];
        q.xu = m == 3 ? c.XLn : c.XL[m == 3 ? 3 : m + 1];
        rn[e] = q.gs(c.B[m]);
    }
}

// Black cells P, P + 2 of plane s - 1.  XM1 = the quad on plane s - 1 (black
// cells old, red ones new), XM2 = the new red values of plane s - 2 at P, P + 2,
// rn = the new red values of plane s at P, P + 2; rim / rip = the new red values
// of the rows i -/+ 1 on plane s - 1 at P, P + 2; radj = the red longitude
// neighbour outside the quad; c = plane s - 1's coefficients; EU = plane s's
// lower radius faces (zero when plane s does not exist).
template <int P>
__device__ __forceinline__ void rb7_black(const RB7Plane& c, const float (&EU)[4], const float (&XM1)[4],
                                          const float (&XM2)[2], const float (&rn)[2], float2 rim, float2 rip,
                                          float radj, bool jl, bool ju, bool il, bool iu, float (&bn)[2]) {
    const float RIM[2] = {rim.x, rim.y}, RIP[2] = {rip.x, rip.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int m = P + 2 * e;
        Cell7<float> q;
        q.xc = XM1[m];
        q.xjm = jl ? XM2[e] : q.xc;
        q.xjp = ju ? rn[e] : q.xc;
        q.xim = il ? RIM[e] : q.xc;
        q.xip = iu ? RIP[e] : q.xc;
        q.xkm = m == 0 ? radj : XM1[m == 0 ? 0 : m - 1];
        q.xkp = m == 3 ? radj : XM1[m == 3 ? 3 : m + 1];
        q.el = c.EL[m], q.eu = EU[m], q.zl = c.ZL[m], q.zu = c.ZU[m], q.xl = c.XL[m];
        q.xu = m == 3 ? c.XLn : c.XL[m == 3 ? 3 : m + 1];
        bn[e] = q.gs(c.B[m]);
    }
}

// The finished quad of plane s - 1: the black cells P, P + 2 new (bn), the red
// ones from XM1.
__device__ __forceinline__ void rb7_store(float* dst, int P, const float (&bn)[2], const float (&XM1)[4]) {
    *reinterpret_cast<float4*>(dst) = P ? make_float4(XM1[0], bn[0], XM1[2], bn[1])
                                        : make_float4(bn[0], XM1[1], bn[1], XM1[3]);
}

template <typename CT>
__device__ __forceinline__ void rb7_tile(const BTask& tk, int lb, unsigned char* smem) {
    const Dims D = tk.v.D;
    const int nph = D.nph, NQ = nph >> 2;
    const int TI = tk.tile[0], TJ = tk.tile[1];
    const int nI = (D.nth + TI - 1) / TI;
    const int it = lb % nI, jc = lb / nI;
    const int i0 = it * TI, iend = min(i0 + TI, D.nth);
    const int j0 = jc * TJ, jend = min(j0 + TJ, D.nr);
    const int plo = max(j0 - 2, 0), phi = min(jend + 1, D.nr - 1);
    const RB7Layout Ly = rb7_layout(TI, nph, RB7Coef<CT>::kBytes);
    const float sel = RB7Coef<CT>::scale(tk.v, 4), szl = RB7Coef<CT>::scale(tk.v, 0),
                sxl = RB7Coef<CT>::scale(tk.v, 8);
    const unsigned char* maps = (const unsigned char*)tk.tmap;   // x, b, el, zl, xl (128 bytes each)
    float* out = (float*)tk.y;
    float2* R = reinterpret_cast<float2*>(smem + Ly.roff);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + Ly.boff_bars);   // a plane's copies landed
    uint64_t* empty = full + kRB7Slots;                                  // every compute warp is done with it
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kRB7Slots);
    auto slot = [&](int p) { return smem + (size_t)((p - plo) % kRB7Slots) * Ly.slot; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncw = (int)(blockDim.x >> 5) - 1;   // compute warps; the last warp copies
    const int s0 = max(j0 - 1, 0);

    if (threadIdx.x == 0) {
        for (int w = 0; w < kRB7Slots; ++w) {
            mbar_init(&full[w], 1);
            mbar_init(&empty[w], ncw);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == ncw) {
        // the copy warp: plane p into slot (p - plo) mod 4 once the compute
        // warps have released the plane four before it
        if (lane == 0) {
            for (int m = 0; m < 5; ++m) tmap_acquire(maps + 128 * m);
            int end = plo;   // planes plo .. end - 1 copied
            for (int p = plo; p <= phi && !*abort_flag; ++p) {
                const int w = (p - plo) % kRB7Slots, k = (p - plo) / kRB7Slots;
                if (k > 0 && !mbar_wait(&empty[w], (unsigned)((k - 1) & 1))) break;
                unsigned char* sl = smem + (size_t)w * Ly.slot;
                mbar_expect_tx(&full[w], Ly.tx);
                tma_load_3d(sl + Ly.xoff, maps, 0, i0 - 2, p, &full[w]);
                tma_load_3d(sl + Ly.boff, maps + 128, 0, i0 - 1, p, &full[w]);
                tma_load_3d(sl + Ly.eoff, maps + 256, 0, i0 - 1, p, &full[w]);
                tma_load_3d(sl + Ly.zoff, maps + 384, 0, i0 - 1, p, &full[w]);
                tma_load_3d(sl + Ly.loff, maps + 512, 0, i0 - 1, p, &full[w]);
                end = p + 1;
            }
            // the compute warps stopped early (a copy that did not land): the
            // copies in flight still write the slots; wait for them (bounded)
            if (*abort_flag)
                for (int p = max(plo, end - kRB7Slots); p < end; ++p)   // the last copy into each slot
                    mbar_wait(&full[(p - plo) % kRB7Slots], (unsigned)(((p - plo) / kRB7Slots) & 1));
        }
    } else {
        // this thread's quad: unit row r (colatitude i0 - 1 + r), quad q
        const int u = threadIdx.x;
        const int r = u / NQ, q = u - r * NQ;
        const int i = i0 - 1 + r;
        const bool valid = u < (TI + 2) * NQ && i >= 0 && i <= iend && i < D.nth;
        const bool interior = valid && i >= i0 && i < iend;
        const int k0 = 4 * q;
        const bool il = i > 0, iu = i + 1 < D.nth;
        const int xr = (r + 1) * nph;                 // own row in the x buffers
        const int cr = r * nph;                       // own row in the b and coefficient buffers
        const int km = k0 == 0 ? nph - 1 : k0 - 1;    // longitude neighbours outside the quad
        const int kp = k0 + 4 == nph ? 0 : k0 + 4;
        const int qm = q == 0 ? NQ - 1 : q - 1, qp = q + 1 == NQ ? 0 : q + 1;
        const unsigned nct = (unsigned)(ncw * 32);
        auto sync_compute = [&]() { asm volatile("bar.sync 1, %0;\n" ::"r"(nct) : "memory"); };
        auto release = [&](int p) {   // this warp has read plane p for the last time
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[(p - plo) % kRB7Slots]);
        };
        int waited = plo - 1;
        auto wait_upto = [&](int need) {
            bool ok = true;
            while (waited < need && ok) {
                const int p = waited + 1;
                ok = mbar_wait(&full[(p - plo) % kRB7Slots], (unsigned)(((p - plo) / kRB7Slots) & 1));
                if (ok) waited = p;
            }
            if (!ok) *abort_flag = 1;
            return ok;
        };

        // state at the first step s0: the quad on planes s0 - 1 and s0 (old)
        float xm2[2] = {0.f, 0.f}, xm1[4] = {0.f, 0.f, 0.f, 0.f}, x0[4] = {0.f, 0.f, 0.f, 0.f};
        RB7Plane kc;   // coefficients of plane s - 1 (its black cells are updated in step s)
        for (int m = 0; m < 4; ++m) kc.B[m] = kc.EL[m] = kc.ZL[m] = kc.ZU[m] = kc.XL[m] = 0.f;
        kc.XLn = 0.f;
        if (wait_upto(min(s0, phi)) && valid) {
            if (s0 > 0) lds4(reinterpret_cast<const float*>(slot(s0 - 1) + Ly.xoff) + xr + k0, xm1);
            lds4(reinterpret_cast<const float*>(slot(s0) + Ly.xoff) + xr + k0, x0);
        }
        if (s0 > plo) release(plo);
        sync_compute();

        for (int s = s0; s <= jend && !*abort_flag; ++s) {
            const bool ok = wait_upto(min(s + 1, phi));
            const bool red = s < D.nr;          // plane s exists
            const bool ju = s + 1 < D.nr;       // plane s + 1 exists
            const bool blk = interior && s - 1 >= j0;
            const int P = (i + s) & 1;
            float rn[2] = {0.f, 0.f};
            RB7Plane c;
            float EU[4] = {0.f, 0.f, 0.f, 0.f};   // lower radius faces of plane s + 1
            float ELs[4] = {0.f, 0.f, 0.f, 0.f};  // lower radius faces of plane s (black's upper faces)
            if (ok && valid && red) {
                const unsigned char* sl = slot(s);
                const float* X = reinterpret_cast<const float*>(sl + Ly.xoff);
                const CT* EL = reinterpret_cast<const CT*>(sl + Ly.eoff);
                const CT* ZL = reinterpret_cast<const CT*>(sl + Ly.zoff);
                const CT* XL = reinterpret_cast<const CT*>(sl + Ly.loff);
                lds4(reinterpret_cast<const float*>(sl + Ly.boff) + cr + k0, c.B);
                RB7Coef<CT>::quad(EL + cr, k0, sel, c.EL);
                RB7Coef<CT>::quad(ZL + cr, k0, szl, c.ZL);
                if (iu) RB7Coef<CT>::quad(ZL + cr + nph, k0, szl, c.ZU);
                else c.ZU[0] = c.ZU[1] = c.ZU[2] = c.ZU[3] = 0.f;
                RB7Coef<CT>::quad(XL + cr, k0, sxl, c.XL);
                c.XLn = RB7Coef<CT>::one(XL + cr, kp, sxl);
                for (int m = 0; m < 4; ++m) ELs[m] = c.EL[m];
                float X1[4] = {0.f, 0.f, 0.f, 0.f}, XIM[4], XIP[4];
                if (ju) {
                    const unsigned char* sl1 = slot(s + 1);
                    lds4(reinterpret_cast<const float*>(sl1 + Ly.xoff) + xr + k0, X1);
                    RB7Coef<CT>::quad(reinterpret_cast<const CT*>(sl1 + Ly.eoff) + cr, k0, sel, EU);
                }
                lds4(X + xr - nph + k0, XIM);
                lds4(X + xr + nph + k0, XIP);
                const float xadj = X[xr + (P == 0 ? km : kp)];
                if (P == 0) rb7_red<0>(c, EU, x0, xm1, X1, XIM, XIP, xadj, s > 0, ju, il, iu, rn);
                else rb7_red<1>(c, EU, x0, xm1, X1, XIM, XIP, xadj, s > 0, ju, il, iu, rn);
                R[(s & 1) * (TI + 2) * NQ + r * NQ + q] = make_float2(rn[0], rn[1]);
                if (blk) {
                    const float2* Rp = R + ((s - 1) & 1) * (TI + 2) * NQ;
                    const float2 rim = il ? Rp[(r - 1) * NQ + q] : make_float2(0.f, 0.f);
                    const float2 rip = iu ? Rp[(r + 1) * NQ + q] : make_float2(0.f, 0.f);
                    const float radj = P == 0 ? Rp[r * NQ + qm].y : Rp[r * NQ + qp].x;
                    float bn[2];
                    if (P == 0) rb7_black<0>(kc, ELs, xm1, xm2, rn, rim, rip, radj, s - 1 > 0, true, il, iu, bn);
                    else rb7_black<1>(kc, ELs, xm1, xm2, rn, rim, rip, radj, s - 1 > 0, true, il, iu, bn);
                    rb7_store(out + ((i64)(s - 1) * D.nth + i) * nph + k0, P, bn, xm1);
                }
                // shift: plane s - 1's red values become the next step's plane
                // s - 2 values, plane s (red new, black old) the next plane
                // s - 1, plane s + 1 the next plane s; plane s's coefficients
                // the next step's black ones (selects, not indexing by P: the
                // arrays stay in registers)
                xm2[0] = P ? xm1[0] : xm1[1];
                xm2[1] = P ? xm1[2] : xm1[3];
                xm1[0] = P ? x0[0] : rn[0];
                xm1[1] = P ? rn[0] : x0[1];
                xm1[2] = P ? x0[2] : rn[1];
                xm1[3] = P ? rn[1] : x0[3];
                x0[0] = X1[0], x0[1] = X1[1], x0[2] = X1[2], x0[3] = X1[3];
                kc = c;
            } else if (ok && blk) {
                // the last plane's black cells (s == nr: no plane above them)
                const float2* Rp = R + ((s - 1) & 1) * (TI + 2) * NQ;
                const float2 rim = il ? Rp[(r - 1) * NQ + q] : make_float2(0.f, 0.f);
                const float2 rip = iu ? Rp[(r + 1) * NQ + q] : make_float2(0.f, 0.f);
                const float radj = P == 0 ? Rp[r * NQ + qm].y : Rp[r * NQ + qp].x;
                float bn[2];
                if (P == 0) rb7_black<0>(kc, ELs, xm1, xm2, rn, rim, rip, radj, s - 1 > 0, false, il, iu, bn);
                else rb7_black<1>(kc, ELs, xm1, xm2, rn, rim, rip, radj, s - 1 > 0, false, il, iu, bn);
                rb7_store(out + ((i64)(s - 1) * D.nth + i) * nph + k0, P, bn, xm1);
            }
            if (ok && s <= phi) release(s);   // plane s is not read again
            sync_compute();                   // the red values of plane s are in R
        }
        if (*abort_flag) {
            const float nan = __int_as_float(0x7fc00000);
            const int per = (iend - i0) * nph;
            for (int p = j0; p < jend; ++p)
                for (int t = threadIdx.x; t < per; t += (int)nct) out[((i64)p * D.nth + i0) * nph + t] = nan;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*abort_flag) atomicOr(&g_sweep_fault, 1u);
        for (int w = 0; w < kRB7Slots; ++w) {
            mbar_inval(&full[w]);
            mbar_inval(&empty[w]);
        }
    }
    __syncthreads();
}

template <typename CT>
__global__ void __launch_bounds__(kRB7Max, 1) k_rb7(const BTask* __restrict__ tasks, int ntasks, int total,
                                                    const int* __restrict__ active, int early_trigger,
        unsigned long long* stamp) {
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(16) unsigned char tk_raw[sizeof(BTask)];
    __shared__ int tk_index;
    const BTask& tk = *reinterpret_cast<const BTask*>(tk_raw);
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    stamp_start(stamp);
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
            for (int w = threadIdx.x; w < (int)(sizeof(BTask) / 4); w += blockDim.x) dst[w] = __ldg(src + w);
        }
        __syncthreads();
        if (!active || active[tk.shell]) {
            const BTask t = tk;   // register copy: the stages write shared memory
            rb7_tile<CT>(t, vb - t.block0, dyn);
        }
        __syncthreads();
    }
    stamp_end(stamp);
    if (!early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename CT>
cudaError_t rb7_launch(const BTask* tasks, int ntasks, int total, const int* active, size_t smem, int threads,
                       cudaStream_t s, unsigned long long* stamp) {
    if (threads < 32 || threads > kRB7Max) return cudaErrorInvalidConfiguration;
    int per_sm = 0;
    cudaError_t e = sweep_per_sm(k_rb7<CT>, threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::min(total, 152 * per_sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = sweep_pdl() ? 1 : 0;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_rb7<CT>, tasks, ntasks, total, active, grid >= total ? 1 : 0, stamp);
}

bool rb7_path(int stencil, int prec) { return stencil == 7 && prec != PREC64; }

}  // namespace

bool sweep_tile_ok(const Dims& D, int stencil, int prec, const int tile[3]) {
    const int vb = prec == PREC64 ? 8 : 4;
    const int TI = tile[0], TJ = tile[1], TK = tile[2];
    if (TI < 1 || TJ < 1 || TK < 1 || D.cut) return false;
    if (rb7_path(stencil, prec)) {
        // whole rows of quads; every copy's rows a multiple of 16 bytes and at
        // most 256 elements wide; one thread per quad of TI + 2 rows
        const int cbytes = prec == PREC16 ? 2 : 4;
        if (TK != D.nph || D.nph % 4 != 0 || (D.nph * cbytes) % 16 != 0 || D.nph > 256) return false;
        if ((TI + 2) * (D.nph / 4) > kRB7MaxThreads || TI + 4 > 256) return false;
        return sweep_smem_bytes(stencil, prec, D, tile) <= 227 * 1024;
    }
    if ((D.nph * vb) % 16 != 0) return false;                  // row stride of the map
    if (D.nph % TK != 0 || (TK * vb) % 16 != 0) return false;  // whole 16-byte stores
    const bool full = TK == D.nph;
    const int cols = full ? D.nph : TK + 2 * halo_cols(stencil, vb);
    const int rows = TI + 2 * halo_rows(stencil);
    if (cols > 256 || rows > 256) return false;                // box limits of the copy
    if (!full && TK < halo_cols(stencil, vb)) return false;
    // the widest stage (colour 0, widened by its ring) within the cells a
    // thread holds in registers
    const int ring = stencil == 7 ? 1 : 3;
    const int srows = std::min(TI + 2 * ring, D.nth);
    const int rows_c = stencil == 7 ? srows : (srows + 1) / 2;
    const int half = (full ? D.nph : TK + 2 * ring) / 2;
    const int cap = (stencil == 7 ? StageSize<7>::kCells : StageSize<19>::kCells) * kSW;
    if (rows_c * half > cap) return false;
    return sweep_smem_bytes(stencil, prec, D, tile) <= 227 * 1024;
}

size_t sweep_smem_bytes(int stencil, int prec, const Dims& D, const int tile[3]) {
    if (rb7_path(stencil, prec)) return rb7_layout(tile[0], D.nph, prec == PREC16 ? 2 : 4).total;
    const int vb = prec == PREC64 ? 8 : 4;
    const bool full = tile[2] == D.nph;
    const size_t cols = full ? D.nph : tile[2] + 2 * halo_cols(stencil, vb);
    const size_t rows = tile[0] + 2 * halo_rows(stencil);
    const size_t pbytes = (rows * cols * vb + 127) & ~(size_t)127;
    return pbytes * ring_planes(stencil) + 8 * ring_planes(stencil);
}

int sweep_units(const Dims& D, const int tile[3]) {
    return ((D.nr + tile[1] - 1) / tile[1]) * ((D.nth + tile[0] - 1) / tile[0]) * (D.nph / tile[2]);
}

int sweep_threads(int stencil, int prec, const Dims& D, const int tile[3]) {
    if (!rb7_path(stencil, prec)) return kSW;
    return ((tile[0] + 2) * (D.nph / 4) + 31) / 32 * 32 + 32;   // the quads' warps and the copy warp
}

int sweep_map_count(int stencil, int prec) { return rb7_path(stencil, prec) ? 5 : 1; }

namespace {

// One 3-D map (longitude, colatitude, radius) of an [nr][nth][nph] array with
// boxes of whole rows: `rows` rows, one plane.
cudaError_t encode_rows(void* map, const void* base, const Dims& D, CUtensorMapDataType dt, int ebytes, int cols,
                        int rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)D.nph, (cuuint64_t)D.nth, (cuuint64_t)D.nr};
    const cuuint64_t strides[2] = {(cuuint64_t)D.nph * ebytes, (cuuint64_t)D.nph * D.nth * ebytes};
    const cuuint32_t box[3] = {(cuuint32_t)cols, (cuuint32_t)rows, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t encode_sweep_maps(void* maps, const BTask& t, int stencil, int prec) {
    const Dims& D = t.v.D;
    unsigned char* m = static_cast<unsigned char*>(maps);
    if (rb7_path(stencil, prec)) {
        // x (rows i0 - 2 .. i0 + TI + 1), b and the lower radius, colatitude and
        // longitude faces (rows i0 - 1 .. i0 + TI + 1)
        const int TI = t.tile[0];
        const bool h = prec == PREC16;
        const CUtensorMapDataType ct = h ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        const int cb = h ? 2 : 4;
        const void* c[3] = {h ? (const void*)t.v.c16.g[4] : (const void*)t.v.c32.g[4],
                            h ? (const void*)t.v.c16.g[0] : (const void*)t.v.c32.g[0],
                            h ? (const void*)t.v.c16.g[8] : (const void*)t.v.c32.g[8]};
        cudaError_t e = encode_rows(m, t.x, D, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, D.nph, TI + 4);
        if (e == cudaSuccess) e = encode_rows(m + 128, t.b, D, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, D.nph, TI + 3);
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = encode_rows(m + 256 + 128 * a, c[a], D, ct, cb, D.nph, TI + 3);
        return e;
    }
    const int vb = prec == PREC64 ? 8 : 4;
    const bool full = t.tile[2] == D.nph;
    return encode_rows(m, t.x, D, vb == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, vb,
                       full ? D.nph : t.tile[2] + 2 * halo_cols(stencil, vb), t.tile[0] + 2 * halo_rows(stencil));
}

cudaError_t launch_sweep(const BTask* tasks, int ntasks, int total, const int* active, int stencil, bool axi,
                         int prec, size_t smem, int threads, cudaStream_t s, unsigned long long* stamp) {
    if (ntasks <= 0 || total <= 0) return cudaSuccess;
    cudaError_t e;
    if (rb7_path(stencil, prec)) {
        if (prec == PREC16) e = rb7_launch<__half>(tasks, ntasks, total, active, smem, threads, s, stamp);
        else e = rb7_launch<float>(tasks, ntasks, total, active, smem, threads, s, stamp);
    } else if (stencil == 7) {   // FP64 (FP32 / FP16 take the red-black kernel above)
        e = sweep_launch<7, PREC64, false>(tasks, ntasks, total, active, smem, s, stamp);
    } else if (axi) {
        if (prec == PREC64) e = sweep_launch<19, PREC64, true>(tasks, ntasks, total, active, smem, s, stamp);
        else if (prec == PREC32) e = sweep_launch<19, PREC32, true>(tasks, ntasks, total, active, smem, s, stamp);
        else e = sweep_launch<19, PREC16, true>(tasks, ntasks, total, active, smem, s, stamp);
    } else {
        if (prec == PREC64) e = sweep_launch<19, PREC64, false>(tasks, ntasks, total, active, smem, s, stamp);
        else if (prec == PREC32) e = sweep_launch<19, PREC32, false>(tasks, ntasks, total, active, smem, s, stamp);
        else e = sweep_launch<19, PREC16, false>(tasks, ntasks, total, active, smem, s, stamp);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t sweep_fault_read(unsigned* out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_sweep_fault, sizeof(unsigned));
    if (e != cudaSuccess || !clear) return e;
    const unsigned z = 0;
    return cudaMemcpyToSymbol(g_sweep_fault, &z, sizeof(unsigned));
}

}  // namespace mgs

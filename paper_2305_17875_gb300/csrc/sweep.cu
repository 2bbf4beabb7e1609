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

// Face rows of one cell held in registers (the layout of StageSize<19>:
// v[1 + a] = component a of the cell's own rows, v[10 + q] = component 3 + q
// of the radius-upper row, v[13 + q] = component q of the colatitude-upper
// row, v[16 + q] = component 6 + q of the longitude-upper row), read by the
// formulas of mg_internal.cuh through CellRows' interface.
template <typename T, bool AXI>
struct RegRows {
    const T* v;
    __device__ __forceinline__ static constexpr bool stored(int a) {
        return !AXI || (a != 2 && a != 5 && a != 6 && a != 7);
    }
    __device__ __forceinline__ bool has(int a) const { return stored(a); }
    template <int F>
    __device__ __forceinline__ T at(int a) const {
        return F == 0 ? v[1 + a] : (F == 1 ? v[10 + a - 3] : (F == 2 ? v[13 + a] : v[16 + a - 6]));
    }
};

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
                                               const int* __restrict__ active, int early_trigger) {
    typedef typename SPrec<P>::T T;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(16) unsigned char tk_raw[sizeof(BTask)];
    __shared__ int tk_index;
    const BTask& tk = *reinterpret_cast<const BTask*>(tk_raw);
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
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
    if (!early_trigger) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

bool sweep_pdl() {
    static const bool on = std::getenv("MG_NO_PDL") == nullptr;
    return on;
}

template <int S, int P, bool AXI>
cudaError_t sweep_launch(const BTask* tasks, int ntasks, int total, const int* active, size_t smem, cudaStream_t s) {
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<S, P, AXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<S, P, AXI>, kSW, smem);
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
    return cudaLaunchKernelEx(&cfg, k_sweep<S, P, AXI>, tasks, ntasks, total, active, grid >= total ? 1 : 0);
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

}  // namespace

bool sweep_tile_ok(const Dims& D, int stencil, int prec, const int tile[3]) {
    const int vb = prec == PREC64 ? 8 : 4;
    const int TI = tile[0], TJ = tile[1], TK = tile[2];
    if (TI < 1 || TJ < 1 || TK < 1 || D.cut) return false;
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

cudaError_t encode_sweep_map(void* map, const void* x, const Dims& D, int stencil, int prec, const int tile[3]) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int vb = prec == PREC64 ? 8 : 4;
    const bool full = tile[2] == D.nph;
    const cuuint64_t dims[3] = {(cuuint64_t)D.nph, (cuuint64_t)D.nth, (cuuint64_t)D.nr};
    const cuuint64_t strides[2] = {(cuuint64_t)D.nph * vb, (cuuint64_t)D.nph * D.nth * vb};
    const cuuint32_t box[3] = {(cuuint32_t)(full ? D.nph : tile[2] + 2 * halo_cols(stencil, vb)),
                               (cuuint32_t)(tile[0] + 2 * halo_rows(stencil)), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(reinterpret_cast<CUtensorMap*>(map),
                          vb == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                          const_cast<void*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_sweep(const BTask* tasks, int ntasks, int total, const int* active, int stencil, bool axi,
                         int prec, size_t smem, cudaStream_t s) {
    if (ntasks <= 0 || total <= 0) return cudaSuccess;
    cudaError_t e;
    if (stencil == 7) {
        if (prec == PREC64) e = sweep_launch<7, PREC64, false>(tasks, ntasks, total, active, smem, s);
        else if (prec == PREC32) e = sweep_launch<7, PREC32, false>(tasks, ntasks, total, active, smem, s);
        else e = sweep_launch<7, PREC16, false>(tasks, ntasks, total, active, smem, s);
    } else if (axi) {
        if (prec == PREC64) e = sweep_launch<19, PREC64, true>(tasks, ntasks, total, active, smem, s);
        else if (prec == PREC32) e = sweep_launch<19, PREC32, true>(tasks, ntasks, total, active, smem, s);
        else e = sweep_launch<19, PREC16, true>(tasks, ntasks, total, active, smem, s);
    } else {
        if (prec == PREC64) e = sweep_launch<19, PREC64, false>(tasks, ntasks, total, active, smem, s);
        else if (prec == PREC32) e = sweep_launch<19, PREC32, false>(tasks, ntasks, total, active, smem, s);
        else e = sweep_launch<19, PREC16, false>(tasks, ntasks, total, active, smem, s);
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

// Vortex-grid transfer kernels shared by the regularization entry points and
// the tile-ordered vortex state (internal; every translation unit that
// includes it gets its own copies of these kernels).
#pragma once
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int BIN_THREADS = 256;
constexpr int BIN_UNROLL = 4;        // vortices per thread whose loads are issued together

// Per-vortex cell record (original order).  Mixed path: packed cell and the
// 32-bit cell fractions as fixed-point integers; FP64: cell and fractions.
template <typename T> struct Pos;
template <> struct __align__(16) Pos<float> {
    unsigned cell;        // ci | cj << 16
    unsigned fxw, fyw;    // fraction * 2^32 (truncated)
    float g;
};
template <> struct __align__(16) Pos<double> {
    int ci, cj;
    double fx, fy, g;
};
// Per-tile record: cell relative to the tile origin (lx, ly in [-2, 32]),
// fractions, Gamma and the vortex's original index q.  Mixed path: each
// fraction keeps 24 bits, fixed point, with the biased local cell lx + 2 in the
// low 8 bits of the same word (16 bytes in all, like the FP64 record's 32).
template <typename T> struct Rec;
template <> struct __align__(16) Rec<float> {
    unsigned xw, yw;      // (fraction * 2^32) & ~0xFF | (local cell + 2)
    float g;
    int q;
};
template <> struct __align__(16) Rec<double> {
    short lx, ly;
    int q;
    double fx, fy, g;
};

__device__ __forceinline__ int pos_ci(const Pos<float>& p) { return (int)(p.cell & 0xFFFFu); }
__device__ __forceinline__ int pos_cj(const Pos<float>& p) { return (int)(p.cell >> 16); }
__device__ __forceinline__ int pos_ci(const Pos<double>& p) { return p.ci; }
__device__ __forceinline__ int pos_cj(const Pos<double>& p) { return p.cj; }

__device__ __forceinline__ int rec_lx(const Rec<float>& r) { return (int)(r.xw & 0xFFu) - 2; }
__device__ __forceinline__ int rec_ly(const Rec<float>& r) { return (int)(r.yw & 0xFFu) - 2; }
__device__ __forceinline__ float rec_fx(const Rec<float>& r) { return __uint2float_rn(r.xw >> 8) * 0x1p-24f; }
__device__ __forceinline__ float rec_fy(const Rec<float>& r) { return __uint2float_rn(r.yw >> 8) * 0x1p-24f; }
__device__ __forceinline__ int rec_lx(const Rec<double>& r) { return r.lx; }
__device__ __forceinline__ int rec_ly(const Rec<double>& r) { return r.ly; }
__device__ __forceinline__ double rec_fx(const Rec<double>& r) { return r.fx; }
__device__ __forceinline__ double rec_fy(const Rec<double>& r) { return r.fy; }

__device__ __forceinline__ Rec<float> make_rec(const Pos<float>& p, int lx, int ly, int q) {
    Rec<float> r;
    r.xw = (p.fxw & ~0xFFu) | (unsigned)(lx + 2);
    r.yw = (p.fyw & ~0xFFu) | (unsigned)(ly + 2);
    r.g = p.g;
    r.q = q;
    return r;
}
__device__ __forceinline__ Rec<double> make_rec(const Pos<double>& p, int lx, int ly, int q) {
    Rec<double> r;
    r.lx = (short)lx;
    r.ly = (short)ly;
    r.q = q;
    r.fx = p.fx;
    r.fy = p.fy;
    r.g = p.g;
    return r;
}

// M4' weights of the four nodes floor(g)-1 .. floor(g)+2 for fractional part f
template <typename T>
__device__ __forceinline__ void m4p_weights(T f, T w[4]) {
    const T a0 = T(1) + f, a1 = f, a2 = T(1) - f, a3 = T(2) - f;
    w[0] = T(0.5) * (T(2) - a0) * (T(2) - a0) * (T(1) - a0);
    w[1] = T(1) - T(2.5) * a1 * a1 + T(1.5) * a1 * a1 * a1;
    w[2] = T(1) - T(2.5) * a2 * a2 + T(1.5) * a2 * a2 * a2;
    w[3] = T(0.5) * (T(2) - a3) * (T(2) - a3) * (T(1) - a3);
}

// Grid coordinate g of a position; the stencil floor(g)-1 .. floor(g)+2 lies in
// [0, n) iff 1 <= g < n - 2.  FP64 path: g = (X - x0)/dx, fraction g - floor(g)
// exact.  Mixed path: one FMA, then the integer and fractional parts are read
// from the bits of g (no further FP64 work); the fraction is truncated to 24 bits.
__device__ __forceinline__ bool split(double X, double x0, double dx, double, double, int n, long long, int& c,
                                      double& f) {
    const double g = (X - x0) / dx;
    if (!(g >= 1.0 && g < (double)(n - 2))) return false;
    const double fl = floor(g);
    c = (int)fl;
    f = g - fl;
    return true;
}
__device__ __forceinline__ bool split(double X, double, double, double inv_dx, double c0, int, long long lim, int& c,
                                      float& f) {
    const double g = fma(X, inv_dx, c0);
    // 1 <= g < n - 2 compared on the bit patterns (monotone for non-negative
    // doubles; negative values and NaN fail; lim = bits of (double)(n - 2)),
    // keeping the FP64 pipe for the FMA
    const long long gb = __double_as_longlong(g);
    if (gb < 0x3FF0000000000000ll || gb >= lim) return false;
    // g = 2^e (1 + m 2^-52), 0 <= e <= 10 since g < 2048: the integer part is the
    // top e fraction bits with the hidden bit, the cell fraction the next 32
    const unsigned hi = (unsigned)((unsigned long long)gb >> 32), lo = (unsigned)gb;
    const int e = (int)(hi >> 20) - 1023;
    const unsigned m20 = hi & 0xFFFFFu;
    c = (int)((m20 | 0x100000u) >> (20 - e));
    f = __uint2float_rz(__funnelshift_l(lo, m20, 12 + e)) * 0x1p-32f;
    return true;
}

// Mixed path of the binning passes: as split, but the cell fraction is returned
// as a 32-bit fixed-point integer (fraction * 2^32, truncated).
__device__ __forceinline__ bool split_fixed(double X, double inv_dx, double c0, long long lim, int& c, unsigned& fr) {
    const double g = fma(X, inv_dx, c0);
    const long long gb = __double_as_longlong(g);
    if (gb < 0x3FF0000000000000ll || gb >= lim) return false;
    const unsigned hi = (unsigned)((unsigned long long)gb >> 32), lo = (unsigned)gb;
    const int e = (int)(hi >> 20) - 1023;
    const unsigned m20 = hi & 0xFFFFFu;
    c = (int)((m20 | 0x100000u) >> (20 - e));
    fr = __funnelshift_l(lo, m20, 12 + e);
    return true;
}

// double -> float rounded to nearest even with integer instructions only (the
// FP64 pipe is 1/64 rate); zero, and values outside the normal FP32 range,
// take the hardware conversion.  Bitwise equal to (float)d.
__device__ __forceinline__ float d2f(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    if (e <= 0 || e >= 255) return (float)d;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;     // 52 fraction bits
    const unsigned top = (unsigned)(m >> 29);                // the 23 kept
    const unsigned rest = (unsigned)(m & 0x1FFFFFFFull);     // the 29 dropped
    unsigned out = sign | ((unsigned)e << 23) | top;
    if (rest > 0x10000000u || (rest == 0x10000000u && (top & 1u))) ++out;   // carries into the exponent
    return __uint_as_float(out);
}

__device__ __forceinline__ void make_pos(Pos<float>& p, int ci, int cj, unsigned fxw, unsigned fyw, double g) {
    p.cell = (unsigned)ci | ((unsigned)cj << 16);
    p.fxw = fxw;
    p.fyw = fyw;
    p.g = d2f(g);
}
__device__ __forceinline__ void make_pos(Pos<double>& p, int ci, int cj, double fx, double fy, double g) {
    p.ci = ci;
    p.cj = cj;
    p.fx = fx;
    p.fy = fy;
    p.g = g;
}

struct Geo {
    double x0, y0, dx;
    double inv_dx, cx, cy;     // 1/dx, -x0/dx, -y0/dx (host computed)
    double inv_dx2;            // 1/dx^2
    long long xlim, ylim;      // bit patterns of (double)(nx - 2), (double)(ny - 2)
    int nx, ny, ntx, ntiles;
};

// the split used by the locate pass: fixed-point fraction (mixed), exact (FP64)
__device__ __forceinline__ bool loc_split(double X, const Geo& g, int axis, int& c, unsigned& fr) {
    return split_fixed(X, g.inv_dx, axis ? g.cy : g.cx, axis ? g.ylim : g.xlim, c, fr);
}
__device__ __forceinline__ bool loc_split(double X, const Geo& g, int axis, int& c, double& f) {
    return split(X, axis ? g.y0 : g.x0, g.dx, 0.0, 0.0, axis ? g.ny : g.nx, 0, c, f);
}
template <typename T> using Frac = typename std::conditional<sizeof(T) == 4, unsigned, double>::type;

// The vortex count and block span of a binning pass: the launch's own, or,
// when dn is given (a captured step replayed at a growing count), dn[0] with
// the span bin_span computes for it; blocks past the count bin nothing.
// (max_blocks: the launch's partition mode, BIN_MAX_BLOCKS or BIN_WIDE_BLOCKS,
// chosen on the host for the capacity.)
__device__ __forceinline__ void bin_count(const int64_t* dn, int min_span, int max_blocks, int64_t& nv,
                                          int64_t& span) {
    if (!dn) return;
    nv = *dn;
    const int64_t s = (nv + max_blocks - 1) / max_blocks;
    span = s < min_span ? min_span : s;
}

template <typename T, int TILE, int NT>
__global__ void __launch_bounds__(NT) k_locate(const double* __restrict__ X, const double* __restrict__ Y,
                                                       const double* __restrict__ G, int64_t nv, int64_t span,
                                                       const int64_t* __restrict__ dn, int min_span, int max_blocks, Geo geo,
                                                       Pos<T>* __restrict__ pos, int* __restrict__ hist,
                                                       double* __restrict__ gmax_blk, int* __restrict__ status,
                                                       unsigned long long* __restrict__ oob, T* __restrict__ zu,
                                                       T* __restrict__ zv) {
    extern __shared__ unsigned sm[];
    __shared__ T wmax[NT / 32];
    unsigned* cnt = sm;
    T gm = T(0);          // in the record's precision: no FP64 instruction per vortex in the mixed path
    for (int i = threadIdx.x; i < geo.ntiles; i += NT) cnt[i] = 0u;
    pdl_wait();
    bin_count(dn, min_span, max_blocks, nv, span);
    __syncthreads();
    const int64_t lo = (int64_t)blockIdx.x * span;
    const int64_t hi = lo + span < nv ? lo + span : nv;
    int bad = 0;
    for (int64_t base = lo; base < hi; base += NT * BIN_UNROLL) {
        // issue the loads of BIN_UNROLL vortices before using any of them
        double xs[BIN_UNROLL], ys[BIN_UNROLL], gs[BIN_UNROLL];
#pragma unroll
        for (int k = 0; k < BIN_UNROLL; ++k) {   // clamped: a thread past the end reloads the last vortex
            int64_t q = base + k * NT + threadIdx.x;
            q = q < hi ? q : hi - 1;
            xs[k] = X[q];
            ys[k] = Y[q];
            gs[k] = G[q];
        }
#pragma unroll
        for (int k = 0; k < BIN_UNROLL; ++k) {
            const int64_t q = base + k * NT + threadIdx.x;
            if (q >= hi) break;
            int ci = 0, cj = 0;
            Frac<T> fx = 0, fy = 0;
            Pos<T> p;
            if (!loc_split(xs[k], geo, 0, ci, fx) || !loc_split(ys[k], geo, 1, cj, fy)) {
                ++bad;
                make_pos(p, 0xFFFF, 0xFFFF, Frac<T>(0), Frac<T>(0), 0.0);   // marker: skipped by scatter
                pos[q] = p;
                if (zu) {                             // no E_v record: its velocity is zero
                    zu[q] = T(0);
                    zv[q] = T(0);
                }
                continue;
            }
            make_pos(p, ci, cj, fx, fy, gs[k]);
            pos[q] = p;
            gm = fmax(gm, (T)fabs(p.g));           // |Gamma| as the record carries it
            const int tx0 = (ci - 1) / TILE, tx1 = (ci + 2) / TILE;
            const int ty0 = (cj - 1) / TILE, ty1 = (cj + 2) / TILE;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&cnt[ty * geo.ntx + tx], 1u);
        }
    }
    if (bad) {
        atomicAdd(oob, (unsigned long long)bad);
        atomicOr(status, ST_OUT_OF_DOMAIN);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = T(0);
        for (int i = 0; i < NT / 32; ++i) m = fmax(m, wmax[i]);
        gmax_blk[blockIdx.x] = (double)m;
    }
    int* row = hist + (size_t)blockIdx.x * geo.ntiles;
    for (int i = threadIdx.x; i < geo.ntiles; i += NT) row[i] = (int)cnt[i];
}

// Fixed-point exponent of a tile: every node sum is bounded by
// count * max|Gamma| < 2^e and is scaled to stay below 2^61.
__device__ __forceinline__ int tile_shift_of(unsigned count, double gmax) {
    const double bound = (double)count * gmax;
    int e = 0;
    if (bound > 0.0) frexp(bound, &e);
    const int sh = 61 - e;
    return sh > 100 ? 100 : (sh < -60 ? -60 : sh);
}

// k_offsets: a block covers OFF_TILES tiles; its OFF_SEGS x OFF_TILES threads
// each own a run of at most OFF_RUN consecutive vortex blocks of one tile.
constexpr int OFF_TILES = 8, OFF_SEGS = 128, OFF_RUN = 5;
static_assert(OFF_SEGS * OFF_RUN >= BIN_MAX_BLOCKS && BIN_MAX_BLOCKS <= 1024, "k_offsets covers every block");
static_assert(OFF_TILES * OFF_SEGS == 1024, "k_offsets runs 1024 threads");

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Per-tile totals and per-(block, tile) offsets within the tile: tile_count
// and, in place over the block histograms, off[b][t] = sum_{b' < b} hist[b'][t].
// Blocks are independent (the tiles' first slots are added by the scatter pass).
__global__ void __launch_bounds__(1024) k_offsets(int ntiles, int nb, int* __restrict__ hist_off,
                                                  unsigned* __restrict__ tile_count, const double* __restrict__ gmax_blk,
                                                  double* __restrict__ gmax_all) {
    __shared__ int part[OFF_SEGS][OFF_TILES + 1];
    __shared__ double wmax[32];
    const int tx = threadIdx.x % OFF_TILES, ty = threadIdx.x / OFF_TILES;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int t0 = blockIdx.x * OFF_TILES, t = t0 + tx;
    const int S = (nb + OFF_SEGS - 1) / OFF_SEGS;   // <= OFF_RUN
    const int b0 = ty * S;
    pdl_wait();
    // block 0: the largest |Gamma| over the locate blocks, one load a thread
    // (nb <= 1024), issued with the histogram loads and reduced after them
    double gm = blockIdx.x == 0 && (int)threadIdx.x < nb ? gmax_blk[threadIdx.x] : 0.0;
    int v[OFF_RUN];
    int seg = 0;
#pragma unroll
    for (int k = 0; k < OFF_RUN; ++k) {              // all loads in flight together (clamped index)
        const bool in = k < S && b0 + k < nb && t < ntiles;
        v[k] = nb > 0 ? hist_off[in ? (size_t)(b0 + k) * ntiles + t : 0] : 0;
        v[k] = in ? v[k] : 0;
        seg += v[k];
    }
    if (blockIdx.x == 0) {                           // block-uniform
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if (lane == 0) wmax[wid] = gm;
    }
    part[ty][tx] = seg;
    __syncthreads();
    if (blockIdx.x == 0 && wid == OFF_TILES) {       // OFF_TILES < 32: a warp that scans nothing
        double m = wmax[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) *gmax_all = m;
    }
    if (wid < OFF_TILES) {                            // exclusive scan over the runs of tile t0 + wid
        const int a0 = part[4 * lane][wid], a1 = part[4 * lane + 1][wid];
        const int a2 = part[4 * lane + 2][wid], a3 = part[4 * lane + 3][wid];
        const int sum4 = a0 + a1 + a2 + a3;
        const int incl = warp_incl_scan(sum4, lane);
        const int ex = incl - sum4;
        part[4 * lane][wid] = ex;
        part[4 * lane + 1][wid] = ex + a0;
        part[4 * lane + 2][wid] = ex + a0 + a1;
        part[4 * lane + 3][wid] = ex + a0 + a1 + a2;
        if (lane == 31 && t0 + wid < ntiles) tile_count[t0 + wid] = (unsigned)incl;
    }
    __syncthreads();
    if (t < ntiles) {
        int run = part[ty][tx];
#pragma unroll
        for (int k = 0; k < OFF_RUN; ++k) {
            if (k < S && b0 + k < nb) hist_off[(size_t)(b0 + k) * ntiles + t] = run;
            run += v[k];
        }
    }
}

// Every block scans the tile totals itself (block 0 publishes the tiles' first
// slots for the deposit and interpolation passes), adds them to its offsets
// and places its records.
constexpr int SCAN_PER = 16;     // tiles per thread in the block scan: 256 * 16 = 64 * 64 tiles at most
// vortices a thread loads at a time: at 1024 threads the eight FP32 records
// spill (64 registers at most), so four (FP64: four and two)
template <typename T, int NT> struct ScatterUnroll {
    static constexpr int value = (sizeof(T) == 4 ? 8 : 4) / (NT == 1024 ? 2 : 1);
};
static_assert((2048 / BIN_TILE) * (2048 / BIN_TILE) <= BIN_THREADS * SCAN_PER, "scan covers every tile");
constexpr int MAX_SCAN_TILES = BIN_THREADS * SCAN_PER;   // smaller tiles are offered only up to this count

template <typename T, int TILE, int NT>
__global__ void __launch_bounds__(NT, NT == 1024 ? 1 : 4) k_scatter(const Pos<T>* __restrict__ pos, int64_t nv, int64_t span,
                                                        const int64_t* __restrict__ dn, int min_span, int max_blocks,
                                                        Geo geo, const int* __restrict__ off,
                                                        const unsigned* __restrict__ tile_count,
                                                        int* __restrict__ tile_start, Rec<T>* __restrict__ recs,
                                                        int64_t rec_cap, int* __restrict__ status) {
    extern __shared__ unsigned sm[];
    __shared__ int wsum[NT / 32];
    unsigned* cnt = sm;
    int* first = (int*)(sm + geo.ntiles);
    pdl_wait();
    bin_count(dn, min_span, max_blocks, nv, span);
    const int64_t lo = (int64_t)blockIdx.x * span;
    const int64_t hi = lo + span < nv ? lo + span : nv;
    // this thread's first records (in flight during the scan)
    Pos<T> p[ScatterUnroll<T, NT>::value];
#pragma unroll
    for (int k = 0; k < ScatterUnroll<T, NT>::value; ++k) {     // clamped loads; past the end: no vortex
        const int64_t q = lo + k * NT + threadIdx.x;
        p[k] = pos[q < hi ? q : (hi > 0 ? hi - 1 : 0)];
        if (q >= hi) make_pos(p[k], 0xFFFF, 0xFFFF, Frac<T>(0), Frac<T>(0), 0.0);
    }
    // exclusive scan of tile_count: thread i owns tiles [i * per, i * per + per)
    const int per = (geo.ntiles + NT - 1) / NT;   // <= SCAN_PER
    const int t0 = threadIdx.x * per;
    int mine = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k)
        if (k < per && t0 + k < geo.ntiles) mine += (int)tile_count[t0 + k];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int run = incl - mine;
    for (int w = 0; w < wid; ++w) run += wsum[w];
    const int* row = off + (size_t)blockIdx.x * geo.ntiles;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        const int i = t0 + k;
        if (k < per && i < geo.ntiles) {
            cnt[i] = 0u;
            first[i] = run + row[i];
            if (blockIdx.x == 0) tile_start[i] = run;
            run += (int)tile_count[i];
        }
    }
    __syncthreads();
    for (int64_t base = lo; base < hi; base += NT * ScatterUnroll<T, NT>::value) {
        if (base != lo) {
#pragma unroll
            for (int k = 0; k < ScatterUnroll<T, NT>::value; ++k) {     // loads first (clamped)
                const int64_t q = base + k * NT + threadIdx.x;
                p[k] = pos[q < hi ? q : hi - 1];
                if (q >= hi) make_pos(p[k], 0xFFFF, 0xFFFF, Frac<T>(0), Frac<T>(0), 0.0);
            }
        }
#pragma unroll
        for (int k = 0; k < ScatterUnroll<T, NT>::value; ++k) {
            const int ci = pos_ci(p[k]), cj = pos_cj(p[k]);
            if (ci == 0xFFFF) continue;
            const int64_t q = base + k * NT + threadIdx.x;
            const int tx0 = (ci - 1) / TILE, tx1 = (ci + 2) / TILE;
            const int ty0 = (cj - 1) / TILE, ty1 = (cj + 2) / TILE;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) {
                    const int t = ty * geo.ntx + tx;
                    const int slot = first[t] + (int)atomicAdd(&cnt[t], 1u);
                    if (slot < 0 || slot >= rec_cap) {      // counts and histograms disagree
                        atomicOr(status, ST_INTERNAL);
                        continue;
                    }
                    recs[slot] = make_rec(p[k], ci - tx * TILE, cj - ty * TILE, (int)q);
                }
        }
    }
}

// fixed-point scale 2^sh as a floating-point number, sh in [-60, 100]
template <typename T> __device__ __forceinline__ T pow2(int sh);
template <> __device__ __forceinline__ float pow2<float>(int sh) { return __int_as_float((sh + 127) << 23); }
template <> __device__ __forceinline__ double pow2<double>(int sh) { return __longlong_as_double((long long)(sh + 1023) << 52); }

// x = hi * 2^16 + lo + e, |lo| <= 2^15, |e| <= 1/2, for |x| < 2^38, with FP32
// adds only (no conversion instructions, which issue at 1/8 rate): adding
// 1.5 * 2^39 rounds x to a multiple of 2^16 (h), x - h is exact, and adding
// 1.5 * 2^23 to an integer-valued (or rounded) float of magnitude < 2^22 leaves
// it in the low mantissa bits.
__device__ __forceinline__ void split_hilo(float x, int& hi, int& lo) {
    const float h = __fsub_rn(__fadd_rn(x, 0x1.8p39f), 0x1.8p39f);
    const float l = __fsub_rn(x, h);
    hi = __float_as_int(__fmaf_rn(h, 0x1p-16f, 0x1.8p23f)) - 0x4B400000;
    lo = __float_as_int(__fadd_rn(l, 0x1.8p23f)) - 0x4B400000;
}

// Deposit: one block per node tile accumulates its records in shared memory as
// fixed-point integers.  FP32 path: each term v 2^sh, rounded to an integer
// hi 2^16 + lo, goes into two native 32-bit shared adds (exact while the tile
// has fewer than 65536 records and |sum| < 2^38); otherwise, and for FP64, one
// 64-bit add.  Integer sums are exact, so the result does not depend on the
// order of the adds.  The scale bounds every node sum by the tile's record
// count times the largest |Gamma| of the whole regularization (reduced by
// k_offsets from the locate blocks' maxima).  (A one-add variant with a
// node-window bound measured no faster and lost seven bits on clustered
// vortices; shared adds are not what bounds this kernel.)
//
// A record's local cell (lx, ly) lies in [-2, TILE], so its nodes lie in
// [-3, TILE + 2]: the accumulator covers that range (acc_w^2 nodes) and the
// adds need no bounds tests; only the tile's own TILE x TILE nodes are written
// out.
constexpr int ACC_HALO = 3;
template <int TILE> struct AccW { static constexpr int value = TILE + 6; };

enum { DEP_SPLIT32 = 0, DEP_F32_64 = 1, DEP_F64_64 = 2 };

template <int MODE, int ACC_W, typename T>
__device__ __forceinline__ void deposit_one(const Rec<T>& rc, T scale, unsigned long long* acc) {
    int* acc_hi = reinterpret_cast<int*>(acc);
    int* acc_lo = reinterpret_cast<int*>(acc) + ACC_W * ACC_W;
    T wx[4], wy[4];
    m4p_weights<T>(rec_fx(rc), wx);
    m4p_weights<T>(rec_fy(rc), wy);
    const T gs = rc.g * scale;
    const int base = (rec_ly(rc) - 1 + ACC_HALO) * ACC_W + (rec_lx(rc) - 1 + ACC_HALO);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const T gy = gs * wy[b];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int node = base + b * ACC_W + a;
            const T x = gy * wx[a];
            if (MODE == DEP_SPLIT32) {
                int hi, lo;
                split_hilo((float)x, hi, lo);
                atomicAdd(&acc_hi[node], hi);
                atomicAdd(&acc_lo[node], lo);
            } else if (MODE == DEP_F32_64) {
                atomicAdd(&acc[node], (unsigned long long)__float2ll_rn((float)x));
            } else {
                atomicAdd(&acc[node], (unsigned long long)__double2ll_rn((double)x));
            }
        }
    }
}

// U records per thread at a time, the next U loaded while these are used (a
// thread past the end reloads the last record, which it then skips)
constexpr int REC_U = 4;
template <typename T, int U>
__device__ __forceinline__ void load_recs(const Rec<T>* __restrict__ recs, int r0, int cnt, Rec<T> (&rc)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int r = r0 + u * (int)blockDim.x + (int)threadIdx.x;
        rc[u] = recs[r < cnt ? r : cnt - 1];
    }
}

// every record of the tile; rc holds this thread's first REC_U (load_recs at 0)
template <int MODE, int ACC_W, typename T>
__device__ __forceinline__ void deposit_records(const Rec<T>* __restrict__ recs, int cnt, T scale,
                                                unsigned long long* acc, Rec<T> (&rc)[REC_U]) {
    const int stride = REC_U * (int)blockDim.x;
    for (int r0 = 0; r0 < cnt; r0 += stride) {
        Rec<T> cur[REC_U];
#pragma unroll
        for (int u = 0; u < REC_U; ++u) cur[u] = rc[u];
        if (r0 + stride < cnt) load_recs(recs, r0 + stride, cnt, rc);
#pragma unroll
        for (int u = 0; u < REC_U; ++u)
            if (r0 + u * (int)blockDim.x + (int)threadIdx.x < cnt) deposit_one<MODE, ACC_W, T>(cur[u], scale, acc);
    }
}

// Split-32 deposit in bank order.  The shared adds of one warp instruction
// (the same stencil term of 32 records) conflict when two lanes' records put
// their stencils' first nodes in the same bank, which for records in random
// cells costs about 3.7 passes an add.  So each chunk of REC_U x blockDim
// records is first counting-sorted by that bank (one shared add a record
// into 32 counters), and lane l of row i takes sorted record l R + i (R rows
// of 32 in the chunk): the lanes of a row lie about one bucket, so one bank,
// apart.  The chunk is stored transposed (sorted record l R + i in slot
// 32 i + l) so a row reads 32 consecutive records.  Only the order of the
// integer adds changes, so the sums are those of the unsorted deposit.
constexpr int DEP_MAX_THREADS = 256;
constexpr int DEP_SORT_MIN = 256;     // fewer records: too few adds for the sort's three barriers to pay
constexpr int DEP_SORT_SLOTS = REC_U * DEP_MAX_THREADS + 32;

template <int ACC_W, typename T>
__device__ __forceinline__ void deposit_records_banked(const Rec<T>* __restrict__ recs, int cnt, T scale,
                                                       unsigned long long* acc, Rec<T> (&rc)[REC_U],
                                                       Rec<T>* srt, int* bcnt, int* bstart) {
    const int stride = REC_U * (int)blockDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
    for (int r0 = 0; r0 < cnt; r0 += stride) {
        const int n = cnt - r0 < stride ? cnt - r0 : stride;
        const int R = (n + 31) >> 5;
        int bank[REC_U], pos[REC_U];
#pragma unroll
        for (int u = 0; u < REC_U; ++u) {
            const int r = u * (int)blockDim.x + (int)threadIdx.x;     // index within the chunk
            bank[u] = ((rec_ly(rc[u]) - 1 + ACC_HALO) * ACC_W + (rec_lx(rc[u]) - 1 + ACC_HALO)) & 31;
            pos[u] = r < n ? atomicAdd(&bcnt[bank[u]], 1) : 0;
        }
        __syncthreads();
        if (wid == 0) {                               // bucket starts; counters cleared for the next chunk
            const int c = bcnt[lane];
            bstart[lane] = warp_incl_scan(c, lane) - c;
            bcnt[lane] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < REC_U; ++u) {
            const int r = u * (int)blockDim.x + (int)threadIdx.x;
            if (r < n) {
                const int idx = bstart[bank[u]] + pos[u];
                srt[(idx % R) * 32 + idx / R] = rc[u];
            }
        }
        if (r0 + stride < cnt) load_recs(recs, r0 + stride, cnt, rc);   // the next chunk in flight
        __syncthreads();
        for (int i = wid; i < R; i += nw)
            if (lane * R + i < n) deposit_one<DEP_SPLIT32, ACC_W, T>(srt[i * 32 + lane], scale, acc);
        __syncthreads();                              // srt and the counters are reused
    }
}

template <typename T, int TILE>
__global__ void __launch_bounds__(256) k_deposit(const Rec<T>* __restrict__ recs, const int* __restrict__ tile_start,
                                                 const unsigned* __restrict__ tile_count,
                                                 const double* __restrict__ gmax_all, Geo geo, T* __restrict__ w,
                                                 int64_t rec_cap, int* __restrict__ status) {
    constexpr int ACC_W = AccW<TILE>::value;
    __shared__ unsigned long long acc[ACC_W * ACC_W];
    __shared__ Rec<T> srt[sizeof(T) == 4 ? DEP_SORT_SLOTS : 1];   // the bank-ordered chunk (mixed path)
    __shared__ int bcnt[32], bstart[32];
    const int t = blockIdx.x;
    const int tx = t % geo.ntx, ty = t / geo.ntx;
    for (int i = threadIdx.x; i < ACC_W * ACC_W; i += blockDim.x) acc[i] = 0ull;
    if (threadIdx.x < 32) bcnt[threadIdx.x] = 0;
    pdl_wait();
    int start = tile_start[t], cnt = (int)tile_count[t];
    if (start < 0 || cnt < 0 || (int64_t)start + cnt > rec_cap) {     // block-uniform
        if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
        start = cnt = 0;
    }
    Rec<T> rc[REC_U];
    if (cnt > 0) load_recs(recs + start, 0, cnt, rc);               // in flight across the barrier
    const bool split32 = sizeof(T) == 4 && cnt < 65536;
    const int sh = tile_shift_of((unsigned)cnt, *gmax_all) - (split32 ? 23 : 0);   // 2^61 -> 2^38 when split
    const T scale = pow2<T>(sh);
    __syncthreads();
    if (sizeof(T) == 8) deposit_records<DEP_F64_64, ACC_W>(recs + start, cnt, scale, acc, rc);
    else if (split32 && cnt >= DEP_SORT_MIN)        // block-uniform
        deposit_records_banked<ACC_W>(recs + start, cnt, scale, acc, rc, srt, bcnt, bstart);
    else if (split32) deposit_records<DEP_SPLIT32, ACC_W>(recs + start, cnt, scale, acc, rc);
    else deposit_records<DEP_F32_64, ACC_W>(recs + start, cnt, scale, acc, rc);
    __syncthreads();
    const int* acc_hi = reinterpret_cast<const int*>(acc);
    const int* acc_lo = reinterpret_cast<const int*>(acc) + ACC_W * ACC_W;
    const float inv_dx2f = (float)geo.inv_dx2;
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
        const int lx = i % TILE, ly = i / TILE;
        const int gi = tx * TILE + lx, gj = ty * TILE + ly;
        const int node = (ly + ACC_HALO) * ACC_W + lx + ACC_HALO;
        if (gi < geo.nx && gj < geo.ny) {
            long long a;
            if (split32) a = (long long)acc_hi[node] * 65536ll + (long long)acc_lo[node];
            else a = (long long)acc[node];
            T v;
            if (sizeof(T) == 4) v = (T)(__ll2float_rn(a) * pow2<float>(-sh) * inv_dx2f);
            else v = (T)(ldexp((double)a, -sh) * geo.inv_dx2);
            w[(size_t)gj * geo.nx + gi] = v;
        }
    }
}

template <typename T>
__device__ __forceinline__ void gather16(const T* __restrict__ uv, int nx, int ci, int cj, T fx, T fy, T& su, T& sv) {
    T wx[4], wy[4];
    m4p_weights<T>(fx, wx);
    m4p_weights<T>(fy, wy);
    su = 0;
    sv = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const T* row = uv + 2 * ((size_t)(cj - 1 + b) * nx + (ci - 1));
        T ru = 0, rv = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            ru += wx[a] * row[2 * a];
            rv += wx[a] * row[2 * a + 1];
        }
        su += wy[b] * ru;
        sv += wy[b] * rv;
    }
}

// E_v at the vortices of the last regularization, in tile order: one block per
// tile stages the (u, v) nodes its resident vortices can touch (the tile plus
// one node before and two after, per direction) in shared memory, then every
// record whose cell lies in the tile (each vortex has exactly one such record)
// gathers its 4x4 stencil there and writes its result at its original index.
template <typename T, int TILE>
__global__ void __launch_bounds__(256) k_interp_tiles(const Rec<T>* __restrict__ recs,
                                                      const int* __restrict__ tile_start,
                                                      const unsigned* __restrict__ tile_count, const C_t<T>* __restrict__ uv,
                                                      Geo geo, T* __restrict__ uq, T* __restrict__ vq, int64_t rec_cap,
                                                      int64_t nq, int* __restrict__ status) {
    using C = C_t<T>;
    constexpr int PATCH = TILE + 3;
    __shared__ C patch[PATCH * PATCH];
    const int t = blockIdx.x;
    pdl_wait();
    const int cnt = (int)tile_count[t];
    if (cnt == 0) return;
    const int start = tile_start[t];
    if (start < 0 || cnt < 0 || (int64_t)start + cnt > rec_cap) {     // block-uniform
        if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
        return;
    }
    const int tx = t % geo.ntx, ty = t / geo.ntx;
    const int gi0 = tx * TILE - 1, gj0 = ty * TILE - 1;
    for (int i = threadIdx.x; i < PATCH * PATCH; i += blockDim.x) {
        const int gi = gi0 + i % PATCH, gj = gj0 + i / PATCH;
        C v = cmake<C>(T(0), T(0));
        if (gi >= 0 && gi < geo.nx && gj >= 0 && gj < geo.ny) v = uv[(size_t)gj * geo.nx + gi];
        patch[i] = v;
    }
    __syncthreads();
    constexpr int U = 4;
    for (int r0 = 0; r0 < cnt; r0 += U * blockDim.x) {
        Rec<T> rc[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {           // loads first (clamped index)
            const int r = r0 + u * blockDim.x + threadIdx.x;
            ok[u] = r < cnt;
            rc[u] = recs[start + (ok[u] ? r : cnt - 1)];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!ok[u]) continue;
            const int lx = rec_lx(rc[u]), ly = rec_ly(rc[u]);
            if (lx < 0 || lx >= TILE || ly < 0 || ly >= TILE) continue;  // not home
            T wx[4], wy[4];
            m4p_weights<T>(rec_fx(rc[u]), wx);
            m4p_weights<T>(rec_fy(rc[u]), wy);
            T su = 0, sv = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const C* row = patch + (ly + b) * PATCH + lx;    // node (lx - 1 + a, ly - 1 + b)
                T ru = 0, rv = 0;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const C c = row[a];
                    ru += wx[a] * c.x;
                    rv += wx[a] * c.y;
                }
                su += wy[b] * ru;
                sv += wy[b] * rv;
            }
            if (rc[u].q < 0 || rc[u].q >= nq) {
                atomicOr(status, ST_INTERNAL);
                continue;
            }
            uq[rc[u].q] = su;
            vq[rc[u].q] = sv;
        }
    }
}

// FP32 variant of k_interp_tiles that reads each stencil row with two 16-byte
// shared loads: the patch is staged twice as node pairs, starting at even and
// at odd local x, so that the four nodes px .. px + 3 of a row are the pairs
// E[px / 2], E[px / 2 + 1] (px even) or O[(px - 1) / 2], O[(px + 1) / 2].
//
// The home records of each chunk of REC_U x blockDim records are counting-
// sorted by the shared-memory bank of their first patch row (as the deposit's
// records are, same transposed layout), so the eight lanes of each quarter-
// warp, whose 16-byte loads are served together, read eight different bank
// groups; non-home records (a vortex's other tiles) drop out in the same pass.
// U records a thread a chunk.  Dynamic shared memory: (U x blockDim + 32)
// records.
template <int TILE, int U>
__global__ void __launch_bounds__(256) k_interp_tiles_f32(const Rec<float>* __restrict__ recs,
                                                          const int* __restrict__ tile_start,
                                                          const unsigned* __restrict__ tile_count,
                                                          const float2* __restrict__ uv, Geo geo,
                                                          float* __restrict__ uq, float* __restrict__ vq,
                                                          int64_t rec_cap, int64_t nq, int* __restrict__ status) {
    constexpr int PATCH = TILE + 3, PAIRS = (PATCH + 1) / 2;   // 18 pairs per patch row at TILE 32
    __shared__ float4 pe[PATCH * PAIRS];
    __shared__ float4 po[PATCH * PAIRS];
    __shared__ int bcnt[32], bstart[32], nhome;
    extern __shared__ __align__(16) unsigned char interp_dyn[];
    Rec<float>* srt = reinterpret_cast<Rec<float>*>(interp_dyn);
    const int t = blockIdx.x;
    pdl_wait();
    const int cnt = (int)tile_count[t];
    if (cnt == 0) return;
    const int start = tile_start[t];
    if (start < 0 || cnt < 0 || (int64_t)start + cnt > rec_cap) {     // block-uniform
        if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
        return;
    }
    Rec<float> rc[U];
    load_recs(recs + start, 0, cnt, rc);          // in flight while the patch is staged
    if (threadIdx.x < 32) bcnt[threadIdx.x] = 0;
    const int tx = t % geo.ntx, ty = t / geo.ntx;
    const int gi0 = tx * TILE - 1, gj0 = ty * TILE - 1;
    // patch nodes px, py in [0, 2 PAIRS) x [0, PATCH); px = 2 PAIRS - 1 only pads
    for (int i = threadIdx.x; i < PATCH * 2 * PAIRS; i += blockDim.x) {
        const int px = i % (2 * PAIRS), py = i / (2 * PAIRS);
        const int gi = gi0 + px, gj = gj0 + py;
        float2 v = make_float2(0.f, 0.f);
        if (px < PATCH && gi >= 0 && gi < geo.nx && gj >= 0 && gj < geo.ny) v = uv[(size_t)gj * geo.nx + gi];
        float* e = reinterpret_cast<float*>(&pe[py * PAIRS + px / 2]) + 2 * (px & 1);
        e[0] = v.x;
        e[1] = v.y;
        if (px >= 1) {
            float* o = reinterpret_cast<float*>(&po[py * PAIRS + (px - 1) / 2]) + 2 * ((px - 1) & 1);
            o[0] = v.x;
            o[1] = v.y;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
    const int stride = U * (int)blockDim.x;
    for (int r0 = 0; r0 < cnt; r0 += stride) {
        const int n = cnt - r0 < stride ? cnt - r0 : stride;
        int key[U], pos[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int lx = rec_lx(rc[u]), ly = rec_ly(rc[u]);
            const bool home = u * (int)blockDim.x + (int)threadIdx.x < n && lx >= 0 && lx < TILE && ly >= 0 &&
                              ly < TILE;
            const float4* row = ((lx & 1) ? po + (lx - 1) / 2 : pe + lx / 2) + ly * PAIRS;
            key[u] = home ? (int)((__cvta_generic_to_shared(row) >> 4) & 31) : -1;
            pos[u] = home ? atomicAdd(&bcnt[key[u]], 1) : 0;
        }
        __syncthreads();
        if (wid == 0) {                               // bucket starts; counters cleared for the next chunk
            const int c = bcnt[lane];
            const int incl = warp_incl_scan(c, lane);
            bstart[lane] = incl - c;
            bcnt[lane] = 0;
            if (lane == 31) nhome = incl;
        }
        __syncthreads();
        const int nh = nhome, R = (nh + 31) >> 5;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (key[u] >= 0) {
                const int idx = bstart[key[u]] + pos[u];
                srt[(idx % R) * 32 + idx / R] = rc[u];
            }
        }
        if (r0 + stride < cnt) load_recs(recs + start, r0 + stride, cnt, rc);   // the next chunk in flight
        __syncthreads();
        for (int i = wid; i < R; i += nw) {
            if (lane * R + i >= nh) continue;
            const Rec<float> rcu = srt[i * 32 + lane];
            const int lx = rec_lx(rcu), ly = rec_ly(rcu);
            float wx[4], wy[4];
            m4p_weights<float>(rec_fx(rcu), wx);
            m4p_weights<float>(rec_fy(rcu), wy);
            const float4* rows = (lx & 1) ? po + (lx - 1) / 2 : pe + lx / 2;   // node px = lx is the first
            float su = 0.f, sv = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float4 p0 = rows[(ly + b) * PAIRS], p1 = rows[(ly + b) * PAIRS + 1];
                const float ru = wx[0] * p0.x + wx[1] * p0.z + wx[2] * p1.x + wx[3] * p1.z;
                const float rv = wx[0] * p0.y + wx[1] * p0.w + wx[2] * p1.y + wx[3] * p1.w;
                su += wy[b] * ru;
                sv += wy[b] * rv;
            }
            if (rcu.q < 0 || rcu.q >= nq) {
                atomicOr(status, ST_INTERNAL);
                continue;
            }
            uq[rcu.q] = su;
            vq[rcu.q] = sv;
        }
        __syncthreads();                              // srt and the counters are reused
    }
}

// E_v at arbitrary points
template <typename T>
__global__ void k_interp_xy(const T* __restrict__ uv, const double* __restrict__ X, const double* __restrict__ Y,
                            int64_t nq, Geo geo, T* __restrict__ uq, T* __restrict__ vq, int* __restrict__ status,
                            unsigned long long* __restrict__ oob) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        int ci = 0, cj = 0;
        T fx = 0, fy = 0;
        T su = 0, sv = 0;
        if (split(X[q], geo.x0, geo.dx, geo.inv_dx, geo.cx, geo.nx, geo.xlim, ci, fx) &&
            split(Y[q], geo.y0, geo.dx, geo.inv_dx, geo.cy, geo.ny, geo.ylim, cj, fy)) {
            gather16<T>(uv, geo.nx, ci, cj, fx, fy, su, sv);
        } else {
            atomicAdd(oob, 1ull);
            atomicOr(status, ST_OUT_OF_DOMAIN);
        }
        uq[q] = su;
        vq[q] = sv;
    }
}

// Scratch used by one regularization: owned by a plan, or carved from the
// static array of the allocation-free entry point.
struct BinWork {
    int* status;
    unsigned long long* oob;
    unsigned* tile_count;     // written by k_offsets
    double* gmax;             // [0]: largest |Gamma| (k_offsets); [1 + b]: that of locate block b
    int* tile_start;
    int* bin_off;             // bin_blocks(nv) * ntiles
    void* pos;
    void* recs;
    int64_t rec_cap;          // record slots in recs
    void* zu = nullptr;       // optional E_v outputs (plan precision): zeroed for every vortex off the grid
    void* zv = nullptr;
};

inline Geo make_geo(int nx, int ny, double dx, double x0, double y0, int tile = BIN_TILE) {
    Geo g;
    g.x0 = x0; g.y0 = y0; g.dx = dx; g.nx = nx; g.ny = ny;
    g.inv_dx = 1.0 / dx;
    g.cx = -x0 / dx;
    g.cy = -y0 / dx;
    g.inv_dx2 = 1.0 / (dx * dx);
    const double lx = (double)(nx - 2), ly = (double)(ny - 2);
    memcpy(&g.xlim, &lx, sizeof(double));
    memcpy(&g.ylim, &ly, sizeof(double));
    g.ntx = ceil_div(nx, tile);
    g.ntiles = g.ntx * ceil_div(ny, tile);
    return g;
}

// Bin nv vortices by tile (locate, offsets, scatter) into bw; `p` (may be
// null) only supplies the timing records and the error text.
// With dn (device count, see bin_count), nv is the capacity the launch is sized for.
template <typename T, int TILE, int NT>
pf_status bin_launch_nt(pf_plan p, const Geo& geo, const BinWork& bw, const double* X, const double* Y,
                        const double* G, int64_t nv, cudaStream_t s, int min_span, const int64_t* dn) {
    const int nb = bin_blocks(nv, min_span);
    const int64_t span = bin_span(nv, min_span);
    const int mb = bin_max_blocks(nv);
    const size_t sh_loc = (size_t)geo.ntiles * sizeof(unsigned);
    const size_t sh_sc = 2 * (size_t)geo.ntiles * sizeof(unsigned);
    if (set_smem(k_locate<T, TILE, NT>, sh_loc) != cudaSuccess || set_smem(k_scatter<T, TILE, NT>, sh_sc) != cudaSuccess)
        return PF_ERR_CUDA;
    Pos<T>* pos = (Pos<T>*)bw.pos;
    if (nb > 0) {
        PF_KERNEL(p, "bin_locate", PF_CUDA(p, pf_launch(k_locate<T, TILE, NT>, nb, NT, sh_loc, s, X, Y, G, nv,
                                                       span, dn, min_span, mb, geo, pos, bw.bin_off, bw.gmax + 1,
                                                       bw.status, bw.oob, (T*)bw.zu, (T*)bw.zv)));
    }
    PF_KERNEL(p, "bin_offsets", PF_CUDA(p, pf_launch(k_offsets, ceil_div(geo.ntiles, OFF_TILES), 1024, 0, s,
                                                     geo.ntiles, nb, bw.bin_off, bw.tile_count,
                                                     (const double*)(bw.gmax + 1), bw.gmax)));
    if (nb > 0) {
        PF_KERNEL(p, "bin_scatter", PF_CUDA(p, pf_launch(k_scatter<T, TILE, NT>, nb, NT, sh_sc, s, pos, nv,
                                                         span, dn, min_span, mb, geo, bw.bin_off, bw.tile_count,
                                                         bw.tile_start, (Rec<T>*)bw.recs, bw.rec_cap, bw.status)));
    } else if (cudaMemsetAsync(bw.tile_start, 0, (size_t)geo.ntiles * sizeof(int), s) != cudaSuccess) {
        return PF_ERR_CUDA;
    }
    return PF_OK;
}

template <typename T, int TILE = BIN_TILE>
pf_status bin_launch(pf_plan p, const Geo& geo, const BinWork& bw, const double* X, const double* Y,
                     const double* G, int64_t nv, cudaStream_t s, int min_span = BIN_MIN_SPAN,
                     const int64_t* dn = nullptr) {
    if (geo.ntiles > MAX_SCAN_TILES) return PF_ERR_ARG;
    if (bin_max_blocks(nv) == BIN_WIDE_BLOCKS)
        return bin_launch_nt<T, TILE, 1024>(p, geo, bw, X, Y, G, nv, s, min_span, dn);
    return bin_launch_nt<T, TILE, BIN_THREADS>(p, geo, bw, X, Y, G, nv, s, min_span, dn);
}

// Deposit the binned records of bw into w.
template <typename T, int TILE = BIN_TILE>
pf_status deposit_launch(pf_plan p, const Geo& geo, const Rec<T>* recs, const int* tile_start,
                         const unsigned* tile_count, const double* gmax, int64_t rec_cap, int* status, T* w,
                         cudaStream_t s, int threads = 256) {
    PF_KERNEL(p, "regularize", PF_CUDA(p, pf_launch(k_deposit<T, TILE>, geo.ntiles, threads, 0, s, recs, tile_start, tile_count,
                                                    gmax, geo, w, rec_cap, status)));
    return PF_OK;
}

// The four regularization kernels.
template <typename T, int TILE = BIN_TILE>
pf_status regularize_launch(pf_plan p, const Geo& geo, const BinWork& bw, const double* X, const double* Y,
                            const double* G, int64_t nv, T* w, cudaStream_t s, int min_span = BIN_MIN_SPAN,
                            int threads = 256, const int64_t* dn = nullptr) {
    PF_TRY((bin_launch<T, TILE>(p, geo, bw, X, Y, G, nv, s, min_span, dn)));
    return deposit_launch<T, TILE>(p, geo, (const Rec<T>*)bw.recs, bw.tile_start, bw.tile_count,
                                   (const double*)bw.gmax, bw.rec_cap, bw.status, w, s, threads);
}

}  // namespace

// Vortex <-> grid transfer with the M4' kernel (Sec. 2.1):
//   R_v (Eq. vortexregularization): w_ij = dx^-2 sum_q Gamma_q d((x_i-X_q)/dx) d((y_j-Y_q)/dx)
//   E_v = R_v^T:                    u_q  = sum_ij d d u_ij
//
// Regularization is a binned scatter in four kernels:
//   locate   FP64 position -> integer cell + fraction (one pass, FP64 used only
//            for g = (X - x0)/dx), compact per-vortex record, per-block tile
//            histogram in shared memory flushed with one reduction per tile;
//   scan     exclusive scan of the tile counts, fixed-point exponent per tile;
//   scatter  per-block ranks in shared memory, one cursor reservation per
//            (block, tile), records written into their tiles; a vortex whose
//            4x4 stencil straddles tiles is entered in every tile it touches;
//   deposit  one block per BIN_TILE^2 node tile sums its records in shared
//            memory as fixed-point integers with a per-tile scale chosen from
//            the tile's record count and largest |Gamma|.  Integer sums are
//            exact, so the result does not depend on the order of the adds.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int CHUNK = 2048;          // vortices per block in the locate / scatter passes
constexpr int BIN_THREADS = 256;
constexpr int PER_THREAD = CHUNK / BIN_THREADS;

// per-vortex cell record (original order)
template <typename T> struct Pos;
template <> struct __align__(16) Pos<float> {
    unsigned cell;    // ci | cj << 16
    float fx, fy, g;
};
template <> struct __align__(16) Pos<double> {
    int ci, cj;
    double fx, fy, g;
};
// per-tile record
template <typename T> struct Rec;
template <> struct __align__(16) Rec<float> {
    short lx, ly;     // cell index relative to the tile origin
    float fx, fy, g;
};
template <> struct __align__(16) Rec<double> {
    int lx, ly;
    double fx, fy, g;
};

__device__ __forceinline__ int pos_ci(const Pos<float>& p) { return (int)(p.cell & 0xFFFFu); }
__device__ __forceinline__ int pos_cj(const Pos<float>& p) { return (int)(p.cell >> 16); }
__device__ __forceinline__ int pos_ci(const Pos<double>& p) { return p.ci; }
__device__ __forceinline__ int pos_cj(const Pos<double>& p) { return p.cj; }

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
__device__ __forceinline__ bool split(double X, double x0, double dx, double, double, int n, int& c, double& f) {
    const double g = (X - x0) / dx;
    if (!(g >= 1.0 && g < (double)(n - 2))) return false;
    const double fl = floor(g);
    c = (int)fl;
    f = g - fl;
    return true;
}
__device__ __forceinline__ bool split(double X, double, double, double inv_dx, double c0, int n, int& c, float& f) {
    const double g = fma(X, inv_dx, c0);
    // 1 <= g < n - 2 compared on the bit patterns (monotone for non-negative
    // doubles; negative values and NaN fail), keeping the FP64 pipe for the FMA
    const long long gb = __double_as_longlong(g);
    if (gb < 0x3FF0000000000000ll || gb >= __double_as_longlong((double)(n - 2))) return false;
    const unsigned long long bits = (unsigned long long)gb;
    const int sh = 52 - ((int)(bits >> 52) - 1023);                  // g >= 1: sign 0, exponent 0..10
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    c = (int)(mant >> sh);
    const unsigned long long fr = mant & ((1ull << sh) - 1);
    f = __uint2float_rz((unsigned)((fr << (64 - sh)) >> 32)) * 0x1p-32f;
    return true;
}

__device__ __forceinline__ void make_pos(Pos<float>& p, int ci, int cj, float fx, float fy, double g) {
    p.cell = (unsigned)ci | ((unsigned)cj << 16);
    p.fx = fx;
    p.fy = fy;
    p.g = (float)g;
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
    int nx, ny, ntx, ntiles;
};

template <typename T>
__global__ void __launch_bounds__(BIN_THREADS) k_locate(const double* __restrict__ X, const double* __restrict__ Y,
                                                       const double* __restrict__ G, int64_t nv, Geo geo,
                                                       Pos<T>* __restrict__ pos, unsigned* __restrict__ tile_count,
                                                       unsigned* __restrict__ tile_gmax, int* __restrict__ status,
                                                       unsigned long long* __restrict__ oob) {
    extern __shared__ unsigned sm[];
    unsigned* cnt = sm;
    unsigned* gmx = sm + geo.ntiles;
    for (int i = threadIdx.x; i < geo.ntiles; i += BIN_THREADS) {
        cnt[i] = 0u;
        gmx[i] = 0u;
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * CHUNK;
    int bad = 0;
    // issue every load of this thread's vortices before using any of them
    double xs[PER_THREAD], ys[PER_THREAD], gs[PER_THREAD];
#pragma unroll
    for (int k = 0; k < PER_THREAD; ++k) {
        const int64_t q = base + k * BIN_THREADS + threadIdx.x;
        xs[k] = ys[k] = gs[k] = 0.0;
        if (q < nv) {
            xs[k] = X[q];
            ys[k] = Y[q];
            gs[k] = G[q];
        }
    }
#pragma unroll
    for (int k = 0; k < PER_THREAD; ++k) {
        const int64_t q = base + k * BIN_THREADS + threadIdx.x;
        if (q >= nv) break;
        int ci = 0, cj = 0;
        T fx = 0, fy = 0;
        const double gq = gs[k];
        Pos<T> p;
        if (!split(xs[k], geo.x0, geo.dx, geo.inv_dx, geo.cx, geo.nx, ci, fx) ||
            !split(ys[k], geo.y0, geo.dx, geo.inv_dx, geo.cy, geo.ny, cj, fy)) {
            ++bad;
            make_pos(p, 0xFFFF, 0xFFFF, T(0), T(0), 0.0);   // marker: skipped by scatter and interpolation
            pos[q] = p;
            continue;
        }
        make_pos(p, ci, cj, fx, fy, gq);
        pos[q] = p;
        // |Gamma| rounded to FP32 and widened by two ulps: an upper bound of |Gamma|
        const unsigned gb = __float_as_uint(fabsf((float)gq) * 1.0000003f);
        const int tx0 = (ci - 1) / BIN_TILE, tx1 = (ci + 2) / BIN_TILE;
        const int ty0 = (cj - 1) / BIN_TILE, ty1 = (cj + 2) / BIN_TILE;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                const int t = ty * geo.ntx + tx;
                atomicAdd(&cnt[t], 1u);
                atomicMax(&gmx[t], gb);
            }
    }
    if (bad) {
        atomicAdd(oob, (unsigned long long)bad);
        atomicOr(status, ST_OUT_OF_DOMAIN);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < geo.ntiles; i += BIN_THREADS)
        if (cnt[i]) {
            atomicAdd(&tile_count[i], cnt[i]);
            atomicMax(&tile_gmax[i], gmx[i]);
        }
}

// Fixed-point exponent of a tile: every node sum is bounded by
// count * max|Gamma| < 2^e and is scaled to stay below 2^61.
__device__ __forceinline__ int tile_shift_of(unsigned count, unsigned gmax_bits) {
    const double bound = (double)count * (double)__uint_as_float(gmax_bits);
    int e = 0;
    if (bound > 0.0) frexp(bound, &e);
    const int sh = 61 - e;
    return sh > 100 ? 100 : (sh < -60 ? -60 : sh);
}

// Exclusive scan of the tile counts by one block of BIN_THREADS threads; thread
// tid owns tiles [tid*per, tid*per + per) and gets their first offset in *first.
__device__ __forceinline__ void block_scan_tiles(const unsigned* __restrict__ tile_count, int ntiles, int per,
                                                 int* __restrict__ wsum, int& first) {
    const int lo = threadIdx.x * per, hi = min(ntiles, lo + per);
    int s = 0;
    for (int t = lo; t < hi; ++t) s += (int)tile_count[t];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int wofs = 0;
    for (int k = 0; k < wid; ++k) wofs += wsum[k];
    first = wofs + incl - s;
}

template <typename T>
__global__ void __launch_bounds__(BIN_THREADS) k_scatter(const Pos<T>* __restrict__ pos, int64_t nv, Geo geo,
                                                        const unsigned* __restrict__ tile_count,
                                                        int* __restrict__ tile_start,
                                                        unsigned* __restrict__ tile_cursor, Rec<T>* __restrict__ recs,
                                                        int* __restrict__ ridx) {
    __shared__ int wsum[BIN_THREADS / 32];
    extern __shared__ unsigned sm[];
    unsigned* cnt = sm;
    int* bas = (int*)(sm + geo.ntiles);
    for (int i = threadIdx.x; i < geo.ntiles; i += BIN_THREADS) cnt[i] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * CHUNK;
    unsigned long long rk[PER_THREAD];     // up to four 16-bit ranks per vortex
    int cell[PER_THREAD][2];
#pragma unroll
    for (int k = 0; k < PER_THREAD; ++k) {     // loads first
        const int64_t q = base + k * BIN_THREADS + threadIdx.x;
        cell[k][0] = 0xFFFF;
        if (q < nv) {
            const Pos<T> p = pos[q];
            cell[k][0] = pos_ci(p);
            cell[k][1] = pos_cj(p);
        }
    }
#pragma unroll
    for (int k = 0; k < PER_THREAD; ++k) {
        rk[k] = 0ull;
        const int ci = cell[k][0], cj = cell[k][1];
        if (ci == 0xFFFF) continue;
        const int tx0 = (ci - 1) / BIN_TILE, tx1 = (ci + 2) / BIN_TILE;
        const int ty0 = (cj - 1) / BIN_TILE, ty1 = (cj + 2) / BIN_TILE;
        int s = 0;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx, ++s) {
                const unsigned r = atomicAdd(&cnt[ty * geo.ntx + tx], 1u);
                rk[k] |= (unsigned long long)r << (16 * s);
            }
    }
    // every block scans the tile totals itself (block 0 publishes them for the
    // deposit and interpolation kernels), then reserves its run in each tile
    const int per = (geo.ntiles + BIN_THREADS - 1) / BIN_THREADS;
    int first = 0;
    block_scan_tiles(tile_count, geo.ntiles, per, wsum, first);   // contains __syncthreads
    for (int i = threadIdx.x * per, e = min(geo.ntiles, threadIdx.x * per + per); i < e; ++i) {
        if (blockIdx.x == 0) tile_start[i] = first;
        if (cnt[i]) bas[i] = first + (int)atomicAdd(&tile_cursor[i], cnt[i]);
        first += (int)tile_count[i];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER_THREAD; ++k) {
        const int64_t q = base + k * BIN_THREADS + threadIdx.x;
        if (q >= nv) continue;
        const Pos<T> p = pos[q];
        const int ci = pos_ci(p), cj = pos_cj(p);
        if (ci == 0xFFFF) continue;
        const int tx0 = (ci - 1) / BIN_TILE, tx1 = (ci + 2) / BIN_TILE;
        const int ty0 = (cj - 1) / BIN_TILE, ty1 = (cj + 2) / BIN_TILE;
        Rec<T> r;
        r.fx = p.fx;
        r.fy = p.fy;
        r.g = p.g;
        int s = 0;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx, ++s) {
                const unsigned rank = (unsigned)(rk[k] >> (16 * s)) & 0xFFFFu;
                r.lx = (decltype(r.lx))(ci - tx * BIN_TILE);
                r.ly = (decltype(r.ly))(cj - ty * BIN_TILE);
                const int slot = bas[ty * geo.ntx + tx] + (int)rank;
                recs[slot] = r;
                if (ridx) ridx[slot] = (int)q;
            }
    }
}

// fixed-point scale 2^sh as a floating-point number, sh in [-60, 100]
template <typename T> __device__ __forceinline__ T pow2(int sh);
template <> __device__ __forceinline__ float pow2<float>(int sh) { return __int_as_float((sh + 127) << 23); }
template <> __device__ __forceinline__ double pow2<double>(int sh) { return __longlong_as_double((long long)(sh + 1023) << 52); }

// round(x) = hi * 2^16 + lo with 0 <= lo < 2^16, for |x| < 2^46, in FP32 and
// 32-bit integer arithmetic only: h = floor(x / 2^16) and x - h 2^16 are exact
__device__ __forceinline__ void split_hilo(float x, int& hi, unsigned& lo) {
    float h = floorf(x * 0x1p-16f);
    const float l = fmaf(-h, 65536.0f, x);
    unsigned li = __float2uint_rn(l);
    if (li >= 65536u) {
        li -= 65536u;
        h += 1.0f;
    }
    hi = __float2int_rz(h);
    lo = li;
}

// Deposit: one block per node tile accumulates its records in shared memory as
// fixed-point integers.  FP32 path: each term round(v 2^sh) = hi 2^16 + lo goes
// into two native 32-bit shared adds (exact while the tile has fewer than 65536
// records and |sum| < 2^46); otherwise, and for FP64, one 64-bit add.  Integer
// sums are exact, so the result does not depend on the order of the adds.
template <typename T>
__global__ void __launch_bounds__(256) k_deposit(const Rec<T>* __restrict__ recs, const int* __restrict__ tile_start,
                                                 const unsigned* __restrict__ tile_count,
                                                 const unsigned* __restrict__ tile_gmax, Geo geo, T* __restrict__ w) {
    __shared__ unsigned long long acc[BIN_TILE * BIN_TILE];
    const int t = blockIdx.x;
    const int tx = t % geo.ntx, ty = t / geo.ntx;
    for (int i = threadIdx.x; i < BIN_TILE * BIN_TILE; i += blockDim.x) acc[i] = 0ull;
    __syncthreads();
    const int start = tile_start[t], cnt = (int)tile_count[t];
    const bool split32 = sizeof(T) == 4 && cnt < 65536;
    const int sh = tile_shift_of((unsigned)cnt, tile_gmax[t]) - (split32 ? 15 : 0);   // 2^61 -> 2^46 when split
    const T scale = pow2<T>(sh);
    int* acc_hi = reinterpret_cast<int*>(acc);
    unsigned* acc_lo = reinterpret_cast<unsigned*>(acc) + BIN_TILE * BIN_TILE;
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const Rec<T> rc = recs[start + r];
        T wx[4], wy[4];
        m4p_weights<T>(rc.fx, wx);
        m4p_weights<T>(rc.fy, wy);
        const T gs = rc.g * scale;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int ly = rc.ly - 1 + b;
            if (ly < 0 || ly >= BIN_TILE) continue;
            const T gy = gs * wy[b];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int lx = rc.lx - 1 + a;
                if (lx < 0 || lx >= BIN_TILE) continue;
                const int node = ly * BIN_TILE + lx;
                const T x = gy * wx[a];
                if (sizeof(T) == 4 && split32) {
                    int hi;
                    unsigned lo;
                    split_hilo((float)x, hi, lo);
                    atomicAdd(&acc_hi[node], hi);
                    atomicAdd(&acc_lo[node], lo);
                } else if (sizeof(T) == 4) {
                    atomicAdd(&acc[node], (unsigned long long)__float2ll_rn((float)x));
                } else {
                    atomicAdd(&acc[node], (unsigned long long)__double2ll_rn((double)x));
                }
            }
        }
    }
    __syncthreads();
    const double inv_dx2 = geo.inv_dx2;
    const float inv_dx2f = (float)geo.inv_dx2;
    for (int i = threadIdx.x; i < BIN_TILE * BIN_TILE; i += blockDim.x) {
        const int gi = tx * BIN_TILE + (i % BIN_TILE), gj = ty * BIN_TILE + (i / BIN_TILE);
        if (gi < geo.nx && gj < geo.ny) {
            long long a;
            if (split32) a = (long long)acc_hi[i] * 65536ll + (long long)acc_lo[i];
            else a = (long long)acc[i];
            T v;
            if (sizeof(T) == 4) v = (T)(__ll2float_rn(a) * pow2<float>(-sh) * inv_dx2f);
            else v = (T)(ldexp((double)a, -sh) * inv_dx2);
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
constexpr int PATCH = BIN_TILE + 3;

template <typename T>
__global__ void __launch_bounds__(256) k_interp_tiles(const Rec<T>* __restrict__ recs, const int* __restrict__ ridx,
                                                      const int* __restrict__ tile_start,
                                                      const unsigned* __restrict__ tile_count, const C_t<T>* __restrict__ uv,
                                                      Geo geo, T* __restrict__ uq, T* __restrict__ vq) {
    using C = C_t<T>;
    __shared__ C patch[PATCH * PATCH];
    const int t = blockIdx.x;
    const int cnt = (int)tile_count[t];
    if (cnt == 0) return;
    const int tx = t % geo.ntx, ty = t / geo.ntx;
    const int gi0 = tx * BIN_TILE - 1, gj0 = ty * BIN_TILE - 1;
    for (int i = threadIdx.x; i < PATCH * PATCH; i += blockDim.x) {
        const int gi = gi0 + i % PATCH, gj = gj0 + i / PATCH;
        C v = cmake<C>(T(0), T(0));
        if (gi >= 0 && gi < geo.nx && gj >= 0 && gj < geo.ny) v = uv[(size_t)gj * geo.nx + gi];
        patch[i] = v;
    }
    __syncthreads();
    const int start = tile_start[t];
    constexpr int U = 4;
    for (int r0 = 0; r0 < cnt; r0 += U * blockDim.x) {
        Rec<T> rc[U];
        int qi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {           // loads first
            const int r = r0 + u * blockDim.x + threadIdx.x;
            rc[u].lx = -1;
            if (r < cnt) {
                rc[u] = recs[start + r];
                qi[u] = ridx[start + r];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (rc[u].lx < 0 || rc[u].lx >= BIN_TILE || rc[u].ly < 0 || rc[u].ly >= BIN_TILE) continue;  // not home
            T wx[4], wy[4];
            m4p_weights<T>(rc[u].fx, wx);
            m4p_weights<T>(rc[u].fy, wy);
            T su = 0, sv = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const C* row = patch + (rc[u].ly + b) * PATCH + rc[u].lx;    // node (lx - 1 + a, ly - 1 + b)
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
            uq[qi[u]] = su;
            vq[qi[u]] = sv;
        }
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
        if (split(X[q], geo.x0, geo.dx, geo.inv_dx, geo.cx, geo.nx, ci, fx) &&
            split(Y[q], geo.y0, geo.dx, geo.inv_dx, geo.cy, geo.ny, cj, fy)) {
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
    unsigned* tile_count;
    unsigned* tile_gmax;
    int* tile_start;
    unsigned* tile_cursor;
    void* pos;
    void* recs;
    int* ridx;          // original index of every binned record (may be null)
};

inline Geo make_geo(int nx, int ny, double dx, double x0, double y0) {
    Geo g;
    g.x0 = x0; g.y0 = y0; g.dx = dx; g.nx = nx; g.ny = ny;
    g.inv_dx = 1.0 / dx;
    g.cx = -x0 / dx;
    g.cy = -y0 / dx;
    g.inv_dx2 = 1.0 / (dx * dx);
    g.ntx = ceil_div(nx, BIN_TILE);
    g.ntiles = g.ntx * ceil_div(ny, BIN_TILE);
    return g;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    static size_t done = 0;
    if (bytes <= done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done = bytes;
    return e;
}

// Launch the four regularization kernels; `p` (may be null) only supplies the
// timing records and the error text.
template <typename T>
pf_status regularize_launch(pf_plan p, const Geo& geo, const BinWork& bw, const double* X, const double* Y,
                            const double* G, int64_t nv, T* w, cudaStream_t s) {
    // tile_count, tile_gmax and tile_cursor are contiguous: one clear
    if (cudaMemsetAsync(bw.tile_count, 0, 3 * (size_t)geo.ntiles * sizeof(unsigned), s) != cudaSuccess) return PF_ERR_CUDA;
    const int nb = nv > 0 ? ceil_div(nv, CHUNK) : 0;
    const size_t sh = 2 * (size_t)geo.ntiles * sizeof(unsigned);
    if (set_smem(k_locate<T>, sh) != cudaSuccess || set_smem(k_scatter<T>, sh) != cudaSuccess) return PF_ERR_CUDA;
    Pos<T>* pos = (Pos<T>*)bw.pos;
    if (nb > 0) {
        PF_KERNEL(p, "bin_locate", k_locate<T><<<nb, BIN_THREADS, sh, s>>>(X, Y, G, nv, geo, pos, bw.tile_count,
                                                                           bw.tile_gmax, bw.status, bw.oob));
    }
    if (nb > 0) {
        PF_KERNEL(p, "bin_scatter", k_scatter<T><<<nb, BIN_THREADS, sh, s>>>(pos, nv, geo, bw.tile_count,
                                                                             bw.tile_start, bw.tile_cursor,
                                                                             (Rec<T>*)bw.recs, bw.ridx));
    }
    if (nb == 0 && cudaMemsetAsync(bw.tile_start, 0, geo.ntiles * sizeof(int), s) != cudaSuccess) return PF_ERR_CUDA;
    PF_KERNEL(p, "regularize", k_deposit<T><<<geo.ntiles, 256, 0, s>>>((const Rec<T>*)bw.recs, bw.tile_start,
                                                                      bw.tile_count, bw.tile_gmax, geo, w));
    return PF_OK;
}

pf_status plan_bin_reserve(pf_plan p, int64_t nv) {
    const size_t psz = p->prec == PF_FP64 ? sizeof(Pos<double>) : sizeof(Pos<float>);
    const size_t rsz = p->prec == PF_FP64 ? sizeof(Rec<double>) : sizeof(Rec<float>);
    // capacities grow geometrically so a slowly growing vortex set (shedding)
    // does not reallocate every step
    if (nv > p->pos_cap) {
        const int64_t cap = std::max<int64_t>(std::max<int64_t>(nv, 2 * p->pos_cap), 4096);
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        if (p->pos) cudaFree(p->pos);
        p->pos = nullptr;
        p->pos_cap = 0;
        PF_CUDA(p, cudaMalloc(&p->pos, (size_t)cap * psz));
        p->pos_cap = cap;
    }
    if (4 * nv > p->rec_cap) {   // a vortex is entered in at most four tiles
        const int64_t cap = 4 * p->pos_cap;
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        if (p->recs) cudaFree(p->recs);
        if (p->ridx) cudaFree(p->ridx);
        p->recs = nullptr;
        p->ridx = nullptr;
        p->rec_cap = 0;
        PF_CUDA(p, cudaMalloc(&p->recs, (size_t)cap * rsz));
        PF_CUDA(p, cudaMalloc(&p->ridx, (size_t)cap * sizeof(int)));
        p->rec_cap = cap;
    }
    return PF_OK;
}

BinWork plan_binwork(pf_plan p) {
    BinWork b;
    b.status = p->d_status;
    b.oob = p->d_oob;
    b.tile_count = p->tile_count;
    b.tile_gmax = p->tile_gmax;
    b.tile_start = p->tile_start;
    b.tile_cursor = p->tile_cursor;
    b.pos = p->pos;
    b.recs = p->recs;
    b.ridx = p->ridx;
    return b;
}

}  // namespace

// size the plan's vortex buffers for nv vortices ahead of time
pf_status plan_reserve_vortices(pf_plan p, int64_t nv) { return plan_bin_reserve(p, nv); }

pf_status vortex_regularize(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, void* w) {
    pf_status st = plan_bin_reserve(p, nv);
    if (st != PF_OK) return st;
    const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0);
    const BinWork bw = plan_binwork(p);
    if (p->prec == PF_FP64) return regularize_launch<double>(p, geo, bw, X, Y, G, nv, (double*)w, p->stream);
    return regularize_launch<float>(p, geo, bw, X, Y, G, nv, (float*)w, p->stream);
}

// E_v at the vortices the last vortex_regularize call binned
pf_status vortex_interpolate_located(pf_plan p, const void* uv, int64_t nq, void* uq, void* vq) {
    if (nq == 0) return PF_OK;
    const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0);
    if (p->prec == PF_FP64)
        PF_KERNEL(p, "interpolate", k_interp_tiles<double><<<geo.ntiles, 256, 0, p->stream>>>(
                                        (const Rec<double>*)p->recs, p->ridx, p->tile_start, p->tile_count,
                                        (const double2*)uv, geo, (double*)uq, (double*)vq));
    else
        PF_KERNEL(p, "interpolate", k_interp_tiles<float><<<geo.ntiles, 256, 0, p->stream>>>(
                                        (const Rec<float>*)p->recs, p->ridx, p->tile_start, p->tile_count,
                                        (const float2*)uv, geo, (float*)uq, (float*)vq));
    return PF_OK;
}

pf_status vortex_interpolate(pf_plan p, const void* uv, const double* X, const double* Y, int64_t nq, void* uq, void* vq) {
    if (nq == 0) return PF_OK;
    const int nb = (int)std::min<int64_t>(ceil_div(nq, 256), 152 * 16);
    const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0);
    if (p->prec == PF_FP64)
        PF_KERNEL(p, "interpolate", k_interp_xy<double><<<nb, 256, 0, p->stream>>>((const double*)uv, X, Y, nq, geo,
                                                                                   (double*)uq, (double*)vq,
                                                                                   p->d_status, p->d_oob));
    else
        PF_KERNEL(p, "interpolate", k_interp_xy<float><<<nb, 256, 0, p->stream>>>((const float*)uv, X, Y, nq, geo,
                                                                                  (float*)uq, (float*)vq, p->d_status,
                                                                                  p->d_oob));
    return PF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free regularization.
//
// Same kernels as pf_regularize, but every piece of scratch (tile counters,
// fixed-point exponents, status words, the per-vortex cell records and the
// binned records) lives in one file-scope device array, so the entry point
// needs no plan and makes no allocation.  The array is part of the library
// image: each GPU that loads the library holds NOALLOC_SCRATCH_BYTES of it
// until the process exits.
namespace {

constexpr int64_t NOALLOC_MAX_VORTICES = 65536;
constexpr int NOALLOC_MAX_TILES = (2048 / BIN_TILE) * (2048 / BIN_TILE);
constexpr size_t NOALLOC_HEADER = 256;   // status int + out-of-domain counter, padded
constexpr size_t NOALLOC_TILE_BYTES = (size_t)NOALLOC_MAX_TILES * 5 * sizeof(int);
constexpr size_t NOALLOC_POS_BYTES = (size_t)NOALLOC_MAX_VORTICES * sizeof(Pos<double>);
constexpr size_t NOALLOC_SCRATCH_BYTES =
    NOALLOC_HEADER + NOALLOC_TILE_BYTES + NOALLOC_POS_BYTES + (size_t)4 * NOALLOC_MAX_VORTICES * sizeof(Rec<double>);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
unsigned char* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Resolve the array's device address for the current device (first call per
// device only).  The host-side name g_noalloc_scratch is not a device address.
cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = (unsigned char*)ptr;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

BinWork noalloc_binwork(unsigned char* base, int ntiles) {
    BinWork b;
    b.status = (int*)base;
    b.oob = (unsigned long long*)(base + 8);
    unsigned* t = (unsigned*)(base + NOALLOC_HEADER);
    const int nt = ntiles;         // <= NOALLOC_MAX_TILES
    b.tile_count = t;              // count, gmax and cursor contiguous for one clear
    b.tile_gmax = t + nt;
    b.tile_cursor = t + 2 * nt;
    b.tile_start = (int*)(t + 3 * nt);
    b.pos = base + NOALLOC_HEADER + NOALLOC_TILE_BYTES;
    b.recs = base + NOALLOC_HEADER + NOALLOC_TILE_BYTES + NOALLOC_POS_BYTES;
    b.ridx = nullptr;   // no interpolation follows an allocation-free regularization
    return b;
}

}  // namespace

extern "C" pf_status pf_regularize_noalloc(const pf_grid_desc* d, const double* X, const double* Y, const double* G,
                                           int64_t nv, void* w, int64_t* out_of_domain, void* stream) {
    if (!d || !w || nv < 0 || (nv > 0 && (!X || !Y || !G))) return PF_ERR_ARG;
    if (d->nx < 8 || d->ny < 8 || d->nx > 2048 || d->ny > 2048 || !(d->dx > 0) || !isfinite(d->x0) ||
        !isfinite(d->y0) || (d->precision != PF_FP64 && d->precision != PF_MIXED))
        return PF_ERR_ARG;
    if (nv > NOALLOC_MAX_VORTICES) return PF_ERR_CAPACITY;
    unsigned char* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return PF_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Geo geo = make_geo(d->nx, d->ny, d->dx, d->x0, d->y0);
    const BinWork bw = noalloc_binwork(base, geo.ntiles);
    // the array keeps the previous call's contents: clear the status words
    if (cudaMemsetAsync(base, 0, NOALLOC_HEADER, s) != cudaSuccess) return PF_ERR_CUDA;
    pf_status st = d->precision == PF_FP64
                       ? regularize_launch<double>(nullptr, geo, bw, X, Y, G, nv, (double*)w, s)
                       : regularize_launch<float>(nullptr, geo, bw, X, Y, G, nv, (float*)w, s);
    if (st != PF_OK) return st;
    if (cudaGetLastError() != cudaSuccess) return PF_ERR_CUDA;
    if (out_of_domain &&
        cudaMemcpyAsync(out_of_domain, bw.oob, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return PF_ERR_CUDA;
    return PF_OK;
}

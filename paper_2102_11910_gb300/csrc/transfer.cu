// Vortex <-> grid transfer with the M4' kernel (Sec. 2.1):
//   R_v (Eq. vortexregularization): w_ij = dx^-2 sum_q Gamma_q d((x_i-X_q)/dx) d((y_j-Y_q)/dx)
//   E_v = R_v^T:                    u_q  = sum_ij d d u_ij
//
// Regularization is a binned scatter.  Vortices are binned by BIN_TILE^2
// node tiles; a vortex whose 4x4 stencil straddles tiles is entered in every
// tile it touches (at most 4).  One block per tile accumulates its nodes in
// shared memory as 64-bit fixed point with a per-tile scale chosen from the
// tile's vortex count and largest |Gamma|, so the integer sums are exact and
// the result does not depend on the order in which blocks or threads add.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

template <typename T> struct Rec;
template <> struct Rec<float> {
    short lx, ly;     // cell index relative to the tile origin
    float fx, fy, g;  // fractional offset in the cell, strength
};
template <> struct Rec<double> {
    int lx, ly;
    double fx, fy, g;
};

// M4' weights of the four nodes floor(g)-1 .. floor(g)+2 for fractional part f
template <typename T>
__device__ __forceinline__ void m4p_weights(T f, T w[4]) {
    const T a0 = T(1) + f, a1 = f, a2 = T(1) - f, a3 = T(2) - f;
    w[0] = T(0.5) * (T(2) - a0) * (T(2) - a0) * (T(1) - a0);
    w[1] = T(1) - T(2.5) * a1 * a1 + T(1.5) * a1 * a1 * a1;
    w[2] = T(1) - T(2.5) * a2 * a2 + T(1.5) * a2 * a2 * a2;
    w[3] = T(0.5) * (T(2) - a3) * (T(2) - a3) * (T(1) - a3);
}

struct Cell {
    int ci, cj;
    double fx, fy;
    bool ok;
};

__device__ __forceinline__ Cell locate(double X, double Y, double x0, double y0, double inv_dx, int nx, int ny) {
    Cell c;
    const double gx = (X - x0) * inv_dx, gy = (Y - y0) * inv_dx;
    const double fgx = floor(gx), fgy = floor(gy);
    // stencil floor(g)-1 .. floor(g)+2 must lie in [0, n): floor(g) in [1, n-3]
    c.ok = (fgx >= 1.0) && (fgx <= nx - 3.0) && (fgy >= 1.0) && (fgy <= ny - 3.0);
    c.ci = c.ok ? (int)fgx : 0;
    c.cj = c.ok ? (int)fgy : 0;
    c.fx = gx - fgx;
    c.fy = gy - fgy;
    return c;
}

__global__ void k_bin_count(const double* __restrict__ X, const double* __restrict__ Y, const double* __restrict__ G,
                            int64_t nv, double x0, double y0, double inv_dx, int nx, int ny, int ntx,
                            int* __restrict__ tile_count, unsigned long long* __restrict__ tile_gmax,
                            int* __restrict__ status, unsigned long long* __restrict__ oob) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        const Cell c = locate(X[q], Y[q], x0, y0, inv_dx, nx, ny);
        if (!c.ok) {
            atomicAdd(oob, 1ull);
            atomicOr(status, ST_OUT_OF_DOMAIN);
            continue;
        }
        const unsigned long long gbits = (unsigned long long)__double_as_longlong(fabs(G[q]));
        const int tx0 = (c.ci - 1) / BIN_TILE, tx1 = (c.ci + 2) / BIN_TILE;
        const int ty0 = (c.cj - 1) / BIN_TILE, ty1 = (c.cj + 2) / BIN_TILE;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                const int t = ty * ntx + tx;
                atomicAdd(&tile_count[t], 1);
                atomicMax(&tile_gmax[t], gbits);
            }
    }
}

// exclusive scan of tile counts (one block), fixed-point exponent per tile,
// cursors reset
__global__ void k_bin_scan(const int* __restrict__ tile_count, const unsigned long long* __restrict__ tile_gmax,
                           int* __restrict__ tile_start, int* __restrict__ tile_cursor, int* __restrict__ tile_shift,
                           int ntiles) {
    __shared__ int part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (ntiles + nt - 1) / nt;
    const int lo = tid * per, hi = min(ntiles, lo + per);
    int s = 0;
    for (int t = lo; t < hi; ++t) s += tile_count[t];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int i = 0; i < nt; ++i) {
            const int v = part[i];
            part[i] = run;
            run += v;
        }
    }
    __syncthreads();
    int run = part[tid];
    for (int t = lo; t < hi; ++t) {
        tile_start[t] = run;
        tile_cursor[t] = 0;
        run += tile_count[t];
        // every node sum is bounded by count * max|Gamma| < 2^e; scale so it stays below 2^61
        const double bound = (double)tile_count[t] * __longlong_as_double((long long)tile_gmax[t]);
        int e = 0;
        if (bound > 0.0) frexp(bound, &e);
        int sh = 61 - e;
        sh = sh > 100 ? 100 : (sh < -60 ? -60 : sh);
        tile_shift[t] = sh;
    }
}

template <typename T>
__global__ void k_bin_scatter(const double* __restrict__ X, const double* __restrict__ Y, const double* __restrict__ G,
                              int64_t nv, double x0, double y0, double inv_dx, int nx, int ny, int ntx,
                              const int* __restrict__ tile_start, int* __restrict__ tile_cursor, Rec<T>* __restrict__ recs) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        const Cell c = locate(X[q], Y[q], x0, y0, inv_dx, nx, ny);
        if (!c.ok) continue;
        const int tx0 = (c.ci - 1) / BIN_TILE, tx1 = (c.ci + 2) / BIN_TILE;
        const int ty0 = (c.cj - 1) / BIN_TILE, ty1 = (c.cj + 2) / BIN_TILE;
        Rec<T> r;
        r.fx = (T)c.fx;
        r.fy = (T)c.fy;
        r.g = (T)G[q];
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) {
                const int t = ty * ntx + tx;
                const int slot = tile_start[t] + atomicAdd(&tile_cursor[t], 1);
                r.lx = (decltype(r.lx))(c.ci - tx * BIN_TILE);
                r.ly = (decltype(r.ly))(c.cj - ty * BIN_TILE);
                recs[slot] = r;
            }
    }
}

template <typename T> __device__ __forceinline__ long long to_fixed(T v, int sh);
template <> __device__ __forceinline__ long long to_fixed<float>(float v, int sh) { return __float2ll_rn(ldexpf(v, sh)); }
template <> __device__ __forceinline__ long long to_fixed<double>(double v, int sh) { return __double2ll_rn(ldexp(v, sh)); }

template <typename T>
__global__ void __launch_bounds__(256) k_regularize(const Rec<T>* __restrict__ recs, const int* __restrict__ tile_start,
                                                    const int* __restrict__ tile_count, const int* __restrict__ tile_shift,
                                                    int nx, int ny, int ntx, double inv_dx2, T* __restrict__ w) {
    __shared__ unsigned long long acc[BIN_TILE * BIN_TILE];
    const int t = blockIdx.x;
    const int tx = t % ntx, ty = t / ntx;
    for (int i = threadIdx.x; i < BIN_TILE * BIN_TILE; i += blockDim.x) acc[i] = 0ull;
    __syncthreads();
    const int start = tile_start[t], cnt = tile_count[t], sh = tile_shift[t];
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const Rec<T> rc = recs[start + r];
        T wx[4], wy[4];
        m4p_weights<T>(rc.fx, wx);
        m4p_weights<T>(rc.fy, wy);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int ly = rc.ly - 1 + b;
            if (ly < 0 || ly >= BIN_TILE) continue;
            const T gy = rc.g * wy[b];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int lx = rc.lx - 1 + a;
                if (lx < 0 || lx >= BIN_TILE) continue;
                atomicAdd(&acc[ly * BIN_TILE + lx], (unsigned long long)to_fixed<T>(gy * wx[a], sh));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < BIN_TILE * BIN_TILE; i += blockDim.x) {
        const int gi = tx * BIN_TILE + (i % BIN_TILE), gj = ty * BIN_TILE + (i / BIN_TILE);
        if (gi < nx && gj < ny) {
            const long long a = (long long)acc[i];
            T v;
            if (sizeof(T) == 4) v = (T)(ldexpf(__ll2float_rn(a), -sh) * (float)inv_dx2);
            else v = (T)(ldexp((double)a, -sh) * inv_dx2);
            w[(size_t)gj * nx + gi] = v;
        }
    }
}

template <typename T>
__global__ void k_interpolate(const T* __restrict__ uv, const double* __restrict__ X, const double* __restrict__ Y,
                              int64_t nq, double x0, double y0, double inv_dx, int nx, int ny, T* __restrict__ uq,
                              T* __restrict__ vq, int* __restrict__ status, unsigned long long* __restrict__ oob) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const Cell c = locate(X[q], Y[q], x0, y0, inv_dx, nx, ny);
        if (!c.ok) {
            atomicAdd(oob, 1ull);
            atomicOr(status, ST_OUT_OF_DOMAIN);
            uq[q] = T(0);
            vq[q] = T(0);
            continue;
        }
        T wx[4], wy[4];
        m4p_weights<T>((T)c.fx, wx);
        m4p_weights<T>((T)c.fy, wy);
        T su = 0, sv = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const T* row = uv + 2 * ((size_t)(c.cj - 1 + b) * nx + (c.ci - 1));
            T ru = 0, rv = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                ru += wx[a] * row[2 * a];
                rv += wx[a] * row[2 * a + 1];
            }
            su += wy[b] * ru;
            sv += wy[b] * rv;
        }
        uq[q] = su;
        vq[q] = sv;
    }
}

template <typename T>
pf_status regularize_t(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, T* w) {
    const double inv_dx = 1.0 / p->dx;
    PF_CUDA(p, cudaMemsetAsync(p->tile_count, 0, p->ntiles * sizeof(int), p->stream));
    PF_CUDA(p, cudaMemsetAsync(p->tile_gmax, 0, p->ntiles * sizeof(unsigned long long), p->stream));
    const int nb = nv > 0 ? (int)std::min<int64_t>(ceil_div(nv, 256), 152 * 16) : 0;
    if (nb > 0) {
        PF_KERNEL(p, "bin_count", k_bin_count<<<nb, 256, 0, p->stream>>>(X, Y, G, nv, p->x0, p->y0, inv_dx, p->nx, p->ny, p->ntx,
                                                p->tile_count, p->tile_gmax, p->d_status, p->d_oob));
    }
    PF_KERNEL(p, "bin_scan", k_bin_scan<<<1, 1024, 0, p->stream>>>(p->tile_count, p->tile_gmax, p->tile_start, p->tile_cursor,
                                                              p->tile_shift, p->ntiles));
    if (nb > 0) {
        PF_KERNEL(p, "bin_scatter", k_bin_scatter<T><<<nb, 256, 0, p->stream>>>(X, Y, G, nv, p->x0, p->y0, inv_dx, p->nx, p->ny,
                                                     p->ntx, p->tile_start, p->tile_cursor, (Rec<T>*)p->recs));
    }
    PF_KERNEL(p, "regularize", k_regularize<T><<<p->ntiles, 256, 0, p->stream>>>((const Rec<T>*)p->recs, p->tile_start,
                                                       p->tile_count, p->tile_shift, p->nx, p->ny, p->ntx, inv_dx * inv_dx, w));
    return PF_OK;
}

}  // namespace

pf_status vortex_regularize(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, void* w) {
    const size_t rsz = p->prec == PF_FP64 ? sizeof(Rec<double>) : sizeof(Rec<float>);
    if (4 * nv > p->rec_cap) {
        // a vortex is entered in at most four tiles
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        if (p->recs) cudaFree(p->recs);
        p->recs = nullptr;
        p->rec_cap = 0;
        PF_CUDA(p, cudaMalloc(&p->recs, (size_t)4 * nv * rsz));
        p->rec_cap = 4 * nv;
    }
    if (p->prec == PF_FP64) return regularize_t<double>(p, X, Y, G, nv, (double*)w);
    return regularize_t<float>(p, X, Y, G, nv, (float*)w);
}

pf_status vortex_interpolate(pf_plan p, const void* uv, const double* X, const double* Y, int64_t nq, void* uq, void* vq) {
    if (nq == 0) return PF_OK;
    const int nb = (int)std::min<int64_t>(ceil_div(nq, 256), 152 * 16);
    const double inv_dx = 1.0 / p->dx;
    if (p->prec == PF_FP64)
        PF_KERNEL(p, "interpolate", k_interpolate<double><<<nb, 256, 0, p->stream>>>((const double*)uv, X, Y, nq, p->x0, p->y0,
                                                         inv_dx, p->nx, p->ny, (double*)uq, (double*)vq, p->d_status, p->d_oob));
    else
        PF_KERNEL(p, "interpolate", k_interpolate<float><<<nb, 256, 0, p->stream>>>((const float*)uv, X, Y, nq, p->x0, p->y0,
                                                        inv_dx, p->nx, p->ny, (float*)uq, (float*)vq, p->d_status, p->d_oob));
    return PF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free regularization.
//
// Same binned fixed-point kernels as pf_regularize, but every piece of scratch
// (tile counters, fixed-point exponents, status words and the binned vortex
// records) lives in one file-scope device array, so the entry point needs no
// plan and makes no allocation.  The array is part of the library image: each
// GPU that loads the library holds NOALLOC_SCRATCH_BYTES of it until exit.
namespace {

constexpr int64_t NOALLOC_MAX_VORTICES = 65536;
constexpr int NOALLOC_MAX_TILES = (2048 / BIN_TILE) * (2048 / BIN_TILE);
constexpr size_t NOALLOC_HEADER = 256;   // status int + out-of-domain counter, padded
constexpr size_t NOALLOC_TILE_BYTES = (size_t)NOALLOC_MAX_TILES * (4 * sizeof(int) + sizeof(unsigned long long));
constexpr size_t NOALLOC_SCRATCH_BYTES =
    NOALLOC_HEADER + NOALLOC_TILE_BYTES + (size_t)4 * NOALLOC_MAX_VORTICES * sizeof(Rec<double>);

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

template <typename T>
pf_status regularize_noalloc_t(const pf_grid_desc* d, const double* X, const double* Y, const double* G, int64_t nv,
                               T* w, int64_t* out_of_domain, cudaStream_t s, unsigned char* base) {
    const int ntx = ceil_div(d->nx, BIN_TILE), nty = ceil_div(d->ny, BIN_TILE), ntiles = ntx * nty;
    int* status = (int*)base;
    unsigned long long* oob = (unsigned long long*)(base + 8);
    int* tile_count = (int*)(base + NOALLOC_HEADER);
    int* tile_start = tile_count + NOALLOC_MAX_TILES;
    int* tile_cursor = tile_start + NOALLOC_MAX_TILES;
    int* tile_shift = tile_cursor + NOALLOC_MAX_TILES;
    unsigned long long* tile_gmax = (unsigned long long*)(tile_shift + NOALLOC_MAX_TILES);
    Rec<T>* recs = (Rec<T>*)(base + NOALLOC_HEADER + NOALLOC_TILE_BYTES);
    const double inv_dx = 1.0 / d->dx;
    // the array keeps the previous call's contents: clear what accumulates
    if (cudaMemsetAsync(base, 0, NOALLOC_HEADER, s) != cudaSuccess) return PF_ERR_CUDA;
    if (cudaMemsetAsync(tile_count, 0, ntiles * sizeof(int), s) != cudaSuccess) return PF_ERR_CUDA;
    if (cudaMemsetAsync(tile_gmax, 0, ntiles * sizeof(unsigned long long), s) != cudaSuccess) return PF_ERR_CUDA;
    const int nb = nv > 0 ? (int)std::min<int64_t>(ceil_div(nv, 256), 152 * 16) : 0;
    if (nb > 0)
        k_bin_count<<<nb, 256, 0, s>>>(X, Y, G, nv, d->x0, d->y0, inv_dx, d->nx, d->ny, ntx, tile_count, tile_gmax,
                                       status, oob);
    k_bin_scan<<<1, 1024, 0, s>>>(tile_count, tile_gmax, tile_start, tile_cursor, tile_shift, ntiles);
    if (nb > 0)
        k_bin_scatter<T><<<nb, 256, 0, s>>>(X, Y, G, nv, d->x0, d->y0, inv_dx, d->nx, d->ny, ntx, tile_start,
                                            tile_cursor, recs);
    k_regularize<T><<<ntiles, 256, 0, s>>>(recs, tile_start, tile_count, tile_shift, d->nx, d->ny, ntx,
                                           inv_dx * inv_dx, w);
    if (cudaGetLastError() != cudaSuccess) return PF_ERR_CUDA;
    if (out_of_domain &&
        cudaMemcpyAsync(out_of_domain, oob, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return PF_ERR_CUDA;
    return PF_OK;
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
    if (d->precision == PF_FP64)
        return regularize_noalloc_t<double>(d, X, Y, G, nv, (double*)w, out_of_domain, s, base);
    return regularize_noalloc_t<float>(d, X, Y, G, nv, (float*)w, out_of_domain, s, base);
}

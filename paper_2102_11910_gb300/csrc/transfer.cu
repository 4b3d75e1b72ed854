// Vortex <-> grid transfer with the M4' kernel (Sec. 2.1):
//   R_v (Eq. vortexregularization): w_ij = dx^-2 sum_q Gamma_q d((x_i-X_q)/dx) d((y_j-Y_q)/dx)
//   E_v = R_v^T:                    u_q  = sum_ij d d u_ij
//
// Regularization is a binned scatter in four kernels:
//   locate   FP64 position -> integer cell + fraction (one pass, FP64 used only
//            for g = (X - x0)/dx), compact per-vortex record, per-block tile
//            histogram in shared memory, written out as one row per block;
//   offsets  column scan of the block histograms: the tile totals and the first
//            record slot of every (block, tile) pair within its tile;
//   scatter  per-block ranks in shared memory, records written into their
//            tiles at the block's offsets (no global atomics); a vortex whose
//            4x4 stencil straddles tiles is entered in every tile it touches;
//   deposit  one block per BIN_TILE^2 node tile sums its records in shared
//            memory as fixed-point integers with a per-tile scale chosen from
//            the tile's record count and largest |Gamma|.  Integer sums are
//            exact, so the result does not depend on the order of the adds.
//
#include <math.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "transfer.cuh"

namespace {

pf_status plan_bin_reserve(pf_plan p, int64_t nv) {
    const size_t psz = p->prec == PF_FP64 ? sizeof(Pos<double>) : sizeof(Pos<float>);
    const size_t rsz = p->prec == PF_FP64 ? sizeof(Rec<double>) : sizeof(Rec<float>);
    if (nv > (int64_t)1 << 29) {   // record slots are 32-bit
        snprintf(p->err, sizeof(p->err), "%lld vortices exceed the 2^29 a plan can bin", (long long)nv);
        return PF_ERR_CAPACITY;
    }
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
        p->recs = nullptr;
        p->rec_cap = 0;
        PF_CUDA(p, cudaMalloc(&p->recs, (size_t)cap * rsz));
        p->rec_cap = cap;
    }
    const int64_t ntiles = (int64_t)ceil_div(p->nx, p->tile) * ceil_div(p->ny, p->tile);
    const int64_t need = (int64_t)bin_blocks(nv, p->min_span) * ntiles;
    if (need > p->bin_off_cap) {
        const int64_t cap = std::max<int64_t>(need, (int64_t)bin_blocks(p->pos_cap, p->min_span) * ntiles);
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        if (p->bin_off) cudaFree(p->bin_off);
        p->bin_off = nullptr;
        p->bin_off_cap = 0;
        PF_CUDA(p, cudaMalloc(&p->bin_off, (size_t)cap * sizeof(int)));
        p->bin_off_cap = cap;
    }
    return PF_OK;
}

BinWork plan_binwork(pf_plan p) {
    BinWork b;
    b.status = p->d_status;
    b.oob = p->d_oob;
    b.tile_count = p->tile_count;
    b.gmax = p->gmax;
    b.tile_start = p->tile_start;
    b.bin_off = p->bin_off;
    b.pos = p->pos;
    b.recs = p->recs;
    b.rec_cap = p->rec_cap;
    return b;
}

template <typename T>
pf_status regularize_configured(pf_plan p, const BinWork& bw, const double* X, const double* Y, const double* G,
                                int64_t nv, T* w, const int64_t* dn) {
    const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0, p->tile);
    p->bin_tile = p->tile;
    if (p->tile == BIN_TILE_SMALL)
        return regularize_launch<T, BIN_TILE_SMALL>(p, geo, bw, X, Y, G, nv, w, p->stream, p->min_span,
                                                    p->tile_threads, dn);
    return regularize_launch<T, BIN_TILE>(p, geo, bw, X, Y, G, nv, w, p->stream, p->min_span, p->tile_threads, dn);
}

template <int TILE>
pf_status interpolate_tiles(pf_plan p, const Geo& geo, const void* uv, int64_t nq, void* uq, void* vq) {
    if (p->prec == PF_FP64)
        PF_KERNEL(p, "interpolate", PF_CUDA(p, pf_launch(k_interp_tiles<double, TILE>, geo.ntiles, p->tile_threads, 0,
                                                         p->stream, (const Rec<double>*)p->recs, p->tile_start,
                                                         p->tile_count, (const double2*)uv, geo, (double*)uq,
                                                         (double*)vq, p->rec_cap, nq, p->d_status)));
    else
        // 256 threads whatever the plan's tile_threads: four records a thread
        // make the sort's chunks 1024 records (128-thread blocks with eight a
        // thread fit six blocks an SM, a second wave at 1024 tiles: 28.7 us
        // against 24.5 us at 1024^2 / 1e6)
        PF_KERNEL(p, "interpolate", PF_CUDA(p, pf_launch(k_interp_tiles_f32<TILE, 4>, geo.ntiles, 256,
                                                         (size_t)(4 * 256 + 32) * sizeof(Rec<float>), p->stream,
                                                         (const Rec<float>*)p->recs, p->tile_start, p->tile_count,
                                                         (const float2*)uv, geo, (float*)uq, (float*)vq, p->rec_cap,
                                                         nq, p->d_status)));
    return PF_OK;
}

}  // namespace

// the plan's binning scratch (cell records, histograms, status words)
BinWork plan_binwork_for(pf_plan p) { return plan_binwork(p); }

// size the plan's vortex buffers for nv vortices ahead of time
pf_status plan_reserve_vortices(pf_plan p, int64_t nv) { return plan_bin_reserve(p, nv); }

// R_v in the plan's launch configuration (tile edge, block partition, threads).
// With dn, the count is read on the device from dn[0] and nv (the capacity)
// only sizes the launches.  With zu, zv (the E_v outputs that follow), every
// vortex off the grid gets a zero velocity there.
pf_status vortex_regularize(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, void* w,
                            const int64_t* dn, void* zu, void* zv) {
    pf_status st = plan_bin_reserve(p, nv);
    if (st != PF_OK) return st;
    BinWork bw = plan_binwork(p);
    bw.zu = zu;
    bw.zv = zv;
    if (p->prec == PF_FP64) return regularize_configured<double>(p, bw, X, Y, G, nv, (double*)w, dn);
    return regularize_configured<float>(p, bw, X, Y, G, nv, (float*)w, dn);
}

// E_v at the vortices the last vortex_regularize call binned (in that call's tiles)
pf_status vortex_interpolate_located(pf_plan p, const void* uv, int64_t nq, void* uq, void* vq) {
    if (nq == 0) return PF_OK;
    const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0, p->bin_tile);
    if (p->bin_tile == BIN_TILE_SMALL) return interpolate_tiles<BIN_TILE_SMALL>(p, geo, uv, nq, uq, vq);
    return interpolate_tiles<BIN_TILE>(p, geo, uv, nq, uq, vq);
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
// status words, the per-vortex cell records and the binned records) lives in
// one file-scope device array, so the entry point needs no plan and makes no
// allocation.  The array is part of the library image: each GPU that loads the
// library holds NOALLOC_SCRATCH_BYTES of it until the process exits.
namespace {

constexpr int64_t NOALLOC_MAX_VORTICES = 65536;
constexpr int NOALLOC_MAX_TILES = (2048 / BIN_TILE) * (2048 / BIN_TILE);
constexpr int NOALLOC_MAX_BLOCKS = (int)(NOALLOC_MAX_VORTICES / 1024);   // bin_blocks() at the maximum
// every region starts on a 256-byte boundary (the records are stored 16 bytes at a time)
constexpr size_t noalloc_round(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NOALLOC_HEADER = 256;   // status int + out-of-domain counter, padded
constexpr size_t NOALLOC_TILE_BYTES = noalloc_round((size_t)NOALLOC_MAX_TILES * 2 * sizeof(int) + (NOALLOC_MAX_BLOCKS + 1) * 8);
constexpr size_t NOALLOC_OFF_BYTES = noalloc_round((size_t)NOALLOC_MAX_BLOCKS * NOALLOC_MAX_TILES * sizeof(int));
constexpr size_t NOALLOC_POS_BYTES = noalloc_round((size_t)NOALLOC_MAX_VORTICES * sizeof(Pos<double>));
static_assert((size_t)NOALLOC_MAX_TILES * 2 * sizeof(int) % 8 == 0, "the |Gamma| maxima are 8-byte aligned");
static_assert(NOALLOC_HEADER % 256 == 0 && NOALLOC_TILE_BYTES % 256 == 0 && NOALLOC_OFF_BYTES % 256 == 0 &&
                  NOALLOC_POS_BYTES % 256 == 0,
              "scratch regions stay 256-byte aligned");
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_HEADER + NOALLOC_TILE_BYTES + NOALLOC_OFF_BYTES + NOALLOC_POS_BYTES +
                                         (size_t)4 * NOALLOC_MAX_VORTICES * sizeof(Rec<double>);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {nullptr};

// Resolve the array's device address for the current device (first call per
// device only; later calls read the cached address under the same lock).  The
// host-side name g_noalloc_scratch is not a device address.
cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = (unsigned char*)ptr;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

BinWork noalloc_binwork(unsigned char* base) {
    BinWork b;
    b.status = (int*)base;
    b.oob = (unsigned long long*)(base + 8);
    unsigned* t = (unsigned*)(base + NOALLOC_HEADER);
    b.tile_count = t;
    b.tile_start = (int*)(t + NOALLOC_MAX_TILES);
    b.gmax = (double*)(t + 2 * NOALLOC_MAX_TILES);
    b.bin_off = (int*)(base + NOALLOC_HEADER + NOALLOC_TILE_BYTES);
    b.pos = base + NOALLOC_HEADER + NOALLOC_TILE_BYTES + NOALLOC_OFF_BYTES;
    b.recs = base + NOALLOC_HEADER + NOALLOC_TILE_BYTES + NOALLOC_OFF_BYTES + NOALLOC_POS_BYTES;
    b.rec_cap = 4 * NOALLOC_MAX_VORTICES;
    return b;
}

// status word bits -> the pf_status the call reports (the same order as pf_sync)
__global__ void k_noalloc_status(const int* __restrict__ bits, int32_t* __restrict__ out) {
    const int st = *bits;
    *out = (st & ST_INTERNAL) ? PF_ERR_INTERNAL : (st & ST_OUT_OF_DOMAIN) ? PF_ERR_OUT_OF_DOMAIN : PF_OK;
}

}  // namespace

extern "C" pf_status pf_regularize_noalloc(const pf_grid_desc* d, const double* X, const double* Y, const double* G,
                                           int64_t nv, void* w, int64_t* out_of_domain, int32_t* status,
                                           void* stream) {
    if (!d || !w || nv < 0 || (nv > 0 && (!X || !Y || !G))) return PF_ERR_ARG;
    if (d->nx < 8 || d->ny < 8 || d->nx > 2048 || d->ny > 2048 || !(d->dx > 0) || !isfinite(d->x0) ||
        !isfinite(d->y0) || (d->precision != PF_FP64 && d->precision != PF_MIXED))
        return PF_ERR_ARG;
    if (nv > NOALLOC_MAX_VORTICES || bin_blocks(nv) > NOALLOC_MAX_BLOCKS) return PF_ERR_CAPACITY;
    unsigned char* base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) return PF_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Geo geo = make_geo(d->nx, d->ny, d->dx, d->x0, d->y0);
    const BinWork bw = noalloc_binwork(base);
    // the array keeps the previous call's contents: clear the status words
    // (every other piece of scratch is written before it is read)
    if (cudaMemsetAsync(base, 0, NOALLOC_HEADER, s) != cudaSuccess) return PF_ERR_CUDA;
    pf_status st = d->precision == PF_FP64
                       ? regularize_launch<double>(nullptr, geo, bw, X, Y, G, nv, (double*)w, s)
                       : regularize_launch<float>(nullptr, geo, bw, X, Y, G, nv, (float*)w, s);
    if (st != PF_OK) return st;
    if (cudaGetLastError() != cudaSuccess) return PF_ERR_CUDA;
    if (out_of_domain &&
        cudaMemcpyAsync(out_of_domain, bw.oob, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return PF_ERR_CUDA;
    if (status) {
        k_noalloc_status<<<1, 1, 0, s>>>(bw.status, status);
        if (cudaGetLastError() != cudaSuccess) return PF_ERR_CUDA;
    }
    return PF_OK;
}

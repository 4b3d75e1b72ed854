// Tile-ordered vortex state for body-free vortex-in-cell time stepping
// (Sec. 2.1 operators R_v, L^-1, E_v; vortices advected with the local
// velocity, forward Euler as in Sec. 2.4.2).
//
// The state keeps its vortices as binned records: every vortex has a home
// record in the 32 x 32 node tile holding its cell, and a copy in each other
// tile its 4 x 4 stencil reaches, exactly the layout one regularization pass
// builds from positions.  A step therefore needs no binning from scratch:
//
//   deposit    R_v from the records (the regularization kernel);
//   velocity   the spectral node velocity (the FFT convolution);
//   advect     per tile: E_v at every home record from the tile's velocity
//              patch, the position moved by dt (u, v) in fixed point, the new
//              record kept at the old slot, the number of records bound for
//              each tile of the 5 x 5 block around it, added into the new
//              tile counts;
//   offsets    one block: the new tile starts (a scan of the counts);
//   scatter    per source tile: a slice of every destination tile claimed with
//              one atomic add, records copied to their new tiles (home and
//              straddled), into the other record buffer.  The order of the
//              source slices inside a tile is arbitrary; nothing depends on it
//              (the deposit sums integers, everything else is per record).
//
// A vortex's home tile may move by at most one tile a step (always true for
// moves under 32 cells); a faster vortex, and one whose stencil leaves the
// grid, is dropped and reported (PF_ERR_CAPACITY / PF_ERR_OUT_OF_DOMAIN at
// pf_sync).
#include "transfer.cuh"

struct pf_vic_state_s {
    pf_plan plan = nullptr;           // grid, precision, stream (not owned)
    int64_t cap = 0;                  // vortex capacity
    int64_t nv0 = 0;                  // vortices given to the last set call (original indices 0 .. nv0-1)
    int64_t rec_cap = 0;              // record slots per buffer
    void* recs[2] = {nullptr, nullptr};
    void* moved = nullptr;            // rec_cap advected records (slot of the old buffer)
    unsigned* tcount[2] = {nullptr, nullptr};
    int* tstart[2] = {nullptr, nullptr};
    int* dcount = nullptr;            // 25 x ntiles: records per (destination, source tile), direction-major
    int* fill = nullptr;              // ntiles: next free slot of each new tile
    double* gmax = nullptr;           // [0]: bound on |Gamma| (fixed by set; vortices keep their strengths)
    long long* nrec = nullptr;        // [0] records, [1] vortices after the last step
    int cur = 0;
    double t = 0.0;
};

namespace {

constexpr int NDIR = 25;               // destinations: tiles (dx, dy) in [-2, 2]^2 around the source
constexpr int PATCH = BIN_TILE + 3;     // staged (u, v) nodes per tile edge: one before, two after
constexpr int MOVE_BIAS = 34;          // moved mixed records keep lx + 34, ly + 34 (cells -34 .. 221 of the source tile)

__device__ __forceinline__ int dir_of(int dtx, int dty) { return (dty + 2) * 5 + (dtx + 2); }

// advected record, local cell relative to the SOURCE tile
template <typename T> struct Moved;
template <> struct __align__(16) Moved<float> {
    unsigned xw, yw;      // (fraction * 2^32) & ~0xFF | (local cell + MOVE_BIAS)
    float g;
    int q;                // original index; -1: no record (a copy, or a dropped vortex)
};
template <> struct __align__(16) Moved<double> {
    short lx, ly;
    int q;
    double fx, fy, g;
};

__device__ __forceinline__ int mv_lx(const Moved<float>& m) { return (int)(m.xw & 0xFFu) - MOVE_BIAS; }
__device__ __forceinline__ int mv_ly(const Moved<float>& m) { return (int)(m.yw & 0xFFu) - MOVE_BIAS; }
__device__ __forceinline__ int mv_lx(const Moved<double>& m) { return m.lx; }
__device__ __forceinline__ int mv_ly(const Moved<double>& m) { return m.ly; }

__device__ __forceinline__ Rec<float> rec_at(const Moved<float>& m, int lx, int ly) {
    Rec<float> r;
    r.xw = (m.xw & ~0xFFu) | (unsigned)(lx + 2);
    r.yw = (m.yw & ~0xFFu) | (unsigned)(ly + 2);
    r.g = m.g;
    r.q = m.q;
    return r;
}
__device__ __forceinline__ Rec<double> rec_at(const Moved<double>& m, int lx, int ly) {
    Rec<double> r;
    r.lx = (short)lx;
    r.ly = (short)ly;
    r.q = m.q;
    r.fx = m.fx;
    r.fy = m.fy;
    r.g = m.g;
    return r;
}

// Move one coordinate by d cells: local cell c with fraction f (mixed: the top
// 24 bits of a 32-bit fixed-point word; FP64: a double in [0, 1)).
__device__ __forceinline__ void move_axis(unsigned word, float d, int& c, unsigned& out) {
    // the fraction and the displacement in units of 2^-24 cell, added exactly
    const long long f = (long long)(word >> 8);
    const long long dd = __float2ll_rn(d * 0x1p24f);
    const long long s = f + dd;
    const long long cs = s >> 24;                    // floor
    c += (int)cs;
    out = (unsigned)((s - (cs << 24)) << 8);
}
__device__ __forceinline__ void move_axis(double f, double d, int& c, double& out) {
    const double s = f + d;
    const double fl = floor(s);
    c += (int)fl;
    out = s - fl;
}

// Destinations of a record whose new cell is (ci, cj) relative to the source
// tile: the tiles its stencil cells ci-1 .. ci+2 touch.  Returns false if one
// lies outside the 5 x 5 block (the vortex moved too far).
__device__ __forceinline__ bool dest_range(int ci, int cj, int& x0, int& x1, int& y0, int& y1) {
    x0 = (ci - 1 + 64) / BIN_TILE - 2;     // floor division for ci - 1 >= -64
    x1 = (ci + 2 + 64) / BIN_TILE - 2;
    y0 = (cj - 1 + 64) / BIN_TILE - 2;
    y1 = (cj + 2 + 64) / BIN_TILE - 2;
    return x0 >= -2 && x1 <= 2 && y0 >= -2 && y1 <= 2;
}

// A home record of the source tile after the move: returns false (and reports)
// if the vortex left the grid or moved too far; else its destinations.
__device__ __forceinline__ bool moved_dest(int ci, int cj, int tx, int ty, const Geo& geo, int& x0, int& x1, int& y0,
                                           int& y1, int* status, unsigned long long* oob) {
    const int gi = tx * BIN_TILE + ci, gj = ty * BIN_TILE + cj;
    if (gi < 1 || gi > geo.nx - 3 || gj < 1 || gj > geo.ny - 3) {
        atomicAdd(oob, 1ull);
        atomicOr(status, ST_OUT_OF_DOMAIN);
        return false;
    }
    if (ci < -BIN_TILE || ci >= 2 * BIN_TILE || cj < -BIN_TILE || cj >= 2 * BIN_TILE || !dest_range(ci, cj, x0, x1, y0, y1)) {
        atomicOr(status, ST_CAPACITY);
        return false;
    }
    return true;
}

// E_v and the Euler move of every home record of a tile.  The tile's velocity
// patch (nodes -1 .. 33 in each direction) is staged in shared memory; the
// advected record goes to moved[slot]; the block counts its records per
// destination tile (a vortex whose new stencil straddles tiles is counted in
// each of them).  Optionally writes the velocity at the vortex's original
// index.
template <typename T>
__global__ void __launch_bounds__(256) k_vic_advect(const Rec<T>* __restrict__ recs, const int* __restrict__ tile_start,
                                                    const unsigned* __restrict__ tile_count,
                                                    const C_t<T>* __restrict__ uv, Geo geo, T dt_dx,
                                                    Moved<T>* __restrict__ moved, int* __restrict__ dcount,
                                                    unsigned* __restrict__ tcount_next,
                                                    T* __restrict__ uq, T* __restrict__ vq, int64_t rec_cap,
                                                    int64_t nq, int* __restrict__ status,
                                                    unsigned long long* __restrict__ oob) {
    using C = C_t<T>;
    __shared__ C patch[PATCH * PATCH];
    __shared__ int lcnt[NDIR];
    const int t = blockIdx.x;
    const int tx = t % geo.ntx, ty = t / geo.ntx;
    if (threadIdx.x < NDIR) lcnt[threadIdx.x] = 0;
    pdl_wait();
    const int cnt = (int)tile_count[t];
    const int start = tile_start[t];
    const bool ok = start >= 0 && cnt >= 0 && (int64_t)start + cnt <= rec_cap;     // block-uniform
    if (!ok && threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    const int n = ok ? cnt : 0;
    if (n > 0) {
        const int gi0 = tx * BIN_TILE - 1, gj0 = ty * BIN_TILE - 1;
        for (int i = threadIdx.x; i < PATCH * PATCH; i += blockDim.x) {
            const int gi = gi0 + i % PATCH, gj = gj0 + i / PATCH;
            C v = cmake<C>(T(0), T(0));
            if (gi >= 0 && gi < geo.nx && gj >= 0 && gj < geo.ny) v = uv[(size_t)gj * geo.nx + gi];
            patch[i] = v;
        }
    }
    __syncthreads();
    constexpr int U = 4;
    for (int r0 = 0; r0 < n; r0 += U * 256) {
      Rec<T> rcs[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {          // clamped: a thread past the end reloads the last record
          const int r = r0 + u * 256 + (int)threadIdx.x;
          rcs[u] = recs[start + (r < n ? r : n - 1)];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u * 256 + threadIdx.x;
        if (r >= n) break;
        const Rec<T> rc = rcs[u];
        const int lx = rec_lx(rc), ly = rec_ly(rc);
        Moved<T> m = {};
        m.q = -1;
        if (lx >= 0 && lx < BIN_TILE && ly >= 0 && ly < BIN_TILE) {
            T wx[4], wy[4];
            m4p_weights<T>(rec_fx(rc), wx);
            m4p_weights<T>(rec_fy(rc), wy);
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
            if (uq != nullptr && rc.q >= 0 && rc.q < nq) {
                uq[rc.q] = su;
                vq[rc.q] = sv;
            }
            int ci = lx, cj = ly;
            Moved<T> mv = {};
            if constexpr (sizeof(T) == 4) {
                move_axis(rc.xw, su * dt_dx, ci, mv.xw);
                move_axis(rc.yw, sv * dt_dx, cj, mv.yw);
            } else {
                move_axis(rc.fx, su * dt_dx, ci, mv.fx);
                move_axis(rc.fy, sv * dt_dx, cj, mv.fy);
            }
            int x0, x1, y0, y1;
            if (moved_dest(ci, cj, tx, ty, geo, x0, x1, y0, y1, status, oob)) {
                if constexpr (sizeof(T) == 4) {
                    mv.xw = (mv.xw & ~0xFFu) | (unsigned)(ci + MOVE_BIAS);
                    mv.yw = (mv.yw & ~0xFFu) | (unsigned)(cj + MOVE_BIAS);
                } else {
                    mv.lx = (short)ci;
                    mv.ly = (short)cj;
                }
                mv.g = rc.g;
                mv.q = rc.q;
                m = mv;
                for (int dy = y0; dy <= y1; ++dy)
                    for (int dx = x0; dx <= x1; ++dx) atomicAdd(&lcnt[dir_of(dx, dy)], 1);
            }
        }
        moved[start + r] = m;
      }
    }
    __syncthreads();
    if (threadIdx.x < NDIR) {
        const int c = lcnt[threadIdx.x];
        dcount[(size_t)threadIdx.x * gridDim.x + t] = c;
        if (c) {          // destination tiles exist: every counted record lies inside the grid
            const int T = t + (threadIdx.x / 5 - 2) * geo.ntx + (threadIdx.x % 5 - 2);
            atomicAdd(&tcount_next[T], (unsigned)c);
        }
    }
}

// New tile starts: one block scans the new tile counts (coalesced), and sets
// each tile's fill pointer to its start.
constexpr int OFF_PER = 4;              // tiles per thread: 1024 * 4 >= 64 * 64 tiles
__global__ void __launch_bounds__(1024) k_vic_offsets(const unsigned* __restrict__ tcount, int ntiles,
                                                      int* __restrict__ tstart, int* __restrict__ fill,
                                                      int64_t rec_cap, long long* __restrict__ nrec,
                                                      int* __restrict__ status) {
    __shared__ int wsum[32];
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;     // <= OFF_PER
    const int t0 = threadIdx.x * per;
    pdl_wait();
    if (threadIdx.x == 0) nrec[1] = 0;       // vortices: counted by the scatter pass
    int c[OFF_PER];
    int mine = 0;
#pragma unroll
    for (int k = 0; k < OFF_PER; ++k) {
        const int T = t0 + k;
        const bool in = k < per && T < ntiles;
        c[k] = (int)tcount[in ? T : 0];
        c[k] = in ? c[k] : 0;
        mine += c[k];
    }
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
#pragma unroll
    for (int k = 0; k < OFF_PER; ++k) {
        const int T = t0 + k;
        if (k < per && T < ntiles) {
            tstart[T] = run;
            fill[T] = run;
        }
        run += c[k];
    }
    if (threadIdx.x == blockDim.x - 1) {
        nrec[0] = run;
        if (run > rec_cap) atomicOr(status, ST_CAPACITY);
    }
}
static_assert(1024 * OFF_PER >= (2048 / BIN_TILE) * (2048 / BIN_TILE), "the offsets block covers every tile");

// Copy every advected record of a source tile to its destination tiles.  The
// tile's slices are claimed into shared memory once; records are loaded four
// per thread at a time.
template <typename T>
__device__ __forceinline__ void scatter_one(const Moved<T>& m, bool live, const int* base, int* lcnt, int64_t rec_cap,
                                            Rec<T>* __restrict__ out, int& homes, int* status) {
    int ci = 0, cj = 0, x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    if (live) {
        ci = mv_lx(m);
        cj = mv_ly(m);
        dest_range(ci, cj, x0, x1, y0, y1);
        ++homes;
    }
    // the home tile (the one holding the cell): records that stay in the
    // source tile (nearly all) take their slots with one shared add per warp
    const int hx = live ? (ci + 64) / BIN_TILE - 2 : 0, hy = live ? (cj + 64) / BIN_TILE - 2 : 0;
    const int hd = dir_of(hx, hy);
    const bool stay = live && hd == dir_of(0, 0);
    const unsigned peers = __ballot_sync(0xffffffffu, stay);
    int hslot = 0;
    if (peers) {
        const int leader = __ffs(peers) - 1;
        const int lane = threadIdx.x & 31;
        int b = 0;
        if (lane == leader) b = atomicAdd(&lcnt[dir_of(0, 0)], __popc(peers));
        b = __shfl_sync(0xffffffffu, b, leader);
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        hslot = b + __popc(peers & lt);
    }
    if (!live) return;
    if (!stay) hslot = atomicAdd(&lcnt[hd], 1);
    for (int dy = y0; dy <= y1; ++dy)
        for (int dx = x0; dx <= x1; ++dx) {
            const int d = dir_of(dx, dy);
            const int k = (d == hd) ? hslot : atomicAdd(&lcnt[d], 1);
            const long long slot = (long long)base[d] + k;
            if (slot < 0 || slot >= rec_cap) {
                atomicOr(status, ST_INTERNAL);
                continue;
            }
            out[slot] = rec_at(m, ci - dx * BIN_TILE, cj - dy * BIN_TILE);
        }
}

template <typename T>
__global__ void __launch_bounds__(256) k_vic_scatter(const Moved<T>* __restrict__ moved,
                                                     const int* __restrict__ tile_start,
                                                     const unsigned* __restrict__ tile_count,
                                                     const int* __restrict__ dcount, int ntx,
                                                     int* __restrict__ fill, int64_t rec_cap,
                                                     Rec<T>* __restrict__ out, long long* __restrict__ nrec,
                                                     int* __restrict__ status) {
    __shared__ int lcnt[NDIR];
    __shared__ int base[NDIR];
    __shared__ int nhome;
    const int t = blockIdx.x;
    pdl_wait();
    if (threadIdx.x < NDIR) {               // this source tile's slice of each destination tile
        lcnt[threadIdx.x] = 0;
        const int c = dcount[(size_t)threadIdx.x * gridDim.x + t];
        base[threadIdx.x] = c ? atomicAdd(&fill[t + (threadIdx.x / 5 - 2) * ntx + (threadIdx.x % 5 - 2)], c) : 0;
    }
    if (threadIdx.x == 0) nhome = 0;
    __syncthreads();
    const int cnt = (int)tile_count[t];
    const int start = tile_start[t];
    if (!(start >= 0 && cnt >= 0 && (int64_t)start + cnt <= rec_cap)) return;   // reported by the advect pass
    constexpr int U = 4;
    int homes = 0;
    for (int r0 = 0; r0 < cnt; r0 += U * 256) {              // trip count uniform over the block
        Moved<T> m[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {          // clamped loads; past the end counts as no record
            const int r = r0 + u * 256 + (int)threadIdx.x;
            m[u] = moved[start + (r < cnt ? r : cnt - 1)];
            if (r >= cnt) m[u].q = -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) scatter_one<T>(m[u], m[u].q >= 0, base, lcnt, rec_cap, out, homes, status);
    }
    for (int o = 16; o > 0; o >>= 1) homes += __shfl_xor_sync(0xffffffffu, homes, o);
    if ((threadIdx.x & 31) == 0 && homes) atomicAdd(&nhome, homes);
    __syncthreads();
    if (threadIdx.x == 0 && nhome)
        atomicAdd(reinterpret_cast<unsigned long long*>(nrec + 1), (unsigned long long)nhome);
}

// FP64 positions of the home records at their original indices.
template <typename T>
__global__ void k_vic_get(const Rec<T>* __restrict__ recs, const int* __restrict__ tile_start,
                          const unsigned* __restrict__ tile_count, Geo geo, double* __restrict__ X,
                          double* __restrict__ Y, double* __restrict__ G, int64_t nq) {
    const int t = blockIdx.x;
    const int tx = t % geo.ntx, ty = t / geo.ntx;
    const int cnt = (int)tile_count[t], start = tile_start[t];
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const Rec<T> rc = recs[start + r];
        const int lx = rec_lx(rc), ly = rec_ly(rc);
        if (lx < 0 || lx >= BIN_TILE || ly < 0 || ly >= BIN_TILE || rc.q < 0 || rc.q >= nq) continue;
        X[rc.q] = geo.x0 + ((double)(tx * BIN_TILE + lx) + (double)rec_fx(rc)) * geo.dx;
        Y[rc.q] = geo.y0 + ((double)(ty * BIN_TILE + ly) + (double)rec_fy(rc)) * geo.dx;
        G[rc.q] = (double)rc.g;
    }
}

__global__ void k_fill_nan(double* a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = __longlong_as_double(0x7FF8000000000000ll);
}

void free_state(pf_vic_state s) {
    void* own[] = {s->recs[0], s->recs[1], s->moved, s->tcount[0], s->tcount[1], s->tstart[0], s->tstart[1],
                   s->dcount, s->fill, s->gmax, s->nrec};
    for (void* q : own)
        if (q) cudaFree(q);
}

template <typename T>
pf_status vic_step_t(pf_vic_state s, double dt, double Uinf, double Vinf, T* uq, T* vq) {
    pf_plan p = s->plan;
    const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0);
    const int c = s->cur, n = c ^ 1;
    const Rec<T>* rc = (const Rec<T>*)s->recs[c];
    PF_TRY((deposit_launch<T, BIN_TILE>(p, geo, rc, s->tstart[c], s->tcount[c], s->gmax, s->rec_cap, p->d_status,
                                        (T*)p->w, p->stream)));
    PF_TRY(conv_solve(p, p->w, p->uv, CONV_UV, Uinf, Vinf));
    PF_CUDA(p, cudaMemsetAsync(s->tcount[n], 0, (size_t)geo.ntiles * sizeof(unsigned), p->stream));
    PF_KERNEL(p, "vic_advect", PF_CUDA(p, pf_launch(k_vic_advect<T>, geo.ntiles, 256, 0, p->stream, rc, s->tstart[c],
                                                   s->tcount[c], (const C_t<T>*)p->uv, geo, (T)(dt / p->dx),
                                                   (Moved<T>*)s->moved, s->dcount, s->tcount[n], uq, vq, s->rec_cap,
                                                   s->nv0, p->d_status, p->d_oob)));
    PF_KERNEL(p, "vic_offsets", PF_CUDA(p, pf_launch(k_vic_offsets, 1, 1024, 0, p->stream,
                                                    (const unsigned*)s->tcount[n], geo.ntiles, s->tstart[n], s->fill,
                                                    s->rec_cap, s->nrec, p->d_status)));
    PF_KERNEL(p, "vic_scatter", PF_CUDA(p, pf_launch(k_vic_scatter<T>, geo.ntiles, 256, 0, p->stream,
                                                    (const Moved<T>*)s->moved, s->tstart[c], s->tcount[c],
                                                    (const int*)s->dcount, geo.ntx, s->fill, s->rec_cap,
                                                    (Rec<T>*)s->recs[n], s->nrec, p->d_status)));
    s->cur = n;
    s->t += dt;
    return PF_OK;
}

}  // namespace

BinWork plan_binwork_for(pf_plan p);                       // transfer.cu

extern "C" {

pf_status pf_vic_state_create(pf_plan p, int64_t capacity, pf_vic_state* out) {
    if (!p || !out || capacity < 1 || capacity > ((int64_t)1 << 27)) return PF_ERR_ARG;
    *out = nullptr;
    pf_vic_state s = new (std::nothrow) pf_vic_state_s();
    if (!s) return PF_ERR_OOM;
    s->plan = p;
    s->cap = capacity;
    s->rec_cap = 4 * capacity;      // a vortex has at most four records
    const size_t rsz = p->prec == PF_FP64 ? sizeof(Rec<double>) : sizeof(Rec<float>);
    auto fail = [&](cudaError_t e) {
        snprintf(p->err, sizeof(p->err), "pf_vic_state_create: %s", cudaGetErrorString(e));
        free_state(s);
        delete s;
        return e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
    };
    cudaError_t e = cudaSuccess;
    const size_t nt = (size_t)p->ntiles;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMalloc(&s->recs[i], (size_t)s->rec_cap * rsz);
        if (e == cudaSuccess) e = cudaMalloc(&s->tcount[i], nt * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMalloc(&s->tstart[i], nt * sizeof(int));
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->moved, (size_t)s->rec_cap * rsz);
    if (e == cudaSuccess) e = cudaMalloc(&s->dcount, nt * NDIR * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&s->fill, nt * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&s->gmax, (BIN_MAX_BLOCKS + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->nrec, 2 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->tcount[0], 0, nt * sizeof(unsigned), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->tstart[0], 0, nt * sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->gmax, 0, sizeof(double), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->nrec, 0, 2 * sizeof(long long), p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(e);
    *out = s;
    return PF_OK;
}

pf_status pf_vic_state_destroy(pf_vic_state s) {
    if (!s) return PF_ERR_ARG;
    cudaStreamSynchronize(s->plan->stream);
    free_state(s);
    delete s;
    return PF_OK;
}

pf_status pf_vic_state_set(pf_vic_state s, const double* X, const double* Y, const double* G, int64_t nv) {
    if (!s || nv < 0 || nv > s->cap || (nv > 0 && (!X || !Y || !G))) return PF_ERR_ARG;
    pf_plan p = s->plan;
    PF_TRY(plan_reserve_vortices(p, nv));        // the plan's per-vortex cell records and histograms
    BinWork bw = plan_binwork_for(p);
    bw.recs = s->recs[0];
    bw.rec_cap = s->rec_cap;
    bw.tile_count = s->tcount[0];
    bw.tile_start = s->tstart[0];
    bw.gmax = s->gmax;
    const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0);
    if (p->prec == PF_FP64) PF_TRY(bin_launch<double>(p, geo, bw, X, Y, G, nv, p->stream));
    else PF_TRY(bin_launch<float>(p, geo, bw, X, Y, G, nv, p->stream));
    const long long cnt[2] = {0, (long long)nv};
    PF_CUDA(p, cudaMemcpyAsync(s->nrec, cnt, sizeof(cnt), cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));      // cnt is a host local
    s->cur = 0;
    s->nv0 = nv;
    s->t = 0.0;
    return PF_OK;
}

pf_status pf_vic_state_get(pf_vic_state s, double* X, double* Y, double* G, int64_t* nv, double* t) {
    if (!s) return PF_ERR_ARG;
    pf_plan p = s->plan;
    if (s->nv0 > 0 && (X || Y || G)) {
        if (!X || !Y || !G) return PF_ERR_ARG;
        const Geo geo = make_geo(p->nx, p->ny, p->dx, p->x0, p->y0);
        const int nb = (int)std::min<int64_t>(ceil_div(s->nv0, 256), 1024);
        for (double* a : {X, Y, G}) {
            k_fill_nan<<<nb, 256, 0, p->stream>>>(a, s->nv0);
            PF_LAUNCH_CHECK(p);
        }
        if (p->prec == PF_FP64)
            k_vic_get<double><<<geo.ntiles, 256, 0, p->stream>>>((const Rec<double>*)s->recs[s->cur], s->tstart[s->cur],
                                                                  s->tcount[s->cur], geo, X, Y, G, s->nv0);
        else
            k_vic_get<float><<<geo.ntiles, 256, 0, p->stream>>>((const Rec<float>*)s->recs[s->cur], s->tstart[s->cur],
                                                                 s->tcount[s->cur], geo, X, Y, G, s->nv0);
        PF_LAUNCH_CHECK(p);
    }
    if (nv) {
        long long cnt[2] = {0, 0};
        PF_CUDA(p, cudaMemcpyAsync(cnt, s->nrec, sizeof(cnt), cudaMemcpyDeviceToHost, p->stream));
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        *nv = (int64_t)cnt[1];
    }
    if (t) *t = s->t;
    return PF_OK;
}

pf_status pf_vic_step(pf_vic_state s, double dt, double Uinf, double Vinf, void* uq, void* vq) {
    if (!s || !(dt >= 0.0) || !isfinite(dt) || !isfinite(Uinf) || !isfinite(Vinf) || (!uq) != (!vq))
        return PF_ERR_ARG;
    if (s->plan->prec == PF_FP64) return vic_step_t<double>(s, dt, Uinf, Vinf, (double*)uq, (double*)vq);
    return vic_step_t<float>(s, dt, Uinf, Vinf, (float*)uq, (float*)vq);
}

}  // extern "C"

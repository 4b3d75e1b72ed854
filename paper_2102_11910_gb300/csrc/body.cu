// Immersed body: surface transfer, Schur complement and the constrained sheet
// solves of Sec. 2.2-2.4, in FP64.
//
//   E_s / R_s       smoothed three-point kernel (Sec. 2.2.1), E weights carry no
//                   dx factor, R_s carries dS/dx^2 (so R_s = E_s^T in the node and
//                   surface inner products)
//   S = -E L^-1 R_s (Eq. vsheet): S[p,q] = -dS_q sum_{16 x 16 node pairs} d_p G d_q,
//                   from the plan's FP64 LGF table (L^-1 = dx^2 G*)
//   S^-1            Gauss-Jordan with partial pivoting, one pivot per pair of
//                   kernel launches (no device-side waiting)
//   f0 = S^-1 1, f0hat = dS o f0, Gamma0 = <1, f0>  (Eqs. f0, circ0)
//   solves          given s0 (Eq. vsheet), circulation (Eq. circsystem), steady
//                   Kutta (Eqs. kuttasystem, s0), shedding at one edge
//                   (Eq. kuttasystem2) or two edges (Eq. twovortex)
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "body.cuh"

namespace {

// smoothed three-point delta of Yang et al. (2009), support |r| < 2
__device__ double yang3(double r) {
    const double a = fabs(r);
    const double s3 = 1.7320508075688772;
    if (a <= 1.0) {
        const double q = -12.0 * a * a + 12.0 * a + 1.0;
        return 17.0 / 48.0 + s3 * M_PI / 108.0 + a / 4.0 - a * a / 4.0 + (1.0 - 2.0 * a) / 16.0 * sqrt(q > 0 ? q : 0.0) -
               s3 / 12.0 * asin(s3 / 2.0 * (2.0 * a - 1.0));
    }
    if (a < 2.0) {
        const double q = -12.0 * a * a + 36.0 * a - 23.0;
        return 55.0 / 48.0 - s3 * M_PI / 108.0 - 13.0 * a / 12.0 + a * a / 4.0 +
               (2.0 * a - 3.0) / 48.0 * sqrt(q > 0 ? q : 0.0) + s3 / 36.0 * asin(s3 / 2.0 * (2.0 * a - 3.0));
    }
    return 0.0;
}

__device__ __forceinline__ double m4p(double r) {
    const double a = fabs(r);
    if (a <= 1.0) return 1.0 - 2.5 * a * a + 1.5 * a * a * a;
    if (a <= 2.0) return 0.5 * (2.0 - a) * (2.0 - a) * (1.0 - a);
    return 0.0;
}

__device__ __forceinline__ double lgf(const double* __restrict__ G, int nx, int m, int n) {
    return G[(size_t)(n < 0 ? -n : n) * (nx + 1) + (m < 0 ? -m : m)];
}

// four-node stencil of a point: nodes floor(g)-1 .. floor(g)+2, g = (x - x0)/dx
__device__ __forceinline__ bool stencil(double x, double x0, double dx, int n, int* idx, double* wt, bool surface) {
    const double g = (x - x0) / dx;
    const double c = floor(g);
    if (!(c >= 1.0 && c <= n - 3.0)) return false;
    const int ci = (int)c;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        idx[a] = ci - 1 + a;
        wt[a] = surface ? yang3((double)(ci - 1 + a) - g) : m4p((double)(ci - 1 + a) - g);
    }
    return true;
}

// one thread per (point p, axis, node a): the FP64 smoothed-three-point weights
// (square root and arcsine) run at the GPU's low FP64 rate, so they are spread
// over many blocks; a point whose stencil leaves the grid on either axis gets
// index 1 and weight 0 on both axes and raises the out-of-domain status
__global__ void k_surface_stencil(const double* __restrict__ x, const double* __restrict__ y, int ns, double x0,
                                  double y0, double dx, int nx, int ny, int* __restrict__ six, int* __restrict__ siy,
                                  double* __restrict__ swx, double* __restrict__ swy, int* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * ns) return;
    const int p = t >> 3, axis = (t >> 2) & 1, a = t & 3;
    const double gx = (x[p] - x0) / dx, gy = (y[p] - y0) / dx;
    const double cx = floor(gx), cy = floor(gy);
    const bool ok = cx >= 1.0 && cx <= nx - 3.0 && cy >= 1.0 && cy <= ny - 3.0;
    if (!ok && t == 8 * p) atomicOr(status, ST_OUT_OF_DOMAIN);
    const double g = axis ? gy : gx;
    const int c = ok ? (int)(axis ? cy : cx) : 0;
    const int idx = ok ? c - 1 + a : 1;
    const double wt = ok ? yang3((double)(c - 1 + a) - g) : 0.0;
    if (axis) {
        siy[4 * p + a] = idx;
        swy[4 * p + a] = wt;
    } else {
        six[4 * p + a] = idx;
        swx[4 * p + a] = wt;
    }
}

// S[p, q] = -dS_q sum_{a,b,a',b'} wx_p[a] wy_p[b] G(ix_p[a]-ix_q[a'], iy_p[b]-iy_q[b']) wx_q[a'] wy_q[b']
// A stencil's nodes are consecutive (ix_p[a] = ix_p[0] + a), so the node
// offsets are ix_p[0] - ix_q[0] + d, d = a - a' in -3..3, and the sum is
// sum_{d,e} cx[d] cy[e] G(...) with cx[d] = sum_{a-a'=d} wx_p[a] wx_q[a'] (and
// cy alike): 49 table reads instead of 256.  (A point outside the grid has
// zero weights, so its placeholder indices contribute nothing.)  The kernel
// K = S / dS_q is symmetric: the thread of (p, q >= p) writes both entries.
__device__ __forceinline__ double stencil_pair_lgf(const int* __restrict__ six, const int* __restrict__ siy,
                                                   const double* __restrict__ swx, const double* __restrict__ swy,
                                                   int p, const int* ixq, const int* iyq, const double* wxq,
                                                   const double* wyq, const double* __restrict__ G, int nx) {
    double cx[7], cy[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) cx[d] = cy[d] = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2) {
            cx[a - a2 + 3] += swx[4 * p + a] * wxq[a2];
            cy[a - a2 + 3] += swy[4 * p + a] * wyq[a2];
        }
    const int bi = six[4 * p] - ixq[0] - 3, bj = siy[4 * p] - iyq[0] - 3;
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < 7; ++e) {
        double r = 0.0;
#pragma unroll
        for (int d = 0; d < 7; ++d) r += cx[d] * lgf(G, nx, bi + d, bj + e);
        acc += cy[e] * r;
    }
    return acc;
}

__global__ void k_schur_build(const int* __restrict__ six, const int* __restrict__ siy, const double* __restrict__ swx,
                              const double* __restrict__ swy, const double* __restrict__ ds, int ns,
                              const double* __restrict__ G, int nx, double* __restrict__ A, int lda) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (q >= ns || q < p) return;
    int ixq[4], iyq[4];
    double wxq[4], wyq[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ixq[a] = six[4 * q + a];
        iyq[a] = siy[4 * q + a];
        wxq[a] = swx[4 * q + a];
        wyq[a] = swy[4 * q + a];
    }
    const double k = stencil_pair_lgf(six, siy, swx, swy, p, ixq, iyq, wxq, wyq, G, nx);
    A[(size_t)p * lda + q] = -ds[q] * k;
    if (q != p) A[(size_t)q * lda + p] = -ds[p] * k;
}

// augmented [S | I] for Gauss-Jordan
__global__ void k_augment(const double* __restrict__ S, double* __restrict__ A, int ns) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= 2 * ns) return;
    A[(size_t)i * 2 * ns + j] = j < ns ? S[(size_t)i * ns + j] : (j - ns == i ? 1.0 : 0.0);
}

// pivot k: choose the row of largest |A[i,k]|, i >= k (lowest index on ties), swap
// it into row k and scale row k by the inverse pivot (one block)
__global__ void k_gj_pivot(double* __restrict__ A, int ns, int k, double tiny, int* __restrict__ status) {
    __shared__ double bv[256];
    __shared__ int bi[256];
    __shared__ double piv_s;
    __shared__ int p_s;
    const int W = 2 * ns, tid = threadIdx.x;
    double best = -1.0;
    int bidx = k;
    for (int i = k + tid; i < ns; i += blockDim.x) {
        const double v = fabs(A[(size_t)i * W + k]);
        if (v > best) { best = v; bidx = i; }
    }
    bv[tid] = best;
    bi[tid] = bidx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) {
            const double v2 = bv[tid + o];
            const int i2 = bi[tid + o];
            if (v2 > bv[tid] || (v2 == bv[tid] && i2 < bi[tid])) { bv[tid] = v2; bi[tid] = i2; }
        }
        __syncthreads();
    }
    if (tid == 0) {
        p_s = bi[0];
        piv_s = A[(size_t)bi[0] * W + k];
        if (!(fabs(piv_s) > tiny)) {
            atomicOr(status, ST_SINGULAR);
            piv_s = piv_s == 0.0 ? 1.0 : piv_s;
        }
    }
    __syncthreads();
    const int p = p_s;
    const double inv = 1.0 / piv_s;
    for (int j = tid; j < W; j += blockDim.x) {
        const double ak = A[(size_t)k * W + j], ap = A[(size_t)p * W + j];
        if (p != k) A[(size_t)p * W + j] = ak;
        A[(size_t)k * W + j] = ap * inv;
    }
}

// eliminate column k from every row i != k (one block per row)
__global__ void k_gj_eliminate(double* __restrict__ A, int ns, int k) {
    const int i = blockIdx.x;
    if (i == k) return;
    const int W = 2 * ns;
    const double f = A[(size_t)i * W + k];
    __syncthreads();     // every thread has read the factor before column k is overwritten
    if (f == 0.0) return;
    for (int j = threadIdx.x; j < W; j += blockDim.x) A[(size_t)i * W + j] -= f * A[(size_t)k * W + j];
}

__global__ void k_extract_inverse(const double* __restrict__ A, double* __restrict__ Sinv, int ns) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= ns) return;
    Sinv[(size_t)i * ns + j] = A[(size_t)i * 2 * ns + ns + j];
}

// ------------------------------------------------ blocked Gauss-Jordan inverse
//
// S^-1 by Gauss-Jordan elimination with row interchanges, 32 columns (a panel
// K) at a time, out of place between two ns x ns buffers.  Per panel:
//   P  one block picks the panel's pivot rows by partial pivoting on an FP32
//      copy of the panel (magnitudes only decide the order) and factors the
//      row-permuted pivot block X_KK = L U in FP64 (no further pivoting: the
//      pivots are the elimination's own);
//   V  per column j: y = L^-1 x_j, z = U^-1 y, with x_j = X_Kj outside the
//      panel and the unit vector e_j inside it; per row r outside the
//      panel: the multipliers l_r = X_rK U^-1;
//   U  the sweep of the permuted X:
//        X'_rj = X_rj - l_r . y_j (r, j outside K),  X'_rj = -l_r . y_j (j in K),
//        X'_Kj = z_j.
// The trailing update goes through the LU factors (as a blocked LU does), not
// through (X_KK)^-1, whose rounding would be amplified by cond(X_KK).  After
// the last panel, undoing the accumulated row permutation on the columns
// gives S^-1.  Three launches per 32 columns instead of two per column; the
// FP64 work stays ~ns^3 multiply-adds, spread over full warps on every SM.
constexpr int BGJ_B = 32;              // panel width
constexpr int BGJ_MAX = 1024;          // ns handled by one panel block (panel rows in shared memory)
constexpr int BGJ_PANEL_THREADS = 1024;

__global__ void __launch_bounds__(BGJ_PANEL_THREADS) k_bgj_panel(const double* __restrict__ X, int n, int k0, int kb,
                                                                  int* __restrict__ perm, int* __restrict__ gperm,
                                                                  double* __restrict__ LU, double tiny,
                                                                  int* __restrict__ status) {
    static_assert(BGJ_PANEL_THREADS == 32 * 32 && BGJ_MAX <= 32 * 32,
                  "32 warps; a lane's rows lane + 32 k (k < 32) fit one bit mask");
    extern __shared__ float sp[];                  // (n - k0) x 33 FP32 copy of the panel
    __shared__ int used[BGJ_MAX];
    __shared__ int rowid[BGJ_MAX];                 // local row i of the permuted panel = local row rowid[i]
    __shared__ int gp[BGJ_MAX];
    __shared__ int wsum[32];
    __shared__ double A[BGJ_B][BGJ_B + 1];
    __shared__ double rpiv[BGJ_B];
    const int m = n - k0, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    pdl_wait();
    for (int idx = tid; idx < m * kb; idx += blockDim.x) {
        const int i = idx / kb, j = idx - (idx / kb) * kb;
        sp[i * 33 + j] = (float)X[(size_t)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    // Pivot rows by partial pivoting on the FP32 copy.  Rows are not moved:
    // warp 0 keeps, lane by lane, a bit mask of the rows lane + 32 k already
    // taken as pivots, finds each pivot and publishes it with the masks; the
    // block then eliminates the pivot's column from the rows not taken.  (The
    // kernel runs on one SM and is bound by instruction issue, so the search
    // is done once, not by every warp.)
    __shared__ unsigned tk[32];
    __shared__ int piv_s;
    unsigned taken = 0u;
    if (tid < 32) tk[tid] = 0u;
    for (int c = 0; c < kb; ++c) {
        if (wid == 0) {
            // the largest |panel[i][c]| over rows i not yet taken, lowest i on
            // ties; all NaN: the lowest row not taken
            float best = -1.f;
            int bi = m, first = m;
            for (int k = 0, i = lane; i < m; ++k, i += 32) {
                if ((taken >> k) & 1u) continue;
                first = min(first, i);
                const float v = fabsf(sp[i * 33 + c]);
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(0xffffffffu, best, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
                if (v2 > best || (v2 == best && i2 < bi)) {
                    best = v2;
                    bi = i2;
                }
            }
            const int pr = bi < m ? bi : (first < m ? first : 0);   // a row not taken exists: c < kb <= m
            if (lane == (pr & 31)) {
                taken |= 1u << (pr >> 5);
                tk[lane] = taken;
            }
            if (lane == 0) {
                piv_s = pr;
                rowid[c] = pr;
            }
        }
        __syncthreads();
        // lane = column, warp w takes the rows w + 32 k not taken
        const int pr = piv_s;
        const unsigned rows_taken = tk[wid];
        const float pv = sp[pr * 33 + c];
        if (pv != 0.f && lane > c && lane < kb) {
            const float q = sp[pr * 33 + lane] / pv;
            for (int k = 0, i = wid; i < m; ++k, i += 32)
                if (!((rows_taken >> k) & 1u)) sp[i * 33 + lane] -= sp[i * 33 + c] * q;
        }
        __syncthreads();
    }
    // the rows not taken follow the pivots, in ascending order
    for (int i = tid; i < m; i += blockDim.x) used[i] = (int)((tk[i & 31] >> (i >> 5)) & 1u);
    __syncthreads();
    const int free_i = tid < m && !used[tid] ? 1 : 0;
    int incl = free_i;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int before = incl - free_i;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    if (free_i) rowid[kb + before] = tid;
    __syncthreads();
    // this panel's permutation (rows < k0 stay) and the accumulated one
    for (int i = tid; i < m; i += blockDim.x) {
        perm[k0 + i] = k0 + rowid[i];
        gp[i] = gperm[k0 + rowid[i]];
    }
    __syncthreads();
    for (int i = tid; i < m; i += blockDim.x) gperm[k0 + i] = gp[i];
    // FP64 LU of the permuted pivot block, thread (i, j) = (warp, lane) owning
    // entry (i, j), one block barrier per column: at step c, rows i > c take
    // l_i = A[i][c] / U_cc (kept apart in Lf, so A[i][c] is never written while
    // it is read) and update A[i][j], j > c, from row c, which no thread writes
    // in this step.  The thread of entry (c + 1, c + 1) forms the next pivot's
    // reciprocal as soon as its last update is done (FP64 division is a long
    // sequence at this GPU's FP64 rate: one thread per pivot).
    __shared__ double Lf[BGJ_B][BGJ_B + 1];
    const int i = tid >> 5, j = lane;
    const bool mine = i < kb && j < kb;
    if (mine) A[i][j] = X[(size_t)(k0 + rowid[i]) * n + k0 + j];
    __syncthreads();
    auto pivot = [&](int c) {
        const double pv = A[c][c];
        if (!(fabs(pv) > tiny)) atomicOr(status, ST_SINGULAR);
        rpiv[c] = 1.0 / (pv == 0.0 ? 1.0 : pv);
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
        if (mine && i > c && j >= c) {
            const double l = A[i][c] * rpiv[c];
            if (j == c) Lf[i][c] = l;
            else A[i][j] -= l * A[c][j];
            if (i == c + 1 && j == c + 1) pivot(c + 1);
        }
        __syncthreads();
    }
    if (mine) LU[i * BGJ_B + j] = j < i ? Lf[i][j] : A[i][j];
    if (tid < kb) LU[BGJ_B * BGJ_B + tid] = rpiv[tid];
}

// One warp per column j < n (y_j, z_j) and per row r < n outside the panel
// (l_r); lanes over the panel's kb entries.  Blocks of 8 warps.
__global__ void __launch_bounds__(256) k_bgj_subst(const double* __restrict__ X, int n, int k0, int kb,
                                                    const int* __restrict__ perm, const double* __restrict__ LU,
                                                    double* __restrict__ Y, double* __restrict__ Z,
                                                    double* __restrict__ Lr) {
    __shared__ double F[BGJ_B][BGJ_B + 1];
    __shared__ double rd[BGJ_B];                   // 1 / U_ll
    const int lane = threadIdx.x & 31;
    const int wg = blockIdx.x * 8 + (threadIdx.x >> 5);
    pdl_wait();
    for (int t = threadIdx.x; t < BGJ_B * BGJ_B; t += blockDim.x) {
        const int a = t >> 5, b = t & 31;
        F[a][b] = (a < kb && b < kb) ? LU[a * BGJ_B + b] : (a == b ? 1.0 : 0.0);
    }
    if (threadIdx.x < BGJ_B) rd[threadIdx.x] = (int)threadIdx.x < kb ? LU[BGJ_B * BGJ_B + threadIdx.x] : 1.0;
    __syncthreads();
    const bool act = lane < kb;
    if (wg < n) {
        const int j = wg;
        double v;
        if (j >= k0 && j < k0 + kb) v = lane == j - k0 ? 1.0 : 0.0;
        else v = act ? X[(size_t)perm[k0 + lane] * n + j] : 0.0;
        for (int l = 0; l < kb; ++l) {            // y = L^-1 x (unit lower)
            const double yl = __shfl_sync(0xffffffffu, v, l);
            if (lane > l) v -= F[lane][l] * yl;
        }
        if (act) Y[(size_t)lane * n + j] = v;
        for (int l = kb - 1; l >= 0; --l) {       // z = U^-1 y
            if (lane == l) v *= rd[l];
            const double zl = __shfl_sync(0xffffffffu, v, l);
            if (lane < l) v -= F[lane][l] * zl;
        }
        if (act) Z[(size_t)lane * n + j] = v;
    } else if (wg < 2 * n) {
        const int r = wg - n;
        if (r >= k0 && r < k0 + kb) return;
        const int src = r < k0 ? r : perm[r];
        double v = act ? X[(size_t)src * n + k0 + lane] : 0.0;
        for (int l = 0; l < kb; ++l) {            // l_r U = x_r
            if (lane == l) v *= rd[l];
            const double al = __shfl_sync(0xffffffffu, v, l);
            if (lane > l) v -= al * F[l][lane];
        }
        if (act) Lr[(size_t)r * BGJ_B + lane] = v;
    }
}

// The sweep into Y: tile of 8 rows x 32 columns, one entry per thread
__global__ void __launch_bounds__(256) k_bgj_sweep(const double* __restrict__ X, int n, int k0, int kb,
                                                    const int* __restrict__ perm, const double* __restrict__ Yk,
                                                    const double* __restrict__ Zk, const double* __restrict__ Lr,
                                                    double* __restrict__ Out) {
    __shared__ double Ls[8][BGJ_B];
    __shared__ double Ys[BGJ_B][32];
    const int j = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
    pdl_wait();
    const bool rk = r >= k0 && r < k0 + kb;
    Ls[threadIdx.y][threadIdx.x] = (r < n && !rk && (int)threadIdx.x < kb) ? Lr[(size_t)r * BGJ_B + threadIdx.x] : 0.0;
    for (int l = threadIdx.y; l < BGJ_B; l += 8)
        Ys[l][threadIdx.x] = (l < kb && j < n) ? Yk[(size_t)l * n + j] : 0.0;
    __syncthreads();
    if (r >= n || j >= n) return;
    double out;
    if (rk) {
        out = Zk[(size_t)(r - k0) * n + j];
    } else {
        double acc = 0.0;
        for (int l = 0; l < kb; ++l) acc += Ls[threadIdx.y][l] * Ys[l][threadIdx.x];
        const bool jk = j >= k0 && j < k0 + kb;
        const int src = r < k0 ? r : perm[r];
        out = (jk ? 0.0 : X[(size_t)src * n + j]) - acc;
    }
    Out[(size_t)r * n + j] = out;
}

// S^-1[i][gperm[r]] = X[i][r]
__global__ void k_bgj_unpermute(const double* __restrict__ X, int n, const int* __restrict__ gperm,
                                double* __restrict__ Sinv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    pdl_wait();
    if (r >= n) return;
    Sinv[(size_t)i * n + gperm[r]] = X[(size_t)i * n + r];
}

__global__ void k_iota(int* __restrict__ v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

// deterministic block reduction of a double (fixed tree)
__device__ double block_sum(double v, double* sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) sh[tid] += sh[tid + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// f0 = S^-1 1 (row sums of S^-1): one warp per row, lanes over strided
// columns, then a fixed shuffle tree (deterministic)
__global__ void k_f0_rows(const double* __restrict__ Sinv, int ns, double* __restrict__ f0) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= ns) return;
    double s = 0.0;
    for (int q = lane; q < ns; q += 32) s += Sinv[(size_t)row * ns + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) f0[row] = s;
}

// f0hat = dS f0 and Gamma0 = sum f0hat (one block of 256, fixed order)
__global__ void k_f0_final(const double* __restrict__ f0, const double* __restrict__ ds, int ns,
                           double* __restrict__ f0hat, double* __restrict__ gamma0) {
    __shared__ double sh[256];
    double part = 0.0;
    for (int p = threadIdx.x; p < ns; p += blockDim.x) {
        const double h = ds[p] * f0[p];
        f0hat[p] = h;
        part += h;
    }
    const double g = block_sum(part, sh);
    if (threadIdx.x == 0) *gamma0 = g;
}

// Rows of a dense ns x ns matrix A against nc vectors x_c (stride ns), one
// warp per row, three vectors per blockIdx.y, a fixed shuffle tree:
//   MODE 0  out_c  = A x_c
//   MODE 1  out_c  = v_c - A x_c     (v_c = 1 when v is null)
//   MODE 2  out_c += A x_c
// One step of iterative refinement of y ~ S^-1 v is MODE 1 with A = S (the
// residual against S itself) and then MODE 2 with A = S^-1: the refined y is
// as accurate as FP64 and cond(S) allow, whatever rounding the inverse carries.
template <int MODE>
__global__ void k_rows(const double* __restrict__ A, int ns, const double* __restrict__ x, int nc,
                       const double* __restrict__ v, double* __restrict__ out) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    const int c0 = 3 * blockIdx.y;
    if (row >= ns) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int q = lane; q < ns; q += 32) {
        const double a = A[(size_t)row * ns + q];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (c0 + c < nc) acc[c] += a * x[(size_t)(c0 + c) * ns + q];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c0 + c >= nc) continue;
            const size_t i = (size_t)(c0 + c) * ns + row;
            if (MODE == 0) out[i] = acc[c];
            else if (MODE == 1) out[i] = (v ? v[i] : 1.0) - acc[c];
            else out[i] += acc[c];
        }
}

inline dim3 rows_grid(int ns, int nc) { return dim3((unsigned)ceil_div(ns, 8), (unsigned)ceil_div(nc, 3)); }

// Order of the sheet deposit: the 16 ns stencil entries e = 16 p + 4 b + a
// sorted by (grid node, e), so that each node's entries are contiguous and in
// index order.  One block; bitonic sort of the 64-bit keys node 2^16 + e
// (e < 2^14, node < 2^22) in shared memory, padded to n2 = 2^k >= 16 ns.
constexpr int SHEET_SORT_MAX = 1024;
constexpr int SHEET_SORT_THREADS = 1024;

__global__ void __launch_bounds__(SHEET_SORT_THREADS) k_sheet_order(const int* __restrict__ six,
                                                                     const int* __restrict__ siy, int ns, int nx,
                                                                     int n2, int* __restrict__ sorder,
                                                                     int* __restrict__ snode) {
    extern __shared__ unsigned long long key[];
    const int ne = 16 * ns;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) {
        if (e < ne) {
            const int p = e >> 4, a = e & 3, b = (e >> 2) & 3;
            const unsigned long long node = (unsigned long long)siy[4 * p + b] * nx + six[4 * p + a];
            key[e] = (node << 16) | (unsigned long long)e;
        } else {
            key[e] = ~0ull;
        }
    }
    __syncthreads();
    // Stages whose partner distance j is below SEG stay inside SEG-key
    // segments; warp w owns segments w, w + 32, ... and runs them with warp
    // barriers only, so block barriers remain for the j >= SEG stages.
    // Pair p of a stage (p < n2 / 2) is the key index with a zero bit
    // inserted at bit log2(j), and its partner has that bit set.
    constexpr int SEG = 64;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    auto cmpx = [&](int p, int j, int k) {
        const int lo = p & (j - 1);
        const int i = ((p - lo) << 1) | lo, l = i | j;
        const unsigned long long x = key[i], y = key[l];
        if ((x > y) == ((i & k) == 0)) {
            key[i] = y;
            key[l] = x;
        }
    };
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= SEG) {
                for (int p = threadIdx.x; p < (n2 >> 1); p += blockDim.x) cmpx(p, j, k);
                __syncthreads();
            } else {
                // this warp's segments: SEG / 2 pairs each, one per lane
                for (int sgm = wid; sgm * SEG < n2; sgm += nw) cmpx(sgm * (SEG / 2) + lane, j, k);
                __syncwarp();
                if (j == 1) __syncthreads();   // the next k begins with a block-wide distance
            }
        }
    for (int i = threadIdx.x; i < ne; i += blockDim.x) {
        sorder[i] = (int)(key[i] & 0xFFFFull);
        snode[i] = (int)(key[i] >> 16);
    }
}

// E_s L^-1 w at surface point p = dx^2 sum_nodes w_m sum_{16 stencil nodes s} d_p(s) G(s - m),
// summed in FP64 over the nonzero nodes of w (any precision of w).  Evaluating
// it directly keeps FFT rounding (white noise on psi, amplified by the
// ill-conditioned S) out of the sheet strength.  One block per surface point;
// per-thread partial sums in a fixed order and a fixed reduction tree.
template <typename T>
__global__ void __launch_bounds__(256) k_surface_einvlw(const T* __restrict__ w, int nx, int ny,
                                                        const int* __restrict__ six, const int* __restrict__ siy,
                                                        const double* __restrict__ swx, const double* __restrict__ swy,
                                                        const double* __restrict__ G, double dx2,
                                                        double* __restrict__ out) {
    __shared__ double sh[256];
    const int p = blockIdx.x;
    int ix[4], iy[4];
    double wx[4], wy[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ix[a] = six[4 * p + a];
        iy[a] = siy[4 * p + a];
        wx[a] = swx[4 * p + a];
        wy[a] = swy[4 * p + a];
    }
    double acc = 0.0;
    const int M = nx * ny;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const double wm = (double)w[m];
        if (wm == 0.0) continue;
        const int i = m % nx, j = m / nx;
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double r = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) r += wx[a] * lgf(G, nx, ix[a] - i, iy[b] - j);
            s += wy[b] * r;
        }
        acc += wm * s;
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) out[p] = dx2 * tot;
}

// Sparse route of the same sum for a field with few nonzero nodes: the
// nonzero nodes are listed once, in node order (deterministic compaction in
// two passes over fixed chunks), and every surface point sums over the list
// only, 16 ns nnz multiply-adds instead of a scan of all nx ny nodes per point.
constexpr int NZ_BLOCKS = 304;

template <typename T>
__global__ void __launch_bounds__(256) k_nz_count(const T* __restrict__ w, int M, int chunk, int* __restrict__ counts) {
    __shared__ int sh[8];
    const int lo = blockIdx.x * chunk, hi = min(M, lo + chunk);
    int c = 0;
    for (int m = lo + threadIdx.x; m < hi; m += blockDim.x) c += w[m] != (T)0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        counts[blockIdx.x] = t;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_nz_write(const T* __restrict__ w, int M, int chunk,
                                                  const int* __restrict__ counts, int* __restrict__ idx,
                                                  double* __restrict__ val, int* __restrict__ total) {
    __shared__ int wsum[8];
    __shared__ int base_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int b = 0;
        for (int i = 0; i < (int)blockIdx.x; ++i) b += counts[i];
        base_s = b;
        if (blockIdx.x == gridDim.x - 1) *total = b + counts[blockIdx.x];
    }
    __syncthreads();
    int base = base_s;
    const int lo = blockIdx.x * chunk, hi = min(M, lo + chunk);
    for (int m0 = lo; m0 < hi; m0 += blockDim.x) {
        const int m = m0 + threadIdx.x;
        const bool nz = m < hi && w[m] != (T)0;
        const unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int before = 0, all = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            before += i < wid ? wsum[i] : 0;
            all += wsum[i];
        }
        if (nz) {
            const int r = base + before + __popc(bal & ((1u << lane) - 1u));
            idx[r] = m;
            val[r] = (double)w[m];
        }
        base += all;
        __syncthreads();
    }
}

// The nonzero entries are split into gridDim.y chunks, so that few surface
// points still fill the GPU (64 points made 64 blocks); each block writes its
// chunk's partial sum, and the last block of a point to finish (a counter per
// point, reset by that block) adds the partials in chunk order: the result
// does not depend on which block finishes last.
__global__ void __launch_bounds__(256) k_surface_einvlw_sparse(const int* __restrict__ idx, const double* __restrict__ val,
                                                               const int* __restrict__ total, int nx,
                                                               const int* __restrict__ six, const int* __restrict__ siy,
                                                               const double* __restrict__ swx,
                                                               const double* __restrict__ swy,
                                                               const double* __restrict__ G, double dx2,
                                                               double* __restrict__ part, unsigned* __restrict__ done,
                                                               double* __restrict__ out) {
    __shared__ double sh[256];
    __shared__ bool last;
    const int p = blockIdx.x, c = blockIdx.y, nc = gridDim.y;
    int ix[4], iy[4];
    double wx[4], wy[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ix[a] = six[4 * p + a];
        iy[a] = siy[4 * p + a];
        wx[a] = swx[4 * p + a];
        wy[a] = swy[4 * p + a];
    }
    const int n = *total;
    const int chunk = (n + nc - 1) / nc;
    const int q0 = c * chunk, q1 = q0 + chunk < n ? q0 + chunk : n;
    double acc = 0.0;
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const int m = idx[q];
        const int i = m % nx, j = m / nx;
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            double r = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) r += wx[a] * lgf(G, nx, ix[a] - i, iy[b] - j);
            s += wy[b] * r;
        }
        acc += val[q] * s;
    }
    const double tot = block_sum(acc, sh);
    if (nc == 1) {
        if (threadIdx.x == 0) out[p] = dx2 * tot;
        return;
    }
    if (threadIdx.x == 0) {
        part[(size_t)p * nc + c] = tot;
        __threadfence();
        last = atomicAdd(&done[p], 1u) == (unsigned)(nc - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (int k = 0; k < nc; ++k) t += __ldcg(&part[(size_t)p * nc + k]);
        out[p] = dx2 * t;
        done[p] = 0u;                                 // ready for the next call (and a graph's next replay)
    }
}

// chunks of the sparse surface sum per surface point: about one block an SM
// (a function of ns alone, so a captured step and pf_step split alike; more
// chunks cost the batched instances, which fill the GPU together, more than
// they gave one instance)
inline int ew_split(int ns) { return std::max(1, std::min(EW_SPLIT_MAX, ceil_div(152, ns))); }

// Vortex route of the same sum: the node entries of R_v Gamma listed straight
// from the FP64 positions, sixteen per vortex (M4' weights in FP64, Eq.
// vortexregularization), duplicates and all (the sum is linear), for the
// sparse kernel.  A vortex whose stencil leaves the grid gives zero entries
// (regularization skips it as well).
__global__ void k_vortex_entries(const double* __restrict__ X, const double* __restrict__ Y,
                                 const double* __restrict__ G, int64_t n, int nx, int ny, double x0, double y0,
                                 double dx, int* __restrict__ idx, double* __restrict__ val, int* __restrict__ total) {
    const double inv_dx2 = 1.0 / (dx * dx);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        int ix[4], iy[4];
        double wx[4], wy[4];
        const bool in = stencil(X[q], x0, dx, nx, ix, wx, false) && stencil(Y[q], y0, dx, ny, iy, wy, false);
        const double g = in ? G[q] * inv_dx2 : 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                idx[16 * q + 4 * b + a] = in ? iy[b] * nx + ix[a] : 0;
                val[16 * q + 4 * b + a] = in ? g * wy[b] * wx[a] : 0.0;
            }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *total = (int)(16 * n);
}

// The same quantity from an FP64 psi = -L^-1 w on the grid: E_s L^-1 w = -E_s psi.
// lowest and highest row among n stencil rows (one block)
__global__ void k_stencil_rows(const int* __restrict__ siy, int n, int* __restrict__ rows) {
    __shared__ int lo[8], hi[8];
    int a = 1 << 30, b = -1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a = min(a, siy[i]);
        b = max(b, siy[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
        lo[threadIdx.x >> 5] = a;
        hi[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a = min(a, lo[w]);
            b = max(b, hi[w]);
        }
        rows[0] = a;
        rows[1] = b;
    }
}

__global__ void k_surface_from_psi(const double* __restrict__ psi, int nx, int ns, const int* __restrict__ six,
                                   const int* __restrict__ siy, const double* __restrict__ swx,
                                   const double* __restrict__ swy, double* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ns) return;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        double r = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) r += swx[4 * p + a] * psi[(size_t)siy[4 * p + b] * nx + six[4 * p + a]];
        s += swy[4 * p + b] * r;
    }
    out[p] = -s;
}

// s'_b = (U - Uinf) y - (V - Vinf) x - Omega/2 (x^2 + y^2)   (Eq. sfsurf with the uniform flow removed)
__global__ void k_sbprime(const double* __restrict__ x, const double* __restrict__ y, int ns, pf_motion m,
                          double* __restrict__ sb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ns) return;
    sb[p] = (m.U - m.Uinf) * y[p] - (m.V - m.Vinf) * x[p] - 0.5 * m.Omega * (x[p] * x[p] + y[p] * y[p]);
}

// s'_b of several bodies: each point with its own body's motion, the free
// stream of motion[0]
__global__ void k_sbprime_multi(const double* __restrict__ x, const double* __restrict__ y, int ns, pf_multibody mb,
                                double* __restrict__ sb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ns) return;
    int b = 0;
    while (b + 1 < mb.n_bodies && p >= mb.start[b + 1]) ++b;
    const pf_motion m = mb.motion[b];
    sb[p] = (m.U - mb.motion[0].Uinf) * y[p] - (m.V - mb.motion[0].Vinf) * x[p] -
            0.5 * m.Omega * (x[p] * x[p] + y[p] * y[p]);
}

// the body indicators 1_b as columns out[b*ns + p]
__global__ void k_indicators(int ns, pf_multibody mb, double* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (p >= ns || b >= mb.n_bodies) return;
    out[(size_t)b * ns + p] = (p >= mb.start[b] && p < mb.start[b + 1]) ? 1.0 : 0.0;
}

// E_s L^-1 d_j for unit point vortices at (vx[j], vy[j]), j < nj: out[j*ns + p]
__global__ void k_unit_vortex(const double* __restrict__ vx, const double* __restrict__ vy, int nj,
                              const int* __restrict__ six, const int* __restrict__ siy, const double* __restrict__ swx,
                              const double* __restrict__ swy, int ns, const double* __restrict__ G, int nx, int ny,
                              double x0, double y0, double dx, double* __restrict__ out, int* __restrict__ status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (p >= ns || j >= nj) return;
    int vix[4], viy[4];
    double vwx[4], vwy[4];
    if (!(stencil(vx[j], x0, dx, nx, vix, vwx, false) && stencil(vy[j], y0, dx, ny, viy, vwy, false))) {
        if (p == 0) atomicOr(status, ST_OUT_OF_DOMAIN);
        out[(size_t)j * ns + p] = 0.0;
        return;
    }
    // L^-1 d_j = dx^2 G * (dx^-2 M4' M4'): the dx factors cancel; separable sum as k_schur_build
    const double acc = stencil_pair_lgf(six, siy, swx, swy, p, vix, viy, vwx, vwy, G, nx);
    out[(size_t)j * ns + p] = acc;
}

// y_c = S^-1 v_c for nc right-hand sides (vectors of length ns, stride ns)
__global__ void k_gemv(const double* __restrict__ Sinv, int ns, const double* __restrict__ v, int nc,
                       double* __restrict__ y) {
    const int p = blockIdx.x;
    __shared__ double sh[4][128];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < ns; q += blockDim.x) {
        const double s = Sinv[(size_t)p * ns + q];
        for (int c = 0; c < nc; ++c) acc[c] += s * v[(size_t)c * ns + q];
    }
    for (int c = 0; c < nc; ++c) sh[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < nc; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < nc) y[(size_t)threadIdx.x * ns + p] = sh[threadIdx.x][0];
}

}  // namespace

// ---------------------------------------------------------------- constraint algebra
// One block.  Inputs (device): sb = s'_b, ew = E L^-1 w, y = S^-1 applied to
// [rhs0, e_1, e_2] (rhs0 depends on the mode, set by the host sequence).
// Modes (Sec. 2.3-2.4), with ftilde(v) = (S^-1 v)/f0:
//   GIVEN_S0      f = S^-1 (sb - s0 1 + ew)                      (y0 computed with that rhs)
//   CIRCULATION   fs = S^-1 (sb + ew), s0 = (<1, fs> - Gamma_b)/Gamma0, f = fs - s0 f0
//   KUTTA_STEADY  ft* = ftilde(P^Gamma sb + ew), s0 = ft*_k, f = f0 o (ft* - s0)
//   KUTTA_SHED    ft* as above, ft_j = ftilde(e_j); one edge:
//                 G1 = (-Gw - f0hat^T P_k ft*) / (1 + f0hat^T P_k ft_1), g = ft* + G1 ft_1, s0 = g_k;
//                 two edges: 2x2 system of Eq. twovortex, g = ft* + G1 ft_1 + G2 ft_2,
//                 s0 = (g_k1 + g_k2)/2;  f = f0 o (g - s0)
//                 With edge bounds (Sec. 2.5, Eq. twovortex-gen) an edge whose ft*_k lies
//                 inside [lo, hi] sheds nothing (G = 0, its row dropped) and an active
//                 edge's row gets + Gamma0 target on the right and s0 = g_k - target;
//                 with no active edge Kelvin alone gives s0 = (f0hat^T ft* + Gw)/Gamma0.
__global__ void k_constraints(int mode, int ns, int nedge, int k1, int k2, EdgeBounds eb, double param_h,
                              const double* __restrict__ param_d, const double* __restrict__ ds,
                              const double* __restrict__ f0, const double* __restrict__ f0hat,
                              const double* __restrict__ gamma0p, const double* __restrict__ y,
                              double* __restrict__ f, double* __restrict__ out_scalars) {
    __shared__ double sh[256];
    __shared__ double sc[8];
    const double param = param_d ? *param_d : param_h;
    const double Gamma0 = *gamma0p;
    const double* y0 = y;
    const double* y1 = y + ns;
    const double* y2 = y + 2 * ns;
    if (mode == PF_SHEET_GIVEN_S0) {
        for (int p = threadIdx.x; p < ns; p += blockDim.x) f[p] = y0[p];
        if (threadIdx.x == 0) { out_scalars[0] = param; out_scalars[1] = 0.0; out_scalars[2] = 0.0; }
        return;
    }
    if (mode == PF_SHEET_CIRCULATION) {
        double part = 0.0;
        for (int p = threadIdx.x; p < ns; p += blockDim.x) part += ds[p] * y0[p];
        const double circ = block_sum(part, sh);
        const double s0 = (circ - param) / Gamma0;
        for (int p = threadIdx.x; p < ns; p += blockDim.x) f[p] = y0[p] - s0 * f0[p];
        if (threadIdx.x == 0) { out_scalars[0] = s0; out_scalars[1] = 0.0; out_scalars[2] = 0.0; }
        return;
    }
    // Kutta modes: ftilde = y / f0;  f0hat^T ftilde(y_c) = sum ds y_c (since f0hat = ds f0)
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int p = threadIdx.x; p < ns; p += blockDim.x) {
        a0 += ds[p] * y0[p];
        if (mode == PF_SHEET_KUTTA_SHED) {
            a1 += ds[p] * y1[p];
            if (nedge == 2) a2 += ds[p] * y2[p];
        }
    }
    const double h0 = block_sum(a0, sh);             // f0hat^T ft*
    const double h1 = block_sum(a1, sh);             // f0hat^T ft_1
    const double h2 = block_sum(a2, sh);             // f0hat^T ft_2
    if (threadIdx.x == 0) {
        const double fs1 = y0[k1] / f0[k1];
        double G1 = 0.0, G2 = 0.0, s0;
        if (mode == PF_SHEET_KUTTA_STEADY) {
            s0 = fs1;
        } else if (nedge == 1) {
            const double t1 = y1[k1] / f0[k1];
            const bool act = !eb.on || !(eb.lo[0] <= fs1 && fs1 <= eb.hi[0]);
            const double tg = (eb.on && fs1 < eb.lo[0]) ? eb.lo[0] : (eb.on ? eb.hi[0] : 0.0);
            if (act) {
                G1 = (-param - (h0 - Gamma0 * fs1) - Gamma0 * tg) / (1.0 + (h1 - Gamma0 * t1));
                s0 = fs1 + G1 * t1 - tg;
            } else {
                s0 = (h0 + param) / Gamma0;
            }
        } else {
            const double fs2 = y0[k2] / f0[k2];
            const double t11 = y1[k1] / f0[k1], t12 = y2[k1] / f0[k1];
            const double t21 = y1[k2] / f0[k2], t22 = y2[k2] / f0[k2];
            const bool act1 = !eb.on || !(eb.lo[0] <= fs1 && fs1 <= eb.hi[0]);
            const bool act2 = !eb.on || !(eb.lo[1] <= fs2 && fs2 <= eb.hi[1]);
            const double tg1 = (eb.on && fs1 < eb.lo[0]) ? eb.lo[0] : (eb.on ? eb.hi[0] : 0.0);
            const double tg2 = (eb.on && fs2 < eb.lo[1]) ? eb.lo[1] : (eb.on ? eb.hi[1] : 0.0);
            // A_ij = 1 + f0hat^T P_ki ft_j,  b_i = -(Gw + f0hat^T P_ki ft* + Gamma0 target_i),
            // f0hat^T P_k v = f0hat^T v - Gamma0 v_k
            const double A11 = 1.0 + h1 - Gamma0 * t11, A12 = 1.0 + h2 - Gamma0 * t12;
            const double A21 = 1.0 + h1 - Gamma0 * t21, A22 = 1.0 + h2 - Gamma0 * t22;
            const double b1 = -(param + h0 - Gamma0 * fs1 + Gamma0 * tg1);
            const double b2 = -(param + h0 - Gamma0 * fs2 + Gamma0 * tg2);
            if (act1 && act2) {
                const double det = A11 * A22 - A12 * A21;
                G1 = (b1 * A22 - A12 * b2) / det;
                G2 = (A11 * b2 - A21 * b1) / det;
                const double g1 = fs1 + G1 * t11 + G2 * t12;
                const double g2 = fs2 + G1 * t21 + G2 * t22;
                s0 = 0.5 * ((g1 - tg1) + (g2 - tg2));
            } else if (act1) {
                G1 = b1 / A11;
                s0 = fs1 + G1 * t11 - tg1;
            } else if (act2) {
                G2 = b2 / A22;
                s0 = fs2 + G2 * t22 - tg2;
            } else {
                s0 = (h0 + param) / Gamma0;
            }
        }
        sc[0] = s0;
        sc[1] = G1;
        sc[2] = G2;
        out_scalars[0] = s0;
        out_scalars[1] = G1;
        out_scalars[2] = G2;
    }
    __syncthreads();
    const double s0 = sc[0], G1 = sc[1], G2 = sc[2];
    for (int p = threadIdx.x; p < ns; p += blockDim.x) {
        double g = y0[p] / f0[p];
        if (mode == PF_SHEET_KUTTA_SHED) {
            g += G1 * y1[p] / f0[p];
            if (nedge == 2) g += G2 * y2[p] / f0[p];
        }
        f[p] = f0[p] * (g - s0);
    }
}

namespace {

// rhs0 for the mode: GIVEN_S0: sb - s0 + ew; CIRCULATION: sb + ew;
// Kutta: P^Gamma sb + ew = sb - (f0hat^T sb / Gamma0) + ew   (one block)
__global__ void k_rhs0(int mode, int ns, double param_h, const double* __restrict__ param_d,
                       const double* __restrict__ sb, const double* __restrict__ ew,
                       const double* __restrict__ f0hat, const double* __restrict__ gamma0p, double* __restrict__ rhs) {
    __shared__ double sh[256];
    const double param = param_d ? *param_d : param_h;
    double shift = 0.0;
    if (mode == PF_SHEET_GIVEN_S0) shift = param;
    else if (mode == PF_SHEET_KUTTA_STEADY || mode == PF_SHEET_KUTTA_SHED) {
        double part = 0.0;
        for (int p = threadIdx.x; p < ns; p += blockDim.x) part += f0hat[p] * sb[p];
        shift = block_sum(part, sh) / *gamma0p;
    }
    for (int p = threadIdx.x; p < ns; p += blockDim.x) rhs[p] = sb[p] - shift + ew[p];
}

}  // namespace

// R_s f added into a node field: w_n += dx^-2 sum_p dS_p f_p d_p(n) (Sec. 2.2.1).
// Deterministic: thread (p, s) handles stencil entry s of point p; the first
// (p, s) in index order that maps to a node sums every entry mapping to it, in
// index order, and writes the node alone.
template <typename T>
__global__ void k_sheet_deposit(const int* __restrict__ six, const int* __restrict__ siy, const double* __restrict__ swx,
                                const double* __restrict__ swy, const double* __restrict__ ds,
                                const double* __restrict__ f, int ns, double inv_dx2, int nx, T* __restrict__ w) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 16 * ns) return;
    const int p = e >> 4, a = e & 3, b = (e >> 2) & 3;
    const int ni = six[4 * p + a], nj = siy[4 * p + b];
    for (int e2 = 0; e2 < e; ++e2) {
        const int p2 = e2 >> 4;
        if (six[4 * p2 + (e2 & 3)] == ni && siy[4 * p2 + ((e2 >> 2) & 3)] == nj) return;   // not the owner
    }
    double acc = 0.0;
    for (int e2 = e; e2 < 16 * ns; ++e2) {
        const int p2 = e2 >> 4, a2 = e2 & 3, b2 = (e2 >> 2) & 3;
        if (six[4 * p2 + a2] == ni && siy[4 * p2 + b2] == nj) acc += ds[p2] * f[p2] * swx[4 * p2 + a2] * swy[4 * p2 + b2];
    }
    const size_t n = (size_t)nj * nx + ni;
    w[n] = (T)((double)w[n] + acc * inv_dx2);
}

// The same sum from the sorted entries: the first entry of each node sums the
// node's run in index order (the order of k_sheet_deposit), in O(16 ns).
template <typename T>
__global__ void k_sheet_deposit_sorted(const int* __restrict__ sorder, const int* __restrict__ snode,
                                       const double* __restrict__ swx, const double* __restrict__ swy,
                                       const double* __restrict__ ds, const double* __restrict__ f, int ne,
                                       double inv_dx2, T* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int node = snode[i];
    if (i > 0 && snode[i - 1] == node) return;    // not the node's first entry
    double acc = 0.0;
    for (int j = i; j < ne && snode[j] == node; ++j) {
        const int e2 = sorder[j];
        const int p2 = e2 >> 4, a2 = e2 & 3, b2 = (e2 >> 2) & 3;
        acc += ds[p2] * f[p2] * swx[4 * p2 + a2] * swy[4 * p2 + b2];
    }
    w[node] = (T)((double)w[node] + acc * inv_dx2);
}

pf_status sheet_deposit(pf_plan p, pf_schur s, const double* f, void* w) {
    const int n = 16 * s->ns;
    const double inv_dx2 = 1.0 / (p->dx * p->dx);
    if (s->snode) {
        if (p->prec == PF_FP64)
            k_sheet_deposit_sorted<double><<<ceil_div(n, 256), 256, 0, p->stream>>>(s->sorder, s->snode, s->swx, s->swy,
                                                                                      s->ds, f, n, inv_dx2, (double*)w);
        else
            k_sheet_deposit_sorted<float><<<ceil_div(n, 256), 256, 0, p->stream>>>(s->sorder, s->snode, s->swx, s->swy,
                                                                                     s->ds, f, n, inv_dx2, (float*)w);
        PF_LAUNCH_CHECK(p);
        return PF_OK;
    }
    if (p->prec == PF_FP64)
        k_sheet_deposit<double><<<ceil_div(n, 128), 128, 0, p->stream>>>(s->six, s->siy, s->swx, s->swy, s->ds, f, s->ns,
                                                                          inv_dx2, p->nx, (double*)w);
    else
        k_sheet_deposit<float><<<ceil_div(n, 128), 128, 0, p->stream>>>(s->six, s->siy, s->swx, s->swy, s->ds, f, s->ns,
                                                                         inv_dx2, p->nx, (float*)w);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

// ---------------------------------------------------------------- host side

static void free_schur(pf_schur s) {
    void* ptrs[] = {s->x, s->y, s->ds, s->six, s->siy, s->swx, s->swy, s->S, s->A, s->Sinv, s->f0, s->f0hat,
                    s->dgamma0, s->sorder, s->snode, s->gj, s->work, s->mwork, s->scal, s->pnx, s->pny,
                    s->fidx, s->fwt, s->ci, s->cj, s->cw, s->rows, s->ewpart, s->ewdone};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (s->jump) {
        free_schur(s->jump);
        delete s->jump;
    }
}

// S^-1 of s->S into s->Sinv: blocked Gauss-Jordan with row interchanges for
// ns <= BGJ_MAX, the column-at-a-time form beyond
pf_status invert_schur_matrix(pf_plan p, pf_schur s) {
    const int ns = s->ns;
    cudaStream_t st = p->stream;
    // pivots of magnitude 1e-300 or less are reported as singular
    if (ns <= BGJ_MAX) {
        double* LU = s->gj;                       // 32 x 32 factors, then 1 / U_ll
        double* Yk = LU + BGJ_B * BGJ_B + BGJ_B;
        double* Zk = Yk + (size_t)BGJ_B * ns;
        double* Lr = Zk + (size_t)BGJ_B * ns;
        int* perm = (int*)(Lr + (size_t)BGJ_B * ns);
        int* gperm = perm + ns;
        double* buf[2] = {s->A, s->A + (size_t)ns * ns};
        k_iota<<<ceil_div(ns, 256), 256, 0, st>>>(gperm, ns);
        PF_LAUNCH_CHECK(p);
        const double* X = s->S;
        int cur = 0;
        for (int k0 = 0; k0 < ns; k0 += BGJ_B) {
            const int kb = std::min(BGJ_B, ns - k0);
            const size_t sh = (size_t)(ns - k0) * 33 * sizeof(float);
            PF_CUDA(p, set_smem(k_bgj_panel, sh));
            PF_CUDA(p, pf_launch(k_bgj_panel, 1, BGJ_PANEL_THREADS, sh, st, X, ns, k0, kb, perm, gperm, LU, 1e-300,
                                 p->d_status));
            PF_CUDA(p, pf_launch(k_bgj_subst, ceil_div(2 * ns, 8), 256, 0, st, X, ns, k0, kb, (const int*)perm,
                                 (const double*)LU, Yk, Zk, Lr));
            PF_CUDA(p, pf_launch(k_bgj_sweep, dim3(ceil_div(ns, 32), ceil_div(ns, 8)), dim3(32, 8), 0, st, X, ns, k0,
                                 kb, (const int*)perm, (const double*)Yk, (const double*)Zk, (const double*)Lr,
                                 buf[cur]));
            X = buf[cur];
            cur ^= 1;
        }
        PF_CUDA(p, pf_launch(k_bgj_unpermute, dim3(ceil_div(ns, 256), ns), dim3(256), 0, st, X, ns,
                             (const int*)gperm, s->Sinv));
    } else {
        k_augment<<<dim3(ceil_div(2 * ns, 256), ns), 256, 0, st>>>(s->S, s->A, ns);
        PF_LAUNCH_CHECK(p);
        for (int k = 0; k < ns; ++k) {
            k_gj_pivot<<<1, 256, 0, st>>>(s->A, ns, k, 1e-300, p->d_status);
            k_gj_eliminate<<<ns, 256, 0, st>>>(s->A, ns, k);
        }
        PF_LAUNCH_CHECK(p);
        k_extract_inverse<<<dim3(ceil_div(ns, 256), ns), 256, 0, st>>>(s->A, s->Sinv, ns);
        PF_LAUNCH_CHECK(p);
    }
    return PF_OK;
}

pf_status schur_factor_device(pf_plan p, pf_schur s) {
    const int ns = s->ns;
    cudaStream_t st = p->stream;
    k_surface_stencil<<<ceil_div(8 * ns, 32), 32, 0, st>>>(s->x, s->y, ns, p->x0, p->y0, p->dx, p->nx, p->ny, s->six,
                                                            s->siy, s->swx, s->swy, p->d_status);
    k_stencil_rows<<<1, 256, 0, st>>>(s->siy, 4 * ns, s->rows);
    PF_LAUNCH_CHECK(p);
    if (s->snode) {
        int n2 = 1;
        while (n2 < 16 * ns) n2 <<= 1;
        const size_t sh = (size_t)n2 * sizeof(unsigned long long);
        PF_CUDA(p, set_smem(k_sheet_order, sh));
        k_sheet_order<<<1, SHEET_SORT_THREADS, sh, st>>>(s->six, s->siy, ns, p->nx, n2, s->sorder, s->snode);
        PF_LAUNCH_CHECK(p);
    }
    k_schur_build<<<dim3(ceil_div(ns, 128), ns), 128, 0, st>>>(s->six, s->siy, s->swx, s->swy, s->ds, ns, p->G, p->nx,
                                                                s->S, ns);
    PF_LAUNCH_CHECK(p);
    PF_TRY(invert_schur_matrix(p, s));
    // f0 = S^-1 1 with one refinement step (scratch: the solve workspace)
    k_f0_rows<<<ceil_div(ns, 8), 256, 0, st>>>(s->Sinv, ns, s->f0);
    k_rows<1><<<rows_grid(ns, 1), 256, 0, st>>>(s->S, ns, s->f0, 1, nullptr, s->work);
    k_rows<2><<<rows_grid(ns, 1), 256, 0, st>>>(s->Sinv, ns, s->work, 1, nullptr, s->f0);
    k_f0_final<<<1, 256, 0, st>>>(s->f0, s->ds, ns, s->f0hat, s->dgamma0);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

pf_status schur_create(pf_plan p, int ns, pf_schur* out) {
    pf_schur s = new (std::nothrow) pf_schur_s();
    if (!s) return PF_ERR_OOM;
    s->plan = p;
    s->ns = ns;
    auto fail = [&](pf_status st) { free_schur(s); delete s; return st; };
#define PF_ALLOC(ptr, bytes)                                                                      \
    do {                                                                                          \
        cudaError_t e_ = cudaMalloc(&(ptr), (bytes));                                             \
        if (e_ != cudaSuccess) {                                                                  \
            snprintf(p->err, sizeof(p->err), "cudaMalloc: %s", cudaGetErrorString(e_));           \
            return fail(e_ == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA);               \
        }                                                                                         \
    } while (0)
    const size_t v = (size_t)ns * sizeof(double);
    PF_ALLOC(s->x, v);
    PF_ALLOC(s->y, v);
    PF_ALLOC(s->ds, v);
    PF_ALLOC(s->six, 4 * (size_t)ns * sizeof(int));
    PF_ALLOC(s->siy, 4 * (size_t)ns * sizeof(int));
    PF_ALLOC(s->swx, 4 * v);
    PF_ALLOC(s->swy, 4 * v);
    PF_ALLOC(s->S, (size_t)ns * v);
    PF_ALLOC(s->A, 2 * (size_t)ns * v);
    PF_ALLOC(s->Sinv, (size_t)ns * v);
    PF_ALLOC(s->f0, v);
    PF_ALLOC(s->f0hat, v);
    PF_ALLOC(s->dgamma0, sizeof(double));
    if (ns <= BGJ_MAX)
        PF_ALLOC(s->gj, (BGJ_B * BGJ_B + BGJ_B + 3 * (size_t)BGJ_B * ns) * sizeof(double) + 2 * (size_t)ns * sizeof(int));
    if (ns <= SHEET_SORT_MAX) {
        PF_ALLOC(s->sorder, 16 * (size_t)ns * sizeof(int));
        PF_ALLOC(s->snode, 16 * (size_t)ns * sizeof(int));
    }
    PF_ALLOC(s->work, 12 * v);
    PF_ALLOC(s->scal, 8 * sizeof(double));
    PF_ALLOC(s->rows, 2 * sizeof(int));
    PF_ALLOC(s->ewpart, (size_t)EW_SPLIT_MAX * v);
    PF_ALLOC(s->ewdone, (size_t)ns * sizeof(unsigned));
    if (cudaMemsetAsync(s->ewdone, 0, (size_t)ns * sizeof(unsigned), p->stream) != cudaSuccess) return fail(PF_ERR_CUDA);
#undef PF_ALLOC
    *out = s;
    return PF_OK;
}

void schur_free(pf_schur s) {
    free_schur(s);
    delete s;
}

// Full sheet solve on device.  psi_w: real field; vx, vy: device positions of
// the new vortices (mode KUTTA_SHED).  Results: f (device, ns) and scal[0..2] =
// (s0, Gamma1, Gamma2) on the device.
// E_s L^-1 w into ew (ns doubles).  The direct FP64 sum costs 16 ns nx ny
// multiply-adds at the GPU's low FP64 rate; on larger grids the same quantity
// comes from an FP64 FFT solve psi = -L^-1 w (FP64 rounding, far below what
// the ill-conditioned S amplifies into the sheet) read at the stencils.
// Route of E_s L^-1 w from the field w (no vortex source): the sparse sum when
// the caller bounds the nonzero nodes and the sum is small (below 2^24
// multiply-adds its few blocks finish sooner than an FFT's passes), else the
// FFT solve where the padded torus allows it, else the direct sum.  The sums
// run on the FP64 pipe; the FFT of an FP64 plan too, so an FP64 plan keeps
// the direct sum on small grids; that of a mixed plan runs in double-float on
// the FP32 pipe (about sixty times the FP64 rate on this GPU) and is taken
// whenever it fits.
enum FieldRoute { ROUTE_SPARSE, ROUTE_DIRECT, ROUTE_FFT };

FieldRoute field_route(pf_plan p, int ns, int64_t nnz_bound) {
    const int64_t M = (int64_t)p->nx * p->ny;
    const bool fft_ok = p->P >= 256 && p->Q >= 256;
    const bool mixed = p->prec != PF_FP64;
    const int64_t sparse_max = (int64_t)1 << 24;
    if (p->rhs_route == PF_RHS_SPARSE ||
        (p->rhs_route == PF_RHS_AUTO && nnz_bound >= 0 && 16 * (int64_t)ns * nnz_bound < sparse_max))
        return ROUTE_SPARSE;
    if (fft_ok && (p->rhs_route == PF_RHS_FFT ||
                   (p->rhs_route == PF_RHS_AUTO && (mixed || (int64_t)ns * M > ((int64_t)1 << 22)))))
        return ROUTE_FFT;
    return ROUTE_DIRECT;
}

// the scratch a field route allocates on first use: the sparse route's node
// list, the mixed plan's FP64 field, streamfunction and spectra for the FFT
pf_status field_route_buffers(pf_plan p, FieldRoute r) {
    const int64_t M = (int64_t)p->nx * p->ny;
    if (r == ROUTE_SPARSE && !p->nz_idx) {
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        PF_CUDA(p, cudaMalloc(&p->nz_idx, (size_t)M * sizeof(int) + (NZ_BLOCKS + 1) * sizeof(int)));
        PF_CUDA(p, cudaMalloc(&p->nz_val, (size_t)M * sizeof(double)));
    }
    if (r == ROUTE_FFT && p->prec != PF_FP64) {
        if (!p->rhs64) {
            const size_t spec = (size_t)p->ldK * p->ldT * 2 * sizeof(double);
            PF_CUDA(p, cudaStreamSynchronize(p->stream));
            PF_CUDA(p, cudaMalloc(&p->rhs64, 2 * (size_t)M * sizeof(double) + 2 * spec));
        }
        PF_TRY(df_tables_ready(p));
    }
    return PF_OK;
}

pf_status surface_rhs(pf_plan p, pf_schur s, const void* w, double* ew, int64_t nnz_bound,
                      const VortexSource* vs = nullptr) {
    const int ns = s->ns;
    cudaStream_t st = p->stream;
    const int64_t M = (int64_t)p->nx * p->ny;
    // the vortex route: forced, or for mixed plans while 256 ns nv multiply-adds stay below 2^31
    if (vs && vs->n > 0 && (vs->force || (p->prec != PF_FP64 && 256 * (int64_t)ns * vs->n < ((int64_t)1 << 31)))) {
        const int64_t ne = 16 * vs->n;
        if (ne > ((int64_t)1 << 30)) {
            snprintf(p->err, sizeof(p->err), "%lld vortices exceed the vortex route's entry list",
                     (long long)vs->n);
            return PF_ERR_CAPACITY;
        }
        if (ne > p->vent_cap) {
            PF_CUDA(p, cudaStreamSynchronize(st));
            if (p->vent_idx) cudaFree(p->vent_idx);
            if (p->vent_val) cudaFree(p->vent_val);
            p->vent_idx = nullptr;
            p->vent_val = nullptr;
            p->vent_cap = 0;
            const int64_t cap = std::max<int64_t>(ne, 2 * p->vent_cap);
            PF_CUDA(p, cudaMalloc(&p->vent_idx, (size_t)cap * sizeof(int) + 16));
            PF_CUDA(p, cudaMalloc(&p->vent_val, (size_t)cap * sizeof(double)));
            p->vent_cap = cap;
        }
        int* total = p->vent_idx + p->vent_cap;
        const int nb = (int)std::min<int64_t>(ceil_div(vs->n, 256), 152 * 8);
        k_vortex_entries<<<nb, 256, 0, st>>>(vs->X, vs->Y, vs->G, vs->n, p->nx, p->ny, p->x0, p->y0, p->dx,
                                             p->vent_idx, p->vent_val, total);
        k_surface_einvlw_sparse<<<dim3(ns, ew_split(ns)), 256, 0, st>>>(p->vent_idx, p->vent_val, total, p->nx, s->six,
                                                                        s->siy, s->swx, s->swy, p->G, p->dx * p->dx,
                                                                        s->ewpart, s->ewdone, ew);
        PF_LAUNCH_CHECK(p);
        return PF_OK;
    }
    const FieldRoute route = field_route(p, ns, nnz_bound);
    PF_TRY(field_route_buffers(p, route));
    if (route == ROUTE_SPARSE) {
        int* counts = p->nz_idx + M;
        int* total = counts + NZ_BLOCKS;
        const int chunk = ceil_div(M, NZ_BLOCKS);
        if (p->prec == PF_FP64) {
            k_nz_count<double><<<NZ_BLOCKS, 256, 0, st>>>((const double*)w, (int)M, chunk, counts);
            k_nz_write<double><<<NZ_BLOCKS, 256, 0, st>>>((const double*)w, (int)M, chunk, counts, p->nz_idx, p->nz_val,
                                                          total);
        } else {
            k_nz_count<float><<<NZ_BLOCKS, 256, 0, st>>>((const float*)w, (int)M, chunk, counts);
            k_nz_write<float><<<NZ_BLOCKS, 256, 0, st>>>((const float*)w, (int)M, chunk, counts, p->nz_idx, p->nz_val,
                                                         total);
        }
        k_surface_einvlw_sparse<<<dim3(ns, ew_split(ns)), 256, 0, st>>>(p->nz_idx, p->nz_val, total, p->nx, s->six,
                                                                        s->siy, s->swx, s->swy, p->G, p->dx * p->dx,
                                                                        s->ewpart, s->ewdone, ew);
        PF_LAUNCH_CHECK(p);
        return PF_OK;
    }
    if (route == ROUTE_DIRECT) {
        const double dx2 = p->dx * p->dx;
        if (p->prec == PF_FP64)
            k_surface_einvlw<double><<<ns, 256, 0, st>>>((const double*)w, p->nx, p->ny, s->six, s->siy, s->swx,
                                                          s->swy, p->G, dx2, ew);
        else
            k_surface_einvlw<float><<<ns, 256, 0, st>>>((const float*)w, p->nx, p->ny, s->six, s->siy, s->swx,
                                                         s->swy, p->G, dx2, ew);
        PF_LAUNCH_CHECK(p);
        return PF_OK;
    }
    const size_t spec = (size_t)p->ldK * p->ldT * 2 * sizeof(double);
    const double* w64;
    double* psi;
    void *T1, *T2;
    if (p->prec == PF_FP64) {      // the plan's own buffers are free during a sheet solve
        w64 = (const double*)w;
        psi = (double*)p->uv;
        T1 = p->T1;
        T2 = p->T2a;
    } else {
        double* b = (double*)p->rhs64;
        psi = b + M;
        T1 = b + 2 * M;
        T2 = (char*)T1 + spec;
        w64 = nullptr;
    }
    // FP64 plans: FP64 passes; mixed plans: double-float passes on the FP32 w
    if (w64) PF_TRY(conv_psi_f64(p, w64, psi, T1, T2));
    else PF_TRY(conv_psi_df(p, (const float*)w, psi, T1, T2, p->rhs64, s->rows));
    k_surface_from_psi<<<ceil_div(ns, 128), 128, 0, st>>>(psi, p->nx, ns, s->six, s->siy, s->swx, s->swy, ew);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

// allocate ahead of time what a sheet solve with this nonzero bound would
// allocate on first use (a step captured for replay may not allocate)
pf_status sheet_solve_reserve(pf_plan p, pf_schur s, int64_t nnz_bound) {
    return field_route_buffers(p, field_route(p, s->ns, nnz_bound));
}

// Several bodies (Sec. 2.7, Eq. kuttasystem4), one block of 256.  y holds
// S^-1 of [rhs0 | E L^-1 d_1 .. d_E | 1_1 .. 1_B] (refined).  With ftilde_c =
// y_c / f0, the Kutta rows e_k^T ftilde = 0 and the Kelvin rows
//   f0hat_b^T ftilde + sum_{i of b} Gamma_i = -gamma_w[b],
// where f0hat_b^T ftilde_c = sum_{p in b} dS_p y_c[p], form the (E + B) system
// in (Gamma, s0), solved by thread 0 with partial pivoting; then
// f = f0 o ftilde = y_0 + sum_i Gamma_i y_i - sum_b s0_b y_(E+b).
// gamma_w comes from gw_dev (device, B values) when it is not null.
// out: s0 (B) then Gamma (E).
constexpr int MB_COLS = 1 + 3 * PF_MAX_BODIES;    // right-hand sides: rhs0, one per edge, one per body
constexpr int MB_N = 3 * PF_MAX_BODIES;           // unknowns: edges + bodies
constexpr int MB_EDGES = 2 * PF_MAX_BODIES;

__global__ void __launch_bounds__(256) k_constraints_multi(int ns, pf_multibody mb, int ne, const double* __restrict__ y,
                                                           const double* __restrict__ f0, const double* __restrict__ ds,
                                                           const double* __restrict__ gw_dev, double* __restrict__ f,
                                                           double* __restrict__ out, int* __restrict__ status) {
    __shared__ double circ[MB_COLS * PF_MAX_BODIES];
    __shared__ double sol[MB_N];
    const int nb = mb.n_bodies, nc = 1 + ne + nb;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int t = wid; t < nc * nb; t += blockDim.x >> 5) {
        const int c = t / nb, b = t - (t / nb) * nb;
        double a = 0.0;
        for (int p = mb.start[b] + lane; p < mb.start[b + 1]; p += 32) a += ds[p] * y[(size_t)c * ns + p];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) circ[t] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int n = ne + nb;
        double M[MB_N][MB_N + 1];
        int kk[2 * PF_MAX_BODIES], own[2 * PF_MAX_BODIES];
        int e = 0;
        for (int b = 0; b < nb; ++b)
            for (int j = 0; j < mb.n_edges[b]; ++j) {
                kk[e] = mb.edge[b][j];
                own[e++] = b;
            }
        for (int r = 0; r < ne; ++r) {                 // Kutta rows
            const int k = kk[r];
            const double inv = 1.0 / f0[k];
            for (int i = 0; i < ne; ++i) M[r][i] = y[(size_t)(1 + i) * ns + k] * inv;
            for (int b = 0; b < nb; ++b) M[r][ne + b] = -y[(size_t)(1 + ne + b) * ns + k] * inv;
            M[r][n] = -y[k] * inv;
        }
        for (int c = 0; c < nb; ++c) {                 // Kelvin rows
            for (int i = 0; i < ne; ++i) M[ne + c][i] = circ[(1 + i) * nb + c] + (own[i] == c ? 1.0 : 0.0);
            for (int b = 0; b < nb; ++b) M[ne + c][ne + b] = -circ[(1 + ne + b) * nb + c];
            M[ne + c][n] = -(gw_dev ? gw_dev[c] : mb.gamma_w[c]) - circ[c];
        }
        for (int col = 0; col < n; ++col) {            // Gaussian elimination, partial pivoting
            int pr = col;
            for (int r = col + 1; r < n; ++r)
                if (fabs(M[r][col]) > fabs(M[pr][col])) pr = r;
            if (pr != col)
                for (int j = 0; j <= n; ++j) {
                    const double t = M[col][j];
                    M[col][j] = M[pr][j];
                    M[pr][j] = t;
                }
            if (!(fabs(M[col][col]) > 1e-300)) {
                atomicOr(status, ST_SINGULAR);
                M[col][col] = 1.0;
            }
            for (int r = col + 1; r < n; ++r) {
                const double l = M[r][col] / M[col][col];
                for (int j = col; j <= n; ++j) M[r][j] -= l * M[col][j];
            }
        }
        for (int r = n - 1; r >= 0; --r) {
            double a = M[r][n];
            for (int j = r + 1; j < n; ++j) a -= M[r][j] * sol[j];
            sol[r] = a / M[r][r];
        }
        for (int b = 0; b < nb; ++b) out[b] = sol[ne + b];
        for (int i = 0; i < ne; ++i) out[nb + i] = sol[i];
    }
    __syncthreads();
    for (int p = threadIdx.x; p < ns; p += blockDim.x) {
        double v = y[p];
        for (int i = 0; i < ne; ++i) v += sol[i] * y[(size_t)(1 + i) * ns + p];
        for (int b = 0; b < nb; ++b) v -= sol[ne + b] * y[(size_t)(1 + ne + b) * ns + p];
        f[p] = v;
    }
}

pf_status sheet_solve_device(pf_plan p, pf_schur s, const void* w, const pf_motion& m, int mode, double param,
                             const double* param_dev, int n_edges, const int* edges, const double* vx,
                             const double* vy, double* f, const EdgeBounds& eb, int64_t nnz_bound,
                             const VortexSource* vs) {
    const int ns = s->ns;
    cudaStream_t st = p->stream;
    double* sb = s->work;
    double* ew = sb + ns;
    double* rhs = ew + ns;          // rhs0 | e_1 | e_2 contiguous
    double* y = rhs + 3 * ns;       // S^-1 [rhs0 | e_1 | e_2]
    double* res = y + 3 * ns;       // refinement residuals
    k_sbprime<<<ceil_div(ns, 128), 128, 0, st>>>(s->x, s->y, ns, m, sb);
    PF_LAUNCH_CHECK(p);
    PF_TRY(surface_rhs(p, s, w, ew, nnz_bound, vs));
    k_rhs0<<<1, 256, 0, st>>>(mode, ns, param, param_dev, sb, ew, s->f0hat, s->dgamma0, rhs);
    PF_LAUNCH_CHECK(p);
    int nc = 1;
    if (mode == PF_SHEET_KUTTA_SHED) {
        nc = 1 + n_edges;
        k_unit_vortex<<<dim3(ceil_div(ns, 128), n_edges), 128, 0, st>>>(vx, vy, n_edges, s->six, s->siy, s->swx,
                                                                           s->swy, ns, p->G, p->nx, p->ny, p->x0, p->y0,
                                                                           p->dx, rhs + ns, p->d_status);
        PF_LAUNCH_CHECK(p);
    }
    k_gemv<<<ns, 128, 0, st>>>(s->Sinv, ns, rhs, nc, y);
    k_rows<1><<<rows_grid(ns, nc), 256, 0, st>>>(s->S, ns, y, nc, rhs, res);
    k_rows<2><<<rows_grid(ns, nc), 256, 0, st>>>(s->Sinv, ns, res, nc, nullptr, y);
    PF_LAUNCH_CHECK(p);
    k_constraints<<<1, 256, 0, st>>>(mode, ns, n_edges, n_edges > 0 ? edges[0] : 0, n_edges > 1 ? edges[1] : 0, eb,
                                     param, param_dev, s->ds, s->f0, s->f0hat, s->dgamma0, y, f, s->scal);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

// ------------------------------------------------ surface pressure (Sec. 2.6.1)
//
// Staggered grid: u = d psi/dy on the x-faces (x_i, y_j + dx/2) as
// (psi[j+1][i] - psi[j][i]) / dx, v = -d psi/dx on the y-faces (x_i + dx/2, y_j)
// as -(psi[j][i+1] - psi[j][i]) / dx (the discrete curl C).  E_f interpolates
// each component from its own face lattice with the smoothed three-point
// function; C_s = n . E_f C is then a 64-node stencil per surface point, and
// the jump operator C_s L^-1 C_s^T = A G A^T D_dS (L^-1 = dx^2 G *, C_s^T =
// C^T R_f (n o .) with R_f carrying dS / dx^2).

// face stencils: thread per (point, lattice l, node a); lattice l = 0: u's x
// (nodes), 1: u's y (half-shifted, ny - 1 rows), 2: v's x (half-shifted,
// nx - 1 columns), 3: v's y (nodes)
__global__ void k_face_stencil(const double* __restrict__ x, const double* __restrict__ y, int ns, double x0,
                               double y0, double dx, int nx, int ny, int* __restrict__ fidx, double* __restrict__ fwt,
                               int* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 16 * ns) return;
    const int p = t >> 4, l = (t >> 2) & 3, a = t & 3;
    const double pos = (l == 0 || l == 2) ? x[p] : y[p];
    const double org = l == 0 ? x0 : (l == 1 ? y0 + 0.5 * dx : (l == 2 ? x0 + 0.5 * dx : y0));
    const int n = l == 0 ? nx : (l == 1 ? ny - 1 : (l == 2 ? nx - 1 : ny));
    const double g = (pos - org) / dx;
    const double c = floor(g);
    const bool ok = c >= 1.0 && c <= n - 3.0;
    if (!ok && a == 0) atomicOr(status, ST_OUT_OF_DOMAIN);
    const int ci = ok ? (int)c : 0;
    fidx[t] = ok ? ci - 1 + a : 1;
    fwt[t] = ok ? yang3((double)(ci - 1 + a) - g) : 0.0;
}

// C_s node stencils: thread per (point, entry k < 64), entries in the order
// (b, a) of the two face stencils, four per pair: u's upper and lower node,
// v's right and left node
__global__ void k_curl_stencil(const int* __restrict__ fidx, const double* __restrict__ fwt,
                               const double* __restrict__ nxs, const double* __restrict__ nys, int ns, double dx,
                               int* __restrict__ ci, int* __restrict__ cj, double* __restrict__ cw) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 64 * ns) return;
    const int p = t >> 6, k = t & 63, pair = k >> 2, r = k & 3, b = pair >> 2, a = pair & 3;
    const int* fi = fidx + 16 * p;
    const double* fw = fwt + 16 * p;
    int i, j;
    double w;
    if (r < 2) {                      // u = (psi[j+1] - psi[j]) / dx on lattice (0, 1)
        const double wu = nxs[p] * fw[a] * fw[4 + b] / dx;
        i = fi[a];
        j = fi[4 + b] + (r == 0 ? 1 : 0);
        w = r == 0 ? wu : -wu;
    } else {                          // v = -(psi[i+1] - psi[i]) / dx on lattice (2, 3)
        const double wv = nys[p] * fw[8 + a] * fw[12 + b] / dx;
        i = fi[8 + a] + (r == 2 ? 1 : 0);
        j = fi[12 + b];
        w = r == 2 ? -wv : wv;
    }
    ci[t] = i;
    cj[t] = j;
    cw[t] = w;
}

// the augmented jump matrix, leading dimension ns + 1:
//   A[p][q] = dS_q sum_k sum_l cw[p][k] G(node_pk - node_ql) cw[q][l],
//   A[p][ns] = 1 (multiplier of the uniform null space), A[ns][q] = dS_q, A[ns][ns] = 0
__global__ void __launch_bounds__(256) k_jump_build(const int* __restrict__ ci, const int* __restrict__ cj,
                                                    const double* __restrict__ cw, const double* __restrict__ ds, int ns,
                                                    const double* __restrict__ G, int nx, double* __restrict__ A) {
    __shared__ int pi[64], pj[64];
    __shared__ double pw[64];
    __shared__ double sh[256];
    const int p = blockIdx.y, q = blockIdx.x, n1 = ns + 1;
    if (p == ns || q == ns) {
        if (threadIdx.x == 0) A[(size_t)p * n1 + q] = p == ns ? (q == ns ? 0.0 : ds[q]) : 1.0;
        return;
    }
    if (threadIdx.x < 64) {
        pi[threadIdx.x] = ci[64 * p + threadIdx.x];
        pj[threadIdx.x] = cj[64 * p + threadIdx.x];
        pw[threadIdx.x] = cw[64 * p + threadIdx.x];
    }
    __syncthreads();
    double acc = 0.0;
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int k = e >> 6, l = e & 63;
        acc += pw[k] * lgf(G, nx, pi[k] - ci[64 * q + l], pj[k] - cj[64 * q + l]) * cw[64 * q + l];
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) A[(size_t)p * n1 + q] = ds[q] * tot;
}

// right-hand side of the jump: r_p = -C_s L^-1 R_s f
//   = -sum_k cw[p][k] sum_q dS_q f_q sum_(a,b) G(node_pk - (ix_qa, iy_qb)) wx_qa wy_qb ; r_ns = 0
__global__ void __launch_bounds__(256) k_jump_rhs(const int* __restrict__ ci, const int* __restrict__ cj,
                                                  const double* __restrict__ cw, const int* __restrict__ six,
                                                  const int* __restrict__ siy, const double* __restrict__ swx,
                                                  const double* __restrict__ swy, const double* __restrict__ ds,
                                                  const double* __restrict__ f, int ns, const double* __restrict__ G,
                                                  int nx, double* __restrict__ r) {
    __shared__ int pi[64], pj[64];
    __shared__ double pw[64];
    __shared__ double sh[256];
    const int p = blockIdx.x;
    if (p == ns) {
        if (threadIdx.x == 0) r[ns] = 0.0;
        return;
    }
    if (threadIdx.x < 64) {
        pi[threadIdx.x] = ci[64 * p + threadIdx.x];
        pj[threadIdx.x] = cj[64 * p + threadIdx.x];
        pw[threadIdx.x] = cw[64 * p + threadIdx.x];
    }
    __syncthreads();
    double acc = 0.0;
    for (int e = threadIdx.x; e < 16 * ns; e += blockDim.x) {
        const int q = e >> 4, a = e & 3, b = (e >> 2) & 3;
        const int mi = six[4 * q + a], mj = siy[4 * q + b];
        const double src = ds[q] * f[q] * swx[4 * q + a] * swy[4 * q + b];
        double g = 0.0;
        for (int k = 0; k < 64; ++k) g += pw[k] * lgf(G, nx, pi[k] - mi, pj[k] - mj);
        acc += g * src;
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) r[p] = -tot;
}

// Delta p = -rho (E_f u - v_s) . (f z x n) - rho d(Delta phi)/dt, u from psi on the faces
template <typename T>
__global__ void k_pressure_jump(const T* __restrict__ psi, int nx, double dx, const int* __restrict__ fidx,
                                const double* __restrict__ fwt, const double* __restrict__ x,
                                const double* __restrict__ y, const double* __restrict__ nxs,
                                const double* __restrict__ nys, const double* __restrict__ f,
                                const double* __restrict__ dphi_dt, pf_motion m, double rho, int ns,
                                double* __restrict__ dp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ns) return;
    const int* fi = fidx + 16 * p;
    const double* fw = fwt + 16 * p;
    double us = 0.0, vs = 0.0;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
            const size_t ju = (size_t)fi[4 + b] * nx + fi[a];
            us += fw[a] * fw[4 + b] * ((double)psi[ju + nx] - (double)psi[ju]) / dx;
            const size_t jv = (size_t)fi[12 + b] * nx + fi[8 + a];
            vs += fw[8 + a] * fw[12 + b] * -((double)psi[jv + 1] - (double)psi[jv]) / dx;
        }
    us += m.Uinf;
    vs += m.Vinf;
    const double vsx = m.U - m.Omega * y[p], vsy = m.V + m.Omega * x[p];
    const double tx = -nys[p], ty = nxs[p];
    dp[p] = -rho * ((us - vsx) * f[p] * tx + (vs - vsy) * f[p] * ty) - rho * (dphi_dt ? dphi_dt[p] : 0.0);
}

// Pressure field at the cell centres (Eq. pgrid, the surface term inside the
// divergence):  p = -rho/2 |u|^2 - rho L^-1 D [w x u + R_f(n o dDphi/dt - v_s x f)].
// Faces outside the grid count as zero, as in the oracle.
template <typename T>
struct FaceField {
    const T* psi;
    const T* w;
    int nx, ny;
    double dx, Uinf, Vinf;
    __device__ double u(int i, int j) const {            // x-face (i, j + 1/2)
        if (i < 0 || i >= nx || j < 0 || j >= ny - 1) return 0.0;
        return ((double)psi[(size_t)(j + 1) * nx + i] - (double)psi[(size_t)j * nx + i]) / dx + Uinf;
    }
    __device__ double v(int i, int j) const {            // y-face (i + 1/2, j)
        if (i < 0 || i >= nx - 1 || j < 0 || j >= ny) return 0.0;
        return -((double)psi[(size_t)j * nx + i + 1] - (double)psi[(size_t)j * nx + i]) / dx + Vinf;
    }
    __device__ double lx(int i, int j) const {           // -w v on the x-face (i, j + 1/2)
        const double wf = 0.5 * ((double)w[(size_t)j * nx + i] + (double)w[(size_t)(j + 1) * nx + i]);
        return -wf * 0.25 * (v(i - 1, j) + v(i, j) + v(i - 1, j + 1) + v(i, j + 1));
    }
    __device__ double ly(int i, int j) const {           // w u on the y-face (i + 1/2, j)
        const double wf = 0.5 * ((double)w[(size_t)j * nx + i] + (double)w[(size_t)j * nx + i + 1]);
        return wf * 0.25 * (u(i, j - 1) + u(i, j) + u(i + 1, j - 1) + u(i + 1, j));
    }
};

// one thread per centre: the Lamb-vector divergence and the kinetic energy
template <typename T>
__global__ void k_pressure_src(FaceField<T> F, double* __restrict__ src, double* __restrict__ ke) {
    const int nc = F.nx - 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * (F.ny - 1)) return;
    const int i = t % nc, j = t / nc;
    src[t] = (F.lx(i + 1, j) - F.lx(i, j) + F.ly(i, j + 1) - F.ly(i, j)) / F.dx;
    const double u0 = F.u(i, j), u1 = F.u(i + 1, j), v0 = F.v(i, j), v1 = F.v(i, j + 1);
    ke[t] = 0.5 * (u0 * u0 + u1 * u1) + 0.5 * (v0 * v0 + v1 * v1);
}

// surface faces R_f(n o dDphi/dt - v_s x f) gathered by each centre of the box
// from every surface point in index order (deterministic), their divergence
// added to src
__device__ __forceinline__ double face_weight(const int* fi, const double* fw, int lx, int ly, int ii, int jj) {
    const int a = ii - fi[lx], b = jj - fi[ly];
    return (a >= 0 && a < 4 && b >= 0 && b < 4) ? fw[lx + a] * fw[ly + b] : 0.0;
}

__global__ void k_surface_src(const int* __restrict__ fidx, const double* __restrict__ fwt,
                              const double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ nxs, const double* __restrict__ nys,
                              const double* __restrict__ ds, const double* __restrict__ dphi_dt,
                              const double* __restrict__ f, pf_motion m, int ns, int nx, double dx, int i0, int j0,
                              int bw, int bh, double* __restrict__ src) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= bw * bh) return;
    const int i = i0 + t % bw, j = j0 + t / bw;
    double qx0 = 0.0, qx1 = 0.0, qy0 = 0.0, qy1 = 0.0;
    for (int p = 0; p < ns; ++p) {
        const double dd = dphi_dt ? dphi_dt[p] : 0.0, ff = f ? f[p] : 0.0;
        const double vsx = m.U - m.Omega * y[p], vsy = m.V + m.Omega * x[p];
        const double ax = ds[p] * (nxs[p] * dd - vsy * ff), ay = ds[p] * (nys[p] * dd + vsx * ff);
        const int* fi = fidx + 16 * p;
        const double* fw = fwt + 16 * p;
        qx0 += ax * face_weight(fi, fw, 0, 4, i, j);
        qx1 += ax * face_weight(fi, fw, 0, 4, i + 1, j);
        qy0 += ay * face_weight(fi, fw, 8, 12, i, j);
        qy1 += ay * face_weight(fi, fw, 8, 12, i, j + 1);
    }
    src[(size_t)j * (nx - 1) + i] += (qx1 - qx0 + qy1 - qy0) / (dx * dx * dx);
}

template <typename T>
__global__ void k_to_plan(const double* __restrict__ a, int64_t n, T* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)a[i];
}

// p = -rho/2 ke - rho L^-1 src = -rho/2 ke + rho psi_c with psi_c = -L^-1 src
template <typename T>
__global__ void k_pressure_final(const double* __restrict__ ke, const T* __restrict__ psic, int64_t n, double rho,
                                 double* __restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = -0.5 * rho * ke[i] + rho * (double)psic[i];
}

pf_status multibody_check(const pf_multibody& mb, int ns, int* n_edges_total) {
    const int nb = mb.n_bodies;
    if (nb < 1 || nb > PF_MAX_BODIES || mb.start[0] != 0 || mb.start[nb] != ns) return PF_ERR_ARG;
    int ne = 0;
    for (int b = 0; b < nb; ++b) {
        if (mb.start[b + 1] <= mb.start[b] || mb.n_edges[b] < 0 || mb.n_edges[b] > 2) return PF_ERR_ARG;
        for (int j = 0; j < mb.n_edges[b]; ++j)
            if (mb.edge[b][j] < mb.start[b] || mb.edge[b][j] >= mb.start[b + 1]) return PF_ERR_ARG;
        ne += mb.n_edges[b];
    }
    *n_edges_total = ne;
    return PF_OK;
}

// the several-body scratch of a factor: sb, ew, then MB_COLS columns each of
// rhs, y, res, then new vortices (x, y: MB_EDGES each) and the outputs
pf_status multibody_scratch(pf_plan p, pf_schur s) {
    if (s->mwork) return PF_OK;
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    PF_CUDA(p, cudaMalloc(&s->mwork, ((2 + 3 * (size_t)MB_COLS) * s->ns + 2 * MB_EDGES + MB_N) * sizeof(double)));
    return PF_OK;
}

double* multibody_newpos(pf_schur s) { return s->mwork + (2 + 3 * (size_t)MB_COLS) * s->ns; }

pf_status sheet_solve_multi_device(pf_plan p, pf_schur s, const void* w, const pf_multibody& mb, int ne,
                                   const double* vx, const double* vy, double* f, const double* gw_dev,
                                   double** out_dev, int64_t nnz_bound, const VortexSource* vs) {
    const int nb = mb.n_bodies, ns = s->ns, nc = 1 + ne + nb;
    cudaStream_t st = p->stream;
    PF_TRY(multibody_scratch(p, s));
    double* sb = s->mwork;
    double* ew = sb + ns;
    double* rhs = ew + ns;                       // rhs0 | E L^-1 d_i | 1_b
    double* y = rhs + (size_t)MB_COLS * ns;
    double* res = y + (size_t)MB_COLS * ns;
    double* out = multibody_newpos(s) + 2 * MB_EDGES;   // s0 (B), Gamma (E)
    k_sbprime_multi<<<ceil_div(ns, 128), 128, 0, st>>>(s->x, s->y, ns, mb, sb);
    PF_LAUNCH_CHECK(p);
    PF_TRY(surface_rhs(p, s, w, ew, nnz_bound, vs));
    k_rhs0<<<1, 256, 0, st>>>(PF_SHEET_KUTTA_SHED, ns, 0.0, nullptr, sb, ew, s->f0hat, s->dgamma0, rhs);
    if (ne > 0)
        k_unit_vortex<<<dim3(ceil_div(ns, 128), ne), 128, 0, st>>>(vx, vy, ne, s->six, s->siy, s->swx, s->swy, ns,
                                                                    p->G, p->nx, p->ny, p->x0, p->y0, p->dx, rhs + ns,
                                                                    p->d_status);
    k_indicators<<<dim3(ceil_div(ns, 256), nb), 256, 0, st>>>(ns, mb, rhs + (size_t)(1 + ne) * ns);
    k_rows<0><<<rows_grid(ns, nc), 256, 0, st>>>(s->Sinv, ns, rhs, nc, nullptr, y);
    k_rows<1><<<rows_grid(ns, nc), 256, 0, st>>>(s->S, ns, y, nc, rhs, res);
    k_rows<2><<<rows_grid(ns, nc), 256, 0, st>>>(s->Sinv, ns, res, nc, nullptr, y);
    k_constraints_multi<<<1, 256, 0, st>>>(ns, mb, ne, y, s->f0, s->ds, gw_dev, f, out, p->d_status);
    PF_LAUNCH_CHECK(p);
    *out_dev = out;
    return PF_OK;
}

extern "C" {

pf_status pf_schur_factor(pf_plan p, const pf_body_desc* b, pf_schur* out) {
    if (!p || !b || !out || b->ns < 4 || b->ns > PF_MAX_SURFACE_POINTS || !b->x || !b->y || !b->ds) return PF_ERR_ARG;
    *out = nullptr;
    pf_schur s = nullptr;
    pf_status st = schur_create(p, b->ns, &s);
    if (st != PF_OK) return st;
    const size_t v = (size_t)b->ns * sizeof(double);
    if (cudaMemcpyAsync(s->x, b->x, v, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->y, b->y, v, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->ds, b->ds, v, cudaMemcpyHostToDevice, p->stream) != cudaSuccess) {
        schur_free(s);
        return PF_ERR_CUDA;
    }
    st = schur_factor_device(p, s);
    if (st != PF_OK) {
        schur_free(s);
        return st;
    }
    int status = 0;
    if (cudaMemcpyAsync(&s->gamma0, s->dgamma0, sizeof(double), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaMemcpyAsync(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
        schur_free(s);
        return PF_ERR_CUDA;
    }
    if (status & (ST_SINGULAR | ST_OUT_OF_DOMAIN)) {
        cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream);
        cudaStreamSynchronize(p->stream);
        schur_free(s);
        return (status & ST_OUT_OF_DOMAIN) ? PF_ERR_OUT_OF_DOMAIN : PF_ERR_SINGULAR;
    }
    *out = s;
    return PF_OK;
}

pf_status pf_schur_destroy(pf_schur s) {
    if (!s) return PF_ERR_ARG;
    cudaStreamSynchronize(s->plan->stream);
    schur_free(s);
    return PF_OK;
}

pf_status pf_schur_info(pf_schur s, double* gamma0, double* f0, double* S) {
    if (!s) return PF_ERR_ARG;
    pf_plan p = s->plan;
    if (gamma0) *gamma0 = s->gamma0;
    if (f0) PF_CUDA(p, cudaMemcpyAsync(f0, s->f0, (size_t)s->ns * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    if (S)
        PF_CUDA(p, cudaMemcpyAsync(S, s->S, (size_t)s->ns * s->ns * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    return PF_OK;
}

pf_status pf_sheet_solve(pf_plan p, pf_schur s, const void* w, const pf_motion* m, int32_t mode, double param,
                         int32_t n_edges, const int32_t* edges, const double* Xnew, const double* Ynew, double* f,
                         double* gamma_new, double* s0) {
    if (!p || !w || !m || !f || mode < PF_SHEET_GIVEN_S0 || mode > PF_SHEET_KUTTA_SHED) return PF_ERR_ARG;
    if (!s) return PF_ERR_NOT_FACTORED;
    const bool kutta = mode == PF_SHEET_KUTTA_STEADY || mode == PF_SHEET_KUTTA_SHED;
    if (kutta && (n_edges < 1 || n_edges > 2 || !edges || (mode == PF_SHEET_KUTTA_STEADY && n_edges != 1)))
        return PF_ERR_ARG;
    if (!kutta) n_edges = 0;
    for (int e = 0; e < n_edges; ++e)
        if (edges[e] < 0 || edges[e] >= s->ns) return PF_ERR_ARG;
    if (mode == PF_SHEET_KUTTA_SHED && (!Xnew || !Ynew)) return PF_ERR_ARG;
    double* vxy = s->scal + 4;   // device slots for up to two new vortices: x at [4,5], y at [6,7]
    if (mode == PF_SHEET_KUTTA_SHED) {
        PF_CUDA(p, cudaMemcpyAsync(vxy, Xnew, n_edges * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(vxy + 2, Ynew, n_edges * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    }
    pf_status st = sheet_solve_device(p, s, w, *m, mode, param, nullptr, n_edges, edges, vxy, vxy + 2, f);
    if (st != PF_OK) return st;
    double sc[3];
    PF_CUDA(p, cudaMemcpyAsync(sc, s->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    if (s0) *s0 = sc[0];
    if (gamma_new)
        for (int e = 0; e < (mode == PF_SHEET_KUTTA_SHED ? n_edges : 0); ++e) gamma_new[e] = sc[1 + e];
    return PF_OK;
}

pf_status pf_sheet_solve_vortices(pf_plan p, pf_schur s, const double* X, const double* Y, const double* Gam,
                                  int64_t nv, const pf_motion* m, int32_t mode, double param, int32_t n_edges,
                                  const int32_t* edges, const double* Xnew, const double* Ynew, double* f,
                                  double* gamma_new, double* s0) {
    if (!p || !m || !f || nv < 0 || (nv > 0 && (!X || !Y || !Gam)) || mode < PF_SHEET_GIVEN_S0 ||
        mode > PF_SHEET_KUTTA_SHED)
        return PF_ERR_ARG;
    if (!s) return PF_ERR_NOT_FACTORED;
    const bool kutta = mode == PF_SHEET_KUTTA_STEADY || mode == PF_SHEET_KUTTA_SHED;
    if (kutta && (n_edges < 1 || n_edges > 2 || !edges || (mode == PF_SHEET_KUTTA_STEADY && n_edges != 1)))
        return PF_ERR_ARG;
    if (!kutta) n_edges = 0;
    for (int e = 0; e < n_edges; ++e)
        if (edges[e] < 0 || edges[e] >= s->ns) return PF_ERR_ARG;
    if (mode == PF_SHEET_KUTTA_SHED && (!Xnew || !Ynew)) return PF_ERR_ARG;
    double* vxy = s->scal + 4;
    if (mode == PF_SHEET_KUTTA_SHED) {
        PF_CUDA(p, cudaMemcpyAsync(vxy, Xnew, n_edges * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(vxy + 2, Ynew, n_edges * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    }
    VortexSource vs;
    vs.X = X;
    vs.Y = Y;
    vs.G = Gam;
    vs.n = nv;
    vs.force = true;
    // with no vortices the free vorticity is zero: the plan's zeroed field stands in for w
    if (nv == 0) PF_CUDA(p, cudaMemsetAsync(p->w, 0, (size_t)p->nx * p->ny * p->esz, p->stream));
    pf_status st = sheet_solve_device(p, s, p->w, *m, mode, param, nullptr, n_edges, edges, vxy, vxy + 2, f,
                                      EdgeBounds(), -1, nv > 0 ? &vs : nullptr);
    if (st != PF_OK) return st;
    double sc[3];
    PF_CUDA(p, cudaMemcpyAsync(sc, s->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    if (s0) *s0 = sc[0];
    if (gamma_new)
        for (int e = 0; e < (mode == PF_SHEET_KUTTA_SHED ? n_edges : 0); ++e) gamma_new[e] = sc[1 + e];
    return PF_OK;
}

pf_status pf_sheet_solve_multi(pf_plan p, pf_schur s, const void* w, const pf_multibody* mb, const double* Xnew,
                               const double* Ynew, double* f, double* gamma_new, double* s0) {
    if (!p || !w || !mb || !f) return PF_ERR_ARG;
    if (!s) return PF_ERR_NOT_FACTORED;
    const int nb = mb->n_bodies;
    int ne = 0;
    PF_TRY(multibody_check(*mb, s->ns, &ne));
    if (ne > 0 && (!Xnew || !Ynew)) return PF_ERR_ARG;
    cudaStream_t st = p->stream;
    PF_TRY(multibody_scratch(p, s));
    double* vx = multibody_newpos(s);
    if (ne > 0) {
        PF_CUDA(p, cudaMemcpyAsync(vx, Xnew, ne * sizeof(double), cudaMemcpyHostToDevice, st));
        PF_CUDA(p, cudaMemcpyAsync(vx + MB_EDGES, Ynew, ne * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    double* out = nullptr;
    PF_TRY(sheet_solve_multi_device(p, s, w, *mb, ne, vx, vx + MB_EDGES, f, nullptr, &out));
    double h[MB_N];
    int status = 0;
    PF_CUDA(p, cudaMemcpyAsync(h, out, (nb + ne) * sizeof(double), cudaMemcpyDeviceToHost, st));
    PF_CUDA(p, cudaMemcpyAsync(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PF_CUDA(p, cudaStreamSynchronize(st));
    if (status & ST_SINGULAR) {
        const int keep = status & ~ST_SINGULAR;
        PF_CUDA(p, cudaMemcpyAsync(p->d_status, &keep, sizeof(int), cudaMemcpyHostToDevice, st));
        PF_CUDA(p, cudaStreamSynchronize(st));
        return PF_ERR_SINGULAR;
    }
    if (s0)
        for (int b = 0; b < nb; ++b) s0[b] = h[b];
    if (gamma_new)
        for (int i = 0; i < ne; ++i) gamma_new[i] = h[nb + i];
    return PF_OK;
}

pf_status pf_sheet_regularize(pf_plan p, pf_schur s, const double* f, void* w) {
    if (!p || !f || !w) return PF_ERR_ARG;
    if (!s) return PF_ERR_NOT_FACTORED;
    return sheet_deposit(p, s, f, w);
}

pf_status pf_pressure_setup(pf_plan p, pf_schur s, const double* nxs, const double* nys) {
    if (!p || !nxs || !nys) return PF_ERR_ARG;
    if (!s) return PF_ERR_NOT_FACTORED;
    const int ns = s->ns;
    cudaStream_t st = p->stream;
    PF_CUDA(p, cudaStreamSynchronize(st));
    if (!s->pnx) {
        PF_CUDA(p, cudaMalloc(&s->pnx, ns * sizeof(double)));
        PF_CUDA(p, cudaMalloc(&s->pny, ns * sizeof(double)));
        PF_CUDA(p, cudaMalloc(&s->fidx, 16 * (size_t)ns * sizeof(int)));
        PF_CUDA(p, cudaMalloc(&s->fwt, 16 * (size_t)ns * sizeof(double)));
        PF_CUDA(p, cudaMalloc(&s->ci, 64 * (size_t)ns * sizeof(int)));
        PF_CUDA(p, cudaMalloc(&s->cj, 64 * (size_t)ns * sizeof(int)));
        PF_CUDA(p, cudaMalloc(&s->cw, 64 * (size_t)ns * sizeof(double)));
    }
    if (!s->jump) PF_TRY(schur_create(p, ns + 1, &s->jump));
    PF_CUDA(p, cudaMemcpyAsync(s->pnx, nxs, ns * sizeof(double), cudaMemcpyHostToDevice, st));
    PF_CUDA(p, cudaMemcpyAsync(s->pny, nys, ns * sizeof(double), cudaMemcpyHostToDevice, st));
    k_face_stencil<<<ceil_div(16 * ns, 64), 64, 0, st>>>(s->x, s->y, ns, p->x0, p->y0, p->dx, p->nx, p->ny, s->fidx,
                                                          s->fwt, p->d_status);
    k_curl_stencil<<<ceil_div(64 * ns, 256), 256, 0, st>>>(s->fidx, s->fwt, s->pnx, s->pny, ns, p->dx, s->ci, s->cj,
                                                            s->cw);
    k_jump_build<<<dim3(ns + 1, ns + 1), 256, 0, st>>>(s->ci, s->cj, s->cw, s->ds, ns, p->G, p->nx, s->jump->S);
    PF_LAUNCH_CHECK(p);
    PF_TRY(invert_schur_matrix(p, s->jump));
    // the cell-centre box the surface faces can reach (stencils of 4 faces from floor - 1)
    std::vector<double> hx(ns), hy(ns);
    PF_CUDA(p, cudaMemcpyAsync(hx.data(), s->x, ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    PF_CUDA(p, cudaMemcpyAsync(hy.data(), s->y, ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    PF_CUDA(p, cudaStreamSynchronize(st));
    const double xlo = *std::min_element(hx.begin(), hx.end()), xhi = *std::max_element(hx.begin(), hx.end());
    const double ylo = *std::min_element(hy.begin(), hy.end()), yhi = *std::max_element(hy.begin(), hy.end());
    s->pbox[0] = std::max(0, (int)floor((xlo - p->x0) / p->dx) - 4);
    s->pbox[1] = std::min(p->nx - 2, (int)floor((xhi - p->x0) / p->dx) + 4);
    s->pbox[2] = std::max(0, (int)floor((ylo - p->y0) / p->dx) - 4);
    s->pbox[3] = std::min(p->ny - 2, (int)floor((yhi - p->y0) / p->dx) + 4);
    return PF_OK;
}

pf_status pf_pressure_field(pf_plan p, pf_schur s, const void* psi, const void* w, const pf_motion* m, const double* f,
                            const double* dphi_dt, double rho, double* pout) {
    if (!p || !psi || !w || !m || !pout) return PF_ERR_ARG;
    if (s && !s->jump) return PF_ERR_NOT_FACTORED;
    cudaStream_t st = p->stream;
    const int64_t nc = (int64_t)(p->nx - 1) * (p->ny - 1);
    if (!p->centres) {
        pf_grid_desc d{p->nx - 1, p->ny - 1, p->dx, p->x0 + 0.5 * p->dx, p->y0 + 0.5 * p->dx, p->prec};
        PF_TRY(pf_plan_create(&d, st, &p->centres));
        PF_CUDA(p, cudaMalloc(&p->pscr, 2 * (size_t)nc * sizeof(double)));
    }
    double* src = p->pscr;
    double* ke = src + nc;
    const int nb = (int)std::min<int64_t>(ceil_div(nc, 256), 152 * 8);
    if (p->prec == PF_FP64)
        k_pressure_src<double><<<ceil_div(nc, 256), 256, 0, st>>>(
            FaceField<double>{(const double*)psi, (const double*)w, p->nx, p->ny, p->dx, m->Uinf, m->Vinf}, src, ke);
    else
        k_pressure_src<float><<<ceil_div(nc, 256), 256, 0, st>>>(
            FaceField<float>{(const float*)psi, (const float*)w, p->nx, p->ny, p->dx, m->Uinf, m->Vinf}, src, ke);
    PF_LAUNCH_CHECK(p);
    if (s && (f || dphi_dt) && s->pbox[1] >= s->pbox[0] && s->pbox[3] >= s->pbox[2]) {
        const int bw = s->pbox[1] - s->pbox[0] + 1, bh = s->pbox[3] - s->pbox[2] + 1;
        k_surface_src<<<ceil_div(bw * bh, 128), 128, 0, st>>>(s->fidx, s->fwt, s->x, s->y, s->pnx, s->pny, s->ds,
                                                               dphi_dt, f, *m, s->ns, p->nx, p->dx, s->pbox[0],
                                                               s->pbox[2], bw, bh, src);
        PF_LAUNCH_CHECK(p);
    }
    pf_plan c = p->centres;
    if (p->prec == PF_FP64) {
        k_to_plan<double><<<nb, 256, 0, st>>>(src, nc, (double*)c->w);
        PF_TRY(conv_solve(c, c->w, c->uv, CONV_PSI, 0.0, 0.0));
        k_pressure_final<double><<<nb, 256, 0, st>>>(ke, (const double*)c->uv, nc, rho, pout);
    } else {
        k_to_plan<float><<<nb, 256, 0, st>>>(src, nc, (float*)c->w);
        PF_TRY(conv_solve(c, c->w, c->uv, CONV_PSI, 0.0, 0.0));
        k_pressure_final<float><<<nb, 256, 0, st>>>(ke, (const float*)c->uv, nc, rho, pout);
    }
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

pf_status pf_potential_jump(pf_plan p, pf_schur s, const double* f, double* dphi) {
    if (!p || !f || !dphi) return PF_ERR_ARG;
    if (!s || !s->jump) return PF_ERR_NOT_FACTORED;
    const int ns = s->ns, n1 = ns + 1;
    cudaStream_t st = p->stream;
    double* r = s->jump->work;          // right-hand side (n1), then the solution (n1), then the residual
    double* y = r + n1;
    double* res = y + n1;
    k_jump_rhs<<<n1, 256, 0, st>>>(s->ci, s->cj, s->cw, s->six, s->siy, s->swx, s->swy, s->ds, f, ns, p->G, p->nx, r);
    k_rows<0><<<rows_grid(n1, 1), 256, 0, st>>>(s->jump->Sinv, n1, r, 1, nullptr, y);
    k_rows<1><<<rows_grid(n1, 1), 256, 0, st>>>(s->jump->S, n1, y, 1, r, res);
    k_rows<2><<<rows_grid(n1, 1), 256, 0, st>>>(s->jump->Sinv, n1, res, 1, nullptr, y);
    PF_LAUNCH_CHECK(p);
    PF_CUDA(p, cudaMemcpyAsync(dphi, y, ns * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return PF_OK;
}

pf_status pf_pressure_jump(pf_plan p, pf_schur s, const void* psi, const pf_motion* m, const double* f,
                           const double* dphi_dt, double rho, double* dp) {
    if (!p || !psi || !m || !f || !dp) return PF_ERR_ARG;
    if (!s || !s->jump) return PF_ERR_NOT_FACTORED;
    const int ns = s->ns;
    cudaStream_t st = p->stream;
    if (p->prec == PF_FP64)
        k_pressure_jump<double><<<ceil_div(ns, 128), 128, 0, st>>>((const double*)psi, p->nx, p->dx, s->fidx, s->fwt,
                                                                   s->x, s->y, s->pnx, s->pny, f, dphi_dt, *m, rho, ns,
                                                                   dp);
    else
        k_pressure_jump<float><<<ceil_div(ns, 128), 128, 0, st>>>((const float*)psi, p->nx, p->dx, s->fidx, s->fwt,
                                                                  s->x, s->y, s->pnx, s->pny, f, dphi_dt, *m, rho, ns,
                                                                  dp);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

pf_status pf_sheet_solve_edges(pf_plan p, pf_schur s, const void* w, const pf_motion* m, double gamma_w,
                               int32_t n_edges, const int32_t* edges, const double* bounds, const double* Xnew,
                               const double* Ynew, double* f, double* gamma_new, double* s0) {
    if (!p || !w || !m || !f || !bounds || !edges || !Xnew || !Ynew || n_edges < 1 || n_edges > 2) return PF_ERR_ARG;
    if (!s) return PF_ERR_NOT_FACTORED;
    EdgeBounds eb;
    eb.on = 1;
    for (int e = 0; e < n_edges; ++e) {
        if (edges[e] < 0 || edges[e] >= s->ns || !(bounds[2 * e] <= bounds[2 * e + 1])) return PF_ERR_ARG;
        eb.lo[e] = bounds[2 * e];
        eb.hi[e] = bounds[2 * e + 1];
    }
    double* vxy = s->scal + 4;
    PF_CUDA(p, cudaMemcpyAsync(vxy, Xnew, n_edges * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(vxy + 2, Ynew, n_edges * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    pf_status st = sheet_solve_device(p, s, w, *m, PF_SHEET_KUTTA_SHED, gamma_w, nullptr, n_edges, edges, vxy, vxy + 2,
                                      f, eb);
    if (st != PF_OK) return st;
    double sc[3];
    PF_CUDA(p, cudaMemcpyAsync(sc, s->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    if (s0) *s0 = sc[0];
    if (gamma_new)
        for (int e = 0; e < n_edges; ++e) gamma_new[e] = sc[1 + e];
    return PF_OK;
}

}  // extern "C"

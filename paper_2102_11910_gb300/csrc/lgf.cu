// Lattice Green's function of the unit-spacing 5-point Laplacian and its
// spectrum on the padded torus, built once per plan in FP64 (Sec. 2.1, the
// LGF of refs. katsura71 / cserti00 / liska14 that gives L^{-1} with unbounded
// boundary conditions).
//
// G(m,n) = 1/(2 pi) Int_0^pi [1 - exp(-2M u) cos(N t)] / sinh(2u) dt,
//   u = asinh(sin(t/2)), M = max(|m|,|n|), N = min(|m|,|n|),
// which follows from the 2D Fourier definition by integrating one variable by
// residues; G(0,0) = 0.  The integral is evaluated with a double-exponential
// (tanh-sinh type) rule, t = pi / (1 + exp(-pi sinh s)), step 1/64 on
// s in [-5, 3.3]; the rule resolves the exp(-2Mu) layer at t ~ 1/M for every
// grid size the library accepts.  The numerator is split as
// (1 - e^{-2Mu}) + e^{-2Mu} 2 sin^2(N t/2) so both terms are cancellation free.
#include <math.h>

#include <vector>

#include "common.cuh"

pf_status fft2d_inplace_f64(pf_plan p, double2* data);

namespace {

constexpr int DE_STEPS_PER_UNIT = 64;
constexpr double DE_S_MIN = -5.0;
constexpr int DE_NODES = 532;   // s_k = -5 + k/64, k = 0..531

__global__ void k_lgf_table(double* __restrict__ G, int nx, int ny, const double* __restrict__ node_t,
                            const double* __restrict__ node_u, const double* __restrict__ node_c, int nn) {
    extern __shared__ double sh[];
    double* st = sh;
    double* su = sh + nn;
    double* sc = sh + 2 * nn;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        st[k] = node_t[k];
        su[k] = node_u[k];
        sc[k] = node_c[k];
    }
    __syncthreads();
    const int64_t total = (int64_t)(nx + 1) * (ny + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e % (nx + 1));
        const int n = (int)(e / (nx + 1));
        const int M = m > n ? m : n;
        const int N = m > n ? n : m;
        double acc = 0.0;
        if (M > 0) {
            for (int k = 0; k < nn; ++k) {
                const double x = -2.0 * M * su[k];
                double ex, em1;
                if (x > -0.5) {
                    em1 = expm1(x);
                    ex = 1.0 + em1;
                } else {
                    ex = exp(x);
                    em1 = ex - 1.0;
                }
                const double sn = sin(0.5 * N * st[k]);
                acc += sc[k] * (-em1 + ex * 2.0 * sn * sn);
            }
        }
        G[e] = acc;
    }
}

__device__ __forceinline__ double lgf_at(const double* __restrict__ G, int nx, int m, int n) {
    return G[(size_t)(n < 0 ? -n : n) * (nx + 1) + (m < 0 ? -m : m)];
}

// Kernels placed on the P x Q torus (row-major, P fastest) at signed offsets
// (m, n); offsets a linear convolution over the grid never reaches are zero.
//   which = 0: G(m, n)                                     (psi:  -dx^2 G * w)
//   which = 1: G(m, n+1) - G(m, n-1),  |n| <= ny-1          (u:   -dx/2 D_y G * w)
//   which = 2: G(m+1, n) - G(m-1, n),  |m| <= nx-1          (v:   +dx/2 D_x G * w)
// The differenced kernels decay like 1/r, so their FP64 spectra carry far less
// rounding than the derivative symbol applied to the spectrum of G.
__global__ void k_torus(double2* __restrict__ g, const double* __restrict__ G, int nx, int ny, int P, int Q, int which) {
    const int64_t total = (int64_t)P * Q;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int mt = (int)(e % P), nt = (int)(e / P);
        const int m = mt <= P / 2 ? mt : mt - P;
        const int n = nt <= Q / 2 ? nt : nt - Q;
        const int am = m < 0 ? -m : m, an = n < 0 ? -n : n;
        double v = 0.0;
        if (which == 0) {
            if (am <= nx && an <= ny) v = lgf_at(G, nx, m, n);
        } else if (which == 1) {
            if (am <= nx && an <= ny - 1) v = lgf_at(G, nx, m, n + 1) - lgf_at(G, nx, m, n - 1);
        } else {
            if (am <= nx - 1 && an <= ny) v = lgf_at(G, nx, m + 1, n) - lgf_at(G, nx, m - 1, n);
        }
        g[e] = make_double2(v, 0.0);
    }
}

// quadrant k in [0, P/2], l in [0, Q/2] of scale * (Re or Im) of the spectrum
__global__ void k_extract(const double2* __restrict__ g, double* __restrict__ H64, float* __restrict__ H32, int P,
                          int Q, int Hld, double scale, int imag) {
    const int hp = P / 2 + 1, hq = Q / 2 + 1;
    const int64_t total = (int64_t)hp * hq;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e % hq), k = (int)(e / hq);
        const double2 c = g[(size_t)l * P + k];
        const double v = scale * (imag ? c.y : c.x);
        H64[(size_t)k * Hld + l] = v;
        H32[(size_t)k * Hld + l] = (float)v;
    }
}

}  // namespace

pf_status lgf_build(pf_plan p) {
    const int nx = p->nx, ny = p->ny, P = p->P, Q = p->Q;
    // quadrature nodes (host, FP64)
    std::vector<double> t(DE_NODES), u(DE_NODES), c(DE_NODES);
    const double h = 1.0 / DE_STEPS_PER_UNIT;
    for (int k = 0; k < DE_NODES; ++k) {
        const double s = DE_S_MIN + k * h;
        const double z = M_PI * sinh(s);
        const double sig = 1.0 / (1.0 + exp(-z));
        const double sigm = 1.0 / (1.0 + exp(z));
        const double th = M_PI * sig;
        const double dth = M_PI * M_PI * cosh(s) * sig * sigm;
        const double uu = asinh(sin(0.5 * th));
        t[k] = th;
        u[k] = uu;
        c[k] = h * dth / (sinh(2.0 * uu) * 2.0 * M_PI);
    }
    double* dn = nullptr;
    PF_CUDA(p, cudaMalloc(&dn, 3 * DE_NODES * sizeof(double)));
    PF_CUDA(p, cudaMemcpyAsync(dn, t.data(), DE_NODES * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(dn + DE_NODES, u.data(), DE_NODES * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(dn + 2 * DE_NODES, c.data(), DE_NODES * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    const size_t sh = 3 * DE_NODES * sizeof(double);
    k_lgf_table<<<4 * 152, 256, sh, p->stream>>>(p->G, nx, ny, dn, dn + DE_NODES, dn + 2 * DE_NODES, DE_NODES);
    PF_LAUNCH_CHECK(p);

    double2* g = nullptr;
    PF_CUDA(p, cudaMalloc(&g, (size_t)P * Q * sizeof(double2)));
    const double inv_pq = 1.0 / ((double)P * Q);
    // psi: -dx^2 Ghat/(PQ) (real, even);  u: -dx/2 Im(DyG^)/(PQ) (odd in l);  v: +dx/2 Im(DxG^)/(PQ) (odd in k)
    double* H64[3] = {p->H64, p->Hu64, p->Hv64};
    float* H32[3] = {p->H32, p->Hu32, p->Hv32};
    const double scale[3] = {-p->dx * p->dx * inv_pq, -0.5 * p->dx * inv_pq, 0.5 * p->dx * inv_pq};
    for (int which = 0; which < 3; ++which) {
        k_torus<<<4 * 152, 256, 0, p->stream>>>(g, p->G, nx, ny, P, Q, which);
        PF_LAUNCH_CHECK(p);
        pf_status st = fft2d_inplace_f64(p, g);
        if (st != PF_OK) return st;
        k_extract<<<4 * 152, 256, 0, p->stream>>>(g, H64[which], H32[which], P, Q, p->Hld, scale[which], which != 0);
        PF_LAUNCH_CHECK(p);
    }
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    cudaFree(g);
    cudaFree(dn);
    return PF_OK;
}

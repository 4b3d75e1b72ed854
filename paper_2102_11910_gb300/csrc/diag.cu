// Impulse diagnostics (Sec. 2.6.2, Eqs. linimpxd, linimpyd, angimpd).
//
// The node terms are written through the integer moments of w,
//   A00 = sum w,  A10 = sum i w,  A01 = sum j w,  B = sum (i^2 + j^2) w,
// so that with x_i = x0 + i dx, y_j = y0 + j dx
//   <y, w>_N = dx^2 (y0 A00 + dx A01),   <x, w>_N = dx^2 (x0 A00 + dx A10),
//   <x^2 + y^2, w>_N = dx^2 ((x0^2 + y0^2) A00 + 2 dx (x0 A10 + y0 A01) + dx^2 B).
// Each row is summed in the grid's precision (integer weights are exact) in a
// fixed tree order, everything above that in FP64 in a fixed order: the result
// does not depend on the launch.
#include <math.h>

#include "common.cuh"

namespace {

constexpr int IMP_THREADS = 256;
constexpr int IMP_PER = 8;           // nodes of a row per thread: nx <= 2048

// One block per row j: the row's sums of w, i w and i^2 w in the grid's
// precision (tree order), then its contribution to the four moments in FP64.
template <typename T>
__global__ void __launch_bounds__(IMP_THREADS) k_impulse_rows(const T* __restrict__ w, int nx,
                                                              double* __restrict__ part) {
    __shared__ T red[3][IMP_THREADS / 32];
    const int j = blockIdx.x;
    const T* row = w + (size_t)j * nx;
    T v[IMP_PER];
#pragma unroll
    for (int k = 0; k < IMP_PER; ++k) {                  // all loads in flight together
        const int i = threadIdx.x + IMP_THREADS * k;
        v[k] = i < nx ? row[i] : T(0);
    }
    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int k = 0; k < IMP_PER; ++k) {
        const T fi = (T)(threadIdx.x + IMP_THREADS * k);  // exact integer
        s0 += v[k];
        s1 += fi * v[k];
        s2 += fi * fi * v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        red[0][wid] = s0;
        red[1][wid] = s1;
        red[2][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T a = 0, b = 0, c = 0;
        for (int q = 0; q < IMP_THREADS / 32; ++q) {
            a += red[0][q];
            b += red[1][q];
            c += red[2][q];
        }
        const double dj = (double)j, d0 = (double)a;
        double* o = part + (size_t)j * 4;
        o[0] = d0;
        o[1] = (double)b;
        o[2] = dj * d0;
        o[3] = (double)c + dj * dj * d0;
    }
}

// One block: the node moments from the per-row partials (fixed order), the
// surface terms, and the three impulses.
__global__ void __launch_bounds__(IMP_THREADS) k_impulse_final(const double* __restrict__ part, int nparts, double dx,
                                                               double x0, double y0, int ns,
                                                               const double* __restrict__ xs,
                                                               const double* __restrict__ ys,
                                                               const double* __restrict__ ds,
                                                               const double* __restrict__ f,
                                                               const double* __restrict__ nxs,
                                                               const double* __restrict__ nys, double U, double V,
                                                               double Omega, double* __restrict__ out) {
    __shared__ double red[7][IMP_THREADS / 32];
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll 8
    for (int q = threadIdx.x; q < nparts; q += IMP_THREADS)
        for (int k = 0; k < 4; ++k) v[k] += part[(size_t)q * 4 + k];
#pragma unroll 4
    for (int p = threadIdx.x; p < ns; p += IMP_THREADS) {
        double dens = f[p];
        if (nxs) {
            const double vx = U - Omega * ys[p], vy = V + Omega * xs[p];
            dens += nxs[p] * vy - nys[p] * vx;
        }
        const double a = ds[p] * dens;
        v[4] += a * ys[p];
        v[5] += a * xs[p];
        v[6] += a * (xs[p] * xs[p] + ys[p] * ys[p]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[k][wid] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[7];
        for (int k = 0; k < 7; ++k) {
            s[k] = 0.0;
            for (int q = 0; q < IMP_THREADS / 32; ++q) s[k] += red[k][q];
        }
        const double A00 = s[0], A10 = s[1], A01 = s[2], B = s[3], dA = dx * dx;
        out[0] = dA * (y0 * A00 + dx * A01) + s[4];
        out[1] = -dA * (x0 * A00 + dx * A10) - s[5];
        out[2] = -0.5 * dA * ((x0 * x0 + y0 * y0) * A00 + 2.0 * dx * (x0 * A10 + y0 * A01) + dx * dx * B) - 0.5 * s[6];
    }
}

}  // namespace

extern "C" pf_status pf_impulse(pf_plan p, const void* w, const pf_body_desc* body, const double* nxs,
                                const double* nys, const double* f, const pf_motion* m, double* out) {
    if (!p || !w || !out) return PF_ERR_ARG;
    if (body && (body->ns < 0 || body->ns > PF_MAX_SURFACE_POINTS ||
                 (body->ns > 0 && (!body->x || !body->y || !body->ds || !f))))
        return PF_ERR_ARG;
    if ((nxs == nullptr) != (nys == nullptr)) return PF_ERR_ARG;
    const int ns = body ? body->ns : 0;
    constexpr int SURF0 = 2048 * 4 + 3;           // per-row partials of up to 2048 rows, results
    static_assert(PF_DIAG_DOUBLES >= SURF0 + 5 * PF_MAX_SURFACE_POINTS, "plan diagnostics buffer");
    double* dev = p->diag;     // partials, the three results, then x, y, dS, n_x, n_y of the surface
    double* sx = dev + SURF0;
    double* sy = sx + PF_MAX_SURFACE_POINTS;
    double* sds = sy + PF_MAX_SURFACE_POINTS;
    double* snx = sds + PF_MAX_SURFACE_POINTS;
    double* sny = snx + PF_MAX_SURFACE_POINTS;
    if (ns > 0) {
        const size_t b = (size_t)ns * sizeof(double);
        PF_CUDA(p, cudaMemcpyAsync(sx, body->x, b, cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(sy, body->y, b, cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(sds, body->ds, b, cudaMemcpyHostToDevice, p->stream));
        if (nxs) {
            PF_CUDA(p, cudaMemcpyAsync(snx, nxs, b, cudaMemcpyHostToDevice, p->stream));
            PF_CUDA(p, cudaMemcpyAsync(sny, nys, b, cudaMemcpyHostToDevice, p->stream));
        }
    }
    static_assert(IMP_THREADS * IMP_PER >= 2048, "a row fits one block");
    const int nb = p->ny;
    if (p->prec == PF_FP64)
        PF_KERNEL(p, "impulse", k_impulse_rows<double><<<nb, IMP_THREADS, 0, p->stream>>>((const double*)w, p->nx,
                                                                                          dev));
    else
        PF_KERNEL(p, "impulse", k_impulse_rows<float><<<nb, IMP_THREADS, 0, p->stream>>>((const float*)w, p->nx,
                                                                                        dev));
    const double U = m ? m->U : 0.0, V = m ? m->V : 0.0, Om = m ? m->Omega : 0.0;
    double* res = dev + (size_t)2048 * 4;
    PF_KERNEL(p, "impulse_final",
              k_impulse_final<<<1, IMP_THREADS, 0, p->stream>>>(dev, nb, p->dx, p->x0, p->y0, ns,
                                                                sx, sy, sds, ns ? f : nullptr,
                                                                (ns && nxs) ? snx : nullptr,
                                                                (ns && nxs) ? sny : nullptr, U, V, Om, res));
    PF_CUDA(p, cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    return PF_OK;
}

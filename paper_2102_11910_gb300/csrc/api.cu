// C-ABI entry points of gridpf (declared in include/gridpf.h).
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "common.cuh"

namespace {

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

void free_plan(pf_plan p) {
    for (cudaEvent_t e : p->tm.ev) cudaEventDestroy(e);
    for (cudaEvent_t e : p->tm.pool) cudaEventDestroy(e);
    void* own[] = {p->T1, p->T2a, p->T2b, p->w, p->uv, p->tile_count, p->gmax, p->tile_start, p->bin_off,
                   p->pos, p->recs, p->stage, p->stage_out, p->diag, p->rhs64, p->nz_idx, p->nz_val, p->vent_idx, p->vent_val,
                   p->d_status, p->d_oob};
    for (void* q : own)
        if (q) cudaFree(q);
    if (p->pscr) cudaFree(p->pscr);
    if (p->centres) {
        free_plan(p->centres);
        delete p->centres;
    }
    if (p->shared && --p->shared->refs == 0) {
        void* tables[] = {p->G, p->H64, p->H32, p->Hu64, p->Hv64, p->Hu32, p->Hv32, p->twP64, p->twQ64, p->twP32,
                          p->twQ32, p->tw256_64, p->tw256_32};
        for (void* q : tables)
            if (q) cudaFree(q);
        if (p->shared->df) cudaFree(p->shared->df);
        delete p->shared;
    }
}

template <typename C>
void twiddles(std::vector<C>& v, int N) {
    v.resize(N);
    for (int m = 0; m < N; ++m) {
        // exp(-2 pi i m / N) with exact values at the quarter points
        double c, s;
        if (m == 0) { c = 1; s = 0; }
        else if (4 * m == N) { c = 0; s = -1; }
        else if (2 * m == N) { c = -1; s = 0; }
        else if (4 * m == 3 * N) { c = 0; s = 1; }
        else { c = cos(2.0 * M_PI * m / N); s = -sin(2.0 * M_PI * m / N); }
        v[m].x = (decltype(v[m].x))c;
        v[m].y = (decltype(v[m].y))s;
    }
}

template <typename T>
pf_status upload(pf_plan p, T** dst, const std::vector<T>& src) {
    PF_CUDA(p, cudaMalloc(dst, src.size() * sizeof(T)));
    PF_CUDA(p, cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return PF_OK;
}


pf_status plan_workspaces(pf_plan p);

pf_status plan_init(pf_plan p) {
    const int nx = p->nx, ny = p->ny, P = p->P, Q = p->Q;
    p->shared = new (std::nothrow) PlanTables();
    if (!p->shared) return PF_ERR_OOM;
    PF_CUDA(p, cudaMalloc(&p->G, (size_t)(nx + 1) * (ny + 1) * sizeof(double)));
    p->Hld = (Q / 2 + 1 + 3) / 4 * 4;
    const size_t hq = (size_t)(P / 2 + 1) * p->Hld;
    for (double** h : {&p->H64, &p->Hu64, &p->Hv64}) {
        PF_CUDA(p, cudaMalloc(h, hq * sizeof(double)));
        PF_CUDA(p, cudaMemsetAsync(*h, 0, hq * sizeof(double), p->stream));
    }
    for (float** h : {&p->H32, &p->Hu32, &p->Hv32}) {
        PF_CUDA(p, cudaMalloc(h, hq * sizeof(float)));
        PF_CUDA(p, cudaMemsetAsync(*h, 0, hq * sizeof(float), p->stream));
    }
    std::vector<double2> tpd, tqd;
    std::vector<float2> tpf, tqf;
    twiddles(tpd, P); twiddles(tqd, Q); twiddles(tpf, P); twiddles(tqf, Q);
    PF_TRY(upload(p, &p->twP64, tpd));
    PF_TRY(upload(p, &p->twQ64, tqd));
    PF_TRY(upload(p, &p->twP32, tpf));
    PF_TRY(upload(p, &p->twQ32, tqf));
    std::vector<double2> t256d;
    std::vector<float2> t256f;
    twiddles(t256d, 256);
    twiddles(t256f, 256);
    PF_TRY(upload(p, &p->tw256_64, t256d));
    PF_TRY(upload(p, &p->tw256_32, t256f));
    PF_TRY(plan_workspaces(p));
    return lgf_build(p);
}

// per-plan buffers (not shared between clones)
pf_status plan_workspaces(pf_plan p) {
    const int nx = p->nx, ny = p->ny, P = p->P;
    p->esz = p->prec == PF_FP64 ? 8 : 4;
    p->ldT = (ny + 3) / 4 * 4;
    p->ldK = (P / 2 + 1 + 3) / 4 * 4;
    const size_t spec = (size_t)p->ldK * p->ldT * 2 * p->esz;
    PF_CUDA(p, cudaMalloc(&p->T1, spec));
    PF_CUDA(p, cudaMalloc(&p->T2a, spec));
    PF_CUDA(p, cudaMalloc(&p->T2b, spec));
    PF_CUDA(p, cudaMalloc(&p->w, (size_t)nx * ny * p->esz));
    PF_CUDA(p, cudaMalloc(&p->uv, (size_t)2 * nx * ny * p->esz));
    p->ntx = ceil_div(nx, BIN_TILE);
    p->nty = ceil_div(ny, BIN_TILE);
    p->ntiles = p->ntx * p->nty;
    const int small = ceil_div(nx, BIN_TILE_SMALL) * ceil_div(ny, BIN_TILE_SMALL);
    p->tile_slots = small <= BIN_MAX_TILES ? small : p->ntiles;
    PF_CUDA(p, cudaMalloc(&p->tile_count, (size_t)p->tile_slots * sizeof(unsigned)));
    PF_CUDA(p, cudaMalloc(&p->gmax, (BIN_MAX_BLOCKS + 1) * sizeof(double)));
    PF_CUDA(p, cudaMalloc(&p->tile_start, (size_t)p->tile_slots * sizeof(int)));
    PF_CUDA(p, cudaMalloc(&p->diag, PF_DIAG_DOUBLES * sizeof(double)));
    PF_CUDA(p, cudaMalloc(&p->d_status, sizeof(int)));
    PF_CUDA(p, cudaMalloc(&p->d_oob, sizeof(unsigned long long)));
    // The status words are read before any kernel writes them.  A plain
    // cudaMemset goes to the legacy stream, which a non-blocking plan stream
    // does not wait for; zero on the plan's stream and wait, so that the plan
    // is ready whatever stream it is later used on.
    PF_CUDA(p, cudaMemsetAsync(p->tile_count, 0, (size_t)p->tile_slots * sizeof(unsigned), p->stream));
    PF_CUDA(p, cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
    PF_CUDA(p, cudaMemsetAsync(p->d_oob, 0, sizeof(unsigned long long), p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    return PF_OK;
}

}  // namespace

cudaError_t ensure_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[std::make_pair(dev, kernel)];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

cudaEvent_t tm_event(pf_plan p) {
    if (!p->tm.pool.empty()) {
        cudaEvent_t e = p->tm.pool.back();
        p->tm.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

extern "C" {

pf_status pf_plan_create(const pf_grid_desc* d, void* stream, pf_plan* out) {
    if (!d || !out) return PF_ERR_ARG;
    *out = nullptr;
    if (d->nx < 8 || d->ny < 8 || d->nx > 2048 || d->ny > 2048 || !(d->dx > 0) || !isfinite(d->x0) ||
        !isfinite(d->y0) || (d->precision != PF_FP64 && d->precision != PF_MIXED))
        return PF_ERR_ARG;
    pf_plan p = new (std::nothrow) pf_plan_s();
    if (!p) return PF_ERR_OOM;
    p->nx = d->nx; p->ny = d->ny; p->dx = d->dx; p->x0 = d->x0; p->y0 = d->y0; p->prec = d->precision;
    p->P = next_pow2(2 * d->nx);
    p->Q = next_pow2(2 * d->ny);
    p->stream = (cudaStream_t)stream;
    pf_status s = plan_init(p);
    if (s != PF_OK) {
        free_plan(p);
        delete p;
        return s;
    }
    *out = p;
    return PF_OK;
}

pf_status pf_plan_clone(pf_plan src, int32_t precision, void* stream, pf_plan* out) {
    if (!src || !out || (precision != PF_FP64 && precision != PF_MIXED)) return PF_ERR_ARG;
    *out = nullptr;
    pf_plan p = new (std::nothrow) pf_plan_s();
    if (!p) return PF_ERR_OOM;
    p->nx = src->nx; p->ny = src->ny; p->P = src->P; p->Q = src->Q; p->Hld = src->Hld; p->dx = src->dx; p->x0 = src->x0;
    p->y0 = src->y0; p->prec = precision;
    p->tile = src->tile; p->min_span = src->min_span; p->tile_threads = src->tile_threads; p->fft_impl = src->fft_impl;
    p->stream = (cudaStream_t)stream;
    p->shared = src->shared;
    p->shared->refs++;
    p->G = src->G; p->H64 = src->H64; p->H32 = src->H32; p->Hu64 = src->Hu64; p->Hv64 = src->Hv64;
    p->Hu32 = src->Hu32; p->Hv32 = src->Hv32; p->twP64 = src->twP64; p->twQ64 = src->twQ64; p->twP32 = src->twP32;
    p->twQ32 = src->twQ32; p->tw256_64 = src->tw256_64; p->tw256_32 = src->tw256_32;
    // make sure the source's tables are complete before another stream reads them
    if (cudaStreamSynchronize(src->stream) != cudaSuccess) {
        free_plan(p);
        delete p;
        return PF_ERR_CUDA;
    }
    pf_status s = plan_workspaces(p);
    if (s != PF_OK) {
        free_plan(p);
        delete p;
        return s;
    }
    *out = p;
    return PF_OK;
}

pf_status pf_plan_destroy(pf_plan p) {
    if (!p) return PF_ERR_ARG;
    cudaStreamSynchronize(p->stream);
    free_plan(p);
    delete p;
    return PF_OK;
}

pf_status pf_plan_set_rhs_route(pf_plan p, int32_t route) {
    if (!p || route < PF_RHS_AUTO || route > PF_RHS_SPARSE) return PF_ERR_ARG;
    if (route == PF_RHS_FFT && (p->P < 256 || p->Q < 256)) return PF_ERR_ARG;
    p->rhs_route = route;
    return PF_OK;
}

pf_status pf_plan_fft_size(pf_plan p, int32_t* P, int32_t* Q) {
    if (!p || !P || !Q) return PF_ERR_ARG;
    *P = p->P;
    *Q = p->Q;
    return PF_OK;
}

pf_status pf_lgf_table(pf_plan p, double* host_out) {
    if (!p || !host_out) return PF_ERR_ARG;
    PF_CUDA(p, cudaMemcpyAsync(host_out, p->G, (size_t)(p->nx + 1) * (p->ny + 1) * sizeof(double),
                               cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    return PF_OK;
}

pf_status pf_sync(pf_plan p, int64_t* out_of_domain) {
    if (!p) return PF_ERR_ARG;
    int st = 0;
    unsigned long long oob = 0;
    // read and clear on the plan's stream: work enqueued after this call sees the cleared flags
    PF_CUDA(p, cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(&oob, p->d_oob, sizeof(oob), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
    PF_CUDA(p, cudaMemsetAsync(p->d_oob, 0, sizeof(unsigned long long), p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    if (out_of_domain) *out_of_domain = (int64_t)oob;
    if (st & ST_INTERNAL) return PF_ERR_INTERNAL;
    if (st & ST_TIMEOUT) return PF_ERR_TIMEOUT;
    if (st & ST_SINGULAR) return PF_ERR_SINGULAR;
    if (st & ST_CAPACITY) return PF_ERR_CAPACITY;
    if (st & ST_OUT_OF_DOMAIN) return PF_ERR_OUT_OF_DOMAIN;
    return PF_OK;
}

const char* pf_last_error(pf_plan p) { return p ? p->err : "null plan"; }

pf_status pf_timing_enable(pf_plan p, int32_t on) {
    if (!p) return PF_ERR_ARG;
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    for (cudaEvent_t e : p->tm.ev) p->tm.pool.push_back(e);
    p->tm.ev.clear();
    p->tm.names.clear();
    p->tm.on = on != 0;
    return PF_OK;
}

pf_status pf_timing_report(pf_plan p, char* buf, int64_t buflen) {
    if (!p || !buf || buflen <= 0) return PF_ERR_ARG;
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    std::vector<const char*> names;
    std::vector<double> ms;
    std::vector<int64_t> cnt;
    for (size_t i = 0; i < p->tm.names.size(); ++i) {
        float t = 0.f;
        PF_CUDA(p, cudaEventElapsedTime(&t, p->tm.ev[2 * i], p->tm.ev[2 * i + 1]));
        size_t k = 0;
        while (k < names.size() && strcmp(names[k], p->tm.names[i]) != 0) ++k;
        if (k == names.size()) { names.push_back(p->tm.names[i]); ms.push_back(0.0); cnt.push_back(0); }
        ms[k] += t;
        cnt[k] += 1;
    }
    int64_t off = 0;
    buf[0] = 0;
    for (size_t k = 0; k < names.size() && off < buflen - 1; ++k)
        off += snprintf(buf + off, (size_t)(buflen - off), "%s %lld %.6f\n", names[k], (long long)cnt[k], ms[k]);
    for (cudaEvent_t e : p->tm.ev) p->tm.pool.push_back(e);
    p->tm.ev.clear();
    p->tm.names.clear();
    return PF_OK;
}

pf_status pf_regularize(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, void* w) {
    if (!p || !w || nv < 0 || (nv > 0 && (!X || !Y || !G))) return PF_ERR_ARG;
    return vortex_regularize(p, X, Y, G, nv, w);
}

pf_status pf_poisson_solve(pf_plan p, const void* w, void* psi) {
    if (!p || !w || !psi) return PF_ERR_ARG;
    return conv_solve(p, w, psi, CONV_PSI, 0.0, 0.0);
}

pf_status pf_velocity_solve(pf_plan p, const void* w, double Uinf, double Vinf, void* uv) {
    if (!p || !w || !uv) return PF_ERR_ARG;
    return conv_solve(p, w, uv, CONV_UV, Uinf, Vinf);
}

pf_status pf_interpolate(pf_plan p, const void* uv, const double* Xq, const double* Yq, int64_t nq, void* uq, void* vq) {
    if (!p || !uv || nq < 0 || (nq > 0 && (!Xq || !Yq || !uq || !vq))) return PF_ERR_ARG;
    return vortex_interpolate(p, uv, Xq, Yq, nq, uq, vq);
}

pf_status pf_vic_velocity(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, double Uinf,
                          double Vinf, void* uq, void* vq) {
    if (!p || nv < 0 || (nv > 0 && (!X || !Y || !G || !uq || !vq))) return PF_ERR_ARG;
    PF_TRY(vortex_regularize(p, X, Y, G, nv, p->w, nullptr, uq, vq));
    PF_TRY(conv_solve(p, p->w, p->uv, CONV_UV, Uinf, Vinf));
    return vortex_interpolate_located(p, p->uv, nv, uq, vq);
}

// Device-accessible address of a page-locked host array, or null for pageable
// memory (which has to be staged through a copy).
static const double* pinned_device_ptr(const double* h) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return (const double*)at.devicePointer;
}

// device staging buffers for nv vortices: inputs (3 nv doubles), outputs (2 nv reals)
static pf_status ensure_stage(pf_plan p, int64_t nv) {
    if (nv > p->stage_cap) {
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        if (p->stage) cudaFree(p->stage);
        if (p->stage_out) cudaFree(p->stage_out);
        p->stage = nullptr;
        p->stage_out = nullptr;
        p->stage_cap = 0;
        PF_CUDA(p, cudaMalloc(&p->stage, (size_t)3 * nv * sizeof(double)));
        PF_CUDA(p, cudaMalloc(&p->stage_out, (size_t)2 * nv * p->esz));
        p->stage_cap = nv;
    }
    return PF_OK;
}

pf_status pf_vic_velocity_host(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, double Uinf,
                               double Vinf, void* uq, void* vq) {
    if (!p || nv < 0 || (nv > 0 && (!X || !Y || !G || !uq || !vq))) return PF_ERR_ARG;
    if (nv == 0) return PF_OK;
    // page-locked inputs are read by the locate pass directly over the host link
    // (one transfer, no staging copy); pageable inputs are copied first
    const double* dXp = pinned_device_ptr(X);
    const double* dYp = dXp ? pinned_device_ptr(Y) : nullptr;
    const double* dGp = dYp ? pinned_device_ptr(G) : nullptr;
    PF_TRY(ensure_stage(p, nv));
    char* du = (char*)p->stage_out;
    char* dv = du + (size_t)nv * p->esz;
    if (dGp) {
        PF_TRY(pf_vic_velocity(p, dXp, dYp, dGp, nv, Uinf, Vinf, du, dv));
    } else {
        double* dX = p->stage;
        double* dY = dX + nv;
        double* dG = dY + nv;
        PF_CUDA(p, cudaMemcpyAsync(dX, X, nv * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(dY, Y, nv * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(dG, G, nv * sizeof(double), cudaMemcpyHostToDevice, p->stream));
        PF_TRY(pf_vic_velocity(p, dX, dY, dG, nv, Uinf, Vinf, du, dv));
    }
    PF_CUDA(p, cudaMemcpyAsync(uq, du, nv * p->esz, cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(vq, dv, nv * p->esz, cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    return PF_OK;
}

pf_status pf_vic_velocity_host_async(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv,
                                     double Uinf, double Vinf, void* uq, void* vq) {
    if (!p || nv < 0 || (nv > 0 && (!X || !Y || !G || !uq || !vq))) return PF_ERR_ARG;
    if (nv == 0) return PF_OK;
    PF_TRY(ensure_stage(p, nv));
    double* dX = p->stage;
    double* dY = dX + nv;
    double* dG = dY + nv;
    char* du = (char*)p->stage_out;
    char* dv = du + (size_t)nv * p->esz;
    // copy-engine transfers: the SMs stay free for another plan's kernels
    PF_CUDA(p, cudaMemcpyAsync(dX, X, nv * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(dY, Y, nv * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(dG, G, nv * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    PF_TRY(pf_vic_velocity(p, dX, dY, dG, nv, Uinf, Vinf, du, dv));
    PF_CUDA(p, cudaMemcpyAsync(uq, du, nv * p->esz, cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(vq, dv, nv * p->esz, cudaMemcpyDeviceToHost, p->stream));
    return PF_OK;
}

}  // extern "C"

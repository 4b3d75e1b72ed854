// Launch configuration of a plan and the autotuner that picks it.
//
// The tunables change how the transfer passes (R_v binning and deposit, E_v;
// Sec. 2.1) and the Poisson solve (L^-1, Sec. 2.3) are cut into thread
// blocks: the node tile edge, the fewest vortices per binning block, the
// threads per tile block and the FFT kernel family.  The tuner times one
// body-free velocity evaluation per candidate on synthetic vortices and keeps
// the fastest; results are cached in a text file keyed by device, grid,
// precision and the vortex count's power of two.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

constexpr int SPANS[] = {256, 512, 1024, 2048, 4096};
constexpr int CACHE_VERSION = 1;

bool config_ok(pf_plan p, const pf_launch_config& c) {
    const bool tile_ok = c.tile == BIN_TILE ||
                         (c.tile == BIN_TILE_SMALL &&
                          ceil_div(p->nx, BIN_TILE_SMALL) * ceil_div(p->ny, BIN_TILE_SMALL) <= p->tile_slots);
    const bool span_ok = std::find(std::begin(SPANS), std::end(SPANS), c.min_span) != std::end(SPANS);
    return tile_ok && span_ok && (c.tile_threads == 128 || c.tile_threads == 256) && (c.fft == 0 || c.fft == 1);
}

pf_launch_config config_of(pf_plan p) { return pf_launch_config{p->tile, p->min_span, p->tile_threads, p->fft_impl}; }

void apply(pf_plan p, const pf_launch_config& c) {
    p->tile = c.tile;
    p->min_span = c.min_span;
    p->tile_threads = c.tile_threads;
    p->fft_impl = c.fft;
}

// splitmix64 (Steele, Lea and Flood, 2014): the q-th value of the stream
// `seed` as a uniform double in [0, 1)
__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long q) {
    unsigned long long z = seed + (q + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1p-53;
}

// nv vortices uniform in [x0 + 2 dx, x0 + (nx - 4) dx] x [y0 + 2 dx, y0 + (ny - 4) dx]
// (every stencil inside the grid), strengths uniform in [-1e-3, 1e-3]
__global__ void k_tune_vortices(double* X, double* Y, double* G, int64_t nv, double x0, double y0, double dx, int nx,
                                int ny) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        X[q] = x0 + dx * (2.0 + (nx - 6) * uniform01(1, q));
        Y[q] = y0 + dx * (2.0 + (ny - 6) * uniform01(2, q));
        G[q] = 1e-3 * (2.0 * uniform01(3, q) - 1.0);
    }
}

std::string cache_key(pf_plan p, int64_t nv) {
    int dev = 0;
    cudaDeviceProp prop;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        snprintf(prop.name, sizeof(prop.name), "unknown");
        prop.major = prop.minor = 0;
    }
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    int lg = 0;
    while (lg < 62 && ((int64_t)1 << (lg + 1)) <= nv) ++lg;
    char buf[384];
    snprintf(buf, sizeof(buf), "gridpf-launch-config %d %s sm_%d%d %d %d %s %d", CACHE_VERSION, name.c_str(),
             prop.major, prop.minor, p->nx, p->ny, p->prec == PF_FP64 ? "fp64" : "mixed", lg);
    return std::string(buf);
}

std::mutex g_cache_mu;   // one reader or appender of a cache file per process at a time

// the configuration stored under `key` (the last such line wins)
bool cache_lookup(const char* path, const std::string& key, pf_launch_config& c, double& us) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        if (strncmp(line, key.c_str(), key.size()) != 0 || line[key.size()] != ' ') continue;
        pf_launch_config t;
        double u = 0.0;
        if (sscanf(line + key.size(), " tile=%d min_span=%d tile_threads=%d fft=%d us=%lf", &t.tile, &t.min_span,
                   &t.tile_threads, &t.fft, &u) == 5) {
            c = t;
            us = u;
            found = true;
        }
    }
    fclose(f);
    return found;
}

bool cache_append(const char* path, const std::string& key, const pf_launch_config& c, double us) {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    FILE* f = fopen(path, "a");
    if (!f) return false;
    const int n = fprintf(f, "%s tile=%d min_span=%d tile_threads=%d fft=%d us=%.3f\n", key.c_str(), c.tile,
                          c.min_span, c.tile_threads, c.fft, us);
    return fclose(f) == 0 && n > 0;
}

// the sticky status of the plan, read and cleared (as pf_sync)
pf_status take_status(pf_plan p) {
    int st = 0;
    PF_CUDA(p, cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    PF_CUDA(p, cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
    PF_CUDA(p, cudaMemsetAsync(p->d_oob, 0, sizeof(unsigned long long), p->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    if (st & ST_INTERNAL) return PF_ERR_INTERNAL;
    if (st & ST_CAPACITY) return PF_ERR_CAPACITY;
    if (st & ST_OUT_OF_DOMAIN) return PF_ERR_OUT_OF_DOMAIN;
    return PF_OK;
}

struct TuneBuffers {
    double* X = nullptr;
    double* Y = nullptr;
    double* G = nullptr;
    void* u = nullptr;
    void* v = nullptr;
    void* flush = nullptr;          // written before every timed call: the call starts with a cold L2
    size_t flush_bytes = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    ~TuneBuffers() {
        for (void* q : {(void*)X, (void*)Y, (void*)G, u, v, flush})
            if (q) cudaFree(q);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

pf_status velocity_once(pf_plan p, const TuneBuffers& tb, int64_t nv) {
    PF_TRY(vortex_regularize(p, tb.X, tb.Y, tb.G, nv, p->w));
    PF_TRY(conv_solve(p, p->w, p->uv, CONV_UV, 1.0, 0.0));
    return vortex_interpolate_located(p, p->uv, nv, tb.u, tb.v);
}

// median time (microseconds) of `reps` evaluations in configuration c
pf_status time_config(pf_plan p, const TuneBuffers& tb, int64_t nv, int reps, const pf_launch_config& c, double& us) {
    apply(p, c);
    PF_TRY(velocity_once(p, tb, nv));
    PF_TRY(take_status(p));
    std::vector<double> t;
    for (int r = 0; r < reps; ++r) {
        PF_CUDA(p, cudaMemsetAsync(tb.flush, r & 255, tb.flush_bytes, p->stream));
        PF_CUDA(p, cudaEventRecord(tb.a, p->stream));
        PF_TRY(velocity_once(p, tb, nv));
        PF_CUDA(p, cudaEventRecord(tb.b, p->stream));
        PF_CUDA(p, cudaEventSynchronize(tb.b));
        float ms = 0.f;
        PF_CUDA(p, cudaEventElapsedTime(&ms, tb.a, tb.b));
        t.push_back(1e3 * ms);
    }
    PF_TRY(take_status(p));
    std::sort(t.begin(), t.end());
    us = t[t.size() / 2];
    return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_launch_config_get(pf_plan p, pf_launch_config* out) {
    if (!p || !out) return PF_ERR_ARG;
    *out = config_of(p);
    return PF_OK;
}

pf_status pf_launch_config_set(pf_plan p, const pf_launch_config* c) {
    if (!p || !c || !config_ok(p, *c)) return PF_ERR_ARG;
    apply(p, *c);
    return PF_OK;
}

pf_status pf_autotune(pf_plan p, int64_t nv, const char* cache_path, int32_t reps, pf_launch_config* chosen,
                      double* best_us) {
    if (!p || nv < 1 || reps < 1 || nv > ((int64_t)1 << 29)) return PF_ERR_ARG;
    const std::string key = cache_key(p, nv);
    pf_launch_config best = config_of(p);
    double best_t = 0.0;
    if (cache_path && cache_lookup(cache_path, key, best, best_t) && config_ok(p, best)) {
        apply(p, best);
    } else {
        PF_CUDA(p, cudaStreamSynchronize(p->stream));
        TuneBuffers tb;
        const size_t d = (size_t)nv * sizeof(double);
        PF_CUDA(p, cudaMalloc(&tb.X, d));
        PF_CUDA(p, cudaMalloc(&tb.Y, d));
        PF_CUDA(p, cudaMalloc(&tb.G, d));
        PF_CUDA(p, cudaMalloc(&tb.u, (size_t)nv * p->esz));
        PF_CUDA(p, cudaMalloc(&tb.v, (size_t)nv * p->esz));
        PF_CUDA(p, cudaEventCreate(&tb.a));
        PF_CUDA(p, cudaEventCreate(&tb.b));
        int dev = 0, l2 = 0;
        PF_CUDA(p, cudaGetDevice(&dev));
        PF_CUDA(p, cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
        tb.flush_bytes = 2 * (size_t)std::max(l2, 1 << 20);
        PF_CUDA(p, cudaMalloc(&tb.flush, tb.flush_bytes));
        const int nb = (int)std::min<int64_t>(ceil_div(nv, 256), 152 * 8);
        k_tune_vortices<<<nb, 256, 0, p->stream>>>(tb.X, tb.Y, tb.G, nv, p->x0, p->y0, p->dx, p->nx, p->ny);
        PF_LAUNCH_CHECK(p);
        const pf_launch_config start = config_of(p);
        std::vector<pf_launch_config> cand;
        for (int tile : {BIN_TILE, BIN_TILE_SMALL})
            for (int th : {128, 256})
                for (int fft : {0, 1})
                    for (int span : SPANS) {
                        // the FFT family is irrelevant where the padded torus is too small
                        // for the register-resident passes: keep one of the two
                        if (fft == 1 && (p->P < 256 || p->Q < 256)) continue;
                        const pf_launch_config c{tile, span, th, fft};
                        if (config_ok(p, c)) cand.push_back(c);
                    }
        best_t = INFINITY;
        for (const pf_launch_config& c : cand) {
            double us = 0.0;
            const pf_status st = time_config(p, tb, nv, reps, c, us);
            if (st != PF_OK) {
                apply(p, start);
                return st;
            }
            if (us < best_t) {
                best_t = us;
                best = c;
            }
        }
        apply(p, best);
        if (cache_path && !cache_append(cache_path, key, best, best_t)) {
            snprintf(p->err, sizeof(p->err), "pf_autotune: cannot append to %s", cache_path);
            return PF_ERR_CUDA;
        }
    }
    if (chosen) *chosen = best;
    if (best_us) *best_us = best_t;
    return PF_OK;
}

}  // extern "C"

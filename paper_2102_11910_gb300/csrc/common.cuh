// Shared device/host definitions of the gridpf library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "gridpf.h"

// ------------------------------------------------------------ complex helpers
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using C_t = typename cplx<T>::type;

template <typename C> __host__ __device__ __forceinline__ C cmake(decltype(C::x) r, decltype(C::x) i) { C c; c.x = r; c.y = i; return c; }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
template <typename C> __host__ __device__ __forceinline__ C conjc(C a) { a.y = -a.y; return a; }
// multiply by +i / -i
template <typename C> __host__ __device__ __forceinline__ C mul_i(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
template <typename C> __host__ __device__ __forceinline__ C mul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

// ------------------------------------------------------------ status bits
enum : int {
    ST_OUT_OF_DOMAIN = 1,
    ST_TIMEOUT = 2,
    ST_SINGULAR = 4,
    ST_CAPACITY = 8,
    ST_INTERNAL = 16,           // a binning consistency check failed; the work was skipped
};

// ------------------------------------------------------------ kernel timing
// Optional per-kernel CUDA-event timing on the plan's stream (off by default).
struct KTiming {
    bool on = false;
    std::vector<const char*> names;
    std::vector<cudaEvent_t> ev;      // pairs: ev[2i] before, ev[2i+1] after launch i
    std::vector<cudaEvent_t> pool;
};

// ------------------------------------------------------------ plan
constexpr int BIN_TILE = 32;        // node tile edge used by binning and regularization (default)
constexpr int BIN_TILE_SMALL = 16;  // the other tile edge a plan may be configured with
constexpr int BIN_MAX_TILES = 4096; // tiles one binning pass handles (the reach of its block scan)
constexpr int PF_DIAG_DOUBLES = 4 * 2048 + 3 + 5 * 4096;   // impulse scratch: row partials, results, surface

// Vortex partition of the binning passes: block b owns vortices
// [b * span, min(nv, (b + 1) * span)).  Sets of fewer than BIN_WIDE_MIN
// vortices use at most BIN_MAX_BLOCKS blocks of 256 threads (four per SM, all
// resident at once, equal work per SM; small sets fewer blocks of at least
// min_span vortices); larger sets use BIN_WIDE_BLOCKS blocks of 1024 threads,
// one per SM, whose per-block histogram, scan and offsets row are paid once
// an SM (1e6 vortices: 111.6 -> 109.3 us a step; the same blocks cost the
// small body workloads 3-5 %).
constexpr int BIN_MAX_BLOCKS = 608;
constexpr int BIN_WIDE_BLOCKS = 152;
constexpr int64_t BIN_WIDE_MIN = (int64_t)BIN_WIDE_BLOCKS * 4096;
constexpr int BIN_MIN_SPAN = 1024;   // default fewest vortices per block (a tuned plan may use another)
inline int bin_max_blocks(int64_t nv) { return nv >= BIN_WIDE_MIN ? BIN_WIDE_BLOCKS : BIN_MAX_BLOCKS; }
inline int64_t bin_span(int64_t nv, int min_span = BIN_MIN_SPAN) {
    const int64_t mb = bin_max_blocks(nv);
    const int64_t s = (nv + mb - 1) / mb;
    return s < min_span ? min_span : s;
}
inline int bin_blocks(int64_t nv, int min_span = BIN_MIN_SPAN) {
    return nv > 0 ? (int)((nv + bin_span(nv, min_span) - 1) / bin_span(nv, min_span)) : 0;
}

// Read-only tables of one grid shape, shared by a plan and its clones.
struct PlanTables {
    int refs = 1;
    // double-float copies of H64 and of the FP64 twiddles (H | twP | twQ, one
    // allocation) for the mixed plans' FFT route of the surface right-hand
    // side, built by the first plan that needs them
    std::mutex mu;
    void* df = nullptr;
};

struct pf_plan_s {
    PlanTables* shared = nullptr;  // owner of G, H*, twiddles (reference counted)
    int nx = 0, ny = 0, P = 0, Q = 0, prec = PF_FP64;
    double dx = 0, x0 = 0, y0 = 0;
    cudaStream_t stream = nullptr;
    // LGF and spectrum
    double* G = nullptr;           // (nx+1)*(ny+1), index n*(nx+1)+m
    // spectra on the padded torus, quadrant k in [0, P/2], l in [0, Q/2], index k*Hld+l with
    // Hld = Q/2+1 rounded up to 4 (rows start on 16-byte boundaries; the pad is zero),
    // all divided by P*Q (the inverse FFTs are unnormalised):
    int Hld = 0;
    double* H64 = nullptr;         // psi:  -dx^2 Ghat (real, even in k and l)
    double* Hu64 = nullptr;        // u:    spectrum = i * Hu, Hu = -dx/2 Im(DyG^), odd in l
    double* Hv64 = nullptr;        // v:    spectrum = i * Hv, Hv = +dx/2 Im(DxG^), odd in k
    float* H32 = nullptr;
    float* Hu32 = nullptr;
    float* Hv32 = nullptr;
    double2* twP64 = nullptr;      // exp(-2 pi i m / P), m in [0, P)
    double2* twQ64 = nullptr;
    float2* twP32 = nullptr;
    float2* twQ32 = nullptr;
    double2* tw256_64 = nullptr;   // exp(-2 pi i m / 256), m in [0, 256)
    float2* tw256_32 = nullptr;
    // grid work buffers (element size depends on precision)
    size_t esz = 8;
    int ldT = 0;                   // ny rounded up to 4
    int ldK = 0;                   // P/2 + 1 rounded up to 4
    void* T1 = nullptr;            // ldT*ldK complex: half spectra of the rows (layout set by the FFT kernels)
    void* T2a = nullptr;
    void* T2b = nullptr;
    void* w = nullptr;             // nx*ny real
    void* uv = nullptr;            // 2*nx*ny real
    // launch configuration of the transfer and Poisson passes (pf_launch_config_set,
    // pf_autotune): tile edge, fewest vortices per binning block, threads per
    // tile block, FFT kernels (0 register-resident radix-16, 1 shared-memory)
    int tile = BIN_TILE;
    int min_span = BIN_MIN_SPAN;
    int tile_threads = 256;
    int fft_impl = 0;
    int bin_tile = BIN_TILE;           // tile edge of the last binning (its records serve E_v)
    // binning
    int ntx = 0, nty = 0, ntiles = 0;  // tiles at BIN_TILE
    int tile_slots = 0;                // entries of tile_count and tile_start (tiles at the smallest offered edge)
    unsigned* tile_count = nullptr;    // records per tile (written by every binning pass)
    double* gmax = nullptr;            // largest |Gamma| of the last binning, then per locate block
    int* tile_start = nullptr;
    int* bin_off = nullptr;            // per (block, tile): histogram, then first record slot
    int64_t bin_off_cap = 0;           // entries
    void* pos = nullptr;               // per-vortex cell records of the last located set
    int64_t pos_cap = 0;
    void* recs = nullptr;              // records binned by tile (with each vortex's original index)
    int64_t rec_cap = 0;
    // host-input staging for the *_host entry points
    double* stage = nullptr;
    int64_t stage_cap = 0;
    void* stage_out = nullptr;
    // FP64 surface right-hand side by FFT (sheet solves on large grids): the
    // route (PF_RHS_AUTO / PF_RHS_DIRECT / PF_RHS_FFT) and, for mixed plans,
    // lazily allocated FP64 buffers: w, psi (nx*ny each), two spectra
    int rhs_route = 0;
    void* rhs64 = nullptr;
    // sparse route: the nonzero nodes of w (index, FP64 value; nx*ny each), then
    // the per-chunk counts and the total (allocated by the first sparse solve)
    int* nz_idx = nullptr;
    double* nz_val = nullptr;
    // vortex route: sixteen (node, FP64 value) entries per vortex, then the count
    int* vent_idx = nullptr;
    double* vent_val = nullptr;
    int64_t vent_cap = 0;
    // pressure field: the plan of the cell-centre lattice ((nx-1) x (ny-1),
    // origin shifted by dx/2, same stream and precision) and its FP64 source
    // and kinetic-energy scratch, built by the first pf_pressure_field call
    struct pf_plan_s* centres = nullptr;
    double* pscr = nullptr;
    // diagnostics scratch (per-block partial sums and results)
    double* diag = nullptr;            // PF_DIAG_DOUBLES
    // status
    int* d_status = nullptr;
    unsigned long long* d_oob = nullptr;
    KTiming tm;
    char err[512] = {0};
};

cudaEvent_t tm_event(pf_plan p);   // api.cu

// Launch a kernel; when timing is on, bracket it with events on the plan stream.
#define PF_KERNEL(p, name, ...)                                                   \
    do {                                                                          \
        cudaEvent_t a_ = nullptr;                                                 \
        const bool t_ = (p) != nullptr && (p)->tm.on;                             \
        if (t_) {                                                                 \
            a_ = tm_event(p);                                                     \
            cudaEventRecord(a_, (p)->stream);                                     \
        }                                                                         \
        __VA_ARGS__;                                                              \
        PF_LAUNCH_CHECK(p);                                                       \
        if (t_) {                                                                 \
            cudaEvent_t b_ = tm_event(p);                                         \
            cudaEventRecord(b_, (p)->stream);                                     \
            (p)->tm.names.push_back(name);                                        \
            (p)->tm.ev.push_back(a_);                                             \
            (p)->tm.ev.push_back(b_);                                             \
        }                                                                         \
    } while (0)

#define PF_CUDA(plan, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (plan) snprintf((plan)->err, sizeof((plan)->err), "%s:%d %s: %s", __FILE__,    \
                               __LINE__, #call, cudaGetErrorString(e_));                      \
            return e_ == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;                \
        }                                                                                     \
    } while (0)

#define PF_LAUNCH_CHECK(plan) PF_CUDA(plan, cudaGetLastError())

#define PF_TRY(x)                   \
    do {                            \
        pf_status s_ = (x);         \
        if (s_ != PF_OK) return s_; \
    } while (0)

// A phase of a step (several launches) timed like one kernel: events on the
// plan stream at construction and destruction, reported under `name` next to
// the kernel names when timing is on.
struct PhaseSpan {
    pf_plan p;
    const char* name;
    cudaEvent_t a = nullptr;
    PhaseSpan(pf_plan p_, const char* name_) : p(p_), name(name_) {
        if (p && p->tm.on) {
            a = tm_event(p);
            cudaEventRecord(a, p->stream);
        }
    }
    ~PhaseSpan() {
        if (!a) return;
        cudaEvent_t b = tm_event(p);
        cudaEventRecord(b, p->stream);
        p->tm.names.push_back(name);
        p->tm.ev.push_back(a);
        p->tm.ev.push_back(b);
    }
    PhaseSpan(const PhaseSpan&) = delete;
    PhaseSpan& operator=(const PhaseSpan&) = delete;
};

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (once per
// device, kernel and size; safe to call from several host threads).
cudaError_t ensure_smem(const void* kernel, size_t bytes);   // api.cu
template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
    return ensure_smem(reinterpret_cast<const void*>(kernel), bytes);
}

// Programmatic dependent launch.  A kernel launched by pf_launch is queued
// behind the kernel before it on the stream without a full stream barrier; it
// runs only shared-memory set-up before pdl_wait(), which returns once that
// kernel has completed and its writes are visible.  No kernel here signals
// griddepcontrol.launch_dependents early: a dependent grid whose blocks are
// resident while the kernel before it still runs can read lines that the
// earlier kernel's blocks left in the same SM's L1, and the wait does not
// drop them.  That happened with the in-place histogram-to-offset pass of the
// binning (whole tiles of wrong records on the first call after the inputs
// changed, 2048^2 grids); launching dependents at completion removed it and
// was also faster (the waiting blocks no longer hold SM resources).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pf_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------ internal entry points
// (defined in the .cu files, used by api.cu)
pf_status lgf_build(pf_plan p);                                  // lgf.cu
pf_status conv_solve(pf_plan p, const void* w, void* out, int mode, double Uinf, double Vinf);  // fft.cu
pf_status conv_psi_f64(pf_plan p, const double* w, double* psi, void* T1, void* T2);           // fft.cu
pf_status conv_psi_df(pf_plan p, const float* w, double* psi, void* T1, void* T2, void* wdf,
                      const int* rows);                                                        // fft.cu
pf_status df_tables_ready(pf_plan p);                                                          // fft.cu
enum { CONV_PSI = 0, CONV_UV = 1 };
pf_status vortex_regularize(pf_plan p, const double* X, const double* Y, const double* G, int64_t nv, void* w,
                            const int64_t* dn = nullptr, void* zu = nullptr, void* zv = nullptr);  // transfer.cu
pf_status plan_reserve_vortices(pf_plan p, int64_t nv);   // transfer.cu: vortex buffers for nv ahead of time
pf_status vortex_interpolate(pf_plan p, const void* uv, const double* X, const double* Y, int64_t nq, void* uq, void* vq);
pf_status vortex_interpolate_located(pf_plan p, const void* uv, int64_t nq, void* uq, void* vq);

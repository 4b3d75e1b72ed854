// Vortex state and time stepping (Sec. 2.4.2-2.4.3 of the paper's vortex model).
//
// A step with a body (rigid, given in its own frame, pitching about the
// origin) runs entirely on the device:
//   1. surface points at time t; S factored at that pose (reused while the
//      pose does not change);
//   2. w = R_v Gamma of the current vortices;
//   3. new-vortex positions by the placement rule: the first one from an edge
//      10 dt |U_inf| from the edge along the edge normal facing the free stream,
//      later ones one third of the way from the edge to the last one released;
//   4. two-edge Kutta sheet solve (Eq. twovortex) with Gamma_w = sum Gamma read
//      on the device (bodies without edges: circulation -sum Gamma, no release);
//   5. the new vortices are appended, w is rebuilt and R_s f added (Sec. 2.4.3:
//      psi = -L^-1 (w + G1 d1 + G2 d2 + R_s f));
//   6. node velocity, interpolation to every vortex, advection.
// RK2 is Heun's method: stage 2 at t + dt keeps the new strengths and enforces
// Kelvin's theorem with the circulation-constrained system (Eq. circsystem),
// bound circulation -sum Gamma, without shedding.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <thread>

#include <new>
#include <utility>
#include <vector>

#include "body.cuh"
#include "common.cuh"

// host threads of pf_step_batch: at most BATCH_MAX_THREADS, and no more than
// one per BATCH_MIN_PER_THREAD instances (thread start-up costs tens of us);
// only when the process gave the device BATCH_MIN_CONNECTIONS hardware work
// queues (CUDA_DEVICE_MAX_CONNECTIONS, read when the context is created).
// With the default 8 queues, instances enqueued in parallel bursts share
// queues and wait on one another more than when enqueued in turn (256
// instances of 128^2..512^2 on a GB300: 18.1 ms a batch step from 16 threads
// against 16.1 ms from one; with 32 queues, 13.0 against 14.0 ms).
constexpr int BATCH_MAX_THREADS = 16;
constexpr int BATCH_MIN_PER_THREAD = 8;
constexpr int BATCH_MIN_CONNECTIONS = 32;

static int device_connections() {
    const char* e = getenv("CUDA_DEVICE_MAX_CONNECTIONS");
    return e ? atoi(e) : 8;
}

struct pf_state_s {
    pf_plan plan = nullptr;
    int64_t cap = 0, nv = 0;
    double t = 0.0;
    int64_t last[2 * PF_MAX_BODIES];   // index of the last vortex released at each edge (-1: none yet)
    double *X = nullptr, *Y = nullptr, *G = nullptr;
    double *Xs = nullptr, *Ys = nullptr;            // RK2 predictor positions
    void *u1 = nullptr, *v1 = nullptr, *u2 = nullptr, *v2 = nullptr;   // velocities (plan precision)
    double* f = nullptr;            // sheet strength
    double* red = nullptr;          // reduction scratch: [0] sum Gamma, [1] -sum Gamma, [2..] partials
    double* newpos = nullptr;       // device x[MAX_EDGES], y[MAX_EDGES] of the vortices being released,
                                    // then per body the released circulation and gamma_w
    // device copy of the counts: [0] vortices, [1 + e] the last vortex released at
    // edge e (-1: none yet); kept by every step.  While a step is captured for
    // replay (`capture`), the kernels read the counts from here and the
    // launches are sized by the capacity.
    int64_t* dn = nullptr;
    bool capture = false;
    // Schur factors of the two most recent poses, the current one first: an
    // RK2 step's second stage (t + dt) is the next step's first, so a moving
    // body is factored once per step
    struct Factor {
        pf_schur f = nullptr;
        std::vector<double> alpha;              // pose of each body
        std::vector<int> ns;
        std::vector<const double*> xb;          // bodies the factor belongs to
    } fac[2];
    pf_state_s() {
        for (auto& l : last) l = -1;
    }
};


namespace {

constexpr int RED_BLOCKS = 64;

// sum of Gamma over nv vortices: fixed partition, fixed reduction tree
__global__ void k_sum_partial(const double* __restrict__ G, int64_t nv, const int64_t* __restrict__ dn,
                              double* __restrict__ part) {
    __shared__ double sh[256];
    if (dn) nv = dn[0];
    double s = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x)
        s += G[q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double* __restrict__ part, int n, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        out[0] = s;
        out[1] = -s;
    }
}

constexpr int MAX_EDGES = 2 * PF_MAX_BODIES;

struct EdgeGeo {
    int n;                            // edges releasing a vortex
    double ex[MAX_EDGES], ey[MAX_EDGES];   // geometric edge points
    double nx[MAX_EDGES], ny[MAX_EDGES];   // unit normal facing the free stream
    double first_dist;                // 10 dt |U_inf|
    long long last[MAX_EDGES];
};

// release positions: out[k] = x, out[MAX_EDGES + k] = y of edge k's new vortex
// (the last released vortex from e.last, or from dn[1 + k] when dn is given)
__global__ void k_place(const double* __restrict__ X, const double* __restrict__ Y, EdgeGeo e,
                        const int64_t* __restrict__ dn, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= e.n) return;
    const long long last = dn ? (long long)dn[1 + k] : e.last[k];
    double x, y;
    if (last < 0) {
        x = e.ex[k] + e.first_dist * e.nx[k];
        y = e.ey[k] + e.first_dist * e.ny[k];
    } else {
        x = e.ex[k] + (X[last] - e.ex[k]) / 3.0;
        y = e.ey[k] + (Y[last] - e.ey[k]) / 3.0;
    }
    out[k] = x;
    out[MAX_EDGES + k] = y;
}

// append the n released vortices at index nv (dn[0] when use_dn): positions
// from pos (as k_place), strengths gam[0..n); the device counts follow.  One
// warp.  A release past the capacity is dropped and flagged (the host checks
// the capacity first, so only a corrupted count gets here).
__global__ void k_append(double* __restrict__ X, double* __restrict__ Y, double* __restrict__ G, int64_t nv,
                         const double* __restrict__ pos, const double* __restrict__ gam, int n,
                         int64_t* __restrict__ dn, int use_dn, int64_t cap, int* __restrict__ status) {
    const int k = threadIdx.x;
    if (use_dn) nv = dn[0];
    const bool fits = nv >= 0 && nv + n <= cap;
    if (k < n && fits) {
        X[nv + k] = pos[k];
        Y[nv + k] = pos[MAX_EDGES + k];
        G[nv + k] = gam[k];
        dn[1 + k] = nv + k;
    }
    __syncwarp();                       // every lane has read dn[0]
    if (k == 0) {
        if (fits) dn[0] = nv + n;
        else atomicOr(status, ST_CAPACITY);
    }
}

// the device counts of a loaded state: nv vortices, nothing released yet
__global__ void k_set_counts(int64_t* __restrict__ dn, int64_t nv) {
    const int k = threadIdx.x;
    if (k == 0) dn[0] = nv;
    if (k < MAX_EDGES) dn[1 + k] = -1;
}

// several bodies: gamma_w of body b >= 1 is the circulation it released, body 0
// takes the rest of the flow's (red[0] = sum Gamma)
__global__ void k_gamma_w(const double* __restrict__ red, const double* __restrict__ rel, int nb,
                          double* __restrict__ gw) {
    if (threadIdx.x != 0) return;
    double other = 0.0;
    for (int b = 1; b < nb; ++b) {
        other += rel[b];
        gw[b] = rel[b];
    }
    gw[0] = red[0] - other;
}

// add each body's new strengths (gam, edges in body order) to its released circulation
__global__ void k_released(const double* __restrict__ gam, pf_multibody mb, double* __restrict__ rel) {
    if (threadIdx.x != 0) return;
    int e = 0;
    for (int b = 0; b < mb.n_bodies; ++b)
        for (int j = 0; j < mb.n_edges[b]; ++j) rel[b] += gam[e++];
}

template <typename T>
__global__ void k_euler(double* __restrict__ X, double* __restrict__ Y, const T* __restrict__ u, const T* __restrict__ v,
                        int64_t nv, const int64_t* __restrict__ dn, double dt) {
    if (dn) nv = dn[0];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        X[q] += dt * (double)u[q];
        Y[q] += dt * (double)v[q];
    }
}

template <typename T>
__global__ void k_predict(const double* __restrict__ X, const double* __restrict__ Y, const T* __restrict__ u,
                          const T* __restrict__ v, int64_t nv, const int64_t* __restrict__ dn, double dt,
                          double* __restrict__ Xs, double* __restrict__ Ys) {
    if (dn) nv = dn[0];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        Xs[q] = X[q] + dt * (double)u[q];
        Ys[q] = Y[q] + dt * (double)v[q];
    }
}

template <typename T>
__global__ void k_heun(double* __restrict__ X, double* __restrict__ Y, const T* __restrict__ u1, const T* __restrict__ v1,
                       const T* __restrict__ u2, const T* __restrict__ v2, int64_t nv, const int64_t* __restrict__ dn,
                       double dt) {
    if (dn) nv = dn[0];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        X[q] += 0.5 * dt * ((double)u1[q] + (double)u2[q]);
        Y[q] += 0.5 * dt * ((double)v1[q] + (double)v2[q]);
    }
}

void free_state(pf_state s) {
    void* ptrs[] = {s->X, s->Y, s->G, s->Xs, s->Ys, s->u1, s->v1, s->u2, s->v2, s->f, s->red, s->newpos, s->dn};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (auto& c : s->fac)
        if (c.f) schur_free(c.f);
}

int nblocks(int64_t n) { return (int)std::min<int64_t>(ceil_div(n > 0 ? n : 1, 256), 152 * 8); }

// body at time t: world points (body frame turned by -alpha), rotation rate
struct Pose {
    std::vector<double> x, y;
    double alpha, Omega;
};

Pose body_pose(const pf_body_kinematics& k, double t) {
    Pose P;
    P.alpha = k.alpha0 + k.amp * sin(k.omega * t);
    P.Omega = -k.amp * k.omega * cos(k.omega * t);     // the body turns by -alpha
    const double ca = cos(P.alpha), sa = sin(P.alpha);
    P.x.resize(k.ns);
    P.y.resize(k.ns);
    for (int i = 0; i < k.ns; ++i) {
        P.x[i] = ca * k.xb[i] + sa * k.yb[i];
        P.y[i] = -sa * k.xb[i] + ca * k.yb[i];
    }
    return P;
}

// the concatenated surface of one or several bodies at their poses
struct Surface {
    std::vector<double> x, y, ds;
    std::vector<double> alpha;
    std::vector<int> ns;
    std::vector<const double*> xb;
};

Surface surface_of(const pf_body_kinematics* k, int nb, const std::vector<Pose>& P) {
    Surface S;
    for (int b = 0; b < nb; ++b) {
        S.x.insert(S.x.end(), P[b].x.begin(), P[b].x.end());
        S.y.insert(S.y.end(), P[b].y.begin(), P[b].y.end());
        S.ds.insert(S.ds.end(), k[b].ds, k[b].ds + k[b].ns);
        S.alpha.push_back(P[b].alpha);
        S.ns.push_back(k[b].ns);
        S.xb.push_back(k[b].xb);
    }
    return S;
}

// factor S at the pose, asynchronously (errors surface at pf_sync); the
// factors of the two latest poses are kept while the bodies are unchanged
pf_status ensure_schur(pf_plan p, pf_state s, const Surface& B) {
    auto fits = [&](const pf_state_s::Factor& c) { return c.f && c.alpha == B.alpha && c.ns == B.ns && c.xb == B.xb; };
    if (fits(s->fac[0])) return PF_OK;
    std::swap(s->fac[0], s->fac[1]);
    if (fits(s->fac[0])) return PF_OK;
    // refactor the older entry, now in front, at this pose
    pf_state_s::Factor& c = s->fac[0];
    const int ns = (int)B.x.size();
    if (!c.f || c.f->ns != ns) {
        if (c.f) {
            PF_CUDA(p, cudaStreamSynchronize(p->stream));
            schur_free(c.f);
            c.f = nullptr;
        }
        PF_TRY(schur_create(p, ns, &c.f));
    }
    c.ns.clear();                 // invalid until factored
    c.xb.clear();
    const size_t v = (size_t)ns * sizeof(double);
    // pageable host sources: the copies complete before the calls return
    PF_CUDA(p, cudaMemcpyAsync(c.f->x, B.x.data(), v, cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(c.f->y, B.y.data(), v, cudaMemcpyHostToDevice, p->stream));
    PF_CUDA(p, cudaMemcpyAsync(c.f->ds, B.ds.data(), v, cudaMemcpyHostToDevice, p->stream));
    PF_TRY(schur_factor_device(p, c.f));
    c.alpha = B.alpha;
    c.ns = B.ns;
    c.xb = B.xb;
    return PF_OK;
}

// geometric edge, unit normal facing the stream, and history of edge point kp
// of a body whose world points are (x, y), n of them
void edge_geometry(const std::vector<double>& x, const std::vector<double>& y, int off, int n, int kp, double Uinf,
                   double Vinf, EdgeGeo& e, int j) {
    // the neighbour along the surface away from the edge, on the same body
    const int nb = kp == 0 ? 1 : (kp == n - 1 ? n - 2 : kp + 1);
    const double tx = x[off + kp] - x[off + nb], ty = y[off + kp] - y[off + nb];
    e.ex[j] = x[off + kp] + 0.5 * tx;
    e.ey[j] = y[off + kp] + 0.5 * ty;
    double nxv = -ty, nyv = tx;
    const double nn = hypot(nxv, nyv);
    nxv /= nn;
    nyv /= nn;
    if (nxv * Uinf + nyv * Vinf < 0.0) { nxv = -nxv; nyv = -nyv; }
    e.nx[j] = nxv;
    e.ny[j] = nyv;
}

pf_status sum_gamma(pf_plan p, pf_state s, int64_t n, const int64_t* dn) {
    k_sum_partial<<<RED_BLOCKS, 256, 0, p->stream>>>(s->G, n, dn, s->red + 2);
    k_sum_final<<<1, 32, 0, p->stream>>>(s->red + 2, RED_BLOCKS, s->red);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

// Launch size and device count of a stage: the host count, or while the step
// is captured for replay, the capacity with the count read from s->dn.  (The
// sheet's right-hand-side route is chosen for the capacity in both cases, 16
// nodes of w per vortex, so a captured step computes exactly what pf_step
// does.)
struct Count {
    int64_t n;
    const int64_t* dn;
};
Count count_of(pf_state s) { return s->capture ? Count{s->cap, s->dn} : Count{s->nv, nullptr}; }

// velocity (plan precision) at the n vortices (X, Y, G) of the current arrays,
// optionally with a body sheet f added to the source
pf_status velocities(pf_plan p, pf_state s, const double* X, const double* Y, Count c, pf_schur sch,
                     const double* f, double Uinf, double Vinf, void* u, void* v) {
    PF_TRY(vortex_regularize(p, X, Y, s->G, c.n, p->w, c.dn, u, v));
    if (sch) PF_TRY(sheet_deposit(p, sch, f, p->w));
    PF_TRY(conv_solve(p, p->w, p->uv, CONV_UV, Uinf, Vinf));
    return vortex_interpolate_located(p, p->uv, c.n, u, v);
}

enum { ADV_EULER = 0, ADV_PREDICT = 1, ADV_HEUN = 2 };

template <typename T>
void advance_t(pf_plan p, pf_state s, int kind, Count c, double dt) {
    const int nb = nblocks(c.n);
    const T *u1 = (const T*)s->u1, *v1 = (const T*)s->v1;
    if (kind == ADV_EULER)
        k_euler<T><<<nb, 256, 0, p->stream>>>(s->X, s->Y, u1, v1, c.n, c.dn, dt);
    else if (kind == ADV_PREDICT)
        k_predict<T><<<nb, 256, 0, p->stream>>>(s->X, s->Y, u1, v1, c.n, c.dn, dt, s->Xs, s->Ys);
    else
        k_heun<T><<<nb, 256, 0, p->stream>>>(s->X, s->Y, u1, v1, (const T*)s->u2, (const T*)s->v2, c.n, c.dn, dt);
}

// X += dt u1 (Euler), (Xs, Ys) = X + dt u1 (predictor), X += dt (u1 + u2) / 2 (Heun)
pf_status advance(pf_plan p, pf_state s, int kind, Count c, double dt) {
    PhaseSpan ph(p, "phase_update");
    if (p->prec == PF_FP64) advance_t<double>(p, s, kind, c, dt);
    else advance_t<float>(p, s, kind, c, dt);
    PF_LAUNCH_CHECK(p);
    return PF_OK;
}

// one stage with the body: shed (two-edge Kutta) or Kelvin-constrained
pf_status body_stage(pf_plan p, pf_state s, const pf_body_kinematics& k, double t, double dt, const double* X,
                     const double* Y, bool shed, void* u, void* v) {
    const std::vector<Pose> P{body_pose(k, t)};
    {
        PhaseSpan ph(p, "phase_schur_factor");
        PF_TRY(ensure_schur(p, s, surface_of(&k, 1, P)));
    }
    pf_schur sch = s->fac[0].f;
    const pf_motion m{0.0, 0.0, P[0].Omega, k.Uinf, k.Vinf};
    Count c = count_of(s);
    {
        PhaseSpan ph(p, "phase_regularize");
        PF_TRY(vortex_regularize(p, X, Y, s->G, c.n, p->w, c.dn));
        PF_TRY(sum_gamma(p, s, c.n, c.dn));
    }
    {
        PhaseSpan ph(p, "phase_sheet_solve");
        if (shed) {
            EdgeGeo e;
            e.n = 2;
            const int kk[2] = {k.edge[0], k.edge[1]};
            for (int j = 0; j < 2; ++j) {
                edge_geometry(P[0].x, P[0].y, 0, k.ns, kk[j], k.Uinf, k.Vinf, e, j);
                e.last[j] = s->last[j];
            }
            e.first_dist = 10.0 * dt * hypot(k.Uinf, k.Vinf);
            k_place<<<1, 32, 0, p->stream>>>(X, Y, e, c.dn, s->newpos);
            PF_LAUNCH_CHECK(p);
            EdgeBounds eb;
            eb.on = k.edge_bounded ? 1 : 0;
            for (int j = 0; j < 2; ++j) {
                eb.lo[j] = k.edge_bounds[2 * j];
                eb.hi[j] = k.edge_bounds[2 * j + 1];
            }
            PF_TRY(sheet_solve_device(p, sch, p->w, m, PF_SHEET_KUTTA_SHED, 0.0, s->red, 2, kk, s->newpos,
                                      s->newpos + MAX_EDGES, s->f, eb, 16 * s->cap));
            // release: the new vortices join the arrays X, Y (the caller's position
            // arrays) and G
            k_append<<<1, 32, 0, p->stream>>>(const_cast<double*>(X), const_cast<double*>(Y), s->G, c.n, s->newpos,
                                              sch->scal + 1, 2, s->dn, c.dn != nullptr, s->cap, p->d_status);
            PF_LAUNCH_CHECK(p);
            if (!c.dn) c.n += 2;
        } else {
            PF_TRY(sheet_solve_device(p, sch, p->w, m, PF_SHEET_CIRCULATION, 0.0, s->red + 1, 0, nullptr, nullptr,
                                      nullptr, s->f, EdgeBounds(), 16 * s->cap));
        }
    }
    PhaseSpan ph(p, "phase_velocity");
    return velocities(p, s, X, Y, c, sch, s->f, k.Uinf, k.Vinf, u, v);
}

// one stage with several bodies (Sec. 2.7): each edge releases a vortex under
// the Kutta condition (shed), Kelvin per body; without shedding every body is
// circulation-constrained
pf_status bodies_stage(pf_plan p, pf_state s, const pf_body_kinematics* k, int nb, double t, double dt,
                       const double* X, const double* Y, bool shed, void* u, void* v) {
    std::vector<Pose> P;
    for (int b = 0; b < nb; ++b) P.push_back(body_pose(k[b], t));
    PF_TRY(ensure_schur(p, s, surface_of(k, nb, P)));
    pf_schur sch = s->fac[0].f;
    pf_multibody mb{};
    mb.n_bodies = nb;
    int ne = 0;
    EdgeGeo e;
    for (int b = 0; b < nb; ++b) {
        mb.start[b + 1] = mb.start[b] + k[b].ns;
        mb.n_edges[b] = shed ? k[b].n_edges : 0;
        for (int j = 0; j < mb.n_edges[b]; ++j) {
            mb.edge[b][j] = mb.start[b] + k[b].edge[j];
            edge_geometry(P[b].x, P[b].y, 0, k[b].ns, k[b].edge[j], k[0].Uinf, k[0].Vinf, e, ne);
            e.last[ne] = s->last[ne];
            ++ne;
        }
        mb.motion[b] = pf_motion{0.0, 0.0, P[b].Omega, k[0].Uinf, k[0].Vinf};
    }
    e.n = ne;
    e.first_dist = 10.0 * dt * hypot(k[0].Uinf, k[0].Vinf);
    double* rel = s->newpos + 2 * MAX_EDGES;
    double* gw = rel + PF_MAX_BODIES;
    Count c = count_of(s);
    PF_TRY(vortex_regularize(p, X, Y, s->G, c.n, p->w, c.dn));
    PF_TRY(sum_gamma(p, s, c.n, c.dn));
    k_gamma_w<<<1, 32, 0, p->stream>>>(s->red, rel, nb, gw);
    if (ne > 0) k_place<<<1, 32, 0, p->stream>>>(X, Y, e, c.dn, s->newpos);
    PF_LAUNCH_CHECK(p);
    double* out = nullptr;
    PF_TRY(sheet_solve_multi_device(p, sch, p->w, mb, ne, s->newpos, s->newpos + MAX_EDGES, s->f, gw, &out,
                                    16 * s->cap));
    if (ne > 0) {
        k_append<<<1, 32, 0, p->stream>>>(const_cast<double*>(X), const_cast<double*>(Y), s->G, c.n, s->newpos,
                                          out + nb, ne, s->dn, c.dn != nullptr, s->cap, p->d_status);
        k_released<<<1, 32, 0, p->stream>>>(out + nb, mb, rel);
        PF_LAUNCH_CHECK(p);
        if (!c.dn) c.n += ne;
    }
    return velocities(p, s, X, Y, c, sch, s->f, k[0].Uinf, k[0].Vinf, u, v);
}

}  // namespace

// enqueue a state load from pinned host arrays on the plan's stream (no sync)
pf_status state_load_async(pf_state s, const double* X, const double* Y, const double* G, int64_t nv, double t) {
    if (nv > s->cap) return PF_ERR_CAPACITY;
    pf_plan p = s->plan;
    const size_t b = (size_t)nv * sizeof(double);
    if (nv > 0) {
        PF_CUDA(p, cudaMemcpyAsync(s->X, X, b, cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(s->Y, Y, b, cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(s->G, G, b, cudaMemcpyHostToDevice, p->stream));
    }
    s->nv = nv;
    s->t = t;
    for (auto& l : s->last) l = -1;
    k_set_counts<<<1, 32, 0, p->stream>>>(s->dn, nv);
    PF_LAUNCH_CHECK(p);
    PF_CUDA(s->plan, cudaMemsetAsync(s->newpos + 2 * MAX_EDGES, 0, PF_MAX_BODIES * sizeof(double), s->plan->stream));
    s->fac[0].xb.clear();
    s->fac[1].xb.clear();
    return PF_OK;
}

// enqueue a copy of the current vortices to pinned host arrays (no sync)
pf_status state_store_async(pf_state s, double* X, double* Y, double* G, int64_t* nv) {
    pf_plan p = s->plan;
    const size_t b = (size_t)s->nv * sizeof(double);
    if (s->nv > 0) {
        PF_CUDA(p, cudaMemcpyAsync(X, s->X, b, cudaMemcpyDeviceToHost, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(Y, s->Y, b, cudaMemcpyDeviceToHost, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(G, s->G, b, cudaMemcpyDeviceToHost, p->stream));
    }
    *nv = s->nv;
    return PF_OK;
}

int64_t state_capacity(pf_state s) { return s->cap; }

// A captured batch step (pf_batch_create): the graph and its executable, the
// batch's stream, and what each instance's host counts need after a launch.
struct pf_batch_s {
    std::vector<pf_plan> plans;
    std::vector<pf_state> states;
    std::vector<pf_body_kinematics> bodies;
    std::vector<double> dt;
    std::vector<int> released;          // vortices each instance releases per step
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    std::vector<cudaEvent_t> order;     // one per plan: the plan's earlier work before a launch
};

namespace {

void free_batch(pf_batch b) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->order)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->stream) cudaStreamDestroy(b->stream);
}

bool fixed_in_time(const pf_body_kinematics& k) { return k.ns == 0 || k.amp == 0.0 || k.omega == 0.0; }

// what a captured step of the full capacity needs ready: the vortex buffers,
// the factor at the (fixed) pose and the buffers of the sheet's route
pf_status prepare_capture(pf_plan p, pf_state s, const pf_body_kinematics& k) {
    PF_TRY(plan_reserve_vortices(p, s->cap));
    if (k.ns > 0) {
        PF_TRY(ensure_schur(p, s, surface_of(&k, 1, std::vector<Pose>{body_pose(k, s->t)})));
        PF_TRY(sheet_solve_reserve(p, s->fac[0].f, 16 * s->cap));
    }
    return PF_OK;
}

// one pf_step with the counts read on the device; the host counts are restored
pf_status step_captured(pf_plan p, pf_state s, const pf_body_kinematics& k, double dt, int scheme) {
    const int64_t nv = s->nv;
    const double t = s->t;
    int64_t last[2 * PF_MAX_BODIES];
    std::copy(std::begin(s->last), std::end(s->last), last);
    s->capture = true;
    const pf_status st = pf_step(p, s, &k, dt, scheme);
    s->capture = false;
    s->nv = nv;
    s->t = t;
    std::copy(std::begin(last), std::end(last), s->last);
    return st;
}

// capture one step of every instance into b->graph (the host counts are
// restored afterwards: the capture runs nothing)
pf_status capture_batch(pf_batch b, int scheme) {
    pf_plan p0 = b->plans[0];
    PF_CUDA(p0, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
    pf_status st = PF_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (size_t i = 0; i < b->plans.size() && st == PF_OK && e == cudaSuccess; ++i) {
        pf_plan p = b->plans[i];
        pf_state s = b->states[i];
        e = cudaStreamWaitEvent(p->stream, b->fork, 0);
        if (e != cudaSuccess) break;
        st = step_captured(p, s, b->bodies[i], b->dt[i], scheme);
        if (st != PF_OK && p != p0) snprintf(p0->err, sizeof(p0->err), "instance %zu: %s", i, p->err);
        // join the plan's stream back (also after an error, so that the capture ends cleanly)
        e = cudaEventRecord(b->join, p->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
    }
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &b->graph);
    if (st != PF_OK) return st;
    PF_CUDA(p0, e);
    PF_CUDA(p0, ee);
    PF_CUDA(p0, cudaGraphInstantiate(&b->exec, b->graph, 0));
    PF_CUDA(p0, cudaGraphUpload(b->exec, b->stream));
    return PF_OK;
}

}  // namespace

pf_status step_graph_create(pf_plan p, pf_state s, const pf_body_kinematics& k, double dt, int scheme,
                            cudaGraphExec_t* out, int* released) {
    *out = nullptr;
    if (!fixed_in_time(k) || !p->stream || p->tm.on) return PF_ERR_ARG;
    PF_TRY(prepare_capture(p, s, k));
    cudaGraph_t g = nullptr;
    PF_CUDA(p, cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeRelaxed));
    const pf_status st = step_captured(p, s, k, dt, scheme);
    const cudaError_t e = cudaStreamEndCapture(p->stream, &g);
    if (st != PF_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st != PF_OK) return st;
        PF_CUDA(p, e);
    }
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    PF_CUDA(p, ei);
    *released = k.ns > 0 && k.n_edges == 2 ? 2 : 0;
    return PF_OK;
}

void step_graph_advance(pf_state s, int released, double dt) {
    const int64_t n0 = s->nv;
    s->nv += released;
    for (int e = 0; e < released; ++e) s->last[e] = n0 + e;
    s->t += dt;
}

extern "C" {

pf_status pf_state_create(pf_plan p, int64_t cap, pf_state* out) {
    if (!p || !out || cap < 0) return PF_ERR_ARG;
    *out = nullptr;
    pf_state s = new (std::nothrow) pf_state_s();
    if (!s) return PF_ERR_OOM;
    s->plan = p;
    s->cap = cap;
    const size_t d = (size_t)(cap > 0 ? cap : 1) * sizeof(double), e = (size_t)(cap > 0 ? cap : 1) * p->esz;
    cudaError_t err = cudaSuccess;
    for (double** q : {&s->X, &s->Y, &s->G, &s->Xs, &s->Ys})
        if (err == cudaSuccess) err = cudaMalloc(q, d);
    for (void** q : {&s->u1, &s->v1, &s->u2, &s->v2})
        if (err == cudaSuccess) err = cudaMalloc(q, e);
    if (err == cudaSuccess) err = cudaMalloc(&s->f, PF_MAX_SURFACE_POINTS * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&s->red, (2 + RED_BLOCKS) * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&s->newpos, (2 * MAX_EDGES + 2 * PF_MAX_BODIES) * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&s->dn, (1 + MAX_EDGES) * sizeof(int64_t));
    if (err == cudaSuccess)
        err = cudaMemsetAsync(s->newpos, 0, (2 * MAX_EDGES + 2 * PF_MAX_BODIES) * sizeof(double), p->stream);
    if (err == cudaSuccess) {
        k_set_counts<<<1, 32, 0, p->stream>>>(s->dn, 0);
        err = cudaGetLastError();
    }
    if (err != cudaSuccess) {
        snprintf(p->err, sizeof(p->err), "pf_state_create: %s", cudaGetErrorString(err));
        free_state(s);
        delete s;
        return err == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
    }
    *out = s;
    return PF_OK;
}

pf_status pf_state_destroy(pf_state s) {
    if (!s) return PF_ERR_ARG;
    cudaStreamSynchronize(s->plan->stream);
    free_state(s);
    delete s;
    return PF_OK;
}

pf_status pf_state_set(pf_state s, const double* X, const double* Y, const double* G, int64_t nv, double t) {
    if (!s || nv < 0 || (nv > 0 && (!X || !Y || !G))) return PF_ERR_ARG;
    if (nv > s->cap) return PF_ERR_CAPACITY;
    pf_plan p = s->plan;
    const size_t b = (size_t)nv * sizeof(double);
    if (nv > 0) {
        PF_CUDA(p, cudaMemcpyAsync(s->X, X, b, cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(s->Y, Y, b, cudaMemcpyHostToDevice, p->stream));
        PF_CUDA(p, cudaMemcpyAsync(s->G, G, b, cudaMemcpyHostToDevice, p->stream));
    }
    s->nv = nv;
    s->t = t;
    for (auto& l : s->last) l = -1;
    k_set_counts<<<1, 32, 0, p->stream>>>(s->dn, nv);
    PF_LAUNCH_CHECK(p);
    PF_CUDA(s->plan, cudaMemsetAsync(s->newpos + 2 * MAX_EDGES, 0, PF_MAX_BODIES * sizeof(double), s->plan->stream));
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    s->fac[0].xb.clear();
    s->fac[1].xb.clear();   // a new history may come with a new body
    return PF_OK;
}

pf_status pf_state_get(pf_state s, double* X, double* Y, double* G, int64_t* nv, double* t) {
    if (!s) return PF_ERR_ARG;
    pf_plan p = s->plan;
    const size_t b = (size_t)s->nv * sizeof(double);
    if (s->nv > 0) {
        if (X) PF_CUDA(p, cudaMemcpyAsync(X, s->X, b, cudaMemcpyDeviceToHost, p->stream));
        if (Y) PF_CUDA(p, cudaMemcpyAsync(Y, s->Y, b, cudaMemcpyDeviceToHost, p->stream));
        if (G) PF_CUDA(p, cudaMemcpyAsync(G, s->G, b, cudaMemcpyDeviceToHost, p->stream));
    }
    PF_CUDA(p, cudaStreamSynchronize(p->stream));
    if (nv) *nv = s->nv;
    if (t) *t = s->t;
    return PF_OK;
}

pf_status pf_step(pf_plan p, pf_state s, const pf_body_kinematics* k, double dt, int32_t scheme) {
    if (!p || !s || !k || !(dt > 0) || (scheme != 0 && scheme != 1) || k->ns < 0 || k->ns > PF_MAX_SURFACE_POINTS)
        return PF_ERR_ARG;
    const bool body = k->ns > 0;
    if (body && (k->ns < 4 || !k->xb || !k->yb || !k->ds || (k->n_edges != 0 && k->n_edges != 2))) return PF_ERR_ARG;
    if (body && k->n_edges == 2)
        for (int e = 0; e < 2; ++e)
            if (k->edge[e] < 0 || k->edge[e] >= k->ns ||
                (k->edge_bounded && !(k->edge_bounds[2 * e] <= k->edge_bounds[2 * e + 1])))
                return PF_ERR_ARG;
    const bool release = body && k->n_edges == 2;
    if (release && s->nv + 2 > s->cap) return PF_ERR_CAPACITY;
    const int64_t n0 = s->nv;
    if (!body) {
        const Count c = count_of(s);
        PF_TRY(velocities(p, s, s->X, s->Y, c, nullptr, nullptr, k->Uinf, k->Vinf, s->u1, s->v1));
        if (scheme == 0) {
            PF_TRY(advance(p, s, ADV_EULER, c, dt));
        } else {
            PF_TRY(advance(p, s, ADV_PREDICT, c, dt));
            PF_TRY(velocities(p, s, s->Xs, s->Ys, c, nullptr, nullptr, k->Uinf, k->Vinf, s->u2, s->v2));
            PF_TRY(advance(p, s, ADV_HEUN, c, dt));
        }
        s->t += dt;
        return PF_OK;
    }
    // stage 1 at t: release two vortices (appended to X, Y, G) and get u1 at all n0 + 2
    PF_TRY(body_stage(p, s, *k, s->t, dt, s->X, s->Y, release, s->u1, s->v1));
    s->nv = n0 + (release ? 2 : 0);
    if (scheme == 0) {
        PF_TRY(advance(p, s, ADV_EULER, count_of(s), dt));
    } else {
        PF_TRY(advance(p, s, ADV_PREDICT, count_of(s), dt));
        PF_TRY(body_stage(p, s, *k, s->t + dt, dt, s->Xs, s->Ys, false, s->u2, s->v2));
        PF_TRY(advance(p, s, ADV_HEUN, count_of(s), dt));
    }
    if (release) {
        s->last[0] = n0;
        s->last[1] = n0 + 1;
    }
    s->t += dt;
    return PF_OK;
}

pf_status pf_step_multi(pf_plan p, pf_state s, int32_t n_bodies, const pf_body_kinematics* bodies, double dt,
                        int32_t scheme) {
    if (!p || !s || !bodies || n_bodies < 1 || n_bodies > PF_MAX_BODIES || !(dt > 0) || (scheme != 0 && scheme != 1))
        return PF_ERR_ARG;
    int ns = 0, ne = 0;
    for (int b = 0; b < n_bodies; ++b) {
        const pf_body_kinematics& k = bodies[b];
        if (k.ns < 4 || !k.xb || !k.yb || !k.ds || k.n_edges < 0 || k.n_edges > 2 || k.edge_bounded) return PF_ERR_ARG;
        for (int j = 0; j < k.n_edges; ++j)
            if (k.edge[j] < 0 || k.edge[j] >= k.ns) return PF_ERR_ARG;
        ns += k.ns;
        ne += k.n_edges;
    }
    if (ns > PF_MAX_SURFACE_POINTS) return PF_ERR_ARG;
    if (s->nv + ne > s->cap) return PF_ERR_CAPACITY;
    const int64_t n0 = s->nv;
    // stage 1 at t: one new vortex per edge (appended to X, Y, G), u1 at all n0 + ne
    PF_TRY(bodies_stage(p, s, bodies, n_bodies, s->t, dt, s->X, s->Y, ne > 0, s->u1, s->v1));
    s->nv = n0 + ne;
    if (scheme == 0) {
        PF_TRY(advance(p, s, ADV_EULER, count_of(s), dt));
    } else {
        PF_TRY(advance(p, s, ADV_PREDICT, count_of(s), dt));
        // stage 2 at t + dt: strengths kept, every body circulation-constrained
        PF_TRY(bodies_stage(p, s, bodies, n_bodies, s->t + dt, dt, s->Xs, s->Ys, false, s->u2, s->v2));
        PF_TRY(advance(p, s, ADV_HEUN, count_of(s), dt));
    }
    for (int e = 0; e < ne; ++e) s->last[e] = n0 + e;
    s->t += dt;
    return PF_OK;
}

pf_status pf_step_batch(int32_t n, pf_plan* plans, pf_state* states, const pf_body_kinematics* bodies,
                        const double* dt, int32_t scheme) {
    if (n < 0 || (n > 0 && (!plans || !states || !bodies || !dt))) return PF_ERR_ARG;
    // Every instance is enqueued on its own plan's stream, and distinct streams
    // run concurrently on the device.  Enqueueing one step costs tens of
    // microseconds of host time (launches, kinematics, shedding bookkeeping),
    // so, given enough hardware queues, a large batch is spread over host
    // threads that take the instances in turn from a shared counter; each
    // thread works on the caller's device.
    const unsigned hw = std::thread::hardware_concurrency();
    int nthreads = (int)std::min<int64_t>(std::min<int64_t>(hw ? hw : 1, BATCH_MAX_THREADS),
                                           ((int64_t)n + BATCH_MIN_PER_THREAD - 1) / BATCH_MIN_PER_THREAD);
    if (device_connections() < BATCH_MIN_CONNECTIONS) nthreads = 1;
    if (nthreads > 1) {
        // instances sharing a plan or a state must run in order: one thread
        std::vector<const void*> own;
        own.reserve(2 * (size_t)n);
        for (int32_t i = 0; i < n; ++i) {
            own.push_back(plans[i]);
            own.push_back(states[i]);
        }
        std::sort(own.begin(), own.end());
        if (std::adjacent_find(own.begin(), own.end()) != own.end()) nthreads = 1;
    }
    if (nthreads <= 1) {
        for (int32_t i = 0; i < n; ++i) {
            const pf_status st = pf_step(plans[i], states[i], &bodies[i], dt[i], scheme);
            if (st != PF_OK) return st;
        }
        return PF_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PF_ERR_CUDA;
    std::atomic<int32_t> next{0};
    std::atomic<int> first_err{PF_OK};
    auto work = [&](bool own_thread) {
        if (own_thread && cudaSetDevice(dev) != cudaSuccess) {
            int expect = PF_OK;
            first_err.compare_exchange_strong(expect, PF_ERR_CUDA);
            return;
        }
        for (;;) {
            const int32_t i = next.fetch_add(1);
            if (i >= n || first_err.load() != PF_OK) return;
            const pf_status st = pf_step(plans[i], states[i], &bodies[i], dt[i], scheme);
            if (st != PF_OK) {
                int expect = PF_OK;
                first_err.compare_exchange_strong(expect, (int)st);
            }
        }
    };
    std::vector<std::thread> pool;
    pool.reserve(nthreads - 1);
    for (int k = 1; k < nthreads; ++k) pool.emplace_back(work, true);
    work(false);
    for (auto& t : pool) t.join();
    return (pf_status)first_err.load();
}

pf_status pf_batch_create(int32_t n, pf_plan* plans, pf_state* states, const pf_body_kinematics* bodies,
                          const double* dt, int32_t scheme, pf_batch* out) {
    if (!out) return PF_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !plans || !states || !bodies || !dt || (scheme != 0 && scheme != 1)) return PF_ERR_ARG;
    std::vector<const void*> own;
    for (int32_t i = 0; i < n; ++i) {
        pf_plan p = plans[i];
        pf_state s = states[i];
        const pf_body_kinematics& k = bodies[i];
        if (!p || !s || s->plan != p || !p->stream || p->tm.on || !(dt[i] > 0) || !fixed_in_time(k)) return PF_ERR_ARG;
        if (k.ns != 0 && (k.ns < 4 || k.ns > PF_MAX_SURFACE_POINTS || !k.xb || !k.yb || !k.ds ||
                          (k.n_edges != 0 && k.n_edges != 2)))
            return PF_ERR_ARG;
        own.push_back(p);
        own.push_back(s);
    }
    std::sort(own.begin(), own.end());
    if (std::adjacent_find(own.begin(), own.end()) != own.end()) return PF_ERR_ARG;
    // everything a step of the full capacity allocates, ahead of the capture
    for (int32_t i = 0; i < n; ++i) {
        PF_TRY(prepare_capture(plans[i], states[i], bodies[i]));
        PF_CUDA(plans[i], cudaStreamSynchronize(plans[i]->stream));
    }
    pf_batch b = new (std::nothrow) pf_batch_s();
    if (!b) return PF_ERR_OOM;
    b->plans.assign(plans, plans + n);
    b->states.assign(states, states + n);
    b->bodies.assign(bodies, bodies + n);
    b->dt.assign(dt, dt + n);
    for (int32_t i = 0; i < n; ++i) b->released.push_back(bodies[i].ns > 0 && bodies[i].n_edges == 2 ? 2 : 0);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    b->order.assign(n, nullptr);
    for (int32_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->order[i], cudaEventDisableTiming);
    pf_status st = PF_OK;
    if (e != cudaSuccess) {
        snprintf(plans[0]->err, sizeof(plans[0]->err), "pf_batch_create: %s", cudaGetErrorString(e));
        st = PF_ERR_CUDA;
    }
    if (st == PF_OK) st = capture_batch(b, scheme);
    if (st != PF_OK) {
        free_batch(b);
        delete b;
        return st;
    }
    *out = b;
    return PF_OK;
}

pf_status pf_batch_step(pf_batch b, int32_t nsteps) {
    if (!b || nsteps < 0) return PF_ERR_ARG;
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i)
        if (b->states[i]->nv + (int64_t)nsteps * b->released[i] > b->states[i]->cap) return PF_ERR_CAPACITY;
    if (nsteps == 0) return PF_OK;
    pf_plan p0 = b->plans[0];
    for (size_t i = 0; i < n; ++i) {
        PF_CUDA(p0, cudaEventRecord(b->order[i], b->plans[i]->stream));
        PF_CUDA(p0, cudaStreamWaitEvent(b->stream, b->order[i], 0));
    }
    for (int32_t k = 0; k < nsteps; ++k) PF_CUDA(p0, cudaGraphLaunch(b->exec, b->stream));
    PF_CUDA(p0, cudaEventRecord(b->join, b->stream));
    for (size_t i = 0; i < n; ++i) {
        PF_CUDA(p0, cudaStreamWaitEvent(b->plans[i]->stream, b->join, 0));
        for (int32_t k = 0; k < nsteps; ++k) step_graph_advance(b->states[i], b->released[i], b->dt[i]);
    }
    return PF_OK;
}

pf_status pf_batch_destroy(pf_batch b) {
    if (!b) return PF_ERR_ARG;
    free_batch(b);
    delete b;
    return PF_OK;
}

}  // extern "C"

// Request server: continuous batching of independent time-stepping requests
// on one GPU (host-side scheduler, device-resident instances).
//
// A request carries a grid, a body, initial vortices and a number of steps.
// Requests are admitted in submission order while a slot is free and the
// device memory of all resident slots stays within the budget.  A slot is a
// plan clone (sharing its grid shape's LGF tables and spectra), a stream and a
// vortex state; a finished request leaves its slot idle for the next request
// of the same shape, so grids, spectra and Schur factors stay on the device.
// All of a request's steps are enqueued on its slot's stream at admission:
// the first as a plain step (it factors S and sizes the buffers), the rest,
// for a body fixed in time, as launches of one step captured into a CUDA
// graph (one host call per step instead of a few dozen launches); slots on
// distinct streams overlap on the device.  Completion is detected with
// events, without blocking.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "body.cuh"
#include "common.cuh"


namespace {

constexpr int GRAPH_MIN_STEPS = 2;   // remaining steps from which a request's step is captured

// Slot capacities come in powers of two (at least 1024 vortices), so that an
// idle slot serves any later request of its shape up to that size and slots
// are created (allocations, page-locked staging) far less often.
int64_t slot_capacity(int64_t need) {
    int64_t c = 1024;
    while (c < need) c *= 2;
    return c;
}

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket = 0;
    pf_grid_desc grid{};
    std::vector<double> xb, yb, ds, X, Y, G;
    pf_body_kinematics kin{};
    int64_t capacity = 0;
    int32_t nsteps = 0, scheme = 0;
    double dt = 0;
    double t_submit = 0, latency = 0;
    std::vector<double> Xo, Yo, Go;
    int64_t nv_out = 0;
    pf_status status = PF_OK;
    bool done = false;
};

struct Shape {
    int nx, ny;
    double dx, x0, y0;
    pf_plan base = nullptr;
    cudaStream_t stream = nullptr;
    int64_t table_bytes = 0;
};

struct Slot {
    int shape = -1;
    pf_plan plan = nullptr;
    cudaStream_t stream = nullptr;
    pf_state state = nullptr;
    int64_t cap = 0, bytes = 0;
    double* pinned = nullptr;    // 3 * cap doubles: X | Y | G
    int64_t nv_out = 0;
    cudaEvent_t done = nullptr;
    cudaGraphExec_t graph = nullptr;     // the running request's captured step
    Request* req = nullptr;
    double last_used = 0;
};

// device bytes of a slot: plan workspaces, vortex bins, state, Schur factor
int64_t slot_bytes(const Shape& s, int prec, int64_t cap, int ns) {
    const int64_t esz = prec == PF_FP64 ? 8 : 4;
    const int P = 1 << (32 - __builtin_clz(2 * s.nx - 1)), ldT = (s.ny + 3) / 4 * 4, ldK = (P / 2 + 4) / 4 * 4;
    const int64_t spec = (int64_t)ldK * ldT * 2 * esz;
    const int64_t grid = 3 * spec + 3 * (int64_t)s.nx * s.ny * esz;
    const int64_t c = cap > 4096 ? cap : 4096;
    const int64_t ntiles = (int64_t)((s.nx + 31) / 32) * ((s.ny + 31) / 32);
    const int64_t bins = c * 32 + 4 * c * 32 + 2 * ntiles * 4 + (int64_t)bin_blocks(c) * ntiles * 4;
    const int64_t state = 5 * cap * 8 + 4 * cap * esz + 4096 * 8;
    // two Schur factors (a moving body keeps the last two poses), each S, the
    // ns x 2 ns Gauss-Jordan workspace, S^-1, and O(ns) vectors and orderings
    const int64_t schur = 2 * ((int64_t)ns * ns * 8 * 4 + (int64_t)ns * 328);
    // FP64 buffers of the FFT route of the surface right-hand side (mixed plans)
    const int64_t M = (int64_t)s.nx * s.ny;
    const int Q = 1 << (32 - __builtin_clz(2 * s.ny - 1));
    const bool fft = P >= 256 && Q >= 256 && (int64_t)ns * M > ((int64_t)1 << 22);
    const int64_t rhs = ((fft && prec != PF_FP64) ? 2 * M * 8 + 2 * (int64_t)ldK * ldT * 16 : 0) +
                        M * 12;    // node list of the sparse route
    return grid + bins + state + schur + rhs;
}

int64_t table_bytes(int nx, int ny) {
    const int P = 1 << (32 - __builtin_clz(2 * nx - 1)), Q = 1 << (32 - __builtin_clz(2 * ny - 1));
    return (int64_t)(nx + 1) * (ny + 1) * 8 + 3 * (int64_t)(P / 2 + 1) * ((Q / 2 + 4) / 4 * 4) * 12;
}

}  // namespace

struct pf_server_s {
    pf_server_config cfg{};
    std::vector<Shape> shapes;
    std::vector<Slot*> slots;            // all slots (idle and busy)
    std::deque<Request*> queue;
    std::map<int64_t, Request*> reqs;
    std::vector<int64_t> finished;       // tickets not yet reported by progress
    int64_t next_ticket = 1;
    int64_t used = 0;                    // tables + slots
};

namespace {

int find_shape(pf_server s, const pf_grid_desc& g) {
    for (size_t i = 0; i < s->shapes.size(); ++i) {
        const Shape& h = s->shapes[i];
        if (h.nx == g.nx && h.ny == g.ny && h.dx == g.dx && h.x0 == g.x0 && h.y0 == g.y0) return (int)i;
    }
    return -1;
}

void destroy_slot(pf_server s, Slot* sl) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    if (sl->graph) cudaGraphExecDestroy(sl->graph);
    if (sl->state) pf_state_destroy(sl->state);
    if (sl->plan) pf_plan_destroy(sl->plan);
    if (sl->pinned) cudaFreeHost(sl->pinned);
    if (sl->done) cudaEventDestroy(sl->done);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    s->used -= sl->bytes;
    delete sl;
}

// free idle slots, least recently used first, until `need` more bytes fit
bool make_room(pf_server s, int64_t need) {
    while (s->used + need > s->cfg.hbm_budget_bytes) {
        Slot* victim = nullptr;
        size_t vi = 0;
        for (size_t i = 0; i < s->slots.size(); ++i) {
            Slot* sl = s->slots[i];
            if (!sl->req && (!victim || sl->last_used < victim->last_used)) { victim = sl; vi = i; }
        }
        if (!victim) return false;
        s->slots.erase(s->slots.begin() + vi);
        destroy_slot(s, victim);
    }
    return true;
}

pf_status new_slot(pf_server s, int shape, int64_t cap, int ns, Slot** out) {
    Shape& h = s->shapes[shape];
    const int64_t bytes = slot_bytes(h, s->cfg.precision, cap, ns);
    Slot* sl = new (std::nothrow) Slot();
    if (!sl) return PF_ERR_OOM;
    sl->shape = shape;
    sl->cap = cap;
    sl->bytes = bytes;
    s->used += bytes;
    pf_status st = PF_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl->pinned, 3 * (size_t)(cap > 0 ? cap : 1) * sizeof(double));
    // only a failed allocation is worth waiting on; any other error (a lost
    // context, for one) fails the request
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
    if (st == PF_OK) st = pf_plan_clone(h.base, s->cfg.precision, sl->stream, &sl->plan);
    if (st == PF_OK) st = pf_state_create(sl->plan, cap, &sl->state);
    if (st == PF_OK) st = plan_reserve_vortices(sl->plan, cap);
    if (st != PF_OK) {
        destroy_slot(s, sl);
        return st;
    }
    s->slots.push_back(sl);
    *out = sl;
    return PF_OK;
}

// enqueue a request on a slot: load, nsteps steps, store, completion event
void launch(Slot* sl, Request* r) {
    sl->req = r;
    const int64_t nv = (int64_t)r->X.size();
    double* X = sl->pinned;
    double* Y = X + sl->cap;
    double* G = Y + sl->cap;
    std::copy(r->X.begin(), r->X.end(), X);
    std::copy(r->Y.begin(), r->Y.end(), Y);
    std::copy(r->G.begin(), r->G.end(), G);
    pf_status st = state_load_async(sl->state, X, Y, G, nv, 0.0);
    int k = 0;
    if (st == PF_OK && r->nsteps > 0) {
        st = pf_step(sl->plan, sl->state, &r->kin, r->dt, r->scheme);
        k = 1;
    }
    const bool fixed = r->kin.ns == 0 || r->kin.amp == 0.0 || r->kin.omega == 0.0;
    if (st == PF_OK && fixed && r->nsteps - k >= GRAPH_MIN_STEPS) {
        int released = 0;
        st = step_graph_create(sl->plan, sl->state, r->kin, r->dt, r->scheme, &sl->graph, &released);
        for (; k < r->nsteps && st == PF_OK; ++k) {
            if (cudaGraphLaunch(sl->graph, sl->stream) != cudaSuccess) st = PF_ERR_CUDA;
            else step_graph_advance(sl->state, released, r->dt);
        }
    }
    for (; k < r->nsteps && st == PF_OK; ++k) st = pf_step(sl->plan, sl->state, &r->kin, r->dt, r->scheme);
    if (st == PF_OK) st = state_store_async(sl->state, X, Y, G, &sl->nv_out);
    r->status = st;
    cudaEventRecord(sl->done, sl->stream);
}

void retire(pf_server s) {
    for (Slot* sl : s->slots) {
        if (!sl->req) continue;
        const cudaError_t e = cudaEventQuery(sl->done);
        if (e == cudaErrorNotReady) continue;
        Request* r = sl->req;
        r->latency = now_s() - r->t_submit;
        if (e != cudaSuccess && r->status == PF_OK) r->status = PF_ERR_CUDA;
        if (r->status == PF_OK) {
            int64_t oob = 0;
            const pf_status st = pf_sync(sl->plan, &oob);     // sticky device status of this instance
            if (st != PF_OK) r->status = st;
        }
        const int64_t n = sl->nv_out;
        r->nv_out = n;
        r->Xo.assign(sl->pinned, sl->pinned + n);
        r->Yo.assign(sl->pinned + sl->cap, sl->pinned + sl->cap + n);
        r->Go.assign(sl->pinned + 2 * sl->cap, sl->pinned + 2 * sl->cap + n);
        r->done = true;
        s->finished.push_back(r->ticket);
        sl->req = nullptr;
        sl->last_used = now_s();
        if (sl->graph) {
            cudaGraphExecDestroy(sl->graph);
            sl->graph = nullptr;
        }
    }
}

// finish the request at the head of the queue without running it
void reject(pf_server s, pf_status st) {
    Request* r = s->queue.front();
    s->queue.pop_front();
    r->status = st;
    r->latency = now_s() - r->t_submit;
    r->nv_out = 0;
    r->done = true;
    s->finished.push_back(r->ticket);
}

// Admit queued requests in order.  A request waits while running requests
// hold the slots or the memory it needs; one that cannot be admitted with
// nothing running never will be, and fails with PF_ERR_OOM.  A CUDA error
// fails the request and is returned.
pf_status admit(pf_server s) {
    while (!s->queue.empty()) {
        Request* r = s->queue.front();
        int busy = 0;
        for (Slot* c : s->slots) busy += c->req != nullptr;
        int shape = find_shape(s, r->grid);
        if (shape < 0) {
            const int64_t tb = table_bytes(r->grid.nx, r->grid.ny);
            if (!make_room(s, tb)) {
                if (busy > 0) return PF_OK;
                reject(s, PF_ERR_OOM);
                continue;
            }
            Shape h;
            h.nx = r->grid.nx; h.ny = r->grid.ny; h.dx = r->grid.dx; h.x0 = r->grid.x0; h.y0 = r->grid.y0;
            h.table_bytes = tb;
            if (cudaStreamCreateWithFlags(&h.stream, cudaStreamNonBlocking) != cudaSuccess) {
                reject(s, PF_ERR_CUDA);
                return PF_ERR_CUDA;
            }
            pf_grid_desc g = r->grid;
            g.precision = s->cfg.precision;
            const pf_status st = pf_plan_create(&g, h.stream, &h.base);
            if (st != PF_OK) {
                cudaStreamDestroy(h.stream);
                if (st == PF_ERR_OOM && busy > 0) return PF_OK;   // wait for memory to free up
                reject(s, st);
                if (st == PF_ERR_OOM || st == PF_ERR_ARG) continue;
                return st;
            }
            s->used += tb;
            s->shapes.push_back(h);
            shape = (int)s->shapes.size() - 1;
        }
        if (busy >= s->cfg.max_slots) return PF_OK;
        Slot* sl = nullptr;
        for (Slot* c : s->slots)
            if (!c->req && c->shape == shape && c->cap >= r->capacity) {
                sl = c;
                break;
            }
        if (!sl) {
            const int64_t cap = slot_capacity(r->capacity);
            if (!make_room(s, slot_bytes(s->shapes[shape], s->cfg.precision, cap, r->kin.ns))) {
                if (busy > 0) return PF_OK;
                reject(s, PF_ERR_OOM);
                continue;
            }
            const pf_status st = new_slot(s, shape, cap, r->kin.ns, &sl);
            if (st == PF_ERR_OOM && busy > 0) return PF_OK;    // wait for memory to free up
            if (st != PF_OK) {
                reject(s, st);
                if (st == PF_ERR_OOM) continue;
                return st;
            }
        }
        s->queue.pop_front();
        launch(sl, r);
    }
    return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_server_create(const pf_server_config* cfg, pf_server* out) {
    if (!cfg || !out || cfg->max_slots < 1 || cfg->hbm_budget_bytes <= 0 ||
        (cfg->precision != PF_FP64 && cfg->precision != PF_MIXED))
        return PF_ERR_ARG;
    pf_server s = new (std::nothrow) pf_server_s();
    if (!s) return PF_ERR_OOM;
    s->cfg = *cfg;
    *out = s;
    return PF_OK;
}

pf_status pf_server_destroy(pf_server s) {
    if (!s) return PF_ERR_ARG;
    for (Slot* sl : s->slots) destroy_slot(s, sl);
    for (Shape& h : s->shapes) {
        pf_plan_destroy(h.base);
        cudaStreamDestroy(h.stream);
    }
    for (auto& kv : s->reqs) delete kv.second;
    for (Request* r : s->queue) (void)r;   // owned by reqs
    delete s;
    return PF_OK;
}

pf_status pf_server_submit(pf_server s, const pf_request* q, int64_t* ticket) {
    if (!s || !q || !ticket || q->nv < 0 || q->nsteps < 0 || !(q->dt > 0) || (q->scheme != 0 && q->scheme != 1))
        return PF_ERR_ARG;
    if (q->nv > 0 && (!q->X || !q->Y || !q->Gam)) return PF_ERR_ARG;
    const pf_body_kinematics& b = q->body;
    if (b.ns < 0 || b.ns > PF_MAX_SURFACE_POINTS || (b.ns > 0 && (!b.xb || !b.yb || !b.ds))) return PF_ERR_ARG;
    const int64_t need = q->nv + ((b.ns > 0 && b.n_edges == 2) ? 2 * (int64_t)q->nsteps : 0);
    if (q->capacity < need) return PF_ERR_CAPACITY;
    Request* r = new (std::nothrow) Request();
    if (!r) return PF_ERR_OOM;
    r->ticket = s->next_ticket++;
    r->grid = q->grid;
    r->xb.assign(b.xb, b.xb + b.ns);
    r->yb.assign(b.yb, b.yb + b.ns);
    r->ds.assign(b.ds, b.ds + b.ns);
    r->kin = b;
    r->kin.xb = r->xb.data();
    r->kin.yb = r->yb.data();
    r->kin.ds = r->ds.data();
    r->X.assign(q->X, q->X + q->nv);
    r->Y.assign(q->Y, q->Y + q->nv);
    r->G.assign(q->Gam, q->Gam + q->nv);
    r->capacity = q->capacity;
    r->nsteps = q->nsteps;
    r->dt = q->dt;
    r->scheme = q->scheme;
    r->t_submit = now_s();
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    return admit(s);
}

pf_status pf_server_progress(pf_server s, int32_t max, int64_t* tickets, int32_t* n_done) {
    if (!s || max < 0 || (max > 0 && !tickets) || !n_done) return PF_ERR_ARG;
    retire(s);
    const pf_status st = admit(s);
    int32_t n = 0;
    while (n < max && !s->finished.empty()) {
        tickets[n++] = s->finished.front();
        s->finished.erase(s->finished.begin());
    }
    *n_done = n;
    return st;
}

pf_status pf_server_result(pf_server s, int64_t ticket, double* X, double* Y, double* G, int64_t* nv,
                           double* latency_s) {
    if (!s) return PF_ERR_ARG;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || !it->second->done) return PF_ERR_ARG;
    Request* r = it->second;
    if (X) std::copy(r->Xo.begin(), r->Xo.end(), X);
    if (Y) std::copy(r->Yo.begin(), r->Yo.end(), Y);
    if (G) std::copy(r->Go.begin(), r->Go.end(), G);
    if (nv) *nv = r->nv_out;
    if (latency_s) *latency_s = r->latency;
    const pf_status st = r->status;
    s->reqs.erase(it);
    delete r;
    return st;
}

pf_status pf_server_stats(pf_server s, int32_t* queued, int32_t* active, int64_t* used_bytes) {
    if (!s) return PF_ERR_ARG;
    int a = 0;
    for (Slot* sl : s->slots) a += sl->req != nullptr;
    if (queued) *queued = (int32_t)s->queue.size();
    if (active) *active = a;
    if (used_bytes) *used_bytes = s->used;
    return PF_OK;
}

}  // extern "C"

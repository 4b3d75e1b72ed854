// Internal definitions of the immersed-body path (body.cu).
#pragma once
#include "common.cuh"

struct pf_schur_s {
    pf_plan plan = nullptr;
    int ns = 0;
    double* x = nullptr;      // surface points (device, ns)
    double* y = nullptr;
    double* ds = nullptr;
    int* six = nullptr;       // smoothed three-point stencils: node indices and weights (ns x 4)
    int* siy = nullptr;
    double* swx = nullptr;
    double* swy = nullptr;
    double* S = nullptr;      // Schur complement, row-major ns x ns
    double* A = nullptr;      // Gauss-Jordan workspace ns x 2 ns
    double* Sinv = nullptr;   // S^-1
    double* f0 = nullptr;     // S^-1 1
    double* f0hat = nullptr;  // dS o f0
    double* dgamma0 = nullptr;
    double gamma0 = 0.0;      // host copy of Gamma0
    int* sorder = nullptr;    // the 16 ns stencil entries e = 16 p + 4 b + a sorted by (grid node, e)
    int* snode = nullptr;     // their grid nodes in that order (both null when ns > SHEET_SORT_MAX)
    double* gj = nullptr;     // blocked Gauss-Jordan scratch: LU (32 x 32), Y, Z (32 x ns), L_R (ns x 32), perm, gperm
    double* work = nullptr;   // 12 ns doubles of solve scratch
    double* mwork = nullptr;  // several-body solve scratch (allocated by the first such solve)
    // surface pressure (pf_pressure_setup): unit normals (ns each), the face
    // stencils (per point 16 indices and weights: u lattice x, y then v lattice
    // x, y, 4 nodes each), the node stencils of C_s (ns x 64), and the factor of
    // the jump operator augmented with the gauge row (an (ns + 1) system)
    double* pnx = nullptr;
    double* pny = nullptr;
    int* fidx = nullptr;
    double* fwt = nullptr;
    int* ci = nullptr;
    int* cj = nullptr;
    double* cw = nullptr;
    struct pf_schur_s* jump = nullptr;
    int pbox[4] = {0, -1, 0, -1};   // cell-centre box (i0, i1, j0, j1) the surface faces can reach
    double* scal = nullptr;   // device scalars: s0, Gamma1, Gamma2, -, new-vortex x[2], y[2]
    int* rows = nullptr;      // lowest and highest grid row of the stencils (device): the rows psi is read at
    double* ewpart = nullptr; // sparse surface sum: partial sums (ns x EW_SPLIT_MAX) and a done counter per point
    unsigned* ewdone = nullptr;
};
constexpr int EW_SPLIT_MAX = 16;

pf_status schur_create(pf_plan p, int ns, pf_schur* out);
void schur_free(pf_schur s);
pf_status schur_factor_device(pf_plan p, pf_schur s);
pf_status invert_schur_matrix(pf_plan p, pf_schur s);
// Several bodies (Sec. 2.7): validate a partition (and count its edges); the
// device-level solve of pf_sheet_solve_multi with new vortices at device
// (vx, vy) and, when gw_dev is not null, the bodies' gamma_w read from the
// device; *out_dev receives the device address of s0 (B values) then the new
// strengths (one per edge).
pf_status multibody_check(const pf_multibody& mb, int ns, int* n_edges_total);
// Point vortices (device FP64 arrays of n) whose E_s L^-1 R_v Gamma a sheet
// solve forms directly (the vortex route of surface_rhs): always when force is
// set; otherwise only for mixed plans while the direct sum is cheap.
struct VortexSource {
    const double* X = nullptr;
    const double* Y = nullptr;
    const double* G = nullptr;
    int64_t n = 0;
    bool force = false;
};
pf_status sheet_solve_multi_device(pf_plan p, pf_schur s, const void* w, const pf_multibody& mb, int ne,
                                   const double* vx, const double* vy, double* f, const double* gw_dev,
                                   double** out_dev, int64_t nnz_bound = -1, const VortexSource* vs = nullptr);
// Generalized edge condition (Sec. 2.5) for the shedding mode: with on = 0 every
// edge sheds under the Kutta condition; otherwise edge e sheds only when its
// intermediate value lies outside [lo[e], hi[e]], and ends at the bound crossed.
struct EdgeBounds {
    int on = 0;
    double lo[2] = {0.0, 0.0};
    double hi[2] = {0.0, 0.0};
};
// param_dev (nullable): device copy of `param` read by the kernels instead;
// nnz_bound >= 0: at most that many nodes of w are nonzero (lets the surface
// right-hand side take the sparse route), -1: unknown
pf_status sheet_solve_device(pf_plan p, pf_schur s, const void* w, const pf_motion& m, int mode, double param,
                             const double* param_dev, int n_edges, const int* edges, const double* vx,
                             const double* vy, double* f, const EdgeBounds& eb = EdgeBounds(),
                             int64_t nnz_bound = -1, const VortexSource* vs = nullptr);
// w += R_s f  (device f of ns doubles, w real[nx*ny])
pf_status sheet_deposit(pf_plan p, pf_schur s, const double* f, void* w);
// allocate what a sheet solve with this nonzero bound allocates on first use
pf_status sheet_solve_reserve(pf_plan p, pf_schur s, int64_t nnz_bound);

// step.cu: asynchronous state transfers used by the request server
pf_status state_load_async(pf_state s, const double* X, const double* Y, const double* G, int64_t nv, double t);
pf_status state_store_async(pf_state s, double* X, double* Y, double* G, int64_t* nv);
int64_t state_capacity(pf_state s);
// One pf_step of (p, s, k) captured on the plan's stream and instantiated
// (the capture runs nothing; s's host counts are left as they were).  The
// body must be fixed in time; the factor at its pose and every buffer a step
// of the state's capacity uses are made ready first (this may synchronise the
// plan's stream).  released: the vortices one step appends.
pf_status step_graph_create(pf_plan p, pf_state s, const pf_body_kinematics& k, double dt, int scheme,
                            cudaGraphExec_t* out, int* released);
// the host counts after one launch of a captured step
void step_graph_advance(pf_state s, int released, double dt);

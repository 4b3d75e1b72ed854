/*
 * gridpf: grid-based planar potential flow with point vortices and an
 * immersed body (Beckers & Eldredge, "Planar potential flow on Cartesian
 * grids", arXiv 2102.11910), on one NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Plain pointers and sizes only.  Every entry point returns a
 * pf_status; none throws.  Unless stated otherwise:
 *   - array arguments are DEVICE pointers owned by the caller;
 *   - work is enqueued asynchronously on the plan's CUDA stream, so a call
 *     returning PF_OK means "enqueued"; errors found by kernels (out-of-domain
 *     vortices, a full state, a failed binning check) are recorded in a sticky
 *     device status word and reported by pf_sync;
 *   - node fields are row-major nx*ny arrays, index j*nx + i for node (i, j) at
 *     (x0 + i dx, y0 + j dx);  their element type is double for PF_FP64 plans and
 *     float for PF_MIXED plans ("real" below);
 *   - vortex positions and strengths are always double.
 *
 * Operators (paper notation): L is the 5-point Laplacian scaled by 1/dx^2;
 * L^{-1} is applied with the lattice Green's function G of the unit-spacing
 * Laplacian (L0 G = delta, G(0,0) = 0), so L^{-1} = dx^2 (G *) on the unbounded
 * grid (Sec. 2.1).  R_v / E_v use the M4' kernel (Eq. vortexregularization and
 * E_v = R_v^T), R_s / E_s the smoothed three-point kernel (Sec. 2.2.1).
 */
#ifndef GRIDPF_H
#define GRIDPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PF_OK = 0,
    PF_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad mode)      */
    PF_ERR_OOM = 2,            /* a device allocation failed                               */
    PF_ERR_CUDA = 3,           /* a CUDA runtime call failed; pf_last_error has the text   */
    PF_ERR_OUT_OF_DOMAIN = 4,  /* a point's 4x4 stencil left the grid; it was not used    */
    PF_ERR_SINGULAR = 5,       /* a pivot of the Schur factorisation vanished              */
    PF_ERR_TIMEOUT = 6,        /* a bounded device wait gave up (no kernel here waits on
                                  another: reserved, never returned)                     */
    PF_ERR_NOT_FACTORED = 7,   /* a sheet solve was asked of a body without a factor       */
    PF_ERR_CAPACITY = 8,       /* a state's vortex capacity would be exceeded              */
    PF_ERR_INTERNAL = 9        /* a device-side consistency check of the vortex binning
                                  failed (the offending records were skipped): a bug     */
} pf_status;

typedef enum { PF_FP64 = 0, PF_MIXED = 1 } pf_precision;

typedef struct {
    int32_t nx, ny;        /* nodes per direction, 8 <= nx, ny <= 2048                      */
    double dx;             /* grid spacing                                                  */
    double x0, y0;         /* coordinates of node (0, 0)                                    */
    int32_t precision;     /* pf_precision: element type and arithmetic of the grid path    */
} pf_grid_desc;

typedef struct pf_plan_s* pf_plan;
typedef struct pf_schur_s* pf_schur;
typedef struct pf_state_s* pf_state;
typedef struct pf_vic_state_s* pf_vic_state;

/* ------------------------------------------------------------------ plan */

/* Create a plan for one grid: builds, in FP64 on the device, the LGF table
 * G(m, n) for 0 <= m <= nx, 0 <= n <= ny (Sec. 2.1, refs. katsura71/cserti00)
 * and the real spectrum of G on the zero-padded (P x Q) torus, P, Q the
 * powers of two >= 2 nx, 2 ny.  `stream` is a cudaStream_t (NULL = default).
 * The plan owns all tables and workspaces; the call synchronises the stream. */
pf_status pf_plan_create(const pf_grid_desc* desc, void* stream, pf_plan* out);
pf_status pf_plan_destroy(pf_plan plan);

/* A plan for the same grid that shares the source's read-only tables (LGF
 * table and spectra, reference counted) but has its own workspaces, stream
 * and precision: many instances of one grid shape cost one set of tables.
 * The tables live until the last plan sharing them is destroyed. */
pf_status pf_plan_clone(pf_plan src, int32_t precision, void* stream, pf_plan* out);

/* Padded FFT sizes chosen for the plan (host ints). */
pf_status pf_plan_fft_size(pf_plan plan, int32_t* P, int32_t* Q);

/* How the sheet solves of this plan obtain E_s L^-1 w, the streamfunction of
 * the free vorticity at the surface stencils (Sec. 2.2.2):
 *   PF_RHS_DIRECT  the FP64 lattice-Green's-function sum over every nonzero
 *                  node of w, each surface point scanning all nx ny nodes;
 *   PF_RHS_FFT     a zero-padded FFT solve psi = -L^-1 w (needs P, Q >= 256),
 *                  read at the stencils: FP64 passes for FP64 plans,
 *                  double-float passes (pairs of FP32 words, about 48
 *                  significant bits, run on the FP32 pipe) on the FP32 w of
 *                  mixed plans;
 *   PF_RHS_SPARSE  the direct sum over a list of the nonzero nodes built once
 *                  per solve (16 ns nnz multiply-adds);
 *   PF_RHS_AUTO    (default) in time stepping, where w holds at most 16 nodes
 *                  per vortex, the sparse route while 16 ns (16 capacity) is
 *                  below 2^24 (capacity: the state's, so that a step's route
 *                  does not change as vortices are shed); otherwise the FFT
 *                  when P, Q >= 256 and, for FP64 plans, ns nx ny > 2^22;
 *                  else the direct sum.
 * All are FP64 or better than FP64 in range and within about 30 FP64 ulps in
 * rounding; they differ by rounding only.  Mixed-precision plans that take
 * the FFT route allocate 2 nx ny doubles and two FP64-sized spectra once (and
 * their grid shape one double-float copy of the LGF spectrum); the sparse
 * route allocates nx ny ints and doubles once.
 * PF_ERR_ARG for an unknown route or PF_RHS_FFT on a grid with P or Q < 256. */
enum { PF_RHS_AUTO = 0, PF_RHS_DIRECT = 1, PF_RHS_FFT = 2, PF_RHS_SPARSE = 3 };
pf_status pf_plan_set_rhs_route(pf_plan plan, int32_t route);

/* Copy the plan's FP64 LGF table to a host array of (nx+1)*(ny+1) doubles,
 * index n*(nx+1) + m for G(m, n). Synchronises. */
pf_status pf_lgf_table(pf_plan plan, double* host_out);

/* Wait for the plan's stream; return and clear the sticky status.  If
 * `out_of_domain` is non-null it receives the number of points dropped since
 * the last pf_sync (host int64). */
pf_status pf_sync(pf_plan plan, int64_t* out_of_domain);

/* Text of the last error on this plan (static storage owned by the plan). */
const char* pf_last_error(pf_plan plan);

/* Per-kernel timing (instrumentation; not part of the method).  While on,
 * every kernel the plan launches is bracketed by CUDA events recorded on the
 * plan's stream.  pf_timing_enable(plan, 1) clears the records and turns it
 * on; (plan, 0) turns it off.  pf_timing_report synchronises and writes one
 * line per kernel name, "<name> <launches> <total milliseconds>\n", into the
 * host buffer buf (NUL terminated, truncated to buflen), then clears the
 * records. */
pf_status pf_timing_enable(pf_plan plan, int32_t on);
pf_status pf_timing_report(pf_plan plan, char* buf, int64_t buflen);

/* Launch configuration of a plan's transfer passes (R_v binning and deposit,
 * E_v, Sec. 2.1) and of its Poisson solve L^-1 (Sec. 2.3).  Only how the work
 * is cut into thread blocks changes:
 *   tile          node tile edge of the binning, deposit and E_v passes: 32, or
 *                 16 on grids of at most 4096 such tiles.  The deposit's
 *                 fixed-point scale is per tile, so w differs between edges by
 *                 rounding (within the plan precision's tolerance).
 *   min_span      fewest vortices per binning block: 256, 512, 1024, 2048 or
 *                 4096.  Results are bitwise the same for every value.
 *   tile_threads  threads per tile block of the deposit (and of E_v in FP64
 *                 plans; mixed plans' E_v always runs 256): 128 or 256.
 *                 Results are bitwise the same for both.
 *   fft           0: register-resident radix-16 Stockham passes (grids whose
 *                 padded torus is at least 256 x 256; smaller ones always take
 *                 the shared-memory passes); 1: shared-memory passes.  Results
 *                 differ by rounding.
 * A new plan has {32, 1024, 256, 0}; clones copy their source's. */
typedef struct {
    int32_t tile;
    int32_t min_span;
    int32_t tile_threads;
    int32_t fft;
} pf_launch_config;

pf_status pf_launch_config_get(pf_plan plan, pf_launch_config* out);
/* PF_ERR_ARG (plan unchanged) for a value outside the lists above. */
pf_status pf_launch_config_set(pf_plan plan, const pf_launch_config* cfg);

/* Autotuner: time every valid launch configuration on nv synthetic vortices
 * (uniform in the grid's interior, strengths uniform in [-1e-3, 1e-3], drawn
 * on the device by a counter-based hash) through one body-free velocity
 * evaluation (R_v, L^-1 with the curl, E_v) on the plan's stream: one untimed
 * call, then `reps` calls timed by CUDA events, each after a write of twice
 * the L2 size (so that it starts with a cold cache), the median kept; the
 * fastest is set on the plan.  The plan's grid, precision and the device (name and
 * compute capability) with floor(log2 nv) form the key of one line of the
 * text file `cache_path` (may be null: no file).  A key found there is applied
 * without timing; a new one is appended.  `chosen` and `best_us` (host, may
 * be null) receive the configuration and its median time in microseconds.
 * Synchronises; allocates and frees 5 nv values and the flush buffer of
 * scratch.  PF_ERR_ARG for nv < 1 or reps < 1; PF_ERR_CUDA if the cache file
 * cannot be appended to. */
pf_status pf_autotune(pf_plan plan, int64_t nv, const char* cache_path, int32_t reps, pf_launch_config* chosen,
                      double* best_us);

/* --------------------------------------------------- body-free VIC path */

/* w = R_v Gamma: w_ij = dx^-2 sum_q Gamma_q M4'((x_i-X_q)/dx) M4'((y_j-Y_q)/dx)
 * (Eq. vortexregularization).  X, Y, Gam: nv doubles.  w: real[nx*ny], fully
 * overwritten.  The sum is formed in 64-bit fixed point per tile, so the
 * result is bitwise independent of scheduling.  Vortices whose stencil leaves
 * the grid are skipped and counted (PF_ERR_OUT_OF_DOMAIN at pf_sync). */
pf_status pf_regularize(pf_plan plan, const double* X, const double* Y, const double* Gam,
                        int64_t nv, void* w);

/* psi = -L^{-1} w (Sec. 2.1, particular solution; no homogeneous part).
 * w, psi: real[nx*ny]; they may alias. */
pf_status pf_poisson_solve(pf_plan plan, const void* w, void* psi);

/* Node velocity of psi = -L^{-1} w plus a uniform flow: u = d psi/dy,
 * v = -d psi/dx by centred differences (Eq. velsf with the face-to-node
 * averages of Sec. 2.1), evaluated exactly in spectral form on the padded
 * torus.  uv: real[2*nx*ny], interleaved (u, v) per node. */
pf_status pf_velocity_solve(pf_plan plan, const void* w, double Uinf, double Vinf, void* uv);

/* E_v: velocity at nq points from an interleaved node velocity field:
 * uq[q] = sum_ij M4' M4' u_ij (E_v = R_v^T, Sec. 2.1).  uq, vq: real[nq]. */
pf_status pf_interpolate(pf_plan plan, const void* uv, const double* Xq, const double* Yq,
                         int64_t nq, void* uq, void* vq);

/* The whole body-free step: R_v, psi = -L^{-1} w, curl, E_v at the vortices
 * themselves (plus the uniform flow).  uq, vq: real[nv]; a vortex whose
 * stencil leaves the grid is left out of R_v, counted (pf_sync) and gets
 * uq = vq = 0. */
pf_status pf_vic_velocity(pf_plan plan, const double* X, const double* Y, const double* Gam,
                          int64_t nv, double Uinf, double Vinf, void* uq, void* vq);

/* Same step with HOST input and output buffers, synchronous.  Page-locked
 * inputs (cudaHostAlloc / cudaHostRegister) are read by the first kernel
 * directly over the host link; pageable inputs are first copied to a device
 * staging buffer.  uq, vq (real[nv]) are copied back from the device. */
pf_status pf_vic_velocity_host(pf_plan plan, const double* X, const double* Y, const double* Gam,
                               int64_t nv, double Uinf, double Vinf, void* uq, void* vq);

/* Same step with HOST buffers, asynchronous: the inputs are copied by the
 * copy engine into the plan's device staging buffer, the step runs, and uq,
 * vq are copied back, all queued on the plan's stream; the call returns
 * without waiting.  X, Y, Gam must stay unchanged and uq, vq unread until
 * pf_sync(plan) returns.  With page-locked buffers the copies of one plan
 * overlap the kernels of another, so a caller alternating two plans keeps
 * the host link and the GPU busy together.  Errors of the queued work are
 * reported by pf_sync. */
pf_status pf_vic_velocity_host_async(pf_plan plan, const double* X, const double* Y, const double* Gam,
                                     int64_t nv, double Uinf, double Vinf, void* uq, void* vq);

/* ------------------------------------------------------- immersed body */

#define PF_MAX_SURFACE_POINTS 4096

/* Surface points of one body (HOST arrays of ns doubles): coordinates and
 * the length dS_p of the segment each point represents (Sec. 2.2.1). */
typedef struct {
    int32_t ns;
    const double* x;
    const double* y;
    const double* ds;
} pf_body_desc;

/* Rigid motion of the body and the free stream: translation (U, V), rotation
 * Omega about the origin; (Uinf, Vinf) is the uniform flow whose
 * streamfunction psi_inf = Uinf y - Vinf x is the homogeneous part of the
 * solution (Sec. 2.1, Eqs. velsurf, sfsurf). */
typedef struct {
    double U, V, Omega;
    double Uinf, Vinf;
} pf_motion;

typedef enum {
    PF_SHEET_GIVEN_S0 = 0,     /* Eq. vsheet: f = S^-1 (s'_b - s0 1 + E L^-1 w); param = s0          */
    PF_SHEET_CIRCULATION = 1,  /* Eq. circsystem: bound circulation <1, f> = param; s0 solved for    */
    PF_SHEET_KUTTA_STEADY = 2, /* Eq. kuttasystem: ftilde = P_k Stilde^-1 (P^Gamma s'_b + E L^-1 w),
                                  one edge k = edges[0]; param unused                              */
    PF_SHEET_KUTTA_SHED = 3    /* Eq. kuttasystem2 (one edge) / Eq. twovortex (two edges): new
                                  vortices at (Xnew, Ynew) take the strengths that null ftilde at
                                  the edges and keep the total circulation zero; param = Gamma_w,
                                  the circulation of the existing free vorticity                   */
} pf_sheet_mode;

/* Schur complement S = -E L^-1 R_s of a body on the plan's grid (Eq. vsheet),
 * its FP64 inverse by Gauss-Jordan with partial pivoting, f0 = S^-1 1 and
 * Gamma0 = <1, f0> (Eqs. f0, circ0).  Synchronous.  Every surface point's
 * stencil must lie inside the grid (else PF_ERR_OUT_OF_DOMAIN); a vanishing
 * pivot gives PF_ERR_SINGULAR.  The factor owns its device memory. */
pf_status pf_schur_factor(pf_plan plan, const pf_body_desc* body, pf_schur* out);
pf_status pf_schur_destroy(pf_schur schur);

/* Host copies: Gamma0 (scalar), f0 (ns doubles) and S (ns*ns, row-major); any
 * may be NULL.  Synchronises. */
pf_status pf_schur_info(pf_schur schur, double* gamma0, double* f0, double* S);

/* Bound vortex sheet for the free vorticity w (device real[nx*ny], e.g. from
 * pf_regularize), body motion m and mode (pf_sheet_mode).  E_s L^-1 w, the
 * free vorticity's streamfunction seen by the surface (Eq. intermedsoln), is
 * summed directly with the FP64 LGF over the nonzero nodes of w rather than
 * read from an FFT solve: S is ill-conditioned (Sec. 2.2.2), and FFT rounding,
 * white on psi, would be amplified into the sheet.  edges: n_edges (1 or 2) surface-point indices of the Kutta
 * edges (host), used by the Kutta modes.  Xnew, Ynew: host positions of the
 * n_edges new vortices (mode PF_SHEET_KUTTA_SHED).  Outputs: f (device,
 * ns doubles: the sheet strength gamma, Sec. 2.2.2), gamma_new (host,
 * n_edges: new vortex strengths), s0 (host: the uniform streamfunction value).
 * The sheet solve runs in FP64 for both precisions.  Synchronises. */
pf_status pf_sheet_solve(pf_plan plan, pf_schur schur, const void* w, const pf_motion* m,
                         int32_t mode, double param, int32_t n_edges, const int32_t* edges,
                         const double* Xnew, const double* Ynew, double* f, double* gamma_new,
                         double* s0);

/* The same solve for the free vorticity of point vortices given directly:
 * X, Y, Gam are DEVICE arrays of nv vortices.  E_s L^-1 R_v Gamma is summed
 * in FP64 from the vortices themselves (sixteen M4' node entries each, Eq.
 * vortexregularization, against the FP64 LGF), so no FP32 rounding of a
 * regularized field enters the sheet, whatever the plan's precision: the sheet
 * of a mixed plan then carries only FP64 rounding times cond(S) (Sec. 2.2.2,
 * S ill-conditioned below dS/dx ~ 1).  Cost: 256 ns nv FP64 multiply-adds.
 * Vortices whose stencil leaves the grid are left out.  Other arguments,
 * outputs and errors as pf_sheet_solve.  Synchronises. */
pf_status pf_sheet_solve_vortices(pf_plan plan, pf_schur schur, const double* X, const double* Y,
                                  const double* Gam, int64_t nv, const pf_motion* m, int32_t mode, double param,
                                  int32_t n_edges, const int32_t* edges, const double* Xnew, const double* Ynew,
                                  double* f, double* gamma_new, double* s0);

/* Linear and angular impulse of the fluid about the origin (Sec. 2.6.2,
 * Eqs. linimpxd, linimpyd, angimpd); for a single body the force and moment
 * are F = -rho dP/dt and M_O = -rho dPi_O/dt (Eq. FMimp):
 *   P_x  =  <y, w>_N + <y_s, f + n_x v_y - n_y v_x>_S
 *   P_y  = -<x, w>_N - <x_s, f + n_x v_y - n_y v_x>_S
 *   Pi_O = -1/2 <x^2 + y^2, w>_N - 1/2 <x_s^2 + y_s^2, f + n_x v_y - n_y v_x>_S
 * with <a, b>_N = dx^2 sum over the nodes, <a, b>_S = sum_p dS_p a_p b_p and the
 * rigid surface velocity v = (U - Omega y_s, V + Omega x_s).
 *   w        real[nx*ny] node vorticity of the fluid (device), e.g. from pf_regularize
 *   body     surface points (host arrays, as for pf_schur_factor), or NULL: node
 *            terms only
 *   nxs, nys double[ns] unit normals into the fluid (HOST), or both NULL: the
 *            slip term n x v is left out (a zero-thickness plate, whose two sides
 *            cancel it)
 *   f        double[ns] bound sheet strength (device, e.g. from pf_sheet_solve);
 *            required when body has points
 *   m        body motion (host; U, V, Omega used) or NULL for a body at rest
 *   out      double[3] (host): P_x, P_y, Pi_O
 * Sums run in FP64 in a fixed order (bitwise reproducible).  Synchronises the
 * plan's stream. */
pf_status pf_impulse(pf_plan plan, const void* w, const pf_body_desc* body, const double* nxs,
                     const double* nys, const double* f, const pf_motion* m, double* out);

/* Generalized edge condition (Sec. 2.5, Eq. twovortex-gen): the shedding
 * solve of pf_sheet_solve (mode PF_SHEET_KUTTA_SHED, param = gamma_w, the
 * circulation of w) with bounds on the edge values of the non-singular sheet
 * ftilde.  Edge e (surface point edges[e]) sheds only when the intermediate
 * sheet's value there, e_k^T ftilde*, lies outside [bounds[2e], bounds[2e+1]],
 * and then with the strength that puts the final value at the bound it
 * crossed; an edge inside its range sheds nothing (gamma_new[e] = 0).  Zero
 * bounds are the Kutta condition.  For a flat plate of chord c the bounds
 * follow from the edge suction parameter sigma_k through
 * e_k^T ftilde = -(2 pi c / Gamma0) sigma_k.  bounds: host, 2 n_edges, with
 * lo <= hi (else PF_ERR_ARG).  Other arguments and outputs as for
 * pf_sheet_solve.  Synchronises. */
pf_status pf_sheet_solve_edges(pf_plan plan, pf_schur schur, const void* w, const pf_motion* m, double gamma_w,
                               int32_t n_edges, const int32_t* edges, const double* bounds, const double* Xnew,
                               const double* Ynew, double* f, double* gamma_new, double* s0);

/* Several bodies sharing one factor (Sec. 2.7, Eq. kuttasystem4).  The factor
 * is built (pf_schur_factor) over the surface points of all bodies, body after
 * body; body b owns the points start[b] .. start[b+1]-1.  Each body has its own
 * uniform streamfunction value s0_b, a Kutta condition at each of its edges
 * (0, 1 or 2; one new vortex released per edge) and Kelvin's condition over
 * itself and the vorticity released from it:
 *   <1_b, f> + (strengths of its new vortices) = -gamma_w[b].
 * A body without edges is thereby circulation-constrained: gamma_w[b] is minus
 * its prescribed bound circulation. */
#define PF_MAX_BODIES 4
typedef struct {
    int32_t n_bodies;                    /* 1 .. PF_MAX_BODIES */
    int32_t start[PF_MAX_BODIES + 1];    /* start[0] = 0 < start[1] < ... < start[n_bodies] = ns */
    int32_t n_edges[PF_MAX_BODIES];      /* 0, 1 or 2 per body */
    int32_t edge[PF_MAX_BODIES][2];      /* edge surface indices, inside the body's range */
    pf_motion motion[PF_MAX_BODIES];     /* rigid motion of each body; the free stream (Uinf, Vinf)
                                            is motion[0]'s */
    double gamma_w[PF_MAX_BODIES];       /* circulation released earlier from body b (see above) */
} pf_multibody;

/* The several-body shedding solve: s'_b from each body's motion, the free
 * vorticity w (device, plan precision), new vortices at (Xnew[i], Ynew[i])
 * (HOST, one per edge, edges in body order).  Results: f (device, ns doubles),
 * gamma_new (HOST, one per edge, same order), s0 (HOST, n_bodies).  With one
 * body it is pf_sheet_solve's PF_SHEET_KUTTA_SHED (two or one edge) or
 * PF_SHEET_CIRCULATION (no edge, param = -gamma_w[0]).  FP64 for both
 * precisions; the (edges + bodies)-square constraint system is solved by
 * Gaussian elimination with partial pivoting.  PF_ERR_ARG for an invalid
 * partition or edge, PF_ERR_SINGULAR (at the return) if the constraint system
 * has a vanishing pivot.  Synchronises. */
pf_status pf_sheet_solve_multi(pf_plan plan, pf_schur schur, const void* w, const pf_multibody* mb,
                               const double* Xnew, const double* Ynew, double* f, double* gamma_new, double* s0);

/* w += R_s f (device f of ns doubles, w real[nx*ny] of the plan's precision):
 * the bound sheet regularized onto the nodes (Sec. 2.2.1), as the steps add it
 * before the corrected solve; deterministic. */
pf_status pf_sheet_regularize(pf_plan plan, pf_schur schur, const double* f, void* w);

/* ------------------------------------------------------- surface pressure */

/* Surface pressure (Sec. 2.6.1).  The grid is staggered: u = d psi/dy on the
 * x-faces (x_i, y_j + dx/2), v = -d psi/dx on the y-faces (x_i + dx/2, y_j); E_f
 * interpolates each component from its own faces with the smoothed
 * three-point function, and C_s psi = n . E_f C psi is the normal velocity at
 * the surface points.
 *
 * pf_pressure_setup: unit normals of the factor's surface points (HOST, ns
 * each; + side of the jumps) and the factor of the jump operator
 * C_s L^-1 C_s^T, augmented with the gauge sum_p dS_p Delta phi_p = 0 (its
 * null space is the uniform values); once per geometry.  The regularized
 * double layer needs dS/dx ~ 1: at dS/dx = 2 it leaks and the jump of a
 * cylinder in a uniform stream comes out a third too small.  Synchronises.
 *
 * pf_potential_jump: Delta phi = -(C_s L^-1 C_s^T)^-1 C_s L^-1 R_s f (the jump
 * in scalar potential of the sheet, Eq. gamphi and below), f and dphi device,
 * ns doubles; FP64, with one refinement step.
 *
 * pf_pressure_jump: Eq. surfbernoulli,
 *   Delta p = -rho (E_f u - v_s) . (f z x n) - rho d(Delta phi)/dt,
 * with u from psi (device, real[nx*ny] in the plan's precision: the
 * streamfunction of the whole flow without the free stream, e.g.
 * pf_poisson_solve of w + R_s f + new vortices) plus (m->Uinf, m->Vinf), the
 * rigid surface velocity v_s = (U - Omega y, V + Omega x) of *m, f (device),
 * dphi_dt (device, ns, e.g. the difference of two pf_potential_jump results
 * over a step; NULL: steady) and the density rho; dp: device, ns doubles.
 * The surface pressures are p+/- = E_c p +/- Delta p / 2.
 * PF_ERR_NOT_FACTORED before pf_pressure_setup. */
pf_status pf_pressure_setup(pf_plan plan, pf_schur schur, const double* nxs, const double* nys);
pf_status pf_potential_jump(pf_plan plan, pf_schur schur, const double* f, double* dphi);
pf_status pf_pressure_jump(pf_plan plan, pf_schur schur, const void* psi, const pf_motion* m, const double* f,
                           const double* dphi_dt, double rho, double* dp);

/* Pressure field at the cell centres (x0 + (i + 1/2) dx, y0 + (j + 1/2) dx),
 * i < nx - 1, j < ny - 1 (Eq. pgrid, the surface term read inside the
 * divergence since L^-1 acts on centre data):
 *   p = -rho/2 |u|^2 - rho L^-1 D [ w x u + R_f(n o d(Delta phi)/dt - v_s x f) ]
 * with u on the faces from psi (as pf_pressure_jump) plus (m->Uinf, m->Vinf),
 * w the free vorticity on the nodes (device, plan precision), the Lamb vector
 * w x u on the faces from two-node averages of w and four-face averages of the
 * other component (faces outside the grid count as zero), D the divergence
 * to the centres and L^-1 = dx^2 G * on the centre lattice.  schur (after
 * pf_pressure_setup) with f and dphi_dt (device, ns each, either may be NULL)
 * adds the surface terms; schur = NULL: a flow without body.  p: device,
 * (nx-1)(ny-1) doubles, row-major; defined up to nothing (no free constant:
 * the LGF solve is unique).  The first call builds and keeps a plan of the
 * centre lattice (its LGF table and spectra, same stream and precision);
 * FP64 arithmetic except that Poisson solve, in the plan's precision; the
 * surface terms are gathered per centre in a fixed order (deterministic). */
pf_status pf_pressure_field(pf_plan plan, pf_schur schur, const void* psi, const void* w, const pf_motion* m,
                            const double* f, const double* dphi_dt, double rho, double* p);

/* ------------------------------------------------------- time stepping */

/* Device-resident vortex set (positions and strengths, FP64) with a fixed
 * capacity; owned by the state, stepped on its plan's stream. */
pf_status pf_state_create(pf_plan plan, int64_t capacity, pf_state* out);
pf_status pf_state_destroy(pf_state state);
/* Load nv vortices from HOST arrays and set the time; clears the shedding
 * history.  PF_ERR_CAPACITY if nv exceeds the capacity.  Synchronises. */
pf_status pf_state_set(pf_state state, const double* X, const double* Y, const double* Gam, int64_t nv,
                       double t);
/* Copy the current vortices to HOST arrays (each at least nv long; any may be
 * NULL) and report nv and t.  Synchronises. */
pf_status pf_state_get(pf_state state, double* X, double* Y, double* Gam, int64_t* nv, double* t);

/* Body-free vortex-in-cell time stepping on a tile-ordered vortex set
 * (Sec. 2.1: R_v, L^-1 with the LGF, node velocity, E_v; vortices advected
 * with the local velocity by forward Euler, Sec. 2.4.2).
 *
 * The state keeps its vortices binned by 32 x 32 node tile between steps (a
 * home record per vortex plus a copy in each other tile its 4 x 4 stencil
 * reaches), so a step moves the vortices and re-bins them incrementally
 * instead of binning from positions: pf_vic_step = R_v, the spectral node
 * velocity, E_v with the Euler move, and the re-bin.  Mixed plans keep each
 * position as an integer cell and a 24-bit fixed-point fraction (moved in
 * fixed point, rounded to nearest), FP64 plans as a cell and a double
 * fraction.  The state uses its plan's stream and work buffers; the plan must
 * outlive it.
 *
 *   capacity     the most vortices the state holds (1 .. 2^27); device memory
 *                is about 2 x 4 x capacity records (16 bytes mixed, 32 FP64)
 *                plus per-tile tables
 */
pf_status pf_vic_state_create(pf_plan plan, int64_t capacity, pf_vic_state* out);
pf_status pf_vic_state_destroy(pf_vic_state state);
/* Bin nv vortices given as DEVICE arrays (nv <= capacity; PF_ERR_ARG beyond).
 * Vortex k keeps the index k for pf_vic_state_get and pf_vic_step's optional
 * velocity output.  Vortices whose stencil leaves the grid are skipped and
 * counted (PF_ERR_OUT_OF_DOMAIN at pf_sync).  Resets the time to 0.
 * Synchronises the plan's stream. */
pf_status pf_vic_state_set(pf_vic_state state, const double* X, const double* Y, const double* Gam, int64_t nv);
/* Positions and strengths in DEVICE arrays of at least the nv of the last
 * set call, at the vortices' indices (a dropped vortex reads NaN); any of X,
 * Y, Gam may be NULL only if all are.  nv (host, may be NULL) receives the
 * number of vortices still held and t (host, may be NULL) the time; asking
 * for nv synchronises. */
pf_status pf_vic_state_get(pf_vic_state state, double* X, double* Y, double* Gam, int64_t* nv, double* t);
/* One forward-Euler step of length dt in the uniform flow (Uinf, Vinf).  uq,
 * vq: optional DEVICE arrays (real, both or neither) that receive the
 * velocity each vortex moved with, at its index.  A vortex whose home tile
 * would move by more than one tile in a step (possible only for moves of 32
 * cells or more) is dropped (PF_ERR_CAPACITY at pf_sync); one whose stencil
 * would leave the grid is dropped and counted (PF_ERR_OUT_OF_DOMAIN).
 * Asynchronous on the plan's stream. */
pf_status pf_vic_step(pf_vic_state state, double dt, double Uinf, double Vinf, void* uq, void* vq);

/* A rigid body given in its own frame (HOST arrays of ns points: coordinates
 * and segment lengths), turned by the angle -alpha(t) about the origin,
 * alpha(t) = alpha0 + amp sin(omega t) (for a plate along the body x axis the
 * chord points along (cos alpha, -sin alpha)), in the uniform flow
 * (Uinf, Vinf).  n_edges = 2: vortices are released at surface points
 * edge[0], edge[1] (Kutta, Sec. 2.4.3); n_edges = 0: no release, the bound
 * circulation is -sum Gamma (Kelvin, Eq. circsystem).  ns = 0 means no body. */
typedef struct {
    int32_t ns;
    const double* xb;
    const double* yb;
    const double* ds;
    int32_t n_edges;
    int32_t edge[2];
    double alpha0, amp, omega;
    double Uinf, Vinf;
    int32_t edge_bounded;        /* 0: Kutta at both edges; 1: generalized edge condition  */
    double edge_bounds[4];       /* lo_0, hi_0, lo_1, hi_1 (as pf_sheet_solve_edges)        */
} pf_body_kinematics;

/* Advance the vortex set by dt.  With a body that has two edges, two vortices
 * are released per step with the two-edge Kutta condition and Kelvin's
 * theorem (Eq. twovortex), placed by the rule of Sec. 2.4.2 (first release
 * 10 dt |U| from the edge along the normal facing the stream, later ones one
 * third of the way to the previous release); every vortex is advected with the
 * velocity of psi = -L^-1 (w + new vortices + R_s f) plus the free stream.
 * scheme 0: forward Euler (the paper's); 1: Heun's RK2 whose second stage at
 * t + dt keeps the new strengths and sets the bound circulation to
 * -sum Gamma (Eq. circsystem).  With edge_bounded the release follows the
 * generalized edge condition of pf_sheet_solve_edges (an edge inside its
 * bounds releases a vortex of zero strength).  S is refactored whenever the pose changes
 * (every stage of a pitching body); nothing in a step waits for the host.
 * PF_ERR_CAPACITY if two more vortices do not fit. */
pf_status pf_step(pf_plan plan, pf_state state, const pf_body_kinematics* body, double dt,
                  int32_t scheme);

/* Advance the vortex set by dt around n_bodies bodies (1 .. PF_MAX_BODIES)
 * sharing one factor (Sec. 2.7, Eq. kuttasystem4): every edge of every body
 * (n_edges 0, 1 or 2; edge_bounded must be 0) releases one vortex per step
 * under the Kutta condition, placed by pf_step's rule from its own body's
 * surface; Kelvin's condition holds per body, body b >= 1 balancing the
 * vorticity it released and body 0 the rest of the flow's circulation (with
 * one body this is pf_step); a body without edges is circulation-constrained.
 * The free stream is bodies[0]'s.  scheme as pf_step, whose second stage
 * constrains every body's circulation.  The factor of the concatenated
 * surface is rebuilt when any body's pose changes (the last two poses are
 * kept).  The state's release history is per edge, edges in body order.
 * PF_ERR_ARG for an invalid body, PF_ERR_CAPACITY if the new vortices do
 * not fit. */
pf_status pf_step_multi(pf_plan plan, pf_state state, int32_t n_bodies, const pf_body_kinematics* bodies,
                        double dt, int32_t scheme);

/* Independent instances, one step each: pf_step for plans[i], states[i],
 * bodies[i] and step length dt[i] (host arrays, i < n), each enqueued on its
 * own plan's stream so instances on
 * distinct streams overlap on the device.  When the process runs with
 * CUDA_DEVICE_MAX_CONNECTIONS >= 32 (set before CUDA starts), a batch of more
 * than 8 distinct plans and states is enqueued from several host threads (up
 * to 16, on the caller's device), taking the instances in turn; otherwise,
 * and when a plan or a state appears twice, the calling thread enqueues the
 * instances in order.
 * Returns the first error met; after an error the instances not yet taken
 * are not stepped. */
pf_status pf_step_batch(int32_t n, pf_plan* plans, pf_state* states, const pf_body_kinematics* bodies,
                        const double* dt, int32_t scheme);

/* A batch of independent instances (plan, state, body, step length) whose
 * steps run as one CUDA graph: pf_step's method for each instance (Sec. 2.4),
 * captured once, the instances' kernels in parallel branches, so that one
 * step of every instance is one graph launch and no per-kernel host work.
 * The captured kernels read each instance's vortex count and last releases
 * from the state's device counts and are sized by its capacity, so the graph
 * serves every step until a state is full.
 * Requirements (else PF_ERR_ARG): n >= 1; plans[i] is the plan states[i] was
 * created with; plans and states distinct; no plan on the legacy default
 * stream or with timing on; each body fixed in time (amp = 0 or omega = 0,
 * or no body); dt[i] > 0; scheme 0 (Euler) or 1 (RK2).
 * Creation factors S at each body's pose where the state has no factor for
 * it, reserves every buffer a step of the full capacity uses, synchronises
 * the plans' streams and captures.  The batch copies dt and the kinematics
 * structs; the body arrays they point to must outlive it, and while it lives
 * its states must not be stepped around other bodies.  Each plan's surface
 * right-hand-side route (pf_plan_set_rhs_route) is chosen once, for the
 * state's capacity, as pf_step chooses it: a batch step is bitwise pf_step's.
 * PF_ERR_CUDA if the capture or the instantiation fails (pf_last_error of
 * plans[0] has the text). */
typedef struct pf_batch_s* pf_batch;
pf_status pf_batch_create(int32_t n, pf_plan* plans, pf_state* states, const pf_body_kinematics* bodies,
                          const double* dt, int32_t scheme, pf_batch* out);

/* nsteps steps of every instance: nsteps launches of the graph on the batch's
 * own stream, ordered after the work enqueued so far on every plan's stream
 * and before any enqueued there afterwards (pf_sync on a plan waits for them).
 * PF_ERR_CAPACITY, with nothing launched, if a state would overflow. */
pf_status pf_batch_step(pf_batch batch, int32_t nsteps);
pf_status pf_batch_destroy(pf_batch batch);

/* ------------------------------------------------------- request server */

/* Continuous batching of independent time-stepping requests on one GPU.
 * Requests are admitted in submission order while fewer than max_slots are
 * running and the device memory of the resident instances (their grids'
 * LGF tables and spectra, and per instance the plan workspaces, vortex bins,
 * state and Schur factor) stays within hbm_budget_bytes; an instance holds
 * a power-of-two number of vortices (at least 1024, at least the request's
 * capacity), and idle instances are kept for reuse by later requests of the
 * same grid up to that size and evicted least recently used first.  Every
 * admitted request runs on its own stream, all of its steps enqueued at
 * admission (for a body fixed in time, every step after the first as a launch
 * of one step captured into a CUDA graph, as pf_batch_*), so requests overlap
 * on the device.  The
 * kernels are deterministic and instances share no mutable data: a request's
 * result does not depend on what else is running.  A request waits in the
 * queue only while running requests hold what it needs: one that does not
 * fit the budget with nothing else resident finishes with PF_ERR_OOM, and a
 * CUDA error while admitting finishes the request at the head of the queue
 * with PF_ERR_CUDA and is returned by the call that met it. */
typedef struct pf_server_s* pf_server;

typedef struct {
    int32_t max_slots;
    int64_t hbm_budget_bytes;
    int32_t precision;           /* pf_precision of every instance */
} pf_server_config;

typedef struct {
    pf_grid_desc grid;           /* its precision field is ignored */
    pf_body_kinematics body;     /* ns = 0: no body; arrays are copied at submission */
    const double* X;             /* initial vortices (host, nv each), copied at submission */
    const double* Y;
    const double* Gam;
    int64_t nv;
    int64_t capacity;            /* >= nv (+ 2 nsteps for a body with two edges) */
    int32_t nsteps;
    double dt;
    int32_t scheme;              /* as pf_step */
} pf_request;

pf_status pf_server_create(const pf_server_config* cfg, pf_server* out);
pf_status pf_server_destroy(pf_server server);
/* Queue a request (admitting what fits) and return its ticket. */
pf_status pf_server_submit(pf_server server, const pf_request* req, int64_t* ticket);
/* Non-blocking progress: retire finished requests and admit queued ones.  Up
 * to max tickets of requests finished since the last call are written to
 * tickets (host), their number to n_done. */
pf_status pf_server_progress(pf_server server, int32_t max, int64_t* tickets, int32_t* n_done);
/* A finished request's final vortices (host arrays of at least nv entries; any
 * may be NULL), nv, and latency from submission to completion in seconds.
 * Returns the request's status; the request is then forgotten. */
pf_status pf_server_result(pf_server server, int64_t ticket, double* X, double* Y, double* Gam,
                           int64_t* nv, double* latency_s);
pf_status pf_server_stats(pf_server server, int32_t* queued, int32_t* active, int64_t* used_bytes);

/* ------------------------------------------------ allocation-free variant */

/* Regularization for callers that cannot allocate device memory: code running
 * where cudaMalloc is not allowed or not wanted (inside a host callback, under
 * a memory budget that forbids new allocations, or in a process whose
 * allocator is owned by someone else).  It computes exactly what
 * pf_regularize computes, with the same kernels, but needs no plan and makes
 * no allocation: its scratch (tile counters and offsets, 65536 per-vortex cell
 * records and up to 4 * 65536 binned records) is one static device array of
 * about 11.1 MiB inside this library, which every GPU that loads the library
 * holds until the process exits.  The paper has no counterpart; it is an
 * interface convenience.
 *
 *   desc          grid and precision, as for pf_plan_create (host pointer);
 *                 grids up to 2048 x 2048 nodes
 *   X, Y, Gam     nv doubles each (device); nv <= 65536, larger nv returns
 *                 PF_ERR_CAPACITY without doing anything
 *   w             real[nx*ny] output (device), fully overwritten
 *   out_of_domain optional device int64: receives the number of vortices whose
 *                 stencil left the grid (they are skipped); may be NULL
 *   status        optional device int32: receives, in stream order, the status
 *                 the work ended with: PF_OK, PF_ERR_OUT_OF_DOMAIN (see
 *                 out_of_domain; w holds the other vortices) or
 *                 PF_ERR_INTERNAL (a consistency check of the binning failed;
 *                 the affected tiles were skipped and w is not valid); may be
 *                 NULL
 *   stream        cudaStream_t to enqueue on (NULL = default stream)
 *
 * The return value covers what the host can check (arguments, capacity,
 * launch errors); the device-side outcome arrives through status.  The first
 * call on each device looks up the array's device address with
 * cudaGetSymbolAddress while that device is current, and caches it per device
 * (thread-safe); make that first call before any stream capture on the
 * device.  Calls after cudaDeviceReset on a device are not supported (the
 * cached address belongs to the old context).  All calls share the one array
 * and it keeps the previous call's contents, so calls whose work overlaps on
 * the GPU (different streams, or different host threads on one device) race
 * and must be serialised by the caller. */
pf_status pf_regularize_noalloc(const pf_grid_desc* desc, const double* X, const double* Y,
                                const double* Gam, int64_t nv, void* w, int64_t* out_of_domain,
                                int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GRIDPF_H */

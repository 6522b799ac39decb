/*
 * dg_swe.h -- C ABI of the GB300 (sm_103a) discontinuous Galerkin solver for
 * the shallow-water equations coupled to a regularized Bingham law.
 *
 * Method (arXiv 2301.11238): first-order system dU/dt + div F = div Q + S,
 * E = div G (Sec. 3, Eq. shallowR2/shallowR3) with U = (h, h u) (Eq. Uterm),
 * F (Eq. Fterm), Q = h sigma / rho (Eq. Qterm), S (Eq. Sterm) and the velocity
 * gradient E (Eq. gradientVel); stress sigma = sigma_N + sigma_B
 * (Eq. binghamR) with the regularizations of Sec. 4 (Eq. sigmaTwoA-C); DG weak
 * form per element (Sec. 5, Eq. WeakForm51/52) with the HLL flux for F
 * (Eq. HLLSolver), central fluxes for G and Q, and strong ghost-value
 * boundary conditions (Sec. 5.2).  Unknowns are the primitive variables
 * V = (h, u) and E (Sec. 5).
 *
 * Conventions
 *  - Every call returns dg_status and never aborts or throws.  On failure the
 *    context (if any) keeps a message readable with dg_swe_last_error().
 *  - The library never allocates device memory.  All device storage (state,
 *    geometry, operators, scratch) lives in one caller-provided workspace of
 *    dg_swe_workspace_size() bytes (dg_swe_set_workspace), so a caller's
 *    allocator (e.g. PyTorch's) owns it.  Host memory is allocated in
 *    dg_swe_init and released in dg_swe_destroy.
 *  - Kernels run on the stream set by dg_swe_set_stream (default stream 0).
 *    Calls that only enqueue work return DG_OK at enqueue; device-side errors
 *    (non-finite state) are latched in a device status word and reported by
 *    the next synchronizing call (dg_swe_get_state, dg_swe_run, dg_swe_sync).
 *  - Nodal layout: a field array is [field][element][node] in double
 *    precision, nodes contiguous.  Node j of an element is the equispaced
 *    reference node (line: r_i = -1 + 2i/p; triangle with vertices
 *    (-1,-1), (1,-1), (-1,1): (r, s) = (-1 + 2i/p, -1 + 2j/p), j outer,
 *    i = 0..p-j inner) mapped affinely onto the element (dg_swe_node_coords).
 *    V fields: h, u_1[, u_2].  E fields (2D): component 2*i + j holds
 *    E_ij = d u_j / d x_i; in 1D the single component du/dx.
 */
#ifndef DG_SWE_H
#define DG_SWE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,          /* invalid argument or unsupported combination     */
  DG_ERR_CUDA = 2,         /* a CUDA runtime call failed                      */
  DG_ERR_WORKSPACE = 3,    /* workspace missing, too small or misaligned      */
  DG_ERR_NONFINITE = 4,    /* the state became NaN/Inf (latched on device)    */
  DG_ERR_NEWTON = 5,       /* Newton did not converge (implicit integrator)   */
  DG_ERR_UNSUPPORTED = 6,  /* feature not available for this configuration    */
  DG_ERR_TIMEOUT = 7       /* a bounded in-kernel wait ran out (latched on
                              device; the step's results are not valid)      */
} dg_status;

typedef struct dg_swe_ctx dg_swe_ctx;

#define DG_SWE_MAX_BC 8

/* Boundary-condition modes (Sec. 5.2, ghost values V+ and E+ at boundary faces). */
enum { DG_BC_COPY = 0,       /* V+ = V- (homogeneous Neumann)                          */
       DG_BC_DIRICHLET = 1,  /* V+ = prescribed value                                  */
       DG_BC_WALL = 2 };     /* velocity slots only: u+ = u- - 2 (u-.n) n (extension)  */

/* Regularizations of the Bingham term (Sec. 4).  1-3 are the paper's;
 * 4 and 5 are extensions the paper does not define. */
enum { DG_REG_NONE = 0,       /* Newtonian: sigma_B = 0                                 */
       DG_REG_SMOOTH_MAX = 1, /* Eq. sigmaTwoA/AA                                       */
       DG_REG_LOCAL_QUAD = 2, /* Eq. sigmaTwoB; needs sigma0 = 0 or sigma0 >= 1/(2 beta) */
       DG_REG_TANH = 3,       /* Eq. sigmaTwoC                                          */
       DG_REG_EXP = 4,        /* 2 sigma0 (1 - exp(-m |E|)) sign E  (Papanastasiou)     */
       DG_REG_BIVISC = 5 };   /* min(2 gamma |E|, 2 sigma0) sign E  (bi-viscosity)      */

enum { DG_PREC_FP64 = 0,     /* state, fluxes and contractions in FP64                  */
       DG_PREC_FP32 = 1,     /* FP32 state and arithmetic; FP64 CFL and mass reductions */
       DG_PREC_FP32_TC = 2 };/* as DG_PREC_FP32, but on triangles of order 2 and 3 the
                                volume pass runs its three dense contractions (the
                                interpolation of the nodal fields to the volume points,
                                the test-function contraction of the pointwise fluxes of
                                Eq. WeakForm51 and the h-weighted mass matrix of the
                                primitive-variable time term, Appendix A) on the tensor
                                cores (tcgen05, TF32 operands split into high and low
                                parts, FP32 accumulation; about 22 significant bits per
                                operand against FP32's 24).  Elsewhere (1D, order 1) it equals
                                DG_PREC_FP32.  Results differ from DG_PREC_FP32 by
                                rounding only.                                           */

typedef struct {
  int32_t mode[7];   /* per slot: V fields (h, u_1[, u_2]) then E fields     */
  double value[7];   /* Dirichlet values per slot                            */
} dg_swe_bc;

typedef struct {
  int32_t dim;                  /* 1 (intervals) or 2 (triangles)                        */
  int64_t n_vertices;
  const double *coords;         /* host, [n_vertices][dim]                               */
  int64_t n_elements;
  const int32_t *elem_vertices; /* host, [n_elements][dim+1]; 1D: x1 > x0; 2D: CCW       */
  const int8_t *face_bc;        /* host, [n_elements][dim+1] or NULL (all 0): index into
                                   params.bc used where the face has no neighbour.
                                   Face f of a triangle joins vertices f and (f+1)%3;
                                   face 0 of an interval is its left end, face 1 its right */
  const double *bed;            /* host, nodal bed H [n_elements][Np] or NULL (flat)     */
} dg_swe_mesh;

typedef struct {
  double g, rho, alpha;         /* gravity, density, plane inclination (g_c = g cos a,
                                   g_s = g sin a; Eq. shallow2/3)                        */
  double eta, sigma0;           /* viscosity and yield stress (Eq. bingham)              */
  double gamma, beta, pap_m;    /* regularization parameters (Sec. 4); pap_m for DG_REG_EXP */
  double h_floor;               /* depth floor for wave speeds and the h-weighted mass   */
  double cfl;                   /* explicit step safety factor                           */
  int32_t precision;            /* DG_PREC_*                                             */
  int32_t n_bc;                 /* entries used in bc[] (>= 1)                           */
  dg_swe_bc bc[DG_SWE_MAX_BC];
  int32_t positivity;           /* 1: wet/dry mode (an extension: the paper leaves wet/dry
                                   fronts to future work, Sec. 7).  Each explicit stage is
                                   taken on the moments <N, U> of U = (h, h u), whose
                                   difference the time term of Eq. WeakForm7 holds:
                                   <N, U(y)> = c0 <N, U(V0)> + c1 (<N, U(Vs)> - dt r_V(Vs)).
                                   The new depth passes the depth limiter (per element,
                                   with hbar the cell average of h and m its minimum over
                                   the nodes, volume and face quadrature points: hbar <= 0
                                   gives h = 0; m < 0 < hbar scales h <- hbar + theta
                                   (h - hbar), theta = hbar / (hbar - m), Zhang-Shu
                                   scaling; cell averages kept), then the velocity solves
                                   M_h u = <psi, h u> with M_h = <psi, max(h, h_floor) psi>
                                   of the limited depth, and u = 0 where hbar < h_floor.
                                   Runs dam breaks onto dry beds (depth exactly 0), which
                                   the primitive stages cannot: they divide the momentum
                                   change by the stage's starting depth.  The stage is
                                   formed by a separate kernel after the volume pass (14
                                   launches per step instead of 11), in FP64, or in FP32
                                   for the elements of an FP32 context whose nodal depths
                                   are all at least 1000 h_floor; elements exactly dry
                                   and at rest with a zero residual stay so.  0: off (stages on V through dU/dV, Appendix A)   */
  double flow_index;            /* n of a Herschel-Bulkley viscous part (an extension; the
                                   paper's introduction cites the law, its scheme is
                                   Bingham): the Newtonian 2 eta (D + tr D I) becomes
                                   2 eta max(s, rate_floor)^(n-1) (D + tr D I), eta the
                                   consistency, s = ||D||_c / sqrt(2) (|E| in 1D).
                                   0 or 1: Newtonian (the paper); 0 < n < 1: shear
                                   thinning; other values DG_ERR_ARG                     */
  double rate_floor;            /* s below which the power-law viscosity is frozen
                                   (> 0 when 0 < flow_index < 1)                         */
} dg_swe_params;

typedef struct {
  int64_t steps;                /* time steps taken since the last set_state             */
  double t;                     /* simulated time                                        */
  double dt_last, dt_min, dt_max;
  double mass;                  /* sum over elements of the integral of h (FP64)         */
  double mass0;                 /* mass at set_state                                     */
  int32_t status;               /* latched device status (dg_status value)               */
} dg_swe_stats;

/* Builds the host-side reference operators, geometry and connectivity.
 * order p in {1,2,3}; regularization = DG_REG_*.  Copies every host input.
 * Errors: DG_ERR_ARG for bad sizes, non-conforming or wrongly oriented meshes,
 * boundary tags >= n_bc, or DG_REG_LOCAL_QUAD with 0 < sigma0 < 1/(2 beta). */
dg_status dg_swe_init(const dg_swe_mesh *mesh, int order, int regularization,
                      const dg_swe_params *params, dg_swe_ctx **out);

/* Device bytes the context needs (a multiple of 256). */
size_t dg_swe_workspace_size(const dg_swe_ctx *ctx);

/* Hands the context its device workspace (256-byte aligned, >= workspace
 * size, owned by the caller and kept alive until dg_swe_destroy) and uploads
 * geometry and operators on the context's stream.  DG_ERR_WORKSPACE if too
 * small or misaligned. */
dg_status dg_swe_set_workspace(dg_swe_ctx *ctx, void *dev_ptr, size_t bytes);

/* CUDA stream (cudaStream_t) for all later work; NULL = legacy default stream. */
dg_status dg_swe_set_stream(dg_swe_ctx *ctx, void *cuda_stream);

/* Physical node coordinates, host buffer [n_elements][Np][dim]. */
dg_status dg_swe_node_coords(const dg_swe_ctx *ctx, double *xyz);

/* Sizes: Np nodes per element, nV and nE fields, n_faces unique faces. */
dg_status dg_swe_sizes(const dg_swe_ctx *ctx, int64_t *n_elements, int32_t *np,
                       int32_t *nv, int32_t *ne, int64_t *n_faces);

/* Sets the nodal state V ([nV][K][Np] doubles; device pointer if on_device,
 * else host) and resets time, step count and the mass reference. */
dg_status dg_swe_set_state(dg_swe_ctx *ctx, const double *V, int on_device);

/* Copies the state V (and, if E is not NULL, the velocity gradient E of the
 * last evaluated stage) out, device or host pointers; synchronizes the stream
 * and reports a latched device error. */
dg_status dg_swe_get_state(dg_swe_ctx *ctx, double *V, double *E, int on_device);

/* One evaluation of the semi-discrete right-hand side at V_dev:
 * E-step (Eq. WeakForm52), face fluxes once per face, volume integrals,
 * lift and the primitive-variable mass solve <N, dU/dV N> dV/dt = -r_V
 * (Eq. WeakForm51 with dU/dV of Appendix A).  V_dev, dVdt_dev: device
 * [nV][K][Np] doubles; E_dev (or NULL): device [nE][K][Np].  Enqueued on the
 * context's stream; does not touch the context state. */
dg_status dg_swe_residual(dg_swe_ctx *ctx, const double *V_dev, double *dVdt_dev, double *E_dev);

/* One explicit SSP-RK3 (Shu-Osher) step of the state.  dt > 0 uses that
 * step; dt <= 0 computes the stable step on the device (FP64 min-reduction):
 *   dt = min_e cfl * dx_e / ((2p+1) lam_e + (2p+1)^2 * 2 nu / dx_e),
 * lam_e = max over nodes of |u| + sqrt(g_c max(h, h_floor)),
 * nu = (4 eta + max d sigma_B / dE) / rho.  If dt_taken is not NULL the
 * call synchronizes and returns the step. */
dg_status dg_swe_step(dg_swe_ctx *ctx, double dt, double *dt_taken);

/* Advances n_steps CFL-limited SSP-RK3 steps (t_end > 0 additionally stops
 * at t_end, which requires a host sync per step and is slower).  The steps
 * are replayed from a CUDA graph captured on first use.  Synchronizes, fills
 * stats (may be NULL) and reports a latched device error. */
dg_status dg_swe_run(dg_swe_ctx *ctx, int64_t n_steps, double t_end, dg_swe_stats *stats);

/* Enqueue-only form of dg_swe_run: replays n_steps CFL-limited SSP-RK3
 * steps from the CUDA graph (captured on first use on a private stream that
 * forks from and joins back into the context's stream) and returns without
 * synchronizing.  Device errors surface at the next synchronizing call. */
dg_status dg_swe_advance(dg_swe_ctx *ctx, int64_t n_steps);

/* Profiling aid: average device time in milliseconds of one launch of each
 * kernel of the explicit path, each launched n_iter times back to back on the
 * context's stream and timed with CUDA events: ms[0] E-step, ms[1] face flux,
 * ms[2] volume/lift/mass-solve/update (writes a scratch stage buffer, the
 * state is unchanged), ms[3] stable-step partial reduction, ms[4] mass
 * partial reduction.  Synchronizes. */
dg_status dg_swe_time_kernels(dg_swe_ctx *ctx, int n_iter, double *ms);

/* Enqueues the FP64 mass reduction and synchronizes; fills stats. */
dg_status dg_swe_sync(dg_swe_ctx *ctx, dg_swe_stats *stats);

/* Size of the library's static device scratch array used by
 * dg_swe_residual_static: 16 MiB, held on every GPU that loads the library
 * until the process exits. */
#define DG_SWE_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* Allocation-free variant of dg_swe_residual (the paper has no counterpart;
 * this is a deployment convenience).  It is meant for callers that must not
 * allocate device memory per call: a host application that reserved its whole
 * device-memory budget at start-up, or code on a latency-critical path where
 * cudaMalloc (which may synchronize the device) is off limits.  Same inputs,
 * outputs and result as dg_swe_residual, but the per-call scratch (E and the
 * face fluxes, plus FP32 staging buffers for DG_PREC_FP32 contexts) lives in a
 * file-scope __device__ array of DG_SWE_STATIC_SCRATCH_BYTES instead of the
 * workspace scratch region; the context's geometry and operators are still
 * read from its workspace.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).
 *  - Problems whose scratch need (dg_swe_static_scratch_need) exceeds the
 *    array are rejected with DG_ERR_ARG and a message giving both sizes.
 *  - Call it with the context's device current (the device that was current
 *    at dg_swe_set_workspace); with another device current it returns
 *    DG_ERR_ARG, since the array it would use belongs to that other device.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) for that device; make that first call before any
 *    CUDA stream capture.
 *  - All calls in the process share the one array, which keeps the contents
 *    of the last call; every word is written before it is read, so no
 *    clearing is needed.  Calls whose work overlaps on the GPU (different
 *    streams or contexts without ordering between them) race on the array
 *    and must be serialized by the caller. */
dg_status dg_swe_residual_static(dg_swe_ctx *ctx, const double *V_dev, double *dVdt_dev, double *E_dev);

/* Scratch bytes dg_swe_residual_static needs for this context. */
size_t dg_swe_static_scratch_need(const dg_swe_ctx *ctx);

/* Number of kernel launches one dg_swe_step enqueues (for launch accounting):
 * 11, or 14 in wet/dry mode (positivity). */
int32_t dg_swe_launches_per_step(const dg_swe_ctx *ctx);

const char *dg_swe_last_error(const dg_swe_ctx *ctx);
void dg_swe_destroy(dg_swe_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DG_SWE_H */

/*
 * dg_implicit.h -- the paper's own time integrator on the GPU: backward Euler
 * with Newton-Raphson on the monolithic (V, E) system, one-dimensional
 * (Sec. 5.1, Eq. WeakForm7 and Eq. Newton; tangent blocks of Appendix A).
 *
 * Per element the unknowns are x_e = [h (p+1 nodes), u (p+1 nodes),
 * E (m3+1 nodes)]: nodal values at equispaced points (E of degree m3 <= p;
 * m3 = 0 stores the element's constant).  The residual is
 *   R_V = (1/dt) <N_V, U(V^k) - U(V^{k-1})> + <N_V^-, F_bar.n> - <dN_V/dx, F>
 *         - <N_V^-, Q_bar.n> + <dN_V/dx, Q> - <N_V, S>
 *   R_E = <N_E, E> - <N_E^-, G_bar.n> + <dN_E/dx, G>
 * with the quadrature, fluxes and boundary ghosts of dg_swe.h.  The Jacobian
 * uses the Appendix A tangent terms with the HLL wave speeds held fixed; it
 * is block tridiagonal for a left-to-right ordered mesh (element e's right
 * neighbour is e + 1) and is solved by block Thomas elimination with partial
 * pivoting (the paper does not name its linear solver), either in FP64 or
 * factored in FP32 and refined in FP64 (linear_solver).  Newton stops when
 * ||R||_2 <= rtol ||R^0||_2, ||R||_2 <= atol or
 * ||dx||_inf <= xtol (1 + ||x||_inf), after at most max_it iterations
 * (the paper uses 10, Sec. 6).  Residual and Jacobian are FP64.
 *
 * The whole integration (time steps x Newton iterations: assembly, solve,
 * update, convergence test) runs in one persistent launch with one thread
 * block per instance.  Conventions (status, workspace, stream) follow
 * dg_swe.h.
 */
#ifndef DG_IMPLICIT_H
#define DG_IMPLICIT_H

#include "dg_swe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_implicit dg_implicit;

typedef struct {
  double dt;                 /* time step (> 0)                                   */
  int32_t m3;                /* degree of E, 0..order (-1: same as order)         */
  int32_t max_it;            /* Newton iterations per step (paper: 10)            */
  int32_t on_fail_continue;  /* 1: keep going after max_it (the paper's runs);
                                0: stop and report DG_ERR_NEWTON                  */
  double rtol, atol, xtol;   /* stopping rule above                               */
  int32_t linear_solver;     /* 0: FP64 block Thomas (partial pivoting);
                                1: FP32 block-Thomas factorization with two FP64
                                   iterative-refinement rounds (residual of the
                                   linear system in FP64); needs
                                   2(p+1) + m3 + 1 <= 10                           */
  int32_t n_gamma;           /* > 1: continuation in the regularization parameter
                                within every time step (Sec. 6.3): Newton is run in
                                turn for gamma_i = gamma0 + (i-1)(gamma - gamma0)
                                / (n_gamma - 1), i = 1..n_gamma, each stage from
                                the previous stage's solution; iterations of all
                                stages are counted; <= 1: plain Newton            */
  double gamma0;             /* first continuation value (> 0 when n_gamma > 1)   */
} dg_implicit_params;

typedef struct {
  int64_t steps;             /* completed time steps                              */
  int64_t newton_its;        /* Newton iterations summed over steps               */
  int64_t failed_steps;      /* steps that reached max_it without converging      */
  double t;                  /* simulated time                                    */
  double last_res;           /* ||R||_2 at the end of the last step               */
  int32_t last_its;          /* Newton iterations of the last step                */
  int32_t status;            /* latched dg_status                                 */
} dg_implicit_stats;

/* 1D mesh only (DG_ERR_UNSUPPORTED otherwise, if the mesh is not ordered
 * left to right, or for a Herschel-Bulkley viscous part, flow_index != 1,
 * which the Appendix A tangent does not cover).  Copies the host inputs. */
dg_status dg_implicit_init(const dg_swe_mesh *mesh, int order, int regularization,
                           const dg_swe_params *params, const dg_implicit_params *ip,
                           dg_implicit **out);
size_t dg_implicit_workspace_size(const dg_implicit *s);
dg_status dg_implicit_set_workspace(dg_implicit *s, void *dev_ptr, size_t bytes);
dg_status dg_implicit_set_stream(dg_implicit *s, void *cuda_stream);
/* Node coordinates of the V nodes [K][p+1] (host). */
dg_status dg_implicit_node_coords(const dg_implicit *s, double *x);
/* Sets V ([2][K][p+1] doubles) and computes the consistent E (R_E = 0);
 * resets time and counters. */
dg_status dg_implicit_set_state(dg_implicit *s, const double *V, int on_device);
/* V [2][K][p+1] and E [K][m3+1]; synchronizes. */
dg_status dg_implicit_get_state(dg_implicit *s, double *V, double *E, int on_device);
/* Advances n_steps backward-Euler steps in one persistent launch;
 * synchronizes and fills stats (may be NULL). */
dg_status dg_implicit_run(dg_implicit *s, int64_t n_steps, dg_implicit_stats *stats);
/* Active-region percentage (Sec. 6): 100/|Omega| int H(|E| - sigma0/gamma)
 * evaluated at the volume quadrature points; synchronizes. */
dg_status dg_implicit_active_percent(dg_implicit *s, double *pct);
const char *dg_implicit_last_error(const dg_implicit *s);
void dg_implicit_destroy(dg_implicit *s);

#ifdef __cplusplus
}
#endif
#endif /* DG_IMPLICIT_H */

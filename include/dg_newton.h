/*
 * dg_newton.h -- backward Euler with a Newton-Krylov solve for a dg_swe
 * context in one or two dimensions: the paper's time discretization (Sec.
 * 5.1, Eq. WeakForm7 and Eq. Newton) carried to the two-dimensional scheme,
 * for which the paper gives no tangent blocks (its Appendix A is 1D).
 *
 * The E equation of Eq. WeakForm7 is linear in E and u, so E = E(u) is the
 * E-step of dg_swe.h and the unknowns are the nodal V values only.  Per step
 * from V_old the library solves
 *   R(V) = (1/dt) <l_a, U(V) - U(V_old)> + r_V(V, E(V)) = 0
 * (U = (h, h u), Eq. Uterm; r_V the spatial residual of Eq. WeakForm51 with
 * the quadrature, fluxes and boundary ghosts of dg_swe.h; l_a the nodal
 * basis) by Newton: J dV = -R, V <- V + dV.  J dV is never formed: each
 * product is the directional difference (R(V + eps z) - R(V)) / eps with
 * eps = sqrt(1e-16) (1 + ||V||_2) / ||z||_2, inside restarted-free
 * GMRES(m) with right preconditioning by dt M(V)^{-1}, M(V) the
 * primitive-variable mass matrix of Appendix A (block lower triangular per
 * element), and classical Gram-Schmidt applied twice.  GMRES stops when its
 * residual estimate falls below krylov_rtol ||R||_2 or after krylov_dim
 * iterations; Newton stops when ||R||_2 <= max(rtol ||R^0||_2, atol) or
 * after max_newton iterations (the paper uses 10, Sec. 6).  Everything is
 * FP64; reductions run in a fixed order (run-to-run reproducible).
 *
 * Conventions (status codes, workspace, stream) follow dg_swe.h.  The state
 * is the context's (dg_swe_set_state / dg_swe_get_state); the context's E
 * and face-flux buffers are scratch during dg_newton_run.  The context's
 * time and step counters advance by dt per step.  The depth limiter of
 * dg_swe_params.positivity is not applied.
 */
#ifndef DG_NEWTON_H
#define DG_NEWTON_H

#include "dg_swe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_newton dg_newton;

typedef struct {
  double dt;                 /* time step (> 0)                                    */
  int32_t max_newton;        /* Newton iterations per step (>= 1; paper: 10)       */
  double rtol, atol;         /* Newton stopping rule above                         */
  int32_t krylov_dim;        /* GMRES basis size m, 1..64                          */
  double krylov_rtol;        /* GMRES stopping rule above (0 < krylov_rtol < 1)    */
  int32_t on_fail_continue;  /* 1: keep stepping after max_newton; 0: stop with
                                DG_ERR_NEWTON                                      */
} dg_newton_params;

typedef struct {
  int64_t steps;             /* completed backward-Euler steps                     */
  int64_t newton_its;        /* Newton iterations summed over steps                */
  int64_t krylov_its;        /* GMRES iterations summed over Newton iterations     */
  int64_t failed_steps;      /* steps that reached max_newton unconverged          */
  double t;                  /* simulated time of the context                      */
  double last_res;           /* ||R||_2 at the end of the last step                */
  int32_t last_newton;       /* Newton iterations of the last step                 */
  int32_t status;            /* latched dg_status                                  */
} dg_newton_stats;

/* Creates a solver for an FP64 context (DG_ERR_UNSUPPORTED for FP32).  The
 * context must outlive the solver.  DG_ERR_ARG for invalid parameters. */
dg_status dg_newton_init(dg_swe_ctx *ctx, const dg_newton_params *params, dg_newton **out);
/* Device bytes of the solver's own scratch (Krylov basis, work vectors). */
size_t dg_newton_workspace_size(const dg_newton *nk);
/* 256-byte aligned device buffer of at least that size, owned by the caller. */
dg_status dg_newton_set_workspace(dg_newton *nk, void *dev_ptr, size_t bytes);
/* n_steps backward-Euler steps on the context's stream; synchronizes (the
 * Krylov loop reads its reductions on the host) and fills stats (may be NULL).
 * DG_ERR_NEWTON when a step fails and on_fail_continue is 0; DG_ERR_NONFINITE
 * when a residual norm is not finite. */
dg_status dg_newton_run(dg_newton *nk, int64_t n_steps, dg_newton_stats *stats);
const char *dg_newton_last_error(const dg_newton *nk);
void dg_newton_destroy(dg_newton *nk);

#ifdef __cplusplus
}
#endif
#endif /* DG_NEWTON_H */

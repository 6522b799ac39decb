// Backward Euler + Newton-Raphson for the 1D scheme (Sec. 5.1, Appendix A):
// one persistent thread block per instance runs time steps x Newton
// iterations (assembly, block-Thomas solve, update, convergence test).
// See include/dg_implicit.h.
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dg_implicit.h"
#include "dg_ctx.h"
#include "dg_kernels.cuh"

using namespace dgswe;

namespace {

template <int P, int M3>
struct IS {
  static constexpr int NP = P + 1, NE = M3 + 1, NB = 2 * NP + NE, NQ = (3 * P + 1) / 2;
};

template <int P, int M3>
struct ImplOps {
  using S = IS<P, M3>;
  double Vq[S::NQ * S::NP], dVq[S::NQ * S::NP];   // l_a, dl_a/dr at volume points
  double VEq[S::NQ * S::NE], dVEq[S::NQ * S::NE]; // psi_c, dpsi_c/dr
  double wq[S::NQ];
  double lf[2 * S::NP], lEf[2 * S::NE];           // basis at r = -1 (face 0) and r = +1 (face 1)
};

struct ImplArgs {
  int K;
  double dt, inv_dt, gc, gs, rho_inv, eta, sigma0, gamma, beta, pap_m, h_floor;
  int reg;
  double rtol, atol, xtol;
  int max_it, on_fail_continue;
  int n_gamma;    // > 1: continuation in gamma within each time step (Sec. 6.3)
  double gamma0;
  int mixed;  // 1: FP32 block-Thomas factorization + FP64 iterative refinement
  BCEntry<double> bcL, bcR;
  double *X, *Uold, *R, *D, *L, *U, *W, *Y, *DX;
  float *Wf, *Af;    // mixed: W_e = A_e^-1 U_e and A_e^-1 per element (FP32)
  double *Rr, *Dx2;  // mixed: refinement residual and correction
  const double *J, *bed;
  double* red;  // per-block partials of the residual norm / dx norms
  dg_implicit_stats* st;
};

// sigma(E) and d sigma / dE in 1D (Eq. sigma11D, bingham1D regularized,
// Appendix A): sigma = (2 eta + phi(|E|)/(2|E|)) 2E, sigma' = 4 eta + phi'(|E|).
__device__ __forceinline__ void sigma1d(double e, const ImplArgs& a, double& sig, double& dsig) {
  Phys<double> ph{};
  ph.eta = a.eta;
  ph.sigma0 = a.sigma0;
  ph.gamma = a.gamma;
  ph.beta = a.beta;
  ph.half_inv_beta = 0.5 / a.beta;
  ph.pap_m = a.pap_m;
  ph.reg = a.reg;
  const double s = fabs(e);
  sig = (2.0 * a.eta + bingham_coef<double>(s, ph)) * 2.0 * e;
  double dp = 0.0;
  const double s0 = a.sigma0, g = a.gamma;
  if (a.reg != 0 && s0 != 0.0) {
    switch (a.reg) {
      case 1: {
        const double eps = 0.5 / a.beta, x = g * s - s0;
        const double mb = x >= eps ? x : (x <= -eps ? 0.0 : 0.5 * a.beta * (x + eps) * (x + eps));
        const double dmb = x >= eps ? 1.0 : (x <= -eps ? 0.0 : a.beta * (x + eps));
        const double den = mb + s0;
        dp = 2.0 * s0 * g / den - 2.0 * s0 * g * g * s * dmb / (den * den);
        break;
      }
      case 2: {
        const double eps = 0.5 / a.beta, x = g * s;
        dp = x >= s0 + eps ? 0.0 : (x <= s0 - eps ? 2.0 * g : 2.0 * a.beta * g * (s0 - x + eps));
        break;
      }
      case 3: {
        const double c = cosh(fmin(g * s, 350.0));
        dp = 2.0 * s0 * g / (c * c);
        break;
      }
      case 4: dp = 2.0 * s0 * a.pap_m * exp(-a.pap_m * s); break;
      case 5: dp = g * s < s0 ? 2.0 * g : 0.0; break;
    }
  }
  dsig = 4.0 * a.eta + dp;
}

__device__ __forceinline__ double block_sum(double v, double* sred) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sred[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sred[i];
  return t;
}

__device__ __forceinline__ double block_max(double v, double* sred) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sred[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sred[i]);
  return t;
}

// Residual and Jacobian blocks of element e at X (thread per element).
// Returns the element's squared residual norm.
template <int P, int M3>
__device__ double assemble(int e, const ImplArgs& a, const ImplOps<P, M3>& o) {
  using S = IS<P, M3>;
  constexpr int NP = S::NP, NE = S::NE, NB = S::NB, NQ = S::NQ;
  const int K = a.K;
  const double* x = a.X + (size_t)e * NB;
  const double J = a.J[e];
  double h[NP], u[NP], E[NE];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    h[i] = x[i];
    u[i] = x[NP + i];
  }
#pragma unroll
  for (int i = 0; i < NE; ++i) E[i] = x[2 * NP + i];
  // ---- pointwise quantities at volume points
  double qh[NQ], qu[NQ], qs[NQ], qds[NQ], qdH[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double hh = 0, uu = 0, ee = 0, dH = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      hh += o.Vq[q * NP + i] * h[i];
      uu += o.Vq[q * NP + i] * u[i];
      if (a.bed) dH += o.dVq[q * NP + i] * a.bed[(size_t)e * NP + i];
    }
#pragma unroll
    for (int c = 0; c < NE; ++c) ee += o.VEq[q * NE + c] * E[c];
    qh[q] = hh;
    qu[q] = uu;
    sigma1d(ee, a, qs[q], qds[q]);
    qdH[q] = dH / J;
  }
  // ---- face data: traces, fluxes and their derivatives (frozen HLL speeds)
  double Fh[2], Fu[2], Gb[2];              // F_bar.n (h, u rows incl. -Q_bar.n), G_bar.n
  double Am[2][2][2], Ap[2][2][2];         // d flux(h,u rows)/d (h,u) of - and + side
  double BEm[2], BEp[2], GVm[2], GVp[2];   // d u-row/dE-, dE+;  d(-Gbar n)/du-, du+
  int nb_e[2];
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const double n = f == 0 ? -1.0 : 1.0;
    double hm = 0, um = 0, em = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      hm += o.lf[f * NP + i] * h[i];
      um += o.lf[f * NP + i] * u[i];
    }
#pragma unroll
    for (int c = 0; c < NE; ++c) em += o.lEf[f * NE + c] * E[c];
    double hp, up, ep, dVh = 1.0, dVu = 1.0, dEp = 1.0;
    const int e2 = f == 0 ? e - 1 : e + 1;
    if (e2 >= 0 && e2 < K) {
      const double* x2 = a.X + (size_t)e2 * NB;
      const int f2 = 1 - f;
      hp = up = ep = 0.0;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        hp += o.lf[f2 * NP + i] * x2[i];
        up += o.lf[f2 * NP + i] * x2[NP + i];
      }
#pragma unroll
      for (int c = 0; c < NE; ++c) ep += o.lEf[f2 * NE + c] * x2[2 * NP + c];
      nb_e[f] = e2;
    } else {
      const BCEntry<double>& b = f == 0 ? a.bcL : a.bcR;
      hp = b.mode[0] == 1 ? b.val[0] : hm;
      dVh = b.mode[0] == 1 ? 0.0 : 1.0;
      if (b.mode[1] == 1) {
        up = b.val[1];
        dVu = 0.0;
      } else if (b.mode[1] == 2) {
        up = -um;
        dVu = -1.0;
      } else {
        up = um;
      }
      ep = b.mode[2] == 1 ? b.val[2] : em;
      dEp = b.mode[2] == 1 ? 0.0 : 1.0;
      nb_e[f] = -1;
    }
    const double cm = sqrt(a.gc * fmax(hm, a.h_floor)), cp = sqrt(a.gc * fmax(hp, a.h_floor));
    const double unm = um * n, unp = up * n;
    const double SL = fmin(unm - cm, unp - cp), SR = fmax(unm + cm, unp + cp);
    const double Fm0 = hm * unm, Fm1 = (hm * um * um + 0.5 * a.gc * hm * hm) * n;
    const double Fp0 = hp * unp, Fp1 = (hp * up * up + 0.5 * a.gc * hp * hp) * n;
    const double dFm[2][2] = {{um * n, hm * n}, {(um * um + a.gc * hm) * n, 2.0 * hm * um * n}};
    const double dFp[2][2] = {{up * n, hp * n}, {(up * up + a.gc * hp) * n, 2.0 * hp * up * n}};
    const double dUm[2][2] = {{1.0, 0.0}, {um, hm}};
    const double dUp[2][2] = {{1.0, 0.0}, {up, hp}};
    double F0, F1;
    if (SL >= 0.0) {
      F0 = Fm0;
      F1 = Fm1;
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          Am[f][r][c] = dFm[r][c];
          Ap[f][r][c] = 0.0;
        }
    } else if (SR <= 0.0) {
      F0 = Fp0;
      F1 = Fp1;
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          Am[f][r][c] = 0.0;
          Ap[f][r][c] = dFp[r][c];
        }
    } else {
      const double inv = 1.0 / (SR - SL);
      F0 = (SR * Fm0 - SL * Fp0 + SL * SR * (hp - hm)) * inv;
      F1 = (SR * Fm1 - SL * Fp1 + SL * SR * (hp * up - hm * um)) * inv;
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          Am[f][r][c] = (SR * dFm[r][c] - SL * SR * dUm[r][c]) * inv;
          Ap[f][r][c] = (-SL * dFp[r][c] + SL * SR * dUp[r][c]) * inv;
        }
    }
    double sm, dsm, sp, dsp;
    sigma1d(em, a, sm, dsm);
    sigma1d(ep, a, sp, dsp);
    Fh[f] = F0;
    Fu[f] = F1 - 0.5 * (hm * sm + hp * sp) * a.rho_inv * n;
    Gb[f] = 0.5 * (um + up) * n;
    Am[f][1][0] -= 0.5 * sm * a.rho_inv * n;
    Ap[f][1][0] -= 0.5 * sp * a.rho_inv * n;
    BEm[f] = -0.5 * hm * dsm * a.rho_inv * n;
    BEp[f] = -0.5 * hp * dsp * a.rho_inv * n;
    GVm[f] = -0.5 * n;
    GVp[f] = -0.5 * n;
    // chain rule through boundary ghosts (dV+/dV- diagonal)
    if (nb_e[f] < 0) {
      for (int r = 0; r < 2; ++r) {
        Ap[f][r][0] *= dVh;
        Ap[f][r][1] *= dVu;
      }
      BEp[f] *= dEp;
      GVp[f] *= dVu;
    }
  }
  // ---- residual
  double Rl[NB];
  const double* uo = a.Uold + (size_t)e * 2 * NP;
  double nrm = 0.0;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    double rh = 0, ru = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const double w = o.wq[q], l = o.Vq[q * NP + i], dl = o.dVq[q * NP + i];
      rh += w * J * l * qh[q] * a.inv_dt - w * dl * qh[q] * qu[q];
      ru += w * J * l * qh[q] * qu[q] * a.inv_dt
            + w * dl * (qh[q] * qs[q] * a.rho_inv - (qh[q] * qu[q] * qu[q] + 0.5 * a.gc * qh[q] * qh[q]))
            + w * J * l * (a.gs * qh[q] + a.gc * qh[q] * qdH[q]);
    }
    rh -= uo[i] * a.inv_dt;
    ru -= uo[NP + i] * a.inv_dt;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      rh += o.lf[f * NP + i] * Fh[f];
      ru += o.lf[f * NP + i] * Fu[f];
    }
    Rl[i] = rh;
    Rl[NP + i] = ru;
  }
#pragma unroll
  for (int c = 0; c < NE; ++c) {
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double ee = 0.0;
#pragma unroll
      for (int d = 0; d < NE; ++d) ee += o.VEq[q * NE + d] * E[d];
      r += o.wq[q] * J * o.VEq[q * NE + c] * ee + o.wq[q] * o.dVEq[q * NE + c] * qu[q];
    }
#pragma unroll
    for (int f = 0; f < 2; ++f) r -= o.lEf[f * NE + c] * Gb[f];
    Rl[2 * NP + c] = r;
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    a.R[(size_t)e * NB + i] = Rl[i];
    nrm += Rl[i] * Rl[i];
  }
  // ---- Jacobian blocks: D (own), L (left neighbour), U (right neighbour)
  double* Dm = a.D + (size_t)e * NB * NB;
  double* Lm = a.L + (size_t)e * NB * NB;
  double* Um = a.U + (size_t)e * NB * NB;
  for (int r = 0; r < NB; ++r) {
    const int rb = r < NP ? 0 : (r < 2 * NP ? 1 : 2);  // row block: h, u, E
    const int ri = rb < 2 ? r - rb * NP : r - 2 * NP;
    for (int c = 0; c < NB; ++c) {
      const int cb = c < NP ? 0 : (c < 2 * NP ? 1 : 2);
      const int ci = cb < 2 ? c - cb * NP : c - 2 * NP;
      double dv = 0.0, lv = 0.0, uv = 0.0;
      for (int q = 0; q < NQ; ++q) {
        const double w = o.wq[q];
        const double lr = rb < 2 ? o.Vq[q * NP + ri] : o.VEq[q * NE + ri];
        const double dlr = rb < 2 ? o.dVq[q * NP + ri] : o.dVEq[q * NE + ri];
        const double lc = cb < 2 ? o.Vq[q * NP + ci] : o.VEq[q * NE + ci];
        const double hq = qh[q], uq = qu[q];
        if (rb == 0 && cb == 0) dv += w * J * lr * lc * a.inv_dt - w * dlr * uq * lc;
        else if (rb == 0 && cb == 1) dv += -w * dlr * hq * lc;
        else if (rb == 1 && cb == 0)
          dv += w * J * lr * uq * lc * a.inv_dt - w * dlr * (uq * uq + a.gc * hq) * lc + w * dlr * qs[q] * a.rho_inv * lc
                + w * J * lr * (a.gs + a.gc * qdH[q]) * lc;
        else if (rb == 1 && cb == 1) dv += w * J * lr * hq * lc * a.inv_dt - w * dlr * 2.0 * hq * uq * lc;
        else if (rb == 1 && cb == 2) dv += w * dlr * hq * qds[q] * a.rho_inv * lc;
        else if (rb == 2 && cb == 2) dv += w * J * lr * lc;
        else if (rb == 2 && cb == 1) dv += w * dlr * lc;
      }
      for (int f = 0; f < 2; ++f) {
        const double fr = rb < 2 ? o.lf[f * NP + ri] : o.lEf[f * NE + ri];
        const double fcm = cb < 2 ? o.lf[f * NP + ci] : o.lEf[f * NE + ci];
        const int f2 = 1 - f;
        const double fcp = cb < 2 ? o.lf[f2 * NP + ci] : o.lEf[f2 * NE + ci];
        double vm = 0.0, vp = 0.0;
        if (rb < 2 && cb < 2) {
          vm = Am[f][rb][cb];
          vp = Ap[f][rb][cb];
        } else if (rb == 1 && cb == 2) {
          vm = BEm[f];
          vp = BEp[f];
        } else if (rb == 2 && cb == 1) {
          vm = GVm[f];
          vp = GVp[f];
        }
        dv += fr * fcm * vm;
        if (nb_e[f] < 0) {
          dv += fr * fcm * vp;  // ghost depends on this element's own trace
        } else if (f == 0) {
          lv += fr * fcp * vp;
        } else {
          uv += fr * fcp * vp;
        }
      }
      Dm[r * NB + c] = dv;
      Lm[r * NB + c] = lv;
      Um[r * NB + c] = uv;
    }
  }
  return nrm;
}

// Block Thomas elimination with one warp: lane c owns column c of the
// augmented block [A | U_e | b] (2 NB + 1 <= 32 columns); Gauss-Jordan with
// partial pivoting by shuffles.  Solves J dx = -R; writes dx to a.DX.
template <int NB>
__device__ void thomas_warp(int K, const ImplArgs& a) {
  const int lane = threadIdx.x & 31;
  double col[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) col[r] = 0.0;
  for (int e = 0; e < K; ++e) {
    const double* D = a.D + (size_t)e * NB * NB;
    const double* L = a.L + (size_t)e * NB * NB;
    const double* U = a.U + (size_t)e * NB * NB;
    // previous W_{e-1} column (lane NB + c) for lanes c < NB; y_{e-1} stays on lane 2 NB
    double prev[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) prev[j] = __shfl_sync(0xffffffffu, col[j], lane < NB ? NB + lane : lane);
    double nc[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      double v = 0.0;
      if (lane < NB) v = D[r * NB + lane];
      else if (lane < 2 * NB) v = U[r * NB + (lane - NB)];
      else if (lane == 2 * NB) v = -a.R[(size_t)e * NB + r];
      if (e > 0 && (lane < NB || lane == 2 * NB)) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) s += L[r * NB + j] * prev[j];
        v -= s;
      }
      nc[r] = v;
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) col[r] = nc[r];
    // Gauss-Jordan on the augmented block
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      int piv = k;
      double best = fabs(col[k]);
#pragma unroll
      for (int r = k + 1; r < NB; ++r)
        if (fabs(col[r]) > best) {
          best = fabs(col[r]);
          piv = r;
        }
      piv = __shfl_sync(0xffffffffu, piv, k);
#pragma unroll
      for (int r = k + 1; r < NB; ++r)
        if (r == piv) {
          const double t = col[k];
          col[k] = col[r];
          col[r] = t;
        }
      const double pv = __shfl_sync(0xffffffffu, col[k], k);
      col[k] = col[k] / pv;
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        if (r == k) continue;
        const double fct = __shfl_sync(0xffffffffu, col[r], k);
        col[r] -= fct * col[k];
      }
    }
    // store W_e (lanes NB..2NB-1, column-major) and y_e (lane 2NB)
    if (lane >= NB && lane <= 2 * NB) {
      double* dst = lane < 2 * NB ? a.W + (size_t)e * NB * NB + (size_t)(lane - NB) * NB : a.Y + (size_t)e * NB;
#pragma unroll
      for (int r = 0; r < NB; ++r) dst[r] = col[r];
    }
  }
  __syncwarp();
  // back substitution: dx_{K-1} = y_{K-1}; dx_e = y_e - W_e dx_{e+1}
  double nxt[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) nxt[r] = 0.0;
  for (int e = K - 1; e >= 0; --e) {
    double v = 0.0;
    if (lane < NB) {
      v = a.Y[(size_t)e * NB + lane];
      if (e < K - 1) {
        const double* W = a.W + (size_t)e * NB * NB;
#pragma unroll
        for (int j = 0; j < NB; ++j) v -= W[j * NB + lane] * nxt[j];
      }
      a.DX[(size_t)e * NB + lane] = v;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) nxt[j] = __shfl_sync(0xffffffffu, v, j);
  }
}

// Mixed-precision block Thomas, factorization (one warp): lane c owns
// column c of [A_e | U_e | I] in FP32 (3 NB <= 32 columns) with
// A_e = D_e - L_e W_{e-1}; Gauss-Jordan leaves W_e = A_e^-1 U_e on lanes
// NB..2NB-1 and A_e^-1 on lanes 2NB..3NB-1, both stored.
template <int NB>
__device__ void thomas_factor_f32(int K, const ImplArgs& a) {
  const int lane = threadIdx.x & 31;
  float col[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) col[r] = 0.f;
  for (int e = 0; e < K; ++e) {
    const double* D = a.D + (size_t)e * NB * NB;
    const double* L = a.L + (size_t)e * NB * NB;
    const double* U = a.U + (size_t)e * NB * NB;
    float prev[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) prev[j] = __shfl_sync(0xffffffffu, col[j], lane < NB ? NB + lane : lane);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      float v = 0.f;
      if (lane < NB) {
        v = (float)D[r * NB + lane];
        if (e > 0) {
          float sacc = 0.f;
#pragma unroll
          for (int j = 0; j < NB; ++j) sacc += (float)L[r * NB + j] * prev[j];
          v -= sacc;
        }
      } else if (lane < 2 * NB) {
        v = (float)U[r * NB + (lane - NB)];
      } else if (lane < 3 * NB) {
        v = (r == lane - 2 * NB) ? 1.f : 0.f;
      }
      col[r] = v;
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      int piv = k;
      float best = fabsf(col[k]);
#pragma unroll
      for (int r = k + 1; r < NB; ++r)
        if (fabsf(col[r]) > best) {
          best = fabsf(col[r]);
          piv = r;
        }
      piv = __shfl_sync(0xffffffffu, piv, k);
#pragma unroll
      for (int r = k + 1; r < NB; ++r)
        if (r == piv) {
          const float t = col[k];
          col[k] = col[r];
          col[r] = t;
        }
      const float pv = __shfl_sync(0xffffffffu, col[k], k);
      col[k] = col[k] / pv;
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        if (r == k) continue;
        const float fct = __shfl_sync(0xffffffffu, col[r], k);
        col[r] -= fct * col[k];
      }
    }
    if (lane >= NB && lane < 3 * NB) {
      float* dst = lane < 2 * NB ? a.Wf + ((size_t)e * NB + (lane - NB)) * NB
                                 : a.Af + ((size_t)e * NB + (lane - 2 * NB)) * NB;
#pragma unroll
      for (int r = 0; r < NB; ++r) dst[r] = col[r];  // column-major blocks
    }
  }
}

// Solve J x = b with the stored FP32 factors (one warp; lane r < NB owns row
// r): forward y_e = A_e^-1 (b_e - L_e y_{e-1}), back x_e = y_e - W_e x_{e+1}.
// b and x are FP64 arrays [K][NB]; y is kept in a.Y.
template <int NB>
__device__ void thomas_apply_f32(int K, const ImplArgs& a, const double* b, double* x) {
  const int lane = threadIdx.x & 31;
  float yp[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) yp[j] = 0.f;
  for (int e = 0; e < K; ++e) {
    float t = 0.f;
    if (lane < NB) {
      t = (float)b[(size_t)e * NB + lane];
      if (e > 0) {
        const double* L = a.L + (size_t)e * NB * NB + (size_t)lane * NB;
#pragma unroll
        for (int j = 0; j < NB; ++j) t -= (float)L[j] * yp[j];
      }
    }
    float tt[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) tt[j] = __shfl_sync(0xffffffffu, t, j);
    float y = 0.f;
    if (lane < NB) {
      const float* Ai = a.Af + (size_t)e * NB * NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) y += Ai[j * NB + lane] * tt[j];
      a.Y[(size_t)e * NB + lane] = (double)y;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) yp[j] = __shfl_sync(0xffffffffu, y, j);
  }
  __syncwarp();
  float nx[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) nx[j] = 0.f;
  for (int e = K - 1; e >= 0; --e) {
    float v = 0.f;
    if (lane < NB) {
      v = (float)a.Y[(size_t)e * NB + lane];
      if (e < K - 1) {
        const float* Wm = a.Wf + (size_t)e * NB * NB;
#pragma unroll
        for (int j = 0; j < NB; ++j) v -= Wm[j * NB + lane] * nx[j];
      }
      x[(size_t)e * NB + lane] = (double)v;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) nx[j] = __shfl_sync(0xffffffffu, v, j);
  }
}

// FP64 residual of the linear system, r = -R - J dx (block tridiagonal), all threads.
template <int NB>
__device__ void linear_residual_f64(int K, const ImplArgs& a) {
  for (int i = threadIdx.x; i < K * NB; i += blockDim.x) {
    const int e = i / NB, r = i - e * NB;
    double v = -a.R[i];
    const double* D = a.D + (size_t)e * NB * NB + (size_t)r * NB;
    const double* x = a.DX + (size_t)e * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) v -= D[j] * x[j];
    if (e > 0) {
      const double* L = a.L + (size_t)e * NB * NB + (size_t)r * NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) v -= L[j] * x[j - NB];
    }
    if (e < K - 1) {
      const double* U = a.U + (size_t)e * NB * NB + (size_t)r * NB;
#pragma unroll
      for (int j = 0; j < NB; ++j) v -= U[j] * x[j + NB];
    }
    a.Rr[i] = v;
  }
}

constexpr int kRefinements = 2;

// Newton iteration for one time level (and one continuation stage): returns
// the iteration count, whether it converged and max |x|.
template <int P, int M3>
__device__ void newton_solve(const ImplArgs& a, const ImplOps<P, M3>& o, double* sred, int& its_out,
                             bool& conv_out, double& xmax_out) {
  using S = IS<P, M3>;
  constexpr int NB = S::NB;
  const int K = a.K;
  double r0 = 0.0, dxmax = 0.0, xmax = 0.0;
  int its = 0;
  bool conv = false;
  for (int it = 0;; ++it) {
    double part = 0.0;
    for (int e = threadIdx.x; e < K; e += blockDim.x) part += assemble<P, M3>(e, a, o);
    const double rn = sqrt(block_sum(part, sred));
    if (it == 0) {
      r0 = rn;
      if (rn <= a.atol) {
        conv = true;
        its = 0;
        break;
      }
    } else if (rn <= a.rtol * r0 || rn <= a.atol || dxmax <= a.xtol * (1.0 + xmax)) {
      conv = true;
      its = it;
      break;
    }
    if (it == a.max_it || !(rn == rn)) {
      its = it;
      break;
    }
    __syncthreads();
    if constexpr (3 * NB <= 32) {
      if (a.mixed) {
        // -R into Rr, FP32 factor + solve, then FP64 residual / correction rounds
        for (int i = threadIdx.x; i < K * NB; i += blockDim.x) a.Rr[i] = -a.R[i];
        __syncthreads();
        if (threadIdx.x < 32) {
          thomas_factor_f32<NB>(K, a);
          __syncwarp();
          thomas_apply_f32<NB>(K, a, a.Rr, a.DX);
        }
        __syncthreads();
        for (int ref = 0; ref < kRefinements; ++ref) {
          linear_residual_f64<NB>(K, a);
          __syncthreads();
          if (threadIdx.x < 32) thomas_apply_f32<NB>(K, a, a.Rr, a.Dx2);
          __syncthreads();
          for (int i = threadIdx.x; i < K * NB; i += blockDim.x) a.DX[i] += a.Dx2[i];
          __syncthreads();
        }
      } else {
        if (threadIdx.x < 32) thomas_warp<NB>(K, a);
        __syncthreads();
      }
    } else {
      if (threadIdx.x < 32) thomas_warp<NB>(K, a);
      __syncthreads();
    }
    double dm = 0.0, xm = 0.0;
    for (int i = threadIdx.x; i < K * NB; i += blockDim.x) {
      const double d = a.DX[i];
      const double xn = a.X[i] + d;
      a.X[i] = xn;
      dm = fmax(dm, fabs(d));
      xm = fmax(xm, fabs(xn));
    }
    dxmax = block_max(dm, sred);
    xmax = block_max(xm, sred);
    __syncthreads();
  }
  __syncthreads();
  its_out = its;
  conv_out = conv;
  xmax_out = xmax;
}

template <int P, int M3>
__global__ void __launch_bounds__(256) implicit_kernel(ImplArgs a, ImplOps<P, M3> o, long long n_steps) {
  using S = IS<P, M3>;
  constexpr int NP = S::NP, NB = S::NB, NQ = S::NQ;
  __shared__ double sred[32];
  const int K = a.K;
  for (long long step = 0; step < n_steps; ++step) {
    // <N_V, U(V^{k-1})>
    for (int e = threadIdx.x; e < K; e += blockDim.x) {
      const double* x = a.X + (size_t)e * NB;
      const double J = a.J[e];
      for (int i = 0; i < NP; ++i) {
        double s0 = 0, s1 = 0;
        for (int q = 0; q < NQ; ++q) {
          double hh = 0, uu = 0;
          for (int j = 0; j < NP; ++j) {
            hh += o.Vq[q * NP + j] * x[j];
            uu += o.Vq[q * NP + j] * x[NP + j];
          }
          s0 += o.wq[q] * J * o.Vq[q * NP + i] * hh;
          s1 += o.wq[q] * J * o.Vq[q * NP + i] * hh * uu;
        }
        a.Uold[(size_t)e * 2 * NP + i] = s0;
        a.Uold[(size_t)e * 2 * NP + NP + i] = s1;
      }
    }
    __syncthreads();
    // continuation in gamma (Sec. 6.3): gamma_i = gamma0 + (i-1)(gamma-gamma0)/(n_gamma-1)
    const int ng = a.n_gamma > 1 ? a.n_gamma : 1;
    int its = 0;
    bool conv = true;
    double xmax = 0.0;
    for (int ic = 0; ic < ng; ++ic) {
      ImplArgs b = a;
      if (ng > 1) b.gamma = a.gamma0 + ic * (a.gamma - a.gamma0) / (ng - 1);
      int it_s;
      bool cv_s;
      newton_solve<P, M3>(b, o, sred, it_s, cv_s, xmax);
      its += it_s;
      conv = conv && cv_s;
    }
    if (threadIdx.x == 0) {
      dg_implicit_stats& st = *a.st;
      st.steps += 1;
      st.t += a.dt;
      st.newton_its += its;
      st.last_its = its;
      if (!conv) st.failed_steps += 1;
      if (!(xmax == xmax)) st.status = DG_ERR_NONFINITE;
      else if (!conv && !a.on_fail_continue) st.status = DG_ERR_NEWTON;
    }
    __syncthreads();
    if (a.st->status != 0) break;
  }
}

// E consistent with V (R_E = 0; element-local solve of <N_E, N_E> E = rhs),
// thread per element.  Also the active-region indicator per element.
template <int P, int M3>
__global__ void init_E_kernel(ImplArgs a, ImplOps<P, M3> o, const double* __restrict__ MEinv) {
  using S = IS<P, M3>;
  constexpr int NP = S::NP, NE = S::NE, NB = S::NB, NQ = S::NQ;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.K) return;
  double* x = a.X + (size_t)e * NB;
  const double J = a.J[e];
  double rhs[NE];
#pragma unroll
  for (int c = 0; c < NE; ++c) {
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double uu = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) uu += o.Vq[q * NP + j] * x[NP + j];
      r -= o.wq[q] * o.dVEq[q * NE + c] * uu;
    }
    rhs[c] = r;
  }
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const double n = f == 0 ? -1.0 : 1.0;
    double um = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) um += o.lf[f * NP + j] * x[NP + j];
    double up;
    const int e2 = f == 0 ? e - 1 : e + 1;
    if (e2 >= 0 && e2 < a.K) {
      up = 0.0;
#pragma unroll
      for (int j = 0; j < NP; ++j) up += o.lf[(1 - f) * NP + j] * a.X[(size_t)e2 * NB + NP + j];
    } else {
      const BCEntry<double>& b = f == 0 ? a.bcL : a.bcR;
      up = b.mode[1] == 1 ? b.val[1] : (b.mode[1] == 2 ? -um : um);
    }
#pragma unroll
    for (int c = 0; c < NE; ++c) rhs[c] += o.lEf[f * NE + c] * 0.5 * (um + up) * n;
  }
  // written to a scratch row first: neighbours read this element's u only
#pragma unroll
  for (int c = 0; c < NE; ++c) {
    double v = 0.0;
#pragma unroll
    for (int d = 0; d < NE; ++d) v += MEinv[c * NE + d] * rhs[d];
    a.DX[(size_t)e * NB + c] = v / J;
  }
}

template <int P, int M3>
__global__ void commit_E_kernel(ImplArgs a) {
  using S = IS<P, M3>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.K) return;
#pragma unroll
  for (int c = 0; c < S::NE; ++c) a.X[(size_t)e * S::NB + 2 * S::NP + c] = a.DX[(size_t)e * S::NB + c];
}

template <int P, int M3>
__global__ void active_kernel(ImplArgs a, ImplOps<P, M3> o, double* out) {
  using S = IS<P, M3>;
  constexpr int NE = S::NE, NB = S::NB, NQ = S::NQ;
  __shared__ double sred[32];
  double act = 0.0, tot = 0.0;
  const double thr = a.gamma > 0 ? a.sigma0 / a.gamma : 0.0;
  for (int e = threadIdx.x; e < a.K; e += blockDim.x) {
    const double* x = a.X + (size_t)e * NB + 2 * S::NP;
    for (int q = 0; q < NQ; ++q) {
      double ee = 0.0;
      for (int c = 0; c < NE; ++c) ee += o.VEq[q * NE + c] * x[c];
      const double w = o.wq[q] * a.J[e];
      tot += w;
      if (fabs(ee) - thr >= 0.0) act += w;
    }
  }
  const double A = block_sum(act, sred);
  const double T = block_sum(tot, sred);
  if (threadIdx.x == 0) *out = 100.0 * A / T;
}

struct ImplDrv {
  virtual ~ImplDrv() = default;
  virtual void run(dg_implicit* s, long long n, cudaStream_t st) = 0;
  virtual void init_E(dg_implicit* s, cudaStream_t st) = 0;
  virtual void active(dg_implicit* s, double* out, cudaStream_t st) = 0;
};

}  // namespace

struct dg_implicit {
  int p = 0, m3 = 0, reg = 0;
  int64_t K = 0;
  dg_swe_params prm{};
  dg_implicit_params ip{};
  std::vector<double> J, bed, node_x, MEinv;
  std::vector<double> Vq, dVq, VEq, dVEq, wq, lf, lEf;
  BCEntry<double> bcL{}, bcR{};
  bool has_bed = false;
  size_t ws_need = 0;
  char* ws = nullptr;
  struct {
    size_t X, Uold, R, D, L, U, W, Y, DX, J, bed, red, st, MEinv, act, Wf, Af, Rr, Dx2;
  } off{};
  cudaStream_t stream = nullptr;
  std::unique_ptr<ImplDrv> drv;
  std::string err;
  template <typename T>
  T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
  int nb() const { return 2 * (p + 1) + (m3 + 1); }
};

namespace {

dg_status ifail(dg_implicit* s, dg_status st, const std::string& m) {
  if (s) s->err = m;
  return st;
}
#define IK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return ifail(s, DG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

ImplArgs make_args(dg_implicit* s) {
  ImplArgs a{};
  const auto& p = s->prm;
  a.K = (int)s->K;
  a.dt = s->ip.dt;
  a.inv_dt = 1.0 / s->ip.dt;
  a.gc = p.g * std::cos(p.alpha);
  a.gs = p.g * std::sin(p.alpha);
  a.rho_inv = 1.0 / p.rho;
  a.eta = p.eta;
  a.sigma0 = p.sigma0;
  a.gamma = p.gamma;
  a.beta = p.beta;
  a.pap_m = p.pap_m;
  a.h_floor = p.h_floor;
  a.reg = s->reg;
  a.rtol = s->ip.rtol;
  a.atol = s->ip.atol;
  a.xtol = s->ip.xtol;
  a.max_it = s->ip.max_it;
  a.on_fail_continue = s->ip.on_fail_continue;
  a.mixed = s->ip.linear_solver == 1 ? 1 : 0;
  a.n_gamma = s->ip.n_gamma;
  a.gamma0 = s->ip.gamma0;
  a.Wf = s->at<float>(s->off.Wf);
  a.Af = s->at<float>(s->off.Af);
  a.Rr = s->at<double>(s->off.Rr);
  a.Dx2 = s->at<double>(s->off.Dx2);
  a.bcL = s->bcL;
  a.bcR = s->bcR;
  a.X = s->at<double>(s->off.X);
  a.Uold = s->at<double>(s->off.Uold);
  a.R = s->at<double>(s->off.R);
  a.D = s->at<double>(s->off.D);
  a.L = s->at<double>(s->off.L);
  a.U = s->at<double>(s->off.U);
  a.W = s->at<double>(s->off.W);
  a.Y = s->at<double>(s->off.Y);
  a.DX = s->at<double>(s->off.DX);
  a.J = s->at<double>(s->off.J);
  a.bed = s->has_bed ? s->at<double>(s->off.bed) : nullptr;
  a.red = s->at<double>(s->off.red);
  a.st = s->at<dg_implicit_stats>(s->off.st);
  return a;
}

template <int P, int M3>
struct IDrv final : ImplDrv {
  ImplOps<P, M3> o{};
  explicit IDrv(const dg_implicit& s) {
    using S = IS<P, M3>;
    for (int i = 0; i < S::NQ * S::NP; ++i) {
      o.Vq[i] = s.Vq[i];
      o.dVq[i] = s.dVq[i];
    }
    for (int i = 0; i < S::NQ * S::NE; ++i) {
      o.VEq[i] = s.VEq[i];
      o.dVEq[i] = s.dVEq[i];
    }
    for (int q = 0; q < S::NQ; ++q) o.wq[q] = s.wq[q];
    for (int i = 0; i < 2 * S::NP; ++i) o.lf[i] = s.lf[i];
    for (int i = 0; i < 2 * S::NE; ++i) o.lEf[i] = s.lEf[i];
  }
  void run(dg_implicit* s, long long n, cudaStream_t st) override {
    implicit_kernel<P, M3><<<1, 256, 0, st>>>(make_args(s), o, n);
  }
  void init_E(dg_implicit* s, cudaStream_t st) override {
    const int K = (int)s->K;
    init_E_kernel<P, M3><<<(K + 127) / 128, 128, 0, st>>>(make_args(s), o, s->at<double>(s->off.MEinv));
    commit_E_kernel<P, M3><<<(K + 127) / 128, 128, 0, st>>>(make_args(s));
  }
  void active(dg_implicit* s, double* out, cudaStream_t st) override {
    active_kernel<P, M3><<<1, 256, 0, st>>>(make_args(s), o, out);
  }
};

std::unique_ptr<ImplDrv> make_idrv(const dg_implicit& s) {
#define ICASE(PP, MM) \
  if (s.p == PP && s.m3 == MM) return std::unique_ptr<ImplDrv>(new IDrv<PP, MM>(s));
  ICASE(1, 0) ICASE(1, 1) ICASE(2, 0) ICASE(2, 1) ICASE(2, 2) ICASE(3, 0) ICASE(3, 1) ICASE(3, 2) ICASE(3, 3)
#undef ICASE
  return nullptr;
}

// 1D Lagrange basis on equispaced nodes of degree m (m = 0: the constant 1).
void lagrange1d(int m, double r, double* l, double* dl) {
  if (m == 0) {
    l[0] = 1.0;
    dl[0] = 0.0;
    return;
  }
  for (int k = 0; k <= m; ++k) {
    const double tk = -1.0 + 2.0 * k / m;
    double v = 1.0, d = 0.0;
    for (int j = 0; j <= m; ++j) {
      if (j == k) continue;
      const double tj = -1.0 + 2.0 * j / m;
      double prod = 1.0 / (tk - tj);
      for (int i = 0; i <= m; ++i) {
        if (i == k || i == j) continue;
        const double ti = -1.0 + 2.0 * i / m;
        prod *= (r - ti) / (tk - ti);
      }
      d += prod;
      v *= (r - tj) / (tk - tj);
    }
    l[k] = v;
    dl[k] = d;
  }
}

}  // namespace

extern "C" {

dg_status dg_implicit_init(const dg_swe_mesh* mesh, int order, int regularization, const dg_swe_params* params,
                           const dg_implicit_params* ip, dg_implicit** out) {
  if (!out) return DG_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<dg_implicit> s(new dg_implicit());
  if (!mesh || !params || !ip) {
    *out = s.release();
    return ifail(*out, DG_ERR_ARG, "null argument");
  }
  if (mesh->dim != 1) {
    *out = s.release();
    return ifail(*out, DG_ERR_UNSUPPORTED, "the implicit integrator is one-dimensional");
  }
  const int m3 = ip->m3 < 0 ? order : ip->m3;
  if (!(ip->dt > 0) || ip->max_it < 1 || m3 < 0 || m3 > order || ip->linear_solver < 0 || ip->linear_solver > 1) {
    *out = s.release();
    return ifail(*out, DG_ERR_ARG, "need dt > 0, max_it >= 1, 0 <= m3 <= order, linear_solver in {0, 1}");
  }
  if (ip->n_gamma > 1 && !(ip->gamma0 > 0)) {
    *out = s.release();
    return ifail(*out, DG_ERR_ARG, "continuation needs gamma0 > 0");
  }
  if (params->flow_index != 0.0 && params->flow_index != 1.0) {
    *out = s.release();
    return ifail(*out, DG_ERR_UNSUPPORTED,
                 "the Appendix A tangent covers the Newtonian viscous part only (flow_index 1); "
                 "use dg_newton.h for the Herschel-Bulkley law");
  }
  if (ip->linear_solver == 1 && 3 * (2 * (order + 1) + m3 + 1) > 32) {
    *out = s.release();
    return ifail(*out, DG_ERR_UNSUPPORTED, "the FP32 factorization handles blocks of at most 10 unknowns (2(p+1) + m3 + 1 <= 10)");
  }
  dg_swe_ctx* c = nullptr;
  dg_status st = dg_swe_init(mesh, order, regularization, params, &c);
  if (st != DG_OK) {
    std::string m = c ? dg_swe_last_error(c) : "";
    dg_swe_destroy(c);
    *out = s.release();
    return ifail(*out, st, m);
  }
  const int64_t K = c->mesh.K;
  for (int64_t e = 0; e + 1 < K; ++e)
    if (mesh->elem_vertices[2 * e + 1] != mesh->elem_vertices[2 * (e + 1)]) {
      dg_swe_destroy(c);
      *out = s.release();
      return ifail(*out, DG_ERR_UNSUPPORTED, "1D mesh must be ordered left to right (element e+1 starts where e ends)");
    }
  s->p = order;
  s->m3 = m3;
  s->reg = regularization;
  s->K = K;
  s->prm = *params;
  s->ip = *ip;
  s->ip.m3 = m3;
  const int NP = order + 1, NE = m3 + 1;
  const RefOps& o = c->ops;
  s->wq = o.wq;
  const int NQ = o.Nq;
  s->Vq.assign(NQ * NP, 0);
  s->dVq.assign(NQ * NP, 0);
  s->VEq.assign(NQ * NE, 0);
  s->dVEq.assign(NQ * NE, 0);
  std::vector<double> l(8), dl(8);
  for (int q = 0; q < NQ; ++q) {
    lagrange1d(order, o.rq[q], l.data(), dl.data());
    for (int i = 0; i < NP; ++i) {
      s->Vq[q * NP + i] = l[i];
      s->dVq[q * NP + i] = dl[i];
    }
    lagrange1d(m3, o.rq[q], l.data(), dl.data());
    for (int i = 0; i < NE; ++i) {
      s->VEq[q * NE + i] = l[i];
      s->dVEq[q * NE + i] = dl[i];
    }
  }
  s->lf.assign(2 * NP, 0);
  s->lEf.assign(2 * NE, 0);
  for (int f = 0; f < 2; ++f) {
    lagrange1d(order, f == 0 ? -1.0 : 1.0, l.data(), dl.data());
    for (int i = 0; i < NP; ++i) s->lf[f * NP + i] = l[i];
    lagrange1d(m3, f == 0 ? -1.0 : 1.0, l.data(), dl.data());
    for (int i = 0; i < NE; ++i) s->lEf[f * NE + i] = l[i];
  }
  // reference E mass matrix inverse
  std::vector<double> ME(NE * NE, 0.0);
  for (int q = 0; q < NQ; ++q)
    for (int a = 0; a < NE; ++a)
      for (int b = 0; b < NE; ++b) ME[a * NE + b] += s->wq[q] * s->VEq[q * NE + a] * s->VEq[q * NE + b];
  s->MEinv.assign(NE * NE, 0.0);
  {  // Gauss-Jordan inverse (NE <= 4)
    std::vector<double> A(ME);
    for (int i = 0; i < NE; ++i) s->MEinv[i * NE + i] = 1.0;
    for (int k = 0; k < NE; ++k) {
      int pv = k;
      for (int r = k + 1; r < NE; ++r)
        if (std::fabs(A[r * NE + k]) > std::fabs(A[pv * NE + k])) pv = r;
      for (int j = 0; j < NE; ++j) {
        std::swap(A[k * NE + j], A[pv * NE + j]);
        std::swap(s->MEinv[k * NE + j], s->MEinv[pv * NE + j]);
      }
      const double d = 1.0 / A[k * NE + k];
      for (int j = 0; j < NE; ++j) {
        A[k * NE + j] *= d;
        s->MEinv[k * NE + j] *= d;
      }
      for (int r = 0; r < NE; ++r) {
        if (r == k) continue;
        const double f = A[r * NE + k];
        for (int j = 0; j < NE; ++j) {
          A[r * NE + j] -= f * A[k * NE + j];
          s->MEinv[r * NE + j] -= f * s->MEinv[k * NE + j];
        }
      }
    }
  }
  s->J.assign(K, 0.0);
  for (int64_t e = 0; e < K; ++e) s->J[e] = c->mesh.geo[4 * K + e];
  s->node_x.assign(c->mesh.node_xyz.begin(), c->mesh.node_xyz.end());
  if (mesh->bed) {
    s->has_bed = true;
    s->bed.assign(mesh->bed, mesh->bed + K * NP);
  }
  auto bc_of = [&](int64_t e, int f) {
    const int id = mesh->face_bc ? mesh->face_bc[e * 2 + f] : 0;
    BCEntry<double> b{};
    for (int k = 0; k < 7; ++k) {
      b.mode[k] = params->bc[id].mode[k];
      b.val[k] = params->bc[id].value[k];
    }
    return b;
  };
  s->bcL = bc_of(0, 0);
  s->bcR = bc_of(K - 1, 1);
  dg_swe_destroy(c);
  s->drv = make_idrv(*s);
  const int NB = s->nb();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off += (bytes + 255) & ~size_t(255);
    return r;
  };
  s->off.X = take(K * NB * 8);
  s->off.Uold = take(K * 2 * NP * 8);
  s->off.R = take(K * NB * 8);
  s->off.D = take(K * NB * NB * 8);
  s->off.L = take(K * NB * NB * 8);
  s->off.U = take(K * NB * NB * 8);
  s->off.W = take(K * NB * NB * 8);
  s->off.Y = take(K * NB * 8);
  s->off.DX = take(K * NB * 8);
  s->off.J = take(K * 8);
  s->off.bed = take(s->has_bed ? K * NP * 8 : 0);
  s->off.red = take(64 * 8);
  s->off.st = take(sizeof(dg_implicit_stats));
  s->off.MEinv = take(NE * NE * 8);
  s->off.act = take(8);
  s->off.Wf = take(K * NB * NB * 4);
  s->off.Af = take(K * NB * NB * 4);
  s->off.Rr = take(K * NB * 8);
  s->off.Dx2 = take(K * NB * 8);
  s->ws_need = off;
  *out = s.release();
  return DG_OK;
}

size_t dg_implicit_workspace_size(const dg_implicit* s) { return s ? s->ws_need : 0; }

dg_status dg_implicit_set_stream(dg_implicit* s, void* st) {
  if (!s) return DG_ERR_ARG;
  s->stream = (cudaStream_t)st;
  return DG_OK;
}

dg_status dg_implicit_set_workspace(dg_implicit* s, void* ptr, size_t bytes) {
  if (!s) return DG_ERR_ARG;
  if (!ptr || bytes < s->ws_need) return ifail(s, DG_ERR_WORKSPACE, "workspace missing or too small");
  if (((uintptr_t)ptr & 255) != 0) return ifail(s, DG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  s->ws = (char*)ptr;
  cudaStream_t st = s->stream;
  IK(cudaMemsetAsync(s->ws, 0, s->ws_need, st));
  IK(cudaMemcpyAsync(s->ws + s->off.J, s->J.data(), s->J.size() * 8, cudaMemcpyHostToDevice, st));
  if (s->has_bed) IK(cudaMemcpyAsync(s->ws + s->off.bed, s->bed.data(), s->bed.size() * 8, cudaMemcpyHostToDevice, st));
  IK(cudaMemcpyAsync(s->ws + s->off.MEinv, s->MEinv.data(), s->MEinv.size() * 8, cudaMemcpyHostToDevice, st));
  IK(cudaStreamSynchronize(st));
  return DG_OK;
}

dg_status dg_implicit_node_coords(const dg_implicit* s, double* x) {
  if (!s || !x) return DG_ERR_ARG;
  std::memcpy(x, s->node_x.data(), s->node_x.size() * 8);
  return DG_OK;
}

dg_status dg_implicit_set_state(dg_implicit* s, const double* V, int on_device) {
  if (!s || !V) return DG_ERR_ARG;
  if (!s->ws) return ifail(s, DG_ERR_WORKSPACE, "no workspace set");
  const int NP = s->p + 1, NB = s->nb();
  const int64_t K = s->K;
  std::vector<double> hv(2 * K * NP);
  cudaStream_t st = s->stream;
  if (on_device) {
    IK(cudaMemcpyAsync(hv.data(), V, hv.size() * 8, cudaMemcpyDeviceToHost, st));
    IK(cudaStreamSynchronize(st));
  } else {
    std::memcpy(hv.data(), V, hv.size() * 8);
  }
  std::vector<double> X(K * NB, 0.0);
  for (int64_t e = 0; e < K; ++e)
    for (int i = 0; i < NP; ++i) {
      X[e * NB + i] = hv[e * NP + i];
      X[e * NB + NP + i] = hv[K * NP + e * NP + i];
    }
  IK(cudaMemcpyAsync(s->ws + s->off.X, X.data(), X.size() * 8, cudaMemcpyHostToDevice, st));
  IK(cudaMemsetAsync(s->ws + s->off.st, 0, sizeof(dg_implicit_stats), st));
  s->drv->init_E(s, st);
  IK(cudaGetLastError());
  IK(cudaStreamSynchronize(st));
  return DG_OK;
}

dg_status dg_implicit_get_state(dg_implicit* s, double* V, double* E, int on_device) {
  if (!s) return DG_ERR_ARG;
  if (!s->ws) return ifail(s, DG_ERR_WORKSPACE, "no workspace set");
  const int NP = s->p + 1, NE = s->m3 + 1, NB = s->nb();
  const int64_t K = s->K;
  std::vector<double> X(K * NB);
  IK(cudaMemcpyAsync(X.data(), s->ws + s->off.X, X.size() * 8, cudaMemcpyDeviceToHost, s->stream));
  IK(cudaStreamSynchronize(s->stream));
  std::vector<double> hv(2 * K * NP), he(K * NE);
  for (int64_t e = 0; e < K; ++e) {
    for (int i = 0; i < NP; ++i) {
      hv[e * NP + i] = X[e * NB + i];
      hv[K * NP + e * NP + i] = X[e * NB + NP + i];
    }
    for (int c = 0; c < NE; ++c) he[e * NE + c] = X[e * NB + 2 * NP + c];
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  if (V) IK(cudaMemcpy(V, hv.data(), hv.size() * 8, kind));
  if (E) IK(cudaMemcpy(E, he.data(), he.size() * 8, kind));
  return DG_OK;
}

dg_status dg_implicit_run(dg_implicit* s, int64_t n_steps, dg_implicit_stats* stats) {
  if (!s) return DG_ERR_ARG;
  if (!s->ws) return ifail(s, DG_ERR_WORKSPACE, "no workspace set");
  if (n_steps < 0) return ifail(s, DG_ERR_ARG, "n_steps < 0");
  if (n_steps > 0) s->drv->run(s, (long long)n_steps, s->stream);
  IK(cudaGetLastError());
  dg_implicit_stats h{};
  IK(cudaMemcpyAsync(&h, s->ws + s->off.st, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  IK(cudaStreamSynchronize(s->stream));
  if (stats) *stats = h;
  if (h.status != 0)
    return ifail(s, (dg_status)h.status,
                 h.status == DG_ERR_NEWTON ? "Newton did not converge within max_it" : "non-finite state");
  return DG_OK;
}

dg_status dg_implicit_active_percent(dg_implicit* s, double* pct) {
  if (!s || !pct) return DG_ERR_ARG;
  if (!s->ws) return ifail(s, DG_ERR_WORKSPACE, "no workspace set");
  s->drv->active(s, s->at<double>(s->off.act), s->stream);
  IK(cudaGetLastError());
  IK(cudaMemcpyAsync(pct, s->ws + s->off.act, 8, cudaMemcpyDeviceToHost, s->stream));
  IK(cudaStreamSynchronize(s->stream));
  return DG_OK;
}

const char* dg_implicit_last_error(const dg_implicit* s) { return s ? s->err.c_str() : "null context"; }

void dg_implicit_destroy(dg_implicit* s) { delete s; }

}  // extern "C"

// Device kernels of the DG shallow-water / regularized-Bingham hot path.
//
// One explicit stage is three launches:
//   estep_kernel   E = grad u in the weak sense of Eq. WeakForm52, written in
//                  the equivalent strong nodal form E = grad u + LIFT(n [u]/2)
//                  (exact for the E space of degree p); neighbour traces come
//                  through the face-to-node map (one thread per element).
//   face_kernel    the numerical flux once per face point: HLL for F
//                  (Eq. HLLSolver, rotated to the face normal) minus the
//                  central flux of Q (Sec. 5), weighted by the edge quadrature
//                  weight and face Jacobian (one thread per face point).
//   volume_kernel  volume integrals of Eq. WeakForm51 (flux, stress, slope and
//                  bed source), lift of the face fluxes, the primitive-variable
//                  mass solve M dh/dt = -r_h, M_h du/dt = -r_u - M_u dh/dt
//                  (dU/dV of Appendix A) with a per-element Cholesky
//                  factorization, and the SSP-RK3 stage update (one thread per
//                  element).
// plus FP64 reductions for the stable step and the mass integral.
//
// Storage is [field][element][node] (nodes contiguous), R = double or float.
// Reference operators are passed by value as kernel parameters: with the
// loops unrolled every thread of a warp reads the same entry, a broadcast
// from the constant bank.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dg_host.h"

namespace dgswe {

template <int DIM, int P>
struct Sh {
  static constexpr int NP = DIM == 1 ? P + 1 : (P + 1) * (P + 2) / 2;
  static constexpr int NQ1 = (3 * P + 1) / 2;
  static constexpr int NQ = DIM == 1 ? NQ1 : NQ1 * NQ1;
  static constexpr int NF = DIM + 1;
  static constexpr int NFP = DIM == 1 ? 1 : P + 1;
  static constexpr int NFQ = DIM == 1 ? 1 : (3 * P + 2) / 2;
  static constexpr int NV = DIM + 1;
  static constexpr int NE = DIM * DIM;
};

// Physical parameters of one instance (kernel parameter for a single
// context, a per-instance device table for a batch).
template <typename R>
struct Phys {
  R gc, gs, rho_inv, eta, sigma0, gamma, beta, pap_m, h_floor;
  R half_inv_beta;  // 1 / (2 beta), the half-width of the regularizations 1 and 2 (host-computed)
  R h_dry;          // FP32 contexts: depth below which an element's mass solve runs in FP64
                    // (kDryFactor x h_floor)
  R hb_n, hb_floor;  // Herschel-Bulkley flow index and rate floor (dg_swe_params)
  int hb;            // 1: power-law viscous part (flow index != 1)
  int reg;
  int pos;  // wet/dry mode: conservative stages with the depth limiter (dg_swe_params.positivity)
};

// One boundary descriptor: per slot (V fields then E fields) a mode
// (0 copy, 1 Dirichlet, 2 wall) and a Dirichlet value.  Boundary faces carry
// -1 - (index into a device table of these).
template <typename R>
struct BCEntry {
  int mode[7];
  R val[7];
};

template <int DIM, int P, typename R>
struct EstepOps {
  using S = Sh<DIM, P>;
  R Dr[S::NP * S::NP];
  R Ds[S::NP * S::NP];
  R LIFT[S::NP * S::NF * S::NFP];
  int8_t fmask[S::NF * S::NFP];
};

template <int DIM, int P, typename R>
struct FaceOps {
  using S = Sh<DIM, P>;
  R Lf[S::NFQ * S::NFP];
  R wf[S::NFQ];
  int8_t fmask[S::NF * S::NFP];
};

template <int DIM, int P, typename R>
struct VolOps {
  using S = Sh<DIM, P>;
  R Vq[S::NQ * S::NP];   // l_a(q)
  R Wr[S::NQ * S::NP];   // w_q dl_a/dr (q)
  R Ws[S::NQ * S::NP];   // w_q dl_a/ds (q)
  R Wm[S::NQ * S::NP];   // w_q l_a(q)
  R Drq[S::NQ * S::NP];  // dl_a/dr (q) (bed gradient)
  R Dsq[S::NQ * S::NP];
  R wq[S::NQ];
  R Minv[S::NP * S::NP];
  R LfT[S::NFP * S::NFQ];  // Lf transposed: lift of face-point values to face nodes
  R wavg[S::NP];           // cell average = sum_a wavg[a] h_a (integral of l_a / reference measure)
};

struct DevScalars {
  double dt, t, dt_min, dt_max, mass, mass0;
  long long steps;
  int status;
  int pad;
};

// ------------------------------------------------------------------ arithmetic helpers
// FP64 keeps IEEE division and square root and uses the CUDA math library's
// reciprocal square root (1 ulp).  FP32 uses the fast hardware forms
// (division, reciprocal square root and square root within 2 ulp), well
// inside the FP32 path's stated tolerance.
template <typename R>
__device__ __forceinline__ R dg_div(R a, R b) { return a / b; }
template <>
__device__ __forceinline__ float dg_div<float>(float a, float b) { return __fdividef(a, b); }
template <typename R>
__device__ __forceinline__ R dg_rsqrt(R x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float dg_rsqrt<float>(float x) { return rsqrtf(x); }
template <typename R>
__device__ __forceinline__ R dg_sqrt(R x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dg_sqrt<float>(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Loads of data that another thread block writes during the same launch (the
// persistent batch kernel, COH = true) go through L2 (ld.global.cg), which is
// coherent on the GPU; every other kernel (COH = false) loads normally.  A
// macro taking base and index, so that the plain loads keep the form
// base[index] (an index sum added once to the base): the form ptr + a + b
// through a helper compiled the FP32 kernels to more registers and ran
// slower (E-step 64 -> 80 registers, 0.36 -> 0.42 ms on 8.4M triangles).
#define DG_LDC(COH, base, idx) ((COH) ? __ldcg((base) + (idx)) : (base)[idx])

// ------------------------------------------------------------------ physics

// phi_k(s) / (2 s) for s >= 0 (limit phi_k'(0)/2 at s = 0): the Bingham
// coefficient of sigma_B = (phi(s)/(2s)) (D + tr D I), s = ||D||_c / sqrt(2).
template <typename R>
__device__ __forceinline__ R bingham_coef(R s, R s_inv, const Phys<R>& ph) {
  // s_inv = 1 / s (any value when s = 0: every s = 0 case takes a branch
  // that does not use it)
  const R s0 = ph.sigma0, g = ph.gamma;
  if (ph.reg == 0 || s0 == R(0)) return R(0);
  switch (ph.reg) {
    case 1: {  // smooth max, Eq. sigmaTwoA/AA
      R e = ph.half_inv_beta;
      R x = g * s - s0;
      R mb = x >= e ? x : (x <= -e ? R(0) : R(0.5) * ph.beta * (x + e) * (x + e));
      return dg_div<R>(s0 * g, mb + s0);
    }
    case 2: {  // local quadratic, Eq. sigmaTwoB
      R e = ph.half_inv_beta;
      R x = g * s;
      if (x >= s0 + e) return s0 * s_inv;
      if (x <= s0 - e) return g;
      R d = s0 - x + e;
      return (R(2) * s0 - ph.beta * d * d) * (R(0.5) * s_inv);
    }
    case 3: {  // tanh, Eq. sigmaTwoC
      R x = g * s;
      if (x < R(1e-8)) return s0 * g * (R(1) - x * x / R(3));
      return s0 * tanh(x) * s_inv;
    }
    case 4: {  // exponential (extension)
      R x = ph.pap_m * s;
      if (x < R(1e-12)) return s0 * ph.pap_m * (R(1) - R(0.5) * x);
      return -s0 * expm1(-x) * s_inv;
    }
    case 5: {  // bi-viscosity (extension)
      R x = g * s;
      return x < s0 ? g : s0 * s_inv;
    }
  }
  return R(0);
}
template <typename R>
__device__ __forceinline__ R bingham_coef(R s, const Phys<R>& ph) {
  return bingham_coef<R>(s, s > R(0) ? dg_div<R>(R(1), s) : R(0), ph);
}

// Viscosity of the Newtonian part: eta, or the Herschel-Bulkley power law
// eta max(s, rate_floor)^(n-1) (dg_swe_params.flow_index, an extension).
template <typename R>
__device__ __forceinline__ R viscous_eta(R s, const Phys<R>& ph) {
  return ph.hb ? ph.eta * pow(fmax(s, ph.hb_floor), ph.hb_n - R(1)) : ph.eta;
}

// sigma from E (component 2i+j = du_j/dx_i); returns sig[i][j].
template <int DIM, typename R>
__device__ __forceinline__ void stress(const R* E, const Phys<R>& ph, R sig[DIM][DIM]) {
  if constexpr (DIM == 1) {
    R e = E[0];
    R mu = R(2) * viscous_eta<R>(fabs(e), ph) + bingham_coef<R>(fabs(e), ph);
    sig[0][0] = mu * R(2) * e;
  } else {
    R d11 = E[0], d22 = E[3], d12 = R(0.5) * (E[1] + E[2]);
    R tr = d11 + d22;
    R nc2 = d11 * d11 + R(2) * d12 * d12 + d22 * d22 + tr * tr;
    const R s2 = R(0.5) * nc2;
    R mu;
    if (ph.reg == 5 && !ph.hb) {
      // bi-viscosity with the Newtonian viscous part: gamma below the yield
      // rate (gamma s < sigma0, tested on s^2) and sigma0 / s above it, so
      // the reciprocal square root is taken only where the material yields
      const R g = ph.gamma, s0 = ph.sigma0;
      const R coef = s0 == R(0) ? R(0) : (g * g * s2 < s0 * s0 ? g : s0 * dg_rsqrt<R>(s2));
      mu = R(2) * ph.eta + coef;
    } else {
      // s = sqrt(nc2 / 2) and 1 / s from one reciprocal square root
      const R s_inv = s2 > R(0) ? dg_rsqrt<R>(s2) : R(0);
      const R s = s2 * s_inv;
      mu = R(2) * viscous_eta<R>(s, ph) + bingham_coef<R>(s, s_inv, ph);
    }
    sig[0][0] = mu * (d11 + tr);
    sig[1][1] = mu * (d22 + tr);
    sig[0][1] = mu * d12;
    sig[1][0] = mu * d12;
  }
}

// Exterior state at a boundary face point (Sec. 5.2 ghost values).
template <int DIM, typename R>
__device__ __forceinline__ void ghost_V(const R* Vm, const R* n, const BCEntry<R>& b, R* Vp) {
  bool wall = false;
#pragma unroll
  for (int v = 0; v < DIM + 1; ++v) {
    int md = b.mode[v];
    Vp[v] = md == 1 ? b.val[v] : Vm[v];
    if (v > 0 && md == 2) wall = true;
  }
  if (wall) {
    R un = R(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j) un += Vm[1 + j] * n[j];
#pragma unroll
    for (int j = 0; j < DIM; ++j) Vp[1 + j] = Vm[1 + j] - R(2) * un * n[j];
  }
}

template <int DIM, typename R>
__device__ __forceinline__ void ghost_E(const R* Em, const BCEntry<R>& b, R* Ep) {
#pragma unroll
  for (int c = 0; c < DIM * DIM; ++c) {
    int slot = DIM + 1 + c;
    Ep[c] = b.mode[slot] == 1 ? b.val[slot] : Em[c];
  }
}

// HLL normal flux (Eq. HLLSolver in the face-normal frame; wave speeds with
// sqrt(g_c max(h, h_floor))).
template <int DIM, typename R>
__device__ __forceinline__ void hll(const R* Vm, const R* Vp, const R* n, const Phys<R>& ph, R* Fn) {
  R hm = Vm[0], hp = Vp[0];
  R unm = R(0), unp = R(0);
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    unm += Vm[1 + j] * n[j];
    unp += Vp[1 + j] * n[j];
  }
  R cm = dg_sqrt<R>(ph.gc * fmax(hm, ph.h_floor));
  R cp = dg_sqrt<R>(ph.gc * fmax(hp, ph.h_floor));
  R SL = fmin(unm - cm, unp - cp);
  R SR = fmax(unm + cm, unp + cp);
  R Fm[DIM + 1], Fp[DIM + 1];
  Fm[0] = hm * unm;
  Fp[0] = hp * unp;
  R pm = R(0.5) * ph.gc * hm * hm, pp = R(0.5) * ph.gc * hp * hp;
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    Fm[1 + j] = hm * Vm[1 + j] * unm + pm * n[j];
    Fp[1 + j] = hp * Vp[1 + j] * unp + pp * n[j];
  }
  if (SL >= R(0)) {
#pragma unroll
    for (int v = 0; v < DIM + 1; ++v) Fn[v] = Fm[v];
  } else if (SR <= R(0)) {
#pragma unroll
    for (int v = 0; v < DIM + 1; ++v) Fn[v] = Fp[v];
  } else {
    R inv = dg_div<R>(R(1), SR - SL);
    R Um[DIM + 1], Up[DIM + 1];
    Um[0] = hm;
    Up[0] = hp;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      Um[1 + j] = hm * Vm[1 + j];
      Up[1 + j] = hp * Vp[1 + j];
    }
#pragma unroll
    for (int v = 0; v < DIM + 1; ++v) Fn[v] = (SR * Fm[v] - SL * Fp[v] + SL * SR * (Up[v] - Um[v])) * inv;
  }
}

// Q . n for one side: Q_i row 1+j = h sigma_{j i} / rho (Eq. Qterm).
template <int DIM, typename R>
__device__ __forceinline__ void q_normal(R h, const R* E, const R* n, const Phys<R>& ph, R* Qn) {
  R sig[DIM][DIM];
  stress<DIM, R>(E, ph, sig);
  Qn[0] = R(0);
  R hr = h * ph.rho_inv;
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    R a = R(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) a += sig[j][i] * n[i];
    Qn[1 + j] = hr * a;
  }
}

// ------------------------------------------------------------------ kernels

// E-step of element e (the body of estep_kernel).  PRE: the element's face
// neighbours and their local faces arrive preloaded in pnb / pnbf (one per
// face) instead of being read from nbr / nbrf.
template <int DIM, int P, typename R, bool COH = false, bool PRE = false>
__device__ __forceinline__ void estep_element(int e, int K, const R* __restrict__ V, R* __restrict__ E,
                                              const R* __restrict__ geo, const int32_t* __restrict__ nbr,
                                              const int8_t* __restrict__ nbrf, const R* __restrict__ fn,
                                              const R* __restrict__ fsj, const EstepOps<DIM, P, R>& ops,
                                              const BCEntry<R>* __restrict__ bct, const int* pnb = nullptr,
                                              const int* pnbf = nullptr) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NF = S::NF, NFP = S::NFP, NE = S::NE;
  const size_t KN = (size_t)K * NP;
  R u[DIM][NP];
#pragma unroll
  for (int j = 0; j < DIM; ++j)
#pragma unroll
    for (int a = 0; a < NP; ++a) u[j][a] = DG_LDC(COH, V, (1 + j) * KN + (size_t)e * NP + a);
  R G[2][2];
  G[0][0] = geo[e];
  if constexpr (DIM == 2) {
    G[0][1] = geo[K + e];
    G[1][0] = geo[2 * K + e];
    G[1][1] = geo[3 * K + e];
  }
  const R Jinv = geo[6 * K + e];
  R Eo[NE][NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      R dr = R(0), ds = R(0);
#pragma unroll
      for (int b = 0; b < NP; ++b) {
        dr += ops.Dr[a * NP + b] * u[j][b];
        if constexpr (DIM == 2) ds += ops.Ds[a * NP + b] * u[j][b];
      }
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        R v = G[0][i] * dr;
        if constexpr (DIM == 2) v += G[1][i] * ds;
        Eo[DIM * i + j][a] = v;
      }
    }
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int e2 = PRE ? pnb[f] : nbr[f * K + e];
    R n[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) n[i] = fn[(f * DIM + i) * K + e];
    const R sc = fsj[f * K + e] * Jinv;
    R gj[NFP][DIM];
    if (e2 >= 0) {
      const int f2 = PRE ? pnbf[f] : nbrf[f * K + e];
#pragma unroll
      for (int k = 0; k < NFP; ++k) {
        const int a = face_node(DIM, P, f, k);
        const int b = ops.fmask[f2 * NFP + (NFP - 1 - k)];
#pragma unroll
        for (int j = 0; j < DIM; ++j) gj[k][j] = R(0.5) * (DG_LDC(COH, V, (1 + j) * KN + (size_t)e2 * NP + b) - u[j][a]);
      }
    } else {
      const BCEntry<R> bc = bct[-1 - e2];
#pragma unroll
      for (int k = 0; k < NFP; ++k) {
        const int a = face_node(DIM, P, f, k);
        R Vm[DIM + 1], Vp[DIM + 1];
        Vm[0] = R(1);
#pragma unroll
        for (int j = 0; j < DIM; ++j) Vm[1 + j] = u[j][a];
        ghost_V<DIM, R>(Vm, n, bc, Vp);
#pragma unroll
        for (int j = 0; j < DIM; ++j) gj[k][j] = R(0.5) * (Vp[1 + j] - Vm[1 + j]);
      }
    }
    if constexpr (sizeof(R) == 8) {
      // FP64 (bound by the FP64 pipe): lift each velocity jump once,
      // w_j(a) = sum_k LIFT_a,fk [u_j]_k / 2, then scale by sc n_i: NP DIM
      // (NFP + DIM) multiply-adds per face instead of NP NFP DIM DIM
      R sn[DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i) sn[i] = sc * n[i];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        R w[DIM];
#pragma unroll
        for (int j = 0; j < DIM; ++j) w[j] = R(0);
#pragma unroll
        for (int k = 0; k < NFP; ++k) {
          const R L = ops.LIFT[a * (NF * NFP) + f * NFP + k];
#pragma unroll
          for (int j = 0; j < DIM; ++j) w[j] += L * gj[k][j];
        }
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
          for (int j = 0; j < DIM; ++j) Eo[DIM * i + j][a] += sn[i] * w[j];
      }
    } else {
      // FP32: the face's jump terms sc n_i [u_j]/2, scaled once per face node
      R gt[NFP][DIM][DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        const R sn = sc * n[i];
#pragma unroll
        for (int k = 0; k < NFP; ++k)
#pragma unroll
          for (int j = 0; j < DIM; ++j) gt[k][i][j] = sn * gj[k][j];
      }
#pragma unroll
      for (int a = 0; a < NP; ++a) {
#pragma unroll
        for (int k = 0; k < NFP; ++k) {
          const R L = ops.LIFT[a * (NF * NFP) + f * NFP + k];
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) Eo[DIM * i + j][a] += L * gt[k][i][j];
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NE; ++c)
#pragma unroll
    for (int a = 0; a < NP; ++a) E[c * KN + (size_t)e * NP + a] = Eo[c][a];
}

template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256) estep_kernel(int K, const R* __restrict__ V, R* __restrict__ E,
                                                    const R* __restrict__ geo, const int32_t* __restrict__ nbr,
                                                    const int8_t* __restrict__ nbrf, const R* __restrict__ fn,
                                                    const R* __restrict__ fsj, const EstepOps<DIM, P, R> ops,
                                                    const BCEntry<R>* __restrict__ bct) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  estep_element<DIM, P, R>(e, K, V, E, geo, nbr, nbrf, fn, fsj, ops, bct);
}

// Numerical flux at one face point m from the traces of both sides at the
// face nodes (owner's node order along its face); writes the weighted flux.
template <int DIM, int P, typename R>
__device__ __forceinline__ void face_point(int m, const R (&Tm)[Sh<DIM, P>::NV + Sh<DIM, P>::NE][Sh<DIM, P>::NFP],
                                           const R (&Tp)[Sh<DIM, P>::NV + Sh<DIM, P>::NE][Sh<DIM, P>::NFP],
                                           bool interior, const BCEntry<R>* __restrict__ bct, int bc,
                                           const R* n, R wsj, const FaceOps<DIM, P, R>& ops, const Phys<R>& ph,
                                           R* __restrict__ wflux, size_t FQ, size_t t) {
  using S = Sh<DIM, P>;
  constexpr int NFP = S::NFP, NV = S::NV, NE = S::NE;
  R Vm[NV], Vp[NV], Em[NE], Ep[NE];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    R a = R(0), b = R(0);
#pragma unroll
    for (int k = 0; k < NFP; ++k) {
      a += ops.Lf[m * NFP + k] * Tm[v][k];
      b += ops.Lf[m * NFP + k] * Tp[v][k];
    }
    Vm[v] = a;
    Vp[v] = b;
  }
#pragma unroll
  for (int c = 0; c < NE; ++c) {
    R a = R(0), b = R(0);
#pragma unroll
    for (int k = 0; k < NFP; ++k) {
      a += ops.Lf[m * NFP + k] * Tm[NV + c][k];
      b += ops.Lf[m * NFP + k] * Tp[NV + c][k];
    }
    Em[c] = a;
    Ep[c] = b;
  }
  if (!interior) {
    const BCEntry<R> b = bct[bc];
    ghost_V<DIM, R>(Vm, n, b, Vp);
    ghost_E<DIM, R>(Em, b, Ep);
  }
  R Fn[NV], Qm[NV], Qp[NV];
  hll<DIM, R>(Vm, Vp, n, ph, Fn);
  q_normal<DIM, R>(Vm[0], Em, n, ph, Qm);
  q_normal<DIM, R>(Vp[0], Ep, n, ph, Qp);
  const R w = ops.wf[m] * wsj;
#pragma unroll
  for (int v = 0; v < NV; ++v) wflux[v * FQ + t] = w * (Fn[v] - R(0.5) * (Qm[v] + Qp[v]));
}

// Resident blocks of 256 threads the face kernel asks the compiler to fit
// per SM: three (at most 85 registers a thread) for FP32 at p <= 2, where
// the latency-bound gathers gain from the extra warps (per-face form on 2M
// triangles: 0.235 -> 0.203 ms, with a 16-byte spill); otherwise the
// compiler's choice (FP64 and p = 3 would spill heavily).
template <int DIM, int P, typename R>
constexpr int face_min_blocks() {
  return (sizeof(R) == 4 && P <= 2) ? 3 : 1;
}

// PERFACE = false: one thread per face point (re-reads the face-node traces
// for every point); PERFACE = true: one thread per face, traces read once
// and all edge points evaluated in turn.  Same arithmetic per point.
// Flux work of one face-kernel thread tid (one face point, or one face when
// PERFACE): the body of face_kernel.
template <int DIM, int P, typename R, bool BATCH, bool PERFACE, bool COH = false>
__device__ __forceinline__ void face_item(long long tid, int K, int F, const R* __restrict__ V,
                                          const R* __restrict__ E, const int32_t* __restrict__ fe1,
                                          const int8_t* __restrict__ ff1, const int32_t* __restrict__ fe2,
                                          const int8_t* __restrict__ ff2, const R* __restrict__ fnrm,
                                          const R* __restrict__ fsj, R* __restrict__ wflux,
                                          const FaceOps<DIM, P, R>& ops, const Phys<R>& ph0,
                                          const Phys<R>* __restrict__ ptab, const int32_t* __restrict__ inst,
                                          const BCEntry<R>* __restrict__ bct) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NFP = S::NFP, NFQ = S::NFQ, NV = S::NV, NE = S::NE;
  const int fc = PERFACE ? (int)tid : (int)(tid / NFQ);
  const int m0 = PERFACE ? 0 : (int)(tid - (long long)fc * NFQ);
  const size_t KN = (size_t)K * NP;
  const int e1 = fe1[fc], f1 = ff1[fc], e2 = fe2[fc];
  const Phys<R> ph = BATCH ? ptab[inst[e1]] : ph0;
  R n[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) n[i] = fnrm[(size_t)i * F + fc];
  R Tm[NV + NE][NFP], Tp[NV + NE][NFP];
#pragma unroll
  for (int k = 0; k < NFP; ++k) {
    const size_t a = (size_t)e1 * NP + ops.fmask[f1 * NFP + k];
#pragma unroll
    for (int v = 0; v < NV; ++v) Tm[v][k] = DG_LDC(COH, V, v * KN + a);
#pragma unroll
    for (int c = 0; c < NE; ++c) Tm[NV + c][k] = DG_LDC(COH, E, c * KN + a);
  }
  const bool interior = e2 >= 0;
  if (interior) {
    const int f2 = ff2[fc];
#pragma unroll
    for (int k = 0; k < NFP; ++k) {
      const size_t b = (size_t)e2 * NP + ops.fmask[f2 * NFP + (NFP - 1 - k)];
#pragma unroll
      for (int v = 0; v < NV; ++v) Tp[v][k] = DG_LDC(COH, V, v * KN + b);
#pragma unroll
      for (int c = 0; c < NE; ++c) Tp[NV + c][k] = DG_LDC(COH, E, c * KN + b);
    }
  } else {
#pragma unroll
    for (int r = 0; r < NV + NE; ++r)
#pragma unroll
      for (int k = 0; k < NFP; ++k) Tp[r][k] = Tm[r][k];
  }
  const R wsj = fsj[fc];
  const size_t FQ = (size_t)F * NFQ;
  if (PERFACE) {
#pragma unroll
    for (int m = 0; m < NFQ; ++m)
      face_point<DIM, P, R>(m, Tm, Tp, interior, bct, -1 - e2, n, wsj, ops, ph, wflux, FQ,
                            (size_t)fc * NFQ + m);
  } else {
    face_point<DIM, P, R>(m0, Tm, Tp, interior, bct, -1 - e2, n, wsj, ops, ph, wflux, FQ, (size_t)tid);
  }
}

template <int DIM, int P, typename R, bool BATCH, bool PERFACE>
__global__ void __launch_bounds__(256, face_min_blocks<DIM, P, R>())
    face_kernel(int K, int F, const R* __restrict__ V, const R* __restrict__ E,
                                                   const int32_t* __restrict__ fe1, const int8_t* __restrict__ ff1,
                                                   const int32_t* __restrict__ fe2, const int8_t* __restrict__ ff2,
                                                   const R* __restrict__ fnrm, const R* __restrict__ fsj,
                                                   R* __restrict__ wflux, const FaceOps<DIM, P, R> ops,
                                                   const Phys<R> ph0, const Phys<R>* __restrict__ ptab,
                                                   const int32_t* __restrict__ inst,
                                                   const BCEntry<R>* __restrict__ bct) {
  constexpr int NFQ = Sh<DIM, P>::NFQ;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = PERFACE ? (long long)F : (long long)F * NFQ;
  if (tid >= nthreads) return;
  face_item<DIM, P, R, BATCH, PERFACE>(tid, K, F, V, E, fe1, ff1, fe2, ff2, fnrm, fsj, wflux, ops, ph0, ptab, inst,
                                       bct);
}

// Per-face flux kernel over a grid-stride loop, for batch groups: while a
// thread gathers and evaluates face fc, the connectivity of its next face
// (fc + grid size: both elements and local faces, normal, scaled Jacobian)
// is already on its way, so each face costs one dependent round trip to
// memory (the trace gathers) instead of two.  Same per-point arithmetic as
// face_kernel (face_point).  The gather and evaluation below restate
// face_item's after its connectivity loads, so that face_kernel keeps its
// own compiled form.
template <int DIM, int P, typename R>
__device__ __forceinline__ void face_pf_body(int fc, int e1, int f1, int e2, int f2, const R (&n)[DIM], R wsj,
                                             int K, int F, const R* __restrict__ V, const R* __restrict__ E,
                                             R* __restrict__ wflux, const FaceOps<DIM, P, R>& ops,
                                             const Phys<R>* __restrict__ ptab, const int32_t* __restrict__ inst,
                                             const BCEntry<R>* __restrict__ bct) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NFP = S::NFP, NFQ = S::NFQ, NV = S::NV, NE = S::NE;
  const size_t KN = (size_t)K * NP;
  const Phys<R> ph = ptab[inst[e1]];
  R Tm[NV + NE][NFP], Tp[NV + NE][NFP];
#pragma unroll
  for (int k = 0; k < NFP; ++k) {
    const size_t a = (size_t)e1 * NP + ops.fmask[f1 * NFP + k];
#pragma unroll
    for (int v = 0; v < NV; ++v) Tm[v][k] = V[v * KN + a];
#pragma unroll
    for (int c = 0; c < NE; ++c) Tm[NV + c][k] = E[c * KN + a];
  }
  const bool interior = e2 >= 0;
  if (interior) {
#pragma unroll
    for (int k = 0; k < NFP; ++k) {
      const size_t b = (size_t)e2 * NP + ops.fmask[f2 * NFP + (NFP - 1 - k)];
#pragma unroll
      for (int v = 0; v < NV; ++v) Tp[v][k] = V[v * KN + b];
#pragma unroll
      for (int c = 0; c < NE; ++c) Tp[NV + c][k] = E[c * KN + b];
    }
  } else {
#pragma unroll
    for (int r = 0; r < NV + NE; ++r)
#pragma unroll
      for (int k = 0; k < NFP; ++k) Tp[r][k] = Tm[r][k];
  }
  const size_t FQ = (size_t)F * NFQ;
#pragma unroll
  for (int m = 0; m < NFQ; ++m)
    face_point<DIM, P, R>(m, Tm, Tp, interior, bct, -1 - e2, n, wsj, ops, ph, wflux, FQ, (size_t)fc * NFQ + m);
}

template <int DIM, int P, typename R>
constexpr int face_pf_min_blocks() {
  return (sizeof(R) == 4 && P <= 2) ? 2 : 1;
}

template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256, face_pf_min_blocks<DIM, P, R>())
    face_pf_kernel(int K, int F, const R* __restrict__ V, const R* __restrict__ E, const int32_t* __restrict__ fe1,
                   const int8_t* __restrict__ ff1, const int32_t* __restrict__ fe2, const int8_t* __restrict__ ff2,
                   const R* __restrict__ fnrm, const R* __restrict__ fsj, R* __restrict__ wflux,
                   const FaceOps<DIM, P, R> ops, const Phys<R>* __restrict__ ptab, const int32_t* __restrict__ inst,
                   const BCEntry<R>* __restrict__ bct) {
  const int stride = gridDim.x * blockDim.x;
  int fc = blockIdx.x * blockDim.x + threadIdx.x;
  if (fc >= F) return;
  int e1 = fe1[fc], f1 = ff1[fc], e2 = fe2[fc], f2 = ff2[fc];
  R n[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) n[i] = fnrm[(size_t)i * F + fc];
  R wsj = fsj[fc];
  for (;;) {
    const int nx = fc + stride;
    const bool more = nx < F && nx > fc;  // (nx > fc: no int overflow past F)
    int e1n = 0, f1n = 0, e2n = -1, f2n = 0;
    R nn[DIM], wsjn = R(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) nn[i] = R(0);
    if (more) {
      e1n = fe1[nx];
      f1n = ff1[nx];
      e2n = fe2[nx];
      f2n = ff2[nx];
#pragma unroll
      for (int i = 0; i < DIM; ++i) nn[i] = fnrm[(size_t)i * F + nx];
      wsjn = fsj[nx];
    }
    face_pf_body<DIM, P, R>(fc, e1, f1, e2, f2, n, wsj, K, F, V, E, wflux, ops, ptab, inst, bct);
    if (!more) break;
    fc = nx;
    e1 = e1n;
    f1 = f1n;
    e2 = e2n;
    f2 = f2n;
#pragma unroll
    for (int i = 0; i < DIM; ++i) n[i] = nn[i];
    wsj = wsjn;
  }
}

// E-step over a grid-stride loop, for batch groups: the face neighbours (and
// their local faces) of a thread's next element are loaded while the current
// element is computed, so the neighbour-trace gathers need no dependent
// round trip to the connectivity first.  Same arithmetic as estep_kernel.
template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256) estep_pf_kernel(int K, const R* __restrict__ V, R* __restrict__ E,
                                                       const R* __restrict__ geo, const int32_t* __restrict__ nbr,
                                                       const int8_t* __restrict__ nbrf, const R* __restrict__ fn,
                                                       const R* __restrict__ fsj, const EstepOps<DIM, P, R> ops,
                                                       const BCEntry<R>* __restrict__ bct) {
  constexpr int NF = Sh<DIM, P>::NF;
  const int stride = gridDim.x * blockDim.x;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  int nb[NF], nbf[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    nb[f] = nbr[f * K + e];
    nbf[f] = nbrf[f * K + e];
  }
  for (;;) {
    const int nx = e + stride;
    const bool more = nx < K && nx > e;  // (nx > e: no int overflow past K)
    int nbn[NF], nbfn[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      nbn[f] = more ? nbr[f * K + nx] : 0;
      nbfn[f] = more ? (int)nbrf[f * K + nx] : 0;
    }
    estep_element<DIM, P, R, false, true>(e, K, V, E, geo, nbr, nbrf, fn, fsj, ops, bct, nb, nbf);
    if (!more) break;
    e = nx;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      nb[f] = nbn[f];
      nbf[f] = nbfn[f];
    }
  }
}

// Unroll factor of the wet/dry stage's loops: full below 2D p = 3, none there.
template <int DIM, int P>
constexpr int wd_unroll() {
  return (DIM == 2 && P == 3) ? 1 : 64;
}

// Depth limiter of one element's nodal depths h (in the stage's compute type
// T), part of the wet/dry stage below (Zhang-Shu scaling of h): with hbar the cell average of h and m
// its minimum over the nodes, the volume quadrature points and the face
// quadrature points, hbar <= 0 gives h = 0, m < 0 < hbar gives
// h <- hbar + theta (h - hbar) with theta = hbar / (hbar - m).  Returns hbar.
template <int DIM, int P, typename R, typename T>
__device__ __forceinline__ T limit_depth(T* h, const VolOps<DIM, P, R>& ops) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NQ = S::NQ, NF = S::NF, NFP = S::NFP, NFQ = S::NFQ;
  T hbar = T(0), m = h[0];
#pragma unroll (wd_unroll<DIM, P>())
  for (int a = 0; a < NP; ++a) {
    hbar += (T)ops.wavg[a] * h[a];
    m = fmin(m, h[a]);
  }
#pragma unroll (wd_unroll<DIM, P>())
  for (int q = 0; q < NQ; ++q) {
    T hq = T(0);
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = 0; a < NP; ++a) hq += (T)ops.Vq[q * NP + a] * h[a];
    m = fmin(m, hq);
  }
#pragma unroll (wd_unroll<DIM, P>())
  for (int f = 0; f < NF; ++f)
#pragma unroll (wd_unroll<DIM, P>())
    for (int mq = 0; mq < NFQ; ++mq) {
      T hf = T(0);
#pragma unroll (wd_unroll<DIM, P>())
      for (int k = 0; k < NFP; ++k) hf += (T)ops.LfT[k * NFQ + mq] * h[face_node(DIM, P, f, k)];
      m = fmin(m, hf);
    }
  if (hbar <= T(0)) {
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = 0; a < NP; ++a) h[a] = T(0);
  } else if (m < T(0)) {
    const T theta = hbar / (hbar - m);
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = 0; a < NP; ++a) h[a] = hbar + theta * (h[a] - hbar);
  }
  return hbar;
}

// One explicit stage of wet/dry mode (dg_swe_params.positivity), taken on the
// moments <N, U> of the conservative unknowns U = (h, h u), the quantity whose
// difference the time term of Eq. WeakForm7 holds, instead of on V:
//   <N, U(y)> = c0 <N, U(V0)> + c1 (<N, U(Vs)> - dt r_V(Vs)).
// Solved for y (reference scaling, r times 1/J): the depth from M y_h = ...,
// i.e. y_h = c0 h0 + c1 (hs - dt M^-1 r_h / J); y_h through limit_depth; then
// M_h y_u = c0 <psi, h0 u0> + c1 (<psi, hs us> - dt r_u / J) with
// M_h = <psi, max(y_h, h_floor) psi>, the products formed at the volume
// quadrature points; y_u = 0 where the mean depth is below h_floor.  The
// primitive stage divides the momentum change by the stage's starting depth,
// zero in a dry element; this one divides the new momentum by the new depth.
// Computed in T: FP64 in FP64 contexts and for near-dry elements of FP32
// contexts, FP32 for their wet elements (wetdry_stage_kernel chooses, as
// mass_solve_dispatch does for the primitive stages); loops unrolled up to
// p = 2 (2D p = 3 keeps them rolled: unrolled, its arrays spilled 13 KB per
// thread).  Runs in its own
// kernel (wetdry_stage_kernel) after the volume pass has written r_V, so the
// fused volume kernels carry none of it.  Writes y to
// out (field stride KN, element offset eo).
template <int DIM, int P, typename R, typename T, bool COH = false>
__device__ __forceinline__ void conservative_stage(const R (&Vn)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                                   const R (&r)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                                   const R* const (&V0e)[Sh<DIM, P>::NV], R c0, R c1, double dt_in,
                                                   const VolOps<DIM, P, R>& ops, R h_floor, R Jinv, R* out,
                                                   size_t KN, size_t eo) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NQ = S::NQ, NV = S::NV;
  T V[NV * NP], V0[NV * NP], rr[NV * NP], y[NV * NP], mom[DIM * NP], Mh[NP * NP], dinv[NP], z[NP];
#pragma unroll (wd_unroll<DIM, P>())
  for (int v = 0; v < NV; ++v)
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = 0; a < NP; ++a) {
      V[v * NP + a] = (T)Vn[v][a];
      V0[v * NP + a] = c0 != R(0) ? (T)DG_LDC(COH, V0e[v], a) : T(0);
      rr[v * NP + a] = (T)r[v][a];
    }
  const T jinv = (T)Jinv, hf = (T)h_floor, a0 = (T)c0, a1 = (T)c1;
  const T dt = (T)dt_in;
  // depth
#pragma unroll (wd_unroll<DIM, P>())
  for (int a = 0; a < NP; ++a) {
    T acc = T(0);
#pragma unroll (wd_unroll<DIM, P>())
    for (int b = 0; b < NP; ++b) acc += (T)ops.Minv[a * NP + b] * rr[b];
    y[a] = a1 * (V[a] - dt * acc * jinv) + a0 * V0[a];
  }
  const T hbar = limit_depth<DIM, P, R, T>(y, ops);
  // momentum moments and M_h of the limited depth
#pragma unroll (wd_unroll<DIM, P>())
  for (int i = 0; i < DIM * NP; ++i) mom[i] = -a1 * dt * jinv * rr[NP + i];
#pragma unroll (wd_unroll<DIM, P>())
  for (int i = 0; i < NP * NP; ++i) Mh[i] = T(0);
#pragma unroll (wd_unroll<DIM, P>())
  for (int q = 0; q < NQ; ++q) {
    T hs = T(0), h0 = T(0), hy = T(0), us[DIM], u0[DIM];
#pragma unroll (wd_unroll<DIM, P>())
    for (int j = 0; j < DIM; ++j) us[j] = u0[j] = T(0);
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = 0; a < NP; ++a) {
      const T l = (T)ops.Vq[q * NP + a];
      hs += l * V[a];
      h0 += l * V0[a];
      hy += l * y[a];
#pragma unroll (wd_unroll<DIM, P>())
      for (int j = 0; j < DIM; ++j) {
        us[j] += l * V[(1 + j) * NP + a];
        u0[j] += l * V0[(1 + j) * NP + a];
      }
    }
    const T w = (T)ops.wq[q];
    const T wh = w * fmax(hy, hf);
    T mq[DIM];
#pragma unroll (wd_unroll<DIM, P>())
    for (int j = 0; j < DIM; ++j) mq[j] = w * (a1 * hs * us[j] + a0 * h0 * u0[j]);
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = 0; a < NP; ++a) {
      const T la = (T)ops.Vq[q * NP + a];
#pragma unroll (wd_unroll<DIM, P>())
      for (int j = 0; j < DIM; ++j) mom[j * NP + a] += mq[j] * la;
      const T t = wh * la;
#pragma unroll (wd_unroll<DIM, P>())
      for (int b = 0; b <= a; ++b) Mh[a * NP + b] += t * (T)ops.Vq[q * NP + b];
    }
  }
  // Cholesky of M_h (lower triangle, reciprocal diagonal) and the solves
#pragma unroll (wd_unroll<DIM, P>())
  for (int a = 0; a < NP; ++a) {
#pragma unroll (wd_unroll<DIM, P>())
    for (int b = 0; b < a; ++b) {
      T sum = Mh[a * NP + b];
#pragma unroll (wd_unroll<DIM, P>())
      for (int c = 0; c < b; ++c) sum -= Mh[a * NP + c] * Mh[b * NP + c];
      Mh[a * NP + b] = sum * dinv[b];
    }
    T d = Mh[a * NP + a];
#pragma unroll (wd_unroll<DIM, P>())
    for (int c = 0; c < a; ++c) d -= Mh[a * NP + c] * Mh[a * NP + c];
    dinv[a] = T(1) / sqrt(d);
  }
  const bool dry = hbar < hf;
#pragma unroll (wd_unroll<DIM, P>())
  for (int j = 0; j < DIM; ++j) {
    T* u = y + (1 + j) * NP;
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = 0; a < NP; ++a) {
      T sum = mom[j * NP + a];
#pragma unroll (wd_unroll<DIM, P>())
      for (int c = 0; c < a; ++c) sum -= Mh[a * NP + c] * z[c];
      z[a] = sum * dinv[a];
    }
#pragma unroll (wd_unroll<DIM, P>())
    for (int a = NP - 1; a >= 0; --a) {
      T sum = z[a];
#pragma unroll (wd_unroll<DIM, P>())
      for (int c = a + 1; c < NP; ++c) sum -= Mh[c * NP + a] * u[c];
      u[a] = dry ? T(0) : sum * dinv[a];
    }
  }
#pragma unroll (wd_unroll<DIM, P>())
  for (int i = 0; i < NV * NP; ++i) out[(i / NP) * KN + eo + i % NP] = (R)y[i];
}

// Primitive-variable mass solve of one element (Appendix A, dU/dV):
// dV = -M(V)^{-1} r, i.e. M dh/dt = -r_h and M_h du/dt = -r_u - M_u dh/dt,
// with M_h = <psi, max(h, h_floor) psi> and M_u = <psi, u psi> at the volume
// quadrature points; r in physical scaling, Jinv = 1 / J.
// STASH: the depth and velocity at the volume points arrive in Vqs (kept
// from the volume-integral loop) instead of being interpolated again, and
// M_h is assembled as sum_q max(h_q, h_floor) (w_q l_a l_b), the products
// w_q l_a l_b read from pm (mass_products: the shared operator table) or,
// with pm = nullptr, formed in the same order here.
template <int DIM, int P, typename R>
__host__ __device__ constexpr int mass_products_pad() {
  return (int)(((Sh<DIM, P>::NP * (Sh<DIM, P>::NP + 1) / 2 * sizeof(R) + 15) / 16) * 16 / sizeof(R));
}
template <int DIM, int P, typename R, bool STASH = false>
__device__ __forceinline__ void mass_solve_element(const R (&Vn)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                                   const R (&r)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                                   const VolOps<DIM, P, R>& ops, R h_floor, R Jinv,
                                                   R (&dV)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                                   const R (*Vqs)[Sh<DIM, P>::NV] = nullptr,
                                                   const R* pm = nullptr) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NQ = S::NQ;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    R acc = R(0);
#pragma unroll
    for (int b = 0; b < NP; ++b) acc += ops.Minv[a * NP + b] * r[0][b];
    dV[0][a] = -acc * Jinv;
  }
  R Mh[NP][NP];
  R rhs[DIM][NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = 0; b < NP; ++b) Mh[a][b] = R(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j) rhs[j][a] = -r[1 + j][a] * Jinv;
  }
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    R hq = R(0), hdq = R(0), uq[DIM];
    if constexpr (STASH) {
      hq = Vqs[q][0];
#pragma unroll
      for (int j = 0; j < DIM; ++j) uq[j] = Vqs[q][1 + j];
#pragma unroll
      for (int a = 0; a < NP; ++a) hdq += ops.Vq[q * NP + a] * dV[0][a];
    } else {
#pragma unroll
      for (int j = 0; j < DIM; ++j) uq[j] = R(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        const R l = ops.Vq[q * NP + a];
        hq += l * Vn[0][a];
        hdq += l * dV[0][a];
#pragma unroll
        for (int j = 0; j < DIM; ++j) uq[j] += l * Vn[1 + j][a];
      }
    }
    const R wd = ops.wq[q] * hdq;
    if constexpr (STASH) {
      const R hf = fmax(hq, h_floor);
      constexpr int MPAD = mass_products_pad<DIM, P, R>();
      R pq[MPAD];
      if (pm) {
        const double2* p2 = reinterpret_cast<const double2*>(pm + q * MPAD);
#pragma unroll
        for (int c = 0; c < MPAD / 2; ++c) {
          const double2 v = p2[c];
          pq[2 * c] = v.x;
          pq[2 * c + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int a = 0, i = 0; a < NP; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b, ++i) pq[i] = (ops.wq[q] * ops.Vq[q * NP + a]) * ops.Vq[q * NP + b];
      }
#pragma unroll
      for (int a = 0, i = 0; a < NP; ++a) {
#pragma unroll
        for (int b = 0; b <= a; ++b, ++i) Mh[a][b] += hf * pq[i];
        const R la = ops.Vq[q * NP + a];
#pragma unroll
        for (int j = 0; j < DIM; ++j) rhs[j][a] -= wd * uq[j] * la;
      }
    } else {
      const R wh = ops.wq[q] * fmax(hq, h_floor);
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        const R la = ops.Vq[q * NP + a];
        const R t = wh * la;
#pragma unroll
        for (int b = 0; b <= a; ++b) Mh[a][b] += t * ops.Vq[q * NP + b];
#pragma unroll
        for (int j = 0; j < DIM; ++j) rhs[j][a] -= wd * uq[j] * la;
      }
    }
  }
  // Cholesky of the reference-scaled M_h (lower triangle); the diagonal is
  // kept as reciprocals so the factorization and both triangular solves
  // multiply instead of divide (NP divisions per element instead of
  // NP (NP + 3) / 2 + 2 DIM NP).
  R dinv[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = 0; b < a; ++b) {
      R s = Mh[a][b];
#pragma unroll
      for (int c = 0; c < b; ++c) s -= Mh[a][c] * Mh[b][c];
      Mh[a][b] = s * dinv[b];
    }
    R d = Mh[a][a];
#pragma unroll
    for (int c = 0; c < a; ++c) d -= Mh[a][c] * Mh[a][c];
    dinv[a] = dg_rsqrt<R>(d);
  }
#pragma unroll
  for (int j = 0; j < DIM; ++j) {
    R y[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      R s = rhs[j][a];
#pragma unroll
      for (int c = 0; c < a; ++c) s -= Mh[a][c] * y[c];
      y[a] = s * dinv[a];
    }
#pragma unroll
    for (int a = NP - 1; a >= 0; --a) {
      R s = y[a];
#pragma unroll
      for (int c = a + 1; c < NP; ++c) s -= Mh[c][a] * dV[1 + j][c];
      dV[1 + j][a] = s * dinv[a];
    }
  }
}

// Near-dry treatment of FP32 contexts: an element whose smallest nodal depth
// is below h_dry (kDryFactor x h_floor) assembles and solves its h-weighted
// mass matrix in FP64 (the depths at the quadrature points, M_h = <psi,
// max(h, h_floor) psi>, M_u dh/dt, the Cholesky factorization and both
// triangular solves), from its FP32 nodal values and residual.  There M_h
// has entries of the size of the floor next to entries a thousand times
// larger, and FP32 would lose their relative accuracy.  The FP64 solve runs
// in loops over per-thread local arrays: it is rare (fronts and films only)
// and must not add registers to the FP32 kernels' common path.  FP64
// contexts and wet elements take the working-precision solve
// (mass_solve_element), whose formulas this restates.
constexpr double kDryFactor = 1000.0;

template <int DIM, int P>
__device__ __forceinline__ void mass_solve_dry(const float (&Vn)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                               const float (&r)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                               const VolOps<DIM, P, float>& ops, float h_floor, float Jinv,
                                               float (&dVout)[Sh<DIM, P>::NV][Sh<DIM, P>::NP]) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NQ = S::NQ, NV = S::NV;
  double V[NV * NP], dV[NV * NP], Mh[NP * NP], rhs[DIM * NP], dinv[NP], y[NP];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) V[v * NP + a] = (double)Vn[v][a];
  const double jinv = (double)Jinv, hf = (double)h_floor;
#pragma unroll 1
  for (int a = 0; a < NP; ++a) {
    double acc = 0.0;
#pragma unroll 1
    for (int b = 0; b < NP; ++b) acc += (double)ops.Minv[a * NP + b] * (double)r[0][b];
    dV[a] = -acc * jinv;
  }
#pragma unroll 1
  for (int i = 0; i < NP * NP; ++i) Mh[i] = 0.0;
#pragma unroll 1
  for (int a = 0; a < NP; ++a)
#pragma unroll 1
    for (int j = 0; j < DIM; ++j) rhs[j * NP + a] = -(double)r[1 + j][a] * jinv;
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    double hq = 0.0, hdq = 0.0, uq[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) uq[j] = 0.0;
#pragma unroll 1
    for (int a = 0; a < NP; ++a) {
      const double l = (double)ops.Vq[q * NP + a];
      hq += l * V[a];
      hdq += l * dV[a];
#pragma unroll
      for (int j = 0; j < DIM; ++j) uq[j] += l * V[(1 + j) * NP + a];
    }
    const double wh = (double)ops.wq[q] * fmax(hq, hf);
    const double wd = (double)ops.wq[q] * hdq;
#pragma unroll 1
    for (int a = 0; a < NP; ++a) {
      const double la = (double)ops.Vq[q * NP + a];
      const double t = wh * la;
#pragma unroll 1
      for (int b = 0; b <= a; ++b) Mh[a * NP + b] += t * (double)ops.Vq[q * NP + b];
#pragma unroll
      for (int j = 0; j < DIM; ++j) rhs[j * NP + a] -= wd * uq[j] * la;
    }
  }
#pragma unroll 1
  for (int a = 0; a < NP; ++a) {
#pragma unroll 1
    for (int b = 0; b < a; ++b) {
      double sum = Mh[a * NP + b];
#pragma unroll 1
      for (int c = 0; c < b; ++c) sum -= Mh[a * NP + c] * Mh[b * NP + c];
      Mh[a * NP + b] = sum * dinv[b];
    }
    double d = Mh[a * NP + a];
#pragma unroll 1
    for (int c = 0; c < a; ++c) d -= Mh[a * NP + c] * Mh[a * NP + c];
    dinv[a] = rsqrt(d);
  }
#pragma unroll 1
  for (int j = 0; j < DIM; ++j) {
#pragma unroll 1
    for (int a = 0; a < NP; ++a) {
      double sum = rhs[j * NP + a];
#pragma unroll 1
      for (int c = 0; c < a; ++c) sum -= Mh[a * NP + c] * y[c];
      y[a] = sum * dinv[a];
    }
#pragma unroll 1
    for (int a = NP - 1; a >= 0; --a) {
      double sum = y[a];
#pragma unroll 1
      for (int c = a + 1; c < NP; ++c) sum -= Mh[c * NP + a] * dV[(1 + j) * NP + c];
      dV[(1 + j) * NP + a] = sum * dinv[a];
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) dVout[v][a] = (float)dV[v * NP + a];
}

template <int DIM, int P, typename R>
__device__ __forceinline__ void mass_solve_dispatch(const R (&Vn)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                                    const R (&r)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                                    const VolOps<DIM, P, R>& ops, const Phys<R>& ph, R Jinv,
                                                    R (&dV)[Sh<DIM, P>::NV][Sh<DIM, P>::NP]) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP;
  if constexpr (sizeof(R) == 4) {
    R hmin = Vn[0][0];
#pragma unroll
    for (int a = 1; a < NP; ++a) hmin = fmin(hmin, Vn[0][a]);
    if (hmin < ph.h_dry) {
      mass_solve_dry<DIM, P>(Vn, r, ops, ph.h_floor, Jinv, dV);
      return;
    }
  }
  mass_solve_element<DIM, P, R>(Vn, r, ops, ph.h_floor, Jinv, dV);
}

// Per-volume-point operator rows (Vq, Wr, Ws, Wm) of the direct
// FP64 2D volume kernel, copied once per block into shared memory with each
// row padded to 16 bytes, so that a row arrives in 128-bit loads instead of
// one constant-bank load per value (FP64 headline volume kernel: 0.401 ->
// 0.389 ms).  FP32 keeps the constant-bank reads, which measured faster
// there (0.252 vs 0.386 ms on 2M triangles); so does the staged kernel,
// whose shared memory holds its element tiles (tab = nullptr), and 1D,
// where the fill cost more than it saved (200-element dam break: -5 %).
template <int DIM, int P, typename R>
struct QTab {
  static constexpr int NP = Sh<DIM, P>::NP, NQ = Sh<DIM, P>::NQ, ROWS = 4;
  static constexpr int PAD = (int)(((NP * sizeof(R) + 15) / 16) * 16 / sizeof(R));
  static constexpr bool USED = sizeof(R) == 8 && DIM == 2;
  // after the rows: per volume point the mass products w_q l_a l_b (b <= a,
  // row by row) of the FP64 mass solve, padded to 16 bytes
  static constexpr int MBASE = NQ * ROWS * PAD, MPAD = mass_products_pad<DIM, P, R>();
  static constexpr int SIZE = USED ? MBASE + NQ * MPAD : 2;
};
template <int DIM, int P, typename R>
__device__ __forceinline__ void qtab_fill(R* tab, const VolOps<DIM, P, R>& ops) {
  using T = QTab<DIM, P, R>;
  if constexpr (T::USED) {
    for (int i = threadIdx.x; i < T::MBASE; i += blockDim.x) {
      const int q = i / (T::ROWS * T::PAD), k = (i / T::PAD) % T::ROWS, a = i % T::PAD;
      R v = R(0);
      if (a < T::NP) {
        const int j = q * T::NP + a;
        v = k == 0 ? ops.Vq[j] : k == 1 ? ops.Wr[j] : k == 2 ? ops.Ws[j] : ops.Wm[j];
      }
      tab[i] = v;
    }
    for (int i = threadIdx.x; i < T::NQ * T::MPAD; i += blockDim.x) {
      const int q = i / T::MPAD, idx = i % T::MPAD;
      R v = R(0);
      if (idx < T::NP * (T::NP + 1) / 2) {
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= idx) ++a;
        const int b = idx - a * (a + 1) / 2;
        v = (ops.wq[q] * ops.Vq[q * T::NP + a]) * ops.Vq[q * T::NP + b];
      }
      tab[T::MBASE + i] = v;
    }
  }
}
// Row ROW of volume point q: from the shared table (FP64) or the operator
// parameters (FP32).
template <int DIM, int P, int ROW, typename R>
__device__ __forceinline__ void op_row(const VolOps<DIM, P, R>& ops, const R* tab, int q,
                                       R (&out)[Sh<DIM, P>::NP]) {
  using T = QTab<DIM, P, R>;
  constexpr int NP = T::NP;
  if constexpr (T::USED) {
    if (tab) {
      const double2* p = reinterpret_cast<const double2*>(tab + (q * T::ROWS + ROW) * T::PAD);
      double tmp[T::PAD];
#pragma unroll
      for (int c = 0; c < T::PAD / 2; ++c) {
        const double2 v = p[c];
        tmp[2 * c] = v.x;
        tmp[2 * c + 1] = v.y;
      }
#pragma unroll
      for (int a = 0; a < NP; ++a) out[a] = tmp[a];
      return;
    }
  }
  const R* tabsrc = ROW == 0 ? ops.Vq : ROW == 1 ? ops.Wr : ROW == 2 ? ops.Ws : ops.Wm;
#pragma unroll
  for (int a = 0; a < NP; ++a) out[a] = tabsrc[q * NP + a];
}

// Everything the volume kernels do for one element e once its nodal values
// are in registers: volume integrals, face lift, mass solve and output.
// Bed and slope source S_j = -g_c h dH/dx_j - g_s h delta_1j (Eq. Sterm).
// FP64 contexts read the coefficients c_j = -g_c dH/dx_j - g_s delta_1j at the
// volume points from src ([DIM * NQ][K], host-computed once since the bed does
// not change), which saves the FP64 kernels (bound by the FP64 pipe) the
// interpolation of the bed gradient; FP32 contexts (latency-bound, where the
// extra global loads inside the point loop cost more than the arithmetic)
// interpolate the gradient from the element's nodal bed bed_e.  Both nullptr:
// flat bed (the slope term -g_s h remains).  V0e[v]: the
// element's values of field v of the stage's first state (read in mode 1
// when c0 != 0).  mode 0: write dV/dt to out; mode 1: out = c0 * V0 + c1 * (Vin +
// dt * dV/dt); mode 2: write the spatial residual r_V of Eq. WeakForm51
// (before the mass solve).
template <int DIM, int P, typename R, bool COH = false>
__device__ __forceinline__ void volume_element(int e, int K, int F, const R (&Vn)[Sh<DIM, P>::NV][Sh<DIM, P>::NP],
                                               const R (&En)[Sh<DIM, P>::NE][Sh<DIM, P>::NP],
                                               const R* __restrict__ bed_e, const R* __restrict__ src,
                                               const R* const (&V0e)[Sh<DIM, P>::NV],
                                               R* out,
                                               const R* __restrict__ geo, const int32_t* __restrict__ fid,
                                               const R* __restrict__ wflux, const VolOps<DIM, P, R>& ops,
                                               const Phys<R>& ph, int ins, int mode, R c0, R c1,
                                               const DevScalars* __restrict__ sc, const R* tab) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NQ = S::NQ, NF = S::NF, NFP = S::NFP, NFQ = S::NFQ, NV = S::NV, NE = S::NE;
  const size_t KN = (size_t)K * NP;
  const size_t eo = (size_t)e * NP;
  R G[2][2];
  G[0][0] = geo[e];
  if constexpr (DIM == 2) {
    G[0][1] = geo[K + e];
    G[1][0] = geo[2 * K + e];
    G[1][1] = geo[3 * K + e];
  }
  const R J = geo[4 * K + e];
  R r[NV][NP];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) r[v][a] = R(0);

  const bool has_src = sizeof(R) == 8 && src != nullptr;
  const bool has_bed = sizeof(R) == 4 && bed_e != nullptr;
  // FP64: the depth and velocity at the volume points, kept for the mass
  // solve (per-thread local memory; saves its interpolation of them).  The
  // FP32 kernels, issue-bound, ran slower with it (8.4M-triangle slump
  // volume 0.97 -> 1.07 ms) and interpolate again.
  constexpr bool kStash = sizeof(R) == 8;
  R Vqs[kStash ? NQ : 1][NV];
  R Hn[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) Hn[a] = has_bed ? bed_e[a] : R(0);

  // ---- volume integrals: -<grad N, F - Q> - <N, S>  (Eq. WeakForm51)
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    R Vq[NV], Eq[NE];
#pragma unroll
    for (int v = 0; v < NV; ++v) Vq[v] = R(0);
#pragma unroll
    for (int c = 0; c < NE; ++c) Eq[c] = R(0);
    R Hr = R(0), Hs = R(0);
    if constexpr (QTab<DIM, P, R>::USED) {
    R rvq[NP];
    op_row<DIM, P, 0>(ops, tab, q, rvq);
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const R l = rvq[a];
#pragma unroll
      for (int v = 0; v < NV; ++v) Vq[v] += l * Vn[v][a];
#pragma unroll
      for (int c = 0; c < NE; ++c) Eq[c] += l * En[c][a];
    }
    } else {
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const R l = ops.Vq[q * NP + a];
#pragma unroll
      for (int v = 0; v < NV; ++v) Vq[v] += l * Vn[v][a];
#pragma unroll
      for (int c = 0; c < NE; ++c) Eq[c] += l * En[c][a];
      if (has_bed) {
        Hr += ops.Drq[q * NP + a] * Hn[a];
        if constexpr (DIM == 2) Hs += ops.Dsq[q * NP + a] * Hn[a];
      }
    }
    }
    if constexpr (kStash) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Vqs[q][v] = Vq[v];
    }
    const R h = Vq[0];
    const R hr = h * ph.rho_inv;
    R sig[DIM][DIM];
    stress<DIM, R>(Eq, ph, sig);
    R fx[DIM][NV];  // (Q - F) in direction i
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      fx[i][0] = -h * Vq[1 + i];
#pragma unroll
      for (int j = 0; j < DIM; ++j) fx[i][1 + j] = -h * Vq[1 + i] * Vq[1 + j] + hr * sig[j][i];
      fx[i][1 + i] -= R(0.5) * ph.gc * h * h;
    }
    R Sv[NV];
    Sv[0] = R(0);
    if (has_src) {
#pragma unroll
      for (int jj = 0; jj < DIM; ++jj) Sv[1 + jj] = h * src[(size_t)(jj * NQ + q) * K + e];
    } else {
      R dH[DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        dH[i] = G[0][i] * Hr;
        if constexpr (DIM == 2) dH[i] += G[1][i] * Hs;
      }
#pragma unroll
      for (int j = 0; j < DIM; ++j) Sv[1 + j] = -ph.gc * h * dH[j];
      Sv[1] -= ph.gs * h;
    }
    R fr[NV], fs[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      fr[v] = G[0][0] * fx[0][v];
      fs[v] = R(0);
      if constexpr (DIM == 2) {
        fr[v] += G[0][1] * fx[1][v];
        fs[v] = G[1][0] * fx[0][v] + G[1][1] * fx[1][v];
      }
    }
    R rwr[NP], rws[NP], rwm[NP];
    if constexpr (QTab<DIM, P, R>::USED) {
      op_row<DIM, P, 1>(ops, tab, q, rwr);
      if constexpr (DIM == 2) op_row<DIM, P, 2>(ops, tab, q, rws);
      op_row<DIM, P, 3>(ops, tab, q, rwm);
    }
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const R wr = QTab<DIM, P, R>::USED ? rwr[a] : ops.Wr[q * NP + a];
      const R ws = DIM == 1 ? R(0) : QTab<DIM, P, R>::USED ? rws[a] : ops.Ws[q * NP + a];
      const R wm = QTab<DIM, P, R>::USED ? rwm[a] : ops.Wm[q * NP + a];
      // accumulated straight into r, three fused multiply-adds per entry
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R t = r[v][a];
        t += wr * fr[v];
        if constexpr (DIM == 2) t += ws * fs[v];
        if (v > 0) t -= wm * Sv[v];  // the depth equation has no source
        r[v][a] = t;
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) r[v][a] *= J;

  // ---- face terms <N^-, F_bar.n - Q_bar.n> (weights and sJ folded into wflux)
  const size_t FQ = (size_t)F * NFQ;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const uint32_t raw = (uint32_t)fid[f * K + e];
    const bool own = (raw & 0x80000000u) == 0;
    const size_t base = (size_t)(raw & 0x7fffffffu) * NFQ;
    R fv[NV][NFQ];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int m = 0; m < NFQ; ++m) {
        const R x = DG_LDC(COH, wflux, v * FQ + base + (own ? m : NFQ - 1 - m));
        fv[v][m] = own ? x : -x;
      }
#pragma unroll
    for (int k = 0; k < NFP; ++k) {
      const int a = face_node(DIM, P, f, k);
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < NFQ; ++m) r[v][a] += ops.LfT[k * NFQ + m] * fv[v][m];
    }
  }

  // mode 2: the spatial residual r_V itself (physical scaling), for the
  // implicit integrators that assemble their own time term
  if (mode == 2) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int a = 0; a < NP; ++a) out[v * KN + eo + a] = r[v][a];
    return;
  }

  // ---- mass solve: M dh/dt = -r_h ; M_h du/dt = -r_u - M_u dh/dt
  R dV[NV][NP];
  if constexpr (kStash)
    mass_solve_element<DIM, P, R, true>(Vn, r, ops, ph.h_floor, geo[6 * K + e], dV, Vqs,
                                        (QTab<DIM, P, R>::USED && tab) ? tab + QTab<DIM, P, R>::MBASE : nullptr);
  else
    mass_solve_dispatch<DIM, P, R>(Vn, r, ops, ph, geo[6 * K + e], dV);

  // ---- output
  if (mode == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int a = 0; a < NP; ++a) out[v * KN + eo + a] = dV[v][a];
  } else {
    const R dt = (R)DG_LDC(COH, &sc[ins].dt, 0);
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        const R vi = Vn[v][a];
        R y = c1 * (vi + dt * dV[v][a]);
        if (c0 != R(0)) y += c0 * DG_LDC(COH, V0e[v], a);
        dV[v][a] = y;
      }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int a = 0; a < NP; ++a) out[v * KN + eo + a] = dV[v][a];
  }
}

// Register cap of the direct volume kernel: 168 for FP32 at p = 3, the most
// that keeps three warps on each SM sub-partition (16,384 registers each; the
// autotuner picks 32-thread blocks for this kernel).  Left to the compiler
// it took 171 (176 allocated), two warps per sub-partition, and the p = 3
// bump volume pass ran 0.40 instead of 0.30 ms.  Otherwise no cap.
template <int DIM, int P, typename R>
constexpr int volume_max_regs() {
  return (sizeof(R) == 4 && P == 3) ? 168 : 255;
}

// One thread per element; nodal values read straight from global memory.
template <int DIM, int P, typename R, bool BATCH>
__global__ void __launch_bounds__(256) __maxnreg__((volume_max_regs<DIM, P, R>())) volume_kernel(int K, int F, const R* __restrict__ Vin,
                                                     const R* V0, R* out,
                                                     const R* __restrict__ E, const R* __restrict__ bed, const R* __restrict__ src,
                                                     const R* __restrict__ geo, const int32_t* __restrict__ fid,
                                                     const R* __restrict__ wflux, const VolOps<DIM, P, R> ops,
                                                     const Phys<R> ph0, const Phys<R>* __restrict__ ptab,
                                                     const int32_t* __restrict__ inst, int mode, R c0, R c1,
                                                     const DevScalars* __restrict__ sc) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NV = S::NV, NE = S::NE;
  __shared__ __align__(16) R tab[QTab<DIM, P, R>::SIZE];
  qtab_fill<DIM, P, R>(tab, ops);
  if constexpr (QTab<DIM, P, R>::USED) __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  const int ins = BATCH ? inst[e] : 0;
  const Phys<R> ph = BATCH ? ptab[ins] : ph0;
  const size_t KN = (size_t)K * NP;
  const size_t eo = (size_t)e * NP;
  // the element's nodal values, read once (each is used at every volume point)
  R Vn[NV][NP], En[NE][NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Vn[v][a] = Vin[v * KN + eo + a];
#pragma unroll
    for (int c = 0; c < NE; ++c) En[c][a] = E[c * KN + eo + a];
  }
  const R* V0e[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) V0e[v] = V0 ? V0 + v * KN + eo : nullptr;
  volume_element<DIM, P, R>(e, K, F, Vn, En, bed ? bed + eo : nullptr, src, V0e, out, geo, fid, wflux, ops, ph, ins, mode,
                            c0, c1, sc, tab);
}

// Stage update of wet/dry mode, one thread per element: after a volume pass
// in mode 2 has written the residual r_V of the stage's input state to rbuf,
// out = the conservative stage (conservative_stage) from Vin, V0 and rbuf.
// rbuf and V0 may alias out: each thread reads its element's values of all
// three before it writes.
template <int DIM, int P, typename R, bool BATCH>
__global__ void __launch_bounds__(128) wetdry_stage_kernel(int K, const R* __restrict__ Vin, const R* V0,
                                                           const R* rbuf, R* out, const R* __restrict__ geo,
                                                           const VolOps<DIM, P, R> ops, const Phys<R> ph0,
                                                           const Phys<R>* __restrict__ ptab,
                                                           const int32_t* __restrict__ inst, R c0, R c1,
                                                           const DevScalars* __restrict__ sc) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NV = S::NV;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  const int ins = BATCH ? inst[e] : 0;
  const Phys<R> ph = BATCH ? ptab[ins] : ph0;
  const size_t KN = (size_t)K * NP;
  const size_t eo = (size_t)e * NP;
  R Vn[NV][NP], r[NV][NP];
  const R* V0e[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    V0e[v] = V0 + v * KN + eo;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      Vn[v][a] = Vin[v * KN + eo + a];
      r[v][a] = rbuf[v * KN + eo + a];
    }
  }
  // an element that is exactly dry and at rest in the stage's states with a
  // zero residual (no water reaches it) stays so: the stage below would give
  // y = 0 too
  bool still = true;
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      still = still && Vn[v][a] == R(0) && r[v][a] == R(0);
      if (c0 != R(0)) still = still && V0e[v][a] == R(0);
    }
  if (still) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int a = 0; a < NP; ++a) out[v * KN + eo + a] = R(0);
    return;
  }
  const double dt = sc[ins].dt;
  const R Jinv = geo[6 * K + e];
  if constexpr (sizeof(R) == 4) {
    // FP32 context: FP32 unless a nodal depth of the stage's states is below h_dry
    R hmin = Vn[0][0];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      hmin = fmin(hmin, Vn[0][a]);
      if (c0 != R(0)) hmin = fmin(hmin, V0e[0][a]);
    }
    if (hmin >= ph.h_dry) {
      conservative_stage<DIM, P, R, float>(Vn, r, V0e, c0, c1, dt, ops, ph.h_floor, Jinv, out, KN, eo);
      return;
    }
  }
  conservative_stage<DIM, P, R, double>(Vn, r, V0e, c0, c1, dt, ops, ph.h_floor, Jinv, out, KN, eo);
}

// ------------------------------------------------------------------ backward Euler (Newton-Krylov)

// <l_a, U_v(V)> per element in physical scaling, with U = (h, h u_1, ..,
// h u_d) (Eq. Uterm) at the volume quadrature points.  mode 0: out = that;
// mode 1: out += (that - Uold) * inv_dt, which adds the backward-Euler time
// term of Eq. WeakForm7 to the spatial residual already in out.
template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256) be_time_kernel(int K, const R* __restrict__ V, const R* __restrict__ Uold,
                                                      R* __restrict__ out, const R* __restrict__ geo,
                                                      const VolOps<DIM, P, R> ops, R inv_dt, int mode) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NQ = S::NQ, NV = S::NV;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  const size_t KN = (size_t)K * NP, eo = (size_t)e * NP;
  R Vn[NV][NP], acc[NV][NP];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      Vn[v][a] = V[v * KN + eo + a];
      acc[v][a] = R(0);
    }
  const R J = geo[4 * K + e];
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    R Vq[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      R t = R(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) t += ops.Vq[q * NP + a] * Vn[v][a];
      Vq[v] = t;
    }
    const R w = ops.wq[q] * J;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const R wl = w * ops.Vq[q * NP + a];
      acc[0][a] += wl * Vq[0];
#pragma unroll
      for (int j = 1; j < NV; ++j) acc[j][a] += wl * (Vq[0] * Vq[j]);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const size_t i = v * KN + eo + a;
      out[i] = mode == 0 ? acc[v][a] : out[i] + (acc[v][a] - Uold[i]) * inv_dt;
    }
}

// z = scale * M(V)^{-1} x per element, M(V) the primitive-variable mass
// matrix (Appendix A, dU/dV): the preconditioner of the Newton-Krylov solve.
template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256) mass_precond_kernel(int K, const R* __restrict__ V, const R* __restrict__ x,
                                                           R* __restrict__ z, const R* __restrict__ geo,
                                                           const VolOps<DIM, P, R> ops, R h_floor, R scale) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NV = S::NV;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K) return;
  const size_t KN = (size_t)K * NP, eo = (size_t)e * NP;
  R Vn[NV][NP], xr[NV][NP], dV[NV][NP];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      Vn[v][a] = V[v * KN + eo + a];
      xr[v][a] = x[v * KN + eo + a];
    }
  mass_solve_element<DIM, P, R>(Vn, xr, ops, h_floor, geo[6 * K + e], dV);
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int a = 0; a < NP; ++a) z[v * KN + eo + a] = -scale * dV[v][a];
}

// ------------------------------------------------------------------ staged volume kernel
// Bulk asynchronous copies (global -> shared, completion counted in bytes on
// an mbarrier) and a bounded mbarrier wait.

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase of the given parity to complete; false after
// limit_ns nanoseconds without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_test(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

constexpr uint64_t kStageWaitNs = 1000000000ull;  // 1 s: copies of a few KB take microseconds

// Bytes of one staging slot: a tile's contiguous range of one field plus the
// up-to-15-byte lead of its 16-byte aligned window, rounded up to 16.
template <typename R>
__host__ __device__ constexpr uint32_t staged_slot_bytes(int T, int NP) {
  return (uint32_t)(((size_t)T * NP * sizeof(R) + 16 + 15) & ~size_t(15));
}
// Staged arrays per buffer: V (NV fields), E (NE), bed (FP32 only), V0 (NV).
template <int DIM, int P>
__host__ __device__ constexpr int staged_arrays() {
  return 2 * Sh<DIM, P>::NV + Sh<DIM, P>::NE + 1;
}
template <int DIM, int P, typename R>
__host__ __device__ constexpr size_t staged_smem_bytes(int T) {
  return 2 * (size_t)staged_arrays<DIM, P>() * staged_slot_bytes<R>(T, Sh<DIM, P>::NP) + 2 * sizeof(uint64_t);
}

// Staged form of volume_kernel for batch groups (same arithmetic, bitwise
// equal results).  A persistent grid walks tiles of T = blockDim.x
// consecutive elements.  While a tile is computed, the element-major nodal
// arrays of the CTA's next tile -- V, E, the bed (FP32) and (stages with c0 != 0)
// V0, each a contiguous range per field -- arrive in the other of two
// shared-memory buffers by bulk asynchronous copies, one thread issuing them
// and an mbarrier per buffer counting the bytes.  Each copy covers the
// 16-byte aligned window around the range (workspace arrays are 256-byte
// aligned and padded, so the window stays inside the allocation); readers
// skip the lead.  A wait that exceeds one second latches DG_ERR_TIMEOUT in
// the instance's status, waits (bounded) for the copies in flight and ends
// the CTA.
template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256) volume_staged_kernel(int K, int F, const R* __restrict__ Vin, const R* V0,
                                                            R* out, const R* __restrict__ E,
                                                            const R* __restrict__ bed, const R* __restrict__ src, const R* __restrict__ geo,
                                                            const int32_t* __restrict__ fid,
                                                            const R* __restrict__ wflux, const VolOps<DIM, P, R> ops,
                                                            const Phys<R>* __restrict__ ptab,
                                                            const int32_t* __restrict__ inst, R c0, R c1,
                                                            DevScalars* sc) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NV = S::NV, NE = S::NE;
  constexpr int NARR = staged_arrays<DIM, P>();
  extern __shared__ __align__(128) unsigned char dsm[];
  const int T = blockDim.x;
  const uint32_t slot = staged_slot_bytes<R>(T, NP);
  uint64_t* bar = reinterpret_cast<uint64_t*>(dsm + 2 * (size_t)NARR * slot);
  const size_t KN = (size_t)K * NP;
  const int ntiles = (K + T - 1) / T;
  const bool need_v0 = c0 != R(0);
  // start of field j's range for a tile starting at element e0 (nullptr: not staged)
  auto src_of = [&](int j, int e0) -> const char* {
    const R* base;
    if (j < NV) base = Vin + j * KN;
    else if (j < NV + NE) base = E + (j - NV) * KN;
    else if (j == NV + NE) base = sizeof(R) == 4 ? bed : nullptr;  // FP64 reads the source coefficients instead
    else base = need_v0 ? V0 + (j - NV - NE - 1) * KN : nullptr;
    return base ? reinterpret_cast<const char*>(base + (size_t)e0 * NP) : nullptr;
  };
  auto issue = [&](int tile, int buf) {
    const int e0 = tile * T;
    const size_t len = (size_t)min(T, K - e0) * NP * sizeof(R);
    uint32_t total = 0;
#pragma unroll 1
    for (int j = 0; j < NARR; ++j) {
      const char* p = src_of(j, e0);
      if (!p) continue;
      const uintptr_t lead = (uintptr_t)p & 15u;
      total += (uint32_t)((lead + len + 15) & ~size_t(15));
    }
    mbar_expect_tx(&bar[buf], total);
#pragma unroll 1
    for (int j = 0; j < NARR; ++j) {
      const char* p = src_of(j, e0);
      if (!p) continue;
      const uintptr_t lead = (uintptr_t)p & 15u;
      bulk_copy_g2s(dsm + ((size_t)buf * NARR + j) * slot, p - lead, (uint32_t)((lead + len + 15) & ~size_t(15)),
                    &bar[buf]);
    }
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  // bit b of parity: phase parity to wait for on buffer b; bit b of pending:
  // copies issued into buffer b and not yet waited for
  int tile = blockIdx.x, buf = 0;
  uint32_t parity = 0u, pending = 0u;
  if (tile < ntiles) {
    if (threadIdx.x == 0) issue(tile, 0);
    pending = 1u;
  }
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    if (next < ntiles) {
      if (threadIdx.x == 0) issue(next, buf ^ 1);
      pending |= 1u << (buf ^ 1);
    }
    const bool ok = mbar_wait_bounded(&bar[buf], (parity >> buf) & 1u, kStageWaitNs);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        atomicExch(&sc[inst[tile * T]].status, (int)DG_ERR_TIMEOUT);
        for (int b2 = 0; b2 < 2; ++b2)
          if ((pending >> b2) & 1u) mbar_wait_bounded(&bar[b2], (parity >> b2) & 1u, kStageWaitNs);
      }
      __syncthreads();
      return;
    }
    pending &= ~(1u << buf);
    parity ^= 1u << buf;
    const int e0 = tile * T;
    const int e = e0 + threadIdx.x;
    if (e < K) {
      const int ins = inst[e];
      const Phys<R> ph = ptab[ins];
      const R* sV[NARR];
#pragma unroll
      for (int j = 0; j < NARR; ++j) {
        const char* p = src_of(j, e0);
        const uintptr_t lead = p ? ((uintptr_t)p & 15u) : 0;
        sV[j] = reinterpret_cast<const R*>(dsm + ((size_t)buf * NARR + j) * slot + lead) +
                (size_t)threadIdx.x * NP;
      }
      R Vn[NV][NP], En[NE][NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
#pragma unroll
        for (int v = 0; v < NV; ++v) Vn[v][a] = sV[v][a];
#pragma unroll
        for (int c = 0; c < NE; ++c) En[c][a] = sV[NV + c][a];
      }
      const R* V0e[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) V0e[v] = sV[NV + NE + 1 + v];
      volume_element<DIM, P, R>(e, K, F, Vn, En, (sizeof(R) == 4 && bed) ? sV[NV + NE] : nullptr, src, V0e, out, geo, fid, wflux, ops, ph,
                                ins, 1, c0, c1, sc, nullptr);
    }
    __syncthreads();
    buf ^= 1;
  }
}

// ------------------------------------------------------------------ reductions (FP64)

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Per-element stable step (see dg_swe_step), block minimum to partial[block].
// A non-finite state sets partial to -1 (flag).
template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256) dt_partial_kernel(int K, const R* __restrict__ V, const R* __restrict__ geo,
                                                         double gc, double h_floor, double cfl, double nu,
                                                         double* __restrict__ partial) {
  constexpr int NP = Sh<DIM, P>::NP;
  __shared__ double red[8];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double dte = 1e300;
  if (e < K) {
    const size_t KN = (size_t)K * NP;
    // wave speeds in the state's precision, step and reduction in FP64
    R lam = R(0);
    bool bad = false;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const R h = V[(size_t)e * NP + a];
      R sp2 = R(0);
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const R u = V[(1 + j) * KN + (size_t)e * NP + a];
        sp2 += u * u;
      }
      const R l = sqrt(sp2) + sqrt((R)gc * fmax(h, (R)h_floor));
      if (!isfinite(l) || !isfinite(h)) bad = true;
      lam = fmax(lam, l);
    }
    // per-element bound in the state's precision; min and time sum in FP64
    const R dx = geo[5 * K + e];
    const R qq = R(2 * P + 1);
    dte = (double)((R)cfl * dx / (qq * lam + qq * qq * R(2) * (R)nu / dx));
    if (bad) dte = -1.0;
  }
  double v = warp_min(dte);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 1e300;
    v = warp_min(v);
    if (lane == 0) partial[blockIdx.x] = v;
  }
}

// Final step size: fixed dt (> 0) or min of the partials; advances t and the
// step counter.  A negative partial latches DG_ERR_NONFINITE (4).
static __global__ void dt_finalize_kernel(int nblocks, const double* __restrict__ partial, double fixed_dt,
                                   DevScalars* __restrict__ sc) {
  __shared__ double red[32];
  double v = 1e300;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v = fmin(v, partial[i]);
  v = warp_min(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 1e300;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmin(m, red[i]);
    if (m < 0.0) {
      sc->status = 4;
      m = 0.0;
    }
    const double dt = fixed_dt > 0.0 ? fixed_dt : m;
    sc->dt = dt;
    sc->t += dt;
    sc->steps += 1;
    sc->dt_min = fmin(sc->dt_min, dt);
    sc->dt_max = fmax(sc->dt_max, dt);
  }
}

// Mass integral: sum_e J_e sum_a wint_a h_a (FP64 partial sums per block).
template <int NP, typename R>
__global__ void __launch_bounds__(256) mass_partial_kernel(int K, const R* __restrict__ V, const R* __restrict__ geo,
                                                           const double* __restrict__ wint,
                                                           double* __restrict__ partial) {
  __shared__ double red[8];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (e < K) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < NP; ++a) s += wint[a] * (double)V[(size_t)e * NP + a];
    m = (double)geo[4 * K + e] * s;
  }
  double v = warp_sum(m);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) partial[blockIdx.x] = v;
  }
}

// Compensated (Kahan) sum of the block partials; which = 0 -> mass, 1 -> mass0 too.
static __global__ void mass_finalize_kernel(int nblocks, const double* __restrict__ partial, int set_ref,
                                     DevScalars* __restrict__ sc) {
  if (threadIdx.x != 0) return;
  double s = 0.0, c = 0.0;
  for (int i = 0; i < nblocks; ++i) {
    double y = partial[i] - c;
    double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  sc->mass = s;
  if (set_ref) sc->mass0 = s;
}


// ------------------------------------------------------------------ per-instance reductions (batches)

// Stable step of a batch: each block takes one contiguous 256-element range
// of one instance (blk_e[b] .. blk_e[b+1]) and writes its FP64 minimum to
// partial[b]; a negative partial flags a non-finite state.
template <int DIM, int P, typename R>
__global__ void __launch_bounds__(256) dt_block_kernel(int K, const int64_t* __restrict__ blk_e,
                                                       const int32_t* __restrict__ blk_gid,
                                                       const R* __restrict__ V, const R* __restrict__ geo,
                                                       const double* __restrict__ iparm,
                                                       double* __restrict__ partial) {
  constexpr int NP = Sh<DIM, P>::NP;
  __shared__ double red[8];
  const int b = blockIdx.x;
  const int g = blk_gid[b];
  const int64_t e = blk_e[b] + threadIdx.x;
  const double gc = iparm[4 * g + 0], h_floor = iparm[4 * g + 1], cfl = iparm[4 * g + 2], nu = iparm[4 * g + 3];
  double dte = 1e300;
  if (e < blk_e[b + 1]) {
    const size_t KN = (size_t)K * NP;
    R lam = R(0);
    bool bad = false;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const R h = V[(size_t)e * NP + a];
      R sp2 = R(0);
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        const R u = V[(1 + j) * KN + (size_t)e * NP + a];
        sp2 += u * u;
      }
      const R l = sqrt(sp2) + sqrt((R)gc * fmax(h, (R)h_floor));
      if (!isfinite(l) || !isfinite(h)) bad = true;
      lam = fmax(lam, l);
    }
    // per-element bound in the state's precision; min and time sum in FP64
    const R dx = geo[5 * K + e];
    const R qq = R(2 * P + 1);
    dte = (double)((R)cfl * dx / (qq * lam + qq * qq * R(2) * (R)nu / dx));
    if (bad) dte = -1.0;
  }
  double v = warp_min(dte);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 1e300;
    v = warp_min(v);
    if (lane == 0) partial[b] = v;
  }
}

// One warp per instance of a group: minimum of its block partials (exact,
// so independent of order), then dt, t, step count and dt_min/max.
static __global__ void dt_members_kernel(int n_members, const int32_t* __restrict__ mblk,
                                         const int32_t* __restrict__ gid, const double* __restrict__ partial,
                                         DevScalars* __restrict__ sc) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n_members) return;
  double m = 1e300;
  for (int b = mblk[i] + lane; b < mblk[i + 1]; b += 32) m = fmin(m, partial[b]);
  m = warp_min(m);
  if (lane == 0) {
    DevScalars& s = sc[gid[i]];
    if (m < 0.0) {
      s.status = 4;
      m = 0.0;
    }
    s.dt = m;
    s.t += m;
    s.steps += 1;
    s.dt_min = fmin(s.dt_min, m);
    s.dt_max = fmax(s.dt_max, m);
  }
}

static __global__ void reset_scalars_array_kernel(int n, DevScalars* sc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  sc[i].dt = 0.0;
  sc[i].t = 0.0;
  sc[i].dt_min = 1e300;
  sc[i].dt_max = 0.0;
  sc[i].steps = 0;
  sc[i].status = 0;
}

// ------------------------------------------------------------------ host: operator tables

template <int DIM, int P, typename R>
void fill_ops(const RefOps& o, EstepOps<DIM, P, R>& eo, FaceOps<DIM, P, R>& fo, VolOps<DIM, P, R>& vo) {
  using S = Sh<DIM, P>;
  const int NP = S::NP, NQ = S::NQ;
  for (int i = 0; i < NP * NP; ++i) {
    eo.Dr[i] = (R)o.Dr[i];
    eo.Ds[i] = (R)o.Ds[i];
    vo.Minv[i] = (R)o.Minv[i];
  }
  for (int i = 0; i < NP * S::NF * S::NFP; ++i) eo.LIFT[i] = (R)o.LIFT[i];
  for (int i = 0; i < S::NF * S::NFP; ++i) {
    eo.fmask[i] = (int8_t)o.fmask[i];
    fo.fmask[i] = (int8_t)o.fmask[i];
  }
  {
    double area = 0.0;
    for (int a = 0; a < NP; ++a) area += o.wint[a];
    for (int a = 0; a < NP; ++a) vo.wavg[a] = (R)(o.wint[a] / area);
  }
  for (int m = 0; m < S::NFQ; ++m) {
    fo.wf[m] = (R)o.wf[m];
    for (int k = 0; k < S::NFP; ++k) {
      fo.Lf[m * S::NFP + k] = (R)o.Lf[m * S::NFP + k];
      vo.LfT[k * S::NFQ + m] = (R)o.Lf[m * S::NFP + k];
    }
  }
  for (int q = 0; q < NQ; ++q) {
    vo.wq[q] = (R)o.wq[q];
    for (int a = 0; a < NP; ++a) {
      vo.Vq[q * NP + a] = (R)o.Vq[q * NP + a];
      vo.Drq[q * NP + a] = (R)o.Drq[q * NP + a];
      vo.Dsq[q * NP + a] = (R)o.Dsq[q * NP + a];
      vo.Wr[q * NP + a] = (R)(o.wq[q] * o.Drq[q * NP + a]);
      vo.Ws[q * NP + a] = (R)(o.wq[q] * o.Dsq[q * NP + a]);
      vo.Wm[q * NP + a] = (R)(o.wq[q] * o.Vq[q * NP + a]);
    }
  }
}

// Maximum d sigma_B / dE over E (attained at E = 0) for the step bound.
// Largest d sigma_N / dE of the viscous part over E, divided by 4: eta, or
// eta rate_floor^(n-1) for the Herschel-Bulkley power law with 0 < n < 1
// (its slope 4 eta n |E|^(n-1) above the floor is smaller).
inline double max_viscous_eta(const dg_swe_params& p) {
  const double n = p.flow_index;
  if (n == 0.0 || n == 1.0) return p.eta;
  return p.eta * std::pow(p.rate_floor, n - 1.0);
}

inline double max_bingham_slope(int reg, double sigma0, double gamma, double pap_m) {
  if (!(sigma0 > 0.0)) return 0.0;
  switch (reg) {
    case 1: case 2: case 5: return 2.0 * gamma;
    case 3: return 2.0 * sigma0 * gamma;
    case 4: return 2.0 * sigma0 * pap_m;
    default: return 0.0;
  }
}

template <typename Rin, typename Rout>
__global__ void convert_kernel(size_t n, const Rin* __restrict__ in, Rout* __restrict__ out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (Rout)in[i];
}

static __global__ void reset_scalars_kernel(DevScalars* sc) {
  sc->dt = 0.0;
  sc->t = 0.0;
  sc->dt_min = 1e300;
  sc->dt_max = 0.0;
  sc->steps = 0;
  sc->status = 0;
}

}  // namespace dgswe

// Persistent form of one SSP-RK3 step of a batch group (dg_batch_set_persistent).
//
// The graph form launches, per group and step, the step-size reduction and
// then, for each of the three stages, the E-step, face-flux and volume
// kernels: 11 launches whose tails and launch gaps dominate small instances.
// Here one launch does all of it.  Its thread blocks claim work items from a
// global counter in a fixed order, phase-major:
//   phase 0          step-bound tiles (128 elements: FP64 minimum of the
//                    per-element bound, as dt_block_kernel),
//   phase 1          one item per instance: minimum over its tiles, then dt,
//                    t and the step count (as dt_members_kernel),
//   phases 2 + 3 s   E-step tiles of stage s (128 elements),
//   phases 3 + 3 s   face-flux tiles of stage s (128 face points),
//   phases 4 + 3 s   volume tiles of stage s (128 elements),
// with per-instance completion counters.  An item waits only for the phase
// before it of the same instance (the volume of stage 0 also for the
// instance's step size), so different instances' phases overlap.  Items are
// claimed in order, so every item waited on was claimed earlier by a running
// block that itself only waits on earlier items: the wait always ends.  Each
// wait is still bounded (one second, %globaltimer); a block that gives up
// latches DG_ERR_TIMEOUT for its instance and moves the counter past the last
// item, so that no block claims further work.
//
// The per-element and per-face-point arithmetic is the graph form's own
// (estep_element, face_item, volume_element); compiled into this kernel, some
// multiply-adds may be fused differently, so results agree to rounding.  Data that another block writes during the launch (stage states, E,
// face fluxes, tile bounds, dt) is read through L2 (ld.global.cg): the
// producer's block barrier, fence and counter increment, and the consumer's
// counter read, fence and block barrier, order the accesses.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dg_kernels.cuh"

namespace dgswe {
namespace persist {

constexpr int kThreads = 128;
constexpr int kPhases = 11;
constexpr uint64_t kWaitNs = 1000000000ull;

// Device view of one group's plan (pointers into the batch workspace).
struct Plan {
  int n_members;
  int pstart[kPhases + 1];      // item range of each phase
  const int32_t* etile_pre;     // [n_members + 1] prefix of element tiles
  const int32_t* ftile_pre;     // [n_members + 1] prefix of face-point tiles
  const int64_t* ebeg;          // [n_members + 1] first element of each member (group-local) and the end
  const int64_t* fbeg;          // [n_members + 1] first face of each member and the end
  const int32_t* gid;           // [n_members] global instance id
  double* tile_dt;              // [element tiles] step bound of each tile
  int* done;                    // [n_members][kPhases] completed items, zeroed before each launch
  int* next;                    // next item to claim, zeroed before each launch
};

// Arrays of one group (pointers into the batch workspace).
template <typename R>
struct Arrays {
  R* V[3];
  R* E;
  R* wflux;
  const R *bed, *src, *geo, *fn, *fsj, *fnrm, *fsjf;
  const int32_t *nbr, *fid, *fe1, *fe2, *inst;
  const int8_t *nbrf, *ff1, *ff2;
  const Phys<R>* ptab;
  const BCEntry<R>* bct;
  const double* iparm;
  DevScalars* sc;
  int K, F;
};

// Phase on which phase ph depends (-1: none) and whether its items are face tiles.
__host__ __device__ constexpr int dep_of(int ph) { return ph == 0 || ph == 2 ? -1 : ph - 1; }
__host__ __device__ constexpr bool face_phase(int ph) { return ph >= 2 && (ph - 2) % 3 == 1; }

__device__ __forceinline__ int upper_member(const int32_t* pre, int n, int j) {
  int lo = 0, hi = n;  // largest m with pre[m] <= j
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= j) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Items of phase ph that instance m completes.
__device__ __forceinline__ int items_of(const Plan& pl, int ph, int m) {
  if (ph == 1) return 1;
  const int32_t* pre = face_phase(ph) ? pl.ftile_pre : pl.etile_pre;
  return pre[m + 1] - pre[m];
}

// Bounded wait (thread 0) until counter >= need.
__device__ __forceinline__ bool wait_count(const int* counter, int need) {
  const volatile int* c = counter;
  if (*c >= need) return true;
  const uint64_t t0 = global_ns();
  while (*c < need)
    if (global_ns() - t0 > kWaitNs) return false;
  return true;
}

template <int DIM, int P, typename R>
__global__ void __launch_bounds__(kThreads) step_kernel(const Plan pl, const Arrays<R> A,
                                                        const EstepOps<DIM, P, R> eo, const FaceOps<DIM, P, R> fo,
                                                        const VolOps<DIM, P, R> vo) {
  using S = Sh<DIM, P>;
  constexpr int NP = S::NP, NV = S::NV, NE = S::NE, NFQ = S::NFQ;
  __shared__ __align__(16) R tab[QTab<DIM, P, R>::SIZE];
  __shared__ double red[kThreads / 32];
  __shared__ int s_item, s_ok;
  qtab_fill<DIM, P, R>(tab, vo);
  const int tid = threadIdx.x;
  const int K = A.K, F = A.F;
  const size_t KN = (size_t)K * NP;
  const int total = pl.pstart[kPhases];
  __syncthreads();
  for (;;) {
    if (tid == 0) s_item = atomicAdd(pl.next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    int ph = 0;
    while (item >= pl.pstart[ph + 1]) ++ph;
    const int j = item - pl.pstart[ph];
    int m = j, t = 0;
    if (ph != 1) {
      const int32_t* pre = face_phase(ph) ? pl.ftile_pre : pl.etile_pre;
      m = upper_member(pre, pl.n_members + 1, j);
      t = j - pre[m];
    }
    // dependencies: the previous phase of this instance (and, for the first
    // volume phase, the instance's step size)
    if (tid == 0) {
      bool ok = true;
      const int d = dep_of(ph);
      if (d >= 0) ok = wait_count(&pl.done[m * kPhases + d], items_of(pl, d, m));
      if (ok && ph == 4) ok = wait_count(&pl.done[m * kPhases + 1], 1);
      if (!ok) {
        atomicExch(&A.sc[pl.gid[m]].status, (int)DG_ERR_TIMEOUT);
        atomicAdd(pl.next, total);  // no block claims further items
      }
      __threadfence();
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) break;
    const int64_t e_lo = pl.ebeg[m], e_hi = pl.ebeg[m + 1];
    if (ph == 0) {
      // step bound of one 128-element tile (dt_block_kernel's per-element bound)
      const int64_t e = e_lo + (int64_t)t * kThreads + tid;
      double dte = 1e300;
      if (e < e_hi) {
        const int g = pl.gid[m];
        const double gc = A.iparm[4 * g + 0], h_floor = A.iparm[4 * g + 1], cfl = A.iparm[4 * g + 2],
                     nu = A.iparm[4 * g + 3];
        R lam = R(0);
        bool bad = false;
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          const R h = DG_LDC(true, A.V[0], (size_t)e * NP + a);
          R sp2 = R(0);
#pragma unroll
          for (int jj = 0; jj < DIM; ++jj) {
            const R u = DG_LDC(true, A.V[0], (1 + jj) * KN + (size_t)e * NP + a);
            sp2 += u * u;
          }
          const R l = sqrt(sp2) + sqrt((R)gc * fmax(h, (R)h_floor));
          if (!isfinite(l) || !isfinite(h)) bad = true;
          lam = fmax(lam, l);
        }
        const R dx = A.geo[5 * K + e];
        const R qq = R(2 * P + 1);
        dte = (double)((R)cfl * dx / (qq * lam + qq * qq * R(2) * (R)nu / dx));
        if (bad) dte = -1.0;
      }
      double v = warp_min(dte);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double mn = red[0];
        for (int w = 1; w < kThreads / 32; ++w) mn = fmin(mn, red[w]);
        pl.tile_dt[pl.etile_pre[m] + t] = mn;
      }
    } else if (ph == 1) {
      // the instance's step (dt_members_kernel)
      double v = 1e300;
      for (int b = pl.etile_pre[m] + tid; b < pl.etile_pre[m + 1]; b += kThreads) v = fmin(v, __ldcg(pl.tile_dt + b));
      v = warp_min(v);
      if ((tid & 31) == 0) red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double mn = red[0];
        for (int w = 1; w < kThreads / 32; ++w) mn = fmin(mn, red[w]);
        DevScalars& s = A.sc[pl.gid[m]];
        if (mn < 0.0) {
          s.status = 4;
          mn = 0.0;
        }
        s.dt = mn;
        s.t += mn;
        s.steps += 1;
        s.dt_min = fmin(s.dt_min, mn);
        s.dt_max = fmax(s.dt_max, mn);
      }
    } else {
      const int st = (ph - 2) / 3, kind = (ph - 2) % 3;
      const int vin = st, vout = st == 2 ? 0 : st + 1;
      if (kind == 0) {
        const int64_t e = e_lo + (int64_t)t * kThreads + tid;
        if (e < e_hi)
          estep_element<DIM, P, R, true>((int)e, K, A.V[vin], A.E, A.geo, A.nbr, A.nbrf, A.fn, A.fsj, eo, A.bct);
      } else if (kind == 1) {
        const int64_t fp = (int64_t)t * kThreads + tid;
        if (fp < (pl.fbeg[m + 1] - pl.fbeg[m]) * NFQ)
          face_item<DIM, P, R, true, false, true>(pl.fbeg[m] * NFQ + fp, K, F, A.V[vin], A.E, A.fe1, A.ff1, A.fe2,
                                                  A.ff2, A.fnrm, A.fsjf, A.wflux, fo, Phys<R>{}, A.ptab, A.inst,
                                                  A.bct);
      } else {
        const int64_t e = e_lo + (int64_t)t * kThreads + tid;
        if (e < e_hi) {
          const R c0 = st == 0 ? R(0.0) : st == 1 ? R(0.75) : R(1.0 / 3.0);
          const R c1 = st == 0 ? R(1.0) : st == 1 ? R(0.25) : R(2.0 / 3.0);
          const int ins = A.inst[e];
          const Phys<R> phy = A.ptab[ins];
          const size_t eo2 = (size_t)e * NP;
          R Vn[NV][NP], En[NE][NP];
#pragma unroll
          for (int a = 0; a < NP; ++a) {
#pragma unroll
            for (int v = 0; v < NV; ++v) Vn[v][a] = DG_LDC(true, A.V[vin], v * KN + eo2 + a);
#pragma unroll
            for (int c = 0; c < NE; ++c) En[c][a] = DG_LDC(true, A.E, c * KN + eo2 + a);
          }
          const R* V0e[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) V0e[v] = A.V[0] + v * KN + eo2;
          volume_element<DIM, P, R, true>((int)e, K, F, Vn, En, A.bed ? A.bed + eo2 : nullptr, A.src, V0e, A.V[vout],
                                          A.geo, A.fid, A.wflux, vo, phy, ins, 1, c0, c1, A.sc, tab);
        }
      }
    }
    __syncthreads();  // the item's writes are done
    if (tid == 0) {
      __threadfence();
      atomicAdd(&pl.done[m * kPhases + ph], 1);
    }
  }
}

}  // namespace persist
}  // namespace dgswe

// Backward Euler with a Jacobian-free Newton-Krylov solve on a dg_swe
// context (1D and 2D).  See include/dg_newton.h for the method and contract.
//
// Residual evaluations reuse the context's stage kernels (E-step, face flux,
// volume pass returning the raw spatial residual) plus the backward-Euler
// time term; the preconditioner is the per-element primitive mass solve.
// The Krylov vectors, Gram-Schmidt reductions and updates are FP64 kernels
// here; the small Hessenberg least-squares problem is solved on the host.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/dg_newton.h"
#include "dg_ctx.h"
#include "dg_kernels.cuh"

using namespace dgswe;

namespace {

constexpr int kVecBlock = 256;
constexpr int kMaxKrylov = 64;

inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------------ FP64 vector kernels

// partial[i * G + b] = block b's share of <x, Y_i>, Y_i = Y + i * n.
__global__ void __launch_bounds__(kVecBlock) dots_partial_kernel(size_t n, const double* __restrict__ x,
                                                                 const double* __restrict__ Y,
                                                                 double* __restrict__ partial) {
  const int i = blockIdx.y;
  const double* y = Y + (size_t)i * n;
  double acc = 0.0;
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    acc += x[j] * y[j];
  __shared__ double sh[kVecBlock / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kVecBlock / 32 ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = v;
  }
}

// out[i] = sum over the G partials of dot i (fixed order).
__global__ void dots_finalize_kernel(int G, int k, const double* __restrict__ partial, double* __restrict__ out) {
  const int i = blockIdx.x;
  if (i >= k) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < G; b += 32) acc += partial[(size_t)i * G + b];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[i] = acc;
}

// w -= sum_i c[i] Y_i
__global__ void multi_axpy_kernel(size_t n, int k, const double* __restrict__ c, const double* __restrict__ Y,
                                  double* __restrict__ w) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    double s = w[j];
    for (int i = 0; i < k; ++i) s -= c[i] * Y[(size_t)i * n + j];
    w[j] = s;
  }
}

// out = sum_i c[i] Y_i
__global__ void combine_kernel(size_t n, int k, const double* __restrict__ c, const double* __restrict__ Y,
                               double* __restrict__ out) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += c[i] * Y[(size_t)i * n + j];
    out[j] = s;
  }
}

// y = a * x
__global__ void scale_kernel(size_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    y[j] = a * x[j];
}

// y = x / sqrt(*nrm2)
__global__ void normalize_kernel(size_t n, const double* __restrict__ nrm2, const double* __restrict__ x,
                                 double* __restrict__ y) {
  const double a = 1.0 / sqrt(*nrm2);
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    y[j] = a * x[j];
}

// eps = sqrt(1e-16) (1 + ||V||) / ||z|| ; Vp = V + eps z
__global__ void fd_point_kernel(size_t n, const double* __restrict__ V, const double* __restrict__ z,
                                const double* __restrict__ vn2, const double* __restrict__ zn2,
                                double* __restrict__ Vp, double* __restrict__ eps_out) {
  const double eps = 1e-8 * (1.0 + sqrt(*vn2)) / sqrt(*zn2);
  if (blockIdx.x == 0 && threadIdx.x == 0) *eps_out = eps;
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    Vp[j] = V[j] + eps * z[j];
}

// w = (R1 - R0) / eps
__global__ void fd_diff_kernel(size_t n, const double* __restrict__ R1, const double* __restrict__ R0,
                               const double* __restrict__ eps, double* __restrict__ w) {
  const double a = 1.0 / *eps;
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    w[j] = (R1[j] - R0[j]) * a;
}

// V += d
__global__ void add_kernel(size_t n, const double* __restrict__ d, double* __restrict__ V) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x)
    V[j] += d[j];
}

__global__ void advance_time_kernel(DevScalars* sc, double dt) {
  sc->t += dt;
  sc->dt = dt;
  sc->dt_min = fmin(sc->dt_min, dt);
  sc->dt_max = fmax(sc->dt_max, dt);
  sc->steps += 1;
}

}  // namespace

struct dg_newton {
  dg_swe_ctx* c = nullptr;
  dg_newton_params prm{};
  size_t n = 0;
  int m = 0;
  int G = 0;  // blocks of the vector kernels and dot partials
  size_t ws_need = 0;
  char* ws = nullptr;
  struct {
    size_t Uold, R0, R1, Vp, z, w, u, basis, partial, dots, scal;
  } off{};
  dg_newton_stats st{};
  std::string err;
  template <typename T>
  T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
};

namespace {

dg_status nfail(dg_newton* k, dg_status s, const std::string& m) {
  if (k) {
    k->err = m;
    if (!k->st.status) k->st.status = s;
  }
  return s;
}
#define NK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return nfail(k, DG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// scalar slots
enum { S_VN2 = 0, S_ZN2 = 1, S_EPS = 2, S_WN2 = 3, S_COUNT = 8 };

struct Ctx {
  dg_newton* k;
  dg_swe_ctx* c;
  cudaStream_t s;
  size_t n;
  unsigned grid;
  double* V;  // the context's state
  double* E;
  void residual(const double* Vx, double* out) {
    c->drv->estep(c, Vx, E, s);
    c->drv->face(c, Vx, E, s);
    c->drv->volume(c, Vx, nullptr, out, 2, 0.0, 0.0, s);
    c->drv->be_time(c, Vx, k->at<double>(k->off.Uold), out, 1.0 / k->prm.dt, 1, s);
  }
  // dots of x against k vectors Y_i into out[0..k) (device)
  void dots(const double* x, const double* Y, int cnt, double* out) {
    dots_partial_kernel<<<dim3((unsigned)k->G, (unsigned)cnt), kVecBlock, 0, s>>>(n, x, Y,
                                                                                 k->at<double>(k->off.partial));
    dots_finalize_kernel<<<cnt, 32, 0, s>>>(k->G, cnt, k->at<double>(k->off.partial), out);
  }
};

}  // namespace

extern "C" {

dg_status dg_newton_init(dg_swe_ctx* c, const dg_newton_params* p, dg_newton** out) {
  if (!c || !p || !out) return DG_ERR_ARG;
  *out = nullptr;
  if (c->prec != DG_PREC_FP64) return DG_ERR_UNSUPPORTED;
  if (!(p->dt > 0.0) || p->max_newton < 1 || p->krylov_dim < 1 || p->krylov_dim > kMaxKrylov ||
      !(p->krylov_rtol > 0.0 && p->krylov_rtol < 1.0) || p->rtol < 0.0 || p->atol < 0.0)
    return DG_ERR_ARG;
  auto* k = new dg_newton();
  k->c = c;
  k->prm = *p;
  k->m = p->krylov_dim;
  k->n = (size_t)(c->dim + 1) * (size_t)c->mesh.K * (size_t)c->ops.Np;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  k->G = std::max(1, std::min(2 * std::max(nsm, 1), (int)((k->n + kVecBlock - 1) / kVecBlock)));
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += a256(bytes);
    return r;
  };
  const size_t vb = k->n * sizeof(double);
  k->off.Uold = take(vb);
  k->off.R0 = take(vb);
  k->off.R1 = take(vb);
  k->off.Vp = take(vb);
  k->off.z = take(vb);
  k->off.w = take(vb);
  k->off.u = take(vb);
  k->off.basis = take((size_t)(k->m + 1) * vb);
  k->off.partial = take((size_t)(k->m + 1) * k->G * sizeof(double));
  k->off.dots = take(2 * (size_t)(k->m + 1) * sizeof(double));
  k->off.scal = take(S_COUNT * sizeof(double));
  k->ws_need = o;
  *out = k;
  return DG_OK;
}

size_t dg_newton_workspace_size(const dg_newton* k) { return k ? k->ws_need : 0; }

dg_status dg_newton_set_workspace(dg_newton* k, void* ptr, size_t bytes) {
  if (!k) return DG_ERR_ARG;
  if (!ptr || ((uintptr_t)ptr & 255) != 0 || bytes < k->ws_need)
    return nfail(k, DG_ERR_WORKSPACE, "workspace missing, misaligned or smaller than dg_newton_workspace_size");
  k->ws = static_cast<char*>(ptr);
  return DG_OK;
}

dg_status dg_newton_run(dg_newton* k, int64_t n_steps, dg_newton_stats* stats) {
  if (!k) return DG_ERR_ARG;
  dg_swe_ctx* c = k->c;
  if (!k->ws || !c->ws) return nfail(k, DG_ERR_WORKSPACE, "solver or context workspace not set");
  if (n_steps < 0) return nfail(k, DG_ERR_ARG, "n_steps must be >= 0");
  Ctx x{k, c, c->stream, k->n, (unsigned)k->G, c->at<double>(c->off.V0), c->at<double>(c->off.E)};
  const size_t n = k->n;
  const int m = k->m;
  double* Uold = k->at<double>(k->off.Uold);
  double* R0 = k->at<double>(k->off.R0);
  double* R1 = k->at<double>(k->off.R1);
  double* Vp = k->at<double>(k->off.Vp);
  double* z = k->at<double>(k->off.z);
  double* w = k->at<double>(k->off.w);
  double* u = k->at<double>(k->off.u);
  double* Bv = k->at<double>(k->off.basis);
  double* dots = k->at<double>(k->off.dots);
  double* sc = k->at<double>(k->off.scal);
  const unsigned G = x.grid;
  cudaStream_t s = x.s;
  std::vector<double> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), y(m), hbuf(2 * (m + 1) + 1);
  auto norm2 = [&](const double* v, double* slot, double& host) -> dg_status {
    x.dots(v, v, 1, slot);
    NK(cudaMemcpyAsync(&host, slot, sizeof(double), cudaMemcpyDeviceToHost, s));
    NK(cudaStreamSynchronize(s));
    return DG_OK;
  };
  for (int64_t step = 0; step < n_steps; ++step) {
    c->drv->be_time(c, x.V, nullptr, Uold, 0.0, 0, s);
    x.residual(x.V, R0);
    double r2 = 0.0;
    dg_status e = norm2(R0, sc + S_WN2, r2);
    if (e != DG_OK) return e;
    const double res0 = std::sqrt(r2);
    double res = res0;
    int its = 0;
    bool ok = res <= std::max(k->prm.rtol * res0, k->prm.atol);
    while (!ok && its < k->prm.max_newton) {
      if (!std::isfinite(res)) return nfail(k, DG_ERR_NONFINITE, "non-finite Newton residual");
      // ---- GMRES on J d = -R0, right preconditioned by dt M(V)^{-1}
      x.dots(x.V, x.V, 1, sc + S_VN2);
      const double beta = res;
      scale_kernel<<<G, kVecBlock, 0, s>>>(n, -1.0 / beta, R0, Bv);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int jn = 0;
      for (int j = 0; j < m; ++j) {
        double* vj = Bv + (size_t)j * n;
        c->drv->precond(c, x.V, vj, z, k->prm.dt, s);
        x.dots(z, z, 1, sc + S_ZN2);
        fd_point_kernel<<<G, kVecBlock, 0, s>>>(n, x.V, z, sc + S_VN2, sc + S_ZN2, Vp, sc + S_EPS);
        x.residual(Vp, R1);
        fd_diff_kernel<<<G, kVecBlock, 0, s>>>(n, R1, R0, sc + S_EPS, w);
        // classical Gram-Schmidt, twice
        x.dots(w, Bv, j + 1, dots);
        multi_axpy_kernel<<<G, kVecBlock, 0, s>>>(n, j + 1, dots, Bv, w);
        x.dots(w, Bv, j + 1, dots + (m + 1));
        multi_axpy_kernel<<<G, kVecBlock, 0, s>>>(n, j + 1, dots + (m + 1), Bv, w);
        x.dots(w, w, 1, sc + S_WN2);
        NK(cudaMemcpyAsync(hbuf.data(), dots, 2 * (m + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
        NK(cudaMemcpyAsync(hbuf.data() + 2 * (m + 1), sc + S_WN2, sizeof(double), cudaMemcpyDeviceToHost, s));
        NK(cudaStreamSynchronize(s));
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hbuf[i] + hbuf[(m + 1) + i];
        const double hn = std::sqrt(hbuf[2 * (m + 1)]);
        H[(size_t)(j + 1) * m + j] = hn;
        // Givens rotations
        for (int i = 0; i < j; ++i) {
          const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
        }
        const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
        const double r = std::hypot(a, b);
        cs[j] = r > 0.0 ? a / r : 1.0;
        sn[j] = r > 0.0 ? b / r : 0.0;
        H[(size_t)j * m + j] = r;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        jn = j + 1;
        k->st.krylov_its += 1;
        if (!std::isfinite(g[j + 1])) return nfail(k, DG_ERR_NONFINITE, "non-finite Krylov residual");
        if (std::fabs(g[j + 1]) <= k->prm.krylov_rtol * beta || hn == 0.0) break;
        if (j + 1 < m) normalize_kernel<<<G, kVecBlock, 0, s>>>(n, sc + S_WN2, w, Bv + (size_t)(j + 1) * n);
      }
      for (int i = jn - 1; i >= 0; --i) {
        double t = g[i];
        for (int l = i + 1; l < jn; ++l) t -= H[(size_t)i * m + l] * y[l];
        y[i] = t / H[(size_t)i * m + i];
      }
      NK(cudaMemcpyAsync(dots, y.data(), jn * sizeof(double), cudaMemcpyHostToDevice, s));
      combine_kernel<<<G, kVecBlock, 0, s>>>(n, jn, dots, Bv, u);
      c->drv->precond(c, x.V, u, z, k->prm.dt, s);
      add_kernel<<<G, kVecBlock, 0, s>>>(n, z, x.V);
      // ---- new residual
      x.residual(x.V, R0);
      e = norm2(R0, sc + S_WN2, r2);
      if (e != DG_OK) return e;
      res = std::sqrt(r2);
      ++its;
      ok = res <= std::max(k->prm.rtol * res0, k->prm.atol);
    }
    if (!std::isfinite(res)) return nfail(k, DG_ERR_NONFINITE, "non-finite Newton residual");
    advance_time_kernel<<<1, 1, 0, s>>>(c->at<DevScalars>(c->off.sc), k->prm.dt);
    NK(cudaGetLastError());
    k->st.steps += 1;
    k->st.newton_its += its;
    k->st.last_newton = its;
    k->st.last_res = res;
    if (!ok) {
      k->st.failed_steps += 1;
      if (!k->prm.on_fail_continue) {
        if (stats) *stats = k->st;
        return nfail(k, DG_ERR_NEWTON, "Newton did not converge in max_newton iterations");
      }
    }
  }
  DevScalars h{};
  NK(cudaMemcpyAsync(&h, c->at<DevScalars>(c->off.sc), sizeof(h), cudaMemcpyDeviceToHost, s));
  NK(cudaStreamSynchronize(s));
  k->st.t = h.t;
  if (stats) *stats = k->st;
  return DG_OK;
}

const char* dg_newton_last_error(const dg_newton* k) { return k ? k->err.c_str() : "null solver"; }

void dg_newton_destroy(dg_newton* k) { delete k; }

}  // extern "C"

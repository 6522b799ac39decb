// C ABI of the GB300 DG shallow-water / regularized-Bingham solver.
// See include/dg_swe.h for the contract of every entry point.
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dg_swe.h"
#include "dg_ctx.h"
#include "dg_kernels.cuh"
#include "dg_tc.cuh"

using namespace dgswe;

namespace {

constexpr int kBlock = 128;
constexpr int kRedBlock = 256;
constexpr int kWetDryBlock = 128;
constexpr int kGraphSteps = 16;

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

namespace dgswe {
void DriverDeleter::operator()(Driver* d) const { delete d; }
}  // namespace dgswe

namespace {

dg_status fail(dg_swe_ctx* c, dg_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

dg_status cuda_fail(dg_swe_ctx* c, cudaError_t e, const char* where) {
  return fail(c, DG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)



template <typename R>
Phys<R> make_phys(const dg_swe_params& p, int reg) {
  Phys<R> ph{};
  ph.gc = (R)(p.g * std::cos(p.alpha));
  ph.gs = (R)(p.g * std::sin(p.alpha));
  ph.rho_inv = (R)(1.0 / p.rho);
  ph.eta = (R)p.eta;
  ph.sigma0 = (R)p.sigma0;
  ph.gamma = (R)p.gamma;
  ph.beta = (R)p.beta;
  ph.half_inv_beta = (R)(0.5 / p.beta);
  ph.pap_m = (R)p.pap_m;
  ph.h_floor = (R)p.h_floor;
  ph.h_dry = (R)(kDryFactor * p.h_floor);
  ph.reg = reg;
  ph.pos = p.positivity ? 1 : 0;
  ph.hb = (p.flow_index != 0.0 && p.flow_index != 1.0) ? 1 : 0;
  ph.hb_n = (R)(ph.hb ? p.flow_index : 1.0);
  ph.hb_floor = (R)p.rate_floor;
  return ph;
}

template <typename R>
std::vector<BCEntry<R>> make_bc_table(const dg_swe_params& p) {
  std::vector<BCEntry<R>> t(p.n_bc);
  for (int b = 0; b < p.n_bc; ++b)
    for (int s = 0; s < 7; ++s) {
      t[b].mode[s] = p.bc[b].mode[s];
      t[b].val[s] = (R)p.bc[b].value[s];
    }
  return t;
}

template <int DIM, int P, typename R>
struct Impl final : Driver {
  using S = Sh<DIM, P>;
  // the tensor-core volume form exists for FP32 triangles of order >= 2
  static constexpr bool kTcForm = DIM == 2 && P >= 2 && sizeof(R) == 4;
  EstepOps<DIM, P, R> eo{};
  FaceOps<DIM, P, R> fo{};
  VolOps<DIM, P, R> vo{};
  Phys<R> ph{};
  bool tc = false;
  std::unique_ptr<tc::Launcher<(P >= 2 ? P : 2), false>> tcl;

  explicit Impl(const dg_swe_ctx& c) {
    fill_ops<DIM, P, R>(c.ops, eo, fo, vo);
    ph = make_phys<R>(c.prm, c.reg);
    if constexpr (kTcForm) {
      tc = c.prec == DG_PREC_FP32_TC;
      if (tc) tcl.reset(new tc::Launcher<P, false>());
    }
  }
  // the tensor-core volume pass (mode as volume_kernel); false if not used
  bool volume_tc(dg_swe_ctx* c, const void* Vin, const void* V0, void* out, const void* E, const void* wflux, int mode,
                 double c0, double c1, cudaStream_t s) {
    if constexpr (kTcForm) {
      if (!tc) return false;
      (*tcl)((int)c->mesh.K, (int)c->mesh.F, (const float*)Vin, (const float*)V0, (float*)out, (const float*)E,
             c->has_bed ? c->at<float>(c->off.bed) : nullptr, c->at<float>(c->off.geo), c->at<int32_t>(c->off.fid),
             (const float*)wflux, vo, c->at<float>(c->off.tcimg), ph, nullptr, nullptr, mode, (float)c0, (float)c1,
             c->at<DevScalars>(c->off.sc), s);
      return true;
    }
    return false;
  }

  void estep(dg_swe_ctx* c, const void* V, void* E, cudaStream_t s) override {
    const int K = (int)c->mesh.K;
    estep_kernel<DIM, P, R><<<(K + kBlock - 1) / kBlock, kBlock, 0, s>>>(
        K, (const R*)V, (R*)E, c->at<R>(c->off.geo), c->at<int32_t>(c->off.nbr), c->at<int8_t>(c->off.nbrf),
        c->at<R>(c->off.fn), c->at<R>(c->off.fsj), eo, c->at<BCEntry<R>>(c->off.bct));
  }
  void face(dg_swe_ctx* c, const void* V, const void* E, cudaStream_t s) override {
    const int K = (int)c->mesh.K, F = (int)c->mesh.F;
    const long long n = (long long)F * S::NFQ;
    face_kernel<DIM, P, R, false, false><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        K, F, (const R*)V, (const R*)E, c->at<int32_t>(c->off.fe1), c->at<int8_t>(c->off.ff1),
        c->at<int32_t>(c->off.fe2), c->at<int8_t>(c->off.ff2), c->at<R>(c->off.fnrm), c->at<R>(c->off.fsjf),
        c->at<R>(c->off.wflux), fo, ph, nullptr, nullptr, c->at<BCEntry<R>>(c->off.bct));
  }
  void volume(dg_swe_ctx* c, const void* Vin, const void* V0, void* out, int mode, double c0, double c1,
              cudaStream_t s) override {
    if (volume_tc(c, Vin, V0, out, c->ws + c->off.E, c->ws + c->off.wflux, mode, c0, c1, s)) return;
    const int K = (int)c->mesh.K, F = (int)c->mesh.F;
    volume_kernel<DIM, P, R, false><<<(K + kBlock - 1) / kBlock, kBlock, 0, s>>>(
        K, F, (const R*)Vin, (const R*)V0, (R*)out, c->at<R>(c->off.E),
        c->has_bed ? c->at<R>(c->off.bed) : nullptr, c->has_bed ? c->at<R>(c->off.src) : nullptr,
        c->at<R>(c->off.geo), c->at<int32_t>(c->off.fid),
        c->at<R>(c->off.wflux), vo, ph, nullptr, nullptr, mode, (R)c0, (R)c1, c->at<DevScalars>(c->off.sc));
  }
  void wetdry_stage(dg_swe_ctx* c, const void* Vin, const void* V0, const void* rbuf, void* out, double c0,
                    double c1, cudaStream_t s) override {
    const int K = (int)c->mesh.K;
    wetdry_stage_kernel<DIM, P, R, false><<<(K + kWetDryBlock - 1) / kWetDryBlock, kWetDryBlock, 0, s>>>(
        K, (const R*)Vin, (const R*)V0, (const R*)rbuf, (R*)out, c->at<R>(c->off.geo), vo, ph, nullptr, nullptr,
        (R)c0, (R)c1, c->at<DevScalars>(c->off.sc));
  }
  void face_into(dg_swe_ctx* c, const void* V, const void* E, void* wflux, cudaStream_t s) override {
    const int K = (int)c->mesh.K, F = (int)c->mesh.F;
    const long long n = (long long)F * S::NFQ;
    face_kernel<DIM, P, R, false, false><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        K, F, (const R*)V, (const R*)E, c->at<int32_t>(c->off.fe1), c->at<int8_t>(c->off.ff1),
        c->at<int32_t>(c->off.fe2), c->at<int8_t>(c->off.ff2), c->at<R>(c->off.fnrm), c->at<R>(c->off.fsjf),
        (R*)wflux, fo, ph, nullptr, nullptr, c->at<BCEntry<R>>(c->off.bct));
  }
  void be_time(dg_swe_ctx* c, const void* V, const void* Uold, void* out, double inv_dt, int mode,
               cudaStream_t s) override {
    const int K = (int)c->mesh.K;
    be_time_kernel<DIM, P, R><<<(K + kBlock - 1) / kBlock, kBlock, 0, s>>>(
        K, (const R*)V, (const R*)Uold, (R*)out, c->at<R>(c->off.geo), vo, (R)inv_dt, mode);
  }
  void precond(dg_swe_ctx* c, const void* V, const void* x, void* z, double scale, cudaStream_t s) override {
    const int K = (int)c->mesh.K;
    mass_precond_kernel<DIM, P, R><<<(K + kBlock - 1) / kBlock, kBlock, 0, s>>>(
        K, (const R*)V, (const R*)x, (R*)z, c->at<R>(c->off.geo), vo, ph.h_floor, (R)scale);
  }
  void residual_from(dg_swe_ctx* c, const void* V, const void* E, const void* wflux, void* out,
                     cudaStream_t s) override {
    if (volume_tc(c, V, nullptr, out, E, wflux, 0, 0.0, 0.0, s)) return;
    const int K = (int)c->mesh.K, F = (int)c->mesh.F;
    volume_kernel<DIM, P, R, false><<<(K + kBlock - 1) / kBlock, kBlock, 0, s>>>(
        K, F, (const R*)V, nullptr, (R*)out, (const R*)E, c->has_bed ? c->at<R>(c->off.bed) : nullptr,
        c->has_bed ? c->at<R>(c->off.src) : nullptr,
        c->at<R>(c->off.geo), c->at<int32_t>(c->off.fid), (const R*)wflux, vo, ph, nullptr, nullptr, 0, R(0), R(0),
        c->at<DevScalars>(c->off.sc));
  }
  void dt_partial(dg_swe_ctx* c, const void* V, cudaStream_t s) override {
    const int K = (int)c->mesh.K;
    const auto& p = c->prm;
    const double slope = max_bingham_slope(c->reg, p.sigma0, p.gamma, p.pap_m);
    const double nu = (4.0 * max_viscous_eta(p) + slope) / p.rho;
    dt_partial_kernel<DIM, P, R><<<c->nblk_dt, kRedBlock, 0, s>>>(
        K, (const R*)V, c->at<R>(c->off.geo), p.g * std::cos(p.alpha), p.h_floor, p.cfl, nu,
        c->at<double>(c->off.partial));
  }
  void mass_partial(dg_swe_ctx* c, const void* V, cudaStream_t s) override {
    const int K = (int)c->mesh.K;
    mass_partial_kernel<S::NP, R><<<c->nblk_mass, kRedBlock, 0, s>>>(
        K, (const R*)V, c->at<R>(c->off.geo), c->at<double>(c->off.wint), c->at<double>(c->off.partial));
  }
};

template <typename R>
DriverPtr make_driver(const dg_swe_ctx& c) {
#define DG_CASE(D, P) \
  if (c.dim == D && c.p == P) return DriverPtr(new Impl<D, P, R>(c));
  DG_CASE(1, 1) DG_CASE(1, 2) DG_CASE(1, 3) DG_CASE(2, 1) DG_CASE(2, 2) DG_CASE(2, 3)
#undef DG_CASE
  return nullptr;
}

cudaStream_t work_stream(dg_swe_ctx* c) { return c->stream; }

// One SSP-RK3 stage.  Wet/dry mode (positivity) splits the volume pass: the
// volume kernel writes r_V (mode 2) to rbuf, a buffer the stage does not
// otherwise read (its own output, or a free stage buffer when the output is
// V0), and wetdry_stage_kernel forms the conservative stage from it.
void enqueue_stage(dg_swe_ctx* c, const void* Vin, const void* V0, void* Vout, void* rbuf, double c0, double c1,
                   cudaStream_t s) {
  c->drv->estep(c, Vin, c->ws + c->off.E, s);
  c->drv->face(c, Vin, c->ws + c->off.E, s);
  if (c->prm.positivity) {
    c->drv->volume(c, Vin, nullptr, rbuf, 2, 0.0, 0.0, s);
    c->drv->wetdry_stage(c, Vin, V0, rbuf, Vout, c0, c1, s);
  } else {
    c->drv->volume(c, Vin, V0, Vout, 1, c0, c1, s);
  }
}

void enqueue_step(dg_swe_ctx* c, double fixed_dt, cudaStream_t s) {
  void* V0 = c->ws + c->off.V0;
  void* V1 = c->ws + c->off.V1;
  void* V2 = c->ws + c->off.V2;
  c->drv->dt_partial(c, V0, s);
  dt_finalize_kernel<<<1, 256, 0, s>>>(c->nblk_dt, c->at<double>(c->off.partial), fixed_dt,
                                       c->at<DevScalars>(c->off.sc));
  enqueue_stage(c, V0, V0, V1, V1, 0.0, 1.0, s);
  enqueue_stage(c, V1, V0, V2, V2, 0.75, 0.25, s);
  enqueue_stage(c, V2, V0, V0, V1, 1.0 / 3.0, 2.0 / 3.0, s);
}

void enqueue_mass(dg_swe_ctx* c, int set_ref, cudaStream_t s) {
  c->drv->mass_partial(c, c->ws + c->off.V0, s);
  mass_finalize_kernel<<<1, 32, 0, s>>>(c->nblk_mass, c->at<double>(c->off.partial), set_ref,
                                        c->at<DevScalars>(c->off.sc));
}

dg_status check_ws(dg_swe_ctx* c) {
  if (!c) return DG_ERR_ARG;
  if (!c->ws) return fail(c, DG_ERR_WORKSPACE, "no workspace set (dg_swe_set_workspace)");
  return DG_OK;
}

template <typename Rin, typename Rout>
void convert(const void* in, void* out, size_t n, cudaStream_t s) {
  if (n == 0) return;
  convert_kernel<Rin, Rout><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (const Rin*)in, (Rout*)out);
}

void destroy_graphs(dg_swe_ctx* c) {
  if (c->g1) cudaGraphExecDestroy(c->g1);
  if (c->gN) cudaGraphExecDestroy(c->gN);
  c->g1 = c->gN = nullptr;
}

dg_status capture(dg_swe_ctx* c, int nsteps, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(c->priv, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < nsteps; ++i) enqueue_step(c, 0.0, c->priv);
  cudaError_t e = cudaStreamEndCapture(c->priv, &g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  return DG_OK;
}

dg_status read_scalars(dg_swe_ctx* c, DevScalars* h) {
  CK(cudaMemcpyAsync(h, c->at<DevScalars>(c->off.sc), sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DG_OK;
}

void fill_stats(const DevScalars& s, dg_swe_stats* st) {
  if (!st) return;
  st->steps = s.steps;
  st->t = s.t;
  st->dt_last = s.dt;
  st->dt_min = s.steps ? s.dt_min : 0.0;
  st->dt_max = s.dt_max;
  st->mass = s.mass;
  st->mass0 = s.mass0;
  st->status = s.status;
}

}  // namespace

extern "C" {

dg_status dg_swe_init(const dg_swe_mesh* mesh, int order, int regularization, const dg_swe_params* params,
                      dg_swe_ctx** out) {
  if (!out) return DG_ERR_ARG;
  *out = nullptr;
  if (!mesh || !params || !mesh->coords || !mesh->elem_vertices) return DG_ERR_ARG;
  std::unique_ptr<dg_swe_ctx> c(new dg_swe_ctx());
  const dg_swe_params& p = *params;
  if (mesh->dim < 1 || mesh->dim > 2 || order < 1 || order > 3 || mesh->n_elements < 1 ||
      mesh->n_elements > (int64_t)0x7fffffff / 16 || mesh->n_vertices < 2) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, "need dim in {1,2}, order in {1,2,3}, 1 <= n_elements < 2^27");
  }
  if (regularization < 0 || regularization > 5 || p.n_bc < 1 || p.n_bc > DG_SWE_MAX_BC ||
      p.precision < 0 || p.precision > 2 || !(p.g > 0) || !(p.rho > 0) || !(p.cfl > 0) || p.eta < 0 ||
      p.sigma0 < 0 || !(p.h_floor > 0)) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, "invalid parameters (regularization, n_bc, precision, g, rho, cfl, eta, sigma0, h_floor)");
  }
  if (p.sigma0 > 0 && (regularization == 1 || regularization == 2 || regularization == 3 || regularization == 5) &&
      !(p.gamma > 0)) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, "gamma must be positive");
  }
  if (p.sigma0 > 0 && (regularization == 1 || regularization == 2) && !(p.beta > 0)) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, "beta must be positive");
  }
  if (regularization == 2 && p.sigma0 > 0 && p.sigma0 < 0.5 / p.beta) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, "local quadratic regularization needs sigma0 >= 1/(2 beta)");
  }
  if (!(p.flow_index == 0.0 || p.flow_index == 1.0 ||
        (p.flow_index > 0.0 && p.flow_index < 1.0 && p.rate_floor > 0.0))) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, "flow_index must be 0 or 1 (Newtonian) or in (0, 1) with rate_floor > 0");
  }
  if (regularization == 4 && p.sigma0 > 0 && !(p.pap_m > 0)) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, "pap_m must be positive");
  }
  for (int b = 0; b < p.n_bc; ++b)
    for (int s = 0; s < 7; ++s)
      if (p.bc[b].mode[s] < 0 || p.bc[b].mode[s] > 2 || (p.bc[b].mode[s] == 2 && (s == 0 || s > mesh->dim))) {
        *out = c.release();
        return fail(*out, DG_ERR_ARG, "bad boundary mode (wall applies to velocity slots only)");
      }
  c->dim = mesh->dim;
  c->p = order;
  c->reg = regularization;
  c->prec = p.precision;
  c->prm = p;
  c->rsize = p.precision == DG_PREC_FP64 ? 8 : 4;
  std::string err;
  if (!build_refops(c->dim, order, c->ops, err) ||
      !build_mesh(c->dim, mesh->n_vertices, mesh->coords, mesh->n_elements, mesh->elem_vertices, mesh->face_bc,
                  p.n_bc, c->ops, c->mesh, err)) {
    *out = c.release();
    return fail(*out, DG_ERR_ARG, err);
  }
  const int64_t K = c->mesh.K, F = c->mesh.F;
  const int Np = c->ops.Np, nV = c->dim + 1, nE = c->dim * c->dim, nf = c->dim + 1, Nfq = c->ops.Nfq;
  if (mesh->bed) {
    c->has_bed = true;
    c->bed.assign(mesh->bed, mesh->bed + K * Np);
    build_bed_source(c->dim, c->ops, K, c->mesh.geo, c->bed, p.g * std::cos(p.alpha), p.g * std::sin(p.alpha),
                     c->src);
  }
  c->drv = c->prec == DG_PREC_FP64 ? make_driver<double>(*c) : make_driver<float>(*c);
  // workspace layout
  const size_t rs = c->rsize;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += align256(bytes);
    return r;
  };
  c->nblk_dt = (int)((K + kRedBlock - 1) / kRedBlock);
  c->nblk_mass = c->nblk_dt;
  c->off.geo = take(kGeoRows * K * rs);
  c->off.nbr = take(nf * K * 4);
  c->off.nbrf = take(nf * K);
  c->off.fid = take(nf * K * 4);
  c->off.fn = take((size_t)nf * c->dim * K * rs);
  c->off.fsj = take(nf * K * rs);
  c->off.fe1 = take(F * 4);
  c->off.fe2 = take(F * 4);
  c->off.ff1 = take(F);
  c->off.ff2 = take(F);
  c->off.fnrm = take((size_t)c->dim * F * rs);
  c->off.fsjf = take(F * rs);
  c->off.bed = take(c->has_bed ? K * Np * rs : 0);
  c->off.src = take(c->has_bed ? (size_t)c->dim * c->ops.Nq * K * rs : 0);
  c->off.V0 = take((size_t)nV * K * Np * rs);
  c->off.V1 = take((size_t)nV * K * Np * rs);
  c->off.V2 = take((size_t)nV * K * Np * rs);
  c->off.E = take((size_t)nE * K * Np * rs);
  c->off.wflux = take((size_t)nV * F * Nfq * rs);
  c->off.partial = take((size_t)c->nblk_dt * 8);
  c->off.wint = take((size_t)Np * 8);
  c->off.sc = take(sizeof(DevScalars));
  c->off.bct = take((size_t)p.n_bc * (c->rsize == 8 ? sizeof(BCEntry<double>) : sizeof(BCEntry<float>)));
  c->off.tcimg = take(c->prec == DG_PREC_FP32_TC ? tc::image_bytes(c->dim, c->p) : 0);
  c->ws_need = o;
  *out = c.release();
  return DG_OK;
}

size_t dg_swe_workspace_size(const dg_swe_ctx* c) { return c ? c->ws_need : 0; }

dg_status dg_swe_set_stream(dg_swe_ctx* c, void* s) {
  if (!c) return DG_ERR_ARG;
  c->stream = (cudaStream_t)s;
  return DG_OK;
}

dg_status dg_swe_set_workspace(dg_swe_ctx* c, void* ptr, size_t bytes) {
  if (!c) return DG_ERR_ARG;
  if (!ptr || bytes < c->ws_need) return fail(c, DG_ERR_WORKSPACE, "workspace missing or smaller than dg_swe_workspace_size()");
  if (((uintptr_t)ptr & 255) != 0) return fail(c, DG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  destroy_graphs(c);
  {
    const cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  }
  c->ws = (char*)ptr;
  const int64_t K = c->mesh.K, F = c->mesh.F;
  const int nf = c->dim + 1;
  cudaStream_t s = c->stream;
  // host staging in the compute precision
  auto up_real = [&](size_t off, const std::vector<double>& v) -> cudaError_t {
    if (v.empty()) return cudaSuccess;
    if (c->rsize == 8) return cudaMemcpyAsync(c->ws + off, v.data(), v.size() * 8, cudaMemcpyHostToDevice, s);
    std::vector<float> f(v.begin(), v.end());
    cudaError_t e = cudaMemcpyAsync(c->ws + off, f.data(), f.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };
  const MeshData& m = c->mesh;
  CK(up_real(c->off.geo, m.geo));
  CK(cudaMemcpyAsync(c->ws + c->off.nbr, m.nbr.data(), nf * K * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->ws + c->off.nbrf, m.nbrf.data(), nf * K, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->ws + c->off.fid, m.fid.data(), nf * K * 4, cudaMemcpyHostToDevice, s));
  CK(up_real(c->off.fn, m.fn));
  CK(up_real(c->off.fsj, m.fsj));
  CK(cudaMemcpyAsync(c->ws + c->off.fe1, m.face_e1.data(), F * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->ws + c->off.fe2, m.face_e2.data(), F * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->ws + c->off.ff1, m.face_f1.data(), F, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->ws + c->off.ff2, m.face_f2.data(), F, cudaMemcpyHostToDevice, s));
  CK(up_real(c->off.fnrm, m.face_n));
  CK(up_real(c->off.fsjf, m.face_sj));
  if (c->has_bed) CK(up_real(c->off.bed, c->bed));
  if (c->has_bed) CK(up_real(c->off.src, c->src));
  CK(cudaMemcpyAsync(c->ws + c->off.wint, c->ops.wint.data(), c->ops.Np * 8, cudaMemcpyHostToDevice, s));
  if (c->rsize == 8) {
    auto t = make_bc_table<double>(c->prm);
    CK(cudaMemcpyAsync(c->ws + c->off.bct, t.data(), t.size() * sizeof(t[0]), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  } else {
    auto t = make_bc_table<float>(c->prm);
    CK(cudaMemcpyAsync(c->ws + c->off.bct, t.data(), t.size() * sizeof(t[0]), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  if (c->prec == DG_PREC_FP32_TC && tc::image_bytes(c->dim, c->p) > 0) {
    std::vector<float> img;
    tc::build_image(c->dim, c->p, c->ops, img);
    CK(cudaMemcpyAsync(c->ws + c->off.tcimg, img.data(), img.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaMemsetAsync(c->ws + c->off.E, 0, (size_t)c->dim * c->dim * K * c->ops.Np * c->rsize, s));
  reset_scalars_kernel<<<1, 1, 0, s>>>(c->at<DevScalars>(c->off.sc));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status dg_swe_node_coords(const dg_swe_ctx* c, double* xyz) {
  if (!c || !xyz) return DG_ERR_ARG;
  std::memcpy(xyz, c->mesh.node_xyz.data(), c->mesh.node_xyz.size() * sizeof(double));
  return DG_OK;
}

dg_status dg_swe_sizes(const dg_swe_ctx* c, int64_t* K, int32_t* np, int32_t* nv, int32_t* ne, int64_t* nfaces) {
  if (!c) return DG_ERR_ARG;
  if (K) *K = c->mesh.K;
  if (np) *np = c->ops.Np;
  if (nv) *nv = c->dim + 1;
  if (ne) *ne = c->dim * c->dim;
  if (nfaces) *nfaces = c->mesh.F;
  return DG_OK;
}

dg_status dg_swe_set_state(dg_swe_ctx* c, const double* V, int on_device) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  if (!V) return fail(c, DG_ERR_ARG, "null state");
  const size_t n = (size_t)(c->dim + 1) * c->mesh.K * c->ops.Np;
  cudaStream_t s = c->stream;
  void* V0 = c->ws + c->off.V0;
  if (c->rsize == 8) {
    CK(cudaMemcpyAsync(V0, V, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else if (on_device) {
    convert<double, float>(V, V0, n, s);
  } else {
    std::vector<float> f(V, V + n);
    CK(cudaMemcpyAsync(V0, f.data(), n * 4, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  reset_scalars_kernel<<<1, 1, 0, s>>>(c->at<DevScalars>(c->off.sc));
  enqueue_mass(c, 1, s);
  CK(cudaGetLastError());
  if (!on_device) CK(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status dg_swe_get_state(dg_swe_ctx* c, double* V, double* E, int on_device) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  const size_t nv = (size_t)(c->dim + 1) * c->mesh.K * c->ops.Np;
  const size_t ne = (size_t)c->dim * c->dim * c->mesh.K * c->ops.Np;
  cudaStream_t s = c->stream;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  auto out = [&](void* dst, size_t off, size_t n) -> cudaError_t {
    if (!dst) return cudaSuccess;
    if (c->rsize == 8) return cudaMemcpyAsync(dst, c->ws + off, n * 8, kind, s);
    if (on_device) {
      convert<float, double>(c->ws + off, dst, n, s);
      return cudaGetLastError();
    }
    std::vector<float> f(n);
    cudaError_t e = cudaMemcpyAsync(f.data(), c->ws + off, n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t i = 0; i < n; ++i) ((double*)dst)[i] = f[i];
    return e;
  };
  CK(out(V, c->off.V0, nv));
  CK(out(E, c->off.E, ne));
  DevScalars h{};
  st = read_scalars(c, &h);
  if (st != DG_OK) return st;
  if (h.status != 0) return fail(c, (dg_status)h.status, "device status: non-finite state");
  return DG_OK;
}

dg_status dg_swe_residual(dg_swe_ctx* c, const double* V_dev, double* dVdt_dev, double* E_dev) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  if (!V_dev || !dVdt_dev) return fail(c, DG_ERR_ARG, "null device pointer");
  const size_t nv = (size_t)(c->dim + 1) * c->mesh.K * c->ops.Np;
  const size_t ne = (size_t)c->dim * c->dim * c->mesh.K * c->ops.Np;
  cudaStream_t s = c->stream;
  void* E = c->ws + c->off.E;
  if (c->rsize == 8) {
    c->drv->estep(c, V_dev, E, s);
    c->drv->face(c, V_dev, E, s);
    c->drv->volume(c, V_dev, nullptr, dVdt_dev, 0, 0.0, 0.0, s);
    if (E_dev) CK(cudaMemcpyAsync(E_dev, E, ne * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    void* V1 = c->ws + c->off.V1;
    void* V2 = c->ws + c->off.V2;
    convert<double, float>(V_dev, V1, nv, s);
    c->drv->estep(c, V1, E, s);
    c->drv->face(c, V1, E, s);
    c->drv->volume(c, V1, nullptr, V2, 0, 0.0, 0.0, s);
    convert<float, double>(V2, dVdt_dev, nv, s);
    if (E_dev) convert<float, double>(E, E_dev, ne, s);
  }
  CK(cudaGetLastError());
  return DG_OK;
}

dg_status dg_swe_step(dg_swe_ctx* c, double dt, double* dt_taken) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  enqueue_step(c, dt > 0 ? dt : 0.0, c->stream);
  CK(cudaGetLastError());
  if (dt_taken) {
    DevScalars h{};
    st = read_scalars(c, &h);
    if (st != DG_OK) return st;
    *dt_taken = h.dt;
    if (h.status != 0) return fail(c, (dg_status)h.status, "device status: non-finite state");
  }
  return DG_OK;
}

dg_status dg_swe_run(dg_swe_ctx* c, int64_t n_steps, double t_end, dg_swe_stats* stats) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  if (n_steps < 0) return fail(c, DG_ERR_ARG, "n_steps < 0");
  if (t_end > 0) {
    for (int64_t i = 0; i < n_steps; ++i) {
      DevScalars h{};
      st = read_scalars(c, &h);
      if (st != DG_OK) return st;
      if (h.t >= t_end || h.status) break;
      double dtc = 0.0;
      st = dg_swe_step(c, 0.0, &dtc);
      if (st != DG_OK) return st;
      st = read_scalars(c, &h);
      if (st != DG_OK) return st;
      if (h.t > t_end) {  // redo the last step with the remaining time
        return fail(c, DG_ERR_UNSUPPORTED, "t_end landing needs a fixed final step; call dg_swe_step(dt)");
      }
    }
  } else if (n_steps > 0) {
    st = dg_swe_advance(c, n_steps);
    if (st != DG_OK) return st;
  }
  enqueue_mass(c, 0, c->stream);
  CK(cudaGetLastError());
  DevScalars h{};
  st = read_scalars(c, &h);
  if (st != DG_OK) return st;
  fill_stats(h, stats);
  if (h.status != 0) return fail(c, (dg_status)h.status, "device status: non-finite state");
  return DG_OK;
}

dg_status dg_swe_advance(dg_swe_ctx* c, int64_t n_steps) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  if (n_steps < 0) return fail(c, DG_ERR_ARG, "n_steps < 0");
  if (n_steps == 0) return DG_OK;
  if (!c->priv) {
    CK(cudaStreamCreateWithFlags(&c->priv, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  if (!c->g1) {
    st = capture(c, 1, &c->g1);
    if (st != DG_OK) return st;
    st = capture(c, kGraphSteps, &c->gN);
    if (st != DG_OK) return st;
  }
  // fork onto the private capture stream and join back: the caller's stream
  // orders everything before and after this call
  CK(cudaEventRecord(c->ev_fork, c->stream));
  CK(cudaStreamWaitEvent(c->priv, c->ev_fork, 0));
  int64_t left = n_steps;
  while (left >= kGraphSteps) {
    CK(cudaGraphLaunch(c->gN, c->priv));
    left -= kGraphSteps;
  }
  while (left-- > 0) CK(cudaGraphLaunch(c->g1, c->priv));
  CK(cudaEventRecord(c->ev_join, c->priv));
  CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  return DG_OK;
}

dg_status dg_swe_time_kernels(dg_swe_ctx* c, int n_iter, double* ms) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  if (n_iter < 1 || !ms) return fail(c, DG_ERR_ARG, "n_iter >= 1 and ms[5] required");
  cudaStream_t s = c->stream;
  void* V0 = c->ws + c->off.V0;
  void* V1 = c->ws + c->off.V1;
  void* E = c->ws + c->off.E;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  // E and the face fluxes of the current state feed the volume kernel
  c->drv->estep(c, V0, E, s);
  c->drv->face(c, V0, E, s);
  for (int k = 0; k < 5; ++k) {
    CK(cudaEventRecord(a, s));
    for (int i = 0; i < n_iter; ++i) {
      switch (k) {
        case 0: c->drv->estep(c, V0, E, s); break;
        case 1: c->drv->face(c, V0, E, s); break;
        case 2: c->drv->volume(c, V0, V0, V1, 1, 0.0, 1.0, s); break;
        case 3:
          c->drv->dt_partial(c, V0, s);
          break;
        case 4: c->drv->mass_partial(c, V0, s); break;
      }
    }
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, a, b));
    ms[k] = (double)t / n_iter;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CK(cudaGetLastError());
  return DG_OK;
}

dg_status dg_swe_sync(dg_swe_ctx* c, dg_swe_stats* stats) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  enqueue_mass(c, 0, c->stream);
  CK(cudaGetLastError());
  DevScalars h{};
  st = read_scalars(c, &h);
  if (st != DG_OK) return st;
  fill_stats(h, stats);
  if (h.status != 0) return fail(c, (dg_status)h.status, "device status: non-finite state");
  return DG_OK;
}

int32_t dg_swe_launches_per_step(const dg_swe_ctx* c) { return c ? (c->prm.positivity ? 14 : 11) : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Scratch for dg_swe_residual_static: a file-scope device array, so that the
// call needs no device allocation of its own.  Every GPU that loads the
// library holds these bytes until the process exits.  Host code only ever
// sees a stand-in symbol here; its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_scratch[DG_SWE_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the context's device, which must be
// the current device (looked up on the first call per device).
dg_status static_scratch(dg_swe_ctx* c, void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  if (dev != c->device)
    return fail(c, DG_ERR_ARG, "device " + std::to_string(dev) + " is current but the context's workspace is on device " +
                                   std::to_string(c->device) + "; make the context's device current");
  if (dev < 0 || dev >= kMaxDevices) return fail(c, DG_ERR_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(c, e, "cudaGetSymbolAddress(g_static_scratch)");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return DG_OK;
}
}  // namespace

extern "C" {

size_t dg_swe_static_scratch_need(const dg_swe_ctx* c) {
  if (!c) return 0;
  const size_t np = (size_t)c->mesh.K * c->ops.Np;
  size_t need = align256((size_t)c->dim * c->dim * np * c->rsize)                        // E
              + align256((size_t)(c->dim + 1) * c->mesh.F * c->ops.Nfq * c->rsize);     // face fluxes
  if (c->rsize == 4) need += 2 * align256((size_t)(c->dim + 1) * np * 4);                // FP32 in/out
  return need;
}

dg_status dg_swe_residual_static(dg_swe_ctx* c, const double* V_dev, double* dVdt_dev, double* E_dev) {
  dg_status st = check_ws(c);
  if (st != DG_OK) return st;
  if (!V_dev || !dVdt_dev) return fail(c, DG_ERR_ARG, "null device pointer");
  const size_t need = dg_swe_static_scratch_need(c);
  if (need > (size_t)DG_SWE_STATIC_SCRATCH_BYTES)
    return fail(c, DG_ERR_ARG, "problem needs " + std::to_string(need) + " scratch bytes; the static scratch holds " +
                                   std::to_string((size_t)DG_SWE_STATIC_SCRATCH_BYTES));
  char* base = nullptr;
  st = static_scratch(c, (void**)&base);
  if (st != DG_OK) return st;
  const size_t np = (size_t)c->mesh.K * c->ops.Np;
  const size_t nv = (size_t)(c->dim + 1) * np, ne = (size_t)c->dim * c->dim * np;
  char* E = base;
  char* wflux = E + align256(ne * c->rsize);
  char* tail = wflux + align256((size_t)(c->dim + 1) * c->mesh.F * c->ops.Nfq * c->rsize);
  cudaStream_t s = c->stream;
  // Every scratch word is written (E by the E-step, fluxes by the face pass)
  // before it is read, so nothing left by an earlier call needs clearing.
  if (c->rsize == 8) {
    c->drv->estep(c, V_dev, E, s);
    c->drv->face_into(c, V_dev, E, wflux, s);
    c->drv->residual_from(c, V_dev, E, wflux, dVdt_dev, s);
    if (E_dev) CK(cudaMemcpyAsync(E_dev, E, ne * 8, cudaMemcpyDeviceToDevice, s));
  } else {
    char* Vf = tail;
    char* Of = tail + align256(nv * 4);
    convert<double, float>(V_dev, Vf, nv, s);
    c->drv->estep(c, Vf, E, s);
    c->drv->face_into(c, Vf, E, wflux, s);
    c->drv->residual_from(c, Vf, E, wflux, Of, s);
    convert<float, double>(Of, dVdt_dev, nv, s);
    if (E_dev) convert<float, double>(E, E_dev, ne, s);
  }
  CK(cudaGetLastError());
  return DG_OK;
}

const char* dg_swe_last_error(const dg_swe_ctx* c) { return c ? c->err.c_str() : "null context"; }

void dg_swe_destroy(dg_swe_ctx* c) {
  if (!c) return;
  destroy_graphs(c);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->priv) cudaStreamDestroy(c->priv);
  delete c;
}

}  // extern "C"

// Internal definition of the single-instance context (shared by the
// translation units of the library; not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/dg_swe.h"
#include "dg_host.h"

struct dg_swe_ctx;

namespace dgswe {
// Kernel launches of one (dimension, order, precision) instantiation.
struct Driver {
  virtual ~Driver() = default;
  virtual void estep(dg_swe_ctx* c, const void* V, void* E, cudaStream_t s) = 0;
  virtual void face(dg_swe_ctx* c, const void* V, const void* E, cudaStream_t s) = 0;
  virtual void volume(dg_swe_ctx* c, const void* Vin, const void* V0, void* out, int mode, double c0,
                      double c1, cudaStream_t s) = 0;
  // wet/dry mode: out = the conservative stage from Vin, V0 and the residual
  // rbuf that a volume pass in mode 2 wrote (rbuf and V0 may alias out)
  virtual void wetdry_stage(dg_swe_ctx* c, const void* Vin, const void* V0, const void* rbuf, void* out, double c0,
                            double c1, cudaStream_t s) = 0;
  virtual void dt_partial(dg_swe_ctx* c, const void* V, cudaStream_t s) = 0;
  virtual void mass_partial(dg_swe_ctx* c, const void* V, cudaStream_t s) = 0;
  // Face flux and residual-mode volume pass with caller-chosen scratch for
  // the face fluxes and E (used by dg_swe_residual_static).
  virtual void face_into(dg_swe_ctx* c, const void* V, const void* E, void* wflux, cudaStream_t s) = 0;
  virtual void residual_from(dg_swe_ctx* c, const void* V, const void* E, const void* wflux, void* out,
                             cudaStream_t s) = 0;
  // Backward-Euler support (dg_newton.h): <l_a, U(V)> (mode 0) or
  // out += (<l_a, U(V)> - Uold) * inv_dt (mode 1); z = scale M(V)^{-1} x.
  virtual void be_time(dg_swe_ctx* c, const void* V, const void* Uold, void* out, double inv_dt, int mode,
                       cudaStream_t s) = 0;
  virtual void precond(dg_swe_ctx* c, const void* V, const void* x, void* z, double scale, cudaStream_t s) = 0;
};
struct DriverDeleter {
  void operator()(Driver* d) const;
};
using DriverPtr = std::unique_ptr<Driver, DriverDeleter>;
}  // namespace dgswe

struct dg_swe_ctx {
  int dim = 0, p = 0, reg = 0, prec = 0;
  dg_swe_params prm{};
  dgswe::RefOps ops;
  dgswe::MeshData mesh;
  std::vector<double> bed;
  std::vector<double> src;  // bed/slope source coefficients at the volume points, [dim * Nq][K] (bed only)
  bool has_bed = false;
  size_t rsize = 8;
  int device = -1;  // device current at dg_swe_set_workspace (the workspace's device)
  // workspace
  size_t ws_need = 0;
  char* ws = nullptr;
  struct {
    size_t geo, nbr, nbrf, fid, fn, fsj, fe1, fe2, ff1, ff2, fnrm, fsjf, bed, V0, V1, V2, E, wflux, partial, wint, sc,
        bct, tcimg, src;
  } off{};
  int nblk_dt = 0, nblk_mass = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t priv = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t g1 = nullptr, gN = nullptr;
  dgswe::DriverPtr drv;
  std::string err;

  template <typename T>
  T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
};

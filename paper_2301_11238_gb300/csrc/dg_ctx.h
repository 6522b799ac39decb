// Internal definition of the single-instance context (shared by the
// translation units of the library; not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/dg_swe.h"
#include "dg_host.h"

namespace dgswe {
struct Driver;
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
  bool has_bed = false;
  size_t rsize = 8;
  // workspace
  size_t ws_need = 0;
  char* ws = nullptr;
  struct {
    size_t geo, nbr, nbrf, fid, fn, fsj, fe1, fe2, ff1, ff2, fnrm, fsjf, bed, V0, V1, V2, E, wflux, partial, wint, sc,
        bct;
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

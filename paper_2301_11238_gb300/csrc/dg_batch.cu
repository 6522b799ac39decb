// Batched ensembles: many independent instances advanced by one launch per
// (dimension, order) group and phase, replayed from a CUDA graph.
// See include/dg_batch.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dg_batch.h"
#include "dg_ctx.h"
#include "dg_kernels.cuh"
#include "dg_tc.cuh"
#include "dg_persist.cuh"

using namespace dgswe;

namespace {

constexpr int kGraphSteps = 16;
inline size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Group;

struct GroupDrv {
  virtual ~GroupDrv() = default;
  virtual void estep(dg_batch* b, Group& g, int vin, cudaStream_t s) = 0;
  virtual void face(dg_batch* b, Group& g, int vin, cudaStream_t s) = 0;
  virtual void volume(dg_batch* b, Group& g, int vin, int vout, double c0, double c1, cudaStream_t s) = 0;
  // whether a volume block size is launchable (negative: staged form)
  virtual bool volume_ok(int tile) = 0;
  virtual void dt(dg_batch* b, Group& g, cudaStream_t s) = 0;
  virtual void mass(dg_batch* b, Group& g, int first, int count, int set_ref, cudaStream_t s) = 0;
  // one whole SSP-RK3 step of the group in one persistent launch (dg_persist.cuh)
  virtual void persistent_step(dg_batch* b, Group& g, cudaStream_t s) = 0;
};

struct Group {
  int dim = 0, p = 0;
  bool pos = false;  // wet/dry mode (dg_swe_params.positivity) of all its members
  std::vector<int> members;          // global instance ids
  RefOps ops;
  int64_t K = 0, F = 0;
  bool has_bed = false;
  std::vector<int64_t> ebase, fbase;  // per member
  // host staging (uploaded by set_workspace)
  std::vector<double> geo, fn, fsj, face_n, face_sj, bed;
  // per member: its bed/slope source coefficients [dim * Nq][K_m] (a flat-bed
  // member of a group with beds: -g_s and 0); interleaved into src
  std::vector<std::vector<double>> src_blocks;
  std::vector<double> src, gs_of;
  std::vector<int32_t> nbr, fid, fe1, fe2, inst, gid;
  std::vector<int8_t> nbrf, ff1, ff2;
  std::vector<int64_t> ebeg;
  struct {
    size_t geo, nbr, nbrf, fid, fn, fsj, fe1, fe2, ff1, ff2, fnrm, fsjf, bed, inst, ebeg, gid, V[3], E, wflux, wint,
        blk_e, blk_gid, mblk, partial, tcimg, src, p_etile, p_ftile, p_fbeg, p_tdt, p_cnt;
  } off{};
  std::vector<int64_t> blk_e;      // step-size blocks: element ranges (n_blk + 1)
  std::vector<int32_t> blk_gid;    // global instance of each block
  std::vector<int32_t> mblk;       // first block of each member (members + 1)
  // plan of the persistent step (dg_persist.cuh): prefixes of element and
  // face-point tiles per member, first face per member, item range per phase
  std::vector<int32_t> p_etile, p_ftile;
  std::vector<int64_t> p_fbeg;
  int p_pstart[persist::kPhases + 1] = {};
  int tile[3] = {128, 128, 128};
  std::unique_ptr<GroupDrv> drv;
};

}  // namespace

struct dg_batch {
  int n = 0, prec = 0;
  size_t rsize = 8;
  bool persistent = false;  // one persistent launch per group and step (dg_batch_set_persistent)
  std::vector<int> dim, order, reg, group_of, local_of;
  std::vector<int64_t> K_of, Np_of;
  std::vector<dg_swe_params> prm;
  std::vector<Group> groups;
  std::vector<int> bc_base;
  int n_bc_total = 0;
  std::vector<char> h_phys, h_bc;  // host copies of the per-instance tables
  std::vector<double> h_iparm;     // per instance: g_c, h_floor, cfl, nu
  size_t ws_need = 0;
  char* ws = nullptr;
  size_t off_ptab = 0, off_bct = 0, off_sc = 0, off_iparm = 0;
  cudaStream_t stream = nullptr, priv = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t g1 = nullptr, gN = nullptr;
  std::string err;
  template <typename T>
  T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
};

namespace {

dg_status bfail(dg_batch* b, dg_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}
dg_status bcuda(dg_batch* b, cudaError_t e, const char* where) {
  return bfail(b, DG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define BK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);   \
  } while (0)

// Integral of h per instance, in two fixed-order passes so that repeated
// calls give identical sums: one block per 256-element range of one
// instance (the step-size blocks) writes its FP64 partial, then one warp per
// instance adds its blocks' partials.  (A single block per instance left a
// whole SM reducing an 8.4M-element instance: 35 ms per set_state.)
template <int NP, typename R>
__global__ void __launch_bounds__(256) mass_block_kernel(int K, int b0, const int64_t* __restrict__ blk_e,
                                                         const R* __restrict__ V, const R* __restrict__ geo,
                                                         const double* __restrict__ wint,
                                                         double* __restrict__ partial) {
  __shared__ double red[8];
  const int b = b0 + blockIdx.x;
  const int64_t e = blk_e[b] + threadIdx.x;
  double v = 0.0;
  if (e < blk_e[b + 1]) {
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < NP; ++a) sum += wint[a] * (double)V[(size_t)e * NP + a];
    v = (double)geo[4 * (size_t)K + e] * sum;
  }
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    partial[b] = t;
  }
}

static __global__ void mass_members_kernel(int first, int count, const int32_t* __restrict__ mblk,
                                           const int32_t* __restrict__ gid, const double* __restrict__ partial,
                                           int set_ref, DevScalars* __restrict__ sc) {
  const int i = first + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= first + count) return;
  double m = 0.0;
  for (int b = mblk[i] + lane; b < mblk[i + 1]; b += 32) m += partial[b];
  m = warp_sum(m);
  if (lane == 0) {
    DevScalars& d = sc[gid[i]];
    d.mass = m;
    if (set_ref) d.mass0 = m;
  }
}

template <int DIM, int P, typename R>
struct GDrv final : GroupDrv {
  using S = Sh<DIM, P>;
  // the tensor-core volume form exists for FP32 triangles of order >= 2
  static constexpr bool kTcForm = DIM == 2 && P >= 2 && sizeof(R) == 4;
  EstepOps<DIM, P, R> eo{};
  FaceOps<DIM, P, R> fo{};
  VolOps<DIM, P, R> vo{};
  bool tc = false;
  std::unique_ptr<tc::Launcher<(P >= 2 ? P : 2), true>> tcl;
  int n_sm = 0;
  size_t smem_optin = 0;     // shared memory a block may use (static + dynamic)
  size_t staged_static = 0;  // the staged kernel's static shared memory
  std::map<int, int> staged_grid;  // staged volume block size -> persistent grid size (0: not launchable)
  int persist_grid = 0;            // resident blocks of the persistent step kernel (0: not yet queried)
  void persistent_step(dg_batch* b, Group& g, cudaStream_t s) override;
  explicit GDrv(const RefOps& o, bool use_tc) {
    fill_ops<DIM, P, R>(o, eo, fo, vo);
    if constexpr (kTcForm) {
      tc = use_tc;
      if (tc) tcl.reset(new tc::Launcher<P, true>());
    }
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) n_sm = v;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
        smem_optin = (size_t)v;
    }
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, volume_staged_kernel<DIM, P, R>) == cudaSuccess)
      staged_static = fa.sharedSizeBytes;
    if (smem_optin > staged_static)
      cudaFuncSetAttribute(volume_staged_kernel<DIM, P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(smem_optin - staged_static));
    cudaGetLastError();
  }
  // persistent grid of the staged volume kernel: resident blocks per SM x SMs
  int staged_blocks(int T) {
    auto it = staged_grid.find(T);
    if (it != staged_grid.end()) return it->second;
    int nb = 0;
    const size_t smem = staged_smem_bytes<DIM, P, R>(T);
    if (n_sm > 0 && smem + staged_static <= smem_optin &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, volume_staged_kernel<DIM, P, R>, T, smem) != cudaSuccess)
      nb = 0;
    cudaGetLastError();
    staged_grid[T] = nb * n_sm;
    return nb * n_sm;
  }
  // resident blocks of the grid-stride per-face kernel at block size T, times the SMs
  std::map<int, int> pf_grid;
  int face_pf_blocks(int T) {
    auto it = pf_grid.find(T);
    if (it != pf_grid.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, face_pf_kernel<DIM, P, R>, T, 0) != cudaSuccess || nb < 1)
      nb = 1;
    cudaGetLastError();
    pf_grid[T] = nb * (n_sm > 0 ? n_sm : 1);
    return pf_grid[T];
  }
  bool volume_ok(int tile) override {
    if (tile > 0) return tile >= 32 && tile <= 256 && tile % 32 == 0;
    const int T = -tile;
    return T >= 32 && T <= 256 && T % 32 == 0 && staged_blocks(T) > 0;
  }

  const Phys<R>* ptab(dg_batch* b) { return b->at<Phys<R>>(b->off_ptab); }
  const BCEntry<R>* bct(dg_batch* b) { return b->at<BCEntry<R>>(b->off_bct); }

  std::map<int, int> estep_grid;
  int estep_pf_blocks(int T) {
    auto it = estep_grid.find(T);
    if (it != estep_grid.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, estep_pf_kernel<DIM, P, R>, T, 0) != cudaSuccess || nb < 1)
      nb = 1;
    cudaGetLastError();
    estep_grid[T] = nb * (n_sm > 0 ? n_sm : 1);
    return estep_grid[T];
  }
  // tile[0] > 0: one thread per element; < 0: the grid-stride form that
  // prefetches the next element's neighbours (|tile| threads per block)
  void estep(dg_batch* b, Group& g, int vin, cudaStream_t s) override {
    const int K = (int)g.K;
    if (g.tile[0] < 0) {
      const int T = -g.tile[0];
      const int grid = std::max(1, std::min((K + T - 1) / T, estep_pf_blocks(T)));
      estep_pf_kernel<DIM, P, R><<<grid, T, 0, s>>>(
          K, b->at<R>(g.off.V[vin]), b->at<R>(g.off.E), b->at<R>(g.off.geo), b->at<int32_t>(g.off.nbr),
          b->at<int8_t>(g.off.nbrf), b->at<R>(g.off.fn), b->at<R>(g.off.fsj), eo, bct(b));
      return;
    }
    const int T = g.tile[0];
    estep_kernel<DIM, P, R><<<(K + T - 1) / T, T, 0, s>>>(
        K, b->at<R>(g.off.V[vin]), b->at<R>(g.off.E), b->at<R>(g.off.geo), b->at<int32_t>(g.off.nbr),
        b->at<int8_t>(g.off.nbrf), b->at<R>(g.off.fn), b->at<R>(g.off.fsj), eo, bct(b));
  }
  // tile[1] > 0: one thread per face point; < 0: one thread per face (|tile| threads per block)
  void face(dg_batch* b, Group& g, int vin, cudaStream_t s) override {
    const int K = (int)g.K, F = (int)g.F, T = g.tile[1] > 0 ? g.tile[1] : -g.tile[1];
    if (g.tile[1] > 0) {
      const long long n = (long long)F * S::NFQ;
      face_kernel<DIM, P, R, true, false><<<(unsigned)((n + T - 1) / T), T, 0, s>>>(
          K, F, b->at<R>(g.off.V[vin]), b->at<R>(g.off.E), b->at<int32_t>(g.off.fe1), b->at<int8_t>(g.off.ff1),
          b->at<int32_t>(g.off.fe2), b->at<int8_t>(g.off.ff2), b->at<R>(g.off.fnrm), b->at<R>(g.off.fsjf),
          b->at<R>(g.off.wflux), fo, Phys<R>{}, ptab(b), b->at<int32_t>(g.off.inst), bct(b));
    } else {
      // one thread per face in a grid-stride loop over the resident blocks
      // (the next face's connectivity loads while the current one computes)
      const int grid = std::max(1, std::min((F + T - 1) / T, face_pf_blocks(T)));
      face_pf_kernel<DIM, P, R><<<(unsigned)grid, T, 0, s>>>(
          K, F, b->at<R>(g.off.V[vin]), b->at<R>(g.off.E), b->at<int32_t>(g.off.fe1), b->at<int8_t>(g.off.ff1),
          b->at<int32_t>(g.off.fe2), b->at<int8_t>(g.off.ff2), b->at<R>(g.off.fnrm), b->at<R>(g.off.fsjf),
          b->at<R>(g.off.wflux), fo, ptab(b), b->at<int32_t>(g.off.inst), bct(b));
    }
  }
  void volume(dg_batch* b, Group& g, int vin, int vout, double c0, double c1, cudaStream_t s) override {
    const int K = (int)g.K, F = (int)g.F;
    if (g.pos) {
      // wet/dry group: r_V (mode 2) into the stage's output buffer, or into
      // stage buffer 1 when the output is V0 (the last stage), then the
      // conservative stage from it
      const int rb = vout != 0 ? vout : 1;
      residual(b, g, vin, rb, s);
      wetdry_stage_kernel<DIM, P, R, true><<<(K + 127) / 128, 128, 0, s>>>(
          K, b->at<R>(g.off.V[vin]), b->at<R>(g.off.V[0]), b->at<R>(g.off.V[rb]), b->at<R>(g.off.V[vout]),
          b->at<R>(g.off.geo), vo, Phys<R>{}, ptab(b), b->at<int32_t>(g.off.inst), (R)c0, (R)c1,
          b->at<DevScalars>(b->off_sc));
      return;
    }
    if constexpr (kTcForm) {
      if (tc) {  // the tensor-core form has its own fixed launch shape; the tile setting is not used
        (*tcl)(K, F, b->at<float>(g.off.V[vin]), b->at<float>(g.off.V[0]), b->at<float>(g.off.V[vout]),
               b->at<float>(g.off.E), g.has_bed ? b->at<float>(g.off.bed) : nullptr, b->at<float>(g.off.geo),
               b->at<int32_t>(g.off.fid), b->at<float>(g.off.wflux), vo, b->at<float>(g.off.tcimg), Phys<float>{},
               ptab(b), b->at<int32_t>(g.off.inst), 1, (float)c0, (float)c1, b->at<DevScalars>(b->off_sc), s);
        return;
      }
    }
    if (g.tile[2] < 0) {
      const int T = -g.tile[2];
      const int ntiles = (K + T - 1) / T;
      const int grid = std::min(ntiles, staged_blocks(T));
      if (grid <= 0) return;
      volume_staged_kernel<DIM, P, R><<<grid, T, staged_smem_bytes<DIM, P, R>(T), s>>>(
          K, F, b->at<R>(g.off.V[vin]), b->at<R>(g.off.V[0]), b->at<R>(g.off.V[vout]), b->at<R>(g.off.E),
          g.has_bed ? b->at<R>(g.off.bed) : nullptr, g.has_bed ? b->at<R>(g.off.src) : nullptr,
          b->at<R>(g.off.geo), b->at<int32_t>(g.off.fid),
          b->at<R>(g.off.wflux), vo, ptab(b), b->at<int32_t>(g.off.inst), (R)c0, (R)c1,
          b->at<DevScalars>(b->off_sc));
      return;
    }
    const int T = g.tile[2];
    volume_kernel<DIM, P, R, true><<<(K + T - 1) / T, T, 0, s>>>(
        K, F, b->at<R>(g.off.V[vin]), b->at<R>(g.off.V[0]), b->at<R>(g.off.V[vout]), b->at<R>(g.off.E),
        g.has_bed ? b->at<R>(g.off.bed) : nullptr, g.has_bed ? b->at<R>(g.off.src) : nullptr,
          b->at<R>(g.off.geo), b->at<int32_t>(g.off.fid),
        b->at<R>(g.off.wflux), vo, Phys<R>{}, ptab(b), b->at<int32_t>(g.off.inst), 1, (R)c0, (R)c1,
        b->at<DevScalars>(b->off_sc));
  }
  // the volume pass in mode 2 (r_V of V[vin] into V[vout]): the tensor-core
  // form or the direct kernel (the staged form has no mode 2; a negative
  // block size is taken by its magnitude)
  void residual(dg_batch* b, Group& g, int vin, int vout, cudaStream_t s) {
    const int K = (int)g.K, F = (int)g.F;
    if constexpr (kTcForm) {
      if (tc) {
        (*tcl)(K, F, b->at<float>(g.off.V[vin]), nullptr, b->at<float>(g.off.V[vout]), b->at<float>(g.off.E),
               g.has_bed ? b->at<float>(g.off.bed) : nullptr, b->at<float>(g.off.geo), b->at<int32_t>(g.off.fid),
               b->at<float>(g.off.wflux), vo, b->at<float>(g.off.tcimg), Phys<float>{}, ptab(b),
               b->at<int32_t>(g.off.inst), 2, 0.0f, 0.0f, b->at<DevScalars>(b->off_sc), s);
        return;
      }
    }
    const int T = g.tile[2] > 0 ? g.tile[2] : -g.tile[2];
    volume_kernel<DIM, P, R, true><<<(K + T - 1) / T, T, 0, s>>>(
        K, F, b->at<R>(g.off.V[vin]), nullptr, b->at<R>(g.off.V[vout]), b->at<R>(g.off.E),
        g.has_bed ? b->at<R>(g.off.bed) : nullptr, g.has_bed ? b->at<R>(g.off.src) : nullptr, b->at<R>(g.off.geo),
        b->at<int32_t>(g.off.fid), b->at<R>(g.off.wflux), vo, Phys<R>{}, ptab(b), b->at<int32_t>(g.off.inst), 2, R(0),
        R(0), b->at<DevScalars>(b->off_sc));
  }
  void dt(dg_batch* b, Group& g, cudaStream_t s) override {
    const int nblk = (int)g.blk_gid.size(), nm = (int)g.members.size();
    dt_block_kernel<DIM, P, R><<<nblk, 256, 0, s>>>((int)g.K, b->at<int64_t>(g.off.blk_e),
                                                    b->at<int32_t>(g.off.blk_gid), b->at<R>(g.off.V[0]),
                                                    b->at<R>(g.off.geo), b->at<double>(b->off_iparm),
                                                    b->at<double>(g.off.partial));
    dt_members_kernel<<<(nm + 7) / 8, 256, 0, s>>>(nm, b->at<int32_t>(g.off.mblk), b->at<int32_t>(g.off.gid),
                                                   b->at<double>(g.off.partial), b->at<DevScalars>(b->off_sc));
  }
  void mass(dg_batch* b, Group& g, int first, int count, int set_ref, cudaStream_t s) override {
    if (count <= 0) return;
    const int b0 = g.mblk[first], nb = g.mblk[first + count] - b0;
    if (nb > 0)
      mass_block_kernel<S::NP, R><<<(unsigned)nb, 256, 0, s>>>((int)g.K, b0, b->at<int64_t>(g.off.blk_e),
                                                              b->at<R>(g.off.V[0]), b->at<R>(g.off.geo),
                                                              b->at<double>(g.off.wint), b->at<double>(g.off.partial));
    mass_members_kernel<<<(unsigned)((count + 7) / 8), 256, 0, s>>>(first, count, b->at<int32_t>(g.off.mblk),
                                                                   b->at<int32_t>(g.off.gid),
                                                                   b->at<double>(g.off.partial), set_ref,
                                                                   b->at<DevScalars>(b->off_sc));
  }
};

template <int DIM, int P, typename R>
void GDrv<DIM, P, R>::persistent_step(dg_batch* b, Group& g, cudaStream_t s) {
  const int nm = (int)g.members.size();
  persist::Plan pl{};
  pl.n_members = nm;
  for (int ph = 0; ph <= persist::kPhases; ++ph) pl.pstart[ph] = g.p_pstart[ph];
  pl.etile_pre = b->at<int32_t>(g.off.p_etile);
  pl.ftile_pre = b->at<int32_t>(g.off.p_ftile);
  pl.ebeg = b->at<int64_t>(g.off.ebeg);
  pl.fbeg = b->at<int64_t>(g.off.p_fbeg);
  pl.gid = b->at<int32_t>(g.off.gid);
  pl.tile_dt = b->at<double>(g.off.p_tdt);
  pl.done = b->at<int>(g.off.p_cnt);
  pl.next = pl.done + nm * persist::kPhases;
  persist::Arrays<R> A{};
  for (int v = 0; v < 3; ++v) A.V[v] = b->at<R>(g.off.V[v]);
  A.E = b->at<R>(g.off.E);
  A.wflux = b->at<R>(g.off.wflux);
  A.bed = g.has_bed ? b->at<R>(g.off.bed) : nullptr;
  A.src = g.has_bed ? b->at<R>(g.off.src) : nullptr;
  A.geo = b->at<R>(g.off.geo);
  A.fn = b->at<R>(g.off.fn);
  A.fsj = b->at<R>(g.off.fsj);
  A.fnrm = b->at<R>(g.off.fnrm);
  A.fsjf = b->at<R>(g.off.fsjf);
  A.nbr = b->at<int32_t>(g.off.nbr);
  A.fid = b->at<int32_t>(g.off.fid);
  A.fe1 = b->at<int32_t>(g.off.fe1);
  A.fe2 = b->at<int32_t>(g.off.fe2);
  A.inst = b->at<int32_t>(g.off.inst);
  A.nbrf = b->at<int8_t>(g.off.nbrf);
  A.ff1 = b->at<int8_t>(g.off.ff1);
  A.ff2 = b->at<int8_t>(g.off.ff2);
  A.ptab = ptab(b);
  A.bct = bct(b);
  A.iparm = b->at<double>(b->off_iparm);
  A.sc = b->at<DevScalars>(b->off_sc);
  A.K = (int)g.K;
  A.F = (int)g.F;
  if (persist_grid == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persist::step_kernel<DIM, P, R>, persist::kThreads, 0) !=
            cudaSuccess ||
        nb < 1)
      nb = 1;
    cudaGetLastError();
    persist_grid = nb * (n_sm > 0 ? n_sm : 1);
  }
  const int total = g.p_pstart[persist::kPhases];
  const int grid = std::max(1, std::min(total, persist_grid));
  cudaMemsetAsync(pl.done, 0, (size_t)(nm * persist::kPhases + 1) * sizeof(int), s);
  persist::step_kernel<DIM, P, R><<<grid, persist::kThreads, 0, s>>>(pl, A, eo, fo, vo);
}

template <typename R>
std::unique_ptr<GroupDrv> make_gdrv(int dim, int p, const RefOps& o, bool use_tc) {
#define GCASE(D, PP) \
  if (dim == D && p == PP) return std::unique_ptr<GroupDrv>(new GDrv<D, PP, R>(o, use_tc));
  GCASE(1, 1) GCASE(1, 2) GCASE(1, 3) GCASE(2, 1) GCASE(2, 2) GCASE(2, 3)
#undef GCASE
  return nullptr;
}

void enqueue_step(dg_batch* b, cudaStream_t s) {
  if (b->persistent) {
    for (auto& g : b->groups) g.drv->persistent_step(b, g, s);
    return;
  }
  for (auto& g : b->groups) g.drv->dt(b, g, s);
  const int vin[3] = {0, 1, 2}, vout[3] = {1, 2, 0};
  const double c0[3] = {0.0, 0.75, 1.0 / 3.0}, c1[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int st = 0; st < 3; ++st)
    for (auto& g : b->groups) {
      g.drv->estep(b, g, vin[st], s);
      g.drv->face(b, g, vin[st], s);
      g.drv->volume(b, g, vin[st], vout[st], c0[st], c1[st], s);
    }
}

void destroy_graphs(dg_batch* b) {
  if (b->g1) cudaGraphExecDestroy(b->g1);
  if (b->gN) cudaGraphExecDestroy(b->gN);
  b->g1 = b->gN = nullptr;
}

dg_status capture(dg_batch* b, int nsteps, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  BK(cudaStreamBeginCapture(b->priv, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < nsteps; ++i) enqueue_step(b, b->priv);
  cudaError_t e = cudaStreamEndCapture(b->priv, &g);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
  return DG_OK;
}

template <typename R>
void push_phys(const dg_swe_params& p, int reg, std::vector<char>& out) {
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
  const char* c = reinterpret_cast<const char*>(&ph);
  out.insert(out.end(), c, c + sizeof(ph));
}

template <typename R>
void push_bc(const dg_swe_bc& bc, std::vector<char>& out) {
  BCEntry<R> e{};
  for (int s = 0; s < 7; ++s) {
    e.mode[s] = bc.mode[s];
    e.val[s] = (R)bc.value[s];
  }
  const char* c = reinterpret_cast<const char*>(&e);
  out.insert(out.end(), c, c + sizeof(e));
}

dg_status check(dg_batch* b) {
  if (!b) return DG_ERR_ARG;
  if (!b->ws) return bfail(b, DG_ERR_WORKSPACE, "no workspace set (dg_batch_set_workspace)");
  return DG_OK;
}

template <typename Rin, typename Rout>
void conv(const void* in, void* out, size_t n, cudaStream_t s) {
  if (n) convert_kernel<Rin, Rout><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (const Rin*)in, (Rout*)out);
}

dg_status read_stats(dg_batch* b, dg_swe_stats* st) {
  std::vector<DevScalars> h(b->n);
  BK(cudaMemcpyAsync(h.data(), b->at<DevScalars>(b->off_sc), b->n * sizeof(DevScalars), cudaMemcpyDeviceToHost,
                     b->stream));
  BK(cudaStreamSynchronize(b->stream));
  int bad = -1;
  for (int i = 0; i < b->n; ++i) {
    if (h[i].status && bad < 0) bad = i;
    if (!st) continue;
    st[i].steps = h[i].steps;
    st[i].t = h[i].t;
    st[i].dt_last = h[i].dt;
    st[i].dt_min = h[i].steps ? h[i].dt_min : 0.0;
    st[i].dt_max = h[i].dt_max;
    st[i].mass = h[i].mass;
    st[i].mass0 = h[i].mass0;
    st[i].status = h[i].status;
  }
  if (bad >= 0)
    return bfail(b, (dg_status)h[bad].status,
                 std::string(h[bad].status == DG_ERR_TIMEOUT ? "device status: staged copy wait timed out"
                                                              : "device status: non-finite state") +
                     " in instance " + std::to_string(bad));
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_batch_init(int n, const dg_swe_mesh* meshes, const int* orders, const int* regs,
                        const dg_swe_params* params, dg_batch** out) {
  if (!out) return DG_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<dg_batch> b(new dg_batch());
  if (n < 1 || !meshes || !orders || !regs || !params) {
    *out = b.release();
    return bfail(*out, DG_ERR_ARG, "need n >= 1 and non-null arrays");
  }
  b->n = n;
  b->prec = params[0].precision;
  b->rsize = b->prec == DG_PREC_FP64 ? 8 : 4;
  std::map<std::tuple<int, int, int>, int> gidx;
  b->group_of.assign(n, -1);
  b->local_of.assign(n, -1);
  b->K_of.assign(n, 0);
  b->Np_of.assign(n, 0);
  b->bc_base.assign(n, 0);
  std::vector<char> phys_bytes, bc_bytes;
  std::vector<double> iparm;
  for (int i = 0; i < n; ++i) {
    if (params[i].precision != b->prec) {
      *out = b.release();
      return bfail(*out, DG_ERR_ARG, "instance " + std::to_string(i) + ": all instances need the same precision");
    }
    // validate and build through the single-instance setup (host only)
    dg_swe_ctx* c = nullptr;
    dg_status st = dg_swe_init(&meshes[i], orders[i], regs[i], &params[i], &c);
    if (st != DG_OK) {
      std::string m = c ? dg_swe_last_error(c) : "";
      dg_swe_destroy(c);
      *out = b.release();
      return bfail(*out, st, "instance " + std::to_string(i) + ": " + m);
    }
    b->dim.push_back(c->dim);
    b->order.push_back(c->p);
    b->reg.push_back(c->reg);
    b->prm.push_back(params[i]);
    // wet/dry instances form groups of their own: their stages take the
    // split volume pass (residual, then wetdry_stage_kernel)
    const int pos = params[i].positivity ? 1 : 0;
    auto key = std::make_tuple(c->dim, c->p, pos);
    if (!gidx.count(key)) {
      gidx[key] = (int)b->groups.size();
      b->groups.emplace_back();
      Group& g = b->groups.back();
      g.dim = c->dim;
      g.p = c->p;
      g.pos = pos != 0;
      g.ops = c->ops;
      g.drv = b->prec == DG_PREC_FP64 ? make_gdrv<double>(g.dim, g.p, g.ops, false)
                                      : make_gdrv<float>(g.dim, g.p, g.ops, b->prec == DG_PREC_FP32_TC);
    }
    const int gi = gidx[key];
    Group& g = b->groups[gi];
    b->group_of[i] = gi;
    b->local_of[i] = (int)g.members.size();
    b->K_of[i] = c->mesh.K;
    b->Np_of[i] = c->ops.Np;
    b->bc_base[i] = b->n_bc_total;
    b->n_bc_total += params[i].n_bc;
    g.members.push_back(i);
    g.ebase.push_back(g.K);
    g.fbase.push_back(g.F);
    // append this instance's mesh to the group (SoA over the group)
    const MeshData& m = c->mesh;
    const int64_t K = m.K, F = m.F, eb = g.K, fb = g.F;
    const int nf = c->dim + 1, Np = c->ops.Np;
    auto remap_nbr = [&](int32_t v) -> int32_t {
      return v >= 0 ? (int32_t)(v + eb) : (int32_t)(-1 - (b->bc_base[i] + (-1 - v)));
    };
    // element-face arrays: [nf][K] per instance -> [nf][Kg] (rebuilt below)
    g.K += K;
    g.F += F;
    g.inst.insert(g.inst.end(), (size_t)K, (int32_t)i);
    g.gid.push_back(i);
    // per-member SoA blocks, interleaved into group SoA arrays below
    g.geo.insert(g.geo.end(), m.geo.begin(), m.geo.end());            // [kGeoRows][K] blocks, interleaved later
    for (int64_t k = 0; k < nf * K; ++k) g.nbr.push_back(remap_nbr(m.nbr[k]));
    g.nbrf.insert(g.nbrf.end(), m.nbrf.begin(), m.nbrf.end());
    for (int64_t k = 0; k < nf * K; ++k) {
      uint32_t raw = (uint32_t)m.fid[k];
      uint32_t id = (raw & 0x7fffffffu) + (uint32_t)fb;
      g.fid.push_back((int32_t)(id | (raw & 0x80000000u)));
    }
    g.fn.insert(g.fn.end(), m.fn.begin(), m.fn.end());
    g.fsj.insert(g.fsj.end(), m.fsj.begin(), m.fsj.end());
    for (int64_t f = 0; f < F; ++f) {
      g.fe1.push_back((int32_t)(m.face_e1[f] + eb));
      g.fe2.push_back(remap_nbr(m.face_e2[f]));
    }
    g.ff1.insert(g.ff1.end(), m.face_f1.begin(), m.face_f1.end());
    g.ff2.insert(g.ff2.end(), m.face_f2.begin(), m.face_f2.end());
    g.face_n.insert(g.face_n.end(), m.face_n.begin(), m.face_n.end());
    g.face_sj.insert(g.face_sj.end(), m.face_sj.begin(), m.face_sj.end());
    if (c->has_bed) {
      if (!g.has_bed) {
        g.bed.assign((size_t)(eb)*Np, 0.0);
        g.has_bed = true;
      }
      g.bed.insert(g.bed.end(), c->bed.begin(), c->bed.end());
    } else if (g.has_bed) {
      g.bed.insert(g.bed.end(), (size_t)K * Np, 0.0);
    }
    g.src_blocks.push_back(c->has_bed ? c->src : std::vector<double>());
    g.gs_of.push_back(params[i].g * std::sin(params[i].alpha));
    // per-instance tables
    if (b->rsize == 8) push_phys<double>(params[i], regs[i], phys_bytes);
    else push_phys<float>(params[i], regs[i], phys_bytes);
    for (int k = 0; k < params[i].n_bc; ++k) {
      if (b->rsize == 8) push_bc<double>(params[i].bc[k], bc_bytes);
      else push_bc<float>(params[i].bc[k], bc_bytes);
    }
    const auto& pp = params[i];
    iparm.push_back(pp.g * std::cos(pp.alpha));
    iparm.push_back(pp.h_floor);
    iparm.push_back(pp.cfl);
    iparm.push_back((4.0 * max_viscous_eta(pp) + max_bingham_slope(regs[i], pp.sigma0, pp.gamma, pp.pap_m)) /
                    pp.rho);
    dg_swe_destroy(c);
  }
  // interleave per-member SoA blocks into group SoA arrays
  for (auto& g : b->groups) {
    const int nf = g.dim + 1, dim = g.dim;
    const int64_t Kg = g.K, Fg = g.F;
    std::vector<double> geo(kGeoRows * Kg), fn((size_t)nf * dim * Kg), fsj(nf * Kg), fnm((size_t)dim * Fg);
    std::vector<int32_t> nbr(nf * Kg), fid(nf * Kg);
    std::vector<int8_t> nbrf(nf * Kg);
    size_t pg = 0, pn = 0, pfn = 0, pfs = 0, pfnm = 0;
    for (size_t mi = 0; mi < g.members.size(); ++mi) {
      const int64_t eb = g.ebase[mi], fb = g.fbase[mi];
      const int64_t K = (mi + 1 < g.members.size() ? g.ebase[mi + 1] : Kg) - eb;
      const int64_t F = (mi + 1 < g.members.size() ? g.fbase[mi + 1] : Fg) - fb;
      for (int c = 0; c < kGeoRows; ++c)
        for (int64_t e = 0; e < K; ++e) geo[c * Kg + eb + e] = g.geo[pg + c * K + e];
      pg += kGeoRows * K;
      for (int f = 0; f < nf; ++f)
        for (int64_t e = 0; e < K; ++e) {
          nbr[f * Kg + eb + e] = g.nbr[pn + f * K + e];
          nbrf[f * Kg + eb + e] = g.nbrf[pn + f * K + e];
          fid[f * Kg + eb + e] = g.fid[pn + f * K + e];
          fsj[f * Kg + eb + e] = g.fsj[pfs + f * K + e];
          for (int d = 0; d < dim; ++d) fn[(f * dim + d) * Kg + eb + e] = g.fn[pfn + (f * dim + d) * K + e];
        }
      pn += nf * K;
      pfs += nf * K;
      pfn += (size_t)nf * dim * K;
      for (int d = 0; d < dim; ++d)
        for (int64_t f = 0; f < F; ++f) fnm[d * Fg + fb + f] = g.face_n[pfnm + d * F + f];
      pfnm += (size_t)dim * F;
    }
    if (g.has_bed) {  // source coefficients, [dim * Nq][Kg]
      const int rows = dim * g.ops.Nq;
      g.src.assign((size_t)rows * Kg, 0.0);
      for (size_t mi = 0; mi < g.members.size(); ++mi) {
        const int64_t eb = g.ebase[mi];
        const int64_t K = (mi + 1 < g.members.size() ? g.ebase[mi + 1] : Kg) - eb;
        const std::vector<double>& blk = g.src_blocks[mi];
        for (int r = 0; r < rows; ++r)
          for (int64_t e = 0; e < K; ++e)
            g.src[(size_t)r * Kg + eb + e] =
                blk.empty() ? (r < g.ops.Nq ? -g.gs_of[mi] : 0.0) : blk[(size_t)r * K + e];
      }
    }
    g.src_blocks.clear();
    g.geo.swap(geo);
    g.fn.swap(fn);
    g.fsj.swap(fsj);
    g.face_n.swap(fnm);
    g.nbr.swap(nbr);
    g.nbrf.swap(nbrf);
    g.fid.swap(fid);
    g.ebeg = g.ebase;
    g.ebeg.push_back(Kg);
    {  // persistent-step plan
      const int nfq = g.ops.Nfq, T = persist::kThreads;
      const size_t nm = g.members.size();
      g.p_etile.assign(nm + 1, 0);
      g.p_ftile.assign(nm + 1, 0);
      g.p_fbeg.assign(nm + 1, 0);
      for (size_t mi = 0; mi < nm; ++mi) {
        const int64_t Km = g.ebeg[mi + 1] - g.ebeg[mi];
        const int64_t Fm = (mi + 1 < nm ? g.fbase[mi + 1] : Fg) - g.fbase[mi];
        g.p_etile[mi + 1] = g.p_etile[mi] + (int32_t)((Km + T - 1) / T);
        g.p_ftile[mi + 1] = g.p_ftile[mi] + (int32_t)((Fm * nfq + T - 1) / T);
        g.p_fbeg[mi] = g.fbase[mi];
      }
      g.p_fbeg[nm] = Fg;
      const int ne = g.p_etile[nm], nfp = g.p_ftile[nm];
      int acc = 0;
      for (int ph = 0; ph < persist::kPhases; ++ph) {
        g.p_pstart[ph] = acc;
        acc += ph == 1 ? (int)nm : persist::face_phase(ph) ? nfp : ne;
      }
      g.p_pstart[persist::kPhases] = acc;
    }
    g.blk_e.clear();
    g.blk_gid.clear();
    g.mblk.clear();
    for (size_t mi = 0; mi < g.members.size(); ++mi) {
      g.mblk.push_back((int32_t)g.blk_gid.size());
      for (int64_t e = g.ebeg[mi]; e < g.ebeg[mi + 1]; e += 256) {
        g.blk_e.push_back(e);
        g.blk_gid.push_back(g.members[mi]);
      }
    }
    g.mblk.push_back((int32_t)g.blk_gid.size());
    g.blk_e.push_back(Kg);
    if (g.K > 0x7fffffff / 16 || g.F > 0x7fffffff / 8) {
      *out = b.release();
      return bfail(*out, DG_ERR_ARG, "group too large for 32-bit indexing");
    }
  }
  // workspace layout
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += a256(bytes);
    return r;
  };
  const size_t rs = b->rsize;
  for (auto& g : b->groups) {
    const int64_t K = g.K, F = g.F;
    const int nf = g.dim + 1, Np = g.ops.Np, nV = g.dim + 1, nE = g.dim * g.dim;
    g.off.geo = take(kGeoRows * K * rs);
    g.off.nbr = take(nf * K * 4);
    g.off.nbrf = take(nf * K);
    g.off.fid = take(nf * K * 4);
    g.off.fn = take((size_t)nf * g.dim * K * rs);
    g.off.fsj = take(nf * K * rs);
    g.off.fe1 = take(F * 4);
    g.off.fe2 = take(F * 4);
    g.off.ff1 = take(F);
    g.off.ff2 = take(F);
    g.off.fnrm = take((size_t)g.dim * F * rs);
    g.off.fsjf = take(F * rs);
    g.off.bed = take(g.has_bed ? K * Np * rs : 0);
    g.off.src = take(g.has_bed ? g.src.size() * rs : 0);
    g.off.inst = take(K * 4);
    g.off.ebeg = take(g.ebeg.size() * 8);
    g.off.gid = take(g.gid.size() * 4);
    for (int v = 0; v < 3; ++v) g.off.V[v] = take((size_t)nV * K * Np * rs);
    g.off.E = take((size_t)nE * K * Np * rs);
    g.off.wflux = take((size_t)nV * F * g.ops.Nfq * rs);
    g.off.wint = take(Np * 8);
    g.off.blk_e = take(g.blk_e.size() * 8);
    g.off.blk_gid = take(g.blk_gid.size() * 4);
    g.off.mblk = take(g.mblk.size() * 4);
    g.off.partial = take(g.blk_gid.size() * 8);
    g.off.p_etile = take(g.p_etile.size() * 4);
    g.off.p_ftile = take(g.p_ftile.size() * 4);
    g.off.p_fbeg = take(g.p_fbeg.size() * 8);
    g.off.p_tdt = take((size_t)g.p_etile.back() * 8);
    g.off.p_cnt = take((g.members.size() * persist::kPhases + 1) * 4);
    g.off.tcimg = take(b->prec == DG_PREC_FP32_TC ? tc::image_bytes(g.dim, g.p) : 0);
  }
  b->off_ptab = take(phys_bytes.size());
  b->off_bct = take(bc_bytes.size());
  b->off_sc = take((size_t)n * sizeof(DevScalars));
  b->off_iparm = take(iparm.size() * 8);
  b->ws_need = o;
  b->h_phys = std::move(phys_bytes);
  b->h_bc = std::move(bc_bytes);
  b->h_iparm = std::move(iparm);
  *out = b.release();
  return DG_OK;
}

size_t dg_batch_workspace_size(const dg_batch* b) { return b ? b->ws_need : 0; }

dg_status dg_batch_set_stream(dg_batch* b, void* s) {
  if (!b) return DG_ERR_ARG;
  b->stream = (cudaStream_t)s;
  return DG_OK;
}

dg_status dg_batch_set_workspace(dg_batch* b, void* ptr, size_t bytes) {
  if (!b) return DG_ERR_ARG;
  if (!ptr || bytes < b->ws_need) return bfail(b, DG_ERR_WORKSPACE, "workspace missing or smaller than dg_batch_workspace_size()");
  if (((uintptr_t)ptr & 255) != 0) return bfail(b, DG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  destroy_graphs(b);
  b->ws = (char*)ptr;
  cudaStream_t s = b->stream;
  auto up = [&](size_t off, const void* src, size_t n) -> cudaError_t {
    return n ? cudaMemcpyAsync(b->ws + off, src, n, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  auto upr = [&](size_t off, const std::vector<double>& v) -> cudaError_t {
    if (v.empty()) return cudaSuccess;
    if (b->rsize == 8) return up(off, v.data(), v.size() * 8);
    std::vector<float> f(v.begin(), v.end());
    cudaError_t e = up(off, f.data(), f.size() * 4);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };
  for (auto& g : b->groups) {
    BK(upr(g.off.geo, g.geo));
    BK(up(g.off.nbr, g.nbr.data(), g.nbr.size() * 4));
    BK(up(g.off.nbrf, g.nbrf.data(), g.nbrf.size()));
    BK(up(g.off.fid, g.fid.data(), g.fid.size() * 4));
    BK(upr(g.off.fn, g.fn));
    BK(upr(g.off.fsj, g.fsj));
    BK(up(g.off.fe1, g.fe1.data(), g.fe1.size() * 4));
    BK(up(g.off.fe2, g.fe2.data(), g.fe2.size() * 4));
    BK(up(g.off.ff1, g.ff1.data(), g.ff1.size()));
    BK(up(g.off.ff2, g.ff2.data(), g.ff2.size()));
    BK(upr(g.off.fnrm, g.face_n));
    BK(upr(g.off.fsjf, g.face_sj));
    if (g.has_bed) BK(upr(g.off.bed, g.bed));
    if (g.has_bed) BK(upr(g.off.src, g.src));
    BK(up(g.off.inst, g.inst.data(), g.inst.size() * 4));
    BK(up(g.off.ebeg, g.ebeg.data(), g.ebeg.size() * 8));
    BK(up(g.off.gid, g.gid.data(), g.gid.size() * 4));
    BK(up(g.off.wint, g.ops.wint.data(), g.ops.wint.size() * 8));
    BK(up(g.off.blk_e, g.blk_e.data(), g.blk_e.size() * 8));
    BK(up(g.off.blk_gid, g.blk_gid.data(), g.blk_gid.size() * 4));
    BK(up(g.off.mblk, g.mblk.data(), g.mblk.size() * 4));
    BK(up(g.off.p_etile, g.p_etile.data(), g.p_etile.size() * 4));
    BK(up(g.off.p_ftile, g.p_ftile.data(), g.p_ftile.size() * 4));
    BK(up(g.off.p_fbeg, g.p_fbeg.data(), g.p_fbeg.size() * 8));
    if (b->prec == DG_PREC_FP32_TC && tc::image_bytes(g.dim, g.p) > 0) {
      std::vector<float> img;
      tc::build_image(g.dim, g.p, g.ops, img);
      BK(up(g.off.tcimg, img.data(), img.size() * 4));
      BK(cudaStreamSynchronize(s));
    }
    BK(cudaMemsetAsync(b->ws + g.off.E, 0, (size_t)g.dim * g.dim * g.K * g.ops.Np * b->rsize, s));
    for (int v = 0; v < 3; ++v)
      BK(cudaMemsetAsync(b->ws + g.off.V[v], 0, (size_t)(g.dim + 1) * g.K * g.ops.Np * b->rsize, s));
  }
  BK(up(b->off_ptab, b->h_phys.data(), b->h_phys.size()));
  BK(up(b->off_bct, b->h_bc.data(), b->h_bc.size()));
  BK(up(b->off_iparm, b->h_iparm.data(), b->h_iparm.size() * 8));
  reset_scalars_array_kernel<<<(b->n + 127) / 128, 128, 0, s>>>(b->n, b->at<DevScalars>(b->off_sc));
  BK(cudaGetLastError());
  BK(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status dg_batch_set_state(dg_batch* b, int i, const double* V, int on_device) {
  dg_status st = check(b);
  if (st != DG_OK) return st;
  if (i < 0 || i >= b->n || !V) return bfail(b, DG_ERR_ARG, "bad instance index or null state");
  Group& g = b->groups[b->group_of[i]];
  const int mi = b->local_of[i];
  const int64_t K = b->K_of[i], Np = b->Np_of[i], eb = g.ebase[mi];
  const int nV = g.dim + 1;
  cudaStream_t s = b->stream;
  for (int f = 0; f < nV; ++f) {
    char* dst = b->ws + g.off.V[0] + ((size_t)f * g.K + eb) * Np * b->rsize;
    const double* src = V + (size_t)f * K * Np;
    if (b->rsize == 8) {
      BK(cudaMemcpyAsync(dst, src, K * Np * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    } else if (on_device) {
      conv<double, float>(src, dst, K * Np, s);
    } else {
      std::vector<float> h(src, src + K * Np);
      BK(cudaMemcpyAsync(dst, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s));
      BK(cudaStreamSynchronize(s));
    }
  }
  reset_scalars_array_kernel<<<1, 1, 0, s>>>(1, b->at<DevScalars>(b->off_sc) + i);
  g.drv->mass(b, g, mi, 1, 1, s);
  BK(cudaGetLastError());
  if (!on_device) BK(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status dg_batch_get_state(dg_batch* b, int i, double* V, int on_device) {
  dg_status st = check(b);
  if (st != DG_OK) return st;
  if (i < 0 || i >= b->n || !V) return bfail(b, DG_ERR_ARG, "bad instance index or null output");
  Group& g = b->groups[b->group_of[i]];
  const int mi = b->local_of[i];
  const int64_t K = b->K_of[i], Np = b->Np_of[i], eb = g.ebase[mi];
  const int nV = g.dim + 1;
  cudaStream_t s = b->stream;
  for (int f = 0; f < nV; ++f) {
    const char* src = b->ws + g.off.V[0] + ((size_t)f * g.K + eb) * Np * b->rsize;
    double* dst = V + (size_t)f * K * Np;
    if (b->rsize == 8) {
      BK(cudaMemcpyAsync(dst, src, K * Np * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    } else if (on_device) {
      conv<float, double>(src, dst, K * Np, s);
    } else {
      std::vector<float> h(K * Np);
      BK(cudaMemcpyAsync(h.data(), src, h.size() * 4, cudaMemcpyDeviceToHost, s));
      BK(cudaStreamSynchronize(s));
      for (size_t k = 0; k < h.size(); ++k) dst[k] = h[k];
    }
  }
  BK(cudaGetLastError());
  return read_stats(b, nullptr);
}

dg_status dg_batch_advance(dg_batch* b, int64_t n_steps) {
  dg_status st = check(b);
  if (st != DG_OK) return st;
  if (n_steps < 0) return bfail(b, DG_ERR_ARG, "n_steps < 0");
  if (n_steps == 0) return DG_OK;
  if (!b->priv) {
    BK(cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking));
    BK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    BK(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
  }
  if (!b->g1) {
    st = capture(b, 1, &b->g1);
    if (st != DG_OK) return st;
    st = capture(b, kGraphSteps, &b->gN);
    if (st != DG_OK) return st;
  }
  BK(cudaEventRecord(b->ev_fork, b->stream));
  BK(cudaStreamWaitEvent(b->priv, b->ev_fork, 0));
  int64_t left = n_steps;
  while (left >= kGraphSteps) {
    BK(cudaGraphLaunch(b->gN, b->priv));
    left -= kGraphSteps;
  }
  while (left-- > 0) BK(cudaGraphLaunch(b->g1, b->priv));
  BK(cudaEventRecord(b->ev_join, b->priv));
  BK(cudaStreamWaitEvent(b->stream, b->ev_join, 0));
  return DG_OK;
}

dg_status dg_batch_stats(dg_batch* b, dg_swe_stats* stats) {
  dg_status st = check(b);
  if (st != DG_OK) return st;
  for (auto& g : b->groups) g.drv->mass(b, g, 0, (int)g.members.size(), 0, b->stream);
  BK(cudaGetLastError());
  return read_stats(b, stats);
}

dg_status dg_batch_run(dg_batch* b, int64_t n_steps, dg_swe_stats* stats) {
  dg_status st = dg_batch_advance(b, n_steps);
  if (st != DG_OK) return st;
  return dg_batch_stats(b, stats);
}

dg_status dg_batch_autotune(dg_batch* b, int n_iter) {
  dg_status st = check(b);
  if (st != DG_OK) return st;
  if (n_iter < 1) return bfail(b, DG_ERR_ARG, "n_iter >= 1");
  static const int cand[8] = {32, 64, 128, 256, -32, -64, -128, -256};
  cudaStream_t s = b->stream;
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  // the step-size scalars are left as they are: the volume pass below writes
  // stage buffer 1 from buffer 0 and leaves the state untouched
  for (auto& g : b->groups) {
    g.drv->estep(b, g, 0, s);
    g.drv->face(b, g, 0, s);
    for (int k = 0; k < 3; ++k) {
      float best = 1e30f;
      int best_t = g.tile[k];
      // each kernel also tries its other form (negative block size): the
      // E-step's grid-stride form, the per-face flux form, the staged volume form
      const int ncand = 8;
      for (int ci = 0; ci < ncand; ++ci) {
        if (k == 2 && !g.drv->volume_ok(cand[ci])) continue;
        g.tile[k] = cand[ci];
        auto launch = [&]() {
          if (k == 0) g.drv->estep(b, g, 0, s);
          else if (k == 1) g.drv->face(b, g, 0, s);
          else g.drv->volume(b, g, 0, 1, 0.0, 1.0, s);
        };
        launch();  // warm-up
        BK(cudaEventRecord(e0, s));
        for (int it = 0; it < n_iter; ++it) launch();
        BK(cudaEventRecord(e1, s));
        BK(cudaEventSynchronize(e1));
        float ms = 0.f;
        BK(cudaEventElapsedTime(&ms, e0, e1));
        BK(cudaGetLastError());
        if (ms < best) {
          best = ms;
          best_t = cand[ci];
        }
      }
      g.tile[k] = best_t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  destroy_graphs(b);
  return DG_OK;
}

dg_status dg_batch_time_kernels(dg_batch* b, int n_iter, double* ms, int cap) {
  dg_status st = check(b);
  if (st != DG_OK) return st;
  if (n_iter < 1 || !ms || cap < 4 * (int)b->groups.size()) return bfail(b, DG_ERR_ARG, "need n_iter >= 1 and 4 slots per group");
  cudaStream_t s = b->stream;
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  std::vector<DevScalars> saved(b->n);
  BK(cudaMemcpyAsync(saved.data(), b->at<DevScalars>(b->off_sc), b->n * sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    Group& g = b->groups[gi];
    g.drv->estep(b, g, 0, s);
    g.drv->face(b, g, 0, s);
    for (int k = 0; k < 4; ++k) {
      BK(cudaEventRecord(e0, s));
      for (int it = 0; it < n_iter; ++it) {
        if (k == 0) g.drv->estep(b, g, 0, s);
        else if (k == 1) g.drv->face(b, g, 0, s);
        else if (k == 2) g.drv->volume(b, g, 0, 1, 0.0, 1.0, s);
        else g.drv->dt(b, g, s);
      }
      BK(cudaEventRecord(e1, s));
      BK(cudaEventSynchronize(e1));
      float t = 0.f;
      BK(cudaEventElapsedTime(&t, e0, e1));
      ms[4 * gi + k] = (double)t / n_iter;
    }
  }
  // the dt kernel advanced t and the step counters: restore them
  BK(cudaMemcpyAsync(b->at<DevScalars>(b->off_sc), saved.data(), b->n * sizeof(DevScalars), cudaMemcpyHostToDevice, s));
  BK(cudaStreamSynchronize(s));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BK(cudaGetLastError());
  return DG_OK;
}

dg_status dg_batch_tiles(const dg_batch* b, int32_t* out, int cap, int32_t* n_groups) {
  if (!b) return DG_ERR_ARG;
  if (n_groups) *n_groups = (int32_t)b->groups.size();
  if (out)
    for (size_t g = 0; g < b->groups.size(); ++g)
      for (int k = 0; k < 3; ++k)
        if ((int)(3 * g + k) < cap) out[3 * g + k] = b->groups[g].tile[k];
  return DG_OK;
}

dg_status dg_batch_set_tiles(dg_batch* b, const int32_t* tiles, int n) {
  if (!b || !tiles || n != 3 * (int)b->groups.size()) return bfail(b, DG_ERR_ARG, "need 3 block sizes per group");
  for (int i = 0; i < n; ++i) {
    const int v = tiles[i] < 0 ? -tiles[i] : tiles[i];
    if (v < 32 || v > 256 || v % 32)
      return bfail(b, DG_ERR_ARG,
                   "block sizes must be 32..256, multiples of 32 (negative E-step entry: grid-stride form; negative "
                   "face entry: per-face form; negative volume entry: staged form)");
    if (i % 3 == 2 && !b->groups[i / 3].drv->volume_ok(tiles[i]))
      return bfail(b, DG_ERR_ARG, "staged volume block size " + std::to_string(v) +
                                      " does not fit in shared memory for this group");
  }
  for (size_t g = 0; g < b->groups.size(); ++g)
    for (int k = 0; k < 3; ++k) b->groups[g].tile[k] = tiles[3 * g + k];
  destroy_graphs(b);
  return DG_OK;
}

dg_status dg_batch_info(const dg_batch* b, int64_t* elements, int64_t* dofs, int32_t* n_groups) {
  if (!b) return DG_ERR_ARG;
  int64_t K = 0, D = 0;
  for (int i = 0; i < b->n; ++i) {
    K += b->K_of[i];
    D += b->K_of[i] * b->Np_of[i] * (b->dim[i] + 1);
  }
  if (elements) *elements = K;
  if (dofs) *dofs = D;
  if (n_groups) *n_groups = (int32_t)b->groups.size();
  return DG_OK;
}

int32_t dg_batch_launches_per_step(const dg_batch* b) {
  if (!b) return 0;
  if (b->persistent) return (int32_t)b->groups.size();
  int32_t n = 0;
  for (const auto& g : b->groups) n += g.pos ? 14 : 11;  // wet/dry: a stage kernel after each volume pass
  return n;
}

dg_status dg_batch_set_persistent(dg_batch* b, int on) {
  if (!b) return DG_ERR_ARG;
  if (on && b->prec == DG_PREC_FP32_TC)
    return bfail(b, DG_ERR_UNSUPPORTED, "the persistent step runs the CUDA-core volume pass; use DG_PREC_FP32");
  if (on)
    for (const auto& g : b->groups)
      if (g.pos)
        return bfail(b, DG_ERR_UNSUPPORTED, "the persistent step has no wet/dry (positivity) stage");
  b->persistent = on != 0;
  destroy_graphs(b);
  return DG_OK;
}

const char* dg_batch_last_error(const dg_batch* b) { return b ? b->err.c_str() : "null batch"; }

void dg_batch_destroy(dg_batch* b) {
  if (!b) return;
  destroy_graphs(b);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->priv) cudaStreamDestroy(b->priv);
  delete b;
}

}  // extern "C"

// Tensor-core (tcgen05, TF32) form of the 2D volume kernel for p >= 2
// (precision mode DG_PREC_FP32_TC).
//
// The volume integrals of Eq. WeakForm51 on triangles contain three dense
// contractions per element that are batched over elements here as GEMMs
// with the elements of a tile as the M dimension (128 rows):
//   1. interpolation of the nodal fields to the volume quadrature points,
//      X_f[e][q] = sum_a V_f[e][a] l_a(q): A = nodal values (K = Np padded to
//      a multiple of 8), B = Vq (N = Nq padded to a multiple of 16); the bed
//      gives its reference gradients with B = Drq and B = Dsq;
//   2. the test-function contraction of the pointwise fluxes,
//      r_v[e][a] = sum_q (Wr[q][a] fr_v + Ws[q][a] fs_v - Wm[q][a] S_v)[e][q]:
//      A = pointwise values (K = points, 8 per chunk), B = weighted basis
//      derivatives and values (N = Np padded to 16);
//   3. the h-weighted mass matrix of the primitive-variable time term
//      (Appendix A, dU/dV): Mh[e][(a,b)] = sum_q w_q max(h, h_floor)[e][q]
//      l_a(q) l_b(q): A = w_q max(h_q, h_floor), B = products l_a l_b (N =
//      Np (Np + 1) / 2 padded to a multiple of 16).
// Each operand is split into TF32 high and low parts (hi = the nearest TF32
// value, lo = the nearest TF32 value of the exact remainder) and each
// product is accumulated in FP32 in tensor memory as hi*hi + hi*lo + lo*hi,
// so each operand keeps about 22 significant bits (FP32 has 24) instead of
// TF32's 11.
//
// Work split: a persistent grid with one 256-thread CTA per SM walks tiles of
// 128 elements.  Threads t and t + 128 serve element row t of the tile
// (tensor-memory lane t): each writes half of the operand rows and evaluates
// the pointwise physics at half of the quadrature points; the MMAs sum over
// both halves.  One thread issues the MMAs; tcgen05.commit arrives on an
// mbarrier that the CTA waits on (bounded: a wait longer than one second
// latches DG_ERR_TIMEOUT, waits for the copies and MMAs in flight, frees the
// tensor memory and ends the CTA).  The epilogue (face lift, the inverse mass
// matrix of dh/dt, the M_u dh/dt term, the Cholesky solve of Mh, the stage
// update and the optional depth limiter) runs on threads 0..127 in FP32 with
// the same formulas as the CUDA-core kernel.
//
// Shared-memory operands use the K-major canonical layout without swizzle:
// 8-row x 16-byte core matrices, consecutive along K (leading-byte offset
// 128 B) and then along the rows (stride-byte offset = 128 B x K / 4).
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>

#include "dg_kernels.cuh"

namespace dgswe {
namespace tc {

constexpr int kRows = 128;    // elements per tile (MMA M)
constexpr int kThreads = 256;  // two threads per element row
constexpr int kChunk = 8;      // quadrature points per contraction chunk (MMA K of tf32)
constexpr int kSlabs = 8;      // (field, term) slabs of one chunk: v0: r, s; v1, v2: r, s, m

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <int P>
struct Shape {
  using S = Sh<2, P>;
  static constexpr int NP = S::NP, NQ = S::NQ;
  static constexpr int KP = round_up(NP, 8);             // MMA-1 K
  static constexpr int NQP = round_up(NQ, 16);           // MMA-1 N, MMA-3 K
  static constexpr int NPAIR = NP * (NP + 1) / 2;        // lower triangle of Mh
  static constexpr int N3 = round_up(NPAIR, 16);         // MMA-3 N
  static constexpr int NCH = (NQ + kChunk - 1) / kChunk;  // contraction chunks
  static constexpr int NFLD = 8;                         // h, u1, u2, E0..E3, bed
  static constexpr int ND1 = 9;                          // interpolation outputs: 7 fields, dH/dr, dH/ds
  // tensor-memory columns
  static constexpr int D1 = 0;                           // 9 blocks of NQP
  static constexpr int D2 = ND1 * NQP;                   // 3 blocks of 16
  static constexpr int D3 = D2 + 48;                     // N3
  static constexpr int COLS_USED = D3 + N3;
  static constexpr int TMEM_COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                                   : COLS_USED <= 256 ? 256 : 512;
  // shared memory (bytes)
  static constexpr int A1_BYTES = NFLD * 2 * kRows * KP * 4;
  static constexpr int A2_BUF = kSlabs * 2 * kRows * kChunk * 4;
  static constexpr int A_BYTES = A1_BYTES > 2 * A2_BUF ? A1_BYTES : 2 * A2_BUF;
  static constexpr int A3_BYTES = 2 * kRows * NQP * 4;
  static constexpr int B1_ONE = NQP * KP * 4;            // one of Vq, Drq, Dsq (hi or lo)
  static constexpr int B1_BYTES = 3 * 2 * B1_ONE;
  static constexpr int B2_ONE = 16 * kChunk * 4;         // one (term, chunk) slab (hi or lo)
  static constexpr int B2_BYTES = NCH * 3 * 2 * B2_ONE;
  static constexpr int B3_BYTES = 2 * N3 * NQP * 4;
  static constexpr int B_BYTES = B1_BYTES + B2_BYTES + B3_BYTES;  // the global operand image
  static constexpr int OFF_A3 = A_BYTES;
  static constexpr int OFF_B = OFF_A3 + A3_BYTES;
  static constexpr int OFF_BAR = OFF_B + B_BYTES;
  static constexpr int SMEM = OFF_BAR + 64;
  static_assert(TMEM_COLS >= COLS_USED, "tensor memory");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(B_BYTES % 16 == 0, "operand image");
};

// float index of element (row r, column k) in a K-major no-swizzle operand
// with kg = K / 4 core matrices per 8-row group
__host__ __device__ __forceinline__ int cm_index(int r, int k, int kg) {
  return ((r >> 3) * kg + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

// Nearest TF32 value of x (ties away from zero): the high part of the split.
// The low part x - hi is exact in FP32 and is itself rounded to TF32 the same
// way, so each operand carries about 22 significant bits.
__host__ __device__ __forceinline__ float tf32_rn(float x) {
#ifdef __CUDA_ARCH__
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;  // finite: round the magnitude
  float y;
  std::memcpy(&y, &u, 4);
  return y;
#endif
}

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture; no swizzle, base offset 0
  return d;
}
// kind::tf32 instruction descriptor: D in FP32, A and B in TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N]);
template <>
__device__ __forceinline__ void tmem_ld<4>(uint32_t ta, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t ta, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t ta, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ host: operand image

// B operands in the shared-memory layout, high then low part of each:
// B1 = Vq, Drq, Dsq as (NQP rows x KP), B2 = per chunk and term
// (16 rows = nodes x 8 points) of Wr, Ws, -Wm, B3 = (N3 rows = node pairs x
// NQP points) of l_a l_b.  Padding is zero.
template <int P>
void build_operand_image(const RefOps& o, std::vector<float>& img) {
  using T = Shape<P>;
  constexpr int NP = T::NP, NQ = T::NQ;
  img.assign(T::B_BYTES / 4, 0.0f);
  auto put = [&](size_t base_hi, size_t one, int r, int k, int kg, double v) {
    const float f = (float)v, hi = tf32_rn(f), lo = tf32_rn(f - hi);
    img[base_hi + cm_index(r, k, kg)] = hi;
    img[base_hi + one + cm_index(r, k, kg)] = lo;
  };
  const size_t b1 = 0, b1one = T::B1_ONE / 4;
  for (int sel = 0; sel < 3; ++sel)
    for (int q = 0; q < NQ; ++q)
      for (int a = 0; a < NP; ++a) {
        const double v = sel == 0 ? o.Vq[q * NP + a] : sel == 1 ? o.Drq[q * NP + a] : o.Dsq[q * NP + a];
        put(b1 + sel * 2 * b1one, b1one, q, a, T::KP / 4, v);
      }
  const size_t b2 = T::B1_BYTES / 4, b2one = T::B2_ONE / 4;
  for (int c = 0; c < T::NCH; ++c)
    for (int t = 0; t < 3; ++t)
      for (int k = 0; k < kChunk; ++k) {
        const int q = c * kChunk + k;
        if (q >= NQ) continue;
        for (int a = 0; a < NP; ++a) {
          const double w = o.wq[q];
          const double v = t == 0 ? w * o.Drq[q * NP + a] : t == 1 ? w * o.Dsq[q * NP + a] : -w * o.Vq[q * NP + a];
          put(b2 + (size_t)(c * 3 + t) * 2 * b2one, b2one, a, k, kChunk / 4, v);
        }
      }
  const size_t b3 = (T::B1_BYTES + T::B2_BYTES) / 4, b3one = (size_t)T::N3 * T::NQP;
  for (int a = 0; a < NP; ++a)
    for (int b = 0; b <= a; ++b)
      for (int q = 0; q < NQ; ++q)
        put(b3, b3one, a * (a + 1) / 2 + b, q, T::NQP / 4, o.Vq[q * NP + a] * o.Vq[q * NP + b]);
}

// ------------------------------------------------------------------ device helpers

// Writes the hi and lo parts of 4 consecutive K values of row r.
__device__ __forceinline__ void put4(float* hi_base, float* lo_base, int r, int k, int kg, const float (&x)[4]) {
  float4 h, l;
  h.x = tf32_rn(x[0]);
  h.y = tf32_rn(x[1]);
  h.z = tf32_rn(x[2]);
  h.w = tf32_rn(x[3]);
  l.x = tf32_rn(x[0] - h.x);
  l.y = tf32_rn(x[1] - h.y);
  l.z = tf32_rn(x[2] - h.z);
  l.w = tf32_rn(x[3] - h.w);
  const int i = cm_index(r, k, kg);
  *reinterpret_cast<float4*>(hi_base + i) = h;
  *reinterpret_cast<float4*>(lo_base + i) = l;
}

// Bounded wait on an mbarrier phase, uniform over the CTA: false (for every
// thread) when any thread gave up.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity) {
  const bool ok = mbar_wait_bounded(bar, parity, kStageWaitNs);
  return __syncthreads_and(ok) != 0;
}

template <int P, bool BATCH>
__global__ void __launch_bounds__(kThreads, 1)
    volume_tc_kernel(int K, int F, const float* __restrict__ Vin, const float* V0, float* out,
                     const float* __restrict__ E, const float* __restrict__ bed, const float* __restrict__ geo,
                     const int32_t* __restrict__ fid, const float* __restrict__ wflux,
                     const VolOps<2, P, float> ops, const float* __restrict__ bimg, const Phys<float> ph0,
                     const Phys<float>* __restrict__ ptab, const int32_t* __restrict__ inst, int mode, float c0,
                     float c1, DevScalars* sc) {
  using T = Shape<P>;
  using S = Sh<2, P>;
  constexpr int NP = S::NP, NQ = S::NQ, NF = S::NF, NFP = S::NFP, NFQ = S::NFQ, NV = S::NV;
  constexpr int KP = T::KP, NQP = T::NQP;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* sA = reinterpret_cast<float*>(smem);
  float* sA3 = reinterpret_cast<float*>(smem + T::OFF_A3);
  float* sB = reinterpret_cast<float*>(smem + T::OFF_B);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + T::OFF_BAR);  // 0: MMA 1, 1-2: A2 buffers, 3: MMA 3
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + T::OFF_BAR + 48);
  const int tid = threadIdx.x;
  const int row = tid & (kRows - 1);
  const int half = tid >> 7;
  const int warp = tid >> 5;
  const size_t KN = (size_t)K * NP;
  const int ntiles = (K + kRows - 1) / kRows;
  const bool has_bed = bed != nullptr;

  // operand image -> shared memory (once per CTA)
  for (int i = tid; i < T::B_BYTES / 16; i += kThreads)
    reinterpret_cast<float4*>(sB)[i] = reinterpret_cast<const float4*>(bimg)[i];
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
    mbar_init_fence();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"((uint32_t)T::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  const uint32_t sA_addr = smem_addr(sA), sA3_addr = smem_addr(sA3), sB_addr = smem_addr(sB);
  const uint32_t b2_addr = sB_addr + T::B1_BYTES, b3_addr = b2_addr + T::B2_BYTES;
  uint32_t par = 0u;  // phase parity per barrier (bit i)
  bool failed = false;

  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int e = tile * kRows + row;
    const bool valid = e < K;
    const int ins = BATCH ? (valid ? inst[e] : 0) : 0;
    const Phys<float> ph = BATCH ? ptab[ins] : ph0;

    // ---- A1: nodal values of 4 fields per thread (half 0: h, u1, u2, E0; half 1: E1, E2, E3, bed)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = half * 4 + j;
      const float* src = f < NV ? Vin + f * KN : f < 7 ? E + (f - NV) * KN : bed;
      float x[KP];
#pragma unroll
      for (int a = 0; a < KP; ++a) x[a] = (valid && src && a < NP) ? src[(size_t)e * NP + a] : 0.0f;
      float* hi = sA + (size_t)f * 2 * kRows * KP;
      float* lo = hi + kRows * KP;
#pragma unroll
      for (int k4 = 0; k4 < KP / 4; ++k4) {
        const float y[4] = {x[4 * k4], x[4 * k4 + 1], x[4 * k4 + 2], x[4 * k4 + 3]};
        put4(hi, lo, row, 4 * k4, KP / 4, y);
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      constexpr uint32_t id1 = idesc_tf32(kRows, NQP);
#pragma unroll 1
      for (int d = 0; d < (has_bed ? T::ND1 : 7); ++d) {
        const int f = d < 7 ? d : 7;
        const int bsel = d < 7 ? 0 : d - 6;
        const uint32_t a_hi = sA_addr + (uint32_t)f * 2 * kRows * KP * 4, a_lo = a_hi + kRows * KP * 4;
        const uint32_t b_hi = sB_addr + (uint32_t)bsel * 2 * T::B1_ONE, b_lo = b_hi + T::B1_ONE;
        const uint32_t dcol = tmem + (uint32_t)(T::D1 + d * NQP);
        const uint32_t sbo = (KP / 4) * 128;
#pragma unroll 1
        for (int j = 0; j < KP / 8; ++j) {
          const uint32_t o = (uint32_t)j * 256;
          mma_tf32(dcol, sdesc(a_hi + o, 128, sbo), sdesc(b_hi + o, 128, sbo), id1, j > 0 ? 1u : 0u);
          mma_tf32(dcol, sdesc(a_hi + o, 128, sbo), sdesc(b_lo + o, 128, sbo), id1, 1u);
          mma_tf32(dcol, sdesc(a_lo + o, 128, sbo), sdesc(b_hi + o, 128, sbo), id1, 1u);
        }
      }
      mma_commit(&bar[0]);
    }
    if (!cta_wait(&bar[0], par & 1u)) {
      failed = true;
      break;
    }
    par ^= 1u;
    fence_after();

    // ---- pointwise physics, chunk by chunk (8 points; this thread: 4 of them)
    float G00 = 0.f, G01 = 0.f, G10 = 0.f, G11 = 0.f;
    if (valid) {
      G00 = geo[e];
      G01 = geo[K + e];
      G10 = geo[2 * K + e];
      G11 = geo[3 * K + e];
    }
#pragma unroll 1
    for (int c = 0; c < T::NCH; ++c) {
      const int buf = c & 1;
      if (c >= 2) {  // the buffer's previous MMAs must be done before it is rewritten
        if (!cta_wait(&bar[1 + buf], (par >> (1 + buf)) & 1u)) {
          failed = true;
          break;
        }
        par ^= 1u << (1 + buf);
      }
      const int q0 = c * kChunk + half * 4;
      float X[T::ND1][4];
#pragma unroll
      for (int d = 0; d < T::ND1; ++d) tmem_ld<4>(lane_base + (uint32_t)(T::D1 + d * NQP + q0), X[d]);
      tmem_wait_ld();
      float slab[kSlabs][4], wh[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int q = q0 + i;
        if (!valid || q >= NQ) {
#pragma unroll
          for (int s = 0; s < kSlabs; ++s) slab[s][i] = 0.0f;
          wh[i] = 0.0f;
          continue;
        }
        const float h = X[0][i];
        const float u[2] = {X[1][i], X[2][i]};
        const float Eq[4] = {X[3][i], X[4][i], X[5][i], X[6][i]};
        const float Hr = has_bed ? X[7][i] : 0.0f, Hs = has_bed ? X[8][i] : 0.0f;
        const float hr = h * ph.rho_inv;
        float sig[2][2];
        stress<2, float>(Eq, ph, sig);
        float fx[2][NV];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          fx[a][0] = -h * u[a];
#pragma unroll
          for (int j = 0; j < 2; ++j) fx[a][1 + j] = -h * u[a] * u[j] + hr * sig[j][a];
          fx[a][1 + a] -= 0.5f * ph.gc * h * h;
        }
        const float dH0 = G00 * Hr + G10 * Hs, dH1 = G01 * Hr + G11 * Hs;
        float Sv[NV];
        Sv[0] = 0.0f;
        Sv[1] = -ph.gc * h * dH0 - ph.gs * h;
        Sv[2] = -ph.gc * h * dH1;
        float fr[NV], fs[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          fr[v] = G00 * fx[0][v] + G01 * fx[1][v];
          fs[v] = G10 * fx[0][v] + G11 * fx[1][v];
        }
        // slabs: (v0, r), (v0, s), (v1, r), (v1, s), (v1, m), (v2, r), (v2, s), (v2, m)
        slab[0][i] = fr[0];
        slab[1][i] = fs[0];
        slab[2][i] = fr[1];
        slab[3][i] = fs[1];
        slab[4][i] = Sv[1];
        slab[5][i] = fr[2];
        slab[6][i] = fs[2];
        slab[7][i] = Sv[2];
        wh[i] = ops.wq[q] * fmaxf(h, ph.h_floor);
      }
      float* A2 = sA + (size_t)buf * (T::A2_BUF / 4);
#pragma unroll
      for (int s = 0; s < kSlabs; ++s) {
        float* hi = A2 + (size_t)s * 2 * kRows * kChunk;
        put4(hi, hi + kRows * kChunk, row, half * 4, kChunk / 4, slab[s]);
      }
      put4(sA3, sA3 + kRows * NQP, row, q0, NQP / 4, wh);
      fence_async_smem();
      fence_before();
      __syncthreads();
      if (tid == 0) {
        fence_after();
        constexpr uint32_t id2 = idesc_tf32(kRows, 16);
        const uint32_t a2 = sA_addr + (uint32_t)buf * T::A2_BUF;
#pragma unroll 1
        for (int s = 0; s < kSlabs; ++s) {
          const int v = s < 2 ? 0 : s < 5 ? 1 : 2;
          const int t = s < 2 ? s : s < 5 ? s - 2 : s - 5;
          const uint32_t a_hi = a2 + (uint32_t)s * 2 * kRows * kChunk * 4, a_lo = a_hi + kRows * kChunk * 4;
          const uint32_t b_hi = b2_addr + (uint32_t)(c * 3 + t) * 2 * T::B2_ONE, b_lo = b_hi + T::B2_ONE;
          const uint32_t dcol = tmem + (uint32_t)(T::D2 + 16 * v);
          const uint32_t first = (c == 0 && t == 0) ? 0u : 1u;
          mma_tf32(dcol, sdesc(a_hi, 128, 256), sdesc(b_hi, 128, 256), id2, first);
          mma_tf32(dcol, sdesc(a_hi, 128, 256), sdesc(b_lo, 128, 256), id2, 1u);
          mma_tf32(dcol, sdesc(a_lo, 128, 256), sdesc(b_hi, 128, 256), id2, 1u);
        }
        mma_commit(&bar[1 + buf]);
      }
    }
    if (failed) break;
    // ---- MMA 3: Mh = (w_q max(h, floor)) x (l_a l_b)
    if (tid == 0) {
      fence_after();
      constexpr uint32_t id3 = idesc_tf32(kRows, T::N3);
      const uint32_t sbo = (NQP / 4) * 128;
      const uint32_t a_hi = sA3_addr, a_lo = sA3_addr + kRows * NQP * 4;
      const uint32_t b_hi = b3_addr, b_lo = b3_addr + T::N3 * NQP * 4;
      const uint32_t dcol = tmem + (uint32_t)T::D3;
#pragma unroll 1
      for (int j = 0; j < NQP / 8; ++j) {
        const uint32_t o = (uint32_t)j * 256;
        mma_tf32(dcol, sdesc(a_hi + o, 128, sbo), sdesc(b_hi + o, 128, sbo), id3, j > 0 ? 1u : 0u);
        mma_tf32(dcol, sdesc(a_hi + o, 128, sbo), sdesc(b_lo + o, 128, sbo), id3, 1u);
        mma_tf32(dcol, sdesc(a_lo + o, 128, sbo), sdesc(b_hi + o, 128, sbo), id3, 1u);
      }
      mma_commit(&bar[3]);
    }
    // the commit of MMA 3 covers every earlier MMA of this tile; the A2
    // buffers' own barriers still complete a phase each, which is consumed
    // here so that their parities stay in step
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int uses = (T::NCH - b + 1) / 2;  // chunks that used buffer b
      const int waited = uses > 1 ? uses - 1 : 0;
      if (uses - waited > 0) {
        if (!cta_wait(&bar[1 + b], (par >> (1 + b)) & 1u)) failed = true;
        par ^= 1u << (1 + b);
      }
    }
    if (failed) break;
    if (!cta_wait(&bar[3], (par >> 3) & 1u)) {
      failed = true;
      break;
    }
    par ^= 1u << 3;
    fence_after();

    // ---- epilogue on threads 0..127 (warps 0-3: their tensor-memory lanes are the tile's rows)
    if (half == 0) {
      float d2[NV][16];
#pragma unroll
      for (int v = 0; v < NV; ++v) tmem_ld<16>(lane_base + (uint32_t)(T::D2 + 16 * v), d2[v]);
      float d3[T::N3];
#pragma unroll
      for (int j = 0; j < T::N3 / 16; ++j) {
        float t16[16];
        tmem_ld<16>(lane_base + (uint32_t)(T::D3 + 16 * j), t16);
#pragma unroll
        for (int i = 0; i < 16; ++i) d3[16 * j + i] = t16[i];
      }
      float uqs[2][NQP];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int c16 = 0; c16 < NQP / 16; ++c16) {
          float t16[16];
          tmem_ld<16>(lane_base + (uint32_t)(T::D1 + (1 + j) * NQP + 16 * c16), t16);
#pragma unroll
          for (int i = 0; i < 16; ++i) uqs[j][16 * c16 + i] = t16[i];
        }
      tmem_wait_ld();
      if (valid) {
        const size_t eo = (size_t)e * NP;
        const float J = geo[4 * K + e];
        float r[NV][NP];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int a = 0; a < NP; ++a) r[v][a] = d2[v][a] * J;
        // face terms <N^-, F_bar.n - Q_bar.n> (weights and sJ folded into wflux)
        const size_t FQ = (size_t)F * NFQ;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const uint32_t raw = (uint32_t)fid[f * K + e];
          const bool own = (raw & 0x80000000u) == 0;
          const size_t base = (size_t)(raw & 0x7fffffffu) * NFQ;
          float fv[NV][NFQ];
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int m = 0; m < NFQ; ++m) {
              const float x = wflux[v * FQ + base + (own ? m : NFQ - 1 - m)];
              fv[v][m] = own ? x : -x;
            }
#pragma unroll
          for (int k = 0; k < NFP; ++k) {
            const int a = face_node(2, P, f, k);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              float acc = 0.0f;
#pragma unroll
              for (int m = 0; m < NFQ; ++m) acc += ops.LfT[k * NFQ + m] * fv[v][m];
              r[v][a] += acc;
            }
          }
        }
        if (mode == 2) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int a = 0; a < NP; ++a) out[v * KN + eo + a] = r[v][a];
        } else {
          // M dh/dt = -r_h ; M_h du/dt = -r_u - M_u dh/dt (Appendix A, dU/dV)
          const float Jinv = geo[6 * K + e];
          float dV[NV][NP];
#pragma unroll
          for (int a = 0; a < NP; ++a) {
            float acc = 0.0f;
#pragma unroll
            for (int b = 0; b < NP; ++b) acc += ops.Minv[a * NP + b] * r[0][b];
            dV[0][a] = -acc * Jinv;
          }
          float rhs[2][NP];
#pragma unroll
          for (int a = 0; a < NP; ++a)
#pragma unroll
            for (int j = 0; j < 2; ++j) rhs[j][a] = -r[1 + j][a] * Jinv;
#pragma unroll 1
          for (int q = 0; q < NQ; ++q) {
            float hdq = 0.0f;
#pragma unroll
            for (int a = 0; a < NP; ++a) hdq += ops.Vq[q * NP + a] * dV[0][a];
            const float wd = ops.wq[q] * hdq;
#pragma unroll
            for (int a = 0; a < NP; ++a) {
              const float la = ops.Vq[q * NP + a];
#pragma unroll
              for (int j = 0; j < 2; ++j) rhs[j][a] -= wd * uqs[j][q] * la;
            }
          }
          // near-dry element (smallest nodal depth below h_dry): the whole
          // mass solve again in FP64 from the nodal values, as in the
          // CUDA-core kernel (mass_solve_dispatch)
          float hmin = Vin[eo];
#pragma unroll
          for (int a = 1; a < NP; ++a) hmin = fminf(hmin, Vin[eo + a]);
          const bool dry = hmin < ph.h_dry;
          if (dry) {
            float Vn[NV][NP];
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
              for (int a = 0; a < NP; ++a) Vn[v][a] = Vin[v * KN + eo + a];
            mass_solve_dry<2, P>(Vn, r, ops, ph.h_floor, Jinv, dV);
          }
          float Mh[NP][NP];
#pragma unroll
          for (int a = 0; a < NP; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) Mh[a][b] = d3[a * (a + 1) / 2 + b];
          float dinv[NP];
          if (!dry) {
#pragma unroll
          for (int a = 0; a < NP; ++a) {
#pragma unroll
            for (int b = 0; b < a; ++b) {
              float s = Mh[a][b];
#pragma unroll
              for (int cc = 0; cc < b; ++cc) s -= Mh[a][cc] * Mh[b][cc];
              Mh[a][b] = s * dinv[b];
            }
            float dd = Mh[a][a];
#pragma unroll
            for (int cc = 0; cc < a; ++cc) dd -= Mh[a][cc] * Mh[a][cc];
            dinv[a] = dg_rsqrt<float>(dd);
          }
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            float y[NP];
#pragma unroll
            for (int a = 0; a < NP; ++a) {
              float s = rhs[j][a];
#pragma unroll
              for (int cc = 0; cc < a; ++cc) s -= Mh[a][cc] * y[cc];
              y[a] = s * dinv[a];
            }
#pragma unroll
            for (int a = NP - 1; a >= 0; --a) {
              float s = y[a];
#pragma unroll
              for (int cc = a + 1; cc < NP; ++cc) s -= Mh[cc][a] * dV[1 + j][cc];
              dV[1 + j][a] = s * dinv[a];
            }
          }
          }
          if (mode == 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
              for (int a = 0; a < NP; ++a) out[v * KN + eo + a] = dV[v][a];
          } else {
            const float dt = (float)sc[ins].dt;
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
              for (int a = 0; a < NP; ++a) {
                float y = c1 * (Vin[v * KN + eo + a] + dt * dV[v][a]);
                if (c0 != 0.0f) y += c0 * V0[v * KN + eo + a];
                dV[v][a] = y;
              }
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
              for (int a = 0; a < NP; ++a) out[v * KN + eo + a] = dV[v][a];
          }
        }
      }
      fence_before();
    }
    __syncthreads();  // tensor memory and the A regions are free for the next tile
    fence_after();
  }

  if (failed) {
    if (tid == 0) {
      const int e0 = min((int)blockIdx.x * kRows, K - 1);
      atomicExch(&sc[BATCH ? inst[e0] : 0].status, (int)DG_ERR_TIMEOUT);
      // let MMAs in flight finish before the tensor memory is released
      for (int b = 0; b < 4; ++b) mbar_wait_bounded(&bar[b], (par >> b) & 1u, kStageWaitNs);
    }
    __syncthreads();
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)T::TMEM_COLS));
}

// ------------------------------------------------------------------ host: launch

// Bytes of the operand image of the (dim, p) tensor-core form; 0 where there
// is none (1D, p = 1: the contractions are too small for the tensor cores).
inline size_t image_bytes(int dim, int p) {
  if (dim != 2) return 0;
  if (p == 2) return Shape<2>::B_BYTES;
  if (p == 3) return Shape<3>::B_BYTES;
  return 0;
}
inline void build_image(int dim, int p, const RefOps& o, std::vector<float>& img) {
  img.clear();
  if (dim == 2 && p == 2) build_operand_image<2>(o, img);
  if (dim == 2 && p == 3) build_operand_image<3>(o, img);
}

// Persistent grid: one CTA per SM (the kernel holds 512 or 256 tensor-memory
// columns and most of the shared memory), never more CTAs than tiles.
template <int P, bool BATCH>
struct Launcher {
  int n_sm = 0;
  Launcher() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      n_sm = v;
    cudaFuncSetAttribute(volume_tc_kernel<P, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, Shape<P>::SMEM);
    cudaGetLastError();
  }
  void operator()(int K, int F, const float* Vin, const float* V0, float* out, const float* E, const float* bed,
                  const float* geo, const int32_t* fid, const float* wflux, const VolOps<2, P, float>& ops,
                  const float* bimg, const Phys<float>& ph, const Phys<float>* ptab, const int32_t* inst, int mode,
                  float c0, float c1, DevScalars* sc, cudaStream_t s) const {
    const int ntiles = (K + kRows - 1) / kRows;
    const int grid = std::min(ntiles, n_sm > 0 ? n_sm : 1);
    volume_tc_kernel<P, BATCH><<<grid, kThreads, Shape<P>::SMEM, s>>>(K, F, Vin, V0, out, E, bed, geo, fid, wflux,
                                                                       ops, bimg, ph, ptab, inst, mode, c0, c1, sc);
  }
};

}  // namespace tc
}  // namespace dgswe

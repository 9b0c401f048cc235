// Hot-path kernels of the aRDG right-hand side, templated on the order N and the arithmetic
// type T.  Included by one translation unit per (order, precision), which defines RDG_TAB, a
// __constant__ array holding that order's reference matrices Dr, Ds, Wr, Ws (Np x Np each)
// and LIFT (Np x 3 Nfp), in that order.  With N a template parameter every loop below is
// fully unrolled, so each matrix entry is an immediate constant-bank operand of an FMA.
//
//  edge_flux_kernel   (one thread per edge)  flux_e = W_e [u_k1; u_k2]
//      W_e = J_f ( -D~ (kappa_R DR + kappa_S DS) A+ blkdiag(P_1, P_2) + upwind trace ),
//      the per-edge operator of Sec. 4 / Algorithm aRDG built at setup; streamed from HBM
//      in 16-byte words laid out [tile of 32 edges][word][lane] so a warp reads 512
//      contiguous bytes per load.
//  elem_kernel        (one thread per element)  volume term M^{-1} S^T . F with
//      F = v u - D grad u, minus sum_f (1/J) LIFT_f (J_f F*.n)_f, plus sources, fused with
//      the SSP-RK3 stage combination (Eq. NDG_diffusion_once_matrixForm_Fullyreference).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace rdg {
namespace dev {

__device__ __forceinline__ double tau_of(int kind, double omega, double t) {
  return kind == RDG_TAU_COS ? cos(omega * t) : (kind == RDG_TAU_SIN ? sin(omega * t) : 1.0);
}

__device__ __forceinline__ double stage_time(const TimeArg& ta) {
  if (ta.ts) return ta.ts->t0 + ((double)ta.ts->n + ta.off) * ta.dt;
  return ta.t0 + ta.off * ta.dt;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
  __device__ static float get(const float4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
  __device__ static double get(const double2& v, int c) { return c == 0 ? v.x : v.y; }
};

// streaming (evict-first) 16-byte load for data read once per kernel
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }

// ---------------------------------------------------------------------------------------
// mbarrier / bulk-copy (TMA unit) helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Orders this thread's generic-proxy shared-memory reads before later async-proxy (bulk
// copy) writes: a slot read with ordinary loads must not be refilled by the copy engine
// before those loads have read it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of an mbarrier, giving up after about two seconds.
constexpr uint64_t kWaitLimitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}
// L2 policy for data streamed once per kernel: evict first, so the operator stream does not
// push the (L2-resident) state, flux and index arrays out of L2
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void report(int* err, int bit) {
  if (err) atomicOr(err, bit);
}

// Geometry of the streamed operator pipeline for one (T, N); VOL adds the volume warps.
// Each edge warp owns DEPTH shared-memory slots and keeps DEPTH operator tiles in flight.
template <typename T, int N, bool VOL = false>
struct EdgePipe {
  static constexpr int NP = np_of(N), NFP = nfp_of(N), NW = NFP * 2 * NP;
  static constexpr int VW = 16 / (int)sizeof(T);
  static constexpr int QW = (NW + VW - 1) / VW;          // 16-byte words per edge
  static constexpr int TILE_BYTES = QW * kTile * 16;     // one warp tile of W (contiguous)
  static constexpr int NV = VOL ? (N <= 4 ? 4 : 2) : 0;  // volume warps
  static constexpr int VOL_BYTES = NV * kTile * NP * (int)sizeof(T);
  static constexpr int BAR_BYTES = 1024;
  static constexpr int BUDGET = 226 * 1024 - BAR_BYTES - VOL_BYTES;
  static constexpr int SLOTS_RAW = BUDGET / TILE_BYTES;
  static constexpr int DEPTH = SLOTS_RAW >= 16 ? 3 : 2;  // tiles in flight per edge warp
  static constexpr int NE_RAW = SLOTS_RAW / DEPTH;
  static constexpr int NE = NE_RAW > 12 ? 12 : (NE_RAW < 1 ? 1 : NE_RAW);  // edge warps
  static constexpr int SLOTS = NE * DEPTH;
  static constexpr int THREADS = 32 * (NE + NV);
  static constexpr int SMEM = BAR_BYTES + SLOTS * TILE_BYTES + VOL_BYTES;
  static_assert(SLOTS * 8 + 16 <= BAR_BYTES, "barrier area too small");
};

// Volume term of one element: M^{-1} S^T . F with F = v u - D grad u, written with the
// metric-folded coefficients F_r = a_r u - (g_rr u_r + g_rs u_s), F_s = a_s u - (g_rs u_r +
// g_ss u_s), vol = Wr F_r + Ws F_s (Wr = M^{-1} Dr^T M, Ws = M^{-1} Ds^T M).
template <typename T, int N>
__device__ __forceinline__ void volume_row(const T (&u)[np_of(N)], T ar, T as, T grr, T grs, T gss,
                                           T (&vol)[np_of(N)]) {
  constexpr int NP = np_of(N);
  constexpr int ODR = 0, ODS = NP * NP, OWR = 2 * NP * NP, OWS = 3 * NP * NP;
  T fr[NP], fs[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    T ur = T(0), us = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      ur = fma((T)RDG_TAB[ODR + i * NP + j], u[j], ur);
      us = fma((T)RDG_TAB[ODS + i * NP + j], u[j], us);
    }
    fr[i] = ar * u[i] - (grr * ur + grs * us);
    fs[i] = as * u[i] - (grs * ur + gss * us);
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      acc = fma((T)RDG_TAB[OWR + i * NP + j], fr[j], acc);
      acc = fma((T)RDG_TAB[OWS + i * NP + j], fs[j], acc);
    }
    vol[i] = acc;
  }
}

// Persistent edge-flux kernel, one CTA per SM (tile = blockIdx.x + m gridDim.x, m taken
// from a CTA-local counter, so the CTA's warps share its tiles dynamically).  Each edge warp
// owns DEPTH shared-memory slots: its lane 0 claims a tile, starts a cp.async.bulk of the
// tile's operator words into a slot (mbarrier completion), and the warp consumes its slots
// round-robin -- one edge per lane: gather u_k1, u_k2 (L2 resident) while the copy is in
// flight, wait on the slot's barrier (phase parity = use count, the slot having no other
// consumer), flux_e = W_e [u1; u2] from shared memory, then fence its shared-memory reads
// against the async proxy and refill the slot.  Every wait is bounded: on a timeout the
// kernel sets kErrWaitTimeout, waits (bounded) for the warp's copies in flight and stops.
//
// VOL = true (fused form) adds NV volume warps that compute the volume term of element tiles
// of 32 (tile j = blockIdx.x + m gridDim.x, m = volume warp + NV t) and store it to a.vol;
// they share the SM with the memory-bound operator stream, so their FMA work is hidden.
template <typename T, int N, bool VOL>
__global__ void __launch_bounds__(EdgePipe<T, N, VOL>::THREADS, 1) edge_flux_kernel(EdgeArgs<T> a) {
  using P = EdgePipe<T, N, VOL>;
  constexpr int NP = P::NP, NFP = P::NFP, NW = P::NW, QW = P::QW, DEPTH = P::DEPTH, NE = P::NE;
  using V = Vec16<T>;
  using VT = typename V::type;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  int* next_tile = reinterpret_cast<int*>(smem + P::SLOTS * 8);
  unsigned char* ring = smem + P::BAR_BYTES;
  const int64_t ntiles = (a.E + kTile - 1) / kTile;
  const int64_t my_n = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P::SLOTS; ++s) mbar_init(&full[s], 1);
    *next_tile = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if constexpr (VOL) {
    if (warp >= NE) {
      const int vw = warp - NE;
      T* sv = reinterpret_cast<T*>(ring + (size_t)P::SLOTS * P::TILE_BYTES) + vw * kTile * NP;
      const int64_t nvt = (a.K + kTile - 1) / kTile;
      for (int64_t j = blockIdx.x + (int64_t)vw * gridDim.x; j < nvt; j += (int64_t)P::NV * gridDim.x) {
        const int64_t k0 = j * kTile;
        const int nk = (int)min((int64_t)kTile, a.K - k0);
        const T* src = a.u + k0 * NP;
        for (int x = lane; x < nk * NP; x += 32) sv[x] = src[x];
        __syncwarp();
        T u[NP];
#pragma unroll
        for (int jj = 0; jj < NP; ++jj) u[jj] = lane < nk ? sv[lane * NP + jj] : T(0);
        __syncwarp();
        if (lane < nk) {
          const int64_t k = k0 + lane;
          T vol[NP];
          volume_row<T, N>(u, a.geo[k], a.geo[a.K + k], a.geo[2 * a.K + k], a.geo[3 * a.K + k], a.geo[4 * a.K + k],
                           vol);
#pragma unroll
          for (int ii = 0; ii < NP; ++ii) sv[lane * NP + ii] = vol[ii];
        }
        __syncwarp();
        T* dst = a.vol + k0 * NP;
        for (int x = lane; x < nk * NP; x += 32) dst[x] = sv[x];
        __syncwarp();
      }
      return;
    }
  }

  const unsigned char* W = static_cast<const unsigned char*>(a.W);
  const uint64_t pol = l2_evict_first_policy();
  // claim the CTA's next tile and start its copy into this warp's slot `slot`; returns the
  // claimed local tile index (warp-uniform) or -1 when the CTA's tiles are exhausted
  auto issue = [&](int slot) -> long long {
    long long m = -1;
    if (lane == 0) {
      const long long c = atomicAdd(next_tile, 1);
      if (c < my_n) {
        m = c;
        mbar_expect_tx(&full[slot], P::TILE_BYTES);
        bulk_g2s(ring + (size_t)slot * P::TILE_BYTES, W + (blockIdx.x + c * gridDim.x) * P::TILE_BYTES,
                 P::TILE_BYTES, &full[slot], pol);
      }
    }
    return __shfl_sync(0xffffffffu, m, 0);
  };
  long long ids[DEPTH];
#pragma unroll
  for (int d = 0; d < DEPTH; ++d) ids[d] = issue(warp * DEPTH + d);

  // gather u_k1, u_k2 of local tile m into uu (lane = edge); e < 0 when the lane has no edge
  auto gather = [&](long long m, T (&uu)[2 * NP], int64_t& e) {
#pragma unroll
    for (int j = 0; j < 2 * NP; ++j) uu[j] = T(0);
    e = -1;
    if (m < 0) return;
    const int64_t ee = (blockIdx.x + m * gridDim.x) * kTile + lane;
    if (ee >= a.E) return;
    e = ee;
    const int k1 = a.k1[ee], k2 = a.k2[ee];
    // self-check of the edge table: a bad index is recorded and its access skipped
    if (k1 < 0 || k1 >= a.K || (k2 >= 0 ? k2 >= a.K : (-1 - (int64_t)k2) >= a.B)) {
      report(a.err, kErrBadIndex);
      return;
    }
    const T* p1 = a.u + (int64_t)k1 * NP;
#pragma unroll
    for (int j = 0; j < NP; ++j) uu[j] = __ldg(p1 + j);
    if (k2 >= 0) {
      const T* p2 = a.u + (int64_t)k2 * NP;
#pragma unroll
      for (int j = 0; j < NP; ++j) uu[NP + j] = __ldg(p2 + j);
    } else {
      // ghost side of a boundary edge: g = sum_m G_m tau_m(t)
      const int64_t b = -1 - (int64_t)k2;
      const double t = stage_time(a.time);
      for (int mm = 0; mm < a.frc.nghost; ++mm) {
        const T tm = (T)tau_of(a.frc.gkind[mm], a.frc.gomega[mm], t);
        const T* g = a.G + ((int64_t)mm * a.B + b) * NP;
#pragma unroll
        for (int j = 0; j < NP; ++j) uu[NP + j] += tm * g[j];
      }
    }
  };

  // one tile: prefetch the next tile's gathers into nxt, wait for this tile's operator words,
  // flux = W [u1; u2] with cur, refill the slot; false when the warp has no tile left
  auto step = [&](int k, T (&cur)[2 * NP], int64_t ecur, T (&nxt)[2 * NP], int64_t& enxt) -> bool {
    const int d = k % DEPTH;
    const int slot = warp * DEPTH + d;
    if (ids[d] < 0) return false;
    gather(ids[(k + 1) % DEPTH], nxt, enxt);
    const bool landed = __all_sync(0xffffffffu, mbar_wait_bounded(&full[slot], (uint32_t)(k / DEPTH) & 1u));
    if (!landed) {
      if (lane == 0) {
        report(a.err, kErrWaitTimeout);
        // let this warp's other copies in flight land before it leaves
        for (int dd = 1; dd < DEPTH; ++dd) {
          const int kk = k + dd;
          if (ids[kk % DEPTH] >= 0) mbar_wait_bounded(&full[warp * DEPTH + kk % DEPTH], (uint32_t)(kk / DEPTH) & 1u);
        }
      }
      return false;
    }
    const VT* w = reinterpret_cast<const VT*>(ring + (size_t)slot * P::TILE_BYTES) + lane;
    T acc[NFP];
#pragma unroll
    for (int i2 = 0; i2 < NFP; ++i2) acc[i2] = T(0);
#pragma unroll
    for (int q = 0; q < QW; ++q) {
      const VT v = w[q * kTile];
#pragma unroll
      for (int cc = 0; cc < V::n; ++cc) {
        const int idx = q * V::n + cc;
        if (idx < NW) acc[idx / (2 * NP)] = fma(V::get(v, cc), cur[idx % (2 * NP)], acc[idx / (2 * NP)]);
      }
    }
    // the slot's reads (generic proxy) must be ordered before the copy engine refills it
    fence_proxy_async_smem();
    __syncwarp();
    ids[d] = issue(slot);
    if (ecur >= 0) {
      T* o = a.flux + ecur * NFP;
#pragma unroll
      for (int r = 0; r < NFP; ++r) o[r] = acc[r];
    }
    return true;
  };

  T ua[2 * NP], ub[2 * NP];
  int64_t ea, eb;
  gather(ids[0], ua, ea);
  for (int k = 0;; k += 2) {
    if (!step(k, ua, ea, ub, eb)) break;
    if (!step(k + 1, ub, eb, ua, ea)) break;
  }
}

// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void stage_in(T* sh, const T* g, int n) {
  constexpr int V = 16 / sizeof(T);
  const int nv = n / V;
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float4* s4 = reinterpret_cast<float4*>(sh);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) s4[i] = __ldcs(g4 + i);
  for (int i = nv * V + threadIdx.x; i < n; i += blockDim.x) sh[i] = g[i];
}

template <typename T>
__device__ __forceinline__ void stage_out(T* g, const T* sh, int n) {
  constexpr int V = 16 / sizeof(T);
  const int nv = n / V;
  float4* g4 = reinterpret_cast<float4*>(g);
  const float4* s4 = reinterpret_cast<const float4*>(sh);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) __stcs(g4 + i, s4[i]);
  for (int i = nv * V + threadIdx.x; i < n; i += blockDim.x) g[i] = sh[i];
}

// Resident blocks per SM asked of the compiler for the surface-only form (VOLIN): FP32 orders
// up to 4 fit 8 blocks of 128 threads (<= 64 registers), so a 131072-element stage runs in
// one wave.
template <typename T, int N, bool VOLIN>
constexpr int elem_min_blocks() {
  return (VOLIN && sizeof(T) == 4 && N <= 4) ? 8 : 1;
}

// Element update.  VOLIN = false: volume term computed here; VOLIN = true: read from a.vol
// (computed by the fused edge kernel).  Then surface terms, sources and the stage.
template <typename T, int N, int MODE, bool VOLIN>
__global__ void __launch_bounds__(kElemBlock, elem_min_blocks<T, N, VOLIN>()) elem_kernel(ElemArgs<T> a) {
  constexpr int NP = np_of(N), NFP = nfp_of(N);
  constexpr int OLIFT = 4 * NP * NP;
  __shared__ __align__(16) T sh[kElemBlock * NP];
  __shared__ __align__(16) T shv[VOLIN ? kElemBlock * NP : 4];
  __shared__ T tau_s[RDG_MAX_FORCING_TERMS];
  const int64_t k0 = (int64_t)blockIdx.x * kElemBlock;
  const int nk = (int)min((int64_t)kElemBlock, a.K - k0);
  const int tid = threadIdx.x;
  const bool active = tid < nk;
  const int64_t k = k0 + tid;

  if (!VOLIN || MODE >= 1) stage_in(sh, a.us + k0 * NP, nk * NP);
  if (VOLIN) stage_in(shv, a.vol + k0 * NP, nk * NP);
  if (tid < a.frc.nsrc) tau_s[tid] = (T)tau_of(a.frc.kind[tid], a.frc.omega[tid], stage_time(a.time));
  __syncthreads();

  T rhs[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) rhs[i] = T(0);
  if (active) {
    const T ij = a.geo[5 * a.K + k];
    if constexpr (VOLIN) {
#pragma unroll
      for (int i = 0; i < NP; ++i) rhs[i] = shv[tid * NP + i];
    } else {
      T u[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) u[j] = sh[tid * NP + j];
      volume_row<T, N>(u, a.geo[k], a.geo[a.K + k], a.geo[2 * a.K + k], a.geo[3 * a.K + k], a.geo[4 * a.K + k],
                       rhs);
    }
    // surface terms: side 1 takes J_f F*.n1 in its face order, side 2 the negated reverse
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      int er = a.eref[(int64_t)f * a.K + k];
      if (er < 0 || (er >> 1) >= a.E) {     // self-check: record and read edge 0 instead
        report(a.err, kErrBadIndex);
        er = 0;
      }
      const T* fl = a.flux + (int64_t)(er >> 1) * NFP;
      const bool side2 = er & 1;
      T q[NFP], qv[NFP];
#pragma unroll
      for (int i = 0; i < NFP; ++i) q[i] = fl[i];
#pragma unroll
      for (int i = 0; i < NFP; ++i) qv[i] = side2 ? -q[NFP - 1 - i] : q[i];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < NFP; ++c) acc = fma((T)RDG_TAB[OLIFT + i * 3 * NFP + f * NFP + c], qv[c], acc);
        rhs[i] -= ij * acc;
      }
    }
    for (int m = 0; m < a.frc.nsrc; ++m) {
      const T* S = a.S + ((int64_t)m * a.K + k) * NP;
#pragma unroll
      for (int i = 0; i < NP; ++i) rhs[i] = fma(tau_s[m], S[i], rhs[i]);
    }
  }
  // stage value u_s + dt L(u_s), with u_s re-read from shared memory
  if (MODE >= 1) {
#pragma unroll
    for (int i = 0; i < NP; ++i) rhs[i] = fma(a.dt, rhs[i], sh[tid * NP + i]);
  }
  if (MODE >= 2) {
    __syncthreads();
    stage_in(sh, a.un + k0 * NP, nk * NP);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if (MODE == 2) rhs[i] = T(0.75) * sh[tid * NP + i] + T(0.25) * rhs[i];
      else rhs[i] = T(1.0 / 3.0) * sh[tid * NP + i] + T(2.0 / 3.0) * rhs[i];
    }
  }
  T* res = rhs;
  __syncthreads();
  if (active) {
#pragma unroll
    for (int i = 0; i < NP; ++i) sh[tid * NP + i] = res[i];
  }
  __syncthreads();
  stage_out(a.out + k0 * NP, sh, nk * NP);
}

// Surface-only element update of the fused form: rhs = vol - (1/J) sum_f LIFT_f q_f + s,
// then the stage.  All of the block's inputs are requested up front (edge ids and face
// fluxes into registers, volume term / stage input / step start through shared memory), so
// one memory round trip covers the kernel.
// Elements per block of the surface-only kernel: 128, or 64 where three staged arrays of
// 128 rows would pass the 48 KB static shared-memory limit (FP64, N >= 5).
template <typename T, int N>
__host__ __device__ constexpr int lite_block() {
  return 3 * 128 * np_of(N) * (int)sizeof(T) > 46 * 1024 ? 64 : 128;
}

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(lite_block<T, N>(), elem_min_blocks<T, N, true>()) elem_lite_kernel(ElemArgs<T> a) {
  constexpr int NP = np_of(N), NFP = nfp_of(N);
  constexpr int OLIFT = 4 * NP * NP;
  constexpr int BLK = lite_block<T, N>();
  __shared__ __align__(16) T shv[BLK * NP];
  __shared__ __align__(16) T shs[MODE >= 1 ? BLK * NP : 4];
  __shared__ __align__(16) T shn[MODE >= 2 ? BLK * NP : 4];
  __shared__ T tau_s[RDG_MAX_FORCING_TERMS];
  const int64_t k0 = (int64_t)blockIdx.x * BLK;
  const int nk = (int)min((int64_t)BLK, a.K - k0);
  const int tid = threadIdx.x;
  const bool active = tid < nk;
  const int64_t k = k0 + tid;

  int er[3] = {0, 0, 0};
  T ij = T(0);
  if (active) {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      er[f] = a.eref[(int64_t)f * a.K + k];
      if (er[f] < 0 || (er[f] >> 1) >= a.E) {     // self-check: record and read edge 0 instead
        report(a.err, kErrBadIndex);
        er[f] = 0;
      }
    }
    ij = a.geo[5 * a.K + k];
  }
  stage_in(shv, a.vol + k0 * NP, nk * NP);
  if (MODE >= 1) stage_in(shs, a.us + k0 * NP, nk * NP);
  if (MODE >= 2) stage_in(shn, a.un + k0 * NP, nk * NP);
  T q[3][NFP];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const T* fl = a.flux + (int64_t)(er[f] >> 1) * NFP;
#pragma unroll
    for (int c = 0; c < NFP; ++c) q[f][c] = active ? fl[c] : T(0);
  }
  if (tid < a.frc.nsrc) tau_s[tid] = (T)tau_of(a.frc.kind[tid], a.frc.omega[tid], stage_time(a.time));
  __syncthreads();

  T rhs[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) rhs[i] = shv[tid * NP + i];
  // surface terms: side 1 takes J_f F*.n1 in its face order, side 2 the negated reverse
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const bool side2 = er[f] & 1;
    T qv[NFP];
#pragma unroll
    for (int c = 0; c < NFP; ++c) qv[c] = side2 ? -q[f][NFP - 1 - c] : q[f][c];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < NFP; ++c) acc = fma((T)RDG_TAB[OLIFT + i * 3 * NFP + f * NFP + c], qv[c], acc);
      rhs[i] -= ij * acc;
    }
  }
  if (active) {
    for (int m = 0; m < a.frc.nsrc; ++m) {
      const T* S = a.S + ((int64_t)m * a.K + k) * NP;
#pragma unroll
      for (int i = 0; i < NP; ++i) rhs[i] = fma(tau_s[m], S[i], rhs[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    if (MODE >= 1) rhs[i] = fma(a.dt, rhs[i], shs[tid * NP + i]);
    if (MODE == 2) rhs[i] = T(0.75) * shn[tid * NP + i] + T(0.25) * rhs[i];
    if (MODE == 3) rhs[i] = T(1.0 / 3.0) * shn[tid * NP + i] + T(2.0 / 3.0) * rhs[i];
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int i = 0; i < NP; ++i) shv[tid * NP + i] = rhs[i];
  }
  __syncthreads();
  stage_out(a.out + k0 * NP, shv, nk * NP);
}

}  // namespace dev

// Host-side launch helpers instantiated by the including translation unit.
inline int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 1;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

template <typename T, int N, bool VOL = false>
inline int launch_edge_t(const EdgeArgs<T>& a, cudaStream_t s) {
  using P = dev::EdgePipe<T, N, VOL>;
  if (a.E == 0) return RDG_OK;
  static bool attr_set[64] = {false};   // per instantiation and device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return RDG_EINVAL;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(dev::edge_flux_kernel<T, N, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             P::SMEM) != cudaSuccess)
      return RDG_ECUDA;
    attr_set[dev] = true;
  }
  const int64_t ntiles = (a.E + kTile - 1) / kTile;
  int64_t cap = sm_count();
  if (a.max_ctas > 0 && a.max_ctas < cap) cap = a.max_ctas;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, cap);
  dev::edge_flux_kernel<T, N, VOL><<<grid, P::THREADS, P::SMEM, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

template <typename T, int N, bool VOLIN = false>
inline int launch_elem_t(int mode, const ElemArgs<T>& a, cudaStream_t s) {
  if (a.K == 0) return RDG_OK;
  const unsigned grid = (unsigned)((a.K + kElemBlock - 1) / kElemBlock);
  if constexpr (VOLIN) {
    constexpr int BLK = dev::lite_block<T, N>();
    const unsigned g2 = (unsigned)((a.K + BLK - 1) / BLK);
    switch (mode) {
      case 0: dev::elem_lite_kernel<T, N, 0><<<g2, BLK, 0, s>>>(a); break;
      case 1: dev::elem_lite_kernel<T, N, 1><<<g2, BLK, 0, s>>>(a); break;
      case 2: dev::elem_lite_kernel<T, N, 2><<<g2, BLK, 0, s>>>(a); break;
      case 3: dev::elem_lite_kernel<T, N, 3><<<g2, BLK, 0, s>>>(a); break;
      default: return RDG_EINVAL;
    }
  } else {
    switch (mode) {
      case 0: dev::elem_kernel<T, N, 0, false><<<grid, kElemBlock, 0, s>>>(a); break;
      case 1: dev::elem_kernel<T, N, 1, false><<<grid, kElemBlock, 0, s>>>(a); break;
      case 2: dev::elem_kernel<T, N, 2, false><<<grid, kElemBlock, 0, s>>>(a); break;
      case 3: dev::elem_kernel<T, N, 3, false><<<grid, kElemBlock, 0, s>>>(a); break;
      default: return RDG_EINVAL;
    }
  }
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

// Reference matrices of order N in the kernel-table layout.
template <typename T>
inline std::vector<T> pack_elem_table(int N) {
  std::vector<T> t;
  const RefOps* o = get_refops(N, nullptr);
  if (!o) return t;
  for (const std::vector<double>* m : {&o->Dr, &o->Ds, &o->Wr, &o->Ws, &o->LIFT})
    for (double v : *m) t.push_back((T)v);
  return t;
}

}  // namespace rdg

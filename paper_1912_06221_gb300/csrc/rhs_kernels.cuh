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
#include <utility>

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

// 16-byte load that asks L2 to keep the line (evict-last policy): operator words reread by
// every stage stay L2-resident up to the keep budget instead of streaming from HBM again
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float4 ld_keep(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_keep(const double2* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while its predecessor in the stream finishes; it must wait here before touching any
// data the predecessor reads or writes (a no-op for an ordinary launch).
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel in the stream launch once every block of this grid has executed it
// (or exited); the next kernel still waits for this grid's completion and memory before it
// reads anything this grid writes.
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void report(int* err, int bit) {
  if (err) atomicOr(err, bit);
}

// Volume term of one element: M^{-1} S^T . F with F = v u - D grad u, written with the
// metric-folded coefficients F_r = a_r u - (g_rr u_r + g_rs u_s), F_s = a_s u - (g_rs u_r +
// g_ss u_s), vol = Wr F_r + Ws F_s (Wr = M^{-1} Dr^T M, Ws = M^{-1} Ds^T M).  The derivatives
// are taken of u - u_0 (Dr, Ds annihilate constants), so the rounding of their large entries
// multiplies differences of nearby values rather than u itself.  Evaluated node by node as a
// running outer product (F_r, F_s at node j, then their column j of Wr, Ws into vol), so only
// u - u_0 and vol are live: 2 Np values instead of 5 Np.
//
// NODAL: D given at the nodes (dn, the element's Np values; the coefficients g_rr, g_rs, g_ss
// then hold the metric alone), F_r = a_r u - D_j (g_rr u_r + g_rs u_s) node by node.
template <typename T, int N, bool NODAL = false>
__device__ __forceinline__ void volume_row(const T (&u)[np_of(N)], T ar, T as, T grr, T grs, T gss,
                                           T (&vol)[np_of(N)], const T* __restrict__ dn = nullptr) {
  constexpr int NP = np_of(N);
  constexpr int ODR = 0, ODS = NP * NP, OWR = 2 * NP * NP, OWS = 3 * NP * NP;
  T du[NP];
#pragma unroll
  for (int j = 1; j < NP; ++j) du[j] = u[j] - u[0];
#pragma unroll
  for (int i = 0; i < NP; ++i) vol[i] = T(0);
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    T ur = T(0), us = T(0);
#pragma unroll
    for (int k = 1; k < NP; ++k) {
      ur = fma((T)RDG_TAB[ODR + j * NP + k], du[k], ur);
      us = fma((T)RDG_TAB[ODS + j * NP + k], du[k], us);
    }
    const T uj = j == 0 ? u[0] : du[j] + u[0];
    T fr, fs;
    if constexpr (NODAL) {
      const T dj = __ldg(dn + j);
      fr = ar * uj - dj * (grr * ur + grs * us);
      fs = as * uj - dj * (grs * ur + gss * us);
    } else {
      fr = ar * uj - (grr * ur + grs * us);
      fs = as * uj - (grs * ur + gss * us);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      vol[i] = fma((T)RDG_TAB[OWR + i * NP + j], fr, vol[i]);
      vol[i] = fma((T)RDG_TAB[OWS + i * NP + j], fs, vol[i]);
    }
  }
}

// The same volume term for the largest order, with the four reference matrices staged in
// shared memory (from RDG_VOLTAB: Dr, Ds row-major, then Wr^T, Ws^T, rows padded to 16 bytes)
// and the node loop unrolled only twice: fully unrolled with constant-bank operands the
// N = 6 row is over 3000 FMAs of straight-line code beside the edge role's, and the stage
// measured 155 us on 131072 triangles against 125 us this way (unroll 1: 134, 4: 125).
template <typename T, int N>
struct VolTab {
  static constexpr int NP = np_of(N);
  static constexpr int NPP = (NP * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
  static constexpr int SIZE = 4 * NP * NPP;
};

template <typename T, int N, bool NODAL = false>
__device__ __forceinline__ void volume_row_smem(const T (&u)[np_of(N)], T ar, T as, T grr, T grs, T gss,
                                                const T* __restrict__ tab, T (&vol)[np_of(N)],
                                                const T* __restrict__ dn = nullptr) {
  using VT = VolTab<T, N>;
  constexpr int NP = VT::NP, NPP = VT::NPP;
  T du[NP];
#pragma unroll
  for (int j = 1; j < NP; ++j) du[j] = u[j] - u[0];
  du[0] = T(0);
#pragma unroll
  for (int i = 0; i < NP; ++i) vol[i] = T(0);
#pragma unroll 2
  for (int j = 0; j < NP; ++j) {
    const T* Dr = tab + j * NPP;
    const T* Ds = tab + NP * NPP + j * NPP;
    const T* WrT = tab + 2 * NP * NPP + j * NPP;
    const T* WsT = tab + 3 * NP * NPP + j * NPP;
    T ur = T(0), us = T(0);
#pragma unroll
    for (int k = 1; k < NP; ++k) {
      ur = fma(Dr[k], du[k], ur);
      us = fma(Ds[k], du[k], us);
    }
    T uj = u[0];
#pragma unroll
    for (int k = 1; k < NP; ++k) uj = (k == j) ? du[k] + u[0] : uj;
    T fr, fs;
    if constexpr (NODAL) {
      const T dj = __ldg(dn + j);
      fr = ar * uj - dj * (grr * ur + grs * us);
      fs = as * uj - dj * (grs * ur + gss * us);
    } else {
      fr = ar * uj - (grr * ur + grs * us);
      fs = as * uj - (grs * ur + gss * us);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      vol[i] = fma(WrT[i], fr, vol[i]);
      vol[i] = fma(WsT[i], fs, vol[i]);
    }
  }
}

// Convex combination of SSP-RK3 stages 2 and 3: (1 - c) u_n + c v with c = 1/4 or 2/3,
// evaluated as u_n + c (v - u_n).  Written as c1 u_n + c2 v with the coefficients rounded to
// FP32, c1 + c2 = 1 + 3e-8 for c = 2/3 and every step would scale the state by that factor
// (a 1.5e-5 drift over 500 steps); here the rounding of c only touches the increment.
template <typename T, int MODE>
__device__ __forceinline__ T rk_combine(T un, T v) {
  const T c = MODE == 2 ? T(0.25) : T(2.0 / 3.0);
  return fma(c, v - un, un);
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

// Batched staging: every thread first issues all of its 16-byte loads of a block's rows
// (n values, n <= BLK * NP, 16-byte aligned start) into registers, and only then stores them
// to shared memory, so a tile costs one memory round trip instead of one per loop trip.
template <typename T, int BLK, int NP>
struct Staged {
  static constexpr int V = 16 / (int)sizeof(T);
  static constexpr int IT = ((BLK * NP + V - 1) / V + BLK - 1) / BLK;
  float4 r[IT];
  T tail0;
  __device__ __forceinline__ void load(const T* g, int n) {
    const int nv = n / V;
    const float4* g4 = reinterpret_cast<const float4*>(g);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int i = threadIdx.x + it * BLK;
      if (i < nv) r[it] = __ldcs(g4 + i);
    }
    const int i = nv * V + threadIdx.x;
    if (threadIdx.x < V && i < n) tail0 = g[i];
  }
  __device__ __forceinline__ void store(T* sh, int n) const {
    const int nv = n / V;
    float4* s4 = reinterpret_cast<float4*>(sh);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int i = threadIdx.x + it * BLK;
      if (i < nv) s4[i] = r[it];
    }
    const int i = nv * V + threadIdx.x;
    if (threadIdx.x < V && i < n) sh[i] = tail0;
  }
};

template <typename T>
__device__ __forceinline__ void stage_out(T* g, const T* sh, int n) {
  constexpr int V = 16 / sizeof(T);
  const int nv = n / V;
  float4* g4 = reinterpret_cast<float4*>(g);
  const float4* s4 = reinterpret_cast<const float4*>(sh);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) __stcs(g4 + i, s4[i]);
  for (int i = nv * V + threadIdx.x; i < n; i += blockDim.x) g[i] = sh[i];
}

// Volume role of the stage kernel: element tile v (one thread per element, rows staged
// through shared memory), vol = M^{-1} S^T . F written to a.vol.  Kept out of line so its
// register demand does not set the edge role's.
template <typename T, int N, bool NODAL = false>
__device__ __noinline__ void stage_volume_tile(const EdgeArgs<T>& a, int64_t v, T* sh) {
  constexpr int NP = np_of(N);
  constexpr bool SMEM_TAB = N >= 6 && sizeof(T) == 4;   // (FP64: 25 KB of tables, and FP64-bound anyway)
  __shared__ __align__(16) T tab[SMEM_TAB ? VolTab<T, N>::SIZE : 4];
  const int tid = threadIdx.x;
  const int64_t k0 = v * kStageBlock;
  const int nk = (int)min((int64_t)kStageBlock, (a.Kvol > 0 ? a.Kvol : a.K) - k0);
  {
    Staged<T, kStageBlock, NP> g;
    g.load(a.u + k0 * NP, nk * NP);
    if constexpr (SMEM_TAB) {
      constexpr int NV = VolTab<T, N>::SIZE * (int)sizeof(T) / 16;
      const float4* src = reinterpret_cast<const float4*>(RDG_VOLTAB);
      float4* dst = reinterpret_cast<float4*>(tab);
      for (int i = tid; i < NV; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    g.store(sh, nk * NP);
  }
  __syncthreads();
  if (tid < nk) {
    const int64_t k = k0 + tid;
    T u[NP], vol[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) u[j] = sh[tid * NP + j];
    const T* dn = NODAL ? a.Dn + k * NP : nullptr;
    if constexpr (SMEM_TAB)
      volume_row_smem<T, N, NODAL>(u, a.geo[k], a.geo[a.K + k], a.geo[2 * a.K + k], a.geo[3 * a.K + k],
                                   a.geo[4 * a.K + k], tab, vol, dn);
    else
      volume_row<T, N, NODAL>(u, a.geo[k], a.geo[a.K + k], a.geo[2 * a.K + k], a.geo[3 * a.K + k], a.geo[4 * a.K + k],
                              vol, dn);
#pragma unroll
    for (int j = 0; j < NP; ++j) sh[tid * NP + j] = vol[j];   // a thread rewrites only its own row
  }
  __syncthreads();
  stage_out(a.vol + k0 * NP, sh, nk * NP);
}

// Stored operator words of one edge (difference form, see edge_flux_core).
template <typename T, int N>
struct EdgeWords {
  static constexpr int NWS = nfp_of(N) * (2 * np_of(N) - 1) + 1;   // stored values per edge
  static constexpr int QW = (NWS + Vec16<T>::n - 1) / Vec16<T>::n;  // 16-byte words per edge
  typename Vec16<T>::type v[QW];
};

// The edge's operator words: streamed with evict-first 16-byte loads (in the stage kernel a
// warp reads 512 contiguous bytes per load of its tile), or kept in L2 for the first
// keep_tiles tiles.
template <typename T, int N>
__device__ __forceinline__ void edge_words(const EdgeArgs<T>& a, int64_t e, EdgeWords<T, N>& w) {
  using VT = typename Vec16<T>::type;
  constexpr int QW = EdgeWords<T, N>::QW;
  const VT* p = reinterpret_cast<const VT*>(a.W) + ((e >> 5) * QW) * kTile + (e & 31);
  const bool keep = (e >> 5) < a.keep_tiles;
  const uint64_t pol = keep ? l2_keep_policy() : 0;
#pragma unroll
  for (int q = 0; q < QW; ++q) w.v[q] = keep ? ld_keep(p + q * kTile, pol) : ld_stream(p + q * kTile);
}

// The two elements' rows of edge e (k1, k2 from the edge table; a boundary edge's ghost side
// sum_m G_m tau_m(t)); a bad index is recorded and its rows left zero.
template <typename T, int N>
__device__ __forceinline__ void edge_rows(const EdgeArgs<T>& a, int k1, int k2, T (&u1)[np_of(N)], T (&u2)[np_of(N)]) {
  constexpr int NP = np_of(N);
#pragma unroll
  for (int j = 0; j < NP; ++j) u1[j] = u2[j] = T(0);
  if (k1 < 0 || k1 >= a.K || (k2 >= 0 ? k2 >= a.K : (-1 - (int64_t)k2) >= a.B)) {
    report(a.err, kErrBadIndex);
    return;
  }
  const T* p1 = a.u + (int64_t)k1 * NP;
#pragma unroll
  for (int j = 0; j < NP; ++j) u1[j] = __ldg(p1 + j);
  if (k2 >= 0) {
    const T* p2 = a.u + (int64_t)k2 * NP;
#pragma unroll
    for (int j = 0; j < NP; ++j) u2[j] = __ldg(p2 + j);
  } else {
    const int64_t bb = -1 - (int64_t)k2;
    const double t = stage_time(a.time);
    for (int mm = 0; mm < a.frc.nghost; ++mm) {
      const T tm = (T)tau_of(a.frc.gkind[mm], a.frc.gomega[mm], t);
      const T* g = a.G + ((int64_t)mm * a.B + bb) * NP;
#pragma unroll
      for (int j = 0; j < NP; ++j) u2[j] += tm * g[j];
    }
  }
}

// flux_e = W_e [u1; u2] (Nfp values in side 1's face order) in the difference form of the
// stored operator: each row holds the coefficients of (u1_1 - u_0, ..., u1_{Np-1} - u_0,
// u2_0 - u_0, ..., u2_{Np-1} - u_0), u_0 = u1_0, and the edge's last value s = J_f (v.n1)
// multiplies u_0 in every row.
template <typename T, int N>
__device__ __forceinline__ void edge_flux_core(T (&u1)[np_of(N)], T (&u2)[np_of(N)], const EdgeWords<T, N>& w,
                                               T (&acc)[nfp_of(N)]) {
  constexpr int NP = np_of(N), NFP = nfp_of(N);
  constexpr int RW = 2 * NP - 1, NWS = EdgeWords<T, N>::NWS, QW = EdgeWords<T, N>::QW;
  using V = Vec16<T>;
  const T ub = u1[0];
#pragma unroll
  for (int j = 1; j < NP; ++j) u1[j] -= ub;
#pragma unroll
  for (int j = 0; j < NP; ++j) u2[j] -= ub;
#pragma unroll
  for (int r = 0; r < NFP; ++r) acc[r] = T(0);
  T srow = T(0);
#pragma unroll
  for (int q = 0; q < QW; ++q) {
#pragma unroll
    for (int cc = 0; cc < V::n; ++cc) {
      const int idx = q * V::n + cc;
      if (idx < NWS - 1) {
        const int r = idx / RW, j = idx % RW;
        acc[r] = fma(V::get(w.v[q], cc), j < NP - 1 ? u1[j + 1] : u2[j - (NP - 1)], acc[r]);
      } else if (idx == NWS - 1) {
        srow = V::get(w.v[q], cc);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NFP; ++r) acc[r] = fma(srow, ub, acc[r]);
}

// Flux of edge e with its two element ids: rows, operator words, arithmetic.  Shared by the
// stage kernel's edge role and the one-kernel stage, so both give the same bits.
template <typename T, int N>
__device__ __forceinline__ void edge_acc(const EdgeArgs<T>& a, int64_t e, T (&acc)[nfp_of(N)], int& k1, int& k2) {
  constexpr int NP = np_of(N);
  k1 = a.k1[e];
  k2 = a.k2[e];
  T u1[NP], u2[NP];
  edge_rows<T, N>(a, k1, k2, u1, u2);
  EdgeWords<T, N> w;
  edge_words<T, N>(a, e, w);
  edge_flux_core<T, N>(u1, u2, w, acc);
}

// Edge role of the stage kernel: edge e (one thread per edge), its flux scattered to the two
// elements' face slots (FB) or written to the edge's row of a.flux.
template <typename T, int N, bool FB>
__device__ __noinline__ void stage_edge(const EdgeArgs<T>& a, int64_t e) {
  constexpr int NFP = nfp_of(N);
  T acc[NFP];
  int k1, k2;
  edge_acc<T, N>(a, e, acc, k1, k2);
  if constexpr (FB) {
    // scatter to the two elements' face slots: side 1 in its face order, side 2 (outward
    // normal -n1, face traversed the other way) negated and reversed
    const int f12 = a.f12[e];
    if (k1 >= 0 && k1 < a.K) {
      T* o1 = a.fb + ((int64_t)k1 * 3 + (f12 & 3)) * NFP;
#pragma unroll
      for (int r = 0; r < NFP; ++r) o1[r] = acc[r];
    }
    if (k2 >= 0 && k2 < a.K) {
      T* o2 = a.fb + ((int64_t)k2 * 3 + ((f12 >> 2) & 3)) * NFP;
#pragma unroll
      for (int r = 0; r < NFP; ++r) o2[r] = -acc[NFP - 1 - r];
    }
  } else {
    T* o = a.flux + e * NFP;
#pragma unroll
    for (int r = 0; r < NFP; ++r) o[r] = acc[r];
  }
}

// Stage kernel: one block per tile.  Without VOL every block is an edge block; with VOL (the
// fused form) the ceil(E/128) edge blocks and ceil(K/128) volume blocks are interleaved
// evenly over the grid (block b is a volume block when floor((b+1) nv / nb) steps up), so
// the volume FMAs run on the same SMs while the operator stream keeps HBM busy.
// Resident stage blocks per SM asked of the compiler (FP32: 5 blocks up to N = 4, <= 102
// registers; 6 above, where more warps in flight measured faster than more registers per
// thread; FP64: 4 up to N = 3, 3 above), so the operator stream keeps enough loads in flight.
// The edge-only form (kind 2) runs beside the tensor-core volume kernel with fewer, larger
// blocks: registers that would hold the volume role's values keep more operator loads in
// flight (order 6 measured 85, 83, 86 us per stage at 2, 3, 4 blocks per SM; orders 4 and 5
// in that form were fastest at 5 and 4).
constexpr int kEdgeOnlyBlocks[7] = {0, 5, 5, 5, 5, 4, 3};
template <typename T, int N, int KIND = 1>
constexpr int stage_min_blocks() {
  if (KIND == 2 && sizeof(T) == 4) return kEdgeOnlyBlocks[N];
  return sizeof(T) == 4 ? (N <= 4 ? 5 : 6) : (N <= 3 ? 4 : 3);
}

// Operator stream kinds: 0 edge blocks only, fluxes to the per-edge buffer (allocation-free
// entry point); 1 the fused form (edge and volume blocks interleaved, fluxes to the face
// slots); 2 edge blocks only, fluxes to the face slots (the volume term from its own
// kernel).
template <typename T, int N, int KIND>
__global__ void __launch_bounds__(kStageBlock, stage_min_blocks<T, N, KIND>()) edge_flux_kernel(EdgeArgs<T> a) {
  constexpr int NP = np_of(N);
  wait_for_predecessor();
  // the element kernel may start its independent loads on SMs that the last wave leaves idle
  if constexpr (KIND != 0) allow_dependents();
  int64_t eblk = blockIdx.x;
  if constexpr (KIND == 1) {
    __shared__ __align__(16) T sh[kStageBlock * NP];
    const int64_t nb = gridDim.x;
    const int64_t nv = ((a.Kvol > 0 ? a.Kvol : a.K) + kStageBlock - 1) / kStageBlock;
    const int64_t b = blockIdx.x;
    const int64_t v0 = (b * nv) / nb, v1 = ((b + 1) * nv) / nb;
    if (v1 > v0) {
      if (a.Dn) stage_volume_tile<T, N, true>(a, v0, sh);    // D given at the nodes
      else stage_volume_tile<T, N, false>(a, v0, sh);
      return;
    }
    eblk = b - v1;    // edge blocks so far = blocks so far minus volume blocks so far
  }
  const int64_t e = eblk * kStageBlock + threadIdx.x;
  if (e < a.E) stage_edge<T, N, KIND != 0>(a, e);
}


// Resident blocks per SM asked of the compiler for the surface-only form (VOLIN): FP32 orders
// up to 4 fit 7 blocks of 128 threads (<= 73 registers), so a 131072-element stage (1024
// blocks) runs in one wave on 152 SMs.
template <typename T, int N, bool VOLIN>
constexpr int elem_min_blocks() {
  return (VOLIN && sizeof(T) == 4 && N <= 4) ? 7 : 1;
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
    for (int i = 0; i < NP; ++i) rhs[i] = rk_combine<T, MODE>(sh[tid * NP + i], rhs[i]);
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
// then the stage.  The edge kernel has already scattered each edge's flux into both
// elements' face slots (q), so every input is a contiguous [K][.] row: the block stages its
// rows of the volume term, face fluxes, stage input and step start in one round trip.
template <typename T, int N>
__host__ __device__ constexpr int lite_block() {
  return 128 * (3 * np_of(N) + 3 * nfp_of(N)) * (int)sizeof(T) <= 46 * 1024
             ? 128
             : (64 * (3 * np_of(N) + 3 * nfp_of(N)) * (int)sizeof(T) <= 46 * 1024 ? 64 : 32);
}

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(lite_block<T, N>(), elem_min_blocks<T, N, true>()) elem_lite_kernel(ElemArgs<T> a) {
  constexpr int NP = np_of(N), NFP = nfp_of(N), NQ = 3 * NFP;
  constexpr int OLIFT = 4 * NP * NP;
  constexpr int BLK = lite_block<T, N>();
  __shared__ __align__(16) T shv[BLK * NP];
  __shared__ __align__(16) T shq[BLK * NQ];
  __shared__ __align__(16) T shs[MODE >= 1 ? BLK * NP : 4];
  __shared__ __align__(16) T shn[MODE >= 2 ? BLK * NP : 4];
  __shared__ T tau_s[RDG_MAX_FORCING_TERMS];
  const int64_t k0 = (int64_t)blockIdx.x * BLK;
  const int nk = (int)min((int64_t)BLK, a.K - k0);
  const int tid = threadIdx.x;
  const bool active = tid < nk;
  const int64_t k = k0 + tid;
  // The stage input and the step start are written by no kernel of this stage (they come from
  // the previous stage's element kernel, which the edge kernel waited for before it let this
  // grid launch), so they are staged before the dependency wait, overlapping the edge
  // kernel's last wave.
  {
    Staged<T, BLK, NP> gs, gn;
    if (MODE >= 1) gs.load(a.us + k0 * NP, nk * NP);
    if (MODE == 2 || MODE == 3 || (MODE == 4 && a.rka != T(0))) gn.load(a.un + k0 * NP, nk * NP);
    if (MODE >= 1) gs.store(shs, nk * NP);
    if (MODE == 2 || MODE == 3 || (MODE == 4 && a.rka != T(0))) gn.store(shn, nk * NP);
  }
  const T ij = active ? a.geo[5 * a.K + k] : T(0);
  wait_for_predecessor();
  {
    Staged<T, BLK, NP> gv;
    Staged<T, BLK, NQ> gq;
    gv.load(a.vol + k0 * NP, nk * NP);
    gq.load(a.fb + k0 * NQ, nk * NQ);
    gv.store(shv, nk * NP);
    gq.store(shq, nk * NQ);
  }
  if (tid < a.frc.nsrc) tau_s[tid] = (T)tau_of(a.frc.kind[tid], a.frc.omega[tid], stage_time(a.time));
  __syncthreads();

  T rhs[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) rhs[i] = shv[tid * NP + i];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    T q[NFP];
#pragma unroll
    for (int c = 0; c < NFP; ++c) q[c] = shq[tid * NQ + f * NFP + c];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < NFP; ++c) acc = fma((T)RDG_TAB[OLIFT + i * 3 * NFP + f * NFP + c], q[c], acc);
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
  if constexpr (MODE == 4) {
    // low-storage stage: du' = rka du + dt L, u' = u + rkb du' (both rows written in place)
    const bool rd = a.rka != T(0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const T du = rd ? fma(a.rka, shn[tid * NP + i], a.dt * rhs[i]) : a.dt * rhs[i];
      rhs[i] = du;
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < NP; ++i) shv[tid * NP + i] = fma(a.rkb, rhs[i], shs[tid * NP + i]);
    }
    __syncthreads();
    stage_out(a.out + k0 * NP, shv, nk * NP);
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < NP; ++i) shv[tid * NP + i] = rhs[i];
    }
    __syncthreads();
    stage_out(a.out2 + k0 * NP, shv, nk * NP);
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if (MODE >= 1) rhs[i] = fma(a.dt, rhs[i], shs[tid * NP + i]);
      if (MODE >= 2) rhs[i] = rk_combine<T, MODE>(shn[tid * NP + i], rhs[i]);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < NP; ++i) shv[tid * NP + i] = rhs[i];
    }
    __syncthreads();
    stage_out(a.out + k0 * NP, shv, nk * NP);
  }
}

// One-kernel stage for low orders: thread = element.  Each element computes the fluxes of its
// three edges itself (edge_acc, the same arithmetic as the stage kernel's edge role, so an
// edge's two elements use bitwise the same flux and the scheme stays conservative), then its
// volume term, LIFT, sources and the stage.  An edge's operator is read by both of its
// elements (the second read mostly hits L2: elements are ordered along a space-filling
// curve); in exchange the stage is one launch with no face-flux or volume-term round trip,
// which pays where a stage's work is small against a launch.  The edge ids and operator words
// are written by no stage, so at order 1 (few registers for them) they are loaded before the
// dependency wait, overlapping the previous stage's tail, with 8 blocks per SM asked of the
// compiler (circle pulse, 131072 triangles: 5.26 us per stage, against 5.52 without the early
// loads and 6.58 with them at the registers the compiler picks; at order 2 the early loads
// cost 2x); the rows wait for the predecessor.  Modes 0..3 only: its
// output must not be a buffer that other blocks gather from (the low-storage stage updates its
// input in place, so it keeps the two-kernel form).
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(kElemBlock, (N == 1 ? 8 : 1)) elem_fused_kernel(EdgeArgs<T> ea, ElemArgs<T> a) {
  static_assert(MODE >= 0 && MODE <= 3, "SSP-RK3 stages and the right-hand side only");
  constexpr int NP = np_of(N), NFP = nfp_of(N);
  constexpr int OLIFT = 4 * NP * NP;
  constexpr int BLK = kElemBlock;
  constexpr bool NEED_UN = MODE == 2 || MODE == 3;
  __shared__ __align__(16) T shs[BLK * NP];
  __shared__ __align__(16) T shn[NEED_UN ? BLK * NP : 4];
  __shared__ T tau_s[RDG_MAX_FORCING_TERMS];
  constexpr bool PRE = N == 1;
  const int64_t k0 = (int64_t)blockIdx.x * BLK;
  const int nk = (int)min((int64_t)BLK, a.K - k0);
  const int tid = threadIdx.x;
  const bool active = tid < nk;
  const int64_t k = active ? k0 + tid : k0;
  int er[3], kk1[3], kk2[3];
  EdgeWords<T, N> w[PRE ? 3 : 1];
  auto edge_ids = [&]() {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      er[f] = a.eref[(int64_t)f * a.K + k];
      if (er[f] < 0 || (er[f] >> 1) >= a.E) {   // self-check: record and use edge 0 instead
        report(a.err, kErrBadIndex);
        er[f] = 0;
      }
      kk1[f] = ea.k1[er[f] >> 1];
      kk2[f] = ea.k2[er[f] >> 1];
      if constexpr (PRE) edge_words<T, N>(ea, er[f] >> 1, w[f]);
    }
  };
  if constexpr (PRE) edge_ids();
  wait_for_predecessor();
  allow_dependents();
  if constexpr (!PRE) edge_ids();
  {
    Staged<T, BLK, NP> gs, gn;
    gs.load(a.us + k0 * NP, nk * NP);
    if (NEED_UN) gn.load(a.un + k0 * NP, nk * NP);
    gs.store(shs, nk * NP);
    if (NEED_UN) gn.store(shn, nk * NP);
  }
  if (tid < a.frc.nsrc) tau_s[tid] = (T)tau_of(a.frc.kind[tid], a.frc.omega[tid], stage_time(a.time));
  __syncthreads();
  T rhs[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) rhs[i] = T(0);
  if (active) {
    T u[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) u[j] = shs[tid * NP + j];
    if (ea.Dn)
      volume_row<T, N, true>(u, a.geo[k], a.geo[a.K + k], a.geo[2 * a.K + k], a.geo[3 * a.K + k], a.geo[4 * a.K + k],
                             rhs, ea.Dn + k * NP);
    else
      volume_row<T, N>(u, a.geo[k], a.geo[a.K + k], a.geo[2 * a.K + k], a.geo[3 * a.K + k], a.geo[4 * a.K + k], rhs);
    const T ij = a.geo[5 * a.K + k];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      T acc[NFP], q[NFP], u1[NP], u2[NP];
      edge_rows<T, N>(ea, kk1[f], kk2[f], u1, u2);
      if constexpr (PRE) {
        edge_flux_core<T, N>(u1, u2, w[f], acc);
      } else {
        edge_words<T, N>(ea, er[f] >> 1, w[0]);
        edge_flux_core<T, N>(u1, u2, w[0], acc);
      }
      // side 1 in its face order; side 2 (outward normal -n1, face traversed the other way)
      // negated and reversed
#pragma unroll
      for (int c = 0; c < NFP; ++c) q[c] = (er[f] & 1) ? -acc[NFP - 1 - c] : acc[c];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < NFP; ++c) s = fma((T)RDG_TAB[OLIFT + i * 3 * NFP + f * NFP + c], q[c], s);
        rhs[i] -= ij * s;
      }
    }
    for (int m = 0; m < a.frc.nsrc; ++m) {
      const T* S = a.S + ((int64_t)m * a.K + k) * NP;
#pragma unroll
      for (int i = 0; i < NP; ++i) rhs[i] = fma(tau_s[m], S[i], rhs[i]);
    }
  }
  {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if (MODE >= 1) rhs[i] = fma(a.dt, rhs[i], shs[tid * NP + i]);
      if (MODE >= 2) rhs[i] = rk_combine<T, MODE>(shn[tid * NP + i], rhs[i]);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < NP; ++i) shs[tid * NP + i] = rhs[i];
    }
    __syncthreads();
    stage_out(a.out + k0 * NP, shs, nk * NP);
  }
}

}  // namespace dev

// Host-side launch helpers instantiated by the including translation unit.
// Launch with programmatic stream serialization (the kernel waits for its predecessor with
// griddepcontrol.wait), so its launch and block scheduling overlap the predecessor's tail.
template <typename... KArgs, typename... Args>
inline int launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...) == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

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
  const int64_t kv = a.Kvol > 0 ? a.Kvol : a.K;
  if (a.E == 0 && (!VOL || kv == 0)) return RDG_OK;
  const int64_t ge = (a.E + kStageBlock - 1) / kStageBlock, gv = (kv + kStageBlock - 1) / kStageBlock;
  if constexpr (VOL) return launch_pdl(dev::edge_flux_kernel<T, N, 1>, (unsigned)(ge + gv), kStageBlock, s, a);
  dev::edge_flux_kernel<T, N, 0><<<(unsigned)ge, kStageBlock, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

// Edge blocks only, fluxes to the face slots, programmatic launch.
template <typename T, int N>
inline int launch_edge_fb_t(const EdgeArgs<T>& a, cudaStream_t s) {
  if (a.E == 0) return RDG_OK;
  const int64_t ge = (a.E + kStageBlock - 1) / kStageBlock;
  return launch_pdl(dev::edge_flux_kernel<T, N, 2>, (unsigned)ge, kStageBlock, s, a);
}

// One-kernel stage (elem_fused_kernel), programmatic launch.
template <typename T, int N>
inline int launch_fused_t(int mode, const EdgeArgs<T>& ea, const ElemArgs<T>& a, cudaStream_t s) {
  if (a.K == 0) return RDG_OK;
  const unsigned g = (unsigned)((a.K + kElemBlock - 1) / kElemBlock);
  switch (mode) {
    case 0: return launch_pdl(dev::elem_fused_kernel<T, N, 0>, g, kElemBlock, s, ea, a);
    case 1: return launch_pdl(dev::elem_fused_kernel<T, N, 1>, g, kElemBlock, s, ea, a);
    case 2: return launch_pdl(dev::elem_fused_kernel<T, N, 2>, g, kElemBlock, s, ea, a);
    case 3: return launch_pdl(dev::elem_fused_kernel<T, N, 3>, g, kElemBlock, s, ea, a);
    default: return RDG_EINVAL;   // the low-storage stage updates its input in place
  }
}

template <typename T, int N, bool VOLIN = false>
inline int launch_elem_t(int mode, const ElemArgs<T>& a, cudaStream_t s) {
  if (a.K == 0) return RDG_OK;
  const unsigned grid = (unsigned)((a.K + kElemBlock - 1) / kElemBlock);
  if constexpr (VOLIN) {
    constexpr int BLK = dev::lite_block<T, N>();
    const unsigned g2 = (unsigned)((a.K + BLK - 1) / BLK);
    switch (mode) {
      case 0: return launch_pdl(dev::elem_lite_kernel<T, N, 0>, g2, BLK, s, a);
      case 1: return launch_pdl(dev::elem_lite_kernel<T, N, 1>, g2, BLK, s, a);
      case 2: return launch_pdl(dev::elem_lite_kernel<T, N, 2>, g2, BLK, s, a);
      case 3: return launch_pdl(dev::elem_lite_kernel<T, N, 3>, g2, BLK, s, a);
      case 4: return launch_pdl(dev::elem_lite_kernel<T, N, 4>, g2, BLK, s, a);
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

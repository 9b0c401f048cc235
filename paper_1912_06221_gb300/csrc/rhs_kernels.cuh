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
template <typename T, int N>
__global__ void __launch_bounds__(kEdgeBlock) edge_flux_kernel(EdgeArgs<T> a) {
  constexpr int NP = np_of(N), NFP = nfp_of(N), NW = NFP * 2 * NP;
  using V = Vec16<T>;
  constexpr int VW = V::n, QW = (NW + VW - 1) / VW;
  const int64_t e = (int64_t)blockIdx.x * kEdgeBlock + threadIdx.x;
  if (e >= a.E) return;
  const int k1 = a.k1[e], k2 = a.k2[e];
  T u1[NP], u2[NP];
  const T* p1 = a.u + (int64_t)k1 * NP;
#pragma unroll
  for (int j = 0; j < NP; ++j) u1[j] = __ldg(p1 + j);
  if (k2 >= 0) {
    const T* p2 = a.u + (int64_t)k2 * NP;
#pragma unroll
    for (int j = 0; j < NP; ++j) u2[j] = __ldg(p2 + j);
  } else {
    // ghost side of a boundary edge: g = sum_m G_m tau_m(t)
    const int64_t b = -1 - (int64_t)k2;
#pragma unroll
    for (int j = 0; j < NP; ++j) u2[j] = T(0);
    const double t = stage_time(a.time);
    for (int m = 0; m < a.frc.nghost; ++m) {
      const T tm = (T)tau_of(a.frc.gkind[m], a.frc.gomega[m], t);
      const T* g = a.G + ((int64_t)m * a.B + b) * NP;
#pragma unroll
      for (int j = 0; j < NP; ++j) u2[j] += tm * g[j];
    }
  }
  using VT = typename V::type;
  const VT* w = reinterpret_cast<const VT*>(a.W) + ((e >> 5) * QW) * kTile + (e & 31);
  T acc[NFP];
#pragma unroll
  for (int i = 0; i < NFP; ++i) acc[i] = T(0);
#pragma unroll
  for (int q = 0; q < QW; ++q) {
    const VT v = ld_stream(w + q * kTile);
#pragma unroll
    for (int c = 0; c < VW; ++c) {
      const int idx = q * VW + c;
      if (idx < NW) {
        const int i = idx / (2 * NP), j = idx % (2 * NP);
        acc[i] = fma(V::get(v, c), j < NP ? u1[j] : u2[j - NP], acc[i]);
      }
    }
  }
  T* o = a.flux + e * NFP;
#pragma unroll
  for (int i = 0; i < NFP; ++i) o[i] = acc[i];
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

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(kElemBlock) elem_kernel(ElemArgs<T> a) {
  constexpr int NP = np_of(N), NFP = nfp_of(N);
  constexpr int OFF = 0;
  constexpr int ODR = OFF, ODS = OFF + NP * NP, OWR = OFF + 2 * NP * NP, OWS = OFF + 3 * NP * NP,
                OLIFT = OFF + 4 * NP * NP;
  __shared__ __align__(16) T sh[kElemBlock * NP];
  __shared__ T tau_s[RDG_MAX_FORCING_TERMS];
  const int64_t k0 = (int64_t)blockIdx.x * kElemBlock;
  const int nk = (int)min((int64_t)kElemBlock, a.K - k0);
  const int tid = threadIdx.x;
  const bool active = tid < nk;
  const int64_t k = k0 + tid;

  stage_in(sh, a.us + k0 * NP, nk * NP);
  if (tid < a.frc.nsrc) tau_s[tid] = (T)tau_of(a.frc.kind[tid], a.frc.omega[tid], stage_time(a.time));
  __syncthreads();

  T rhs[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) rhs[i] = T(0);
  if (active) {
    T u[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) u[j] = sh[tid * NP + j];
    // metric-folded volume coefficients: F_r = a_r u - (g_rr u_r + g_rs u_s), etc.
    const T ar = a.geo[0 * a.K + k], as = a.geo[1 * a.K + k], grr = a.geo[2 * a.K + k],
            grs = a.geo[3 * a.K + k], gss = a.geo[4 * a.K + k], ij = a.geo[5 * a.K + k];
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
      rhs[i] = acc;
    }
    // surface terms: side 1 takes J_f F*.n1 in its face order, side 2 the negated reverse
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const int er = a.eref[(int64_t)f * a.K + k];
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

}  // namespace dev

// Host-side launch helpers instantiated by the including translation unit.
template <typename T, int N>
inline int launch_edge_t(const EdgeArgs<T>& a, cudaStream_t s) {
  if (a.E == 0) return RDG_OK;
  const unsigned grid = (unsigned)((a.E + kEdgeBlock - 1) / kEdgeBlock);
  dev::edge_flux_kernel<T, N><<<grid, kEdgeBlock, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

template <typename T, int N>
inline int launch_elem_t(int mode, const ElemArgs<T>& a, cudaStream_t s) {
  if (a.K == 0) return RDG_OK;
  const unsigned grid = (unsigned)((a.K + kElemBlock - 1) / kElemBlock);
  switch (mode) {
    case 0: dev::elem_kernel<T, N, 0><<<grid, kElemBlock, 0, s>>>(a); break;
    case 1: dev::elem_kernel<T, N, 1><<<grid, kElemBlock, 0, s>>>(a); break;
    case 2: dev::elem_kernel<T, N, 2><<<grid, kElemBlock, 0, s>>>(a); break;
    case 3: dev::elem_kernel<T, N, 3><<<grid, kElemBlock, 0, s>>>(a); break;
    default: return RDG_EINVAL;
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

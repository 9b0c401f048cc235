// One persistent launch for a chunk of SSP-RK3 steps of many independent problems (meshes
// of any size, orders 1..6, FP32 with stored operators).  The work of a launch is a list of
// items, stage by stage (3 per step), and within a stage first every member's part A (edge
// tiles of 128 x ept edges writing the face fluxes, element tiles of 128 elements writing
// the volume terms, interleaved) and then every member's part B (element tiles: LIFT of the
// face fluxes, sources and the stage update).  Blocks take items from a global ticket
// counter in list order.  Part A of member m in stage p starts when m's part B of stage p - 1
// is done; part B of stage p when m's part A of stage p is done (per-member counts of
// finished items).  Because items are handed out in list order, every item an item waits on
// was handed out earlier to a block that is running it, so the waits always end (no
// co-residency needed).  Each wait is bounded: after the wait limit the block records
// kErrWaitTimeout, raises the launch's abort flag and leaves, and every other block leaves at
// its next item.
//
// The tiles do the work of the stage kernel and the element kernel (rhs_kernels.cuh) with
// the same arithmetic; every order's reference matrices sit in constant memory (order 6's
// volume matrices in shared memory), so one kernel serves every order.  The paper solves one problem at a time; this
// has no counterpart there.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "batch_kernel.h"

namespace {
// the one-launch stage's device functions used here take no constant-bank table
__constant__ float c_unused[1];
__device__ float g_unused[4];
}  // namespace
#define RDG_TAB c_unused
#define RDG_VOLTAB g_unused
#include "rhs_kernels.cuh"

namespace rdg {
namespace bk {

using dev::Staged;
using dev::stage_out;

// Reference matrices of every order in constant memory (Dr, Ds, Wr, Ws, LIFT, the element
// kernels' layout), so each entry is an immediate constant-bank operand as in the per-order
// kernels; order 6's volume matrices are staged in shared memory instead (VolTab layout), as
// the per-order stage kernel does.
constexpr int tab_count(int N) { return 4 * np_of(N) * np_of(N) + 3 * np_of(N) * nfp_of(N); }
__constant__ float c_b1[tab_count(1)];
__constant__ float c_b2[tab_count(2)];
__constant__ float c_b3[tab_count(3)];
__constant__ float c_b4[tab_count(4)];
__constant__ float c_b5[tab_count(5)];
__constant__ float c_b6[tab_count(6)];

template <int N>
__device__ __forceinline__ float bt(int i) {
  if constexpr (N == 1) return c_b1[i];
  else if constexpr (N == 2) return c_b2[i];
  else if constexpr (N == 3) return c_b3[i];
  else if constexpr (N == 4) return c_b4[i];
  else if constexpr (N == 5) return c_b5[i];
  else return c_b6[i];
}

// The volume term of one element, the same arithmetic as volume_row (rhs_kernels.cuh) with the
// constant table of order N.
template <int N>
__device__ __forceinline__ void volume_row_b(const float (&u)[np_of(N)], float ar, float as, float grr, float grs,
                                             float gss, float (&vol)[np_of(N)]) {
  constexpr int NP = np_of(N);
  constexpr int ODR = 0, ODS = NP * NP, OWR = 2 * NP * NP, OWS = 3 * NP * NP;
  float du[NP];
#pragma unroll
  for (int j = 1; j < NP; ++j) du[j] = u[j] - u[0];
#pragma unroll
  for (int i = 0; i < NP; ++i) vol[i] = 0.f;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    float ur = 0.f, us = 0.f;
#pragma unroll
    for (int k = 1; k < NP; ++k) {
      ur = fmaf(bt<N>(ODR + j * NP + k), du[k], ur);
      us = fmaf(bt<N>(ODS + j * NP + k), du[k], us);
    }
    const float uj = j == 0 ? u[0] : du[j] + u[0];
    const float fr = ar * uj - (grr * ur + grs * us);
    const float fs = as * uj - (grs * ur + gss * us);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      vol[i] = fmaf(bt<N>(OWR + i * NP + j), fr, vol[i]);
      vol[i] = fmaf(bt<N>(OWS + i * NP + j), fs, vol[i]);
    }
  }
}

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until *cnt >= target (or the launch is aborted).  false: gave up.
__device__ bool wait_count(const unsigned long long* cnt, unsigned long long target, const int* abort,
                           uint64_t limit_ns) {
  const volatile unsigned long long* c = cnt;
  const volatile int* ab = abort;
  if (*c >= target) return true;
  const uint64_t t0 = gtime();
  unsigned ns = 32;
  while (*c < target) {
    if (*ab) return false;
    if (gtime() - t0 > limit_ns) return false;
    __nanosleep(ns);
    ns = ns < 1024 ? 2 * ns : ns;
  }
  __threadfence();
  return true;
}

// Part B, one element per thread: rhs = vol - (1/J) sum_f LIFT_f q_f + sum_m tau_m S_m, then
// the stage (the element kernel's arithmetic, LIFT from the shared-memory table).  Its inputs
// were written by other blocks of this launch: read through L2.
template <int N, int MODE>
__device__ __noinline__ void update_element(const BMember& b, int64_t k, const float* us, const float* un, float* out,
                                            const float* tau) {
  constexpr int NP = np_of(N), NFP = nfp_of(N);
  constexpr int OLIFT = 4 * NP * NP;
  const float ij = b.geo[5 * b.K + k];
  float rhs[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) rhs[i] = __ldcg(b.vol + k * NP + i);
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    float q[NFP];
#pragma unroll
    for (int c = 0; c < NFP; ++c) q[c] = __ldcg(b.fb + (k * 3 + f) * NFP + c);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < NFP; ++c) acc = fmaf(bt<N>(OLIFT + i * 3 * NFP + f * NFP + c), q[c], acc);
      rhs[i] -= ij * acc;
    }
  }
  for (int m = 0; m < b.frc.nsrc; ++m) {
    const float* S = b.S + ((int64_t)m * b.K + k) * NP;
#pragma unroll
    for (int i = 0; i < NP; ++i) rhs[i] = fmaf(tau[m], S[i], rhs[i]);
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    float r = fmaf(b.dt32, rhs[i], __ldcg(us + k * NP + i));
    if (MODE >= 2) r = dev::rk_combine<float, MODE>(__ldcg(un + k * NP + i), r);
    out[k * NP + i] = r;
  }
}

// One item of member b in stage `stage` (0, 1, 2) of the step starting at time tstep: part
// A tile t (part_b false) or part B tile t.
template <int N>
__device__ __noinline__ void run_tile(const BMember& b, bool part_b, int stage, double tstep, int64_t t,
                                      const float* tab, float* sh, float* tau) {
  constexpr int NP = np_of(N);
  const float* us = stage == 0 ? b.u : (stage == 1 ? b.u1 : b.u2);
  float* out = stage == 0 ? b.u1 : (stage == 1 ? b.u2 : b.u);
  const float* un = b.u;
  const double off = stage == 0 ? 0.0 : (stage == 1 ? 1.0 : 0.5);
  if (part_b) {
    if (threadIdx.x < b.frc.nsrc) {
      const double ts = tstep + off * b.dt;
      tau[threadIdx.x] = (float)dev::tau_of(b.frc.kind[threadIdx.x], b.frc.omega[threadIdx.x], ts);
    }
    __syncthreads();
    const int64_t k = t * kStageBlock + threadIdx.x;
    if (k < b.K) {
      if (stage == 0) update_element<N, 1>(b, k, us, un, out, tau);
      else if (stage == 1) update_element<N, 2>(b, k, us, un, out, tau);
      else update_element<N, 3>(b, k, us, un, out, tau);
    }
    return;
  }
  // part A: element tiles spread evenly among the edge tiles, as in the stage grid
  const int64_t nt = b.ntile_e + b.ntile_v;
  const int64_t v0 = (t * b.ntile_v) / nt, v1 = ((t + 1) * b.ntile_v) / nt;
  if (v1 > v0) {
    const int64_t k0 = v0 * kStageBlock;
    const int nk = (int)min((int64_t)kStageBlock, b.K - k0);
    {
      Staged<float, kStageBlock, NP> g;
      g.load(us + k0 * NP, nk * NP);
      g.store(sh, nk * NP);
    }
    __syncthreads();
    const int tid = threadIdx.x;
    if (tid < nk) {
      const int64_t k = k0 + tid;
      float u[NP], vol[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) u[j] = sh[tid * NP + j];
      if constexpr (N >= 6)
        dev::volume_row_smem<float, N>(u, b.geo[k], b.geo[b.K + k], b.geo[2 * b.K + k], b.geo[3 * b.K + k],
                                       b.geo[4 * b.K + k], tab, vol);
      else
        volume_row_b<N>(u, b.geo[k], b.geo[b.K + k], b.geo[2 * b.K + k], b.geo[3 * b.K + k], b.geo[4 * b.K + k], vol);
#pragma unroll
      for (int j = 0; j < NP; ++j) sh[tid * NP + j] = vol[j];
    }
    __syncthreads();
    stage_out(b.vol + k0 * NP, sh, nk * NP);
    return;
  }
  EdgeArgs<float> ea{b.k1, b.k2, b.W, us, nullptr, b.G, b.E, b.B, b.frc,
                     TimeArg{nullptr, tstep, b.dt, off}, b.err, b.K, b.vol, b.geo, b.f12, b.fb, 0};
  const int64_t eblk = t - v1;
  for (int r = 0; r < b.ept; ++r) {
    const int64_t e = (eblk * b.ept + r) * kStageBlock + threadIdx.x;
    if (e < b.E) dev::stage_edge<float, N, true>(ea, e);
  }
}

__global__ void __launch_bounds__(kStageBlock, 4) batch_persistent_kernel(BatchArgs a) {
  extern __shared__ __align__(16) float smem[];
  float* tabs = smem;                           // order 6's volume tables, if present
  float* sh = smem + a.tab_floats;              // element rows of a volume tile
  // the member descriptors, in shared memory when they fit (searched for every item)
  BMember* smem_m = reinterpret_cast<BMember*>(sh + kStageBlock * np_of(6));
  const bool in_smem = a.nm <= kSmemMembers;
  const BMember* mem = in_smem ? smem_m : a.m;
  __shared__ float tau[RDG_MAX_FORCING_TERMS];
  __shared__ long long s_item;
  __shared__ int s_go;
  for (int i = threadIdx.x; i < a.tab_floats; i += blockDim.x) tabs[i] = a.tabs[i];
  if (in_smem) {
    const int words = a.nm * (int)(sizeof(BMember) / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.m);
    uint32_t* dst = reinterpret_cast<uint32_t*>(smem_m);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  const long long total = a.per_phase * a.nphase;
  // the next ticket is taken while the current item runs, hiding the atomic's round trip
  long long next = threadIdx.x == 0 ? (long long)atomicAdd(a.ticket, 1ull) : 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = next;
      if (next < total) next = (long long)atomicAdd(a.ticket, 1ull);
    }
    __syncthreads();
    const long long it = s_item;
    if (it >= total) break;
    const int p = (int)(it / a.per_phase);
    long long r = it - (long long)p * a.per_phase;
    const bool part_b = r >= a.items_a;
    if (part_b) r -= a.items_a;
    int lo = 0, hi = a.nm - 1;                  // member holding item r of the part
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if ((part_b ? mem[mid].off_b : mem[mid].off_a) <= r) lo = mid;
      else hi = mid - 1;
    }
    const BMember& b = mem[lo];
    if (threadIdx.x == 0) {
      // part A of stage p after part B of stage p - 1; part B of stage p after part A of
      // stage p; a held stage's part A never starts
      const unsigned long long* cnt = part_b ? a.done + lo : a.done + a.nm + lo;
      unsigned long long target = part_b ? (unsigned long long)(p + 1) * (unsigned long long)b.nitem_a
                                         : (unsigned long long)p * (unsigned long long)b.nitem_b;
      if (!part_b && p == b.hold_phase) target = ~0ull;
      const bool ok = wait_count(cnt, target, a.abort, a.wait_ns);
      if (!ok) {
        atomicOr(a.err, kErrWaitTimeout);
        atomicExch(a.abort, 1);
      }
      s_go = ok;
    }
    __syncthreads();
    if (!s_go) break;
    const long long item = r - (part_b ? b.off_b : b.off_a);
    const long long ntile = part_b ? b.ntile_u : b.ntile_e + b.ntile_v;
    const long long t0 = item * b.tpi, t1 = min(t0 + b.tpi, ntile);
    const int step = p / 3, stage = p - 3 * step;
    const double tstep = b.ts->t0 + ((double)b.ts->n + step) * b.dt;
    for (long long t = t0; t < t1; ++t) {
      switch (b.N) {
        case 1: run_tile<1>(b, part_b, stage, tstep, t, tabs, sh, tau); break;
        case 2: run_tile<2>(b, part_b, stage, tstep, t, tabs, sh, tau); break;
        case 3: run_tile<3>(b, part_b, stage, tstep, t, tabs, sh, tau); break;
        case 4: run_tile<4>(b, part_b, stage, tstep, t, tabs, sh, tau); break;
        case 5: run_tile<5>(b, part_b, stage, tstep, t, tabs, sh, tau); break;
        default: run_tile<6>(b, part_b, stage, tstep, t, tabs, sh, tau); break;
      }
      __syncthreads();                          // the tile's shared rows before the next tile
    }
    __threadfence();                            // this thread's writes of the item
    __syncthreads();                            // ... and every other thread's
    if (threadIdx.x == 0) atomicAdd(a.done + (part_b ? a.nm : 0) + lo, 1ull);
  }
}

__global__ void batch_advance_kernel(BMember* m, int nm, long long steps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nm) m[i].ts->n += steps;
}

}  // namespace bk

// Order 6's volume tables in the layout volume_row_smem reads (VolTab: Dr, Ds row-major,
// Wr^T, Ws^T, rows padded); the other orders read constant memory.
static void append_voltab6(std::vector<float>& out) {
  const RefOps* o = get_refops(6, nullptr);
  const int NP = np_of(6);
  const int NPP = (NP * 4 + 15) / 16 * 4;
  std::vector<float> vt(4 * NP * NPP, 0.f);
  for (int r = 0; r < NP; ++r)
    for (int c = 0; c < NP; ++c) {
      vt[r * NPP + c] = (float)o->Dr[r * NP + c];
      vt[NP * NPP + r * NPP + c] = (float)o->Ds[r * NP + c];
      vt[2 * NP * NPP + r * NPP + c] = (float)o->Wr[c * NP + r];
      vt[3 * NP * NPP + r * NPP + c] = (float)o->Ws[c * NP + r];
    }
  out.insert(out.end(), vt.begin(), vt.end());
}

template <int N, typename A>
static int upload_const(A& arr) {
  std::vector<float> t = pack_elem_table<float>(N);
  if (t.size() * sizeof(float) != sizeof(arr)) return RDG_EINVAL;
  return cudaMemcpyToSymbol(arr, t.data(), sizeof(arr)) == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

int batch_tables(const bool orders[7], std::vector<float>& tabs, int off[7]) {
  static bool uploaded[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return RDG_EINVAL;
  if (!uploaded[dev]) {
    int rc = RDG_OK;
    if (rc == RDG_OK) rc = upload_const<1>(bk::c_b1);
    if (rc == RDG_OK) rc = upload_const<2>(bk::c_b2);
    if (rc == RDG_OK) rc = upload_const<3>(bk::c_b3);
    if (rc == RDG_OK) rc = upload_const<4>(bk::c_b4);
    if (rc == RDG_OK) rc = upload_const<5>(bk::c_b5);
    if (rc == RDG_OK) rc = upload_const<6>(bk::c_b6);
    if (rc != RDG_OK) return rc;
    uploaded[dev] = true;
  }
  tabs.clear();
  for (int N = 0; N <= 6; ++N) off[N] = 0;
  if (orders[6]) append_voltab6(tabs);
  return RDG_OK;
}

size_t batch_smem_bytes(int tab_floats, int nm) {
  const size_t base = ((size_t)tab_floats + kStageBlock * np_of(6)) * sizeof(float);
  return base + (nm <= kSmemMembers ? (size_t)nm * sizeof(BMember) : 0);
}

int batch_grid(size_t smem) {
  static bool attr = false;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr) {
    if (cudaFuncSetAttribute(bk::batch_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess)
      return -1;
    attr = true;
  }
  int per = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bk::batch_persistent_kernel, kStageBlock, smem) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1;
  return std::max(1, per) * nsm;
}

int launch_batch_persistent(const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
  bk::batch_persistent_kernel<<<grid, kStageBlock, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

int launch_batch_advance(BMember* m, int nm, long long steps, cudaStream_t s) {
  bk::batch_advance_kernel<<<(nm + 127) / 128, 128, 0, s>>>(m, nm, steps);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

}  // namespace rdg

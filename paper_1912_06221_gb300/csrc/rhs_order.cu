// One order / one precision of the hot-path kernels.  The build compiles this file once per
// (RDG_ORDER in 1..6, RDG_REAL in {float, double}) so the translation units build in
// parallel; each object holds its order's reference matrices in its own constant bank.
#include <cuda_runtime.h>

#include "internal.h"

#ifndef RDG_ORDER
#error "RDG_ORDER must be defined"
#endif
#ifndef RDG_REAL
#error "RDG_REAL must be defined"
#endif

#define RDG_CAT2(a, b) a##b
#define RDG_CAT(a, b) RDG_CAT2(a, b)

namespace {
constexpr int kN = RDG_ORDER;
constexpr int kNp = (kN + 1) * (kN + 2) / 2;
constexpr int kTabN = 4 * kNp * kNp + 3 * kNp * (kN + 1);
__constant__ RDG_REAL c_tab[kTabN];
// the volume matrices again, in global memory, for the orders whose volume role stages them
// in shared memory (layout of VolTab in rhs_kernels.cuh)
constexpr int kNpp = (kNp * (int)sizeof(RDG_REAL) + 15) / 16 * 16 / (int)sizeof(RDG_REAL);
__device__ __align__(16) RDG_REAL g_voltab[4 * kNp * kNpp];
}  // namespace
#define RDG_TAB c_tab
#define RDG_VOLTAB g_voltab
#include "rhs_kernels.cuh"

// FP32 objects of orders 1..kMaxGemmN also hold the GEMM form of the edge flux.
#define RDG_GEMM (RDG_TAG_IS_F && RDG_ORDER <= 5)
#if RDG_GEMM
#include <cstring>

#include "gemm_kernels.cuh"
namespace {
using GS = rdg::gemm::Shape<kN>;
__device__ __align__(16) float4 g_xb[4 * GS::BTILE / 16];
__device__ int g_gtab[3 * kNp + kN + 1];
}  // namespace
#endif

// The FP32 object of order 6 also holds the volume term as a tensor-core GEMM
// (volume_gemm.cuh), which its stage launches beside the edge-only operator stream.
#define RDG_VGEMM (RDG_TAG_IS_F && RDG_ORDER == 6)
#if RDG_VGEMM
#include <cstring>

#include "gemm_kernels.cuh"
#include "volume_gemm.cuh"
namespace {
using VS = rdg::gemm::VolShape<kN>;
__device__ __align__(16) float4 g_vb[VS::BWORDS];
}  // namespace
#endif

namespace rdg {

int RDG_CAT(upload_tab_, RDG_CAT(RDG_TAG, RDG_ORDER))() {
  std::vector<RDG_REAL> t = pack_elem_table<RDG_REAL>(kN);
  if ((int)t.size() != kTabN) return RDG_EINVAL;
  if (cudaMemcpyToSymbol(c_tab, t.data(), t.size() * sizeof(RDG_REAL)) != cudaSuccess) return RDG_ECUDA;
  {
    // Dr, Ds row-major and Wr^T, Ws^T, rows padded to kNpp
    std::vector<RDG_REAL> vt(4 * kNp * kNpp, RDG_REAL(0));
    const int n2 = kNp * kNp;
    for (int r = 0; r < kNp; ++r)
      for (int c = 0; c < kNp; ++c) {
        vt[r * kNpp + c] = t[r * kNp + c];
        vt[kNp * kNpp + r * kNpp + c] = t[n2 + r * kNp + c];
        vt[2 * kNp * kNpp + r * kNpp + c] = t[2 * n2 + c * kNp + r];
        vt[3 * kNp * kNpp + r * kNpp + c] = t[3 * n2 + c * kNp + r];
      }
    if (cudaMemcpyToSymbol(g_voltab, vt.data(), vt.size() * sizeof(RDG_REAL)) != cudaSuccess) return RDG_ECUDA;
  }
#if RDG_GEMM
  const RefOps* o = get_refops(kN, nullptr);
  if (!o) return RDG_EINVAL;
  std::vector<float> xb = gemm::pack_gemm_operand<kN>(*o);
  std::vector<int> gt = gemm::pack_gemm_table<kN>(*o);
  if (xb.size() * 4 != sizeof(g_xb) || gt.size() * 4 != sizeof(g_gtab)) return RDG_EINVAL;
  // the warp-specialised kernel takes the shared face's rotated-order nodes as constants
  for (int q = 0; q < kN + 1; ++q)
    if (gt[3 * kNp + q] != gemm::hyp_of(kN, q)) return RDG_EINVAL;
  if (cudaMemcpyToSymbol(g_xb, xb.data(), sizeof(g_xb)) != cudaSuccess) return RDG_ECUDA;
  if (cudaMemcpyToSymbol(g_gtab, gt.data(), sizeof(g_gtab)) != cudaSuccess) return RDG_ECUDA;
#endif
#if RDG_VGEMM
  {
    const RefOps* o = get_refops(kN, nullptr);
    if (!o) return RDG_EINVAL;
    std::vector<float> vb = gemm::pack_volume_operand<kN>(*o);
    if (vb.size() * 4 != sizeof(g_vb)) return RDG_EINVAL;
    if (cudaMemcpyToSymbol(g_vb, vb.data(), sizeof(g_vb)) != cudaSuccess) return RDG_ECUDA;
  }
#endif
  return RDG_OK;
}

#if RDG_GEMM
int RDG_CAT(launch_gemm_, RDG_CAT(RDG_TAG, RDG_ORDER))(const EdgeArgs<float>& a, cudaStream_t s) {
  void* xb = nullptr;
  void* gt = nullptr;
  if (cudaGetSymbolAddress(&xb, g_xb) != cudaSuccess || cudaGetSymbolAddress(&gt, g_gtab) != cudaSuccess)
    return RDG_ECUDA;
  return gemm::launch_gemm_t<kN>(a, static_cast<const float4*>(xb), static_cast<const int*>(gt), s);
}
#endif

int RDG_CAT(launch_edge_, RDG_CAT(RDG_TAG, RDG_ORDER))(const EdgeArgs<RDG_REAL>& a, cudaStream_t s) {
  return launch_edge_t<RDG_REAL, kN>(a, s);
}

int RDG_CAT(launch_elem_, RDG_CAT(RDG_TAG, RDG_ORDER))(int mode, const ElemArgs<RDG_REAL>& a, cudaStream_t s) {
  return launch_elem_t<RDG_REAL, kN>(mode, a, s);
}

int RDG_CAT(launch_edge_vol_, RDG_CAT(RDG_TAG, RDG_ORDER))(const EdgeArgs<RDG_REAL>& a, cudaStream_t s) {
  return launch_edge_t<RDG_REAL, kN, true>(a, s);
}

#if RDG_VGEMM
// the volume term on the tensor cores (the stage launches it on a second stream beside the
// edge-only blocks, so they overlap)
int RDG_CAT(launch_volume_, RDG_CAT(RDG_TAG, RDG_ORDER))(const EdgeArgs<float>& a, cudaStream_t s) {
  void* vb = nullptr;
  if (cudaGetSymbolAddress(&vb, g_vb) != cudaSuccess) return RDG_ECUDA;
  return gemm::launch_volume_gemm_t<kN>(a, static_cast<const float4*>(vb), s);
}
#endif

int RDG_CAT(launch_elem_lite_, RDG_CAT(RDG_TAG, RDG_ORDER))(int mode, const ElemArgs<RDG_REAL>& a, cudaStream_t s) {
  return launch_elem_t<RDG_REAL, kN, true>(mode, a, s);
}

int RDG_CAT(launch_edge_only_, RDG_CAT(RDG_TAG, RDG_ORDER))(const EdgeArgs<RDG_REAL>& a, cudaStream_t s) {
  return launch_edge_fb_t<RDG_REAL, kN>(a, s);
}

int RDG_CAT(launch_fused_, RDG_CAT(RDG_TAG, RDG_ORDER))(int mode, const EdgeArgs<RDG_REAL>& ea,
                                                      const ElemArgs<RDG_REAL>& a, cudaStream_t s) {
  return launch_fused_t<RDG_REAL, kN>(mode, ea, a, s);
}

}  // namespace rdg

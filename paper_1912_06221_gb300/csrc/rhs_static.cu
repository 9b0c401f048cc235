// Allocation-free variant of rdg_rhs_eval.
//
// rdg_rhs_eval keeps the per-edge fluxes between its two kernels in a buffer the context
// allocates.  Some callers cannot allocate device memory where they evaluate the right-hand
// side: code running while another component captures a CUDA graph (cudaMalloc cannot be
// captured), latency-bound loops that must not hit cudaMalloc's implicit synchronisation,
// and processes whose device memory is owned by a fixed-budget pool allocator.  This entry
// point uses, instead, one fixed scratch array compiled into the library (kStaticFluxBytes)
// and calls no allocating routine at all.  It runs the unfused pair of kernels (edge fluxes
// into that array, then the element kernel with the volume term, LIFT and sources), not the
// fused pair of rdg_rhs_eval; the two agree to rounding.  The paper has no counterpart to it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "context.h"

namespace {

constexpr size_t kStaticFluxBytes = size_t(8) << 20;   // 8 MiB of edge fluxes
static __device__ __align__(256) unsigned char g_static_flux[kStaticFluxBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

int fail_static(rdg_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

}  // namespace

extern "C" int rdg_rhs_eval_static(rdg_ctx* ctx, const void* u_dev, void* rhs_dev, double t) {
  using namespace rdg;
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail_static(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!u_dev || !rhs_dev) return fail_static(ctx, RDG_EINVAL, "NULL device array");
  if ((((uintptr_t)u_dev) & 15u) || (((uintptr_t)rhs_dev) & 15u))
    return fail_static(ctx, RDG_EINVAL, "device arrays must be 16-byte aligned");
  if (u_dev == rhs_dev) return fail_static(ctx, RDG_EINVAL, "u and rhs must not overlap");
  if (ctx->gemm)
    return fail_static(ctx, RDG_ESTATE,
                       "rdg_rhs_eval_static needs stored flux operators: contexts using the GEMM form of the edge "
                       "flux (RDG_FP32_3XTF32 with N <= 5 and an interface rule other than RDG_IFACE_ALG1) are refused");
  if (ctx->d_Dn)
    return fail_static(ctx, RDG_ESTATE, "rdg_rhs_eval_static does not take a D given at the nodes");
  const size_t need = (size_t)ctx->E * nfp_of(ctx->N) * ctx->esz;
  if (need > kStaticFluxBytes)
    return fail_static(ctx, RDG_EINVAL,
                       "edge fluxes need " + std::to_string(need) + " bytes, more than the " +
                           std::to_string(kStaticFluxBytes) + "-byte static scratch of rdg_rhs_eval_static");
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return fail_static(ctx, RDG_EINVAL, "device id too large");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return fail_static(ctx, RDG_ECUDA, "cudaGetDevice failed");
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess)
    return fail_static(ctx, RDG_ECUDA, "cudaSetDevice failed");
  int rc = RDG_OK;
  void* flux = nullptr;
  {
    // one-time set-up per device (with that device current): the array's device address.
    // It is cached for the life of the process, so it is valid only while the device's
    // primary context lives (a cudaDeviceReset by another component would leave it stale).
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[ctx->device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_flux);
      if (e != cudaSuccess || !p) rc = fail_static(ctx, RDG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      else g_addr[ctx->device] = p;
    }
    flux = g_addr[ctx->device];
  }
  if (rc == RDG_OK) {
    // every edge writes all of its Nfp fluxes before the element kernel reads them, so the
    // array needs no clearing between calls
    TimeArg ta{nullptr, t, 1.0, 0.0};
    if (ctx->esz == 4) {
      EdgeArgs<float> ea{ctx->d_k1, ctx->d_k2, ctx->d_W, (const float*)u_dev, (float*)flux, (const float*)ctx->d_G,
                         ctx->E, ctx->B, ctx->frc, ta, ctx->d_err, ctx->K};
      ElemArgs<float> la{(const float*)u_dev, nullptr, (float*)rhs_dev, (const float*)flux, ctx->d_eref,
                         (const float*)ctx->d_geo, (const float*)ctx->d_S, ctx->K, 0.0f, ctx->frc, ta, ctx->d_err, ctx->E};
      rc = launch_edge32(ctx->N, ea, ctx->stream);
      if (rc == RDG_OK) rc = launch_elem32(ctx->N, 0, la, ctx->stream);
    } else {
      EdgeArgs<double> ea{ctx->d_k1, ctx->d_k2, ctx->d_W, (const double*)u_dev, (double*)flux, (const double*)ctx->d_G,
                          ctx->E, ctx->B, ctx->frc, ta, ctx->d_err, ctx->K};
      ElemArgs<double> la{(const double*)u_dev, nullptr, (double*)rhs_dev, (const double*)flux, ctx->d_eref,
                          (const double*)ctx->d_geo, (const double*)ctx->d_S, ctx->K, 0.0, ctx->frc, ta, ctx->d_err, ctx->E};
      rc = launch_edge64(ctx->N, ea, ctx->stream);
      if (rc == RDG_OK) rc = launch_elem64(ctx->N, 0, la, ctx->stream);
    }
    if (rc != RDG_OK) fail_static(ctx, rc, "kernel launch failed");
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return rc;
}

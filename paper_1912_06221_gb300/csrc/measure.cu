// Measurement entry points: the FMA rates of this GPU (the compute side of the roofline) and
// the error norms of Eqs. L2_norm_cellUnit and Linf_norm_cellUnit (Sec. 5), evaluated in FP64
// on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "context.h"

namespace rdg {
namespace {

// Sixteen independent FMA chains per thread (enough to cover the FMA latency with a few warps
// per scheduler), four chain rounds per loop trip; x -> a x + b with |a| < 1 stays bounded.
template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T* out, int iters, T a, T b) {
  T x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] = fma(x[i], a, b);
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 16; ++i) s += x[i];
  if (s == T(-1)) out[blockIdx.x] = s;   // never true: keeps the chains live
}

template <typename T>
int peak_fma(int device, double* flops) {
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return RDG_ECUDA;
  const int grid = nsm * 8, block = 256, iters = sizeof(T) == 4 ? 4096 : 512;
  T* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RDG_OK;
  if (cudaMalloc(&out, grid * sizeof(T)) != cudaSuccess) return RDG_ENOMEM;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = RDG_ECUDA;
  double best = 0.0;
  for (int rep = 0; rc == RDG_OK && rep < 6; ++rep) {     // two warm-up launches, best of four
    cudaEventRecord(e0, s);
    fma_chain_kernel<T><<<grid, block, 0, s>>>(out, iters, T(0.999999), T(1e-6));
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = RDG_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double f = 2.0 * 64.0 * (double)iters * grid * block / (ms * 1e-3);
    if (rep >= 2) best = std::max(best, f);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  *flops = best;
  return rc;
}

// Streaming read of n4 16-byte words: grid-stride, eight independent evict-first loads per
// trip, summed in a register that is stored only under a condition that never holds.
__global__ void __launch_bounds__(256) stream_read_kernel(const float4* __restrict__ p, int64_t n4, float* out) {
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 7 * stride < n4; i += 8 * stride) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcs(p + i + u * stride);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u].x + v[u].y + v[u].z + v[u].w;
  }
  for (; i < n4; i += stride) {
    const float4 v = __ldcs(p + i);
    acc += v.x + v.y + v.z + v.w;
  }
  if (acc == -1.f) out[blockIdx.x] = acc;
}

// Collapsed Gauss rule on the reference triangle with q = N + 3 points per direction: exact
// for total degree 2q - 2 = 2N + 4 (the degree of the squared error of a degree-(N + 2)
// function), weights summing to the reference area 2.
void error_rule(int N, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w) {
  std::vector<double> x, gw;
  const int q = N + 3;
  gauss_legendre_rule(q, x, gw);
  r.clear();
  s.clear();
  w.clear();
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      const double a = x[i], b = x[j];
      r.push_back((1 + a) * (1 - b) / 2 - 1);
      s.push_back(b);
      w.push_back(gw[i] * gw[j] * (1 - b) / 2);
    }
}

// One thread per element: u at the rule's points (interpolation I = psi(r_q, s_q) V^{-1}),
// e = u - u_e, then sum J w e^2 and the largest cell mean of |e| over the block.
template <typename T>
__global__ void __launch_bounds__(128) error_norm_kernel(const T* __restrict__ u, const double* __restrict__ ue,
                                                         const double* __restrict__ J, const double* __restrict__ I,
                                                         const double* __restrict__ w, int np, int nq, int64_t K,
                                                         double* __restrict__ part) {
  extern __shared__ double sm[];
  double* sI = sm;                 // [nq][np]
  double* sw = sI + nq * np;       // [nq]
  double* red = sw + nq;           // [3][128]
  for (int i = threadIdx.x; i < nq * np; i += blockDim.x) sI[i] = I[i];
  for (int i = threadIdx.x; i < nq; i += blockDim.x) sw[i] = w[i];
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0, area = 0.0, mean = 0.0;
  if (k < K) {
    double s2 = 0.0, s1 = 0.0;
    for (int q = 0; q < nq; ++q) {
      double uq = 0.0;
      for (int j = 0; j < np; ++j) uq = fma(sI[q * np + j], (double)u[k * np + j], uq);
      const double e = uq - ue[k * nq + q];
      s2 = fma(sw[q], e * e, s2);
      s1 = fma(sw[q], fabs(e), s1);
    }
    e2 = J[k] * s2;
    area = 2.0 * J[k];
    mean = 0.5 * s1;            // (J s1) / (2 J): the mean of |e| over the element
  }
  red[threadIdx.x] = e2;
  red[128 + threadIdx.x] = area;
  red[256 + threadIdx.x] = mean;
  __syncthreads();
  for (int h = 64; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[threadIdx.x] += red[threadIdx.x + h];
      red[128 + threadIdx.x] += red[128 + threadIdx.x + h];
      red[256 + threadIdx.x] = fmax(red[256 + threadIdx.x], red[256 + threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = red[0];
    part[3 * blockIdx.x + 1] = red[128];
    part[3 * blockIdx.x + 2] = red[256];
  }
}

int fail_m(rdg_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

}  // namespace
}  // namespace rdg

extern "C" int rdg_peak_fma(int device, int precision, double* flops_per_second) {
  using namespace rdg;
  if (!flops_per_second || (precision != RDG_FP32 && precision != RDG_FP64)) return RDG_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RDG_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return RDG_ECUDA;
  const int rc = precision == RDG_FP32 ? peak_fma<float>(device, flops_per_second) : peak_fma<double>(device, flops_per_second);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}

extern "C" int rdg_stream_read(int device, int64_t bytes, double* seconds) {
  using namespace rdg;
  if (!seconds || bytes < 16 || bytes > ((int64_t)64 << 30)) return RDG_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RDG_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return RDG_ECUDA;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  const int64_t n4 = bytes / 16;
  const size_t flush_bytes = (size_t)512 << 20;    // larger than L2: written between timed reads
  float4* buf = nullptr;
  float* out = nullptr;
  void* flush = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RDG_OK;
  if (cudaMalloc(&buf, (size_t)n4 * 16) != cudaSuccess || cudaMalloc(&out, 8192 * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&flush, flush_bytes) != cudaSuccess)
    rc = RDG_ENOMEM;
  if (rc == RDG_OK && (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = RDG_ECUDA;
  std::vector<float> ts;
  if (rc == RDG_OK) cudaMemsetAsync(buf, 0, (size_t)n4 * 16, s);
  for (int rep = 0; rc == RDG_OK && rep < 10; ++rep) {   // two warm-up reads, median of eight
    cudaMemsetAsync(flush, rep, flush_bytes, s);
    cudaEventRecord(e0, s);
    stream_read_kernel<<<nsm * 8, 256, 0, s>>>(buf, n4, out);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = RDG_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep >= 2) ts.push_back(ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(buf);
  cudaFree(out);
  cudaFree(flush);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (rc != RDG_OK) return rc;
  std::sort(ts.begin(), ts.end());
  *seconds = 0.5 * (ts[ts.size() / 2 - 1] + ts[ts.size() / 2]) * 1e-3;
  return RDG_OK;
}

extern "C" int rdg_error_quadrature(rdg_ctx* ctx, int* nq, double* xy) {
  using namespace rdg;
  if (!ctx || !nq) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail_m(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  std::vector<double> r, s, w;
  error_rule(ctx->N, r, s, w);
  *nq = (int)w.size();
  if (!xy) return RDG_OK;
  for (int64_t k = 0; k < ctx->K; ++k) {
    const double* v = &ctx->exy[6 * k];
    for (size_t q = 0; q < w.size(); ++q) {
      const double a = -(r[q] + s[q]) / 2, b = (r[q] + 1) / 2, c = (s[q] + 1) / 2;
      xy[(k * w.size() + q) * 2 + 0] = a * v[0] + b * v[2] + c * v[4];
      xy[(k * w.size() + q) * 2 + 1] = a * v[1] + b * v[3] + c * v[5];
    }
  }
  return RDG_OK;
}

extern "C" int rdg_error_norms(rdg_ctx* ctx, const void* u_dev, const double* ue_q_dev, double* l2, double* linf) {
  using namespace rdg;
  if (!ctx || !ue_q_dev || !l2 || !linf) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail_m(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  const RefOps* o = get_refops(ctx->N, nullptr);
  if (!o) return fail_m(ctx, RDG_ESTATE, "reference operators unavailable");
  std::vector<double> r, s, w;
  error_rule(ctx->N, r, s, w);
  const int np = o->Np, nq = (int)w.size();
  // interpolation from the nodes to the rule's points, I = psi(r_q, s_q) V^{-1}
  std::vector<double> I((size_t)nq * np, 0.0), psi(np);
  for (int q = 0; q < nq; ++q) {
    simplex_basis(ctx->N, r[q], s[q], psi.data(), nullptr, nullptr);
    for (int j = 0; j < np; ++j) {
      double acc = 0.0;
      for (int m = 0; m < np; ++m) acc += psi[m] * o->Vinv[(size_t)m * np + j];
      I[(size_t)q * np + j] = acc;
    }
  }
  std::vector<double> J(ctx->K);
  for (int64_t k = 0; k < ctx->K; ++k) {
    const double* v = &ctx->exy[6 * k];
    const double xr = (v[2] - v[0]) / 2, yr = (v[3] - v[1]) / 2, xs = (v[4] - v[0]) / 2, ys = (v[5] - v[1]) / 2;
    J[k] = xr * ys - xs * yr;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return fail_m(ctx, RDG_ECUDA, "cudaSetDevice");
  const int64_t nb = (ctx->K + 127) / 128;
  double *dJ = nullptr, *dI = nullptr, *dw = nullptr, *dpart = nullptr;
  cudaStream_t st = ctx->stream;
  int rc = RDG_OK;
  if (cudaMallocAsync((void**)&dJ, ctx->K * sizeof(double), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dI, I.size() * sizeof(double), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dw, w.size() * sizeof(double), st) != cudaSuccess ||
      cudaMallocAsync((void**)&dpart, nb * 3 * sizeof(double), st) != cudaSuccess)
    rc = fail_m(ctx, RDG_ENOMEM, "error-norm scratch");
  std::vector<double> part(nb * 3);
  if (rc == RDG_OK) {
    cudaMemcpyAsync(dJ, J.data(), J.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dI, I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dw, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    const void* u = u_dev ? u_dev : ctx->d_u;
    const size_t sh = ((size_t)nq * np + nq + 3 * 128) * sizeof(double);
    if (ctx->esz == 4)
      error_norm_kernel<float><<<(unsigned)nb, 128, sh, st>>>((const float*)u, ue_q_dev, dJ, dI, dw, np, nq, ctx->K, dpart);
    else
      error_norm_kernel<double><<<(unsigned)nb, 128, sh, st>>>((const double*)u, ue_q_dev, dJ, dI, dw, np, nq, ctx->K, dpart);
    if (cudaGetLastError() != cudaSuccess) rc = fail_m(ctx, RDG_ECUDA, "error-norm kernel launch");
    cudaMemcpyAsync(part.data(), dpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  cudaFreeAsync(dJ, st);
  cudaFreeAsync(dI, st);
  cudaFreeAsync(dw, st);
  cudaFreeAsync(dpart, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == RDG_OK) rc = fail_m(ctx, RDG_ECUDA, "error-norm kernel");
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  if (rc != RDG_OK) return rc;
  double se = 0.0, sa = 0.0, mx = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    se += part[3 * b];
    sa += part[3 * b + 1];
    mx = std::max(mx, part[3 * b + 2]);
  }
  *l2 = std::sqrt(se / sa);
  *linf = mx;
  return RDG_OK;
}

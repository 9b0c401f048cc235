// Row gather and scatter for the halo exchange of a mesh split across ranks: before every
// right-hand-side stage a rank sends the stage-input rows of its elements that border another
// rank (gathered into a contiguous buffer) and receives the rows of its halo elements, because
// the reconstruction of every edge reads all 2 Np values of both neighbours (Sec. 4,
// Algorithm aRDG), not only their traces.
#include <cuda_runtime.h>

#include "context.h"

namespace rdg {
namespace {

// One thread per value; a warp covers consecutive values of consecutive rows, so both the
// contiguous side and each indexed row are read or written in whole segments.
template <typename T>
__global__ void rows_kernel(const T* __restrict__ src, const int32_t* __restrict__ idx, int64_t n, int np,
                            T* __restrict__ dst, bool scatter, int64_t nrows, int* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * np) return;
  const int64_t row = i / np;
  const int c = (int)(i - row * np);
  const int64_t k = idx[row];
  if (k < 0 || k >= nrows) {
    if (err) atomicOr(err, kErrBadIndex);   // recorded like the other kernels' index self-checks
    return;
  }
  if (scatter) dst[k * np + c] = src[row * np + c];
  else dst[row * np + c] = src[k * np + c];
}

}  // namespace

int launch_rows(int esz, int np, const void* src, const int32_t* idx, int64_t n, void* dst, bool scatter,
                int64_t nrows, int* err, cudaStream_t s) {
  const int64_t total = n * np;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (esz == 4)
    rows_kernel<float><<<grid, 256, 0, s>>>((const float*)src, idx, n, np, (float*)dst, scatter, nrows, err);
  else
    rows_kernel<double><<<grid, 256, 0, s>>>((const double*)src, idx, n, np, (double*)dst, scatter, nrows, err);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

}  // namespace rdg

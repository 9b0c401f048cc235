// Volume term as a tensor-core GEMM (tcgen05, split 3xTF32), for the largest order.
//
// The volume term of element k is a fixed linear combination of five products of the
// element's values with shared reference matrices (the metric-folded form of M^{-1} S^T . F,
// F = v u - D grad u, with Dr, Ds applied to d = u - u_0, which they annihilate the constant
// part of):
//     vol = a_r Wr u + a_s Ws u - g_rr (Wr Dr) d - g_rs (Wr Ds + Ws Dr) d - g_ss (Ws Ds) d,
// Wr = M^{-1} Dr^T M, Ws = M^{-1} Ds^T M, and d_0 = 0 so only d_1..d_{Np-1} enter.  So a tile
// of 128 elements is one GEMM
//     D[k][(b,i)] = sum_c A[k][c] B[(b,i)][c],   A[k] = (u_0..u_{Np-1}, d_1..d_{Np-1}),
// with B the five stacked matrices (zero where a block does not act), and the epilogue sums
// the five blocks with the element's a_r, a_s, -g_rr, -g_rs, -g_ss.  Operands are split into
// TF32 hi + lo and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in tensor memory, as in
// the edge GEMM form (gemm_kernels.cuh, whose helpers this uses).  At N = 6 the element-by-
// element form runs 3136 FMAs per element with a distinct constant operand each.
#pragma once

namespace rdg {
namespace gemm {

template <int N>
struct VolShape {
  static constexpr int NP = np_of(N);
  static constexpr int KR = 2 * NP - 1;                   // u_0..u_{Np-1}, d_1..d_{Np-1}
  static constexpr int KP = (KR + 7) / 8 * 8;
  static constexpr int NR = 5 * NP;                       // five blocks of Np rows
  static constexpr int NPAD = (NR + 15) / 16 * 16;
  static constexpr int M = 128;
  static constexpr int SBO = KP / 4 * 128;
  static constexpr int ATILE = M * KP * 4;
  static constexpr int BTILE = NPAD * KP * 4;
  static constexpr int TCOLS = NPAD <= 32 ? 32 : NPAD <= 64 ? 64 : NPAD <= 128 ? 128 : NPAD <= 256 ? 256 : 512;
  static constexpr int CTAS = 512 / TCOLS;
  static constexpr int OFF_B = 2 * ATILE;                 // A hi, lo; then B hi, lo
  static constexpr int OFF_BAR = OFF_B + 2 * BTILE;
  static constexpr int OFF_STAGE = OFF_BAR + 16;          // element rows staged for coalesced I/O
  static constexpr int DATA = OFF_STAGE + M * NP * 4;
  static constexpr int FLOOR = 233472 / (CTAS + 1) - 1024 + 16;
  static constexpr int SMEM = DATA > FLOOR ? DATA : FLOOR;
  static_assert(NPAD <= 256, "MMA N limit");
  static_assert(SMEM <= 232448, "shared memory per block");
  static_assert(OFF_STAGE % 16 == 0, "staging alignment");
};

// Persistent: B (hi, lo) copied into shared memory once, tensor-memory columns taken once
// after the dependency wait, then element tiles blockIdx.x, blockIdx.x + gridDim.x, ...
template <int N>
__global__ void __launch_bounds__(128, 1) volume_gemm_kernel(EdgeArgs<float> a, const float4* vb) {
  using S = VolShape<N>;
  constexpr int NP = S::NP;
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    float4* dst = reinterpret_cast<float4*>(smem + S::OFF_B);
    for (int i = tid; i < 2 * S::BTILE / 16; i += blockDim.x) dst[i] = vb[i];
  }
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + S::OFF_BAR + 8);
  const uint32_t bar = smem_u32(smem + S::OFF_BAR);
  if (tid == 0) mbar_init(bar, 1);
  dev::wait_for_predecessor();
  if (tid < 32) tmem_alloc(smem_u32(slot), S::TCOLS);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  float* stage = reinterpret_cast<float*>(smem + S::OFF_STAGE);
  const int64_t ntiles = (a.K + S::M - 1) / S::M;
  uint32_t phase = 0;
  bool ok = true;
  // the next tile's element rows are loaded into registers while this tile's MMAs run
  dev::Staged<float, S::M, NP> g;
  int64_t t = blockIdx.x;
  if (t < ntiles) g.load(a.u + t * S::M * NP, (int)min((int64_t)S::M, a.K - t * S::M) * NP);
  for (; t < ntiles && ok; t += gridDim.x) {
    const int64_t k0 = t * S::M;
    const int nk = (int)min((int64_t)S::M, a.K - k0);
    g.store(stage, nk * NP);
    __syncthreads();
    // operand row of this thread's element, split into TF32 hi + lo
    {
      float row[S::KP];
#pragma unroll
      for (int c = 0; c < S::KP; ++c) row[c] = 0.f;
      if (tid < nk) {
#pragma unroll
        for (int j = 0; j < NP; ++j) row[j] = stage[tid * NP + j];
#pragma unroll
        for (int j = 1; j < NP; ++j) row[NP + j - 1] = row[j] - row[0];
      }
      uint8_t* hi = smem + (tid >> 3) * S::SBO + (tid & 7) * 16;
      uint8_t* lo = smem + S::ATILE + (tid >> 3) * S::SBO + (tid & 7) * 16;
#pragma unroll
      for (int k4 = 0; k4 < S::KP / 4; ++k4) {
        float4 h, o;
        split_tf32(row[4 * k4 + 0], h.x, o.x);
        split_tf32(row[4 * k4 + 1], h.y, o.y);
        split_tf32(row[4 * k4 + 2], h.z, o.z);
        split_tf32(row[4 * k4 + 3], h.w, o.w);
        *reinterpret_cast<float4*>(hi + k4 * 128) = h;
        *reinterpret_cast<float4*>(lo + k4 * 128) = o;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      constexpr uint32_t idesc = idesc_tf32<S::NPAD>();
      const uint32_t sa = smem_u32(smem), sb = smem_u32(smem + S::OFF_B);
#pragma unroll
      for (int ks = 0; ks < S::KP / 8; ++ks) {
        const uint32_t ah = sa + ks * 256, al = ah + S::ATILE;
        const uint32_t bh = sb + ks * 256, bl = bh + S::BTILE;
        mma_tf32(tmem, smem_desc(ah, 128, S::SBO), smem_desc(bh, 128, S::SBO), idesc, ks > 0);
        mma_tf32(tmem, smem_desc(ah, 128, S::SBO), smem_desc(bl, 128, S::SBO), idesc, 1);
        mma_tf32(tmem, smem_desc(al, 128, S::SBO), smem_desc(bh, 128, S::SBO), idesc, 1);
      }
      mma_commit(bar);
    }
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) g.load(a.u + tn * S::M * NP, (int)min((int64_t)S::M, a.K - tn * S::M) * NP);
    // epilogue coefficients a_r, a_s, -g_rr, -g_rs, -g_ss
    float co[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (tid < nk) {
      const int64_t k = k0 + tid;
      co[0] = a.geo[k];
      co[1] = a.geo[a.K + k];
      co[2] = -a.geo[2 * a.K + k];
      co[3] = -a.geo[3 * a.K + k];
      co[4] = -a.geo[4 * a.K + k];
    }
    bool done = mbar_wait(bar, phase, 1000000000ull);
    if (!done) mbar_wait(bar, phase, 1000000000ull);   // give the tensor core a second chance to drain
    // every thread leaves the loop together if any of them gave up
    ok = __syncthreads_and(done ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) dev::report(a.err, kErrWaitTimeout);
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    // vol_i = a_r D[i] + a_s D[Np+i] - g_rr D[2Np+i] - g_rs D[3Np+i] - g_ss D[4Np+i]
    float vol[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) vol[i] = 0.f;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < S::NPAD / 16; ++c) {
      float v[16];
      tmem_ld16(lane_base + c * 16, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = c * 16 + j;
        if (n < S::NR) vol[n % NP] = fmaf(co[n / NP], v[j], vol[n % NP]);
      }
    }
    tc_fence_before();
    if (tid < nk) {
#pragma unroll
      for (int i = 0; i < NP; ++i) stage[tid * NP + i] = vol[i];   // a thread rewrites only its own row
    }
    __syncthreads();
    dev::stage_out(a.vol + k0 * NP, stage, nk * NP);
    __syncthreads();   // staging, operand tiles and tensor memory free for the next tile
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(tmem, S::TCOLS);
}

// B of order N in the shared-memory layout the kernel copies verbatim: [hi, lo][NPAD rows
// (b, i)][KP columns c] in core-matrix order; blocks Wr, Ws on the u columns and Wr Dr,
// Wr Ds + Ws Dr, Ws Ds on the d columns (d_j, j >= 1, at column Np + j - 1).
template <int N>
std::vector<float> pack_volume_operand(const RefOps& o) {
  using S = VolShape<N>;
  constexpr int NP = S::NP;
  auto at = [&](const std::vector<double>& m, int i, int j) { return m[(size_t)i * NP + j]; };
  std::vector<double> A1((size_t)NP * NP, 0.0), A2((size_t)NP * NP, 0.0), A3((size_t)NP * NP, 0.0);
  for (int i = 0; i < NP; ++i)
    for (int j = 0; j < NP; ++j)
      for (int m = 0; m < NP; ++m) {
        A1[(size_t)i * NP + j] += at(o.Wr, i, m) * at(o.Dr, m, j);
        A2[(size_t)i * NP + j] += at(o.Wr, i, m) * at(o.Ds, m, j) + at(o.Ws, i, m) * at(o.Dr, m, j);
        A3[(size_t)i * NP + j] += at(o.Ws, i, m) * at(o.Ds, m, j);
      }
  std::vector<float> out(2 * S::BTILE / 4, 0.f);
  auto put = [&](int n, int c, double x) {
    float hf = (float)x;
    uint32_t bits;
    std::memcpy(&bits, &hf, 4);
    bits &= 0xFFFFE000u;
    std::memcpy(&hf, &bits, 4);
    const float lf = (float)(x - (double)hf);
    const size_t off = (size_t)(n / 8) * S::SBO + (c / 4) * 128 + (n % 8) * 16 + (c % 4) * 4;
    out[off / 4] = hf;
    out[(S::BTILE + off) / 4] = lf;
  };
  for (int i = 0; i < NP; ++i) {
    for (int j = 0; j < NP; ++j) {
      put(0 * NP + i, j, at(o.Wr, i, j));
      put(1 * NP + i, j, at(o.Ws, i, j));
    }
    for (int j = 1; j < NP; ++j) {
      put(2 * NP + i, NP + j - 1, A1[(size_t)i * NP + j]);
      put(3 * NP + i, NP + j - 1, A2[(size_t)i * NP + j]);
      put(4 * NP + i, NP + j - 1, A3[(size_t)i * NP + j]);
    }
  }
  return out;
}

template <int N>
int launch_volume_gemm_t(const EdgeArgs<float>& a, const float4* vb, cudaStream_t s) {
  using S = VolShape<N>;
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    if (cudaFuncSetAttribute(volume_gemm_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) !=
        cudaSuccess)
      return RDG_ECUDA;
    attr_done[dev] = true;
  }
  const int64_t ntiles = (a.K + S::M - 1) / S::M;
  if (ntiles == 0) return RDG_OK;
  // one wave of persistent blocks: as many per SM as both shared memory (1 KB reserved per
  // block) and tensor memory allow
  const int per_sm = std::max(1, std::min(S::CTAS, 233472 / (S::SMEM + 1024)));
  int64_t grid = std::min<int64_t>(ntiles, (int64_t)per_sm * sm_count());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = S::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, volume_gemm_kernel<N>, a, vb) == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

}  // namespace gemm
}  // namespace rdg

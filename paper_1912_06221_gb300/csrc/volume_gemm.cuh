// Volume term as a tensor-core GEMM (tcgen05, split 3xTF32).  Written for any order (rows
// of whole 16-byte words load as vectors, others element by element); the library builds it
// for FP32 order 6, where it is faster than the fused stage kernel's volume role (at orders
// 4 and 5 the split form measured 45.6 and 73.2 us per stage against 31.0 and 58.6 fused).
//
// The volume term of element k is a fixed linear combination of five products of the
// element's values with shared reference matrices (the metric-folded form of M^{-1} S^T . F,
// F = v u - D grad u, with Dr, Ds applied to d = u - u_0, which they annihilate the constant
// part of):
//     vol = a_r Wr u + a_s Ws u - g_rr (Wr Dr) d - g_rs (Wr Ds + Ws Dr) d - g_ss (Ws Ds) d,
// Wr = M^{-1} Dr^T M, Ws = M^{-1} Ds^T M, and d_0 = 0 so only d_1..d_{Np-1} enter.  So a tile
// of 128 elements is two GEMMs on one operand A[k] = (u_0..u_{Np-1} | d_1..d_{Np-1}):
//     D1[k][(b,i)] = sum_j u_j B1[(b,i)][j],        B1 = [Wr; Ws],
//     D2[k][(b,i)] = sum_j d_j B2[(b,i)][j],        B2 = [Wr Dr; Wr Ds + Ws Dr; Ws Ds],
// and the epilogue sums the five blocks with the element's a_r, a_s, -g_rr, -g_rs, -g_ss.
// Operands are split into TF32 hi + lo and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates
// in tensor memory, as in the edge GEMM form (gemm_kernels.cuh, whose helpers this uses).  At
// N = 6 the element-by-element form runs 3136 FMAs per element with a distinct constant
// operand each.
#pragma once

namespace rdg {
namespace gemm {

// Persistent volume blocks per SM at most (shared and tensor memory allow two at order 6;
// at lower orders the edge-only blocks running beside them keep the rest of the SM).
constexpr int kVolumeBlocksPerSm = 2;

template <int N>
struct VolShape {
  static constexpr int NP = np_of(N);
  static constexpr int KU = (NP + 7) / 8 * 8;             // u block of A (TF32 k-step 8)
  static constexpr int KD = (NP - 1 + 7) / 8 * 8;         // d block of A
  static constexpr int KP = KU + KD;
  static constexpr int N1 = 2 * NP, N2 = 3 * NP;          // rows of B1, B2
  static constexpr int NPAD1 = (N1 + 31) / 32 * 32, NPAD2 = (N2 + 31) / 32 * 32;   // MMA N, epilogue reads
  static constexpr int M = 128;
  static constexpr int SBO_A = KP / 4 * 128;              // bytes between 8-row groups of A
  static constexpr int SBO_B1 = KU / 4 * 128, SBO_B2 = KD / 4 * 128;
  static constexpr int ATILE = M * KP * 4;
  static constexpr int BT1 = NPAD1 * KU * 4, BT2 = NPAD2 * KD * 4;
  static constexpr int BWORDS = 2 * (BT1 + BT2) / 16;     // B1 hi, lo, B2 hi, lo (16-byte words)
  static constexpr int COLS = NPAD1 + NPAD2;
  static constexpr int TCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static constexpr int CTAS = 512 / TCOLS;
  static constexpr int OFF_B = 2 * ATILE;                 // A hi, lo; then B
  static constexpr int OFF_BAR = OFF_B + 2 * (BT1 + BT2);
  static constexpr int DATA = OFF_BAR + 16;
  // shared-memory floor that keeps tensor memory from being oversubscribed (checked below for
  // every mix): a block of four or more per SM's worth of columns takes a 1/CTAS share
  static constexpr int FLOOR = CTAS >= 4 ? 233472 / CTAS - 1024 : 233472 / (CTAS + 1) - 1024 + 16;
  static constexpr int SMEM = DATA > FLOOR ? DATA : FLOOR;
  static constexpr bool VEC = NP * 4 % 16 == 0;           // element rows of whole 16-byte words
  static_assert(NPAD1 <= 256 && NPAD2 <= 256, "MMA N limit");
  static_assert(NPAD1 % 32 == 0 && NPAD2 % 32 == 0, "epilogue reads 32 columns at a time");
  static_assert(SMEM <= 232448, "shared memory per block");
};

// Tensor-memory columns: every mix of blocks of the tcgen05 kernels (edge GEMM form of orders
// 1..5, this volume kernel at order 6) that fits one SM's 228 KB of shared memory (1 KB reserved per
// block) holds at most the SM's 512 columns, so an allocation never waits for another block.
struct TmemUser {
  int smem, cols;
};
constexpr int kNumTmemUsers = 6;
constexpr TmemUser kTmemUsers[kNumTmemUsers] = {
    {Shape<1>::SMEM, Shape<1>::TCOLS}, {Shape<2>::SMEM, Shape<2>::TCOLS}, {Shape<3>::SMEM, Shape<3>::TCOLS},
    {Shape<4>::SMEM, Shape<4>::TCOLS}, {Shape<5>::SMEM, Shape<5>::TCOLS}, {VolShape<6>::SMEM, VolShape<6>::TCOLS}};
constexpr int max_tmem_cols(int i, int smem_left) {
  if (i == kNumTmemUsers) return 0;
  int best = 0;
  for (int c = 0; c * (kTmemUsers[i].smem + 1024) <= smem_left; ++c) {
    const int v = c * kTmemUsers[i].cols + max_tmem_cols(i + 1, smem_left - c * (kTmemUsers[i].smem + 1024));
    best = v > best ? v : best;
  }
  return best;
}
static_assert(max_tmem_cols(0, 233472) <= 512, "co-resident tcgen05 blocks could oversubscribe tensor memory");

// 32 consecutive FP32 columns of this thread's tensor-memory lane (warp w reads lanes
// 32w..32w+31), one completion wait per 32 columns.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Persistent: B (hi, lo) copied into shared memory once, tensor-memory columns taken once
// after the dependency wait, then element tiles blockIdx.x, blockIdx.x + gridDim.x, ...  Each
// thread owns one element: its row is read straight into registers (the next tile's while
// this tile's MMAs run), and its volume row is written straight back.
template <int N>
__global__ void __launch_bounds__(128, 1) volume_gemm_kernel(EdgeArgs<float> a, const float4* vb) {
  using S = VolShape<N>;
  constexpr int NP = S::NP;
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    float4* dst = reinterpret_cast<float4*>(smem + S::OFF_B);
    for (int i = tid; i < S::BWORDS; i += blockDim.x) dst[i] = vb[i];
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
  const int64_t ntiles = (a.K + S::M - 1) / S::M;
  uint32_t phase = 0;
  float nxt[NP];
  int64_t t = blockIdx.x;
  auto load_row = [&](int64_t tt) {
    const int64_t kk = tt * S::M + tid;
    if (tt < ntiles && kk < a.K) {
      if constexpr (S::VEC) {
        const float4* p = reinterpret_cast<const float4*>(a.u + kk * NP);
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) {
          const float4 w = __ldg(p + q);
          nxt[4 * q] = w.x;
          nxt[4 * q + 1] = w.y;
          nxt[4 * q + 2] = w.z;
          nxt[4 * q + 3] = w.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < NP; ++j) nxt[j] = __ldg(a.u + kk * NP + j);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NP; ++j) nxt[j] = 0.f;
    }
  };
  load_row(t);
  for (; t < ntiles; t += gridDim.x) {
    const int64_t k = t * S::M + tid;
    const bool live = k < a.K;
    // operand row (u | d) of this thread's element, split into TF32 hi + lo
    {
      float row[S::KP];
#pragma unroll
      for (int c = 0; c < S::KP; ++c) row[c] = 0.f;
#pragma unroll
      for (int j = 0; j < NP; ++j) row[j] = nxt[j];
#pragma unroll
      for (int j = 1; j < NP; ++j) row[S::KU + j - 1] = row[j] - row[0];
      uint8_t* hi = smem + (tid >> 3) * S::SBO_A + (tid & 7) * 16;
      uint8_t* lo = hi + S::ATILE;
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
    if (tid == 0 && t + 1 != a.hold_tile) {   // (test hook: a held tile's MMAs are never issued)
      tc_fence_after();
      constexpr uint32_t id1 = idesc_tf32<S::NPAD1>(), id2 = idesc_tf32<S::NPAD2>();
      const uint32_t sa = smem_u32(smem), sb = smem_u32(smem + S::OFF_B);
      const uint32_t b1h = sb, b1l = sb + S::BT1, b2h = sb + 2 * S::BT1, b2l = b2h + S::BT2;
#pragma unroll
      for (int ks = 0; ks < S::KU / 8; ++ks) {
        const uint32_t ah = sa + ks * 256, al = ah + S::ATILE;
        mma_tf32(tmem, smem_desc(ah, 128, S::SBO_A), smem_desc(b1h + ks * 256, 128, S::SBO_B1), id1, ks > 0);
        mma_tf32(tmem, smem_desc(ah, 128, S::SBO_A), smem_desc(b1l + ks * 256, 128, S::SBO_B1), id1, 1);
        mma_tf32(tmem, smem_desc(al, 128, S::SBO_A), smem_desc(b1h + ks * 256, 128, S::SBO_B1), id1, 1);
      }
#pragma unroll
      for (int ks = 0; ks < S::KD / 8; ++ks) {
        const uint32_t ah = sa + (S::KU / 4) * 128 + ks * 256, al = ah + S::ATILE;
        const uint32_t d2 = tmem + S::NPAD1;
        mma_tf32(d2, smem_desc(ah, 128, S::SBO_A), smem_desc(b2h + ks * 256, 128, S::SBO_B2), id2, ks > 0);
        mma_tf32(d2, smem_desc(ah, 128, S::SBO_A), smem_desc(b2l + ks * 256, 128, S::SBO_B2), id2, 1);
        mma_tf32(d2, smem_desc(al, 128, S::SBO_A), smem_desc(b2h + ks * 256, 128, S::SBO_B2), id2, 1);
      }
      mma_commit(bar);
    }
    load_row(t + gridDim.x);
    // epilogue coefficients a_r, a_s, -g_rr, -g_rs, -g_ss
    float co[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (live) {
      co[0] = a.geo[k];
      co[1] = a.geo[a.K + k];
      co[2] = -a.geo[2 * a.K + k];
      co[3] = -a.geo[3 * a.K + k];
      co[4] = -a.geo[4 * a.K + k];
    }
    bool done = mbar_wait(bar, phase, 1000000000ull);
    if (!done) done = mbar_wait(bar, phase, 1000000000ull);   // a second chance to drain
    // the block agrees on the outcome, so every thread leaves the loop together
    if (__syncthreads_and(done ? 1 : 0) == 0) {
      if (tid == 0) dev::report(a.err, kErrWaitTimeout);
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    // vol_i = a_r D1[i] + a_s D1[Np+i] - g_rr D2[i] - g_rs D2[Np+i] - g_ss D2[2Np+i]
    float vol[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) vol[i] = 0.f;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < S::NPAD1 / 32; ++c) {
      float v[32];
      tmem_ld32(lane_base + c * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = c * 32 + j;
        if (n < S::N1) vol[n % NP] = fmaf(co[n / NP], v[j], vol[n % NP]);
      }
    }
#pragma unroll
    for (int c = 0; c < S::NPAD2 / 32; ++c) {
      float v[32];
      tmem_ld32(lane_base + S::NPAD1 + c * 32, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = c * 32 + j;
        if (n < S::N2) vol[n % NP] = fmaf(co[2 + n / NP], v[j], vol[n % NP]);
      }
    }
    tc_fence_before();
    if (live) {
      if constexpr (S::VEC) {
        float4* o = reinterpret_cast<float4*>(a.vol + k * NP);
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) o[q] = make_float4(vol[4 * q], vol[4 * q + 1], vol[4 * q + 2], vol[4 * q + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) a.vol[k * NP + i] = vol[i];
      }
    }
    __syncthreads();   // operand tiles and tensor memory free for the next tile
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(tmem, S::TCOLS);
}

// B1 and B2 of order N in the shared-memory layout the kernel copies verbatim: [B1 hi, B1 lo,
// B2 hi, B2 lo], each [NPAD rows (b, i)][K columns] in core-matrix order; B1 = [Wr; Ws] on
// u_0..u_{Np-1}, B2 = [Wr Dr; Wr Ds + Ws Dr; Ws Ds] on d_1..d_{Np-1} (column j - 1).
template <int N>
std::vector<float> pack_volume_operand(const RefOps& o) {
  using S = VolShape<N>;
  constexpr int NP = S::NP;
  auto at = [&](const std::vector<double>& m, int i, int j) { return m[(size_t)i * NP + j]; };
  std::vector<double> P[3];
  for (auto& p : P) p.assign((size_t)NP * NP, 0.0);
  for (int i = 0; i < NP; ++i)
    for (int j = 0; j < NP; ++j)
      for (int m = 0; m < NP; ++m) {
        P[0][(size_t)i * NP + j] += at(o.Wr, i, m) * at(o.Dr, m, j);
        P[1][(size_t)i * NP + j] += at(o.Wr, i, m) * at(o.Ds, m, j) + at(o.Ws, i, m) * at(o.Dr, m, j);
        P[2][(size_t)i * NP + j] += at(o.Ws, i, m) * at(o.Ds, m, j);
      }
  std::vector<float> out(S::BWORDS * 4, 0.f);
  // base: byte offset of the hi matrix; its lo copy follows `tile` bytes later
  auto put = [&](size_t base, size_t tile, int sbo, int n, int c, double x) {
    float hf = (float)x;
    uint32_t bits;
    std::memcpy(&bits, &hf, 4);
    bits &= 0xFFFFE000u;
    std::memcpy(&hf, &bits, 4);
    const float lf = (float)(x - (double)hf);
    const size_t off = base + (size_t)(n / 8) * sbo + (c / 4) * 128 + (n % 8) * 16 + (c % 4) * 4;
    out[off / 4] = hf;
    out[(off + tile) / 4] = lf;
  };
  const size_t b2 = 2 * (size_t)S::BT1;
  for (int i = 0; i < NP; ++i) {
    for (int j = 0; j < NP; ++j) {
      put(0, S::BT1, S::SBO_B1, i, j, at(o.Wr, i, j));
      put(0, S::BT1, S::SBO_B1, NP + i, j, at(o.Ws, i, j));
    }
    for (int j = 1; j < NP; ++j)
      for (int b = 0; b < 3; ++b) put(b2, S::BT2, S::SBO_B2, b * NP + i, j - 1, P[b][(size_t)i * NP + j]);
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
  const int per_sm = std::max(1, std::min({S::CTAS, 233472 / (S::SMEM + 1024), kVolumeBlocksPerSm}));
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)per_sm * sm_count());
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

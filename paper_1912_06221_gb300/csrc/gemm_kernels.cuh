// GEMM form of the edge flux on the fifth-generation tensor cores (tcgen05, split 3xTF32).
//
// The per-edge diffusive operator is not streamed from memory.  Side k's part of the edge
// gradient in rotated node order is
//     sum_rho kappa_rho sum_m psi_m(alpha_k, beta_k) X_k[m][i][rho][l]
// (Sec. 4.4-4.5: the projection V^{-1} V_p V_rf^{-1} of Eq. totalProjection is a polynomial
// of degree <= N in the parallelogram apex coordinates (alpha_k, beta_k), expanded once per
// order in the orthonormal basis psi_m).  So one tile of 128 edges is a GEMM
//     D_k[e][(m,i)] = sum_(rho,l) A_k[e][(rho,l)] X_k[(m,i)][(rho,l)],
//     A_k[e][(rho,l)] = kappa_rho(e) (u_k,rot[l] - u_0)
// against the shared reference matrix X_k, and the epilogue contracts D_k with the edge's
// psi_m(alpha_k, beta_k) and scales by -J_f D~_i; the upwind term J_f (v.n1) u_up is added
// from the gathered traces.  Per edge the hot path reads a 2Np + Nfp + 3 float parameter
// record instead of the Nfp x 2Np operator.
//
// FP32 accuracy from TF32 inputs: every operand is split x = hi + lo with hi the leading 10
// mantissa bits, and D = A_hi X_hi + A_hi X_lo + A_lo X_hi is accumulated in FP32 in tensor
// memory (the dropped lo*lo term and the truncation of lo are below FP32 rounding).
//
// Operands live in shared memory in the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, [row/8][k/4][row%8][k%4], so a descriptor's leading byte offset
// (next core matrix along K) is 128 B and its stride byte offset (next 8-row group) is
// KP/4 x 128 B.  The accumulators of the two sides occupy 2 x NPAD tensor-memory columns.
// Included by rhs_order.cu for FP32 orders 1..5, after rhs_kernels.cuh.
#pragma once

namespace rdg {
namespace gemm {

template <int N>
struct Shape {
  static constexpr int NP = np_of(N), NFP = nfp_of(N);
  static constexpr int KR = 2 * NP;                        // (rho, l)
  static constexpr int KP = (KR + 7) / 8 * 8;              // K padded to the TF32 k-step (8)
  static constexpr int NR = NP * NFP;                      // (m, i)
  static constexpr int NPAD = (NR + 15) / 16 * 16;         // MMA N: a multiple of 16 for M = 128
  static constexpr int M = 128;                            // edges per tile (one per thread)
  static constexpr int SBO = KP / 4 * 128;                 // bytes between 8-row groups
  static constexpr int ATILE = M * KP * 4;
  static constexpr int BTILE = NPAD * KP * 4;
  static constexpr int COLS = 2 * NPAD;
  static constexpr int TCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static constexpr int PW = 2 * NP + NFP + 3;              // parameter record (floats)
  static constexpr int PW4 = (PW + 3) / 4;                 // ... in 16-byte words
  static constexpr int CTAS = 512 / TCOLS;                 // CTAs whose columns fit one SM
  // Dynamic shared memory: the operands, the barrier and the tables; then at least enough
  // that no more than CTAS blocks of any kernel with this much shared memory fit one SM
  // (228 KB per SM, 1 KB reserved per block), so a tensor-memory allocation never waits.
  static constexpr int OFF_B = 4 * ATILE;
  static constexpr int OFF_BAR = OFF_B + 4 * BTILE;
  static constexpr int OFF_TAB = OFF_BAR + 16;
  static constexpr int DATA = OFF_TAB + 4 * (3 * NP + NFP) + 16;
  static constexpr int FLOOR = 233472 / (CTAS + 1) - 1024 + 16;
  static constexpr int SMEM = DATA > FLOOR ? DATA : FLOOR;
  static_assert(NPAD <= 256, "MMA N limit");
  static_assert(SMEM <= 232448, "shared memory per block");
};

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B
// TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <int NN>
__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading and stride byte offsets
// (all >> 4), descriptor version 1 at bits 46-47, layout type 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the barrier phase: false if it did not complete within `ns` nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try(bar, parity))
    if (global_ns() - t0 > ns) return false;
  return true;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on the barrier once every previously issued MMA of this thread has completed
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane (warp w reads lanes
// 32w..32w+31).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// x = hi + lo, hi keeping the sign, exponent and leading 10 mantissa bits (a TF32 value)
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}


// Edge role, one tile of 128 edges (thread = edge): gather, operand tiles, MMAs, epilogue.
// Returns false if the MMA completion wait gave up (the error word is then set).
template <int N>
__device__ __forceinline__ bool gemm_edge_tile(const EdgeArgs<float>& a, int64_t t, uint8_t* smem, uint32_t tmem,
                                               uint32_t& phase) {
  using S = Shape<N>;
  constexpr int NP = S::NP, NFP = S::NFP;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int* sperm = reinterpret_cast<const int*>(smem + S::OFF_TAB);   // [3][NP] rotated -> natural
  const int* shyp = sperm + 3 * NP;                                     // [NFP]
  const int64_t e = t * S::M + tid;
  const bool live = e < a.E;
  float ur1[NP], ur2[NP];
#pragma unroll
  for (int l = 0; l < NP; ++l) ur1[l] = ur2[l] = 0.f;
  int k1 = -1, k2 = -1, f12 = 0;
  float pr[S::PW4 * 4];
#pragma unroll
  for (int q = 0; q < S::PW4 * 4; ++q) pr[q] = 0.f;
  if (live) {
    k1 = a.k1[e];
    k2 = a.k2[e];
    f12 = a.f12[e];
    if (k1 < 0 || k1 >= a.K || (k2 >= 0 ? k2 >= a.K : (-1 - (int64_t)k2) >= a.B)) {
      dev::report(a.err, kErrBadIndex);
      k1 = -1;
      k2 = -1;
    } else {
      const float4* P = reinterpret_cast<const float4*>(a.W) + ((e >> 5) * S::PW4) * kTile + (e & 31);
#pragma unroll
      for (int q = 0; q < S::PW4; ++q) {
        const float4 w = dev::ld_stream(P + q * kTile);
        pr[4 * q] = w.x;
        pr[4 * q + 1] = w.y;
        pr[4 * q + 2] = w.z;
        pr[4 * q + 3] = w.w;
      }
      const int f1 = f12 & 3, f2 = (f12 >> 2) & 3;
      const float* p1 = a.u + (int64_t)k1 * NP;
#pragma unroll
      for (int l = 0; l < NP; ++l) ur1[l] = __ldg(p1 + sperm[f1 * NP + l]);
      if (k2 >= 0) {
        const float* p2 = a.u + (int64_t)k2 * NP;
#pragma unroll
        for (int l = 0; l < NP; ++l) ur2[l] = __ldg(p2 + sperm[f2 * NP + l]);
      } else {
        // ghost side (its shared face is face 1): g = sum_m G_m tau_m(t), in rotated order
        const int64_t bb = -1 - (int64_t)k2;
        const double tt = dev::stage_time(a.time);
        for (int mm = 0; mm < a.frc.nghost; ++mm) {
          const float tm = (float)dev::tau_of(a.frc.gkind[mm], a.frc.gomega[mm], tt);
          const float* g = a.G + ((int64_t)mm * a.B + bb) * NP;
#pragma unroll
          for (int l = 0; l < NP; ++l) ur2[l] += tm * g[sperm[NP + l]];
        }
      }
    }
  }
  // operand rows: kappa_rho (u_rot - u_0), split into TF32 hi + lo
  {
    const float ub = ur1[0], kR = pr[2 * NP], kS = pr[2 * NP + 1];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      float row[S::KP];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        const float d = (side == 0 ? ur1[l] : ur2[l]) - ub;
        row[l] = kR * d;
        row[NP + l] = kS * d;
      }
#pragma unroll
      for (int k = 2 * NP; k < S::KP; ++k) row[k] = 0.f;
      uint8_t* hi = smem + (side * 2 + 0) * S::ATILE + (tid >> 3) * S::SBO + (tid & 7) * 16;
      uint8_t* lo = smem + (side * 2 + 1) * S::ATILE + (tid >> 3) * S::SBO + (tid & 7) * 16;
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
  }
  fence_async_smem();
  __syncthreads();
  const uint32_t bar = smem_u32(smem + S::OFF_BAR);
  if (tid == 0) {
    tc_fence_after();
    constexpr uint32_t idesc = idesc_tf32<S::NPAD>();
    const uint32_t sa = smem_u32(smem), sb = smem_u32(smem + S::OFF_B);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const uint32_t d = tmem + side * S::NPAD;
#pragma unroll
      for (int ks = 0; ks < S::KP / 8; ++ks) {
        const uint32_t ah = sa + (side * 2) * S::ATILE + ks * 256, al = ah + S::ATILE;
        const uint32_t bh = sb + (side * 2) * S::BTILE + ks * 256, bl = bh + S::BTILE;
        mma_tf32(d, smem_desc(ah, 128, S::SBO), smem_desc(bh, 128, S::SBO), idesc, ks > 0);
        mma_tf32(d, smem_desc(ah, 128, S::SBO), smem_desc(bl, 128, S::SBO), idesc, 1);
        mma_tf32(d, smem_desc(al, 128, S::SBO), smem_desc(bh, 128, S::SBO), idesc, 1);
      }
    }
    mma_commit(bar);
  }
  const bool done = mbar_wait(bar, phase, 1000000000ull);
  if (!done) mbar_wait(bar, phase, 1000000000ull);   // give the tensor core a second chance to drain
  // the block agrees on the outcome, so every thread leaves the tile loop together
  const bool ok = __syncthreads_and(done ? 1 : 0) != 0;
  if (!ok && tid == 0) dev::report(a.err, kErrWaitTimeout);
  phase ^= 1u;
  tc_fence_after();
  // epilogue: acc_i = sum_side sum_m psi_m(side) D_side[(m, i)]
  float acc[NFP];
#pragma unroll
  for (int i = 0; i < NFP; ++i) acc[i] = 0.f;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
  for (int side = 0; side < 2; ++side) {
#pragma unroll
    for (int c = 0; c < S::NPAD / 16; ++c) {
      float v[16];
      tmem_ld16(lane_base + side * S::NPAD + c * 16, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = c * 16 + j;
        if (n < S::NR) acc[n % NFP] = fmaf(pr[side * NP + n / NFP], v[j], acc[n % NFP]);
      }
    }
  }
  tc_fence_before();
  if (live && k1 >= 0) {
    const float jv = pr[2 * NP + 2 + NFP];
    float fl[NFP];
#pragma unroll
    for (int i = 0; i < NFP; ++i) {
      // upwind trace: side 1's face node i, or side 2's node NFP-1-i (the face runs the
      // other way there)
      const int h1 = shyp[i], h2 = shyp[NFP - 1 - i];
      float up1 = 0.f, up2 = 0.f;
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        up1 = (l == h1) ? ur1[l] : up1;
        up2 = (l == h2) ? ur2[l] : up2;
      }
      fl[i] = fmaf(pr[2 * NP + 2 + i], acc[i], jv * (jv >= 0.f ? up1 : up2));
    }
    float* o1 = a.fb + ((int64_t)k1 * 3 + (f12 & 3)) * NFP;
#pragma unroll
    for (int i = 0; i < NFP; ++i) o1[i] = fl[i];
    if (k2 >= 0) {
      float* o2 = a.fb + ((int64_t)k2 * 3 + ((f12 >> 2) & 3)) * NFP;
#pragma unroll
      for (int i = 0; i < NFP; ++i) o2[i] = -fl[NFP - 1 - i];
    }
  }
  __syncthreads();   // tensor memory and the operand tiles are free for the next tile
  return ok;
}

// Persistent kernel: the CTA loads the reference operands X (hi, lo; both sides) into shared
// memory and allocates its tensor-memory columns once, then runs edge tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and afterwards the element volume tiles the same
// way (the volume term M^{-1} S^T . F into a.vol, one thread per element).
template <int N>
__global__ void __launch_bounds__(128, 1) edge_gemm_kernel(EdgeArgs<float> a, const float4* xb, const int* tab) {
  using S = Shape<N>;
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x;
  {
    float4* dst = reinterpret_cast<float4*>(smem + S::OFF_B);
    for (int i = tid; i < 4 * S::BTILE / 16; i += blockDim.x) dst[i] = xb[i];
    int* st = reinterpret_cast<int*>(smem + S::OFF_TAB);
    for (int i = tid; i < 3 * S::NP + S::NFP; i += blockDim.x) st[i] = tab[i];
  }
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + S::OFF_BAR + 8);
  if (tid == 0) mbar_init(smem_u32(smem + S::OFF_BAR), 1);
  // tensor memory is taken only after the predecessor grid has finished, so this block never
  // holds columns while it waits on another kernel
  dev::wait_for_predecessor();
  // the element kernel's blocks may fill SMs as these persistent blocks finish
  dev::allow_dependents();
  if (threadIdx.x < 32) tmem_alloc(smem_u32(slot), S::TCOLS);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const int64_t ntiles = (a.E + S::M - 1) / S::M;
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) ok = gemm_edge_tile<N>(a, t, smem, tmem, phase);
  if (ok) {
    const int64_t nvol = (a.K + kStageBlock - 1) / kStageBlock;
    float* sh = reinterpret_cast<float*>(smem);   // the A tiles are free now
    for (int64_t v = blockIdx.x; v < nvol; v += gridDim.x) {
      dev::stage_volume_tile<float, N>(a, v, sh);
      __syncthreads();
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(tmem, S::TCOLS);
}

// ---------------------------------------------------------------------------------------
// Warp-specialised form (orders whose double-buffered tiles fit one SM: N <= 4).  One CTA
// per SM, persistent over the edge tiles, with four roles that run concurrently:
//   producers  two groups of four warps; group g takes the CTA's tiles i = g, g + 2, ...
//              (thread = edge): gathers the tile, builds its operand rows into stage i % 2
//              of shared memory (hi, lo; both sides) and the epilogue's per-edge values
//              (psi_m of both sides, -J_f D~_i, the upwind flux, the element ids) into stash
//              i % 2; after a group barrier one of its threads issues the tile's split-TF32
//              MMAs into tensor-memory buffer i % 2 and commits them to done[i % 2].  The
//              group's next element ids are loaded while this tile's values are in flight.
//   epilogue   four warps (warp % 4 = the tensor-memory lane quadrant they may read): waits
//              done[s], contracts its 32 rows with psi_m, scatters the face fluxes, arrives
//              on empty[s] (stage, stash and buffer s free again).
//   volume     four warps: the element volume tiles (thread = element), the next tile's
//              rows loaded before this tile's arithmetic.
// So two tiles are gathered while a third is multiplied and a fourth written out, and the
// volume arithmetic runs beside them.  Every wait is bounded: on a timeout the CTA sets a
// shared abort flag (the other roles' waits then return at once) and the error word, drains
// its MMAs (bounded) and frees its tensor memory.
// Rotated-order index of the shared face's node q: the last node of row q of the
// row-by-row node numbering (checked against the reference operators when they are packed).
__host__ __device__ constexpr int hyp_of(int N, int q) { return (q + 1) * (N + 1) - q * (q + 1) / 2 - 1; }

template <int N>
struct Pipe {
  using S = Shape<N>;
  static constexpr int NP = S::NP, NFP = S::NFP;
  static constexpr int SW = 2 * NP + 2 * NFP + 3;            // stash words per edge
  static constexpr int OFF_B = 0;                            // X: [side][hi, lo]
  static constexpr int OFF_A = 4 * S::BTILE;                 // A: [stage][side][hi, lo]
  static constexpr int OFF_ST = OFF_A + 8 * S::ATILE;        // stash: [stage][word][edge]
  static constexpr int NVOLW = 4;                            // volume warps
  static constexpr int VT = NVOLW * 32;                      // elements per volume tile
  static constexpr int OFF_VOL = OFF_ST + 2 * SW * 128 * 4;  // volume rows [VT][NP]
  static constexpr int OFF_TAB = OFF_VOL + VT * NP * 4;      // rotated-order tables
  static constexpr int OFF_BAR = (OFF_TAB + 4 * (3 * NP + NFP) + 15) / 16 * 16;
  // barriers done[2], empty[2]; then the tensor-memory slot and the abort flag
  static constexpr int SMEM = OFF_BAR + 4 * 8 + 16;
  static constexpr int COLS = 4 * S::NPAD;                   // two buffers x two sides
  static constexpr int TCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static constexpr int PG = 2;                               // producer groups (4 warps each)
  static constexpr int W_EPI = 4 * PG, W_VOL = W_EPI + 4;   // 16 warps in all (128 registers)
  static constexpr int THREADS = (W_VOL + NVOLW) * 32;
  static constexpr bool FITS = SMEM <= 232448 && COLS <= 512;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
// Named barrier that also returns whether every participating thread passed `v`.
__device__ __forceinline__ bool named_and(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// mbarrier test that may suspend the thread (up to about 20 us, woken early when the phase
// completes) instead of returning at once, so waiting warps do not take issue slots from the
// working ones.
__device__ __forceinline__ bool mbar_try_suspend(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(20000)
      : "memory");
  return ok != 0;
}

// Bounded wait of a pipeline role: false (and the CTA's abort flag set) if the phase did not
// complete within `ns` nanoseconds, or false at once when another role has aborted.
__device__ __forceinline__ bool pipe_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint64_t ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_suspend(bar, parity)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > ns) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane, without the wait.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

constexpr uint64_t kPipeWaitNs = 1000000000ull;

// The split-TF32 MMAs of one tile: A (stage s, both sides, hi and lo) against the reference
// operand X into tensor-memory buffer s (issued by one thread).
template <int N>
__device__ __forceinline__ void issue_tile_mma(uint8_t* smem, uint32_t tmem, int s) {
  using S = Shape<N>;
  using P = Pipe<N>;
  constexpr uint32_t idesc = idesc_tf32<S::NPAD>();
  const uint32_t sb = smem_u32(smem + P::OFF_B);
  const uint32_t sa = smem_u32(smem + P::OFF_A + s * 4 * S::ATILE);
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const uint32_t d = tmem + s * 2 * S::NPAD + side * S::NPAD;
#pragma unroll
    for (int ks = 0; ks < S::KP / 8; ++ks) {
      const uint32_t ah = sa + (side * 2) * S::ATILE + ks * 256, al = ah + S::ATILE;
      const uint32_t bh = sb + (side * 2) * S::BTILE + ks * 256, bl = bh + S::BTILE;
      mma_tf32(d, smem_desc(ah, 128, S::SBO), smem_desc(bh, 128, S::SBO), idesc, ks > 0);
      mma_tf32(d, smem_desc(ah, 128, S::SBO), smem_desc(bl, 128, S::SBO), idesc, 1);
      mma_tf32(d, smem_desc(al, 128, S::SBO), smem_desc(bh, 128, S::SBO), idesc, 1);
    }
  }
}

// Producer role (warps 0 .. 4 PG - 1), thread = edge of each tile of its group.
template <int N>
__device__ __forceinline__ void pipe_producer(const EdgeArgs<float>& a, uint8_t* smem, uint32_t tmem,
                                              volatile int* abort_flag) {
  using S = Shape<N>;
  using P = Pipe<N>;
  constexpr int NP = S::NP, NFP = S::NFP;
  const int tid = threadIdx.x & 127, grp = threadIdx.x >> 7;
  const int* sperm = reinterpret_cast<const int*>(smem + P::OFF_TAB);
  const uint32_t bar = smem_u32(smem + P::OFF_BAR);
  const int64_t ntiles = (a.E + S::M - 1) / S::M;
  const int64_t tstep = (int64_t)P::PG * gridDim.x;
  int64_t t = blockIdx.x + (int64_t)grp * gridDim.x;
  int nk1 = -1, nk2 = -1, nf12 = 0, last = -1;
  if (t < ntiles && t * S::M + tid < a.E) {
    nk1 = a.k1[t * S::M + tid];
    nk2 = a.k2[t * S::M + tid];
    nf12 = a.f12[t * S::M + tid];
  }
  for (int i = grp; t < ntiles; i += P::PG, t += tstep) {
    const int s = i & 1;
    if (t + 1 == a.hold_tile) break;    // test hook: this tile is never released (group-uniform)
    const int64_t e = t * S::M + tid;
    int k1 = nk1, k2 = nk2;
    const int f12 = nf12;
    float ur1[NP], ur2[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) ur1[l] = ur2[l] = 0.f;
    float pr[S::PW4 * 4];
#pragma unroll
    for (int q = 0; q < S::PW4 * 4; ++q) pr[q] = 0.f;
    if (e < a.E) {
      if (k1 < 0 || k1 >= a.K || (k2 >= 0 ? k2 >= a.K : (-1 - (int64_t)k2) >= a.B)) {
        dev::report(a.err, kErrBadIndex);
        k1 = -1;
        k2 = -1;
      } else {
        const float4* Pp = reinterpret_cast<const float4*>(a.W) + ((e >> 5) * S::PW4) * kTile + (e & 31);
#pragma unroll
        for (int q = 0; q < S::PW4; ++q) {
          const float4 w = dev::ld_stream(Pp + q * kTile);
          pr[4 * q] = w.x;
          pr[4 * q + 1] = w.y;
          pr[4 * q + 2] = w.z;
          pr[4 * q + 3] = w.w;
        }
        const int f1 = f12 & 3, f2 = (f12 >> 2) & 3;
        const float* p1 = a.u + (int64_t)k1 * NP;
#pragma unroll
        for (int l = 0; l < NP; ++l) ur1[l] = __ldg(p1 + sperm[f1 * NP + l]);
        if (k2 >= 0) {
          const float* p2 = a.u + (int64_t)k2 * NP;
#pragma unroll
          for (int l = 0; l < NP; ++l) ur2[l] = __ldg(p2 + sperm[f2 * NP + l]);
        } else {
          // ghost side (its shared face is face 1): g = sum_m G_m tau_m(t), in rotated order
          const int64_t bb = -1 - (int64_t)k2;
          const double tt = dev::stage_time(a.time);
          for (int mm = 0; mm < a.frc.nghost; ++mm) {
            const float tm = (float)dev::tau_of(a.frc.gkind[mm], a.frc.gomega[mm], tt);
            const float* g = a.G + ((int64_t)mm * a.B + bb) * NP;
#pragma unroll
            for (int l = 0; l < NP; ++l) ur2[l] += tm * g[sperm[NP + l]];
          }
        }
      }
    } else {
      k1 = -1;
    }
    // the next tile's element ids, in flight while this tile is written
    {
      const int64_t tn = t + tstep, en = tn * S::M + tid;
      if (tn < ntiles && en < a.E) {
        nk1 = a.k1[en];
        nk2 = a.k2[en];
        nf12 = a.f12[en];
      }
    }
    // stage s and stash s are free once the epilogue of tile i - 2 has finished with them;
    // the group agrees on the outcome, so its named barriers below always see 128 threads
    const bool free_ok = i < 2 || pipe_wait(bar + 16 + 8 * s, ((i >> 1) - 1) & 1, abort_flag, kPipeWaitNs);
    if (!named_and(2 + grp, 128, free_ok)) break;
    {
      const float ub = ur1[0], kR = pr[2 * NP], kS = pr[2 * NP + 1];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        float row[S::KP];
#pragma unroll
        for (int l = 0; l < NP; ++l) {
          const float d = (side == 0 ? ur1[l] : ur2[l]) - ub;
          row[l] = kR * d;
          row[NP + l] = kS * d;
        }
#pragma unroll
        for (int k = 2 * NP; k < S::KP; ++k) row[k] = 0.f;
        uint8_t* base = smem + P::OFF_A + (s * 4 + side * 2) * S::ATILE + (tid >> 3) * S::SBO + (tid & 7) * 16;
#pragma unroll
        for (int k4 = 0; k4 < S::KP / 4; ++k4) {
          float4 h, o;
          split_tf32(row[4 * k4 + 0], h.x, o.x);
          split_tf32(row[4 * k4 + 1], h.y, o.y);
          split_tf32(row[4 * k4 + 2], h.z, o.z);
          split_tf32(row[4 * k4 + 3], h.w, o.w);
          *reinterpret_cast<float4*>(base + k4 * 128) = h;
          *reinterpret_cast<float4*>(base + S::ATILE + k4 * 128) = o;
        }
      }
    }
    {
      float* st = reinterpret_cast<float*>(smem + P::OFF_ST) + s * P::SW * 128;
#pragma unroll
      for (int m = 0; m < 2 * NP; ++m) st[m * 128 + tid] = pr[m];
      const float jv = pr[2 * NP + 2 + NFP];
#pragma unroll
      for (int q = 0; q < NFP; ++q) {
        // upwind trace: side 1's face node q, or side 2's node NFP-1-q (the face runs the
        // other way there)
        const float up1 = ur1[hyp_of(N, q)], up2 = ur2[hyp_of(N, NFP - 1 - q)];
        st[(2 * NP + q) * 128 + tid] = pr[2 * NP + 2 + q];
        st[(2 * NP + NFP + q) * 128 + tid] = jv * (jv >= 0.f ? up1 : up2);
      }
      int* sti = reinterpret_cast<int*>(st);
      sti[(2 * NP + 2 * NFP) * 128 + tid] = k1;
      sti[(2 * NP + 2 * NFP + 1) * 128 + tid] = k2;
      sti[(2 * NP + 2 * NFP + 2) * 128 + tid] = f12;
    }
    // the group's writes, visible to the tensor core, then one thread issues the tile's MMAs
    // (the thread is held while the tensor core works through them; the rest of the group
    // goes on to its next tile's loads)
    fence_async_smem();
    named_sync(2 + grp, 128);
    if (tid == 0) {
      tc_fence_after();
      issue_tile_mma<N>(smem, tmem, s);
      mma_commit(bar + 8 * s);
      last = i;
    }
  }
  // nothing may be in flight when the columns are freed (bounded even after an abort)
  if (tid == 0 && last >= 0) mbar_wait(bar + 8 * (last & 1), (last >> 1) & 1, kPipeWaitNs);
}

// Epilogue role (four warps): quadrant q = warp % 4 of every tile's rows.
template <int N>
__device__ __forceinline__ void pipe_epilogue(const EdgeArgs<float>& a, uint8_t* smem, uint32_t tmem,
                                              volatile int* abort_flag) {
  using S = Shape<N>;
  using P = Pipe<N>;
  constexpr int NP = S::NP, NFP = S::NFP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3;
  const int r = 32 * q + lane;
  const uint32_t bar = smem_u32(smem + P::OFF_BAR);
  const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
  const int64_t ntiles = (a.E + S::M - 1) / S::M;
  int64_t t = blockIdx.x;
  for (int i = 0; t < ntiles; ++i, t += gridDim.x) {
    const int s = i & 1;
    // the warp agrees before its collective tensor-memory loads
    const bool ok = pipe_wait(bar + 8 * s, (i >> 1) & 1, abort_flag, kPipeWaitNs);
    if (!__all_sync(0xffffffffu, ok)) break;
    tc_fence_after();
    const float* st = reinterpret_cast<const float*>(smem + P::OFF_ST) + s * P::SW * 128;
    float acc[NFP];
#pragma unroll
    for (int k = 0; k < NFP; ++k) acc[k] = 0.f;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      uint32_t v[S::NPAD];
#pragma unroll
      for (int c = 0; c < S::NPAD / 16; ++c)
        tmem_ld16_async(lane_base + s * 2 * S::NPAD + side * S::NPAD + c * 16,
                        *reinterpret_cast<uint32_t(*)[16]>(&v[16 * c]));
      tmem_wait_ld();
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const float psi = st[(side * NP + m) * 128 + r];
#pragma unroll
        for (int k = 0; k < NFP; ++k) acc[k] = fmaf(psi, __uint_as_float(v[m * NFP + k]), acc[k]);
      }
    }
    float fl[NFP];
#pragma unroll
    for (int k = 0; k < NFP; ++k) fl[k] = fmaf(st[(2 * NP + k) * 128 + r], acc[k], st[(2 * NP + NFP + k) * 128 + r]);
    const int* sti = reinterpret_cast<const int*>(st);
    const int k1 = sti[(2 * NP + 2 * NFP) * 128 + r];
    const int k2 = sti[(2 * NP + 2 * NFP + 1) * 128 + r];
    const int f12 = sti[(2 * NP + 2 * NFP + 2) * 128 + r];
    tc_fence_before();
    mbar_arrive(bar + 16 + 8 * s);
    if (k1 >= 0) {
      float* o1 = a.fb + ((int64_t)k1 * 3 + (f12 & 3)) * NFP;
#pragma unroll
      for (int k = 0; k < NFP; ++k) o1[k] = fl[k];
      if (k2 >= 0) {
        float* o2 = a.fb + ((int64_t)k2 * 3 + ((f12 >> 2) & 3)) * NFP;
#pragma unroll
        for (int k = 0; k < NFP; ++k) o2[k] = -fl[NFP - 1 - k];
      }
    }
  }
}

// Volume role (NVOLW warps, thread vt = element of each tile of VT elements, named barrier 1):
// rows staged through shared memory with 16-byte loads and stores, the next tile's rows in
// flight during this tile's arithmetic.
template <int N>
__device__ __forceinline__ void pipe_volume(const EdgeArgs<float>& a, uint8_t* smem) {
  using P = Pipe<N>;
  constexpr int NP = np_of(N), VT = P::VT;
  constexpr int IT = (VT * NP / 4 + VT - 1) / VT;   // 16-byte words of a full tile per thread
  const int vt = threadIdx.x - P::W_VOL * 32;
  float* sh = reinterpret_cast<float*>(smem + P::OFF_VOL);
  const int64_t nvol = (a.K + VT - 1) / VT;
  float4 rg[IT];
  float tail = 0.f;
  auto load = [&](int64_t v) {
    const int64_t k0 = v * VT;
    const int n = (int)min((int64_t)VT, a.K - k0) * NP, nv = n / 4;
    const float4* g4 = reinterpret_cast<const float4*>(a.u + k0 * NP);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int j = vt + it * VT;
      if (j < nv) rg[it] = __ldcs(g4 + j);
    }
    if (vt < 4 && nv * 4 + vt < n) tail = a.u[k0 * NP + nv * 4 + vt];
  };
  int64_t v = blockIdx.x;
  if (v < nvol) load(v);
  for (; v < nvol; v += gridDim.x) {
    const int64_t k0 = v * VT;
    const int nk = (int)min((int64_t)VT, a.K - k0), n = nk * NP, nv = n / 4;
    named_sync(1, VT);                             // the previous tile's rows are written out
    {
      float4* s4 = reinterpret_cast<float4*>(sh);
#pragma unroll
      for (int it = 0; it < IT; ++it) {
        const int j = vt + it * VT;
        if (j < nv) s4[j] = rg[it];
      }
      if (vt < 4 && nv * 4 + vt < n) sh[nv * 4 + vt] = tail;
    }
    named_sync(1, VT);
    if (v + gridDim.x < nvol) load(v + gridDim.x);  // next tile in flight during the arithmetic
    if (vt < nk) {
      const int64_t k = k0 + vt;
      float u[NP], vol[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) u[j] = sh[vt * NP + j];
      dev::volume_row<float, N>(u, a.geo[k], a.geo[a.K + k], a.geo[2 * a.K + k], a.geo[3 * a.K + k],
                                a.geo[4 * a.K + k], vol);
#pragma unroll
      for (int j = 0; j < NP; ++j) sh[vt * NP + j] = vol[j];   // a thread rewrites only its own row
    }
    named_sync(1, VT);
    {
      float4* g4 = reinterpret_cast<float4*>(a.vol + k0 * NP);
      const float4* s4 = reinterpret_cast<const float4*>(sh);
      for (int j = vt; j < nv; j += VT) __stcs(g4 + j, s4[j]);
      for (int j = nv * 4 + vt; j < n; j += VT) a.vol[k0 * NP + j] = sh[j];
    }
  }
}

template <int N>
__global__ void __launch_bounds__(Pipe<N>::THREADS, 1) edge_gemm_pipe_kernel(EdgeArgs<float> a, const float4* xb,
                                                                            const int* tab) {
  using S = Shape<N>;
  using P = Pipe<N>;
  extern __shared__ __align__(128) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    float4* dst = reinterpret_cast<float4*>(smem + P::OFF_B);
    for (int i = tid; i < 4 * S::BTILE / 16; i += blockDim.x) dst[i] = xb[i];
    int* st = reinterpret_cast<int*>(smem + P::OFF_TAB);
    for (int i = tid; i < 3 * S::NP + S::NFP; i += blockDim.x) st[i] = tab[i];
  }
  const uint32_t bar = smem_u32(smem + P::OFF_BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + P::OFF_BAR + 32);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + P::OFF_BAR + 36);
  if (tid == 0) {
    *abort_flag = 0;
    mbar_init(bar + 0, 1);      // done[0], done[1]: the MMA commit
    mbar_init(bar + 8, 1);
    mbar_init(bar + 16, 128);   // empty[0], empty[1]: every epilogue thread
    mbar_init(bar + 24, 128);
  }
  // tensor memory is taken only after the predecessor grid has finished, so this block never
  // holds columns while it waits on another kernel
  dev::wait_for_predecessor();
  dev::allow_dependents();
  if (warp == 0) tmem_alloc(smem_u32(slot), P::TCOLS);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (warp < P::W_EPI) pipe_producer<N>(a, smem, tmem, abort_flag);
  else if (warp < P::W_VOL) pipe_epilogue<N>(a, smem, tmem, abort_flag);
  else pipe_volume<N>(a, smem);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *abort_flag) dev::report(a.err, kErrWaitTimeout);
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, P::TCOLS);
  }
}

// Reference operand X of order N in the shared-memory layout the kernel copies verbatim:
// [side][hi, lo][NPAD rows (m, i)][KP columns (rho, l)] in core-matrix order.
template <int N>
std::vector<float> pack_gemm_operand(const RefOps& o) {
  using S = Shape<N>;
  std::vector<float> out(4 * S::BTILE / 4, 0.f);
  for (int side = 0; side < 2; ++side)
    for (int m = 0; m < S::NP; ++m)
      for (int i = 0; i < S::NFP; ++i)
        for (int rho = 0; rho < 2; ++rho)
          for (int l = 0; l < S::NP; ++l) {
            const double x = o.X[side][(((size_t)m * S::NFP + i) * 2 + rho) * S::NP + l];
            const int n = m * S::NFP + i, k = rho * S::NP + l;
            const size_t off = (size_t)(n / 8) * S::SBO + (k / 4) * 128 + (n % 8) * 16 + (k % 4) * 4;
            float hf = (float)x;
            uint32_t bits;
            std::memcpy(&bits, &hf, 4);
            bits &= 0xFFFFE000u;
            std::memcpy(&hf, &bits, 4);
            const float lf = (float)(x - (double)hf);
            out[((size_t)(side * 2 + 0) * S::BTILE + off) / 4] = hf;
            out[((size_t)(side * 2 + 1) * S::BTILE + off) / 4] = lf;
          }
  return out;
}

// Tables for the kernel: rotated -> natural node index per face [3][Np], then the rotated
// indices of the shared face's nodes [Nfp].
template <int N>
std::vector<int> pack_gemm_table(const RefOps& o) {
  using S = Shape<N>;
  std::vector<int> t(3 * S::NP + S::NFP);
  for (int f = 0; f < 3; ++f)
    for (int i = 0; i < S::NP; ++i) t[f * S::NP + o.perm[f * S::NP + i]] = i;
  for (int q = 0; q < S::NFP; ++q) t[3 * S::NP + q] = o.hyp[q];
  return t;
}

template <int N>
int launch_gemm_t(const EdgeArgs<float>& a, const float4* xb, const int* tab, cudaStream_t s) {
  using S = Shape<N>;
  using P = Pipe<N>;
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  const int64_t ntiles = (a.E + S::M - 1) / S::M;
  const int64_t nvol = (a.K + kStageBlock - 1) / kStageBlock;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.stream = s;
  if constexpr (P::FITS) {
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
      if (cudaFuncSetAttribute(edge_gemm_pipe_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM) !=
          cudaSuccess)
        return RDG_ECUDA;
      attr_done[dev] = true;
    }
    int64_t grid = std::min<int64_t>(sm_count(), std::max(ntiles, nvol));
    if (grid < 1) grid = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(P::THREADS);
    cfg.dynamicSmemBytes = P::SMEM;
    return cudaLaunchKernelEx(&cfg, edge_gemm_pipe_kernel<N>, a, xb, tab) == cudaSuccess ? RDG_OK : RDG_ECUDA;
  } else {
    if (dev >= 0 && dev < 64 && !attr_done[dev]) {
      if (cudaFuncSetAttribute(edge_gemm_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM) !=
          cudaSuccess)
        return RDG_ECUDA;
      attr_done[dev] = true;
    }
    int64_t grid = (int64_t)S::CTAS * sm_count();
    grid = std::min(grid, std::max(ntiles, nvol));
    if (grid < 1) grid = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = S::SMEM;
    return cudaLaunchKernelEx(&cfg, edge_gemm_kernel<N>, a, xb, tab) == cudaSuccess ? RDG_OK : RDG_ECUDA;
  }
}

}  // namespace gemm
}  // namespace rdg

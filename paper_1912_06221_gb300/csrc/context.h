// Definition of the library context (shared by the translation units that enqueue work).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "internal.h"

struct EdgeRec {
  int32_t k1, f1, k2, f2;  // k2 = -1 - b for boundary edge b
  double shx, shy;
};

struct rdg_ctx {
  using Forcing = rdg::Forcing;
  using TimeState = rdg::TimeState;
  int device = 0;
  cudaStream_t stream = nullptr;     // the caller's stream (may be the legacy default stream)
  cudaStream_t cap_stream = nullptr; // private stream used only to capture graphs
  bool capturing = false;
  bool own_stream = false;
  // forked stream for a volume kernel that runs beside the edge kernel (FP32, order 6)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
  // mesh (host)
  bool mesh_ok = false;
  int64_t K = 0, E = 0, B = 0;
  int64_t n_owned = 0;            // elements [n_owned, K) are halo copies (partitioned upload)
  int bc = 0;
  std::vector<double> exy;       // [K][6]
  std::vector<EdgeRec> edges;    // interior edges first, then boundary edges (a split mesh:
                                 // first the e_split edges with no halo side)
  std::vector<int64_t> bedge;    // edge of ghost b (boundary edge b)
  int64_t e_split = 0;           // edges [0, e_split) touch no halo element (a multiple of 32)
  std::vector<int32_t> eref;     // [3][K]
  // operators
  bool ops_ok = false;
  int N = 0, prec = RDG_FP32, esz = 4, iface = RDG_IFACE_ALG2;
  double vx = 0, vy = 0;
  std::vector<double> Dk;           // element diffusion (x diffusion when Dy is set)
  std::vector<double> Dy;           // y diffusion of a diagonal tensor (Dx, Dy); empty: isotropic
  std::vector<double> Dn;           // D at the nodes [K][Np]; empty: D per element
  void* d_Dn = nullptr;             // the same on the device, in the context's precision
  // device buffers
  int integrator = RDG_INTEGRATOR_SSP_RK3;
  int stage_form = RDG_STAGE_AUTO;     // kernel form of a right-hand-side stage
  int64_t gemm_hold = 0;               // test hook: GEMM-form edge tile gemm_hold - 1 never released
  bool gemm = false;                // GEMM form of the edge flux (RDG_FP32_3XTF32, N <= kMaxGemmN)
  void* d_W = nullptr;              // tiled per-edge operators, or the GEMM-form parameter records
  int32_t *d_k1 = nullptr, *d_k2 = nullptr, *d_eref = nullptr;
  void *d_geo = nullptr, *d_flux = nullptr, *d_u = nullptr, *d_u1 = nullptr, *d_u2 = nullptr;
  void *d_S = nullptr, *d_G = nullptr;
  void* d_vol = nullptr;            // volume terms of the current stage [K][Np]
  void* d_fb = nullptr;             // face fluxes of the current stage [K][3][Nfp]
  int32_t* d_f12 = nullptr;         // per edge f1 | f2 << 2
  TimeState* d_time = nullptr;
  int* d_err = nullptr;            // device error bits (kernel self-checks)
  int64_t l2_keep_bytes = -1;       // operator bytes kept L2-resident (-1: default)
  Forcing frc;
  // per-kernel event timing (class 0 edge flux, 1 element update)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[2];
  double prof_ms[2] = {0, 0};
  int64_t prof_n[2] = {0, 0};
  // graph of a chunk of steps for one dt
  cudaGraphExec_t gexec = nullptr;
  double g_dt = 0;
  int g_chunk = 0;
};

namespace rdg {
// One SSP-RK3 step of ctx's resident state with every launch on stream s (which may be
// capturing); used by the batch, whose member steps run on per-member branch streams.
int enqueue_rk_step_on(rdg_ctx* ctx, cudaStream_t s, const TimeArg& base, double dt);
// Row gather (dst[i] = src[idx[i]]) or scatter (dst[idx[i]] = src[i]) of np-value rows of
// esz-byte values; indices outside 0..nrows-1 are recorded in err and skipped.
int launch_rows(int esz, int np, const void* src, const int32_t* idx, int64_t n, void* dst, bool scatter,
                int64_t nrows, int* err, cudaStream_t s);
}  // namespace rdg

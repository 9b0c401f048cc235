// Internal declarations shared by the host code and the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rdg.h"
#include "refops.h"

namespace rdg {

constexpr int kTile = 32;            // edges per W tile (one warp, one edge per lane)
constexpr int kElemBlock = 128;      // elements per element-kernel block
constexpr int kStageBlock = 128;     // threads per block of the stage (edge/volume) kernel

// Stored values of one edge's flux operator in its difference form: per row, side 1's
// columns 1..Np-1 and side 2's Np columns (2 Np - 1 values), then the one value J_f (v.n1)
// that every row's column 0 (the row sum) would hold.
inline int w_stored_values(int N) { return nfp_of(N) * (2 * np_of(N) - 1) + 1; }

// Words (of 16 bytes) per edge row block of the tiled flux operator.
inline int w_vecs_per_edge(int N, int elem_bytes) {
  int nw = w_stored_values(N);
  int per = 16 / elem_bytes;
  return (nw + per - 1) / per;
}

struct Forcing {
  int nsrc = 0, nghost = 0;
  int kind[RDG_MAX_FORCING_TERMS] = {0}, gkind[RDG_MAX_FORCING_TERMS] = {0};
  double omega[RDG_MAX_FORCING_TERMS] = {0}, gomega[RDG_MAX_FORCING_TERMS] = {0};
};

// Device-resident time origin of a captured graph: step n of the replay starts at t0 + n dt.
struct TimeState {
  double t0;
  long long n;
};

// Stage time: ts ? ts->t0 + (ts->n + off) dt : t0 + off dt
struct TimeArg {
  const TimeState* ts;
  double t0, dt, off;
};

template <typename T>
struct EdgeArgs {
  const int32_t* k1;
  const int32_t* k2;   // >= 0 element, or -1-b for boundary edge b (ghost data)
  const void* W;       // tiled operator
  const T* u;
  T* flux;             // [E][Nfp]
  const T* G;          // [nghost][B][Np]
  int64_t E, B;
  Forcing frc;
  TimeArg time;
  int* err;            // device error word (kErr* bits); may be null
  int64_t K;           // elements (for the index self-check)
  T* vol;              // fused form: volume term of every element, [K][Np] (else null)
  const T* geo;        // fused form: element coefficients [6][K]
  const int32_t* f12;  // fused form: per edge f1 | f2 << 2 (local faces of the two sides)
  T* fb;               // fused form: face fluxes [K][3][Nfp] in each element's own face order
  int64_t keep_tiles;  // operator tiles [0, keep_tiles) are loaded evict-last (kept in L2)
  const T* Dn;         // D at the nodes [K][Np] when given so (geo then holds the metric alone), else null
  int64_t Kvol;        // fused form: volume terms of elements [0, Kvol) only (0: all K)
  int64_t hold_tile;   // test hook of the GEMM form: edge tile hold_tile - 1 is never released (0: none)
};

// Device error bits reported through rdg_synchronize.
constexpr int kErrWaitTimeout = 1;   // a bounded wait for the tensor core gave up
constexpr int kErrBadIndex = 2;

template <typename T>
struct ElemArgs {
  const T* us;         // stage input
  const T* un;         // step start (RK combination)
  T* out;
  const T* flux;
  const int32_t* eref; // [3][K]: 2*edge + (1 if the element is side 2)
  const T* geo;        // [6][K]: a_r, a_s, g_rr, g_rs, g_ss, 1/J
  const T* S;          // [nsrc][K][Np]
  int64_t K;
  T dt;
  Forcing frc;
  TimeArg time;
  int* err;            // device error word; may be null
  int64_t E;           // edges (for the index self-check)
  const T* vol;        // fused form: precomputed volume term [K][Np] (else null)
  const T* fb;         // fused form: face fluxes [K][3][Nfp]
  // low-storage Runge-Kutta stage (mode 4): un is the residual register du (read only when
  // rka != 0), du' = rka du + dt L(us) is written to out2 and us + rkb du' to out
  T* out2;
  T rka, rkb;
};

// mode: 0 rhs only; 1..3 the three SSP-RK3 stage combinations; 4 a low-storage RK stage
int launch_edge32(int N, const EdgeArgs<float>& a, cudaStream_t s);
int launch_edge64(int N, const EdgeArgs<double>& a, cudaStream_t s);
int launch_elem32(int N, int mode, const ElemArgs<float>& a, cudaStream_t s);
int launch_elem64(int N, int mode, const ElemArgs<double>& a, cudaStream_t s);
// Fused form: the edge kernel's extra warps also compute the element volume terms (hidden
// under the operator stream) and the element kernel adds the surface terms and the stage.
int launch_edge_vol32(int N, const EdgeArgs<float>& a, cudaStream_t s);
int launch_edge_vol64(int N, const EdgeArgs<double>& a, cudaStream_t s);
int launch_elem_lite32(int N, int mode, const ElemArgs<float>& a, cudaStream_t s);
int launch_elem_lite64(int N, int mode, const ElemArgs<double>& a, cudaStream_t s);
// One-kernel stage (elem_fused_kernel): modes 0..3.
int launch_fused32(int N, int mode, const EdgeArgs<float>& ea, const ElemArgs<float>& a, cudaStream_t s);
int launch_fused64(int N, int mode, const EdgeArgs<double>& ea, const ElemArgs<double>& a, cudaStream_t s);
int upload_elem_tables(int device);
// GEMM form of the edge flux (FP32 state, tcgen05 split 3xTF32), orders 1..kMaxGemmN: the
// edge kernel reads per-edge parameter records (EdgeArgs::W) and also computes the volume
// terms; the element kernel is the same as the stored-operator form's.
constexpr int kMaxGemmN = 5;
int launch_gemm32(int N, const EdgeArgs<float>& a, cudaStream_t s);
// Orders whose FP32 volume term is its own tensor-core kernel (volume_gemm.cuh), launched
// beside the edge-only operator stream (kind 2) instead of the fused stage kernel (order 6).
bool split_volume32(int N);
int launch_volume32(int N, const EdgeArgs<float>& a, cudaStream_t s);
// Edge blocks only (fluxes into the face slots), every order and precision.
int launch_edge_only32(int N, const EdgeArgs<float>& a, cudaStream_t s);
int launch_edge_only64(int N, const EdgeArgs<double>& a, cudaStream_t s);
int gemm_param_words(int N);   // 16-byte words of an edge's parameter record

// ---- setup (FP64) -------------------------------------------------------------------
struct EdgeSetupIn {
  const double* xy;        // [K][6] element vertex coordinates
  const int32_t* k1;
  const int32_t* f1;
  const int32_t* k2;       // -1-b for boundary edge b
  const int32_t* f2;
  const double* shift;     // [E][2]
  const double* D;         // [K] (x diffusion when Dy is set)
  const double* Dy;        // [K] y diffusion of the diagonal tensor (Dx, Dy), or null: isotropic
  const double* Dn;        // [K][Np] D at the nodes, or null (D then per element)
  const double* nodal_refs;  // with Dn: RVV [2][Nfp][Np], GR [2][2][Np][Np], GS [2][2][Np][Np]
  const double* refs;      // per-order reference constants (layout in setup.cu)
  int64_t E;
  double vx, vy;
  int iface;               // RDG_IFACE_*
  int64_t nrefs;           // doubles in refs (checked against the order's layout)
};

// Per edge: the tiled operator W (W_tiled, elem_bytes per value), the dense FP64 operator
// (W_dense), and/or the GEMM-form parameter record (P_tiled, FP32); any may be null.
int setup_edges(int N, const EdgeSetupIn& in, void* W_tiled, int elem_bytes, double* W_dense, float* P_tiled,
                cudaStream_t s);
int setup_elements(int64_t K, const double* xy, const double* D, const double* Dy, double vx, double vy, void* geo,
                   int elem_bytes,
                   cudaStream_t s);
// Reference constants for the setup kernel, flattened in the order setup.cu reads them.
std::vector<double> pack_setup_refs(const RefOps& o);
int advance_time(TimeState* ts, long long by, cudaStream_t s);
int set_time(TimeState* ts, double t0, cudaStream_t s);

}  // namespace rdg

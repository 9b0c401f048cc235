// Device-side descriptors and host entry points of the persistent batch launch
// (batch_kernel.cu), shared with the batch host code (batch.cpp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.h"

namespace rdg {

// One member problem as the persistent kernel sees it (FP32, stored operators, SSP-RK3).
// A stage of a member is two parts of work items: part A, its edge tiles (fluxes into the
// face slots) and element tiles (volume terms); part B, its element tiles again (surface
// terms and the stage update).
struct BMember {
  const void* W;             // tiled per-edge operators
  const int32_t* k1;
  const int32_t* k2;
  const int32_t* f12;
  float *u, *u1, *u2;        // state and the two stage buffers
  float *vol, *fb;           // volume terms, face slots
  const float* geo;
  const float* S;            // sources [nsrc][K][Np]
  const float* G;            // Dirichlet ghost data [nghost][B][Np]
  int* err;                  // the member's device error word
  TimeState* ts;             // time origin and steps done before this launch
  int64_t K, E, B;
  Forcing frc;
  double dt;
  float dt32;
  int N;
  int ept;                   // edges per thread in an edge tile (1 or 2)
  int tpi;                   // tiles per work item (1, 2 or 4)
  int64_t ntile_e, ntile_v;  // part A: edge and element tiles per stage
  int64_t ntile_u;           // part B: element tiles per stage
  int64_t nitem_a, nitem_b;  // work items of part A / part B per stage (tiles / tpi, rounded up)
  int64_t off_a, off_b;      // first item of this member within part A / part B of a stage
  int64_t hold_phase;        // a stage whose part A is never released (test hook), or -1
};

struct BatchArgs {
  const BMember* m;          // device array [nm], ascending off_a and off_b
  int nm;
  int64_t items_a;           // part-A items of all members in one stage
  int64_t per_phase;         // items of one stage: every member's part A, then every part B
  int nphase;                // stages of this launch (3 x steps)
  unsigned long long* ticket;
  unsigned long long* done;  // [2 nm]: part-A items finished per member, then part-B items
  int* abort;
  int* err;                  // the batch's device error word
  const float* tabs;         // order 6's volume tables for shared memory (batch_tables), if present
  int tab_floats;
  uint64_t wait_ns;          // bound on every dependency wait
};

// Uploads every order's reference matrices to the kernel's constant banks (once per device)
// and returns the shared-memory tables the kernel stages (order 6's volume matrices, when
// orders[6]); off is unused (all zero).
int batch_tables(const bool orders[7], std::vector<float>& tabs, int off[7]);
// Dynamic shared memory of the kernel: the tables, a volume tile's rows, and the member
// descriptors when there are at most kSmemMembers of them.
constexpr int kSmemMembers = 64;
size_t batch_smem_bytes(int tab_floats, int nm);
int batch_grid(size_t smem);   // resident blocks of the persistent kernel (-1 on error)
int launch_batch_persistent(const BatchArgs& a, int grid, size_t smem, cudaStream_t s);
int launch_batch_advance(BMember* m, int nm, long long steps, cudaStream_t s);

}  // namespace rdg

/*
 * rdg.h -- C ABI of the GB300 (sm_103a) affine reconstructed nodal DG library.
 *
 * Method: Song & Srinivasan, "An efficient reconstruction algorithm for diffusion on
 * triangular grids using the nodal discontinuous Galerkin method" (arXiv 1912.06221).
 * The library evaluates the semi-discrete right-hand side of
 *
 *     u_t + div(v u) - div(D grad u) = s                       (Eq. convection_diffusion)
 *
 * on a triangle mesh in the reference-domain form of Eq.
 * NDG_diffusion_once_matrixForm_Fullyreference: a volume term M^{-1} S^T . F with
 * F = v u - D grad u, and surface terms (J_f / J) LIFT_f (F*.n) whose diffusive part is the
 * normal gradient of the polynomial reconstructed on the enclosed parallelogram of each
 * interior edge (Sec. 4, Algorithm aRDG).  Element-wise D enters the edge flux by the paper's
 * Algorithm 2 (D~ = RDG(D1,D2)) or Algorithm 1 (Sec. 3), chosen at rdg_operator_setup.
 * Time stepping is the three-stage SSP-RK3 scheme.
 *
 * Conventions shared with every caller:
 *  - order N in 1..6; Np = (N+1)(N+2)/2 nodes per triangle, Nfp = N+1 per face.
 *  - nodes: Warp & Blend points with alpha = 0 on the reference triangle
 *    {r,s >= -1, r+s <= 0} with vertices v1=(-1,-1), v2=(1,-1), v3=(-1,1), ordered row by
 *    row (for i = 0..N, for j = 0..N-i); element vertex k maps to v_k through the affine map
 *    x = -(r+s)/2 x1 + (r+1)/2 x2 + (s+1)/2 x3 (Eq. mapping_tri).
 *  - nodal arrays are row-major [K][Np] (element-major), in the precision chosen at
 *    rdg_operator_setup (double for RDG_FP64, float for RDG_FP32 and RDG_FP32_3XTF32).
 *  - triangles must be counter-clockwise; faces are (x1,x2), (x2,x3), (x3,x1).
 *
 * Status: every call returns 0 (RDG_OK) or a negative RDG_E* code; rdg_last_error() gives a
 * message.  Ownership: host arrays passed in are copied and stay the caller's; device
 * pointers passed in are borrowed for the duration of the call (work is enqueued on the
 * context's stream, so they must stay valid until that stream reaches it) and are never
 * freed by the library; the library owns and frees everything it allocates in
 * rdg_destroy.  Threading: one context per host thread at a time; all device work of a
 * context runs on its stream.
 */
#ifndef RDG_H
#define RDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rdg_ctx rdg_ctx;
typedef struct rdg_batch rdg_batch;

enum {
  RDG_OK = 0,
  RDG_EINVAL = -1,   /* bad argument (range, null pointer, size) */
  RDG_ENOMEM = -2,   /* device or host allocation failed */
  RDG_ECUDA = -3,    /* a CUDA runtime call failed */
  RDG_EMESH = -4,    /* mesh not valid: clockwise/degenerate triangle, non-manifold or unmatched edge */
  RDG_ERANK = -5,    /* reconstruction system not of full column rank */
  RDG_ETIMEOUT = -6, /* a bounded device wait (for the tensor core, 1 s) gave up */
  RDG_ESTATE = -7    /* call made in the wrong order (e.g. rhs before operator setup) */
};

enum { RDG_BC_PERIODIC = 0, RDG_BC_DIRICHLET = 1 };
/* Precision of the state and the hot path.  RDG_FP32_3XTF32: FP32 state with the edge flux in
 * its GEMM form on the tensor cores (split 3xTF32 products against shared reference
 * matrices, per-edge parameters instead of stored operators, see rdg_operator_setup); orders
 * N = 1..5 with RDG_IFACE_ALG2 or RDG_IFACE_HARMONIC (otherwise the RDG_FP32 path runs). */
enum { RDG_FP64 = 0, RDG_FP32 = 1, RDG_FP32_3XTF32 = 2 };
enum { RDG_TAU_CONST = 0, RDG_TAU_COS = 1, RDG_TAU_SIN = 2 };
/* Edge diffusion for element-wise D: the paper's Algorithm 2 (D~ = RDG(D1, D2) on the
 * diagonal times n . grad u~), the harmonic mean 2 D1 D2 / (D1 + D2) times n . grad u~ (not
 * in the paper: stable for high-contrast jumps, where Algorithm 2 gives growing modes), or
 * the paper's Algorithm 1 (n . RDG(D1 grad u~^1, D2 grad u~^2), u~^k the L2 projection of u~
 * onto sub-triangle k; also stable for such jumps).  Algorithm 2 and the harmonic rule agree
 * when D1 = D2; Algorithm 1 agrees with them on linear data. */
enum { RDG_IFACE_ALG2 = 0, RDG_IFACE_HARMONIC = 1, RDG_IFACE_ALG1 = 2 };
#define RDG_MAX_FORCING_TERMS 4

/* Library version string. */
const char* rdg_version(void);

/* Message for the last failing call on ctx (or for rdg_create when ctx is NULL). */
const char* rdg_last_error(const rdg_ctx* ctx);

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to run on (the
 * legacy default stream, cudaStreamLegacy, is accepted), or NULL for a stream the library
 * creates (non-blocking) and destroys.  Graphs are captured on a private stream and
 * launched on this one.  Also uploads the
 * reference operators of every order to the device on first use of that device.
 * Errors: RDG_EINVAL (device out of range), RDG_ECUDA, RDG_ENOMEM. */
int rdg_create(rdg_ctx** out, int device, void* cuda_stream);

/* Free every buffer the context owns and the context itself (NULL is accepted). */
int rdg_destroy(rdg_ctx* ctx);

/* Mesh (the triangulation of Sec. 3, affine elements of Eq. mapping_tri; the interior edges
 * are the ones Algorithm aRDG of Sec. 4 reconstructs on): nv vertices xy[2*nv]
 * (x0,y0,x1,y1,...), nt counter-clockwise triangles tri[3*nt]
 * (0-based vertex ids).  Two faces with the same pair of vertex ids form an edge; the faces
 * left over are matched by coincident midpoints.  bc = RDG_BC_PERIODIC: every face must meet
 * another face whose midpoint agrees modulo period[0..1] (period must be non-NULL); the neighbour's vertex
 * coordinates are translated onto the shared face.  bc = RDG_BC_DIRICHLET: faces met by no
 * other face are boundary edges whose outer side is the ghost triangle, the point
 * reflection of the element about the edge midpoint (period may be NULL).
 * Errors: RDG_EINVAL, RDG_EMESH (non-CCW or degenerate triangle, an edge shared by more
 * than two faces, an unmatched periodic face), RDG_ENOMEM. */
int rdg_mesh_upload(rdg_ctx* ctx, int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                    int32_t bc, const double* period);

/* One mesh split across ranks (Sec. 4, Algorithm aRDG: every edge reads all 2 Np values of
 * both neighbours, so a rank needs the full state of the other ranks' elements next to its
 * own).  Like rdg_mesh_upload, but triangles [n_owned, nt) are halo copies of elements that
 * other ranks own: faces of halo triangles that meet no other face become boundary edges
 * (ghost data zero unless set), so only the rows of halo triangles depend on them; a face of
 * an owned triangle left unmatched on a periodic mesh is still RDG_EMESH.  Every right-hand
 * side and stage then computes all nt rows, and the rows [0, n_owned) are exact as long as
 * the halo rows of each stage's input hold the owners' values (rdg_stage_buffer,
 * rdg_rows_gather/rdg_rows_scatter, rdg_rk_stage).  Errors: as rdg_mesh_upload, and
 * RDG_EINVAL for n_owned outside 0..nt. */
int rdg_mesh_upload_partition(rdg_ctx* ctx, int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                              int32_t bc, const double* period, int64_t n_owned);

/* Operators for order N (1..6) with element-wise diffusion D_elem[nt] (> 0), constant
 * velocity (vx, vy), arithmetic precision RDG_FP64, RDG_FP32 or RDG_FP32_3XTF32, interface rule
 * RDG_IFACE_ALG2, RDG_IFACE_ALG1 or RDG_IFACE_HARMONIC for the edge diffusion (Algorithm 1
 * folds D1 and D2 into the operator in place of D~).  Builds, in FP64 on the GPU,
 * the element metric terms and for every edge the enclosed parallelogram (Sec. 4.2), the
 * projections V^{-1} V_p V_rf^{-1} of both sides (Eq. totalProjection), the least-squares
 * reconstruction (Sec. 4.5) and the edge-normal gradient, folded with D~ = RDG(D1, D2)
 * (Algorithm 2), the edge Jacobian J_f and the upwind convective trace into one
 * Nfp x 2Np flux operator per edge, stored in the chosen precision.  With RDG_FP32_3XTF32
 * (N <= 5) no operator is stored: each edge keeps a parameter record (the orthonormal basis
 * at both sides' apex coordinates, kappa_R, kappa_S, -J_f D~_i, J_f v.n1), and the edge
 * kernel forms the flux as a tensor-core GEMM against reference matrices of the order (see
 * rdg_reference_operator which = 6).
 * Errors: RDG_ESTATE (no mesh), RDG_EINVAL, RDG_ERANK, RDG_ENOMEM, RDG_ECUDA. */
int rdg_operator_setup(rdg_ctx* ctx, int N, const double* D_elem, double vx, double vy, int precision,
                       int interface_rule);

/* rdg_operator_setup for the diagonal diffusion tensor D = (Dx, Dy) of Eq.
 * NDG_diffusion_once_matrixForm_reference_general (Sec. 3): element-wise Dx[nt], Dy[nt] (> 0),
 * volume flux F = v u - (Dx u_x, Dy u_y), and on every edge the chosen interface rule applied
 * per component (Algorithm 2: n . (D~x u~_x, D~y u~_y) with D~x = RDG(Dx1, Dx2) and likewise
 * for y; Algorithm 1: n . RDG((Dx^1 u~^1_x, Dy^1 u~^1_y), (Dx^2 u~^2_x, Dy^2 u~^2_y)); harmonic:
 * the per-component harmonic means), folded into the per-edge operators as for scalar D.
 * Stored operators only: with RDG_FP32_3XTF32 the RDG_FP32 path runs.  Errors: as
 * rdg_operator_setup (RDG_EINVAL when Dy is NULL). */
int rdg_operator_setup_aniso(rdg_ctx* ctx, int N, const double* Dx, const double* Dy, double vx, double vy,
                             int precision, int interface_rule);

/* rdg_operator_setup for a spatially varying D given at the nodes (Sec. 3: D a function of
 * space in Eq. NDG_diffusion_once_matrixForm_reference_general): D_nodal[nt][Np] (> 0) in the
 * element's node order.  The volume flux is the nodal product v u - D grad u; the edge
 * diffusion is, for RDG_IFACE_ALG2, D~ reconstructed on the diagonal from both elements'
 * nodal D (Algorithm 2), for RDG_IFACE_ALG1 each element's D evaluated at its sub-triangle's
 * nodes and multiplied into that sub-triangle's gradient before the second reconstruction
 * (Algorithm 1), for RDG_IFACE_HARMONIC the harmonic mean of the two elements' D at each face
 * node; a Dirichlet ghost's D is its element's D at the point reflections.  Stored operators
 * only (with RDG_FP32_3XTF32 the RDG_FP32 path runs; order 6 in FP32 forms the volume term on
 * the CUDA cores); not for rdg_rhs_eval_static or the persistent batch form.  Device memory:
 * rdg_query_bytes plus nt x Np values.  Errors: as rdg_operator_setup. */
int rdg_operator_setup_nodal(rdg_ctx* ctx, int N, const double* D_nodal, double vx, double vy, int precision,
                             int interface_rule);

/* Separable forcing (after rdg_operator_setup).  Source s(x,t) = sum_m S_m(x) tau_m(t) with
 * S given as nodal values S[nsrc][nt][Np] (host, double), tau_m = 1, cos(w t) or sin(w t)
 * per src_kind[m], src_omega[m].  Dirichlet ghost data g(x,t) = sum_m G_m(x) tau_m(t) with
 * G[nghost][nb][Np] (host, double) at the ghost nodes returned by rdg_get_ghost_coords.
 * nsrc, nghost <= RDG_MAX_FORCING_TERMS; 0 clears.  Errors: RDG_ESTATE, RDG_EINVAL. */
int rdg_set_forcing(rdg_ctx* ctx, int nsrc, const double* S, const int32_t* src_kind, const double* src_omega,
                    int nghost, const double* G, const int32_t* ghost_kind, const double* ghost_omega);

/* Counts after rdg_mesh_upload: triangles, edges (interior + boundary), boundary edges. */
int rdg_mesh_counts(const rdg_ctx* ctx, int64_t* nt, int64_t* n_edges, int64_t* n_boundary);

/* Physical node coordinates xy[nt][Np][2] (host, double) after rdg_operator_setup. */
int rdg_get_node_coords(rdg_ctx* ctx, double* xy);

/* Ghost-triangle node coordinates xy[nb][Np][2] (host, double) of the boundary edges, in the
 * order rdg_set_forcing expects G. */
int rdg_get_ghost_coords(rdg_ctx* ctx, double* xy);

/* Resident state u[nt][Np] in the context's precision; on_device != 0: u is a device
 * pointer (copied device to device), else a host pointer.  Errors: RDG_ESTATE, RDG_EINVAL. */
int rdg_set_state(rdg_ctx* ctx, const void* u, int on_device);
int rdg_get_state(rdg_ctx* ctx, void* out, int to_device);

/* rhs = L(u, t), the semi-discrete right-hand side of Eq. NDG_diffusion_once_matrixForm_Fullyreference
 * (Sec. 4.2; volume term M^{-1} S^T . F, surface terms (J_f/J) LIFT_f (F*.n) with the
 * reconstructed edge gradient of Algorithm aRDG and the interface rule chosen at setup,
 * plus the source s of Eq. convection_diffusion), for device arrays u, rhs [nt][Np] in the
 * context's precision (no host
 * synchronisation; enqueued on the context's stream).  Both must be 16-byte aligned and must
 * not overlap (RDG_EINVAL otherwise). */
int rdg_rhs_eval(rdg_ctx* ctx, const void* u_dev, void* rhs_dev, double t);

/* Allocation-free rhs = L(u, t), for callers that cannot allocate device memory where they
 * evaluate the right-hand side (inside another component's CUDA-graph capture, in loops
 * that must not hit cudaMalloc's implicit synchronisation, or under a pool allocator that
 * owns all device memory).  It computes the same right-hand side as rdg_rhs_eval, to rounding,
 * with the unfused pair of kernels (per-edge fluxes, then an element kernel that forms the
 * volume term, LIFT and sources), and keeps the per-edge fluxes in one static device array
 * compiled into the library, 8 MiB,
 * held by every GPU that loads the library until the process exits; it calls no allocating
 * routine.  Meshes needing more than 8 MiB of fluxes (n_edges x Nfp x element size) get
 * RDG_EINVAL with a message.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress with the device current) and caches it for the life of the
 * process, so the address is valid only while that device's primary context lives (not after
 * a cudaDeviceReset); make that first call before any stream capture.  Contexts using the
 * GEMM form of the edge flux (RDG_FP32_3XTF32 with N <= 5 and an interface rule other than
 * RDG_IFACE_ALG1) have no stored operators and get RDG_ESTATE.  All calls share the array, which keeps the last call's contents (every
 * flux is rewritten before it is read, so nothing is cleared): calls whose GPU work
 * overlaps (different streams or devices' contexts sharing a device) race on it.  The paper
 * has no counterpart to this entry point. */
int rdg_rhs_eval_static(rdg_ctx* ctx, const void* u_dev, void* rhs_dev, double t);

/* Time integrator of rdg_rk_step, rdg_solve_to_time and batch steps:
 * RDG_INTEGRATOR_SSP_RK3 (default) three-stage SSP-RK3, stages at t, t+dt, t+dt/2;
 * RDG_INTEGRATOR_LSRK54 the five-stage fourth-order low-storage scheme of Carpenter and
 * Kennedy (1994) that the paper's results use (Sec. 5), in its two-register form (the state
 * and one residual).  Errors: RDG_EINVAL for another value. */
enum { RDG_INTEGRATOR_SSP_RK3 = 0, RDG_INTEGRATOR_LSRK54 = 1 };
int rdg_set_integrator(rdg_ctx* ctx, int integrator);

/* Kernel form of a right-hand-side stage (Algorithm aRDG, Sec. 4.5, and the SSP-RK3 update;
 * the arithmetic is the same in every form):
 * RDG_STAGE_TWO_KERNELS  a stage kernel (edge fluxes into the two elements' face slots,
 *                        volume terms) and an element kernel (LIFT, sources, stage update);
 * RDG_STAGE_ONE_KERNEL   one element kernel that also computes its three edges' fluxes (each
 *                        edge's operator read by both of its elements; one launch per stage);
 * RDG_STAGE_AUTO         (default) the form measured faster for the context's order and
 *                        precision on GB300 (one kernel for FP32 order 1, two otherwise).
 * The one-kernel form serves rdg_rhs_eval and SSP-RK3 stages of contexts with stored
 * operators; the low-storage integrator (which updates its input in place), the GEMM form
 * and FP32 order 6 (tensor-core volume term) keep two kernels whatever is set.  Errors:
 * RDG_EINVAL for another value.  rdg_get_stage_form reports the form in use for a
 * right-hand-side stage (RDG_STAGE_ONE_KERNEL or RDG_STAGE_TWO_KERNELS) in *form. */
enum { RDG_STAGE_AUTO = 0, RDG_STAGE_TWO_KERNELS = 1, RDG_STAGE_ONE_KERNEL = 2 };
int rdg_set_stage_form(rdg_ctx* ctx, int form);
int rdg_get_stage_form(const rdg_ctx* ctx, int* form);

/* Test hook of the tensor-core kernels' bounded waits (no counterpart in the paper): from
 * the next stage on, tile `tile` of every launch of the context's tensor-core kernel is never
 * released (the GEMM form of the edge flux: edge tile of 128 edges, never handed to the MMAs
 * by its producer; FP32 order 6: element tile of 128 elements of the volume term, whose MMAs
 * are never issued), so the threads that wait for it give up after 1-2 s, the launch leaves
 * early (its results undefined) and the next rdg_synchronize returns RDG_ETIMEOUT; tile = -1
 * removes the hold.  Other contexts ignore it.  Errors: RDG_EINVAL for tile < -1. */
int rdg_gemm_hold_tile(rdg_ctx* ctx, int64_t tile);

/* One step of the resident state from time t with step dt with the selected integrator;
 * enqueued, no host synchronisation. */
int rdg_rk_step(rdg_ctx* ctx, double t, double dt);

/* One stage of one step of the selected integrator from step start t with step dt
 * (SSP-RK3: stage 0, 1, 2 at t, t+dt, t+dt/2; the low-storage scheme: stages 0..4): the same
 * launches as the stage inside rdg_rk_step, enqueued.  Stages 0..last in order make one step.
 * For a mesh split across ranks the caller refreshes the halo rows of rdg_stage_buffer(stage)
 * before each stage.  Errors: RDG_ESTATE, RDG_EINVAL (stage out of range, bad dt). */
int rdg_rk_stage(rdg_ctx* ctx, int stage, double t, double dt);

/* The same stage in two parts, so that a split mesh's halo exchange overlaps the work that
 * does not need it (the per-stage exchange of the partitioned Algorithm aRDG, Sec. 4.5: an
 * edge reads all 2 Np values of both neighbours).  Part 0 enqueues the edges with no halo
 * side (the first e_split edges of a partitioned upload; e_split is a multiple of 32) and the
 * owned elements' volume terms: it reads owned rows of the stage input only.  Part 1 enqueues
 * the remaining edges and the element update; the caller writes the halo rows of
 * rdg_stage_buffer(stage) between the two (rdg_rows_scatter).  Parts 0 then 1 give the same
 * owned rows as rdg_rk_stage (halo rows of the stage output are not defined).  Contexts that
 * cannot split a stage (not partitioned, the GEMM form, FP32 order 6, the one-kernel form)
 * run the whole stage in part 1 and nothing in part 0.  Errors: as rdg_rk_stage, RDG_EINVAL
 * for a part other than 0 or 1. */
int rdg_rk_stage_part(rdg_ctx* ctx, int stage, int part, double t, double dt);

/* Owned elements and e_split (edges [0, e_split) touch no halo element) of the uploaded
 * mesh: n_owned = nt and e_split = the edge count for an unsplit upload.  Errors:
 * RDG_ESTATE before a mesh upload. */
int rdg_split_counts(const rdg_ctx* ctx, int64_t* n_owned, int64_t* e_split);

/* Device pointer of the input buffer [nt][Np] of stage `stage` (SSP-RK3: the state, then the
 * two stage buffers; the low-storage scheme: the state for every stage), owned by the context
 * and valid until the next rdg_operator_setup or rdg_destroy. */
int rdg_stage_buffer(rdg_ctx* ctx, int stage, void** dev_ptr);

/* Rows of Np values in the context's precision on the device: gather dst[i][:] =
 * src[idx[i]][:] or scatter dst[idx[i]][:] = src[i][:] for i < n (idx: device int32).  The
 * halo exchange of a split mesh: gather the rows a neighbour rank needs into a contiguous
 * send buffer, scatter received rows into the halo rows.  Indexes outside 0..nt-1 are
 * skipped and reported by rdg_synchronize.  Enqueued on the context stream. */
int rdg_rows_gather(rdg_ctx* ctx, const void* src_dev, const int32_t* idx_dev, int64_t n, void* dst_dev);
int rdg_rows_scatter(rdg_ctx* ctx, const void* src_dev, const int32_t* idx_dev, int64_t n, void* dst_dev);

/* nsteps steps of the selected integrator from t0 with step dt, replayed from a CUDA
 * graph of a fixed chunk of steps (captured on first use for a given dt); enqueued. */
int rdg_solve_to_time(rdg_ctx* ctx, double t0, double dt, int64_t nsteps);

/* Bytes of the per-edge flux operators that every stage loads with an evict-last L2 policy,
 * so they stay L2-resident from one stage to the next instead of streaming from HBM again
 * (the rest is streamed evict-first).  -1 (the default) and 0 stream everything.  Affects
 * speed only, never results. */
int rdg_set_l2_resident_bytes(rdg_ctx* ctx, int64_t bytes);

/* Per-kernel timing.  With enable != 0 every later edge-flux and element-update kernel launch
 * of ctx is bracketed by CUDA events on the context stream (rdg_solve_to_time then steps
 * without its graph).  rdg_kernel_stats waits for the stream and returns, for kernel class
 * 0 (edge flux) and 1 (element update), the number of launches and the summed device
 * milliseconds since the last reset; reset != 0 clears them afterwards. */
int rdg_profile(rdg_ctx* ctx, int enable);
int rdg_kernel_stats(rdg_ctx* ctx, int64_t* launches, double* ms, int reset);

/* Wait for the context's stream; returns RDG_ECUDA if device work failed or a kernel's
 * index self-check found a corrupt edge table (the device error word is then cleared). */
int rdg_synchronize(rdg_ctx* ctx);

/* Device bytes a context allocates for order N, nt triangles, n_edges edges (n_boundary of
 * them boundary edges), precision, nsrc/nghost forcing terms: the admission figure a
 * scheduler compares with its memory budget. */
int rdg_query_bytes(int N, int64_t nt, int64_t n_edges, int64_t n_boundary, int precision, int nsrc, int nghost,
                    int64_t* bytes);

/* Reference operators of order N as the library computed them (host FP64), for checks:
 * which = 0 nodes r,s [2][Np]; 1 Dr [Np][Np]; 2 Ds; 3 LIFT [Np][3 Nfp]; 4 pseudo-inverse of
 * the reconstruction system [Mp][2Np]; 5 mass matrix [Np][Np]; 6 the reference factors of
 * the GEMM form of the edge operator, X[2 sides][Np m][Nfp i][2 (d_R, d_S)][Np l]: side k's
 * diffusive edge gradient in rotated node order is
 * sum_rho kappa_rho sum_m psi_m(alpha_k, beta_k) X[k][m][i][rho][l] (Sec. 4.4-4.5, Eq.
 * totalProjection: the projection is polynomial in the apex coordinates); 7 the node
 * permutations [3][Np] (rotated node i of face f is node perm[f][i]); 8 the rotated-order
 * indices of the shared face's nodes [Nfp]; for a nodal D (rdg_operator_setup_nodal):
 * 9 RVV[2 sides j][Nfp][Np] = Phi_diag A+_j Vinv, the reconstruction on the diagonal of side
 * j's modal data, brought to nodal input; 10 GR[2 j][2 k][Np][Np] = Dr V A_j A+_k Vinv and
 * 11 GS (Ds in place of Dr): Algorithm 1's edge gradient with D at the sub-triangle nodes is
 * sum_j s_j RVV[j] diag(D_p^j) (kappa_R GR[j][k] + kappa_S GS[j][k]) u_k,rot, s_1 = 1,
 * s_2 = -1 (Sec. 3, Algorithm 1; Sec. 4.5).  out must hold the stated number of doubles. */
int rdg_reference_operator(int N, int which, double* out);

/* Per-edge flux operators in FP64 as built on the GPU: W[n_edges][Nfp][2Np] (host,
 * double), plus per edge (k1, f1, k2, f2) into ids[n_edges][4] (k2 = -1-b for the b-th
 * boundary edge).  For checks and tooling; not needed for solving. */
int rdg_get_edge_operators(rdg_ctx* ctx, double* W, int32_t* ids);

/* ---- Measurement ---------------------------------------------------------------------------
 * Points of the error norms: a collapsed Gauss rule on every triangle, exact for total degree
 * 2N + 4 ((N + 3)^2 points per triangle).  *nq receives the number of points per triangle;
 * xy (may be NULL) receives their physical coordinates [nt][nq][2] (host, double), where the
 * caller evaluates the exact solution for rdg_error_norms.  Errors: RDG_ESTATE, RDG_EINVAL. */
int rdg_error_quadrature(rdg_ctx* ctx, int* nq, double* xy);

/* Error norms of Eq. L2_norm_cellUnit and Eq. Linf_norm_cellUnit (Sec. 5), in FP64 on the GPU:
 * with e = u - u_e on each triangle k, *l2 = sqrt(sum_k int_k e^2 / sum_k |k|) and *linf =
 * max_k (1/|k|) int_k |e| (the largest cell mean, as the paper defines its L_inf norm).
 * u_dev: nodal values [nt][Np] in the context's precision on the device, or NULL for the
 * resident state; ue_q_dev: the exact solution at the points of rdg_error_quadrature, device
 * double [nt][nq].  Allocates its scratch on the context stream and waits for it.  Errors:
 * RDG_ESTATE, RDG_EINVAL, RDG_ENOMEM, RDG_ECUDA. */
int rdg_error_norms(rdg_ctx* ctx, const void* u_dev, const double* ue_q_dev, double* l2, double* linf);

/* FMA rate of device `device` in FLOP/s (an FMA counts 2) for precision RDG_FP32 or RDG_FP64:
 * independent FMA chains on every SM, timed with CUDA events, best of four launches after two
 * warm-up launches, at whatever clocks the GPU runs (nothing is locked or changed).  The
 * compute side of the right-hand side's roofline.  Errors: RDG_EINVAL, RDG_ENOMEM, RDG_ECUDA. */
int rdg_peak_fma(int device, int precision, double* flops_per_second);

/* Time of a plain streaming read of `bytes` (16..64 GiB) from device memory on `device`:
 * 16-byte evict-first loads, grid-stride over 8 blocks per SM, a 512 MiB buffer written
 * between timed reads (larger than L2), median of eight launches after two warm-up ones,
 * CUDA events.  The size-matched bound of an HBM-streaming kernel: a standalone launch pays a
 * fixed ramp-up and tail, so a read of 100 MB reaches well under the copy peak measured on
 * gigabytes.  Allocates bytes + 512 MiB and frees them.  Errors: RDG_EINVAL, RDG_ENOMEM,
 * RDG_ECUDA. */
int rdg_stream_read(int device, int64_t bytes, double* seconds);

/* ---- Batched stepping of independent problems ------------------------------------------
 * Many independent solves (different meshes, orders N = 1..6, precisions, dt) advanced
 * together: every member is a context set up as for a single solve (mesh, operators,
 * forcing, state); a batch step advances every member by the same number of SSP-RK3 steps
 * (Sec. 2.1 time integration of each problem's semi-discrete system, each with its own dt).
 * The members' kernels are captured as parallel branches of one CUDA graph of `chunk` steps
 * and replayed with one launch per chunk, so problems of all sizes and orders run
 * concurrently.  The paper solves one problem at a time and has no counterpart.
 * Ownership: the batch borrows its member contexts; remove a member (or destroy the batch)
 * before destroying the context.  Ordering: a batch step runs after the work already
 * enqueued on every member's stream, and later work on a member's stream runs after it. */

/* Create an empty batch on `device`.  cuda_stream: stream the graph is launched on (NULL: an
 * own non-blocking stream).  chunk: steps per captured graph (1..1024).  RDG_EINVAL on a
 * bad argument, RDG_ECUDA if stream/event creation fails. */
int rdg_batch_create(rdg_batch** out, int device, void* cuda_stream, int chunk);
/* Wait for the batch's work and free it (not the member contexts).  NULL is a no-op. */
int rdg_batch_destroy(rdg_batch* b);
/* Text of the batch's last error. */
const char* rdg_batch_last_error(const rdg_batch* b);
/* Add a context whose operators are set up: its resident state is stepped from time t0
 * with step dt.  RDG_ESTATE without operators; RDG_EINVAL for another device, a
 * non-positive dt, a non-finite t0, or a context already in the batch. */
int rdg_batch_add(rdg_batch* b, rdg_ctx* ctx, double t0, double dt);
/* Remove a member (waits for its branch); RDG_EINVAL if ctx is not a member. */
int rdg_batch_remove(rdg_batch* b, rdg_ctx* ctx);
/* Steps per captured graph from now on (1..1024; the graph is captured again on the next
 * step).  RDG_EINVAL outside the range. */
int rdg_batch_set_chunk(rdg_batch* b, int chunk);
/* Number of members into *n. */
int rdg_batch_size(const rdg_batch* b, int* n);
/* Enqueue nsteps SSP-RK3 steps of every member: floor(nsteps/chunk) replays of the graph
 * (captured on first use after the membership changed) and the remainder as direct
 * launches on the branch streams.  Each member continues from its own time. */
int rdg_batch_step(rdg_batch* b, int64_t nsteps);
/* Wait for the batch stream, then check every member as rdg_synchronize does.  Returns
 * RDG_ETIMEOUT if a dependency wait of the persistent form gave up (the members' states are
 * then undefined; the batch's error word is cleared). */
int rdg_batch_synchronize(rdg_batch* b);

/* Form of a batch step.  RDG_BATCH_GRAPH: the members' own stage launches as parallel
 * branches of one CUDA graph.  RDG_BATCH_PERSISTENT: one persistent launch per chunk of steps
 * for all members (captured in the CUDA graph like the branches): blocks take work items
 * (member, stage, part, tile) from a ticket counter in stage order; part A of a stage (edge
 * fluxes, volume terms) starts once the member's previous stage is done, part B (surface
 * terms and stage update per element) once the member's part A is done; every wait is
 * bounded (see rdg_batch_set_wait_limit).  It needs every member FP32 with stored operators and the
 * SSP-RK3 integrator (order 6 then forms its volume term on the CUDA cores).  RDG_BATCH_AUTO
 * (the default): persistent when every member fits, else the graph.  The persistent form
 * takes each member's set-up (forcing, dt, tiles) when the membership last changed.
 * Errors: RDG_EINVAL (unknown mode, or RDG_BATCH_PERSISTENT with a member that does not fit). */
enum { RDG_BATCH_AUTO = 0, RDG_BATCH_GRAPH = 1, RDG_BATCH_PERSISTENT = 2 };
int rdg_batch_set_mode(rdg_batch* b, int mode);
/* The form the next step uses (RDG_BATCH_GRAPH or RDG_BATCH_PERSISTENT) into *mode. */
int rdg_batch_get_mode(const rdg_batch* b, int* mode);
/* Tile mapping of the persistent form for members of order N: edges_per_thread (1 or 2)
 * edges per thread of an edge tile (128 or 256 edges per tile; element tiles are 128
 * elements) and tiles_per_item (1, 2 or 4) consecutive tiles per work item, which amortises
 * an item's dependency check over more work.  Chosen per order by the autotuner.  Errors:
 * RDG_EINVAL. */
int rdg_batch_set_tiles(rdg_batch* b, int N, int edges_per_thread, int tiles_per_item);
/* Bound on every dependency wait of the persistent kernel (default 1 s; (0, 60]): a wait that
 * runs out records the timeout, and the launch ends without finishing its work. */
int rdg_batch_set_wait_limit(rdg_batch* b, double seconds);
/* Test hook for the bounded waits: the persistent kernel never releases stage `phase`
 * (3 x step + stage within a launch) of member `member` (index in the order of
 * rdg_batch_add), so that stage's items wait until the wait limit and the step reports
 * RDG_ETIMEOUT.  member = -1 removes the hold. */
int rdg_batch_hold_phase(rdg_batch* b, int member, int64_t phase);

#ifdef __cplusplus
}
#endif

#endif /* RDG_H */

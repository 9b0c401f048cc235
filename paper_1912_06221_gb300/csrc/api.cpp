// C ABI of the aRDG library: context, mesh connectivity, operator setup, forcing, state,
// right-hand side, SSP-RK3 stepping and CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "context.h"

using namespace rdg;

namespace {

std::mutex g_err_mu;
std::string g_create_err;
std::mutex g_tab_mu;
std::vector<bool> g_tab_uploaded;

int fail(rdg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_err = msg;
  }
  return code;
}

int cuda_fail(rdg_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? RDG_ENOMEM : RDG_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);  \
  } while (0)

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the context stream):
// a plain cudaFree waits for the whole device, which would stall every other context's
// queued work whenever one context is set up or released.
template <typename T>
cudaError_t dalloc(T** p, size_t bytes, cudaStream_t s) {
  return cudaMallocAsync(reinterpret_cast<void**>(p), bytes, s);
}
template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

void free_ops(rdg_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  dfree(ctx->d_W, s);
  dfree(ctx->d_k1, s);
  dfree(ctx->d_k2, s);
  dfree(ctx->d_eref, s);
  dfree(ctx->d_geo, s);
  dfree(ctx->d_flux, s);
  dfree(ctx->d_u, s);
  dfree(ctx->d_u1, s);
  dfree(ctx->d_u2, s);
  dfree(ctx->d_S, s);
  dfree(ctx->d_G, s);
  dfree(ctx->d_vol, s);
  dfree(ctx->d_fb, s);
  dfree(ctx->d_f12, s);
  dfree(ctx->d_Dn, s);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  ctx->ops_ok = false;
  ctx->frc = Forcing();
}

cudaEvent_t take_event(rdg_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Sum the elapsed times of completed event pairs (the caller has synchronised the stream).
void drain_events(rdg_ctx* ctx) {
  for (int c = 0; c < 2; ++c) {
    for (auto& pr : ctx->ev_pending[c]) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
        ctx->prof_ms[c] += ms;
        ctx->prof_n[c] += 1;
      }
      ctx->ev_pool.push_back(pr.first);
      ctx->ev_pool.push_back(pr.second);
    }
    ctx->ev_pending[c].clear();
  }
}

void free_events(rdg_ctx* ctx) {
  cudaStreamSynchronize(ctx->stream);
  drain_events(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  ctx->ev_pool.clear();
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int64_t w_bytes(int N, int64_t E, int esz) {
  const int64_t tiles = (E + kTile - 1) / kTile;
  return tiles * w_vecs_per_edge(N, esz) * kTile * 16;
}

bool uses_gemm(int N, int precision, int iface = RDG_IFACE_ALG2) {
  return precision == RDG_FP32_3XTF32 && N <= kMaxGemmN && iface != RDG_IFACE_ALG1;
}

// bytes of the per-edge data the edge kernel streams: operators or GEMM-form parameters
int64_t edge_data_bytes(int N, int64_t E, int precision) {
  if (uses_gemm(N, precision)) return (E + kTile - 1) / kTile * gemm_param_words(N) * kTile * 16;
  return w_bytes(N, E, precision == RDG_FP64 ? 8 : 4);
}

bool valid_precision(int p) { return p == RDG_FP32 || p == RDG_FP64 || p == RDG_FP32_3XTF32; }

const int kFaceA[3] = {0, 1, 2}, kFaceB[3] = {1, 2, 0};

}  // namespace

extern "C" {

const char* rdg_version(void) { return "rdg-gb300 0.1 (sm_103a)"; }

const char* rdg_last_error(const rdg_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_create_err.c_str();
}

int rdg_create(rdg_ctx** out, int device, void* cuda_stream) {
  if (!out) return fail(nullptr, RDG_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return fail(nullptr, RDG_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (device < 0 || device >= n) return fail(nullptr, RDG_EINVAL, "device out of range");
  DeviceGuard g(device);
  {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if ((int)g_tab_uploaded.size() < n) g_tab_uploaded.resize(n, false);
    if (!g_tab_uploaded[device]) {
      for (int N = 1; N <= kMaxN; ++N) {
        const char* msg = "";
        if (!get_refops(N, &msg)) return fail(nullptr, RDG_ERANK, msg);
      }
      if (upload_elem_tables(device) != RDG_OK)
        return fail(nullptr, RDG_ECUDA, "uploading reference operators failed");
      g_tab_uploaded[device] = true;
    }
  }
  rdg_ctx* c = new (std::nothrow) rdg_ctx();
  if (!c) return fail(nullptr, RDG_ENOMEM, "host allocation failed");
  c->device = device;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, RDG_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  e = dalloc(&c->d_time, sizeof(TimeState), c->stream);
  if (e == cudaSuccess) e = dalloc(&c->d_err, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    dfree(c->d_time, c->stream);
    dfree(c->d_err, c->stream);
    cudaStreamSynchronize(c->stream);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return fail(nullptr, RDG_ENOMEM, "device allocation failed");
  }
  *out = c;
  return RDG_OK;
}

int rdg_destroy(rdg_ctx* ctx) {
  if (!ctx) return RDG_OK;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_ops(ctx);
  free_events(ctx);
  dfree(ctx->d_time, ctx->stream);
  dfree(ctx->d_err, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return RDG_OK;
}

}  // extern "C"

// Mesh upload; elements [n_owned, nt) are halo copies of another rank's elements, whose faces
// may stay unmatched (they become boundary edges that only the halo rows depend on).
static int mesh_upload_impl(rdg_ctx* ctx, int64_t nv, const double* xy, int64_t nt, const int32_t* tri, int32_t bc,
                            const double* period, int64_t n_owned) {
  if (!ctx) return RDG_EINVAL;
  if (nv <= 0 || nt <= 0 || !xy || !tri) return fail(ctx, RDG_EINVAL, "empty mesh or NULL arrays");
  if (nt > (int64_t)1 << 30) return fail(ctx, RDG_EINVAL, "too many triangles (max 2^30)");
  if (bc != RDG_BC_PERIODIC && bc != RDG_BC_DIRICHLET) return fail(ctx, RDG_EINVAL, "bc must be PERIODIC or DIRICHLET");
  if (bc == RDG_BC_PERIODIC && (!period || !(period[0] > 0) || !(period[1] > 0)))
    return fail(ctx, RDG_EINVAL, "periodic mesh needs a positive period");
  if (n_owned < 0 || n_owned > nt) return fail(ctx, RDG_EINVAL, "n_owned must be in 0..nt");
  free_ops(ctx);
  ctx->mesh_ok = false;
  ctx->K = nt;
  ctx->n_owned = n_owned;
  ctx->bc = bc;
  ctx->exy.assign(nt * 6, 0.0);
  double hmin = 1e300;
  for (int64_t k = 0; k < nt; ++k) {
    for (int c = 0; c < 3; ++c) {
      int32_t v = tri[3 * k + c];
      if (v < 0 || v >= nv) return fail(ctx, RDG_EMESH, "vertex id out of range in triangle " + std::to_string(k));
      ctx->exy[6 * k + 2 * c] = xy[2 * v];
      ctx->exy[6 * k + 2 * c + 1] = xy[2 * v + 1];
    }
    const double* p = &ctx->exy[6 * k];
    double J = (p[2] - p[0]) * (p[5] - p[1]) - (p[4] - p[0]) * (p[3] - p[1]);
    double l2 = std::max({(p[2] - p[0]) * (p[2] - p[0]) + (p[3] - p[1]) * (p[3] - p[1]),
                          (p[4] - p[2]) * (p[4] - p[2]) + (p[5] - p[3]) * (p[5] - p[3]),
                          (p[0] - p[4]) * (p[0] - p[4]) + (p[1] - p[5]) * (p[1] - p[5])});
    if (!(J > 1e-12 * l2)) return fail(ctx, RDG_EMESH, "triangle " + std::to_string(k) + " is clockwise or degenerate");
    hmin = std::min(hmin, std::sqrt(l2));
  }
  (void)hmin;
  // Faces are matched first by their vertex ids: a counting sort of the faces by their lower
  // vertex id, then equal upper ids within each (small) bucket.  The faces left over (domain
  // boundary, periodic images, vertices duplicated at one point) are matched by their
  // midpoint modulo the period.  Linear in the mesh size for any vertex numbering.
  const int64_t nf = 3 * nt;
  std::vector<int64_t> partner(nf, -1);
  {
    auto lo_hi = [&](int64_t i, int32_t* lo, int32_t* hi) {
      const int32_t a = tri[3 * (i / 3) + kFaceA[i % 3]], b = tri[3 * (i / 3) + kFaceB[i % 3]];
      *lo = std::min(a, b);
      *hi = std::max(a, b);
    };
    std::vector<int64_t> start(nv + 1, 0);
    for (int64_t i = 0; i < nf; ++i) {
      int32_t lo, hi;
      lo_hi(i, &lo, &hi);
      start[lo + 1]++;
    }
    for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
    std::vector<int64_t> fill(start.begin(), start.end() - 1), bucket(nf);
    for (int64_t i = 0; i < nf; ++i) {
      int32_t lo, hi;
      lo_hi(i, &lo, &hi);
      bucket[fill[lo]++] = i;
    }
    std::vector<std::pair<int32_t, int64_t>> run;
    for (int64_t v = 0; v < nv; ++v) {
      const int64_t b0 = start[v], n = start[v + 1] - b0;
      if (n < 2) continue;
      run.clear();
      for (int64_t j = 0; j < n; ++j) {
        int32_t lo, hi;
        lo_hi(bucket[b0 + j], &lo, &hi);
        run.push_back({hi, bucket[b0 + j]});
      }
      std::sort(run.begin(), run.end());
      for (int64_t j = 0; j < n;) {
        int64_t q = j + 1;
        while (q < n && run[q].first == run[j].first) ++q;
        if (q - j > 2) return fail(ctx, RDG_EMESH, "non-manifold edge (shared by more than two faces)");
        if (q - j == 2) {
          partner[run[j].second] = run[j + 1].second;
          partner[run[j + 1].second] = run[j].second;
        }
        j = q;
      }
    }
  }
  {
    struct Key {
      long long x, y;
      bool operator==(const Key& o) const { return x == o.x && y == o.y; }
    };
    struct KeyHash {
      size_t operator()(const Key& k) const { return std::hash<long long>()(k.x * 1000003LL ^ k.y); }
    };
    const double scale = (bc == RDG_BC_PERIODIC) ? 1e9 : 1e12;
    auto canon = [&](double x, double y) {
      if (bc == RDG_BC_PERIODIC) {
        x = std::fmod(x, period[0]);
        if (x < 0) x += period[0];
        if (std::fabs(x - period[0]) < 1e-9) x = 0;
        y = std::fmod(y, period[1]);
        if (y < 0) y += period[1];
        if (std::fabs(y - period[1]) < 1e-9) y = 0;
      }
      return Key{std::llround(x * scale), std::llround(y * scale)};
    };
    std::unordered_map<Key, std::vector<int64_t>, KeyHash> table;
    for (int64_t i = 0; i < nf; ++i) {
      if (partner[i] >= 0) continue;
      const double* p = &ctx->exy[6 * (i / 3)];
      const int f = (int)(i % 3);
      double mx = 0.5 * (p[2 * kFaceA[f]] + p[2 * kFaceB[f]]), my = 0.5 * (p[2 * kFaceA[f] + 1] + p[2 * kFaceB[f] + 1]);
      table[canon(mx, my)].push_back(i);
    }
    for (auto& kv : table) {
      auto& l = kv.second;
      if (l.size() > 2) return fail(ctx, RDG_EMESH, "non-manifold edge (shared by more than two faces)");
      if (l.size() == 2) {
        partner[l[0]] = l[1];
        partner[l[1]] = l[0];
      }
    }
  }
  // edges in the order of their first face (sorted by first element, for locality of the
  // neighbour gathers): interior edges, then boundary edges
  std::vector<EdgeRec> inner, bnd;
  inner.reserve(nf / 2 + 1);
  for (int64_t i = 0; i < nf; ++i) {
    const int64_t j = partner[i];
    if (j >= 0 && j < i) continue;
    if (j < 0) {
      if (bc == RDG_BC_PERIODIC && i / 3 < n_owned) return fail(ctx, RDG_EMESH, "unmatched face on a periodic mesh");
      bnd.push_back(EdgeRec{(int32_t)(i / 3), (int32_t)(i % 3), -1, 1, 0.0, 0.0});
      continue;
    }
    EdgeRec r;
    r.k1 = (int32_t)(i / 3);
    r.f1 = (int32_t)(i % 3);
    r.k2 = (int32_t)(j / 3);
    r.f2 = (int32_t)(j % 3);
    const double* p1 = &ctx->exy[6 * r.k1];
    const double* p2 = &ctx->exy[6 * r.k2];
    // the two faces must run in opposite directions over the same segment
    double ax = p1[2 * kFaceA[r.f1]], ay = p1[2 * kFaceA[r.f1] + 1];
    double bx = p1[2 * kFaceB[r.f1]], by = p1[2 * kFaceB[r.f1] + 1];
    double cx = p2[2 * kFaceA[r.f2]], cy = p2[2 * kFaceA[r.f2] + 1];
    double dx = p2[2 * kFaceB[r.f2]], dy = p2[2 * kFaceB[r.f2] + 1];
    r.shx = 0.5 * (ax + bx) - 0.5 * (cx + dx);
    r.shy = 0.5 * (ay + by) - 0.5 * (cy + dy);
    double tol = 1e-9 * std::sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
    if (std::fabs(dx + r.shx - ax) > tol || std::fabs(dy + r.shy - ay) > tol ||
        std::fabs(cx + r.shx - bx) > tol || std::fabs(cy + r.shy - by) > tol)
      return fail(ctx, RDG_EMESH, "faces meeting at an edge do not coincide or run the same way");
    inner.push_back(r);
  }
  for (size_t b = 0; b < bnd.size(); ++b) bnd[b].k2 = -1 - (int32_t)b;
  ctx->edges = inner;
  ctx->edges.insert(ctx->edges.end(), bnd.begin(), bnd.end());
  ctx->E = (int64_t)ctx->edges.size();
  ctx->B = (int64_t)bnd.size();
  ctx->e_split = ctx->E;
  if (n_owned < nt) {
    // a split mesh: first a multiple of 32 (whole operator tiles) of the edges with no halo
    // side, which a stage may process while the halo rows are still in flight, then the rest
    // (order otherwise kept)
    auto no_halo = [&](const EdgeRec& r) { return r.k1 < n_owned && r.k2 < n_owned; };
    std::vector<EdgeRec> a, rest;
    for (const EdgeRec& r : ctx->edges) (no_halo(r) ? a : rest).push_back(r);
    ctx->e_split = (int64_t)a.size() / kTile * kTile;
    rest.insert(rest.begin(), a.begin() + ctx->e_split, a.end());
    a.resize(ctx->e_split);
    a.insert(a.end(), rest.begin(), rest.end());
    ctx->edges.swap(a);
  }
  ctx->bedge.assign(ctx->B, -1);
  for (int64_t e = 0; e < ctx->E; ++e)
    if (ctx->edges[e].k2 < 0) ctx->bedge[-1 - (int64_t)ctx->edges[e].k2] = e;
  ctx->eref.assign(3 * nt, -1);
  for (int64_t e = 0; e < ctx->E; ++e) {
    const EdgeRec& r = ctx->edges[e];
    ctx->eref[(int64_t)r.f1 * nt + r.k1] = (int32_t)(2 * e);
    if (r.k2 >= 0) ctx->eref[(int64_t)r.f2 * nt + r.k2] = (int32_t)(2 * e + 1);
  }
  for (int64_t i = 0; i < 3 * nt; ++i)
    if (ctx->eref[i] < 0) return fail(ctx, RDG_EMESH, "a face has no edge");
  if (2 * ctx->E > (int64_t)INT32_MAX) return fail(ctx, RDG_EINVAL, "too many edges");
  ctx->mesh_ok = true;
  return RDG_OK;
}

extern "C" {

int rdg_mesh_upload(rdg_ctx* ctx, int64_t nv, const double* xy, int64_t nt, const int32_t* tri, int32_t bc,
                    const double* period) {
  return mesh_upload_impl(ctx, nv, xy, nt, tri, bc, period, nt);
}

int rdg_mesh_upload_partition(rdg_ctx* ctx, int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                              int32_t bc, const double* period, int64_t n_owned) {
  return mesh_upload_impl(ctx, nv, xy, nt, tri, bc, period, n_owned);
}

int rdg_mesh_counts(const rdg_ctx* ctx, int64_t* nt, int64_t* n_edges, int64_t* n_boundary) {
  if (!ctx || !ctx->mesh_ok) return RDG_ESTATE;
  if (nt) *nt = ctx->K;
  if (n_edges) *n_edges = ctx->E;
  if (n_boundary) *n_boundary = ctx->B;
  return RDG_OK;
}

int rdg_query_bytes(int N, int64_t nt, int64_t n_edges, int64_t n_boundary, int precision, int nsrc, int nghost,
                    int64_t* bytes) {
  if (!bytes || N < 1 || N > kMaxN || nt < 0 || n_edges < 0 || n_boundary < 0) return RDG_EINVAL;
  if (!valid_precision(precision)) return RDG_EINVAL;
  const int64_t esz = precision == RDG_FP64 ? 8 : 4;
  const int64_t Np = np_of(N), Nfp = nfp_of(N);
  // the stored operators: an upper bound for every mode (the GEMM form's parameter records
  // are smaller, and it falls back to stored operators for N = 6 and Algorithm 1)
  int64_t b = w_bytes(N, n_edges, (int)esz);
  b += 3 * 4 * n_edges + 3 * 4 * nt;          // k1, k2, face pairs, eref
  b += 3 * nt * Nfp * esz;                     // face fluxes (fused form)
  b += 6 * esz * nt;                           // element coefficients
  b += n_edges * Nfp * esz;                    // edge fluxes
  b += 4 * nt * Np * esz;                      // state, two stage buffers, volume terms
  b += (int64_t)nsrc * nt * Np * esz + (int64_t)nghost * n_boundary * Np * esz;
  *bytes = b;
  return RDG_OK;
}

}  // extern "C"

static int build_edge_ops(rdg_ctx* ctx, const RefOps* o, void* W_tiled, int esz, double* W_dense,
                          float* P_tiled = nullptr) {
  const int64_t K = ctx->K, E = ctx->E;
  std::vector<int32_t> k1(E), f1(E), k2(E), f2(E);
  std::vector<double> sh(2 * E);
  for (int64_t e = 0; e < E; ++e) {
    k1[e] = ctx->edges[e].k1;
    f1[e] = ctx->edges[e].f1;
    k2[e] = ctx->edges[e].k2;
    f2[e] = ctx->edges[e].f2;
    sh[2 * e] = ctx->edges[e].shx;
    sh[2 * e + 1] = ctx->edges[e].shy;
  }
  std::vector<double> refs = pack_setup_refs(*o);
  double *d_xy = nullptr, *d_sh = nullptr, *d_D = nullptr, *d_Dy = nullptr, *d_refs = nullptr;
  double *d_Dn64 = nullptr, *d_nref = nullptr;
  const bool aniso = !ctx->Dy.empty();
  const bool nodal = !ctx->Dn.empty();
  std::vector<double> nref;
  if (nodal) {   // RVV [2][Nfp][Np], GR [2][2][Np][Np], GS [2][2][Np][Np]
    for (int j = 0; j < 2; ++j) nref.insert(nref.end(), o->RVV[j].begin(), o->RVV[j].end());
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k) nref.insert(nref.end(), o->GR[j][k].begin(), o->GR[j][k].end());
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k) nref.insert(nref.end(), o->GS[j][k].begin(), o->GS[j][k].end());
  }
  int32_t *d_i = nullptr;
  int rc = RDG_OK;
  cudaError_t e;
  cudaStream_t s = ctx->stream;
  auto cleanup = [&]() {
    dfree(d_xy, s);
    dfree(d_sh, s);
    dfree(d_D, s);
    dfree(d_Dy, s);
    dfree(d_Dn64, s);
    dfree(d_nref, s);
    dfree(d_refs, s);
    dfree(d_i, s);
    cudaStreamSynchronize(s);
  };
  if ((e = dalloc(&d_xy, K * 6 * sizeof(double), s)) != cudaSuccess ||
      (e = dalloc(&d_sh, 2 * E * sizeof(double), s)) != cudaSuccess ||
      (e = dalloc(&d_D, K * sizeof(double), s)) != cudaSuccess ||
      (aniso && (e = dalloc(&d_Dy, K * sizeof(double), s)) != cudaSuccess) ||
      (nodal && (e = dalloc(&d_Dn64, ctx->Dn.size() * sizeof(double), s)) != cudaSuccess) ||
      (nodal && (e = dalloc(&d_nref, nref.size() * sizeof(double), s)) != cudaSuccess) ||
      (e = dalloc(&d_refs, refs.size() * sizeof(double), s)) != cudaSuccess ||
      (e = dalloc(&d_i, 4 * E * sizeof(int32_t), s)) != cudaSuccess) {
    cleanup();
    return cuda_fail(ctx, e, "setup buffers");
  }
  if ((e = cudaMemcpyAsync(d_xy, ctx->exy.data(), K * 6 * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_sh, sh.data(), 2 * E * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_D, ctx->Dk.data(), K * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (aniso && (e = cudaMemcpyAsync(d_Dy, ctx->Dy.data(), K * sizeof(double), cudaMemcpyHostToDevice, s)) !=
                    cudaSuccess) ||
      (nodal && (e = cudaMemcpyAsync(d_Dn64, ctx->Dn.data(), ctx->Dn.size() * sizeof(double), cudaMemcpyHostToDevice,
                                     s)) != cudaSuccess) ||
      (nodal && (e = cudaMemcpyAsync(d_nref, nref.data(), nref.size() * sizeof(double), cudaMemcpyHostToDevice, s)) !=
                    cudaSuccess) ||
      (e = cudaMemcpyAsync(d_refs, refs.data(), refs.size() * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_i, k1.data(), E * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_i + E, f1.data(), E * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_i + 2 * E, k2.data(), E * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_i + 3 * E, f2.data(), E * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    cleanup();
    return cuda_fail(ctx, e, "setup upload");
  }
  if (W_tiled) {
    if ((e = cudaMemsetAsync(W_tiled, 0, w_bytes(ctx->N, E, esz), s)) != cudaSuccess) {
      cleanup();
      return cuda_fail(ctx, e, "W clear");
    }
  }
  EdgeSetupIn in{d_xy, d_i, d_i + E, d_i + 2 * E, d_i + 3 * E, d_sh, d_D, d_Dy, d_Dn64, d_nref, d_refs, E, ctx->vx,
                 ctx->vy, ctx->iface, (int64_t)refs.size()};
  rc = setup_edges(ctx->N, in, W_tiled, esz, W_dense, P_tiled, s);
  if (rc == RDG_OK && ctx->d_geo && !W_dense)
    rc = setup_elements(K, d_xy, nodal ? nullptr : d_D, d_Dy, ctx->vx, ctx->vy, ctx->d_geo, esz, s);
  e = cudaStreamSynchronize(s);
  cleanup();
  if (rc != RDG_OK) return fail(ctx, rc, "setup kernel launch failed");
  if (e != cudaSuccess) return cuda_fail(ctx, e, "setup kernels");
  return RDG_OK;
}

extern "C" {

}  // extern "C"

// Operator set-up; Dy (may be null) is the y diffusion of a diagonal tensor (D_elem then
// holds the x diffusion), which needs the stored operators.
static int operator_setup_impl(rdg_ctx* ctx, int N, const double* D_elem, const double* Dy, double vx, double vy,
                               int precision, int interface_rule, const double* Dn = nullptr) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->mesh_ok) return fail(ctx, RDG_ESTATE, "rdg_mesh_upload must come first");
  if (N < 1 || N > kMaxN) return fail(ctx, RDG_EINVAL, "order N must be in 1..6");
  if (!valid_precision(precision))
    return fail(ctx, RDG_EINVAL, "precision must be RDG_FP32, RDG_FP64 or RDG_FP32_3XTF32");
  if (!D_elem) return fail(ctx, RDG_EINVAL, "D_elem is NULL");
  if (interface_rule != RDG_IFACE_ALG2 && interface_rule != RDG_IFACE_HARMONIC && interface_rule != RDG_IFACE_ALG1)
    return fail(ctx, RDG_EINVAL, "interface rule must be RDG_IFACE_ALG2, RDG_IFACE_HARMONIC or RDG_IFACE_ALG1");
  if (!std::isfinite(vx) || !std::isfinite(vy)) return fail(ctx, RDG_EINVAL, "velocity not finite");
  for (int64_t k = 0; k < ctx->K; ++k)
    if (!(D_elem[k] > 0) || !std::isfinite(D_elem[k]) || (Dy && (!(Dy[k] > 0) || !std::isfinite(Dy[k]))))
      return fail(ctx, RDG_EINVAL, "D must be positive and finite");
  const char* msg = "";
  const RefOps* o = get_refops(N, &msg);
  if (!o) return fail(ctx, RDG_ERANK, msg);
  DeviceGuard g(ctx->device);
  free_ops(ctx);
  ctx->N = N;
  ctx->prec = precision;
  ctx->esz = precision == RDG_FP64 ? 8 : 4;
  // the GEMM form folds one isotropic element-wise D~
  ctx->gemm = uses_gemm(N, precision, interface_rule) && !Dy && !Dn;
  ctx->vx = vx;
  ctx->vy = vy;
  ctx->iface = interface_rule;
  ctx->Dk.assign(D_elem, D_elem + ctx->K);
  if (Dy) ctx->Dy.assign(Dy, Dy + ctx->K);
  else ctx->Dy.clear();
  if (Dn) ctx->Dn.assign(Dn, Dn + ctx->K * np_of(N));
  else ctx->Dn.clear();
  const int64_t K = ctx->K, E = ctx->E, Np = o->Np, Nfp = o->Nfp, esz = ctx->esz;
  const int64_t stb = K * Np * esz;
  CK(dalloc(&ctx->d_W, ctx->gemm ? edge_data_bytes(N, E, precision) : w_bytes(N, E, (int)esz), ctx->stream));
  CK(dalloc(&ctx->d_k1, E * 4, ctx->stream));
  CK(dalloc(&ctx->d_k2, E * 4, ctx->stream));
  CK(dalloc(&ctx->d_eref, 3 * K * 4, ctx->stream));
  CK(dalloc(&ctx->d_geo, 6 * K * esz, ctx->stream));
  CK(dalloc(&ctx->d_flux, E * Nfp * esz, ctx->stream));
  CK(dalloc(&ctx->d_u, stb, ctx->stream));
  CK(dalloc(&ctx->d_u1, stb, ctx->stream));
  CK(dalloc(&ctx->d_u2, stb, ctx->stream));
  CK(dalloc(&ctx->d_vol, stb, ctx->stream));
  CK(dalloc(&ctx->d_fb, K * 3 * Nfp * esz, ctx->stream));
  CK(dalloc(&ctx->d_f12, E * 4, ctx->stream));
  if (Dn) {   // the volume term's nodal D, in the context's precision
    CK(dalloc(&ctx->d_Dn, K * Np * esz, ctx->stream));
    if (esz == 8) {
      CK(cudaMemcpyAsync(ctx->d_Dn, Dn, K * Np * 8, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    } else {
      std::vector<float> f(Dn, Dn + K * Np);
      CK(cudaMemcpyAsync(ctx->d_Dn, f.data(), K * Np * 4, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
  }
  std::vector<int32_t> k1(E), k2(E), f12(E);
  for (int64_t e = 0; e < E; ++e) {
    k1[e] = ctx->edges[e].k1;
    k2[e] = ctx->edges[e].k2;
    f12[e] = ctx->edges[e].f1 | ((ctx->edges[e].k2 >= 0 ? ctx->edges[e].f2 : 0) << 2);
  }
  CK(cudaMemcpyAsync(ctx->d_f12, f12.data(), E * 4, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_k1, k1.data(), E * 4, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_k2, k2.data(), E * 4, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_eref, ctx->eref.data(), 3 * K * 4, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_u, 0, stb, ctx->stream));
  int rc = ctx->gemm ? build_edge_ops(ctx, o, nullptr, (int)esz, nullptr, static_cast<float*>(ctx->d_W))
                     : build_edge_ops(ctx, o, ctx->d_W, (int)esz, nullptr);
  if (rc != RDG_OK) {
    free_ops(ctx);
    return rc;
  }
  ctx->ops_ok = true;
  return RDG_OK;
}

extern "C" {

int rdg_operator_setup(rdg_ctx* ctx, int N, const double* D_elem, double vx, double vy, int precision,
                       int interface_rule) {
  return operator_setup_impl(ctx, N, D_elem, nullptr, vx, vy, precision, interface_rule);
}

int rdg_operator_setup_aniso(rdg_ctx* ctx, int N, const double* Dx, const double* Dy, double vx, double vy,
                             int precision, int interface_rule) {
  if (ctx && !Dy) return fail(ctx, RDG_EINVAL, "Dy is NULL");
  return operator_setup_impl(ctx, N, Dx, Dy, vx, vy, precision, interface_rule);
}

int rdg_operator_setup_nodal(rdg_ctx* ctx, int N, const double* D_nodal, double vx, double vy, int precision,
                             int interface_rule) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->mesh_ok) return fail(ctx, RDG_ESTATE, "rdg_mesh_upload must come first");
  if (!D_nodal) return fail(ctx, RDG_EINVAL, "D_nodal is NULL");
  if (N < 1 || N > kMaxN) return fail(ctx, RDG_EINVAL, "order N must be in 1..6");
  const int64_t Np = np_of(N);
  std::vector<double> mean(ctx->K, 0.0);   // per element, only to keep every kernel argument defined
  for (int64_t k = 0; k < ctx->K; ++k) {
    for (int64_t j = 0; j < Np; ++j) {
      const double d = D_nodal[k * Np + j];
      if (!(d > 0) || !std::isfinite(d)) return fail(ctx, RDG_EINVAL, "D must be positive and finite");
      mean[k] += d / Np;
    }
  }
  return operator_setup_impl(ctx, N, mean.data(), nullptr, vx, vy, precision, interface_rule, D_nodal);
}

int rdg_get_edge_operators(rdg_ctx* ctx, double* W, int32_t* ids) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  DeviceGuard g(ctx->device);
  const RefOps* o = get_refops(ctx->N, nullptr);
  const int64_t nw = (int64_t)o->Nfp * 2 * o->Np * ctx->E;
  if (W) {
    double* d = nullptr;
    CK(dalloc(&d, nw * sizeof(double), ctx->stream));
    int rc = build_edge_ops(ctx, o, nullptr, 8, d);
    if (rc == RDG_OK) {
      cudaError_t e = cudaMemcpyAsync(W, d, nw * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
      dfree(d, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "copy W");
    } else {
      dfree(d, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      return rc;
    }
  }
  if (ids)
    for (int64_t e = 0; e < ctx->E; ++e) {
      ids[4 * e] = ctx->edges[e].k1;
      ids[4 * e + 1] = ctx->edges[e].f1;
      ids[4 * e + 2] = ctx->edges[e].k2;
      ids[4 * e + 3] = ctx->edges[e].f2;
    }
  return RDG_OK;
}

int rdg_get_node_coords(rdg_ctx* ctx, double* xy) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!xy) return fail(ctx, RDG_EINVAL, "xy is NULL");
  const RefOps* o = get_refops(ctx->N, nullptr);
  for (int64_t k = 0; k < ctx->K; ++k) {
    const double* p = &ctx->exy[6 * k];
    for (int i = 0; i < o->Np; ++i) {
      double r = o->r[i], s = o->s[i];
      double a = -(r + s) / 2, b = (r + 1) / 2, c = (s + 1) / 2;
      xy[(k * o->Np + i) * 2] = a * p[0] + b * p[2] + c * p[4];
      xy[(k * o->Np + i) * 2 + 1] = a * p[1] + b * p[3] + c * p[5];
    }
  }
  return RDG_OK;
}

int rdg_get_ghost_coords(rdg_ctx* ctx, double* xy) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!xy && ctx->B) return fail(ctx, RDG_EINVAL, "xy is NULL");
  const RefOps* o = get_refops(ctx->N, nullptr);
  const int kc[3] = {2, 0, 1};
  for (int64_t b = 0; b < ctx->B; ++b) {
    const EdgeRec& r = ctx->edges[ctx->bedge[b]];
    const double* p = &ctx->exy[6 * r.k1];
    double e1x = p[2 * kFaceA[r.f1]], e1y = p[2 * kFaceA[r.f1] + 1];
    double e2x = p[2 * kFaceB[r.f1]], e2y = p[2 * kFaceB[r.f1] + 1];
    double qx = p[2 * kc[r.f1]], qy = p[2 * kc[r.f1] + 1];
    // ghost vertices: v1 = reflected apex, v2 = e2, v3 = e1
    double g[6] = {e1x + e2x - qx, e1y + e2y - qy, e2x, e2y, e1x, e1y};
    for (int i = 0; i < o->Np; ++i) {
      double rr = o->r[i], ss = o->s[i];
      double a = -(rr + ss) / 2, bb = (rr + 1) / 2, c = (ss + 1) / 2;
      xy[(b * o->Np + i) * 2] = a * g[0] + bb * g[2] + c * g[4];
      xy[(b * o->Np + i) * 2 + 1] = a * g[1] + bb * g[3] + c * g[5];
    }
  }
  return RDG_OK;
}

}  // extern "C"

static int upload_converted(rdg_ctx* ctx, void** dst, const double* src, int64_t n) {
  dfree(*dst, ctx->stream);
  if (n == 0) return RDG_OK;
  CK(dalloc(dst, n * ctx->esz, ctx->stream));
  if (ctx->esz == 8) {
    CK(cudaMemcpyAsync(*dst, src, n * 8, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    std::vector<float> f(src, src + n);
    CK(cudaMemcpyAsync(*dst, f.data(), n * 4, cudaMemcpyHostToDevice, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));   // the converted host copy goes out of scope
  return RDG_OK;
}

extern "C" {

int rdg_set_forcing(rdg_ctx* ctx, int nsrc, const double* S, const int32_t* src_kind, const double* src_omega,
                    int nghost, const double* G, const int32_t* ghost_kind, const double* ghost_omega) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (nsrc < 0 || nsrc > RDG_MAX_FORCING_TERMS || nghost < 0 || nghost > RDG_MAX_FORCING_TERMS)
    return fail(ctx, RDG_EINVAL, "at most 4 source and 4 ghost terms");
  if ((nsrc && (!S || !src_kind || !src_omega)) || (nghost && (!G || !ghost_kind || !ghost_omega)))
    return fail(ctx, RDG_EINVAL, "NULL forcing array");
  if (nghost && ctx->B == 0) return fail(ctx, RDG_EINVAL, "ghost data given but the mesh has no boundary edges");
  for (int m = 0; m < nsrc; ++m)
    if (src_kind[m] < 0 || src_kind[m] > 2) return fail(ctx, RDG_EINVAL, "bad source kind");
  for (int m = 0; m < nghost; ++m)
    if (ghost_kind[m] < 0 || ghost_kind[m] > 2) return fail(ctx, RDG_EINVAL, "bad ghost kind");
  DeviceGuard g(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  const int64_t Np = np_of(ctx->N);
  int rc = upload_converted(ctx, &ctx->d_S, S, (int64_t)nsrc * ctx->K * Np);
  if (rc != RDG_OK) return rc;
  rc = upload_converted(ctx, &ctx->d_G, G, (int64_t)nghost * ctx->B * Np);
  if (rc != RDG_OK) return rc;
  Forcing f;
  f.nsrc = nsrc;
  f.nghost = nghost;
  for (int m = 0; m < nsrc; ++m) {
    f.kind[m] = src_kind[m];
    f.omega[m] = src_omega[m];
  }
  for (int m = 0; m < nghost; ++m) {
    f.gkind[m] = ghost_kind[m];
    f.gomega[m] = ghost_omega[m];
  }
  ctx->frc = f;
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  return RDG_OK;
}

int rdg_set_state(rdg_ctx* ctx, const void* u, int on_device) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!u) return fail(ctx, RDG_EINVAL, "u is NULL");
  DeviceGuard g(ctx->device);
  const int64_t bytes = ctx->K * np_of(ctx->N) * ctx->esz;
  CK(cudaMemcpyAsync(ctx->d_u, u, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
  return RDG_OK;
}

int rdg_get_state(rdg_ctx* ctx, void* out, int to_device) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!out) return fail(ctx, RDG_EINVAL, "out is NULL");
  DeviceGuard g(ctx->device);
  const int64_t bytes = ctx->K * np_of(ctx->N) * ctx->esz;
  CK(cudaMemcpyAsync(out, ctx->d_u, bytes, to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!to_device) CK(cudaStreamSynchronize(ctx->stream));
  return RDG_OK;
}

}  // extern "C"

namespace {

// stream kernels go to: the capture stream while a graph is being recorded
cudaStream_t ls(const rdg_ctx* ctx) { return ctx->capturing ? ctx->cap_stream : ctx->stream; }

// Operator tiles loaded evict-last: the leading tiles up to the keep budget.  The default
// is none: on the 131072-triangle N=4 workload (119 MB of operators) keeping 32-96 MB
// resident measured no faster and 64 MB or more measured slower than streaming it all.
int64_t keep_tiles(const rdg_ctx* ctx) {
  int64_t bytes = ctx->l2_keep_bytes;
  if (bytes < 0) bytes = 0;
  const int64_t tile = (int64_t)w_vecs_per_edge(ctx->N, ctx->esz) * kTile * 16;
  return tile > 0 ? bytes / tile : 0;
}

// Volume kernel on a stream forked from `st` and joined back after the edge kernel, so the
// tensor-core volume term and the HBM-bound operator stream share the SMs.  Works the same
// eagerly and under graph capture (the fork and join become graph edges).
// Edges [e0, e1) of a stage's edge arguments (e0 a multiple of the 32-edge operator tile):
// the edge ids, face ids and operator tiles offset by e0.
template <typename T>
EdgeArgs<T> edge_subrange(const rdg_ctx* ctx, const EdgeArgs<T>& ea, int64_t e0, int64_t e1) {
  EdgeArgs<T> r = ea;
  const int64_t t0 = e0 / kTile;
  const int64_t tile_bytes = (int64_t)w_vecs_per_edge(ctx->N, ctx->esz) * kTile * 16;
  r.k1 = ea.k1 + e0;
  r.k2 = ea.k2 + e0;
  r.f12 = ea.f12 + e0;
  r.W = static_cast<const char*>(ea.W) + t0 * tile_bytes;
  r.E = e1 - e0;
  r.keep_tiles = std::max<int64_t>(0, ea.keep_tiles - t0);
  return r;
}

int enqueue_split_stage(rdg_ctx* ctx, const EdgeArgs<float>& ea, cudaStream_t st) {
  // created on first use; each one again on a later call if its creation failed
  if (!ctx->side_stream && cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->side_stream = nullptr;
    return RDG_ECUDA;
  }
  if (!ctx->ev_fork && cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    ctx->ev_fork = nullptr;
    return RDG_ECUDA;
  }
  if (!ctx->ev_join && cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    ctx->ev_join = nullptr;
    return RDG_ECUDA;
  }
  if (cudaEventRecord(ctx->ev_fork, st) != cudaSuccess) return RDG_ECUDA;
  if (cudaStreamWaitEvent(ctx->side_stream, ctx->ev_fork, 0) != cudaSuccess) return RDG_ECUDA;
  int rc = launch_volume32(ctx->N, ea, ctx->side_stream);
  // the join is recorded even after a failed launch, so a capture never ends with the side
  // stream still attached
  if (cudaEventRecord(ctx->ev_join, ctx->side_stream) != cudaSuccess && rc == RDG_OK) rc = RDG_ECUDA;
  if (rc == RDG_OK) rc = launch_edge_only32(ctx->N, ea, st);
  if (cudaStreamWaitEvent(st, ctx->ev_join, 0) != cudaSuccess && rc == RDG_OK) rc = RDG_ECUDA;
  return rc;
}

// Whether a right-hand-side stage of this context runs as one kernel (elem_fused_kernel):
// stored operators, not FP32 order 6 (its volume term runs on the tensor cores beside the
// edge stream); by default at FP32 order 1 only, the one case where it measured faster on
// GB300 (circle pulse, 131072 triangles: 5.26 against 7.41 us per stage; order 2 10.4-12.6
// against 10.6-10.7, FP64 slower at every order).
bool one_kernel_stage(const rdg_ctx* ctx) {
  if (ctx->gemm || (ctx->esz == 4 && split_volume32(ctx->N))) return false;
  const bool fast = ctx->esz == 4 && ctx->N == 1;
  const int form = ctx->stage_form == RDG_STAGE_AUTO ? (fast ? RDG_STAGE_ONE_KERNEL : RDG_STAGE_TWO_KERNELS)
                                                     : ctx->stage_form;
  return form == RDG_STAGE_ONE_KERNEL;
}

// Whether a stage of this context can run in two parts around a halo exchange (the stage
// kernel and element kernel form on a split mesh).
bool splittable_stage(const rdg_ctx* ctx, int mode) {
  return ctx->n_owned < ctx->K && !ctx->gemm && !(ctx->esz == 4 && split_volume32(ctx->N)) &&
         !(mode <= 3 && one_kernel_stage(ctx));
}

// part -1: the whole stage.  On a split mesh, part 0: the edges with no halo side and the owned
// elements' volume terms (they read owned rows only); part 1: the remaining edges and the
// element update.  A stage that cannot be split runs whole in part 1 (part 0 enqueues nothing).
template <typename T>
int enqueue_stage(rdg_ctx* ctx, const void* us, const void* un, void* out, int mode, T dt, const TimeArg& ta,
                  void* out2 = nullptr, T rka = T(0), T rkb = T(0), int part = -1) {
  EdgeArgs<T> ea{ctx->d_k1, ctx->d_k2, ctx->d_W, (const T*)us, (T*)ctx->d_flux, (const T*)ctx->d_G,
                 ctx->E, ctx->B, ctx->frc, ta, ctx->d_err, ctx->K, (T*)ctx->d_vol,
                 (const T*)ctx->d_geo, ctx->d_f12, (T*)ctx->d_fb, keep_tiles(ctx), (const T*)ctx->d_Dn};
  ElemArgs<T> la{(const T*)us, (const T*)un, (T*)out, (const T*)ctx->d_flux, ctx->d_eref, (const T*)ctx->d_geo,
                 (const T*)ctx->d_S, ctx->K, dt, ctx->frc, ta, ctx->d_err, ctx->E, (const T*)ctx->d_vol,
                 (const T*)ctx->d_fb, (T*)out2, rka, rkb};
  cudaStream_t st = ls(ctx);
  if (part >= 0 && splittable_stage(ctx, mode)) {
    int rc = RDG_OK;
    if (part == 0) {
      if (ctx->n_owned == 0) return RDG_OK;
      EdgeArgs<T> e0 = ea;
      e0.E = ctx->e_split;
      e0.Kvol = ctx->n_owned;
      if constexpr (sizeof(T) == 4) rc = launch_edge_vol32(ctx->N, e0, st);
      else rc = launch_edge_vol64(ctx->N, e0, st);
      return rc;
    }
    const EdgeArgs<T> e1 = edge_subrange(ctx, ea, ctx->e_split, ctx->E);
    if constexpr (sizeof(T) == 4) rc = launch_edge_only32(ctx->N, e1, st);
    else rc = launch_edge_only64(ctx->N, e1, st);
    if (rc == RDG_OK) {
      if constexpr (sizeof(T) == 4) rc = launch_elem_lite32(ctx->N, mode, la, st);
      else rc = launch_elem_lite64(ctx->N, mode, la, st);
    }
    return rc;
  }
  if (part == 0) return RDG_OK;
  const bool prof = ctx->prof && !ctx->capturing;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  if (prof)
    for (auto& e : ev) e = take_event(ctx);
  int rc;
  if (mode <= 3 && one_kernel_stage(ctx)) {
    // one launch: the edge part of the timing is empty
    if (prof) {
      cudaEventRecord(ev[0], st);
      cudaEventRecord(ev[1], st);
      cudaEventRecord(ev[2], st);
    }
    if constexpr (sizeof(T) == 4) rc = launch_fused32(ctx->N, mode, ea, la, st);
    else rc = launch_fused64(ctx->N, mode, ea, la, st);
    if (prof) {
      cudaEventRecord(ev[3], st);
      ctx->ev_pending[0].push_back({ev[0], ev[1]});
      ctx->ev_pending[1].push_back({ev[2], ev[3]});
    }
    return rc;
  }
  if (prof) cudaEventRecord(ev[0], st);
  if constexpr (sizeof(T) == 4) {
    if (ctx->gemm) {
      EdgeArgs<T> eg = ea;
      eg.hold_tile = ctx->gemm_hold;
      rc = launch_gemm32(ctx->N, eg, st);
    }
    else if (split_volume32(ctx->N) && !ctx->d_Dn) {
      EdgeArgs<T> eg = ea;
      eg.hold_tile = ctx->gemm_hold;
      rc = enqueue_split_stage(ctx, eg, st);
    }
    else rc = launch_edge_vol32(ctx->N, ea, st);
  } else {
    rc = launch_edge_vol64(ctx->N, ea, st);
  }
  if (prof) {
    cudaEventRecord(ev[1], st);
    cudaEventRecord(ev[2], st);
  }
  if (rc == RDG_OK) {
    if constexpr (sizeof(T) == 4) rc = launch_elem_lite32(ctx->N, mode, la, st);
    else rc = launch_elem_lite64(ctx->N, mode, la, st);
  }
  if (prof) {
    cudaEventRecord(ev[3], st);
    ctx->ev_pending[0].push_back({ev[0], ev[1]});
    ctx->ev_pending[1].push_back({ev[2], ev[3]});
  }
  return rc;
}

// Five-stage fourth-order low-storage Runge-Kutta scheme (Carpenter and Kennedy 1994, the
// integrator of the paper's Sec. 5): published coefficients a_i, b_i and stage times c_i.
constexpr double kLsrkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                              -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
constexpr double kLsrkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                              1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                              2277821191437.0 / 14882151754819.0};
constexpr double kLsrkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                              2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

template <typename T>
int enqueue_lsrk_step(rdg_ctx* ctx, const TimeArg& base, double dt) {
  // two registers: u (d_u) and the residual du (d_u1), both updated in place per stage
  int rc = RDG_OK;
  for (int i = 0; i < 5 && rc == RDG_OK; ++i) {
    TimeArg ti = base;
    ti.off = base.off + kLsrkC[i];
    rc = enqueue_stage<T>(ctx, ctx->d_u, ctx->d_u1, ctx->d_u, 4, (T)dt, ti, ctx->d_u1, (T)kLsrkA[i], (T)kLsrkB[i]);
  }
  return rc;
}

int enqueue_rk_step(rdg_ctx* ctx, const TimeArg& base, double dt) {
  if (ctx->integrator == RDG_INTEGRATOR_LSRK54)
    return ctx->esz == 4 ? enqueue_lsrk_step<float>(ctx, base, dt) : enqueue_lsrk_step<double>(ctx, base, dt);
  // stage times t, t + dt, t + dt/2 (as offsets in units of dt)
  TimeArg t1 = base, t2 = base, t3 = base;
  t2.off = base.off + 1.0;
  t3.off = base.off + 0.5;
  int rc;
  if (ctx->esz == 4) {
    float d = (float)dt;
    rc = enqueue_stage<float>(ctx, ctx->d_u, nullptr, ctx->d_u1, 1, d, t1);
    if (rc == RDG_OK) rc = enqueue_stage<float>(ctx, ctx->d_u1, ctx->d_u, ctx->d_u2, 2, d, t2);
    if (rc == RDG_OK) rc = enqueue_stage<float>(ctx, ctx->d_u2, ctx->d_u, ctx->d_u, 3, d, t3);
  } else {
    rc = enqueue_stage<double>(ctx, ctx->d_u, nullptr, ctx->d_u1, 1, dt, t1);
    if (rc == RDG_OK) rc = enqueue_stage<double>(ctx, ctx->d_u1, ctx->d_u, ctx->d_u2, 2, dt, t2);
    if (rc == RDG_OK) rc = enqueue_stage<double>(ctx, ctx->d_u2, ctx->d_u, ctx->d_u, 3, dt, t3);
  }
  return rc;
}

// Input buffer of stage `stage` of the selected integrator (SSP-RK3: u, u1, u2; the
// low-storage scheme updates u in place every stage).
void* stage_input(rdg_ctx* ctx, int stage) {
  if (ctx->integrator == RDG_INTEGRATOR_LSRK54) return ctx->d_u;
  return stage == 0 ? ctx->d_u : (stage == 1 ? ctx->d_u1 : ctx->d_u2);
}

// One stage of the selected integrator, the same launches as the stage inside
// enqueue_rk_step (time offsets in units of dt from the step start in base).
int enqueue_one_stage(rdg_ctx* ctx, int stage, const TimeArg& base, double dt, int part = -1) {
  TimeArg ts = base;
  if (ctx->integrator == RDG_INTEGRATOR_LSRK54) {
    ts.off = base.off + kLsrkC[stage];
    if (ctx->esz == 4)
      return enqueue_stage<float>(ctx, ctx->d_u, ctx->d_u1, ctx->d_u, 4, (float)dt, ts, ctx->d_u1, (float)kLsrkA[stage],
                                  (float)kLsrkB[stage], part);
    return enqueue_stage<double>(ctx, ctx->d_u, ctx->d_u1, ctx->d_u, 4, dt, ts, ctx->d_u1, kLsrkA[stage], kLsrkB[stage],
                                 part);
  }
  static const double off[3] = {0.0, 1.0, 0.5};
  ts.off = base.off + off[stage];
  void* in = stage_input(ctx, stage);
  void* out = stage == 0 ? ctx->d_u1 : (stage == 1 ? ctx->d_u2 : ctx->d_u);
  const void* un = stage == 0 ? nullptr : ctx->d_u;
  if (ctx->esz == 4) return enqueue_stage<float>(ctx, in, un, out, stage + 1, (float)dt, ts, nullptr, 0.0f, 0.0f, part);
  return enqueue_stage<double>(ctx, in, un, out, stage + 1, dt, ts, nullptr, 0.0, 0.0, part);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

namespace rdg {

int enqueue_rk_step_on(rdg_ctx* ctx, cudaStream_t s, const TimeArg& base, double dt) {
  cudaStream_t saved = ctx->cap_stream;
  const bool was = ctx->capturing;
  ctx->cap_stream = s;
  ctx->capturing = true;
  int rc = enqueue_rk_step(ctx, base, dt);
  ctx->cap_stream = saved;
  ctx->capturing = was;
  return rc;
}

}  // namespace rdg

extern "C" {

int rdg_rhs_eval(rdg_ctx* ctx, const void* u_dev, void* rhs_dev, double t) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!u_dev || !rhs_dev) return fail(ctx, RDG_EINVAL, "NULL device array");
  if (!aligned16(u_dev) || !aligned16(rhs_dev)) return fail(ctx, RDG_EINVAL, "device arrays must be 16-byte aligned");
  if (u_dev == rhs_dev) return fail(ctx, RDG_EINVAL, "u and rhs must not overlap");
  DeviceGuard g(ctx->device);
  TimeArg ta{nullptr, t, 1.0, 0.0};
  int rc = ctx->esz == 4 ? enqueue_stage<float>(ctx, u_dev, nullptr, rhs_dev, 0, 0.0f, ta)
                         : enqueue_stage<double>(ctx, u_dev, nullptr, rhs_dev, 0, 0.0, ta);
  return rc == RDG_OK ? RDG_OK : fail(ctx, rc, "kernel launch failed");
}

int rdg_rk_step(rdg_ctx* ctx, double t, double dt) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!(dt > 0) || !std::isfinite(t)) return fail(ctx, RDG_EINVAL, "dt must be positive and t finite");
  DeviceGuard g(ctx->device);
  TimeArg ta{nullptr, t, dt, 0.0};
  int rc = enqueue_rk_step(ctx, ta, dt);
  return rc == RDG_OK ? RDG_OK : fail(ctx, rc, "kernel launch failed");
}

int rdg_rk_stage(rdg_ctx* ctx, int stage, double t, double dt) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!(dt > 0) || !std::isfinite(t)) return fail(ctx, RDG_EINVAL, "dt must be positive and t finite");
  const int nst = ctx->integrator == RDG_INTEGRATOR_LSRK54 ? 5 : 3;
  if (stage < 0 || stage >= nst) return fail(ctx, RDG_EINVAL, "stage out of range for the integrator");
  DeviceGuard g(ctx->device);
  TimeArg ta{nullptr, t, dt, 0.0};
  int rc = enqueue_one_stage(ctx, stage, ta, dt);
  return rc == RDG_OK ? RDG_OK : fail(ctx, rc, "kernel launch failed");
}

int rdg_rk_stage_part(rdg_ctx* ctx, int stage, int part, double t, double dt) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!(dt > 0) || !std::isfinite(t)) return fail(ctx, RDG_EINVAL, "dt must be positive and t finite");
  const int nst = ctx->integrator == RDG_INTEGRATOR_LSRK54 ? 5 : 3;
  if (stage < 0 || stage >= nst) return fail(ctx, RDG_EINVAL, "stage out of range for the integrator");
  if (part != 0 && part != 1) return fail(ctx, RDG_EINVAL, "part must be 0 or 1");
  DeviceGuard g(ctx->device);
  TimeArg ta{nullptr, t, dt, 0.0};
  int rc = enqueue_one_stage(ctx, stage, ta, dt, part);
  return rc == RDG_OK ? RDG_OK : fail(ctx, rc, "kernel launch failed");
}

int rdg_split_counts(const rdg_ctx* ctx, int64_t* n_owned, int64_t* e_split) {
  if (!ctx || !ctx->mesh_ok) return RDG_ESTATE;
  if (n_owned) *n_owned = ctx->n_owned;
  if (e_split) *e_split = ctx->e_split;
  return RDG_OK;
}

int rdg_stage_buffer(rdg_ctx* ctx, int stage, void** dev_ptr) {
  if (!ctx || !dev_ptr) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  const int nst = ctx->integrator == RDG_INTEGRATOR_LSRK54 ? 5 : 3;
  if (stage < 0 || stage >= nst) return fail(ctx, RDG_EINVAL, "stage out of range for the integrator");
  *dev_ptr = stage_input(ctx, stage);
  return RDG_OK;
}

int rdg_rows_gather(rdg_ctx* ctx, const void* src_dev, const int32_t* idx_dev, int64_t n, void* dst_dev) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (n < 0 || (n > 0 && (!src_dev || !idx_dev || !dst_dev))) return fail(ctx, RDG_EINVAL, "bad row gather arguments");
  if (n == 0) return RDG_OK;
  DeviceGuard g(ctx->device);
  int rc = launch_rows(ctx->esz, np_of(ctx->N), src_dev, idx_dev, n, dst_dev, false, ctx->K, ctx->d_err, ctx->stream);
  return rc == RDG_OK ? RDG_OK : fail(ctx, rc, "kernel launch failed");
}

int rdg_rows_scatter(rdg_ctx* ctx, const void* src_dev, const int32_t* idx_dev, int64_t n, void* dst_dev) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (n < 0 || (n > 0 && (!src_dev || !idx_dev || !dst_dev))) return fail(ctx, RDG_EINVAL, "bad row scatter arguments");
  if (n == 0) return RDG_OK;
  DeviceGuard g(ctx->device);
  int rc = launch_rows(ctx->esz, np_of(ctx->N), src_dev, idx_dev, n, dst_dev, true, ctx->K, ctx->d_err, ctx->stream);
  return rc == RDG_OK ? RDG_OK : fail(ctx, rc, "kernel launch failed");
}

int rdg_solve_to_time(rdg_ctx* ctx, double t0, double dt, int64_t nsteps) {
  if (!ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return fail(ctx, RDG_ESTATE, "rdg_operator_setup must come first");
  if (!(dt > 0) || !std::isfinite(t0) || nsteps < 0) return fail(ctx, RDG_EINVAL, "bad t0, dt or nsteps");
  if (nsteps == 0) return RDG_OK;
  DeviceGuard g(ctx->device);
  const int chunk = ctx->prof ? (int)(nsteps + 1) : 16;   // profiling steps without the graph
  if (nsteps >= chunk && (!ctx->gexec || ctx->g_dt != dt)) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    cudaGraph_t graph;
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = true;
    int rc = RDG_OK;
    for (int i = 0; i < chunk && rc == RDG_OK; ++i) {
      // the captured steps read their time origin and step count from device memory
      TimeArg ta{ctx->d_time, 0.0, dt, (double)i};
      rc = enqueue_rk_step(ctx, ta, dt);
    }
    if (rc == RDG_OK) rc = advance_time(ctx->d_time, chunk, ctx->cap_stream);
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    ctx->capturing = false;
    if (rc != RDG_OK) return fail(ctx, rc, "capture failed");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->g_dt = dt;
    ctx->g_chunk = chunk;
  }
  int64_t done = 0;
  if (nsteps >= chunk) {
    int rc = set_time(ctx->d_time, t0, ctx->stream);
    if (rc != RDG_OK) return fail(ctx, rc, "kernel launch failed");
    for (; done + chunk <= nsteps; done += chunk) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
  }
  for (; done < nsteps; ++done) {
    TimeArg ta{nullptr, t0 + done * dt, dt, 0.0};
    int rc = enqueue_rk_step(ctx, ta, dt);
    if (rc != RDG_OK) return fail(ctx, rc, "kernel launch failed");
  }
  return RDG_OK;
}

int rdg_set_integrator(rdg_ctx* ctx, int integrator) {
  if (!ctx) return RDG_EINVAL;
  if (integrator != RDG_INTEGRATOR_SSP_RK3 && integrator != RDG_INTEGRATOR_LSRK54)
    return fail(ctx, RDG_EINVAL, "integrator must be RDG_INTEGRATOR_SSP_RK3 or RDG_INTEGRATOR_LSRK54");
  ctx->integrator = integrator;
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  return RDG_OK;
}

int rdg_set_stage_form(rdg_ctx* ctx, int form) {
  if (!ctx) return RDG_EINVAL;
  if (form != RDG_STAGE_AUTO && form != RDG_STAGE_TWO_KERNELS && form != RDG_STAGE_ONE_KERNEL)
    return fail(ctx, RDG_EINVAL, "form must be RDG_STAGE_AUTO, RDG_STAGE_TWO_KERNELS or RDG_STAGE_ONE_KERNEL");
  ctx->stage_form = form;
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  return RDG_OK;
}

int rdg_gemm_hold_tile(rdg_ctx* ctx, int64_t tile) {
  if (!ctx) return RDG_EINVAL;
  if (tile < -1) return fail(ctx, RDG_EINVAL, "tile must be >= -1");
  ctx->gemm_hold = tile + 1;
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  return RDG_OK;
}

int rdg_get_stage_form(const rdg_ctx* ctx, int* form) {
  if (!ctx || !form) return RDG_EINVAL;
  *form = one_kernel_stage(ctx) ? RDG_STAGE_ONE_KERNEL : RDG_STAGE_TWO_KERNELS;
  return RDG_OK;
}

int rdg_set_l2_resident_bytes(rdg_ctx* ctx, int64_t bytes) {
  if (!ctx) return RDG_EINVAL;
  if (bytes < -1) return fail(ctx, RDG_EINVAL, "bytes must be >= -1");
  ctx->l2_keep_bytes = bytes;
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  return RDG_OK;
}

int rdg_profile(rdg_ctx* ctx, int enable) {
  if (!ctx) return RDG_EINVAL;
  ctx->prof = enable != 0;
  return RDG_OK;
}

int rdg_kernel_stats(rdg_ctx* ctx, int64_t* launches, double* ms, int reset) {
  if (!ctx) return RDG_EINVAL;
  DeviceGuard g(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  drain_events(ctx);
  for (int c = 0; c < 2; ++c) {
    if (launches) launches[c] = ctx->prof_n[c];
    if (ms) ms[c] = ctx->prof_ms[c];
    if (reset) {
      ctx->prof_n[c] = 0;
      ctx->prof_ms[c] = 0;
    }
  }
  return RDG_OK;
}

int rdg_synchronize(rdg_ctx* ctx) {
  if (!ctx) return RDG_EINVAL;
  DeviceGuard g(ctx->device);
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h) {
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h & kErrBadIndex) return fail(ctx, RDG_ECUDA, "a kernel's index self-check failed (corrupt edge tables)");
    return fail(ctx, RDG_ETIMEOUT, "a bounded wait for the tensor core gave up (more than 1 s)");
  }
  return RDG_OK;
}

int rdg_reference_operator(int N, int which, double* out) {
  if (!out) return RDG_EINVAL;
  const char* msg = "";
  const RefOps* o = get_refops(N, &msg);
  if (!o) return RDG_EINVAL;
  const std::vector<double>* src = nullptr;
  switch (which) {
    case 0:
      std::copy(o->r.begin(), o->r.end(), out);
      std::copy(o->s.begin(), o->s.end(), out + o->Np);
      return RDG_OK;
    case 1: src = &o->Dr; break;
    case 2: src = &o->Ds; break;
    case 3: src = &o->LIFT; break;
    case 4: src = &o->Apinv; break;
    case 5: src = &o->M; break;
    case 6:
      std::copy(o->X[0].begin(), o->X[0].end(), out);
      std::copy(o->X[1].begin(), o->X[1].end(), out + o->X[0].size());
      return RDG_OK;
    case 7:
      for (size_t i = 0; i < o->perm.size(); ++i) out[i] = o->perm[i];
      return RDG_OK;
    case 8:
      for (size_t i = 0; i < o->hyp.size(); ++i) out[i] = o->hyp[i];
      return RDG_OK;
    case 9:
      std::copy(o->RVV[0].begin(), o->RVV[0].end(), out);
      std::copy(o->RVV[1].begin(), o->RVV[1].end(), out + o->RVV[0].size());
      return RDG_OK;
    case 10:
    case 11: {
      size_t off = 0;
      for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) {
          const std::vector<double>& g = which == 10 ? o->GR[j][k] : o->GS[j][k];
          std::copy(g.begin(), g.end(), out + off);
          off += g.size();
        }
      return RDG_OK;
    }
    default: return RDG_EINVAL;
  }
  std::copy(src->begin(), src->end(), out);
  return RDG_OK;
}

}  // extern "C"

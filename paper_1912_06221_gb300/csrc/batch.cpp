// Batched stepping of independent problems.  Every member context keeps its own mesh,
// order, precision, operators and resident state; a step of the batch advances every member
// by the same number of SSP-RK3 steps with its own dt.  The members' stage kernels are
// captured as parallel branches of one CUDA graph (fork on the batch stream, one branch
// stream per member, join back), so one graph launch runs a chunk of steps of all members
// and kernels of small and large problems, of different orders, overlap on the GPU.  Each
// member's launches keep their per-order kernels, register budgets and launch shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "batch_kernel.h"
#include "context.h"

struct rdg_batch {
  struct Member {
    rdg_ctx* ctx;
    double dt;
    cudaEvent_t ev_in;    // member stream -> batch stream (work enqueued on the member before a step)
    cudaEvent_t ev_join;  // branch -> fork stream
    cudaStream_t branch;
  };
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int chunk = 16;
  std::string err;
  std::vector<Member> members;
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_out = nullptr;
  cudaStream_t cap = nullptr;     // private stream the graph is captured on
  cudaGraphExec_t gexec = nullptr;
  int g_chunk = 0;
  // persistent form: one launch per chunk of steps of every member
  int mode = RDG_BATCH_AUTO;
  int ept[7] = {1, 1, 1, 1, 1, 1, 1};   // edges per thread of an edge tile, per order
  int tpi[7] = {1, 1, 1, 1, 1, 1, 1};   // tiles per work item, per order
  double wait_s = 1.0;                  // bound on every dependency wait of the kernel
  int hold_member = -1;                 // test hook: this member's phase hold_phase never starts
  int64_t hold_phase = -1;
  bool dirty = true;                    // descriptors to rebuild before the next launch
  rdg::BMember* d_members = nullptr;
  unsigned long long* d_ticket = nullptr;   // ticket, then one count per member
  int* d_flags = nullptr;               // abort flag, error word
  float* d_tabs = nullptr;
  int nm_alloc = 0;
  rdg::BatchArgs args{};
  int grid = 0;
  size_t smem = 0;
};

namespace {

struct DevGuard {
  int prev = 0;
  explicit DevGuard(int d) {
    cudaGetDevice(&prev);
    cudaSetDevice(d);
  }
  ~DevGuard() { cudaSetDevice(prev); }
};

int bfail(rdg_batch* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}

int bcuda(rdg_batch* b, cudaError_t e, const char* what) {
  return bfail(b, RDG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void drop_graph(rdg_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->g_chunk = 0;
}

void release_member(rdg_batch::Member& m) {
  if (m.ev_in) cudaEventDestroy(m.ev_in);
  if (m.ev_join) cudaEventDestroy(m.ev_join);
  if (m.branch) cudaStreamDestroy(m.branch);
}

// The persistent form applies when every member is FP32 with stored operators and SSP-RK3.
bool persistent_fits(const rdg_batch* b) {
  for (const auto& m : b->members) {
    const rdg_ctx* c = m.ctx;
    if (c->esz != 4 || c->gemm || c->integrator != RDG_INTEGRATOR_SSP_RK3 || c->d_Dn) return false;
  }
  return !b->members.empty();
}

bool use_persistent(const rdg_batch* b) {
  if (b->mode == RDG_BATCH_GRAPH) return false;
  return persistent_fits(b);
}

void free_persistent(rdg_batch* b) {
  cudaFree(b->d_members);
  cudaFree(b->d_ticket);
  cudaFree(b->d_flags);
  cudaFree(b->d_tabs);
  b->d_members = nullptr;
  b->d_ticket = nullptr;
  b->d_flags = nullptr;
  b->d_tabs = nullptr;
  b->nm_alloc = 0;
  b->dirty = true;
}

// Descriptors, tables and counters of the persistent launch (after a membership change).
int prepare_persistent(rdg_batch* b) {
  if (!b->dirty) return RDG_OK;
  free_persistent(b);
  const int nm = (int)b->members.size();
  std::vector<rdg::BMember> hm(nm);
  bool orders[7] = {false, false, false, false, false, false, false};
  int64_t off = 0, offb = 0;
  for (int i = 0; i < nm; ++i) {
    const rdg_ctx* c = b->members[i].ctx;
    rdg::BMember& d = hm[i];
    d.W = c->d_W;
    d.k1 = c->d_k1;
    d.k2 = c->d_k2;
    d.f12 = c->d_f12;
    d.u = (float*)c->d_u;
    d.u1 = (float*)c->d_u1;
    d.u2 = (float*)c->d_u2;
    d.vol = (float*)c->d_vol;
    d.fb = (float*)c->d_fb;
    d.geo = (const float*)c->d_geo;
    d.S = (const float*)c->d_S;
    d.G = (const float*)c->d_G;
    d.err = c->d_err;
    d.ts = c->d_time;
    d.K = c->K;
    d.E = c->E;
    d.B = c->B;
    d.frc = c->frc;
    d.dt = b->members[i].dt;
    d.dt32 = (float)b->members[i].dt;
    d.N = c->N;
    d.ept = b->ept[c->N];
    d.ntile_v = (c->K + rdg::kStageBlock - 1) / rdg::kStageBlock;
    const int64_t per_tile = (int64_t)rdg::kStageBlock * d.ept;
    d.ntile_e = (c->E + per_tile - 1) / per_tile;
    d.ntile_u = d.ntile_v;
    d.tpi = b->tpi[c->N];
    d.nitem_a = (d.ntile_e + d.ntile_v + d.tpi - 1) / d.tpi;
    d.nitem_b = (d.ntile_u + d.tpi - 1) / d.tpi;
    d.off_a = off;
    d.off_b = offb;
    d.hold_phase = i == b->hold_member ? b->hold_phase : -1;
    off += d.nitem_a;
    offb += d.nitem_b;
    orders[c->N] = true;
  }
  std::vector<float> tabs;
  int toff[7];
  int rc = rdg::batch_tables(orders, tabs, toff);
  if (rc != RDG_OK) return bfail(b, rc, "reference tables");
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_members, nm * sizeof(rdg::BMember))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_ticket, (2 * nm + 1) * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_flags, 2 * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_tabs, std::max<size_t>(tabs.size(), 4) * sizeof(float))) != cudaSuccess) {
    free_persistent(b);
    return bcuda(b, e, "persistent batch buffers");
  }
  if ((e = cudaMemcpy(b->d_members, hm.data(), nm * sizeof(rdg::BMember), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_tabs, tabs.data(), tabs.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(b->d_flags, 0, 2 * sizeof(int))) != cudaSuccess) {
    free_persistent(b);
    return bcuda(b, e, "persistent batch upload");
  }
  rdg::BatchArgs& a = b->args;
  a.m = b->d_members;
  a.nm = nm;
  a.items_a = off;
  a.per_phase = off + offb;
  a.ticket = b->d_ticket;
  a.done = b->d_ticket + 1;
  a.abort = b->d_flags;
  a.err = b->d_flags + 1;
  a.tabs = b->d_tabs;
  a.tab_floats = (int)tabs.size();
  a.wait_ns = (uint64_t)(b->wait_s * 1e9);
  b->smem = rdg::batch_smem_bytes(a.tab_floats, nm);
  b->grid = rdg::batch_grid(b->smem);
  if (b->grid <= 0) {
    free_persistent(b);
    return bfail(b, RDG_ECUDA, "persistent batch kernel occupancy");
  }
  b->nm_alloc = nm;
  b->dirty = false;
  return RDG_OK;
}

// nsteps steps of every member in one persistent launch on `root`, then the time origins.
int enqueue_persistent(rdg_batch* b, cudaStream_t root, int nsteps) {
  cudaError_t e = cudaMemsetAsync(b->d_ticket, 0, (2 * b->nm_alloc + 1) * sizeof(unsigned long long), root);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flags, 0, sizeof(int), root);   // abort flag only
  if (e != cudaSuccess) return bcuda(b, e, "cudaMemsetAsync");
  rdg::BatchArgs a = b->args;
  a.nphase = 3 * nsteps;
  int rc = rdg::launch_batch_persistent(a, b->grid, b->smem, root);
  if (rc == RDG_OK) rc = rdg::launch_batch_advance(b->d_members, b->nm_alloc, nsteps, root);
  return rc == RDG_OK ? RDG_OK : bfail(b, rc, "kernel launch failed");
}

// Fork from `root` to every member's branch, enqueue nsteps steps per member (each reads its
// time origin from its device time state, which the branch then advances), join on `root`.
int enqueue_all(rdg_batch* b, cudaStream_t root, int nsteps) {
  if (use_persistent(b)) return enqueue_persistent(b, root, nsteps);
  cudaError_t e = cudaEventRecord(b->ev_fork, root);
  if (e != cudaSuccess) return bcuda(b, e, "cudaEventRecord");
  for (auto& m : b->members) {
    if ((e = cudaStreamWaitEvent(m.branch, b->ev_fork, 0)) != cudaSuccess) return bcuda(b, e, "cudaStreamWaitEvent");
    for (int k = 0; k < nsteps; ++k) {
      rdg::TimeArg ta{m.ctx->d_time, 0.0, m.dt, (double)k};
      int rc = rdg::enqueue_rk_step_on(m.ctx, m.branch, ta, m.dt);
      if (rc != RDG_OK) return bfail(b, rc, "kernel launch failed");
    }
    int rc = rdg::advance_time(m.ctx->d_time, nsteps, m.branch);
    if (rc != RDG_OK) return bfail(b, rc, "kernel launch failed");
    if ((e = cudaEventRecord(m.ev_join, m.branch)) != cudaSuccess) return bcuda(b, e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(root, m.ev_join, 0)) != cudaSuccess) return bcuda(b, e, "cudaStreamWaitEvent");
  }
  return RDG_OK;
}

int capture(rdg_batch* b, int chunk) {
  drop_graph(b);
  if (use_persistent(b)) {
    int rc = prepare_persistent(b);
    if (rc != RDG_OK) return rc;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamBeginCapture");
  int rc = enqueue_all(b, b->cap, chunk);
  e = cudaStreamEndCapture(b->cap, &graph);
  if (rc != RDG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->gexec = nullptr;
    return bcuda(b, e, "cudaGraphInstantiate");
  }
  b->g_chunk = chunk;
  return RDG_OK;
}

}  // namespace

extern "C" {

int rdg_batch_create(rdg_batch** out, int device, void* cuda_stream, int chunk) {
  if (!out) return RDG_EINVAL;
  *out = nullptr;
  if (chunk < 1 || chunk > 1024) return RDG_EINVAL;
  rdg_batch* b = new (std::nothrow) rdg_batch();
  if (!b) return RDG_ENOMEM;
  b->device = device;
  b->chunk = chunk;
  DevGuard g(device);
  bool ok = true;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess;
    b->own_stream = ok;
  }
  ok = ok && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return RDG_ECUDA;
  }
  *out = b;
  return RDG_OK;
}

int rdg_batch_destroy(rdg_batch* b) {
  if (!b) return RDG_OK;
  DevGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& m : b->members) {
    cudaStreamSynchronize(m.branch);
    release_member(m);
  }
  free_persistent(b);
  cudaEventDestroy(b->ev_fork);
  cudaEventDestroy(b->ev_out);
  cudaStreamDestroy(b->cap);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return RDG_OK;
}

const char* rdg_batch_last_error(const rdg_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

int rdg_batch_add(rdg_batch* b, rdg_ctx* ctx, double t0, double dt) {
  if (!b || !ctx) return RDG_EINVAL;
  if (!ctx->ops_ok) return bfail(b, RDG_ESTATE, "member context has no operators (rdg_operator_setup first)");
  if (ctx->device != b->device) return bfail(b, RDG_EINVAL, "member context is on another device");
  if (!(dt > 0) || !std::isfinite(dt) || !std::isfinite(t0)) return bfail(b, RDG_EINVAL, "dt must be positive, t0 finite");
  for (auto& m : b->members)
    if (m.ctx == ctx) return bfail(b, RDG_EINVAL, "context is already in the batch");
  DevGuard g(b->device);
  rdg_batch::Member m{ctx, dt, nullptr, nullptr, nullptr};
  bool ok = cudaEventCreateWithFlags(&m.ev_in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&m.ev_join, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&m.branch, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    release_member(m);
    return bfail(b, RDG_ECUDA, "event or stream creation failed");
  }
  // the member's time origin, ordered after whatever the caller enqueued on its stream
  int rc = rdg::set_time(ctx->d_time, t0, ctx->stream);
  if (rc != RDG_OK) {
    release_member(m);
    return bfail(b, rc, "kernel launch failed");
  }
  b->members.push_back(m);
  drop_graph(b);
  b->dirty = true;
  return RDG_OK;
}

int rdg_batch_remove(rdg_batch* b, rdg_ctx* ctx) {
  if (!b || !ctx) return RDG_EINVAL;
  DevGuard g(b->device);
  for (size_t i = 0; i < b->members.size(); ++i) {
    if (b->members[i].ctx != ctx) continue;
    cudaStreamSynchronize(b->members[i].branch);
    release_member(b->members[i]);
    cudaStreamSynchronize(b->stream);   // a persistent launch reads every member's descriptor
    b->members.erase(b->members.begin() + (ptrdiff_t)i);
    drop_graph(b);
    b->dirty = true;
    return RDG_OK;
  }
  return bfail(b, RDG_EINVAL, "context is not in the batch");
}

int rdg_batch_set_chunk(rdg_batch* b, int chunk) {
  if (!b) return RDG_EINVAL;
  if (chunk < 1 || chunk > 1024) return bfail(b, RDG_EINVAL, "chunk must be in 1..1024");
  if (chunk != b->chunk) {
    DevGuard g(b->device);
    cudaStreamSynchronize(b->stream);   // the replaced graph may still be running
    drop_graph(b);
    b->chunk = chunk;
  }
  return RDG_OK;
}

int rdg_batch_size(const rdg_batch* b, int* n) {
  if (!b || !n) return RDG_EINVAL;
  *n = (int)b->members.size();
  return RDG_OK;
}

int rdg_batch_step(rdg_batch* b, int64_t nsteps) {
  if (!b) return RDG_EINVAL;
  if (nsteps < 0) return bfail(b, RDG_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0 || b->members.empty()) return RDG_OK;
  DevGuard g(b->device);
  cudaError_t e;
  // order after the work already enqueued on every member's own stream
  for (auto& m : b->members) {
    if ((e = cudaEventRecord(m.ev_in, m.ctx->stream)) != cudaSuccess) return bcuda(b, e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(b->stream, m.ev_in, 0)) != cudaSuccess) return bcuda(b, e, "cudaStreamWaitEvent");
  }
  int64_t done = 0;
  if (nsteps >= b->chunk) {
    if (b->g_chunk != b->chunk || !b->gexec) {
      int rc = capture(b, b->chunk);
      if (rc != RDG_OK) return rc;
    }
    for (; done + b->chunk <= nsteps; done += b->chunk)
      if ((e = cudaGraphLaunch(b->gexec, b->stream)) != cudaSuccess) return bcuda(b, e, "cudaGraphLaunch");
  }
  if (done < nsteps) {
    if (use_persistent(b)) {
      int rc = prepare_persistent(b);
      if (rc != RDG_OK) return rc;
    }
    int rc = enqueue_all(b, b->stream, (int)(nsteps - done));
    if (rc != RDG_OK) return rc;
  }
  // later work on a member's stream (state reads, its own steps) waits for the batch
  if ((e = cudaEventRecord(b->ev_out, b->stream)) != cudaSuccess) return bcuda(b, e, "cudaEventRecord");
  for (auto& m : b->members)
    if ((e = cudaStreamWaitEvent(m.ctx->stream, b->ev_out, 0)) != cudaSuccess) return bcuda(b, e, "cudaStreamWaitEvent");
  return RDG_OK;
}

int rdg_batch_synchronize(rdg_batch* b) {
  if (!b) return RDG_EINVAL;
  {
    DevGuard g(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "cudaStreamSynchronize");
    if (b->d_flags) {
      int fl[2] = {0, 0};
      if ((e = cudaMemcpy(fl, b->d_flags, sizeof(fl), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bcuda(b, e, "cudaMemcpy");
      if (fl[1] & rdg::kErrWaitTimeout) {
        // the launch gave up part-way: the members' states are undefined; clear the error word
        if ((e = cudaMemset(b->d_flags, 0, 2 * sizeof(int))) != cudaSuccess) return bcuda(b, e, "cudaMemset");
        return bfail(b, RDG_ETIMEOUT, "a dependency wait of the persistent batch kernel gave up");
      }
    }
  }
  for (auto& m : b->members) {
    int rc = rdg_synchronize(m.ctx);
    if (rc != RDG_OK) return bfail(b, rc, std::string("member: ") + rdg_last_error(m.ctx));
  }
  return RDG_OK;
}

int rdg_batch_set_mode(rdg_batch* b, int mode) {
  if (!b) return RDG_EINVAL;
  if (mode != RDG_BATCH_AUTO && mode != RDG_BATCH_GRAPH && mode != RDG_BATCH_PERSISTENT)
    return bfail(b, RDG_EINVAL, "mode must be RDG_BATCH_AUTO, RDG_BATCH_GRAPH or RDG_BATCH_PERSISTENT");
  if (mode == RDG_BATCH_PERSISTENT && !b->members.empty() && !persistent_fits(b))
    return bfail(b, RDG_EINVAL, "the persistent form needs FP32 members with stored operators and SSP-RK3");
  DevGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  b->mode = mode;
  drop_graph(b);
  return RDG_OK;
}

int rdg_batch_get_mode(const rdg_batch* b, int* mode) {
  if (!b || !mode) return RDG_EINVAL;
  *mode = use_persistent(b) ? RDG_BATCH_PERSISTENT : RDG_BATCH_GRAPH;
  return RDG_OK;
}

int rdg_batch_set_tiles(rdg_batch* b, int N, int edges_per_thread, int tiles_per_item) {
  if (!b) return RDG_EINVAL;
  if (N < 1 || N > 6 || edges_per_thread < 1 || edges_per_thread > 2 ||
      (tiles_per_item != 1 && tiles_per_item != 2 && tiles_per_item != 4))
    return bfail(b, RDG_EINVAL, "N must be in 1..6, edges_per_thread 1 or 2, tiles_per_item 1, 2 or 4");
  DevGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  b->ept[N] = edges_per_thread;
  b->tpi[N] = tiles_per_item;
  b->dirty = true;
  drop_graph(b);
  return RDG_OK;
}

int rdg_batch_set_wait_limit(rdg_batch* b, double seconds) {
  if (!b) return RDG_EINVAL;
  if (!(seconds > 0) || seconds > 60) return bfail(b, RDG_EINVAL, "wait limit must be in (0, 60] seconds");
  DevGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  b->wait_s = seconds;
  b->dirty = true;
  drop_graph(b);
  return RDG_OK;
}

int rdg_batch_hold_phase(rdg_batch* b, int member, int64_t phase) {
  if (!b) return RDG_EINVAL;
  if (member < -1 || member >= (int)b->members.size()) return bfail(b, RDG_EINVAL, "no such member");
  DevGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  b->hold_member = member;
  b->hold_phase = phase;
  b->dirty = true;
  drop_graph(b);
  return RDG_OK;
}

}  // extern "C"

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

// Fork from `root` to every member's branch, enqueue nsteps steps per member (each reads its
// time origin from its device time state, which the branch then advances), join on `root`.
int enqueue_all(rdg_batch* b, cudaStream_t root, int nsteps) {
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
  return RDG_OK;
}

int rdg_batch_remove(rdg_batch* b, rdg_ctx* ctx) {
  if (!b || !ctx) return RDG_EINVAL;
  DevGuard g(b->device);
  for (size_t i = 0; i < b->members.size(); ++i) {
    if (b->members[i].ctx != ctx) continue;
    cudaStreamSynchronize(b->members[i].branch);
    release_member(b->members[i]);
    b->members.erase(b->members.begin() + (ptrdiff_t)i);
    drop_graph(b);
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
  }
  for (auto& m : b->members) {
    int rc = rdg_synchronize(m.ctx);
    if (rc != RDG_OK) return bfail(b, rc, std::string("member: ") + rdg_last_error(m.ctx));
  }
  return RDG_OK;
}

}  // extern "C"

// Batches of independent systems (sog_batch_* in sog.h): one plan per system,
// all systems' evaluations captured into one CUDA graph and replayed with one
// cudaGraphLaunch.  Inside the graph every system forks from a common event
// onto its plan's own streams, so small systems fill the GPU together.
#include <cuda_runtime.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "sog_internal.h"

struct sog_batch {
  int nsys = 0;
  int prec = SOG_PREC_MIXED;
  std::vector<sog_plan*> plans;
  cudaStream_t origin = nullptr;   // capture origin
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_done;
  std::vector<const void*> key;    // pointers of the captured graph
  cudaGraphExec_t exec = nullptr;
  cudaStream_t last_stream = nullptr;
  int launch_error = 0;
  int64_t launches = 0;
};

namespace {

void destroy_batch(sog_batch* b) {
  if (!b) return;
  if (b->exec) {
    cudaStreamSynchronize(b->last_stream);
    cudaGraphExecDestroy(b->exec);
  }
  for (sog_plan* p : b->plans)
    if (p) sog_plan_destroy(p);
  for (cudaEvent_t e : b->ev_done)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

}  // namespace

extern "C" {

sog_status sog_batch_create(sog_batch** out, int32_t nsys, const int64_t* N, const double* L,
                            const double* tol, const sog_opts* opts) {
  if (!out || nsys < 1 || !N || !L || !tol) return SOG_ERR_ARG;
  if (opts && opts->manual) return SOG_ERR_ARG;  // parameters differ between systems
  *out = nullptr;
  sog_batch* b = new sog_batch;
  b->nsys = nsys;
  b->prec = opts ? opts->precision : SOG_PREC_MIXED;
  b->plans.assign(nsys, nullptr);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    delete b;
    return SOG_ERR_CUDA;
  }
  // plan tables are built on the host: create the plans on several threads
  std::vector<sog_status> st(nsys, SOG_OK);
  const int nthr = std::max(1, std::min<int>(nsys, (int)std::min(16u, std::thread::hardware_concurrency())));
  std::vector<std::thread> pool;
  for (int t = 0; t < nthr; ++t)
    pool.emplace_back([&, t]() {
      cudaSetDevice(dev);
      for (int i = t; i < nsys; i += nthr)
        st[i] = sog_plan_create(&b->plans[i], N[i], L[3 * i], L[3 * i + 1], L[3 * i + 2], tol[i], opts);
    });
  for (auto& th : pool) th.join();
  for (int i = 0; i < nsys; ++i)
    if (st[i] != SOG_OK) {
      const sog_status s = st[i];
      destroy_batch(b);
      return s;
    }
  b->ev_done.assign(nsys, nullptr);
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    destroy_batch(b);
    return SOG_ERR_CUDA;
  }
  for (int i = 0; i < nsys; ++i)
    if (cudaEventCreateWithFlags(&b->ev_done[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      destroy_batch(b);
      return SOG_ERR_CUDA;
    }
  *out = b;
  return SOG_OK;
}

int32_t sog_batch_size(const sog_batch* b) { return b ? b->nsys : 0; }

sog_plan* sog_batch_plan(sog_batch* b, int32_t i) {
  return (b && i >= 0 && i < b->nsys) ? b->plans[i] : nullptr;
}

sog_status sog_batch_eval(sog_batch* b, const void* const* q, const void* const* r,
                          void* const* phi, double* E, void* const* F, void* stream) {
  if (!b || !q || !r) return SOG_ERR_ARG;
  for (int i = 0; i < b->nsys; ++i)
    if (!q[i] || !r[i]) return SOG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const void*> key;
  key.reserve(4 * b->nsys + 1);
  for (int i = 0; i < b->nsys; ++i) {
    key.push_back(q[i]);
    key.push_back(r[i]);
    key.push_back(phi ? phi[i] : nullptr);
    key.push_back(F ? F[i] : nullptr);
  }
  key.push_back(E);
  if (!b->exec || key != b->key) {
    if (b->exec) {
      cudaStreamSynchronize(b->last_stream);
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, b->origin);
    cudaError_t e1 = e;
    int64_t launches = 0;
    for (int i = 0; i < b->nsys && e1 == cudaSuccess; ++i) {
      sog_plan* p = b->plans[i];
      e1 = cudaStreamWaitEvent(p->cap_stream, b->ev_fork, 0);
      if (e1 == cudaSuccess)
        e1 = sogk::enqueue_eval(p, q[i], r[i], phi ? phi[i] : nullptr, E ? E + i : nullptr,
                                F ? F[i] : nullptr, p->cap_stream);
      if (e1 == cudaSuccess) e1 = cudaEventRecord(b->ev_done[i], p->cap_stream);
      if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(b->origin, b->ev_done[i], 0);
      launches += p->launches;
    }
    const cudaError_t e2 = cudaStreamEndCapture(b->origin, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (e2 == cudaSuccess) cudaGraphDestroy(graph);
      cudaGetLastError();
      b->launch_error = 1;
      return SOG_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
      b->launch_error = 1;
      return SOG_ERR_CUDA;
    }
    b->key = key;
    b->launches = launches;
  }
  if (cudaGraphLaunch(b->exec, s) != cudaSuccess) {
    cudaGetLastError();
    b->launch_error = 1;
    return SOG_ERR_CUDA;
  }
  b->last_stream = s;
  for (sog_plan* p : b->plans) p->last_stream = s;
  return SOG_OK;
}

sog_status sog_batch_check(sog_batch* b, int32_t* first_bad) {
  if (!b) return SOG_ERR_ARG;
  if (first_bad) *first_bad = -1;
  if (b->last_stream && cudaStreamSynchronize(b->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return SOG_ERR_CUDA;
  }
  sog_status worst = SOG_OK;
  for (int i = 0; i < b->nsys; ++i) {
    const sog_status st = sog_plan_check(b->plans[i]);
    if (st != SOG_OK && worst == SOG_OK) {
      worst = st;
      if (first_bad) *first_bad = i;
    }
  }
  if (b->launch_error) {
    b->launch_error = 0;
    if (worst == SOG_OK) worst = SOG_ERR_CUDA;
  }
  return worst;
}

int64_t sog_batch_launches(const sog_batch* b) { return b ? b->launches : 0; }

void sog_batch_destroy(sog_batch* b) { destroy_batch(b); }

}  // extern "C"

// Many independent problems stepped together (a batch of CN-WSGD solves of
// different sizes, orders and coefficients). The problems share nothing, so
// the batch runs them concurrently: W host worker threads, each with its own
// CUDA stream, drive disjoint subsets of the handles (FGMRES keeps its small
// Hessenberg least-squares problem on the host, so every solve needs a host
// thread of its own to overlap with the others). Problems are assigned by
// longest-processing-time-first on an n log n cost estimate.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fde.h"

namespace fde {
void set_global_error(const char* msg);
struct GroupEngine;
GroupEngine* group_engine_create(const std::vector<fde_handle*>& hs, cudaStream_t st,
                                 std::string& why);
void group_engine_destroy(GroupEngine* e);
int group_engine_step(GroupEngine* e, const double* const* u_prev, const double* const* v_half,
                      double* const* u_next, cudaStream_t st, std::vector<int>& rc,
                      fde_stats* stats);
long long group_engine_launches(const GroupEngine* e);
}  // namespace fde

struct fde_batch {
  int device = 0;
  cudaStream_t user = nullptr;
  std::vector<fde_handle*> h;
  std::vector<cudaStream_t> streams;     // one per worker
  std::vector<std::vector<int>> work;    // problem indices per worker
  std::vector<cudaEvent_t> done;         // one per worker
  cudaEvent_t start = nullptr;
  std::vector<int> rc;                   // last status per problem
  // grouped engine (fde_group.cu): built at the first step when every problem
  // qualifies and FDE_BATCH_ENGINE is not "threads"; engine_state 0 = not
  // decided, 1 = grouped, 2 = worker threads
  fde::GroupEngine* engine = nullptr;
  int engine_state = 0;
  std::string engine_why;
};

namespace {
constexpr int kMaxWorkers = 16;

void destroy(fde_batch* b) {
  if (!b) return;
  if (b->engine) {
    cudaStreamSynchronize(b->user);
    fde::group_engine_destroy(b->engine);
  }
  for (fde_handle* h : b->h) fde_destroy(h);
  for (cudaStream_t s : b->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : b->done) cudaEventDestroy(e);
  if (b->start) cudaEventDestroy(b->start);
  delete b;
}
}  // namespace

extern "C" {

int fde_batch_create(const fde_params* p, int count, void* stream, fde_batch** out) {
  if (!out) return FDE_ERR_ARG;
  *out = nullptr;
  if (!p || count <= 0) {
    fde::set_global_error("fde_batch_create: null params or count <= 0");
    return FDE_ERR_ARG;
  }
  fde_batch* b = new fde_batch();
  b->user = (cudaStream_t)stream;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    fde::set_global_error("fde_batch_create: no CUDA device");
    return FDE_ERR_CUDA;
  }
  int maxw = kMaxWorkers;
  if (const char* env = std::getenv("FDE_BATCH_WORKERS")) {
    const int v = std::atoi(env);
    if (v >= 1 && v <= 256) maxw = v;
  }
  const int W = std::min(count, maxw);
  b->streams.resize(W, nullptr);
  b->done.resize(W, nullptr);
  b->work.resize(W);
  for (int w = 0; w < W; ++w) {
    if (cudaStreamCreateWithFlags(&b->streams[w], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done[w], cudaEventDisableTiming) != cudaSuccess) {
      destroy(b);
      fde::set_global_error("fde_batch_create: stream or event creation failed");
      return FDE_ERR_CUDA;
    }
  }
  if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
    destroy(b);
    fde::set_global_error("fde_batch_create: event creation failed");
    return FDE_ERR_CUDA;
  }
  // longest processing time first: heaviest problem to the least-loaded worker
  std::vector<int> order(count);
  std::vector<double> cost(count);
  for (int i = 0; i < count; ++i) {
    const double N = (double)p[i].n1 * (double)p[i].n2;
    cost[i] = N * std::log2(N + 2.0);
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<double> load(W, 0.0);
  std::vector<int> owner(count);
  for (int i : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[w] += cost[i];
    owner[i] = w;
  }
  b->h.assign(count, nullptr);
  b->rc.assign(count, FDE_OK);
  for (int i = 0; i < count; ++i) {
    const int rc = fde_create(&p[i], b->streams[owner[i]], &b->h[i]);
    if (rc != FDE_OK) {
      char buf[600];
      snprintf(buf, sizeof(buf), "fde_batch_create: problem %d: %s", i, fde_last_error(nullptr));
      destroy(b);
      fde::set_global_error(buf);
      return rc;
    }
    b->work[owner[i]].push_back(i);
  }
  *out = b;
  return FDE_OK;
}

void fde_batch_destroy(fde_batch* b) { destroy(b); }

int fde_batch_size(const fde_batch* b) { return b ? (int)b->h.size() : 0; }

fde_handle* fde_batch_handle(fde_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->h.size()) return nullptr;
  return b->h[i];
}

int fde_batch_engine(const fde_batch* b) { return b ? b->engine_state : 0; }

const char* fde_batch_engine_note(const fde_batch* b) {
  return b ? b->engine_why.c_str() : "";
}

long long fde_batch_launch_count(const fde_batch* b) {
  if (!b) return 0;
  long long n = fde::group_engine_launches(b->engine);
  for (fde_handle* h : b->h) n += fde_launch_count(h);
  return n;
}

int fde_batch_status(const fde_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->rc.size()) return FDE_ERR_ARG;
  return b->rc[i];
}

int fde_batch_step(fde_batch* b, const double* const* u_prev, const double* const* v_half,
                   double* const* u_next, fde_stats* st) {
  if (!b) return FDE_ERR_ARG;
  const int count = (int)b->h.size();
  if (!u_prev || !v_half || !u_next) {
    fde::set_global_error("fde_batch_step: null pointer array");
    return FDE_ERR_ARG;
  }
  if (b->engine_state == 0) {
    const char* env = std::getenv("FDE_BATCH_ENGINE");
    b->engine_state = 2;
    if (!(env && std::string(env) == "threads")) {
      // coefficients may still be in flight on the problems' own streams
      for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
      b->engine = fde::group_engine_create(b->h, b->user, b->engine_why);
      if (b->engine) b->engine_state = 1;
    } else {
      b->engine_why = "FDE_BATCH_ENGINE=threads";
    }
  }
  if (b->engine_state == 1) {
    // the problems' own streams may hold coefficient updates: the caller's
    // stream waits for them, then runs the grouped step
    for (int w = 0; w < (int)b->streams.size(); ++w) {
      if (cudaEventRecord(b->done[w], b->streams[w]) != cudaSuccess ||
          cudaStreamWaitEvent(b->user, b->done[w], 0) != cudaSuccess)
        return FDE_ERR_CUDA;
    }
    const int r = fde::group_engine_step(b->engine, u_prev, v_half, u_next, b->user, b->rc, st);
    if (r != FDE_OK) {
      fde::set_global_error("fde_batch_step: the grouped engine failed");
      return r;
    }
    for (int i = 0; i < count; ++i)
      if (b->rc[i] != FDE_OK) {
        char buf[600];
        snprintf(buf, sizeof(buf), "fde_batch_step: problem %d: %s", i, fde_last_error(b->h[i]));
        fde::set_global_error(buf);
        return b->rc[i];
      }
    return FDE_OK;
  }
  // the workers' streams start after the caller's stream work that precedes this call
  if (cudaEventRecord(b->start, b->user) != cudaSuccess) return FDE_ERR_CUDA;
  for (cudaStream_t s : b->streams)
    if (cudaStreamWaitEvent(s, b->start, 0) != cudaSuccess) return FDE_ERR_CUDA;
  const int W = (int)b->streams.size();
  std::vector<std::thread> pool;
  pool.reserve(W);
  for (int w = 0; w < W; ++w) {
    pool.emplace_back([b, w, u_prev, v_half, u_next, st]() {
      cudaSetDevice(b->device);
      for (int i : b->work[w]) {
        fde_stats s{0, 0, 0, 0.0, 0};
        b->rc[i] = fde_step(b->h[i], u_prev[i], v_half[i], u_next[i], &s);
        if (st) st[i] = s;
      }
      cudaEventRecord(b->done[w], b->streams[w]);
    });
  }
  for (auto& t : pool) t.join();
  // the caller's stream continues after every worker's work
  for (int w = 0; w < W; ++w)
    if (cudaStreamWaitEvent(b->user, b->done[w], 0) != cudaSuccess) return FDE_ERR_CUDA;
  for (int i = 0; i < count; ++i)
    if (b->rc[i] != FDE_OK) {
      char buf[600];
      snprintf(buf, sizeof(buf), "fde_batch_step: problem %d: %s", i, fde_last_error(b->h[i]));
      fde::set_global_error(buf);
      return b->rc[i];
    }
  return FDE_OK;
}

}  // extern "C"

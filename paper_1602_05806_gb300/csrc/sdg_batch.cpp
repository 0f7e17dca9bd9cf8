// Batches of independent problems (sdg_batch_*): every member is a full
// sdg_handle with its own CUDA stream, and a step advances the members
// concurrently from a pool of host threads.  Each member's CG loop keeps
// its own host synchronisation, so while one thread waits on its stream the
// others keep launching: the small problems of a batch fill the GPU
// together instead of one after another.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sdg.h"

namespace sdg {
void set_last_error(const char* msg);
}

struct sdg_batch {
  int nprob = 0;
  int device = 0;
  int nthreads = 1;
  std::vector<sdg_handle*> h;
  std::vector<cudaStream_t> s;
  std::vector<cudaEvent_t> done;
  std::vector<int> order;  // members by size, largest first
  cudaEvent_t start = nullptr;
};

namespace {

void destroy(sdg_batch* b) {
  if (!b) return;
  for (auto e : b->done)
    if (e) cudaEventDestroy(e);
  for (auto s : b->s)
    if (s) cudaStreamDestroy(s);
  for (auto h : b->h)
    if (h) sdg_destroy(h);
  if (b->start) cudaEventDestroy(b->start);
  delete b;
}

}  // namespace

extern "C" {

int sdg_batch_create(const sdg_grid* grids, const int* N, const double* nu, int nprob, double theta, double dt,
                     sdg_batch** out) {
  if (!grids || !N || !nu || !out || nprob < 1) {
    sdg::set_last_error("sdg_batch_create: NULL argument or nprob < 1");
    return SDG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sdg_batch* b = new (std::nothrow) sdg_batch();
  if (!b) return SDG_ERR_CUDA;
  b->nprob = nprob;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    destroy(b);
    sdg::set_last_error("sdg_batch_create: no current device");
    return SDG_ERR_CUDA;
  }
  b->h.assign(nprob, nullptr);
  b->s.assign(nprob, nullptr);
  b->done.assign(nprob, nullptr);
  std::vector<long long> size(nprob, 0);
  for (int i = 0; i < nprob; ++i) {
    const int rc = sdg_create(&grids[i], N[i], nu[i], theta, dt, &b->h[i]);
    if (rc != SDG_OK) {
      const std::string msg = std::string("sdg_batch_create: member ") + std::to_string(i) + ": " + sdg_last_error();
      destroy(b);
      sdg::set_last_error(msg.c_str());
      return rc;
    }
    size[i] = sdg_ndof(b->h[i]);
    if (cudaStreamCreateWithFlags(&b->s[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess) {
      destroy(b);
      sdg::set_last_error("sdg_batch_create: stream or event creation failed");
      return SDG_ERR_CUDA;
    }
  }
  if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
    destroy(b);
    sdg::set_last_error("sdg_batch_create: event creation failed");
    return SDG_ERR_CUDA;
  }
  b->order.resize(nprob);
  for (int i = 0; i < nprob; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return size[a] > size[c]; });
  const unsigned hw = std::thread::hardware_concurrency();
  b->nthreads = std::max(1, std::min(nprob, std::min(16, (int)(hw ? hw : 4))));
  *out = b;
  return SDG_OK;
}

int sdg_batch_destroy(sdg_batch* b) {
  if (!b) return SDG_OK;
  for (auto s : b->s)
    if (s) cudaStreamSynchronize(s);
  destroy(b);
  return SDG_OK;
}

int sdg_batch_size(const sdg_batch* b) { return b ? b->nprob : 0; }

int sdg_batch_member(sdg_batch* b, int i, sdg_handle** h) {
  if (!b || !h || i < 0 || i >= b->nprob) {
    sdg::set_last_error("sdg_batch_member: bad batch, index or output");
    return SDG_ERR_INVALID_ARG;
  }
  *h = b->h[i];
  return SDG_OK;
}

int sdg_batch_set_threads(sdg_batch* b, int nthreads) {
  if (!b || nthreads < 1 || nthreads > 256) {
    sdg::set_last_error("sdg_batch_set_threads: nthreads must be in [1, 256]");
    return SDG_ERR_INVALID_ARG;
  }
  b->nthreads = std::min(nthreads, b->nprob);
  return SDG_OK;
}

int sdg_batch_step(sdg_batch* b, int nsteps, sdg_step_info* info, void* stream) {
  if (!b || nsteps < 0) {
    sdg::set_last_error("sdg_batch_step: bad arguments");
    return SDG_ERR_INVALID_ARG;
  }
  cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
  if (cudaEventRecord(b->start, caller) != cudaSuccess) return SDG_ERR_CUDA;
  for (int i = 0; i < b->nprob; ++i)
    if (cudaStreamWaitEvent(b->s[i], b->start, 0) != cudaSuccess) return SDG_ERR_CUDA;
  std::vector<int> rc(b->nprob, SDG_OK);
  std::vector<std::string> err(b->nprob);
  std::vector<sdg_step_info> local(b->nprob);
  std::atomic<int> next{0};
  auto worker = [&]() {
    if (cudaSetDevice(b->device) != cudaSuccess) return;
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= b->nprob) break;
      const int i = b->order[k];
      rc[i] = sdg_step(b->h[i], nsteps, &local[i], b->s[i]);
      if (rc[i] != SDG_OK) err[i] = sdg_last_error();
      if (cudaEventRecord(b->done[i], b->s[i]) != cudaSuccess && rc[i] == SDG_OK) {
        rc[i] = SDG_ERR_CUDA;
        err[i] = "event record failed";
      }
    }
  };
  std::vector<std::thread> pool;
  const int nt = std::min(b->nthreads, b->nprob);
  pool.reserve(nt);
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  if (next.load() < b->nprob) {  // a worker could not select the device
    sdg::set_last_error("sdg_batch_step: cudaSetDevice failed in a worker thread");
    return SDG_ERR_CUDA;
  }
  int first = SDG_OK;
  for (int i = 0; i < b->nprob; ++i) {
    if (cudaStreamWaitEvent(caller, b->done[i], 0) != cudaSuccess) return SDG_ERR_CUDA;
    if (info) info[i] = local[i];
    if (rc[i] != SDG_OK && first == SDG_OK) {
      first = rc[i];
      const std::string msg = std::string("sdg_batch_step: member ") + std::to_string(i) + ": " + err[i];
      sdg::set_last_error(msg.c_str());
    }
  }
  return first;
}

}  // extern "C"

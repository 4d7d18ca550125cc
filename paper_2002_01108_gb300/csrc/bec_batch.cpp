// Batched solves of many independent all-at-once problems of uneven size.
//
// Each instance is a bec_problem with its own workspace, bound to one of a
// few internal CUDA streams.  bec_batch_solve advances every instance's
// GMRES state machine in rounds: it enqueues the next step of every active
// instance on its stream (Arnoldi iterations replayed from per-iteration CUDA
// graphs when enabled), then waits once per stream, then lets every instance
// read its scalars and decide.  Host synchronisation is per round, not per
// instance and iteration, and instances on different streams overlap on the
// GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "bec_internal.h"

struct bec_batch {
  std::vector<bec_problem*> probs;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_of;
  int use_graphs = 1;
  long long total_U = 0;
};

namespace {

void batch_release(bec_batch* b) {
  for (bec_problem* p : b->probs) bec_free_problem(p);
  b->probs.clear();
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  b->streams.clear();
}

bec_status batch_einval(const char* msg) {
  bec::set_error(msg);
  return BEC_EINVAL;
}

}  // namespace

extern "C" {

bec_status bec_batch_create(const bec_problem_desc* descs, const double* eps, int count,
                            int nstreams, int use_graphs, bec_batch** out) {
  if (descs == nullptr || eps == nullptr || out == nullptr) return batch_einval("null argument");
  *out = nullptr;
  if (count < 1) return batch_einval("count must be >= 1");
  if (nstreams < 1 || nstreams > 64) return batch_einval("nstreams must lie in [1, 64]");
  bec_batch* b = new (std::nothrow) bec_batch();
  if (b == nullptr) return BEC_ENOMEM;
  b->use_graphs = use_graphs ? 1 : 0;
  const int ns = std::min(nstreams, count);
  for (int i = 0; i < ns; ++i) {
    cudaStream_t s = nullptr;
    const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      batch_release(b);
      delete b;
      return bec::cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    b->streams.push_back(s);
  }
  for (int i = 0; i < count; ++i) {
    bec_problem* p = nullptr;
    const int si = i % ns;
    bec_status st = bec_allocate_problem(&descs[i], b->streams[si], &p);
    if (st == BEC_OK) st = bec_set_eps(p, eps[i]);
    if (st == BEC_OK) st = bec_autotune(p, 0, nullptr);   // once per distinct shape (cached)
    if (st != BEC_OK) {
      if (p) bec_free_problem(p);
      const std::string msg = "instance " + std::to_string(i) + ": " + bec_last_error();
      batch_release(b);
      delete b;
      bec::set_error(msg);
      return st;
    }
    b->probs.push_back(p);
    b->stream_of.push_back(si);
    b->total_U += bec_problem_size(p);
  }
  *out = b;
  return BEC_OK;
}

bec_status bec_batch_problem(bec_batch* b, int i, bec_problem** out) {
  if (b == nullptr || out == nullptr) return batch_einval("null argument");
  if (i < 0 || i >= (int)b->probs.size()) return batch_einval("instance index out of range");
  *out = b->probs[i];
  return BEC_OK;
}

long long bec_batch_unknowns(const bec_batch* b) { return b ? b->total_U : 0; }

long long bec_batch_kernel_launches(const bec_batch* b) {
  long long n = 0;
  if (b)
    for (const bec_problem* p : b->probs) n += bec_kernel_launches(p);
  return n;
}

bec_status bec_batch_solve(bec_batch* b, const double* const* f, double* const* u,
                           const bec_gmres_opts* opts, bec_gmres_info* infos) {
  if (b == nullptr || f == nullptr || u == nullptr || opts == nullptr)
    return batch_einval("null argument");
  const int n = (int)b->probs.size();
  std::vector<bec::GmresRun> runs(n);
  for (int i = 0; i < n; ++i) {
    bec_problem* p = b->probs[i];
    const bec_status st = bec::check_gmres_opts(p, opts);
    if (st != BEC_OK) return st;
    if (f[i] == nullptr || u[i] == nullptr) return batch_einval("null vector pointer");
    if ((reinterpret_cast<uintptr_t>(f[i]) & 15u) || (reinterpret_cast<uintptr_t>(u[i]) & 15u))
      return batch_einval("f[i] and u[i] must be 16-byte aligned");
    bec::gmres_run_init(runs[i], p, f[i], u[i], *opts, b->use_graphs != 0);
  }
  bec_status first_error = BEC_OK;
  std::vector<char> busy(b->streams.size());
  while (true) {
    std::fill(busy.begin(), busy.end(), 0);
    int active = 0;
    for (int i = 0; i < n; ++i) {
      bec::GmresRun& r = runs[i];
      bool enq = false;
      // host-only steps run back to back; stop at the first one that enqueues
      while (r.state != bec::GmresRun::DONE && !enq) {
        const bec_status st = bec::gmres_run_step(r, &enq);
        if (st != BEC_OK) {
          if (first_error == BEC_OK) first_error = st;
          r.state = bec::GmresRun::DONE;
          r.status = st;
        }
      }
      if (enq) {
        busy[b->stream_of[i]] = 1;
        ++active;
      }
    }
    if (active == 0) break;
    for (size_t s = 0; s < b->streams.size(); ++s)
      if (busy[s]) {
        const cudaError_t e = cudaStreamSynchronize(b->streams[s]);
        if (e != cudaSuccess) return bec::cuda_fail(e, "cudaStreamSynchronize");
      }
  }
  bool all_conv = true;
  for (int i = 0; i < n; ++i) {
    if (infos) bec::gmres_run_info(runs[i], &infos[i]);
    all_conv = all_conv && runs[i].converged;
    if (b->probs[i]->net) {
      const bec_status st = bec::net_check(b->probs[i]);
      if (st != BEC_OK && first_error == BEC_OK) first_error = st;
    }
  }
  if (first_error != BEC_OK) return first_error;
  return all_conv ? BEC_OK : BEC_ENOTCONV;
}

bec_status bec_batch_free(bec_batch* b) {
  if (b == nullptr) return BEC_OK;
  batch_release(b);
  delete b;
  return BEC_OK;
}

}  // extern "C"

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
  int persistent = 0;                   // BEC_BATCH_PERSISTENT
  long long total_U = 0;
  // persistent mode: the job table (pinned host and device copies), the
  // queue counters and the error words of a round's launches
  bec::PersistJob* jobs_host = nullptr;
  bec::PersistJob* jobs_dev = nullptr;
  int* ctr_dev = nullptr;
  int* err_host = nullptr;
  long long persist_launches = 0;
};

namespace {

void batch_release(bec_batch* b) {
  for (bec_problem* p : b->probs) bec_free_problem(p);
  b->probs.clear();
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  b->streams.clear();
  if (b->jobs_host) cudaFreeHost(b->jobs_host);
  if (b->err_host) cudaFreeHost(b->err_host);
  if (b->jobs_dev) cudaFree(b->jobs_dev);
  if (b->ctr_dev) cudaFree(b->ctr_dev);
  b->jobs_host = nullptr;
  b->err_host = nullptr;
  b->jobs_dev = nullptr;
  b->ctr_dev = nullptr;
}

constexpr int kCtrInts = 4 + 5 * bec::kPersistMaxJobs;   // queue counters of one launch

// the persistent mode's job table (one entry per instance) and the counters
// and error words of up to `count` launches per round
bec_status persist_alloc(bec_batch* b, int count) {
  BEC_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&b->jobs_host),
                              (size_t)count * sizeof(bec::PersistJob)));
  BEC_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&b->err_host), (size_t)count * sizeof(int)));
  BEC_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&b->jobs_dev),
                          (size_t)count * sizeof(bec::PersistJob)));
  BEC_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&b->ctr_dev), (size_t)count * kCtrInts * sizeof(int)));
  return BEC_OK;
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
  if (use_graphs < 0 || use_graphs > BEC_BATCH_PERSISTENT)
    return batch_einval("mode must be BEC_BATCH_STREAMS, BEC_BATCH_GRAPHS or BEC_BATCH_PERSISTENT");
  bec_batch* b = new (std::nothrow) bec_batch();
  if (b == nullptr) return BEC_ENOMEM;
  b->use_graphs = use_graphs ? 1 : 0;
  b->persistent = use_graphs == BEC_BATCH_PERSISTENT ? 1 : 0;
  if (b->persistent) {
    const bec_status st = persist_alloc(b, count);
    if (st != BEC_OK) {
      batch_release(b);
      delete b;
      return st;
    }
  }
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
    if (st == BEC_OK && b->persistent && !bec::persist_supported(p)) {
      bec::set_error("BEC_BATCH_PERSISTENT needs FP32 sine-transform instances in 2D (finite "
                     "differences, backward Euler) with sides 31..255 and N 4..512");
      st = BEC_EINVAL;
    }
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
  if (b) {
    for (const bec_problem* p : b->probs) n += bec_kernel_launches(p);
    n += b->persist_launches;
  }
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
    const bec_status sp = bec::net_prepare(p);
    if (sp != BEC_OK) return sp;
    bec::gmres_run_init(runs[i], p, f[i], u[i], *opts, b->use_graphs != 0);
  }
  if (b->persistent) {
    if (opts->left_pc) return batch_einval("BEC_BATCH_PERSISTENT needs right preconditioning");
    for (auto& r : runs) r.ext_pinv = true;
  }
  bec_status first_error = BEC_OK;
  std::vector<char> busy(b->streams.size());
  std::vector<int> at_iter;
  while (true) {
    std::fill(busy.begin(), busy.end(), 0);
    at_iter.clear();
    int active = 0;
    for (int i = 0; i < n; ++i) {
      bec::GmresRun& r = runs[i];
      bool enq = false;
      // host-only steps run back to back; stop at the first one that
      // enqueues (or, in persistent mode, at an Arnoldi step: its P_eps^{-1}
      // goes into the round's shared launch first)
      while (r.state != bec::GmresRun::DONE && !enq) {
        if (b->persistent && r.state == bec::GmresRun::ITER) {
          at_iter.push_back(i);
          break;
        }
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
    int launches = 0;
    if (!at_iter.empty()) {
      // per stream, the P_eps^{-1} of every instance of that stream that takes
      // an Arnoldi step, in shared launches of up to kPersistMaxJobs jobs on
      // the stream itself; then the rest of each step, in stream order.
      // Different streams' launches and Krylov steps overlap on the GPU.
      int slot = 0;   // next free entry of the job table
      for (size_t si = 0; si < b->streams.size(); ++si) {
        std::vector<int> mine;
        for (int i : at_iter)
          if (b->stream_of[i] == (int)si) mine.push_back(i);
        for (size_t c0 = 0; c0 < mine.size(); c0 += bec::kPersistMaxJobs) {
          const int nj = (int)std::min<size_t>(bec::kPersistMaxJobs, mine.size() - c0);
          bec::PersistJob* jh = b->jobs_host + slot;
          for (int k = 0; k < nj; ++k) {
            const double* y = nullptr;
            double* z = nullptr;
            const double* sc = nullptr;
            bec::gmres_run_pinv_operands(runs[mine[c0 + k]], &y, &z, &sc);
            bec::persist_make_job(runs[mine[c0 + k]].p, y, z, sc, &jh[k]);
          }
          bec::PersistQueue q;
          int* ctr = b->ctr_dev + (size_t)launches * kCtrInts;
          const bec_status st = bec::persist_launch(jh, b->jobs_dev + slot, nj, &q, ctr,
                                                    bec::persist_take_withhold(), b->streams[si]);
          if (st != BEC_OK) return st;
          ++b->persist_launches;
          // the launch's error word, read once the round has drained
          BEC_CUDA_TRY(cudaMemcpyAsync(b->err_host + launches, ctr + 1, sizeof(int),
                                       cudaMemcpyDeviceToHost, b->streams[si]));
          slot += nj;
          ++launches;
        }
        for (int i : mine) {
          bool enq = false;
          const bec_status st = bec::gmres_run_step(runs[i], &enq);   // the rest of the step
          if (st != BEC_OK) {
            if (first_error == BEC_OK) first_error = st;
            runs[i].state = bec::GmresRun::DONE;
            runs[i].status = st;
          }
          busy[si] = 1;
          if (enq) ++active;
        }
      }
    }
    if (active == 0 && launches == 0) break;
    for (size_t s = 0; s < b->streams.size(); ++s)
      if (busy[s]) {
        const cudaError_t e = cudaStreamSynchronize(b->streams[s]);
        if (e != cudaSuccess) return bec::cuda_fail(e, "cudaStreamSynchronize");
      }
    for (int c = 0; c < launches; ++c)
      if (b->err_host[c] != 0) {
        bec::set_error("persistent batch launch: a bounded wait for an earlier pass ran out");
        return BEC_ETIMEOUT;
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
    const bec_status pst = bec::pc_check(b->probs[i]);
    if (pst != BEC_OK && first_error == BEC_OK) first_error = pst;
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

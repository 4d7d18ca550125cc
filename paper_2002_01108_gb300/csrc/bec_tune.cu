// Autotuning of the block widths of the P_eps^{-1} passes (bec_autotune).
//
// Each pass (x-DST, y-DST, time pass) is launched with 4, 8 or 16 warps per
// block on the problem's own workspace (the Krylov basis and the FP32
// scratch, zeroed first; no solve is running), timed with CUDA events over
// 5 launches after 2 warm-up launches, and the fastest width is kept.  A
// width whose shared memory does not fit a block is skipped.  The width only
// changes how lines are grouped into blocks, not what each warp computes, so
// every choice gives the same result bit for bit.  Choices are cached per
// (precision, dim, nx, N) for the process, so the instances of a batch that
// share a shape are tuned once.  When the environment variable
// BEC_TUNE_CACHE names a file, earlier choices are read from it once per
// process and every new choice is appended to it ("fp64 dim nx N rows cols
// time" per line), so other processes reuse them without timing again.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "bec_fft.cuh"
#include "bec_internal.h"
#include "bec_passes.cuh"

namespace bec {
namespace {

using Key = std::tuple<int, int, int, int>;

std::mutex& cache_mutex() {
  static std::mutex m;
  return m;
}

std::map<Key, TileChoice>& cache() {
  static std::map<Key, TileChoice> c;
  return c;
}

const char* cache_file() {
  const char* f = std::getenv("BEC_TUNE_CACHE");
  return (f != nullptr && f[0] != '\0') ? f : nullptr;
}

bool valid_width(int w) { return w == 0 || w == 4 || w == 8 || w == 16; }

// reads the cache file into the process cache (once; under cache_mutex)
void load_cache_file() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = cache_file();
  if (path == nullptr) return;
  FILE* fh = std::fopen(path, "r");
  if (fh == nullptr) return;
  char line[256];
  while (std::fgets(line, sizeof line, fh) != nullptr) {   // a malformed line is skipped
    int f64, dim, m, N, r, c, t;
    if (std::sscanf(line, "%d %d %d %d %d %d %d", &f64, &dim, &m, &N, &r, &c, &t) == 7 &&
        valid_width(r) && valid_width(c) && valid_width(t))
      cache()[Key{f64, dim, m, N}] = TileChoice{r, c, t};
  }
  std::fclose(fh);
}

void append_cache_file(const Key& k, const TileChoice& t) {
  const char* path = cache_file();
  if (path == nullptr) return;
  FILE* fh = std::fopen(path, "a");
  if (fh == nullptr) return;
  std::fprintf(fh, "%d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
               std::get<3>(k), t.rows, t.cols, t.time);
  std::fclose(fh);
}

int default_width(int which, int tsize) {
  return which == 0 ? kRowsWarps : which == 1 ? default_cols_warps(tsize) : default_time_warps(tsize);
}

}  // namespace

size_t pass_smem_bytes(int which, int logn, int fp64, int w) {
  const int tsize = fp64 ? 8 : 4;
  if (w == 0) w = default_width(which, tsize);
  const int slots = which == 2 ? line_slots(logn) : dst_line_stride(logn, tsize);
  return (size_t)w * 2 * slots * tsize;
}

bec_status autotune(bec_problem* p, int force, bec_tune_report* rep) {
  NvtxRange range("bec autotune");
  bec_tune_report r = {};
  const int fp64 = p->desc.precision == BEC_PC_FP64;
  const int tsize = fp64 ? 8 : 4;
  const Key key{fp64, p->dim, p->m, p->N};
  if (p->desc.route != BEC_ROUTE_FST) {   // the other routes have no tunable pass
    if (rep) *rep = r;
    return BEC_OK;
  }
  if (!force) {
    std::lock_guard<std::mutex> g(cache_mutex());
    load_cache_file();
    auto it = cache().find(key);
    if (it != cache().end()) {
      p->tile = it->second;
      r.rows_warps = p->tile.rows ? p->tile.rows : default_width(0, tsize);
      r.cols_warps = cols16_applies(p) ? kD16Threads / 32
                     : p->tile.cols ? p->tile.cols : default_width(1, tsize);
      r.time_warps = time16_applies(p) ? kT16Threads / 32
                     : p->tile.time ? p->tile.time : default_width(2, tsize);
      r.cached = 1;
      if (rep) *rep = r;
      return BEC_OK;
    }
  }
  int dev = 0, limit = 0;
  BEC_CUDA_TRY(cudaGetDevice(&dev));
  BEC_CUDA_TRY(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  double* x = p->V;
  void* s = p->pc_scratch;
  BEC_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)p->U * sizeof(double), p->stream));
  if (!fp64) BEC_CUDA_TRY(cudaMemsetAsync(s, 0, (size_t)p->N * p->Jp * sizeof(float), p->stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BEC_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  }
  const long long rows = p->J / p->m * p->N;
  const int cand[3] = {4, 8, 16};
  float* out_ms[3] = {r.rows_ms, r.cols_ms, r.time_ms};
  int best[3] = {0, 0, 0};
  bec_status st = BEC_OK;
  for (int which = 0; which < 3 && st == BEC_OK; ++which) {
    if (which == 1 && p->dim < 2) continue;
    if (which == 2 && time16_applies(p)) continue;   // fixed block of 8 warps
    if (which == 1 && cols16_applies(p)) continue;   // likewise
    const int logn = which == 2 ? p->tab.time.logn : p->tab.space.logn;
    if (logn < 5) continue;                       // short transforms: default width only
    float best_ms = -1.f;
    for (int c = 0; c < 3 && st == BEC_OK; ++c) {
      const int w = cand[c];
      if (pass_smem_bytes(which, logn, fp64, w) > (size_t)limit) continue;
      auto launch = [&]() -> bec_status {
        if (which == 0)
          return fp64 ? launch_dst_rows_w(p, x, 1, x, 1, rows, 1, w)
                      : launch_dst_rows_w(p, x, 1, s, 0, rows, 0, w);
        if (which == 1) return launch_dst_cols_w(p, fp64 ? (void*)x : s, fp64, w);
        return launch_time_pass_w(p, fp64 ? (void*)x : s, fp64, 1.0, nullptr, w);
      };
      for (int i = 0; i < 2 && st == BEC_OK; ++i) st = launch();
      if (st != BEC_OK) break;
      if (cudaEventRecord(e0, p->stream) != cudaSuccess) st = BEC_ECUDA;
      for (int i = 0; i < 5 && st == BEC_OK; ++i) st = launch();
      if (st == BEC_OK && cudaEventRecord(e1, p->stream) != cudaSuccess) st = BEC_ECUDA;
      if (st == BEC_OK && cudaEventSynchronize(e1) != cudaSuccess) st = BEC_ECUDA;
      float ms = 0.f;
      if (st == BEC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = BEC_ECUDA;
      if (st != BEC_OK) break;
      out_ms[which][c] = ms / 5.f;
      if (best_ms < 0.f || ms / 5.f < best_ms) {
        best_ms = ms / 5.f;
        best[which] = w;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BEC_OK) {
    if (st == BEC_ECUDA) set_error("autotune: event timing failed");
    return st;
  }
  p->tile.rows = best[0];
  p->tile.cols = best[1];
  p->tile.time = best[2];
  {
    std::lock_guard<std::mutex> g(cache_mutex());
    cache()[key] = p->tile;
    append_cache_file(key, p->tile);
  }
  r.rows_warps = best[0] ? best[0] : default_width(0, tsize);
  r.cols_warps = cols16_applies(p) ? kD16Threads / 32 : best[1] ? best[1] : default_width(1, tsize);
  r.time_warps = time16_applies(p) ? kT16Threads / 32 : best[2] ? best[2] : default_width(2, tsize);
  if (rep) *rep = r;
  return BEC_OK;
}

bec_status set_tiles(bec_problem* p, int rows, int cols, int time) {
  const int v[3] = {rows, cols, time};
  const int fp64 = p->desc.precision == BEC_PC_FP64;
  int dev = 0, limit = 0;
  BEC_CUDA_TRY(cudaGetDevice(&dev));
  BEC_CUDA_TRY(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  for (int which = 0; which < 3; ++which) {
    if (v[which] != 0 && v[which] != 4 && v[which] != 8 && v[which] != 16) {
      set_error("block widths must be 0 (default), 4, 8 or 16 warps");
      return BEC_EINVAL;
    }
    const int logn = which == 2 ? p->tab.time.logn : p->tab.space.logn;
    if (v[which] != 0 && logn < 5) {
      set_error("block widths are tunable only for transforms of length >= 32");
      return BEC_EINVAL;
    }
    if (pass_smem_bytes(which, logn, fp64, v[which]) > (size_t)limit) {
      set_error("block width needs more shared memory than a block has");
      return BEC_EINVAL;
    }
  }
  p->tile.rows = rows;
  p->tile.cols = cols;
  p->tile.time = time;
  return BEC_OK;
}

}  // namespace bec

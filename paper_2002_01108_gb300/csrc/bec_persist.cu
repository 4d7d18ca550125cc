// Persistent batched P_eps^{-1}: the FP32 sine-transform preconditioner
// (Sec. 4: scale and FFT in time, shifted solves by the 2D DST-I, inverse FFT
// and unscale) of every active instance of a batch in ONE kernel launch.
//
// Work is a queue of items (pass p, instance i, tile t), numbered pass-major:
// all x-DST tiles of every instance, then all y-DST tiles, the time-pass
// tiles, the inverse y-DST and the inverse x-DST tiles.  The launch has one
// block per item, and every block takes its item from one atomic counter
// (a device work queue), not from its block index.  Before an item of pass
// p > 0 a block waits until every tile of pass p - 1 of the same instance has
// been signalled done; after its item it signals its own.  Items are handed
// out in order, so every item a block waits for was taken earlier by a block
// that is already running: the waits always end unless a block stops.  Each
// wait is bounded (about 0.2 s): on running out it sets an error word and an
// abort flag, every later block leaves at once, and the host reports
// BEC_ETIMEOUT.  (A loop of items per resident block was tried first: the
// tiles of all shapes inside one loop made the compiler spill; one item per
// block needs 64 registers.)
//
// The tiles are those of the per-instance pass kernels (bec_passes.cuh) at 8
// warps per block (for N = 256 the time pass, and for n = 256 the y-DST,
// take the four-step tiles of 32 modes or columns, as the per-instance FP32
// passes do); sizes: sides 31..255
// (n = 32..256) and N = 4..512.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "bec_fft.cuh"
#include "bec_internal.h"
#include "bec_passes.cuh"

namespace bec {
namespace {

constexpr int kPWarps = 8;
constexpr int kPThreads = kPWarps * 32;
constexpr int kPasses = 5;
constexpr long long kPSpinCycles = 400000000ll;   // ~0.2 s at 2 GHz

// counters: [0] queue head, [1] error word, [2] abort flag, [3] unused,
// then done[i * kPasses + p]
constexpr int kCHead = 0, kCErr = 1, kCAbort = 2, kCDone = 4;

__device__ __forceinline__ int ld_volatile(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// waits until *cnt >= target or the abort flag is set; false on running out
// or abort (the caller then sets the abort flag)
__device__ bool wait_count(int* ctr, const int* cnt, int target) {
  const long long t0 = clock64();
  while (true) {
    if (ld_volatile(cnt) >= target) return true;
    if (ld_volatile(ctr + kCAbort)) return false;
    if (clock64() - t0 > kPSpinCycles) {
      atomicExch(ctr + kCErr, 1);
      return false;
    }
    __nanosleep(64);
  }
}

// pass p of job j on tile t (LOGN: spatial transform length, LOGT: time).
// One tile per item: a loop over several tiles per block made the compiler
// keep every shape's per-thread values live and spill.
template <int LOGN>
__device__ __forceinline__ void space_pass(const PersistJob& j, int p, long long t,
                                           unsigned char* sm) {
  const long long rows = (long long)j.N * j.m;
  const int tid = threadIdx.x;
  if (p == 0) {
    dst_rows_tile<float, double, float, LOGN, kPWarps>(j.y, j.s, rows, j.m, j.m, j.ld, j.sin2, j.tws,
                                                       t, sm, tid);
  } else if (p == 4) {
    dst_rows_tile<float, float, double, LOGN, kPWarps>(j.s, j.z, rows, j.m, j.ld, j.m, j.sin2, j.tws,
                                                       t, sm, tid);
  } else if constexpr (LOGN == 8) {
    // the four-step column tile of the per-instance kernel (32 columns of one
    // slice), its stage filled and emptied with plain 16-byte copies
    static_assert(kPThreads == kD16Threads, "the n = 256 column tile takes 256 threads");
    const int cb = j.ld / kD16Cols;
    float* const st = reinterpret_cast<float*>(sm);
    float* const base = j.s + (t / cb) * (long long)j.m * j.ld + (t % cb) * kD16Cols;
    for (int e = tid; e < j.m * (kD16Cols / 4); e += kPThreads) {
      const int row = e / (kD16Cols / 4), c4 = e - row * (kD16Cols / 4);
      reinterpret_cast<float4*>(st)[e] =
          *reinterpret_cast<const float4*>(base + (long long)row * j.ld + 4 * c4);
    }
    __syncthreads();
    dst16_cols_core(st, nullptr, reinterpret_cast<float2*>(sm + kD16StageBytes), j.sin2, j.tws,
                    tid);
    __syncthreads();
    for (int e = tid; e < j.m * (kD16Cols / 4); e += kPThreads) {
      const int row = e / (kD16Cols / 4), c4 = e - row * (kD16Cols / 4);
      *reinterpret_cast<float4*>(base + (long long)row * j.ld + 4 * c4) =
          reinterpret_cast<const float4*>(st)[e];
    }
  } else {
    const long long cb = (j.m + 2 * kPWarps - 1) / (2 * kPWarps);
    dst_cols_tile<float, LOGN, kPWarps>(j.s, j.m, j.m, j.ld, (long long)j.m * j.ld, t % cb, t / cb,
                                        j.sin2, j.tws, sm,
                                        tid);
  }
}

template <int LOGT>
__device__ __forceinline__ void time_pass(const PersistJob& j, long long t, unsigned char* sm) {
  if constexpr (LOGT == 8) {       // the four-step tile of the per-instance kernel (256 threads)
    static_assert(kPThreads == kT16Threads, "the N = 256 time tile takes 256 threads");
    time_pass16_tile<false, false>(j.s, nullptr, j.J, j.m, j.ld, 2, j.es, j.eis, j.lamf, ModeEigs<float>{j.mu, nullptr},
                            j.tau, j.scale_h, j.scale_dev, j.twt, t, sm, threadIdx.x);
    return;
  }
  time_pass_tile<float, LOGT, kPWarps, false>(j.s, j.J, j.m, j.ld, 2, j.es, j.eis, j.lamf,
                                              ModeEigs<float>{j.mu, nullptr}, j.tau, j.scale_h,
                                              j.scale_dev, j.twt, nullptr, t, sm, threadIdx.x);
}

__device__ __forceinline__ void run_item(const PersistJob& j, int p, long long t,
                                         unsigned char* sm) {
  if (p == 2) {
    switch (j.logt) {
      case 2: time_pass<2>(j, t, sm); break;
      case 3: time_pass<3>(j, t, sm); break;
      case 4: time_pass<4>(j, t, sm); break;
      case 5: time_pass<5>(j, t, sm); break;
      case 6: time_pass<6>(j, t, sm); break;
      case 7: time_pass<7>(j, t, sm); break;
      case 8: time_pass<8>(j, t, sm); break;
      case 9: time_pass<9>(j, t, sm); break;
      default: break;
    }
    return;
  }
  switch (j.logn) {
    case 5: space_pass<5>(j, p, t, sm); break;
    case 6: space_pass<6>(j, p, t, sm); break;
    case 7: space_pass<7>(j, p, t, sm); break;
    case 8: space_pass<8>(j, p, t, sm); break;
    default: break;
  }
}

// One block per item: the block takes the next item number from the queue
// counter (not its block index), so items start in queue order whatever
// order the hardware starts the blocks in.
__global__ void __launch_bounds__(kPThreads, 4)
persist_pinv_kernel(const PersistJob* __restrict__ jobs, const __grid_constant__ PersistQueue q,
                    int* ctr) {
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  __shared__ int s_item, s_p, s_i, s_go;
  if (threadIdx.x == 0) {
    const int item = ld_volatile(ctr + kCAbort) ? q.total : atomicAdd(ctr + kCHead, 1);
    int go = item < q.total ? 1 : 0;
    int p = 0, i = 0;
    if (go) {
      while (p + 1 < kPasses && item >= q.pass_start[p + 1]) ++p;
      const int* st = q.job_start + p * (q.njobs + 1);
      while (i + 1 < q.njobs && item >= st[i + 1]) ++i;
      if (p > 0) {
        const int target = q.target[i * kPasses + p - 1];
        if (!wait_count(ctr, ctr + kCDone + i * kPasses + p - 1, target)) {
          atomicExch(ctr + kCAbort, 1);
          go = 0;
        }
        __threadfence();
      }
    }
    s_item = item;
    s_p = p;
    s_i = i;
    s_go = go;
  }
  __syncthreads();
  if (!s_go) return;
  const int p = s_p, i = s_i;
  const long long t = s_item - q.job_start[p * (q.njobs + 1) + i];
  run_item(jobs[i], p, t, smem_bytes);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr + kCDone + i * kPasses + p, 1);
  }
}

// Dynamic shared memory of one job's largest tile.
size_t job_smem(int logn, int logt) {
  const size_t sp = logn == 8 ? kD16StageBytes + kD16TotBytes
                              : (size_t)kPWarps * 2 * dst_line_stride(logn, 4) * sizeof(float);
  const size_t tm = logt == 8 ? kT16Smem : (size_t)kPWarps * 2 * line_slots(logt) * sizeof(float);
  return std::max(sp, tm);
}

std::mutex g_attr_mutex;
bool g_attr_set = false;
std::atomic<int> g_withhold{0};   // set by bec_inject_fault, taken by the next launch

}  // namespace

void persist_withhold_next() { g_withhold.store(1); }
int persist_take_withhold() { return g_withhold.exchange(0); }

bool persist_supported(const bec_problem* p) {
  const int logn = p->tab.space.logn, logt = p->tab.time.logn;
  return p->desc.route == BEC_ROUTE_FST && p->desc.precision == BEC_PC_FP32 && p->dim == 2 &&
         p->desc.space == BEC_SPACE_FD && p->desc.time_scheme == BEC_TIME_BDF1 && logn >= 5 &&
         logn <= 8 && logt >= 2 && logt <= 9;
}

void persist_make_job(const bec_problem* p, const double* y, double* z, const double* scale_dev,
                      PersistJob* j) {
  const double n = (double)(p->m + 1);
  const double per_axis = (2.0 / n) / 16.0;   // (orthonormal / raw)^2 for one forward+inverse pair
  const double scale = 0.5 / p->N * per_axis * per_axis;
  j->y = y;
  j->z = z;
  j->s = static_cast<float*>(p->pc_scratch);
  j->scale_dev = scale_dev;
  j->sin2 = p->tab.sin2_32;
  j->tws = p->tab.space.tw32;
  j->twt = p->tab.time.tw32;
  j->es = p->tab.es32;
  j->eis = p->tab.eis32;
  j->lamf = p->tab.lamf32;
  j->mu = p->tab.mu32;
  j->J = p->Jp;   // the scratch in the layout of the per-instance passes
  j->ld = p->ld;
  j->tau = (float)p->tau;
  j->scale_h = (float)scale;
  j->m = p->m;
  j->N = p->N;
  j->logn = p->tab.space.logn;
  j->logt = p->tab.time.logn;
  const long long rows = (long long)p->N * p->m;
  const long long row_tiles = (rows + 2 * kPWarps - 1) / (2 * kPWarps);
  const long long col_tiles = p->tab.space.logn == 8
                                  ? (long long)(p->ld / kD16Cols) * p->N
                                  : (long long)((p->m + 2 * kPWarps - 1) / (2 * kPWarps)) * p->N;
  const long long time_modes = p->N == 256 ? kT16Modes : 2 * kPWarps;   // modes per time tile
  const long long time_tiles = (p->Jp + time_modes - 1) / time_modes;
  j->tiles[0] = (int)row_tiles;
  j->tiles[1] = (int)col_tiles;
  j->tiles[2] = (int)time_tiles;
  j->tiles[3] = (int)col_tiles;
  j->tiles[4] = (int)row_tiles;
}

bec_status persist_launch(const PersistJob* jobs_host, PersistJob* jobs_dev, int njobs,
                          PersistQueue* qh, int* ctr_dev, int withhold, cudaStream_t st) {
  if (njobs < 1 || njobs > kPersistMaxJobs) {
    set_error("persistent batch: job count outside [1, 64]");
    return BEC_EINVAL;
  }
  PersistQueue& q = *qh;
  q.njobs = njobs;
  int item = 0;
  size_t smem = 0;
  for (int p = 0; p < kPasses; ++p) {
    q.pass_start[p] = item;
    for (int i = 0; i < njobs; ++i) {
      q.job_start[p * (njobs + 1) + i] = item;
      item += jobs_host[i].tiles[p];
    }
    q.job_start[p * (njobs + 1) + njobs] = item;
  }
  q.pass_start[kPasses] = item;
  q.total = item;
  for (int i = 0; i < njobs; ++i) {
    for (int p = 0; p < kPasses; ++p) q.target[i * kPasses + p] = jobs_host[i].tiles[p];
    smem = std::max(smem, job_smem(jobs_host[i].logn, jobs_host[i].logt));
  }
  // a test of the bounded waits: instance 0's x-DST is never reported
  // complete, so its y-DST items wait until they run out
  if (withhold) q.target[0] += 1;
  BEC_CUDA_TRY(cudaMemcpyAsync(jobs_dev, jobs_host, (size_t)njobs * sizeof(PersistJob),
                               cudaMemcpyHostToDevice, st));
  BEC_CUDA_TRY(cudaMemsetAsync(ctr_dev, 0, (size_t)(kCDone + njobs * kPasses) * sizeof(int), st));
  {
    // once per process: room for the largest tile any supported job needs
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (!g_attr_set) {
      BEC_CUDA_TRY(cudaFuncSetAttribute(persist_pinv_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)std::max(job_smem(8, 9), job_smem(8, 8))));
      g_attr_set = true;
    }
  }
  persist_pinv_kernel<<<q.total, kPThreads, smem, st>>>(jobs_dev, q, ctr_dev);
  BEC_CUDA_TRY(cudaGetLastError());
  return BEC_OK;
}

}  // namespace bec

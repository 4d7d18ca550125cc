// Time pass of P_eps^{-1} (Sec. 4, eqs. ytild, blockdiaginv, zcompt), run in
// the sine basis where every B_k = lambda_k I + tau K is diagonal:
//   for each spatial mode q with FD eigenvalue mu_q, and its column w_j (j < N),
//     a_j = eps^{j/N} w_j                       (D_eps, Step 1)
//     A_k = sum_j a_j e^{-2 pi i jk/N}          (FFT along time, Step 1)
//     B_k = A_k / (lambda'_k + tau mu_q)        (Step 2; lambda'_k = 1 - eps^{1/N}
//                                                e^{-2 pi i k/N} is the eigenvalue that
//                                                pairs with this FFT sign)
//     z_j = eps^{-j/N} N^{-1} sum_k B_k e^{+2 pi i jk/N}   (Step 3)
// Two real modes share one complex FFT; their spectra are separated, divided
// and recombined for the pairs (k, N-k), k = 0..N/2, so only ceil((N+1)/2)
// distinct shifted solves are done (half-spectrum remark of Sec. 4).
#include <cuda_runtime.h>

#include "bec_fft.cuh"
#include "bec_internal.h"
#include "bec_passes.cuh"
#include "bec_tma.cuh"

#include <cudaTypedefs.h>

#include <atomic>

namespace bec {
namespace {

template <typename T>
constexpr int time_warps() { return default_time_warps(sizeof(T)); }

// rinv[q][k] = 1 / |lambda'_k + tau mu_q|^2 (same arithmetic as the division
// it replaces in time_pass_kernel)
__global__ void rinv_table_kernel(double* __restrict__ rinv, long long J, int NK, int m, int dim,
                                  const double2* __restrict__ lamf, ModeEigs<double> me,
                                  double tau) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= J * NK) return;
  const long long q = g / NK;
  const int k = (int)(g - q * NK);
  const double2 L = lamf[k];
  double muM, muK;
  mode_eigs(q, J, m, m, dim, me, muM, muK);
  const bool fe = me.m != nullptr;
  const double dr = fe ? fma(L.x, muM, tau * muK) : L.x + tau * muK, di = fe ? L.y * muM : L.y;
  rinv[g] = 1.0 / fma(dr, dr, di * di);
}

// data: [N][J] in place, rows of ld slots; a block owns W = 2 x warps
// adjacent modes (time_pass_tile).  registers: 128 per thread in FP64 and 64 in FP32 for
// N <= 256 (the block count the bound asks for fills the 64K-register
// file), free above.  FE: the mass eigenvalues are present (Q1 elements);
// finite differences (M = I) take the other instantiation, without the
// products by mu^M.
template <typename T, int LOGN, int WARPS, bool FE>
__global__ void __launch_bounds__(WARPS * 32, LOGN <= 8 ? (sizeof(T) == 8 ? 16 : 32) / WARPS : 1)
time_pass_kernel(T* __restrict__ data, long long J, int m, int ld, int dim,
                 const T* __restrict__ es,
                 const T* __restrict__ eis, const v2_t<T>* __restrict__ lamf,
                 ModeEigs<T> me, T tau, T scale_h, const double* __restrict__ scale_dev,
                 const v2_t<T>* __restrict__ tw, const double* __restrict__ rinv) {
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  time_pass_tile<T, LOGN, WARPS, FE>(data, J, m, ld, dim, es, eis, lamf, me, tau, scale_h, scale_dev,
                                     tw, rinv, blockIdx.x, smem_bytes, threadIdx.x);
}

template <typename T, int LOGN, int WARPS>
bec_status time_launch(bec_problem* p, void* data, double scale, const double* scale_dev,
                       const T* es, const T* eis, const v2_t<T>* lamf, ModeEigs<T> me,
                       const v2_t<T>* tw, const double* rinv) {
  constexpr int warps = WARPS;
  const size_t smem = (size_t)warps * 2 * line_slots(LOGN) * sizeof(T);
  auto k = me.m != nullptr ? time_pass_kernel<T, LOGN, WARPS, true>
                           : time_pass_kernel<T, LOGN, WARPS, false>;
  if (smem > 48 * 1024)
    BEC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // FP32 data is the preconditioner's scratch, in its layout
  const long long J = sizeof(T) == 4 ? p->Jp : p->J;
  const int ld = sizeof(T) == 4 ? p->ld : p->m;
  const long long W = 2 * warps;
  const unsigned grid = (unsigned)((J + W - 1) / W);
  BEC_LAUNCH_BEGIN(p);
  k<<<grid, warps * 32, smem, p->stream>>>(static_cast<T*>(data), J, p->m, ld, p->dim, es, eis,
                                           lamf, me, (T)p->tau, (T)scale, scale_dev, tw, rinv);
  BEC_LAUNCH_CHECK(p, "time_pass_kernel");
  return BEC_OK;
}

// FP32 time pass for N = 256 as a four-step FFT in registers
// (time_pass16_tile): 256 threads per block, 32 modes per block, the
// block's values loaded and stored by the threads.  128 registers a thread
// (two blocks per SM): the 16-point transforms and their twiddles keep many
// values live; a bound of 80 spilled and ran slower.
template <bool FE>
__global__ void __launch_bounds__(kT16Threads, 2)
time_pass16_kernel(float* __restrict__ data, long long J, int m, int ld, int dim,
                   const float* __restrict__ es, const float* __restrict__ eis,
                   const float2* __restrict__ lamf, ModeEigs<float> me, float tau, float scale_h,
                   const double* __restrict__ scale_dev, const float2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  time_pass16_tile<FE, false>(data, nullptr, J, m, ld, dim, es, eis, lamf, me, tau, scale_h,
                              scale_dev, tw, blockIdx.x, smem_bytes, threadIdx.x);
}

// The same pass with the tiles moved by TMA: each block copies the pass's
// tables to shared memory, then walks tiles blk, blk + grid, ...; while it transforms one tile in shared memory (stage b)
// the next one arrives in the other stage, and the results leave by a TMA
// store from the stage they were computed in.  Before a stage is refilled
// its store must have read it (bulk wait_group.read).  A wait for a tile
// that runs out (about 0.2 s) sets *err and ends the block.
constexpr size_t kT16StageBytes = (size_t)kT16Modes * 256 * sizeof(float);   // 32 KB
// tables copied to shared memory once per block: es, eis (256 floats each),
// tw (256 float2), lamf (129 float2)
constexpr size_t kT16TabBytes = 2 * 256 * sizeof(float) + (256 + 129) * sizeof(float2);
constexpr size_t kT16TmaSmem = 2 * kT16StageBytes + kT16Smem + 16 + kT16TabBytes;

template <bool FE>
__global__ void __launch_bounds__(kT16Threads, 2)
time_pass16_tma_kernel(const __grid_constant__ CUtensorMap map, long long J, int m, int ld,
                       int dim, const float* __restrict__ es, const float* __restrict__ eis,
                       const float2* __restrict__ lamf, ModeEigs<float> me, float tau,
                       float scale_h, const double* __restrict__ scale_dev,
                       const float2* __restrict__ tw, long long ntiles, int withhold,
                       int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char t16_smem[];
  float* const stage0 = reinterpret_cast<float*>(t16_smem);
  float* const stage1 = stage0 + kT16StageBytes / sizeof(float);
  unsigned char* const xbuf = t16_smem + 2 * kT16StageBytes;
  const uint32_t bar0 = tma_smem_u32(xbuf + kT16Smem), bar1 = bar0 + 8;
  float* const s_es = reinterpret_cast<float*>(xbuf + kT16Smem + 16);
  float* const s_eis = s_es + 256;
  float2* const s_tw = reinterpret_cast<float2*>(s_eis + 256);
  float2* const s_lam = s_tw + 256;
  const int tid = threadIdx.x;
  if (tid == 0) {
    tma_mbar_init(bar0, 1);
    tma_mbar_init(bar1, 1);
    tma_fence_mbar_init();
  }
  s_es[tid] = es[tid];
  s_eis[tid] = eis[tid];
  s_tw[tid] = tw[tid];
  if (tid <= 128) s_lam[tid] = lamf[tid];
  __syncthreads();
  long long t = blockIdx.x;
  if (tid == 0 && t < ntiles && !withhold) {
    tma_mbar_expect_tx(bar0, (uint32_t)kT16StageBytes);
    tma_load_2d(tma_smem_u32(stage0), &map, (int)(t * kT16Modes), 0, bar0);
  }
  int it = 0;
  bool ok = true;
  for (; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    float* const st = b ? stage1 : stage0;
    if (tid == 0 && t + gridDim.x < ntiles && !withhold) {   // prefetch the next tile
      tma_wait_group_read0();
      const uint32_t nb = b ? bar0 : bar1;
      tma_mbar_expect_tx(nb, (uint32_t)kT16StageBytes);
      tma_load_2d(tma_smem_u32(b ? stage0 : stage1), &map, (int)((t + gridDim.x) * kT16Modes), 0,
                  nb);
    }
    const bool got = tma_mbar_wait(b ? bar1 : bar0, (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    time_pass16_tile<FE, true>(nullptr, st, J, m, ld, dim, s_es, s_eis, s_lam, me, tau, scale_h,
                               scale_dev, s_tw, t, xbuf, tid);
    tma_fence_proxy_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_2d(&map, (int)(t * kT16Modes), 0, tma_smem_u32(st));
      tma_commit_group();
    }
  }
  if (tid == 0) {
    if (!ok) {
      atomicExch(err, 1);
      // the prefetch issued in the failed iteration may still be in flight
      if (t + gridDim.x < ntiles && !withhold) tma_mbar_wait(((it + 1) & 1) ? bar1 : bar0,
                                                (uint32_t)(((it + 1) >> 1) & 1));
    }
    tma_wait_group0();
  }
}

bec_status time16_launch(bec_problem* p, void* data, double scale, const double* scale_dev) {
  const PcTables& t = p->tab;
  const ModeEigs<float> me{t.mu32, t.mum32};
  const long long ntiles = (p->Jp + kT16Modes - 1) / kT16Modes;
  if (p->time_map_ok && data == p->pc_scratch) {
    auto k = me.m != nullptr ? time_pass16_tma_kernel<true> : time_pass16_tma_kernel<false>;
    static bool attr_set = false;
    if (!attr_set) {
      BEC_CUDA_TRY(cudaFuncSetAttribute(time_pass16_tma_kernel<true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kT16TmaSmem));
      BEC_CUDA_TRY(cudaFuncSetAttribute(time_pass16_tma_kernel<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kT16TmaSmem));
      attr_set = true;
    }
    int sms = 0;
    BEC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    const long long grid = ntiles < 2LL * sms ? ntiles : 2LL * sms;
    BEC_LAUNCH_BEGIN(p);
    k<<<(unsigned)grid, kT16Threads, kT16TmaSmem, p->stream>>>(
        p->time_map, p->Jp, p->m, p->ld, p->dim, t.es32, t.eis32, t.lamf32, me, (float)p->tau,
        (float)scale, scale_dev, t.time.tw32, ntiles, tma_take_withhold(), p->pc_err);
    BEC_LAUNCH_CHECK(p, "time_pass16_tma_kernel");
    return BEC_OK;
  }
  auto k = me.m != nullptr ? time_pass16_kernel<true> : time_pass16_kernel<false>;
  BEC_LAUNCH_BEGIN(p);
  k<<<(unsigned)ntiles, kT16Threads, kT16Smem, p->stream>>>(
      static_cast<float*>(data), p->Jp, p->m, p->ld, p->dim, t.es32, t.eis32, t.lamf32, me,
      (float)p->tau, (float)scale, scale_dev, t.time.tw32);
  BEC_LAUNCH_CHECK(p, "time_pass16_kernel");
  return BEC_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 time_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    else
      cudaGetLastError();
  }
  return fn;
}

// The block width w (warps per block) is tunable for N >= 32; shorter
// transforms always use the default.
template <typename T, int LOGN>
bec_status time_w(bec_problem* p, int w, void* data, double scale, const double* scale_dev,
                  const T* es, const T* eis, const v2_t<T>* lamf, ModeEigs<T> me,
                  const v2_t<T>* tw, const double* rinv) {
  if constexpr (LOGN >= 5) {
    if (w == 4) return time_launch<T, LOGN, 4>(p, data, scale, scale_dev, es, eis, lamf, me, tw, rinv);
    if (w == 8) return time_launch<T, LOGN, 8>(p, data, scale, scale_dev, es, eis, lamf, me, tw, rinv);
    if (w == 16) return time_launch<T, LOGN, 16>(p, data, scale, scale_dev, es, eis, lamf, me, tw, rinv);
  }
  return time_launch<T, LOGN, time_warps<T>()>(p, data, scale, scale_dev, es, eis, lamf, me, tw,
                                                rinv);
}

template <typename T>
bec_status time_dispatch(bec_problem* p, int w, void* data, double scale, const double* scale_dev,
                         const T* es, const T* eis, const v2_t<T>* lamf, ModeEigs<T> me,
                         const v2_t<T>* tw, const double* rinv) {
  switch (p->tab.time.logn) {
#define BEC_TIME_CASE(L) \
  case L: return time_w<T, L>(p, w, data, scale, scale_dev, es, eis, lamf, me, tw, rinv);
    BEC_TIME_CASE(1) BEC_TIME_CASE(2) BEC_TIME_CASE(3) BEC_TIME_CASE(4) BEC_TIME_CASE(5)
    BEC_TIME_CASE(6) BEC_TIME_CASE(7) BEC_TIME_CASE(8) BEC_TIME_CASE(9) BEC_TIME_CASE(10)
#undef BEC_TIME_CASE
    default: break;
  }
  set_error("unsupported number of time steps");
  return BEC_EUNSUPPORTED;
}

// Step 1 alone (multigrid route): for every spatial point q the half
// spectrum  S[k][q] = scale sum_j e^{-2 pi i jk/N} eps^{j/N} y[j][q],
// k = 0..N/2, written to HBM as [N/2+1][J] complex.  Two points share one
// complex FFT and are separated as (C_k + conj C_{N-k}) / 2 and
// (C_k - conj C_{N-k}) / (2i).
template <typename T, int LOGN>
__global__ void __launch_bounds__(time_warps<T>() * 32)
time_fwd_kernel(const double* __restrict__ y, v2_t<T>* __restrict__ spec, long long J,
                const T* __restrict__ es, T scale_h, const double* __restrict__ scale_dev,
                const v2_t<T>* __restrict__ tw) {
  using V = v2_t<T>;
  constexpr int N = 1 << LOGN;
  constexpr int LSC = line_slots(LOGN);
  constexpr int WARPS = time_warps<T>();
  constexpr int W = 2 * WARPS;
  constexpr int NK = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  T* sm = reinterpret_cast<T*>(smem_bytes);
  V* out = reinterpret_cast<V*>(sm + (size_t)WARPS * 2 * LSC);   // [NK][W]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long q0 = (long long)blockIdx.x * W;
  const T scale = scale_dev ? (T)((double)scale_h * scale_dev[0]) : scale_h;
#pragma unroll 4
  for (int e = threadIdx.x; e < N * W; e += WARPS * 32) {
    const int j = e / W, c = e % W;
    const long long q = q0 + c;
    sm[(c >> 1) * 2 * LSC + 2 * j + (c & 1)] = q < J ? convert<T>(y[(long long)j * J + q]) * es[j] : T(0);
  }
  __syncthreads();
  V* line = reinterpret_cast<V*>(sm + (size_t)warp * 2 * LSC);
  warp_fft<T, -1, LOGN>(line, tw, lane);
  const T half = scale * T(0.5);
  for (int k = lane; k < NK; k += 32) {
    const V C = line[k], Cn = line[(N - k) & (N - 1)];
    out[k * W + 2 * warp] = {(C.x + Cn.x) * half, (C.y - Cn.y) * half};
    out[k * W + 2 * warp + 1] = {(C.y + Cn.y) * half, (Cn.x - C.x) * half};
  }
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.x; e < NK * W; e += WARPS * 32) {
    const int k = e / W, c = e % W;
    const long long q = q0 + c;
    if (q < J) spec[(long long)k * J + q] = out[e];
  }
}

// Step 3 alone (multigrid route): z[j][q] = scale eps^{-j/N} sum_k Z_k
// e^{+2 pi i jk/N} with Z_{N-k} = conj(Z_k), from the half spectrum; the
// imaginary parts of Z_0 and Z_{N/2} are ignored (complex-to-real inverse).
template <typename T, int LOGN>
__global__ void __launch_bounds__(time_warps<T>() * 32)
time_inv_kernel(const v2_t<T>* __restrict__ spec, double* __restrict__ z, long long J,
                const T* __restrict__ eis, T scale, const v2_t<T>* __restrict__ tw) {
  using V = v2_t<T>;
  constexpr int N = 1 << LOGN;
  constexpr int LSC = line_slots(LOGN);
  constexpr int WARPS = time_warps<T>();
  constexpr int W = 2 * WARPS;
  constexpr int NK = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  T* sm = reinterpret_cast<T*>(smem_bytes);
  V* in = reinterpret_cast<V*>(sm + (size_t)WARPS * 2 * LSC);    // [NK][W]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long q0 = (long long)blockIdx.x * W;
#pragma unroll 4
  for (int e = threadIdx.x; e < NK * W; e += WARPS * 32) {
    const int k = e / W, c = e % W;
    const long long q = q0 + c;
    in[e] = q < J ? spec[(long long)k * J + q] : V{0, 0};
  }
  __syncthreads();
  V* line = reinterpret_cast<V*>(sm + (size_t)warp * 2 * LSC);
  for (int k = lane; k < NK; k += 32) {
    const V A = in[k * W + 2 * warp], B = in[k * W + 2 * warp + 1];
    if (k > 0 && k < N / 2) {
      line[k] = {A.x - B.y, A.y + B.x};                  // A + i B
      line[N - k] = {A.x + B.y, B.x - A.y};              // conj(A) + i conj(B)
    } else {
      // k = 0 and N/2 of a real signal are real: their imaginary parts are
      // dropped (a complex-to-real inverse), not mixed into the other line
      line[k] = {A.x, B.x};
    }
  }
  __syncwarp();
  warp_fft<T, +1, LOGN>(line, tw, lane);
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.x; e < N * W; e += WARPS * 32) {
    const int j = e / W, c = e % W;
    const long long q = q0 + c;
    if (q < J)
      z[(long long)j * J + q] = convert<double>(sm[(c >> 1) * 2 * LSC + 2 * j + (c & 1)] * eis[j] * scale);
  }
}

template <typename T, int LOGN>
bec_status time_fwd_launch(bec_problem* p, const double* y, void* spec, double scale,
                           const double* scale_dev, const T* es, const v2_t<T>* tw) {
  constexpr int N = 1 << LOGN;
  constexpr int warps = time_warps<T>();
  const size_t smem = (size_t)warps * 2 * line_slots(LOGN) * sizeof(T) +
                      (size_t)(N / 2 + 1) * 2 * warps * sizeof(v2_t<T>);
  auto k = time_fwd_kernel<T, LOGN>;
  if (smem > 48 * 1024)
    BEC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long W = 2 * warps;
  BEC_LAUNCH_BEGIN(p);
  k<<<(unsigned)((p->J + W - 1) / W), warps * 32, smem, p->stream>>>(
      y, static_cast<v2_t<T>*>(spec), p->J, es, (T)scale, scale_dev, tw);
  BEC_LAUNCH_CHECK(p, "time_fwd_kernel");
  return BEC_OK;
}

template <typename T, int LOGN>
bec_status time_inv_launch(bec_problem* p, const void* spec, double* z, double scale,
                           const T* eis, const v2_t<T>* tw) {
  constexpr int N = 1 << LOGN;
  constexpr int warps = time_warps<T>();
  const size_t smem = (size_t)warps * 2 * line_slots(LOGN) * sizeof(T) +
                      (size_t)(N / 2 + 1) * 2 * warps * sizeof(v2_t<T>);
  auto k = time_inv_kernel<T, LOGN>;
  if (smem > 48 * 1024)
    BEC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long W = 2 * warps;
  BEC_LAUNCH_BEGIN(p);
  k<<<(unsigned)((p->J + W - 1) / W), warps * 32, smem, p->stream>>>(
      static_cast<const v2_t<T>*>(spec), z, p->J, eis, (T)scale, tw);
  BEC_LAUNCH_CHECK(p, "time_inv_kernel");
  return BEC_OK;
}

#define BEC_TIME_SWITCH(logn, CALL)                                                    \
  switch (logn) {                                                                     \
    case 1: return CALL(1);                                                           \
    case 2: return CALL(2);                                                           \
    case 3: return CALL(3);                                                           \
    case 4: return CALL(4);                                                           \
    case 5: return CALL(5);                                                           \
    case 6: return CALL(6);                                                           \
    case 7: return CALL(7);                                                           \
    case 8: return CALL(8);                                                           \
    case 9: return CALL(9);                                                           \
    default: break;                                                                   \
  }

}  // namespace

bec_status launch_time_fwd(bec_problem* p, const double* y, void* spec, int fp64,
                           const double* scale_dev) {
  const PcTables& t = p->tab;
  if (fp64) {
#define BEC_FWD64(L) time_fwd_launch<double, L>(p, y, spec, 1.0, scale_dev, t.es64, t.time.tw64)
    BEC_TIME_SWITCH(t.time.logn, BEC_FWD64)
#undef BEC_FWD64
  } else {
#define BEC_FWD32(L) time_fwd_launch<float, L>(p, y, spec, 1.0, scale_dev, t.es32, t.time.tw32)
    BEC_TIME_SWITCH(t.time.logn, BEC_FWD32)
#undef BEC_FWD32
  }
  set_error("the multigrid route supports N <= 512");
  return BEC_EUNSUPPORTED;
}

bec_status launch_time_inv(bec_problem* p, const void* spec, double* z, int fp64) {
  const PcTables& t = p->tab;
  const double scale = 1.0 / p->N;
  if (fp64) {
#define BEC_INV64(L) time_inv_launch<double, L>(p, spec, z, scale, t.eis64, t.time.tw64)
    BEC_TIME_SWITCH(t.time.logn, BEC_INV64)
#undef BEC_INV64
  } else {
#define BEC_INV32(L) time_inv_launch<float, L>(p, spec, z, scale, t.eis32, t.time.tw32)
    BEC_TIME_SWITCH(t.time.logn, BEC_INV32)
#undef BEC_INV32
  }
  set_error("the multigrid route supports N <= 512");
  return BEC_EUNSUPPORTED;
}

bec_status launch_time_pass_w(bec_problem* p, void* data, int fp64, double scale,
                              const double* scale_dev, int w) {
  const PcTables& t = p->tab;
  if (fp64)
    return time_dispatch<double>(p, w, data, scale, scale_dev, t.es64, t.eis64, t.lamf64,
                                 ModeEigs<double>{t.mu64, t.mum64}, t.time.tw64, t.rinv64);
  if (time16_applies(p)) return time16_launch(p, data, scale, scale_dev);
  return time_dispatch<float>(p, w, data, scale, scale_dev, t.es32, t.eis32, t.lamf32,
                              ModeEigs<float>{t.mu32, t.mum32}, t.time.tw32, nullptr);
}

bool time16_applies(const bec_problem* p) {
  return p->desc.precision == BEC_PC_FP32 && p->tab.time.logn == 8;
}

bec_status time16_make_map(bec_problem* p) {
  p->time_map_ok = false;
  // a TMA tile needs 16-byte aligned time slices (Jp a multiple of 4 floats)
  if (!time16_applies(p) || p->pc_scratch == nullptr || p->Jp % 4 != 0) return BEC_OK;
  auto fn = time_encode_fn();
  if (fn == nullptr) return BEC_OK;              // the per-thread-load kernel runs instead
  const cuuint64_t dims[2] = {(cuuint64_t)p->Jp, (cuuint64_t)p->N};
  const cuuint64_t strides[1] = {(cuuint64_t)p->Jp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kT16Modes, 256};
  const cuuint32_t es[2] = {1, 1};
  if (fn(&p->time_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->pc_scratch, dims, strides, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (time pass)");
    return BEC_ECUDA;
  }
  p->time_map_ok = true;
  return BEC_OK;
}

namespace {
std::atomic<int> g_withhold_tma{0};   // set by bec_inject_fault, taken by the next launch
}  // namespace

void tma_withhold_next() { g_withhold_tma.store(1); }
int tma_take_withhold() { return g_withhold_tma.exchange(0); }

bec_status pc_check(bec_problem* p) {
  if (p->pc_err == nullptr) return BEC_OK;
  int v = 0;
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  BEC_CUDA_TRY(cudaMemcpy(&v, p->pc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v == 0) return BEC_OK;
  BEC_CUDA_TRY(cudaMemset(p->pc_err, 0, sizeof(int)));
  set_error("a bounded wait for a time-pass tile ran out");
  return BEC_ETIMEOUT;
}

bec_status launch_time_pass(bec_problem* p, void* data, int fp64, double scale,
                            const double* scale_dev) {
  return launch_time_pass_w(p, data, fp64, scale, scale_dev, p->tile.time);
}

bec_status launch_rinv_table(bec_problem* p) {
  const long long total = p->J * (long long)(p->N / 2 + 1);
  BEC_LAUNCH_BEGIN(p);
  rinv_table_kernel<<<(unsigned)((total + 255) / 256), 256, 0, p->stream>>>(
      p->tab.rinv64, p->J, p->N / 2 + 1, p->m, p->dim, p->tab.lamf64,
      ModeEigs<double>{p->tab.mu64, p->tab.mum64}, p->tau);
  BEC_LAUNCH_CHECK(p, "rinv_table_kernel");
  return BEC_OK;
}

}  // namespace bec

// Spatial sine-transform passes of P_eps^{-1} (Sec. 4: the shifted systems
// B_k = lambda_k I + tau K are diagonalised by the 2D DST-I when a is constant
// on a uniform grid).  Both passes compute 4 x the unnormalised DST-I; the
// normalisation is folded into the divide of the time pass.
#include <cuda_runtime.h>

#include "bec_fft.cuh"
#include "bec_internal.h"

namespace bec {
namespace {

template <typename T>
constexpr int rows_warps() { return 8; }
template <typename T>
constexpr int cols_warps() { return sizeof(T) == 8 ? 8 : 16; }

// DST along x: one warp per pair of contiguous rows of length m = n - 1.
// `in` and `out` may be the same array (each warp reads its rows before
// writing them); in that case TI == TO.
template <typename T, typename TI, typename TO, int LOGN>
__global__ void __launch_bounds__(rows_warps<T>() * 32)
dst_rows_kernel(const TI* in, TO* out, long long rows, int m, const T* __restrict__ sin2,
                const v2_t<T>* __restrict__ tw) {
  constexpr int n = 1 << LOGN;
  constexpr int LSC = line_slots(LOGN);      // complex slots per line
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  T* sm = reinterpret_cast<T*>(smem_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* raw = sm + (size_t)warp * 2 * LSC;
  const long long r0 = 2 * ((long long)blockIdx.x * rows_warps<T>() + warp);
  if (r0 >= rows) return;                    // whole warp leaves; no block barrier below
  const bool hasb = r0 + 1 < rows;
  const TI* ia = in + r0 * m;
  for (int j = lane; j < m; j += 32) {
    raw[j] = (T)ia[j];
    raw[LSC + j] = hasb ? (T)ia[m + j] : T(0);
  }
  __syncwarp();
  warp_dst_pair<T, LOGN>(raw, LSC, sin2, tw, lane);
  TO* oa = out + r0 * m;
  for (int j = lane; j < m; j += 32) {
    oa[j] = (TO)raw[j];
    if (hasb) oa[m + j] = (TO)raw[LSC + j];
  }
}

// DST along y, in place, for every slice of `nslices` [m][m] slices: a block
// owns W = 2 x warps adjacent columns of one slice; the tile is loaded and
// stored with coalesced row segments, each warp transforms one column pair.
template <typename T, int LOGN>
__global__ void __launch_bounds__(cols_warps<T>() * 32)
dst_cols_kernel(T* data, int m, long long J, const T* __restrict__ sin2,
                const v2_t<T>* __restrict__ tw) {
  constexpr int n = 1 << LOGN;
  constexpr int LSC = line_slots(LOGN);
  constexpr int WARPS = cols_warps<T>();
  constexpr int W = 2 * WARPS;
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  T* sm = reinterpret_cast<T*>(smem_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x0 = blockIdx.x * W;
  T* base = data + (long long)blockIdx.y * J;
  const int total = m * W;
  for (int e = threadIdx.x; e < total; e += WARPS * 32) {
    const int j = e / W, c = e % W;
    const int x = x0 + c;
    sm[c * LSC + j] = x < m ? base[(long long)j * m + x] : T(0);
  }
  __syncthreads();
  warp_dst_pair<T, LOGN>(sm + (size_t)warp * 2 * LSC, LSC, sin2, tw, lane);
  __syncthreads();
  for (int e = threadIdx.x; e < total; e += WARPS * 32) {
    const int j = e / W, c = e % W;
    const int x = x0 + c;
    if (x < m) base[(long long)j * m + x] = sm[c * LSC + j];
  }
}

template <typename Kern>
cudaError_t prepare(Kern k, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <typename T, typename TI, typename TO, int LOGN>
bec_status rows_launch(bec_problem* p, const void* in, void* out, long long rows,
                       const T* sin2, const v2_t<T>* tw) {
  constexpr int n = 1 << LOGN;
  const int warps = rows_warps<T>();
  const size_t smem = (size_t)warps * 2 * line_slots(LOGN) * sizeof(T);
  auto k = dst_rows_kernel<T, TI, TO, LOGN>;
  BEC_CUDA_TRY(prepare(k, smem));
  const long long pairs = (rows + 1) / 2;
  const unsigned grid = (unsigned)((pairs + warps - 1) / warps);
  BEC_LAUNCH_BEGIN(p);
  k<<<grid, warps * 32, smem, p->stream>>>(static_cast<const TI*>(in), static_cast<TO*>(out), rows,
                                           p->m, sin2, tw);
  BEC_LAUNCH_CHECK(p, "dst_rows_kernel");
  return BEC_OK;
}

template <typename T, int LOGN>
bec_status cols_launch(bec_problem* p, void* data, const T* sin2, const v2_t<T>* tw) {
  constexpr int n = 1 << LOGN;
  constexpr int warps = cols_warps<T>();
  const size_t smem = (size_t)warps * 2 * line_slots(LOGN) * sizeof(T);
  auto k = dst_cols_kernel<T, LOGN>;
  BEC_CUDA_TRY(prepare(k, smem));
  dim3 grid((unsigned)((p->m + 2 * warps - 1) / (2 * warps)), (unsigned)p->N);
  BEC_LAUNCH_BEGIN(p);
  k<<<grid, warps * 32, smem, p->stream>>>(static_cast<T*>(data), p->m, p->J, sin2, tw);
  BEC_LAUNCH_CHECK(p, "dst_cols_kernel");
  return BEC_OK;
}

#define BEC_LOGN_SWITCH(logn, CALL)         \
  switch (logn) {                           \
    case 2: return CALL(2);                 \
    case 3: return CALL(3);                 \
    case 4: return CALL(4);                 \
    case 5: return CALL(5);                 \
    case 6: return CALL(6);                 \
    case 7: return CALL(7);                 \
    case 8: return CALL(8);                 \
    case 9: return CALL(9);                 \
    case 10: return CALL(10);               \
    default: break;                         \
  }

template <typename T, typename TI, typename TO>
bec_status rows_dispatch(bec_problem* p, const void* in, void* out, long long rows,
                         const T* sin2, const v2_t<T>* tw) {
#define BEC_ROWS_CALL(L) rows_launch<T, TI, TO, L>(p, in, out, rows, sin2, tw)
  BEC_LOGN_SWITCH(p->tab.space.logn, BEC_ROWS_CALL)
#undef BEC_ROWS_CALL
  set_error("unsupported spatial transform length");
  return BEC_EUNSUPPORTED;
}

template <typename T>
bec_status cols_dispatch(bec_problem* p, void* data, const T* sin2, const v2_t<T>* tw) {
#define BEC_COLS_CALL(L) cols_launch<T, L>(p, data, sin2, tw)
  BEC_LOGN_SWITCH(p->tab.space.logn, BEC_COLS_CALL)
#undef BEC_COLS_CALL
  set_error("unsupported spatial transform length");
  return BEC_EUNSUPPORTED;
}

}  // namespace

bec_status launch_dst_rows(bec_problem* p, const void* in, int in_fp64, void* out, int out_fp64,
                           long long rows, int fp64) {
  if (fp64) {
    if (!in_fp64 || !out_fp64) return BEC_EINVAL;
    return rows_dispatch<double, double, double>(p, in, out, rows, p->tab.sin2_64,
                                                 p->tab.space.tw64);
  }
  const float* s = p->tab.sin2_32;
  const float2* tw = p->tab.space.tw32;
  if (in_fp64 && !out_fp64) return rows_dispatch<float, double, float>(p, in, out, rows, s, tw);
  if (!in_fp64 && out_fp64) return rows_dispatch<float, float, double>(p, in, out, rows, s, tw);
  if (!in_fp64 && !out_fp64) return rows_dispatch<float, float, float>(p, in, out, rows, s, tw);
  set_error("FP32 row pass needs a float input or a float output");
  return BEC_EINVAL;
}

bec_status launch_dst_cols(bec_problem* p, void* data, int fp64) {
  if (fp64) return cols_dispatch<double>(p, data, p->tab.sin2_64, p->tab.space.tw64);
  return cols_dispatch<float>(p, data, p->tab.sin2_32, p->tab.space.tw32);
}

}  // namespace bec

// Spatial sine-transform passes of P_eps^{-1} (Sec. 4: the shifted systems
// B_k = lambda_k I + tau K are diagonalised by the 2D DST-I when a is constant
// on a uniform grid).  Both passes compute 4 x the unnormalised DST-I; the
// normalisation is folded into the divide of the time pass.
#include <cuda_runtime.h>

#include "bec_fft.cuh"
#include "bec_internal.h"
#include "bec_passes.cuh"
#include "bec_tma.cuh"

#include <cudaTypedefs.h>

namespace bec {
namespace {


// Blocks per SM that the register bound of dst_rows_kernel asks for, as warps
// per SM over the block's warps (at least one block): in FP64 32 warps for
// n <= 256 (64 registers) and 16 for n = 512; in FP32 40 warps for n <= 256,
// 32 for n = 512 and 16 above; longer FP64 transforms are left free.
__host__ __device__ constexpr int rows_min_blocks(int bytes, int logn, int warps) {
  const int w = bytes == 8 ? (logn <= 8 ? 32 : logn == 9 ? 16 : warps)
                           : (logn <= 8 ? 40 : logn == 9 ? 32 : 16);
  return w / warps > 0 ? w / warps : 1;
}

// DST along x: one warp per pair of contiguous rows of length m = n - 1
// (dst_rows_tile, one tile per block).  `in` and `out` may be the same array;
// in that case TI == TO.
template <typename T, typename TI, typename TO, int LOGN, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, rows_min_blocks(sizeof(T), LOGN, WARPS))
dst_rows_kernel(const TI* in, TO* out, long long rows, int m, int in_ld, int out_ld,
                const T* __restrict__ sin2, const v2_t<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  dst_rows_tile<T, TI, TO, LOGN, WARPS>(in, out, rows, m, in_ld, out_ld, sin2, tw, blockIdx.x,
                                        smem_bytes, threadIdx.x);
}

// Blocks per SM that the register bound of dst_cols_kernel asks for, as warps
// per SM over the block's warps (at least one block): for n <= 256, 40 warps
// in FP32 (48 registers a thread) and 24 in FP64 (80 registers); for n = 512,
// 16 warps in FP32; longer transforms are left free.
__host__ __device__ constexpr int cols_min_blocks(int bytes, int logn, int warps) {
  return (bytes == 4 ? (logn <= 8 ? 40 : logn == 9 ? 16 : warps) : (logn <= 8 ? 24 : warps)) / warps;
}

// DST along the rows of every slice, in place: slice s (s < nslices, at
// data + s * slice_stride) holds m rows of ncols values, row j at j *
// row_stride, and the transform runs down each column (along j); a block
// owns W = 2 x warps adjacent columns (dst_cols_tile) and walks the slices.
// 2D: the y-DST of [ny][nx] slices; 3D: the y-DST of every [ny][nx] plane
// and the z-DST of [nz][ny nx] slices.
template <typename T, int LOGN, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, cols_min_blocks(sizeof(T), LOGN, WARPS))
dst_cols_kernel(T* data, int m, int ncols, long long row_stride, long long slice_stride,
                long long nslices, const T* __restrict__ sin2, const v2_t<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  for (long long sl = blockIdx.y; sl < nslices; sl += gridDim.y)
    dst_cols_tile<T, LOGN, WARPS>(data, m, ncols, row_stride, slice_stride, blockIdx.x, sl, sin2,
                                  tw, smem_bytes, threadIdx.x);
}

// FP32 y-DST for n = 256 (2D) on the four-step tile (dst16_cols_core), the
// tiles moved by TMA, with an exchange buffer of its own (four block
// barriers per tile instead of six): each block copies sin2 and the
// twiddles to shared memory, then walks tiles blk, blk + grid, ... (tile t:
// columns 32 (t mod tiles_x) .. + 31 of slice t / tiles_x), transforming one
// in its shared-memory stage while the next arrives in the other stage;
// results leave by a TMA store from the stage they were computed in, which
// is refilled only after the store has read it.  A wait that runs out
// (about 0.2 s) sets *err and ends the block.
// sin2 (256 floats) and tw (256 float2) copied to shared memory once per block
constexpr size_t kD16TabBytes = 256 * sizeof(float) + 256 * sizeof(float2);
constexpr size_t kD16XBytes = 16 * 256 * sizeof(float2);   // the exchange buffer (32 KB)
constexpr size_t kD16TmaSmem = 2 * kD16StageBytes + kD16TotBytes + 16 + kD16TabBytes + kD16XBytes;

__global__ void __launch_bounds__(kD16Threads, 2)
dst_cols16_tma_kernel(const __grid_constant__ CUtensorMap map, const float* __restrict__ sin2,
                      const float2* __restrict__ tw, int tiles_x, long long ntiles,
                      uint32_t tile_bytes, int withhold, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char d16_smem[];
  float* const stage0 = reinterpret_cast<float*>(d16_smem);
  float* const stage1 = stage0 + kD16StageBytes / sizeof(float);
  float2* const tot = reinterpret_cast<float2*>(d16_smem + 2 * kD16StageBytes);
  const uint32_t bar0 = tma_smem_u32(d16_smem + 2 * kD16StageBytes + kD16TotBytes), bar1 = bar0 + 8;
  float* const s_sin2 = reinterpret_cast<float*>(d16_smem + 2 * kD16StageBytes + kD16TotBytes + 16);
  float2* const s_tw = reinterpret_cast<float2*>(s_sin2 + 256);
  float2* const xbuf = s_tw + 256;
  const int tid = threadIdx.x;
  if (tid == 0) {
    tma_mbar_init(bar0, 1);
    tma_mbar_init(bar1, 1);
    tma_fence_mbar_init();
  }
  s_sin2[tid] = sin2[tid];
  s_tw[tid] = tw[tid];
  __syncthreads();
  long long t = blockIdx.x;
  if (tid == 0 && t < ntiles && !withhold) {
    tma_mbar_expect_tx(bar0, tile_bytes);
    tma_load_3d(tma_smem_u32(stage0), &map, (int)(t % tiles_x) * kD16Cols, 0, (int)(t / tiles_x),
                bar0);
  }
  int it = 0;
  bool ok = true;
  for (; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    float* const st = b ? stage1 : stage0;
    const long long tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles && !withhold) {    // prefetch the next tile into the other stage
      tma_wait_group_read0();
      const uint32_t nb = b ? bar0 : bar1;
      tma_mbar_expect_tx(nb, tile_bytes);
      tma_load_3d(tma_smem_u32(b ? stage0 : stage1), &map, (int)(tn % tiles_x) * kD16Cols, 0,
                  (int)(tn / tiles_x), nb);
    }
    const bool got = tma_mbar_wait(b ? bar1 : bar0, (uint32_t)((it >> 1) & 1));
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    dst16_cols_core(st, xbuf, tot, s_sin2, s_tw, tid);
    tma_fence_proxy_smem();
    __syncthreads();
    if (tid == 0) {
      tma_store_3d(&map, (int)(t % tiles_x) * kD16Cols, 0, (int)(t / tiles_x), tma_smem_u32(st));
      tma_commit_group();
    }
  }
  if (tid == 0) {
    if (!ok) {
      atomicExch(err, 1);
      if (t + gridDim.x < ntiles && !withhold) tma_mbar_wait(((it + 1) & 1) ? bar1 : bar0,
                                                (uint32_t)(((it + 1) >> 1) & 1));
    }
    tma_wait_group0();
  }
}

bec_status cols16_launch(bec_problem* p) {
  static bool attr_set = false;
  if (!attr_set) {
    BEC_CUDA_TRY(cudaFuncSetAttribute(dst_cols16_tma_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kD16TmaSmem));
    attr_set = true;
  }
  const int tiles_x = (p->ld + kD16Cols - 1) / kD16Cols;
  const long long ntiles = (long long)tiles_x * p->N;
  int sms = 0;
  BEC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  const long long grid = ntiles < 2LL * sms ? ntiles : 2LL * sms;
  const uint32_t tile_bytes = (uint32_t)(kD16Cols * p->m * sizeof(float));
  BEC_LAUNCH_BEGIN(p);
  dst_cols16_tma_kernel<<<(unsigned)grid, kD16Threads, kD16TmaSmem, p->stream>>>(
      p->cols_map, p->tab.sin2_32, p->tab.space.tw32, tiles_x, ntiles, tile_bytes,
      tma_take_withhold(), p->pc_err);
  BEC_LAUNCH_CHECK(p, "dst_cols16_tma_kernel");
  return BEC_OK;
}

template <typename Kern>
cudaError_t prepare(Kern k, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <typename T, typename TI, typename TO, int LOGN, int WARPS>
bec_status rows_launch(bec_problem* p, const void* in, void* out, long long rows,
                       const T* sin2, const v2_t<T>* tw) {
  const size_t smem = (size_t)WARPS * 2 * dst_line_stride(LOGN, sizeof(T)) * sizeof(T);
  auto k = dst_rows_kernel<T, TI, TO, LOGN, WARPS>;
  BEC_CUDA_TRY(prepare(k, smem));
  const long long pairs = (rows + 1) / 2;
  const unsigned grid = (unsigned)((pairs + WARPS - 1) / WARPS);
  // FP32 arrays are the preconditioner's scratch, in its layout (rows of ld)
  const int in_ld = sizeof(TI) == 4 ? p->ld : p->m, out_ld = sizeof(TO) == 4 ? p->ld : p->m;
  BEC_LAUNCH_BEGIN(p);
  k<<<grid, WARPS * 32, smem, p->stream>>>(static_cast<const TI*>(in), static_cast<TO*>(out), rows,
                                           p->m, in_ld, out_ld, sin2, tw);
  BEC_LAUNCH_CHECK(p, "dst_rows_kernel");
  return BEC_OK;
}

template <typename T, int LOGN, int WARPS>
bec_status cols_launch(bec_problem* p, void* data, const T* sin2, const v2_t<T>* tw) {
  const size_t smem = (size_t)WARPS * 2 * dst_line_stride(LOGN, sizeof(T)) * sizeof(T);
  auto k = dst_cols_kernel<T, LOGN, WARPS>;
  BEC_CUDA_TRY(prepare(k, smem));
  // FP32 data is the preconditioner's scratch: rows of ld slots
  const long long m = p->m, ld = sizeof(T) == 4 ? p->ld : p->m, m2 = m * ld;
  const long long J = sizeof(T) == 4 ? p->Jp : p->J;
  // 2D: y over [ny][nx] slices; 3D: y over every [ny][nx] plane, then z over
  // [nz][ny nx] slices (a plane's pad slots are zeros and stay zeros)
  const int passes = p->dim == 3 ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    const bool zpass = pass == 1;
    const int ncols = (int)(zpass ? m2 : m);
    const long long row_stride = zpass ? m2 : ld;
    const long long slice_stride = zpass ? J : m2;
    const long long nslices = zpass ? (long long)p->N : (long long)p->N * (p->dim == 3 ? m : 1);
    dim3 grid((unsigned)((ncols + 2 * WARPS - 1) / (2 * WARPS)),
              (unsigned)(nslices < 65535 ? nslices : 65535));
    BEC_LAUNCH_BEGIN(p);
    k<<<grid, WARPS * 32, smem, p->stream>>>(static_cast<T*>(data), p->m, ncols, row_stride,
                                             slice_stride, nslices, sin2, tw);
    BEC_LAUNCH_CHECK(p, "dst_cols_kernel");
  }
  return BEC_OK;
}

// The block width w (warps per block) is tunable for n >= 32; shorter
// transforms always use the default.
template <typename T, typename TI, typename TO, int LOGN>
bec_status rows_w(bec_problem* p, int w, const void* in, void* out, long long rows, const T* sin2,
                  const v2_t<T>* tw) {
  if constexpr (LOGN >= 5) {
    if (w == 4) return rows_launch<T, TI, TO, LOGN, 4>(p, in, out, rows, sin2, tw);
    if (w == 16) return rows_launch<T, TI, TO, LOGN, 16>(p, in, out, rows, sin2, tw);
  }
  return rows_launch<T, TI, TO, LOGN, kRowsWarps>(p, in, out, rows, sin2, tw);
}

template <typename T, int LOGN>
bec_status cols_w(bec_problem* p, int w, void* data, const T* sin2, const v2_t<T>* tw) {
  if constexpr (LOGN >= 5) {
    if (w == 4) return cols_launch<T, LOGN, 4>(p, data, sin2, tw);
    if (w == 8) return cols_launch<T, LOGN, 8>(p, data, sin2, tw);
    if (w == 16) return cols_launch<T, LOGN, 16>(p, data, sin2, tw);
  }
  return cols_launch<T, LOGN, default_cols_warps(sizeof(T))>(p, data, sin2, tw);
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
bec_status rows_dispatch(bec_problem* p, int w, const void* in, void* out, long long rows,
                         const T* sin2, const v2_t<T>* tw) {
#define BEC_ROWS_CALL(L) rows_w<T, TI, TO, L>(p, w, in, out, rows, sin2, tw)
  BEC_LOGN_SWITCH(p->tab.space.logn, BEC_ROWS_CALL)
#undef BEC_ROWS_CALL
  set_error("unsupported spatial transform length");
  return BEC_EUNSUPPORTED;
}

template <typename T>
bec_status cols_dispatch(bec_problem* p, int w, void* data, const T* sin2, const v2_t<T>* tw) {
#define BEC_COLS_CALL(L) cols_w<T, L>(p, w, data, sin2, tw)
  BEC_LOGN_SWITCH(p->tab.space.logn, BEC_COLS_CALL)
#undef BEC_COLS_CALL
  set_error("unsupported spatial transform length");
  return BEC_EUNSUPPORTED;
}

__global__ void convert_kernel_f32(const double* __restrict__ x, float* __restrict__ y, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) y[g] = f64_to_f32(x[g]);
}

__global__ void convert_kernel_f64(const float* __restrict__ x, double* __restrict__ y, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) y[g] = f32_to_f64(x[g]);
}

}  // namespace

__global__ void rcp64_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) y[g] = rcp64(x[g]);
}

cudaError_t launch_rcp64(const double* x, double* y, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  rcp64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* x, void* y, long long n, int to_float, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (to_float)
    convert_kernel_f32<<<grid, 256, 0, st>>>(static_cast<const double*>(x), static_cast<float*>(y), n);
  else
    convert_kernel_f64<<<grid, 256, 0, st>>>(static_cast<const float*>(x), static_cast<double*>(y), n);
  return cudaGetLastError();
}

bec_status launch_dst_rows_w(bec_problem* p, const void* in, int in_fp64, void* out, int out_fp64,
                             long long rows, int fp64, int w) {
  if (fp64) {
    if (!in_fp64 || !out_fp64) return BEC_EINVAL;
    return rows_dispatch<double, double, double>(p, w, in, out, rows, p->tab.sin2_64,
                                                 p->tab.space.tw64);
  }
  const float* s = p->tab.sin2_32;
  const float2* tw = p->tab.space.tw32;
  if (in_fp64 && !out_fp64) return rows_dispatch<float, double, float>(p, w, in, out, rows, s, tw);
  if (!in_fp64 && out_fp64) return rows_dispatch<float, float, double>(p, w, in, out, rows, s, tw);
  if (!in_fp64 && !out_fp64) return rows_dispatch<float, float, float>(p, w, in, out, rows, s, tw);
  set_error("FP32 row pass needs a float input or a float output");
  return BEC_EINVAL;
}

bool cols16_applies(const bec_problem* p) {
  return p->desc.precision == BEC_PC_FP32 && p->dim == 2 && p->tab.space.logn == 8 &&
         p->cols_map_ok;
}

bec_status cols16_make_map(bec_problem* p) {
  p->cols_map_ok = false;
  if (p->desc.precision != BEC_PC_FP32 || p->dim != 2 || p->tab.space.logn != 8 ||
      p->pc_scratch == nullptr || p->ld % 4 != 0)
    return BEC_OK;
  void* ptr = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return BEC_OK;                                  // the per-warp column kernel runs instead
  }
  auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  // the scratch as [N][m][ld] floats; a box is 32 columns of one slice
  const cuuint64_t dims[3] = {(cuuint64_t)p->ld, (cuuint64_t)p->m, (cuuint64_t)p->N};
  const cuuint64_t strides[2] = {(cuuint64_t)p->ld * sizeof(float),
                                 (cuuint64_t)p->ld * p->m * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)kD16Cols, (cuuint32_t)p->m, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  if (fn(&p->cols_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p->pc_scratch, dims, strides, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (column pass)");
    return BEC_ECUDA;
  }
  p->cols_map_ok = true;
  return BEC_OK;
}

bec_status launch_dst_cols_w(bec_problem* p, void* data, int fp64, int w) {
  if (!fp64 && data == p->pc_scratch && cols16_applies(p)) return cols16_launch(p);
  if (fp64) return cols_dispatch<double>(p, w, data, p->tab.sin2_64, p->tab.space.tw64);
  return cols_dispatch<float>(p, w, data, p->tab.sin2_32, p->tab.space.tw32);
}

bec_status launch_dst_rows(bec_problem* p, const void* in, int in_fp64, void* out, int out_fp64,
                           long long rows, int fp64) {
  return launch_dst_rows_w(p, in, in_fp64, out, out_fp64, rows, fp64, p->tile.rows);
}

bec_status launch_dst_cols(bec_problem* p, void* data, int fp64) {
  return launch_dst_cols_w(p, data, fp64, p->tile.cols);
}

}  // namespace bec

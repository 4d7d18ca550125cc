// 3 x 3 convolution with 32 input and 32 output channels on the 5th-generation
// tensor cores (tcgen05), BF16 operands, FP32 accumulation in tensor memory:
// the hot layers of the learned correction's network (7 of its 9 layers).
//
// Implicit GEMM.  One tile is 8 x 16 output pixels of one image = the MMA's
// M = 128 rows; N = 32 output channels; K = 9 taps x 32 input channels, issued
// as 9 x 2 MMAs of K = 16.  For tap (dy, dx) the A operand is the input box
// shifted by (dy, dx): TMA loads it from the NHWC activation (channels
// innermost, 64 bytes per pixel) with the 64-byte swizzle, and the tensor
// map's out-of-range fill supplies the zero padding at the borders.  The B
// operand (the weights of all taps, [tap][c_out][c_in]) is loaded once per
// CTA by TMA with the same swizzle.  Both operands are K-major, so the shared
// memory descriptors describe rows of 64 bytes in 8-row swizzle atoms
// (stride 512 bytes), the second K-step starting 32 bytes into the row.
//
// The CTA is persistent over tiles: while the epilogue of tile t reads the
// accumulator from tensor memory (tcgen05.ld), applies ReLU and stores BF16,
// the loads of tile t + grid are already in flight.  Two CTAs share an SM.
//
// Every wait is bounded (about 0.2 s of SM clock); a wait that runs
// out sets *err, every thread leaves the tile loop at the next CTA barrier,
// the CTA waits (bounded) for its copies and MMAs in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bec_internal.h"

namespace bec {
namespace {

constexpr int kTileX = 16, kTileY = 8;             // 128 output pixels
constexpr int kC = 32;                             // channels in and out
constexpr int kTaps = 9;
constexpr int kABytes = kTileX * kTileY * kC * 2;  // 8192 per tap
constexpr int kBBytes = kC * kC * 2;               // 2048 per tap
constexpr int kSmemBytes = kTaps * (kABytes + kBBytes) + 1024 + 64;
constexpr int kThreads = 128;
constexpr long long kSpinCycles = 400000000LL;     // ~0.2 s at 2 GHz
constexpr uint32_t kTmemCols = 32;

// instruction descriptor of tcgen05.mma kind::f16: D F32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Waits for the phase of parity ph; false when it ran out or another thread
// of the CTA gave up (*abort).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t ph, volatile int* abort) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(ph)
        : "memory");
    if (done) return true;
    if (*abort) return false;
    if (clock64() - t0 > kSpinCycles) return false;
  }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// shared memory descriptor: K-major, 64-byte swizzle, 8-row atoms 512 bytes
// apart (SBO); LBO is not used by swizzled K-major layouts (set to 1);
// bits 46-48 hold the fixed value 0b001; swizzle mode 4 = 64 bytes.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 columns of FP32 from tensor memory: thread t of the warp gets
// row (lane base + t), columns col .. col + 31.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct TileCoord {
  int img, x0, y0;
};

__device__ __forceinline__ TileCoord tile_coord(int t, int tiles_x, int tiles_img) {
  TileCoord c;
  c.img = t / tiles_img;
  const int r = t - c.img * tiles_img;
  const int ty = r / tiles_x;
  c.x0 = (r - ty * tiles_x) * kTileX;
  c.y0 = ty * kTileY;
  return c;
}

__device__ __forceinline__ void issue_tile(const CUtensorMap* in_map, uint32_t sA, uint32_t bar,
                                           TileCoord c) {
  mbar_expect_tx(bar, kTaps * kABytes);
#pragma unroll 1
  for (int tap = 0; tap < kTaps; ++tap) {
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    tma_load_4d(sA + tap * kABytes, in_map, 0, c.x0 + dx, c.y0 + dy, c.img, bar);
  }
}

__global__ void __launch_bounds__(kThreads, 2)
conv3x3_tc_kernel(const __grid_constant__ CUtensorMap in_map,
                  const __grid_constant__ CUtensorMap w_map, int layer,
                  __nv_bfloat16* __restrict__ out, int m, int tiles_x, int tiles_img, int ntiles,
                  int relu, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t sA = smem_u32(base);
  const uint32_t sB = sA + kTaps * kABytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kTaps * (kABytes + kBBytes));
  const uint32_t bar_ld = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]),
                 bar_w = smem_u32(&bars[2]);
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(bar_ld, 1);
    mbar_init(bar_mma, 1);
    mbar_init(bar_w, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  int t = blockIdx.x;
  bool pending_ld = false;   // a tile's loads were issued and not yet waited for
  bool pending_mma = false;  // MMAs were committed and not yet waited for
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar_w, kTaps * kBBytes);
    tma_load_3d(sB, &w_map, 0, 0, layer * kTaps, bar_w);
    if (t < ntiles) {
      issue_tile(&in_map, sA, bar_ld, tile_coord(t, tiles_x, tiles_img));
      pending_ld = true;
    }
    if (!mbar_wait(bar_w, 0, &abort_flag)) abort_flag = 1;
  }
  uint32_t ph = 0;
  bool failed = false;
  for (; t < ntiles; t += gridDim.x) {
    if (threadIdx.x == 0 && !abort_flag) {
      if (mbar_wait(bar_ld, ph, &abort_flag)) {
        pending_ld = false;
        fence_after();
#pragma unroll 1
        for (int tap = 0; tap < kTaps; ++tap) {
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t off = ks * 32;
            mma_bf16(tmem, sdesc(sA + tap * kABytes + off), sdesc(sB + tap * kBBytes + off),
                     (tap | ks) != 0);
          }
        }
        mma_commit(bar_mma);
        pending_mma = true;
      } else {
        abort_flag = 1;
      }
    }
    const bool ok = mbar_wait(bar_mma, ph, &abort_flag);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    pending_mma = false;
    fence_after();
    const int tn = t + gridDim.x;
    if (threadIdx.x == 0 && tn < ntiles) {
      issue_tile(&in_map, sA, bar_ld, tile_coord(tn, tiles_x, tiles_img));
      pending_ld = true;
    }
    // epilogue: row 32 warp + lane of the accumulator = tile pixel
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
    const TileCoord c = tile_coord(t, tiles_x, tiles_img);
    const int row = 32 * warp + lane;
    const int y = c.y0 + row / kTileX, x = c.x0 + row % kTileX;
    if (y < m && x < m) {
      uint4 pk[4];
      uint32_t* w32 = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float a = v[2 * i], b = v[2 * i + 1];
        if (relu) {
          a = fmaxf(a, 0.f);
          b = fmaxf(b, 0.f);
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        w32[i] = *reinterpret_cast<const uint32_t*>(&h);
      }
      uint4* dst = reinterpret_cast<uint4*>(out + (((long long)c.img * m + y) * m + x) * kC);
#pragma unroll
      for (int i = 0; i < 4; ++i) dst[i] = pk[i];
    }
    fence_before();
    __syncthreads();
    ph ^= 1;
  }
  if (failed && threadIdx.x == 0) {
    atomicExch(err, 1);
    // let copies and MMAs in flight land before the shared and tensor memory
    // are released (bounded again)
    volatile int never = 0;
    if (pending_ld) mbar_wait(bar_ld, ph, &never);
    if (pending_mma) mbar_wait(bar_mma, ph, &never);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// wt[l][tap][co][ci] = bf16(W[l][tap][ci][co]) for the 32 -> 32 layers
__global__ void tc_weights_kernel(const float* __restrict__ W, __nv_bfloat16* __restrict__ wt,
                                  int nlayers) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nlayers * kTaps * kC * kC) return;
  const int ci = g % kC, co = (g / kC) % kC, lt = g / (kC * kC);
  wt[g] = __float2bfloat16(W[(long long)lt * kC * kC + ci * kC + co]);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

bool tc_conv_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

bec_status tc_convert_weights(bec_problem* p, const float* W_first, int nlayers,
                              __nv_bfloat16* wt) {
  const int n = nlayers * kTaps * kC * kC;
  BEC_LAUNCH_BEGIN(p);
  tc_weights_kernel<<<(n + 255) / 256, 256, 0, p->stream>>>(W_first, wt, nlayers);
  BEC_LAUNCH_CHECK(p, "net_tc_weights_kernel");
  return BEC_OK;
}

bec_status tc_conv3x3(bec_problem* p, const __nv_bfloat16* in, const __nv_bfloat16* wt,
                      int nlayers, int layer, __nv_bfloat16* out, int m, int B, int bmax, bool relu,
                      int* err) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (enc == nullptr || m < kTileX || B < 1 || B > bmax || layer < 0 || layer >= nlayers) {
    set_error("tensor-core convolution: unsupported request");
    return BEC_EUNSUPPORTED;
  }
  alignas(64) CUtensorMap in_map, w_map;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)kC, (cuuint64_t)m, (cuuint64_t)m, (cuuint64_t)bmax};
    const cuuint64_t strides[3] = {(cuuint64_t)kC * 2, (cuuint64_t)kC * 2 * m,
                                   (cuuint64_t)kC * 2 * m * m};
    const cuuint32_t box[4] = {(cuuint32_t)kC, kTileX, kTileY, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&in_map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(in), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled (activations)");
      return BEC_ECUDA;
    }
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)kC, (cuuint64_t)kC, (cuuint64_t)nlayers * kTaps};
    const cuuint64_t strides[2] = {(cuuint64_t)kC * 2, (cuuint64_t)kC * kC * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kC, (cuuint32_t)kC, (cuuint32_t)kTaps};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(&w_map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(wt), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled (weights)");
      return BEC_ECUDA;
    }
  }
  static bool attr_set = false;
  if (!attr_set) {
    BEC_CUDA_TRY(cudaFuncSetAttribute(conv3x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kSmemBytes));
    attr_set = true;
  }
  int dev = 0, sms = 0;
  BEC_CUDA_TRY(cudaGetDevice(&dev));
  BEC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int tiles_x = (m + kTileX - 1) / kTileX, tiles_y = (m + kTileY - 1) / kTileY;
  const int tiles_img = tiles_x * tiles_y;
  const int ntiles = tiles_img * B;
  const int grid = ntiles < 2 * sms ? ntiles : 2 * sms;
  BEC_LAUNCH_BEGIN(p);
  conv3x3_tc_kernel<<<grid, kThreads, kSmemBytes, p->stream>>>(
      in_map, w_map, layer, out, m, tiles_x, tiles_img, ntiles, relu ? 1 : 0, err);
  BEC_LAUNCH_CHECK(p, "net_conv_tc_kernel");
  return BEC_OK;
}

}  // namespace bec

// RES = ||f - L u|| / ||f|| without any device allocation: bec_relres_noalloc.
//
// Some callers cannot allocate device memory when they need this check: their
// device memory is owned by another allocator (a framework's caching pool),
// their memory budget is fixed at start-up, their policy forbids allocation
// after initialisation, or the device is nearly full.  Such callers may hold
// no bec_problem either, since bec_allocate_problem allocates.  This entry
// point takes the geometry and the two vectors directly and keeps its block
// partial sums in a file-scope device array, so it allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "bec_internal.h"

namespace bec {
namespace {

constexpr int kStaticThreads = 256;
constexpr int kStaticTimeChunk = 8;
constexpr int kRelresMaxBlocks = 16384;   // partial-sum pairs the array holds
constexpr int kMaxDevices = 64;

// Partial sums of (f - L u)^2 and f^2, one pair per block.  Every GPU that
// loads the library holds this array (256 KiB) until the process exits.
static __device__ __align__(256) double g_relres_partials[2 * kRelresMaxBlocks];

// Device address of g_relres_partials for each device, looked up once.
std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {};

struct StaticGeom {
  long long J;
  int m, N, dim;
  double cdiag, c;
};

__device__ __forceinline__ double static_row(const double* __restrict__ us, long long q, int ix,
                                             int iy, const StaticGeom& g, double center) {
  double nb = (ix > 0 ? us[q - 1] : 0.0) + (ix < g.m - 1 ? us[q + 1] : 0.0);
  if (g.dim == 2) nb += (iy > 0 ? us[q - g.m] : 0.0) + (iy < g.m - 1 ? us[q + g.m] : 0.0);
  return g.cdiag * center - g.c * nb;
}

// One block per 256 spatial points x 8 time slices; writes one partial pair.
__global__ void __launch_bounds__(kStaticThreads)
relres_partials_static_kernel(const double* __restrict__ f, const double* __restrict__ u,
                              double* __restrict__ partials, StaticGeom g) {
  const long long q = (long long)blockIdx.x * kStaticThreads + threadIdx.x;
  double rr = 0.0, ff = 0.0;
  if (q < g.J) {
    const int n0 = blockIdx.y * kStaticTimeChunk;
    const int n1 = min(g.N, n0 + kStaticTimeChunk);
    const int iy = g.dim == 2 ? (int)(q / g.m) : 0;
    const int ix = (int)(q - (long long)iy * g.m);
    double prev = n0 > 0 ? u[(long long)(n0 - 1) * g.J + q] : 0.0;
    for (int n = n0; n < n1; ++n) {
      const double* us = u + (long long)n * g.J;
      const double center = us[q];
      const long long o = (long long)n * g.J + q;
      const double fo = f[o];
      const double r = fo - (static_row(us, q, ix, iy, g, center) - prev);
      rr += r * r;
      ff += fo * fo;
      prev = center;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, off);
    ff += __shfl_down_sync(0xffffffffu, ff, off);
  }
  __shared__ double s_rr[kStaticThreads / 32], s_ff[kStaticThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_rr[warp] = rr;
    s_ff[warp] = ff;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kStaticThreads / 32; ++w) {
      a += s_rr[w];
      b += s_ff[w];
    }
    const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    partials[2 * blk] = a;
    partials[2 * blk + 1] = b;
  }
}

// res_out[0] = sqrt(sum rr) / sqrt(sum ff), summed in a fixed order.
__global__ void relres_finish_static_kernel(const double* __restrict__ partials, long long nblk,
                                            double* __restrict__ res_out) {
  __shared__ double s_a[256], s_b[256];
  double a = 0.0, b = 0.0;
  for (long long i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  s_a[threadIdx.x] = a;
  s_b[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      s_a[threadIdx.x] += s_a[threadIdx.x + s];
      s_b[threadIdx.x] += s_b[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) res_out[0] = sqrt(s_a[0]) / sqrt(s_b[0]);
}

bec_status static_einval(const char* msg) {
  set_error(msg);
  return BEC_EINVAL;
}

// Looks up (once per device, with that device current) the device address of
// the file-scope partials array.
bec_status static_scratch(double** out) {
  int dev = 0;
  BEC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return static_einval("device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (g_static_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_relres_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_relres_partials)");
    g_static_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_static_ptr[dev];
  return BEC_OK;
}

bool pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace
}  // namespace bec

extern "C" bec_status bec_relres_noalloc(int dim, int nx, int N, double T, double a,
                                         const double* f, const double* u, double* res_out,
                                         void* stream) {
  using namespace bec;
  if (dim != 1 && dim != 2) return static_einval("dim must be 1 or 2");
  if (!pow2((long long)nx + 1) || nx + 1 < 4 || nx + 1 > 1024)
    return static_einval("nx + 1 must be a power of two in [4, 1024]");
  if (!pow2(N) || N < 2 || N > 1024) return static_einval("N must be a power of two in [2, 1024]");
  if (!(T > 0.0) || !(a > 0.0) || T != T || a != a) return static_einval("T and a must be > 0");
  if (f == nullptr || u == nullptr || res_out == nullptr) return static_einval("null pointer");
  const long long J = dim == 2 ? (long long)nx * nx : nx;
  const dim3 grid((unsigned)((J + kStaticThreads - 1) / kStaticThreads),
                  (unsigned)((N + kStaticTimeChunk - 1) / kStaticTimeChunk));
  const long long nblk = (long long)grid.x * grid.y;
  if (nblk > kRelresMaxBlocks)
    return static_einval("problem too large for bec_relres_noalloc: needs ceil(J/256) * "
                         "ceil(N/8) <= 16384 partial sums (about 33.5M unknowns)");
  double* partials = nullptr;
  const bec_status s = static_scratch(&partials);
  if (s != BEC_OK) return s;
  StaticGeom g;
  g.J = J;
  g.m = nx;
  g.N = N;
  g.dim = dim;
  const double h = 1.0 / (nx + 1);
  g.c = (T / N) * a / (h * h);
  g.cdiag = 1.0 + 2.0 * dim * g.c;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  relres_partials_static_kernel<<<grid, kStaticThreads, 0, st>>>(f, u, partials, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "relres_partials_static_kernel");
  relres_finish_static_kernel<<<1, 256, 0, st>>>(partials, nblk, res_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "relres_finish_static_kernel");
  return BEC_OK;
}

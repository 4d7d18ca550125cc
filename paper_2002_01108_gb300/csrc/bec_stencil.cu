// All-at-once stencil kernels (Sec. 2, eq. allatoncesystem): L v, P_eps v,
// the right-hand side f and the true residual RES of Sec. 5.
//
// With M = I and K = (a/h^2) x (3- or 5-point Laplacian), block row n of L is
//     (L v)^n = (1 + 2 dim c) v^n - c (sum of the 2 dim neighbours of v^n) - v^{n-1},
// c = tau a / h^2, with no v^0 term; P_eps adds -eps v^N to block row 1.
// A thread owns one spatial point and walks a chunk of time slices, keeping
// v^{n-1} in a register, so v is read from memory once.
#include <cuda_runtime.h>

#include "bec_internal.h"

namespace bec {
namespace {

constexpr int kStencilThreads = 256;
constexpr int kTimeChunk = 8;

struct StencilGeom {
  long long J;
  int m, N, dim;
  double c;       // tau a / h^2 (constant a)
  double alpha;   // (1 + 2 dim c) / c
  const double* __restrict__ kc;   // variable a: tau K row [centre, W, E, S, N] x J, or null
};

// (L v)^n at one point: c (alpha v - sum of neighbours) - v^{n-1}, which is
// (1 + 2 dim c) v - c (sum) - v^{n-1} in 3 FP64 adds and 2 FMAs.
__device__ __forceinline__ double apply_row(const double* __restrict__ vs, long long q, int ix,
                                            int iy, const StencilGeom& g, double center,
                                            double prev) {
  if (g.kc != nullptr) {   // variable coefficient: v + tau K v - v^{n-1}
    const long long J = g.J;
    double t = fma(g.kc[q], center, center - prev);
    if (ix > 0) t = fma(-g.kc[J + q], vs[q - 1], t);
    if (ix < g.m - 1) t = fma(-g.kc[2 * J + q], vs[q + 1], t);
    if (iy > 0) t = fma(-g.kc[3 * J + q], vs[q - g.m], t);
    if (iy < g.m - 1) t = fma(-g.kc[4 * J + q], vs[q + g.m], t);
    return t;
  }
  double nb = (ix > 0 ? vs[q - 1] : 0.0) + (ix < g.m - 1 ? vs[q + 1] : 0.0);
  if (g.dim == 2) nb += (iy > 0 ? vs[q - g.m] : 0.0) + (iy < g.m - 1 ? vs[q + g.m] : 0.0);
  return fma(g.c, fma(g.alpha, center, -nb), -prev);
}

// y = L v (corner = 0) or y = P_eps v (corner = eps), times *out_scale if given.
__global__ void __launch_bounds__(kStencilThreads)
apply_L_kernel(const double* __restrict__ v, double* __restrict__ y, StencilGeom g,
               double corner, const double* __restrict__ out_scale) {
  const long long q = (long long)blockIdx.x * kStencilThreads + threadIdx.x;
  if (q >= g.J) return;
  const int n0 = blockIdx.y * kTimeChunk;
  const int n1 = min(g.N, n0 + kTimeChunk);
  const int iy = g.dim == 2 ? (int)(q / g.m) : 0;
  const int ix = (int)(q - (long long)iy * g.m);
  double prev = n0 > 0 ? v[(long long)(n0 - 1) * g.J + q]
                       : (corner != 0.0 ? corner * v[(long long)(g.N - 1) * g.J + q] : 0.0);
  const double sc = out_scale ? out_scale[0] : 1.0;
  for (int n = n0; n < n1; ++n) {
    const double* vs = v + (long long)n * g.J;
    const double center = vs[q];
    const double r = apply_row(vs, q, ix, iy, g, center, prev);
    y[(long long)n * g.J + q] = out_scale ? sc * r : r;
    prev = center;
  }
}

// w = L z and, for v < NV, the block sums of V_v . w: the first Gram-Schmidt
// pass fused with the operator.  A fixed grid walks the (256-point tile, time
// chunk) pairs in a fixed order, so the partial sums are reproducible.
template <int NV>
__global__ void __launch_bounds__(kStencilThreads)
stencil_dots_kernel(const double* __restrict__ z, double* __restrict__ w, StencilGeom g, VecList V,
                    const double* __restrict__ vshift, const double* __restrict__ sshift,
                    double* __restrict__ partials) {
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  double accn = 0.0;
  const double ss = vshift ? sshift[0] : 0.0;
  const long long jt = (g.J + kStencilThreads - 1) / kStencilThreads;
  const long long tiles = jt * ((g.N + kTimeChunk - 1) / kTimeChunk);
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const long long q = (t % jt) * kStencilThreads + threadIdx.x;
    if (q >= g.J) continue;
    const int n0 = (int)(t / jt) * kTimeChunk;
    const int n1 = min(g.N, n0 + kTimeChunk);
    const int iy = g.dim == 2 ? (int)(q / g.m) : 0;
    const int ix = (int)(q - (long long)iy * g.m);
    double prev = n0 > 0 ? z[(long long)(n0 - 1) * g.J + q] : 0.0;
    for (int n = n0; n < n1; ++n) {
      const double* zs = z + (long long)n * g.J;
      const double center = zs[q];
      const long long o = (long long)n * g.J + q;
      double y = apply_row(zs, q, ix, iy, g, center, prev);
      if (vshift) y = fma(-ss, vshift[o], y);
      w[o] = y;
      prev = center;
      accn = fma(y, y, accn);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fma(V.v[v][o], y, acc[v]);
    }
  }
  __shared__ double red[kStencilThreads / 32][NV + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = acc[v];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) red[warp][v] = s;
  }
  for (int off = 16; off > 0; off >>= 1) accn += __shfl_down_sync(0xffffffffu, accn, off);
  if (lane == 0) red[warp][NV] = accn;
  __syncthreads();
  if ((int)threadIdx.x <= NV) {
    double s = 0.0;
#pragma unroll
    for (int wi = 0; wi < kStencilThreads / 32; ++wi) s += red[wi][threadIdx.x];
    partials[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;   // row NV: sum of w^2
  }
}

// r = f - L u (u == nullptr: r = f)
__global__ void __launch_bounds__(kStencilThreads)
residual_kernel(const double* __restrict__ f, const double* __restrict__ u,
                double* __restrict__ r, StencilGeom g) {
  const long long q = (long long)blockIdx.x * kStencilThreads + threadIdx.x;
  if (q >= g.J) return;
  const int n0 = blockIdx.y * kTimeChunk;
  const int n1 = min(g.N, n0 + kTimeChunk);
  const int iy = g.dim == 2 ? (int)(q / g.m) : 0;
  const int ix = (int)(q - (long long)iy * g.m);
  if (u == nullptr) {
    for (int n = n0; n < n1; ++n) r[(long long)n * g.J + q] = f[(long long)n * g.J + q];
    return;
  }
  double prev = n0 > 0 ? u[(long long)(n0 - 1) * g.J + q] : 0.0;
  for (int n = n0; n < n1; ++n) {
    const double* us = u + (long long)n * g.J;
    const double center = us[q];
    const long long o = (long long)n * g.J + q;
    r[o] = f[o] - apply_row(us, q, ix, iy, g, center, prev);
    prev = center;
  }
}

// Block sums of (f - L u)^2 and f^2 for RES (Sec. 5).  One partial pair per
// block, reduced in a fixed order by finish_norms_kernel: deterministic.
__global__ void __launch_bounds__(kStencilThreads)
residual_norms_kernel(const double* __restrict__ f, const double* __restrict__ u,
                      double* __restrict__ partials, StencilGeom g) {
  const long long q = (long long)blockIdx.x * kStencilThreads + threadIdx.x;
  double rr = 0.0, ff = 0.0;
  if (q < g.J) {
    const int n0 = blockIdx.y * kTimeChunk;
    const int n1 = min(g.N, n0 + kTimeChunk);
    const int iy = g.dim == 2 ? (int)(q / g.m) : 0;
    const int ix = (int)(q - (long long)iy * g.m);
    double prev = n0 > 0 ? u[(long long)(n0 - 1) * g.J + q] : 0.0;
    for (int n = n0; n < n1; ++n) {
      const double* us = u + (long long)n * g.J;
      const double center = us[q];
      const long long o = (long long)n * g.J + q;
      const double fo = f[o];
      const double r = fo - apply_row(us, q, ix, iy, g, center, prev);
      rr += r * r;
      ff += fo * fo;
      prev = center;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, off);
    ff += __shfl_down_sync(0xffffffffu, ff, off);
  }
  __shared__ double s_rr[kStencilThreads / 32], s_ff[kStencilThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_rr[warp] = rr;
    s_ff[warp] = ff;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kStencilThreads / 32; ++w) {
      a += s_rr[w];
      b += s_ff[w];
    }
    const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    partials[2 * blk] = a;
    partials[2 * blk + 1] = b;
  }
}

__global__ void finish_norms_kernel(const double* __restrict__ partials, long long nblk,
                                    double* __restrict__ scal, int slot) {
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
  if (threadIdx.x == 0) {
    scal[slot] = sqrt(s_a[0]);
    scal[slot + 1] = sqrt(s_b[0]);
  }
}

// f = tau fsrc, plus u0 in slice 1 (Sec. 2).
__global__ void build_rhs_kernel(const double* __restrict__ u0, const double* __restrict__ fsrc,
                                 double* __restrict__ f, long long J, long long U, double tau) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < U;
       i += (long long)gridDim.x * blockDim.x) {
    double v = tau * fsrc[i];
    if (i < J) v += u0[i];
    f[i] = v;
  }
}

StencilGeom geom(const bec_problem* p) {
  StencilGeom g;
  g.J = p->J;
  g.m = p->m;
  g.N = p->N;
  g.dim = p->dim;
  g.c = p->tau * p->a / (p->h * p->h);
  g.alpha = (1.0 + 2.0 * p->dim * g.c) / g.c;
  g.kc = p->kcoef;
  return g;
}

dim3 stencil_grid(const bec_problem* p) {
  return dim3((unsigned)((p->J + kStencilThreads - 1) / kStencilThreads),
              (unsigned)((p->N + kTimeChunk - 1) / kTimeChunk));
}

}  // namespace

long long stencil_blocks(const bec_problem* p) {
  const dim3 g = stencil_grid(p);
  return (long long)g.x * g.y;
}

bec_status launch_apply_L(bec_problem* p, const double* v, double* y, double corner,
                          const double* out_scale) {
  BEC_LAUNCH_BEGIN(p);
  apply_L_kernel<<<stencil_grid(p), kStencilThreads, 0, p->stream>>>(v, y, geom(p), corner,
                                                                     out_scale);
  BEC_LAUNCH_CHECK(p, "apply_L_kernel");
  return BEC_OK;
}

bec_status launch_stencil_dots(bec_problem* p, const double* z, double* w,
                               const double* const* V, int nv, const double* sigma,
                               double* hout, const double* vshift, const double* sshift,
                               int norm_slot) {
  const int n = nv < kMaxVec ? nv : kMaxVec;
  VecList L;
  for (int i = 0; i < kMaxVec; ++i) L.v[i] = i < n ? V[i] : V[0];
  BEC_LAUNCH_BEGIN(p);
  switch (n) {
#define BEC_SD_CASE(NV)                                                                     \
  case NV:                                                                                  \
    stencil_dots_kernel<NV><<<kStencilDotBlocks, kStencilThreads, 0, p->stream>>>(          \
        z, w, geom(p), L, vshift, sshift, p->partials);                                     \
    break;
    BEC_SD_CASE(1) BEC_SD_CASE(2) BEC_SD_CASE(3) BEC_SD_CASE(4) BEC_SD_CASE(5) BEC_SD_CASE(6)
    BEC_SD_CASE(7) BEC_SD_CASE(8) BEC_SD_CASE(9) BEC_SD_CASE(10) BEC_SD_CASE(11) BEC_SD_CASE(12)
    BEC_SD_CASE(13) BEC_SD_CASE(14) BEC_SD_CASE(15) BEC_SD_CASE(16) BEC_SD_CASE(17)
    BEC_SD_CASE(18) BEC_SD_CASE(19) BEC_SD_CASE(20) BEC_SD_CASE(21) BEC_SD_CASE(22)
    BEC_SD_CASE(23) BEC_SD_CASE(24) BEC_SD_CASE(25) BEC_SD_CASE(26) BEC_SD_CASE(27)
    BEC_SD_CASE(28) BEC_SD_CASE(29) BEC_SD_CASE(30) BEC_SD_CASE(31) BEC_SD_CASE(32)
#undef BEC_SD_CASE
    default: return BEC_EINVAL;
  }
  BEC_LAUNCH_CHECK(p, "stencil_dots_kernel");
  bec_status s = BEC_OK;
  if (norm_slot >= 0) {
    s = launch_finish_sqrt(p, p->partials + (long long)n * kStencilDotBlocks, kStencilDotBlocks,
                           norm_slot, nullptr);
    if (s != BEC_OK) return s;
  }
  s = launch_finish_dots(p, n, kStencilDotBlocks, sigma, hout);
  if (s != BEC_OK || nv <= kMaxVec) return s;
  // more vectors than one fused launch holds: the rest as plain dots
  return launch_dots(p, w, V + kMaxVec, nv - kMaxVec, sigma ? sigma + kMaxVec : nullptr,
                     hout + kMaxVec);
}

bec_status launch_residual(bec_problem* p, const double* f, const double* u, double* r) {
  BEC_LAUNCH_BEGIN(p);
  residual_kernel<<<stencil_grid(p), kStencilThreads, 0, p->stream>>>(f, u, r, geom(p));
  BEC_LAUNCH_CHECK(p, "residual_kernel");
  return BEC_OK;
}

bec_status launch_residual_norms(bec_problem* p, const double* f, const double* u, int slot) {
  const dim3 grid = stencil_grid(p);
  BEC_LAUNCH_BEGIN(p);
  residual_norms_kernel<<<grid, kStencilThreads, 0, p->stream>>>(f, u, p->partials, geom(p));
  BEC_LAUNCH_CHECK(p, "residual_norms_kernel");
  BEC_LAUNCH_BEGIN(p);
  finish_norms_kernel<<<1, 256, 0, p->stream>>>(p->partials, (long long)grid.x * grid.y, p->scal,
                                                 slot);
  BEC_LAUNCH_CHECK(p, "finish_norms_kernel");
  return BEC_OK;
}

bec_status launch_build_rhs(bec_problem* p, const double* u0, const double* fsrc, double* f) {
  BEC_LAUNCH_BEGIN(p);
  build_rhs_kernel<<<4 * 152, 256, 0, p->stream>>>(u0, fsrc, f, p->J, p->U, p->tau);
  BEC_LAUNCH_CHECK(p, "build_rhs_kernel");
  return BEC_OK;
}

}  // namespace bec

// All-at-once stencil kernels (Sec. 2, eq. allatoncesystem): L v, P_eps v,
// the right-hand side f and the true residual RES of Sec. 5.
//
// With M = I and K = (a/h^2) x (3- or 5-point Laplacian), block row n of L is
//     (L v)^n = (1 + 2 dim c) v^n - c (sum of the 2 dim neighbours of v^n) - v^{n-1},
// c = tau a / h^2, with no v^0 term; P_eps adds -eps v^N to block row 1.  With
// Q1 elements (Example 1 of Sec. 5) it is (M + tau K) v^n - M v^{n-1}, with the
// 9-point stencils of M and K, and P_eps adds -eps M v^N.  The two-step
// scheme (eq. pstepscheme with r = (3/2, -2, 1/2), template parameter P = 2)
// has block rows (r0 M + tau K) v^n + r1 M v^{n-1} + r2 M v^{n-2}, and P_eps
// wraps the missing terms around with the factor eps (eq.
// pstepbecpreconditioner).
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
  // Q1 elements (q1 != 0): the 9-point (2D) or 3-point (1D) stencils of
  // M + tau K and of M, as centre / edge / corner weights
  int q1;
  double ac, ae, ak, mc, me, mk;
  // two-step scheme: r1, r2 of the rows; rhs1, rhs2 = the multiples of M u^0
  // that the right-hand side adds to slices 1 and 2 (BDF1: 1 and 0)
  double r1, r2, rhs1, rhs2;
};

// sums of the 4 edge and 4 corner neighbours of point q of slice s (zero
// outside the interior; 1D: the 2 neighbours, no corners)
__device__ __forceinline__ void neighbour_sums(const double* __restrict__ s, long long q, int ix,
                                               int iy, const StencilGeom& g, double& edge,
                                               double& corner) {
  const int m = g.m;
  const bool w = ix > 0, e = ix < m - 1;
  edge = (w ? s[q - 1] : 0.0) + (e ? s[q + 1] : 0.0);
  corner = 0.0;
  if (g.dim == 2) {
    const bool so = iy > 0, no = iy < m - 1;
    edge += (so ? s[q - m] : 0.0) + (no ? s[q + m] : 0.0);
    corner = ((so && w) ? s[q - m - 1] : 0.0) + ((so && e) ? s[q - m + 1] : 0.0) +
             ((no && w) ? s[q + m - 1] : 0.0) + ((no && e) ? s[q + m + 1] : 0.0);
  }
}

// Q1 elements: (M + tau K) v^n - ps_scale M ps at one point (ps = the slice
// before, or the wrapped last slice of P_eps, or null).
__device__ __forceinline__ double apply_row_q1(const double* __restrict__ vs,
                                               const double* __restrict__ ps, double ps_scale,
                                               long long q, int ix, int iy, const StencilGeom& g,
                                               double center) {
  double e, k;
  neighbour_sums(vs, q, ix, iy, g, e, k);
  double y = fma(g.ac, center, fma(g.ae, e, g.ak * k));
  if (ps != nullptr) {
    double pe, pk;
    neighbour_sums(ps, q, ix, iy, g, pe, pk);
    y = fma(-ps_scale, fma(g.mc, ps[q], fma(g.me, pe, g.mk * pk)), y);
  }
  return y;
}

// Q1 elements, two-step scheme: (r0 M + tau K) v^n + s1 M ps + s2 M ps2 at one
// point (ps, ps2 = the slices one and two back, wrapped or null).
__device__ __forceinline__ double apply_row_q1_p2(const double* __restrict__ vs,
                                                  const double* __restrict__ ps, double s1,
                                                  const double* __restrict__ ps2, double s2,
                                                  long long q, int ix, int iy, const StencilGeom& g,
                                                  double center) {
  double e, k;
  neighbour_sums(vs, q, ix, iy, g, e, k);
  double y = fma(g.ac, center, fma(g.ae, e, g.ak * k));
  if (ps != nullptr) {
    double pe, pk;
    neighbour_sums(ps, q, ix, iy, g, pe, pk);
    y = fma(s1, fma(g.mc, ps[q], fma(g.me, pe, g.mk * pk)), y);
  }
  if (ps2 != nullptr) {
    double pe, pk;
    neighbour_sums(ps2, q, ix, iy, g, pe, pk);
    y = fma(s2, fma(g.mc, ps2[q], fma(g.me, pe, g.mk * pk)), y);
  }
  return y;
}

// M u at one point (Q1 elements)
__device__ __forceinline__ double mass_row_q1(const double* __restrict__ us, long long q, int ix,
                                              int iy, const StencilGeom& g) {
  double e, k;
  neighbour_sums(us, q, ix, iy, g, e, k);
  return fma(g.mc, us[q], fma(g.me, e, g.mk * k));
}

// The operator a kernel instantiation applies: finite differences in 1D or
// 2D (constant or variable a), Q1 elements (1D or 2D), finite differences in 3D.
enum { kFD = 0, kQ1 = 1, kFD3 = 2 };

// point q of a slice as (ix, iy, iz): x fastest, rows of m points
template <int KIND>
__device__ __forceinline__ void decompose(long long q, const StencilGeom& g, int& ix, int& iy,
                                          int& iz) {
  if constexpr (KIND == kFD3) {
    const long long r = q / g.m;
    ix = (int)(q - r * g.m);
    iz = (int)(r / g.m);
    iy = (int)(r - (long long)iz * g.m);
  } else {
    iy = g.dim == 2 ? (int)(q / g.m) : 0;
    ix = (int)(q - (long long)iy * g.m);
    iz = 0;
  }
}

// (L v)^n at one point: c (alpha v - sum of neighbours) - v^{n-1}, which is
// (1 + 2 dim c) v - c (sum) - v^{n-1} in 3 FP64 adds and 2 FMAs (2D).
__device__ __forceinline__ double apply_row(const double* __restrict__ vs, long long q, int ix,
                                            int iy, int iz, const StencilGeom& g, double center,
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

// 3D finite differences (7-point): (1 + 6c) v - c (sum of the 6 neighbours) - v^{n-1}
__device__ __forceinline__ double apply_row3(const double* __restrict__ vs, long long q, int ix,
                                             int iy, int iz, const StencilGeom& g, double center,
                                             double prev) {
  const long long m2 = (long long)g.m * g.m;
  const double nb = (ix > 0 ? vs[q - 1] : 0.0) + (ix < g.m - 1 ? vs[q + 1] : 0.0) +
                    (iy > 0 ? vs[q - g.m] : 0.0) + (iy < g.m - 1 ? vs[q + g.m] : 0.0) +
                    (iz > 0 ? vs[q - m2] : 0.0) + (iz < g.m - 1 ? vs[q + m2] : 0.0);
  return fma(g.c, fma(g.alpha, center, -nb), -prev);
}

// the row of L (or P_eps without the wrap) of kernel kind KIND and P-step
// scheme at one point; ps, ps2 = the slices one and two back (Q1 only; null
// before the first slice); prev, prev2 = v^{n-1}, v^{n-2} at the point (FD)
template <int KIND, int P>
__device__ __forceinline__ double row_of(const double* __restrict__ vs,
                                         const double* __restrict__ ps,
                                         const double* __restrict__ ps2, long long q, int ix,
                                         int iy, int iz, const StencilGeom& g, double center,
                                         double prev, double prev2) {
  if constexpr (P == 2) {
    static_assert(KIND != kFD3, "the two-step scheme is 1D or 2D");
    if constexpr (KIND == kQ1) {
      return apply_row_q1_p2(vs, ps, g.r1, ps2, g.r2, q, ix, iy, g, center);
    } else {
      double nb = (ix > 0 ? vs[q - 1] : 0.0) + (ix < g.m - 1 ? vs[q + 1] : 0.0);
      if (g.dim == 2) nb += (iy > 0 ? vs[q - g.m] : 0.0) + (iy < g.m - 1 ? vs[q + g.m] : 0.0);
      return fma(g.c, fma(g.alpha, center, -nb), fma(g.r1, prev, g.r2 * prev2));
    }
  } else if constexpr (KIND == kQ1) {
    return apply_row_q1(vs, ps, 1.0, q, ix, iy, g, center);
  } else if constexpr (KIND == kFD3) {
    return apply_row3(vs, q, ix, iy, iz, g, center, prev);
  } else {
    return apply_row(vs, q, ix, iy, iz, g, center, prev);
  }
}

// slice n - j of v for row n, or the slice wrapped around by P_eps (corner
// != 0) with *scale multiplied by corner; null when there is none
__device__ __forceinline__ const double* back_slice(const double* __restrict__ v, int n, int j,
                                                    const StencilGeom& g, double corner,
                                                    double& scale) {
  if (n - j >= 0) return v + (long long)(n - j) * g.J;
  if (corner == 0.0) return nullptr;
  scale *= corner;
  return v + (long long)(n - j + g.N) * g.J;
}

// y = L v (corner = 0) or y = P_eps v (corner = eps), times *out_scale if given.
template <int KIND, int P>
__global__ void __launch_bounds__(kStencilThreads)
apply_L_kernel(const double* __restrict__ v, double* __restrict__ y, StencilGeom g,
               double corner, const double* __restrict__ out_scale) {
  const long long q = (long long)blockIdx.x * kStencilThreads + threadIdx.x;
  if (q >= g.J) return;
  const int n0 = blockIdx.y * kTimeChunk;
  const int n1 = min(g.N, n0 + kTimeChunk);
  int ix, iy, iz;
  decompose<KIND>(q, g, ix, iy, iz);
  // v^{n0-1} and v^{n0-2} at this point, wrapped around (times corner) by P_eps
  double prev = n0 > 0 ? v[(long long)(n0 - 1) * g.J + q]
                       : (corner != 0.0 ? corner * v[(long long)(g.N - 1) * g.J + q] : 0.0);
  double prev2 = 0.0;
  if constexpr (P == 2) {
    prev2 = n0 > 1 ? v[(long long)(n0 - 2) * g.J + q]
                   : (corner != 0.0 ? corner * v[(long long)(n0 - 2 + g.N) * g.J + q] : 0.0);
  }
  const double sc = out_scale ? out_scale[0] : 1.0;
  for (int n = n0; n < n1; ++n) {
    const double* vs = v + (long long)n * g.J;
    const double center = vs[q];
    double r;
    if constexpr (KIND == kQ1 && P == 2) {
      double s1 = g.r1, s2 = g.r2;
      const double* ps = back_slice(v, n, 1, g, corner, s1);
      const double* ps2 = back_slice(v, n, 2, g, corner, s2);
      r = apply_row_q1_p2(vs, ps, s1, ps2, s2, q, ix, iy, g, center);
    } else if constexpr (KIND == kQ1) {
      const double* ps = n > 0 ? vs - g.J : (corner != 0.0 ? v + (long long)(g.N - 1) * g.J : nullptr);
      r = apply_row_q1(vs, ps, n > 0 ? 1.0 : corner, q, ix, iy, g, center);
    } else {
      r = row_of<KIND, P>(vs, nullptr, nullptr, q, ix, iy, iz, g, center, prev, prev2);
    }
    y[(long long)n * g.J + q] = out_scale ? sc * r : r;
    prev2 = prev;
    prev = center;
  }
}

// w = L z and, for v < NV, the block sums of V_v . w: the first Gram-Schmidt
// pass fused with the operator.  A fixed grid walks the (256-point tile, time
// chunk) pairs in a fixed order, so the partial sums are reproducible.
template <int NV, int KIND, int P>
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
    int ix, iy, iz;
    decompose<KIND>(q, g, ix, iy, iz);
    double prev = n0 > 0 ? z[(long long)(n0 - 1) * g.J + q] : 0.0;
    double prev2 = (P == 2 && n0 > 1) ? z[(long long)(n0 - 2) * g.J + q] : 0.0;
    for (int n = n0; n < n1; ++n) {
      const double* zs = z + (long long)n * g.J;
      const double center = zs[q];
      const long long o = (long long)n * g.J + q;
      double y = row_of<KIND, P>(zs, n > 0 ? zs - g.J : nullptr, n > 1 ? zs - 2 * g.J : nullptr, q,
                                 ix, iy, iz, g, center, prev, prev2);
      if (vshift) y = fma(-ss, vshift[o], y);
      w[o] = y;
      prev2 = prev;
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
template <int KIND, int P>
__global__ void __launch_bounds__(kStencilThreads)
residual_kernel(const double* __restrict__ f, const double* __restrict__ u,
                double* __restrict__ r, StencilGeom g) {
  const long long q = (long long)blockIdx.x * kStencilThreads + threadIdx.x;
  if (q >= g.J) return;
  const int n0 = blockIdx.y * kTimeChunk;
  const int n1 = min(g.N, n0 + kTimeChunk);
  int ix, iy, iz;
  decompose<KIND>(q, g, ix, iy, iz);
  if (u == nullptr) {
    for (int n = n0; n < n1; ++n) r[(long long)n * g.J + q] = f[(long long)n * g.J + q];
    return;
  }
  double prev = n0 > 0 ? u[(long long)(n0 - 1) * g.J + q] : 0.0;
  double prev2 = (P == 2 && n0 > 1) ? u[(long long)(n0 - 2) * g.J + q] : 0.0;
  for (int n = n0; n < n1; ++n) {
    const double* us = u + (long long)n * g.J;
    const double center = us[q];
    const long long o = (long long)n * g.J + q;
    r[o] = f[o] - row_of<KIND, P>(us, n > 0 ? us - g.J : nullptr, n > 1 ? us - 2 * g.J : nullptr,
                                  q, ix, iy, iz, g, center, prev, prev2);
    prev2 = prev;
    prev = center;
  }
}

// Block sums of (f - L u)^2 and f^2 for RES (Sec. 5).  One partial pair per
// block, reduced in a fixed order by finish_norms_kernel: deterministic.
template <int KIND, int P>
__global__ void __launch_bounds__(kStencilThreads)
residual_norms_kernel(const double* __restrict__ f, const double* __restrict__ u,
                      double* __restrict__ partials, StencilGeom g) {
  const long long q = (long long)blockIdx.x * kStencilThreads + threadIdx.x;
  double rr = 0.0, ff = 0.0;
  if (q < g.J) {
    const int n0 = blockIdx.y * kTimeChunk;
    const int n1 = min(g.N, n0 + kTimeChunk);
    int ix, iy, iz;
    decompose<KIND>(q, g, ix, iy, iz);
    double prev = n0 > 0 ? u[(long long)(n0 - 1) * g.J + q] : 0.0;
    double prev2 = (P == 2 && n0 > 1) ? u[(long long)(n0 - 2) * g.J + q] : 0.0;
    for (int n = n0; n < n1; ++n) {
      const double* us = u + (long long)n * g.J;
      const double center = us[q];
      const long long o = (long long)n * g.J + q;
      const double fo = f[o];
      const double r = fo - row_of<KIND, P>(us, n > 0 ? us - g.J : nullptr,
                                            n > 1 ? us - 2 * g.J : nullptr, q, ix, iy, iz, g,
                                            center, prev, prev2);
      rr += r * r;
      ff += fo * fo;
      prev2 = prev;
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

// f = tau fsrc, plus M u0 in slice 1 (Sec. 2; M = I for finite differences);
// two-step scheme: plus rhs1 M u0 in slice 1 and rhs2 M u0 in slice 2.
__global__ void build_rhs_kernel(const double* __restrict__ u0, const double* __restrict__ fsrc,
                                 double* __restrict__ f, StencilGeom g, double tau) {
  const long long U = g.J * g.N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < U;
       i += (long long)gridDim.x * blockDim.x) {
    double v = tau * fsrc[i];
    const double coef = i < g.J ? g.rhs1 : (i < 2 * g.J ? g.rhs2 : 0.0);
    if (coef != 0.0) {
      const long long q = i < g.J ? i : i - g.J;
      double mu;
      if (g.q1) {
        int ix, iy, iz;
        decompose<kQ1>(q, g, ix, iy, iz);
        mu = mass_row_q1(u0, q, ix, iy, g);
      } else {
        mu = u0[q];
      }
      v = coef == 1.0 ? v + mu : fma(coef, mu, v);
    }
    f[i] = v;
  }
}

StencilGeom geom(const bec_problem* p) {
  StencilGeom g;
  g.J = p->J;
  g.m = p->m;
  g.N = p->N;
  g.dim = p->dim;
  // r0, r1, r2 of the time scheme (BDF1: 1, -1, 0; BDF2: 3/2, -2, 1/2)
  const bool bdf2 = p->desc.time_scheme == BEC_TIME_BDF2;
  const double r0 = bdf2 ? 1.5 : 1.0;
  g.r1 = bdf2 ? -2.0 : -1.0;
  g.r2 = bdf2 ? 0.5 : 0.0;
  // pre-start values taken equal to u^0: slice n gains -(r_n + ... + r_p) M u^0
  g.rhs1 = -(g.r1 + g.r2);
  g.rhs2 = -g.r2;
  g.c = p->tau * p->a / (p->h * p->h);
  g.alpha = (r0 + 2.0 * p->dim * g.c) / g.c;
  g.kc = p->kcoef;
  g.q1 = p->desc.space == BEC_SPACE_Q1;
  g.ac = g.ae = g.ak = g.mc = g.me = g.mk = 0.0;
  if (g.q1) {
    const double h = p->h, a = p->a, tau = p->tau;
    double kc, ke, kk;
    if (p->dim == 2) {   // M = h^2/36 [1 4 1; 4 16 4; 1 4 1], K = a/3 [-1 -1 -1; -1 8 -1; -1 -1 -1]
      g.mc = 16.0 * h * h / 36.0;
      g.me = 4.0 * h * h / 36.0;
      g.mk = h * h / 36.0;
      kc = 8.0 * a / 3.0;
      ke = -a / 3.0;
      kk = -a / 3.0;
    } else {             // M = h/6 [1 4 1], K = a/h [-1 2 -1]
      g.mc = 4.0 * h / 6.0;
      g.me = h / 6.0;
      g.mk = 0.0;
      kc = 2.0 * a / h;
      ke = -a / h;
      kk = 0.0;
    }
    g.ac = r0 * g.mc + tau * kc;
    g.ae = r0 * g.me + tau * ke;
    g.ak = r0 * g.mk + tau * kk;
  }
  return g;
}

int kind_of(const bec_problem* p) {
  if (p->desc.space == BEC_SPACE_Q1) return kQ1;
  return p->dim == 3 ? kFD3 : kFD;
}

// the kernel instantiation a problem uses: operator kind and time-scheme steps
enum { kVarFD = 0, kVarQ1, kVarFD3, kVarFD2, kVarQ12 };
int variant_of(const bec_problem* p) {
  const int k = kind_of(p);
  if (p->desc.time_scheme == BEC_TIME_BDF2) return k == kQ1 ? kVarQ12 : kVarFD2;
  return k == kQ1 ? kVarQ1 : (k == kFD3 ? kVarFD3 : kVarFD);
}

// LAUNCH(KIND, P) for the problem's variant
#define BEC_STENCIL_SWITCH(var, LAUNCH) \
  switch (var) {                         \
    case kVarQ1: LAUNCH(kQ1, 1); break;  \
    case kVarFD3: LAUNCH(kFD3, 1); break; \
    case kVarFD2: LAUNCH(kFD, 2); break; \
    case kVarQ12: LAUNCH(kQ1, 2); break; \
    default: LAUNCH(kFD, 1);             \
  }

template <int NV>
void stencil_dots_launch(int var, cudaStream_t st, const double* z, double* w,
                         const StencilGeom& g, const VecList& L, const double* vshift,
                         const double* sshift, double* partials) {
#define BEC_SD_LAUNCH(K, P)                                                      \
  stencil_dots_kernel<NV, K, P><<<kStencilDotBlocks, kStencilThreads, 0, st>>>( \
      z, w, g, L, vshift, sshift, partials)
  BEC_STENCIL_SWITCH(var, BEC_SD_LAUNCH)
#undef BEC_SD_LAUNCH
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
  const StencilGeom g = geom(p);
  BEC_LAUNCH_BEGIN(p);
#define BEC_L_LAUNCH(K, P)                                                \
  apply_L_kernel<K, P><<<stencil_grid(p), kStencilThreads, 0, p->stream>>>( \
      v, y, g, corner, out_scale)
  BEC_STENCIL_SWITCH(variant_of(p), BEC_L_LAUNCH)
#undef BEC_L_LAUNCH
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
  const int var = variant_of(p);
  const StencilGeom g = geom(p);
  BEC_LAUNCH_BEGIN(p);
  switch (n) {
#define BEC_SD_CASE(NV)                                                                  \
  case NV:                                                                               \
    stencil_dots_launch<NV>(var, p->stream, z, w, g, L, vshift, sshift, p->partials);   \
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
  const StencilGeom g = geom(p);
  BEC_LAUNCH_BEGIN(p);
#define BEC_R_LAUNCH(K, P) \
  residual_kernel<K, P><<<stencil_grid(p), kStencilThreads, 0, p->stream>>>(f, u, r, g)
  BEC_STENCIL_SWITCH(variant_of(p), BEC_R_LAUNCH)
#undef BEC_R_LAUNCH
  BEC_LAUNCH_CHECK(p, "residual_kernel");
  return BEC_OK;
}

bec_status launch_residual_norms(bec_problem* p, const double* f, const double* u, int slot) {
  const dim3 grid = stencil_grid(p);
  const StencilGeom g = geom(p);
  BEC_LAUNCH_BEGIN(p);
#define BEC_RN_LAUNCH(K, P) \
  residual_norms_kernel<K, P><<<grid, kStencilThreads, 0, p->stream>>>(f, u, p->partials, g)
  BEC_STENCIL_SWITCH(variant_of(p), BEC_RN_LAUNCH)
#undef BEC_RN_LAUNCH
  BEC_LAUNCH_CHECK(p, "residual_norms_kernel");
  BEC_LAUNCH_BEGIN(p);
  finish_norms_kernel<<<1, 256, 0, p->stream>>>(p->partials, (long long)grid.x * grid.y, p->scal,
                                                 slot);
  BEC_LAUNCH_CHECK(p, "finish_norms_kernel");
  return BEC_OK;
}

bec_status launch_build_rhs(bec_problem* p, const double* u0, const double* fsrc, double* f) {
  BEC_LAUNCH_BEGIN(p);
  build_rhs_kernel<<<4 * 152, 256, 0, p->stream>>>(u0, fsrc, f, geom(p), p->tau);
  BEC_LAUNCH_CHECK(p, "build_rhs_kernel");
  return BEC_OK;
}

}  // namespace bec

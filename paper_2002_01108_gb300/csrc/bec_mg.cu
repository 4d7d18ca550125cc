// Multigrid route of P_eps^{-1} (Sec. 4: "efficient spatial solvers, such as
// a multigrid method"; Example 2 of Sec. 5: one V-cycle per shifted system,
// one pre- and one post-smoothing step, piecewise-linear interpolation and
// its transpose).  For every frequency k <= N/2 the V-cycle approximates
//     (lambda'_k M_l + tau K_l) x = b
// on levels l = 0..L-1 with m_0 = nx, m_{l+1} = (m_l - 1)/2, down to 1 x 1:
//   * M_0 = I and K_0 = the conservative 5-point -div(a grad) / h^2;
//   * P_l bilinear interpolation, R_l = P_l^T / 4 (full weighting);
//   * M_{l+1} = R_l M_l P_l and K_{l+1} = R_l K_l P_l (Galerkin, 9-point);
//   * damped Jacobi, x <- x + omega D^{-1} (b - B x), D = diag(B), or the ILU
//     smoother x <- x + M^{-1} (b - B x), M = (D + L) D^{-1} (D + U) with L, U
//     the strictly lower and upper parts of B and D chosen so that diag(M) =
//     diag(B) (ILU(0) on the 5-point finest grid);
//   * the 1 x 1 level is solved exactly.
// K_0 may also carry a convection term w . grad u by first-order upwind
// differences (Example 3 of Sec. 5, whose multigrid smooths with ILU).
// The Galerkin stencils are real and do not depend on k; they are built once
// on the host and read by every frequency.  Each thread owns one grid point
// and walks a chunk of frequencies with its 18 stencil coefficients in
// registers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "bec_fft.cuh"
#include "bec_internal.h"

namespace bec {
namespace {

constexpr int kMgThreads = 256;
constexpr int kFreqChunk = 8;

template <typename T>
struct MgArgs {
  const T* SM;            // [9][J]
  const T* SK;            // [9][J]
  const v2_t<T>* lam;     // lambda'_k, k < K
  int m;
  long long J;
  int K;
  T tau;
  T omega;
};

template <typename V, typename T>
__device__ __forceinline__ V cscale(V a, T s) { return {a.x * s, a.y * s}; }

// L0: the finest grid, where M = I and K is a 5-point stencil: the mass
// product is the centre value and the corner slots are skipped (fewer loads
// and registers; the same sums, since those entries are zero).
__host__ __device__ constexpr bool mg_corner(int s) { return s == 0 || s == 2 || s == 6 || s == 8; }

// B x at point q for frequency k with the stencil coefficients in registers.
template <typename T, bool L0>
__device__ __forceinline__ v2_t<T> apply_b(const v2_t<T>* __restrict__ xk, const T (&sm)[9],
                                           const T (&sk)[9], const int (&off)[9],
                                           const bool (&ok)[9], v2_t<T> lam, T tau) {
  using V = v2_t<T>;
  V am = {0, 0}, ak = {0, 0};
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    if (L0 && mg_corner(s)) continue;
    if (ok[s]) {
      const V xv = xk[off[s]];
      if (L0) {
        if (s == 4) am = xv;
      } else {
        am.x += sm[s] * xv.x;
        am.y += sm[s] * xv.y;
      }
      ak.x += sk[s] * xv.x;
      ak.y += sk[s] * xv.y;
    }
  }
  const V lm = cmul(lam, am);
  return {lm.x + tau * ak.x, lm.y + tau * ak.y};
}

template <typename T, bool L0>
__device__ __forceinline__ void load_point(const MgArgs<T>& a, long long q, T (&sm)[9], T (&sk)[9],
                                           int (&off)[9], bool (&ok)[9]) {
  const int iy = (int)(q / a.m), ix = (int)(q - (long long)iy * a.m);
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    const int dy = s / 3 - 1, dx = s % 3 - 1;
    ok[s] = iy + dy >= 0 && iy + dy < a.m && ix + dx >= 0 && ix + dx < a.m;
    off[s] = (int)q + dy * a.m + dx;
    sm[s] = (L0 ? (s == 4 ? T(1) : T(0)) : a.SM[(long long)s * a.J + q]);
    sk[s] = (L0 && mg_corner(s)) ? T(0) : a.SK[(long long)s * a.J + q];
  }
}

// ZERO: xo = omega D^{-1} b (one sweep from x = 0);
// else: xo = x + omega D^{-1} (b - B x)      (xo != x)
template <typename T, bool ZERO, bool L0>
__global__ void __launch_bounds__(kMgThreads)
mg_smooth_kernel(v2_t<T>* __restrict__ xo, const v2_t<T>* __restrict__ x,
                 const v2_t<T>* __restrict__ b, MgArgs<T> a) {
  using V = v2_t<T>;
  const long long q = (long long)blockIdx.x * kMgThreads + threadIdx.x;
  if (q >= a.J) return;
  T sm[9], sk[9];
  int off[9];
  bool ok[9];
  load_point<T, L0>(a, q, sm, sk, off, ok);
  const int k0 = blockIdx.y * kFreqChunk, k1 = min(a.K, k0 + kFreqChunk);
  for (int k = k0; k < k1; ++k) {
    const long long base = (long long)k * a.J;
    const V lam = a.lam[k];
    const V D = {lam.x * sm[4] + a.tau * sk[4], lam.y * sm[4]};
    const T d2 = D.x * D.x + D.y * D.y;
    T inv;
    if constexpr (sizeof(T) == 8) inv = a.omega * rcp64(d2);   // no FP64 division
    else inv = a.omega / d2;
    V rr = b[base + q];
    V x0 = {0, 0};
    if (!ZERO) {
      x0 = x[base + q];
      const V bx = apply_b<T, L0>(x + base, sm, sk, off, ok, lam, a.tau);
      rr = {rr.x - bx.x, rr.y - bx.y};
    }
    const V c = cmulc(rr, D);     // rr conj(D); times omega / |D|^2 = omega rr / D
    xo[base + q] = {x0.x + c.x * inv, x0.y + c.y * inv};
  }
}

// r = b - B x
template <typename T, bool L0>
__global__ void __launch_bounds__(kMgThreads)
mg_residual_kernel(v2_t<T>* __restrict__ r, const v2_t<T>* __restrict__ x,
                   const v2_t<T>* __restrict__ b, MgArgs<T> a) {
  using V = v2_t<T>;
  const long long q = (long long)blockIdx.x * kMgThreads + threadIdx.x;
  if (q >= a.J) return;
  T sm[9], sk[9];
  int off[9];
  bool ok[9];
  load_point<T, L0>(a, q, sm, sk, off, ok);
  const int k0 = blockIdx.y * kFreqChunk, k1 = min(a.K, k0 + kFreqChunk);
  for (int k = k0; k < k1; ++k) {
    const long long base = (long long)k * a.J;
    const V bx = apply_b<T, L0>(x + base, sm, sk, off, ok, a.lam[k], a.tau);
    const V bb = b[base + q];
    r[base + q] = {bb.x - bx.x, bb.y - bx.y};
  }
}

// bc = R r, R = P^T / 4: coarse (cy, cx) weighs the 3 x 3 fine block around
// fine (2cy+1, 2cx+1) with 1/4 (centre), 1/8 (edges), 1/16 (corners).
template <typename T>
__global__ void __launch_bounds__(kMgThreads)
mg_restrict_kernel(v2_t<T>* __restrict__ bc, const v2_t<T>* __restrict__ r, int mc, int mf,
                   int K) {
  using V = v2_t<T>;
  const long long Jc = (long long)mc * mc, Jf = (long long)mf * mf;
  const long long c = (long long)blockIdx.x * kMgThreads + threadIdx.x;
  if (c >= Jc) return;
  const int cy = (int)(c / mc), cx = (int)(c - (long long)cy * mc);
  const long long f0 = (long long)(2 * cy + 1) * mf + (2 * cx + 1);
  const int k0 = blockIdx.y * kFreqChunk, k1 = min(K, k0 + kFreqChunk);
  for (int k = k0; k < k1; ++k) {
    const V* rk = r + (long long)k * Jf;
    V acc = {0, 0};
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const T w = (dy == 0 ? T(0.5) : T(0.25)) * (dx == 0 ? T(0.5) : T(0.25));
        const V v = rk[f0 + dy * mf + dx];
        acc.x += w * v.x;
        acc.y += w * v.y;
      }
    }
    bc[(long long)k * Jc + c] = acc;
  }
}

// x += P xc (bilinear): fine 2i+1 takes coarse i, fine 2i the mean of i-1, i.
template <typename T>
__global__ void __launch_bounds__(kMgThreads)
mg_prolong_add_kernel(v2_t<T>* __restrict__ x, const v2_t<T>* __restrict__ xc, int mf, int mc,
                      int K) {
  using V = v2_t<T>;
  const long long Jc = (long long)mc * mc, Jf = (long long)mf * mf;
  const long long f = (long long)blockIdx.x * kMgThreads + threadIdx.x;
  if (f >= Jf) return;
  const int fy = (int)(f / mf), fx = (int)(f - (long long)fy * mf);
  int cyv[2], cxv[2];
  T wy[2], wx[2];
  int ny, nx;
  if (fy & 1) { ny = 1; cyv[0] = (fy - 1) / 2; wy[0] = 1; } else {
    ny = 2; cyv[0] = fy / 2 - 1; cyv[1] = fy / 2; wy[0] = wy[1] = T(0.5);
  }
  if (fx & 1) { nx = 1; cxv[0] = (fx - 1) / 2; wx[0] = 1; } else {
    nx = 2; cxv[0] = fx / 2 - 1; cxv[1] = fx / 2; wx[0] = wx[1] = T(0.5);
  }
  const int k0 = blockIdx.y * kFreqChunk, k1 = min(K, k0 + kFreqChunk);
  for (int k = k0; k < k1; ++k) {
    const V* ck = xc + (long long)k * Jc;
    V acc = x[(long long)k * Jf + f];
    for (int a = 0; a < ny; ++a) {
      if (cyv[a] < 0 || cyv[a] >= mc) continue;
      for (int b = 0; b < nx; ++b) {
        if (cxv[b] < 0 || cxv[b] >= mc) continue;
        const T w = wy[a] * wx[b];
        const V v = ck[(long long)cyv[a] * mc + cxv[b]];
        acc.x += w * v.x;
        acc.y += w * v.y;
      }
    }
    x[(long long)k * Jf + f] = acc;
  }
}

// The 1 x 1 level: x = b / (lambda'_k M + tau K).
template <typename T>
__global__ void mg_coarsest_kernel(v2_t<T>* __restrict__ x, const v2_t<T>* __restrict__ b,
                                   MgArgs<T> a) {
  using V = v2_t<T>;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.K) return;
  const V lam = a.lam[k];
  const T sm = a.SM[4], sk = a.SK[4];
  const V D = {lam.x * sm + a.tau * sk, lam.y * sm};
  const T inv = T(1) / (D.x * D.x + D.y * D.y);
  const V c = cmulc(b[k], D);
  x[k] = {c.x * inv, c.y * inv};
}

// ------------------------------------------------- fused coarse-grid cycle
// The levels from lc down to the 1 x 1 grid of one V-cycle in a single
// kernel: one block per frequency, every level's x, b and r in shared memory,
// the steps separated by block barriers.  Each step is the per-point
// arithmetic of the per-level kernels above (same formulas, same order), so
// the result is the same bit for bit; it replaces 3 + pre + post launches per
// level, whose run time on these small grids is mostly launch latency.
constexpr int kMgCoarseMax = 8;        // fused levels at most
// threads of the fused cycle's one block per frequency: the block is alone
// on its SM (its levels fill the shared memory), so its warps are the SM's
// only latency hiding; FP32 (64 registers) takes 1024, FP64 (80) 512
template <typename T>
constexpr int kMgCoarseThreads = sizeof(T) == 4 ? 1024 : 512;

template <typename T>
struct MgCoarseArgs {
  const T* SM[kMgCoarseMax];
  const T* SK[kMgCoarseMax];
  int m[kMgCoarseMax];
  int nlev;                      // fused levels (the last is 1 x 1)
  const v2_t<T>* lam;
  T tau, omega;
  int pre, post;
  const v2_t<T>* b_in;           // [K][J_0] right-hand side of the first fused level
  v2_t<T>* x_out;                // [K][J_0] its V-cycle result
};

// xo = x + omega D^{-1} (b - B x) (ZERO: x = 0) at every point of one level
template <typename T, bool ZERO>
__device__ __forceinline__ void cc_smooth(v2_t<T>* xo, const v2_t<T>* x, const v2_t<T>* b,
                                          const T* SMl, const T* SKl, int m, v2_t<T> lam, T tau,
                                          T omega) {
  using V = v2_t<T>;
  MgArgs<T> a;
  a.SM = SMl;
  a.SK = SKl;
  a.m = m;
  a.J = (long long)m * m;
  for (long long q = threadIdx.x; q < a.J; q += kMgCoarseThreads<T>) {
    T sm[9], sk[9];
    int off[9];
    bool ok[9];
    load_point<T, false>(a, q, sm, sk, off, ok);
    const V D = {lam.x * sm[4] + tau * sk[4], lam.y * sm[4]};
    const T d2 = D.x * D.x + D.y * D.y;
    T inv;
    if constexpr (sizeof(T) == 8) inv = omega * rcp64(d2);
    else inv = omega / d2;
    V rr = b[q];
    V x0 = {0, 0};
    if (!ZERO) {
      x0 = x[q];
      const V bx = apply_b<T, false>(x, sm, sk, off, ok, lam, tau);
      rr = {rr.x - bx.x, rr.y - bx.y};
    }
    const V c = cmulc(rr, D);
    xo[q] = {x0.x + c.x * inv, x0.y + c.y * inv};
  }
}

template <typename T>
__device__ __forceinline__ void cc_residual(v2_t<T>* r, const v2_t<T>* x, const v2_t<T>* b,
                                            const T* SMl, const T* SKl, int m, v2_t<T> lam, T tau) {
  using V = v2_t<T>;
  MgArgs<T> a;
  a.SM = SMl;
  a.SK = SKl;
  a.m = m;
  a.J = (long long)m * m;
  for (long long q = threadIdx.x; q < a.J; q += kMgCoarseThreads<T>) {
    T sm[9], sk[9];
    int off[9];
    bool ok[9];
    load_point<T, false>(a, q, sm, sk, off, ok);
    const V bx = apply_b<T, false>(x, sm, sk, off, ok, lam, tau);
    const V bb = b[q];
    r[q] = {bb.x - bx.x, bb.y - bx.y};
  }
}

template <typename T>
__device__ __forceinline__ void cc_restrict(v2_t<T>* bc, const v2_t<T>* r, int mc, int mf) {
  using V = v2_t<T>;
  for (int c = threadIdx.x; c < mc * mc; c += kMgCoarseThreads<T>) {
    const int cy = c / mc, cx = c - cy * mc;
    const int f0 = (2 * cy + 1) * mf + (2 * cx + 1);
    V acc = {0, 0};
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const T w = (dy == 0 ? T(0.5) : T(0.25)) * (dx == 0 ? T(0.5) : T(0.25));
        const V v = r[f0 + dy * mf + dx];
        acc.x += w * v.x;
        acc.y += w * v.y;
      }
    }
    bc[c] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void cc_prolong_add(v2_t<T>* x, const v2_t<T>* xc, int mf, int mc) {
  using V = v2_t<T>;
  for (int f = threadIdx.x; f < mf * mf; f += kMgCoarseThreads<T>) {
    const int fy = f / mf, fx = f - fy * mf;
    int cyv[2], cxv[2];
    T wy[2], wx[2];
    int ny, nx;
    if (fy & 1) { ny = 1; cyv[0] = (fy - 1) / 2; wy[0] = 1; } else {
      ny = 2; cyv[0] = fy / 2 - 1; cyv[1] = fy / 2; wy[0] = wy[1] = T(0.5);
    }
    if (fx & 1) { nx = 1; cxv[0] = (fx - 1) / 2; wx[0] = 1; } else {
      nx = 2; cxv[0] = fx / 2 - 1; cxv[1] = fx / 2; wx[0] = wx[1] = T(0.5);
    }
    V acc = x[f];
    for (int a = 0; a < ny; ++a) {
      if (cyv[a] < 0 || cyv[a] >= mc) continue;
      for (int b = 0; b < nx; ++b) {
        if (cxv[b] < 0 || cxv[b] >= mc) continue;
        const T w = wy[a] * wx[b];
        const V v = xc[cyv[a] * mc + cxv[b]];
        acc.x += w * v.x;
        acc.y += w * v.y;
      }
    }
    x[f] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kMgCoarseThreads<T>)
mg_coarse_cycle_kernel(const __grid_constant__ MgCoarseArgs<T> a) {
  using V = v2_t<T>;
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  const int k = blockIdx.x;
  const V lam = a.lam[k];
  // per level: x, b, r (J_l complex each), levels one after another
  V* xs[kMgCoarseMax];
  V* bs[kMgCoarseMax];
  V* rs[kMgCoarseMax];
  {
    V* p = reinterpret_cast<V*>(smem_bytes);
#pragma unroll
    for (int l = 0; l < kMgCoarseMax; ++l) {
      if (l < a.nlev) {
        const int J = a.m[l] * a.m[l];
        xs[l] = p;
        bs[l] = p + J;
        rs[l] = p + 2 * J;
        p += 3 * J;
      }
    }
  }
  const int J0 = a.m[0] * a.m[0];
  for (int q = threadIdx.x; q < J0; q += kMgCoarseThreads<T>) bs[0][q] = a.b_in[(long long)k * J0 + q];
  __syncthreads();
  for (int l = 0; l + 1 < a.nlev; ++l) {
    cc_smooth<T, true>(xs[l], nullptr, bs[l], a.SM[l], a.SK[l], a.m[l], lam, a.tau, a.omega);
    __syncthreads();
    for (int s = 1; s < a.pre; ++s) {
      cc_smooth<T, false>(rs[l], xs[l], bs[l], a.SM[l], a.SK[l], a.m[l], lam, a.tau, a.omega);
      __syncthreads();
      V* t = xs[l];
      xs[l] = rs[l];
      rs[l] = t;
    }
    cc_residual<T>(rs[l], xs[l], bs[l], a.SM[l], a.SK[l], a.m[l], lam, a.tau);
    __syncthreads();
    cc_restrict<T>(bs[l + 1], rs[l], a.m[l + 1], a.m[l]);
    __syncthreads();
  }
  {
    // the 1 x 1 level: x = b / (lambda'_k M + tau K)
    const int l = a.nlev - 1;
    if (threadIdx.x == 0) {
      const T sm = a.SM[l][4], sk = a.SK[l][4];
      const V D = {lam.x * sm + a.tau * sk, lam.y * sm};
      const T inv = T(1) / (D.x * D.x + D.y * D.y);
      const V c = cmulc(bs[l][0], D);
      xs[l][0] = {c.x * inv, c.y * inv};
    }
    __syncthreads();
  }
  for (int l = a.nlev - 2; l >= 0; --l) {
    cc_prolong_add<T>(xs[l], xs[l + 1], a.m[l], a.m[l + 1]);
    __syncthreads();
    for (int s = 0; s < a.post; ++s) {
      cc_smooth<T, false>(rs[l], xs[l], bs[l], a.SM[l], a.SK[l], a.m[l], lam, a.tau, a.omega);
      __syncthreads();
      V* t = xs[l];
      xs[l] = rs[l];
      rs[l] = t;
    }
  }
  for (int q = threadIdx.x; q < J0; q += kMgCoarseThreads<T>) a.x_out[(long long)k * J0 + q] = xs[0][q];
}

// shared memory of the fused cycle from level l of the hierarchy down
size_t coarse_cycle_smem(const std::vector<MgLevel>& lv, int l, size_t vsize) {
  size_t b = 0;
  for (size_t i = l; i < lv.size(); ++i) b += 3 * (size_t)lv[i].J * vsize;
  return b;
}

// the first level the fused cycle takes: the largest below the finest grid
// (which keeps its 5-point kernels) whose x, b and r for it and every coarser
// level fit in kMgCoarseSmem bytes (at least two levels; -1: none, or the
// ILU smoother)
constexpr size_t kMgCoarseSmem = 160 * 1024;
int coarse_cycle_level(const bec_problem* p, size_t vsize) {
  const std::vector<MgLevel>& lv = p->mg.lv;
  const int L = (int)lv.size();
  if (p->mg.ilu || L < 3) return -1;
  for (int l = 1; l + 1 < L; ++l)
    if (L - l <= kMgCoarseMax && coarse_cycle_smem(lv, l, vsize) <= kMgCoarseSmem) return l;
  return -1;
}

// ---------------------------------------------------------------- ILU smoother
// The triangular recurrences of M run over the wavefronts t = x + 2y of a
// level's grid (x fastest): every lower neighbour of (x, y) (W, SE on t - 1;
// S on t - 2; SW on t - 3) lies on an earlier wavefront, every upper one (E,
// NW on t + 1; N on t + 2; NE on t + 3) on a later one.  One block per
// frequency walks the 3 (m - 1) + 1 wavefronts; a thread owns the points of
// a wavefront by their row y, and the values of the last three wavefronts
// stay in a shared-memory ring indexed by [t mod 4][y].
constexpr int kIluThreads = 128;

// entry s (stencil slot (dy+1)*3 + dx+1) of row q of lambda M + tau K
template <typename T>
__device__ __forceinline__ v2_t<T> ilu_coef(const MgArgs<T>& a, int s, long long q, v2_t<T> lam) {
  const T sm = a.SM[(long long)s * a.J + q], sk = a.SK[(long long)s * a.J + q];
  return {lam.x * sm + a.tau * sk, lam.y * sm};
}

template <typename T>
__device__ __forceinline__ v2_t<T> cinv(v2_t<T> d) {
  const T s = T(1) / (d.x * d.x + d.y * d.y);
  return {d.x * s, -d.y * s};
}

// 1/d_i, d_i = b_ii - sum over the lower neighbours j of b_ij b_ji / d_j
template <typename T>
__global__ void __launch_bounds__(kIluThreads)
ilu_setup_kernel(v2_t<T>* __restrict__ dinv, MgArgs<T> a) {
  using V = v2_t<T>;
  extern __shared__ __align__(16) unsigned char ilu_smem[];
  V* ring = reinterpret_cast<V*>(ilu_smem);     // [4][m]
  const int k = blockIdx.x, m = a.m;
  const V lam = a.lam[k];
  V* dk = dinv + (long long)k * a.J;
  for (int t = 0; t <= 3 * (m - 1); ++t) {
    const int ylo = t > m - 1 ? (t - (m - 1) + 1) / 2 : 0;
    const int yhi = min(m - 1, t / 2);
    for (int y = ylo + (int)threadIdx.x; y <= yhi; y += blockDim.x) {
      const int x = t - 2 * y;
      const long long q = (long long)y * m + x;
      V d = ilu_coef(a, 4, q, lam);
      // (slot at i, slot at j, neighbour offset, ring wavefront, ring row)
      if (x > 0) {                                   // W
        const V p = cmul(ilu_coef(a, 3, q, lam), ilu_coef(a, 5, q - 1, lam));
        const V e = cmul(p, ring[((t - 1) & 3) * m + y]);
        d.x -= e.x;
        d.y -= e.y;
      }
      if (y > 0) {
        const V p = cmul(ilu_coef(a, 1, q, lam), ilu_coef(a, 7, q - m, lam));   // S
        const V e = cmul(p, ring[((t - 2) & 3) * m + y - 1]);
        d.x -= e.x;
        d.y -= e.y;
        if (x + 1 < m) {                             // SE
          const V p2 = cmul(ilu_coef(a, 2, q, lam), ilu_coef(a, 6, q - m + 1, lam));
          const V e2 = cmul(p2, ring[((t - 1) & 3) * m + y - 1]);
          d.x -= e2.x;
          d.y -= e2.y;
        }
        if (x > 0) {                                 // SW
          const V p3 = cmul(ilu_coef(a, 0, q, lam), ilu_coef(a, 8, q - m - 1, lam));
          const V e3 = cmul(p3, ring[((t - 3) & 3) * m + y - 1]);
          d.x -= e3.x;
          d.y -= e3.y;
        }
      }
      const V di = cinv<T>(d);
      ring[(t & 3) * m + y] = di;
      dk[q] = di;
    }
    __syncthreads();
  }
}

// One ILU smoothing step for every frequency: z = M^{-1} rin, then x = z
// (ACC false) or x += z (ACC true); rin may alias work, which holds the
// forward result y between the two sweeps.  A thread owns one point per
// wavefront (the block has a thread per point of the longest one).  The
// operands that do not depend on the recurrence are staged by cp.async: at
// wavefront t a thread starts the copies of its point on wavefront t + 3
// (backward: t - 3) into its own slot of a 4-stage buffer in shared memory
// and waits only for the group of wavefront t.  Slot layout: the 8 neighbour entries, then rhs / forward value,
// 1/d and (ACC, backward) the old x.
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The slot stride (80 or 144 bytes, an odd number of 16-byte units) puts the
// slots of 8 consecutive threads on distinct 16-byte bank groups, so the
// 16-byte reads of a warp are free of bank conflicts.
template <typename T>
struct IluSlot {
  static constexpr int kNb = 0, kV = 8 * (int)sizeof(T), kD = kV + 2 * (int)sizeof(T),
                       kX = kD + 2 * (int)sizeof(T), kBytes = sizeof(T) == 4 ? 80 : 144;
};

// starts the copies of the operands of this thread's point on wavefront t
// (nothing when it has none), then commits one group
template <typename T, bool FWD, bool ACC>
__device__ __forceinline__ void ilu_issue(unsigned char* slot, int t, const MgArgs<T>& a,
                                          const v2_t<T>* src, const v2_t<T>* dk,
                                          const v2_t<T>* xk, const T* nb) {
  using S = IluSlot<T>;
  const int m = a.m;
  const int ylo = t > m - 1 ? (t - (m - 1) + 1) / 2 : 0;
  const int yhi = min(m - 1, t / 2);
  const int y = ylo + (int)threadIdx.x;
  if (t >= 0 && t <= 3 * (m - 1) && y <= yhi) {
    const long long q = (long long)y * m + (t - 2 * y);
    const unsigned char* e = reinterpret_cast<const unsigned char*>(nb + ((FWD ? 0 : a.J) + q) * 8);
#pragma unroll
    for (int i = 0; i < 8 * (int)sizeof(T) / 16; ++i) cp_async(slot + S::kNb + 16 * i, e + 16 * i, 16);
    cp_async(slot + S::kV, src + q, 2 * (int)sizeof(T));
    cp_async(slot + S::kD, dk + q, 2 * (int)sizeof(T));
    if (!FWD && ACC) cp_async(slot + S::kX, xk + q, 2 * (int)sizeof(T));
  }
  cp_async_commit();
}

// reads a slot with 16-byte loads: the 8 neighbour entries, the value and 1/d
template <typename T>
__device__ __forceinline__ void ilu_read(const unsigned char* sl, T (&e)[8], v2_t<T>& v,
                                         v2_t<T>& d) {
  using S = IluSlot<T>;
  if constexpr (sizeof(T) == 4) {
    const float4 a = reinterpret_cast<const float4*>(sl + S::kNb)[0];
    const float4 b = reinterpret_cast<const float4*>(sl + S::kNb)[1];
    const float4 c = *reinterpret_cast<const float4*>(sl + S::kV);   // v, then d
    e[0] = a.x; e[1] = a.y; e[2] = a.z; e[3] = a.w;
    e[4] = b.x; e[5] = b.y; e[6] = b.z; e[7] = b.w;
    v = make_float2(c.x, c.y);
    d = make_float2(c.z, c.w);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 u = reinterpret_cast<const double2*>(sl + S::kNb)[i];
      e[2 * i] = u.x;
      e[2 * i + 1] = u.y;
    }
    v = *reinterpret_cast<const double2*>(sl + S::kV);
    d = *reinterpret_cast<const double2*>(sl + S::kD);
  }
}

template <typename T, bool ACC>
__global__ void __launch_bounds__(512)
ilu_sweep_async_kernel(v2_t<T>* __restrict__ x, v2_t<T>* work, const v2_t<T>* rin,
                       const v2_t<T>* __restrict__ dinv, const T* __restrict__ nb, MgArgs<T> a) {
  using V = v2_t<T>;
  using S = IluSlot<T>;
  extern __shared__ __align__(16) unsigned char ilu_smem[];
  V* ring = reinterpret_cast<V*>(ilu_smem);                       // [4][m]
  const int k = blockIdx.x, m = a.m;
  unsigned char* stage = ilu_smem + ((4 * (size_t)m * sizeof(V) + 127) & ~(size_t)127);
  auto slot = [&](int t) { return stage + ((size_t)(t & 3) * blockDim.x + threadIdx.x) * S::kBytes; };
  const V lam = a.lam[k];
  const long long base = (long long)k * a.J;
  const V* dk = dinv + base;
  const V* rk = rin + base;
  V* wk = work + base;
  V* xk = x + base;
  const int tmax = 3 * (m - 1);
  auto coefv = [&](T sm, T sk) -> V { return {lam.x * sm + a.tau * sk, lam.y * sm}; };
  auto point = [&](int t, int& y, int& xx) {
    const int ylo = t > m - 1 ? (t - (m - 1) + 1) / 2 : 0;
    const int yhi = min(m - 1, t / 2);
    y = ylo + (int)threadIdx.x;
    xx = t - 2 * y;
    return y <= yhi;
  };
  // forward: (D + L) y = rin
  for (int t = 0; t < 3; ++t) ilu_issue<T, true, ACC>(slot(t), t, a, rk, dk, xk, nb);
  for (int t = 0; t <= tmax; ++t) {
    ilu_issue<T, true, ACC>(slot(t + 3), t + 3, a, rk, dk, xk, nb);
    cp_async_wait<3>();
    int y, xx;
    if (point(t, y, xx)) {
      const unsigned char* sl = slot(t);
      T e[8];
      V acc, dv;
      ilu_read<T>(sl, e, acc, dv);
      if (xx > 0) {                                   // W
        const V c = cmul(coefv(e[0], e[4]), ring[((t - 1) & 3) * m + y]);
        acc.x -= c.x;
        acc.y -= c.y;
      }
      if (y > 0) {
        const V c = cmul(coefv(e[1], e[5]), ring[((t - 2) & 3) * m + y - 1]);   // S
        acc.x -= c.x;
        acc.y -= c.y;
        if (xx + 1 < m) {                             // SE
          const V c2 = cmul(coefv(e[2], e[6]), ring[((t - 1) & 3) * m + y - 1]);
          acc.x -= c2.x;
          acc.y -= c2.y;
        }
        if (xx > 0) {                                 // SW
          const V c3 = cmul(coefv(e[3], e[7]), ring[((t - 3) & 3) * m + y - 1]);
          acc.x -= c3.x;
          acc.y -= c3.y;
        }
      }
      const V yv = cmul(acc, dv);
      ring[(t & 3) * m + y] = yv;
      wk[(long long)y * m + xx] = yv;
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  // backward: (D + U) z = D y, i.e. z = y - D^{-1} U z
  for (int i = 0; i < 3; ++i) ilu_issue<T, false, ACC>(slot(tmax - i), tmax - i, a, wk, dk, xk, nb);
  for (int t = tmax; t >= 0; --t) {
    ilu_issue<T, false, ACC>(slot(t - 3), t - 3, a, wk, dk, xk, nb);
    cp_async_wait<3>();
    int y, xx;
    if (point(t, y, xx)) {
      const unsigned char* sl = slot(t);
      T e[8];
      V yv, dv;
      ilu_read<T>(sl, e, yv, dv);
      V acc = {0, 0};
      if (xx + 1 < m) {                               // E
        const V c = cmul(coefv(e[0], e[4]), ring[((t + 1) & 3) * m + y]);
        acc.x += c.x;
        acc.y += c.y;
      }
      if (y + 1 < m) {
        const V c = cmul(coefv(e[1], e[5]), ring[((t + 2) & 3) * m + y + 1]);   // N
        acc.x += c.x;
        acc.y += c.y;
        if (xx > 0) {                                 // NW
          const V c2 = cmul(coefv(e[2], e[6]), ring[((t + 1) & 3) * m + y + 1]);
          acc.x += c2.x;
          acc.y += c2.y;
        }
        if (xx + 1 < m) {                             // NE
          const V c3 = cmul(coefv(e[3], e[7]), ring[((t + 3) & 3) * m + y + 1]);
          acc.x += c3.x;
          acc.y += c3.y;
        }
      }
      const V cc = cmul(acc, dv);
      const V z = {yv.x - cc.x, yv.y - cc.y};
      ring[(t & 3) * m + y] = z;
      const long long q = (long long)y * m + xx;
      if (ACC) {
        const V xo = *reinterpret_cast<const V*>(sl + S::kX);
        xk[q] = {xo.x + z.x, xo.y + z.y};
      } else {
        xk[q] = z;
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- host side
// Coarse 9-point stencil Ac = R Af P with R = P^T / 4 (layout [s][J], s =
// (dy+1)*3 + (dx+1)).  Fine point f of a 1D grid of mf points belongs to
// coarse node c with weight 1 if f = 2c+1 and 1/2 if f = 2c or 2c+2.
void galerkin(const std::vector<double>& Af, int mf, std::vector<double>& Ac, int mc) {
  const long long Jf = (long long)mf * mf, Jc = (long long)mc * mc;
  Ac.assign(9 * Jc, 0.0);
  auto w1 = [](int f, int c) -> double {
    if (f == 2 * c + 1) return 1.0;
    if (f == 2 * c || f == 2 * c + 2) return 0.5;
    return 0.0;
  };
  for (int cy = 0; cy < mc; ++cy)
    for (int cx = 0; cx < mc; ++cx) {
      const long long C = (long long)cy * mc + cx;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int fy = 2 * cy + 1 + dy, fx = 2 * cx + 1 + dx;
          const double wr = 0.25 * w1(fy, cy) * w1(fx, cx);
          const long long F = (long long)fy * mf + fx;
          for (int s = 0; s < 9; ++s) {
            const double av = Af[s * Jf + F];
            if (av == 0.0) continue;
            const int gy = fy + s / 3 - 1, gx = fx + s % 3 - 1;
            if (gy < 0 || gy >= mf || gx < 0 || gx >= mf) continue;
            for (int ey = -1; ey <= 1; ++ey)
              for (int ex = -1; ex <= 1; ++ex) {
                const int c2y = cy + ey, c2x = cx + ex;
                if (c2y < 0 || c2y >= mc || c2x < 0 || c2x >= mc) continue;
                const double wp = w1(gy, c2y) * w1(gx, c2x);
                if (wp == 0.0) continue;
                Ac[(long long)((ey + 1) * 3 + (ex + 1)) * Jc + C] += wr * av * wp;
              }
          }
        }
    }
}

template <typename T>
bec_status upload_stencil(void** dst, const std::vector<double>& src) {
  std::vector<T> h(src.begin(), src.end());
  cudaError_t e = cudaMalloc(dst, h.size() * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    set_error("cudaMalloc (multigrid stencils)");
    return BEC_ENOMEM;
  }
  BEC_CUDA_TRY(cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return BEC_OK;
}

template <typename T>
MgArgs<T> level_args(const bec_problem* p, const MgLevel& L) {
  MgArgs<T> a;
  a.SM = static_cast<const T*>(L.SM);
  a.SK = static_cast<const T*>(L.SK);
  a.lam = reinterpret_cast<const v2_t<T>*>(sizeof(T) == 8 ? (const void*)p->tab.lamf64
                                                          : (const void*)p->tab.lamf32);
  a.m = L.m;
  a.J = L.J;
  a.K = p->mg.K;
  a.tau = (T)p->tau;
  a.omega = (T)p->mg.omega;
  return a;
}

// Profile names per level (level 0 is the finest grid).
#define BEC_LV_NAMES(base)                                                                \
  {base "[l0]", base "[l1]", base "[l2]", base "[l3]", base "[l4]", base "[l5]", base "[l6]", \
   base "[l7]", base "[l8]", base "[l9]", base "[l10]"}
const char* const kSmooth0Names[] = BEC_LV_NAMES("mg_smooth0_kernel");
const char* const kSmoothNames[] = BEC_LV_NAMES("mg_smooth_kernel");
const char* const kResidNames[] = BEC_LV_NAMES("mg_residual_kernel");
const char* const kRestrictNames[] = BEC_LV_NAMES("mg_restrict_kernel");
const char* const kProlongNames[] = BEC_LV_NAMES("mg_prolong_add_kernel");
const char* const kIluSweepNames[] = BEC_LV_NAMES("ilu_sweep_kernel");
const char* const kIluSetupNames[] = BEC_LV_NAMES("ilu_setup_kernel");
#undef BEC_LV_NAMES

dim3 mg_grid(long long J, int K) {
  return dim3((unsigned)((J + kMgThreads - 1) / kMgThreads),
              (unsigned)((K + kFreqChunk - 1) / kFreqChunk));
}

#define BEC_TRY_MG(expr)         \
  do {                           \
    bec_status _s = (expr);      \
    if (_s != BEC_OK) return _s; \
  } while (0)

size_t ilu_smem_bytes(int m, size_t vsize) { return 4 * (size_t)m * vsize; }

// a thread per point of the longest wavefront ((m + 1) / 2 points), in warps
int ilu_threads(int m) { return (((m + 1) / 2 + 31) / 32) * 32; }

// the wavefront ring (rounded up to 128 bytes) plus 4 operand slots per thread
size_t ilu_sweep_smem_bytes(int m, int threads, size_t vsize) {
  const size_t slot = vsize == 8 ? 80 : 144;
  return ((4 * (size_t)m * vsize + 127) & ~(size_t)127) + 4 * (size_t)threads * slot;
}

// one ILU smoothing step on level l: x = M^{-1} rin (acc false) or x += M^{-1} rin;
// r is the work array (rin may be r)
template <typename T>
bec_status ilu_sweep(bec_problem* p, MgLevel& c, int l, const void* rin, bool acc) {
  using V = v2_t<T>;
  const MgArgs<T> a = level_args<T>(p, c);
  const int threads = ilu_threads(c.m);
  const size_t smem = ilu_sweep_smem_bytes(c.m, threads, sizeof(V));
  BEC_LAUNCH_BEGIN(p);
  if (acc)
    ilu_sweep_async_kernel<T, true><<<p->mg.K, threads, smem, p->stream>>>(
        static_cast<V*>(c.x), static_cast<V*>(c.r), static_cast<const V*>(rin),
        static_cast<const V*>(c.dinv), static_cast<const T*>(c.ilu_nb), a);
  else
    ilu_sweep_async_kernel<T, false><<<p->mg.K, threads, smem, p->stream>>>(
        static_cast<V*>(c.x), static_cast<V*>(c.r), static_cast<const V*>(rin),
        static_cast<const V*>(c.dinv), static_cast<const T*>(c.ilu_nb), a);
  BEC_LAUNCH_CHECK(p, kIluSweepNames[l]);
  return BEC_OK;
}

template <typename T>
bec_status ilu_setup_t(bec_problem* p) {
  using V = v2_t<T>;
  // the ring and the operand slots of the largest grid may exceed the default 48 KB
  const int m0 = p->mg.lv[0].m;
  const int big = (int)ilu_smem_bytes(m0, sizeof(V));
  if (big > 48 * 1024)
    BEC_CUDA_TRY(cudaFuncSetAttribute(ilu_setup_kernel<T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  const int bigs = (int)ilu_sweep_smem_bytes(m0, ilu_threads(m0), sizeof(V));
  if (bigs > 48 * 1024) {
    BEC_CUDA_TRY(cudaFuncSetAttribute(ilu_sweep_async_kernel<T, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bigs));
    BEC_CUDA_TRY(cudaFuncSetAttribute(ilu_sweep_async_kernel<T, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bigs));
  }
  for (size_t l = 0; l + 1 < p->mg.lv.size(); ++l) {
    MgLevel& c = p->mg.lv[l];
    BEC_LAUNCH_BEGIN(p);
    ilu_setup_kernel<T><<<p->mg.K, kIluThreads, ilu_smem_bytes(c.m, sizeof(V)), p->stream>>>(
        static_cast<V*>(c.dinv), level_args<T>(p, c));
    BEC_LAUNCH_CHECK(p, kIluSetupNames[l]);
  }
  return BEC_OK;
}

// f = tau fsrc + sum over the W, E, S, N boundary nodes of bcoef g (+ u0 in slice 1)
__global__ void build_rhs_dirichlet_kernel(const double* __restrict__ u0,
                                           const double* __restrict__ fsrc,
                                           const double* __restrict__ g,
                                           const double* __restrict__ bcoef,
                                           double* __restrict__ f, int m, int N, double tau) {
  const long long J = (long long)m * m, U = J * N;
  const long long n2 = (long long)(m + 2) * (m + 2);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < U;
       i += (long long)gridDim.x * blockDim.x) {
    const long long n = i / J, q = i - n * J;
    const int iy = (int)(q / m), ix = (int)(q - (long long)iy * m);
    const double* gn = g + n * n2;
    const long long node = (long long)(iy + 1) * (m + 2) + (ix + 1);
    double v = tau * fsrc[i];
    if (ix == 0) v = fma(bcoef[q], gn[node - 1], v);
    if (ix == m - 1) v = fma(bcoef[J + q], gn[node + 1], v);
    if (iy == 0) v = fma(bcoef[2 * J + q], gn[node - (m + 2)], v);
    if (iy == m - 1) v = fma(bcoef[3 * J + q], gn[node + (m + 2)], v);
    if (n == 0) v += u0[q];
    f[i] = v;
  }
}

// stencil launches of level l (level 0 takes the finest-grid specialisation)
template <typename T>
void residual_launch(int l, dim3 g, cudaStream_t st, v2_t<T>* r, const v2_t<T>* x,
                     const v2_t<T>* b, const MgArgs<T>& a) {
  if (l == 0) mg_residual_kernel<T, true><<<g, kMgThreads, 0, st>>>(r, x, b, a);
  else mg_residual_kernel<T, false><<<g, kMgThreads, 0, st>>>(r, x, b, a);
}

template <typename T, bool ZERO>
void smooth_launch(int l, dim3 g, cudaStream_t st, v2_t<T>* xo, const v2_t<T>* x,
                   const v2_t<T>* b, const MgArgs<T>& a) {
  if (l == 0) mg_smooth_kernel<T, ZERO, true><<<g, kMgThreads, 0, st>>>(xo, x, b, a);
  else mg_smooth_kernel<T, ZERO, false><<<g, kMgThreads, 0, st>>>(xo, x, b, a);
}

// One V-cycle for every frequency on levels l0.. (level l0's b -> its x).
template <typename T>
bec_status vcycle_t(bec_problem* p, int l0) {
  using V = v2_t<T>;
  std::vector<MgLevel>& lv = p->mg.lv;
  const int L = (int)lv.size();
  const int K = p->mg.K;
  // levels >= lc run in one fused kernel (the whole coarse part of the cycle)
  int lc = coarse_cycle_level(p, sizeof(V));
  if (lc >= 0 && lc < l0) lc = L - l0 >= 2 ? l0 : -1;
  const int ltop = lc >= 0 ? lc : L - 1;   // levels above it run per level
  for (int l = l0; l < ltop; ++l) {
    MgLevel& c = lv[l];
    const MgArgs<T> a = level_args<T>(p, c);
    const dim3 g = mg_grid(c.J, K);
    if (p->mg.ilu) {
      BEC_TRY_MG(ilu_sweep<T>(p, c, l, c.b, false));        // x = M^{-1} b
      for (int s = 1; s < p->mg.pre; ++s) {
        BEC_LAUNCH_BEGIN(p);
        residual_launch<T>(l, g, p->stream, 
            static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
        BEC_LAUNCH_CHECK(p, kResidNames[l]);
        BEC_TRY_MG(ilu_sweep<T>(p, c, l, c.r, true));
      }
    } else {
      BEC_LAUNCH_BEGIN(p);
      smooth_launch<T, true>(l, g, p->stream, 
          static_cast<V*>(c.x), nullptr, static_cast<const V*>(c.b), a);
      BEC_LAUNCH_CHECK(p, kSmooth0Names[l]);
      for (int s = 1; s < p->mg.pre; ++s) {
        BEC_LAUNCH_BEGIN(p);
        smooth_launch<T, false>(l, g, p->stream, 
            static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
        BEC_LAUNCH_CHECK(p, kSmoothNames[l]);
        std::swap(c.x, c.r);
      }
    }
    BEC_LAUNCH_BEGIN(p);
    residual_launch<T>(l, g, p->stream, 
        static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
    BEC_LAUNCH_CHECK(p, kResidNames[l]);
    MgLevel& n = lv[l + 1];
    BEC_LAUNCH_BEGIN(p);
    mg_restrict_kernel<T><<<mg_grid(n.J, K), kMgThreads, 0, p->stream>>>(
        static_cast<V*>(n.b), static_cast<const V*>(c.r), n.m, c.m, K);
    BEC_LAUNCH_CHECK(p, kRestrictNames[l]);
  }
  if (lc >= 0) {
    MgCoarseArgs<T> ca;
    ca.nlev = L - lc;
    for (int i = 0; i < ca.nlev; ++i) {
      ca.SM[i] = static_cast<const T*>(lv[lc + i].SM);
      ca.SK[i] = static_cast<const T*>(lv[lc + i].SK);
      ca.m[i] = lv[lc + i].m;
    }
    ca.lam = level_args<T>(p, lv[lc]).lam;
    ca.tau = (T)p->tau;
    ca.omega = (T)p->mg.omega;
    ca.pre = p->mg.pre;
    ca.post = p->mg.post;
    ca.b_in = static_cast<const V*>(lv[lc].b);
    ca.x_out = static_cast<V*>(lv[lc].x);
    const size_t smem = coarse_cycle_smem(lv, lc, sizeof(V));
    if (smem > 48 * 1024)
      BEC_CUDA_TRY(cudaFuncSetAttribute(mg_coarse_cycle_kernel<T>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BEC_LAUNCH_BEGIN(p);
    mg_coarse_cycle_kernel<T><<<K, kMgCoarseThreads<T>, smem, p->stream>>>(ca);
    BEC_LAUNCH_CHECK(p, "mg_coarse_cycle_kernel");
  } else {
    MgLevel& c = lv[L - 1];
    BEC_LAUNCH_BEGIN(p);
    mg_coarsest_kernel<T><<<(K + 127) / 128, 128, 0, p->stream>>>(
        static_cast<V*>(c.x), static_cast<const V*>(c.b), level_args<T>(p, c));
    BEC_LAUNCH_CHECK(p, "mg_coarsest_kernel");
  }
  for (int l = ltop - 1; l >= l0; --l) {
    MgLevel& c = lv[l];
    const MgLevel& n = lv[l + 1];
    const dim3 g = mg_grid(c.J, K);
    BEC_LAUNCH_BEGIN(p);
    mg_prolong_add_kernel<T><<<g, kMgThreads, 0, p->stream>>>(
        static_cast<V*>(c.x), static_cast<const V*>(n.x), c.m, n.m, K);
    BEC_LAUNCH_CHECK(p, kProlongNames[l]);
    const MgArgs<T> a = level_args<T>(p, c);
    for (int s = 0; s < p->mg.post; ++s) {
      if (p->mg.ilu) {
        BEC_LAUNCH_BEGIN(p);
        residual_launch<T>(l, g, p->stream, 
            static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
        BEC_LAUNCH_CHECK(p, kResidNames[l]);
        BEC_TRY_MG(ilu_sweep<T>(p, c, l, c.r, true));
        continue;
      }
      BEC_LAUNCH_BEGIN(p);
      smooth_launch<T, false>(l, g, p->stream, 
          static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
      BEC_LAUNCH_CHECK(p, kSmoothNames[l]);
      std::swap(c.x, c.r);
    }
  }
  return BEC_OK;
}

}  // namespace

bec_status mg_setup(bec_problem* p, const double* a_nodes, const double* wind) {
  const int m = p->m;
  const double side = p->desc.side == 0.0 ? 1.0 : p->desc.side;
  const double hp = side / (m + 1);   // physical spacing
  const double h2 = hp * hp;
  // node coefficients (constant a when a_nodes is null)
  const int n2 = m + 2;
  std::vector<double> an((size_t)n2 * n2, p->a);
  if (a_nodes != nullptr)
    for (size_t i = 0; i < an.size(); ++i) an[i] = a_nodes[i];
  for (double v : an)
    if (!(v > 0.0) || !std::isfinite(v)) {
      set_error("a_nodes must be finite and > 0");
      return BEC_EINVAL;
    }
  if (wind != nullptr)
    for (size_t i = 0; i < 2 * an.size(); ++i)
      if (!std::isfinite(wind[i])) {
        set_error("wind must be finite");
        return BEC_EINVAL;
      }
  // level 0: M = I, K = conservative 5-point with face means, plus the upwind
  // convection w_x (u - u_W)/h where w_x > 0, w_x (u_E - u)/h where w_x < 0
  // (likewise in y) when a wind is given; also the tau K row for the stencil
  // kernels, [centre, W, E, S, N] x J (off-diagonals negated), and -tau x the
  // couplings to boundary nodes for the Dirichlet right-hand side
  const long long J = (long long)m * m;
  std::vector<double> SM0(9 * J, 0.0), SK0(9 * J, 0.0), kc(5 * J, 0.0), bc(4 * J, 0.0);
  for (int iy = 0; iy < m; ++iy)
    for (int ix = 0; ix < m; ++ix) {
      const long long q = (long long)iy * m + ix;
      const int gy = iy + 1, gx = ix + 1;
      const size_t node = (size_t)gy * n2 + gx;
      const double ac = an[node];
      const double aw = 0.5 * (ac + an[node - 1]);
      const double ae = 0.5 * (ac + an[node + 1]);
      const double as = 0.5 * (ac + an[node - n2]);
      const double anf = 0.5 * (ac + an[node + n2]);
      const double wx = wind ? wind[node] : 0.0;
      const double wy = wind ? wind[an.size() + node] : 0.0;
      // row entries: centre, W, E, S, N
      const double cW = -aw / h2 - std::max(wx, 0.0) / hp;
      const double cE = -ae / h2 + std::min(wx, 0.0) / hp;
      const double cS = -as / h2 - std::max(wy, 0.0) / hp;
      const double cN = -anf / h2 + std::min(wy, 0.0) / hp;
      const double cC = (aw + ae + as + anf) / h2 + (std::fabs(wx) + std::fabs(wy)) / hp;
      SM0[4 * J + q] = 1.0;
      SK0[4 * J + q] = cC;
      if (ix > 0) SK0[3 * J + q] = cW;
      if (ix < m - 1) SK0[5 * J + q] = cE;
      if (iy > 0) SK0[1 * J + q] = cS;
      if (iy < m - 1) SK0[7 * J + q] = cN;
      kc[0 * J + q] = p->tau * cC;
      kc[1 * J + q] = ix > 0 ? -p->tau * cW : 0.0;
      kc[2 * J + q] = ix < m - 1 ? -p->tau * cE : 0.0;
      kc[3 * J + q] = iy > 0 ? -p->tau * cS : 0.0;
      kc[4 * J + q] = iy < m - 1 ? -p->tau * cN : 0.0;
      bc[0 * J + q] = ix == 0 ? -p->tau * cW : 0.0;
      bc[1 * J + q] = ix == m - 1 ? -p->tau * cE : 0.0;
      bc[2 * J + q] = iy == 0 ? -p->tau * cS : 0.0;
      bc[3 * J + q] = iy == m - 1 ? -p->tau * cN : 0.0;
    }
  for (int which = 0; which < 2; ++which) {
    double** dst = which == 0 ? &p->kcoef : &p->bcoef;
    const std::vector<double>& src = which == 0 ? kc : bc;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), src.size() * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      *dst = nullptr;
      set_error("cudaMalloc (coefficients)");
      return BEC_ENOMEM;
    }
    BEC_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice));
  }

  const bool fp64 = p->desc.precision == BEC_PC_FP64;
  const size_t csz = fp64 ? sizeof(double2) : sizeof(float2);
  p->mg.K = p->N / 2 + 1;
  if (m > 2047) return BEC_EINVAL;   // at most 11 levels (profile names)
  std::vector<double> SM = SM0, SK = SK0;
  int ml = m;
  while (true) {
    MgLevel L;
    L.m = ml;
    L.J = (long long)ml * ml;
    bec_status s = fp64 ? upload_stencil<double>(&L.SM, SM) : upload_stencil<float>(&L.SM, SM);
    if (s == BEC_OK) s = fp64 ? upload_stencil<double>(&L.SK, SK) : upload_stencil<float>(&L.SK, SK);
    if (s == BEC_OK && p->mg.ilu && ml > 1) {
      // the ILU sweeps' neighbour entries, [dir][q][M W, S, SE, SW | K same]
      // (dir 0) and [M E, N, NW, NE | K same] (dir 1)
      const int lo[4] = {3, 1, 2, 0}, up[4] = {5, 7, 6, 8};
      std::vector<double> nbv((size_t)16 * L.J);
      for (long long q = 0; q < L.J; ++q)
        for (int i = 0; i < 4; ++i) {
          nbv[(size_t)q * 8 + i] = SM[(size_t)lo[i] * L.J + q];
          nbv[(size_t)q * 8 + 4 + i] = SK[(size_t)lo[i] * L.J + q];
          nbv[(size_t)(L.J + q) * 8 + i] = SM[(size_t)up[i] * L.J + q];
          nbv[(size_t)(L.J + q) * 8 + 4 + i] = SK[(size_t)up[i] * L.J + q];
        }
      s = fp64 ? upload_stencil<double>(&L.ilu_nb, nbv) : upload_stencil<float>(&L.ilu_nb, nbv);
    }
    const size_t bytes = (size_t)p->mg.K * L.J * csz;
    void* bufs[4] = {nullptr, nullptr, nullptr, nullptr};
    const int nbuf = (p->mg.ilu && ml > 1) ? 4 : 3;   // + 1/D of the ILU smoother
    for (int i = 0; i < nbuf && s == BEC_OK; ++i) {
      if (cudaMalloc(&bufs[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc (multigrid levels)");
        s = BEC_ENOMEM;
      }
    }
    L.x = bufs[0];
    L.b = bufs[1];
    L.r = bufs[2];
    L.dinv = bufs[3];
    p->mg.lv.push_back(L);
    if (s != BEC_OK) return s;
    if (ml == 1) break;
    const int mc = (ml - 1) / 2;
    std::vector<double> SMc, SKc;
    galerkin(SM, ml, SMc, mc);
    galerkin(SK, ml, SKc, mc);
    SM.swap(SMc);
    SK.swap(SKc);
    ml = mc;
  }
  return BEC_OK;
}

void mg_free(bec_problem* p) {
  for (MgLevel& L : p->mg.lv) {
    void* ptrs[] = {L.SM, L.SK, L.x, L.b, L.r, L.dinv, L.ilu_nb};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
  p->mg.lv.clear();
  if (p->kcoef) cudaFree(p->kcoef);
  p->kcoef = nullptr;
  if (p->bcoef) cudaFree(p->bcoef);
  p->bcoef = nullptr;
}

bec_status mg_residual_level0(bec_problem* p, void* r, const void* x, const void* b) {
  const MgLevel& L = p->mg.lv[0];
  if (p->desc.precision == BEC_PC_FP64) {
    BEC_LAUNCH_BEGIN(p);
    mg_residual_kernel<double, true><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
        static_cast<double2*>(r), static_cast<const double2*>(x), static_cast<const double2*>(b),
        level_args<double>(p, L));
  } else {
    BEC_LAUNCH_BEGIN(p);
    mg_residual_kernel<float, true><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
        static_cast<float2*>(r), static_cast<const float2*>(x), static_cast<const float2*>(b),
        level_args<float>(p, L));
  }
  BEC_LAUNCH_CHECK(p, "mg_residual_kernel[l0]");
  return BEC_OK;
}

bec_status mg_smooth_level0(bec_problem* p, void* xo, const void* x, const void* b) {
  const MgLevel& L = p->mg.lv[0];
  if (p->desc.precision == BEC_PC_FP64) {
    BEC_LAUNCH_BEGIN(p);
    mg_smooth_kernel<double, false, true><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
        static_cast<double2*>(xo), static_cast<const double2*>(x), static_cast<const double2*>(b),
        level_args<double>(p, L));
  } else {
    BEC_LAUNCH_BEGIN(p);
    mg_smooth_kernel<float, false, true><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
        static_cast<float2*>(xo), static_cast<const float2*>(x), static_cast<const float2*>(b),
        level_args<float>(p, L));
  }
  BEC_LAUNCH_CHECK(p, "mg_smooth_kernel[l0]");
  return BEC_OK;
}

bec_status mg_ilu_setup(bec_problem* p) {
  if (p->desc.precision == BEC_PC_FP64) return ilu_setup_t<double>(p);
  return ilu_setup_t<float>(p);
}

bec_status launch_build_rhs_dirichlet(bec_problem* p, const double* u0, const double* fsrc,
                                      const double* g, double* f) {
  BEC_LAUNCH_BEGIN(p);
  build_rhs_dirichlet_kernel<<<4 * 152, 256, 0, p->stream>>>(u0, fsrc, g, p->bcoef, f, p->m, p->N,
                                                             p->tau);
  BEC_LAUNCH_CHECK(p, "build_rhs_dirichlet_kernel");
  return BEC_OK;
}

bec_status mg_vcycle(bec_problem* p) { return mg_vcycle_from(p, 0); }

bec_status mg_vcycle_from(bec_problem* p, int l0) {
  NvtxRange range("bec V-cycle");
  if (l0 < 0 || l0 + 1 >= (int)p->mg.lv.size()) return BEC_EINVAL;
  if (p->desc.precision == BEC_PC_FP64) return vcycle_t<double>(p, l0);
  return vcycle_t<float>(p, l0);
}

bec_status mg_residual_level(bec_problem* p, int l, void* r, const void* x, const void* b) {
  if (l == 0) return mg_residual_level0(p, r, x, b);
  const MgLevel& L = p->mg.lv[l];
  const dim3 g = mg_grid(L.J, p->mg.K);
  BEC_LAUNCH_BEGIN(p);
  if (p->desc.precision == BEC_PC_FP64)
    residual_launch<double>(l, g, p->stream, static_cast<double2*>(r),
                            static_cast<const double2*>(x), static_cast<const double2*>(b),
                            level_args<double>(p, L));
  else
    residual_launch<float>(l, g, p->stream, static_cast<float2*>(r), static_cast<const float2*>(x),
                           static_cast<const float2*>(b), level_args<float>(p, L));
  BEC_LAUNCH_CHECK(p, kResidNames[l]);
  return BEC_OK;
}

bec_status mg_restrict_to(bec_problem* p, int lf, void* bc, const void* rf) {
  const MgLevel& f = p->mg.lv[lf];
  const MgLevel& c = p->mg.lv[lf + 1];
  const int K = p->mg.K;
  BEC_LAUNCH_BEGIN(p);
  if (p->desc.precision == BEC_PC_FP64)
    mg_restrict_kernel<double><<<mg_grid(c.J, K), kMgThreads, 0, p->stream>>>(
        static_cast<double2*>(bc), static_cast<const double2*>(rf), c.m, f.m, K);
  else
    mg_restrict_kernel<float><<<mg_grid(c.J, K), kMgThreads, 0, p->stream>>>(
        static_cast<float2*>(bc), static_cast<const float2*>(rf), c.m, f.m, K);
  BEC_LAUNCH_CHECK(p, kRestrictNames[lf]);
  return BEC_OK;
}

}  // namespace bec

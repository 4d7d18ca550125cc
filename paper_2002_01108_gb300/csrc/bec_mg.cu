// Multigrid route of P_eps^{-1} (Sec. 4: "efficient spatial solvers, such as
// a multigrid method"; Example 2 of Sec. 5: one V-cycle per shifted system,
// one pre- and one post-smoothing step, piecewise-linear interpolation and
// its transpose).  For every frequency k <= N/2 the V-cycle approximates
//     (lambda'_k M_l + tau K_l) x = b
// on levels l = 0..L-1 with m_0 = nx, m_{l+1} = (m_l - 1)/2, down to 1 x 1:
//   * M_0 = I and K_0 = the conservative 5-point -div(a grad) / h^2;
//   * P_l bilinear interpolation, R_l = P_l^T / 4 (full weighting);
//   * M_{l+1} = R_l M_l P_l and K_{l+1} = R_l K_l P_l (Galerkin, 9-point);
//   * damped Jacobi, x <- x + omega D^{-1} (b - B x), D = diag(B);
//   * the 1 x 1 level is solved exactly.
// The Galerkin stencils are real and do not depend on k; they are built once
// on the host and read by every frequency.  Each thread owns one grid point
// and walks a chunk of frequencies with its 18 stencil coefficients in
// registers.
#include <cuda_runtime.h>

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

// B x at point q for frequency k with the stencil coefficients in registers.
template <typename T>
__device__ __forceinline__ v2_t<T> apply_b(const v2_t<T>* __restrict__ xk, const T (&sm)[9],
                                           const T (&sk)[9], const int (&off)[9],
                                           const bool (&ok)[9], v2_t<T> lam, T tau) {
  using V = v2_t<T>;
  V am = {0, 0}, ak = {0, 0};
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    if (ok[s]) {
      const V xv = xk[off[s]];
      am.x += sm[s] * xv.x;
      am.y += sm[s] * xv.y;
      ak.x += sk[s] * xv.x;
      ak.y += sk[s] * xv.y;
    }
  }
  const V lm = cmul(lam, am);
  return {lm.x + tau * ak.x, lm.y + tau * ak.y};
}

template <typename T>
__device__ __forceinline__ void load_point(const MgArgs<T>& a, long long q, T (&sm)[9], T (&sk)[9],
                                           int (&off)[9], bool (&ok)[9]) {
  const int iy = (int)(q / a.m), ix = (int)(q - (long long)iy * a.m);
#pragma unroll
  for (int s = 0; s < 9; ++s) {
    const int dy = s / 3 - 1, dx = s % 3 - 1;
    ok[s] = iy + dy >= 0 && iy + dy < a.m && ix + dx >= 0 && ix + dx < a.m;
    off[s] = (int)q + dy * a.m + dx;
    sm[s] = a.SM[(long long)s * a.J + q];
    sk[s] = a.SK[(long long)s * a.J + q];
  }
}

// ZERO: xo = omega D^{-1} b (one sweep from x = 0);
// else: xo = x + omega D^{-1} (b - B x)      (xo != x)
template <typename T, bool ZERO>
__global__ void __launch_bounds__(kMgThreads)
mg_smooth_kernel(v2_t<T>* __restrict__ xo, const v2_t<T>* __restrict__ x,
                 const v2_t<T>* __restrict__ b, MgArgs<T> a) {
  using V = v2_t<T>;
  const long long q = (long long)blockIdx.x * kMgThreads + threadIdx.x;
  if (q >= a.J) return;
  T sm[9], sk[9];
  int off[9];
  bool ok[9];
  load_point(a, q, sm, sk, off, ok);
  const int k0 = blockIdx.y * kFreqChunk, k1 = min(a.K, k0 + kFreqChunk);
  for (int k = k0; k < k1; ++k) {
    const long long base = (long long)k * a.J;
    const V lam = a.lam[k];
    const V D = {lam.x * sm[4] + a.tau * sk[4], lam.y * sm[4]};
    const T inv = a.omega / (D.x * D.x + D.y * D.y);
    V rr = b[base + q];
    V x0 = {0, 0};
    if (!ZERO) {
      x0 = x[base + q];
      const V bx = apply_b<T>(x + base, sm, sk, off, ok, lam, a.tau);
      rr = {rr.x - bx.x, rr.y - bx.y};
    }
    const V c = cmulc(rr, D);     // rr conj(D); times omega / |D|^2 = omega rr / D
    xo[base + q] = {x0.x + c.x * inv, x0.y + c.y * inv};
  }
}

// r = b - B x
template <typename T>
__global__ void __launch_bounds__(kMgThreads)
mg_residual_kernel(v2_t<T>* __restrict__ r, const v2_t<T>* __restrict__ x,
                   const v2_t<T>* __restrict__ b, MgArgs<T> a) {
  using V = v2_t<T>;
  const long long q = (long long)blockIdx.x * kMgThreads + threadIdx.x;
  if (q >= a.J) return;
  T sm[9], sk[9];
  int off[9];
  bool ok[9];
  load_point(a, q, sm, sk, off, ok);
  const int k0 = blockIdx.y * kFreqChunk, k1 = min(a.K, k0 + kFreqChunk);
  for (int k = k0; k < k1; ++k) {
    const long long base = (long long)k * a.J;
    const V bx = apply_b<T>(x + base, sm, sk, off, ok, a.lam[k], a.tau);
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
#undef BEC_LV_NAMES

dim3 mg_grid(long long J, int K) {
  return dim3((unsigned)((J + kMgThreads - 1) / kMgThreads),
              (unsigned)((K + kFreqChunk - 1) / kFreqChunk));
}

template <typename T>
bec_status vcycle_t(bec_problem* p) {
  using V = v2_t<T>;
  std::vector<MgLevel>& lv = p->mg.lv;
  const int L = (int)lv.size();
  const int K = p->mg.K;
  for (int l = 0; l + 1 < L; ++l) {
    MgLevel& c = lv[l];
    const MgArgs<T> a = level_args<T>(p, c);
    const dim3 g = mg_grid(c.J, K);
    BEC_LAUNCH_BEGIN(p);
    mg_smooth_kernel<T, true><<<g, kMgThreads, 0, p->stream>>>(
        static_cast<V*>(c.x), nullptr, static_cast<const V*>(c.b), a);
    BEC_LAUNCH_CHECK(p, kSmooth0Names[l]);
    for (int s = 1; s < p->mg.pre; ++s) {
      BEC_LAUNCH_BEGIN(p);
      mg_smooth_kernel<T, false><<<g, kMgThreads, 0, p->stream>>>(
          static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
      BEC_LAUNCH_CHECK(p, kSmoothNames[l]);
      std::swap(c.x, c.r);
    }
    BEC_LAUNCH_BEGIN(p);
    mg_residual_kernel<T><<<g, kMgThreads, 0, p->stream>>>(
        static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
    BEC_LAUNCH_CHECK(p, kResidNames[l]);
    MgLevel& n = lv[l + 1];
    BEC_LAUNCH_BEGIN(p);
    mg_restrict_kernel<T><<<mg_grid(n.J, K), kMgThreads, 0, p->stream>>>(
        static_cast<V*>(n.b), static_cast<const V*>(c.r), n.m, c.m, K);
    BEC_LAUNCH_CHECK(p, kRestrictNames[l]);
  }
  {
    MgLevel& c = lv[L - 1];
    BEC_LAUNCH_BEGIN(p);
    mg_coarsest_kernel<T><<<(K + 127) / 128, 128, 0, p->stream>>>(
        static_cast<V*>(c.x), static_cast<const V*>(c.b), level_args<T>(p, c));
    BEC_LAUNCH_CHECK(p, "mg_coarsest_kernel");
  }
  for (int l = L - 2; l >= 0; --l) {
    MgLevel& c = lv[l];
    const MgLevel& n = lv[l + 1];
    const dim3 g = mg_grid(c.J, K);
    BEC_LAUNCH_BEGIN(p);
    mg_prolong_add_kernel<T><<<g, kMgThreads, 0, p->stream>>>(
        static_cast<V*>(c.x), static_cast<const V*>(n.x), c.m, n.m, K);
    BEC_LAUNCH_CHECK(p, kProlongNames[l]);
    const MgArgs<T> a = level_args<T>(p, c);
    for (int s = 0; s < p->mg.post; ++s) {
      BEC_LAUNCH_BEGIN(p);
      mg_smooth_kernel<T, false><<<g, kMgThreads, 0, p->stream>>>(
          static_cast<V*>(c.r), static_cast<const V*>(c.x), static_cast<const V*>(c.b), a);
      BEC_LAUNCH_CHECK(p, kSmoothNames[l]);
      std::swap(c.x, c.r);
    }
  }
  return BEC_OK;
}

}  // namespace

bec_status mg_setup(bec_problem* p, const double* a_nodes) {
  const int m = p->m;
  const double h2 = p->h * p->h;
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
  // level 0: M = I, K = conservative 5-point with face means; also the tau K
  // row for the stencil kernels: [centre, W, E, S, N] x J
  const long long J = (long long)m * m;
  std::vector<double> SM0(9 * J, 0.0), SK0(9 * J, 0.0), kc(5 * J, 0.0);
  for (int iy = 0; iy < m; ++iy)
    for (int ix = 0; ix < m; ++ix) {
      const long long q = (long long)iy * m + ix;
      const int gy = iy + 1, gx = ix + 1;
      const double ac = an[(size_t)gy * n2 + gx];
      const double aw = 0.5 * (ac + an[(size_t)gy * n2 + gx - 1]);
      const double ae = 0.5 * (ac + an[(size_t)gy * n2 + gx + 1]);
      const double as = 0.5 * (ac + an[(size_t)(gy - 1) * n2 + gx]);
      const double anf = 0.5 * (ac + an[(size_t)(gy + 1) * n2 + gx]);
      SM0[4 * J + q] = 1.0;
      SK0[4 * J + q] = (aw + ae + as + anf) / h2;
      if (ix > 0) SK0[3 * J + q] = -aw / h2;
      if (ix < m - 1) SK0[5 * J + q] = -ae / h2;
      if (iy > 0) SK0[1 * J + q] = -as / h2;
      if (iy < m - 1) SK0[7 * J + q] = -anf / h2;
      kc[0 * J + q] = p->tau * (aw + ae + as + anf) / h2;
      kc[1 * J + q] = ix > 0 ? p->tau * aw / h2 : 0.0;
      kc[2 * J + q] = ix < m - 1 ? p->tau * ae / h2 : 0.0;
      kc[3 * J + q] = iy > 0 ? p->tau * as / h2 : 0.0;
      kc[4 * J + q] = iy < m - 1 ? p->tau * anf / h2 : 0.0;
    }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->kcoef), kc.size() * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    p->kcoef = nullptr;
    set_error("cudaMalloc (coefficients)");
    return BEC_ENOMEM;
  }
  BEC_CUDA_TRY(cudaMemcpy(p->kcoef, kc.data(), kc.size() * sizeof(double), cudaMemcpyHostToDevice));

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
    const size_t bytes = (size_t)p->mg.K * L.J * csz;
    void* bufs[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3 && s == BEC_OK; ++i) {
      if (cudaMalloc(&bufs[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc (multigrid levels)");
        s = BEC_ENOMEM;
      }
    }
    L.x = bufs[0];
    L.b = bufs[1];
    L.r = bufs[2];
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
    void* ptrs[] = {L.SM, L.SK, L.x, L.b, L.r};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
  p->mg.lv.clear();
  if (p->kcoef) cudaFree(p->kcoef);
  p->kcoef = nullptr;
}

bec_status mg_residual_level0(bec_problem* p, void* r, const void* x, const void* b) {
  const MgLevel& L = p->mg.lv[0];
  if (p->desc.precision == BEC_PC_FP64) {
    BEC_LAUNCH_BEGIN(p);
    mg_residual_kernel<double><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
        static_cast<double2*>(r), static_cast<const double2*>(x), static_cast<const double2*>(b),
        level_args<double>(p, L));
  } else {
    BEC_LAUNCH_BEGIN(p);
    mg_residual_kernel<float><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
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
    mg_smooth_kernel<double, false><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
        static_cast<double2*>(xo), static_cast<const double2*>(x), static_cast<const double2*>(b),
        level_args<double>(p, L));
  } else {
    BEC_LAUNCH_BEGIN(p);
    mg_smooth_kernel<float, false><<<mg_grid(L.J, p->mg.K), kMgThreads, 0, p->stream>>>(
        static_cast<float2*>(xo), static_cast<const float2*>(x), static_cast<const float2*>(b),
        level_args<float>(p, L));
  }
  BEC_LAUNCH_CHECK(p, "mg_smooth_kernel[l0]");
  return BEC_OK;
}

bec_status mg_vcycle(bec_problem* p) {
  NvtxRange range("bec V-cycle");
  if (p->desc.precision == BEC_PC_FP64) return vcycle_t<double>(p);
  return vcycle_t<float>(p);
}

}  // namespace bec

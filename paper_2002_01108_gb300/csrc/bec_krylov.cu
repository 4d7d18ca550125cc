// FP64 Krylov kernels for restarted GMRES / FGMRES on the device: block
// multi-dot and multi-axpy for classical Gram-Schmidt (applied twice), norms,
// scaling, and the one-thread Hessenberg / Givens / least-squares updates.
// Every reduction writes one partial per block of a fixed grid and is summed
// in a fixed order, so results are bitwise reproducible run to run.
#include <cuda_runtime.h>

#include "bec_internal.h"

namespace bec {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kDotChunk = 32;   // vectors per multi-dot launch

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// partials[v * gridDim.x + b] = sum over block b of V_v . w, v < nv <= K.
// U is even (N is a power of two), so double2 loads are aligned.
template <int K>
__global__ void __launch_bounds__(kThreads)
mdot_kernel(const double* __restrict__ Vb, int nv, long long U, const double* __restrict__ w,
            double* __restrict__ partials) {
  double acc[K];
#pragma unroll
  for (int v = 0; v < K; ++v) acc[v] = 0.0;
  const long long U2 = U / 2;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < U2;
       i += (long long)gridDim.x * kThreads) {
    const double2 wv = w2[i];
#pragma unroll
    for (int v = 0; v < K; ++v) {
      if (v < nv) {
        const double2 x = reinterpret_cast<const double2*>(Vb + (long long)v * U)[i];
        acc[v] = fma(x.x, wv.x, fma(x.y, wv.y, acc[v]));
      }
    }
  }
  __shared__ double red[kWarps][K];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < K; ++v) {
    const double s = warp_sum(acc[v]);
    if (lane == 0) red[warp][v] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x < nv) {
    double s = 0.0;
#pragma unroll
    for (int wi = 0; wi < kWarps; ++wi) s += red[wi][threadIdx.x];
    partials[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

// out[v] = sum_b partials[v * nb + b]   (block v, fixed tree order)
__global__ void __launch_bounds__(kThreads)
finish_rows_kernel(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  __shared__ double s[kThreads];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) a += partials[(long long)blockIdx.x * nb + b];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// y += sign * sum_{v < nv} coef[v] V_v; partials[b] = block sum of y^2 (if non-null)
__global__ void __launch_bounds__(kThreads)
maxpy_kernel(double* __restrict__ y, const double* __restrict__ Vb, int nv, long long U,
             const double* __restrict__ coef, double sign, double* __restrict__ partials) {
  __shared__ double c[kMaxRestart + 2];
  for (int v = threadIdx.x; v < nv; v += kThreads) c[v] = sign * coef[v];
  __syncthreads();
  const long long U2 = U / 2;
  double2* y2 = reinterpret_cast<double2*>(y);
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < U2;
       i += (long long)gridDim.x * kThreads) {
    double2 a = y2[i];
    for (int v = 0; v < nv; ++v) {
      const double2 x = reinterpret_cast<const double2*>(Vb + (long long)v * U)[i];
      a.x = fma(c[v], x.x, a.x);
      a.y = fma(c[v], x.y, a.y);
    }
    y2[i] = a;
    nrm = fma(a.x, a.x, fma(a.y, a.y, nrm));
  }
  if (partials == nullptr) return;
  __shared__ double red[kWarps];
  const double s = warp_sum(nrm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wi = 0; wi < kWarps; ++wi) t += red[wi];
    partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads)
sumsq_kernel(const double* __restrict__ x, long long U, double* __restrict__ partials) {
  const long long U2 = U / 2;
  const double2* x2 = reinterpret_cast<const double2*>(x);
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < U2;
       i += (long long)gridDim.x * kThreads) {
    const double2 a = x2[i];
    nrm = fma(a.x, a.x, fma(a.y, a.y, nrm));
  }
  __shared__ double red[kWarps];
  const double s = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wi = 0; wi < kWarps; ++wi) t += red[wi];
    partials[blockIdx.x] = t;
  }
}

// scal[slot] = sqrt(sum partials)
__global__ void __launch_bounds__(kThreads)
finish_sqrt_kernel(const double* __restrict__ partials, int nb, double* __restrict__ scal,
                   int slot) {
  __shared__ double s[kThreads];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) a += partials[b];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) scal[slot] = sqrt(s[0]);
}

__global__ void __launch_bounds__(kThreads)
scale_by_inv_kernel(const double* __restrict__ x, double* __restrict__ y, long long U,
                    const double* __restrict__ scal, int slot) {
  const double inv = 1.0 / scal[slot];
  const long long U2 = U / 2;
  const double2* x2 = reinterpret_cast<const double2*>(x);
  double2* y2 = reinterpret_cast<double2*>(y);
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < U2;
       i += (long long)gridDim.x * kThreads) {
    const double2 a = x2[i];
    y2[i] = make_double2(a.x * inv, a.y * inv);
  }
}

// Column j of the Arnoldi Hessenberg matrix (leading dimension ldh), the
// Givens rotations that keep it upper triangular, and the rotated
// right-hand side g whose entry j+1 is the GMRES residual norm.
__global__ void hessenberg_kernel(double* __restrict__ H, int ldh, int j,
                                  const double* __restrict__ h1, const double* __restrict__ h2,
                                  double* __restrict__ scal, int norm_slot, int res_slot,
                                  double* __restrict__ cs, double* __restrict__ sn,
                                  double* __restrict__ g) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (long long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  col[j + 1] = scal[norm_slot];
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[j], b = col[j + 1];
  double c = 1.0, s = 0.0;
  if (b != 0.0) {
    const double r = hypot(a, b);
    c = a / r;
    s = b / r;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = c * a + s * b;
  col[j + 1] = 0.0;
  const double gj = g[j];
  g[j] = c * gj;
  g[j + 1] = -s * gj;
  scal[res_slot] = fabs(g[j + 1]);
}

__global__ void gmres_start_kernel(double* __restrict__ g, int len,
                                   const double* __restrict__ scal, int slot) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = i == 0 ? scal[slot] : 0.0;
}

// back substitution y = R^{-1} g with R = H(0:k, 0:k) upper triangular
__global__ void least_squares_kernel(const double* __restrict__ H, int ldh, int k,
                                     const double* __restrict__ g, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(long long)c * ldh + i] * y[c];
    y[i] = s / H[(long long)i * ldh + i];
  }
}

}  // namespace

bec_status launch_mdot(bec_problem* p, const double* Vb, int nv, const double* w,
                       double* hcol) {
  const int nb = kReduceBlocks;
  for (int v0 = 0; v0 < nv; v0 += kDotChunk) {
    const int cnt = nv - v0 < kDotChunk ? nv - v0 : kDotChunk;
    const double* base = Vb + (long long)v0 * p->U;
    BEC_LAUNCH_BEGIN(p);
    if (cnt <= 4)
      mdot_kernel<4><<<nb, kThreads, 0, p->stream>>>(base, cnt, p->U, w, p->partials);
    else if (cnt <= 8)
      mdot_kernel<8><<<nb, kThreads, 0, p->stream>>>(base, cnt, p->U, w, p->partials);
    else if (cnt <= 16)
      mdot_kernel<16><<<nb, kThreads, 0, p->stream>>>(base, cnt, p->U, w, p->partials);
    else
      mdot_kernel<32><<<nb, kThreads, 0, p->stream>>>(base, cnt, p->U, w, p->partials);
    BEC_LAUNCH_CHECK(p, "mdot_kernel");
    BEC_LAUNCH_BEGIN(p);
    finish_rows_kernel<<<cnt, kThreads, 0, p->stream>>>(p->partials, nb, hcol + v0);
    BEC_LAUNCH_CHECK(p, "finish_rows_kernel");
  }
  return BEC_OK;
}

bec_status launch_maxpy(bec_problem* p, double* w, const double* Vb, int nv, const double* coef,
                        double sign, int norm_slot) {
  double* part = norm_slot >= 0 ? p->partials : nullptr;
  BEC_LAUNCH_BEGIN(p);
  maxpy_kernel<<<kReduceBlocks, kThreads, 0, p->stream>>>(w, Vb, nv, p->U, coef, sign, part);
  BEC_LAUNCH_CHECK(p, "maxpy_kernel");
  if (norm_slot >= 0) {
    BEC_LAUNCH_BEGIN(p);
    finish_sqrt_kernel<<<1, kThreads, 0, p->stream>>>(p->partials, kReduceBlocks, p->scal,
                                                       norm_slot);
    BEC_LAUNCH_CHECK(p, "finish_sqrt_kernel");
  }
  return BEC_OK;
}

bec_status launch_norm(bec_problem* p, const double* x, int slot) {
  BEC_LAUNCH_BEGIN(p);
  sumsq_kernel<<<kReduceBlocks, kThreads, 0, p->stream>>>(x, p->U, p->partials);
  BEC_LAUNCH_CHECK(p, "sumsq_kernel");
  BEC_LAUNCH_BEGIN(p);
  finish_sqrt_kernel<<<1, kThreads, 0, p->stream>>>(p->partials, kReduceBlocks, p->scal, slot);
  BEC_LAUNCH_CHECK(p, "finish_sqrt_kernel");
  return BEC_OK;
}

bec_status launch_scale_by_inv(bec_problem* p, const double* x, double* y, int slot) {
  BEC_LAUNCH_BEGIN(p);
  scale_by_inv_kernel<<<kReduceBlocks, kThreads, 0, p->stream>>>(x, y, p->U, p->scal, slot);
  BEC_LAUNCH_CHECK(p, "scale_by_inv_kernel");
  return BEC_OK;
}

bec_status launch_hessenberg(bec_problem* p, int j, const double* h1, const double* h2,
                             int norm_slot, int res_slot) {
  BEC_LAUNCH_BEGIN(p);
  hessenberg_kernel<<<1, 32, 0, p->stream>>>(p->H, p->max_restart + 1, j, h1, h2, p->scal,
                                             norm_slot, res_slot, p->cs, p->sn, p->g);
  BEC_LAUNCH_CHECK(p, "hessenberg_kernel");
  return BEC_OK;
}

bec_status launch_gmres_start(bec_problem* p, int slot) {
  BEC_LAUNCH_BEGIN(p);
  gmres_start_kernel<<<1, 64, 0, p->stream>>>(p->g, p->max_restart + 1, p->scal, slot);
  BEC_LAUNCH_CHECK(p, "gmres_start_kernel");
  return BEC_OK;
}

bec_status launch_least_squares(bec_problem* p, int k) {
  BEC_LAUNCH_BEGIN(p);
  least_squares_kernel<<<1, 32, 0, p->stream>>>(p->H, p->max_restart + 1, k, p->g, p->ycoef);
  BEC_LAUNCH_CHECK(p, "least_squares_kernel");
  return BEC_OK;
}

bec_status launch_copy(bec_problem* p, const double* x, double* y) {
  BEC_CUDA_TRY(cudaMemcpyAsync(y, x, (size_t)p->U * sizeof(double), cudaMemcpyDeviceToDevice,
                               p->stream));
  return BEC_OK;
}

bec_status launch_zero(bec_problem* p, double* x) {
  BEC_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)p->U * sizeof(double), p->stream));
  return BEC_OK;
}

}  // namespace bec

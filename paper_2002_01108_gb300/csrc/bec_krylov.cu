// FP64 Krylov kernels for restarted GMRES / FGMRES on the device.
//
// The Arnoldi basis is orthogonalised by classical Gram-Schmidt applied twice
// (CGS2), fused into few passes over the vectors:
//   pass 1: w = L z  and  h1 = V^T w             (stencil_dots, bec_stencil.cu)
//   pass 2: w -= V h1  and  h2 = V^T w           (update_dots)
//   pass 3: v_{j+1} = w - V h2  and  ||v_{j+1}|| (combine)
// Basis vectors are stored unnormalised; sigma_i = 1 / ||stored V_i|| is
// applied wherever V_i is read, which removes the separate scaling pass.
// Every reduction writes one partial per block of a fixed grid and is summed
// in a fixed order, so results are bitwise reproducible run to run.
// Kernels that keep one dot accumulator per vector are instantiated for the
// exact vector count (no work for unused slots).
#include <cuda_runtime.h>

#include "bec_internal.h"

namespace bec {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Block-reduce NV accumulators; partials[v * gridDim.x + blockIdx.x].
template <int NV>
__device__ __forceinline__ void block_store_dots(double (&acc)[NV], double* __restrict__ partials) {
  __shared__ double red[kWarps][NV];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double s = warp_sum(acc[v]);
    if (lane == 0) red[warp][v] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int wi = 0; wi < kWarps; ++wi) s += red[wi][threadIdx.x];
    partials[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__device__ __forceinline__ void block_store_sum(double v, double* __restrict__ partials) {
  __shared__ double red[kWarps];
  const double s = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int wi = 0; wi < kWarps; ++wi) t += red[wi];
    partials[blockIdx.x] = t;
  }
}

// Plain dots <V_v, w> for v < NV.  U is even (N is a power of two) and every
// vector is 16-byte aligned, so double2 loads are used.
template <int NV>
__global__ void __launch_bounds__(kThreads)
dots_kernel(const double* __restrict__ w, VecList V, long long U, double* __restrict__ partials,
            const int* __restrict__ flag) {
  if (flag && *flag == 0) return;
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  const long long U2 = U / 2;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < U2;
       i += (long long)gridDim.x * kThreads) {
    const double2 a = w2[i];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double2 x = reinterpret_cast<const double2*>(V.v[v])[i];
      acc[v] = fma(x.x, a.x, fma(x.y, a.y, acc[v]));
    }
  }
  block_store_dots<NV>(acc, partials);
}

// w -= sum_v c_v V_v, then dots <V_v, w_new>.  c_v = coef_v sigma_v.
template <int NV>
__global__ void __launch_bounds__(kThreads)
update_dots_kernel(double* __restrict__ w, VecList V, long long U, const double* __restrict__ coef,
                   const double* __restrict__ sigma, double* __restrict__ partials) {
  double c[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) c[v] = coef[v] * (sigma ? sigma[v] : 1.0);
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  const long long U2 = U / 2;
  double2* w2 = reinterpret_cast<double2*>(w);
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < U2;
       i += (long long)gridDim.x * kThreads) {
    double2 x[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = reinterpret_cast<const double2*>(V.v[v])[i];
    double2 a = w2[i];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      a.x = fma(-c[v], x[v].x, a.x);
      a.y = fma(-c[v], x[v].y, a.y);
    }
    w2[i] = a;
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = fma(x[v].x, a.x, fma(x[v].y, a.y, acc[v]));
  }
  block_store_dots<NV>(acc, partials);
}

// out = w + sign sum_{v<nv} coef_v sigma_v V_v (w null: 0); optional sum of out^2.
__global__ void __launch_bounds__(kThreads)
combine_kernel(double* out, const double* w, VecList V, int nv, long long U,
               const double* __restrict__ coef, const double* __restrict__ sigma, double sign,
               double* __restrict__ partials, const int* __restrict__ flag) {
  if (flag && *flag == 0) return;
  __shared__ double c[kMaxVec];
  for (int v = threadIdx.x; v < nv; v += kThreads) c[v] = sign * coef[v] * (sigma ? sigma[v] : 1.0);
  __syncthreads();
  const long long U2 = U / 2;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2* o2 = reinterpret_cast<double2*>(out);
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < U2;
       i += (long long)gridDim.x * kThreads) {
    double2 a = w2 ? w2[i] : make_double2(0.0, 0.0);
    for (int v = 0; v < nv; ++v) {
      const double2 x = reinterpret_cast<const double2*>(V.v[v])[i];
      a.x = fma(c[v], x.x, a.x);
      a.y = fma(c[v], x.y, a.y);
    }
    o2[i] = a;
    nrm = fma(a.x, a.x, fma(a.y, a.y, nrm));
  }
  if (partials != nullptr) block_store_sum(nrm, partials);
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
  block_store_sum(nrm, partials);
}

// hout[v] = sigma_v * sum_b partials[v * nb + b]   (block v, fixed tree order)
__global__ void __launch_bounds__(kThreads)
finish_dots_kernel(const double* __restrict__ partials, int nb, const double* __restrict__ sigma,
                   double* __restrict__ hout, const int* __restrict__ flag) {
  if (flag && *flag == 0) {
    if (threadIdx.x == 0) hout[blockIdx.x] = 0.0;
    return;
  }
  __shared__ double s[kThreads];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) a += partials[(long long)blockIdx.x * nb + b];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) hout[blockIdx.x] = s[0] * (sigma ? sigma[blockIdx.x] : 1.0);
}

// scal[slot] = sqrt(sum partials)
__global__ void __launch_bounds__(kThreads)
finish_sqrt_kernel(const double* __restrict__ partials, int nb, double* __restrict__ scal,
                   int slot, const int* __restrict__ flag) {
  if (flag && *flag == 0) return;
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

// Column j of the Arnoldi Hessenberg matrix (leading dimension ldh), the
// Givens rotations that keep it upper triangular, the rotated right-hand side
// g whose entry j+1 is the GMRES residual norm, and sigma_{j+1}.
__global__ void hessenberg_kernel(double* __restrict__ H, int ldh, int j,
                                  const double* __restrict__ h1, const double* __restrict__ h2,
                                  double* __restrict__ scal, int norm_slot, int res_slot,
                                  double* __restrict__ cs, double* __restrict__ sn,
                                  double* __restrict__ g, double* __restrict__ sigma,
                                  double shift) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (long long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
  col[j] += shift;   // Arnoldi on (A - shift I): H(A) = H(A - shift I) + shift I
  const double hn = scal[norm_slot];
  col[j + 1] = hn;
  sigma[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
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

__global__ void reorth_flag_kernel(const double* __restrict__ scal, int before, int after,
                                   int* __restrict__ flag) {
  if (threadIdx.x == 0) flag[0] = scal[after] * scal[after] < 0.5 * scal[before] * scal[before];
}

__global__ void gmres_start_kernel(double* __restrict__ g, int len, const double* __restrict__ scal,
                                   int slot, double* __restrict__ sigma) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = i == 0 ? scal[slot] : 0.0;
  if (threadIdx.x == 0) sigma[0] = scal[slot] > 0.0 ? 1.0 / scal[slot] : 0.0;
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

VecList pack(const double* const* V, int n) {
  VecList l;
  for (int i = 0; i < kMaxVec; ++i) l.v[i] = i < n ? V[i] : V[0];
  return l;
}

#define BEC_NV_CASES(X)                                                                 \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) \
  X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30)   \
  X(31) X(32)

__global__ void publish_scalars_kernel(const double* __restrict__ scal, double* __restrict__ host,
                                       int n) {
  if ((int)threadIdx.x < n) host[threadIdx.x] = scal[threadIdx.x];
}

bec_status launch_dots_chunk(bec_problem* p, const double* w, VecList L, int n, const int* flag) {
  BEC_LAUNCH_BEGIN(p);
  switch (n) {
#define BEC_DOTS_CASE(NV) \
  case NV: dots_kernel<NV><<<kReduceBlocks, kThreads, 0, p->stream>>>(w, L, p->U, p->partials, flag); break;
    BEC_NV_CASES(BEC_DOTS_CASE)
#undef BEC_DOTS_CASE
    default: return BEC_EINVAL;
  }
  BEC_LAUNCH_CHECK(p, "dots_kernel");
  return BEC_OK;
}

}  // namespace

bec_status launch_finish_dots(bec_problem* p, int nv, int nb, const double* sigma, double* hout,
                              const int* flag) {
  BEC_LAUNCH_BEGIN(p);
  finish_dots_kernel<<<nv, kThreads, 0, p->stream>>>(p->partials, nb, sigma, hout, flag);
  BEC_LAUNCH_CHECK(p, "finish_dots_kernel");
  return BEC_OK;
}

bec_status launch_finish_sqrt(bec_problem* p, const double* parts, int nb, int slot,
                              const int* flag) {
  BEC_LAUNCH_BEGIN(p);
  finish_sqrt_kernel<<<1, kThreads, 0, p->stream>>>(parts, nb, p->scal, slot, flag);
  BEC_LAUNCH_CHECK(p, "finish_sqrt_kernel");
  return BEC_OK;
}

bec_status launch_reorth_flag(bec_problem* p, int before_slot, int after_slot) {
  BEC_LAUNCH_BEGIN(p);
  reorth_flag_kernel<<<1, 32, 0, p->stream>>>(p->scal, before_slot, after_slot, p->flag);
  BEC_LAUNCH_CHECK(p, "reorth_flag_kernel");
  return BEC_OK;
}

bec_status launch_dots(bec_problem* p, const double* w, const double* const* V, int nv,
                       const double* sigma, double* hout, const int* flag) {
  for (int v0 = 0; v0 < nv; v0 += kMaxVec) {
    const int n = nv - v0 < kMaxVec ? nv - v0 : kMaxVec;
    bec_status s = launch_dots_chunk(p, w, pack(V + v0, n), n, flag);
    if (s != BEC_OK) return s;
    s = launch_finish_dots(p, n, kReduceBlocks, sigma ? sigma + v0 : nullptr, hout + v0, flag);
    if (s != BEC_OK) return s;
  }
  return BEC_OK;
}

bec_status launch_update_dots(bec_problem* p, double* w, const double* const* V, int nv,
                              const double* sigma, const double* coef, double* hout) {
  if (nv > kMaxVec) {   // unfused: update with every vector, then the dots in chunks
    bec_status s = launch_combine(p, w, w, V, nv, sigma, coef, -1.0, -1);
    if (s != BEC_OK) return s;
    return launch_dots(p, w, V, nv, sigma, hout);
  }
  const VecList L = pack(V, nv);
  BEC_LAUNCH_BEGIN(p);
  switch (nv) {
#define BEC_UPD_CASE(NV)                                                                    \
  case NV:                                                                                  \
    update_dots_kernel<NV><<<kReduceBlocks, kThreads, 0, p->stream>>>(w, L, p->U, coef,      \
                                                                       sigma, p->partials); \
    break;
    BEC_NV_CASES(BEC_UPD_CASE)
#undef BEC_UPD_CASE
    default: return BEC_EINVAL;
  }
  BEC_LAUNCH_CHECK(p, "update_dots_kernel");
  return launch_finish_dots(p, nv, kReduceBlocks, sigma, hout);
}

bec_status launch_combine(bec_problem* p, double* out, const double* w, const double* const* V,
                          int nv, const double* sigma, const double* coef, double sign,
                          int norm_slot, const int* flag) {
  // chunks of kMaxVec vectors; the norm comes from the last chunk
  int v0 = 0;
  do {
    const int n = nv - v0 < kMaxVec ? nv - v0 : kMaxVec;
    const bool last = v0 + kMaxVec >= nv;
    double* part = (last && norm_slot >= 0) ? p->partials : nullptr;
    const double* src = v0 == 0 ? w : out;
    BEC_LAUNCH_BEGIN(p);
    combine_kernel<<<kReduceBlocks, kThreads, 0, p->stream>>>(
        out, src, pack(V + v0, n > 0 ? n : 1), n, p->U, coef + v0, sigma ? sigma + v0 : nullptr,
        sign, part, flag);
    BEC_LAUNCH_CHECK(p, "combine_kernel");
    v0 += kMaxVec;
  } while (v0 < nv);
  if (norm_slot >= 0) return launch_finish_sqrt(p, p->partials, kReduceBlocks, norm_slot, flag);
  return BEC_OK;
}

bec_status launch_norm(bec_problem* p, const double* x, int slot) {
  BEC_LAUNCH_BEGIN(p);
  sumsq_kernel<<<kReduceBlocks, kThreads, 0, p->stream>>>(x, p->U, p->partials);
  BEC_LAUNCH_CHECK(p, "sumsq_kernel");
  return launch_finish_sqrt(p, p->partials, kReduceBlocks, slot, nullptr);
}

bec_status launch_hessenberg(bec_problem* p, int j, const double* h1, const double* h2,
                             int norm_slot, int res_slot, double shift) {
  BEC_LAUNCH_BEGIN(p);
  hessenberg_kernel<<<1, 32, 0, p->stream>>>(p->H, p->max_restart + 1, j, h1, h2, p->scal,
                                             norm_slot, res_slot, p->cs, p->sn, p->g, p->sigma,
                                             shift);
  BEC_LAUNCH_CHECK(p, "hessenberg_kernel");
  return BEC_OK;
}

bec_status launch_gmres_start(bec_problem* p, int slot) {
  BEC_LAUNCH_BEGIN(p);
  gmres_start_kernel<<<1, 64, 0, p->stream>>>(p->g, p->max_restart + 1, p->scal, slot, p->sigma);
  BEC_LAUNCH_CHECK(p, "gmres_start_kernel");
  return BEC_OK;
}

bec_status launch_least_squares(bec_problem* p, int k) {
  BEC_LAUNCH_BEGIN(p);
  least_squares_kernel<<<1, 32, 0, p->stream>>>(p->H, p->max_restart + 1, k, p->g, p->ycoef);
  BEC_LAUNCH_CHECK(p, "least_squares_kernel");
  return BEC_OK;
}

bec_status launch_publish_scalars(bec_problem* p) {
  BEC_LAUNCH_BEGIN(p);
  publish_scalars_kernel<<<1, 32, 0, p->stream>>>(p->scal, p->host_scal_dev, kScalSlots);
  BEC_LAUNCH_CHECK(p, "publish_scalars_kernel");
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

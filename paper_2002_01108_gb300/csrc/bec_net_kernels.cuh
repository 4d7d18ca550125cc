// Kernels of the learned correction network (4-level convolutional network on
// the multigrid hierarchy, 3 x 3 convolutions without bias; the residual path
// is linear, its layer outputs multiplied by gates computed from log a and
// lambda_k, see bec_net.cu).
// Activations are NHWC: act[b][y][x][c] with the channels contiguous, in the
// activation type AT (float or __nv_bfloat16); weights are FP32 [9][cin][cout]
// (tap = (dy+1)*3 + (dx+1)); every sum accumulates in FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace bec {
namespace net {

constexpr int kMaxC = 32;
constexpr int kConvThreads = 128;

template <typename AT> __device__ __forceinline__ float ld(const AT* p);
template <> __device__ __forceinline__ float ld<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <typename AT> __device__ __forceinline__ AT st(float v);
template <> __device__ __forceinline__ float st<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 st<__nv_bfloat16>(float v) {
  return __float2bfloat16(v);
}

// out[b][p][co] = act(sum_{tap, ci} W[tap][ci][co] in[b][p + tap][ci]),
// zero padding; one thread per output pixel, all COUT outputs in registers.
template <typename AT, int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(kConvThreads)
conv3x3_fwd_kernel(const AT* __restrict__ in, const float* __restrict__ W, AT* __restrict__ out,
                   int m, long long npix) {
  __shared__ float sW[9 * CIN * COUT];
  for (int i = threadIdx.x; i < 9 * CIN * COUT; i += kConvThreads) sW[i] = W[i];
  __syncthreads();
  const long long g = (long long)blockIdx.x * kConvThreads + threadIdx.x;
  if (g >= npix) return;
  const long long mm = (long long)m * m;
  const long long b = g / mm;
  const int p = (int)(g - b * mm);
  const int y = p / m, x = p - (p / m) * m;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = 0.f;
  const AT* base = in + b * mm * CIN;
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
    if (yy < 0 || yy >= m || xx < 0 || xx >= m) continue;
    const AT* src = base + ((long long)yy * m + xx) * CIN;
    const float* w = sW + tap * CIN * COUT;
#pragma unroll 2
    for (int ci = 0; ci < CIN; ++ci) {
      const float v = ld(src + ci);
#pragma unroll
      for (int co = 0; co < COUT; ++co) acc[co] = fmaf(v, w[ci * COUT + co], acc[co]);
    }
  }
  AT* dst = out + g * COUT;
#pragma unroll
  for (int co = 0; co < COUT; ++co) dst[co] = st<AT>(RELU ? fmaxf(acc[co], 0.f) : acc[co]);
}

// din[b][p][ci] = sum_{tap, co} W[tap][ci][co] dout[b][p - tap][co]
// (the adjoint of the zero-padded correlation); one thread per input pixel.
template <typename AT, int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads)
conv3x3_bwd_data_kernel(const AT* __restrict__ dout, const float* __restrict__ W,
                        AT* __restrict__ din, int m, long long npix) {
  __shared__ float sW[9 * CIN * COUT];
  for (int i = threadIdx.x; i < 9 * CIN * COUT; i += kConvThreads) sW[i] = W[i];
  __syncthreads();
  const long long g = (long long)blockIdx.x * kConvThreads + threadIdx.x;
  if (g >= npix) return;
  const long long mm = (long long)m * m;
  const long long b = g / mm;
  const int p = (int)(g - b * mm);
  const int y = p / m, x = p - (p / m) * m;
  float acc[CIN];
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.f;
  const AT* base = dout + b * mm * COUT;
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const int yy = y - (tap / 3 - 1), xx = x - (tap % 3 - 1);
    if (yy < 0 || yy >= m || xx < 0 || xx >= m) continue;
    const AT* src = base + ((long long)yy * m + xx) * COUT;
    const float* w = sW + tap * CIN * COUT;
#pragma unroll 2
    for (int co = 0; co < COUT; ++co) {
      const float v = ld(src + co);
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) acc[ci] = fmaf(v, w[ci * COUT + co], acc[ci]);
    }
  }
  AT* dst = din + g * CIN;
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) dst[ci] = st<AT>(acc[ci]);
}

// Partial weight gradients: block j sums in[b][p + tap][ci] dout[b][p][co]
// over its pixel range into part[j][tap][ci][co]; thread t owns entries
// t, t + blockDim, ...
template <typename AT, int CIN, int COUT>
__global__ void __launch_bounds__(256)
conv3x3_bwd_weight_kernel(const AT* __restrict__ in, const AT* __restrict__ dout,
                          float* __restrict__ part, int m, long long npix, long long per_block) {
  constexpr int NW = 9 * CIN * COUT;
  constexpr int PER = (NW + 255) / 256;
  constexpr int TILE = 32;                       // pixels staged per pass
  __shared__ float s_in[TILE][9][CIN];
  __shared__ float s_do[TILE][COUT];
  float acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i] = 0.f;
  const long long mm = (long long)m * m;
  const long long g0 = (long long)blockIdx.x * per_block;
  const long long g1 = g0 + per_block < npix ? g0 + per_block : npix;
  for (long long t0 = g0; t0 < g1; t0 += TILE) {
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * 9 * CIN; e += 256) {
      const int tp = e / (9 * CIN), rem = e % (9 * CIN), tap = rem / CIN, ci = rem % CIN;
      const long long g = t0 + tp;
      float v = 0.f;
      if (g < g1) {
        const long long b = g / mm;
        const int p = (int)(g - b * mm);
        const int yy = p / m + tap / 3 - 1, xx = p % m + tap % 3 - 1;
        if (yy >= 0 && yy < m && xx >= 0 && xx < m) v = ld(in + (b * mm + (long long)yy * m + xx) * CIN + ci);
      }
      s_in[tp][tap][ci] = v;
    }
    for (int e = threadIdx.x; e < TILE * COUT; e += 256) {
      const int tp = e / COUT, co = e % COUT;
      const long long g = t0 + tp;
      s_do[tp][co] = g < g1 ? ld(dout + g * COUT + co) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int w = threadIdx.x + 256 * i;
      if (w < NW) {
        const int tap = w / (CIN * COUT), ci = (w / COUT) % CIN, co = w % COUT;
        float a = acc[i];
        for (int tp = 0; tp < TILE; ++tp) a = fmaf(s_in[tp][tap][ci], s_do[tp][co], a);
        acc[i] = a;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + 256 * i;
    if (w < NW) part[(long long)blockIdx.x * NW + w] = acc[i];
  }
}

// dW[w] = sum_j part[j][w] in a fixed order
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nblk, int nw,
                                    float* __restrict__ dW) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  float s = 0.f;
  for (int j = 0; j < nblk; ++j) s += part[(long long)j * nw + w];
  dW[w] = s;
}

// Channel-wise full weighting R = P^T / 4 from a fine (mf) to a coarse grid;
// out = scale * R in (+ out when ADD).
template <typename AT, bool ADD>
__global__ void restrict_ch_kernel(const AT* __restrict__ in, AT* __restrict__ out, int mf, int mc,
                                   int C, long long n, float scale) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;                    // n = B * mc * mc * C
  const int c = (int)(g % C);
  const long long pix = g / C;
  const long long mcc = (long long)mc * mc;
  const long long b = pix / mcc;
  const int q = (int)(pix - b * mcc);
  const int cy = q / mc, cx = q % mc;
  const AT* src = in + b * (long long)mf * mf * C;
  float acc = 0.f;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const float w = (dy == 0 ? 0.5f : 0.25f) * (dx == 0 ? 0.5f : 0.25f);
      acc = fmaf(w, ld(src + ((long long)(2 * cy + 1 + dy) * mf + (2 * cx + 1 + dx)) * C + c), acc);
    }
  acc *= scale;
  if (ADD) acc += ld(out + g);
  out[g] = st<AT>(acc);
}

// Channel-wise bilinear prolongation from coarse (mc) to fine (mf);
// out = scale * P in (+ add_src when non-null).
template <typename AT>
__global__ void prolong_ch_kernel(const AT* __restrict__ in, const AT* __restrict__ add_src,
                                  AT* __restrict__ out, int mc, int mf, int C, long long n,
                                  float scale) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;                    // n = B * mf * mf * C
  const int c = (int)(g % C);
  const long long pix = g / C;
  const long long mff = (long long)mf * mf;
  const long long b = pix / mff;
  const int f = (int)(pix - b * mff);
  const int fy = f / mf, fx = f % mf;
  const AT* src = in + b * (long long)mc * mc * C;
  float acc = 0.f;
  for (int a = 0; a < 2; ++a) {
    int cy;
    float wy;
    if (fy & 1) { if (a) break; cy = (fy - 1) / 2; wy = 1.f; }
    else { cy = fy / 2 - 1 + a; wy = 0.5f; }
    if (cy < 0 || cy >= mc) continue;
    for (int bb = 0; bb < 2; ++bb) {
      int cx;
      float wx;
      if (fx & 1) { if (bb) break; cx = (fx - 1) / 2; wx = 1.f; }
      else { cx = fx / 2 - 1 + bb; wx = 0.5f; }
      if (cx < 0 || cx >= mc) continue;
      acc = fmaf(wy * wx, ld(src + ((long long)cy * mc + cx) * C + c), acc);
    }
  }
  acc *= scale;
  if (add_src) acc += ld(add_src + g);
  out[g] = st<AT>(acc);
}

// 16-byte groups of channels: V = 16 / sizeof(AT) consecutive channels of one
// pixel, loaded and stored as one uint4 (the pointer must be 16-byte aligned)
template <typename AT>
struct ChVec {
  static constexpr int V = 16 / (int)sizeof(AT);
};

template <typename AT>
__device__ __forceinline__ void ld_vec(const AT* p, float (&v)[ChVec<AT>::V]) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  if constexpr (sizeof(AT) == 4) {
    v[0] = __uint_as_float(u.x);
    v[1] = __uint_as_float(u.y);
    v[2] = __uint_as_float(u.z);
    v[3] = __uint_as_float(u.w);
  } else {
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
}

template <typename AT>
__device__ __forceinline__ void st_vec(AT* p, const float (&v)[ChVec<AT>::V]) {
  uint4 u;
  if constexpr (sizeof(AT) == 4) {
    u = make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]),
                   __float_as_uint(v[3]));
  } else {
    unsigned w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<const unsigned*>(&h);
    }
    u = make_uint4(w[0], w[1], w[2], w[3]);
  }
  *reinterpret_cast<uint4*>(p) = u;
}

// restrict_ch_kernel with a thread per 16-byte channel group (C a multiple of
// ChVec<AT>::V): the same FP32 sums in the same order per channel.
template <typename AT, bool ADD>
__global__ void restrict_ch_vec_kernel(const AT* __restrict__ in, AT* __restrict__ out, int mf,
                                       int mc, int C, long long n, float scale) {
  constexpr int V = ChVec<AT>::V;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;                    // n = B * mc * mc * C / V
  const int G = C / V;
  const int c0 = (int)(g % G) * V;
  const long long pix = g / G;
  const long long mcc = (long long)mc * mc;
  const long long b = pix / mcc;
  const int q = (int)(pix - b * mcc);
  const int cy = q / mc, cx = q % mc;
  const AT* src = in + b * (long long)mf * mf * C;
  float acc[V];
#pragma unroll
  for (int i = 0; i < V; ++i) acc[i] = 0.f;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const float w = (dy == 0 ? 0.5f : 0.25f) * (dx == 0 ? 0.5f : 0.25f);
      float v[V];
      ld_vec<AT>(src + ((long long)(2 * cy + 1 + dy) * mf + (2 * cx + 1 + dx)) * C + c0, v);
#pragma unroll
      for (int i = 0; i < V; ++i) acc[i] = fmaf(w, v[i], acc[i]);
    }
  AT* dst = out + pix * C + c0;
  if (ADD) {
    float o[V];
    ld_vec<AT>(dst, o);
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] = acc[i] * scale + o[i];
  } else {
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] *= scale;
  }
  st_vec<AT>(dst, acc);
}

// prolong_ch_kernel with a thread per 16-byte channel group, same sums.
template <typename AT>
__global__ void prolong_ch_vec_kernel(const AT* __restrict__ in, const AT* __restrict__ add_src,
                                      AT* __restrict__ out, int mc, int mf, int C, long long n,
                                      float scale) {
  constexpr int V = ChVec<AT>::V;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;                    // n = B * mf * mf * C / V
  const int G = C / V;
  const int c0 = (int)(g % G) * V;
  const long long pix = g / G;
  const long long mff = (long long)mf * mf;
  const long long b = pix / mff;
  const int f = (int)(pix - b * mff);
  const int fy = f / mf, fx = f % mf;
  const AT* src = in + b * (long long)mc * mc * C;
  float acc[V];
#pragma unroll
  for (int i = 0; i < V; ++i) acc[i] = 0.f;
  for (int a = 0; a < 2; ++a) {
    int cy;
    float wy;
    if (fy & 1) { if (a) break; cy = (fy - 1) / 2; wy = 1.f; }
    else { cy = fy / 2 - 1 + a; wy = 0.5f; }
    if (cy < 0 || cy >= mc) continue;
    for (int bb = 0; bb < 2; ++bb) {
      int cx;
      float wx;
      if (fx & 1) { if (bb) break; cx = (fx - 1) / 2; wx = 1.f; }
      else { cx = fx / 2 - 1 + bb; wx = 0.5f; }
      if (cx < 0 || cx >= mc) continue;
      float v[V];
      ld_vec<AT>(src + ((long long)cy * mc + cx) * C + c0, v);
#pragma unroll
      for (int i = 0; i < V; ++i) acc[i] = fmaf(wy * wx, v[i], acc[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < V; ++i) acc[i] *= scale;
  AT* dst = out + pix * C + c0;
  if (add_src) {
    float o[V];
    ld_vec<AT>(add_src + pix * C + c0, o);
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] += o[i];
  }
  st_vec<AT>(dst, acc);
}

// d *= (a > 0), elementwise
template <typename AT>
__global__ void relu_mask_kernel(AT* __restrict__ d, const AT* __restrict__ a, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n && !(ld(a + g) > 0.f)) d[g] = st<AT>(0.f);
}

// d += e, elementwise
template <typename AT>
__global__ void add_kernel(AT* __restrict__ d, const AT* __restrict__ e, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) d[g] = st<AT>(ld(d + g) + ld(e + g));
}

// ---------------------------------------------------------------- gates
constexpr int kGates = 8;      // gated layers (0..7)
constexpr int kPoles = 8;      // pole terms of the correction
struct Poles {
  float s[kPoles];             // sigma_j
};
constexpr int kGateAHidden = 8; // hidden channels of an a-gate

// out[b][p][c] = pre[b][p][c] GA[p][c] (out may be pre); grid (x: the
// mmC = m^2 C elements of one image, y: the image b), no index division
template <typename AT>
__global__ void gate_apply_kernel(const AT* __restrict__ pre, AT* __restrict__ out,
                                  const float* __restrict__ GA, long long mmC) {
  const long long pc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pc >= mmC) return;
  const long long g = (long long)blockIdx.y * mmC + pc;
  out[g] = st<AT>(ld(pre + g) * GA[pc]);
}

// d[b][p][c] *= GA[p][c] (the adjoint of the gate multiply), the same grid
template <typename AT>
__global__ void gate_scale_grad_kernel(AT* __restrict__ d, const float* __restrict__ GA,
                                       long long mmC) {
  const long long pc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pc >= mmC) return;
  const long long g = (long long)blockIdx.y * mmC + pc;
  d[g] = st<AT>(ld(d + g) * GA[pc]);
}

// dGA[p][c] = sum_b dout[b][p][c] pre[b][p][c]  (b in order)
template <typename AT>
__global__ void gate_dga_kernel(const AT* __restrict__ dout, const AT* __restrict__ pre,
                                float* __restrict__ dGA, long long mmC, int B) {
  const long long pc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pc >= mmC) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) {
    const long long g = (long long)b * mmC + pc;
    s = fmaf(ld(dout + g), ld(pre + g), s);
  }
  dGA[pc] = s;
}

// a = 1 + tanh(a) in place (the a-gate's output)
__global__ void one_plus_tanh_kernel(float* __restrict__ a, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) a[g] = 1.f + tanhf(a[g]);
}

// d = dG (1 - (G - 1)^2): the derivative through G = 1 + tanh(z)
__global__ void dtanh_kernel(const float* __restrict__ dG, const float* __restrict__ G,
                             float* __restrict__ d, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const float t = G[g] - 1.f;
  d[g] = dG[g] * (1.f - t * t);
}

// where the a-gates' weights A1_i and A2_i start in the flat weight vector
struct GateOffsets {
  long long a1[kGates], a2[kGates];
};

// Adam step on FP32 master weights: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// w -= lr_t m / (sqrt(v) + eps), lr_t = lr sqrt(1-b2^t) / (1-b1^t).
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ mo, float* __restrict__ ve,
                            const float* __restrict__ g, int n, float lr_t, float b1, float b2,
                            float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float m = b1 * mo[i] + (1.f - b1) * gi;
  const float v = b2 * ve[i] + (1.f - b2) * gi * gi;
  mo[i] = m;
  ve[i] = v;
  w[i] -= lr_t * m / (sqrtf(v) + eps);
}

}  // namespace net
}  // namespace bec

// Learned route of P_eps^{-1} (BEC_ROUTE_LEARNED): one multigrid V-cycle per
// shifted system, then a learned correction of what the V-cycle left,
//     x1 = x_k + P_0 ec_k(R_0 (b_k - B_k x_k)),
// one damped-Jacobi sweep x2 = x1 + omega D^{-1} (b_k - B_k x1) (the
// post-smoothing that follows a prolonged correction), and the step
// x_k <- x_k + alpha (x2 - x_k) with one alpha for all frequencies, fixed by
// a calibration apply (the minimal-residual step of all frequencies together
// on a fixed right-hand side; alpha = 0 keeps the V-cycle's iterates: the
// multigrid is the fallback).
//
// The coarse correction is linear in the residual and analytic in the shift:
//     ec_k = sum_j sigma_j / (lambda'_k + sigma_j) Nc_j(rc / sigma_0),
// 8 fixed poles sigma_j (geometric, from the smoothest mode's shift to the
// largest eigenvalue on the grid of spacing 2h) with residue maps Nc_j that
// do not depend on k: real operators, Nc_j(x) = N_j(Re x) + i N_j(Im x), the
// 8 outputs of one 4-level convolutional network of one real plane on the
// grid of spacing 2h, whose layer outputs are multiplied by gates computed
// from log a only.  Real residue operators give ec the exact inverse's
// symmetry ec(conj lambda, conj r) = conj ec(lambda, r), on which the half
// spectrum relies (else the map would jump to its conjugate at k = 0, N/2).
// Why analytic: Step 3 multiplies time step j by eps^{-j/N}.  A dependence of
// the inner solve on conj(lambda'_k) (through Re, Im or |lambda'_k|
// separately, or through conj of the residual) links the first time steps
// to the last ones, and that part comes back amplified by up to 1/eps.  Poles
// on the negative real axis, like those of the exact (lambda M + tau K)^{-1},
// the V-cycle and the sweep, have no such part.
//
// The network is trained on the GPU, by these kernels, on pairs that the
// method's own multigrid generates: r is the residual a V-cycle leaves for
// the right-hand sides that the V-cycles of a multigrid-preconditioned FGMRES
// solve were given (the time spectra of its Krylov vectors), the target the
// coarse-grid correction B_{k,1}^{-1} R_0 r (level 1 of the hierarchy),
// obtained by repeated V-cycles from level 1 (defect correction).
// Requires the FP32 preconditioner.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "bec_fft.cuh"
#include "bec_internal.h"
#include "bec_net_kernels.cuh"

namespace bec {

namespace {

enum Act { A_X, A_H0, A_S0, A_R0, A_S1, A_R1, A_S2, A_R2, A_S3, A_P2, A_U2, A_P1, A_U1, A_P0,
           A_U0, A_Y, NACT };

int act_level(int a) {
  switch (a) {
    case A_X: case A_H0: case A_S0: case A_P0: case A_U0: case A_Y: return 0;
    case A_R0: case A_S1: case A_P1: case A_U1: return 1;
    case A_R1: case A_S2: case A_P2: case A_U2: return 2;
    default: return 3;
  }
}

constexpr int kT = 256;
unsigned grid_for(long long n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace

struct NetState {
  int C = 32;
  bool fp32 = false;
  int mf = 0;                    // fine grid
  int sz[4] = {0, 0, 0, 0};      // network levels, sz[0] = (mf - 1) / 2
  int Bmax = 0;                  // network samples; a frequency takes two (r and i r)
  int cin[9], cout[9];
  long long woff[10];            // the 9 convolutions of the residual path
  net::GateOffsets goff;         // the gate networks' weights
  long long nparam = 0;          // all weights
  float* W = nullptr;            // FP32 master weights, all layers
  float* G = nullptr;            // gradients
  float* Mo = nullptr;           // Adam moments
  float* Ve = nullptr;
  float* wpart = nullptr;        // weight-gradient partials
  long long wpart_n = 0;
  void* act[NACT] = {};
  void* grad[NACT] = {};
  void* pre[net::kGates] = {};   // layer outputs before their gates (training)
  float* la_lv[4] = {};          // centred log a on the 4 network levels
  float* GA[net::kGates] = {};   // a-gates [m_l^2][C] of the gated layers
  float* GAt[net::kGates] = {};  // the same, channel-major [C][m_l^2] (the tensor-core
                                 // epilogue's coalesced reads)
  float* Z1[net::kGates] = {};   // their hidden layer, relu'd, [m_l^2][8]
  float* dGA[net::kGates] = {};  // gradients of the a-gates
  float* dA = nullptr;           // work: [sz0^2][C]
  float* dZ = nullptr;           // work: [sz0^2][8]
  net::Poles poles;              // sigma_j of the pole terms
  bool gates_ok = false;         // GA matches the weights
  bool cal_ok = false;           // alpha matches the weights and eps
  bool bypass = false;           // the route acts as the multigrid route alone
  bool judge = true;             // the calibration's spectral-radius test runs
  bool rejected = false;         // the last calibration kept the V-cycle's iterates
                                 // (read on the host: the applies skip the network)
  double* jrho = nullptr;        // [2K + 2]: the judge's radii per frequency (V-cycle,
                                 // corrected) and their maxima
  int nkry = 0;                  // recorded Krylov vectors (rows of the problem's V)
  double* kf = nullptr;          // U doubles: the recording solve's right-hand side
  double* ku = nullptr;          // U doubles: its solution
  double a_mean = 1.0;
  float* rc = nullptr;           // [Bmax][mc^2] complex
  float* ecb = nullptr;          // [Bmax / 2][mc^2] complex: the coarse correction ec
  int* row = nullptr;            // per sample row of res / etgt (staged from the host)
  int* lam = nullptr;            // per sample frequency index
  int* iota = nullptr;           // 0, 1, ..., K-1 (rows = frequencies, no host staging)
  const int* cur_row = nullptr;  // the index arrays the next features/loss calls use
  const int* cur_lam = nullptr;
  int* h_idx = nullptr;          // pinned staging of row/lam (2 Bmax)
  float* efine = nullptr;        // [Bmax][J] complex: P_0 correction
  float* res = nullptr;          // [K][J] complex residuals
  float* etgt = nullptr;         // [K][mc^2] complex coarse targets
  float* rcall = nullptr;        // [K][mc^2] complex: R_0 res of every frequency
  float* ework = nullptr;        // [K][J] complex: the pair generation's right-hand sides
  float* xnew = nullptr;         // [K][J] complex corrected iterate
  double* part = nullptr;        // per-sample / per-frequency partial sums
  double* jpart = nullptr;       // the calibration's block sums, [K][kMrSplit][4]
  float2* alpha = nullptr;       // the step, one for all frequencies (from the calibration)
  double* h_part = nullptr;      // pinned mirror
  int adam_t = 0;
  unsigned long long rng_ctr = 0;
  bool tc = false;               // every layer on the tensor cores (BF16, C = 32)
  __nv_bfloat16* wt = nullptr;   // BF16 weights of all layers in the operand layout
  __nv_bfloat16* x16 = nullptr;  // input planes padded to 16 channels (tensor-core layer 0)
  int* err = nullptr;            // set by a device wait that ran out
};

namespace {

// ------------------------------------------------------------ net kernels
// rc[b][q] = R_0 res[row[b]] at coarse node q (complex = 2 channels)
__global__ void feat_restrict_kernel(const float2* __restrict__ res, const int* __restrict__ row,
                                     float2* __restrict__ rc, int mf, int mc, int B) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long mcc = (long long)mc * mc;
  if (g >= B * mcc) return;
  const int b = (int)(g / mcc), q = (int)(g - (long long)b * mcc);
  const int cy = q / mc, cx = q % mc;
  const float2* src = res + (long long)row[b] * mf * mf;
  float2 acc = {0.f, 0.f};
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const float w = (dy == 0 ? 0.5f : 0.25f) * (dx == 0 ? 0.5f : 0.25f);
      const float2 v = src[(long long)(2 * cy + 1 + dy) * mf + (2 * cx + 1 + dx)];
      acc.x = fmaf(w, v.x, acc.x);
      acc.y = fmaf(w, v.y, acc.y);
    }
  rc[g] = acc;
}

// The input planes of Bc complex samples as 2 Bc real network samples:
// X[b][q] = Re rc / sigma_0 and X[Bc + b][q] = Im rc / sigma_0, the same scale
// for every frequency (and, when X16 is not null, the same plane padded with
// zeros to 16 BF16 channels: the input of the tensor-core layer 0)
__device__ __forceinline__ void x16_store(__nv_bfloat16* X16, long long g, float f0) {
  const __nv_bfloat162 h01 = __floats2bfloat162_rn(f0, 0.f);
  uint4 lo;
  lo.x = *reinterpret_cast<const unsigned*>(&h01);
  lo.y = 0u;
  lo.z = 0u;
  lo.w = 0u;
  uint4* d16 = reinterpret_cast<uint4*>(X16 + g * 16);
  d16[0] = lo;
  d16[1] = make_uint4(0u, 0u, 0u, 0u);
}

template <typename AT>
__global__ void feat_fill_kernel(const float2* __restrict__ rc, float c, AT* __restrict__ X,
                                 __nv_bfloat16* __restrict__ X16, long long mcc, int Bc) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long half = Bc * mcc;
  if (g >= half) return;
  const float2 v = rc[g];
  const float f0 = c * v.x, f1 = c * v.y;
  X[g] = net::st<AT>(f0);
  X[half + g] = net::st<AT>(f1);
  if (X16 != nullptr) {
    x16_store(X16, g, f0);
    x16_store(X16, half + g, f1);
  }
}

// gt[c][p] = g[p][c] (a gate in channel-major order)
__global__ void gate_transpose_kernel(const float* __restrict__ g, float* __restrict__ gt,
                                      long long mm, int C) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mm * C) return;
  const long long c = e / mm, q = e - c * mm;
  gt[e] = g[q * C + c];
}

// w_j = sigma_j / (lambda + sigma_j) of one frequency
__device__ __forceinline__ void pole_weights(float2 L, const net::Poles& P,
                                             float2 (&w)[net::kPoles]) {
#pragma unroll
  for (int j = 0; j < net::kPoles; ++j) {
    const float dr = L.x + P.s[j], di = L.y;
    const float f = P.s[j] / fmaf(dr, dr, di * di);
    w[j] = make_float2(dr * f, -di * f);
  }
}

// ec = sum_j w_j Nc_j at coarse point q of complex sample b, with
// Nc_j = N_j(Re x) + i N_j(Im x) from the network outputs Y[b] = N(Re x) and
// Y[Bc + b] = N(Im x) (kNetOut = kPoles real channels)
template <typename AT>
__device__ __forceinline__ float2 pole_sum(const AT* __restrict__ Y, long long b, long long q,
                                           long long mcc, int Bc, const float2 (&w)[net::kPoles]) {
  static_assert(kNetOut == net::kPoles, "one output plane per pole");
  const AT* yr = Y + (b * mcc + q) * kNetOut;
  const AT* yi = Y + ((Bc + b) * mcc + q) * kNetOut;
  float ex = 0.f, ey = 0.f;
#pragma unroll
  for (int j = 0; j < net::kPoles; ++j) {
    const float pr = net::ld(yr + j), pi = net::ld(yi + j);
    ex = fmaf(w[j].x, pr, fmaf(-w[j].y, pi, ex));
    ey = fmaf(w[j].x, pi, fmaf(w[j].y, pr, ey));
  }
  return make_float2(ex, ey);
}

// ecb[b][q] = ec of complex sample b (frequency lam[b]) at coarse point q
template <typename AT>
__global__ void pole_sum_kernel(const AT* __restrict__ Y, const int* __restrict__ lam,
                                const float2* __restrict__ lamf, net::Poles P,
                                float2* __restrict__ ecb, long long mcc, int Bc) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Bc * mcc) return;
  const int b = (int)(g / mcc);
  float2 w[net::kPoles];
  pole_weights(lamf[lam[b]], P, w);
  ecb[g] = pole_sum(Y, b, g - (long long)b * mcc, mcc, Bc, w);
}

// efine[b][f] = P_0 ec_b at fine node f for each of Bc complex samples
__global__ void out_prolong_kernel(const float2* __restrict__ ecb, float2* __restrict__ efine,
                                   int mc, int mf, int Bc) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long mff = (long long)mf * mf, mcc = (long long)mc * mc;
  if (g >= Bc * mff) return;
  const int b = (int)(g / mff), f = (int)(g - (long long)b * mff);
  const int fy = f / mf, fx = f % mf;
  float ax = 0.f, ay = 0.f;
  for (int a = 0; a < 2; ++a) {
    int cy;
    float wy;
    if (fy & 1) { if (a) break; cy = (fy - 1) / 2; wy = 1.f; }
    else { cy = fy / 2 - 1 + a; wy = 0.5f; }
    if (cy < 0 || cy >= mc) continue;
    for (int c2 = 0; c2 < 2; ++c2) {
      int cx;
      float wx;
      if (fx & 1) { if (c2) break; cx = (fx - 1) / 2; wx = 1.f; }
      else { cx = fx / 2 - 1 + c2; wx = 0.5f; }
      if (cx < 0 || cx >= mc) continue;
      const float2 v = ecb[(long long)b * mcc + (long long)cy * mc + cx];
      ax = fmaf(wy * wx, v.x, ax);
      ay = fmaf(wy * wx, v.y, ay);
    }
  }
  efine[g] = make_float2(ax, ay);
}

// one block per complex sample: part[2b] = ||ec_b - etgt[row_b]||^2 and
// part[2b+1] = ||etgt[row_b]||^2 on the coarse grid (ec_b: pole_sum at the
// sample's frequency lam[b])
template <typename AT>
__global__ void closs_parts_kernel(const AT* __restrict__ Y, const float2* __restrict__ etgt,
                                   const int* __restrict__ row, const int* __restrict__ lam,
                                   const float2* __restrict__ lamf, net::Poles P,
                                   double* __restrict__ part, long long mcc, int Bc) {
  __shared__ double rn[256], rd[256];
  const int b = blockIdx.x;
  const float2* t = etgt + (long long)row[b] * mcc;
  float2 w[net::kPoles];
  pole_weights(lamf[lam[b]], P, w);
  double num = 0.0, den = 0.0;
  for (long long q = threadIdx.x; q < mcc; q += blockDim.x) {
    const float2 tv = t[q];
    const float2 e = pole_sum(Y, b, q, mcc, Bc, w);
    const double dx = (double)e.x - tv.x, dy = (double)e.y - tv.y;
    num += dx * dx + dy * dy;
    den += (double)tv.x * tv.x + (double)tv.y * tv.y;
  }
  rn[threadIdx.x] = num;
  rd[threadIdx.x] = den;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      rn[threadIdx.x] += rn[threadIdx.x + s];
      rd[threadIdx.x] += rd[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * b] = rn[0];
    part[2 * b + 1] = rd[0];
  }
}

// L = mean_b ||ec_b - t_b||^2 / den_b over Bc complex samples, G = dL/dec_b
// = 2 (ec_b - t_b) / (den_b Bc).  Through ec = sum_j w_j (a_j + i b_j)
// (pole_sum: a_j channel j of Y_b, b_j of Y_{Bc+b}), with h_j = conj(G) w_j:
// dL/da_j = Re h_j,  dL/db_j = -Im h_j
template <typename AT>
__global__ void closs_grad_kernel(const AT* __restrict__ Y, const float2* __restrict__ etgt,
                                  const int* __restrict__ row, const int* __restrict__ lam,
                                  const float2* __restrict__ lamf, net::Poles P,
                                  const double* __restrict__ part, AT* __restrict__ dY,
                                  long long mcc, int Bc) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long half = Bc * mcc;
  if (g >= half) return;
  const int b = (int)(g / mcc);
  const long long q = g - (long long)b * mcc;
  float2 w[net::kPoles];
  pole_weights(lamf[lam[b]], P, w);
  const float2 t = etgt[(long long)row[b] * mcc + q];
  const float2 e = pole_sum(Y, b, q, mcc, Bc, w);
  const double k = 2.0 / (part[2 * b + 1] * Bc);
  const float gx = (float)(k * ((double)e.x - t.x)), gy = (float)(k * ((double)e.y - t.y));
  AT* dr = dY + g * kNetOut;
  AT* di = dY + (half + g) * kNetOut;
#pragma unroll
  for (int j = 0; j < net::kPoles; ++j) {
    const float hr = fmaf(gx, w[j].x, gy * w[j].y), hi = fmaf(gx, w[j].y, -gy * w[j].x);
    dr[j] = net::st<AT>(hr);
    di[j] = net::st<AT>(-hi);
  }
}

// The calibration right-hand side: value i of the interleaved (re, im) array
// of [K][J] complex is (t >> 40) 2^-23 - 1, t = splitmix64(key ^
// splitmix64(i)) (SplitMix64's output function of Steele, Lea and Flood):
// uniform in [-1, 1) and exactly representable in FP32.
constexpr unsigned long long kCalibrationKey = 0xCA11B8A7E5EED001ull;
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void calibration_fill_kernel(float* __restrict__ v, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const unsigned long long t = splitmix64(kCalibrationKey ^ splitmix64((unsigned long long)g));
  v[g] = (float)(int)(t >> 40) * 0x1p-23f - 1.0f;
}

// v[i] = uniform in [-1, 1): (splitmix64(key ^ splitmix64(i)) >> 11) 2^-52 - 1
__global__ void uniform_fill_f64_kernel(double* __restrict__ v, long long n,
                                        unsigned long long key) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const unsigned long long t = splitmix64(key ^ splitmix64((unsigned long long)g));
  v[g] = (double)(t >> 11) * 0x1p-52 - 1.0;
}

// counter-based standard normal pair (splitmix64 hash + Box-Muller)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void gauss_fill_kernel(float2* __restrict__ v, long long n, unsigned long long key) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const unsigned long long h = mix64(key ^ mix64((unsigned long long)g));
  const float u1 = ((float)(h >> 40) + 0.5f) * (1.0f / 16777216.0f);
  const float u2 = ((float)((h >> 16) & 0xFFFFFF) + 0.5f) * (1.0f / 16777216.0f);
  const float r = sqrtf(-2.f * logf(u1));
  float sv, cv;
  sincospif(2.f * u2, &sv, &cv);
  v[g] = make_float2(r * cv, r * sv);
}

__global__ void axpy_c_kernel(float2* __restrict__ y, const float2* __restrict__ x, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) {
    const float2 a = y[g], b = x[g];
    y[g] = make_float2(a.x + b.x, a.y + b.y);
  }
}

// out[k0 + b] = x[k0 + b] + efine[b]
__global__ void add_corr_kernel(float2* __restrict__ out, const float2* __restrict__ x,
                                const float2* __restrict__ efine, long long mff, int k0, int B) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B * mff) return;
  const long long o = (long long)k0 * mff + g;
  const float2 a = x[o], e = efine[g];
  out[o] = make_float2(a.x + e.x, a.y + e.y);
}

// kMrSplit blocks per frequency k: with res = b - B x (the V-cycle's
// residual) and r2 = b - B x2 (the corrected and smoothed iterate),
// B d = res - r2 for the step d = x2 - x.  jpart[(k kMrSplit + s) 4 + i] =
// the block's Re, Im <B d, res>, ||B d||^2, ||res||^2 (<u, v> = u^H v): each
// thread sums its points (mff / (kMrSplit 256) of them) in FP32, the block
// adds the threads' sums in FP64 in a fixed order.
constexpr int kMrSplit = 8;
__global__ void __launch_bounds__(256)
mr_dots_kernel(const float2* __restrict__ res, const float2* __restrict__ r2,
               double* __restrict__ jpart, long long mff) {
  __shared__ double red[4][256];
  const int k = blockIdx.x, sblk = blockIdx.y;
  float cr = 0.f, ci = 0.f, dd = 0.f, rr = 0.f;
  const long long stride = (long long)kMrSplit * blockDim.x;
  for (long long f = (long long)sblk * blockDim.x + threadIdx.x; f < mff; f += stride) {
    const float2 r = res[(long long)k * mff + f];
    const float2 q = r2[(long long)k * mff + f];
    const float bx = r.x - q.x, by = r.y - q.y;
    cr = fmaf(bx, r.x, fmaf(by, r.y, cr));
    ci = fmaf(bx, r.y, fmaf(-by, r.x, ci));
    dd = fmaf(bx, bx, fmaf(by, by, dd));
    rr = fmaf(r.x, r.x, fmaf(r.y, r.y, rr));
  }
  red[0][threadIdx.x] = cr;
  red[1][threadIdx.x] = ci;
  red[2][threadIdx.x] = dd;
  red[3][threadIdx.x] = rr;
  __syncthreads();
  for (int st2 = blockDim.x / 2; st2 > 0; st2 >>= 1) {
    if ((int)threadIdx.x < st2)
      for (int i = 0; i < 4; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + st2];
    __syncthreads();
  }
  if (threadIdx.x < 4)
    jpart[((long long)k * kMrSplit + sblk) * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// One block: per frequency the sums over the kMrSplit blocks (in order) into
// part[4k..]; then the one step alpha = sum_k <B d, res>_k / sum_k ||B d||_k^2
// (k in order; 0 when the sums vanish or are not finite: the V-cycle's
// iterate is kept, one fallback); then ratio[k] = ||res - alpha B d|| / ||res||
// = sqrt(rr - 2 Re(alpha conj<B d, res>) + |alpha|^2 dd) / sqrt(rr).
__global__ void __launch_bounds__(256)
mr_alpha_kernel(const double* __restrict__ jpart, double* __restrict__ part,
                float2* __restrict__ alpha, int K, double* __restrict__ ratio,
                int* __restrict__ fallbacks) {
  __shared__ double al[2];
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double sm[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < kMrSplit; ++b)
      for (int i = 0; i < 4; ++i) sm[i] += jpart[((long long)k * kMrSplit + b) * 4 + i];
    for (int i = 0; i < 4; ++i) part[4 * k + i] = sm[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double cr = 0.0, ci = 0.0, dd = 0.0;
    for (int k = 0; k < K; ++k) {
      cr += part[4 * k];
      ci += part[4 * k + 1];
      dd += part[4 * k + 2];
    }
    const bool ok = dd > 0.0 && isfinite(dd) && isfinite(cr) && isfinite(ci);
    al[0] = ok ? cr / dd : 0.0;
    al[1] = ok ? ci / dd : 0.0;
    alpha[0] = make_float2((float)al[0], (float)al[1]);
    if (!ok) *fallbacks = 1;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double cr = part[4 * k], ci = part[4 * k + 1], dd = part[4 * k + 2], rr = part[4 * k + 3];
    const double after = rr - 2.0 * (al[0] * cr + al[1] * ci) + (al[0] * al[0] + al[1] * al[1]) * dd;
    ratio[k] = rr > 0.0 ? sqrt(fmax(after, 0.0) / rr) : 0.0;
  }
}

// kMrSplit blocks per frequency k: jpart[k kMrSplit + s] = the block's part
// of ||v_k||^2 (FP32 per thread, FP64 across the block's threads in a fixed
// order)
__global__ void __launch_bounds__(256)
knorm_parts_kernel(const float2* __restrict__ v, double* __restrict__ jpart, long long mff) {
  __shared__ double red[256];
  const int k = blockIdx.x, sblk = blockIdx.y;
  float acc = 0.f;
  const long long stride = (long long)kMrSplit * blockDim.x;
  for (long long f = (long long)sblk * blockDim.x + threadIdx.x; f < mff; f += stride) {
    const float2 a = v[(long long)k * mff + f];
    acc = fmaf(a.x, a.x, fmaf(a.y, a.y, acc));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st2 = blockDim.x / 2; st2 > 0; st2 >>= 1) {
    if ((int)threadIdx.x < st2) red[threadIdx.x] += red[threadIdx.x + st2];
    __syncthreads();
  }
  if (threadIdx.x == 0) jpart[(long long)k * kMrSplit + sblk] = red[0];
}

// v_k <- v_k / ||v_k|| (kept when the norm is 0), rho[k] = ||v_k||
__global__ void knorm_scale_kernel(float2* __restrict__ v, const double* __restrict__ jpart,
                                   double* __restrict__ rho, long long mff, int K) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)K * mff) return;
  const int k = (int)(g / mff);
  double ss = 0.0;
  for (int b = 0; b < kMrSplit; ++b) ss += jpart[(long long)k * kMrSplit + b];
  const double nrm = sqrt(ss);
  if (g - (long long)k * mff == 0) rho[k] = nrm;
  if (nrm > 0.0) {
    const float sc = (float)(1.0 / nrm);
    const float2 a = v[g];
    v[g] = make_float2(a.x * sc, a.y * sc);
  }
}

// The judge's decision: the largest radius over the frequencies of the
// V-cycle (rho[0..K)) and of the corrected preconditioner (rho[K..2K)) into
// rho[2K], rho[2K+1]; unless the corrected one is the smaller, alpha = 0 (the
// V-cycle's iterates are kept) and the fallback flag is set.
__global__ void judge_kernel(double* __restrict__ rho, int K, float2* __restrict__ alpha,
                             int* __restrict__ fallback) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double m0 = 0.0, m1 = 0.0;
  for (int k = 0; k < K; ++k) {
    m0 = fmax(m0, rho[k]);
    m1 = fmax(m1, rho[K + k]);
  }
  for (int k = 0; k < K; ++k)
    if (!(rho[K + k] == rho[K + k])) m1 = rho[K + k];   // a NaN radius rejects
  rho[2 * K] = m0;
  rho[2 * K + 1] = m1;
  if (!(m1 < m0)) {
    alpha[0] = make_float2(0.f, 0.f);
    *fallback = 1;
  }
}

// x <- x + alpha (x2 - x) with the calibration's step (mr_alpha_kernel)
__global__ void mr_update_kernel(float2* __restrict__ x, const float2* __restrict__ x2,
                                 const float2* __restrict__ alpha, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const float2 al = alpha[0];
  const float2 a = x[g], c = x2[g];
  const float dx = c.x - a.x, dy = c.y - a.y;
  x[g] = make_float2(a.x + al.x * dx - al.y * dy, a.y + al.x * dy + al.y * dx);
}

// ------------------------------------------------------------ dispatch helpers
// out = conv3x3(in, W) (ReLU when relu: the a-gates' hidden layer) for B images of side m, FP32 weights
// [9][ci][co] at W; the channel pairs of the residual path (C = 4 or 32) and
// of the a-gates
template <typename AT>
bec_status conv_fwd_raw(bec_problem* p, const AT* a, const float* W, int ci, int co, AT* o, int m,
                        int B, bool relu) {
  const long long npix = (long long)B * m * m;
  const unsigned g = (unsigned)((npix + net::kConvThreads - 1) / net::kConvThreads);
  BEC_LAUNCH_BEGIN(p);
#define BEC_CF(CI, CO)                                                                            \
  if (ci == CI && co == CO) {                                                                     \
    if (relu) net::conv3x3_fwd_kernel<AT, CI, CO, true><<<g, net::kConvThreads, 0, p->stream>>>(a, W, o, m, npix); \
    else net::conv3x3_fwd_kernel<AT, CI, CO, false><<<g, net::kConvThreads, 0, p->stream>>>(a, W, o, m, npix); \
  } else
  BEC_CF(1, 4) BEC_CF(4, 4) BEC_CF(4, 8) BEC_CF(1, 32) BEC_CF(32, 32) BEC_CF(32, 8) BEC_CF(1, 8)
  BEC_CF(8, 4) BEC_CF(8, 32) {
    set_error("unsupported network channel count");
    return BEC_EUNSUPPORTED;
  }
#undef BEC_CF
  BEC_LAUNCH_CHECK(p, "net_conv_fwd_kernel");
  return BEC_OK;
}

// layer `layer` of the residual path (no activation).  With gate not null
// the tensor-core path multiplies by the layer's gate in its epilogue; only
// that path takes a gate (the caller applies it otherwise).
template <typename AT>
bec_status conv_fwd(bec_problem* p, const void* in, int layer, void* out, int m, int B,
                    const float* gate = nullptr) {
  NetState& n = *p->net;
  const AT* a = static_cast<const AT*>(in);
  AT* o = static_cast<AT*>(out);
  if constexpr (sizeof(AT) == 2) {
    if (n.tc) {   // every layer (layer 0 reads the 16-channel padded planes)
      const __nv_bfloat16* src =
          layer == 0 ? n.x16 : reinterpret_cast<const __nv_bfloat16*>(a);
      return tc_conv3x3(p, layer, src, n.wt, reinterpret_cast<__nv_bfloat16*>(o), gate, m, B,
                        n.Bmax, n.err);
    }
  }
  return conv_fwd_raw<AT>(p, a, n.W + n.woff[layer], n.cin[layer], n.cout[layer], o, m, B, false);
}

// dW (written, not added) and, when din is not null, din for the loss whose
// gradient with respect to out = conv3x3(in, W) is dout
template <typename AT>
bec_status conv_bwd_raw(bec_problem* p, const AT* a, const AT* d, const float* W, float* dW,
                        int ci, int co, AT* di, int m, int B) {
  NetState& n = *p->net;
  const long long npix = (long long)B * m * m;
  const int nw = 9 * ci * co;
  long long nblk = (npix + 255) / 256;
  if (nblk > 512) nblk = 512;
  const long long per = (npix + nblk - 1) / nblk;
  const unsigned g = (unsigned)((npix + net::kConvThreads - 1) / net::kConvThreads);
#define BEC_CB(CI, CO)                                                                            \
  if (ci == CI && co == CO) {                                                                     \
    BEC_LAUNCH_BEGIN(p);                                                                          \
    net::conv3x3_bwd_weight_kernel<AT, CI, CO><<<(unsigned)nblk, 256, 0, p->stream>>>(a, d, n.wpart, m, npix, per); \
    BEC_LAUNCH_CHECK(p, "net_conv_wgrad_kernel");                                                 \
    if (di) {                                                                                     \
      BEC_LAUNCH_BEGIN(p);                                                                        \
      net::conv3x3_bwd_data_kernel<AT, CI, CO><<<g, net::kConvThreads, 0, p->stream>>>(d, W, di, m, npix); \
      BEC_LAUNCH_CHECK(p, "net_conv_dgrad_kernel");                                               \
    }                                                                                             \
  } else
  BEC_CB(1, 4) BEC_CB(4, 4) BEC_CB(4, 8) BEC_CB(1, 32) BEC_CB(32, 32) BEC_CB(32, 8) BEC_CB(1, 8)
  BEC_CB(8, 4) BEC_CB(8, 32) {
    set_error("unsupported network channel count");
    return BEC_EUNSUPPORTED;
  }
#undef BEC_CB
  BEC_LAUNCH_BEGIN(p);
  net::reduce_parts_kernel<<<(nw + 255) / 256, 256, 0, p->stream>>>(n.wpart, (int)nblk, nw, dW);
  BEC_LAUNCH_CHECK(p, "net_wgrad_reduce_kernel");
  return BEC_OK;
}

template <typename AT>
bec_status conv_bwd(bec_problem* p, const void* in, const void* dout, int layer, void* din, int m,
                    int B) {
  NetState& n = *p->net;
  return conv_bwd_raw<AT>(p, static_cast<const AT*>(in), static_cast<const AT*>(dout),
                          n.W + n.woff[layer], n.G + n.woff[layer], n.cin[layer], n.cout[layer],
                          static_cast<AT*>(din), m, B);
}

bool aligned16p(const void* q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

template <typename AT>
bec_status restrict_ch(bec_problem* p, const void* in, void* out, int lf, int B, float scale,
                       bool add) {
  NetState& n = *p->net;
  const int mf = n.sz[lf], mc = n.sz[lf + 1];
  const long long cnt = (long long)B * mc * mc * n.C;
  constexpr int V = net::ChVec<AT>::V;
  if (n.C % V == 0 && aligned16p(in) && aligned16p(out)) {   // 16-byte channel groups
    const long long cv = cnt / V;
    BEC_LAUNCH_BEGIN(p);
    if (add)
      net::restrict_ch_vec_kernel<AT, true><<<grid_for(cv), kT, 0, p->stream>>>(
          static_cast<const AT*>(in), static_cast<AT*>(out), mf, mc, n.C, cv, scale);
    else
      net::restrict_ch_vec_kernel<AT, false><<<grid_for(cv), kT, 0, p->stream>>>(
          static_cast<const AT*>(in), static_cast<AT*>(out), mf, mc, n.C, cv, scale);
    BEC_LAUNCH_CHECK(p, "net_restrict_kernel");
    return BEC_OK;
  }
  BEC_LAUNCH_BEGIN(p);
  if (add)
    net::restrict_ch_kernel<AT, true><<<grid_for(cnt), kT, 0, p->stream>>>(
        static_cast<const AT*>(in), static_cast<AT*>(out), mf, mc, n.C, cnt, scale);
  else
    net::restrict_ch_kernel<AT, false><<<grid_for(cnt), kT, 0, p->stream>>>(
        static_cast<const AT*>(in), static_cast<AT*>(out), mf, mc, n.C, cnt, scale);
  BEC_LAUNCH_CHECK(p, "net_restrict_kernel");
  return BEC_OK;
}

template <typename AT>
bec_status prolong_ch(bec_problem* p, const void* in, const void* add_src, void* out, int lf, int B,
                      float scale) {
  NetState& n = *p->net;
  const int mf = n.sz[lf], mc = n.sz[lf + 1];
  const long long cnt = (long long)B * mf * mf * n.C;
  constexpr int V = net::ChVec<AT>::V;
  if (n.C % V == 0 && aligned16p(in) && aligned16p(add_src) && aligned16p(out)) {
    const long long cv = cnt / V;
    BEC_LAUNCH_BEGIN(p);
    net::prolong_ch_vec_kernel<AT><<<grid_for(cv), kT, 0, p->stream>>>(
        static_cast<const AT*>(in), static_cast<const AT*>(add_src), static_cast<AT*>(out), mc, mf,
        n.C, cv, scale);
    BEC_LAUNCH_CHECK(p, "net_prolong_kernel");
    return BEC_OK;
  }
  BEC_LAUNCH_BEGIN(p);
  net::prolong_ch_kernel<AT><<<grid_for(cnt), kT, 0, p->stream>>>(
      static_cast<const AT*>(in), static_cast<const AT*>(add_src), static_cast<AT*>(out), mc, mf,
      n.C, cnt, scale);
  BEC_LAUNCH_CHECK(p, "net_prolong_kernel");
  return BEC_OK;
}

template <typename AT>
bec_status add_into(bec_problem* p, void* d, const void* e, int level, int B) {
  NetState& n = *p->net;
  const long long cnt = (long long)B * n.sz[level] * n.sz[level] * n.C;
  BEC_LAUNCH_BEGIN(p);
  net::add_kernel<AT><<<grid_for(cnt), kT, 0, p->stream>>>(static_cast<AT*>(d),
                                                           static_cast<const AT*>(e), cnt);
  BEC_LAUNCH_CHECK(p, "net_add_kernel");
  return BEC_OK;
}

#define BEC_TRY(expr)            \
  do {                           \
    bec_status _s = (expr);      \
    if (_s != BEC_OK) return _s; \
  } while (0)

// features of B samples (rows n.row, frequencies n.lam) from n.res into act[X]
// gated layer i: its input and output activations (its level is
// net::kGateLevel[i])
constexpr int kGateIn[net::kGates] = {A_X, A_H0, A_R0, A_R1, A_R2, A_P2, A_P1, A_P0};
constexpr int kGateOut[net::kGates] = {A_H0, A_S0, A_S1, A_S2, A_S3, A_U2, A_U1, A_U0};
constexpr int kGateLevel[net::kGates] = {0, 0, 1, 2, 3, 2, 1, 0};

// the a-gates of every gated layer from the current weights:
// Z1_i = relu(conv(la_l, A1_i)), GA_i = 1 + tanh(conv(Z1_i, A2_i))
bec_status gates_fwd(bec_problem* p) {
  NetState& n = *p->net;
  for (int i = 0; i < net::kGates; ++i) {
    const int l = kGateLevel[i], m = n.sz[l];
    BEC_TRY(conv_fwd_raw<float>(p, n.la_lv[l], n.W + n.goff.a1[i], 1, net::kGateAHidden, n.Z1[i],
                                m, 1, true));
    BEC_TRY(conv_fwd_raw<float>(p, n.Z1[i], n.W + n.goff.a2[i], net::kGateAHidden, n.C, n.GA[i], m,
                                1, false));
    const long long cnt = (long long)m * m * n.C;
    BEC_LAUNCH_BEGIN(p);
    net::one_plus_tanh_kernel<<<grid_for(cnt), kT, 0, p->stream>>>(n.GA[i], cnt);
    BEC_LAUNCH_CHECK(p, "net_gate_tanh_kernel");
    if (n.GAt[i] != nullptr) {
      BEC_LAUNCH_BEGIN(p);
      gate_transpose_kernel<<<grid_for(cnt), kT, 0, p->stream>>>(n.GA[i], n.GAt[i], (long long)m * m,
                                                                 n.C);
      BEC_LAUNCH_CHECK(p, "net_gate_transpose_kernel");
    }
  }
  n.gates_ok = true;
  return BEC_OK;
}

// input planes of Bc complex samples (rows n.cur_row of n.res, frequencies
// n.cur_lam) as 2 Bc network samples
template <typename AT>
bec_status features(bec_problem* p, int Bc) {
  NetState& n = *p->net;
  const int mc = n.sz[0];
  const long long mcc = (long long)mc * mc;
  BEC_LAUNCH_BEGIN(p);
  feat_restrict_kernel<<<grid_for(Bc * mcc), kT, 0, p->stream>>>(
      reinterpret_cast<const float2*>(n.res), n.cur_row, reinterpret_cast<float2*>(n.rc), n.mf, mc, Bc);
  BEC_LAUNCH_CHECK(p, "net_feat_restrict_kernel");
  BEC_LAUNCH_BEGIN(p);
  feat_fill_kernel<AT><<<grid_for(Bc * mcc), kT, 0, p->stream>>>(
      reinterpret_cast<const float2*>(n.rc), 1.f / n.poles.s[0], static_cast<AT*>(n.act[A_X]),
      (sizeof(AT) == 2 && n.tc) ? n.x16 : nullptr, mcc, Bc);
  BEC_LAUNCH_CHECK(p, "net_feat_fill_kernel");
  return BEC_OK;
}

// gated layer i: out = conv(in, W_i) * GA_i; training keeps the product's
// first factor in n.pre[i] for the backward pass.  Inference on the tensor
// cores applies the gate in the convolution's epilogue (no second pass over
// the layer's output).
template <typename AT>
bec_status gate_layer(bec_problem* p, int i, int B, bool training) {
  NetState& n = *p->net;
  const int m = n.sz[kGateLevel[i]];
  AT* out = static_cast<AT*>(n.act[kGateOut[i]]);
  if (!training && sizeof(AT) == 2 && n.tc)
    return conv_fwd<AT>(p, n.act[kGateIn[i]], i, out, m, B, n.GAt[i]);
  AT* pre = training ? static_cast<AT*>(n.pre[i]) : out;
  BEC_TRY(conv_fwd<AT>(p, n.act[kGateIn[i]], i, pre, m, B));
  const long long mmC = (long long)m * m * n.C;
  BEC_LAUNCH_BEGIN(p);
  net::gate_apply_kernel<AT><<<dim3(grid_for(mmC), B), kT, 0, p->stream>>>(pre, out, n.GA[i], mmC);
  BEC_LAUNCH_CHECK(p, "net_gate_kernel");
  return BEC_OK;
}

template <typename AT>
bec_status forward(bec_problem* p, int B, bool training) {
  NetState& n = *p->net;
  void** a = n.act;
  if (sizeof(AT) == 2 && n.tc) BEC_TRY(tc_convert_weights(p, n.W, n.woff, n.wt));
  BEC_TRY(gate_layer<AT>(p, 0, B, training));
  BEC_TRY(gate_layer<AT>(p, 1, B, training));
  BEC_TRY(restrict_ch<AT>(p, a[A_S0], a[A_R0], 0, B, 1.f, false));
  BEC_TRY(gate_layer<AT>(p, 2, B, training));
  BEC_TRY(restrict_ch<AT>(p, a[A_S1], a[A_R1], 1, B, 1.f, false));
  BEC_TRY(gate_layer<AT>(p, 3, B, training));
  BEC_TRY(restrict_ch<AT>(p, a[A_S2], a[A_R2], 2, B, 1.f, false));
  BEC_TRY(gate_layer<AT>(p, 4, B, training));
  BEC_TRY(prolong_ch<AT>(p, a[A_S3], a[A_S2], a[A_P2], 2, B, 1.f));
  BEC_TRY(gate_layer<AT>(p, 5, B, training));
  BEC_TRY(prolong_ch<AT>(p, a[A_U2], a[A_S1], a[A_P1], 1, B, 1.f));
  BEC_TRY(gate_layer<AT>(p, 6, B, training));
  BEC_TRY(prolong_ch<AT>(p, a[A_U1], a[A_S0], a[A_P0], 0, B, 1.f));
  BEC_TRY(gate_layer<AT>(p, 7, B, training));
  BEC_TRY(conv_fwd<AT>(p, a[A_U0], 8, a[A_Y], n.sz[0], B));
  return BEC_OK;
}

// efine[b] = P_0 ec_b of the last forward pass, b < Bc (frequencies n.cur_lam)
template <typename AT>
bec_status correction_fine(bec_problem* p, int Bc) {
  NetState& n = *p->net;
  const long long mff = (long long)n.mf * n.mf, mcc = (long long)n.sz[0] * n.sz[0];
  BEC_LAUNCH_BEGIN(p);
  pole_sum_kernel<AT><<<grid_for(Bc * mcc), kT, 0, p->stream>>>(
      static_cast<const AT*>(n.act[A_Y]), n.cur_lam, p->tab.lamf32, n.poles,
      reinterpret_cast<float2*>(n.ecb), mcc, Bc);
  BEC_LAUNCH_CHECK(p, "net_pole_sum_kernel");
  BEC_LAUNCH_BEGIN(p);
  out_prolong_kernel<<<grid_for(Bc * mff), kT, 0, p->stream>>>(
      reinterpret_cast<const float2*>(n.ecb), reinterpret_cast<float2*>(n.efine), n.sz[0], n.mf, Bc);
  BEC_LAUNCH_CHECK(p, "net_out_prolong_kernel");
  return BEC_OK;
}

// backward through gated layer i, d = dL/d(out_i) on entry: the gate
// gradient dGA_i (summed over the samples), then d <- d * GA_i = dL/d(pre_i)
template <typename AT>
bec_status gate_bwd(bec_problem* p, int i, void* dv, int B) {
  NetState& n = *p->net;
  const int m = n.sz[kGateLevel[i]];
  const long long mmC = (long long)m * m * n.C;
  AT* d = static_cast<AT*>(dv);
  const AT* pre = static_cast<const AT*>(n.pre[i]);
  BEC_LAUNCH_BEGIN(p);
  net::gate_dga_kernel<AT><<<grid_for(mmC), kT, 0, p->stream>>>(d, pre, n.dGA[i], mmC, B);
  BEC_LAUNCH_CHECK(p, "net_gate_dga_kernel");
  BEC_LAUNCH_BEGIN(p);
  net::gate_scale_grad_kernel<AT><<<dim3(grid_for(mmC), B), kT, 0, p->stream>>>(d, n.GA[i], mmC);
  BEC_LAUNCH_CHECK(p, "net_gate_grad_kernel");
  return BEC_OK;
}

// gradients of every weight for the loss whose dL/dY is in grad[A_Y], over
// B = 2 Bc network samples
template <typename AT>
bec_status backward(bec_problem* p, int B) {
  NetState& n = *p->net;
  void** a = n.act;
  void** d = n.grad;
  BEC_TRY(conv_bwd<AT>(p, a[A_U0], d[A_Y], 8, d[A_U0], n.sz[0], B));
  BEC_TRY(gate_bwd<AT>(p, 7, d[A_U0], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_P0], d[A_U0], 7, d[A_P0], n.sz[0], B));
  // P0 = P U1 + S0:  dU1 = P^T dP0 = 4 R dP0,  dS0 = dP0 (+ more below)
  BEC_TRY(restrict_ch<AT>(p, d[A_P0], d[A_U1], 0, B, 4.f, false));
  BEC_TRY(gate_bwd<AT>(p, 6, d[A_U1], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_P1], d[A_U1], 6, d[A_P1], n.sz[1], B));
  BEC_TRY(restrict_ch<AT>(p, d[A_P1], d[A_U2], 1, B, 4.f, false));
  BEC_TRY(gate_bwd<AT>(p, 5, d[A_U2], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_P2], d[A_U2], 5, d[A_P2], n.sz[2], B));
  BEC_TRY(restrict_ch<AT>(p, d[A_P2], d[A_S3], 2, B, 4.f, false));
  BEC_TRY(gate_bwd<AT>(p, 4, d[A_S3], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_R2], d[A_S3], 4, d[A_R2], n.sz[3], B));
  // S2 feeds R2 = R S2 and P2 = P S3 + S2:  dS2 = R^T dR2 + dP2 = P dR2 / 4 + dP2
  BEC_TRY(prolong_ch<AT>(p, d[A_R2], d[A_P2], d[A_S2], 2, B, 0.25f));
  BEC_TRY(gate_bwd<AT>(p, 3, d[A_S2], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_R1], d[A_S2], 3, d[A_R1], n.sz[2], B));
  BEC_TRY(prolong_ch<AT>(p, d[A_R1], d[A_P1], d[A_S1], 1, B, 0.25f));
  BEC_TRY(gate_bwd<AT>(p, 2, d[A_S1], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_R0], d[A_S1], 2, d[A_R0], n.sz[1], B));
  BEC_TRY(prolong_ch<AT>(p, d[A_R0], d[A_P0], d[A_S0], 0, B, 0.25f));
  BEC_TRY(gate_bwd<AT>(p, 1, d[A_S0], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_H0], d[A_S0], 1, d[A_H0], n.sz[0], B));
  BEC_TRY(gate_bwd<AT>(p, 0, d[A_H0], B));
  BEC_TRY(conv_bwd<AT>(p, a[A_X], d[A_H0], 0, nullptr, n.sz[0], B));
  // the a-gates' weights: through GA = 1 + tanh(conv(Z1, A2)), Z1 = relu(conv(la, A1))
  for (int i = 0; i < net::kGates; ++i) {
    const int l = kGateLevel[i], m = n.sz[l];
    const long long cnt = (long long)m * m * n.C;
    BEC_LAUNCH_BEGIN(p);
    net::dtanh_kernel<<<grid_for(cnt), kT, 0, p->stream>>>(n.dGA[i], n.GA[i], n.dA, cnt);
    BEC_LAUNCH_CHECK(p, "net_gate_dtanh_kernel");
    BEC_TRY(conv_bwd_raw<float>(p, n.Z1[i], n.dA, n.W + n.goff.a2[i], n.G + n.goff.a2[i],
                                net::kGateAHidden, n.C, n.dZ, m, 1));
    const long long hz = (long long)m * m * net::kGateAHidden;
    BEC_LAUNCH_BEGIN(p);
    net::relu_mask_kernel<float><<<grid_for(hz), kT, 0, p->stream>>>(n.dZ, n.Z1[i], hz);
    BEC_LAUNCH_CHECK(p, "net_relu_mask_kernel");
    BEC_TRY(conv_bwd_raw<float>(p, n.la_lv[l], n.dZ, n.W + n.goff.a1[i], n.G + n.goff.a1[i], 1,
                                net::kGateAHidden, nullptr, m, 1));
  }
  return BEC_OK;
}

// loss parts (per complex sample) and dL/dY of the 2 Bc network samples, for
// the Bc complex samples in n.row against the coarse targets n.etgt
template <typename AT>
bec_status loss_and_dy(bec_problem* p, int Bc) {
  NetState& n = *p->net;
  const long long mcc = (long long)n.sz[0] * n.sz[0];
  BEC_LAUNCH_BEGIN(p);
  closs_parts_kernel<AT><<<Bc, 256, 0, p->stream>>>(
      static_cast<const AT*>(n.act[A_Y]), reinterpret_cast<const float2*>(n.etgt), n.cur_row,
      n.cur_lam, p->tab.lamf32, n.poles, n.part, mcc, Bc);
  BEC_LAUNCH_CHECK(p, "net_loss_kernel");
  BEC_LAUNCH_BEGIN(p);
  closs_grad_kernel<AT><<<grid_for(Bc * mcc), kT, 0, p->stream>>>(
      static_cast<const AT*>(n.act[A_Y]), reinterpret_cast<const float2*>(n.etgt), n.cur_row,
      n.cur_lam, p->tab.lamf32, n.poles, n.part, static_cast<AT*>(n.grad[A_Y]), mcc, Bc);
  BEC_LAUNCH_CHECK(p, "net_loss_grad_kernel");
  return BEC_OK;
}

bec_status set_samples(bec_problem* p, const int* rows, const int* lams, int B) {
  NetState& n = *p->net;
  for (int b = 0; b < B; ++b) {
    n.h_idx[b] = rows[b];
    n.h_idx[n.Bmax + b] = lams[b];
  }
  BEC_CUDA_TRY(cudaMemcpyAsync(n.row, n.h_idx, B * sizeof(int), cudaMemcpyHostToDevice, p->stream));
  BEC_CUDA_TRY(cudaMemcpyAsync(n.lam, n.h_idx + n.Bmax, B * sizeof(int), cudaMemcpyHostToDevice,
                               p->stream));
  // the staging buffer is reused by the next call only after a stream sync
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  n.cur_row = n.row;
  n.cur_lam = n.lam;
  return BEC_OK;
}

bec_status adam_step(bec_problem* p, float lr) {
  NetState& n = *p->net;
  n.adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float lr_t = lr * sqrtf(1.f - powf(b2, (float)n.adam_t)) / (1.f - powf(b1, (float)n.adam_t));
  const int nw = (int)n.nparam;
  BEC_LAUNCH_BEGIN(p);
  net::adam_kernel<<<(nw + 255) / 256, 256, 0, p->stream>>>(n.W, n.Mo, n.Ve, n.G, nw, lr_t, b1, b2,
                                                            1e-8f);
  BEC_LAUNCH_CHECK(p, "net_adam_kernel");
  return BEC_OK;
}

// Training pairs for every frequency: res = b - B V(b), and the coarse
// target etgt = B_1^{-1} R_0 res by `sweeps` defect-correction V-cycles from
// level 1 of the hierarchy.  The right-hand sides b: with kry < 0 a random
// Gaussian one per frequency; else the time spectrum (Step 1 of Sec. 4) of
// Krylov vector kry of the recording solve, i.e. exactly what the V-cycles
// of that solve were given.
bec_status make_pairs(bec_problem* p, int sweeps, int kry) {
  NetState& n = *p->net;
  MgLevel& L0 = p->mg.lv[0];
  const long long tot = (long long)p->mg.K * L0.J;
  const long long tot1 = (long long)p->mg.K * p->mg.lv[1].J;
  if (kry < 0) {
    BEC_LAUNCH_BEGIN(p);
    gauss_fill_kernel<<<grid_for(tot), kT, 0, p->stream>>>(
        static_cast<float2*>(L0.b), tot, 0xB5C0FFEEull + (n.rng_ctr++) * 0x100000001ull);
    BEC_LAUNCH_CHECK(p, "net_gauss_fill_kernel");
  } else {
    // V_kry is stored unnormalised; sigma[kry] = 1 / ||V_kry|| scales it as
    // the solve's preconditioner apply did.  V_0 is the right-hand side
    // itself (a solve from zero does not copy it into V).
    const double* v = kry == 0 ? n.kf : p->V + (long long)kry * p->U;
    BEC_TRY(launch_time_fwd(p, v, L0.b, 0, p->sigma + kry));
  }
  // keep the right-hand side: the V-cycle reuses L0.b
  BEC_CUDA_TRY(cudaMemcpyAsync(n.ework, L0.b, tot * sizeof(float2), cudaMemcpyDeviceToDevice, p->stream));
  BEC_TRY(mg_vcycle(p));
  BEC_TRY(mg_residual_level0(p, n.res, L0.x, n.ework));          // res = b - B V(b)
  BEC_TRY(mg_restrict_to(p, 0, n.rcall, n.res));                 // R_0 res
  BEC_CUDA_TRY(cudaMemsetAsync(n.etgt, 0, tot1 * sizeof(float2), p->stream));
  for (int it = 0; it < sweeps; ++it) {
    BEC_TRY(mg_residual_level(p, 1, p->mg.lv[1].b, n.etgt, n.rcall));   // b_1 = R_0 res - B_1 e
    BEC_TRY(mg_vcycle_from(p, 1));
    BEC_LAUNCH_BEGIN(p);
    axpy_c_kernel<<<grid_for(tot1), kT, 0, p->stream>>>(reinterpret_cast<float2*>(n.etgt),
                                                        static_cast<const float2*>(p->mg.lv[1].x), tot1);
    BEC_LAUNCH_CHECK(p, "net_axpy_kernel");
  }
  return BEC_OK;
}

// The recording solve: FGMRES preconditioned by the multigrid alone (the
// route bypassed) on a random right-hand side, to RES 1e-10 within one
// restart cycle.  Its Krylov basis stays in the problem's V: the inputs of
// its preconditioner applies, which the training then turns into pairs.
bec_status record_krylov(bec_problem* p, unsigned long long seed) {
  NetState& n = *p->net;
  BEC_LAUNCH_BEGIN(p);
  uniform_fill_f64_kernel<<<grid_for(p->U), kT, 0, p->stream>>>(n.kf, p->U,
                                                                0x5EEDF00Dull ^ (seed * 0x9E37ull));
  BEC_LAUNCH_CHECK(p, "net_uniform_fill_kernel");
  bec_gmres_opts o{};
  o.restart = p->max_restart;
  o.maxit = p->max_restart;
  o.rtol = 1e-10;
  o.flexible = p->desc.flexible ? 1 : 0;
  bec_gmres_info info{};
  n.bypass = true;
  const bec_status st = gmres_solve_one(p, n.kf, n.ku, &o, &info);
  n.bypass = false;
  if (st != BEC_OK && st != BEC_ENOTCONV) return st;
  n.nkry = info.iters > 0 ? info.iters : 0;
  return BEC_OK;
}

// The learning rate of step s of `steps`: a linear warm-up over the first
// kWarmup steps (the first Adam steps move every weight by about lr whatever
// its gradient), then a cosine decay to lr / 10 at the last step (the final
// weights come from small steps, whatever the loss did on the way).
constexpr int kWarmup = 100;
float lr_at(float lr, int s, int steps) {
  if (s < kWarmup) return lr * (float)(s + 1) / kWarmup;
  const int span = steps - kWarmup;
  const double t = span > 1 ? (double)(s - kWarmup) / (span - 1) : 1.0;
  return (float)(lr * (0.1 + 0.45 * (1.0 + std::cos(M_PI * t))));
}

template <typename AT>
bec_status train_t(bec_problem* p, int steps, int batch, float lr, unsigned long long seed,
                   double* loss_hist) {
  NvtxRange range("bec learned training");
  NetState& n = *p->net;
  const int K = p->mg.K;
  unsigned long long st = seed * 6364136223846793005ull + 1442695040888963407ull;
  std::vector<int> rows(batch);
  const int regen = (K + batch - 1) / batch;   // batches drawn from one set of pairs
  n.gates_ok = false;
  n.cal_ok = false;
  BEC_TRY(record_krylov(p, seed));
  int sets = 0;
  for (int s = 0; s < steps; ++s) {
    // fresh pairs, alternately from the recorded Krylov vectors in turn (what
    // the solve's V-cycles are given) and from a random Gaussian right-hand
    // side per frequency (every mode the V-cycle leaves, so that the
    // correction is trained not to amplify modes outside the Krylov space)
    if (s % regen == 0) {
      const bool krylov = n.nkry > 0 && (sets & 1) == 0;
      BEC_TRY(make_pairs(p, 12, krylov ? (sets / 2) % n.nkry : -1));
      ++sets;
    }
    for (int b = 0; b < batch; ++b) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      rows[b] = (int)((st >> 33) % (unsigned long long)K);
    }
    BEC_TRY(set_samples(p, rows.data(), rows.data(), batch));
    BEC_TRY(gates_fwd(p));
    BEC_TRY(features<AT>(p, batch));
    BEC_TRY(forward<AT>(p, 2 * batch, true));
    BEC_TRY(loss_and_dy<AT>(p, batch));
    BEC_TRY(backward<AT>(p, 2 * batch));
    BEC_TRY(adam_step(p, lr_at(lr, s, steps)));
    if (loss_hist) {
      BEC_CUDA_TRY(cudaMemcpyAsync(n.h_part, n.part, 2 * batch * sizeof(double),
                                   cudaMemcpyDeviceToHost, p->stream));
      BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
      double l = 0.0;
      for (int b = 0; b < batch; ++b) l += n.h_part[2 * b] / n.h_part[2 * b + 1];
      loss_hist[s] = l / batch;
    }
  }
  n.gates_ok = false;   // the weights moved after the last gates_fwd
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  return net_check(p);
}

// x1 = x + P_0 ec(R_0 (b - B x)) for every frequency, into n.xnew, from
// the residual in n.res (batches of Bmax / 2 frequencies, Bmax network
// samples)
template <typename AT>
bec_status corrected_iterate(bec_problem* p) {
  NetState& n = *p->net;
  MgLevel& L0 = p->mg.lv[0];
  const int K = p->mg.K;
  const long long mff = (long long)n.mf * n.mf;
  if (!n.gates_ok) BEC_TRY(gates_fwd(p));
  const int bc = n.Bmax / 2;
  for (int k0 = 0; k0 < K; k0 += bc) {
    const int B = K - k0 < bc ? K - k0 : bc;
    n.cur_row = n.iota + k0;
    n.cur_lam = n.iota + k0;
    BEC_TRY(features<AT>(p, B));
    BEC_TRY(forward<AT>(p, 2 * B, false));
    BEC_TRY(correction_fine<AT>(p, B));
    BEC_LAUNCH_BEGIN(p);
    add_corr_kernel<<<grid_for(B * mff), kT, 0, p->stream>>>(
        reinterpret_cast<float2*>(n.xnew), static_cast<const float2*>(L0.x),
        reinterpret_cast<const float2*>(n.efine), mff, k0, B);
    BEC_LAUNCH_CHECK(p, "net_add_correction_kernel");
  }
  return BEC_OK;
}

// The calibration apply: the V-cycle and the correction on the fixed
// right-hand side of calibration_fill_kernel at every frequency; alpha = the
// minimal-residual step sum_k <B d, res> / sum_k ||B d||^2, d = x2 - x (0
// when the sums vanish or are not finite, the V-cycle's iterates then kept),
// and the residual ratio it reaches per frequency.  Uses the
// multigrid's level-0 arrays, so it runs before an apply's Step 1.
template <typename AT>
bec_status judge_t(bec_problem* p);

template <typename AT>
bec_status calibrate_t(bec_problem* p) {
  NvtxRange range("bec learned calibration");
  NetState& n = *p->net;
  MgLevel& L0 = p->mg.lv[0];
  const int K = p->mg.K;
  const long long mff = (long long)n.mf * n.mf;
  BEC_LAUNCH_BEGIN(p);
  calibration_fill_kernel<<<grid_for(2 * K * mff), kT, 0, p->stream>>>(static_cast<float*>(L0.b),
                                                                       2 * K * mff);
  BEC_LAUNCH_CHECK(p, "net_calibration_fill_kernel");
  BEC_TRY(mg_vcycle(p));
  BEC_TRY(mg_residual_level0(p, n.res, L0.x, L0.b));
  BEC_TRY(corrected_iterate<AT>(p));
  // x2 = one damped-Jacobi sweep on x1 into L0.r; its residual into xnew
  BEC_TRY(mg_smooth_level0(p, L0.r, n.xnew, L0.b));
  BEC_TRY(mg_residual_level0(p, n.xnew, L0.r, L0.b));
  BEC_LAUNCH_BEGIN(p);
  mr_dots_kernel<<<dim3(K, kMrSplit), 256, 0, p->stream>>>(
      reinterpret_cast<const float2*>(n.res), reinterpret_cast<const float2*>(n.xnew), n.jpart, mff);
  BEC_LAUNCH_CHECK(p, "net_calibration_dots_kernel");
  int* fb = reinterpret_cast<int*>(n.part + 5 * K);
  BEC_CUDA_TRY(cudaMemsetAsync(fb, 0, sizeof(int), p->stream));
  BEC_LAUNCH_BEGIN(p);
  mr_alpha_kernel<<<1, 256, 0, p->stream>>>(n.jpart, n.part, n.alpha, K, n.part + 4 * K, fb);
  BEC_LAUNCH_CHECK(p, "net_calibration_alpha_kernel");
  if (n.judge) {
    BEC_TRY(judge_t<AT>(p));
  } else {
    // all bits set: NaN radii (no judgement)
    BEC_CUDA_TRY(cudaMemsetAsync(n.jrho, 0xFF, (2 * K + 2) * sizeof(double), p->stream));
  }
  n.cal_ok = true;
  return BEC_OK;
}

// The multigrid judges the correction: kJudgeIters power iterations per
// frequency on the error operator E_k = I - M_k B_k of one apply, from the
// calibration right-hand side (normalised per frequency), for M_k the
// V-cycle alone and for the corrected preconditioner with the calibrated
// step.  The last ||E_k v|| (||v|| = 1) estimates E_k's spectral radius; the
// correction is kept only when its largest estimate over k is below the
// V-cycle's (one decision for all frequencies: a per-frequency choice would
// depend on k non-analytically).  Uses the calibration's arrays.
constexpr int kJudgeIters = 10;

template <typename AT>
bec_status judge_t(bec_problem* p) {
  NvtxRange range("bec learned judge");
  NetState& n = *p->net;
  MgLevel& L0 = p->mg.lv[0];
  const int K = p->mg.K;
  const long long mff = (long long)n.mf * n.mf, tot = K * mff;
  float2* v = reinterpret_cast<float2*>(n.ework);
  auto normalise = [&](int arm) -> bec_status {
    BEC_LAUNCH_BEGIN(p);
    knorm_parts_kernel<<<dim3(K, kMrSplit), 256, 0, p->stream>>>(v, n.jpart, mff);
    BEC_LAUNCH_CHECK(p, "net_judge_norm_kernel");
    BEC_LAUNCH_BEGIN(p);
    knorm_scale_kernel<<<grid_for(tot), kT, 0, p->stream>>>(v, n.jpart, n.jrho + arm * K, mff, K);
    BEC_LAUNCH_CHECK(p, "net_judge_scale_kernel");
    return BEC_OK;
  };
  for (int arm = 0; arm < 2; ++arm) {
    BEC_LAUNCH_BEGIN(p);
    calibration_fill_kernel<<<grid_for(2 * tot), kT, 0, p->stream>>>(n.ework, 2 * tot);
    BEC_LAUNCH_CHECK(p, "net_calibration_fill_kernel");
    BEC_TRY(normalise(arm));
    for (int it = 0; it < kJudgeIters; ++it) {
      // L0.b = 0 - B v, L0.x = M L0.b, v <- v + L0.x = E v
      BEC_CUDA_TRY(cudaMemsetAsync(n.xnew, 0, tot * sizeof(float2), p->stream));
      BEC_TRY(mg_residual_level0(p, L0.b, n.ework, n.xnew));
      BEC_TRY(mg_vcycle(p));
      if (arm == 1) {
        BEC_TRY(mg_residual_level0(p, n.res, L0.x, L0.b));
        BEC_TRY(corrected_iterate<AT>(p));
        BEC_TRY(mg_smooth_level0(p, L0.r, n.xnew, L0.b));
        BEC_LAUNCH_BEGIN(p);
        mr_update_kernel<<<grid_for(tot), kT, 0, p->stream>>>(
            static_cast<float2*>(L0.x), static_cast<const float2*>(L0.r), n.alpha, tot);
        BEC_LAUNCH_CHECK(p, "net_step_kernel");
      }
      BEC_LAUNCH_BEGIN(p);
      axpy_c_kernel<<<grid_for(tot), kT, 0, p->stream>>>(v, static_cast<const float2*>(L0.x), tot);
      BEC_LAUNCH_CHECK(p, "net_axpy_kernel");
      BEC_TRY(normalise(arm));
    }
  }
  BEC_LAUNCH_BEGIN(p);
  judge_kernel<<<1, 1, 0, p->stream>>>(n.jrho, K, n.alpha, reinterpret_cast<int*>(n.part + 5 * K));
  BEC_LAUNCH_CHECK(p, "net_judge_kernel");
  return BEC_OK;
}

template <typename AT>
bec_status correct_t(bec_problem* p) {
  NvtxRange range("bec learned correction");
  NetState& n = *p->net;
  MgLevel& L0 = p->mg.lv[0];
  const int K = p->mg.K;
  const long long mff = (long long)n.mf * n.mf;
  // residual the V-cycle left, x1 = x + the correction
  BEC_TRY(mg_residual_level0(p, n.res, L0.x, L0.b));
  BEC_TRY(corrected_iterate<AT>(p));
  // x2 = one damped-Jacobi sweep on x1 (the post-smoothing of a prolonged
  // correction) into L0.r, then x <- x + alpha (x2 - x)
  BEC_TRY(mg_smooth_level0(p, L0.r, n.xnew, L0.b));
  BEC_LAUNCH_BEGIN(p);
  mr_update_kernel<<<grid_for(K * mff), kT, 0, p->stream>>>(
      static_cast<float2*>(L0.x), static_cast<const float2*>(L0.r), n.alpha, K * mff);
  BEC_LAUNCH_CHECK(p, "net_step_kernel");
  return BEC_OK;
}

bec_status dalloc(void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("cudaMalloc (learned correction)");
    return BEC_ENOMEM;
  }
  return BEC_OK;
}

}  // namespace

bec_status net_setup(bec_problem* p, const double* a_nodes, int channels, int fp32_acts, int bmax) {
  if (p->desc.precision != BEC_PC_FP32) return BEC_EINVAL;
  if (p->m < 31) {
    set_error("the learned route needs nx >= 31 (4 network levels below the fine grid)");
    return BEC_EINVAL;
  }
  NetState* n = new (std::nothrow) NetState();
  if (n == nullptr) return BEC_ENOMEM;
  p->net = n;
  n->C = channels;
  n->fp32 = fp32_acts != 0;
  n->mf = p->m;
  n->sz[0] = (p->m - 1) / 2;
  for (int l = 1; l < 4; ++l) n->sz[l] = (n->sz[l - 1] - 1) / 2;
  n->Bmax = bmax;
  const int C = channels;
  const int shapes[9][2] = {{1, C}, {C, C}, {C, C}, {C, C}, {C, C},
                            {C, C}, {C, C}, {C, C}, {C, kNetOut}};
  n->woff[0] = 0;
  for (int i = 0; i < 9; ++i) {
    n->cin[i] = shapes[i][0];
    n->cout[i] = shapes[i][1];
    n->woff[i + 1] = n->woff[i] + 9LL * shapes[i][0] * shapes[i][1];
  }
  // then A1_0..7 [3][3][1][8], A2_0..7 [3][3][8][C]
  long long o = n->woff[9];
  for (int i = 0; i < net::kGates; ++i, o += 9LL * net::kGateAHidden) n->goff.a1[i] = o;
  for (int i = 0; i < net::kGates; ++i, o += 9LL * net::kGateAHidden * C) n->goff.a2[i] = o;
  n->nparam = o;
  const long long nw = n->nparam;
  bec_status s = BEC_OK;
  auto chain = [&](bec_status r) { if (s == BEC_OK) s = r; };
  chain(dalloc(reinterpret_cast<void**>(&n->W), nw * sizeof(float)));
  chain(dalloc(reinterpret_cast<void**>(&n->G), nw * sizeof(float)));
  chain(dalloc(reinterpret_cast<void**>(&n->Mo), nw * sizeof(float)));
  chain(dalloc(reinterpret_cast<void**>(&n->Ve), nw * sizeof(float)));
  n->wpart_n = 512LL * 9 * 32 * 32;
  chain(dalloc(reinterpret_cast<void**>(&n->wpart), n->wpart_n * sizeof(float)));
  const size_t asz = n->fp32 ? sizeof(float) : sizeof(__nv_bfloat16);
  for (int a = 0; a < NACT; ++a) {
    const int l = act_level(a);
    const int ch = a == A_X ? 1 : (a == A_Y ? kNetOut : C);
    const size_t bytes = (size_t)bmax * n->sz[l] * n->sz[l] * ch * asz;
    chain(dalloc(&n->act[a], bytes));
    chain(dalloc(&n->grad[a], bytes));
  }
  for (int i = 0; i < net::kGates; ++i) {
    const long long mm = (long long)n->sz[kGateLevel[i]] * n->sz[kGateLevel[i]];
    chain(dalloc(&n->pre[i], (size_t)bmax * mm * C * asz));
    chain(dalloc(reinterpret_cast<void**>(&n->GA[i]), (size_t)mm * C * sizeof(float)));
    if (!n->fp32 && C == 32)   // the tensor-core path (decided below) reads these
      chain(dalloc(reinterpret_cast<void**>(&n->GAt[i]), (size_t)mm * C * sizeof(float)));
    chain(dalloc(reinterpret_cast<void**>(&n->dGA[i]), (size_t)mm * C * sizeof(float)));
    chain(dalloc(reinterpret_cast<void**>(&n->Z1[i]), (size_t)mm * net::kGateAHidden * sizeof(float)));
  }
  const long long mcc = (long long)n->sz[0] * n->sz[0];
  const long long mff = (long long)p->m * p->m;
  const long long K = p->N / 2 + 1;
  for (int l = 0; l < 4; ++l)
    chain(dalloc(reinterpret_cast<void**>(&n->la_lv[l]), (size_t)n->sz[l] * n->sz[l] * sizeof(float)));
  chain(dalloc(reinterpret_cast<void**>(&n->dA), (size_t)mcc * C * sizeof(float)));
  chain(dalloc(reinterpret_cast<void**>(&n->dZ), (size_t)mcc * net::kGateAHidden * sizeof(float)));
  chain(dalloc(reinterpret_cast<void**>(&n->rc), (size_t)bmax * mcc * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->ecb), (size_t)(bmax / 2) * mcc * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->row), bmax * sizeof(int)));
  chain(dalloc(reinterpret_cast<void**>(&n->lam), bmax * sizeof(int)));
  chain(dalloc(reinterpret_cast<void**>(&n->iota), K * sizeof(int)));
  chain(dalloc(reinterpret_cast<void**>(&n->efine), (size_t)bmax * mff * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->res), (size_t)K * mff * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->etgt), (size_t)K * mcc * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->rcall), (size_t)K * mcc * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->ework), (size_t)K * mff * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->xnew), (size_t)K * mff * sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->part), (size_t)(5 * K + 2 * bmax + 2) * sizeof(double)));
  chain(dalloc(reinterpret_cast<void**>(&n->jpart), (size_t)K * kMrSplit * 4 * sizeof(double)));
  chain(dalloc(reinterpret_cast<void**>(&n->alpha), sizeof(float2)));
  chain(dalloc(reinterpret_cast<void**>(&n->jrho), (size_t)(2 * K + 2) * sizeof(double)));
  chain(dalloc(reinterpret_cast<void**>(&n->err), sizeof(int)));
  chain(dalloc(reinterpret_cast<void**>(&n->kf), (size_t)p->U * sizeof(double)));
  chain(dalloc(reinterpret_cast<void**>(&n->ku), (size_t)p->U * sizeof(double)));
  n->tc = !n->fp32 && C == 32 && tc_conv_supported();
  if (n->tc) {
    chain(dalloc(reinterpret_cast<void**>(&n->wt), (size_t)tc_weights_elems() * sizeof(__nv_bfloat16)));
    chain(dalloc(reinterpret_cast<void**>(&n->x16),
                 (size_t)bmax * n->sz[0] * n->sz[0] * 16 * sizeof(__nv_bfloat16)));
  }
  if (s == BEC_OK) {
    if (cudaMallocHost(reinterpret_cast<void**>(&n->h_idx), 2 * bmax * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&n->h_part), (5 * K + 2 * bmax + 2) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      s = BEC_ENOMEM;
    }
  }
  if (s != BEC_OK) return s;
  // log a on the network's levels: level 0 at the coarse nodes (fine node
  // (2i+2, 2j+2)), centred by the mean over all nodes; each next level the
  // full-weighting restriction (1/4, 1/8, 1/16 on the 3 x 3 block around
  // fine (2i+1, 2j+1)) of the one above; and the mean of a
  const int m2 = p->m + 2;
  std::vector<double> la((size_t)m2 * m2);
  double mean_la = 0.0, mean_a = 0.0;
  for (size_t i = 0; i < la.size(); ++i) {
    const double a = a_nodes ? a_nodes[i] : p->a;
    la[i] = std::log(a);
    mean_la += la[i];
    mean_a += a;
  }
  mean_la /= (double)la.size();
  n->a_mean = mean_a / (double)la.size();
  // the poles: sigma_0 = tau a_mean 2 pi^2 (the smoothest mode's shift) up to
  // 2 tau a_mean (m+1)^2 (the largest eigenvalue of the 5-point operator on
  // the grid of spacing 2h), geometric
  {
    const double s0 = p->tau * n->a_mean * 2.0 * M_PI * M_PI;
    const double top = 2.0 * p->tau * n->a_mean * (double)(p->m + 1) * (double)(p->m + 1);
    for (int j = 0; j < net::kPoles; ++j)
      n->poles.s[j] = (float)(s0 * std::pow(top / s0, (double)j / (net::kPoles - 1)));
  }
  std::vector<double> lv((size_t)mcc);
  for (int cy = 0; cy < n->sz[0]; ++cy)
    for (int cx = 0; cx < n->sz[0]; ++cx)
      lv[(size_t)cy * n->sz[0] + cx] = la[(size_t)(2 * cy + 2) * m2 + (2 * cx + 2)] - mean_la;
  for (int l = 0; l < 4; ++l) {
    const int ml = n->sz[l];
    if (l > 0) {
      const int mf = n->sz[l - 1];
      std::vector<double> c((size_t)ml * ml, 0.0);
      for (int cy = 0; cy < ml; ++cy)
        for (int cx = 0; cx < ml; ++cx) {
          double acc = 0.0;
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
              acc += (dy == 0 ? 0.5 : 0.25) * (dx == 0 ? 0.5 : 0.25) *
                     lv[(size_t)(2 * cy + 1 + dy) * mf + (2 * cx + 1 + dx)];
          c[(size_t)cy * ml + cx] = acc;
        }
      lv.swap(c);
    }
    std::vector<float> lf(lv.begin(), lv.end());
    BEC_CUDA_TRY(cudaMemcpy(n->la_lv[l], lf.data(), lf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  std::vector<int> io(K);
  for (long long k = 0; k < K; ++k) io[k] = (int)k;
  BEC_CUDA_TRY(cudaMemcpy(n->iota, io.data(), K * sizeof(int), cudaMemcpyHostToDevice));
  // initial weights from a fixed counter-based normal sequence: the residual
  // path std sqrt(1 / (9 C_in)) (last layer x 0.01: the correction starts
  // small), A1 std 0.3, A2 zero (every gate starts at 1)
  std::vector<float> w(nw, 0.f);
  unsigned long long z = 0x243F6A8885A308D3ull;
  auto normal = [&z]() {
    z = z * 6364136223846793005ull + 1442695040888963407ull;
    const double u1 = ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    z = z * 6364136223846793005ull + 1442695040888963407ull;
    const double u2 = ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
  };
  for (int i = 0; i < 9; ++i) {
    const double sd = std::sqrt(1.0 / (9.0 * n->cin[i])) * (i == 8 ? 0.01 : 1.0);
    for (long long j = n->woff[i]; j < n->woff[i + 1]; ++j) w[j] = (float)(sd * normal());
  }
  for (int i = 0; i < net::kGates; ++i)
    for (long long j = 0; j < 9LL * net::kGateAHidden; ++j) w[n->goff.a1[i] + j] = (float)(0.3 * normal());
  BEC_CUDA_TRY(cudaMemcpy(n->W, w.data(), nw * sizeof(float), cudaMemcpyHostToDevice));
  BEC_CUDA_TRY(cudaMemset(n->Mo, 0, nw * sizeof(float)));
  BEC_CUDA_TRY(cudaMemset(n->Ve, 0, nw * sizeof(float)));
  BEC_CUDA_TRY(cudaMemset(n->err, 0, sizeof(int)));
  return BEC_OK;
}

void net_free(bec_problem* p) {
  NetState* n = p->net;
  if (n == nullptr) return;
  void* ptrs[] = {n->W, n->G, n->Mo, n->Ve, n->wpart, n->rc, n->row, n->lam, n->iota,
                  n->efine, n->res, n->etgt, n->rcall, n->ework, n->xnew, n->part, n->jpart,
                  n->alpha, n->jrho, n->err, n->wt, n->x16, n->dA, n->dZ, n->ecb, n->kf, n->ku};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int l = 0; l < 4; ++l)
    if (n->la_lv[l]) cudaFree(n->la_lv[l]);
  for (int i = 0; i < net::kGates; ++i) {
    void* g[] = {n->pre[i], n->GA[i], n->GAt[i], n->dGA[i], n->Z1[i]};
    for (void* q : g)
      if (q) cudaFree(q);
  }
  for (int a = 0; a < NACT; ++a) {
    if (n->act[a]) cudaFree(n->act[a]);
    if (n->grad[a]) cudaFree(n->grad[a]);
  }
  if (n->h_idx) cudaFreeHost(n->h_idx);
  if (n->h_part) cudaFreeHost(n->h_part);
  delete n;
  p->net = nullptr;
}

bec_status net_correct(bec_problem* p) {
  return p->net->fp32 ? correct_t<float>(p) : correct_t<__nv_bfloat16>(p);
}

bec_status net_calibrate(bec_problem* p) {
  NetState& n = *p->net;
  BEC_TRY(n.fp32 ? calibrate_t<float>(p) : calibrate_t<__nv_bfloat16>(p));
  // read the decision when the stream is not being captured (a capture keeps
  // running the correction, a no-op with alpha = 0)
  n.rejected = false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  BEC_CUDA_TRY(cudaStreamIsCapturing(p->stream, &cs));
  if (cs == cudaStreamCaptureStatusNone) {
    int fb = 0;
    BEC_CUDA_TRY(cudaMemcpyAsync(&fb, reinterpret_cast<int*>(n.part + 5 * p->mg.K), sizeof(int),
                                 cudaMemcpyDeviceToHost, p->stream));
    BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
    n.rejected = fb != 0;
  }
  return BEC_OK;
}

bool net_calibrated(const bec_problem* p) { return p->net != nullptr && p->net->cal_ok; }

bool net_bypassed(const bec_problem* p) { return p->net != nullptr && p->net->bypass; }

void net_invalidate(bec_problem* p) {
  if (p->net) p->net->cal_ok = false;
}

bec_status net_train(bec_problem* p, int steps, int batch, float lr, unsigned long long seed,
                     double* loss_hist) {
  if (batch < 1 || 2 * batch > p->net->Bmax) return BEC_EINVAL;
  return p->net->fp32 ? train_t<float>(p, steps, batch, lr, seed, loss_hist)
                      : train_t<__nv_bfloat16>(p, steps, batch, lr, seed, loss_hist);
}

long long net_num_weights(const bec_problem* p) { return p->net ? p->net->nparam : 0; }

bec_status net_get_weights(bec_problem* p, float* host) {
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  BEC_CUDA_TRY(cudaMemcpy(host, p->net->W, p->net->nparam * sizeof(float), cudaMemcpyDeviceToHost));
  return BEC_OK;
}

bec_status net_set_weights(bec_problem* p, const float* host) {
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  BEC_CUDA_TRY(cudaMemcpy(p->net->W, host, p->net->nparam * sizeof(float), cudaMemcpyHostToDevice));
  p->net->adam_t = 0;
  p->net->gates_ok = false;
  p->net->cal_ok = false;
  BEC_CUDA_TRY(cudaMemset(p->net->Mo, 0, p->net->nparam * sizeof(float)));
  BEC_CUDA_TRY(cudaMemset(p->net->Ve, 0, p->net->nparam * sizeof(float)));
  return BEC_OK;
}

namespace {
__global__ void c128_to_c64_kernel(const double2* __restrict__ a, float2* __restrict__ b,
                                   long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) b[g] = make_float2((float)a[g].x, (float)a[g].y);
}

template <typename AT>
bec_status loss_grad_t(bec_problem* p, int B, const int* lams, const double* r, const double* et,
                       double* loss_out, float* grad_host) {
  NetState& n = *p->net;
  const long long mff = (long long)n.mf * n.mf;
  const long long tot = (long long)B * mff;
  const long long totc = (long long)B * n.sz[0] * n.sz[0];
  BEC_LAUNCH_BEGIN(p);
  c128_to_c64_kernel<<<grid_for(tot), kT, 0, p->stream>>>(reinterpret_cast<const double2*>(r),
                                                          reinterpret_cast<float2*>(n.res), tot);
  BEC_LAUNCH_CHECK(p, "net_convert_kernel");
  BEC_LAUNCH_BEGIN(p);
  c128_to_c64_kernel<<<grid_for(totc), kT, 0, p->stream>>>(reinterpret_cast<const double2*>(et),
                                                           reinterpret_cast<float2*>(n.etgt), totc);
  BEC_LAUNCH_CHECK(p, "net_convert_kernel");
  std::vector<int> rows(B);
  for (int b = 0; b < B; ++b) rows[b] = b;
  BEC_TRY(set_samples(p, rows.data(), lams, B));
  BEC_TRY(gates_fwd(p));
  BEC_TRY(features<AT>(p, B));
  BEC_TRY(forward<AT>(p, 2 * B, true));
  BEC_TRY(loss_and_dy<AT>(p, B));
  BEC_TRY(backward<AT>(p, 2 * B));
  BEC_CUDA_TRY(cudaMemcpyAsync(n.h_part, n.part, 2 * B * sizeof(double), cudaMemcpyDeviceToHost,
                               p->stream));
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  double l = 0.0;
  for (int b = 0; b < B; ++b) l += n.h_part[2 * b] / n.h_part[2 * b + 1];
  *loss_out = l / B;
  if (grad_host)
    BEC_CUDA_TRY(cudaMemcpy(grad_host, n.G, n.nparam * sizeof(float), cudaMemcpyDeviceToHost));
  return net_check(p);
}
}  // namespace

bec_status net_loss_grad(bec_problem* p, int B, const int* lams, const double* r, const double* et,
                         double* loss_out, float* grad_host) {
  if (B < 1 || 2 * B > p->net->Bmax || B > p->mg.K) {   // samples are staged in rows 0..B-1 of K
    set_error("B must lie in [1, min(32, N/2 + 1)]");
    return BEC_EINVAL;
  }
  return p->net->fp32 ? loss_grad_t<float>(p, B, lams, r, et, loss_out, grad_host)
                      : loss_grad_t<__nv_bfloat16>(p, B, lams, r, et, loss_out, grad_host);
}

long long net_fallbacks(bec_problem* p) {
  if (p->net == nullptr) return -1;
  int fb = 0;
  cudaStreamSynchronize(p->stream);
  cudaMemcpy(&fb, reinterpret_cast<int*>(p->net->part + 5 * p->mg.K), sizeof(int),
             cudaMemcpyDeviceToHost);
  return fb;
}

bec_status net_check(bec_problem* p) {
  if (p->net == nullptr || p->net->err == nullptr) return BEC_OK;
  int v = 0;
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  BEC_CUDA_TRY(cudaMemcpy(&v, p->net->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v == 0) return BEC_OK;
  BEC_CUDA_TRY(cudaMemset(p->net->err, 0, sizeof(int)));
  set_error("a bounded wait in the tensor-core convolution ran out");
  return BEC_ETIMEOUT;
}

bool net_rejected(const bec_problem* p) { return p->net != nullptr && p->net->rejected; }

bec_status net_prepare(bec_problem* p) {
  if (p->net == nullptr || p->desc.route != BEC_ROUTE_LEARNED || p->net->bypass || p->net->cal_ok)
    return BEC_OK;
  return net_calibrate(p);
}

void net_set_judge(bec_problem* p, bool on) {
  p->net->judge = on;
  p->net->cal_ok = false;
}

bec_status net_judge_radii(bec_problem* p, double* host) {
  const int K = p->mg.K;
  if (!p->net->cal_ok) {
    for (int i = 0; i < 2 * K + 2; ++i) host[i] = std::nan("");
    return BEC_OK;
  }
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  BEC_CUDA_TRY(cudaMemcpy(host, p->net->jrho, (2 * K + 2) * sizeof(double), cudaMemcpyDeviceToHost));
  return BEC_OK;
}

bec_status net_residual_ratios(bec_problem* p, double* host) {
  BEC_CUDA_TRY(cudaStreamSynchronize(p->stream));
  BEC_CUDA_TRY(cudaMemcpy(host, p->net->part + 4 * p->mg.K, p->mg.K * sizeof(double),
                          cudaMemcpyDeviceToHost));
  return BEC_OK;
}

}  // namespace bec

// The three streaming passes of the sine-transform P_eps^{-1} (Sec. 4, eqs.
// ytild, blockdiaginv, zcompt) as per-tile device functions.  A tile is the
// work of one block of the pass kernels: the kernels in bec_dst.cu and
// bec_time.cu run one tile per block, and the persistent batch kernel in
// bec_persist.cu runs tiles of many problems taken from a work queue.  Each
// function uses `sm` (dynamic shared memory of the size the launchers
// compute), takes the thread's index in the block as `tid`, and leaves no
// pending block barrier.
#pragma once

#include <cuda_runtime.h>

#include "bec_fft.cuh"

namespace bec {
namespace {


// ---------------------------------------------------------------- x-DST
// DST along x: one warp per pair of rows of m = n - 1 values, the tile's
// warps on rows 2 (blk WARPS + warp) and the next; row r of `in` starts at
// r in_ld, of `out` at r out_ld (in_ld, out_ld = m or m + 1; an output row
// of m + 1 slots gets a zero in its last one).  `in` and `out` may be the
// same array (each warp reads its rows before writing them); in that case
// TI == TO and in_ld == out_ld.
template <typename T, typename TI, typename TO, int LOGN, int WARPS>
__device__ __forceinline__ void dst_rows_tile(const TI* in, TO* out, long long rows, int m,
                                              int in_ld, int out_ld, const T* __restrict__ sin2,
                                              const v2_t<T>* __restrict__ tw, long long blk,
                                              unsigned char* smem_bytes, int tid) {
  constexpr int RS = dst_line_stride(LOGN, sizeof(T));   // real slots per line
  T* sm = reinterpret_cast<T*>(smem_bytes);
  const int warp = tid >> 5, lane = tid & 31;
  T* raw = sm + (size_t)warp * 2 * RS;
  const long long r0 = 2 * (blk * WARPS + warp);
  if (r0 >= rows) return;                    // whole warp leaves; no block barrier below
  const bool hasb = r0 + 1 < rows;
  const TI* ia = in + r0 * in_ld;
  // loads in groups of G per row, all issued before the group's conversions
  // (m = n - 1 < 32 PER)
  constexpr int PER = (1 << LOGN) / 32 > 0 ? (1 << LOGN) / 32 : 1;
  constexpr int G = PER < 8 ? PER : 8;
#pragma unroll
  for (int t0 = 0; t0 < PER; t0 += G) {
    TI va[G], vb[G];
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int j = lane + 32 * (t0 + t);
      va[t] = j < m ? ia[j] : TI(0);
      vb[t] = (j < m && hasb) ? ia[in_ld + j] : TI(0);
    }
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int j = lane + 32 * (t0 + t);
      if (j < m) {
        raw[j] = convert<T>(va[t]);
        raw[RS + j] = convert<T>(vb[t]);
      }
    }
  }
  __syncwarp();
  warp_dst_pair<T, LOGN>(raw, RS, sin2, tw, lane);
  TO* oa = out + r0 * out_ld;
#pragma unroll
  for (int t0 = 0; t0 < PER; t0 += G) {
    TO wa[G], wb[G];
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int j = lane + 32 * (t0 + t);
      wa[t] = j < m ? convert<TO>(raw[dst_out<T, LOGN>(j)]) : TO(0);
      wb[t] = j < m ? convert<TO>(raw[RS + dst_out<T, LOGN>(j)]) : TO(0);
    }
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int j = lane + 32 * (t0 + t);
      if (j < m) {
        oa[j] = wa[t];
        if (hasb) oa[out_ld + j] = wb[t];
      } else if (j < out_ld) {             // the pad slot (j = m)
        oa[j] = TO(0);
        if (hasb) oa[out_ld + j] = TO(0);
      }
    }
  }
}

// ---------------------------------------------------------------- y-DST
// DST down the columns of one slice, in place: the slice at data + sl *
// slice_stride holds m rows of ncols values, row j at j * row_stride.  The
// tile owns W = 2 x WARPS adjacent columns starting at bx * W; it is loaded
// and stored with coalesced row segments, and each warp transforms one
// column pair.
template <typename T, int LOGN, int WARPS>
__device__ __forceinline__ void dst_cols_tile(T* data, int m, int ncols, long long row_stride,
                                              long long slice_stride, long long bx, long long sl,
                                              const T* __restrict__ sin2,
                                              const v2_t<T>* __restrict__ tw,
                                              unsigned char* smem_bytes, int tid) {
  constexpr int RS = dst_line_stride(LOGN, sizeof(T));   // real slots per column
  constexpr int W = 2 * WARPS;
  T* sm = reinterpret_cast<T*>(smem_bytes);
  const int warp = tid >> 5, lane = tid & 31;
  // thread t always handles column c = t mod W of the tile and the rows
  // j = t / W + JS i.  In FP32 the tile arrives by asynchronous copies, which
  // hold no registers, so all of a thread's loads are in flight together.
  constexpr int JS = WARPS * 32 / W;
  const int c = tid % W, j0 = tid / W;
  const long long x = bx * W + c;
  const bool xin = x < ncols;
  T* const slot = sm + c * RS;
  T* const col = data + sl * slice_stride + (xin ? x : 0);   // row j at col[j row_stride]
  if constexpr (sizeof(T) == 4) {
#pragma unroll 4
    for (int j = j0; j < m; j += JS) cp_async4(slot + j, col + (long long)j * row_stride, xin);
    cp_async_wait_all();
  } else {                                 // FP64: bound by its arithmetic, not by loads
#pragma unroll 4
    for (int j = j0; j < m; j += JS) slot[j] = xin ? col[(long long)j * row_stride] : T(0);
  }
  __syncthreads();
  warp_dst_pair<T, LOGN>(sm + (size_t)warp * 2 * RS, RS, sin2, tw, lane);
  __syncthreads();
  if (xin) {
#pragma unroll 4
    for (int j = j0; j < m; j += JS) col[(long long)j * row_stride] = slot[dst_out<T, LOGN>(j)];
  }
  __syncthreads();
}

// ---------------------------------------------------------------- time pass
// The 1D eigenvalue tables of the spatial operators on the sine basis:
// stiffness k (times a) and mass m (null: M = I, finite differences).
template <typename T>
struct ModeEigs {
  const T* __restrict__ k;
  const T* __restrict__ m;
};

// Mass and stiffness eigenvalues of spatial mode q: FD (1, k_i + k_l); Q1
// (m_i m_l, m_i k_l + k_i m_l) in 2D, (m_q, k_q) in 1D.  The layout has J
// points per time slice in rows of ld >= m slots (x index i = q mod ld);
// slots past the end or with i >= m are padding.
template <typename T>
__device__ __forceinline__ void mode_eigs(long long q, long long J, int m, int ld, int dim,
                                          ModeEigs<T> e, T& muM, T& muK) {
  const long long row = q / ld;
  const int i = (int)(q - row * ld);
  if (q >= J || i >= m) {                        // padding: any positive value
    muM = T(1);
    muK = T(1);
    return;
  }
  if (dim == 1) {
    muM = e.m ? e.m[i] : T(1);
    muK = e.k[i];
    return;
  }
  if (dim == 3) {                                // FD only: k_i + k_l + k_s
    const int s = (int)(row / m);
    const int l = (int)(row - (long long)s * m);
    muM = T(1);
    muK = e.k[i] + e.k[l] + e.k[s];
    return;
  }
  const int l = (int)row;
  if (e.m == nullptr) {
    muM = T(1);
    muK = e.k[i] + e.k[l];
  } else {
    muM = e.m[i] * e.m[l];
    muK = fma(e.m[i], e.k[l], e.k[i] * e.m[l]);
  }
}

// data: [N][J] in place; the tile owns W = 2 x WARPS adjacent modes from
// q0 = blk W, and warp w transforms modes (q0 + 2w, q0 + 2w + 1) packed as
// real + i imaginary: scale by eps^{j/N} (D_eps, Step 1), FFT along time,
// divide by lambda'_k mu^M + tau mu^K (Step 2), inverse FFT, unscale (Step
// 3).  FE: the mass eigenvalues are present (Q1 elements).
template <typename T, int LOGN, int WARPS, bool FE>
__device__ __forceinline__ void time_pass_tile(T* __restrict__ data, long long J, int m, int ld,
                                               int dim,
                                               const T* __restrict__ es, const T* __restrict__ eis,
                                               const v2_t<T>* __restrict__ lamf, ModeEigs<T> me,
                                               T tau, T scale_h, const double* __restrict__ scale_dev,
                                               const v2_t<T>* __restrict__ tw,
                                               const double* __restrict__ rinv, long long blk,
                                               unsigned char* smem_bytes, int tid) {
  using V = v2_t<T>;
  const T scale = scale_dev ? (T)((double)scale_h * scale_dev[0]) : scale_h;
  constexpr int N = 1 << LOGN;
  constexpr int LSC = line_slots(LOGN);
  constexpr int W = 2 * WARPS;
  T* sm = reinterpret_cast<T*>(smem_bytes);
  const int warp = tid >> 5, lane = tid & 31;
  const long long q0 = blk * W;

  // load + D_eps scaling: mode c of the tile -> line c/2, real (c even) or
  // imaginary part.  Thread t always handles mode c = t mod W and the rows
  // j = t / W + JS i.  In FP32 it issues its loads in groups of up to 16
  // before the group's stores, so that they are in flight together.
  constexpr int JS = WARPS * 32 / W;
  constexpr int NI = (N + JS - 1) / JS;
  const int c = tid % W, j0 = tid / W;
  const bool qin = q0 + c < J;
  T* const slot = sm + (c >> 1) * 2 * LSC + (c & 1);          // element j at slot[2 j]
  T* const col = data + (qin ? q0 + c : 0);                    // element j at col[j J]
  if constexpr (sizeof(T) == 4) {
    constexpr int GMAX = LOGN <= 8 ? 16 : 8;   // loads in flight per group (registers)
    constexpr int G = NI < GMAX ? NI : GMAX;
#pragma unroll
    for (int g = 0; g < NI; g += G) {
      T v[G];
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int j = j0 + JS * (g + i);
        v[i] = (qin && (N % JS == 0 || j < N)) ? col[(long long)j * J] : T(0);
      }
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int j = j0 + JS * (g + i);
        if (N % JS == 0 || j < N) slot[2 * j] = v[i] * es[j];
      }
    }
  } else {                                   // FP64: bound by its arithmetic, not by loads
#pragma unroll 4
    for (int j = j0; j < N; j += JS) slot[2 * j] = qin ? col[(long long)j * J] * es[j] : T(0);
  }
  __syncthreads();

  V* line = reinterpret_cast<V*>(sm + (size_t)warp * 2 * LSC);
  warp_fft<T, -1, LOGN>(line, tw, lane);
  const long long qa = q0 + 2 * warp;
  T ma, mua, mb, mub;                 // mass and stiffness eigenvalues of modes a, b
  mode_eigs(qa, J, m, ld, dim, me, ma, mua);
  if (qa + 1 < J) {
    mode_eigs(qa + 1, J, m, ld, dim, me, mb, mub);
  } else {
    mb = ma;
    mub = mua;
  }
  constexpr int NK = N / 2 + 1;
  constexpr int PERK = (NK + 31) / 32;
#pragma unroll
  for (int t = 0; t < PERK; ++t) {
    const int k = lane + 32 * t;
    if (k < NK) {
      const int kk = (N - k) & (N - 1);
      const V C = line[k], Cn = line[kk];
      // A1 = spectrum of mode a, A2 = spectrum of mode b (each times 2)
      const V A1 = {C.x + Cn.x, C.y - Cn.y};
      const V A2 = {C.y + Cn.y, Cn.x - C.x};
      const V L = lamf[k];
      // d = lambda'_k mu^M + tau mu^K for each mode (mu^M = 1 with FD)
      constexpr bool fe = FE;
      const T d1r = fe ? fma(L.x, ma, tau * mua) : L.x + tau * mua;
      const T d2r = fe ? fma(L.x, mb, tau * mub) : L.x + tau * mub;
      const T d1i = fe ? L.y * ma : L.y, d2i = fe ? L.y * mb : L.y;
      T s1, s2;
      if (rinv != nullptr) {           // 1 / |d|^2 from the table ([q][k], coalesced in k)
        s1 = qa < J ? scale * (T)rinv[qa * NK + k] : T(0);
        s2 = qa + 1 < J ? scale * (T)rinv[(qa + 1) * NK + k] : s1;
      } else if constexpr (sizeof(T) == 4) {
        // |d|^2 lies far inside the normal range, where the approximate
        // division is within 2 units in the last place
        s1 = __fdividef(scale, fma(d1r, d1r, d1i * d1i));
        s2 = __fdividef(scale, fma(d2r, d2r, d2i * d2i));
      } else {
        s1 = scale / fma(d1r, d1r, d1i * d1i);
        s2 = scale / fma(d2r, d2r, d2i * d2i);
      }
      const V q1 = {d1r * s1, -d1i * s1};           // scale / d1
      const V q2 = {d2r * s2, -d2i * s2};
      const V B1 = cmul(A1, q1), B2 = cmul(A2, q2);
      line[k] = {B1.x - B2.y, B1.y + B2.x};         // B1 + i B2
      line[kk] = {B1.x + B2.y, B2.x - B1.y};        // conj(B1) + i conj(B2)
    }
  }
  __syncwarp();
  warp_fft<T, +1, LOGN>(line, tw, lane);
  __syncthreads();

  if (qin) {
#pragma unroll 4
    for (int j = j0; j < N; j += JS) col[(long long)j * J] = slot[2 * j] * eis[j];
  }
}


// ------------------------------------------------- time pass, FP32, N = 256
// The same time pass (Steps 1-3 of Sec. 4 on one tile of spatial modes) as a
// four-step FFT with N = 16 x 16 held in registers: j = j1 + 16 j2 and
// k = k2 + 16 k1, so that
//   X_{k2 + 16 k1} = sum_{j1} w16^{j1 k1} [w^{j1 k2} sum_{j2} x_{j1 + 16 j2} w16^{j2 k2}]
// (w = e^{-2 pi i / N}).  Step A: a thread owns a residue j1 of one line and
// does the 16-point DFT over j2 in registers, then the twiddles w^{j1 k2}.
// One shared-memory exchange hands each thread a class k2, step B does the
// 16-point DFT over j1, the divide, and the inverse DFT over k1; a second
// exchange and the inverse DFT over k2 finish the line.  The half spectrum
// pairs k with N - k: class (16 - k2) mod 16, held by another lane of the
// same half-warp, which passes it by shuffle.  The tile is 16 complex lines
// (32 adjacent modes, two per line as real + i imaginary); 16 threads per
// line, 256 per block.
constexpr int kT16Threads = 256;
constexpr int kT16Modes = 32;                   // modes per tile
constexpr int kT16LineSlots = 16 * 17 + 1;      // complex slots per line: 16 rows of 17, odd
constexpr size_t kT16Smem = (size_t)16 * kT16LineSlots * 8;

// In-register DFT of length 16 with kernel e^{SIGN 2 pi i r k / 16}, natural
// order in and out, as 4 x 4: the 4-point DFTs over the samples a + 4 b
// (b = 0..3), the twiddles w16^{a kb}, then the 4-point DFTs over a; output
// kb + 4 ka.
template <int SIGN, typename V>
__device__ __forceinline__ void dft16(V (&v)[16]) {
  using T = decltype(v[0].x);
  V u[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    V t[4] = {v[a], v[a + 4], v[a + 8], v[a + 12]};
    radix_dft<4, SIGN>(t);
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) u[a][kb] = t[kb];
  }
  // w16^m = cos(m pi / 8) + SIGN i sin(m pi / 8) for m = a kb
  const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173);
  const T h = T(0.70710678118654752440);
  u[1][1] = cmul(u[1][1], V{c1, SIGN * s1});      // m = 1
  u[1][2] = cmul(u[1][2], V{h, SIGN * h});        // m = 2
  u[1][3] = cmul(u[1][3], V{s1, SIGN * c1});      // m = 3
  u[2][1] = cmul(u[2][1], V{h, SIGN * h});        // m = 2
  u[2][2] = cmul_si<SIGN>(u[2][2]);               // m = 4
  u[2][3] = cmul(u[2][3], V{-h, SIGN * h});       // m = 6
  u[3][1] = cmul(u[3][1], V{s1, SIGN * c1});      // m = 3
  u[3][2] = cmul(u[3][2], V{-h, SIGN * h});       // m = 6
  u[3][3] = cmul(u[3][3], V{-c1, -SIGN * s1});    // m = 9
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    V t[4] = {u[0][kb], u[1][kb], u[2][kb], u[3][kb]};
    radix_dft<4, SIGN>(t);
#pragma unroll
    for (int ka = 0; ka < 4; ++ka) v[kb + 4 * ka] = t[ka];
  }
}

// B_k / (lambda'_k mu^M + tau mu^K) of the two modes of a line for one k,
// from the packed spectrum C = X_k and its partner Cn = X_{N-k}: the modes'
// spectra (times 2) are A1 = C + conj Cn and A2 = -i (C - conj Cn); the
// result is the packed value B1 + i B2 at k.  lam = lambda'_k.
template <bool FE>
__device__ __forceinline__ float2 t16_divide(float2 C, float2 Cn, float2 lam, float ma, float tmua,
                                             float mb, float tmub, float scale) {
  const float2 A1 = {C.x + Cn.x, C.y - Cn.y};
  const float2 A2 = {C.y + Cn.y, Cn.x - C.x};
  const float d1r = FE ? fmaf(lam.x, ma, tmua) : lam.x + tmua;
  const float d2r = FE ? fmaf(lam.x, mb, tmub) : lam.x + tmub;
  const float d1i = FE ? lam.y * ma : lam.y, d2i = FE ? lam.y * mb : lam.y;
  // |d|^2 lies far inside the normal range, where the approximate division
  // is within 2 units in the last place
  const float s1 = __fdividef(scale, fmaf(d1r, d1r, d1i * d1i));
  const float s2 = __fdividef(scale, fmaf(d2r, d2r, d2i * d2i));
  const float2 q1 = {d1r * s1, -d1i * s1}, q2 = {d2r * s2, -d2i * s2};
  const float2 B1 = cmul(A1, q1), B2 = cmul(A2, q2);
  return {B1.x - B2.y, B1.y + B2.x};
}

// The same for the pair: nc = the packed result at k, nn = at N - k
// (conj B1 + i conj B2).  nn equals, bit for bit, what t16_divide gives from
// (Cn, C, conj lam): the modes' spectra, the shifts and the products are then
// exact conjugates of these.
template <bool FE>
__device__ __forceinline__ void t16_divide_pair(float2 C, float2 Cn, float2 lam, float ma,
                                                float tmua, float mb, float tmub, float scale,
                                                float2& nc, float2& nn) {
  const float2 A1 = {C.x + Cn.x, C.y - Cn.y};
  const float2 A2 = {C.y + Cn.y, Cn.x - C.x};
  const float d1r = FE ? fmaf(lam.x, ma, tmua) : lam.x + tmua;
  const float d2r = FE ? fmaf(lam.x, mb, tmub) : lam.x + tmub;
  const float d1i = FE ? lam.y * ma : lam.y, d2i = FE ? lam.y * mb : lam.y;
  const float s1 = __fdividef(scale, fmaf(d1r, d1r, d1i * d1i));
  const float s2 = __fdividef(scale, fmaf(d2r, d2r, d2i * d2i));
  const float2 q1 = {d1r * s1, -d1i * s1}, q2 = {d2r * s2, -d2i * s2};
  const float2 B1 = cmul(A1, q1), B2 = cmul(A2, q2);
  nc = {B1.x - B2.y, B1.y + B2.x};
  nn = {B1.x + B2.y, B2.x - B1.y};
}

// data: [N][J] in place, N = 256, rows of ld slots (mode_eigs); the tile
// owns modes q0 .. q0 + 31 from q0 = 32 blk (line L: modes q0 + 2L and
// q0 + 2L + 1).  STAGED: the tile's values are not in `data` but in a
// shared-memory tile `stage` of [256][32] floats (time row j at 32 j), which
// it also returns in; global memory is not touched.  `xbuf` holds kT16Smem
// bytes.  tw[t] = e^{-2 pi i t / N}; lamf[k] = lambda'_k for k = 0..N/2
// (lambda'_{N-k} = conj lambda'_k).
template <bool FE, bool STAGED>
__device__ __forceinline__ void time_pass16_tile(float* __restrict__ data, float* __restrict__ stage,
                                                 long long J, int m, int ld, int dim,
                                                 const float* __restrict__ es,
                                                 const float* __restrict__ eis,
                                                 const float2* __restrict__ lamf,
                                                 ModeEigs<float> me, float tau, float scale_h,
                                                 const double* __restrict__ scale_dev,
                                                 const float2* __restrict__ tw, long long blk,
                                                 unsigned char* xbuf, int tid) {
  using V = float2;
  const float scale = scale_dev ? (float)((double)scale_h * scale_dev[0]) : scale_h;
  V* buf = reinterpret_cast<V*>(xbuf);
  const long long q0 = blk * kT16Modes;
  const bool full = q0 + kT16Modes <= J;
  // Step A layout: line L = tid mod 16, residue r; a warp holds residues w and
  // w + 8 of 16 lines, so its rows j = r + 16 j2 share their parity.  From
  // global memory a pair of modes is one 8-byte load when its offset j J + q
  // is even (J even, or r even; q is even), else two 4-byte loads.
  const int La = tid & 15;
  const int r = ((tid >> 4) & 1) * 8 + (tid >> 5);
  const long long qA = q0 + 2 * La;
  const bool in0 = qA < J, in1 = qA + 1 < J;
  const bool vec = full && ((J & 1) == 0 || (r & 1) == 0);
  float* const colA = STAGED ? stage + 2 * La : data + (in0 ? qA : 0);
  const long long rstride = STAGED ? (long long)kT16Modes : J;   // floats from time row j to j + 1
  V* const rowA = buf + La * kT16LineSlots + r;            // element k2 at rowA[17 k2]
  {
    V v[16];
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {
      const float* pp = colA + (long long)(r + 16 * j2) * rstride;
      if (STAGED || vec) {
        v[j2] = *reinterpret_cast<const V*>(pp);
      } else {
        v[j2].x = in0 ? pp[0] : 0.f;
        v[j2].y = in1 ? pp[1] : 0.f;
      }
    }
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {          // D_eps (Step 1)
      const float e = es[r + 16 * j2];
      v[j2].x *= e;
      v[j2].y *= e;
    }
    dft16<-1>(v);
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw[r * k2]);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) rowA[17 * k2] = v[k2];
  }
  __syncthreads();
  {
    // Step B layout: line L = tid / 16, class k2 = tid mod 16 (a half-warp
    // is one line, so the partner class is a lane of the same half-warp)
    const int lane = tid & 31, k2 = lane & 15, Lb = tid >> 4;
    V* const rowB = buf + Lb * kT16LineSlots + 17 * k2;    // element j1 at rowB[j1]
    V y[16];
#pragma unroll
    for (int j1 = 0; j1 < 16; ++j1) y[j1] = rowB[j1];
    dft16<-1>(y);                              // y[k1] = X_{k2 + 16 k1}
    const long long qa = q0 + 2 * Lb;
    float ma, mua, mb, mub;                    // mass and stiffness eigenvalues of the two modes
    mode_eigs(qa, J, m, ld, dim, me, ma, mua);
    mode_eigs(qa + 1, J, m, ld, dim, me, mb, mub);
    const float tmua = tau * mua, tmub = tau * mub;
    // X_{N-k} for k = k2 + 16 k1: class (16 - k2) mod 16 at k1' = 15 - k1
    // (k2 > 0, from lane (16 - k2) of the half-warp) or (16 - k1) mod 16
    // (k2 = 0, the thread's own).  Each pair (k, N - k) with k < N/2 is done
    // once, by the lane that holds k (k1 < 8); its result at N - k goes back
    // to the partner by the same shuffle.  Lane k2 = 0 also holds k = N/2.
    const int src = (lane & 16) | ((16 - k2) & 15);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
      const V sv = k2 == 0 ? y[(16 - k1) & 15] : y[15 - k1];
      V Cn;
      Cn.x = __shfl_sync(0xffffffffu, sv.x, src);
      Cn.y = __shfl_sync(0xffffffffu, sv.y, src);
      V nc, nn;
      t16_divide_pair<FE>(y[k1], Cn, lamf[k2 + 16 * k1], ma, tmua, mb, tmub, scale, nc, nn);
      V rn;                                    // the partner's result at my N - k'
      rn.x = __shfl_sync(0xffffffffu, nn.x, src);
      rn.y = __shfl_sync(0xffffffffu, nn.y, src);
      y[k1] = nc;
      if (k2 == 0) y[(16 - k1) & 15] = rn;
      else y[15 - k1] = rn;
    }
    if (k2 == 0) {                             // k = N/2, its own partner
      V lam = lamf[128];
      lam.y = -lam.y;
      y[8] = t16_divide<FE>(y[8], y[8], lam, ma, tmua, mb, tmub, scale);
    }
    dft16<+1>(y);                              // y[j1] = sum_k1 Z_{k2 + 16 k1} w16^{-j1 k1}
#pragma unroll
    for (int j1 = 0; j1 < 16; ++j1) rowB[j1] = y[j1];
  }
  __syncthreads();
  {
    V v[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) v[k2] = rowA[17 * k2];
#pragma unroll
    for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmulc(v[k2], tw[r * k2]);
    dft16<+1>(v);                              // v[j2] = z_{r + 16 j2} times N e^{...}
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {          // D_eps^{-1} (Step 3)
      const float e = eis[r + 16 * j2];
      v[j2].x *= e;
      v[j2].y *= e;
    }
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {
      float* pp = colA + (long long)(r + 16 * j2) * rstride;
      if (STAGED || vec) {
        *reinterpret_cast<V*>(pp) = v[j2];
      } else {
        if (in0) pp[0] = v[j2].x;
        if (in1) pp[1] = v[j2].y;
      }
    }
  }
}

// ------------------------------------------------- y-DST, FP32, n = 256
// The DST-I down 32 adjacent columns of one slice (n = 256, m = 255 rows),
// with the same four-step 16 x 16 FFT in registers as the N = 256 time
// pass.  Column pairs (2L, 2L + 1) are one complex line; the DST of a line
// is the length-n FFT of y_j = 2 sin(j pi / n)(x_j + x_{n-j}) + (x_j -
// x_{n-j}), then for k < n/2 the even outputs 4 S_{2k} = e_k and the odd
// ones 4 S_{2k+1} = sum_{k' <= k} r_{k'} (the method of warp_dst_pair).
// The tile sits in a shared-memory stage of [256][32] floats (row i holds
// x_{i+1}; row 255 is not used) and returns there as rows of S (row i holds
// 4 S_{i+1}).  The exchange buffer of the 16 x 16 steps is `xbuf` (32 KB)
// or, when xbuf is null, the stage itself (two more block barriers), in
// either case XOR-swizzled (line L, class k2, index j1 at 256 L + 16 k2 +
// (j1 ^ k2 ^ L)), which keeps both of its access patterns free of bank
// conflicts; `tot` holds 256 float2.  sin2[j] = 2 sin(j pi / n), tw[t] =
// e^{-2 pi i t / n}.
constexpr int kD16Threads = 256;
constexpr int kD16Cols = 32;                                // columns per tile
constexpr size_t kD16StageBytes = (size_t)256 * kD16Cols * sizeof(float);   // 32 KB
constexpr size_t kD16TotBytes = 256 * sizeof(float2);

__device__ __forceinline__ int d16_xs(int L, int k2, int j1) {
  return 256 * L + 16 * k2 + ((j1 ^ k2 ^ L) & 15);
}

__device__ __forceinline__ void dst16_cols_core(float* __restrict__ stage, float2* xbuf,
                                                float2* __restrict__ tot,
                                                const float* __restrict__ sin2,
                                                const float2* __restrict__ tw, int tid) {
  using V = float2;
  V* const sv = reinterpret_cast<V*>(stage);              // row i, line L at sv[16 i + L]
  V* const xv = xbuf != nullptr ? xbuf : sv;              // the exchange buffer
  // Step A layout (as in time_pass16_tile): line L, residue r of j mod 16
  const int La = tid & 15;
  const int r = ((tid >> 4) & 1) * 8 + (tid >> 5);
  V v[16];
#pragma unroll
  for (int j2 = 0; j2 < 16; ++j2) {
    const int j = r + 16 * j2;                            // x_j at row j - 1, x_{n-j} at 255 - j
    V y = {0.f, 0.f};                                     // y_0 = 0 (x_0 = x_n = 0)
    if (j2 > 0 || r > 0) {
      const V xa = sv[16 * (j - 1) + La], xb = sv[16 * (255 - j) + La];
      const float s = sin2[j];
      y.x = fmaf(s, xa.x + xb.x, xa.x - xb.x);
      y.y = fmaf(s, xa.y + xb.y, xa.y - xb.y);
    }
    v[j2] = y;
  }
  if (xbuf == nullptr) __syncthreads();                   // the stage becomes the exchange buffer
  dft16<-1>(v);
#pragma unroll
  for (int k2 = 1; k2 < 16; ++k2) v[k2] = cmul(v[k2], tw[r * k2]);
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) xv[d16_xs(La, k2, r)] = v[k2];
  __syncthreads();
  // Step B layout: line L = tid / 16, class k2 = tid mod 16
  const int lane = tid & 31, k2 = lane & 15, Lb = tid >> 4;
  V y[16];
#pragma unroll
  for (int j1 = 0; j1 < 16; ++j1) y[j1] = xv[d16_xs(Lb, k2, j1)];
  if (xbuf == nullptr) __syncthreads();                   // the stage becomes the r / e buffers
  dft16<-1>(y);                                           // y[k1] = X_{k2 + 16 k1}
  // X_{n-k} for k = k2 + 16 k1 < n/2 (k1 < 8): as in time_pass16_tile
  V* const rb = sv;                                       // r_k of line L at rb[129 L + k]
  V* const eb = sv + 16 * 129;                            // e_k (k >= 1) at eb[127 L + k - 1]
  const int src = (lane & 16) | ((16 - k2) & 15);
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    const V s = k2 == 0 ? y[(16 - k1) & 15] : y[15 - k1];
    V Cn;
    Cn.x = __shfl_sync(0xffffffffu, s.x, src);
    Cn.y = __shfl_sync(0xffffffffu, s.y, src);
    const V C = y[k1];
    const int k = k2 + 16 * k1;
    if (k == 0) {
      rb[129 * Lb] = C;
    } else {
      rb[129 * Lb + k] = {C.x + Cn.x, C.y + Cn.y};
      eb[127 * Lb + k - 1] = {Cn.y - C.y, C.x - Cn.x};
    }
  }
  __syncthreads();
  // Output layout: chunk c = tid / 16 owns k = 8c .. 8c + 7 of line L = tid
  // mod 16: a serial running sum, the chunk totals of the lower chunks, and
  // rows 2k (odd outputs) and 2k - 1 (even outputs) of the stage.
  const int c = tid >> 4, L = tid & 15;
  V P[8], E[8];
  V run = {0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = 8 * c + i;
    const V rv = rb[129 * L + k];
    run.x += rv.x;
    run.y += rv.y;
    P[i] = run;
    E[i] = (k > 0) ? eb[127 * L + k - 1] : V{0.f, 0.f};
  }
  tot[16 * c + L] = run;
  __syncthreads();
  V off = {0.f, 0.f};
  for (int cc = 0; cc < c; ++cc) {
    const V t = tot[16 * cc + L];
    off.x += t.x;
    off.y += t.y;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = 8 * c + i;
    sv[16 * (2 * k) + L] = {off.x + P[i].x, off.y + P[i].y};   // 4 S_{2k+1}
    if (k > 0) sv[16 * (2 * k - 1) + L] = E[i];                // 4 S_{2k}
  }
}

}  // namespace
}  // namespace bec

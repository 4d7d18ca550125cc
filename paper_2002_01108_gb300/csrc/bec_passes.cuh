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
// DST along x: one warp per pair of contiguous rows of length m = n - 1, the
// tile's warps on rows 2 (blk WARPS + warp) and the next.  `in` and `out` may
// be the same array (each warp reads its rows before writing them); in that
// case TI == TO.
template <typename T, typename TI, typename TO, int LOGN, int WARPS>
__device__ __forceinline__ void dst_rows_tile(const TI* in, TO* out, long long rows, int m,
                                              const T* __restrict__ sin2,
                                              const v2_t<T>* __restrict__ tw, long long blk,
                                              unsigned char* smem_bytes, int tid) {
  constexpr int RS = dst_line_stride(LOGN, sizeof(T));   // real slots per line
  T* sm = reinterpret_cast<T*>(smem_bytes);
  const int warp = tid >> 5, lane = tid & 31;
  T* raw = sm + (size_t)warp * 2 * RS;
  const long long r0 = 2 * (blk * WARPS + warp);
  if (r0 >= rows) return;                    // whole warp leaves; no block barrier below
  const bool hasb = r0 + 1 < rows;
  const TI* ia = in + r0 * m;
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
      vb[t] = (j < m && hasb) ? ia[m + j] : TI(0);
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
  TO* oa = out + r0 * m;
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
        if (hasb) oa[m + j] = wb[t];
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
// (m_i m_l, m_i k_l + k_i m_l) in 2D, (m_q, k_q) in 1D.
template <typename T>
__device__ __forceinline__ void mode_eigs(long long q, long long J, int m, int dim,
                                          ModeEigs<T> e, T& muM, T& muK) {
  if (q >= J) {                                  // padding column: any positive value
    muM = T(1);
    muK = T(1);
    return;
  }
  if (dim == 1) {
    muM = e.m ? e.m[q] : T(1);
    muK = e.k[q];
    return;
  }
  if (dim == 3) {                                // FD only: k_i + k_l + k_s
    const long long m2 = (long long)m * m;
    const int s = (int)(q / m2);
    const long long r = q - (long long)s * m2;
    const int l = (int)(r / m), i = (int)(r - (long long)l * m);
    muM = T(1);
    muK = e.k[i] + e.k[l] + e.k[s];
    return;
  }
  const int l = (int)(q / m), i = (int)(q - (long long)l * m);
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
__device__ __forceinline__ void time_pass_tile(T* __restrict__ data, long long J, int m, int dim,
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
  mode_eigs(qa, J, m, dim, me, ma, mua);
  if (qa + 1 < J) {
    mode_eigs(qa + 1, J, m, dim, me, mb, mub);
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

}  // namespace
}  // namespace bec

// Warp-level FFT and DST-I building blocks used by the preconditioner passes.
//
// Each line (one complex sequence of length n = 2^LOGN) lives in shared memory
// and is transformed by a single warp, so only __syncwarp() is needed inside a
// transform.  Two real lines are packed into one complex line (real and
// imaginary parts) and separated afterwards, which halves the work of the
// real-data transforms.
#pragma once

#include <cuda_runtime.h>

namespace bec {

template <typename T> struct V2T;
template <> struct V2T<double> { using type = double2; };
template <> struct V2T<float> { using type = float2; };
template <typename T> using v2_t = typename V2T<T>::type;

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// In-register DFT of length R with kernel e^{SIGN 2 pi i r k / R}.
template <int R, int SIGN, typename V>
__device__ __forceinline__ void radix_dft(V (&v)[R]) {
  if constexpr (R == 2) {
    V a = v[0], b = v[1];
    v[0] = {a.x + b.x, a.y + b.y};
    v[1] = {a.x - b.x, a.y - b.y};
  } else {
    static_assert(R == 4, "radix 2 or 4");
    V a = {v[0].x + v[2].x, v[0].y + v[2].y};
    V b = {v[0].x - v[2].x, v[0].y - v[2].y};
    V c = {v[1].x + v[3].x, v[1].y + v[3].y};
    V d = {v[1].x - v[3].x, v[1].y - v[3].y};
    // w d with w = SIGN * i
    V wd = SIGN < 0 ? V{d.y, -d.x} : V{-d.y, d.x};
    v[0] = {a.x + c.x, a.y + c.y};
    v[2] = {a.x - c.x, a.y - c.y};
    v[1] = {b.x + wd.x, b.y + wd.y};
    v[3] = {b.x - wd.x, b.y - wd.y};
  }
}

// One Stockham autosort pass of radix R = 2^LOGR at span Ns = 2^LOGNS on a
// line of n = 2^LOGN complex values.  Butterfly j reads x[j + r n/R], applies
// the twiddles e^{SIGN 2 pi i (j mod Ns) r / (Ns R)}, does the radix-R DFT and
// writes x[(j div Ns) Ns R + (j mod Ns) + r Ns].  All reads finish before any
// write, so the pass works in place.  tw[t] = e^{-2 pi i t / n}.
template <typename T, int SIGN, int LOGN, int LOGNS, int LOGR>
__device__ __forceinline__ void fft_pass(v2_t<T>* buf, const v2_t<T>* __restrict__ tw,
                                         int lane) {
  using V = v2_t<T>;
  constexpr int n = 1 << LOGN, R = 1 << LOGR, Ns = 1 << LOGNS;
  constexpr int NB = n / R;
  constexpr int PER = (NB + 31) / 32;
  constexpr int TWSTEP = n / (Ns * R);
  V v[PER][R];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int j = lane + 32 * t;
    if (NB % 32 == 0 || j < NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[t][r] = buf[j + r * NB];
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int j = lane + 32 * t;
    if (NB % 32 == 0 || j < NB) {
      const int k = j & (Ns - 1);
      if constexpr (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const V w = tw[k * r * TWSTEP];
          v[t][r] = SIGN < 0 ? cmul(v[t][r], w) : cmulc(v[t][r], w);
        }
      }
      radix_dft<R, SIGN>(v[t]);
      const int base = ((j >> LOGNS) << (LOGNS + LOGR)) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[base + r * Ns] = v[t][r];
    }
  }
  __syncwarp();
}

template <typename T, int SIGN, int LOGN, int LOGNS>
__device__ __forceinline__ void fft_radix4_passes(v2_t<T>* buf, const v2_t<T>* __restrict__ tw,
                                                  int lane) {
  if constexpr (LOGNS + 2 <= LOGN) {
    fft_pass<T, SIGN, LOGN, LOGNS, 2>(buf, tw, lane);
    fft_radix4_passes<T, SIGN, LOGN, LOGNS + 2>(buf, tw, lane);
  }
}

// Complex FFT of length 2^LOGN in place in shared memory, natural order in
// and out, by one warp.  SIGN = -1: X_k = sum_j x_j e^{-2 pi i jk/n};
// SIGN = +1: the unnormalised inverse.  A radix-2 pass (with trivial
// twiddles) comes first when LOGN is odd, radix-4 passes follow.
template <typename T, int SIGN, int LOGN>
__device__ __forceinline__ void warp_fft(v2_t<T>* buf, const v2_t<T>* __restrict__ tw, int lane) {
  if constexpr (LOGN & 1) {
    fft_pass<T, SIGN, LOGN, 0, 1>(buf, tw, lane);
    fft_radix4_passes<T, SIGN, LOGN, 1>(buf, tw, lane);
  } else {
    fft_radix4_passes<T, SIGN, LOGN, 0>(buf, tw, lane);
  }
}

// DST-I of two real lines at once, by one warp.  With n = 2^LOGN, each line
// holds x_1..x_{n-1} (x_0 = x_n = 0): line a at raw[0 .. n-2], line b at
// raw[rs .. rs+n-2] (rs >= n+1).  On return the same slots hold
//     4 S_k = 4 sum_{j=1}^{n-1} x_j sin(pi j k / n),  k = 1..n-1.
// Method: y_j = 2 sin(j pi / n)(x_j + x_{n-j}) + (x_j - x_{n-j}) makes the odd
// outputs the running sums of the real parts and the even outputs the
// imaginary parts of one length-n real DFT; both lines share one complex FFT
// (y^a + i y^b).  `raw` must hold 2n reals (it doubles as the complex line).
// sin2[j] = 2 sin(j pi / n), tw[t] = e^{-2 pi i t / n}.
template <typename T, int LOGN>
__device__ __forceinline__ void warp_dst_pair(T* raw, int rs, const T* __restrict__ sin2,
                                              const v2_t<T>* __restrict__ tw, int lane) {
  using V = v2_t<T>;
  constexpr int n = 1 << LOGN;
  constexpr int PERJ = (n + 31) / 32;
  V c[PERJ];
#pragma unroll
  for (int t = 0; t < PERJ; ++t) {
    const int j = lane + 32 * t;
    if (n % 32 == 0 || j < n) {
      T xa = 0, xan = 0, xb = 0, xbn = 0;
      if (j > 0) {
        xa = raw[j - 1];
        xan = raw[n - j - 1];
        xb = raw[rs + j - 1];
        xbn = raw[rs + n - j - 1];
      }
      const T s = sin2[j];
      c[t] = {s * (xa + xan) + (xa - xan), s * (xb + xbn) + (xb - xbn)};
    }
  }
  __syncwarp();
  V* line = reinterpret_cast<V*>(raw);
#pragma unroll
  for (int t = 0; t < PERJ; ++t) {
    const int j = lane + 32 * t;
    if (n % 32 == 0 || j < n) line[j] = c[t];
  }
  __syncwarp();
  warp_fft<T, -1, LOGN>(line, tw, lane);

  // Separate the two real spectra.  For k in [0, n/2): r_k feeds the running
  // sum of the odd outputs, e_k is the even output S_{2k}.
  constexpr int H = n / 2;
  constexpr int CH = H >= 32 ? H / 32 : 1;
  const int k0 = lane * CH;
  const bool act = k0 < H;
  T ra[CH], rb[CH], ea[CH], eb[CH];
  T sa = 0, sb = 0;
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    ra[i] = rb[i] = ea[i] = eb[i] = 0;
    if (act) {
      const int k = k0 + i;
      const V C = line[k];
      if (k == 0) {
        ra[i] = C.x;
        rb[i] = C.y;
      } else {
        const V Cn = line[n - k];
        ra[i] = C.x + Cn.x;
        rb[i] = C.y + Cn.y;
        ea[i] = Cn.y - C.y;
        eb[i] = C.x - Cn.x;
      }
    }
    sa += ra[i];
    ra[i] = sa;
    sb += rb[i];
    rb[i] = sb;
  }
  // exclusive prefix of the per-lane totals across the warp
  T ta = sa, tb = sb;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T va = __shfl_up_sync(0xffffffffu, ta, off);
    const T vb = __shfl_up_sync(0xffffffffu, tb, off);
    if (lane >= off) {
      ta += va;
      tb += vb;
    }
  }
  ta -= sa;
  tb -= sb;
  __syncwarp();
  if (act) {
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      const int k = k0 + i;
      raw[2 * k] = ra[i] + ta;           // 4 S_{2k+1}
      raw[rs + 2 * k] = rb[i] + tb;
      if (k > 0) {
        raw[2 * k - 1] = ea[i];          // 4 S_{2k}
        raw[rs + 2 * k - 1] = eb[i];
      }
    }
  }
  __syncwarp();
}

}  // namespace bec

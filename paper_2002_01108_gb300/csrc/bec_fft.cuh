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

// Complex products with the fused multiply-adds written out, so that every
// compilation of a kernel (e.g. each block width) rounds them the same way.
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return {fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x)};
}
// a * conj(b)
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {
  return {fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -(a.x * b.y))};
}

// IEEE 754 binary64 <-> binary32 conversions in integer arithmetic.  On this
// GPU the hardware conversion runs on the FP64 pipe (2 per clock per SM),
// which made it the bottleneck of the FP32 passes that read or write the
// FP64 vectors.  Normal results are formed from the bit fields: the float
// exponent is the double's minus 896, and the 29 dropped mantissa bits round
// to nearest, ties to even (a carry into the exponent is the correct
// result, up to infinity).  Zero, subnormal, overflowing, infinite and NaN
// inputs take the hardware conversion.
// the rare cases, out of line so that the hardware conversion is not
// executed (and its result discarded) on the common path
static __device__ __noinline__ float f64_to_f32_slow(double x) { return (float)x; }
static __device__ __noinline__ double f32_to_f64_slow(float x) { return (double)x; }

__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e - 897u <= 253u) {                                  // float exponent 1..254
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    unsigned r = ((e - 896u) << 23) | m;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | r);
  }
  return f64_to_f32_slow(x);
}

__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e - 1u <= 253u) {                                    // normal float
    const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
  }
  return f32_to_f64_slow(x);
}

// value conversion between the preconditioner's storage types
// 1/x in FP64 with few FP64 instructions (a division is a long sequence on
// GB300, whose FP64 pipe issues 2 operations per clock per SM): the float
// reciprocal of the float-rounded x (__frcp_rn, relative error <= 2^-23
// against 1/x), then two Newton-Raphson steps for f(y) = 1/y - x,
// y <- y + y (1 - x y), each of which squares the relative error
// (2^-23 -> 2^-46 -> below the FP64 rounding).  The result is within one
// unit in the last place of 1/x.  |x| outside [2^-120, 2^120] (and zero,
// infinities, NaN) take the division.
static __device__ __noinline__ double rcp64_slow(double x) { return 1.0 / x; }

__device__ __forceinline__ double rcp64(double x) {
  const unsigned e = ((unsigned)__double2hiint(x) >> 20) & 0x7FFu;
  if (e - (1023u - 120u) <= 240u) {
    double y = f32_to_f64(__frcp_rn(f64_to_f32(x)));
    double r = fma(-x, y, 1.0);
    y = fma(y, r, y);
    r = fma(-x, y, 1.0);
    return fma(y, r, y);
  }
  return rcp64_slow(x);
}

// Asynchronous 4-byte copy from global to shared memory (no register holds
// the value, so many can be in flight per thread).  valid = false copies no
// bytes and writes zero.  cp_async_wait_all() makes the thread's own copies
// visible to it; a block barrier after it makes them visible to the block.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem),
               "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename TO, typename TI>
__device__ __forceinline__ TO convert(TI x) {
  if constexpr (sizeof(TO) == 4 && sizeof(TI) == 8) return f64_to_f32(x);
  else if constexpr (sizeof(TO) == 8 && sizeof(TI) == 4) return f32_to_f64(x);
  else return (TO)x;
}

// Complex slots a warp's line of n = 2^LOGN values occupies in shared memory:
// n plus one pad slot per 16 (the padded layout of the intermediate passes),
// made odd so that a block's lines also start on different banks.
__host__ __device__ constexpr int line_slots(int logn) {
  return ((1 << logn) + ((1 << logn) >> 4) + 1) | 1;
}

// position of element i in the padded layout: one slot skipped every 16
template <bool PAD>
__device__ __forceinline__ int pidx(int i) {
  return PAD ? i + (i >> 4) : i;
}

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
// SIGN * i * a
template <int SIGN, typename V>
__device__ __forceinline__ V cmul_si(V a) { return SIGN < 0 ? V{a.y, -a.x} : V{-a.y, a.x}; }

// In-register DFT of length R with kernel e^{SIGN 2 pi i r k / R}.
template <int R, int SIGN, typename V>
__device__ __forceinline__ void radix_dft(V (&v)[R]) {
  if constexpr (R == 2) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const V c = cadd(v[1], v[3]);
    const V wd = cmul_si<SIGN>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, wd);
    v[3] = csub(b, wd);
  } else {
    static_assert(R == 8, "radix 2, 4 or 8");
    // X_k = E_k + w^k O_k, X_{k+4} = E_k - w^k O_k with E, O the 4-point DFTs
    // of the even and odd samples and w = e^{SIGN 2 pi i / 8}
    using T = decltype(v[0].x);
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    radix_dft<4, SIGN>(e);
    radix_dft<4, SIGN>(o);
    const T h = T(0.70710678118654752440);
    // w o1 = h (1 + SIGN i) o1, w^2 o2 = SIGN i o2, w^3 o3 = h (-1 + SIGN i) o3
    // (the factor h is applied inside the final FMAs: e +- h u)
    const V s1 = cmul_si<SIGN>(o[1]);
    const V u1 = {o[1].x + s1.x, o[1].y + s1.y};
    const V t2 = cmul_si<SIGN>(o[2]);
    const V s3 = cmul_si<SIGN>(o[3]);
    const V u3 = {s3.x - o[3].x, s3.y - o[3].y};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = {fma(h, u1.x, e[1].x), fma(h, u1.y, e[1].y)};
    v[5] = {fma(-h, u1.x, e[1].x), fma(-h, u1.y, e[1].y)};
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = {fma(h, u3.x, e[3].x), fma(h, u3.y, e[3].y)};
    v[7] = {fma(-h, u3.x, e[3].x), fma(-h, u3.y, e[3].y)};
  }
}

// One Stockham autosort pass of radix R = 2^LOGR at span Ns = 2^LOGNS on a
// line of n = 2^LOGN complex values.  Butterfly j reads x[j + r n/R], applies
// the twiddles e^{SIGN 2 pi i (j mod Ns) r / (Ns R)}, does the radix-R DFT and
// writes x[(j div Ns) Ns R + (j mod Ns) + r Ns].  All reads finish before any
// write, so the pass works in place; PIN / POUT select the padded layout for
// the reads / writes.  tw[t] = e^{-2 pi i t / n}.  In FP32 one twiddle is read
// per butterfly and its powers are formed by multiplication; in FP64, whose
// arithmetic is the scarce resource, every power is read from the table.
template <typename T, int SIGN, int LOGN, int LOGNS, int LOGR, bool PIN, bool POUT>
__device__ __forceinline__ void fft_pass(v2_t<T>* buf, const v2_t<T>* __restrict__ tw,
                                         int lane) {
  using V = v2_t<T>;
  constexpr int n = 1 << LOGN, R = 1 << LOGR, Ns = 1 << LOGNS;
  constexpr int NB = n / R;
  constexpr int PER = (NB + 31) / 32;
  constexpr int TWSTEP = n / (Ns * R);
  // Padded positions as a per-thread base plus compile-time offsets:
  // pidx(j + r NB) = pidx(j) + r NB + (r NB) / 16 because j < NB and the
  // multiples of 16 are multiples of NB (or NB of 16); likewise for the
  // writes, whose butterfly outputs base + r Ns never straddle a multiple of
  // 16 except at multiples of 16 from base.
  V v[PER][R];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int j = lane + 32 * t;
    if (NB % 32 == 0 || j < NB) {
      const int rb = pidx<PIN>(j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[t][r] = buf[rb + r * NB + (PIN ? (r * NB) >> 4 : 0)];
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int j = lane + 32 * t;
    if (NB % 32 == 0 || j < NB) {
      const int k = j & (Ns - 1);
      if constexpr (Ns > 1) {
        if constexpr (sizeof(T) == 4) {
          V w = tw[k * TWSTEP];
          if (SIGN > 0) w.y = -w.y;
          V wr = w;
#pragma unroll
          for (int r = 1; r < R; ++r) {
            v[t][r] = cmul(v[t][r], wr);
            if (r + 1 < R) wr = cmul(wr, w);
          }
        } else {
#pragma unroll
          for (int r = 1; r < R; ++r) {
            const V w = tw[k * r * TWSTEP];
            v[t][r] = SIGN < 0 ? cmul(v[t][r], w) : cmulc(v[t][r], w);
          }
        }
      }
      radix_dft<R, SIGN>(v[t]);
      const int wb = pidx<POUT>(((j >> LOGNS) << (LOGNS + LOGR)) + k);
#pragma unroll
      for (int r = 0; r < R; ++r) buf[wb + r * Ns + (POUT ? (r * Ns) >> 4 : 0)] = v[t][r];
    }
  }
  __syncwarp();
}

// radix of the pass that starts at span 2^LOGNS: 8 while at least 3 bits
// remain (but not 8 then 2: 4 + 4 instead), else what remains
__host__ __device__ constexpr int pass_logr(int logn, int logns) {
  return (logn - logns >= 3 && logn - logns != 4) ? 3 : (logn - logns >= 2 ? 2 : 1);
}

// PLAST: the last pass also writes the padded layout
template <typename T, int SIGN, int LOGN, int LOGNS, bool PLAST = false>
__device__ __forceinline__ void fft_passes(v2_t<T>* buf, const v2_t<T>* __restrict__ tw,
                                           int lane) {
  if constexpr (LOGNS < LOGN) {
    constexpr int LOGR = pass_logr(LOGN, LOGNS);
    constexpr bool first = LOGNS == 0, last = LOGNS + LOGR == LOGN;
    fft_pass<T, SIGN, LOGN, LOGNS, LOGR, !first, !last || PLAST>(buf, tw, lane);
    fft_passes<T, SIGN, LOGN, LOGNS + LOGR, PLAST>(buf, tw, lane);
  }
}

// Complex FFT of length 2^LOGN in place in shared memory, natural order in
// and out, by one warp; the buffer holds line_slots(LOGN) complex values.
// SIGN = -1: X_k = sum_j x_j e^{-2 pi i jk/n}; SIGN = +1: the unnormalised
// inverse.  Radix-8 passes, then radix 4 or 2 for the remaining bits.
template <typename T, int SIGN, int LOGN>
__device__ __forceinline__ void warp_fft(v2_t<T>* buf, const v2_t<T>* __restrict__ tw, int lane) {
  fft_passes<T, SIGN, LOGN, 0>(buf, tw, lane);
}

// Output layout of warp_dst_pair.  FP64 writes S_k in natural order.  FP32
// writes them with one pad slot after every 2 CH reals, where lane l owns
// the CH = max(1, n/64) consecutive k from CH l: its stores then fall on
// distinct banks.  dst_out<T, LOGN>(j) is the slot of output j of a line;
// dst_line_stride(logn, bytes) the real slots from line a to line b (odd, and
// at least what the padded complex FFT line needs).
template <typename T, int LOGN>
__device__ __forceinline__ int dst_out(int j) {
  if constexpr (sizeof(T) == 8) return j;
  else return j + (j >> (LOGN >= 6 ? LOGN - 5 : 1));
}
__host__ __device__ constexpr int dst_line_stride(int logn, int bytes) {
  if (bytes == 8) return line_slots(logn);
  const int n = 1 << logn, shift = logn >= 6 ? logn - 5 : 1;
  const int need = (n - 2) + ((n - 2) >> shift) + 1;        // last output slot + 1
  return (need > line_slots(logn) ? need : line_slots(logn)) | 1;
}

// DST-I of two real lines at once, by one warp.  With n = 2^LOGN, each line
// holds x_1..x_{n-1} (x_0 = x_n = 0): line a at raw[0 .. n-2], line b at
// raw[rs .. rs+n-2] (rs = dst_line_stride(LOGN, sizeof(T))).  On return
//     4 S_k = 4 sum_{j=1}^{n-1} x_j sin(pi j k / n),  k = 1..n-1,
// of line a is at raw[dst_out(k - 1)] and that of line b at
// raw[rs + dst_out(k - 1)].
// Method: y_j = 2 sin(j pi / n)(x_j + x_{n-j}) + (x_j - x_{n-j}) makes the odd
// outputs the running sums of the real parts and the even outputs the
// imaginary parts of one length-n real DFT; both lines share one complex FFT
// (y^a + i y^b).  `raw` must hold 2 rs reals (it doubles as the complex
// line).  sin2[j] = 2 sin(j pi / n), tw[t] = e^{-2 pi i t / n}.
template <typename T, int LOGN>
__device__ __forceinline__ void warp_dst_pair(T* raw, int rs, const T* __restrict__ sin2,
                                              const v2_t<T>* __restrict__ tw, int lane) {
  using V = v2_t<T>;
  constexpr int n = 1 << LOGN;
  constexpr bool PAD = sizeof(T) == 4;     // FFT output and S_k in the padded layouts
  V* line = reinterpret_cast<V*>(raw);
  // The pre-pass is fused into the first radix pass of the FFT, which reads
  // its inputs y_j straight from the two real lines (no round trip of y
  // through shared memory); the first pass has no twiddles.
  {
    constexpr int LOGR = pass_logr(LOGN, 0), R = 1 << LOGR;
    constexpr int NB = n / R;
    constexpr int PER = (NB + 31) / 32;
    V v[PER][R];
    if constexpr (sizeof(T) == 8 && NB % 32 == 0 && R >= 4 && PER <= 2) {
      // FP64, where the additions are the scarce resource: inputs e and n - e
      // share x_e + x_{n-e} and, with the opposite sign, x_e - x_{n-e}.  A
      // lane forms them for r <= R/2 and takes those for r > R/2 from the lane
      // that holds n - e: lane (32 - l) mod 32, slot t' = PER - 1 - t,
      // r' = R - 1 - r.  Lane 0 holds both ends of its pairs (at t' = PER - t,
      // or r' = R - r when t = 0).  A third of the pre-pass additions go.
      constexpr int RH = R / 2;
      T sa[PER][RH + 1], da[PER][RH + 1], sb[PER][RH + 1], db[PER][RH + 1];
#pragma unroll
      for (int t = 0; t < PER; ++t) {
#pragma unroll
        for (int r = 0; r <= RH; ++r) {
          const int e = lane + 32 * t + r * NB;
          T xa = 0, xan = 0, xb = 0, xbn = 0;
          if (r > 0 || e > 0) {
            xa = raw[e - 1];
            xan = raw[n - e - 1];
            xb = raw[rs + e - 1];
            xbn = raw[rs + n - e - 1];
          }
          sa[t][r] = xa + xan;
          da[t][r] = xa - xan;
          sb[t][r] = xb + xbn;
          db[t][r] = xb - xbn;
        }
      }
      const int pl = (32 - lane) & 31;
      const bool l0 = lane == 0;
#pragma unroll
      for (int t = 0; t < PER; ++t) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int e = lane + 32 * t + r * NB;
          T s1, d1, s2, d2;
          if (r <= RH) {
            s1 = sa[t][r];
            d1 = da[t][r];
            s2 = sb[t][r];
            d2 = db[t][r];
          } else {
            const int tp = PER - 1 - t, rp = R - 1 - r;
            const int t0 = t == 0 ? 0 : PER - t, r0 = t == 0 ? R - r : rp;   // lane 0's own
            const T qs1 = __shfl_sync(0xffffffffu, sa[tp][rp], pl);
            const T qd1 = __shfl_sync(0xffffffffu, da[tp][rp], pl);
            const T qs2 = __shfl_sync(0xffffffffu, sb[tp][rp], pl);
            const T qd2 = __shfl_sync(0xffffffffu, db[tp][rp], pl);
            s1 = l0 ? sa[t0][r0] : qs1;
            d1 = -(l0 ? da[t0][r0] : qd1);
            s2 = l0 ? sb[t0][r0] : qs2;
            d2 = -(l0 ? db[t0][r0] : qd2);
          }
          const T sv = sin2[e];
          v[t][r] = {fma(sv, s1, d1), fma(sv, s2, d2)};
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const int j = lane + 32 * t;
        if (NB % 32 == 0 || j < NB) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int e = j + r * NB;
            T xa = 0, xan = 0, xb = 0, xbn = 0;
            if (r > 0 || e > 0) {
              xa = raw[e - 1];
              xan = raw[n - e - 1];
              xb = raw[rs + e - 1];
              xbn = raw[rs + n - e - 1];
            }
            const T s = sin2[e];
            v[t][r] = {s * (xa + xan) + (xa - xan), s * (xb + xbn) + (xb - xbn)};
          }
        }
      }
    }
    __syncwarp();
    constexpr bool POUT = LOGR < LOGN || PAD;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int j = lane + 32 * t;
      if (NB % 32 == 0 || j < NB) {
        radix_dft<R, -1>(v[t]);
        const int wb = pidx<POUT>(j << LOGR);
#pragma unroll
        for (int r = 0; r < R; ++r) line[wb + r + (POUT ? r >> 4 : 0)] = v[t][r];
      }
    }
    __syncwarp();
    fft_passes<T, -1, LOGN, LOGR, PAD>(line, tw, lane);
  }

  // Separate the two real spectra.  For k in [0, n/2): r_k feeds the running
  // sum of the odd outputs, e_k is the even output S_{2k}.  Lane l owns the
  // CH consecutive k from CH l: a serial running sum and one warp scan of
  // the lane totals.  In FP32 the FFT output and the S_k are in the padded
  // layouts, so these reads and writes are free of bank conflicts.
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
      const V C = line[pidx<PAD>(k)];
      if (k == 0) {
        ra[i] = C.x;
        rb[i] = C.y;
      } else {
        const V Cn = line[pidx<PAD>(n - k)];
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
      raw[dst_out<T, LOGN>(2 * k)] = ra[i] + ta;             // 4 S_{2k+1}
      raw[rs + dst_out<T, LOGN>(2 * k)] = rb[i] + tb;
      if (k > 0) {
        raw[dst_out<T, LOGN>(2 * k - 1)] = ea[i];            // 4 S_{2k}
        raw[rs + dst_out<T, LOGN>(2 * k - 1)] = eb[i];
      }
    }
  }
  __syncwarp();
}

}  // namespace bec

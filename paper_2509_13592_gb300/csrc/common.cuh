// Shared device helpers: complex arithmetic, radix-2/4/8/16 DFT butterflies,
// twiddle tables, error handling.
//
// The FFT convention is the paper's (Section III-B): the forward 2D DFT uses
// exp(-j 2 pi k n / L); the inverse uses exp(+j ...) and is unnormalised here
// (the 1/(L1 L2) factor is folded into the Fourier-domain multiplier).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bccb {

// ------------------------------------------------------------------------------------------
// complex helpers on float2 / double2
// ------------------------------------------------------------------------------------------
template <typename V> struct ScalarOf;
template <> struct ScalarOf<float2> { using T = float; };
template <> struct ScalarOf<double2> { using T = double; };

template <typename V>
__device__ __forceinline__ V cmk(typename ScalarOf<V>::T x, typename ScalarOf<V>::T y) {
  V r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
// complex64 sums as one paired FP32 instruction (add/sub.f32x2, sm_100 and later): half the
// issue slots of two scalar adds, each lane rounded as a scalar add.  A product that feeds such
// a sum is no longer fused into it; where that is the common form, twmadd below keeps the fused
// multiply-adds explicit.
__device__ __forceinline__ unsigned long long pk2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
template <typename V> __device__ __forceinline__ V cneg(V a) { return cmk<V>(-a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return cmk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cscale(V a, typename ScalarOf<V>::T s) {
  return cmk<V>(a.x * s, a.y * s);
}
// a * (-j) for the forward direction, a * (+j) for the inverse
template <bool INV, typename V> __device__ __forceinline__ V mul_mj(V a) {
  return INV ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x);
}
// multiply by the twiddle w (forward) or conj(w) (inverse)
template <bool INV, typename V> __device__ __forceinline__ V twmul(V a, V w) {
  return INV ? cmulc(a, w) : cmul(a, w);
}
// acc + twmul<INV>(a, w) as two fused multiply-adds per lane
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }
template <bool INV, typename V> __device__ __forceinline__ V twmadd(V acc, V a, V w) {
  return INV ? cmk<V>(fmx(a.y, w.y, fmx(a.x, w.x, acc.x)), fmx(-a.x, w.y, fmx(a.y, w.x, acc.y)))
             : cmk<V>(fmx(-a.y, w.y, fmx(a.x, w.x, acc.x)), fmx(a.y, w.x, fmx(a.x, w.y, acc.y)));
}

// ------------------------------------------------------------------------------------------
// compile-time twiddles W_16^p = exp(-j 2 pi p / 16) (forward sign)
// cos(pi/8), sin(pi/8), sqrt(1/2): mathematical constants
// ------------------------------------------------------------------------------------------
#define BCCB_C8 0.92387953251128675613
#define BCCB_S8 0.38268343236508977173
#define BCCB_R2 0.70710678118654752440

__host__ __device__ constexpr double cos16(int p) {
  return p == 0 ? 1.0 : p == 1 ? BCCB_C8 : p == 2 ? BCCB_R2 : p == 3 ? BCCB_S8 : p == 4 ? 0.0
       : p == 5 ? -BCCB_S8 : p == 6 ? -BCCB_R2 : p == 7 ? -BCCB_C8 : p == 8 ? -1.0
       : p == 9 ? -BCCB_C8 : p == 10 ? -BCCB_R2 : p == 11 ? -BCCB_S8 : p == 12 ? 0.0
       : p == 13 ? BCCB_S8 : p == 14 ? BCCB_R2 : BCCB_C8;
}
__host__ __device__ constexpr double sin16(int p) { return cos16((p + 12) & 15); }

// a * W_16^p (forward) or a * W_16^{-p} (inverse)
template <int P, bool INV, typename V> __device__ __forceinline__ V tw16(V a) {
  using T = typename ScalarOf<V>::T;
  constexpr int p = P & 15;
  if constexpr (p == 0) {
    return a;
  } else if constexpr (p == 4) {
    return mul_mj<INV>(a);
  } else if constexpr (p == 8) {
    return cneg(a);
  } else if constexpr (p == 12) {
    return mul_mj<!INV>(a);
  } else if constexpr ((p & 3) == 2) {
    // multiples of pi/4: r2 * (+-1 +- j)
    constexpr T r = (T)BCCB_R2;
    constexpr T c = (T)cos16(p) > 0 ? (T)1 : (T)-1;
    constexpr T s = (INV ? (T)1 : (T)-1) * ((T)sin16(p) > 0 ? (T)1 : (T)-1);
    // (a.x + j a.y)(c + j s) * r
    return cmk<V>(r * (c * a.x - s * a.y), r * (c * a.y + s * a.x));
  } else {
    constexpr T c = (T)cos16(p);
    constexpr T s = INV ? (T)sin16(p) : (T)-sin16(p);
    return cmul(a, cmk<V>(c, s));
  }
}

// ------------------------------------------------------------------------------------------
// radix-R DFT of v[0..R) in registers, natural order in and out:
//   v[k] <- sum_n v[n] exp(-+ j 2 pi n k / R)   (minus: forward, plus: inverse)
// Built from the split R = N1 * N2, n = e + N1 m, k = k' + N2 k'':
//   inner N2-point DFTs over m, twiddle W_R^{e k'}, outer N1-point DFTs over e.
// ------------------------------------------------------------------------------------------
template <bool INV, typename V> __device__ __forceinline__ void dft2(V& a, V& b) {
  V t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV, typename V> __device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
  V t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  // t1 +- (-+j) d lane by lane: a paired form would first have to swap d's lanes
  if (INV) {
    a1 = cmk<V>(t1.x - d.y, t1.y + d.x);
    a3 = cmk<V>(t1.x + d.y, t1.y - d.x);
  } else {
    a1 = cmk<V>(t1.x + d.y, t1.y - d.x);
    a3 = cmk<V>(t1.x - d.y, t1.y + d.x);
  }
}

template <int R, bool INV, typename V> struct Dft;

template <bool INV, typename V> struct Dft<1, INV, V> {
  static __device__ __forceinline__ void run(V*) {}
};
template <bool INV, typename V> struct Dft<2, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft2<INV>(v[0], v[1]); }
};
template <bool INV, typename V> struct Dft<4, INV, V> {
  static __device__ __forceinline__ void run(V* v) { dft4<INV>(v[0], v[1], v[2], v[3]); }
};
template <bool INV, typename V> struct Dft<8, INV, V> {
  // N1 = 2 (e), N2 = 4 (m)
  static __device__ __forceinline__ void run(V* v) {
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    v[3] = tw16<2, INV>(v[3]);  // e=1,k'=1: W_8^1
    v[5] = tw16<4, INV>(v[5]);  // e=1,k'=2: W_8^2
    v[7] = tw16<6, INV>(v[7]);  // e=1,k'=3: W_8^3
    dft2<INV>(v[0], v[1]);
    dft2<INV>(v[2], v[3]);
    dft2<INV>(v[4], v[5]);
    dft2<INV>(v[6], v[7]);
    // X[k' + 4k''] sits at v[2k' + k'']
    V o[8];
#pragma unroll
    for (int kp = 0; kp < 4; ++kp)
#pragma unroll
      for (int kpp = 0; kpp < 2; ++kpp) o[kp + 4 * kpp] = v[2 * kp + kpp];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
  }
};
template <bool INV, typename V> struct Dft<16, INV, V> {
  // N1 = 4 (e), N2 = 4 (m)
  static __device__ __forceinline__ void run(V* v) {
    dft4<INV>(v[0], v[4], v[8], v[12]);
    dft4<INV>(v[1], v[5], v[9], v[13]);
    dft4<INV>(v[2], v[6], v[10], v[14]);
    dft4<INV>(v[3], v[7], v[11], v[15]);
    // E_e[k'] sits at v[e + 4k']; twiddle W_16^{e k'}
    v[5] = tw16<1, INV>(v[5]);
    v[9] = tw16<2, INV>(v[9]);
    v[13] = tw16<3, INV>(v[13]);
    v[6] = tw16<2, INV>(v[6]);
    v[10] = tw16<4, INV>(v[10]);
    v[14] = tw16<6, INV>(v[14]);
    v[7] = tw16<3, INV>(v[7]);
    v[11] = tw16<6, INV>(v[11]);
    v[15] = tw16<9, INV>(v[15]);
    dft4<INV>(v[0], v[1], v[2], v[3]);
    dft4<INV>(v[4], v[5], v[6], v[7]);
    dft4<INV>(v[8], v[9], v[10], v[11]);
    dft4<INV>(v[12], v[13], v[14], v[15]);
    // X[k' + 4k''] sits at v[4k' + k'']
    V o[16];
#pragma unroll
    for (int kp = 0; kp < 4; ++kp)
#pragma unroll
      for (int kpp = 0; kpp < 4; ++kpp) o[kp + 4 * kpp] = v[4 * kp + kpp];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
  }
};

// ------------------------------------------------------------------------------------------
// radix schedule: n = 16 * 16 * ... * rem (rem in {2,4,8,16}); stage s has radix radix_of(n, s)
// ------------------------------------------------------------------------------------------
__host__ __device__ constexpr int log2i(int n) { return n <= 1 ? 0 : 1 + log2i(n / 2); }
__host__ __device__ constexpr int num_stages(int n) { return n <= 1 ? 0 : (log2i(n) + 3) / 4; }
__host__ __device__ constexpr int radix_of(int n, int s) {
  // all stages radix 16 except the last, which takes the remainder
  return (s < num_stages(n) - 1) ? 16 : (1 << (log2i(n) - 4 * (num_stages(n) - 1)));
}

// twiddle table length: W_TW^e for e in [0, TW)
constexpr int kTwiddleLen = 1024;

}  // namespace bccb

// ------------------------------------------------------------------------------------------
// host-side status codes (mirrors include/bccb.h)
// ------------------------------------------------------------------------------------------
#define BCCB_OK 0
#define BCCB_ERR_INVALID_ARG 1
#define BCCB_ERR_UNSUPPORTED 2
#define BCCB_ERR_CUDA 3
#define BCCB_ERR_KKT 4
#define BCCB_ERR_TIMEOUT 5

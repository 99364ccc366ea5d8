// Register-resident DFT building blocks (FP32) for the fused march.
//
// All DFTs take natural-order input and return natural-order output in the
// same registers: X[k] = sum_n x[n] W^{n k}, W = exp(-2 pi i / R) forward,
// exp(+2 pi i / R) inverse (unnormalised).
//
// Accuracy note.  The march applies the same forward/inverse pair tens of
// thousands of times, so any constant rounded to FP32 acts as a fixed
// perturbation of every step and its error grows linearly with the number of
// steps.  Every non-trivial constant (cos(pi/8), sin(pi/8), 1/sqrt(2)) and
// every table twiddle is therefore carried as an unevaluated sum hi + lo of
// two floats and applied with fused multiply-adds, so the only FP32 error
// left is the rounding of results, which varies from step to step.
#pragma once

#include <cuda_runtime.h>

namespace bpm {

constexpr double kC1d = 0.92387953251128673848;  // cos(pi/8)
constexpr double kS1d = 0.38268343236508978178;  // sin(pi/8)
constexpr double kHd = 0.70710678118654752440;   // sqrt(1/2)
constexpr float kC1h = float(kC1d);
constexpr float kC1l = float(kC1d - double(kC1h));
constexpr float kS1h = float(kS1d);
constexpr float kS1l = float(kS1d - double(kS1h));
constexpr float kHh = float(kHd);
constexpr float kHl = float(kHd - double(kHh));

// |p|^2 added to an FP64 band-power sum: the squares of FP32 values are
// exact in FP64, so the sum's only roundings are its FP64 additions.
__device__ __forceinline__ double pow_acc(double s, float2 p) {
  return fma(double(p.x), double(p.x), fma(double(p.y), double(p.y), s));
}

// Complex add / subtract.  PACK = true: one packed FP32x2 instruction (sm_100
// family) each; per component the result is the correctly rounded scalar
// sum or difference (a - b is formed as b * (-1) + a, which rounds once,
// exactly like a - b), so both forms give bit-identical results.  Packing
// halves the issue slots of the adds; whether that pays depends on the
// kernel (register pairing can cost moves), so kernels choose.
template <bool PACK = true>
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  if constexpr (PACK) return __fadd2_rn(a, b);
  else return make_float2(a.x + b.x, a.y + b.y);
}
template <bool PACK = true>
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  if constexpr (PACK) return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
  else return make_float2(a.x - b.x, a.y - b.y);
}

// Multiply by W4 = -i (forward) or +i (inverse): exact.
template <bool INV>
__device__ __forceinline__ float2 mul_w4(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// z * (c + i s) with c = ch + cl, s = sh + sl (double-float constant).
__device__ __forceinline__ float2 cmul_hl(float2 z, float ch, float sh,
                                          float cl, float sl) {
  float re = fmaf(z.x, cl, -(z.y * sl));
  re = fmaf(-z.y, sh, re);
  re = fmaf(z.x, ch, re);
  float im = fmaf(z.x, sl, z.y * cl);
  im = fmaf(z.y, ch, im);
  im = fmaf(z.x, sh, im);
  return make_float2(re, im);
}

// Constant policy: EXACT = true carries every internal constant as hi + lo;
// EXACT = false uses the nearest float (cheaper; adequate when the FFT only
// acts on the small per-step increment, see the fused kernel).
template <bool EXACT>
__device__ __forceinline__ float mul_h(float x) {
  if constexpr (EXACT) return fmaf(x, kHh, x * kHl);
  else return x * kHh;
}

// z * (c + i s) with a plain float constant.
__device__ __forceinline__ float2 cmul_f(float2 z, float c, float s) {
  return make_float2(fmaf(z.x, c, -(z.y * s)), fmaf(z.x, s, z.y * c));
}

template <bool EXACT>
__device__ __forceinline__ float2 cmul_k(float2 z, float ch, float sh, float cl, float sl) {
  if constexpr (EXACT) return cmul_hl(z, ch, sh, cl, sl);
  else return cmul_f(z, ch, sh);
}

// z * W8^1 (forward: (1 - i)/sqrt2; inverse: (1 + i)/sqrt2).
template <bool INV, bool EXACT = true>
__device__ __forceinline__ float2 mul_w8(float2 z) {
  return INV ? make_float2(mul_h<EXACT>(z.x - z.y), mul_h<EXACT>(z.x + z.y))
             : make_float2(mul_h<EXACT>(z.x + z.y), mul_h<EXACT>(z.y - z.x));
}
// z * W8^3 (forward: (-1 - i)/sqrt2; inverse: (-1 + i)/sqrt2).
template <bool INV, bool EXACT = true>
__device__ __forceinline__ float2 mul_w8_3(float2 z) {
  return INV ? make_float2(-mul_h<EXACT>(z.x + z.y), mul_h<EXACT>(z.x - z.y))
             : make_float2(mul_h<EXACT>(z.y - z.x), -mul_h<EXACT>(z.x + z.y));
}
// z * W16^1, W16^3, W16^9 (forward exp(-2 pi i m/16); inverse conjugate).
template <bool INV, bool EXACT = true>
__device__ __forceinline__ float2 mul_w16_1(float2 z) {
  return INV ? cmul_k<EXACT>(z, kC1h, kS1h, kC1l, kS1l)
             : cmul_k<EXACT>(z, kC1h, -kS1h, kC1l, -kS1l);
}
template <bool INV, bool EXACT = true>
__device__ __forceinline__ float2 mul_w16_3(float2 z) {
  return INV ? cmul_k<EXACT>(z, kS1h, kC1h, kS1l, kC1l)
             : cmul_k<EXACT>(z, kS1h, -kC1h, kS1l, -kC1l);
}
template <bool INV, bool EXACT = true>
__device__ __forceinline__ float2 mul_w16_9(float2 z) {
  return INV ? cmul_k<EXACT>(z, -kC1h, -kS1h, -kC1l, -kS1l)
             : cmul_k<EXACT>(z, -kC1h, kS1h, -kC1l, kS1l);
}

template <bool INV, bool PACK = true>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd<PACK>(a, b);
  v[1] = csub<PACK>(a, b);
}

// (the last two outputs add a swapped, negated pair: scalar, which folds the
// negation into the adds)
template <bool INV, bool PACK = true>
__device__ __forceinline__ void dft4_inplace(float2& x0, float2& x1,
                                             float2& x2, float2& x3) {
  float2 t0 = cadd<PACK>(x0, x2), t1 = csub<PACK>(x0, x2);
  float2 t2 = cadd<PACK>(x1, x3), t3 = mul_w4<INV>(csub<PACK>(x1, x3));
  x0 = cadd<PACK>(t0, t2);
  x2 = csub<PACK>(t0, t2);
  x1 = cadd<false>(t1, t3);
  x3 = csub<false>(t1, t3);
}

template <bool INV, bool PACK = true>
__device__ __forceinline__ void dft4(float2* v) {
  dft4_inplace<INV, PACK>(v[0], v[1], v[2], v[3]);
}

// 8 = 4 x 2: n = 2 n1 + n2, k = k1 + 4 k2.
template <bool INV, bool EXACT = true, bool PACK = true>
__device__ __forceinline__ void dft8(float2* v) {
  dft4_inplace<INV, PACK>(v[0], v[2], v[4], v[6]);   // n2 = 0 -> a[k1][0] at v[2 k1]
  dft4_inplace<INV, PACK>(v[1], v[3], v[5], v[7]);   // n2 = 1 -> a[k1][1] at v[2 k1 + 1]
  v[3] = mul_w8<INV, EXACT>(v[3]);
  v[5] = mul_w4<INV>(v[5]);
  v[7] = mul_w8_3<INV, EXACT>(v[7]);
  float2 o[8];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    o[k1] = cadd<PACK>(v[2 * k1], v[2 * k1 + 1]);
    o[k1 + 4] = csub<PACK>(v[2 * k1], v[2 * k1 + 1]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = o[k];
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2, inner twiddles W16^(n2 k1).
template <bool INV, bool EXACT = true, bool PACK = true>
__device__ __forceinline__ void dft16(float2* v) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2)
    dft4_inplace<INV, PACK>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // a[k1][n2] now at v[4 k1 + n2]
  v[5] = mul_w16_1<INV, EXACT>(v[5]);      // k1=1,n2=1: W^1
  v[6] = mul_w8<INV, EXACT>(v[6]);         // k1=1,n2=2: W^2
  v[7] = mul_w16_3<INV, EXACT>(v[7]);      // k1=1,n2=3: W^3
  v[9] = mul_w8<INV, EXACT>(v[9]);         // k1=2,n2=1: W^2
  v[10] = mul_w4<INV>(v[10]);              // k1=2,n2=2: W^4
  v[11] = mul_w8_3<INV, EXACT>(v[11]);     // k1=2,n2=3: W^6
  v[13] = mul_w16_3<INV, EXACT>(v[13]);    // k1=3,n2=1: W^3
  v[14] = mul_w8_3<INV, EXACT>(v[14]);     // k1=3,n2=2: W^6
  v[15] = mul_w16_9<INV, EXACT>(v[15]);    // k1=3,n2=3: W^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
    dft4_inplace<INV, PACK>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // X[k1 + 4 k2] at v[4 k1 + k2]: transpose the 4x4 block.
  float2 o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = o[k];
}

template <int R, bool INV, bool EXACT = true, bool PACK = true>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<INV, PACK>(v);
  else if constexpr (R == 4) dft4<INV, PACK>(v);
  else if constexpr (R == 8) dft8<INV, EXACT, PACK>(v);
  else if constexpr (R == 16) dft16<INV, EXACT, PACK>(v);
}

// z * w for a table twiddle t = (ch, sh, cl, sl) holding W = exp(-i a);
// the inverse uses conj(W).
template <bool INV>
__device__ __forceinline__ float2 mul_tw(float2 z, float4 t) {
  return INV ? cmul_hl(z, t.x, -t.y, t.z, -t.w) : cmul_hl(z, t.x, t.y, t.z, t.w);
}

}  // namespace bpm

// Arithmetic layer of the kernels: complex operations for the three vector
// forms (double2: FP64; float2: FP32; dfc: FP32 pairs) and the accumulators of
// the dot products.
//
// FP32-pair ("double-float") numbers represent x = hi + lo with |lo| <= ulp(hi)/2,
// a 48-bit significand (relative rounding about 2^-48 = 3.6e-15) with FP32's
// exponent range, computed entirely on the FP32 pipes.  The building blocks are
// the error-free transformations of Knuth (TwoSum: a + b = s + e exactly) and
// of Dekker/Ogita-Rump-Oishi with FMA (TwoProd: a * b = p + e exactly).  Each
// operation uses explicitly rounded intrinsics so that no contraction or
// reassociation can change it.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace kw {

struct __align__(8) df {
  float hi, lo;
};
struct __align__(16) dfc {
  df re, im;
};

// ------------------------------------------------------------- error-free transformations
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // requires |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// ------------------------------------------------------------- FP32-pair real arithmetic
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
// Pair addition in Dekker's form: the leading parts are added exactly, the
// trailing parts in plain FP32.  Its error is about 2^-48 (|a| + |b|), the same
// order as the rounding the operands already carry, at 11 operations.
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {   // b an exact FP32 number
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// a*b - c*d with one rounding of the leading parts
__device__ __forceinline__ df df_fms(df a, df b, df c, df d) {
  const df p = two_prod(a.hi, b.hi);
  const df q = two_prod(c.hi, d.hi);
  const df s = two_sum(p.hi, -q.hi);
  float lo = __fadd_rn(s.lo, __fsub_rn(p.lo, q.lo));
  lo = __fmaf_rn(a.hi, b.lo, lo);
  lo = __fmaf_rn(a.lo, b.hi, lo);
  lo = __fmaf_rn(-c.hi, d.lo, lo);
  lo = __fmaf_rn(-c.lo, d.hi, lo);
  return fast_two_sum(s.hi, lo);
}
// a*b + c*d
__device__ __forceinline__ df df_fma2(df a, df b, df c, df d) { return df_fms(a, b, df_neg(c), d); }

__device__ __forceinline__ df df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// ------------------------------------------------------------- complex operations
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ dfc cmul(dfc a, dfc b) {
  return {df_fms(a.re, b.re, a.im, b.im), df_fma2(a.re, b.im, a.im, b.re)};
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ dfc csub(dfc a, dfc b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }

__device__ __forceinline__ double2 vconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 vconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ dfc vconj(dfc a) { return {a.re, df_neg(a.im)}; }

template <class V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ dfc vzero<dfc>() { return {{0.f, 0.f}, {0.f, 0.f}}; }

// A complex FP64 scalar in the vector form.  `pair` is its FP32-pair form
// (x = re.hi, y = re.lo, z = im.hi, w = im.lo), precomputed by whoever wrote
// the scalar so that the kernels do no FP64 conversions per thread.
template <class V> __device__ __forceinline__ V vscalar(double2 d, float4 pair);
template <> __device__ __forceinline__ double2 vscalar<double2>(double2 d, float4) { return d; }
template <> __device__ __forceinline__ float2 vscalar<float2>(double2, float4 p) { return make_float2(p.x, p.z); }
template <> __device__ __forceinline__ dfc vscalar<dfc>(double2, float4 p) { return {{p.x, p.y}, {p.z, p.w}}; }

// A complex vector element from a real FP64 value (initialisation only).
template <class V> __device__ __forceinline__ V vreal(double x);
template <> __device__ __forceinline__ double2 vreal<double2>(double x) { return make_double2(x, 0.0); }
template <> __device__ __forceinline__ float2 vreal<float2>(double x) { return make_float2((float)x, 0.f); }
template <> __device__ __forceinline__ dfc vreal<dfc>(double x) { return {df_from_double(x), {0.f, 0.f}}; }

template <class V> __device__ __forceinline__ double2 vto_double(V v);
template <> __device__ __forceinline__ double2 vto_double<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ double2 vto_double<float2>(float2 v) { return make_double2(v.x, v.y); }
template <> __device__ __forceinline__ double2 vto_double<dfc>(dfc v) {
  return make_double2(df_to_double(v.re), df_to_double(v.im));
}

// Real element types of matrix values and projection rows.
template <class R> __device__ __forceinline__ R rfrom_double(double x);
template <> __device__ __forceinline__ double rfrom_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float rfrom_double<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ df rfrom_double<df>(double x) { return df_from_double(x); }

// ------------------------------------------------------------- acc += v * x (real v, complex x)
__device__ __forceinline__ void mac(double2& acc, double v, double2 x) {
  acc.x = fma(v, x.x, acc.x);
  acc.y = fma(v, x.y, acc.y);
}
__device__ __forceinline__ void mac(double2& acc, float v, double2 x) { mac(acc, (double)v, x); }
__device__ __forceinline__ void mac(float2& acc, float v, float2 x) {
  acc.x = fmaf(v, x.x, acc.x);
  acc.y = fmaf(v, x.y, acc.y);
}
// FP32-pair accumulation with deferred normalisation: acc.hi collects the
// rounded leading terms exactly through TwoSum, acc.lo the errors.
__device__ __forceinline__ void mac_pair(df& acc, float v, df x) {
  const df p = two_prod(v, x.hi);
  const df s = two_sum(acc.hi, p.hi);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, __fmaf_rn(v, x.lo, p.lo)));
}
__device__ __forceinline__ void mac_pair(df& acc, df v, df x) {
  const df p = two_prod(v.hi, x.hi);
  const df s = two_sum(acc.hi, p.hi);
  float e = __fmaf_rn(v.hi, x.lo, p.lo);
  e = __fmaf_rn(v.lo, x.hi, e);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ void mac(dfc& acc, float v, dfc x) {
  mac_pair(acc.re, v, x.re);
  mac_pair(acc.im, v, x.im);
}
__device__ __forceinline__ void mac(dfc& acc, df v, dfc x) {
  mac_pair(acc.re, v, x.re);
  mac_pair(acc.im, v, x.im);
}
// acc += x for vectors; the pair form adds the leading parts exactly (TwoSum)
// and collects every trailing part in acc.lo (normalise once at the end).
__device__ __forceinline__ void vacc(double2& acc, double2 x) {
  acc.x += x.x;
  acc.y += x.y;
}
__device__ __forceinline__ void vacc(float2& acc, float2 x) {
  acc.x += x.x;
  acc.y += x.y;
}
__device__ __forceinline__ void vacc(dfc& acc, dfc x) {
  const df sr = two_sum(acc.re.hi, x.re.hi), si = two_sum(acc.im.hi, x.im.hi);
  acc.re.hi = sr.hi;
  acc.re.lo = __fadd_rn(acc.re.lo, __fadd_rn(sr.lo, x.re.lo));
  acc.im.hi = si.hi;
  acc.im.lo = __fadd_rn(acc.im.lo, __fadd_rn(si.lo, x.im.lo));
}
__device__ __forceinline__ dfc normalize(dfc a) {
  return {fast_two_sum(a.re.hi, a.re.lo), fast_two_sum(a.im.hi, a.im.lo)};
}
__device__ __forceinline__ double2 normalize(double2 a) { return a; }
__device__ __forceinline__ float2 normalize(float2 a) { return a; }

// ------------------------------------------------------------- dot-product accumulators
// Accumulator type A: double (FP64 form), float (FP32 form, FP64 across chunks),
// df (FP32-pair form).
// Bring an accumulator to normalised form (pairs accumulate with deferred
// normalisation, so hi and lo may overlap).
__device__ __forceinline__ double anorm(double a) { return a; }
__device__ __forceinline__ float anorm(float a) { return a; }
__device__ __forceinline__ df anorm(df a) { return two_sum(a.hi, a.lo); }
__device__ __forceinline__ void aadd(double& a, double v) { a += v; }
__device__ __forceinline__ void aadd(float& a, float v) { a += v; }
__device__ __forceinline__ void aadd(df& a, df v) { a = df_add(a, v); }

// rho += r^T r (unconjugated): re += x^2 - y^2, im += 2 x y;  nrm += x^2 + y^2
__device__ __forceinline__ void acc_rho_nrm(double& re, double& im, double& n, double2 r) {
  re += r.x * r.x - r.y * r.y;
  im += 2.0 * r.x * r.y;
  n += r.x * r.x + r.y * r.y;
}
__device__ __forceinline__ void acc_rho_nrm(float& re, float& im, float& n, float2 r) {
  re += r.x * r.x - r.y * r.y;
  im += 2.f * r.x * r.y;
  n += r.x * r.x + r.y * r.y;
}
// acc += a*b for pairs, deferring normalisation: the rounded leading product is
// added exactly (TwoSum), every error term goes to acc.lo.
__device__ __forceinline__ void acc_prod(df& acc, df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const df s = two_sum(acc.hi, p.hi);
  float e = __fmaf_rn(a.hi, b.lo, p.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  acc.hi = s.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ void acc_rho_nrm(df& re, df& im, df& n, dfc r) {
  const df mim = df_neg(r.im);
  acc_prod(re, r.re, r.re);
  acc_prod(re, mim, r.im);
  const df x2 = {2.f * r.re.hi, 2.f * r.re.lo};
  acc_prod(im, x2, r.im);
  acc_prod(n, r.re, r.re);
  acc_prod(n, r.im, r.im);
}
// (re, im) += x^dagger y (one element): re += x.re y.re + x.im y.im, im += x.re y.im - x.im y.re
__device__ __forceinline__ void acc_cdot(double& re, double& im, double2 x, double2 y) {
  re += x.x * y.x + x.y * y.y;
  im += x.x * y.y - x.y * y.x;
}
__device__ __forceinline__ void acc_cdot(float& re, float& im, float2 x, float2 y) {
  re += x.x * y.x + x.y * y.y;
  im += x.x * y.y - x.y * y.x;
}
__device__ __forceinline__ void acc_cdot(df& re, df& im, dfc x, dfc y) {
  acc_prod(re, x.re, y.re);
  acc_prod(re, x.im, y.im);
  acc_prod(im, x.re, y.im);
  acc_prod(im, df_neg(x.im), y.re);
}
// nrm += |r|^2
__device__ __forceinline__ void acc_nrm(double& n, double2 r) { n += r.x * r.x + r.y * r.y; }
__device__ __forceinline__ void acc_nrm(float& n, float2 r) { n += r.x * r.x + r.y * r.y; }
__device__ __forceinline__ void acc_nrm(df& n, dfc r) {
  acc_prod(n, r.re, r.re);
  acc_prod(n, r.im, r.im);
}
// (re, im) += a * r  (real a)
__device__ __forceinline__ void acc_proj(double& re, double& im, double a, double2 r) {
  re = fma(a, r.x, re);
  im = fma(a, r.y, im);
}
__device__ __forceinline__ void acc_proj(float& re, float& im, float a, float2 r) {
  re = fmaf(a, r.x, re);
  im = fmaf(a, r.y, im);
}
__device__ __forceinline__ void acc_proj(df& re, df& im, df a, dfc r) {
  acc_prod(re, a, r.re);
  acc_prod(im, a, r.im);
}
// (re, im) += p
__device__ __forceinline__ void acc_cplx(double& re, double& im, double2 p) {
  re += p.x;
  im += p.y;
}
__device__ __forceinline__ void acc_cplx(float& re, float& im, float2 p) {
  re += p.x;
  im += p.y;
}
__device__ __forceinline__ void acc_cplx(df& re, df& im, dfc p) {
  re = df_add(re, p.re);
  im = df_add(im, p.im);
}

__device__ __forceinline__ double ato_double(double a) { return a; }
__device__ __forceinline__ double ato_double(float a) { return (double)a; }
__device__ __forceinline__ double ato_double(df a) { return df_to_double(a); }   // hi + lo, exact in FP64

template <class A> __device__ __forceinline__ A azero();
template <> __device__ __forceinline__ double azero<double>() { return 0.0; }
template <> __device__ __forceinline__ float azero<float>() { return 0.f; }
template <> __device__ __forceinline__ df azero<df>() { return {0.f, 0.f}; }

// ------------------------------------------------------------- packed FP32 pairs (sm_100 and later)
// The real and imaginary parts of a complex FP32 pair travel together in the
// packed two-lane FP32 instructions (add/mul/fma .f32x2, round to nearest), so
// one instruction does the same error-free step on both parts.  A complex pair
// in this layout is {hi = (re.hi, im.hi), lo = (re.lo, im.lo)}.
struct cpk {
  float2 hi, lo;
};
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ cpk cpk_of(dfc v) { return {make_float2(v.re.hi, v.im.hi), make_float2(v.re.lo, v.im.lo)}; }
__device__ __forceinline__ cpk cpk_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
// acc += a * r for a real pair a and a complex pair r (both parts at once):
// the rounded leading products are added exactly (TwoSum), the product errors
// and the trailing terms go to acc.lo (normalised at the end), as acc_prod.
__device__ __forceinline__ void acc_proj_pk(cpk& acc, df a, const cpk& r) {
  const float2 ah = make_float2(a.hi, a.hi), al = make_float2(a.lo, a.lo);
  const float2 p = pk_mul(ah, r.hi);
  float2 e = pk_fma(ah, r.hi, make_float2(-p.x, -p.y));
  e = pk_fma(ah, r.lo, e);
  e = pk_fma(al, r.hi, e);
  const float2 s = pk_add(acc.hi, p);
  const float2 bb = pk_sub(s, acc.hi);
  const float2 err = pk_add(pk_sub(acc.hi, pk_sub(s, bb)), pk_sub(p, bb));
  acc.hi = s;
  acc.lo = pk_add(acc.lo, pk_add(err, e));
}

// A complex pair coefficient c in the two forms a packed product needs:
// c * v = re * v + im * swap(v) with re = (c.re, c.re), im = (-c.im, c.im)
// (lane 0 the real part, lane 1 the imaginary part).  pair: (re.hi, re.lo,
// im.hi, im.lo); sign = -1 gives the coefficient of -c.
struct cpk_coef {
  cpk re, im;
};
__device__ __forceinline__ cpk_coef cpk_coef_of(float4 pair, float sign) {
  const float rh = sign * pair.x, rl = sign * pair.y, ih = sign * pair.z, il = sign * pair.w;
  return {{make_float2(rh, rh), make_float2(rl, rl)}, {make_float2(-ih, ih), make_float2(-il, il)}};
}
__device__ __forceinline__ cpk cpk_swap(const cpk& v) {
  return {make_float2(v.hi.y, v.hi.x), make_float2(v.lo.y, v.lo.x)};
}
__device__ __forceinline__ dfc dfc_of(const cpk& v) { return {{v.hi.x, v.lo.x}, {v.hi.y, v.lo.y}}; }

// One term x * y of a packed pair sum kept as (S exact sum of the rounded
// leading products, L every error and trailing term): TwoProd of the leading
// parts, TwoSum into S, the cross terms into L (Dekker's form with one
// normalisation at the end, as the sums of dfc products elsewhere).
__device__ __forceinline__ void pk_term(float2& S, float2& L, const cpk& x, const cpk& y) {
  const float2 p = pk_mul(x.hi, y.hi);
  const float2 e = pk_fma(x.hi, y.hi, make_float2(-p.x, -p.y));
  const float2 s = pk_add(S, p);
  const float2 bb = pk_sub(s, S);
  const float2 t = pk_add(pk_sub(S, pk_sub(s, bb)), pk_sub(p, bb));
  S = s;
  L = pk_add(L, pk_add(t, e));
  L = pk_fma(x.hi, y.lo, L);
  L = pk_fma(x.lo, y.hi, L);
}

// r_{n+1} = a r_n - b q - c r_{n-1} (Eq. 16) for complex pairs in one packed
// sum of six products (na = a, nb = -b, nc = -c as cpk_coef), normalised once.
__device__ __forceinline__ cpk three_term_pk(const cpk_coef& na, const cpk_coef& nb, const cpk_coef& nc,
                                             const cpk& rn, const cpk& q, const cpk& rm) {
  float2 S = pk_mul(na.re.hi, rn.hi);
  float2 L = pk_fma(na.re.hi, rn.hi, make_float2(-S.x, -S.y));
  L = pk_fma(na.re.hi, rn.lo, L);
  L = pk_fma(na.re.lo, rn.hi, L);
  pk_term(S, L, na.im, cpk_swap(rn));
  pk_term(S, L, nb.re, q);
  pk_term(S, L, nb.im, cpk_swap(q));
  pk_term(S, L, nc.re, rm);
  pk_term(S, L, nc.im, cpk_swap(rm));
  const float2 h = pk_add(S, L);
  return {h, pk_sub(L, pk_sub(h, S))};   // Fast2Sum: (h, error)
}

// acc += (x.re^2, x.im^2) for a complex pair x (lanes: the squares of the two parts)
__device__ __forceinline__ void acc_sq_pk(cpk& acc, const cpk& x) {
  const float2 p = pk_mul(x.hi, x.hi);
  float2 e = pk_fma(x.hi, x.hi, make_float2(-p.x, -p.y));
  const float2 two_lo = pk_add(x.lo, x.lo);
  e = pk_fma(x.hi, two_lo, e);                       // 2 hi lo
  const float2 s = pk_add(acc.hi, p);
  const float2 bb = pk_sub(s, acc.hi);
  const float2 err = pk_add(pk_sub(acc.hi, pk_sub(s, bb)), pk_sub(p, bb));
  acc.hi = s;
  acc.lo = pk_add(acc.lo, pk_add(err, e));
}

#define KW_FULL_MASK 0xffffffffu
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(KW_FULL_MASK, v, o); }
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(KW_FULL_MASK, v, o); }
__device__ __forceinline__ df shfl_xor(df v, int o) {
  return {__shfl_xor_sync(KW_FULL_MASK, v.hi, o), __shfl_xor_sync(KW_FULL_MASK, v.lo, o)};
}
__device__ __forceinline__ void vshfl_add(double2& a, int o) {
  a.x += shfl_xor(a.x, o);
  a.y += shfl_xor(a.y, o);
}
__device__ __forceinline__ void vshfl_add(float2& a, int o) {
  a.x += shfl_xor(a.x, o);
  a.y += shfl_xor(a.y, o);
}
__device__ __forceinline__ void vshfl_add(dfc& a, int o) {
  a.re = df_add(a.re, shfl_xor(a.re, o));
  a.im = df_add(a.im, shfl_xor(a.im, o));
}

// Warp sum of an accumulator (every lane gets the result).
template <class A> __device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) aadd(v, shfl_xor(v, off));
  return v;
}
template <> __device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(KW_FULL_MASK, v, off);
  return v;
}

}  // namespace kw

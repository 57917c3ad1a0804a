// dw_common.cuh -- device-side building blocks of the Wilson-Dirac CG library:
// complex arithmetic, field storage formats, the batch/system descriptor and
// the deterministic two-level grid reduction with the CG scalar updates.
//
// Storage (per parity block of Vh sites, per right-hand side), structure of
// arrays so that consecutive threads (consecutive even-odd site indices)
// touch consecutive 16-byte words:
//   spinor FP64 : 12 planes of double2       (complex k = 3*spin + colour)
//   spinor FP32 :  6 planes of float4        (complex 2j, 2j+1)
//   spinor F16/BF16: 3 planes of 8 halves (uint4) + 1 plane of FP32 per-site
//                  scale; stored value = component / max|component of site|
//   spinor I16   : the same planes of 16-bit fixed point: round(32767 *
//                  component / max|component of site|), FP32 per-site scale
//   links  (parity p of the base site, direction mu) planes of
//          FP64 18: 9 double2   FP64 12: 6 double2
//          FP32 18: 9 float2    FP32 12: 3 float4
//          F16/BF16 18: uint4, uint4, uint (18 halves)
//          F16/BF16 12: uint4, uint2 (12 halves)
//          I16 as F16/BF16, each entry stored as round(32767 * entry)
//   12-real links keep rows 0 and 1; row 2 = conj(row0 x row1) (SU(3)).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dw {

enum Prec { P64 = 0, P32 = 1, P16 = 2, PB16 = 3, PDF = 4, PI16 = 5 };

// ------------------------------------------------------------------ double-float
// A real as the unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2),
// about 49 significant bits, computed on the FP32 pipes.  The error-free
// transforms are Knuth's TwoSum, Dekker's Fast2Sum and the FMA form of
// TwoProduct; every step uses explicitly rounded intrinsics so the compiler
// cannot contract or reorder them.
// Conversions between binary64 and the (hi, lo) pair use integer bit
// operations (GB300's FP64 pipe runs at 1/61 of the FP32 rate):
//   d -> hi = sign | exponent | top 23 mantissa bits of d (truncated),
//        lo = the low 29 mantissa bits scaled by 2^(e - 1075), rounded to 24
//        bits: |d - (hi + lo)| <= 2^-47 |d|.  Values below 2^-126 flush to 0,
//        lo flushes below 2^-74; infinities and NaN keep their class.
//   (hi, lo) -> d = widen(hi) + widen(lo) with exact bit widening and one
//        FP64 add.
__device__ __forceinline__ void split_double(double d, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const int ef = e - 896;  // float biased exponent
  const unsigned mant23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  if (e == 0x7FF) {
    h = __uint_as_float(sign | 0x7F800000u | (((hw & 0xFFFFFu) | lw) ? 0x400000u : 0u));
    l = 0.f;
    return;
  }
  if (ef <= 0) {
    h = __uint_as_float(sign);
    l = 0.f;
    return;
  }
  if (ef >= 255) {
    h = __uint_as_float(sign | 0x7F800000u);
    l = 0.f;
    return;
  }
  h = __uint_as_float(sign | ((unsigned)ef << 23) | mant23);
  const int es = e - 948;  // biased float exponent of 2^(e - 1075)
  const float r = __uint2float_rn(lw & 0x1FFFFFFFu);
  const float lm = es > 0 ? __fmul_rn(r, __uint_as_float((unsigned)es << 23)) : 0.f;
  l = sign ? -lm : lm;
}
__device__ __forceinline__ double widen_float(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned long long m = (unsigned long long)(b & 0x7FFFFFu) << 29;
  if (e == 0u) return __longlong_as_double((long long)sign);  // zero (FP32 denormals flush)
  const unsigned long long de = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(sign | (de << 52) | m));
}

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ explicit DF(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ explicit DF(float v) : hi(v), lo(0.f) {}
  __device__ explicit DF(double d) { split_double(d, hi, lo); }
  __device__ explicit operator double() const { return widen_float(hi) + widen_float(lo); }
  __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ DF df_make(float h, float l) {
  DF r;
  r.hi = h;
  r.lo = l;
  return r;
}
// a + b exactly as s + e (Knuth)
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// a + b exactly as s + e when |a| >= |b| (Dekker)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ DF operator-(DF a) { return df_make(-a.hi, -a.lo); }
// hi parts added exactly, lo parts added in FP32, renormalised: the error is
// below about 2u^2 (|a| + |b|), u = 2^-24, which is the scale the per-site
// comparisons measure
__device__ __forceinline__ DF operator+(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// a*b + c (the float and double overloads stay visible next to this one)
using ::fma;
__device__ __forceinline__ DF fma(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const DF s = two_sum(p, c.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(c.lo, e)));
}

// Sum with the hi parts added exactly and everything else collected in lo,
// without renormalising: for values that feed further double-float
// operations, which accept any (hi, lo) with |lo| << |hi|.
__device__ __forceinline__ DF add_lazy(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  return df_make(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF renorm(DF a) { return fast_two_sum(a.hi, a.lo); }

// Exact high product and its low-order terms: x*y = p + e (+ x.lo*y.lo).
__device__ __forceinline__ DF prod_terms(DF x, DF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_make(p, e);
}

// Sum of 6 products x_i * y_i: exact high products added pairwise with TwoSum
// (a tree, so the three first-level sums are independent), all low-order
// terms collected in FP32, one renormalisation.
__device__ __forceinline__ DF df_dot6(const DF (&x)[6], const DF (&y)[6]) {
  const DF a = prod_terms(x[0], y[0]), b = prod_terms(x[1], y[1]), c = prod_terms(x[2], y[2]);
  const DF d = prod_terms(x[3], y[3]), e = prod_terms(x[4], y[4]), f = prod_terms(x[5], y[5]);
  const DF ab = two_sum(a.hi, b.hi), cd = two_sum(c.hi, d.hi), ef = two_sum(e.hi, f.hi);
  const DF abcd = two_sum(ab.hi, cd.hi);
  const DF all = two_sum(abcd.hi, ef.hi);
  const float lo1 = __fadd_rn(__fadd_rn(a.lo, b.lo), __fadd_rn(c.lo, d.lo));
  const float lo2 = __fadd_rn(__fadd_rn(e.lo, f.lo), __fadd_rn(ab.lo, cd.lo));
  const float lo3 = __fadd_rn(__fadd_rn(ef.lo, abcd.lo), all.lo);
  return fast_two_sum(all.hi, __fadd_rn(__fadd_rn(lo1, lo2), lo3));
}


// Two independent double-float numbers in the two lanes of packed FP32x2
// registers: each instruction below does the same IEEE operation on both
// lanes (Blackwell's fma/add/mul.rn.f32x2), so one sequence computes two
// double-float results.  Same algorithms as the scalar forms above.
struct DF2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.f), a); }
// a + b exactly as s + e, lane by lane (Knuth)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 bb = sub2(s, a);
  e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// x * y for a double-float x (same in both lanes) and two double-floats y:
// exact high product p and the low-order terms e, x*y = p + e (+ x.lo*y.lo)
__device__ __forceinline__ void prod_terms2(DF x, const DF2& y, float2& p, float2& e) {
  const float2 xh = bc2(x.hi);
  p = __fmul2_rn(xh, y.hi);
  e = __ffma2_rn(xh, y.hi, make_float2(-p.x, -p.y));
  e = __ffma2_rn(xh, y.lo, e);
  e = __ffma2_rn(bc2(x.lo), y.hi, e);
}
// Two six-term dot products sum_i x_i * y_i (lane-wise in y), as df_dot6.
__device__ __forceinline__ DF2 df2_dot6(const DF (&x)[6], const DF2 (&y)[6]) {
  float2 p[6], e[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) prod_terms2(x[i], y[i], p[i], e[i]);
  float2 ab, abe, cd, cde, ef, efe, abcd, abcde, all, alle;
  two_sum2(p[0], p[1], ab, abe);
  two_sum2(p[2], p[3], cd, cde);
  two_sum2(p[4], p[5], ef, efe);
  two_sum2(ab, cd, abcd, abcde);
  two_sum2(abcd, ef, all, alle);
  const float2 lo1 = __fadd2_rn(__fadd2_rn(e[0], e[1]), __fadd2_rn(e[2], e[3]));
  const float2 lo2 = __fadd2_rn(__fadd2_rn(e[4], e[5]), __fadd2_rn(abe, cde));
  const float2 lo3 = __fadd2_rn(__fadd2_rn(efe, abcde), alle);
  const float2 lo = __fadd2_rn(__fadd2_rn(lo1, lo2), lo3);
  DF2 r;
  r.hi = __fadd2_rn(all, lo);
  r.lo = sub2(lo, sub2(r.hi, all));
  return r;
}

// ------------------------------------------------------------------ complex
template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R a, R b) {
  Cx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return cx(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return cx(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return cx(s * a.re, s * a.im); }
// i*a
template <typename R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> a) { return cx(-a.im, a.re); }
// a*b
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return cx(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
// c + a*b
template <typename R>
__device__ __forceinline__ Cx<R> cmadd(Cx<R> a, Cx<R> b, Cx<R> c) {
  return cx(fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im)));
}
// conj(a)*b
template <typename R>
__device__ __forceinline__ Cx<R> cjmul(Cx<R> a, Cx<R> b) {
  return cx(fma(a.re, b.re, a.im * b.im), fma(a.re, b.im, -a.im * b.re));
}
// c + conj(a)*b
template <typename R>
__device__ __forceinline__ Cx<R> cjmadd(Cx<R> a, Cx<R> b, Cx<R> c) {
  return cx(fma(a.re, b.re, fma(a.im, b.im, c.re)), fma(a.re, b.im, fma(-a.im, b.re, c.im)));
}
template <typename R>
__device__ __forceinline__ Cx<R> conjx(Cx<R> a) { return cx(a.re, -a.im); }

// ------------------------------------------------------------------ 16-bit helpers
template <int P>
struct H16;
template <>
struct H16<P16> {
  static constexpr float kUnit = 1.f;  // stored units per 1
  __device__ static __forceinline__ float2 to2(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h);
  }
  __device__ static __forceinline__ uint32_t from2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};
template <>
struct H16<PB16> {
  static constexpr float kUnit = 1.f;
  __device__ static __forceinline__ float2 to2(uint32_t w) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
    return __bfloat1622float2(h);
  }
  __device__ static __forceinline__ uint32_t from2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};

// 16-bit fixed point: q = round(32767 x) for x in [-1, 1], two per word
// (first value in the low half).  to2 returns the integers q themselves
// (kUnit = 32767 units per 1), so the unit folds into the per-site scale.
// (Exact bit-level conversions on the FP32/ALU pipes were measured slower
// than the conversion instructions.)
template <>
struct H16<PI16> {
  static constexpr float kUnit = 32767.f;
  __device__ static __forceinline__ float2 to2(uint32_t w) {
    return make_float2(__int2float_rn((int)(short)(w & 0xFFFFu)), __int2float_rn((int)w >> 16));
  }
  // a, b in [-1, 1] (values already divided by their site maximum)
  __device__ static __forceinline__ uint32_t from2(float a, float b) {
    const int qa = __float2int_rn(a * 32767.f), qb = __float2int_rn(b * 32767.f);
    return ((uint32_t)qa & 0xFFFFu) | ((uint32_t)qb << 16);
  }
};

// ------------------------------------------------------------------ 16-bit word arithmetic
// Operations on 32-bit words holding one complex number as two 16-bit floats
// (real part in the low half).  pm/rot_pm are packed two-lane adds; cmac and
// cmac_adj are FP32-accumulating products of 16-bit operands (the product of
// two 16-bit floats is exact in FP32, so only the accumulation rounds, in FP32).
// A sign flip of one lane is an XOR of its sign bit.
constexpr uint32_t kNegRe = 0x00008000u, kNegIm = 0x80000000u, kNegBoth = 0x80008000u;

__device__ __forceinline__ uint32_t swap_halves(uint32_t w) { return __byte_perm(w, 0u, 0x1032); }

template <int P>
struct HW;

#define DW_HW_SPECIALISE(PREC, TY, PLUS_MINUS, MINUS_PLUS)                                              \
  template <>                                                                                          \
  struct HW<PREC> {                                                                                    \
    /* a + b, a - b per lane */                                                                        \
    __device__ static __forceinline__ uint32_t add(uint32_t a, uint32_t b) {                           \
      uint32_t d;                                                                                      \
      asm("add.rn." TY "x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));                                 \
      return d;                                                                                        \
    }                                                                                                  \
    __device__ static __forceinline__ uint32_t sub(uint32_t a, uint32_t b) {                           \
      uint32_t d;                                                                                      \
      asm("sub.rn." TY "x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));                                 \
      return d;                                                                                        \
    }                                                                                                  \
    /* a + T i b (T = +1 or -1): i b = (-b.im, b.re), one rounding per lane */                         \
    template <int T>                                                                                   \
    __device__ static __forceinline__ uint32_t rot_add(uint32_t a, uint32_t b) {                       \
      uint32_t d;                                                                                      \
      const uint32_t m = T > 0 ? PLUS_MINUS : MINUS_PLUS;                                              \
      asm("fma.rn." TY "x2 %0, %1, %2, %3;" : "=r"(d) : "r"(swap_halves(b)), "r"(m), "r"(a));         \
      return d;                                                                                        \
    }                                                                                                  \
    /* (re, im) += u h, with hn = h whose imaginary lane is negated */                                 \
    __device__ static __forceinline__ void cmac(float& re, float& im, uint32_t u, uint32_t h,          \
                                                uint32_t hn) {                                         \
      asm("{ .reg .b16 ur, ui, hr, hi, nr, ni;\n\t"                                                 \
          "mov.b32 {ur, ui}, %2;\n\tmov.b32 {hr, hi}, %3;\n\tmov.b32 {nr, ni}, %4;\n\t"                \
          "fma.rn.f32." TY " %0, ur, hr, %0;\n\tfma.rn.f32." TY " %0, ui, ni, %0;\n\t"                 \
          "fma.rn.f32." TY " %1, ur, hi, %1;\n\tfma.rn.f32." TY " %1, ui, hr, %1; }"                  \
          : "+f"(re), "+f"(im) : "r"(u), "r"(h), "r"(hn));                                             \
    }                                                                                                  \
    /* (re, im) += conj(u) h, with hm = h whose real lane is negated */                                \
    __device__ static __forceinline__ void cmac_adj(float& re, float& im, uint32_t u, uint32_t h,      \
                                                    uint32_t hm) {                                     \
      asm("{ .reg .b16 ur, ui, hr, hi, mr, mi;\n\t"                                                 \
          "mov.b32 {ur, ui}, %2;\n\tmov.b32 {hr, hi}, %3;\n\tmov.b32 {mr, mi}, %4;\n\t"                \
          "fma.rn.f32." TY " %0, ur, hr, %0;\n\tfma.rn.f32." TY " %0, ui, hi, %0;\n\t"                 \
          "fma.rn.f32." TY " %1, ur, hi, %1;\n\tfma.rn.f32." TY " %1, ui, mr, %1; }"                  \
          : "+f"(re), "+f"(im) : "r"(u), "r"(h), "r"(hm));                                             \
    }                                                                                                  \
    /* conj(a d - b c) in FP32 from 16-bit words; nc, nd = c, d with both lanes negated */             \
    __device__ static __forceinline__ void cross(float& re, float& im, uint32_t a, uint32_t b,         \
                                                 uint32_t c, uint32_t d, uint32_t nc, uint32_t nd) {   \
      re = 0.f;                                                                                        \
      im = 0.f;                                                                                        \
      asm("{ .reg .b16 ar, ai, br, bi, cr, ci, dr, di, ncr, nci, ndr, ndi;\n\t"                     \
          "mov.b32 {ar, ai}, %2;\n\tmov.b32 {br, bi}, %3;\n\tmov.b32 {cr, ci}, %4;\n\t"                \
          "mov.b32 {dr, di}, %5;\n\tmov.b32 {ncr, nci}, %6;\n\tmov.b32 {ndr, ndi}, %7;\n\t"            \
          "fma.rn.f32." TY " %0, ar, dr, %0;\n\tfma.rn.f32." TY " %0, ai, ndi, %0;\n\t"                \
          "fma.rn.f32." TY " %0, br, ncr, %0;\n\tfma.rn.f32." TY " %0, bi, ci, %0;\n\t"                \
          "fma.rn.f32." TY " %1, ar, ndi, %1;\n\tfma.rn.f32." TY " %1, ai, ndr, %1;\n\t"               \
          "fma.rn.f32." TY " %1, br, ci, %1;\n\tfma.rn.f32." TY " %1, bi, cr, %1; }"                  \
          : "+f"(re), "+f"(im) : "r"(a), "r"(b), "r"(c), "r"(d), "r"(nc), "r"(nd));                    \
    }                                                                                                  \
  };

// lane constants (low half first): (-1, +1) and (+1, -1)
DW_HW_SPECIALISE(P16, "f16", 0x3C00BC00u, 0xBC003C00u)
DW_HW_SPECIALISE(PB16, "bf16", 0x3F80BF80u, 0xBF803F80u)
#undef DW_HW_SPECIALISE

// ------------------------------------------------------------------ spinor storage
template <int P>
struct Spin;

template <>
struct Spin<P64> {
  using R = double;
  static constexpr bool kScaled = false;
  static constexpr int kBytes = 192;  // bytes per site
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<double> (&v)[12]) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 t = __ldg(b + (size_t)k * vh + s);
      v[k] = cx(t.x, t.y);
    }
  }
  // a site's stored words, formed in registers before they are written
  struct Packed {
    double2 w[12];
  };
  __device__ static __forceinline__ Packed pack(const Cx<double> (&v)[12]) {
    Packed o;
#pragma unroll
    for (int k = 0; k < 12; ++k) o.w[k] = make_double2(v[k].re, v[k].im);
    return o;
  }
  __device__ static __forceinline__ void store_packed(char* base, int vh, int s, const Packed& o) {
    double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) b[(size_t)k * vh + s] = o.w[k];
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<double> (&v)[12]) {
    store_packed(base, vh, s, pack(v));
  }
  // v <- the value a store followed by a load would give
  __device__ static __forceinline__ void roundtrip(Cx<double> (&)[12]) {}
};

template <>
struct Spin<P32> {
  using R = float;
  static constexpr bool kScaled = false;
  static constexpr int kBytes = 96;
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<float> (&v)[12]) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 t = __ldg(b + (size_t)k * vh + s);
      v[2 * k] = cx(t.x, t.y);
      v[2 * k + 1] = cx(t.z, t.w);
    }
  }
  struct Packed {
    float4 w[6];
  };
  __device__ static __forceinline__ Packed pack(const Cx<float> (&v)[12]) {
    Packed o;
#pragma unroll
    for (int k = 0; k < 6; ++k) o.w[k] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
    return o;
  }
  __device__ static __forceinline__ void store_packed(char* base, int vh, int s, const Packed& o) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; ++k) b[(size_t)k * vh + s] = o.w[k];
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<float> (&v)[12]) {
    store_packed(base, vh, s, pack(v));
  }
  __device__ static __forceinline__ void roundtrip(Cx<float> (&)[12]) {}
};

// Largest component magnitude of a site, the per-site scale of 16-bit
// storage.  Sites whose largest component is below 1e-30 are stored as zero:
// 1/scale would overflow FP32 there (values that small appear at the edge of
// a point source's Krylov support), and they are negligible against any
// residual norm the solver tests.
__device__ __forceinline__ float site_max(const Cx<float> (&v)[12]) {
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
  return m >= 1e-30f ? m : 0.f;
}

template <int P>
struct Spin16 {
  using R = float;
  static constexpr bool kScaled = true;
  static constexpr int kBytes = 52;  // 48 bytes of halves + 4 bytes of scale
  // stored values (unscaled, in stored units) and the site's scale per unit:
  // value = v * sc
  __device__ static __forceinline__ void load_raw(const char* base, int vh, int s, Cx<float> (&v)[12], float& sc) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    sc = __ldg(reinterpret_cast<const float*>(base + (size_t)48 * vh) + s) * (1.f / H16<P>::kUnit);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 t = __ldg(b + (size_t)k * vh + s);
      float2 a = H16<P>::to2(t.x), c = H16<P>::to2(t.y), d = H16<P>::to2(t.z), e = H16<P>::to2(t.w);
      v[4 * k + 0] = cx(a.x, a.y);
      v[4 * k + 1] = cx(c.x, c.y);
      v[4 * k + 2] = cx(d.x, d.y);
      v[4 * k + 3] = cx(e.x, e.y);
    }
  }
  // stored words (one complex per word, see HW) and the site's scale
  __device__ static __forceinline__ void load_words(const char* base, int vh, int s, uint32_t (&w)[12], float& sc) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    sc = __ldg(reinterpret_cast<const float*>(base + (size_t)48 * vh) + s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint4 t = __ldg(b + (size_t)k * vh + s);
      w[4 * k + 0] = t.x;
      w[4 * k + 1] = t.y;
      w[4 * k + 2] = t.z;
      w[4 * k + 3] = t.w;
    }
  }
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<float> (&v)[12]) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    const float sc = __ldg(reinterpret_cast<const float*>(base + (size_t)48 * vh) + s) * (1.f / H16<P>::kUnit);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 t = __ldg(b + (size_t)k * vh + s);
      float2 a = H16<P>::to2(t.x), c = H16<P>::to2(t.y), d = H16<P>::to2(t.z), e = H16<P>::to2(t.w);
      v[4 * k + 0] = cx(a.x * sc, a.y * sc);
      v[4 * k + 1] = cx(c.x * sc, c.y * sc);
      v[4 * k + 2] = cx(d.x * sc, d.y * sc);
      v[4 * k + 3] = cx(e.x * sc, e.y * sc);
    }
  }
  struct Packed {
    uint4 w[3];
    float m;
  };
  __device__ static __forceinline__ Packed pack(const Cx<float> (&v)[12]) {
    Packed o;
    o.m = site_max(v);
    const float inv = o.m > 0.f ? 1.0f / o.m : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o.w[k].x = H16<P>::from2(v[4 * k + 0].re * inv, v[4 * k + 0].im * inv);
      o.w[k].y = H16<P>::from2(v[4 * k + 1].re * inv, v[4 * k + 1].im * inv);
      o.w[k].z = H16<P>::from2(v[4 * k + 2].re * inv, v[4 * k + 2].im * inv);
      o.w[k].w = H16<P>::from2(v[4 * k + 3].re * inv, v[4 * k + 3].im * inv);
    }
    return o;
  }
  __device__ static __forceinline__ void store_packed(char* base, int vh, int s, const Packed& o) {
    uint4* b = reinterpret_cast<uint4*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) b[(size_t)k * vh + s] = o.w[k];
    reinterpret_cast<float*>(base + (size_t)48 * vh)[s] = o.m;
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<float> (&v)[12]) {
    store_packed(base, vh, s, pack(v));
  }
  __device__ static __forceinline__ void roundtrip(Cx<float> (&v)[12]) {
    const float m = site_max(v);
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    const float mu = m * (1.f / H16<P>::kUnit);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      float2 q = H16<P>::to2(H16<P>::from2(v[k].re * inv, v[k].im * inv));
      v[k] = cx(q.x * mu, q.y * mu);
    }
  }
};
template <>
struct Spin<P16> : Spin16<P16> {};
template <>
struct Spin<PB16> : Spin16<PB16> {};
template <>
struct Spin<PI16> : Spin16<PI16> {};

// double-float: 12 planes of float4 (re.hi, re.lo, im.hi, im.lo)
template <>
struct Spin<PDF> {
  using R = DF;
  static constexpr bool kScaled = false;
  static constexpr int kBytes = 192;
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<DF> (&v)[12]) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      float4 t = __ldg(b + (size_t)k * vh + s);
      v[k].re = df_make(t.x, t.y);
      v[k].im = df_make(t.z, t.w);
    }
  }
  struct Packed {
    float4 w[12];
  };
  __device__ static __forceinline__ Packed pack(const Cx<DF> (&v)[12]) {
    Packed o;
#pragma unroll
    for (int k = 0; k < 12; ++k) o.w[k] = make_float4(v[k].re.hi, v[k].re.lo, v[k].im.hi, v[k].im.lo);
    return o;
  }
  __device__ static __forceinline__ void store_packed(char* base, int vh, int s, const Packed& o) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; ++k) b[(size_t)k * vh + s] = o.w[k];
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<DF> (&v)[12]) {
    store_packed(base, vh, s, pack(v));
  }
  // the three colours of one spin
  __device__ static __forceinline__ void load_spin(const char* base, int vh, int s, int spin, Cx<DF> (&v)[3]) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float4 t = __ldg(b + (size_t)(3 * spin + c) * vh + s);
      v[c].re = df_make(t.x, t.y);
      v[c].im = df_make(t.z, t.w);
    }
  }
  __device__ static __forceinline__ void roundtrip(Cx<DF> (&)[12]) {}
};

// ------------------------------------------------------------------ link storage
template <typename R>
__device__ __forceinline__ void rebuild_row2(Cx<R> (&u)[9]) {
  // row2 = conj(row0 x row1)
  u[6] = conjx(cmul(u[1], u[5]) - cmul(u[2], u[4]));
  u[7] = conjx(cmul(u[2], u[3]) - cmul(u[0], u[5]));
  u[8] = conjx(cmul(u[0], u[4]) - cmul(u[1], u[3]));
}

template <int P, bool C12>
struct Link;

template <bool C12>
struct Link<P64, C12> {
  using R = double;
  static constexpr int kBytes = C12 ? 96 : 144;  // per site per direction
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<double> (&u)[9]) {
    const double2* b = reinterpret_cast<const double2*>(base);
    constexpr int n = C12 ? 6 : 9;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      double2 t = __ldg(b + (size_t)k * vh + s);
      u[k] = cx(t.x, t.y);
    }
    if (C12) rebuild_row2(u);
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<double> (&u)[9]) {
    double2* b = reinterpret_cast<double2*>(base);
    constexpr int n = C12 ? 6 : 9;
#pragma unroll
    for (int k = 0; k < n; ++k) b[(size_t)k * vh + s] = make_double2(u[k].re, u[k].im);
  }
};

template <>
struct Link<P32, false> {
  using R = float;
  static constexpr int kBytes = 72;
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<float> (&u)[9]) {
    const float2* b = reinterpret_cast<const float2*>(base);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float2 t = __ldg(b + (size_t)k * vh + s);
      u[k] = cx(t.x, t.y);
    }
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<float> (&u)[9]) {
    float2* b = reinterpret_cast<float2*>(base);
#pragma unroll
    for (int k = 0; k < 9; ++k) b[(size_t)k * vh + s] = make_float2(u[k].re, u[k].im);
  }
};

template <>
struct Link<P32, true> {
  using R = float;
  static constexpr int kBytes = 48;
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<float> (&u)[9]) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 t = __ldg(b + (size_t)k * vh + s);
      u[2 * k] = cx(t.x, t.y);
      u[2 * k + 1] = cx(t.z, t.w);
    }
    rebuild_row2(u);
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<float> (&u)[9]) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      b[(size_t)k * vh + s] = make_float4(u[2 * k].re, u[2 * k].im, u[2 * k + 1].re, u[2 * k + 1].im);
  }
};

template <bool C12>
struct Link<PDF, C12> {
  using R = DF;
  static constexpr int kBytes = C12 ? 96 : 144;
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<DF> (&u)[9]) {
    const float4* b = reinterpret_cast<const float4*>(base);
    constexpr int n = C12 ? 6 : 9;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      float4 t = __ldg(b + (size_t)k * vh + s);
      u[k].re = df_make(t.x, t.y);
      u[k].im = df_make(t.z, t.w);
    }
    if (C12) rebuild_row2(u);
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<DF> (&u)[9]) {
    float4* b = reinterpret_cast<float4*>(base);
    constexpr int n = C12 ? 6 : 9;
#pragma unroll
    for (int k = 0; k < n; ++k) b[(size_t)k * vh + s] = make_float4(u[k].re.hi, u[k].re.lo, u[k].im.hi, u[k].im.lo);
  }
};

template <int P, bool C12>
struct Link16 {
  using R = float;
  static constexpr int kBytes = C12 ? 24 : 36;
  __device__ static __forceinline__ void load(const char* base, int vh, int s, Cx<float> (&u)[9]) {
    constexpr float k = 1.f / H16<P>::kUnit;  // stored units -> entry
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(base) + s);
    float2 f0 = H16<P>::to2(a.x), f1 = H16<P>::to2(a.y), f2 = H16<P>::to2(a.z), f3 = H16<P>::to2(a.w);
    u[0] = cx(f0.x * k, f0.y * k);
    u[1] = cx(f1.x * k, f1.y * k);
    u[2] = cx(f2.x * k, f2.y * k);
    u[3] = cx(f3.x * k, f3.y * k);
    if (C12) {
      const uint2 c = __ldg(reinterpret_cast<const uint2*>(base + (size_t)16 * vh) + s);
      float2 g0 = H16<P>::to2(c.x), g1 = H16<P>::to2(c.y);
      u[4] = cx(g0.x * k, g0.y * k);
      u[5] = cx(g1.x * k, g1.y * k);
      rebuild_row2(u);
    } else {
      const uint4 c = __ldg(reinterpret_cast<const uint4*>(base + (size_t)16 * vh) + s);
      const uint32_t d = __ldg(reinterpret_cast<const uint32_t*>(base + (size_t)32 * vh) + s);
      float2 g0 = H16<P>::to2(c.x), g1 = H16<P>::to2(c.y), g2 = H16<P>::to2(c.z), g3 = H16<P>::to2(c.w);
      float2 g4 = H16<P>::to2(d);
      u[4] = cx(g0.x * k, g0.y * k);
      u[5] = cx(g1.x * k, g1.y * k);
      u[6] = cx(g2.x * k, g2.y * k);
      u[7] = cx(g3.x * k, g3.y * k);
      u[8] = cx(g4.x * k, g4.y * k);
    }
  }
  // 16-bit words; with compression the third row is rebuilt from FP32-accumulated
  // products of the stored rows and rounded once to 16 bits
  __device__ static __forceinline__ void load_words(const char* base, int vh, int s, uint32_t (&u)[9]) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(base) + s);
    u[0] = a.x;
    u[1] = a.y;
    u[2] = a.z;
    u[3] = a.w;
    if (C12) {
      const uint2 c = __ldg(reinterpret_cast<const uint2*>(base + (size_t)16 * vh) + s);
      u[4] = c.x;
      u[5] = c.y;
      const uint32_t n3 = u[3] ^ kNegBoth, n4 = u[4] ^ kNegBoth, n5 = u[5] ^ kNegBoth;
      float re, im;
      HW<P>::cross(re, im, u[1], u[2], u[4], u[5], n4, n5);  // conj(u01 u12 - u02 u11)
      u[6] = H16<P>::from2(re, im);
      HW<P>::cross(re, im, u[2], u[0], u[5], u[3], n5, n3);  // conj(u02 u10 - u00 u12)
      u[7] = H16<P>::from2(re, im);
      HW<P>::cross(re, im, u[0], u[1], u[3], u[4], n3, n4);  // conj(u00 u11 - u01 u10)
      u[8] = H16<P>::from2(re, im);
    } else {
      const uint4 c = __ldg(reinterpret_cast<const uint4*>(base + (size_t)16 * vh) + s);
      u[4] = c.x;
      u[5] = c.y;
      u[6] = c.z;
      u[7] = c.w;
      u[8] = __ldg(reinterpret_cast<const uint32_t*>(base + (size_t)32 * vh) + s);
    }
  }
  __device__ static __forceinline__ void store(char* base, int vh, int s, const Cx<float> (&u)[9]) {
    uint4 a;
    a.x = H16<P>::from2(u[0].re, u[0].im);
    a.y = H16<P>::from2(u[1].re, u[1].im);
    a.z = H16<P>::from2(u[2].re, u[2].im);
    a.w = H16<P>::from2(u[3].re, u[3].im);
    reinterpret_cast<uint4*>(base)[s] = a;
    if (C12) {
      uint2 c;
      c.x = H16<P>::from2(u[4].re, u[4].im);
      c.y = H16<P>::from2(u[5].re, u[5].im);
      reinterpret_cast<uint2*>(base + (size_t)16 * vh)[s] = c;
    } else {
      uint4 c;
      c.x = H16<P>::from2(u[4].re, u[4].im);
      c.y = H16<P>::from2(u[5].re, u[5].im);
      c.z = H16<P>::from2(u[6].re, u[6].im);
      c.w = H16<P>::from2(u[7].re, u[7].im);
      reinterpret_cast<uint4*>(base + (size_t)16 * vh)[s] = c;
      reinterpret_cast<uint32_t*>(base + (size_t)32 * vh)[s] = H16<P>::from2(u[8].re, u[8].im);
    }
  }
};
template <bool C12>
struct Link<P16, C12> : Link16<P16, C12> {};
template <bool C12>
struct Link<PB16, C12> : Link16<PB16, C12> {};
template <bool C12>
struct Link<PI16, C12> : Link16<PI16, C12> {};

// ------------------------------------------------------------------ descriptors
// A field reference inside a system: address of (rhs r, parity par) block is
// p + r*rhs_stride + par*par_stride (bytes).  Parity-only fields use
// par_stride = 0 and are only addressed with the parity they hold.
struct Slot {
  char* p;
  long long rhs_stride;
  long long par_stride;
};

enum SlotId {
  S_LLO = 0,   // inner-precision links
  S_LHI,       // high-precision links (FP64 or double-float)
  S_B,         // source b in the high precision (full)
  S_X,         // high-precision accumulator x (full; the caller's field when high = FP64)
  S_BH,        // prepared even source (high precision)
  S_RT,        // high-precision residual / temporary (full: even = r, odd = t)
  S_XL,        // low-precision solution increment (accumulate precision)
  S_R,         // inner residual
  S_P,         // search direction
  S_Z,         // D^dag r
  S_W,         // D p
  S_T,         // odd temporary (inner)
  S_AUX0,      // operator/API use
  S_AUX1,
  S_AUX2,
  S_AUX3,
  S_XU,        // the caller's solution field (FP64)
  S_BU,        // the caller's source field (FP64)
  S_LF64,      // the caller's FP64 links (final certification)
  kNumSlots
};

// Unsigned division by an invariant divisor d < 2^31 (Granlund & Montgomery
// 1994, branch-free form): q = (t + ((n - t) >> s1)) >> s2, t = umulhi(m, n).
struct FastDiv {
  unsigned m;
  int s1, s2;
};
__device__ __forceinline__ int fdiv(int n, FastDiv f) {
  const unsigned t = __umulhi(f.m, (unsigned)n);
  return (int)((t + (((unsigned)n - t) >> f.s1)) >> f.s2);
}

struct SysDesc {
  int lxh, ly, lz, lt;  // Lx/2, Ly, Lz, Lt
  // kappa and kappa^2 as FP32 (kappa_f = fl(kappa), kappa2_f = fl(kappa^2)) and
  // the low parts of their double-float forms, formed once on the host: GB300's
  // FP64 pipe (about two operations per clock per SM) makes a per-thread
  // double-to-float conversion cost microseconds per launch
  float kappa_f, kappa2_f, kappa_lo, kappa2_lo;
  FastDiv div_lxh, div_ly, div_lz;
  int vh;               // sites per parity
  int nrhs;
  int anti_t;
  int tpp;              // thread blocks per parity for this system
  int tile0;            // first block (within one parity) of this system
  int col0;             // first column (system, rhs) index
  int part0;            // first partial-sum slot (one per block and column)
  int sys;              // system index
  double kappa;
  Slot f[kNumSlots];
};

// All systems of one launch, passed as a __grid_constant__ kernel parameter
// (no descriptor buffers in device memory; CUDA graphs capture it by value).
// Blocks [sd[i].tile0, sd[i].tile0 + sd[i].tpp) of each parity belong to
// system i.
constexpr int kMaxSys = 8;
struct Batch {
  int nsys;  // systems in this launch
  int ntot;  // blocks per parity over all systems (grid x per parity)
  int T;     // sites per block (per right-hand side), multiple of 32
  int RB;    // right-hand sides per block
  int ny;    // right-hand-side blocks, ceil(nrhs / RB): the grid is x = (parity
             // range, tile, rhs block) with the rhs block varying fastest
  int rev;   // 1: blocks walk the grid from its end (see DW_BLOCK_PROLOGUE)
  SysDesc sd[kMaxSys];
};

__device__ __forceinline__ int block_system(const Batch& B, int b) {
  int si = 0;
  while (si + 1 < B.nsys && b >= B.sd[si + 1].tile0) ++si;
  return si;
}

// Per-column (system, right-hand side) CG state, in device memory.
struct ColState {
  double gamma;    // |z|^2, z = A-side residual
  double alpha, beta;
  float alpha_f, beta_f;  // alpha and beta rounded to FP32 by the finalizer
  // alpha of the iteration whose term alpha p is not yet in the low-precision
  // increment xl (added by k_update_p or k_fold_x; 0 once added), and FP32
  double alpha_x;
  float alpha_xf;
  double rr;       // iterated |r|^2
  double rr_ref;   // |r|^2 at the last reliable update
  double bnorm2;   // |b|^2 (full lattice)
  double tol2;     // tol^2 * |b|^2
  double delta2;   // delta^2
  double store[4]; // scalar outputs of plain reductions
  unsigned long long deadline_ns;  // globaltimer deadline (0 = none)
  int iter, maxiter, nrel;
  int defect;      // 1: restart the low-precision CG after every high-precision correction
  int active;      // 1 while iterating
  int do_rel;      // reliable update pending
  int status;      // dw_status of this column
  int xzero;       // initial guess is zero: the first residual is the source itself
  int restart;     // defect correction: the next beta is 0 (new search direction)
  int zsrc;        // zero source: the solution is x = 0
  int pad;
};

// Batch-wide flags.
struct Flags {
  int active;       // number of active columns
  int rel_pending;  // number of columns with a reliable update pending
  int loops;        // iterations run by the device-driven loop
  int max_loops;    // hard cap on loops (maxiter + 2)
  int rel_runs;     // reliable-update passes run by the device-driven loop
  int pad;
};

enum Fin {
  FIN_STORE0 = 0,  // store[0] = v  (plain reductions)
  FIN_STORE1,
  FIN_STORE2,
  FIN_STORE3,
  FIN_BNORM,       // bnorm2 = v, tol2 = tol^2 v (tol^2 kept in tol2 before)
  FIN_ALPHA,       // alpha = gamma / v
  FIN_UPDATE,      // rr = v; iter++; decide on a reliable update
  FIN_RELIABLE,    // rr = rr_ref = v (true residual); convergence decision
  FIN_GAMMA0,      // gamma = v, beta = 0
  FIN_BETA,        // beta = v / gamma; gamma = v
  FIN_XNORM,       // |x0|^2: a zero guess skips the first FP64 residual
  FIN_RESID0,      // first residual = source (zero guess)
};

struct RedArgs {
  double* partial;
  ColState* cols;
  Flags* flags;
  int fin;
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void deactivate(ColState& C, Flags* F, int status) {
  if (C.active) {
    C.active = 0;
    C.status = status;
    atomicSub(&F->active, 1);
  }
}

// CG scalar recurrences, run by one thread of the last block of a system.
__device__ __forceinline__ void finalize(const RedArgs& ra, int col, double v) {
  ColState& C = ra.cols[col];
  switch (ra.fin) {
    case FIN_STORE0: C.store[0] = v; break;
    case FIN_STORE1: C.store[1] = v; break;
    case FIN_STORE2: C.store[2] = v; break;
    case FIN_STORE3: C.store[3] = v; break;
    case FIN_BNORM:
      C.bnorm2 = v;
      C.tol2 = C.tol2 * v;
      if (v == 0.0) {  // D x = 0 has the solution x = 0: nothing to iterate
        C.zsrc = 1;
        deactivate(C, ra.flags, 0);
      }
      break;
    case FIN_ALPHA:
      if (!C.active) break;
      if (!(v > 0.0) || !isfinite(v) || !isfinite(C.gamma)) {
        // p^dag A p <= 0 or not finite: CG cannot continue
        deactivate(C, ra.flags, 7 /* DW_ERR_BREAKDOWN */);
      } else {
        C.alpha = C.gamma / v;
        C.alpha_f = (float)C.alpha;
        C.alpha_x = C.alpha;
        C.alpha_xf = C.alpha_f;
      }
      break;
    case FIN_UPDATE: {
      if (!C.active) break;
      C.rr = v;
      C.iter += 1;
      bool timeout = C.deadline_ns != 0ull && globaltimer_ns() > C.deadline_ns;
      if (!isfinite(v)) {
        deactivate(C, ra.flags, 7);
      } else if (v <= C.tol2 || v < C.delta2 * C.rr_ref || C.iter >= C.maxiter || timeout) {
        C.do_rel = 1;
        atomicAdd(&ra.flags->rel_pending, 1);
      }
      break;
    }
    case FIN_XNORM:
      C.xzero = v == 0.0 ? 1 : 0;
      if (C.xzero && C.do_rel) {
        C.do_rel = 0;
        atomicSub(&ra.flags->rel_pending, 1);
      }
      break;
    case FIN_RESID0:
      if (!C.xzero) break;
      C.xzero = 0;
      C.rr = v;
      C.rr_ref = v;
      if (v <= C.tol2) deactivate(C, ra.flags, 0);
      else if (!isfinite(v)) deactivate(C, ra.flags, 7);
      break;
    case FIN_RELIABLE: {
      if (!C.do_rel) break;
      C.do_rel = 0;
      C.alpha_x = 0.0;  // k_fold_x added alpha p to x
      C.alpha_xf = 0.f;
      atomicSub(&ra.flags->rel_pending, 1);
      C.rr = v;
      C.rr_ref = v;
      C.nrel += 1;
      if (C.defect) C.restart = 1;
      bool timeout = C.deadline_ns != 0ull && globaltimer_ns() > C.deadline_ns;
      if (v <= C.tol2) deactivate(C, ra.flags, 0);
      else if (!isfinite(v)) deactivate(C, ra.flags, 7);
      else if (C.iter >= C.maxiter) deactivate(C, ra.flags, 6 /* NOT_CONVERGED */);
      else if (timeout) deactivate(C, ra.flags, 8 /* TIMEOUT */);
      break;
    }
    case FIN_GAMMA0:
      if (!C.active) break;
      C.gamma = v;
      C.beta = 0.0;
      C.beta_f = 0.f;
      break;
    case FIN_BETA:
      if (!C.active) break;
      C.beta = C.restart ? 0.0 : v / C.gamma;
      C.beta_f = (float)C.beta;
      C.restart = 0;
      C.gamma = v;
      break;
  }
}

// Warp total in lane 0 only (other lanes hold partial sums), fixed order.  Only
// the lanes whose partial is still needed add, 31 FP64 additions per warp
// instead of the butterfly's 160: GB300 executes two FP64 thread operations per
// clock per SM, so the butterfly alone cost several microseconds per launch.
__device__ __forceinline__ double warp_sum_lane0(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_down_sync(0xffffffffu, v, o);
    if (lane < o) v += t;
  }
  return v;
}

// Value reduced inside a block: double-float for FP32 and double-float
// arithmetic (added on the FP32 pipes, about 48 significant bits), IEEE FP64
// for FP64 arithmetic.  Block partials and both grid levels are IEEE FP64.
template <typename R>
struct RedT {
  using type = DF;
};
template <>
struct RedT<double> {
  using type = double;
};
__device__ __forceinline__ DF to_red(float v) { return df_make(v, 0.f); }
__device__ __forceinline__ DF to_red(DF v) { return v; }
__device__ __forceinline__ double to_red(double v) { return v; }
__device__ __forceinline__ double red_double(DF v) { return (double)v; }
__device__ __forceinline__ double red_double(double v) { return v; }
__device__ __forceinline__ DF red_zero(DF) { return df_make(0.f, 0.f); }
__device__ __forceinline__ double red_zero(double) { return 0.0; }
// warp total in lane 0, fixed order, double-float on the FP32 pipes
__device__ __forceinline__ DF warp_sum_lane0(DF v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float th = __shfl_down_sync(0xffffffffu, v.hi, o);
    const float tl = __shfl_down_sync(0xffffffffu, v.lo, o);
    if (lane < o) v = v + df_make(th, tl);
  }
  return v;
}

// Deterministic grid reduction in two kernels.  A block holds RB groups of T
// threads (T a multiple of 32); group g works on right-hand side r = y*RB + g
// for the block's right-hand-side block y.  The producing kernel sums each
// group's values in a fixed order (double-float on the FP32 pipes, or IEEE FP64 for FP64
// arithmetic) and writes one IEEE-FP64 partial per block and right-hand side;
// nothing in it waits.  k_finish, launched next on the same stream (which
// orders the partial writes before it), sums each column's partials in a
// fixed order and runs the finalizer.  Results are bitwise reproducible.
// (A last-block-finishes scheme needs a fence and an arrival atomic in every
// block, whose round trips hold the block's SM slot: measured on GB300, that
// tail cost a 1M-site FP16 stencil about 25 us per launch.)
//
// `store` runs in every thread after the partials are written: a kernel
// writes its outputs there.  Every thread of the block must call this.
struct NoStore {
  __device__ void operator()() const {}
};
template <class V, class Store = NoStore>
__device__ __forceinline__ void reduce_block(const SysDesc& S, int T, int RB, int tile, int ntiles, V v,
                                             const RedArgs& ra, int by, Store store = Store()) {
  __shared__ V wpart[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  v = warp_sum_lane0(v);
  if (lane == 0) wpart[warp] = v;
  __syncthreads();
  if (tid < RB) {
    const int r = by * RB + tid;
    const int wpr = T >> 5;
    if (r < S.nrhs) {
      V s = wpart[tid * wpr];
      for (int w = 1; w < wpr; ++w) s = s + wpart[tid * wpr + w];
      ra.partial[S.part0 + r * ntiles + tile] = red_double(s);
    }
  }
  store();
}

// As reduce_block for a thread holding the values of NV consecutive right-hand
// sides, (by*RB + g)*NV + j for its group g and j < NV.
template <int NV, class V, class Store = NoStore>
__device__ __forceinline__ void reduce_block_n(const SysDesc& S, int T, int RB, int tile, int ntiles,
                                               const V (&v)[NV], const RedArgs& ra, int by, Store store = Store()) {
  __shared__ V wpart[NV][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const V w = warp_sum_lane0(v[j]);
    if (lane == 0) wpart[j][warp] = w;
  }
  __syncthreads();
  if (tid < RB * NV) {
    const int g = tid / NV, j = tid - g * NV;
    const int r = (by * RB + g) * NV + j;
    const int wpr = T >> 5;
    if (r < S.nrhs) {
      V s = wpart[j][g * wpr];
      for (int w = 1; w < wpr; ++w) s = s + wpart[j][g * wpr + w];
      ra.partial[S.part0 + r * ntiles + tile] = red_double(s);
    }
  }
  store();
}

// Finishing kernel: one block (kFinishThreads threads) per column (system,
// right-hand side).  Thread t sums partials t, t + kFinishThreads, ... in
// order (double-float), loading eight at a time so that their L2 round trips
// overlap, then a fixed warp tree and a fixed sum over warps; thread 0 runs
// the finalizer in IEEE FP64.  Columns whose kernel was gated off hold stale
// partials; the finalizer ignores them by the same state the gate tested
// (active, do_rel, xzero).
constexpr int kFinishThreads = 1024;
static __global__ void __launch_bounds__(kFinishThreads) k_finish(const __grid_constant__ Batch B, int par_mode,
                                                           RedArgs ra) {
  __shared__ DF wpart[kFinishThreads / 32];
  const int col = blockIdx.x;
  const int nrhs = B.sd[0].nrhs;
  const int si = col / nrhs, r = col - si * nrhs;
  const SysDesc& S = B.sd[si];
  const int ntiles = par_mode == 2 ? 2 * S.tpp : S.tpp;
  const double* p = ra.partial + S.part0 + (size_t)r * ntiles;
  DF v = df_make(0.f, 0.f);
  for (int i0 = threadIdx.x; i0 < ntiles; i0 += 8 * kFinishThreads) {
    double t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = i0 + j * kFinishThreads;
      t[j] = i < ntiles ? __ldcg(p + i) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) v = v + DF(t[j]);
  }
  v = warp_sum_lane0(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wpart[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    DF t = wpart[0];
    for (int w = 1; w < kFinishThreads / 32; ++w) t = t + wpart[w];
    finalize(ra, S.col0 + r, (double)t);
  }
}

// Cooperative copy of this block's system descriptor into shared memory.
__device__ __forceinline__ void load_desc(SysDesc& S, const SysDesc* __restrict__ sd, int si) {
  const int* src = reinterpret_cast<const int*>(sd + si);
  int* dst = reinterpret_cast<int*>(&S);
  for (int i = threadIdx.x; i < (int)(sizeof(SysDesc) / 4); i += blockDim.x) dst[i] = src[i];
}

}  // namespace dw

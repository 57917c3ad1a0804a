// dw_kernels.cuh -- the hopping-term stencil and the CG vector kernels.
//
// Hopping term (the sum in D = 1 - kappa*H):
//   (H psi)(x) = sum_mu [ (1 - gamma_mu) eta U_mu(x) psi(x+mu)
//                       + (1 + gamma_mu) eta U_mu(x-mu)^dag psi(x-mu) ]
// and for D^dag the two projectors swap.  Per output site and direction the
// kernel spin-projects the neighbour to a half spinor (2 spins x 3 colours),
// multiplies by the link or its adjoint, and reconstructs the lower two spins
// (the four stages of the paper's Fig. 1: load, linear combination, 3x3
// mat-vec, accumulate).  One thread per (output site, right-hand side);
// threads of a warp take consecutive even-odd site indices so every load is
// a coalesced 16-byte (or 8-byte) access.  The boundary sign eta (-1 on links
// crossing t = Lt-1 -> 0 when antiperiodic) is applied in the kernel, so
// links stay SU(3) and 12-real compression stays valid.
//
// Gamma basis (chiral): gamma_mu = [[0, B_mu], [B_mu^dag, 0]] with
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.  Then
//   (1 + s gamma_mu) psi = [ h ; s B^dag h ],  h = psi_up + s B psi_down.
#pragma once

#include <type_traits>

#include "dw_common.cuh"

namespace dw {

enum Coef { C_ONE = 0, C_MK, C_PK, C_MK2, C_PK2 };
// Stencil operator: the Wilson hopping term H, or the spin-diagonal covariant
// hopping term K = sum_mu [U_mu(x) delta_{x+mu} + U_mu(x-mu)^dag delta_{x-mu}]
// of the Laplacian 1 - kappa K (Hermitian: no dagger form).
enum Op { OP_WILSON = 0, OP_LAPLACE = 1 };
enum Gate { G_ACTIVE = 0, G_REL, G_ALL, G_XZERO, G_ZSRC };

template <int C>
__device__ __forceinline__ double coef_of(double kappa) {
  return C == C_ONE ? 1.0 : C == C_MK ? -kappa : C == C_PK ? kappa : C == C_MK2 ? -kappa * kappa : kappa * kappa;
}
// The coefficient in the arithmetic type R, from the system's pre-rounded
// kappa (FP32 and double-float) so that no thread converts from FP64.
template <int C, typename R>
__device__ __forceinline__ R coef(const SysDesc& S) {
  if constexpr (std::is_same<R, double>::value) {
    return coef_of<C>(S.kappa);
  } else if constexpr (std::is_same<R, float>::value) {
    return C == C_ONE ? 1.f : C == C_MK ? -S.kappa_f : C == C_PK ? S.kappa_f : C == C_MK2 ? -S.kappa2_f : S.kappa2_f;
  } else {
    const DF k = df_make(S.kappa_f, S.kappa_lo), k2 = df_make(S.kappa2_f, S.kappa2_lo);
    return C == C_ONE ? DF(1) : C == C_MK ? -k : C == C_PK ? k : C == C_MK2 ? -k2 : k2;
  }
}
// A CG scalar (alpha, beta) in the arithmetic type R: the finalizer's FP32
// rounding for FP32, the FP64 value split exactly for double-float.
template <typename R>
__device__ __forceinline__ R scalar_as(double v, float vf) {
  if constexpr (std::is_same<R, double>::value) return v;
  else if constexpr (std::is_same<R, float>::value) return vf;
  else return DF(v);
}

__device__ __forceinline__ int gate_of(int g, const ColState* cols, int col) {
  if (g == G_ALL) return 1;
  if (g == G_XZERO) return cols[col].xzero;
  if (g == G_ZSRC) return cols[col].zsrc;
  return g == G_ACTIVE ? cols[col].active : cols[col].do_rel;
}

// a + S*b,  S = +1 or -1 (compile time)
template <int S, typename R>
__device__ __forceinline__ Cx<R> pm(Cx<R> a, Cx<R> b) { return S > 0 ? a + b : a - b; }

// half spinor of (1 + S gamma_mu) psi
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const Cx<R> (&p)[12], Cx<R> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {        // h0 = p0 - S i p3, h1 = p1 - S i p2
      h[c] = pm<-S>(p[c], mul_i(p[9 + c]));
      h[3 + c] = pm<-S>(p[3 + c], mul_i(p[6 + c]));
    } else if (MU == 1) { // h0 = p0 - S p3, h1 = p1 + S p2
      h[c] = pm<-S>(p[c], p[9 + c]);
      h[3 + c] = pm<S>(p[3 + c], p[6 + c]);
    } else if (MU == 2) { // h0 = p0 - S i p2, h1 = p1 + S i p3
      h[c] = pm<-S>(p[c], mul_i(p[6 + c]));
      h[3 + c] = pm<S>(p[3 + c], mul_i(p[9 + c]));
    } else {              // h0 = p0 + S p2, h1 = p1 + S p3
      h[c] = pm<S>(p[c], p[6 + c]);
      h[3 + c] = pm<S>(p[3 + c], p[9 + c]);
    }
  }
}

// acc += (1 + S gamma_mu) reconstructed from the multiplied half spinor g
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate(Cx<R> (&acc)[12], const Cx<R> (&g)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = acc[c] + g[c];
    acc[3 + c] = acc[3 + c] + g[3 + c];
    if (MU == 0) {        // lower = S i (g1, g0)
      acc[6 + c] = pm<S>(acc[6 + c], mul_i(g[3 + c]));
      acc[9 + c] = pm<S>(acc[9 + c], mul_i(g[c]));
    } else if (MU == 1) { // lower = S (g1, -g0)
      acc[6 + c] = pm<S>(acc[6 + c], g[3 + c]);
      acc[9 + c] = pm<-S>(acc[9 + c], g[c]);
    } else if (MU == 2) { // lower = S i (g0, -g1)
      acc[6 + c] = pm<S>(acc[6 + c], mul_i(g[c]));
      acc[9 + c] = pm<-S>(acc[9 + c], mul_i(g[3 + c]));
    } else {              // lower = S (g0, g1)
      acc[6 + c] = pm<S>(acc[6 + c], g[c]);
      acc[9 + c] = pm<S>(acc[9 + c], g[3 + c]);
    }
  }
}

// acc + w * g  (w real), componentwise FMA
template <typename R>
__device__ __forceinline__ Cx<R> cfma(R w, Cx<R> g, Cx<R> acc) { return cx(fma(w, g.re, acc.re), fma(w, g.im, acc.im)); }

// acc += w (1 + S gamma_mu) reconstructed from g, w = dequantisation scale times
// the boundary sign (the 16-bit inputs are projected and multiplied unscaled)
template <int MU, int S, typename R>
__device__ __forceinline__ void accumulate_w(Cx<R> (&acc)[12], const Cx<R> (&g)[6], R w) {
  const R ws = S > 0 ? w : -w;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = cfma(w, g[c], acc[c]);
    acc[3 + c] = cfma(w, g[3 + c], acc[3 + c]);
    if (MU == 0) {        // lower = S i (g1, g0)
      acc[6 + c] = cfma(ws, mul_i(g[3 + c]), acc[6 + c]);
      acc[9 + c] = cfma(ws, mul_i(g[c]), acc[9 + c]);
    } else if (MU == 1) { // lower = S (g1, -g0)
      acc[6 + c] = cfma(ws, g[3 + c], acc[6 + c]);
      acc[9 + c] = cfma(-ws, g[c], acc[9 + c]);
    } else if (MU == 2) { // lower = S i (g0, -g1)
      acc[6 + c] = cfma(ws, mul_i(g[c]), acc[6 + c]);
      acc[9 + c] = cfma(-ws, mul_i(g[3 + c]), acc[9 + c]);
    } else {              // lower = S (g0, g1)
      acc[6 + c] = cfma(ws, g[c], acc[6 + c]);
      acc[9 + c] = cfma(ws, g[3 + c], acc[9 + c]);
    }
  }
}

// g = U h (ADJ = false) or U^dag h (ADJ = true), on both half-spinor spins
template <bool ADJ, typename R>
__device__ __forceinline__ void su3_mul(const Cx<R> (&u)[9], const Cx<R> (&h)[6], Cx<R> (&g)[6]) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!ADJ) {
        Cx<R> t = cmul(u[a * 3 + 0], h[3 * k + 0]);
        t = cmadd(u[a * 3 + 1], h[3 * k + 1], t);
        g[3 * k + a] = cmadd(u[a * 3 + 2], h[3 * k + 2], t);
      } else {
        Cx<R> t = cjmul(u[0 * 3 + a], h[3 * k + 0]);
        t = cjmadd(u[1 * 3 + a], h[3 * k + 1], t);
        g[3 * k + a] = cjmadd(u[2 * 3 + a], h[3 * k + 2], t);
      }
    }
}

// 16-bit operand forms.  The projection runs on packed 16-bit lanes (one
// extra rounding to 16 bits per half-spinor component); the mat-vec takes the
// stored 16-bit link and half-spinor components directly into FP32-accumulating
// fused multiply-adds, so no component is converted to FP32 first.
template <int MU, int S, int P>
__device__ __forceinline__ void project_w(const uint32_t (&p)[12], uint32_t (&h)[6]) {
  using W = HW<P>;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) {        // h0 = p0 - S i p3, h1 = p1 - S i p2
      h[c] = W::template rot_add<-S>(p[c], p[9 + c]);
      h[3 + c] = W::template rot_add<-S>(p[3 + c], p[6 + c]);
    } else if (MU == 1) { // h0 = p0 - S p3, h1 = p1 + S p2
      h[c] = S > 0 ? W::sub(p[c], p[9 + c]) : W::add(p[c], p[9 + c]);
      h[3 + c] = S > 0 ? W::add(p[3 + c], p[6 + c]) : W::sub(p[3 + c], p[6 + c]);
    } else if (MU == 2) { // h0 = p0 - S i p2, h1 = p1 + S i p3
      h[c] = W::template rot_add<-S>(p[c], p[6 + c]);
      h[3 + c] = W::template rot_add<S>(p[3 + c], p[9 + c]);
    } else {              // h0 = p0 + S p2, h1 = p1 + S p3
      h[c] = S > 0 ? W::add(p[c], p[6 + c]) : W::sub(p[c], p[6 + c]);
      h[3 + c] = S > 0 ? W::add(p[3 + c], p[9 + c]) : W::sub(p[3 + c], p[9 + c]);
    }
  }
}

template <bool ADJ, int P>
__device__ __forceinline__ void su3_mul_w(const uint32_t (&u)[9], const uint32_t (&h)[6], Cx<float> (&g)[6]) {
  uint32_t hx[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) hx[k] = h[k] ^ (ADJ ? kNegRe : kNegIm);
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (ADJ) HW<P>::cmac_adj(re, im, u[b * 3 + a], h[3 * k + b], hx[3 * k + b]);
        else HW<P>::cmac(re, im, u[a * 3 + b], h[3 * k + b], hx[3 * k + b]);
      }
      g[3 * k + a] = cx(re, im);
    }
}

// Double-float version: each real output is one 6-term dot product.  The two
// spin rows of the half spinor are the two lanes of packed FP32x2 arithmetic,
// so each packed dot product yields one real output for both rows.
#ifndef DW_DF_PACKED
#define DW_DF_PACKED 1
#endif
#if DW_DF_PACKED
template <bool ADJ>
__device__ __forceinline__ void su3_mul(const Cx<DF> (&u)[9], const Cx<DF> (&h)[6], Cx<DF> (&g)[6]) {
  DF2 hr[3], hi[3], hrn[3], hin[3];  // rows k = 0, 1 in the lanes; n: negated
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    hr[b].hi = make_float2(h[b].re.hi, h[3 + b].re.hi);
    hr[b].lo = make_float2(h[b].re.lo, h[3 + b].re.lo);
    hi[b].hi = make_float2(h[b].im.hi, h[3 + b].im.hi);
    hi[b].lo = make_float2(h[b].im.lo, h[3 + b].im.lo);
    hrn[b].hi = make_float2(-hr[b].hi.x, -hr[b].hi.y);
    hrn[b].lo = make_float2(-hr[b].lo.x, -hr[b].lo.y);
    hin[b].hi = make_float2(-hi[b].hi.x, -hi[b].hi.y);
    hin[b].lo = make_float2(-hi[b].lo.x, -hi[b].lo.y);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    DF xr[6], xi[6];
    DF2 yr[6], yi[6];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Cx<DF> m = ADJ ? u[b * 3 + a] : u[a * 3 + b];
      // re = m.re h.re -/+ m.im h.im ; im = m.re h.im +/- m.im h.re  (lower sign: adjoint)
      xr[2 * b] = m.re;
      yr[2 * b] = hr[b];
      xr[2 * b + 1] = m.im;
      yr[2 * b + 1] = ADJ ? hi[b] : hin[b];
      xi[2 * b] = m.re;
      yi[2 * b] = hi[b];
      xi[2 * b + 1] = m.im;
      yi[2 * b + 1] = ADJ ? hrn[b] : hr[b];
    }
    const DF2 re = df2_dot6(xr, yr), im = df2_dot6(xi, yi);
    g[a].re = df_make(re.hi.x, re.lo.x);
    g[a].im = df_make(im.hi.x, im.lo.x);
    g[3 + a].re = df_make(re.hi.y, re.lo.y);
    g[3 + a].im = df_make(im.hi.y, im.lo.y);
  }
}
#else
template <bool ADJ>
__device__ __forceinline__ void su3_mul(const Cx<DF> (&u)[9], const Cx<DF> (&h)[6], Cx<DF> (&g)[6]) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      DF xr[6], yr[6], xi[6], yi[6];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const Cx<DF> m = ADJ ? u[b * 3 + a] : u[a * 3 + b];
        const Cx<DF> v = h[3 * k + b];
        // re = m.re v.re -/+ m.im v.im ; im = m.re v.im +/- m.im v.re  (lower sign: adjoint)
        xr[2 * b] = m.re;
        yr[2 * b] = v.re;
        xr[2 * b + 1] = ADJ ? m.im : -m.im;
        yr[2 * b + 1] = v.im;
        xi[2 * b] = m.re;
        yi[2 * b] = v.im;
        xi[2 * b + 1] = ADJ ? -m.im : m.im;
        yi[2 * b + 1] = v.re;
      }
      g[3 * k + a].re = df_dot6(xr, yr);
      g[3 * k + a].im = df_dot6(xi, yi);
    }
}
#endif

// Runtime-direction form of the spin projection and reconstruction, used by
// the double-float stencil whose unrolled body would not fit the instruction
// cache.  For (1 + s gamma_mu):  h0 = p0 + c0 q0,  h1 = p1 + c1 q1 with
// (q0, q1) = (p3, p2) for mu = x, y and (p2, p3) for mu = z, t; the lower spins
// are d2 (g1 or g0) and d3 (g0 or g1) with the same pairing.  Every factor is
// +-1 or +-i:
//   mu = x: c0 = c1 = -s i;   d2 = d3 = s i
//   mu = y: c0 = -s, c1 = s;  d2 = s, d3 = -s
//   mu = z: c0 = -s i, c1 = s i; d2 = s i, d3 = -s i
//   mu = t: c0 = c1 = s;      d2 = d3 = s
struct UnitFactor {
  bool imag;   // multiply by i
  bool neg;    // then by -1
};
template <typename R>
__device__ __forceinline__ Cx<R> mul_unit(Cx<R> q, UnitFactor f) {
  Cx<R> r = f.imag ? cx(-q.im, q.re) : q;
  return f.neg ? cx(-r.re, -r.im) : r;
}
struct DirSpin {
  bool swap;  // pair spin 0 with spin 3 (x, y)
  UnitFactor c0, c1, d2, d3;
};
__device__ __forceinline__ DirSpin dir_spin(int mu, int s) {
  DirSpin d;
  const bool neg_s = s < 0;
  d.swap = mu <= 1;
  const bool im = (mu == 0 || mu == 2);
  d.c0 = UnitFactor{im, mu == 3 ? neg_s : !neg_s};
  d.c1 = UnitFactor{im, mu == 0 ? !neg_s : neg_s};
  d.d2 = UnitFactor{im, neg_s};
  d.d3 = UnitFactor{im, (mu == 1 || mu == 2) ? !neg_s : neg_s};
  return d;
}
// complex sums for the double-float path: lazy (no renormalisation)
__device__ __forceinline__ Cx<DF> cadd_lazy(Cx<DF> a, Cx<DF> b) { return cx(add_lazy(a.re, b.re), add_lazy(a.im, b.im)); }
template <typename R>
__device__ __forceinline__ void project_rt(const DirSpin& d, const Cx<R> (&p)[12], Cx<R> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<R> q0 = d.swap ? p[9 + c] : p[6 + c];
    const Cx<R> q1 = d.swap ? p[6 + c] : p[9 + c];
    h[c] = cadd_lazy(p[c], mul_unit(q0, d.c0));
    h[3 + c] = cadd_lazy(p[3 + c], mul_unit(q1, d.c1));
  }
}
// The same projection from a double-float field, loading for each half-spinor
// row only the two spins it combines, so that six of the twelve components
// are live at a time.
template <class In>
__device__ __forceinline__ void project_rt_loaded(const DirSpin& d, const In& in, const SysDesc& S, int par, int r,
                                                  int n, Cx<DF> (&h)[6]) {
  const char* base = slot_ptr(S, in.slot, r, par);
  Cx<DF> a[3], q[3];
  Spin<PDF>::load_spin(base, S.vh, n, 0, a);
  Spin<PDF>::load_spin(base, S.vh, n, d.swap ? 3 : 2, q);
#pragma unroll
  for (int c = 0; c < 3; ++c) h[c] = cadd_lazy(a[c], mul_unit(q[c], d.c0));
  Spin<PDF>::load_spin(base, S.vh, n, 1, a);
  Spin<PDF>::load_spin(base, S.vh, n, d.swap ? 2 : 3, q);
#pragma unroll
  for (int c = 0; c < 3; ++c) h[3 + c] = cadd_lazy(a[c], mul_unit(q[c], d.c1));
}
// acc stays unnormalised across the eight directions (renormalised by the caller)
template <typename R>
__device__ __forceinline__ void accumulate_rt(const DirSpin& d, Cx<R> (&acc)[12], const Cx<R> (&g)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = cadd_lazy(acc[c], g[c]);
    acc[3 + c] = cadd_lazy(acc[3 + c], g[3 + c]);
    const Cx<R> g2 = d.swap ? g[3 + c] : g[c];
    const Cx<R> g3 = d.swap ? g[c] : g[3 + c];
    acc[6 + c] = cadd_lazy(acc[6 + c], mul_unit(g2, d.d2));
    acc[9 + c] = cadd_lazy(acc[9 + c], mul_unit(g3, d.d3));
  }
}

// Site coordinates of even-odd index s on parity par.
struct Coord {
  int xh, x, y, z, t, row;  // row = s - xh (start of the x-row in eo indexing)
};

__device__ __forceinline__ Coord coord_of(const SysDesc& S, int s, int par) {
  Coord c;
  int q = fdiv(s, S.div_lxh);
  c.xh = s - q * S.lxh;
  c.row = s - c.xh;
  int q2 = fdiv(q, S.div_ly);
  c.y = q - q2 * S.ly;
  c.t = fdiv(q2, S.div_lz);
  c.z = q2 - c.t * S.lz;
  c.x = 2 * c.xh + ((c.y + c.z + c.t + par) & 1);
  return c;
}

// eo index of the neighbour one step in direction MU (DIR = +1/-1); *eta is
// the boundary sign of the link crossed.
template <int MU, int DIR>
__device__ __forceinline__ int neighbour(const SysDesc& S, const Coord& c, int s, float* eta) {
  *eta = 1.f;
  if (MU == 0) {
    const int lx = 2 * S.lxh;
    int xn = c.x + DIR;
    xn = xn == lx ? 0 : (xn < 0 ? lx - 1 : xn);
    return (xn >> 1) + c.row;
  } else if (MU == 1) {
    const int st = S.lxh;
    if (DIR > 0) return c.y == S.ly - 1 ? s - (S.ly - 1) * st : s + st;
    return c.y == 0 ? s + (S.ly - 1) * st : s - st;
  } else if (MU == 2) {
    const int st = S.lxh * S.ly;
    if (DIR > 0) return c.z == S.lz - 1 ? s - (S.lz - 1) * st : s + st;
    return c.z == 0 ? s + (S.lz - 1) * st : s - st;
  } else {
    const int st = S.lxh * S.ly * S.lz;
    if (DIR > 0) {
      if (c.t == S.lt - 1) {
        if (S.anti_t) *eta = -1.f;
        return s - (S.lt - 1) * st;
      }
      return s + st;
    }
    if (c.t == 0) {
      if (S.anti_t) *eta = -1.f;
      return s + (S.lt - 1) * st;
    }
    return s - st;
  }
}

__device__ __forceinline__ int neighbour_rt(const SysDesc& S, const Coord& c, int s, int mu, int dir, float* eta) {
  switch (mu) {
    case 0: return dir > 0 ? neighbour<0, +1>(S, c, s, eta) : neighbour<0, -1>(S, c, s, eta);
    case 1: return dir > 0 ? neighbour<1, +1>(S, c, s, eta) : neighbour<1, -1>(S, c, s, eta);
    case 2: return dir > 0 ? neighbour<2, +1>(S, c, s, eta) : neighbour<2, -1>(S, c, s, eta);
    default: return dir > 0 ? neighbour<3, +1>(S, c, s, eta) : neighbour<3, -1>(S, c, s, eta);
  }
}

__device__ __forceinline__ const char* slot_ptr(const SysDesc& S, int slot, int r, int par) {
  const Slot& f = S.f[slot];
  return f.p + r * f.rhs_stride + par * f.par_stride;
}
__device__ __forceinline__ char* slot_wptr(const SysDesc& S, int slot, int r, int par) {
  const Slot& f = S.f[slot];
  return f.p + r * f.rhs_stride + par * f.par_stride;
}

template <typename R, typename Q>
__device__ __forceinline__ void convert12(const Cx<Q> (&a)[12], Cx<R> (&b)[12]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) b[k] = cx((R)a[k].re, (R)a[k].im);
}

// ------------------------------------------------------------------ input loaders
// Neighbour spinor from one field.
template <int SP>
struct InOne {
  int slot;
  static constexpr bool kScaled = Spin<SP>::kScaled;
  __host__ double io_bytes() const { return Spin<SP>::kBytes; }
  template <typename R>
  __device__ __forceinline__ void load(const SysDesc& S, int par, int r, int s, Cx<R> (&v)[12]) const {
    Cx<typename Spin<SP>::R> t[12];
    Spin<SP>::load(slot_ptr(S, slot, r, par), S.vh, s, t);
    convert12(t, v);
  }
  // 16-bit storage: stored words and the site scale
  __device__ __forceinline__ void load_words(const SysDesc& S, int par, int r, int s, uint32_t (&w)[12],
                                             float& sc) const {
    Spin<SP>::load_words(slot_ptr(S, slot, r, par), S.vh, s, w, sc);
  }
  // 16-bit storage: unscaled values and the site scale
  template <typename R>
  __device__ __forceinline__ void load_raw(const SysDesc& S, int par, int r, int s, Cx<R> (&v)[12], R& sc) const {
    if constexpr (Spin<SP>::kScaled) {
      Spin<SP>::load_raw(slot_ptr(S, slot, r, par), S.vh, s, v, sc);
    } else {
      load(S, par, r, s, v);
      sc = (R)1;
    }
  }
};

// ------------------------------------------------------------------ epilogues
// write(): forms and stores the output of one site.  Reducing epilogues with
// kSplit also offer prepare() (forms the stored words and the reduced value)
// and commit() (stores them), so that the kernel can publish its block's
// partial sum before the output stores.
// out = coef * H in
template <int SPO, int COEF>
struct EpiOut {
  static constexpr bool kReduce = false;
  static constexpr bool kSplit = false;
  using Packed = int;
  int slot_out;
  int gate;
  __host__ double io_bytes() const { return Spin<SPO>::kBytes; }
  template <typename R, typename V>
  __device__ __forceinline__ void write(const SysDesc& S, int par, int r, int s, Cx<R> (&acc)[12], V&) const {
    using RO = typename Spin<SPO>::R;
    const R c = coef<COEF, R>(S);
    Cx<RO> o[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = cx((RO)(c * acc[k].re), (RO)(c * acc[k].im));
    Spin<SPO>::store(slot_wptr(S, slot_out, r, par), S.vh, s, o);
  }
};

// out = X + coef * H in  (X on the output parity), optional |out|^2 reduction.
// slot_out < 0: nothing stored (norm only).
template <int SPO, int SPX, int COEF, bool RED>
struct EpiXpay {
  static constexpr bool kReduce = RED;
  static constexpr bool kSplit = RED;
  using Packed = typename Spin<SPO>::Packed;
  int slot_out, slot_x;
  int gate;
  __host__ double io_bytes() const { return Spin<SPX>::kBytes + (slot_out >= 0 ? Spin<SPO>::kBytes : 0); }
  template <typename R>
  __device__ __forceinline__ Packed prepare(const SysDesc& S, int par, int r, int s, Cx<R> (&acc)[12],
                                            typename RedT<R>::type& nrm) const {
    using RO = typename Spin<SPO>::R;
    Cx<typename Spin<SPX>::R> xv[12];
    Spin<SPX>::load(slot_ptr(S, slot_x, r, par), S.vh, s, xv);
    const R c = coef<COEF, R>(S);
    Cx<RO> o[12];
    R n = (R)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      R re = fma(c, acc[k].re, (R)xv[k].re), im = fma(c, acc[k].im, (R)xv[k].im);
      o[k] = cx((RO)re, (RO)im);
      n = fma(re, re, fma(im, im, n));
    }
    nrm = to_red(n);
    return Spin<SPO>::pack(o);
  }
  __device__ __forceinline__ void commit(const SysDesc& S, int par, int r, int s, const Packed& o) const {
    if (slot_out >= 0) Spin<SPO>::store_packed(slot_wptr(S, slot_out, r, par), S.vh, s, o);
  }
  template <typename R>
  __device__ __forceinline__ void write(const SysDesc& S, int par, int r, int s, Cx<R> (&acc)[12],
                                        typename RedT<R>::type& nrm) const {
    const Packed o = prepare(S, par, r, s, acc, nrm);
    commit(S, par, r, s, o);
  }
};

// out = x + c*acc with the reduction Re <x, out> (the CG's p^dag A p for a
// Hermitian operator, x = p).
template <int SPO, int SPX, int COEF>
struct EpiXpayDot {
  static constexpr bool kReduce = true;
  static constexpr bool kSplit = true;
  using Packed = typename Spin<SPO>::Packed;
  int slot_out, slot_x;
  int gate;
  __host__ double io_bytes() const { return Spin<SPX>::kBytes + Spin<SPO>::kBytes; }
  __device__ __forceinline__ void commit(const SysDesc& S, int par, int r, int s, const Packed& o) const {
    Spin<SPO>::store_packed(slot_wptr(S, slot_out, r, par), S.vh, s, o);
  }
  template <typename R>
  __device__ __forceinline__ void write(const SysDesc& S, int par, int r, int s, Cx<R> (&acc)[12], double& nrm) const {
    commit(S, par, r, s, prepare(S, par, r, s, acc, nrm));
  }
  template <typename R>
  __device__ __forceinline__ Packed prepare(const SysDesc& S, int par, int r, int s, Cx<R> (&acc)[12],
                                            typename RedT<R>::type& nrm) const {
    using RO = typename Spin<SPO>::R;
    Cx<typename Spin<SPX>::R> xv[12];
    Spin<SPX>::load(slot_ptr(S, slot_x, r, par), S.vh, s, xv);
    const R c = coef<COEF, R>(S);
    Cx<RO> o[12];
    R n = (R)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R xr = (R)xv[k].re, xi = (R)xv[k].im;
      const R re = fma(c, acc[k].re, xr), im = fma(c, acc[k].im, xi);
      o[k] = cx((RO)re, (RO)im);
      n = fma(xr, re, fma(xi, im, n));
    }
    nrm = to_red(n);
    return Spin<SPO>::pack(o);
  }
};

// Residual of the even-odd system in the high precision SPH at even site s,
// once the accumulator x has absorbed the low-precision increment:
//   r_hi = bh - x + kappa^2 * acc  (acc = H_eo t, t = H_oe x);  r_low <- r_hi;
//   reduction |r_hi|^2.  r_hi itself is not stored: the iteration continues
//   from r_low, and the next correction recomputes r_hi.
template <int SPL, int SPH>
struct EpiResidEO {
  static constexpr bool kReduce = true;
  static constexpr bool kSplit = false;
  using Packed = int;
  int gate;
  __host__ double io_bytes() const { return 2.0 * Spin<SPH>::kBytes + Spin<SPL>::kBytes; }
  template <typename RH>
  __device__ __forceinline__ void write(const SysDesc& S, int par, int r, int s, Cx<RH> (&acc)[12],
                                        typename RedT<RH>::type& nrm) const {
    Cx<RH> x[12], bh[12], rv[12];
    Spin<SPH>::load(slot_ptr(S, S_X, r, par), S.vh, s, x);
    Spin<SPH>::load(slot_ptr(S, S_BH, r, par), S.vh, s, bh);
    const RH k2 = coef<C_PK2, RH>(S);
    RH n = (RH)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k] = cx(fma(k2, acc[k].re, bh[k].re - x[k].re), fma(k2, acc[k].im, bh[k].im - x[k].im));
      n = fma(rv[k].re, rv[k].re, fma(rv[k].im, rv[k].im, n));
    }
    nrm = to_red(n);
    Cx<typename Spin<SPL>::R> lo[12];
    convert12(rv, lo);
    Spin<SPL>::store(slot_wptr(S, S_R, r, par), S.vh, s, lo);
  }
};

// Full-lattice residual rt = b - (x - kappa*acc) on the output parity (with
// acc = H x this is b - D x; with acc = Hdag x it is b - D^dag x), in the
// precision SPH of x, b and rt, optionally also r_low <- rt.  Reduction |rt|^2.
template <int SPL, bool STORE_LOW, int SPH>
struct EpiResidFull {
  static constexpr bool kReduce = true;
  static constexpr bool kSplit = false;
  using Packed = int;
  int gate;
  int slot_rt;  // < 0: norm only
  int slot_x;
  int slot_b;
  __host__ double io_bytes() const {
    return 2.0 * Spin<SPH>::kBytes + (slot_rt >= 0 ? Spin<SPH>::kBytes : 0) + (STORE_LOW ? Spin<SPL>::kBytes : 0);
  }
  template <typename RH>
  __device__ __forceinline__ void write(const SysDesc& S, int par, int r, int s, Cx<RH> (&acc)[12],
                                        typename RedT<RH>::type& nrm) const {
    Cx<RH> x[12], b[12], rv[12];
    Spin<SPH>::load(slot_ptr(S, slot_x, r, par), S.vh, s, x);
    Spin<SPH>::load(slot_ptr(S, slot_b, r, par), S.vh, s, b);
    const RH kap = coef<C_PK, RH>(S);
    RH n = (RH)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k] = cx(fma(kap, acc[k].re, b[k].re - x[k].re), fma(kap, acc[k].im, b[k].im - x[k].im));
      n = fma(rv[k].re, rv[k].re, fma(rv[k].im, rv[k].im, n));
    }
    nrm = to_red(n);
    if (slot_rt >= 0) Spin<SPH>::store(slot_wptr(S, slot_rt, r, par), S.vh, s, rv);
    if (STORE_LOW) {
      Cx<typename Spin<SPL>::R> lo[12];
      convert12(rv, lo);
      Spin<SPL>::store(slot_wptr(S, S_R, r, par), S.vh, s, lo);
    }
  }
};

// ------------------------------------------------------------------ block prologue
// System descriptor into shared memory, the gate of every column of the
// system, this thread's site s on output parity par and right-hand side r.
// A block returns at once only when every column of its system is gated off:
// all blocks of a system read the same gates (they change only in the
// system's last block, after every block has read them), so either all of a
// system's blocks arrive at the reduction or none does.
#define DW_BLOCK_PROLOGUE(GATE)                                            \
  __shared__ SysDesc S;                                                    \
  __shared__ int act[64];                                                  \
  const int T = B.T, RB = B.RB;                                            \
  /* the right-hand-side block varies fastest: the blocks of one tile run  \
     together and share its links and neighbours in L2 */                  \
  const unsigned bx_ = B.rev ? gridDim.x - 1u - blockIdx.x : blockIdx.x;   \
  const int by = (int)(bx_ % (unsigned)B.ny);                              \
  int b = (int)(bx_ / (unsigned)B.ny), par;                                \
  if (par_mode == 2) {                                                     \
    par = b >= B.ntot ? 1 : 0;                                             \
    b -= par * B.ntot;                                                     \
  } else {                                                                 \
    par = par_mode;                                                        \
  }                                                                        \
  load_desc(S, B.sd, block_system(B, b));                                  \
  __syncthreads();                                                         \
  for (int i_ = threadIdx.x; i_ < S.nrhs; i_ += blockDim.x)                \
    act[i_] = gate_of(GATE, ra.cols, S.col0 + i_);                         \
  __syncthreads();                                                         \
  int any = 0;                                                             \
  for (int i_ = 0; i_ < S.nrhs; ++i_) any |= act[i_];                      \
  if (!any) return;                                                        \
  const int rl = threadIdx.x / T;                                          \
  const int r = by * RB + rl;                                              \
  const int tile = b - S.tile0;                                            \
  const int s = tile * T + (threadIdx.x - rl * T);                         \
  const bool valid = s < S.vh && r < S.nrhs && act[r < S.nrhs ? r : 0];

#define DW_BLOCK_REDUCE(val)                                               \
  {                                                                        \
    const int ntiles = par_mode == 2 ? 2 * S.tpp : S.tpp;                  \
    const int tt = par_mode == 2 ? par * S.tpp + tile : tile;              \
    reduce_block(S, T, RB, tt, ntiles, val, ra, by);               \
  }
// As DW_BLOCK_REDUCE, with the output stores STORE (a lambda) run after the
// block's partial sums are written.
#define DW_BLOCK_REDUCE_STORE(val, STORE)                                  \
  {                                                                        \
    const int ntiles = par_mode == 2 ? 2 * S.tpp : S.tpp;                  \
    const int tt = par_mode == 2 ? par * S.tpp + tile : tile;              \
    reduce_block(S, T, RB, tt, ntiles, val, ra, by, STORE);        \
  }

// ------------------------------------------------------------------ the Laplacian's directions
// acc = K psi at output site s: the neighbour's whole spinor (no projection)
// times U_mu(x) or U_mu(x-mu)^dag, spin by spin, with the boundary sign.
template <int SPA, int LP, bool C12, class In, typename R>
__device__ __forceinline__ void laplace_dirs(const SysDesc& S, const In& in, const Coord& c, int s, int r, int pin,
                                             const char* ulink_own, const char* ulink_nb, long long mu_stride,
                                             Cx<R> (&acc)[12]) {
  // FP32 and 16-bit: all eight directions unrolled (compile-time neighbour
  // arithmetic); double-float and FP64 keep one copy of the loop body, whose
  // unrolled form would not fit the instruction cache
  constexpr int kUnroll = (SPA == PDF || SPA == P64) ? 1 : 8;
#pragma unroll kUnroll
  for (int d = 0; d < 8; ++d) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    float eta;
    const int n = neighbour_rt(S, c, s, mu, fwd ? +1 : -1, &eta);
    const char* lb = (fwd ? ulink_own : ulink_nb) + mu * mu_stride;
    const int li = fwd ? s : n;
    if constexpr (SPA == P16 || SPA == PB16) {
      uint32_t pw[12], h0[6], h1[6], u[9];
      float sc;
      Cx<float> g0[6], g1[6];
      in.load_words(S, pin, r, n, pw, sc);
      Link<LP, C12>::load_words(lb, S.vh, li, u);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        h0[k] = pw[k];
        h1[k] = pw[6 + k];
      }
      if (fwd) {
        su3_mul_w<false, SPA>(u, h0, g0);
        su3_mul_w<false, SPA>(u, h1, g1);
      } else {
        su3_mul_w<true, SPA>(u, h0, g0);
        su3_mul_w<true, SPA>(u, h1, g1);
      }
      const float w = eta < 0.f ? -sc : sc;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        acc[k] = cfma(w, g0[k], acc[k]);
        acc[6 + k] = cfma(w, g1[k], acc[6 + k]);
      }
    } else {
      Cx<R> p[12], h0[6], h1[6], g0[6], g1[6], u[9];
      in.load(S, pin, r, n, p);
      Link<LP, C12>::load(lb, S.vh, li, u);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        h0[k] = p[k];
        h1[k] = p[6 + k];
      }
      if (eta < 0.f) {  // boundary sign: taken only on the t-boundary slice
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          h0[k] = cx(-h0[k].re, -h0[k].im);
          h1[k] = cx(-h1[k].re, -h1[k].im);
        }
      }
      if (fwd) {
        su3_mul<false>(u, h0, g0);
        su3_mul<false>(u, h1, g1);
      } else {
        su3_mul<true>(u, h0, g0);
        su3_mul<true>(u, h1, g1);
      }
      // double-float: sums left unnormalised, renormalised once after the
      // eight directions (as the Wilson stencil's accumulation)
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if constexpr (std::is_same<R, DF>::value) {
          acc[k] = cadd_lazy(acc[k], g0[k]);
          acc[6 + k] = cadd_lazy(acc[6 + k], g1[k]);
        } else {
          acc[k] = acc[k] + g0[k];
          acc[6 + k] = acc[6 + k] + g1[k];
        }
      }
    }
  }
}

// ------------------------------------------------------------------ the stencil kernel
// par_mode 0/1: output parity fixed, grid = ntot blocks.  par_mode 2: both
// parities, grid = 2*ntot (block b >= ntot works on odd output sites).
// Input is read on the opposite parity.  SPA: arithmetic-precision tag.
// Minimum resident blocks (of 256 threads) per SM requested from the compiler.
// Measured on GB300: capping the double-float stencil at 128 registers (2)
// runs 9% faster despite small spills (more warps to hide its long dependency
// chains); the 16-bit stencils, whose operands stay in packed 16-bit words,
// fit 80 registers without spills (3) and run 5% faster there than at 128.
#ifndef DW_HOP16_MINB
#define DW_HOP16_MINB 3
#endif
#ifndef DW_HOPDF_MINB
#define DW_HOPDF_MINB 2
#endif
template <int SPA>
struct HopOccupancy {
  static constexpr int kMinBlocks = (SPA == P16 || SPA == PB16) ? DW_HOP16_MINB : SPA == PDF ? DW_HOPDF_MINB : 1;
};

template <int SPA, int LP, bool C12, bool DAG, class In, class Epi, int OP = OP_WILSON>
__global__ void __launch_bounds__(256, HopOccupancy<SPA>::kMinBlocks)
    k_hop(const __grid_constant__ Batch B, int par_mode, int link_slot, In in, Epi epi, RedArgs ra) {
  using R = typename Spin<SPA>::R;
  DW_BLOCK_PROLOGUE(epi.gate)
  {
    typename RedT<R>::type nrm = red_zero(typename RedT<R>::type());
    typename Epi::Packed po;
    if (valid) {
      const Coord c = coord_of(S, s, par);
      const int pin = par ^ 1;
      const char* ulink_own = slot_ptr(S, link_slot, 0, par);  // links based at this site
      const char* ulink_nb = slot_ptr(S, link_slot, 0, pin);   // links based at the neighbour
      const long long mu_stride = (long long)Link<LP, C12>::kBytes * S.vh;
      constexpr int SF = DAG ? +1 : -1;  // forward projector sign
      constexpr int SB = -SF;            // backward projector sign
      Cx<R> acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = cx((R)0, (R)0);

#define DW_HOP_DIR(MU)                                                          \
  {                                                                             \
    float eta;                                                                  \
    Cx<R> p[12], h[6], g[6], u[9];                                              \
    R sc;                                                                       \
    const int nf = neighbour<MU, +1>(S, c, s, &eta);                            \
    in.load_raw(S, pin, r, nf, p, sc);                                          \
    project<MU, SF>(p, h);                                                      \
    Link<LP, C12>::load(ulink_own + MU * mu_stride, S.vh, s, u);                 \
    su3_mul<false>(u, h, g);                                                    \
    accumulate_w<MU, SF>(acc, g, eta < 0.f ? -sc : sc);                         \
    const int nb = neighbour<MU, -1>(S, c, s, &eta);                            \
    in.load_raw(S, pin, r, nb, p, sc);                                          \
    project<MU, SB>(p, h);                                                      \
    Link<LP, C12>::load(ulink_nb + MU * mu_stride, S.vh, nb, u);                 \
    su3_mul<true>(u, h, g);                                                     \
    accumulate_w<MU, SB>(acc, g, eta < 0.f ? -sc : sc);                         \
  }
#define DW_HOP_DIR_W(MU)                                                        \
  {                                                                             \
    float eta, sc;                                                              \
    uint32_t p[12], h[6], u[9];                                                 \
    Cx<float> g[6];                                                             \
    const int nf = neighbour<MU, +1>(S, c, s, &eta);                            \
    in.load_words(S, pin, r, nf, p, sc);                                        \
    project_w<MU, SF, SPA>(p, h);                                               \
    Link<LP, C12>::load_words(ulink_own + MU * mu_stride, S.vh, s, u);           \
    su3_mul_w<false, SPA>(u, h, g);                                             \
    accumulate_w<MU, SF>(acc, g, eta < 0.f ? -sc : sc);                         \
    const int nb = neighbour<MU, -1>(S, c, s, &eta);                            \
    in.load_words(S, pin, r, nb, p, sc);                                        \
    project_w<MU, SB, SPA>(p, h);                                               \
    Link<LP, C12>::load_words(ulink_nb + MU * mu_stride, S.vh, nb, u);           \
    su3_mul_w<true, SPA>(u, h, g);                                              \
    accumulate_w<MU, SB>(acc, g, eta < 0.f ? -sc : sc);                         \
  }
      if constexpr (OP == OP_LAPLACE) {
        laplace_dirs<SPA, LP, C12>(S, in, c, s, r, pin, ulink_own, ulink_nb, mu_stride, acc);
        if constexpr (SPA == PDF) {
#pragma unroll
          for (int k = 0; k < 12; ++k) acc[k] = cx(renorm(acc[k].re), renorm(acc[k].im));
        }
      } else if constexpr (SPA == P16 || SPA == PB16) {
        DW_HOP_DIR_W(0)
        DW_HOP_DIR_W(1)
        DW_HOP_DIR_W(2)
        DW_HOP_DIR_W(3)
      } else if constexpr (SPA == PDF) {
        // compact loop: one copy of the double-float mat-vec per (U, U^dag)
#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu) {
          float eta;
          Cx<R> h[6], g[6], u[9];
          const DirSpin df = dir_spin(mu, SF), db = dir_spin(mu, SB);
          const int nf = neighbour_rt(S, c, s, mu, +1, &eta);
          project_rt_loaded(df, in, S, pin, r, nf, h);
          Link<LP, C12>::load(ulink_own + mu * mu_stride, S.vh, s, u);
          if (eta < 0.f) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = cx(-h[k].re, -h[k].im);
          }
          su3_mul<false>(u, h, g);
          accumulate_rt(df, acc, g);
          const int nb = neighbour_rt(S, c, s, mu, -1, &eta);
          project_rt_loaded(db, in, S, pin, r, nb, h);
          Link<LP, C12>::load(ulink_nb + mu * mu_stride, S.vh, nb, u);
          if (eta < 0.f) {
#pragma unroll
            for (int k = 0; k < 6; ++k) h[k] = cx(-h[k].re, -h[k].im);
          }
          su3_mul<true>(u, h, g);
          accumulate_rt(db, acc, g);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = cx(renorm(acc[k].re), renorm(acc[k].im));
      } else {
        DW_HOP_DIR(0)
        DW_HOP_DIR(1)
        DW_HOP_DIR(2)
        DW_HOP_DIR(3)
      }
#undef DW_HOP_DIR
#undef DW_HOP_DIR_W
      if constexpr (Epi::kSplit) po = epi.prepare(S, par, r, s, acc, nrm);
      else epi.write(S, par, r, s, acc, nrm);
    }
    if constexpr (Epi::kSplit) {
      DW_BLOCK_REDUCE_STORE(nrm, [&] {
        if (valid) epi.commit(S, par, r, s, po);
      })
    } else if constexpr (Epi::kReduce) {
      DW_BLOCK_REDUCE(nrm)
    }
  }
}

// 16-bit stencil with two right-hand sides per thread: each link is loaded,
// and with 12-real compression its third row rebuilt, once and applied to
// both; the two neighbour loads of a direction are in flight together.  Block:
// T sites x RB thread groups, group g of right-hand-side block y taking
// right-hand sides 2(y RB + g) and 2(y RB + g) + 1, for ny = ceil(nrhs / (2 RB))
// blocks y; the grid is one-dimensional with y varying fastest.
template <int SPA, bool C12, bool DAG, class Epi>
__global__ void __launch_bounds__(256, 2)
    k_hop_pair(const __grid_constant__ Batch B, int par_mode, int link_slot, int in_slot, Epi epi, RedArgs ra) {
  static_assert(SPA == P16 || SPA == PB16, "two right-hand sides per thread: 16-bit storage");
  __shared__ SysDesc S;
  __shared__ int act[64];
  const int T = B.T, RB = B.RB;
  const unsigned ny = (unsigned)((B.sd[0].nrhs + 2 * RB - 1) / (2 * RB));
  const unsigned bx = B.rev ? gridDim.x - 1u - blockIdx.x : blockIdx.x;
  const int by = (int)(bx % ny);
  int b = (int)(bx / ny), par;
  if (par_mode == 2) {
    par = b >= B.ntot ? 1 : 0;
    b -= par * B.ntot;
  } else {
    par = par_mode;
  }
  load_desc(S, B.sd, block_system(B, b));
  __syncthreads();
  for (int i_ = threadIdx.x; i_ < S.nrhs; i_ += blockDim.x) act[i_] = gate_of(epi.gate, ra.cols, S.col0 + i_);
  __syncthreads();
  int any = 0;
  for (int i_ = 0; i_ < S.nrhs; ++i_) any |= act[i_];
  if (!any) return;
  const int rl = threadIdx.x / T;
  const int r0 = (by * RB + rl) * 2, r1 = r0 + 1;
  const int tile = b - S.tile0;
  const int s = tile * T + (threadIdx.x - rl * T);
  const bool site = s < S.vh;
  const bool v0 = site && r0 < S.nrhs && act[r0 < S.nrhs ? r0 : 0];
  const bool v1 = site && r1 < S.nrhs && act[r1 < S.nrhs ? r1 : 0];
  const int r1l = r1 < S.nrhs ? r1 : r0;  // a missing second column reloads the first
  typename RedT<float>::type nrm[2] = {red_zero(typename RedT<float>::type()), red_zero(typename RedT<float>::type())};
  typename Epi::Packed po0, po1;
  if (v0 || v1) {
    const InOne<SPA> in{in_slot};
    const Coord c = coord_of(S, s, par);
    const int pin = par ^ 1;
    const char* ulink_own = slot_ptr(S, link_slot, 0, par);
    const char* ulink_nb = slot_ptr(S, link_slot, 0, pin);
    const long long mu_stride = (long long)Link<SPA, C12>::kBytes * S.vh;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    Cx<float> acc0[12], acc1[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc0[k] = acc1[k] = cx(0.f, 0.f);
#define DW_HOP_PAIR_DIR(MU)                                                     \
  {                                                                             \
    float eta, sc0, sc1;                                                        \
    uint32_t p0[12], p1[12], h0[6], h1[6], u[9];                                \
    Cx<float> g[6];                                                             \
    const int nf = neighbour<MU, +1>(S, c, s, &eta);                            \
    in.load_words(S, pin, r0, nf, p0, sc0);                                     \
    in.load_words(S, pin, r1l, nf, p1, sc1);                                    \
    Link<SPA, C12>::load_words(ulink_own + MU * mu_stride, S.vh, s, u);         \
    project_w<MU, SF, SPA>(p0, h0);                                             \
    project_w<MU, SF, SPA>(p1, h1);                                             \
    su3_mul_w<false, SPA>(u, h0, g);                                            \
    accumulate_w<MU, SF>(acc0, g, eta < 0.f ? -sc0 : sc0);                      \
    su3_mul_w<false, SPA>(u, h1, g);                                            \
    accumulate_w<MU, SF>(acc1, g, eta < 0.f ? -sc1 : sc1);                      \
    const int nb = neighbour<MU, -1>(S, c, s, &eta);                            \
    in.load_words(S, pin, r0, nb, p0, sc0);                                     \
    in.load_words(S, pin, r1l, nb, p1, sc1);                                    \
    Link<SPA, C12>::load_words(ulink_nb + MU * mu_stride, S.vh, nb, u);         \
    project_w<MU, SB, SPA>(p0, h0);                                             \
    project_w<MU, SB, SPA>(p1, h1);                                             \
    su3_mul_w<true, SPA>(u, h0, g);                                             \
    accumulate_w<MU, SB>(acc0, g, eta < 0.f ? -sc0 : sc0);                      \
    su3_mul_w<true, SPA>(u, h1, g);                                             \
    accumulate_w<MU, SB>(acc1, g, eta < 0.f ? -sc1 : sc1);                      \
  }
    DW_HOP_PAIR_DIR(0)
    DW_HOP_PAIR_DIR(1)
    DW_HOP_PAIR_DIR(2)
    DW_HOP_PAIR_DIR(3)
#undef DW_HOP_PAIR_DIR
    if constexpr (Epi::kSplit) {
      if (v0) po0 = epi.prepare(S, par, r0, s, acc0, nrm[0]);
      if (v1) po1 = epi.prepare(S, par, r1, s, acc1, nrm[1]);
    } else {
      if (v0) epi.write(S, par, r0, s, acc0, nrm[0]);
      if (v1) epi.write(S, par, r1, s, acc1, nrm[1]);
    }
  }
  if constexpr (Epi::kReduce) {
    const int ntiles = par_mode == 2 ? 2 * S.tpp : S.tpp;
    const int tt = par_mode == 2 ? par * S.tpp + tile : tile;
    reduce_block_n<2>(S, T, RB, tt, ntiles, nrm, ra, by, [&] {
      if constexpr (Epi::kSplit) {
        if (v0) epi.commit(S, par, r0, s, po0);
        if (v1) epi.commit(S, par, r1, s, po1);
      }
    });
  }
}

// ------------------------------------------------------------------ site-local kernels
// r -= alpha w;  reduction |r|^2 -> FIN_UPDATE.  The matching x-increment
// xl += alpha p is left to k_update_p (which reads p anyway) or, when a
// reliable update comes first, to k_fold_x: ColState::alpha_x holds it.
template <int SPL>
__global__ void __launch_bounds__(256) k_update_r(const __grid_constant__ Batch B, int par_mode, RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_ACTIVE)
  using RL = typename Spin<SPL>::R;
  typename RedT<RL>::type nrm = red_zero(typename RedT<RL>::type());
  typename Spin<SPL>::Packed rp;
  if (valid) {
    const ColState& C = ra.cols[S.col0 + r];
    Cx<RL> w[12], rv[12];
    Spin<SPL>::load(slot_ptr(S, S_W, r, par), S.vh, s, w);
    Spin<SPL>::load(slot_ptr(S, S_R, r, par), S.vh, s, rv);
    const RL a = scalar_as<RL>(C.alpha, C.alpha_f);
    RL n = (RL)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) rv[k] = cx(fma(-a, w[k].re, rv[k].re), fma(-a, w[k].im, rv[k].im));
    // the norm is taken of the value as stored, so the recursion sees what
    // the next kernels will read
    Spin<SPL>::roundtrip(rv);
    rp = Spin<SPL>::pack(rv);
#pragma unroll
    for (int k = 0; k < 12; ++k) n = fma(rv[k].re, rv[k].re, fma(rv[k].im, rv[k].im, n));
    nrm = to_red(n);
  }
  ra.fin = FIN_UPDATE;
  DW_BLOCK_REDUCE_STORE(nrm, [&] {
    if (valid) Spin<SPL>::store_packed(slot_wptr(S, S_R, r, par), S.vh, s, rp);
  })
}

// xl += alpha_x p (the increment of the iteration that used p, unless a
// reliable update has folded it already: alpha_x = 0);  p = z + beta p
template <int SPL, int SPA>
__global__ void __launch_bounds__(256) k_update_p(const __grid_constant__ Batch B, int par_mode, RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_ACTIVE)
  if (valid) {
    using RL = typename Spin<SPL>::R;
    using RA = typename Spin<SPA>::R;
    const ColState& C = ra.cols[S.col0 + r];
    const RL beta = scalar_as<RL>(C.beta, C.beta_f);
    Cx<RL> p[12], z[12];
    Spin<SPL>::load(slot_ptr(S, S_P, r, par), S.vh, s, p);
    Spin<SPL>::load(slot_ptr(S, S_Z, r, par), S.vh, s, z);
    if (C.alpha_x != 0.0) {
      const RA aa = scalar_as<RA>(C.alpha_x, C.alpha_xf);
      Cx<RA> xl[12];
      Spin<SPA>::load(slot_ptr(S, S_XL, r, par), S.vh, s, xl);
#pragma unroll
      for (int k = 0; k < 12; ++k) xl[k] = cx(fma(aa, (RA)p[k].re, xl[k].re), fma(aa, (RA)p[k].im, xl[k].im));
      Spin<SPA>::store(slot_wptr(S, S_XL, r, par), S.vh, s, xl);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = cx(fma(beta, p[k].re, z[k].re), fma(beta, p[k].im, z[k].im));
    Spin<SPL>::store(slot_wptr(S, S_P, r, par), S.vh, s, p);
  }
}

// First residual for a zero initial guess: r_low = src, reduction |src|^2 -> FIN_RESID0
template <int SPL, int SPH>
__global__ void __launch_bounds__(256) k_init_r(const __grid_constant__ Batch B, int par_mode, int slot_src, RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_XZERO)
  using RH = typename Spin<SPH>::R;
  typename RedT<RH>::type nrm = red_zero(typename RedT<RH>::type());
  if (valid) {
    Cx<RH> v[12];
    Cx<typename Spin<SPL>::R> lo[12];
    Spin<SPH>::load(slot_ptr(S, slot_src, r, par), S.vh, s, v);
    RH n = (RH)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) n = fma(v[k].re, v[k].re, fma(v[k].im, v[k].im, n));
    nrm = to_red(n);
    convert12(v, lo);
    Spin<SPL>::store(slot_wptr(S, S_R, r, par), S.vh, s, lo);
  }
  DW_BLOCK_REDUCE(nrm)
}

// x += xl + alpha_x p; xl = 0 on the launched parities (start of a reliable
// update: the pending increment of the current iteration is added first, in
// the increment's precision, as k_update_p would have)
template <int SPL, int SPA, int SPH>
__global__ void __launch_bounds__(256) k_fold_x(const __grid_constant__ Batch B, int par_mode, RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_REL)
  if (valid) {
    using RL = typename Spin<SPL>::R;
    using RA = typename Spin<SPA>::R;
    using RH = typename Spin<SPH>::R;
    const ColState& C = ra.cols[S.col0 + r];
    Cx<RH> x[12];
    Cx<RA> xl[12];
    Spin<SPH>::load(slot_ptr(S, S_X, r, par), S.vh, s, x);
    Spin<SPA>::load(slot_ptr(S, S_XL, r, par), S.vh, s, xl);
    if (C.alpha_x != 0.0) {
      const RA aa = scalar_as<RA>(C.alpha_x, C.alpha_xf);
      Cx<RL> p[12];
      Spin<SPL>::load(slot_ptr(S, S_P, r, par), S.vh, s, p);
#pragma unroll
      for (int k = 0; k < 12; ++k) xl[k] = cx(fma(aa, (RA)p[k].re, xl[k].re), fma(aa, (RA)p[k].im, xl[k].im));
      Spin<SPA>::roundtrip(xl);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      x[k] = cx(x[k].re + (RH)xl[k].re, x[k].im + (RH)xl[k].im);
      xl[k] = cx((RA)0, (RA)0);
    }
    Spin<SPH>::store(slot_wptr(S, S_X, r, par), S.vh, s, x);
    Spin<SPA>::store(slot_wptr(S, S_XL, r, par), S.vh, s, xl);
  }
}

// |field|^2 of slot over the launched parities -> finalizer ra.fin (gate: all)
template <int SP>
__global__ void __launch_bounds__(256) k_norm(const __grid_constant__ Batch B, int par_mode, int slot, RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_ALL)
  using RS = typename Spin<SP>::R;
  typename RedT<RS>::type nrm = red_zero(typename RedT<RS>::type());
  if (valid) {
    Cx<RS> v[12];
    Spin<SP>::load(slot_ptr(S, slot, r, par), S.vh, s, v);
    RS n = (RS)0;
#pragma unroll
    for (int k = 0; k < 12; ++k) n = fma(v[k].re, v[k].re, fma(v[k].im, v[k].im, n));
    nrm = to_red(n);
  }
  DW_BLOCK_REDUCE(nrm)
}

// Odd-site reconstruction x_o = b_o + kappa t_o, t_o = H_oe x_e as left in the
// odd half of S_RT by the last reliable update, in the high precision SPH.
template <int SPH>
__global__ void __launch_bounds__(256) k_recon_odd(const __grid_constant__ Batch B, int par_mode, RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_ALL)
  if (valid) {
    using RH = typename Spin<SPH>::R;
    Cx<RH> bv[12], tv[12], xv[12];
    Spin<SPH>::load(slot_ptr(S, S_B, r, par), S.vh, s, bv);
    Spin<SPH>::load(slot_ptr(S, S_RT, r, par), S.vh, s, tv);
    const RH k = coef<C_PK, RH>(S);
#pragma unroll
    for (int j = 0; j < 12; ++j) xv[j] = cx(fma(k, tv[j].re, bv[j].re), fma(k, tv[j].im, bv[j].im));
    Spin<SPH>::store(slot_wptr(S, S_X, r, par), S.vh, s, xv);
  }
}

// field <- 0 for the columns with a zero source (gate G_ZSRC)
template <int SP>
__global__ void __launch_bounds__(256) k_zero_zsrc(const __grid_constant__ Batch B, int par_mode, int slot, RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_ZSRC)
  if (valid) {
    Cx<typename Spin<SP>::R> z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) z[k] = cx((typename Spin<SP>::R)0, (typename Spin<SP>::R)0);
    Spin<SP>::store(slot_wptr(S, slot, r, par), S.vh, s, z);
  }
}

// dst = convert(src), over the launched parities (gate: all)
template <int SPD, int SPS>
__global__ void __launch_bounds__(256) k_convert(const __grid_constant__ Batch B, int par_mode, int slot_dst, int slot_src,
                                                 RedArgs ra) {
  DW_BLOCK_PROLOGUE(G_ALL)
  if (valid) {
    Cx<typename Spin<SPS>::R> v[12];
    Cx<typename Spin<SPD>::R> o[12];
    Spin<SPS>::load(slot_ptr(S, slot_src, r, par), S.vh, s, v);
    convert12(v, o);
    Spin<SPD>::store(slot_wptr(S, slot_dst, r, par), S.vh, s, o);
  }
}

}  // namespace dw

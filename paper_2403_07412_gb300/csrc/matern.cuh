// Matérn correlation of Eq. (2) as seen by the likelihood kernels.
//
// rho(u) = C(d)/sigma2 with u = (d/beta)^2, and h(u) = u * drho/du, so that
// dC/dbeta = -(2 sigma2 / beta) h(u).  rho is read from a per-nu table of
// piecewise polynomials (built on the GPU by matern_fit_kernel, see matern.cu):
//   u in [2^e (1 + j/16), 2^e (1 + (j+1)/16)),  e in [kELo, kEHi),  j in 0..15,
//   t = 32 u / 2^e - 33 - 2j in [-1, 1),  rho ~ P(t) = sum_{k<=8} c_k t^k.
// The interval index and t come from the bits of u with integer operations.  On GB300
// an FP64 instruction occupies its pipe about 76 times as long as an FP32 one, so only
// the constant term is added in FP64:
//   P(t) = c0 + t q(t),  q(t) = c1 + t(c2 + t(c3 + t(c4 + t T5(t)))),
//   T5(t) = c5 + c6 t + c7 t^2 + c8 t^3.
// q and t q are evaluated in double-float arithmetic (pairs of floats with error-free
// products and sums, about 2^-47 relative), the tail T5 in plain FP32, and the pair
// (hi, lo) of t q re-enters FP64 by exact bit conversion: two FP64 additions per rho.
// Since |t q| is at most ~|c1| (~1/30 of rho's scale), the result stays within FP64
// rounding of rho.  h = u rho'(u) = 32 M P'(t) (M = mantissa of u) is formed the same
// way with one FP64 addition.  The float coefficients carry a per-interval power-of-two
// scale, so that they keep their relative precision where rho is tiny.
// Below 2^kELo the expansion of rho at u = 0 is used; at and above 2^kEHi, rho = 0.
#pragma once

#include "common.cuh"

namespace vecchia {

struct MaternConst {
  // kind: Matérn 0 = non-integer nu, 1 = nu == 1, 2 = integer nu >= 2;
  //       3 = power exponential (nu holds the exponent alpha).
  int kind;
  double nu, a1, G, b0, b1;
};

// Coefficient words of interval idx (kIntWords float4 each), every float times 2^S:
//   w0: c1 hi, c1 lo, c2 hi, c2 lo      w1: c3 hi, c3 lo, c4 hi, c4 lo
//   w2: c5, c6, c7, c8                   w3: c0 (FP64, low word first), S (int), 0
//   w4: 3c3 hi, 3c3 lo, 5c5, 6c6
__device__ __forceinline__ const float4* table_iv(const double* tab) {
  return reinterpret_cast<const float4*>(tab);
}
__device__ __forceinline__ const double* table_c(const double* tab) { return tab + 2 * kIntWords * kNInt; }

__device__ __forceinline__ MaternConst load_matern_const(const double* __restrict__ tab) {
  const double* c = table_c(tab);
  MaternConst mc;
  mc.kind = (int)__double_as_longlong(c[0]);
  mc.nu = c[1];
  mc.a1 = c[2];
  mc.G = c[3];
  mc.b0 = c[4];
  mc.b1 = c[5];
  return mc;
}

// f 2^adj as a double, exactly, with integer operations (0 for zero, subnormal f, or
// a result below the normal range).
__device__ __forceinline__ double f2d_scaled(float f, int adj) {
  const unsigned fb = __float_as_uint(f);
  const unsigned ab = fb & 0x7FFFFFFFu;
  const int e = (int)(ab >> 23) + 896 + adj;
  if (ab < 0x00800000u || e <= 0) return 0.0;
  const unsigned long long db = ((unsigned long long)(fb & 0x80000000u) << 32) |
                                ((unsigned long long)e << 52) | ((unsigned long long)(ab & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)db);
}

// v 2^-24 as a float, exactly, for v < 2^24 (no int-to-float conversion instruction).
__device__ __forceinline__ float u24_float(unsigned v) {
  return (__uint_as_float(0x3F800000u | (v & 0x7FFFFFu)) - ((v >> 23) ? 0.0f : 1.0f)) * 0.5f;
}

// Bits of u below the sub-interval index: fr (kFracBits = 48 bits), t = fr 2^-47 - 1,
// returned as an exact float pair th + tl (the leading 24 and the trailing 24 bits).
constexpr int kFracBits = 52 - kSub;
__device__ __forceinline__ void local_t_df(long long fr, float& th, float& tl) {
  const unsigned hi = (unsigned)(fr >> 24);
  th = __uint_as_float(0x3F800000u | (hi & 0x7FFFFFu)) - ((hi >> 23) ? 1.0f : 2.0f);
  tl = u24_float((unsigned)fr & 0xFFFFFFu) * 0x1p-23f;
}

// Double-float arithmetic (error-free transformations; the explicit _rn intrinsics keep
// the compiler from fusing the steps whose rounding errors are being captured).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (h, l) = (ah, al) * (bh, bl), dropping al bl.
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  h = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -h);
  e = fmaf(ah, bl, e);
  l = fmaf(al, bh, e);
}

// (ph, pl) <- (ch, cl) + (ph, pl) (th, tl), renormalised.
__device__ __forceinline__ void df_horner(float& ph, float& pl, float th, float tl, float ch, float cl) {
  float xh, xl, s, e;
  df_mul(ph, pl, th, tl, xh, xl);
  two_sum(ch, xh, s, e);
  e = __fadd_rn(e, __fadd_rn(xl, cl));
  ph = __fadd_rn(s, e);
  pl = __fsub_rn(e, __fsub_rn(ph, s));
}

// (ph, pl) = (ch, cl) + p th for a plain float p (the tail), renormalised.
__device__ __forceinline__ void df_start(float& ph, float& pl, float p, float th, float ch, float cl) {
  float s, e;
  two_sum(ch, __fmul_rn(p, th), s, e);
  e = __fadd_rn(e, cl);
  ph = __fadd_rn(s, e);
  pl = __fsub_rn(e, __fsub_rn(ph, s));
}

// Expansion of rho and h at u -> 0 (u < 2^kELo), from the series of x^nu K_nu(x):
//   non-integer nu: rho = 1 + u/(4(1-nu)) - Gamma(1-nu) (u/4)^nu [1/Gamma(1+nu) + (u/4)/Gamma(2+nu)]
//   nu = 1:          rho = 1 + (u/4)(log(u/4) + 2 gamma_E - 1)
//   integer nu >= 2: rho = 1 - u/(4(nu-1))
// Omitted terms are O(u^2 log u) or O(u^(nu+2)), below 1e-17 for u < 2^-30.
// Power exponential, Eq. (3), evaluated directly: with u = (d / beta^(1/alpha))^2,
// rho = exp(-u^(alpha/2)) and h = u rho' = -(alpha/2) u^(alpha/2) rho.
static __device__ __noinline__ void rho_powexp(double u, double alpha, double& rho, double& h) {
  if (u == 0.0) { rho = 1.0; h = 0.0; return; }
  const double w = exp(0.5 * alpha * log(u));
  rho = exp(-w);
  h = -0.5 * alpha * w * rho;
}

static __device__ __noinline__ void rho_small(double u, const MaternConst& mc, double& rho, double& h) {
  if (mc.kind == 3) { rho_powexp(u, mc.nu, rho, h); return; }
  if (u == 0.0) { rho = 1.0; h = 0.0; return; }
  const double q = 0.25 * u;
  if (mc.kind == 1) {
    const double L = log(q) + 1.1544313298030657;  // + 2 gamma_E
    rho = 1.0 + q * (L - 1.0);
    h = q * L;
  } else if (mc.kind == 2) {
    rho = 1.0 + mc.a1 * u;
    h = mc.a1 * u;
  } else {
    const double w = exp(mc.nu * log(q));
    rho = 1.0 + mc.a1 * u - mc.G * w * (mc.b0 + mc.b1 * u);
    h = mc.a1 * u - mc.G * w * (mc.nu * mc.b0 + (mc.nu + 1.0) * mc.b1 * u);
  }
}

// Polynomial part of rho(u) (and h(u) = u rho'(u) when DERIV), branch-free: the
// interval index is clamped, so u outside [2^kELo, 2^kEHi) gets a finite value that
// rho_fix() then replaces.
struct PolyArg {
  long long b;
  int idx;
  float th, tl;
};

__device__ __forceinline__ PolyArg poly_arg(double u) {
  PolyArg a;
  a.b = __double_as_longlong(u);
  const int ex = min(max((int)(a.b >> 52) - 1023, kELo), kEHi - 1);
  a.idx = ((ex - kELo) << kSub) | (int)((a.b >> kFracBits) & ((1 << kSub) - 1));
  local_t_df(a.b & ((1LL << kFracBits) - 1), a.th, a.tl);
  return a;
}

// 32 M P'(t) at scale 2^S as a float pair (M = mantissa of u, leading 47 bits).
__device__ __forceinline__ void h_pair(const PolyArg& a, const float4& w0, const float4& w1, const float4& w2,
                                       const float4& w4, float& hh, float& hl) {
  // P'(t) = c1 + t(2c2 + t(3c3 + t(4c4 + t D5(t)))),  D5 = 5c5 + t(6c6 + t(7c7 + t 8c8))
  const float d5 = fmaf(fmaf(fmaf(8.0f * w2.w, a.th, 7.0f * w2.z), a.th, w4.w), a.th, w4.z);
  float qh, ql;
  df_start(qh, ql, d5, a.th, 4.0f * w1.z, 4.0f * w1.w);
  df_horner(qh, ql, a.th, a.tl, w4.x, w4.y);
  df_horner(qh, ql, a.th, a.tl, 2.0f * w0.z, 2.0f * w0.w);
  df_horner(qh, ql, a.th, a.tl, w0.x, w0.y);
  const float mh = __uint_as_float(0x3F800000u | (unsigned)((a.b >> 29) & 0x7FFFFF));
  const float ml = u24_float((unsigned)(a.b >> 5) & 0xFFFFFFu) * 0x1p-23f;
  df_mul(qh, ql, mh, ml, hh, hl);
}

// t q(t) at scale 2^S as a float pair: the non-constant part of P(t).
__device__ __forceinline__ void tq_pair(const PolyArg& a, const float4& w0, const float4& w1, const float4& w2,
                                        float& xh, float& xl) {
  const float t5 = fmaf(fmaf(fmaf(w2.w, a.th, w2.z), a.th, w2.y), a.th, w2.x);
  float ph, pl;
  df_start(ph, pl, t5, a.th, w1.z, w1.w);
  df_horner(ph, pl, a.th, a.tl, w1.x, w1.y);
  df_horner(ph, pl, a.th, a.tl, w0.z, w0.w);
  df_horner(ph, pl, a.th, a.tl, w0.x, w0.y);
  df_mul(ph, pl, a.th, a.tl, xh, xl);
}

// rho (and h when DERIV) to about FP64 rounding, relative, even where rho is tiny: c0 in
// FP64 plus the pair, two FP64 additions for rho and one for h.
template <bool DERIV>
__device__ __forceinline__ void rho_poly(double u, const double* __restrict__ tab, double& rho, double& h) {
  const PolyArg a = poly_arg(u);
  const float4* __restrict__ w = table_iv(tab) + a.idx * kIntWords;
  const float4 w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3);
  const int S = __float_as_int(w3.z);
  float xh, xl;
  tq_pair(a, w0, w1, w2, xh, xl);
  const double c0 = __hiloint2double(__float_as_int(w3.y), __float_as_int(w3.x));
  rho = (c0 + f2d_scaled(xh, -S)) + f2d_scaled(xl, -S);
  if (DERIV) {
    const float4 w4 = __ldg(w + 4);
    float hh, hl;
    h_pair(a, w0, w1, w2, w4, hh, hl);
    h = f2d_scaled(hh, 5 - S) + f2d_scaled(hl, 5 - S);
  }
}

// h(u) = u rho'(u) alone in FP64 (one FP64 addition), branch-free.
__device__ __forceinline__ double h_poly(double u, const double* __restrict__ tab) {
  const PolyArg a = poly_arg(u);
  const float4* __restrict__ w = table_iv(tab) + a.idx * kIntWords;
  const float4 w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3), w4 = __ldg(w + 4);
  const int S = __float_as_int(w3.z);
  float hh, hl;
  h_pair(a, w0, w1, w2, w4, hh, hl);
  return f2d_scaled(hh, 5 - S) + f2d_scaled(hl, 5 - S);
}

// Replaces rho_poly's value outside the tabulated range (rare): u < 2^kELo -> the
// expansion at zero (Matérn) or direct evaluation (power exponential); u >= 2^kEHi ->
// 0 for the Matérn (below the smallest double), direct evaluation for the power
// exponential (whose far field decays slowly for small exponents).
__device__ __forceinline__ void rho_fix(double u, const MaternConst& mc, double& rho, double& h) {
  const int ex = (int)(__double_as_longlong(u) >> 52) - 1023;
  if (ex >= kEHi) {
    if (mc.kind == 3) rho_powexp(u, mc.nu, rho, h);
    else { rho = 0.0; h = 0.0; }
  } else if (ex < kELo) {
    rho_small(u, mc, rho, h);
  }
}

__device__ __forceinline__ double h_fix(double u, const MaternConst& mc, double h) {
  const int ex = (int)(__double_as_longlong(u) >> 52) - 1023;
  if (ex >= kEHi || ex < kELo) {
    double r = 0.0;
    rho_fix(u, mc, r, h);
  }
  return h;
}

// ---- evaluation from a double-float argument u = uh + ul (likelihood kernels)
// The interval index and t come from uh's float bits: u / 2^e = 1.m, t = 32 u / 2^e -
// 33 - 2j, so th = (m mod 2^19) 2^-18 - 1 exactly and tl = ul 2^(5-e); 32 M = u dt/du is
// (uh, ul) 2^(5-e).  Outside [2^kELo, 2^kEHi) the clamped index gives a finite value that
// the rare path below replaces.
struct PolyArgF {
  int idx, ex;
  float th, tl, mh, ml;  // t and 32 M as float pairs
};

__device__ __forceinline__ PolyArgF poly_arg_df(float uh, float ul) {
  PolyArgF a;
  const unsigned ub = __float_as_uint(uh);
  a.ex = (int)((ub >> 23) & 0xFF) - 127;
  const int ec = min(max(a.ex, kELo), kEHi - 1);
  a.idx = ((ec - kELo) << kSub) | (int)((ub >> 19) & ((1u << kSub) - 1));
  a.th = fmaf(__uint_as_float(0x3F800000u | ((ub & 0x7FFFFu) << 4)), 2.0f, -3.0f);
  const float sc = __uint_as_float((unsigned)(127 + 5 - ec) << 23);
  a.tl = __fmul_rn(ul, sc);
  a.mh = __fmul_rn(uh, sc);
  a.ml = a.tl;
  return a;
}

// u outside the tabulated range as a double (rare path).
__device__ __forceinline__ double df_to_double(float uh, float ul) {
  return f2d_scaled(uh, 0) + f2d_scaled(ul, 0);
}

__device__ __forceinline__ double rho_df(float uh, float ul, const double* __restrict__ tab, const MaternConst& mc) {
  const PolyArgF a = poly_arg_df(uh, ul);
  const float4* __restrict__ w = table_iv(tab) + a.idx * kIntWords;
  const float4 w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3);
  const int S = __float_as_int(w3.z);
  const float t5 = fmaf(fmaf(fmaf(w2.w, a.th, w2.z), a.th, w2.y), a.th, w2.x);
  float ph, pl, xh, xl;
  df_start(ph, pl, t5, a.th, w1.z, w1.w);
  df_horner(ph, pl, a.th, a.tl, w1.x, w1.y);
  df_horner(ph, pl, a.th, a.tl, w0.z, w0.w);
  df_horner(ph, pl, a.th, a.tl, w0.x, w0.y);
  df_mul(ph, pl, a.th, a.tl, xh, xl);
  const double c0 = __hiloint2double(__float_as_int(w3.y), __float_as_int(w3.x));
  double rho = (c0 + f2d_scaled(xh, -S)) + f2d_scaled(xl, -S);
  if (a.ex < kELo || a.ex >= kEHi) {
    double h = 0.0;
    rho_fix(df_to_double(uh, ul), mc, rho, h);
  }
  return rho;
}

// f 2^k for a float, by its exponent field; 0 when the result falls below the normal
// range (|h| is at most a few units, so it never overflows).
__device__ __forceinline__ float fscale(float f, int k) {
  const unsigned fb = __float_as_uint(f);
  const int ne = (int)((fb >> 23) & 0xFF) + k;
  if ((fb & 0x7F800000u) == 0u || ne <= 0) return 0.0f;
  return __uint_as_float((fb & 0x807FFFFFu) | ((unsigned)ne << 23));
}

// h(u) as a float pair (about 2^-46 relative), no FP64 instruction on the common path.
__device__ __forceinline__ void h_df(float uh, float ul, const double* __restrict__ tab, const MaternConst& mc,
                                     float& hh, float& hl) {
  const PolyArgF a = poly_arg_df(uh, ul);
  const float4* __restrict__ w = table_iv(tab) + a.idx * kIntWords;
  const float4 w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3), w4 = __ldg(w + 4);
  const int S = __float_as_int(w3.z);
  const float d5 = fmaf(fmaf(fmaf(8.0f * w2.w, a.th, 7.0f * w2.z), a.th, w4.w), a.th, w4.z);
  float qh, ql;
  df_start(qh, ql, d5, a.th, 4.0f * w1.z, 4.0f * w1.w);
  df_horner(qh, ql, a.th, a.tl, w4.x, w4.y);
  df_horner(qh, ql, a.th, a.tl, 2.0f * w0.z, 2.0f * w0.w);
  df_horner(qh, ql, a.th, a.tl, w0.x, w0.y);
  df_mul(qh, ql, a.mh, a.ml, hh, hl);  // 32 M P'(t), times 2^S
  hh = fscale(hh, -S);
  hl = fscale(hl, -S);
  if (a.ex < kELo || a.ex >= kEHi) {
    double r = 0.0, h = 0.0;
    rho_fix(df_to_double(uh, ul), mc, r, h);
    const float hi = __double2float_rn(h);
    hh = hi;
    hl = __double2float_rn(h - (double)hi);
  }
}

template <bool DERIV>
__device__ __forceinline__ void rho_eval(double u, const double* __restrict__ tab, const MaternConst& mc,
                                         double& rho, double& h) {
  rho_poly<DERIV>(u, tab, rho, h);
  rho_fix(u, mc, rho, h);
}

__device__ __forceinline__ double rho_only(double u, const double* __restrict__ tab, const MaternConst& mc) {
  double r, h;
  rho_eval<false>(u, tab, mc, r, h);
  return r;
}

}  // namespace vecchia

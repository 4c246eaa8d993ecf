// Matérn correlation of Eq. (2) as seen by the likelihood kernels.
//
// rho(u) = C(d)/sigma2 with u = (d/beta)^2, and h(u) = u * drho/du, so that
// dC/dbeta = -(2 sigma2 / beta) h(u).  rho is read from a per-nu table of
// piecewise polynomials (built on the GPU by matern_fit_kernel, see matern.cu):
//   u in [2^e (1 + j/16), 2^e (1 + (j+1)/16)),  e in [kELo, kEHi),  j in 0..15,
//   t = 32 u / 2^e - 33 - 2j in [-1, 1),  rho ~ P(t) = sum_{k<=8} c_k t^k.
// The interval index, t and u dt/du = 32 M (M = mantissa of u) come from the bits of
// u with integer operations.  On GB300 an FP64 instruction costs as much as ~60 others,
// so the polynomial is split by magnitude:
//   P(t) = c0 + t(c1 + t(c2 + t(c3 + t(c4 + t T5(t))))),
//   T5(t) = c5 + c6 t + c7 t^2 + c8 t^3 evaluated in FP32;
//   P'(t) = c1 + t(2 c2 + t R(t)),  R(t) = 3 c3 + 4 c4 t + ... + 8 c8 t^5 in FP32.
// Near the origin the coefficients shrink by ~1/66 per degree, so the FP32 part of rho
// stays below FP64 rounding (measured against exact rational evaluation: within
// 1.7e-16 absolute, as an all-FP64 Horner), and h keeps ~1e-9 relative accuracy where
// rho > 1e-3 (a few 1e-9 below), far below 1e-10 of max |h| in absolute terms, which
// is what the beta-gradient (a sum of h-weighted pair terms) needs.  FP32 results
// re-enter FP64 by exact bit conversion.  Cost: 5 FP64 FMAs for rho, 3 more for h.
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

__device__ __forceinline__ const double* table_d(const double* tab) { return tab; }
__device__ __forceinline__ const double* table_c(const double* tab) { return tab + kNInt * kNDbl; }
__device__ __forceinline__ const float* table_f(const double* tab) {
  return reinterpret_cast<const float*>(tab + kNInt * kNDbl + kNConst);
}

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

// Exact float -> double without the FP64 pipe (F2F is an FP64-pipe instruction).
// Zero and subnormal floats (below 1.2e-38 in magnitude) map to zero.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned fb = __float_as_uint(f);
  const unsigned ab = fb & 0x7FFFFFFFu;
  if (ab < 0x00800000u) return 0.0;
  const unsigned long long db = ((unsigned long long)(fb & 0x80000000u) << 32) |
                                ((unsigned long long)((ab >> 23) + 896u) << 52) |
                                ((unsigned long long)(ab & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)db);
}

// Bits of u below the sub-interval index, and the local variable t = s 2^-kTBits with
// s = those bits - 2^kTBits (|s| <= 2^kTBits), converted exactly with integer operations.
constexpr int kFracBits = 52 - kSub;  // bits of u below the sub-interval index
constexpr int kTBits = kFracBits - 1;
__device__ __forceinline__ double local_t(long long fr) {
  const long long s = fr - (1LL << kTBits);
  if (s == 0) return 0.0;
  const unsigned long long sign = s < 0 ? 0x8000000000000000ULL : 0ULL;
  const unsigned long long a = (unsigned long long)(s < 0 ? -s : s);
  const int lz = __clzll((long long)a);             // leading one at bit 63 - lz
  const unsigned long long e = (unsigned long long)(1023 + (63 - lz) - kTBits);
  const unsigned long long mant = (a << (lz + 1)) >> 12;
  return __longlong_as_double((long long)(sign | (e << 52) | mant));
}

// The same t in FP32 (23 leading bits), for the FP32 tails.
__device__ __forceinline__ float local_t_f32(long long fr) {
  return fmaf(__uint_as_float(0x3F800000u | (unsigned)(fr >> (kFracBits - 23))), 2.0f, -3.0f);
}

// u dt/du = 2^(kSub+1) M, M = mantissa of u in [1, 2): the exponent field set to 1023+kSub+1.
__device__ __forceinline__ double u_dtdu(long long b) {
  return __longlong_as_double(((long long)(1023 + kSub + 1) << 52) | (b & 0xFFFFFFFFFFFFFLL));
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
template <bool DERIV>
__device__ __forceinline__ void rho_poly(double u, const double* __restrict__ tab, double& rho, double& h) {
  const long long b = __double_as_longlong(u);
  const int ex = min(max((int)(b >> 52) - 1023, kELo), kEHi - 1);
  const int idx = ((ex - kELo) << kSub) | (int)((b >> kFracBits) & ((1 << kSub) - 1));
  const long long fr = b & ((1LL << kFracBits) - 1);
  const double t = local_t(fr);
  const float tf = local_t_f32(fr);
  const double2* __restrict__ cd = reinterpret_cast<const double2*>(table_d(tab) + idx * kNDbl);
  const float4* __restrict__ cf = reinterpret_cast<const float4*>(table_f(tab) + idx * kNFlt);
  const double2 c01 = __ldg(cd), c23 = __ldg(cd + 1), c4x = __ldg(cd + 2);
  const float4 f0 = __ldg(cf);
  const float t5 = fmaf(fmaf(fmaf(f0.w, tf, f0.z), tf, f0.y), tf, f0.x);
  double p = f2d_exact(t5);
  p = fma(p, t, c4x.x);
  p = fma(p, t, c23.y);
  p = fma(p, t, c23.x);
  p = fma(p, t, c01.y);
  rho = fma(p, t, c01.x);
  if (DERIV) {
    const float4 f1 = __ldg(cf + 1), f2 = __ldg(cf + 2);
    // R(t) = 3c3 + 4c4 t + 5c5 t^2 + 6c6 t^3 + 7c7 t^4 + 8c8 t^5
    float r = f2.y;
    r = fmaf(r, tf, f2.x);
    r = fmaf(r, tf, f1.w);
    r = fmaf(r, tf, f1.z);
    r = fmaf(r, tf, f1.y);
    r = fmaf(r, tf, f1.x);
    const double dq = fma(t, f2d_exact(r), c4x.y);
    const double dp = fma(t, dq, c01.y);
    h = u_dtdu(b) * dp;
  }
}

// h(u) = u rho'(u) alone (the derivative part of rho_poly<true>), branch-free.
__device__ __forceinline__ double h_poly(double u, const double* __restrict__ tab) {
  const long long b = __double_as_longlong(u);
  const int ex = min(max((int)(b >> 52) - 1023, kELo), kEHi - 1);
  const int idx = ((ex - kELo) << kSub) | (int)((b >> kFracBits) & ((1 << kSub) - 1));
  const long long fr = b & ((1LL << kFracBits) - 1);
  const double t = local_t(fr);
  const float tf = local_t_f32(fr);
  const double2* __restrict__ cd = reinterpret_cast<const double2*>(table_d(tab) + idx * kNDbl);
  const float4* __restrict__ cf = reinterpret_cast<const float4*>(table_f(tab) + idx * kNFlt);
  const double2 c01 = __ldg(cd), c4x = __ldg(cd + 2);
  const float4 f1 = __ldg(cf + 1), f2 = __ldg(cf + 2);
  float r = f2.y;
  r = fmaf(r, tf, f2.x);
  r = fmaf(r, tf, f1.w);
  r = fmaf(r, tf, f1.z);
  r = fmaf(r, tf, f1.y);
  r = fmaf(r, tf, f1.x);
  const double dq = fma(t, f2d_exact(r), c4x.y);
  const double dp = fma(t, dq, c01.y);
  return u_dtdu(b) * dp;
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

// Matérn correlation of Eq. (2) as seen by the likelihood kernels.
//
// rho(u) = C(d)/sigma2 with u = (d/beta)^2, and h(u) = u * drho/du, so that
// dC/dbeta = -(2 sigma2 / beta) h(u).  rho is read from a per-nu table of
// piecewise polynomials (built on the GPU by build_matern_table, see matern.cu):
//   u in [2^e (1 + j/8), 2^e (1 + (j+1)/8)),  e in [kELo, kEHi),  j in 0..7,
//   t = 16 u / 2^e - 17 - 2j in [-1, 1),  rho ~ sum_k c[e,j,k] t^k  (k <= kDeg).
// The interval index, t and u dt/du = 16 M (M = mantissa of u) are formed from the
// bits of u with integer operations, so one evaluation costs kDeg + 1 FP64 FMAs
// (2 kDeg + 1 with the derivative).  Below 2^kELo the two-term expansion of rho at
// u = 0 is used; at and above 2^kEHi, rho = 0 (it is below the smallest double).
#pragma once

#include "common.cuh"

namespace vecchia {

struct MaternConst {
  // kind: 0 = non-integer nu, 1 = nu == 1, 2 = integer nu >= 2.
  int kind;
  double nu, a1, G, b0, b1;
};

__device__ __forceinline__ MaternConst load_matern_const(const double* __restrict__ tab) {
  const double* c = tab + kNInt * kNCoef;
  MaternConst mc;
  mc.kind = (int)__double_as_longlong(c[0]);
  mc.nu = c[1];
  mc.a1 = c[2];
  mc.G = c[3];
  mc.b0 = c[4];
  mc.b1 = c[5];
  return mc;
}

// Expansion of rho and h at u -> 0 (u < 2^kELo), from the series of x^nu K_nu(x):
//   non-integer nu: rho = 1 + u/(4(1-nu)) - Gamma(1-nu) (u/4)^nu [1/Gamma(1+nu) + (u/4)/Gamma(2+nu)]
//   nu = 1:          rho = 1 + (u/4)(log(u/4) + 2 gamma_E - 1)
//   integer nu >= 2: rho = 1 - u/(4(nu-1))
// Omitted terms are O(u^2 log u) or O(u^(nu+2)), below 1e-17 for u < 2^-30.
static __device__ __noinline__ void rho_small(double u, const MaternConst& mc, double& rho, double& h) {
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

// rho(u) only.
__device__ __forceinline__ double rho_eval(double u, const double* __restrict__ tab,
                                           const MaternConst& mc) {
  const long long b = __double_as_longlong(u);
  const int ex = (int)(b >> 52) - 1023;
  if (ex >= kEHi) return 0.0;
  if (ex < kELo) {
    double r, h;
    rho_small(u, mc, r, h);
    return r;
  }
  const int idx = ((ex - kELo) << kSub) | (int)((b >> 49) & 7);
  const double v = __longlong_as_double(0x3FF0000000000000LL | ((b & 0x1FFFFFFFFFFFFLL) << 3));
  const double t = fma(v, 2.0, -3.0);
  const double* __restrict__ c = tab + idx * kNCoef;
  double p = __ldg(c + kDeg);
#pragma unroll
  for (int k = kDeg - 1; k >= 0; --k) p = fma(p, t, __ldg(c + k));
  return p;
}

// rho(u) and h(u) = u rho'(u).
__device__ __forceinline__ void rho_eval_d(double u, const double* __restrict__ tab,
                                           const MaternConst& mc, double& rho, double& h) {
  const long long b = __double_as_longlong(u);
  const int ex = (int)(b >> 52) - 1023;
  if (ex >= kEHi) { rho = 0.0; h = 0.0; return; }
  if (ex < kELo) { rho_small(u, mc, rho, h); return; }
  const int idx = ((ex - kELo) << kSub) | (int)((b >> 49) & 7);
  const double v = __longlong_as_double(0x3FF0000000000000LL | ((b & 0x1FFFFFFFFFFFFLL) << 3));
  const double t = fma(v, 2.0, -3.0);
  const double* __restrict__ c = tab + idx * kNCoef;
  double p = __ldg(c + kDeg), dp = 0.0;
#pragma unroll
  for (int k = kDeg - 1; k >= 0; --k) {
    dp = fma(dp, t, p);
    p = fma(p, t, __ldg(c + k));
  }
  rho = p;
  // u dt/du = 16 M, M = mantissa of u in [1, 2): exponent field set to 1023 + 4.
  const double m16 = __longlong_as_double(0x4030000000000000LL | (b & 0xFFFFFFFFFFFFFLL));
  h = m16 * dp;
}

}  // namespace vecchia

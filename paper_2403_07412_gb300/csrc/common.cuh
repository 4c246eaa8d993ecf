// Shared definitions of the Vecchia CUDA library: status codes, the plan object,
// covariance-table geometry and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vecchia.h"

namespace vecchia {

// ------------------------------------------------------------------ table geometry
// The Matérn correlation rho(u) = C(d)/sigma2 is tabulated in u = (d/beta)^2 as
// piecewise polynomials: for u in [2^e, 2^(e+1)), e in [kELo, kEHi), the octave is
// cut into 2^kSub equal sub-intervals, each carrying a degree-kDeg polynomial in the
// local variable t in [-1, 1).  Interval index and t come straight from the bits of u.
constexpr int kELo = -30;
constexpr int kEHi = 20;
constexpr int kSub = 4;
constexpr int kDeg = 8;
constexpr int kNInt = (kEHi - kELo) << kSub;
// Per interval kIntWords 16-byte words of coefficients (layout in matern.cuh), then
// kNConst doubles of small-u constants: kind, nu, a1, G, b0, b1, I(0).
constexpr int kIntWords = 5;
constexpr int kNConst = 8;
constexpr size_t kTableBytes = (size_t)16 * kIntWords * kNInt + sizeof(double) * kNConst;

// Largest conditioning sets: overall (CTA-per-location kernel) and for the warp kernels.
constexpr int kMaxM = VECCHIA_MAX_M;
constexpr int kMaxMWarp = VECCHIA_MAX_M_WARP;
// Most warps in one CTA of the warp kernels: thirteen 32-lane blocks of m = 60 fill the
// 227 KB of shared memory a CTA may hold.
constexpr int kMaxCtaWarps = 13;
// Largest block (K = m + 1 rows) a group of G lanes per location handles: narrow groups
// keep at most four neighbour slots per lane, so their per-lane register arrays (and the
// selects that index them) stay short.
__host__ __device__ constexpr int max_k_for_lanes(int G) { return G == 4 ? 16 : (G == 8 ? 32 : kMaxMWarp + 1); }

// Covariance families (VECCHIA_KERNEL_*): Matérn, Eq. (2); power exponential, Eq. (3).
constexpr int kFamilyMatern = 0;
constexpr int kFamilyPowExp = 1;

struct Plan {
  int64_t n = 0;
  int32_t m = 0;
  int family = kFamilyMatern;
  int device = 0;
  int metric = 0;             // 0: plane (Euclidean), 1: sphere (great-circle distance)
  double radius = 1.0;        // sphere radius (metric 1)
  double* d_xy = nullptr;     // n x 2, original order (longitude, latitude for metric 1)
  double* d_xyz = nullptr;    // n x 3 unit vectors, original order (metric 1)
  int32_t* d_nbr = nullptr;   // n x m, ORIGINAL indices of J_i, -1 padded (ordered rows)
  int32_t* d_self = nullptr;  // n, original index of ordered location i
  int64_t* h_perm = nullptr;  // n, host copy of the ordering
  int32_t* d_inv = nullptr;   // n, ordered position of each original index
  // reusable scratch
  double* d_partial = nullptr;  // per-CTA partial sums
  int64_t partial_cap = 0;
  unsigned long long* d_errloc = nullptr;  // first failing location (ULLONG_MAX = none)
  cudaStream_t last_stream = nullptr;
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ double rcp_newton(double d) {
  // Reciprocal: hardware approximation of 1/d (about 20 correct bits), then one
  // cubically convergent Newton step y <- y (1 + e + e^2), e = 1 - d y.
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  const double e2 = fma(e, e, e);
  return fma(y, e2, y);
}

// Reciprocal of a pivot with no FP64 instruction (the FP64 pipe is the bottleneck; the
// integer and FP32 pipes are idle most of the time).  For normal d in [2^-1022, 2^1022)
// with mantissa m in [1, 2):
//  1. y0 = 1/m_hi in FP32 (m_hi = m truncated to 24 bits), as a 32-bit fixed-point Y0 =
//     y0 2^32; |1 - m y0| < 2^-21.
//  2. The residual R = 2^84 - M Y0 (M = m 2^52 the 53-bit integer mantissa) is exact in
//     64-bit wrap-around arithmetic, since |R| < 2^63: R = e 2^84 with e = 1 - m y0.
//  3. 1/m = y0 / (1 - e) = y0 (1 + e + e^2 + ...); |e|^3 < 2^-63, so Z = 2^62 y0 (1 + e +
//     e^2) in fixed point is within a few units of 2^62/m, i.e. far below one unit in the
//     53rd bit.
//  4. The double is assembled from Z (rounded to 53 bits) and the exponent; a mantissa of
//     exactly 1 gives a power of two.
// Other inputs (zero, subnormal, >= 2^1022, negative, non-finite) give an unspecified
// finite-or-not value: callers reject them first with pivot_in_range.
__device__ __forceinline__ double rcp_fixed(double d) {
  const unsigned long long D = (unsigned long long)__double_as_longlong(d);
  const unsigned E = (unsigned)(D >> 52) & 0x7FFu;
  const unsigned hi = (unsigned)(D >> 32), lo = (unsigned)D;
  const unsigned Mhi = (hi & 0xFFFFFu) | 0x100000u;  // M = Mhi 2^32 + lo
  const float mh = __uint_as_float(0x3F800000u | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(mh));
  const unsigned rb = __float_as_uint(r);  // r in [1/2, 1]: exponent field 126 or 127
  const unsigned long long Yw = (unsigned long long)((rb & 0x7FFFFFu) | 0x800000u) << ((rb >> 23) - 118u);
  const unsigned Y0 = Yw > 0xFFFFFFFFull ? 0xFFFFFFFFu : (unsigned)Yw;
  const unsigned long long P = (unsigned long long)lo * Y0 + ((unsigned long long)(Mhi * Y0) << 32);
  const long long R = -(long long)P;  // e 2^84
  const int Rh = (int)(R >> 32);
  const unsigned Rl = (unsigned)R;
  long long c1 = ((long long)Y0 * Rh) >> 22;  // Y0 e 2^30, first order
  c1 += (long long)(((unsigned long long)Y0 * Rl) >> 54);
  const long long c2 = ((long long)(int)(c1 >> 10) * Rh) >> 42;  // second order
  const long long Z = ((long long)Y0 << 30) + c1 + c2;        // 2^62 / m, in (2^61, 2^62)
  const unsigned long long out = (D & 0xFFFFFFFFFFFFFull) == 0ull
                                     ? (unsigned long long)(2046u - E) << 52
                                     : ((unsigned long long)(2044u - E) << 52) + (unsigned long long)((Z + 256) >> 9);
  return __longlong_as_double((long long)out);
}

// a b for b a positive normal double (a pivot reciprocal), by integer arithmetic with
// round-to-nearest-even: equal to the FP64 product whenever the exact product is finite
// and at least 2^-1022 in magnitude.  The 106-bit mantissa product is formed from 32-bit
// limbs; a zero or subnormal a, or an exact product below 2^-1022, gives a zero of a's
// sign, and one that rounds beyond the largest double an infinity.
__device__ __forceinline__ double mul_by_positive(double a, double b) {
  const unsigned long long A = (unsigned long long)__double_as_longlong(a);
  const unsigned long long B = (unsigned long long)__double_as_longlong(b);
  const unsigned long long sgn = A & 0x8000000000000000ull;
  const int ea = (int)((A >> 52) & 0x7FFu), eb = (int)((B >> 52) & 0x7FFu);
  const unsigned ah = ((unsigned)(A >> 32) & 0xFFFFFu) | 0x100000u, al = (unsigned)A;
  const unsigned bh = ((unsigned)(B >> 32) & 0xFFFFFu) | 0x100000u, bl = (unsigned)B;
  const unsigned long long lo = (unsigned long long)al * bl;
  const unsigned long long mid = (unsigned long long)ah * bl + (unsigned long long)al * bh;  // < 2^54
  const unsigned long long plo = lo + (mid << 32);
  const unsigned long long phi = (unsigned long long)ah * bh + (mid >> 32) + (plo < lo ? 1ull : 0ull);
  const int top = (int)(phi >> 41) & 1;  // product in [2^105, 2^106)
  const int sh = 52 + top;
  unsigned long long m = (phi << (64 - sh)) | (plo >> sh);
  const unsigned long long rnd = (plo >> (sh - 1)) & 1ull;
  const unsigned long long sticky = (plo & ((1ull << (sh - 1)) - 1ull)) != 0ull ? 1ull : 0ull;
  m += rnd & (sticky | (m & 1ull));  // a carry out of 53 bits moves into the exponent field
  const int e = ea + eb - 1023 + top;
  unsigned long long r = sgn + ((unsigned long long)(e - 1) << 52) + m;
  r = (ea == 0 || e <= 0) ? sgn : r;
  r = e >= 2047 ? (sgn | 0x7FF0000000000000ull) : r;
  return __longlong_as_double((long long)r);
}

// True iff d is a positive normal double below 2^1022 (biased exponent in [1, 2044]),
// the domain of rcp_fixed; decided on the bit pattern.
__device__ __forceinline__ bool pivot_in_range(double d) {
  const long long b = __double_as_longlong(d);
  return b >= 0x0010000000000000LL && b < 0x7FD0000000000000LL;
}

// True iff d is a positive finite double, decided on the bit pattern (no FP64 op).
__device__ __forceinline__ bool positive_finite(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0 && b < 0x7FF0000000000000LL;
}

// True iff d is finite (not an infinity or NaN), decided on the bit pattern.
__device__ __forceinline__ bool finite_bits(double d) {
  return (__double_as_longlong(d) & 0x7FF0000000000000LL) != 0x7FF0000000000000LL;
}

struct Neumaier {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  // Adds another compensated sum (its sum and compensation).
  __device__ __forceinline__ void merge(double s2, double c2) {
    const double t = s + s2;
    const double e = fabs(s) >= fabs(s2) ? (s - t) + s2 : (s2 - t) + s;
    s = t;
    c = (c + c2) + e;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

// ------------------------------------------------------------------ error slot
// A call's error slot holds the smallest code (location << 2 | kind) written by any
// failing location, so the first failing ordered location wins and, at one location, the
// lower kind.  All ones means no failure.
constexpr unsigned kErrIndex = 0;  // a conditioning-set or location index outside [0, n)
constexpr unsigned kErrData = 1;   // a non-finite data value in the block
constexpr unsigned kErrNotPD = 2;  // a block that is not positive definite
__host__ __device__ __forceinline__ unsigned long long err_code(int64_t i, unsigned kind) {
  return ((unsigned long long)i << 2) | kind;
}

// Bounds-checked build (-DVECCHIA_CHECKED): every index the kernels read through (the
// conditioning sets, the location itself, the batched work items) is checked against
// its range before use; a bad one is recorded in the error slot (kErrIndex) and replaced
// by a valid index, and the affected outputs become NaN.  No trap, no fault.  Without the
// flag the single-field kernels check the caller-supplied index arrays only where the
// caller, not a plan, provided them (the allocation-free entry point).
#ifdef VECCHIA_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

}  // namespace vecchia

// The C ABI's opaque plan handle is a Plan.
struct vecchia_plan : public vecchia::Plan {};

#define VECCHIA_CUDA_TRY(expr)                        \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return VECCHIA_ECUDA;      \
  } while (0)

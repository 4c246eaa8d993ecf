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
  double* d_partial = nullptr;  // per-warp partial sums
  int64_t partial_cap = 0;
  unsigned long long* d_errloc = nullptr;  // first failing location (ULLONG_MAX = none)
  cudaStream_t last_stream = nullptr;
  // covariance tables, cached by nu
  static constexpr int kCache = 4;
  double cache_nu[kCache] = {0, 0, 0, 0};
  double* cache_tab[kCache] = {nullptr, nullptr, nullptr, nullptr};
  int cache_next = 0;
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

// True iff d is a positive finite double, decided on the bit pattern (no FP64 op).
__device__ __forceinline__ bool positive_finite(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0 && b < 0x7FF0000000000000LL;
}

struct Neumaier {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

}  // namespace vecchia

// The C ABI's opaque plan handle is a Plan.
struct vecchia_plan : public vecchia::Plan {};

#define VECCHIA_CUDA_TRY(expr)                        \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return VECCHIA_ECUDA;      \
  } while (0)

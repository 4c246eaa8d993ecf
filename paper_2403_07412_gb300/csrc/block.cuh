// One ordered location's Vecchia term, computed by one warp in shared memory
// (Sec. V-B, Algorithm 1), shared by the single-field and the batched kernels.
//
// For location i with conditioning set J (m_i = min(i, m) real neighbours, the rest
// identity padding) the warp builds the bordered (K+1) x (K+1) lower triangle, K = m + 1,
//
//        rows 0..m-1 : neighbours J (pads: identity rows)       | border row K:
//        row  m      : the location itself                        |   y_B
//     M = [ R_B + gamma I      .  ]    R_B = correlation block, gamma = tau2/sigma2
//         [ y_B^T              0  ]
//
// and runs K-1 steps of an in-place L D L^T elimination over the neighbour columns.
// What remains in the trailing 2x2 corner is exactly Algorithm 1's correction:
//   M[m][m] = s_i / sigma2   (conditional variance, lines 20 and 23),
//   M[K][m] = y_i - mu_i      (conditional residual, lines 16-19 and 22),
// so the batched POTRF, the two TRSVs and the two dot products of Algorithm 1 become
// one elimination of the bordered block, and the univariate term (line 24)
//   l_i = -1/2 (y_i - mu_i)^2 / s_i - 1/2 log s_i - 1/2 log 2 pi.
//
// Storage: the triangle is packed column by column from the last column (K) to the
// first, so the columns still to be updated at step j form a prefix [0, off(j)),
// off(c) = (K-c)(K-c+1)/2.  Every FP64 instruction is issued with as many active lanes
// as the trailing prefix allows; pivots use one reciprocal (no square root).
//
// Adjoint (not in the paper).  With w = Sigma_JJ^{-1} v, alpha = Sigma_JJ^{-1} y_J,
// r = y_i - mu_i and s = s_i, write w^ = [-w; 1], a^ = [alpha; 0] and
//   g = (r/s) a^ + 1/2 (r^2/s^2 - 1/s) w^.
// Then dl_i/dtheta_p = w^T (dSigma_B/dtheta_p) g, hence
//   dl_i/dtau2   = w^T g,
//   dl_i/dsigma2 = (1/2 (r^2/s - 1) - tau2 w^T g) / sigma2   (uses Sigma_B w^ = s e_i),
//   dl_i/dbeta   = -(2 sigma2/beta) sum_{p>q} h(u_pq) (w^_p g_q + w^_q g_p),
// where h = u rho'(u).  w and alpha come from two backward solves with the unit
// factor already in shared memory (rows m and K of L are L_J^{-1}-scaled v and y_J).
#pragma once

#include "common.cuh"
#include "matern.cuh"

namespace vecchia {

__host__ __device__ __forceinline__ int tri_off(int K, int c) { return (K - c) * (K - c + 1) / 2; }

__host__ __device__ __forceinline__ int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Schedule sizes for block size K (= m + 1): NT packed slots, NP correlation pairs.
struct SchedSize {
  int NT, NP, sched_bytes, pairs_bytes;
  __host__ __device__ explicit SchedSize(int K) {
    NT = (K + 1) * (K + 2) / 2;
    NP = K * (K - 1) / 2;
    sched_bytes = align_up(NT * 2, 16);
    pairs_bytes = align_up(NP * 4, 16);
  }
};

// Whether the gradient kernel with G lanes per location may gather the block's
// coordinates a second time after the elimination, so that its block fits the forward
// kernel's two vectors (the launch decides, see shape_for in loglik.cu).  With 8 lanes
// (m = 16..31) shared memory can limit the warps per SM: at n = 1M, fwd + grad at m = 25
// went from 13.48 to 12.54 ms (12 -> 16 warps per SM) and at m = 30 from 21.80 to 21.07
// ms (10 -> 12), but at m = 31 (10 -> 11 warps) from 22.24 to 22.33 ms and at m = 20
// (16 warps either way) from 7.69 to 8.05 ms.  With 32 lanes the second gather costs more
// than the thirteenth warp gains (m = 60: 99.0 -> 102.3 ms; m = 45: 48.2 -> 50.0 ms), and
// with 4 lanes the registers, not shared memory, limit the warps.
__host__ __device__ constexpr bool regather_capable(bool grad, int G) { return grad && G == 8; }

// Per-warp shared-memory area for blocks up to size K: the packed triangle A and the
// block rows' coordinates CX, CY (float pairs; on the sphere a third array CZ follows CY).
// The elimination's two column buffers TV and TV1 hold the unscaled entries of columns j
// and j+1:
//  - forward kernel (and the gradient kernel where it gathers twice, see
//    regather_capable): they reuse CX and CY, which are dead after the assembly, and the
//    data go straight into A's border row, so a block takes two vectors besides A (at
//    m = 60, 16.6 KB instead of 17.6 KB: thirteen 32-lane blocks fit on an SM instead of
//    twelve).  The adjoint's weight vectors w^ and g (float pairs) then sit at the start
//    of A once the backward solves have read the factor;
//  - gradient kernel otherwise: TV and TV1 are separate (TV1 holds the data until the
//    assembly), and after the elimination w^ and g take their places.
struct WarpArea {
  double* A;
  float2 *CX, *CY, *CZ;
  double *TV, *TV1;   // elimination: unscaled entries of columns j and j+1
  float2 *WHf, *GVf;  // gradient, after the elimination: w^ and g as float pairs
  bool regather;      // gradient: coordinates gathered again after the elimination
  __host__ __device__ static bool separate(bool grad, int G, bool regather) {
    return grad && !(regather && regather_capable(grad, G));
  }
  __host__ __device__ static int doubles(int K, bool grad, int G, bool sphere = false, bool regather = false) {
    const SchedSize S(K);
    const bool sep = separate(grad, G, regather);
    return align_up(S.NT, 2) + ((sphere ? 3 : 2) + (sep ? 2 : 0)) * align_up(K + 1, 2);
  }
  __device__ WarpArea(double* base, int K, bool grad, int G, bool sphere = false, bool regather_ = false) {
    const SchedSize S(K);
    const int V = align_up(K + 1, 2);
    regather = regather_ && regather_capable(grad, G);
    A = base;
    CX = reinterpret_cast<float2*>(A + align_up(S.NT, 2));
    CY = CX + V;
    CZ = sphere ? CY + V : CY;
    if (separate(grad, G, regather)) {
      TV = reinterpret_cast<double*>(CY + (sphere ? 2 : 1) * V);
      TV1 = TV + V;
      WHf = reinterpret_cast<float2*>(TV1);
      GVf = reinterpret_cast<float2*>(TV);
    } else {
      TV = reinterpret_cast<double*>(CX);
      TV1 = reinterpret_cast<double*>(CY);
      WHf = reinterpret_cast<float2*>(A);  // K entries each; 2K <= NT for every K >= 2
      GVf = WHf + K;
    }
  }
};

// Stride, in doubles, between the areas of a warp's 32/G location groups: the area
// (WarpArea::doubles) plus 16 bytes where the groups would otherwise start on the same
// shared-memory banks.  The groups run one instruction stream, so each access of a warp
// touches the same slot of every group's area; with 8 lanes and an area that is a
// multiple of 128 bytes (m = 16, 27, 29, 30 among others) the four groups' 64-bit
// accesses met on 16 of the 32 banks, four wavefronts where two serve (4 lanes: a
// multiple of 64 bytes puts eight groups on 16 banks).
__host__ __device__ inline int group_doubles(int K, bool grad, int G, bool sphere = false, bool regather = false) {
  const int d = WarpArea::doubles(K, grad, G, sphere, regather);
  const int bytes = 8 * d;
  return ((G == 8 && bytes % 128 == 0) || (G == 4 && bytes % 64 == 0)) ? d + 2 : d;
}

// Element schedules for block size K: sched[e] = (row, col) of packed slot e;
// pairs[q] = (row, col, slot) of the q-th strictly-lower pair of the K x K block.
__device__ __forceinline__ void build_schedules(int K, uint16_t* sched, uint32_t* pairs) {
  for (int c = threadIdx.x; c <= K; c += blockDim.x) {
    const int o = tri_off(K, c);
    for (int r = c; r <= K; ++r) sched[o + r - c] = (uint16_t)(r | (c << 8));
    if (c < K - 1) {
      const int base = (K - 1 - c) * (K - 2 - c) / 2;
      for (int r = c + 1; r <= K - 1; ++r)
        pairs[base + r - c - 1] = (uint32_t)r | ((uint32_t)c << 8) | ((uint32_t)(o + r - c) << 16);
    }
  }
}

// theta-dependent constants of one evaluation.  inv_len scales distances so that
// u = (d inv_len)^2 is the table's variable: 1/beta for the Matérn, beta^(-1/alpha) for
// the power exponential; dbeta_coef turns h = u rho'(u) into dC/dbeta / 1:
// -2 sigma2 / beta (Matérn) or -2 sigma2 / (alpha beta) (power exponential).
struct ThetaConst {
  double sigma2, inv_len, gamma1, inv_sigma2, tau2, dbeta_coef;
  __device__ void set(double s2, double beta, double t2, int family, double nu) {
    sigma2 = s2;
    const bool pe = family == kFamilyPowExp;
    inv_len = pe ? exp(-log(beta) / nu) : 1.0 / beta;
    dbeta_coef = -2.0 * s2 / (beta * (pe ? nu : 1.0));
    gamma1 = 1.0 + t2 / s2;
    inv_sigma2 = 1.0 / s2;
    tau2 = t2;
  }
};

// Running sums of a warp.  The log-likelihood is kept as its parts,
//   sum l_i = -1/2 sum r_i^2/s_i - 1/2 log(prod s_i) - (count) 1/2 log 2 pi,
// with prod s_i held as a mantissa in [1, 2) and an integer binary exponent, so one
// log per warp replaces one per location (identical on all lanes).  Also
// sum 1/2 (r^2/s - 1), and the per-lane partial sums of the beta pair sums and of w^T g.
struct Accum {
  Neumaier Q;
  double P = 1.0;
  long long PE = 0;
  long long count = 0;
  double S = 0.0, B = 0.0, T = 0.0;
  __device__ __forceinline__ void mul_s(double s) {
    const long long b = __double_as_longlong(P * s);
    PE += ((b >> 52) & 0x7FF) - 1023;
    P = __longlong_as_double((b & 0xFFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  }
  __device__ __forceinline__ double loglik() const {
    return -0.5 * Q.value() - 0.5 * (log(P) + 0.69314718055994530942 * (double)PE) -
           0.91893853320467274178 * (double)count;
  }
};

// Field description: device arrays of one field and its plan.
struct FieldView {
  const double2* __restrict__ xy;   // n, original order
  const double* __restrict__ yf;    // n, original order
  const int32_t* __restrict__ nbr;  // n x m original indices
  const int32_t* __restrict__ self; // n
  int64_t n;
  int m;
  // indices into xy / yf must lie in [0, nidx); checked before use when check_idx (a
  // warp-uniform flag) or in a bounds-checked build
  int64_t nidx = 0;
  bool check_idx = false;
  // great-circle distances: unit vectors (n x 3, original order) and K2 = (2 r / len)^2,
  // with len the family's length scale, as a float pair and in FP64
  const double* __restrict__ xyz = nullptr;
  bool sphere = false;
  float2 k2 = make_float2(0.0f, 0.0f);
  double k2d = 0.0;
  // prediction: every location has m conditioning points (all observed points qualify),
  // y of the location itself is 0 (unknown), and the conditional mean and variance are
  // written to pmean / pvar (n each) instead of likelihood terms
  double* pmean = nullptr;
  double* pvar = nullptr;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lanes of a group of G lanes (G divides 32): shuffles and reductions stay in the group.
template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Processes ordered location i of field F with a group of G lanes (sub = lane within
// the group); the 32/G groups of a warp run the same instruction stream on different
// locations, so every loop below has a trip count that depends on K only and no group
// leaves early; inactive groups (active = false) compute a valid location and discard
// it.  When terms_mode (the same for the whole warp), terms (if not null) receives l_i,
// or {l_i, dl_i/dsigma2, dl_i/dbeta, dl_i/dtau2} when GRAD.  A block that is not positive definite gives a NaN term and records i in errloc.
// x as a float pair hi + lo (hi: x's leading 24 bits, lo: the next 24, about 2^-48
// relative), with integer operations; exponents far from 0 take the FP64 route.
__device__ __forceinline__ float2 d2f_pair(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -90 || e > 90) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
  // remainder: mantissa bits 28..5, v 2^(e-47) = (v 2^-24) 2^(e-23)
  const float lo = fscale(u24_float((unsigned)(b >> 5) & 0xFFFFFFu), e - 23);
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

// x as a float pair (hi: x's leading 24 bits, lo: the next 24), by integer operations
// only; |x| below 2^-100 gives (0, 0).  For values of moderate exponent (factor entries).
__device__ __forceinline__ float2 d2f_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
  const float lo = fscale(u24_float((unsigned)(b >> 5) & 0xFFFFFFu), e - 23);
  const bool z = e < -100;
  return make_float2(z ? 0.0f : hi, z ? 0.0f : __uint_as_float(__float_as_uint(lo) | sign));
}

// (h, l) -= (a.x + a.y)(b.x + b.y) in double-float arithmetic (about 2^-46 relative).
__device__ __forceinline__ void df_fms(float& h, float& l, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float pe = fmaf(a.x, b.x, -p);
  pe = fmaf(a.x, b.y, pe);
  pe = fmaf(a.y, b.x, pe);
  float s, e;
  two_sum(h, -p, s, e);
  e = __fadd_rn(e, __fsub_rn(l, pe));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// Squared distance of two block points held as float pairs (x = hi + lo, about 2^-48
// relative), in double-float arithmetic on the FP32 pipe: (uh, ul) within about 2^-46
// of |p_r - p_c|^2 relative, plus 2^-47 of the block's coordinate scale in |p_r - p_c|.
// A covariance entry needs absolute accuracy, and |drho/du| |du| stays far below the
// factorisation's own rounding.  (An exact square of 64-bit integer coordinates costs
// ~70 integer instructions at half rate; this costs ~41 full-rate FP32 ones.)
__device__ __forceinline__ void df_diff(float2 a, float2 b, float& h, float& l) {
  float s, e;
  two_sum(a.x, -b.x, s, e);
  e = __fadd_rn(e, __fsub_rn(a.y, b.y));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

__device__ __forceinline__ void sq_dist_df(float2 xr, float2 xc, float2 yr, float2 yc, float& uh, float& ul) {
  float dxh, dxl, dyh, dyl;
  df_diff(xr, xc, dxh, dxl);
  df_diff(yr, yc, dyh, dyl);
  const float px = __fmul_rn(dxh, dxh), py = __fmul_rn(dyh, dyh);
  float ex = fmaf(dxh, dxh, -px), ey = fmaf(dyh, dyh, -py);
  ex = fmaf(dxh + dxh, dxl, ex);
  ey = fmaf(dyh + dyh, dyl, ey);
  float s, e;
  two_sum(px, py, s, e);
  e = __fadd_rn(e, __fadd_rn(ex, ey));
  uh = __fadd_rn(s, e);
  ul = __fsub_rn(e, __fsub_rn(uh, s));
}

// Squared chord between two points on the unit sphere held as float-pair offsets, in
// double-float arithmetic (as sq_dist_df, with three coordinates).
__device__ __forceinline__ void sq_chord_df(float2 xr, float2 xc, float2 yr, float2 yc, float2 zr, float2 zc,
                                            float& ch, float& cl) {
  float dxh, dxl, dyh, dyl, dzh, dzl;
  df_diff(xr, xc, dxh, dxl);
  df_diff(yr, yc, dyh, dyl);
  df_diff(zr, zc, dzh, dzl);
  const float px = __fmul_rn(dxh, dxh), py = __fmul_rn(dyh, dyh), pz = __fmul_rn(dzh, dzh);
  float ex = fmaf(dxh, dxh, -px), ey = fmaf(dyh, dyh, -py), ez = fmaf(dzh, dzh, -pz);
  ex = fmaf(dxh + dxh, dxl, ex);
  ey = fmaf(dyh + dyh, dyl, ey);
  ez = fmaf(dzh + dzh, dzl, ez);
  float s1, e1, s2, e2;
  two_sum(px, py, s1, e1);
  two_sum(s1, pz, s2, e2);
  float e = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(ex, ey), ez));
  ch = __fadd_rn(s2, e);
  cl = __fsub_rn(e, __fsub_rn(ch, s2));
}

// u = K2 asin^2(c / 2) from the squared chord c^2 = ch + cl of two unit vectors: the
// great-circle distance d = 2 r asin(c / 2) (Sec. VI-C), over the length scale, squared.
// With w = c^2 / 4, asin^2(sqrt(w)) = w + w^2 T(w), T(w) = 1/3 + 8w/45 + 4w^2/35 +
// 128w^3/1575 + 128w^4/2079 (the series sum_k 2^(2k-1) w^k / (k^2 C(2k,k))), whose
// next term is below 2^-50 w for w <= 2^-10, i.e. chords up to 1/16 of the radius;
// longer chords take FP64 asin.  Double-float arithmetic otherwise, as sq_dist_df.
__device__ __forceinline__ void sphere_u_df(float ch, float cl, const FieldView& F, float& uh, float& ul) {
  const float wh = ch * 0.25f, wl = cl * 0.25f;
  if (wh > 0x1p-10f) {
    const double a = asin(sqrt(f2d_scaled(wh, 0) + f2d_scaled(wl, 0)));
    const float2 u = d2f_pair(F.k2d * a * a);
    uh = u.x;
    ul = u.y;
    return;
  }
  constexpr float kThirdH = 1.0f / 3.0f;
  constexpr float kThirdL = (float)(1.0 / 3.0 - (double)(1.0f / 3.0f));
  constexpr float k845H = 8.0f / 45.0f;
  constexpr float k845L = (float)(8.0 / 45.0 - (double)(8.0f / 45.0f));
  const float r = fmaf(fmaf(128.0f / 2079.0f, wh, 128.0f / 1575.0f), wh, 4.0f / 35.0f);
  float t1h, t1l, s, e;
  df_mul(wh, wl, k845H, k845L, t1h, t1l);
  two_sum(kThirdH, t1h, s, e);
  e = __fadd_rn(e, __fadd_rn(__fadd_rn(t1l, kThirdL), __fmul_rn(__fmul_rn(wh, wh), r)));
  const float th = __fadd_rn(s, e), tl = __fsub_rn(e, __fsub_rn(th, s));
  float ah, al, bh, bl;
  df_mul(wh, wl, th, tl, ah, al);  // w T
  df_mul(wh, wl, ah, al, bh, bl);  // w^2 T
  two_sum(wh, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(wl, bl));
  const float vh = __fadd_rn(s, e), vl = __fsub_rn(e, __fsub_rn(vh, s));
  df_mul(F.k2.x, F.k2.y, vh, vl, uh, ul);
}

// u of the pair (r, c) of the block, plane or sphere (a compile-time choice, so that the
// planar kernels carry no trace of the sphere path).
template <bool SPHERE>
__device__ __forceinline__ void pair_u(const FieldView& F, const float2* __restrict__ CX,
                                       const float2* __restrict__ CY, const float2* __restrict__ CZ, int r, int c,
                                       float& uh, float& ul) {
  if constexpr (SPHERE) {
    float ch, cl;
    sq_chord_df(CX[r], CX[c], CY[r], CY[c], CZ[r], CZ[c], ch, cl);
    sphere_u_df(ch, cl, F, uh, ul);
  } else {
    sq_dist_df(CX[r], CX[c], CY[r], CY[c], uh, ul);
  }
}

// (pbh, pbl) += h (w_r g_c + w_c g_r) in double-float arithmetic.
__device__ __forceinline__ void beta_pair_add(float2 wr, float2 wc, float2 gr, float2 gc, float hh, float hl,
                                              float& pbh, float& pbl) {
  float ah, al, bh, bl, s, e;
  df_mul(wr.x, wr.y, gc.x, gc.y, ah, al);
  df_mul(wc.x, wc.y, gr.x, gr.y, bh, bl);
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  const float th = __fadd_rn(s, e);
  const float tl = __fsub_rn(e, __fsub_rn(th, s));
  float ph, pl;
  df_mul(hh, hl, th, tl, ph, pl);
  two_sum(pbh, ph, s, e);
  e = __fadd_rn(e, __fadd_rn(pl, pbl));
  pbh = __fadd_rn(s, e);
  pbl = __fsub_rn(e, __fsub_rn(pbh, s));
}

// The adjoint's beta pair sums of one location: this lane's share of
// sum_{p>q} h(u_pq) (w^_p g_q + w^_q g_p), with h recomputed from the block's float-pair
// coordinates (pads carry zero weights).  Lane `sub` of the G lanes takes pairs
// q = sub + G k, in increasing k; w^ and g are float pairs (WHf, GVf).  One pair per
// iteration: fewer live registers than two (n = 1M, m = 60, l + grad 101.2 -> 99.3 ms;
// at n = 250k, m = 20, 2.03 -> 1.98 ms), with the same sums.
template <int G, bool SPHERE>
__device__ __forceinline__ double beta_pass(const FieldView& F, int NP, const uint32_t* __restrict__ pairs,
                                            const float2* __restrict__ CX, const float2* __restrict__ CY,
                                            const float2* __restrict__ CZ, const float2* __restrict__ WHf,
                                            const float2* __restrict__ GVf, const double* __restrict__ tab,
                                            const MaternConst& mc, int sub) {
  float pbh = 0.0f, pbl = 0.0f;
  for (int q0 = sub; q0 < NP; q0 += G) {
    const uint32_t w0 = pairs[q0];
    const int r0 = w0 & 0xFF, c0 = (w0 >> 8) & 0xFF;
    float u0h, u0l, h0h, h0l;
    pair_u<SPHERE>(F, CX, CY, CZ, r0, c0, u0h, u0l);
    h_df(u0h, u0l, tab, mc, h0h, h0l);
    beta_pair_add(WHf[r0], WHf[c0], GVf[r0], GVf[c0], h0h, h0l, pbh, pbl);
  }
  return f2d_scaled(pbh, 0) + f2d_scaled(pbl, 0);
}

// Offsets of neighbour j from the location js: centred, 1/beta-scaled plane coordinates,
// or unit-vector differences on the sphere (the length scale enters through K2 there).
template <bool SPHERE>
__device__ __forceinline__ void coord_offsets(const FieldView& F, const ThetaConst& tc, double2 ps, int js, int j,
                                              double& xv, double& yv, double& zv) {
  if constexpr (SPHERE) {
    xv = F.xyz[3 * j] - F.xyz[3 * js];
    yv = F.xyz[3 * j + 1] - F.xyz[3 * js + 1];
    zv = F.xyz[3 * j + 2] - F.xyz[3 * js + 2];
  } else {
    const double2 q = F.xy[j];
    xv = (q.x - ps.x) * tc.inv_len;
    yv = (q.y - ps.y) * tc.inv_len;
  }
}

// Returns whether the location's term is valid (positive definite block, finite data,
// indices in range).
template <bool GRAD, int G, bool SPHERE>
__device__ __forceinline__ bool process_location(int64_t i, bool active, const FieldView& F, const SchedSize& S,
                                                 const uint16_t* __restrict__ sched,
                                                 const uint32_t* __restrict__ pairs, const WarpArea& W,
                                                 const double* __restrict__ tab, const MaternConst& mc,
                                                 const ThetaConst& tc, Accum& acc, bool terms_mode,
                                                 double* terms, unsigned long long* errloc, int sub) {
  constexpr int KCAP = max_k_for_lanes(G);
  constexpr int NSG = (KCAP - 1 + G - 1) / G;  // neighbour slots per lane (m <= KCAP - 1)
  const int m = F.m;
  const int K = m + 1;
  double* __restrict__ A = W.A;
  float2* __restrict__ CX = W.CX;
  float2* __restrict__ CY = W.CY;
  float2* __restrict__ CZ = W.CZ;
  double* __restrict__ TV = W.TV;
  const int mi = (i < m && !F.pmean) ? (int)i : m;
  const int32_t* __restrict__ row = F.nbr + i * m;
  const bool check = kChecked || F.check_idx;
  bool bad_idx = false;
  int js = F.self[i];
  if (check && (unsigned long long)(int64_t)js >= (unsigned long long)F.nidx) {
    bad_idx = true;
    js = 0;
  }
  const double2 ps = F.xy[js];
  // ---- gather: centred, 1/beta-scaled coordinates (as float pairs), and the data: with
  // two vectors per block straight into the border row K of A (slot tri_off(K, c) + K - c;
  // the location's own y lands in A[2]), with separate column buffers into TV1, copied to
  // the border by the assembly (that order measured 1% faster there)
  const bool regather = regather_capable(GRAD, G) && W.regather;  // warp-uniform
  const bool sep_buffers = GRAD && !regather;
#pragma unroll
  for (int s = 0; s < NSG; ++s) {
    const int p = sub + G * s;
    if (p < m) {
      double xv = 0.0, yv = 0.0, zv = 0.0, fv = 0.0;
      if (p < mi) {
        int j = row[p];
        if (check && (unsigned long long)(int64_t)j >= (unsigned long long)F.nidx) {
          bad_idx = true;
          j = 0;
        }
        coord_offsets<SPHERE>(F, tc, ps, js, j, xv, yv, zv);
        fv = F.yf[j];
      }
      if (sep_buffers) {
        W.TV1[p] = fv;
      } else {
        A[tri_off(K, p) + K - p] = fv;
      }
      CX[p] = d2f_pair(xv);
      CY[p] = d2f_pair(yv);
      if constexpr (SPHERE) CZ[p] = d2f_pair(zv);
    }
  }
  if (sub == 0) {
    CX[m] = make_float2(0.0f, 0.0f);
    CY[m] = make_float2(0.0f, 0.0f);
    if constexpr (SPHERE) CZ[m] = make_float2(0.0f, 0.0f);
    if (sep_buffers) {
      W.TV1[m] = F.yf[js];
    } else {
      A[tri_off(K, m) + K - m] = F.yf[js];
    }
  }
  if (check) {  // a bad index anywhere in the group fails the group's block
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    bad_idx = (__ballot_sync(0xffffffffu, bad_idx) & gmask) != 0u;
  }
  __syncwarp();
  // ---- assemble: diagonal (and, with separate column buffers, the data border), then
  // the correlation pairs
  for (int c = sub; c < K; c += G) {
    const int o = tri_off(K, c);
    A[o] = (c >= mi && c < m) ? 1.0 : tc.gamma1;
    if (sep_buffers) A[o + K - c] = W.TV1[c];
  }
  if (sub == 0) A[0] = 0.0;
  // Two pairs per lane per iteration so one pair's loads overlap the other's FMAs.
  for (int q0 = sub; q0 < S.NP; q0 += 2 * G) {
    const int q1 = q0 + G;
    const bool has1 = q1 < S.NP;
    const uint32_t w0 = pairs[q0];
    const uint32_t w1 = has1 ? pairs[q1] : w0;
    const int r0 = w0 & 0xFF, c0 = (w0 >> 8) & 0xFF;
    const int r1 = w1 & 0xFF, c1 = (w1 >> 8) & 0xFF;
    const bool v0 = c0 < mi && (r0 < mi || r0 == m);
    const bool v1 = has1 && c1 < mi && (r1 < mi || r1 == m);
    float u0h, u0l, u1h, u1l;
    pair_u<SPHERE>(F, CX, CY, CZ, r0, c0, u0h, u0l);
    pair_u<SPHERE>(F, CX, CY, CZ, r1, c1, u1h, u1l);
    const double val0 = rho_df(u0h, u0l, tab, mc), val1 = rho_df(u1h, u1l, tab, mc);
    A[w0 >> 16] = v0 ? val0 : 0.0;
    if (has1) A[w1 >> 16] = v1 ? val1 : 0.0;
  }
  __syncwarp();
  // ---- L D L^T over the neighbour columns, two columns per step: column j, then column
  // j+1 updated by column j and scaled, then one pass over the remaining prefix applying
  // both (fma(-L1, T1, fma(-L0, T0, a)): the same roundings, in the same order, as two
  // single-column steps, with half the column transitions and shared-memory passes).
  bool ok = true;
  double* __restrict__ TV1 = W.TV1;  // column j+1's unscaled entries
  // Column scaling by the pivot reciprocal: the integer round-to-nearest-even product
  // (mul_by_positive, bit-identical to the DMUL) in the full-warp forward kernel, where
  // it keeps an FP64 instruction off the column step's serial path (n = 1M, m = 60:
  // 89.5 -> 86.4 ms), and in the 4-lane forward kernel (m = 10: 1.266 -> 1.245 ms); the
  // DMUL in the gradient kernel, whose double-float adjoint leaves the FP64 queue shorter
  // (103.4 -> 100.0 ms with the DMUL), and in 8- and 16-lane groups (2.5% faster at
  // m = 30).
  constexpr bool kIntScale = (G == 32 || G == 4) && !GRAD;
  int j = 0;
  for (; j + 2 < K; j += 2) {
    const int oj = tri_off(K, j), o1 = tri_off(K, j + 1);
    const double d0 = A[oj];
    ok = ok && pivot_in_range(d0);  // a failed block runs on (values unused) to stay in step
    const double inv0 = rcp_fixed(d0);
    for (int r = j + 1 + sub; r <= K; r += G) {
      const double tv = A[oj + r - j];
      TV[r] = tv;
      if constexpr (kIntScale) {
        A[oj + r - j] = mul_by_positive(tv, inv0);
      } else {
        A[oj + r - j] = tv * inv0;
      }
    }
    __syncwarp();
    const double* L0 = A + oj - j;  // L0[r] = L[r][j]
    {
      const double t0 = TV[j + 1];
      for (int r = j + 1 + sub; r <= K; r += G) {
        const int e = o1 + r - j - 1;
        A[e] = fma(-L0[r], t0, A[e]);
      }
    }
    __syncwarp();
    const double d1 = A[o1];
    ok = ok && pivot_in_range(d1);
    const double inv1 = rcp_fixed(d1);
    for (int r = j + 2 + sub; r <= K; r += G) {
      const double tv = A[o1 + r - j - 1];
      TV1[r] = tv;
      if constexpr (kIntScale) {
        A[o1 + r - j - 1] = mul_by_positive(tv, inv1);
      } else {
        A[o1 + r - j - 1] = tv * inv1;
      }
    }
    __syncwarp();
    const double* L1 = A + o1 - j - 1;  // L1[r] = L[r][j+1]
    constexpr int U = 4;
    const int nfull = (o1 - 1) / (G * U);
    const int tail0 = 1 + G * U * nfull;
    // Forward kernel: the remainder slots [tail0, o1) (fewer than G U) go first, their
    // loads and FMAs issued ahead of the full batches and their results stored after
    // them, so each remainder chain's latency overlaps the batches' FMAs (slots are
    // disjoint: the same values as any other order).  Measured on GB300 at n = 1M,
    // m = 60: forward 86.9 -> 86.1 ms; in the gradient kernel the extra registers cost
    // more than the overlap gains (103.5 -> 108.5 ms), so there the remainder runs last.
    constexpr bool kTailFirst = !GRAD;
    double tres[U];
    if constexpr (kTailFirst) {
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (tail0 + G * k >= o1) break;  // uniform over the warp
        const int e = tail0 + sub + G * k;
        if (e < o1) {
          const uint32_t rc = sched[e];
          const int r = rc & 0xFF, c = rc >> 8;
          tres[k] = fma(-L1[r], TV1[c], fma(-L0[r], TV[c], A[e]));
        }
      }
    }
    if (nfull > 0) {
      double l0[U], t0[U], l1[U], t1[U], av[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const uint32_t rc = sched[1 + sub + G * k];
        l0[k] = L0[rc & 0xFF];
        l1[k] = L1[rc & 0xFF];
        t0[k] = TV[rc >> 8];
        t1[k] = TV1[rc >> 8];
        av[k] = A[1 + sub + G * k];
      }
      for (int bt = 0; bt < nfull; ++bt) {
        const int base = 1 + sub + G * U * bt;
        double res[U];
#pragma unroll
        for (int k = 0; k < U; ++k) res[k] = fma(-l0[k], t0[k], av[k]);
#pragma unroll
        for (int k = 0; k < U; ++k) res[k] = fma(-l1[k], t1[k], res[k]);
        if (bt + 1 < nfull) {
#pragma unroll
          for (int k = 0; k < U; ++k) {
            const int e = base + G * (U + k);
            const uint32_t rc = sched[e];
            l0[k] = L0[rc & 0xFF];
            l1[k] = L1[rc & 0xFF];
            t0[k] = TV[rc >> 8];
            t1[k] = TV1[rc >> 8];
            av[k] = A[e];
          }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) A[base + G * k] = res[k];
      }
    }
    if constexpr (kTailFirst) {
#pragma unroll
      for (int k = 0; k < U; ++k) {
        if (tail0 + G * k >= o1) break;
        const int e = tail0 + sub + G * k;
        if (e < o1) A[e] = tres[k];
      }
    } else {
      for (int e = tail0 + sub; e < o1; e += G) {
        const uint32_t rc = sched[e];
        const int r = rc & 0xFF, c = rc >> 8;
        A[e] = fma(-L1[r], TV1[c], fma(-L0[r], TV[c], A[e]));
      }
    }
    __syncwarp();
  }
  if (j < K - 1) {  // an odd number of neighbour columns: the last one alone
    const int oj = tri_off(K, j);
    const double d = A[oj];
    ok = ok && pivot_in_range(d);  // a failed block runs on (values unused) to stay in step
    const double inv = rcp_fixed(d);
    for (int r = j + 1 + sub; r <= K; r += G) {
      const double tv = A[oj + r - j];
      TV[r] = tv;
      // integer product in the full-warp forward kernel (no wait behind other warps'
      // FP64 work on the column step's serial path); DMUL elsewhere (kIntScale)
      if constexpr (kIntScale) {
        A[oj + r - j] = mul_by_positive(tv, inv);
      } else {
        A[oj + r - j] = tv * inv;
      }
    }
    __syncwarp();
    // Trailing update of the prefix [1, oj).  Full batches of eight slots per lane are
    // software-pipelined (the next batch's shared-memory loads are issued before this
    // batch's results are stored); the remainder runs one slot at a time, so no FP64
    // instruction is issued for a slot that no lane owns.
    const double* Lc = A + oj - j;  // Lc[r] = L[r][j]
    constexpr int U = 8;
    const int nfull = (oj - 1) / (G * U);
    const int tail0 = 1 + G * U * nfull;
    if (nfull > 0) {
      double lv[U], tv[U], av[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const uint32_t rc = sched[1 + sub + G * k];
        lv[k] = Lc[rc & 0xFF];
        tv[k] = TV[rc >> 8];
        av[k] = A[1 + sub + G * k];
      }
      for (int bt = 0; bt < nfull; ++bt) {
        const int base = 1 + sub + G * U * bt;
        double res[U];
#pragma unroll
        for (int k = 0; k < U; ++k) res[k] = fma(-lv[k], tv[k], av[k]);
        if (bt + 1 < nfull) {
#pragma unroll
          for (int k = 0; k < U; ++k) {
            const int e = base + G * (U + k);
            const uint32_t rc = sched[e];
            lv[k] = Lc[rc & 0xFF];
            tv[k] = TV[rc >> 8];
            av[k] = A[e];
          }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) A[base + G * k] = res[k];
      }
    }
    for (int e = tail0 + sub; e < oj; e += G) {
      const uint32_t rc = sched[e];
      A[e] = fma(-Lc[rc & 0xFF], TV[rc >> 8], A[e]);
    }
    __syncwarp();
  }
  const double st = A[1];  // s_i / sigma2
  const double rr = A[2];  // y_i - mu_i
  // The pivots and s_i depend on the covariance only, the residual on the data: a
  // non-finite residual (with a positive definite block) means a non-finite y in B_i.
  const bool pd = ok && positive_finite(st);
  const bool good = pd && finite_bits(rr) && !bad_idx;
  const double nan = __longlong_as_double(0x7FF8000000000000LL);
  const double s = tc.sigma2 * st;
  const double inv_s = rcp_newton(s);
  const double q = rr * rr * inv_s;
  if (active) {
    if (good) {
      acc.Q.add(q);
      acc.mul_s(s);
      acc.count += 1;
    } else {
      acc.Q.add(nan);
      if (sub == 0 && !F.pmean) atomicMin(errloc, err_code(i, bad_idx ? kErrIndex : (pd ? kErrData : kErrNotPD)));
    }
    if (F.pmean && sub == 0) {
      // y_i = 0 here, so rr = -mu; a variance of 0 (prediction at an observed point
      // without nugget) is valid, so only a failed neighbour factorisation, a bad index
      // or non-finite data gives NaN
      const bool pok = ok && !bad_idx && finite_bits(rr);
      F.pmean[i] = pok ? -rr : nan;
      if (F.pvar) F.pvar[i] = pok ? fmax(s, 0.0) : nan;
      if (!pok) atomicMin(errloc, err_code(i, bad_idx ? kErrIndex : (ok ? kErrData : kErrNotPD)));
    }
  }
  // per-location terms (test and inspection path) pay for their own log
  const double li = terms_mode ? (good ? -0.5 * q - 0.5 * log(s) - 0.91893853320467274178 : nan) : 0.0;
  if (!GRAD) {
    if (terms && active && sub == 0) terms[0] = li;
    __syncwarp();
    return good;
  }
  // ---- adjoint: with two vectors per block, the coordinates again first (the
  // elimination used CX and CY as its column buffers; the same values as the first
  // gather); then w = L_J^{-T} (row m of L) and alpha~ = L_J^{-T} (row K of L)
  if (regather) {
#pragma unroll
    for (int s = 0; s < NSG; ++s) {
      const int p = sub + G * s;
      if (p < m) {
        double xv = 0.0, yv = 0.0, zv = 0.0;
        if (p < mi) {
          int j = row[p];
          if (check && (unsigned long long)(int64_t)j >= (unsigned long long)F.nidx) j = 0;
          coord_offsets<SPHERE>(F, tc, ps, js, j, xv, yv, zv);
        }
        CX[p] = d2f_pair(xv);
        CY[p] = d2f_pair(yv);
      }
    }
    if (sub == 0) {
      CX[m] = make_float2(0.0f, 0.0f);
      CY[m] = make_float2(0.0f, 0.0f);
    }
  }
  constexpr int NS = (KCAP - 1 + G - 1) / G;  // slots of the K-1 <= KCAP-1 neighbour entries
  // The two unit backward solves run in double-float arithmetic on the FP32 pipe: each
  // step of their serial chain would otherwise wait behind the other warps' FP64 work.
  float2 wf[NS], bf[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int c = sub + G * t;
    wf[t] = make_float2(0.0f, 0.0f);
    bf[t] = make_float2(0.0f, 0.0f);
    if (c < K - 1) {
      const int o = tri_off(K, c);
      wf[t] = d2f_trunc(A[o + m - c]);
      bf[t] = d2f_trunc(A[o + K - c]);
    }
  }
  for (int c = K - 2; c >= 1; --c) {
    const int src = c % G, sl = c / G;
    float2 wsel = wf[0], bsel = bf[0];
#pragma unroll
    for (int t = 1; t < NS; ++t)
      if (sl == t) {
        wsel = wf[t];
        bsel = bf[t];
      }
    const float2 wc = make_float2(__shfl_sync(0xffffffffu, wsel.x, src, G), __shfl_sync(0xffffffffu, wsel.y, src, G));
    const float2 bc = make_float2(__shfl_sync(0xffffffffu, bsel.x, src, G), __shfl_sync(0xffffffffu, bsel.y, src, G));
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int cc = sub + G * t;
      if (cc < c) {
        const float2 l = d2f_trunc(A[tri_off(K, cc) + c - cc]);
        df_fms(wf[t].x, wf[t].y, l, wc);
        df_fms(bf[t].x, bf[t].y, l, bc);
      }
    }
  }
  double w[NS], bv[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    w[t] = f2d_scaled(wf[t].x, 0) + f2d_scaled(wf[t].y, 0);
    bv[t] = f2d_scaled(bf[t].x, 0) + f2d_scaled(bf[t].y, 0);
  }
  const double rs = rr * inv_s;
  const double cb = 0.5 * (rs * rs - inv_s);
  const double rsa = rs * tc.inv_sigma2;  // alpha = alpha~ / sigma2
  // w^ and g are kept as float pairs for the beta pair sums below (double-float products
  // there: the same ~2^-46 relative precision as h(u) itself, and no FP64 instruction).
  // With two vectors per block they go to the start of A, which no lane reads any more.
  float2* __restrict__ WHf = W.WHf;
  float2* __restrict__ GVf = W.GVf;
  if (regather) __syncwarp();
  double pT = 0.0;
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int c = sub + G * t;
    if (c < K - 1) {
      const double wh = -w[t], gv = fma(rsa, bv[t], cb * wh);
      WHf[c] = d2f_pair(wh);
      GVf[c] = d2f_pair(gv);
      pT = fma(wh, gv, pT);
    }
  }
  if (sub == 0) {
    WHf[m] = make_float2(1.0f, 0.0f);
    GVf[m] = d2f_pair(cb);
    pT += cb;
  }
  const double sS = 0.5 * (rr * rs - 1.0);
  __syncwarp();
  const double pB = beta_pass<G, SPHERE>(F, S.NP, pairs, CX, CY, CZ, WHf, GVf, tab, mc, sub);
  if (terms_mode) {
    const double tB = group_sum<G>(pB), tT = group_sum<G>(pT);
    if (terms && active && sub == 0) {
      terms[0] = li;
      terms[1] = good ? (sS - tc.tau2 * tT) * tc.inv_sigma2 : nan;
      terms[2] = good ? tc.dbeta_coef * tB : nan;
      terms[3] = good ? tT : nan;
    }
  }
  if (active) {
    if (good) {
      acc.S += sS;
      acc.B += pB;
      acc.T += pT;
    } else {  // every output of a failed term is NaN
      acc.S += nan;
      acc.B += nan;
      acc.T += nan;
    }
  }
  __syncwarp();
  return good;
}

// Combines the warp's sums into the four output slots
// {l, sum 1/2(r^2/s - 1), sum of beta pair sums, sum w^T g}: per-group values are
// added over the 32/G groups in group order, per-lane partials over all lanes.
template <int G>
__device__ __forceinline__ void write_partial(Accum& acc, double* out, int lane) {
  const double B = warp_sum(acc.B);
  const double T = warp_sum(acc.T);
  const double Lg = acc.loglik();
  double L = Lg, Ssum = acc.S;
#pragma unroll
  for (int g = 1; g < 32 / G; ++g) {
    L += __shfl_sync(0xffffffffu, Lg, g * G);
    Ssum += __shfl_sync(0xffffffffu, acc.S, g * G);
  }
  if (lane == 0) {
    out[0] = L;
    out[1] = Ssum;
    out[2] = B;
    out[3] = T;
  }
}

}  // namespace vecchia

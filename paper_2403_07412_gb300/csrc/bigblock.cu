// Large conditioning sets (m > VECCHIA_MAX_M_WARP): one CTA per location.
//
// The paper runs m up to 150 (Sec. VI-D).  A 151-row bordered block is 93 KB of packed
// FP64, too much for a warp's share of shared memory, so here a CTA of kCtaThreads
// threads owns one location at a time and runs the same elimination as block.cuh (the
// bordered L D L^T whose trailing 2x2 corner holds s_i / sigma2 and y_i - mu_i) with
// CTA-wide barriers.  The (row, column) of a packed slot or a pair index is decoded
// arithmetically (a triangular-number inverse) instead of from schedule tables, which
// keeps two CTAs resident per SM.  The adjoint's two backward solves run on the first two
// warps, one each, on vectors in shared memory; everything else is spread over all
// threads.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "block.cuh"
#include "common.cuh"
#include "matern.cuh"

namespace vecchia {

constexpr int kCtaThreads = 128;     // default CTA size (4 warps)
constexpr int kCtaThreadsMax = 256;  // when fewer than 4 CTAs fit on an SM

struct BigArgs {
  const double* __restrict__ xy;
  const double* __restrict__ yf;
  const int32_t* __restrict__ nbr;
  const int32_t* __restrict__ self;
  const double* __restrict__ tab;
  int64_t n;
  int m;
  int family;
  double sigma2, beta, nu, tau2;
  double* partial;  // [gridDim.x][4]
  double* terms;
  unsigned long long* errloc;
  const double* __restrict__ xyz;  // n x 3 unit vectors (sphere plans)
  int metric;                      // 0 plane, 1 sphere
  double radius;
  int64_t i0, i1;                  // ordered locations [i0, i1) are evaluated
};

// Largest w with w(w+1)/2 <= e (e < 2^24).
__device__ __forceinline__ int tri_root(int e) {
  int w = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  if ((w + 1) * (w + 2) / 2 <= e) ++w;
  if (w * (w + 1) / 2 > e) --w;
  return w;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

// B columns j..j+B-1 of the bordered L D L^T, CTA-wide.  Each column in turn is scaled by
// its pivot's reciprocal (its unscaled entries kept in TVs[q]) and applied to the later
// columns of the group; then one pass over the remaining prefix [1, o_{j+B-1}) applies
// all B columns to each slot in column order, fma(-L_q T_q, .) for q = 0..B-1.  Every
// slot sees the same roundings in the same order as with single-column steps, while the
// trailing matrix is read and written once per B columns.  Returns false (uniformly over
// the CTA) at a pivot outside rcp_fixed's domain.
template <int B>
__device__ __forceinline__ bool cta_columns(double* A, double* const* TVs, int K, int j, int tid, int NTH) {
  int o[B];
#pragma unroll
  for (int q = 0; q < B; ++q) o[q] = tri_off(K, j + q);
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const double d = A[o[q]];
    if (!pivot_in_range(d)) return false;  // every thread reads the same pivot
    const double inv = rcp_fixed(d);
    double* T = TVs[q];
    for (int r = j + q + 1 + tid; r <= K; r += NTH) {
      const double tv = A[o[q] + r - j - q];
      T[r] = tv;
      A[o[q] + r - j - q] = tv * inv;
    }
    __syncthreads();
    if (q + 1 < B) {
      const double* Lq = A + o[q] - j - q;
#pragma unroll
      for (int p = q + 1; p < B; ++p) {
        const double tp = T[j + p];
        for (int r = j + p + tid; r <= K; r += NTH) {
          const int e = o[p] + r - j - p;
          A[e] = fma(-Lq[r], tp, A[e]);
        }
      }
      __syncthreads();
    }
  }
  const double* L[B];
#pragma unroll
  for (int q = 0; q < B; ++q) L[q] = A + o[q] - j - q;
  constexpr int U = 8 / B;
  const int end = o[B - 1];
  const int nfull = (end - 1) / (NTH * U);
  const int tail0 = 1 + NTH * U * nfull;
  for (int bt = 0; bt < nfull; ++bt) {
    const int base = 1 + tid + NTH * U * bt;
    double av[U];
    int rr[U], cc[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int e = base + NTH * k;
      const int w = tri_root(e);
      cc[k] = K - w;
      rr[k] = cc[k] + (e - w * (w + 1) / 2);
      av[k] = A[e];
    }
#pragma unroll
    for (int q = 0; q < B; ++q)
#pragma unroll
      for (int k = 0; k < U; ++k) av[k] = fma(-L[q][rr[k]], TVs[q][cc[k]], av[k]);
#pragma unroll
    for (int k = 0; k < U; ++k) A[base + NTH * k] = av[k];
  }
  for (int e = tail0 + tid; e < end; e += NTH) {
    const int w = tri_root(e);
    const int c = K - w, r = c + (e - w * (w + 1) / 2);
    double a = A[e];
#pragma unroll
    for (int q = 0; q < B; ++q) a = fma(-L[q][r], TVs[q][c], a);
    A[e] = a;
  }
  __syncthreads();
  return true;
}

template <bool GRAD, bool SPHERE>
__global__ void __launch_bounds__(kCtaThreadsMax) vecchia_big_kernel(const BigArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = a.m, K = m + 1;
  const int NTd = (K + 1) * (K + 2) / 2, NP = K * (K - 1) / 2;
  double* A = reinterpret_cast<double*>(smem);
  constexpr bool sphere = SPHERE;
  float2* CX = reinterpret_cast<float2*>(A + align_up(NTd, 2));
  float2* CY = CX + align_up(K + 1, 2);
  float2* CZ = sphere ? CY + align_up(K + 1, 2) : CY;
  double* YV = reinterpret_cast<double*>(CY + (sphere ? 2 : 1) * align_up(K + 1, 2));
  double* TV = YV + align_up(K + 1, 2);
  double* WH = TV + align_up(K + 1, 2);
  double* GV = WH + align_up(K + 1, 2);
  double* red = GV + align_up(K + 1, 2);
  float2* WHf = reinterpret_cast<float2*>(WH);  // w^ and g as float pairs for the beta sums
  float2* GVf = reinterpret_cast<float2*>(GV);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int NTH = blockDim.x;
  const MaternConst mc = load_matern_const(a.tab);
  ThetaConst tc;
  tc.set(a.sigma2, a.beta, a.tau2, a.family, a.nu);
  const double2* __restrict__ xy2 = reinterpret_cast<const double2*>(a.xy);
  FieldView F;  // the distance fields pair_u reads
  F.sphere = sphere;
  F.xyz = a.xyz;
  if constexpr (SPHERE) {
    const double k = 2.0 * a.radius * tc.inv_len;
    F.k2d = k * k;
    F.k2 = d2f_pair(F.k2d);
  }
  Accum acc;
  for (int64_t i = a.i0 + blockIdx.x; i < a.i1; i += gridDim.x) {
    const int mi = i < m ? (int)i : m;
    const int32_t* __restrict__ row = a.nbr + i * m;
    bool bad_idx = false;  // bounds-checked builds only: an index outside [0, n)
    int js = a.self[i];
    if (kChecked && (unsigned long long)(int64_t)js >= (unsigned long long)a.n) {
      bad_idx = true;
      js = 0;
    }
    const double2 ps = xy2[js];
    // ---- gather (two slots per thread covers m <= 2 * kCtaThreads): centred,
    // 1/beta-scaled coordinates as float pairs, and data
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int p = tid + NTH * s;
      if (p < m) {
        double xv = 0.0, yv = 0.0, zv = 0.0, fv = 0.0;
        if (p < mi) {
          int j = row[p];
          if (kChecked && (unsigned long long)(int64_t)j >= (unsigned long long)a.n) {
            bad_idx = true;
            j = 0;
          }
          if constexpr (SPHERE) {
            xv = a.xyz[3 * j] - a.xyz[3 * js];
            yv = a.xyz[3 * j + 1] - a.xyz[3 * js + 1];
            zv = a.xyz[3 * j + 2] - a.xyz[3 * js + 2];
          } else {
            const double2 q = xy2[j];
            xv = (q.x - ps.x) * tc.inv_len;
            yv = (q.y - ps.y) * tc.inv_len;
          }
          fv = a.yf[j];
        }
        YV[p] = fv;
        CX[p] = d2f_pair(xv);
        CY[p] = d2f_pair(yv);
        if constexpr (SPHERE) CZ[p] = d2f_pair(zv);
      }
    }
    if (tid == 0) {
      CX[m] = make_float2(0.0f, 0.0f);
      CY[m] = make_float2(0.0f, 0.0f);
      if constexpr (SPHERE) CZ[m] = make_float2(0.0f, 0.0f);
      YV[m] = a.yf[js];
    }
    if (kChecked) bad_idx = __syncthreads_or(bad_idx) != 0;
    __syncthreads();
    // ---- assemble
    for (int c = tid; c < K; c += NTH) {
      const int o = tri_off(K, c);
      A[o] = (c >= mi && c < m) ? 1.0 : tc.gamma1;
      A[o + K - c] = YV[c];
    }
    if (tid == 0) A[0] = 0.0;
    for (int q0 = tid; q0 < NP; q0 += 2 * NTH) {
      const int q1 = q0 + NTH;
      const bool has1 = q1 < NP;
      const int v0 = tri_root(q0), v1 = tri_root(has1 ? q1 : q0);
      const int c0 = K - 2 - v0, r0 = c0 + 1 + (q0 - v0 * (v0 + 1) / 2);
      const int qq1 = has1 ? q1 : q0;
      const int c1 = K - 2 - v1, r1 = c1 + 1 + (qq1 - v1 * (v1 + 1) / 2);
      const bool ok0 = c0 < mi && (r0 < mi || r0 == m);
      const bool ok1 = has1 && c1 < mi && (r1 < mi || r1 == m);
      float u0h, u0l, u1h, u1l;
      pair_u<SPHERE>(F, CX, CY, CZ, r0, c0, u0h, u0l);
      pair_u<SPHERE>(F, CX, CY, CZ, r1, c1, u1h, u1l);
      const double val0 = rho_df(u0h, u0l, a.tab, mc), val1 = rho_df(u1h, u1l, a.tab, mc);
      A[tri_off(K, c0) + r0 - c0] = ok0 ? val0 : 0.0;
      if (has1) A[tri_off(K, c1) + r1 - c1] = ok1 ? val1 : 0.0;
    }
    __syncthreads();
    // ---- L D L^T over the neighbour columns: CTA-wide steps of four columns (then two,
    // then one), bit-identical to single-column steps (cta_columns)
    double* TVs[4] = {TV, YV, WH, GV};  // YV, WH and GV are free during the elimination
    bool ok = true;
    int j = 0;
    for (; ok && j + 4 < K; j += 4) ok = cta_columns<4>(A, TVs, K, j, tid, NTH);
    for (; ok && j + 2 < K; j += 2) ok = cta_columns<2>(A, TVs, K, j, tid, NTH);
    if (ok && j + 1 < K) ok = cta_columns<1>(A, TVs, K, j, tid, NTH);
    const double st = A[1], rr = A[2];
    const bool pd = ok && positive_finite(st);  // a non-finite rr with pd: non-finite data
    const bool good = pd && finite_bits(rr) && !bad_idx;
    const double nan = __longlong_as_double(0x7FF8000000000000LL);
    const double s = tc.sigma2 * st;
    const double inv_s = rcp_newton(s);
    const double q = rr * rr * inv_s;
    if (good) {
      acc.Q.add(q);
      acc.mul_s(s);
      acc.count += 1;
    } else {
      acc.Q.add(nan);
      if (tid == 0) atomicMin(a.errloc, err_code(i, bad_idx ? kErrIndex : (pd ? kErrData : kErrNotPD)));
    }
    const double li = good ? -0.5 * q - 0.5 * log(s) - 0.91893853320467274178 : nan;
    if (!GRAD) {
      if (a.terms && tid == 0) a.terms[i] = li;
      __syncthreads();
      continue;
    }
    // ---- adjoint: the two backward solves on warps 0 (w) and 1 (alpha~) at once, then
    // the pair pass on all threads
    const double rs = rr * inv_s;
    const double cb = 0.5 * (rs * rs - inv_s);
    const double rsa = rs * tc.inv_sigma2;
    double pT = 0.0;
    if (wid < 2 && good) {
      // Double-float solves on the FP32 pipe, as in the warp kernels: each step of the
      // serial chain would otherwise wait behind the other CTAs' FP64 work.  Warp 0
      // solves with row m of the factor (w) in TV, warp 1 with row K (alpha~) in YV (both
      // free after the elimination).  The vectors live in shared memory, not registers:
      // held in registers they took the kernel from 80 to 122 registers per thread and
      // one CTA per SM of occupancy at m = 90 and 120.
      float2* V = reinterpret_cast<float2*>(wid == 0 ? TV : YV);
      const int row = wid == 0 ? m : K;
      for (int c = lane; c < K - 1; c += 32) V[c] = d2f_trunc(A[tri_off(K, c) + row - c]);
      __syncwarp();
      for (int c = K - 2; c >= 1; --c) {
        const float2 vc = V[c];  // final since the previous step (__syncwarp below)
        for (int cc = lane; cc < c; cc += 32) {
          const float2 l = d2f_trunc(A[tri_off(K, cc) + c - cc]);
          float2 v = V[cc];
          df_fms(v.x, v.y, l, vc);
          V[cc] = v;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (wid == 0 && good) {
      const float2* Vw = reinterpret_cast<const float2*>(TV);
      const float2* Va = reinterpret_cast<const float2*>(YV);
      for (int c = lane; c < K - 1; c += 32) {
        const double w = f2d_scaled(Vw[c].x, 0) + f2d_scaled(Vw[c].y, 0);
        const double al = f2d_scaled(Va[c].x, 0) + f2d_scaled(Va[c].y, 0);
        const double wh = -w, gv = fma(rsa, al, cb * wh);
        WHf[c] = d2f_pair(wh);
        GVf[c] = d2f_pair(gv);
        pT = fma(wh, gv, pT);
      }
      if (lane == 0) {
        WHf[m] = make_float2(1.0f, 0.0f);
        GVf[m] = d2f_pair(cb);
        pT += cb;
      }
    }
    __syncthreads();
    float pbh = 0.0f, pbl = 0.0f;
    if (good) {  // one pair per iteration (two took more registers, no less time)
      for (int q0 = tid; q0 < NP; q0 += NTH) {
        const int v0 = tri_root(q0);
        const int c0 = K - 2 - v0, r0 = c0 + 1 + (q0 - v0 * (v0 + 1) / 2);
        float u0h, u0l, h0h, h0l;
        pair_u<SPHERE>(F, CX, CY, CZ, r0, c0, u0h, u0l);
        h_df(u0h, u0l, a.tab, mc, h0h, h0l);
        beta_pair_add(WHf[r0], WHf[c0], GVf[r0], GVf[c0], h0h, h0l, pbh, pbl);
      }
    }
    const double pB = f2d_scaled(pbh, 0) + f2d_scaled(pbl, 0);
    const double sS = 0.5 * (rr * rs - 1.0);
    if (a.terms) {
      const double tB = block_sum(pB, red), tT = block_sum(pT, red);
      if (tid == 0) {
        double* o = a.terms + i * 4;
        o[0] = li;
        o[1] = good ? (sS - tc.tau2 * tT) * tc.inv_sigma2 : nan;
        o[2] = good ? tc.dbeta_coef * tB : nan;
        o[3] = good ? tT : nan;
      }
    }
    if (good) {
      acc.S += sS;
      acc.B += pB;
      acc.T += pT;
    } else {  // every output of a failed term is NaN
      acc.S += nan;
      acc.B += nan;
      acc.T += nan;
    }
    __syncthreads();
  }
  const double B = block_sum(acc.B, red);
  const double T = block_sum(acc.T, red);
  if (tid == 0) {
    double* o = a.partial + (int64_t)blockIdx.x * 4;
    o[0] = acc.loglik();
    o[1] = acc.S;
    o[2] = B;
    o[3] = T;
  }
}

// Shared memory of the CTA kernel for block size K.
int big_smem_bytes(int K, bool sphere) {
  const int NTd = (K + 1) * (K + 2) / 2;
  return 8 * (align_up(NTd, 2) + (sphere ? 7 : 6) * align_up(K + 1, 2) + 32 + 16);
}

// CTA size: 128 threads while at least 4 CTAs fit on an SM (more locations in flight),
// else 256 so that the SM still holds 512 threads.  Measured on GB300 at n = 100k:
// m = 90 (6 CTAs/SM) 128 threads 1.35x faster than 256; m = 150 (2 CTAs/SM) 256
// threads 1.34x faster than 128.  VECCHIA_CTA_THREADS = 128 or 256 forces one.
int big_config(int K, bool grad, int* blocks, int* threads, int* smem, bool sphere) {
  int dev = 0, sms = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  *smem = big_smem_bytes(K, sphere);
  auto kern = grad ? (sphere ? vecchia_big_kernel<true, true> : vecchia_big_kernel<true, false>)
                   : (sphere ? vecchia_big_kernel<false, true> : vecchia_big_kernel<false, false>);
  VECCHIA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, *smem));
  const char* e = getenv("VECCHIA_CTA_THREADS");
  const int forced = e ? atoi(e) : 0;
  int t = (forced == 128 || forced == 256) ? forced : kCtaThreads;
  int per_sm = 0;
  VECCHIA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, t, *smem));
  if (forced != 128 && forced != 256 && per_sm * t < 512) {
    int per_sm2 = 0;
    VECCHIA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, kern, kCtaThreadsMax, *smem));
    if (per_sm2 >= 1) {
      t = kCtaThreadsMax;
      per_sm = per_sm2;
    }
  }
  if (per_sm < 1) return VECCHIA_EINVAL;
  *blocks = per_sm * sms;
  *threads = t;
  return VECCHIA_OK;
}

void launch_big(bool grad, int blocks, int threads, int smem, const BigArgs& a, cudaStream_t s) {
  const bool sph = a.metric == 1;
  if (grad) {
    if (sph) vecchia_big_kernel<true, true><<<blocks, threads, smem, s>>>(a);
    else vecchia_big_kernel<true, false><<<blocks, threads, smem, s>>>(a);
  } else {
    if (sph) vecchia_big_kernel<false, true><<<blocks, threads, smem, s>>>(a);
    else vecchia_big_kernel<false, false><<<blocks, threads, smem, s>>>(a);
  }
}

}  // namespace vecchia

// Fused Vecchia log-likelihood and adjoint kernels (Sec. V-B, Algorithm 1).
//
// One warp owns one ordered location i at a time and keeps everything about it in
// shared memory; nothing per location is written to global memory.  For location i
// with conditioning set J (m_i = min(i, m) real neighbours, the rest identity padding)
// the warp builds the bordered (K+1) x (K+1) lower triangle, K = m + 1,
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
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "matern.cuh"

namespace vecchia {

int get_matern_table(double nu, cudaStream_t stream, const double** out);
int launch_matern_table(double nu, double* tab, cudaStream_t stream);
bool theta_ok(const double* th);

struct LikArgs {
  const double* __restrict__ xy;     // n x 2, original order
  const double* __restrict__ yf;     // n, original order
  const int32_t* __restrict__ nbr;   // n x m original indices
  const int32_t* __restrict__ self;  // n
  const double* __restrict__ tab;    // correlation table for nu
  int64_t n;
  int m;
  double sigma2, beta, tau2;
  double* partial;                   // [nwarps][4]
  double* terms;                     // optional [n][1|4]
  unsigned long long* errloc;
};

__host__ __device__ __forceinline__ int tri_off(int K, int c) { return (K - c) * (K - c + 1) / 2; }

__host__ __device__ __forceinline__ int align_up(int x, int a) { return (x + a - 1) / a * a; }

// Shared-memory layout for block size K (= m + 1) and W warps per CTA.
struct SmemLayout {
  int NT, NP, sched_bytes, pairs_bytes, per_warp_doubles;
  __host__ __device__ SmemLayout(int K, bool grad) {
    NT = (K + 1) * (K + 2) / 2;
    NP = K * (K - 1) / 2;
    sched_bytes = align_up(NT * 2, 16);
    pairs_bytes = align_up(NP * 4, 16);
    // A[NT], X, Y, YV, TV [K+1 each]; grad: H[NP], WH, GV [K+1 each]
    per_warp_doubles = align_up(NT, 2) + 4 * align_up(K + 1, 2);
    if (grad) per_warp_doubles += align_up(NP, 2) + 2 * align_up(K + 1, 2);
  }
  __host__ __device__ int bytes(int W) const { return sched_bytes + pairs_bytes + W * per_warp_doubles * 8; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool GRAD>
__global__ void __launch_bounds__(384) vecchia_lik_kernel(const LikArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = a.m;
  const int K = m + 1;
  const SmemLayout L(K, GRAD);
  uint16_t* sched = reinterpret_cast<uint16_t*>(smem);
  uint32_t* pairs = reinterpret_cast<uint32_t*>(smem + L.sched_bytes);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  double* A = reinterpret_cast<double*>(smem + L.sched_bytes + L.pairs_bytes) + wib * L.per_warp_doubles;
  double* X = A + align_up(L.NT, 2);
  double* Y = X + align_up(K + 1, 2);
  double* YV = Y + align_up(K + 1, 2);
  double* TV = YV + align_up(K + 1, 2);
  double* H = TV + align_up(K + 1, 2);
  double* WH = H + align_up(L.NP, 2);
  double* GV = WH + align_up(K + 1, 2);

  // Element schedules, shared by the CTA: sched[e] = (row, col) of packed slot e;
  // pairs[q] = (row, col, slot) of the q-th strictly-lower pair of the K x K block.
  for (int c = threadIdx.x; c <= K; c += blockDim.x) {
    const int o = tri_off(K, c);
    for (int r = c; r <= K; ++r) sched[o + r - c] = (uint16_t)(r | (c << 8));
    if (c < K - 1) {
      const int base = (K - 1 - c) * (K - 2 - c) / 2;
      for (int r = c + 1; r <= K - 1; ++r)
        pairs[base + r - c - 1] = (uint32_t)r | ((uint32_t)c << 8) | ((uint32_t)(o + r - c) << 16);
    }
  }
  __syncthreads();

  const MaternConst mc = load_matern_const(a.tab);
  const double sigma2 = a.sigma2;
  const double inv_beta = 1.0 / a.beta;
  const double gamma1 = 1.0 + a.tau2 / sigma2;
  const double inv_sigma2 = 1.0 / sigma2;
  const double half_log2pi = 0.91893853320467274178;
  const double2* __restrict__ xy2 = reinterpret_cast<const double2*>(a.xy);
  const int64_t gw = (int64_t)blockIdx.x * W + wib;
  const int64_t nw = (int64_t)gridDim.x * W;

  Neumaier accL;            // sum of l_i (identical on every lane)
  double accS = 0.0;        // sum of 1/2 (r^2/s - 1)
  double accB = 0.0;        // per-lane partial of the beta pair sums
  double accT = 0.0;        // per-lane partial of w^T g

  for (int64_t i = gw; i < a.n; i += nw) {
    const int mi = i < m ? (int)i : m;
    const int32_t* __restrict__ row = a.nbr + i * m;
    const int js = a.self[i];
    const double2 ps = xy2[js];
    // ---- gather: centred, 1/beta-scaled coordinates and data of the block rows
    for (int p = lane; p < m; p += 32) {
      double xv = 0.0, yv = 0.0, fv = 0.0;
      if (p < mi) {
        const int j = row[p];
        const double2 q = xy2[j];
        xv = (q.x - ps.x) * inv_beta;
        yv = (q.y - ps.y) * inv_beta;
        fv = a.yf[j];
      }
      X[p] = xv;
      Y[p] = yv;
      YV[p] = fv;
    }
    if (lane == 0) {
      X[m] = 0.0;
      Y[m] = 0.0;
      YV[m] = a.yf[js];
    }
    __syncwarp();
    // ---- assemble: diagonal, data border, then the correlation pairs
    for (int c = lane; c < K; c += 32) {
      const int o = tri_off(K, c);
      A[o] = (c >= mi && c < m) ? 1.0 : gamma1;
      A[o + K - c] = YV[c];
    }
    if (lane == 0) A[0] = 0.0;
    // Two pairs per lane per iteration so one pair's loads overlap the other's FMAs.
    for (int q0 = lane; q0 < L.NP; q0 += 64) {
      const int q1 = q0 + 32;
      const bool has1 = q1 < L.NP;
      const uint32_t w0 = pairs[q0];
      const uint32_t w1 = has1 ? pairs[q1] : w0;
      const int r0 = w0 & 0xFF, c0 = (w0 >> 8) & 0xFF;
      const int r1 = w1 & 0xFF, c1 = (w1 >> 8) & 0xFF;
      const bool v0 = c0 < mi && (r0 < mi || r0 == m);
      const bool v1 = has1 && c1 < mi && (r1 < mi || r1 == m);
      const double dx0 = X[r0] - X[c0], dy0 = Y[r0] - Y[c0];
      const double dx1 = X[r1] - X[c1], dy1 = Y[r1] - Y[c1];
      const double u0 = fma(dx0, dx0, dy0 * dy0), u1 = fma(dx1, dx1, dy1 * dy1);
      double val0, hv0 = 0.0, val1, hv1 = 0.0;
      rho_poly<GRAD>(u0, a.tab, val0, hv0);
      rho_poly<GRAD>(u1, a.tab, val1, hv1);
      rho_fix(u0, mc, val0, hv0);
      rho_fix(u1, mc, val1, hv1);
      if (!v0) { val0 = 0.0; hv0 = 0.0; }
      if (!v1) { val1 = 0.0; hv1 = 0.0; }
      A[w0 >> 16] = val0;
      if (GRAD) H[q0] = hv0;
      if (has1) {
        A[w1 >> 16] = val1;
        if (GRAD) H[q1] = hv1;
      }
    }
    __syncwarp();
    // ---- L D L^T over the neighbour columns
    bool ok = true;
    for (int j = 0; j < K - 1; ++j) {
      const int oj = tri_off(K, j);
      const double d = A[oj];
      if (!positive_finite(d)) { ok = false; break; }
      const double inv = rcp_newton(d);
      for (int r = j + 1 + lane; r <= K; r += 32) {
        const double tv = A[oj + r - j];
        TV[r] = tv;
        A[oj + r - j] = tv * inv;
      }
      __syncwarp();
      // Trailing update of the prefix [1, oj), four slots per lane per batch: the next
      // batch's shared-memory loads are issued before this batch's results are stored.
      const double* Lc = A + oj - j;  // Lc[r] = L[r][j]
      constexpr int U = 4;
      double lv[U], tv[U], av[U];
      int ee[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        ee[k] = 1 + lane + 32 * k;
        const int ek = ee[k] < oj ? ee[k] : 0;
        const uint32_t rc = sched[ek];
        lv[k] = Lc[rc & 0xFF];
        tv[k] = TV[rc >> 8];
        av[k] = A[ek];
      }
      for (int base = 1 + lane; base < oj; base += 32 * U) {
        double res[U];
#pragma unroll
        for (int k = 0; k < U; ++k) res[k] = fma(-lv[k], tv[k], av[k]);
        int ne[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          ne[k] = base + 32 * (U + k);
          const int ek = ne[k] < oj ? ne[k] : 0;
          const uint32_t rc = sched[ek];
          lv[k] = Lc[rc & 0xFF];
          tv[k] = TV[rc >> 8];
          av[k] = A[ek];
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          if (ee[k] < oj) A[ee[k]] = res[k];
          ee[k] = ne[k];
        }
      }
      __syncwarp();
    }
    const double st = A[1];   // s_i / sigma2
    const double rr = A[2];   // y_i - mu_i
    if (!ok || !positive_finite(st)) {
      if (lane == 0) {
        atomicMin(a.errloc, (unsigned long long)i);
        if (a.terms) {
          const int tw = GRAD ? 4 : 1;
          for (int k = 0; k < tw; ++k) a.terms[i * tw + k] = __longlong_as_double(0x7FF8000000000000LL);
        }
      }
      accL.add(__longlong_as_double(0x7FF8000000000000LL));
      __syncwarp();
      continue;
    }
    const double s = sigma2 * st;
    const double inv_s = rcp_newton(s);
    const double li = -0.5 * rr * rr * inv_s - 0.5 * log(s) - half_log2pi;
    accL.add(li);
    if (!GRAD) {
      if (a.terms && lane == 0) a.terms[i] = li;
      __syncwarp();
      continue;
    }
    // ---- adjoint: w = L_J^{-T} (row m of L), alpha~ = L_J^{-T} (row K of L)
    double w0 = 0.0, w1 = 0.0, b0 = 0.0, b1 = 0.0;
    const int c0 = lane, c1 = lane + 32;
    if (c0 < K - 1) { const int o = tri_off(K, c0); w0 = A[o + m - c0]; b0 = A[o + K - c0]; }
    if (c1 < K - 1) { const int o = tri_off(K, c1); w1 = A[o + m - c1]; b1 = A[o + K - c1]; }
    for (int c = K - 2; c >= 1; --c) {
      const int src = c & 31;
      const double wc = __shfl_sync(0xffffffffu, c >= 32 ? w1 : w0, src);
      const double bc = __shfl_sync(0xffffffffu, c >= 32 ? b1 : b0, src);
      if (c0 < c) {
        const double l = A[tri_off(K, c0) + c - c0];
        w0 = fma(-l, wc, w0);
        b0 = fma(-l, bc, b0);
      }
      if (c1 < c) {
        const double l = A[tri_off(K, c1) + c - c1];
        w1 = fma(-l, wc, w1);
        b1 = fma(-l, bc, b1);
      }
    }
    const double rs = rr * inv_s;
    const double cb = 0.5 * (rs * rs - inv_s);
    const double rsa = rs * inv_sigma2;  // alpha = alpha~ / sigma2
    double pT = 0.0;
    if (c0 < K - 1) {
      const double wh = -w0, gv = fma(rsa, b0, cb * wh);
      WH[c0] = wh; GV[c0] = gv; pT = fma(wh, gv, pT);
    }
    if (c1 < K - 1) {
      const double wh = -w1, gv = fma(rsa, b1, cb * wh);
      WH[c1] = wh; GV[c1] = gv; pT = fma(wh, gv, pT);
    }
    if (lane == 0) { WH[m] = 1.0; GV[m] = cb; pT += cb; }
    const double sS = 0.5 * (rr * rs - 1.0);
    accS += sS;
    __syncwarp();
    double pB = 0.0;
    for (int q = lane; q < L.NP; q += 32) {
      const uint32_t w = pairs[q];
      const int r = w & 0xFF, c = (w >> 8) & 0xFF;
      double t = WH[r] * GV[c];
      t = fma(WH[c], GV[r], t);
      pB = fma(H[q], t, pB);
    }
    if (a.terms) {
      const double tB = warp_sum(pB), tT = warp_sum(pT);
      if (lane == 0) {
        double* o = a.terms + i * 4;
        o[0] = li;
        o[1] = (sS - a.tau2 * tT) * inv_sigma2;
        o[2] = -2.0 * sigma2 * inv_beta * tB;
        o[3] = tT;
      }
    }
    accB += pB;
    accT += pT;
    __syncwarp();
  }
  accB = warp_sum(accB);
  accT = warp_sum(accT);
  if (lane == 0) {
    double* o = a.partial + gw * 4;
    o[0] = accL.value();
    o[1] = accS;
    o[2] = accB;
    o[3] = accT;
  }
}

// Deterministic reduction of the per-warp partials (fixed order, Neumaier).
__global__ void vecchia_finalize_kernel(const double* __restrict__ partial, int64_t nw, double sigma2,
                                        double beta, double tau2, int want_grad, double* out) {
  if (threadIdx.x >= 4) return;
  const int k = threadIdx.x;
  Neumaier acc;
  for (int64_t w = 0; w < nw; ++w) acc.add(partial[w * 4 + k]);
  const double v = acc.value();
  if (!want_grad) {
    if (k == 0) out[0] = v;
    return;
  }
  // Partials: [sum l_i, sum 1/2(r^2/s-1), sum beta pair sums, sum w^T g].
  __shared__ double sv[4];
  sv[k] = v;
  __syncwarp(0xFu);
  if (k == 0) out[0] = sv[0];
  if (k == 1) out[1] = (sv[1] - tau2 * sv[3]) / sigma2;
  if (k == 2) out[2] = -2.0 * sigma2 / beta * sv[2];
  if (k == 3) out[3] = sv[3];
}

// ------------------------------------------------------------------ launch
namespace {
struct LaunchCfg {
  int W = 4, blocks = 0, smem = 0;
};

int pick_config(int K, bool grad, LaunchCfg* cfg) {
  int dev = 0, sms = 0, smem_optin = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const SmemLayout L(K, grad);
  int best_warps = -1;
  // Warps per CTA: the candidate giving the most resident warps per SM wins (ties go
  // to the larger CTA).  VECCHIA_WARPS_PER_CTA forces one value (tuning experiments).
  const char* fenv = getenv("VECCHIA_WARPS_PER_CTA");
  const int forced = fenv ? atoi(fenv) : 0;
  const int cand_all[] = {12, 10, 8, 6, 4, 2, 1};
  for (int W : cand_all) {
    if (forced > 0 && W != forced) continue;
    const int bytes = L.bytes(W);
    if (bytes > smem_optin) continue;
    auto kern = grad ? vecchia_lik_kernel<true> : vecchia_lik_kernel<false>;
    VECCHIA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int per_sm = 0;
    VECCHIA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, bytes));
    const int warps = std::min(per_sm * W, 16);
    if (per_sm > 0 && warps > best_warps) {
      best_warps = warps;
      cfg->W = W;
      cfg->blocks = per_sm * sms;
      cfg->smem = bytes;
    }
  }
  if (best_warps <= 0) return VECCHIA_EINVAL;
  auto kern = grad ? vecchia_lik_kernel<true> : vecchia_lik_kernel<false>;
  VECCHIA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cfg->smem));
  return VECCHIA_OK;
}
}  // namespace

int launch_loglik(Plan* p, const double* y_dev, const double* theta, bool grad, double* out_dev,
                  double* terms_dev, cudaStream_t stream) {
  if (!p || !y_dev || !theta_ok(theta) || (!out_dev && !terms_dev)) return VECCHIA_EINVAL;
  const int K = p->m + 1;
  LaunchCfg cfg;
  int rc = pick_config(K, grad, &cfg);
  if (rc) return rc;
  const int64_t nw = (int64_t)cfg.blocks * cfg.W;
  if (p->partial_cap < nw * 4) {
    if (p->d_partial) cudaFree(p->d_partial);
    p->d_partial = nullptr;
    p->partial_cap = 0;
    if (cudaMalloc(&p->d_partial, sizeof(double) * nw * 4) != cudaSuccess) return VECCHIA_ENOMEM;
    p->partial_cap = nw * 4;
  }
  const double* tab = nullptr;
  rc = get_matern_table(theta[2], stream, &tab);
  if (rc) return rc;
  VECCHIA_CUDA_TRY(cudaMemsetAsync(p->d_errloc, 0xFF, sizeof(unsigned long long), stream));
  LikArgs a;
  a.xy = p->d_xy;
  a.yf = y_dev;
  a.nbr = p->d_nbr;
  a.self = p->d_self;
  a.tab = tab;
  a.n = p->n;
  a.m = p->m;
  a.sigma2 = theta[0];
  a.beta = theta[1];
  a.tau2 = theta[3];
  a.partial = p->d_partial;
  a.terms = terms_dev;
  a.errloc = p->d_errloc;
  if (grad) vecchia_lik_kernel<true><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
  else vecchia_lik_kernel<false><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  if (out_dev) {
    vecchia_finalize_kernel<<<1, 32, 0, stream>>>(p->d_partial, nw, theta[0], theta[1], theta[3], grad ? 1 : 0,
                                                  out_dev);
    VECCHIA_CUDA_TRY(cudaGetLastError());
  }
  p->last_stream = stream;
  return VECCHIA_OK;
}

}  // namespace vecchia

// ------------------------------------------------------------------ allocation-free entry
// Scratch for vecchia_loglik_noalloc: per-warp partial sums for at most
// kNoAllocWarps warps, the error slot and one covariance table, in a file-scope device
// array that every GPU loading the library holds until the process exits.
namespace vecchia {
constexpr int kNoAllocWarps = 4096;
constexpr size_t kNoAllocPartialBytes = sizeof(double) * 4 * kNoAllocWarps;
constexpr size_t kNoAllocErrOff = kNoAllocPartialBytes;
constexpr size_t kNoAllocTabOff = kNoAllocErrOff + 256;
constexpr size_t kNoAllocBytes = kNoAllocTabOff + (kTableBytes + 255) / 256 * 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device;
// the host-side symbol is only a stand-in and must never be passed to a kernel).
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return VECCHIA_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VECCHIA_ECUDA;
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return VECCHIA_OK;
}
}  // namespace
}  // namespace vecchia

extern "C" int vecchia_loglik_noalloc(const double* xy_dev, const double* y_dev, const int32_t* nbr_dev,
                                      const int32_t* self_dev, int64_t n, int32_t m, const double theta[4],
                                      double* out_dev, void* stream) {
  using namespace vecchia;
  if (!xy_dev || !y_dev || !nbr_dev || !self_dev || !out_dev || n < 1 || n > 2147483647LL || m < 1 ||
      m > kMaxM || !theta_ok(theta))
    return VECCHIA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  double* partial = reinterpret_cast<double*>(base);
  unsigned long long* errloc = reinterpret_cast<unsigned long long*>(base + kNoAllocErrOff);
  double* tab = reinterpret_cast<double*>(base + kNoAllocTabOff);
  LaunchCfg cfg;
  rc = pick_config(m + 1, false, &cfg);
  if (rc) return rc;
  // The kernel is persistent (warps stride over locations), so any grid covers any n;
  // it is capped to the warps the scratch can hold.
  const int max_blocks = kNoAllocWarps / cfg.W;
  if (cfg.blocks > max_blocks) cfg.blocks = max_blocks;
  const int64_t nw = (int64_t)cfg.blocks * cfg.W;
  rc = launch_matern_table(theta[2], tab, s);
  if (rc) return rc;
  VECCHIA_CUDA_TRY(cudaMemsetAsync(errloc, 0xFF, sizeof(unsigned long long), s));
  LikArgs a;
  a.xy = xy_dev;
  a.yf = y_dev;
  a.nbr = nbr_dev;
  a.self = self_dev;
  a.tab = tab;
  a.n = n;
  a.m = m;
  a.sigma2 = theta[0];
  a.beta = theta[1];
  a.tau2 = theta[3];
  a.partial = partial;
  a.terms = nullptr;
  a.errloc = errloc;
  vecchia_lik_kernel<false><<<cfg.blocks, cfg.W * 32, cfg.smem, s>>>(a);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  vecchia_finalize_kernel<<<1, 32, 0, s>>>(partial, nw, theta[0], theta[1], theta[3], 0, out_dev);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  return VECCHIA_OK;
}

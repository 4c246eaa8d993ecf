// Construction of the per-nu Matérn correlation table and the stand-alone covariance
// evaluator (vecchia_matern).
//
// rho(u) = 2^{1-nu}/Gamma(nu) x^nu K_nu(x), u = x^2, is computed at the table nodes from
// the integral representation K_nu(z) = (z/2)^nu / 2 int_0^inf exp(-t - z^2/(4t)) t^{-nu-1} dt
// (DLMF 10.32.10).  Substituting t = z^2/(4s) and s = e^tau gives
//   rho(u) = I(u) / I(0),   I(u) = int_R exp(nu tau - e^tau - (u/4) e^{-tau}) dtau,
// (I(0) = Gamma(nu)).  The integrand is analytic in the strip |Im tau| < pi/2 and decays
// double-exponentially, so the trapezoidal rule converges geometrically; the step is
// set from the curvature at the peak and from nu, and terms are summed with Neumaier
// compensation until they fall below e^-45 of the peak.
// Each interval's polynomial is the degree-kDeg Chebyshev interpolant at the
// first-kind Chebyshev points, converted to monomials in t and stored in the split
// FP64/FP32 layout that matern.cuh evaluates.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "matern.cuh"

namespace vecchia {

// I(u) by the trapezoidal rule, computed by a whole warp: lane l takes nodes k = k0 + l
// of each chunk of 32 on either side of the peak; a side ends after the first chunk that
// reaches a node below e^-45 of the peak (the log-integrand is concave, so the tail only
// falls from there).  Each lane keeps a compensated sum; the lanes' sums are merged by a
// fixed shuffle tree and lane 0's result is returned on every lane.  (One FP64
// instruction costs a warp as much with 1 lane active as with 32, so a single thread's
// serial loop would take 32 times longer.)  All 32 lanes must call it together.
__device__ double quad_I_warp(double u, double nu) {
  const int lane = threadIdx.x & 31;
  const double a = 0.25 * u;
  const double et = 0.5 * (nu + sqrt(nu * nu + 4.0 * a));  // e^tau at the peak
  const double tc = log(et);
  const double curv = et + a / et;                          // -(log integrand)'' at the peak
  const double h = fmin(0.2, fmin(0.6 / sqrt(curv), 0.3 / fmax(nu, 1.0)));
  const double lpeak = nu * tc - et - a / et;
  Neumaier acc;
  for (int side = 0; side < 2; ++side) {
    for (int k0 = side; k0 < 200000; k0 += 32) {
      const int k = k0 + lane;
      const double tau = side == 0 ? tc + k * h : tc - k * h;
      const double e = exp(tau);
      const double lv = nu * tau - e - a / e;
      acc.add(exp(lv - lpeak));
      if (__any_sync(0xffffffffu, lv - lpeak < -45.0 && k > 3)) break;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_down_sync(0xffffffffu, acc.s, o);
    const double c2 = __shfl_down_sync(0xffffffffu, acc.c, o);
    acc.merge(s2, c2);
  }
  return __shfl_sync(0xffffffffu, acc.value(), 0) * h * exp(lpeak);
}

// One warp: I(0) and the small-u expansion constants (family Matérn), or the exponent
// (power exponential).
__global__ void matern_const_kernel(double nu, int family, double* tab) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const double I0 = family == kFamilyPowExp ? 1.0 : quad_I_warp(0.0, nu);
  if (threadIdx.x != 0) return;
  double* c = tab + 2 * kIntWords * kNInt;
  if (family == kFamilyPowExp) {
    c[0] = __longlong_as_double(3LL);
    c[1] = nu;
    c[2] = c[3] = c[4] = c[5] = 0.0;
    c[6] = 1.0;
    c[7] = 0.0;
    return;
  }
  const bool integer = (nu == floor(nu));
  long long kind = integer ? (nu == 1.0 ? 1 : 2) : 0;
  c[0] = __longlong_as_double(kind);
  c[1] = nu;
  if (integer) {
    c[2] = nu == 1.0 ? 0.0 : -0.25 / (nu - 1.0);
    c[3] = c[4] = c[5] = 0.0;
  } else {
    c[2] = 0.25 / (1.0 - nu);
    c[3] = tgamma(1.0 - nu);
    c[4] = 1.0 / tgamma(1.0 + nu);
    c[5] = 0.25 / tgamma(2.0 + nu);
  }
  c[6] = I0;
  c[7] = 0.0;
}

// One block per interval, a warp per Chebyshev node.  Node values: the Matérn quadrature,
// or the power exponential exp(-u^(alpha/2)) (u = (d / beta^(1/alpha))^2) evaluated directly.
// One interval's coefficients in the layout of matern.cuh: c0 in FP64; c1..c4 and
// 3 c3 as float pairs (hi = nearest float, lo = nearest float to the rest); c5..c8,
// 5 c5, 6 c6 as floats; all floats scaled by 2^S, |max(c1..c4)| 2^S in [1/2, 1), so
// that they keep their relative precision wherever rho is small.
__device__ void split_float(double x, float* hl) {
  hl[0] = (float)x;
  hl[1] = (float)(x - (double)hl[0]);
}

__device__ void write_interval(const double* mono, float* w) {
  double top = 0.0;
  for (int k = 1; k <= 4; ++k) top = fmax(top, fabs(mono[k]));
  int S = 0;
  if (top > 0.0) {
    frexp(top, &S);
    S = -S;
  }
  double c[kDeg + 1];
  for (int k = 1; k <= kDeg; ++k) c[k] = ldexp(mono[k], S);
  split_float(c[1], w + 0);
  split_float(c[2], w + 2);
  split_float(c[3], w + 4);
  split_float(c[4], w + 6);
  for (int k = 5; k <= 8; ++k) w[8 + k - 5] = (float)c[k];
  const unsigned long long d0 = (unsigned long long)__double_as_longlong(mono[0]);
  w[12] = __uint_as_float((unsigned)(d0 & 0xFFFFFFFFULL));
  w[13] = __uint_as_float((unsigned)(d0 >> 32));
  w[14] = __int_as_float(S);
  w[15] = 0.0f;
  split_float(3.0 * c[3], w + 16);
  w[18] = (float)(5.0 * c[5]);
  w[19] = (float)(6.0 * c[6]);
}

// One CTA of kFitThreads (a warp per node) per interval.
constexpr int kFitThreads = 32 * (kDeg + 1);

__global__ void __launch_bounds__(kFitThreads) matern_fit_kernel(double nu, int family, double* tab) {
  constexpr int N = kDeg + 1;
  __shared__ double f[N], cheb[N], mono[N], tm[N][N];
  const int idx = blockIdx.x;
  const int e = kELo + (idx >> kSub);
  const int j = idx & ((1 << kSub) - 1);
  const int tid = threadIdx.x;
  const double I0 = tab[2 * kIntWords * kNInt + 6];
  const double scale = ldexp(1.0, e);
  const double mid = scale * (1.0 + (2.0 * j + 1.0) / (2.0 * (1 << kSub)));
  const double hw = scale / (2.0 * (1 << kSub));
  {  // node w = warp w: the first-kind Chebyshev point cos(pi (w + 1/2) / N)
    const int w = tid >> 5;
    const double tn = cospi((w + 0.5) / N);
    const double u = mid + hw * tn;
    const double v = family == kFamilyPowExp ? exp(-exp(0.5 * nu * log(u))) : quad_I_warp(u, nu) / I0;
    if ((tid & 31) == 0) f[w] = v;
  }
  if (tid == 0) {
    // Monomial coefficients of T_0..T_kDeg (exact small integers).
    for (int k = 0; k < N; ++k)
      for (int q = 0; q < N; ++q) tm[k][q] = 0.0;
    tm[0][0] = 1.0;
    tm[1][1] = 1.0;
    for (int k = 2; k < N; ++k)
      for (int q = 0; q < N; ++q)
        tm[k][q] = (q > 0 ? 2.0 * tm[k - 1][q - 1] : 0.0) - tm[k - 2][q];
  }
  __syncthreads();
  if (tid < N) {
    double s = 0.0;
    for (int q = 0; q < N; ++q) s += f[q] * cospi(tid * (q + 0.5) / N);
    cheb[tid] = (tid == 0 ? 1.0 : 2.0) * s / N;
  }
  __syncthreads();
  if (tid < N) {
    double a = 0.0;
    for (int k = N - 1; k >= 0; --k) a += cheb[k] * tm[k][tid];
    mono[tid] = a;
  }
  __syncthreads();
  if (tid == 0) write_interval(mono, reinterpret_cast<float*>(tab) + (size_t)idx * 4 * kIntWords);
}

// ------------------------------------------------------------------ table cache
// Tables are cached per (device, family, nu), at most kMaxTables per process; a call that
// needs a table not in the cache builds it on its own stream.  Every launch that reads a
// table records a use event on its stream afterwards (cov_table_used; one event per
// stream that used the table).  When the cache is full, the least recently used table
// that no call is between look-up and launch of is rebuilt in place: the building stream
// first waits on that table's use events, so the new contents are written only after
// every earlier reader has finished.  Nothing synchronises the device or frees memory.
namespace {
struct TableUse {
  cudaStream_t stream;
  cudaEvent_t done;
};
struct TableEntry {
  int device = -1;
  int family = 0;
  double nu = 0.0;
  double* d_tab = nullptr;
  cudaEvent_t ready = nullptr;  // recorded after the build
  std::vector<TableUse> uses;   // recorded after each launch that read the table
  int pending = 0;              // calls between get_cov_table and cov_table_used
  unsigned long long last_use = 0;
};
std::mutex g_mu;
std::vector<TableEntry> g_tables;
unsigned long long g_clock = 0;
constexpr size_t kMaxTables = 32;
constexpr size_t kMaxUseStreams = 8;
}  // namespace

// Returns (building on `stream` if needed) the device table for (family, nu) on the
// current device, and makes `stream` wait until it is built.  The caller launches its
// kernels and then calls cov_table_used(table, stream).
int get_cov_table(int family, double nu, cudaStream_t stream, const double** out) {
  int dev = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& t : g_tables) {
    if (t.device == dev && t.family == family && t.nu == nu) {
      VECCHIA_CUDA_TRY(cudaStreamWaitEvent(stream, t.ready, 0));
      t.last_use = ++g_clock;
      t.pending += 1;
      *out = t.d_tab;
      return VECCHIA_OK;
    }
  }
  TableEntry* slot = nullptr;
  TableEntry* victim = nullptr;
  for (auto& t : g_tables)  // least recently used table of this device not pinned by a call
    if (t.device == dev && t.pending == 0 && (!victim || t.last_use < victim->last_use)) victim = &t;
  if (g_tables.size() >= kMaxTables && victim) {
    // Rebuild in place once every earlier reader of the old contents has finished.
    for (const TableUse& u : victim->uses) {
      VECCHIA_CUDA_TRY(cudaStreamWaitEvent(stream, u.done, 0));
      cudaEventDestroy(u.done);
    }
    victim->uses.clear();
    slot = victim;
  } else {
    double* d = nullptr;
    if (cudaMalloc(&d, kTableBytes) != cudaSuccess) return VECCHIA_ENOMEM;
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaFree(d);
      return VECCHIA_ECUDA;
    }
    g_tables.emplace_back();
    slot = &g_tables.back();
    slot->d_tab = d;
    slot->ready = ev;
  }
  matern_const_kernel<<<1, 32, 0, stream>>>(nu, family, slot->d_tab);
  matern_fit_kernel<<<kNInt, kFitThreads, 0, stream>>>(nu, family, slot->d_tab);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  VECCHIA_CUDA_TRY(cudaEventRecord(slot->ready, stream));
  slot->device = dev;
  slot->family = family;
  slot->nu = nu;
  slot->pending = 1;
  slot->last_use = ++g_clock;
  *out = slot->d_tab;
  return VECCHIA_OK;
}

// Records that the kernels enqueued on `stream` so far have read `tab` (from
// get_cov_table), and releases the call's pin on it.
void cov_table_used(const double* tab, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& t : g_tables) {
    if (t.d_tab != tab) continue;
    if (t.pending > 0) t.pending -= 1;
    for (TableUse& u : t.uses)
      if (u.stream == stream) {
        cudaEventRecord(u.done, stream);
        return;
      }
    if (t.uses.size() >= kMaxUseStreams) {  // fold the oldest stream's use into this one
      cudaStreamWaitEvent(stream, t.uses.front().done, 0);
      cudaEventDestroy(t.uses.front().done);
      t.uses.erase(t.uses.begin());
    }
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return;
    cudaEventRecord(ev, stream);
    t.uses.push_back({stream, ev});
    return;
  }
}

int get_matern_table(double nu, cudaStream_t stream, const double** out) {
  return get_cov_table(kFamilyMatern, nu, stream, out);
}

// Builds the Matérn table for nu into caller-provided device memory (kTableBytes,
// 16-byte aligned) on `stream`, without touching the cache.
int launch_matern_table(double nu, double* tab, cudaStream_t stream) {
  matern_const_kernel<<<1, 32, 0, stream>>>(nu, kFamilyMatern, tab);
  matern_fit_kernel<<<kNInt, kFitThreads, 0, stream>>>(nu, kFamilyMatern, tab);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  return VECCHIA_OK;
}

// ------------------------------------------------------------------ vecchia_matern
// C(d) and dC/dbeta through the kernels' device code.  u = (d * inv_len)^2 with the
// family's length scale (beta for the Matérn, beta^(1/alpha) for the power
// exponential), and dC/dbeta = dcoef h(u), dcoef = -2 sigma2 / (beta a), a = 1 or alpha.
__global__ void matern_eval_kernel(const double* __restrict__ d, int64_t count, double sigma2,
                                   double beta, int family, const double* __restrict__ tab,
                                   double* __restrict__ c, double* __restrict__ dc) {
  const MaternConst mc = load_matern_const(tab);
  const double inv_len = family == kFamilyPowExp ? exp(-log(beta) / mc.nu) : 1.0 / beta;
  const double dcoef = -2.0 * sigma2 / (beta * (family == kFamilyPowExp ? mc.nu : 1.0));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = d[i] * inv_len;
    const double u = x * x;
    double rho, h;
    rho_eval<true>(u, tab, mc, rho, h);
    c[i] = sigma2 * rho;
    if (dc) dc[i] = dcoef * h;
  }
}

bool theta_ok(const double* th) {
  if (!th) return false;
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(th[k])) return false;
  return th[0] > 0.0 && th[1] > 0.0 && th[2] > 0.0 && th[3] >= 0.0;
}

// theta valid for the family: the power exponential needs 0 < alpha <= 2.
bool theta_ok_family(const double* th, int family) {
  return theta_ok(th) && (family != kFamilyPowExp || th[2] <= 2.0);
}

static int covariance(int family, const double* d_dev, int64_t count, const double* theta, double* c_dev,
                      double* dcdbeta_dev, cudaStream_t s) {
  if (count < 0 || (count > 0 && (!d_dev || !c_dev)) || !theta_ok_family(theta, family)) return VECCHIA_EINVAL;
  if (count == 0) return VECCHIA_OK;
  const double* tab = nullptr;
  int rc = get_cov_table(family, theta[2], s, &tab);
  if (rc) return rc;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  matern_eval_kernel<<<(int)blocks, 256, 0, s>>>(d_dev, count, theta[0], theta[1], family, tab, c_dev,
                                                 dcdbeta_dev);
  cov_table_used(tab, s);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  return VECCHIA_OK;
}

}  // namespace vecchia

extern "C" int vecchia_matern(const double* d_dev, int64_t count, const double theta[4], double* c_dev,
                              double* dcdbeta_dev, void* stream) {
  return vecchia::covariance(vecchia::kFamilyMatern, d_dev, count, theta, c_dev, dcdbeta_dev,
                             (cudaStream_t)stream);
}

extern "C" int vecchia_covariance(int kernel, const double* d_dev, int64_t count, const double theta[4],
                                  double* c_dev, double* dcdbeta_dev, void* stream) {
  if (kernel != VECCHIA_KERNEL_MATERN && kernel != VECCHIA_KERNEL_POWEXP) return VECCHIA_EINVAL;
  return vecchia::covariance(kernel, d_dev, count, theta, c_dev, dcdbeta_dev, (cudaStream_t)stream);
}

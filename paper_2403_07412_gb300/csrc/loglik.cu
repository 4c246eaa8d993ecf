// Single-field Vecchia log-likelihood and adjoint launches (Sec. V-B, Algorithm 1).
//
// A persistent grid of warps strides over the n ordered locations; each warp computes
// one location at a time entirely in shared memory (block.cuh) and keeps running sums,
// written once per warp and reduced in a fixed order by vecchia_finalize_kernel, so the
// result does not depend on scheduling.  Nothing per location is written to global
// memory unless per-location terms are requested.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "block.cuh"
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

// Shared-memory layout for block size K (= m + 1) and W warps per CTA.
struct SmemLayout {
  SchedSize S;
  int per_warp_doubles;
  __host__ __device__ SmemLayout(int K, bool grad) : S(K), per_warp_doubles(WarpArea::doubles(K, grad)) {}
  __host__ __device__ int bytes(int W) const { return S.sched_bytes + S.pairs_bytes + W * per_warp_doubles * 8; }
};

template <bool GRAD>
__global__ void __launch_bounds__(384) vecchia_lik_kernel(const LikArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int K = a.m + 1;
  const SmemLayout L(K, GRAD);
  uint16_t* sched = reinterpret_cast<uint16_t*>(smem);
  uint32_t* pairs = reinterpret_cast<uint32_t*>(smem + L.S.sched_bytes);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  const WarpArea area(reinterpret_cast<double*>(smem + L.S.sched_bytes + L.S.pairs_bytes) +
                          wib * L.per_warp_doubles, K);
  build_schedules(K, sched, pairs);
  __syncthreads();

  const MaternConst mc = load_matern_const(a.tab);
  ThetaConst tc;
  tc.set(a.sigma2, a.beta, a.tau2);
  FieldView F;
  F.xy = reinterpret_cast<const double2*>(a.xy);
  F.yf = a.yf;
  F.nbr = a.nbr;
  F.self = a.self;
  F.n = a.n;
  F.m = a.m;
  const int64_t gw = (int64_t)blockIdx.x * W + wib;
  const int64_t nw = (int64_t)gridDim.x * W;
  Accum acc;
  for (int64_t i = gw; i < a.n; i += nw) {
    double* trow = a.terms ? a.terms + i * (GRAD ? 4 : 1) : nullptr;
    process_location<GRAD>(i, F, L.S, sched, pairs, area, a.tab, mc, tc, acc, trow, a.errloc, lane);
  }
  write_partial(acc, a.partial + gw * 4, lane);
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
  const int cand_all[] = {12, 11, 10, 9, 8, 6, 4, 2, 1};
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

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
#include <vector>

#include "block.cuh"
#include "common.cuh"
#include "matern.cuh"

namespace vecchia {

int get_matern_table(double nu, cudaStream_t stream, const double** out);
int get_cov_table(int family, double nu, cudaStream_t stream, const double** out);
void cov_table_used(const double* tab, cudaStream_t stream);

// A covariance table taken from the cache for one call: when the call's scope ends (after
// its launches, or on an early error return) the use is recorded on the stream.
struct TablePin {
  const double* tab = nullptr;
  cudaStream_t stream = nullptr;
  TablePin() = default;
  TablePin(const TablePin&) = delete;
  TablePin& operator=(const TablePin&) = delete;
  int get(int family, double nu, cudaStream_t s) {
    stream = s;
    return get_cov_table(family, nu, s, &tab);
  }
  ~TablePin() {
    if (tab) cov_table_used(tab, stream);
  }
};

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
  double* partial;
  double* terms;
  unsigned long long* errloc;
  const double* __restrict__ xyz;  // n x 3 unit vectors (sphere plans)
  int metric;                      // 0 plane, 1 sphere
  double radius;
  int64_t i0, i1;                  // ordered locations [i0, i1) are evaluated
};
int big_config(int K, bool grad, int* blocks, int* threads, int* smem, bool sphere);
void launch_big(bool grad, int blocks, int threads, int smem, const BigArgs& a, cudaStream_t s);
bool theta_ok_family(const double* th, int family);
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
  int family;                        // kFamilyMatern or kFamilyPowExp
  double sigma2, beta, nu, tau2;
  double* partial;                   // [nwarps][4]
  double* terms;                     // optional [n][1|4]
  unsigned long long* errloc;
  const double* __restrict__ xyz = nullptr;  // n x 3 unit vectors (sphere plans)
  int metric = 0;                    // 0 plane, 1 sphere
  double radius = 1.0;
  double* pmean = nullptr;           // prediction outputs (n), see FieldView
  double* pvar = nullptr;
  int64_t i0 = 0, i1 = 0;            // ordered locations [i0, i1) are evaluated
  int64_t n_index = 0;               // entries of xy / yf (0: n)
  bool check_idx = false;            // check nbr / self entries against [0, n_index)
  bool regather = false;             // gradient, 8 lanes: two vectors per block (WarpArea)
};

// Shared-memory layout for block size K (= m + 1), G lanes per location (32/G locations
// per warp) and W warps per CTA.
struct SmemLayout {
  SchedSize S;
  int group_doubles, per_warp_doubles;
  __host__ __device__ SmemLayout(int K, bool grad, int G, bool sphere = false, bool regather = false)
      : S(K),
        group_doubles(vecchia::group_doubles(K, grad, G, sphere, regather)),
        per_warp_doubles((32 / G) * vecchia::group_doubles(K, grad, G, sphere, regather)) {}
  __host__ __device__ int bytes(int W) const { return S.sched_bytes + S.pairs_bytes + W * per_warp_doubles * 8; }
};

// Up to 13 warps per CTA for the forward pass (its two-vector blocks fit thirteen on an
// SM at m = 60) and 12 for the gradient; the 8-lane gradient kernels are bounded for 16
// warps per SM (two CTAs of 8, at most 128 registers a thread), which their second-gather
// layout reaches at m = 25.
template <bool GRAD, int G, bool SPHERE>
__global__ void __launch_bounds__(GRAD ? (G == 8 ? 512 : 384) : 32 * kMaxCtaWarps) vecchia_lik_kernel(const LikArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NL = 32 / G;
  const int K = a.m + 1;
  constexpr bool sphere = SPHERE;
  const SmemLayout L(K, GRAD, G, sphere, a.regather);
  uint16_t* sched = reinterpret_cast<uint16_t*>(smem);
  uint32_t* pairs = reinterpret_cast<uint32_t*>(smem + L.S.sched_bytes);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int W = blockDim.x >> 5;
  const int grp = lane / G, sub = lane % G;
  const WarpArea area(reinterpret_cast<double*>(smem + L.S.sched_bytes + L.S.pairs_bytes) +
                          wib * L.per_warp_doubles + grp * L.group_doubles, K, GRAD, G, sphere, a.regather);
  build_schedules(K, sched, pairs);
  __syncthreads();

  const MaternConst mc = load_matern_const(a.tab);
  ThetaConst tc;
  tc.set(a.sigma2, a.beta, a.tau2, a.family, a.nu);
  FieldView F;
  F.xy = reinterpret_cast<const double2*>(a.xy);
  F.yf = a.yf;
  F.nbr = a.nbr;
  F.self = a.self;
  F.n = a.n;
  F.m = a.m;
  F.nidx = a.n_index > 0 ? a.n_index : a.n;
  F.check_idx = a.check_idx;
  F.pmean = a.pmean;
  F.pvar = a.pvar;
  if constexpr (SPHERE) {
    F.sphere = true;
    F.xyz = a.xyz;
    const double k = 2.0 * a.radius * tc.inv_len;
    F.k2d = k * k;
    F.k2 = d2f_pair(F.k2d);
  }
  const int64_t gw = (int64_t)blockIdx.x * W + wib;
  const int64_t nw = (int64_t)gridDim.x * W;
  const bool terms_mode = a.terms != nullptr;
  Accum acc;
  for (int64_t base = a.i0 + gw * NL; base < a.i1; base += nw * NL) {
    const int64_t i = base + grp;
    const bool active = i < a.i1;
    const int64_t ii = active ? i : base;
    double* trow = terms_mode ? a.terms + ii * (GRAD ? 4 : 1) : nullptr;
    process_location<GRAD, G, SPHERE>(ii, active, F, L.S, sched, pairs, area, a.tab, mc, tc, acc, terms_mode, trow,
                              a.errloc, sub);
  }
  // The CTA's warps' sums are combined in warp order (compensated), one record per CTA.
  __shared__ double wpart[kMaxCtaWarps][4];
  write_partial<G>(acc, wpart[wib], lane);
  __syncthreads();
  if (threadIdx.x < 4) {
    Neumaier c;
    for (int w = 0; w < W; ++w) c.add(wpart[w][threadIdx.x]);
    a.partial[(int64_t)blockIdx.x * 4 + threadIdx.x] = c.value();
  }
}

// Deterministic reduction of the per-CTA records: warp k sums column k, each lane a
// strided subset (compensated), then the lanes' (sum, compensation) pairs are merged by a
// fixed shuffle tree, so the result depends only on the number of records.
// Records: [sum l_i, sum 1/2(r^2/s-1), sum beta pair sums, sum w^T g]; dbeta_div is 1
// (Matérn) or alpha (power exponential).
__global__ void __launch_bounds__(128) vecchia_finalize_kernel(const double* __restrict__ partial, int64_t np,
                                                               double sigma2, double beta, double tau2,
                                                               double dbeta_div, int want_grad, double* out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Neumaier acc;
  for (int64_t w = lane; w < np; w += 32) acc.add(partial[w * 4 + k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_down_sync(0xffffffffu, acc.s, o);
    const double c2 = __shfl_down_sync(0xffffffffu, acc.c, o);
    acc.merge(s2, c2);
  }
  __shared__ double sv[4];
  if (lane == 0) sv[k] = acc.value();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!want_grad) {
      out[0] = sv[0];
      return;
    }
    out[0] = sv[0];
    out[1] = (sv[1] - tau2 * sv[3]) / sigma2;
    out[2] = -2.0 * sigma2 / (beta * dbeta_div) * sv[2];
    out[3] = sv[3];
  }
}

// ------------------------------------------------------------------ launch
namespace {
struct LaunchCfg {
  int G = 32, W = 4, blocks = 0, smem = 0;
  bool regather = false;  // gradient, 8 lanes: coordinates gathered twice, two vectors per block
  int sms = 0;            // SMs of the device
};

template <bool GRAD, bool SPHERE>
void* kernel_ptr(int G) {
  if (G == 4) return reinterpret_cast<void*>(vecchia_lik_kernel<GRAD, 4, SPHERE>);
  if (G == 8) return reinterpret_cast<void*>(vecchia_lik_kernel<GRAD, 8, SPHERE>);
  if (G == 16) return reinterpret_cast<void*>(vecchia_lik_kernel<GRAD, 16, SPHERE>);
  return reinterpret_cast<void*>(vecchia_lik_kernel<GRAD, 32, SPHERE>);
}

void* lik_kernel(bool grad, int G, bool sphere) {
  if (grad) return sphere ? kernel_ptr<true, true>(G) : kernel_ptr<true, false>(G);
  return sphere ? kernel_ptr<false, true>(G) : kernel_ptr<false, false>(G);
}

// Lanes per location chosen when no tuning result exists: small blocks share a warp.  The
// break points are the fastest measured shapes on GB300 at n = 1e6 (m = 15, 20, 25, 31,
// 45, 60); the adjoint favours wider groups a little earlier than the forward pass.
int default_lanes(int K, bool grad) {
  if (K <= 16) return 4;
  if (K <= 32) return 8;
  if (K <= 48) return grad ? 32 : 16;
  return 32;
}

// Tuning results, per (device, K, grad): lanes per location and warps per CTA.
struct Tuned {
  int dev, K, grad, G, W;
};
std::mutex g_tune_mu;
std::vector<Tuned> g_tuned;

bool tuned_for(int dev, int K, bool grad, int* G, int* W) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const Tuned& t : g_tuned)
    if (t.dev == dev && t.K == K && t.grad == (int)grad) {
      *G = t.G;
      *W = t.W;
      return true;
    }
  return false;
}

void set_tuned(int dev, int K, bool grad, int G, int W) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (Tuned& t : g_tuned)
    if (t.dev == dev && t.K == K && t.grad == (int)grad) {
      t.G = G;
      t.W = W;
      return;
    }
  g_tuned.push_back({dev, K, (int)grad, G, W});
}

// Launch shape for lanes-per-location G: W (forced_W > 0, else the value giving the most
// resident warps per SM, ties to the larger CTA) and a persistent grid of one wave.  An
// 8-lane gradient launch gathers the coordinates twice (two vectors per block) when that
// gives at least 20% more resident warps (regather_capable in block.cuh has the
// measurements behind the threshold).
//
// Shapes are cached per (device, K, kind, G, forced W, metric): the occupancy queries
// behind one cost tens of microseconds of host time.  The dynamic shared-memory limit
// last set on each kernel is recorded, so that a cached shape sets it again only where a
// launch of another block size changed it.
struct ShapeEntry {
  int dev, K, grad, G, W, sphere;
  LaunchCfg cfg;
};
struct SmemLimit {
  int dev;
  void* kern;
  int bytes;
};
std::mutex g_shape_mu;
std::vector<ShapeEntry> g_shapes;
std::vector<SmemLimit> g_smem_limits;

// Sets the kernel's dynamic shared-memory limit to `bytes` unless it already is.
// Called with g_shape_mu held.
int set_smem_limit(int dev, void* kern, int bytes) {
  for (SmemLimit& l : g_smem_limits)
    if (l.dev == dev && l.kern == kern) {
      if (l.bytes != bytes) {
        VECCHIA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        l.bytes = bytes;
      }
      return VECCHIA_OK;
    }
  VECCHIA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  g_smem_limits.push_back({dev, kern, bytes});
  return VECCHIA_OK;
}

int shape_for(int K, bool grad, int G, int forced_W, LaunchCfg* cfg, bool sphere = false) {
  if (K > max_k_for_lanes(G)) return VECCHIA_EINVAL;  // narrow groups hold small blocks only
  int dev = 0, sms = 0, smem_optin = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_shape_mu);
  void* kern = lik_kernel(grad, G, sphere);
  for (const ShapeEntry& e : g_shapes)
    if (e.dev == dev && e.K == K && e.grad == (int)grad && e.G == G && e.W == forced_W && e.sphere == (int)sphere) {
      const int rc = set_smem_limit(dev, kern, e.cfg.smem);
      if (rc) return rc;
      *cfg = e.cfg;
      return VECCHIA_OK;
    }
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  VECCHIA_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));  // the forward kernel takes up to 13 warps
  // most resident warps per SM (capped at 16 by the registers) for one layout, or -1
  auto best_for = [&](bool regather, LaunchCfg* out) -> int {
    const SmemLayout L(K, grad, G, sphere, regather);
    int best_warps = -1;
    for (int W : {13, 12, 11, 10, 9, 8, 6, 4, 2, 1}) {
      if (forced_W > 0 && W != forced_W) continue;
      if (32 * W > fa.maxThreadsPerBlock) continue;
      const int bytes = L.bytes(W);
      if (bytes > smem_optin) continue;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return -2;
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, bytes) != cudaSuccess) return -2;
      const int warps = std::min(per_sm * W, 16);
      if (per_sm > 0 && warps > best_warps) {
        best_warps = warps;
        out->G = G;
        out->W = W;
        out->blocks = per_sm * sms;
        out->sms = sms;
        out->smem = bytes;
        out->regather = regather;
      }
    }
    return best_warps;
  };
  LaunchCfg sep, rg;
  const int ws = best_for(false, &sep);
  const int wr = regather_capable(grad, G) ? best_for(true, &rg) : -1;
  if (ws == -2 || wr == -2) return VECCHIA_ECUDA;
  if (ws <= 0 && wr <= 0) return VECCHIA_EINVAL;
  *cfg = (wr > 0 && 5 * wr >= 6 * ws) ? rg : sep;
  VECCHIA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cfg->smem));
  bool known = false;  // the search above set other limits on the way
  for (SmemLimit& l : g_smem_limits)
    if (l.dev == dev && l.kern == kern) {
      l.bytes = cfg->smem;
      known = true;
    }
  if (!known) g_smem_limits.push_back({dev, kern, cfg->smem});
  g_shapes.push_back({dev, K, (int)grad, G, forced_W, (int)sphere, *cfg});
  return VECCHIA_OK;
}

// Configuration for block size K: the tuned shape if vecchia_autotune recorded one, else
// the default lanes per location.  VECCHIA_LANES_PER_LOCATION / VECCHIA_WARPS_PER_CTA
// force either value (tuning experiments).  `count` (> 0: the call's locations) widens
// the default groups, up to 16 lanes, while they would leave fewer location groups than
// the GPU has sub-partitions: such a call is bound by each warp's serial latency, which
// wider groups shorten (n = 2,000, m = 10, per call: 4 lanes 33.9 us, 8 lanes 30.7, 16
// lanes 28.8, 32 lanes 41.1).
int pick_config(int K, bool grad, LaunchCfg* cfg, bool sphere = false, int64_t count = -1) {
  int dev = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  int G = default_lanes(K, grad), W = 0;
  bool chosen = tuned_for(dev, K, grad, &G, &W);
  if (sphere) W = 0;  // the tuned CTA size was sized for planar blocks
  if (const char* e = getenv("VECCHIA_LANES_PER_LOCATION")) {
    const int v = atoi(e);
    if (v == 4 || v == 8 || v == 16 || v == 32) {
      G = v;
      chosen = true;
    }
  }
  if (const char* e = getenv("VECCHIA_WARPS_PER_CTA")) W = atoi(e);
  if (!chosen && count > 0) {
    int sms = 0;
    VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    while (G < 16 && (count + 32 / G - 1) / (32 / G) < 4 * (int64_t)sms) G *= 2;
  }
  while (K > max_k_for_lanes(G)) G *= 2;
  return shape_for(K, grad, G, W, cfg, sphere);
}

template <bool SPHERE>
void launch_lik_m(const LaunchCfg& cfg, bool grad, const LikArgs& a, cudaStream_t stream) {
  if (grad) {
    if (cfg.G == 4) vecchia_lik_kernel<true, 4, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
    else if (cfg.G == 8) vecchia_lik_kernel<true, 8, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
    else if (cfg.G == 16) vecchia_lik_kernel<true, 16, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
    else vecchia_lik_kernel<true, 32, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
  } else {
    if (cfg.G == 4) vecchia_lik_kernel<false, 4, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
    else if (cfg.G == 8) vecchia_lik_kernel<false, 8, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
    else if (cfg.G == 16) vecchia_lik_kernel<false, 16, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
    else vecchia_lik_kernel<false, 32, SPHERE><<<cfg.blocks, cfg.W * 32, cfg.smem, stream>>>(a);
  }
}

void launch_lik(const LaunchCfg& cfg, bool grad, const LikArgs& a, cudaStream_t stream) {
  if (a.metric == 1) launch_lik_m<true>(cfg, grad, a, stream);
  else launch_lik_m<false>(cfg, grad, a, stream);
}
}  // namespace

// Lanes per location for block size K: the tuned value if any, else the default.
int lanes_for(int K, bool grad) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return default_lanes(K, grad);
  int G = default_lanes(K, grad), W = 0;
  tuned_for(dev, K, grad, &G, &W);
  return G;
}

namespace {
// The launch for `count` locations: with fewer location groups than the shape's resident
// warps, the groups are spread over every SM with fewer warps per CTA.  A full-size CTA
// would put them all on a few SMs, whose FP64 pipes (one warp-instruction per 64 cycles
// per sub-partition, whatever the active lanes) would then run the whole problem while
// the rest of the GPU idles: at n = 2,000, m = 10 the kernel took 35 us that way, 26 us
// spread.  Each warp keeps the same locations (warp w takes group w); only the per-CTA
// grouping of the warps' sums changes, and with it the last bits of the totals.
LaunchCfg fit_to_work(LaunchCfg c, int K, bool grad, bool sphere, int64_t count) {
  const int NL = 32 / c.G;
  const int64_t groups = (count + NL - 1) / NL;
  if (c.sms <= 0 || groups >= (int64_t)c.blocks * c.W) return c;
  const int W = (int)std::max<int64_t>(1, std::min<int64_t>(c.W, (groups + c.sms - 1) / c.sms));
  c.W = W;
  c.blocks = (int)((groups + W - 1) / W);
  c.smem = SmemLayout(K, grad, c.G, sphere, c.regather).bytes(W);
  return c;
}

int launch_with(Plan* p, const double* y_dev, const double* theta, bool grad, const LaunchCfg& shape,
                double* out_dev, double* terms_dev, cudaStream_t stream, int64_t i0, int64_t i1) {
  const LaunchCfg cfg = fit_to_work(shape, p->m + 1, grad, p->metric == 1, i1 - i0);
  const int64_t nw = (int64_t)cfg.blocks * cfg.W;
  if (p->partial_cap < nw * 4) {
    if (p->d_partial) cudaFree(p->d_partial);
    p->d_partial = nullptr;
    p->partial_cap = 0;
    if (cudaMalloc(&p->d_partial, sizeof(double) * nw * 4) != cudaSuccess) return VECCHIA_ENOMEM;
    p->partial_cap = nw * 4;
  }
  TablePin pin;
  int rc = pin.get(p->family, theta[2], stream);
  if (rc) return rc;
  const double* tab = pin.tab;
  VECCHIA_CUDA_TRY(cudaMemsetAsync(p->d_errloc, 0xFF, sizeof(unsigned long long), stream));
  LikArgs a;
  a.xy = p->d_xy;
  a.yf = y_dev;
  a.nbr = p->d_nbr;
  a.self = p->d_self;
  a.tab = tab;
  a.n = p->n;
  a.m = p->m;
  a.family = p->family;
  a.sigma2 = theta[0];
  a.beta = theta[1];
  a.nu = theta[2];
  a.tau2 = theta[3];
  a.partial = p->d_partial;
  a.terms = terms_dev;
  a.errloc = p->d_errloc;
  a.xyz = p->d_xyz;
  a.metric = p->metric;
  a.radius = p->radius;
  a.i0 = i0;
  a.i1 = i1;
  a.regather = cfg.regather;
  launch_lik(cfg, grad, a, stream);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  if (out_dev) {
    const double dbeta_div = p->family == kFamilyPowExp ? theta[2] : 1.0;
    vecchia_finalize_kernel<<<1, 128, 0, stream>>>(p->d_partial, cfg.blocks, theta[0], theta[1], theta[3], dbeta_div,
                                                   grad ? 1 : 0, out_dev);
    VECCHIA_CUDA_TRY(cudaGetLastError());
  }
  p->last_stream = stream;
  return VECCHIA_OK;
}
}  // namespace

// Blocks beyond the warp kernels' size: one CTA per location (bigblock.cu).
static int launch_big_loglik(Plan* p, const double* y_dev, const double* theta, bool grad, double* out_dev,
                             double* terms_dev, cudaStream_t stream, int64_t i0, int64_t i1) {
  int blocks = 0, threads = 0, smem = 0;
  int rc = big_config(p->m + 1, grad, &blocks, &threads, &smem, p->metric == 1);
  if (rc) return rc;
  if (p->partial_cap < (int64_t)blocks * 4) {
    if (p->d_partial) cudaFree(p->d_partial);
    p->d_partial = nullptr;
    p->partial_cap = 0;
    if (cudaMalloc(&p->d_partial, sizeof(double) * blocks * 4) != cudaSuccess) return VECCHIA_ENOMEM;
    p->partial_cap = (int64_t)blocks * 4;
  }
  TablePin pin;
  rc = pin.get(p->family, theta[2], stream);
  if (rc) return rc;
  const double* tab = pin.tab;
  VECCHIA_CUDA_TRY(cudaMemsetAsync(p->d_errloc, 0xFF, sizeof(unsigned long long), stream));
  BigArgs a;
  a.xy = p->d_xy;
  a.yf = y_dev;
  a.nbr = p->d_nbr;
  a.self = p->d_self;
  a.tab = tab;
  a.n = p->n;
  a.m = p->m;
  a.family = p->family;
  a.sigma2 = theta[0];
  a.beta = theta[1];
  a.nu = theta[2];
  a.tau2 = theta[3];
  a.partial = p->d_partial;
  a.terms = terms_dev;
  a.errloc = p->d_errloc;
  a.xyz = p->d_xyz;
  a.metric = p->metric;
  a.radius = p->radius;
  a.i0 = i0;
  a.i1 = i1;
  launch_big(grad, blocks, threads, smem, a, stream);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  if (out_dev) {
    const double dbeta_div = p->family == kFamilyPowExp ? theta[2] : 1.0;
    vecchia_finalize_kernel<<<1, 128, 0, stream>>>(p->d_partial, blocks, theta[0], theta[1], theta[3], dbeta_div,
                                                   grad ? 1 : 0, out_dev);
    VECCHIA_CUDA_TRY(cudaGetLastError());
  }
  p->last_stream = stream;
  return VECCHIA_OK;
}

// Ordered locations [i0, i1) (i1 < 0: all n).  An empty range writes zeros.
int launch_loglik(Plan* p, const double* y_dev, const double* theta, bool grad, double* out_dev,
                  double* terms_dev, cudaStream_t stream, int64_t i0, int64_t i1) {
  if (!p || !y_dev || !theta_ok_family(theta, p->family) || (!out_dev && !terms_dev)) return VECCHIA_EINVAL;
  if (i1 < 0) i1 = p->n;
  if (i0 < 0 || i0 > i1 || i1 > p->n) return VECCHIA_EINVAL;
  if (i0 == i1) {
    if (out_dev) VECCHIA_CUDA_TRY(cudaMemsetAsync(out_dev, 0, sizeof(double) * (grad ? 4 : 1), stream));
    VECCHIA_CUDA_TRY(cudaMemsetAsync(p->d_errloc, 0xFF, sizeof(unsigned long long), stream));
    p->last_stream = stream;
    return VECCHIA_OK;
  }
  if (p->m > kMaxMWarp) return launch_big_loglik(p, y_dev, theta, grad, out_dev, terms_dev, stream, i0, i1);
  LaunchCfg cfg;
  int rc = pick_config(p->m + 1, grad, &cfg, p->metric == 1, i1 - i0);
  if (rc) return rc;
  return launch_with(p, y_dev, theta, grad, cfg, out_dev, terms_dev, stream, i0, i1);
}

int knn_predict(Plan* p, const double* xy_new_host, int64_t n_new, int32_t* d_nbr_new, std::vector<double>* xyz_new_out,
                cudaStream_t stream);

// Kriging at new points (vecchia_predict): conditioning sets from knn_predict, then the
// likelihood kernel over the new points with the observed and new coordinates side by
// side (observed first, so the sets' original indices address them), y = 0 at the new
// points and the prediction outputs in place of the likelihood sums.
int predict(Plan* p, const double* xy_new_host, int64_t n_new, const double* y_dev, const double* theta,
            double* mean_dev, double* var_dev, int32_t* nbr_host, cudaStream_t stream) {
  if (!p || !xy_new_host || n_new < 1 || n_new > 2147483647LL - p->n || !y_dev || !mean_dev ||
      !theta_ok_family(theta, p->family))
    return VECCHIA_EINVAL;
  if (p->m > kMaxMWarp || p->m > p->n) return VECCHIA_EINVAL;
  for (int64_t k = 0; k < 2 * n_new; ++k)
    if (!std::isfinite(xy_new_host[k])) return VECCHIA_EINVAL;
  if (p->metric == 1)
    for (int64_t k = 0; k < n_new; ++k)
      if (!(fabs(xy_new_host[2 * k + 1]) <= 90.0)) return VECCHIA_EINVAL;
  const int64_t n = p->n, nt = n + n_new, m = p->m;
  int32_t* d_nbr = nullptr;
  int32_t* d_self = nullptr;
  double *d_xy = nullptr, *d_y = nullptr, *d_xyz = nullptr;
  int rc = VECCHIA_OK;
  if (cudaMalloc(&d_nbr, sizeof(int32_t) * n_new * m) != cudaSuccess ||
      cudaMalloc(&d_self, sizeof(int32_t) * n_new) != cudaSuccess ||
      cudaMalloc(&d_xy, sizeof(double) * 2 * nt) != cudaSuccess || cudaMalloc(&d_y, sizeof(double) * nt) != cudaSuccess ||
      (p->metric == 1 && cudaMalloc(&d_xyz, sizeof(double) * 3 * nt) != cudaSuccess))
    rc = VECCHIA_ENOMEM;
  std::vector<double> xyz_new;
  if (!rc) rc = knn_predict(p, xy_new_host, n_new, d_nbr, &xyz_new, stream);
  std::vector<int32_t> self(n_new);
  for (int64_t k = 0; k < n_new; ++k) self[k] = (int32_t)(n + k);
  auto cp = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    if (!rc && cudaMemcpyAsync(dst, src, bytes, kind, stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  };
  cp(d_self, self.data(), sizeof(int32_t) * n_new, cudaMemcpyHostToDevice);
  cp(d_xy, p->d_xy, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice);
  cp(d_xy + 2 * n, xy_new_host, sizeof(double) * 2 * n_new, cudaMemcpyHostToDevice);
  cp(d_y, y_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice);
  if (!rc && cudaMemsetAsync(d_y + n, 0, sizeof(double) * n_new, stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  if (p->metric == 1) {
    cp(d_xyz, p->d_xyz, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice);
    cp(d_xyz + 3 * n, xyz_new.data(), sizeof(double) * 3 * n_new, cudaMemcpyHostToDevice);
  }
  LaunchCfg cfg;
  if (!rc) rc = pick_config((int)m + 1, false, &cfg, p->metric == 1, n_new);
  if (!rc) cfg = fit_to_work(cfg, (int)m + 1, false, p->metric == 1, n_new);
  const int64_t nw = (int64_t)cfg.blocks * cfg.W;
  if (!rc && p->partial_cap < nw * 4) {
    if (p->d_partial) cudaFree(p->d_partial);
    p->d_partial = nullptr;
    p->partial_cap = 0;
    if (cudaMalloc(&p->d_partial, sizeof(double) * nw * 4) != cudaSuccess) rc = VECCHIA_ENOMEM;
    else p->partial_cap = nw * 4;
  }
  TablePin pin;
  if (!rc) rc = pin.get(p->family, theta[2], stream);
  const double* tab = pin.tab;
  if (!rc && cudaMemsetAsync(p->d_errloc, 0xFF, sizeof(unsigned long long), stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  if (!rc) {
    LikArgs a;
    a.xy = d_xy;
    a.yf = d_y;
    a.nbr = d_nbr;
    a.self = d_self;
    a.tab = tab;
    a.n = n_new;
    a.m = (int)m;
    a.family = p->family;
    a.sigma2 = theta[0];
    a.beta = theta[1];
    a.nu = theta[2];
    a.tau2 = theta[3];
    a.partial = p->d_partial;
    a.terms = nullptr;
    a.errloc = p->d_errloc;
    a.xyz = d_xyz;
    a.metric = p->metric;
    a.radius = p->radius;
    a.pmean = mean_dev;
    a.pvar = var_dev;
    a.i0 = 0;
    a.i1 = n_new;
    a.n_index = nt;
    launch_lik(cfg, false, a, stream);
    if (cudaGetLastError() != cudaSuccess) rc = VECCHIA_ECUDA;
  }
  if (!rc && nbr_host)
    cp(nbr_host, d_nbr, sizeof(int32_t) * n_new * m, cudaMemcpyDeviceToHost);
  if (cudaStreamSynchronize(stream) != cudaSuccess && !rc) rc = VECCHIA_ECUDA;
  cudaFree(d_nbr);
  cudaFree(d_self);
  cudaFree(d_xy);
  cudaFree(d_y);
  cudaFree(d_xyz);
  p->last_stream = stream;
  return rc;
}

// Times every (lanes per location, warps per CTA) shape on the caller's problem and
// records the fastest for this block size and kind of evaluation.
int autotune(Plan* p, const double* y_dev, const double* theta, bool grad, int* G_out, int* W_out,
             cudaStream_t stream) {
  if (!p || !y_dev || !theta_ok_family(theta, p->family)) return VECCHIA_EINVAL;
  const int K = p->m + 1;
  if (p->m > kMaxMWarp) {  // one CTA per location, sized by occupancy: nothing to time
    int blocks = 0, threads = 0, smem = 0;
    const int rc = big_config(K, grad, &blocks, &threads, &smem, p->metric == 1);
    if (rc) return rc;
    if (G_out) *G_out = threads;
    if (W_out) *W_out = threads / 32;
    return VECCHIA_OK;
  }
  int dev = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * 4) != cudaSuccess) return VECCHIA_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bestG = default_lanes(K, grad), bestW = 0, rc = VECCHIA_OK;
  for (int G : {4, 8, 16, 32}) {
    if (K > max_k_for_lanes(G)) continue;
    for (int W : {13, 12, 11, 10, 9, 8, 6, 4}) {
      LaunchCfg cfg;
      if (shape_for(K, grad, G, W, &cfg, p->metric == 1) != VECCHIA_OK) continue;
      float tmin = 1e30f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {
        cudaEventRecord(e0, stream);
        rc = launch_with(p, y_dev, theta, grad, cfg, out, nullptr, stream, 0, p->n);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = VECCHIA_ECUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tmin = std::min(tmin, ms);
      }
      if (rc) break;
      if (tmin < best) {
        best = tmin;
        bestG = G;
        bestW = W;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) return rc;
  set_tuned(dev, K, grad, bestG, bestW);
  if (G_out) *G_out = bestG;
  if (W_out) *W_out = bestW;
  return VECCHIA_OK;
}

// ------------------------------------------------------------------ vecchia_pivot_reciprocal
// The pivot reciprocal on its own: NaN outside its domain.
__global__ void pivot_reciprocal_kernel(const double* __restrict__ d, int64_t count, double* __restrict__ out) {
  const double nan = __longlong_as_double(0x7FF8000000000000LL);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = d[i];
    out[i] = pivot_in_range(v) ? rcp_fixed(v) : nan;
  }
}

// The column-scaling product of the full-warp kernels on its own.
__global__ void mul_by_positive_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t count,
                                       double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mul_by_positive(a[i], b[i]);
}

}  // namespace vecchia

extern "C" int vecchia_mul_by_positive(const double* a_dev, const double* b_dev, int64_t count, double* out_dev,
                                       void* stream) {
  if (count < 0 || (count > 0 && (!a_dev || !b_dev || !out_dev))) return VECCHIA_EINVAL;
  if (count == 0) return VECCHIA_OK;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  vecchia::mul_by_positive_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(a_dev, b_dev, count, out_dev);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  return VECCHIA_OK;
}

extern "C" int vecchia_pivot_reciprocal(const double* d_dev, int64_t count, double* out_dev, void* stream) {
  if (count < 0 || (count > 0 && (!d_dev || !out_dev))) return VECCHIA_EINVAL;
  if (count == 0) return VECCHIA_OK;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
  vecchia::pivot_reciprocal_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(d_dev, count, out_dev);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  return VECCHIA_OK;
}

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
      m > kMaxMWarp || !theta_ok(theta))
    return VECCHIA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc) return rc;
  double* partial = reinterpret_cast<double*>(base);
  unsigned long long* errloc = reinterpret_cast<unsigned long long*>(base + kNoAllocErrOff);
  double* tab = reinterpret_cast<double*>(base + kNoAllocTabOff);
  LaunchCfg cfg;
  rc = pick_config(m + 1, false, &cfg, false, n);
  if (rc) return rc;
  // The kernel is persistent (warps stride over locations), so any grid covers any n;
  // it is capped to the warps the scratch can hold.
  const int max_blocks = kNoAllocWarps / cfg.W;
  if (cfg.blocks > max_blocks) cfg.blocks = max_blocks;
  cfg = fit_to_work(cfg, m + 1, false, false, n);
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
  a.family = kFamilyMatern;
  a.sigma2 = theta[0];
  a.beta = theta[1];
  a.nu = theta[2];
  a.tau2 = theta[3];
  a.partial = partial;
  a.terms = nullptr;
  a.errloc = errloc;
  a.i0 = 0;
  a.i1 = n;
  a.check_idx = true;  // caller-supplied index arrays: a bad entry fails its block, never reads out of bounds
  launch_lik(cfg, false, a, s);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  vecchia_finalize_kernel<<<1, 128, 0, s>>>(partial, cfg.blocks, theta[0], theta[1], theta[3], 1.0, 0, out_dev);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  return VECCHIA_OK;
}

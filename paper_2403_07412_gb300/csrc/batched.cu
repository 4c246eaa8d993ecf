// Many independent (field, theta) log-likelihood evaluations in one persistent launch.
//
// The paper batches only over the locations of one field (Sec. V-B).  Here the unit of
// work is an item = (field, theta, tile of kTile consecutive ordered locations); a
// persistent grid of warps takes items from a global counter, evaluates each location
// with the same per-location code as the single-field kernel (block.cuh), and writes
// one partial-sum record per item.  Fields may differ in n and m (all block sizes of a
// batch share one shared-memory layout sized for the largest), and each theta picks its
// covariance table by smoothness nu among the tables prepared with
// vecchia_batched_prepare.  Items are laid out so the most expensive fields (largest m)
// are handed out first.  A second kernel reduces each (field, theta)'s records in item
// order, so results do not depend on scheduling.  The launch sequence (two memsets and
// two kernels) allocates nothing and never waits on the host, so it can be captured in
// a CUDA graph once the work layout has been cached by a first call.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "block.cuh"
#include "common.cuh"
#include "matern.cuh"

namespace vecchia {

int launch_matern_table(double nu, double* tab, cudaStream_t stream);
bool theta_ok(const double* th);
int lanes_for(int K, bool grad);

constexpr int kTile = 256;       // ordered locations per work item
constexpr int kMaxNu = 8;        // prepared smoothness values
constexpr int kMaxDistinctK = 4; // distinct block sizes per batch

struct FieldDesc {
  const double2* xy;
  const double* yf;
  const int32_t* nbr;
  const int32_t* self;
  int64_t n;
  int32_t m;
  int32_t kidx;       // index of this field's block size in the batch's K list
  int32_t orig;       // position in the caller's field list
  int32_t tiles;      // ceil(n / kTile)
  int32_t lanes;      // lanes per location (8, 16 or 32)
  int64_t item_base;  // first item of this field
};

struct BatchArgs {
  const FieldDesc* fields;
  int nfields;
  int ntheta;
  const double* thetas;  // [nfields][ntheta][4], caller order
  const double* nus;     // [kMaxNu]
  const double* const* tabs;
  int nnu;
  int64_t total_items;
  unsigned long long* counter;
  unsigned long long* errloc;
  double* partial;  // [total_items][4]
  int nk;
  int kval[kMaxDistinctK];
  int sched_off[kMaxDistinctK];
  int pairs_off[kMaxDistinctK];
  int area_off;
  int area_doubles;
};

// One item with G lanes per location: the 32/G groups of the warp take the tile's
// locations in turn.
template <bool GRAD, int G>
__device__ __forceinline__ void run_item(const FieldDesc& fd, int64_t tile, const unsigned char* smem,
                                         const BatchArgs& a, double* base, const double* tab,
                                         const MaternConst& mc, const ThetaConst& tc, double* out, int lane) {
  constexpr int NL = 32 / G;
  const int grp = lane / G, sub = lane % G;
  FieldView F;
  F.xy = fd.xy;
  F.yf = fd.yf;
  F.nbr = fd.nbr;
  F.self = fd.self;
  F.n = fd.n;
  F.m = fd.m;
  F.nidx = fd.n;
  const int K = fd.m + 1;
  const SchedSize S(K);
  const uint16_t* sched = reinterpret_cast<const uint16_t*>(smem + a.sched_off[fd.kidx]);
  const uint32_t* pairs = reinterpret_cast<const uint32_t*>(smem + a.pairs_off[fd.kidx]);
  const WarpArea area(base + grp * group_doubles(K, GRAD, G), K, GRAD, G);
  Accum acc;
  const int64_t i0 = tile * kTile;
  const int64_t i1 = min(fd.n, i0 + kTile);
  for (int64_t b = i0; b < i1; b += NL) {
    const int64_t i = b + grp;
    const bool active = i < i1;
    process_location<GRAD, G, false>(active ? i : b, active, F, S, sched, pairs, area, tab, mc, tc, acc, false, nullptr,
                              a.errloc, sub);
  }
  write_partial<G>(acc, out, lane);
}

template <bool GRAD>
__global__ void __launch_bounds__(384) vecchia_batched_kernel(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (int k = 0; k < a.nk; ++k)
    build_schedules(a.kval[k], reinterpret_cast<uint16_t*>(smem + a.sched_off[k]),
                    reinterpret_cast<uint32_t*>(smem + a.pairs_off[k]));
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  double* base = reinterpret_cast<double*>(smem + a.area_off) + wib * a.area_doubles;
  while (true) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(a.counter, 1ULL);
    item = __shfl_sync(0xffffffffu, item, 0);
    if ((int64_t)item >= a.total_items) break;
    // field of this item: fields are stored in item order
    int lo = 0, hi = a.nfields - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.fields[mid].item_base <= (int64_t)item) lo = mid; else hi = mid - 1;
    }
    const FieldDesc fd = a.fields[lo];
    const int64_t rel = (int64_t)item - fd.item_base;
    const int t = (int)(rel / fd.tiles);
    const int64_t tile = rel % fd.tiles;
    if (kChecked && (t >= a.ntheta || tile >= fd.tiles || lo < 0 || lo >= a.nfields)) {
      if (lane == 0) {  // a work item outside the layout: record it and skip it
        atomicMin(a.errloc, err_code((int64_t)item, kErrIndex));
      }
      continue;
    }
    const double* th = a.thetas + ((int64_t)fd.orig * a.ntheta + t) * 4;
    const double s2 = th[0], beta = th[1], nu = th[2], t2 = th[3];
    const double* tab = nullptr;
    for (int k = 0; k < a.nnu; ++k)
      if (__double_as_longlong(a.nus[k]) == __double_as_longlong(nu)) tab = a.tabs[k];
    double* out = a.partial + item * 4;
    const bool theta_valid = s2 > 0.0 && beta > 0.0 && t2 >= 0.0 && isfinite(s2) && isfinite(beta) &&
                             isfinite(t2);
    if (!tab || !theta_valid) {
      if (lane == 0) {
        out[0] = out[1] = out[2] = out[3] = __longlong_as_double(0x7FF8000000000000LL);
        atomicMin(a.errloc, err_code(0, kErrData));
      }
      continue;
    }
    const MaternConst mc = load_matern_const(tab);
    ThetaConst tc;
    tc.set(s2, beta, t2, kFamilyMatern, nu);
    if (fd.lanes == 4) run_item<GRAD, 4>(fd, tile, smem, a, base, tab, mc, tc, out, lane);
    else if (fd.lanes == 8) run_item<GRAD, 8>(fd, tile, smem, a, base, tab, mc, tc, out, lane);
    else if (fd.lanes == 16) run_item<GRAD, 16>(fd, tile, smem, a, base, tab, mc, tc, out, lane);
    else run_item<GRAD, 32>(fd, tile, smem, a, base, tab, mc, tc, out, lane);
    __syncwarp();
  }
}

// One warp per (field, theta): the field's tile records, each lane a strided subset in
// item order (compensated), merged by a fixed shuffle tree, so the result depends only
// on the field's tile count.
__global__ void vecchia_batched_finalize(const FieldDesc* __restrict__ fields, int nfields, int ntheta,
                                         const double* __restrict__ thetas, const double* __restrict__ partial,
                                         int want_grad, double* out) {
  const int64_t id = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (id >= (int64_t)nfields * ntheta) return;  // whole warps leave together
  const int fs = (int)(id / ntheta), t = (int)(id % ntheta);
  const FieldDesc fd = fields[fs];
  Neumaier acc[4];
  const double* p = partial + (fd.item_base + (int64_t)t * fd.tiles) * 4;
  for (int k = lane; k < fd.tiles; k += 32)
    for (int c = 0; c < 4; ++c) acc[c].add(p[k * 4 + c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double s2 = __shfl_down_sync(0xffffffffu, acc[c].s, o);
      const double c2 = __shfl_down_sync(0xffffffffu, acc[c].c, o);
      acc[c].merge(s2, c2);
    }
  if (lane != 0) return;
  const int64_t o = (int64_t)fd.orig * ntheta + t;
  if (!want_grad) {
    out[o] = acc[0].value();
    return;
  }
  const double* th = thetas + o * 4;
  double* r = out + o * 4;
  r[0] = acc[0].value();
  r[1] = (acc[1].value() - th[3] * acc[3].value()) / th[0];
  r[2] = -2.0 * th[0] / th[1] * acc[2].value();
  r[3] = acc[3].value();
}

// ------------------------------------------------------------------ host state
namespace {

struct PreparedNu {
  int device = -1;
  int nnu = 0;
  double nus[kMaxNu] = {};
  double* tabs[kMaxNu] = {};
  double* d_nus = nullptr;
  double** d_tabs = nullptr;
};

struct BatchState {
  int device = -1;
  std::vector<const void*> plans;
  std::vector<const double*> ys;
  int ntheta = 0;
  int want_grad = 0;
  FieldDesc* d_fields = nullptr;
  double* d_partial = nullptr;
  unsigned long long* d_counter = nullptr;  // [0] = work counter, [1] = error slot
  int64_t total_items = 0;
  BatchArgs args{};
  int W = 0, blocks = 0, smem = 0;
};

std::mutex g_mu;
std::vector<PreparedNu> g_prepared;
std::vector<BatchState*> g_batches;

void free_batch(BatchState* b) {
  cudaFree(b->d_fields);
  cudaFree(b->d_partial);
  cudaFree(b->d_counter);
  delete b;
}

PreparedNu* prepared_for(int dev) {
  for (auto& p : g_prepared)
    if (p.device == dev) return &p;
  return nullptr;
}

// Warps per CTA with the most resident warps per SM for this shared-memory footprint.
template <bool GRAD>
int batched_config(int fixed_bytes, int per_warp_bytes, int* W, int* blocks, int* smem) {
  int dev = 0, sms = 0, optin = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VECCHIA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  int best = -1;
  for (int w : {12, 11, 10, 9, 8, 6, 4, 2, 1}) {
    const int bytes = fixed_bytes + w * per_warp_bytes;
    if (bytes > optin) continue;
    VECCHIA_CUDA_TRY(cudaFuncSetAttribute(vecchia_batched_kernel<GRAD>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    int per_sm = 0;
    VECCHIA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vecchia_batched_kernel<GRAD>,
                                                                   w * 32, bytes));
    const int warps = std::min(per_sm * w, 16);
    if (per_sm > 0 && warps > best) {
      best = warps;
      *W = w;
      *blocks = per_sm * sms;
      *smem = bytes;
    }
  }
  if (best <= 0) return VECCHIA_EINVAL;
  VECCHIA_CUDA_TRY(cudaFuncSetAttribute(vecchia_batched_kernel<GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        *smem));
  return VECCHIA_OK;
}

int build_batch(const Plan* const* plans, const double* const* ys, int nfields, int ntheta, int want_grad,
                int dev, BatchState** out) {
  BatchState* b = new BatchState();
  b->device = dev;
  b->ntheta = ntheta;
  b->want_grad = want_grad;
  std::vector<int> order(nfields);
  for (int f = 0; f < nfields; ++f) order[f] = f;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return plans[x]->m > plans[y]->m; });
  std::vector<FieldDesc> fd(nfields);
  std::vector<int> kvals;
  int64_t items = 0;
  for (int s = 0; s < nfields; ++s) {
    const Plan* p = plans[order[s]];
    FieldDesc& d = fd[s];
    d.xy = reinterpret_cast<const double2*>(p->d_xy);
    d.yf = ys[order[s]];
    d.nbr = p->d_nbr;
    d.self = p->d_self;
    d.n = p->n;
    d.m = p->m;
    const int K = p->m + 1;
    auto it = std::find(kvals.begin(), kvals.end(), K);
    if (it == kvals.end()) {
      if ((int)kvals.size() == kMaxDistinctK) { delete b; return VECCHIA_EINVAL; }
      kvals.push_back(K);
      it = kvals.end() - 1;
    }
    d.kidx = (int)(it - kvals.begin());
    d.lanes = lanes_for(K, want_grad != 0);
    d.orig = order[s];
    d.tiles = (int)((p->n + kTile - 1) / kTile);
    d.item_base = items;
    items += (int64_t)d.tiles * ntheta;
  }
  // Every warp's shared-memory area is sized for the largest field's share (32/lanes
  // blocks).  A field whose own choice of lanes would need more than the full-warp
  // fields do widens its groups instead, so the launch keeps the occupancy of the
  // largest blocks (which carry most of the flops).
  int full_area = 0;
  for (int f = 0; f < nfields; ++f)
    if (fd[f].lanes == 32) full_area = std::max(full_area, group_doubles(fd[f].m + 1, want_grad != 0, 32));
  if (full_area > 0) {
    for (int f = 0; f < nfields; ++f) {
      const int K = fd[f].m + 1;
      while (fd[f].lanes < 32 && (32 / fd[f].lanes) * group_doubles(K, want_grad != 0, fd[f].lanes) > full_area)
        fd[f].lanes *= 2;
    }
  }
  for (int s = 0; s < nfields; ++s) {
    b->plans.push_back(plans[s]);
    b->ys.push_back(ys[s]);
  }
  b->total_items = items;
  BatchArgs& a = b->args;
  a.nfields = nfields;
  a.ntheta = ntheta;
  a.total_items = items;
  a.nk = (int)kvals.size();
  int off = 0, area = 0;
  for (int k = 0; k < a.nk; ++k) {
    const SchedSize S(kvals[k]);
    a.kval[k] = kvals[k];
    a.sched_off[k] = off;
    off += S.sched_bytes;
    a.pairs_off[k] = off;
    off += S.pairs_bytes;
  }
  for (int f = 0; f < nfields; ++f)  // a warp holds 32/lanes blocks of its field's size
    area = std::max(area, (32 / fd[f].lanes) * group_doubles(fd[f].m + 1, want_grad != 0, fd[f].lanes));
  a.area_off = off;
  a.area_doubles = area;
  int rc = want_grad ? batched_config<true>(off, a.area_doubles * 8, &b->W, &b->blocks, &b->smem)
                     : batched_config<false>(off, a.area_doubles * 8, &b->W, &b->blocks, &b->smem);
  if (rc) { delete b; return rc; }
  if (cudaMalloc(&b->d_fields, sizeof(FieldDesc) * nfields) != cudaSuccess ||
      cudaMalloc(&b->d_partial, sizeof(double) * 4 * std::max<int64_t>(items, 1)) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(unsigned long long) * 2) != cudaSuccess) {
    free_batch(b);
    return VECCHIA_ENOMEM;
  }
  if (cudaMemcpy(b->d_fields, fd.data(), sizeof(FieldDesc) * nfields, cudaMemcpyHostToDevice) != cudaSuccess) {
    free_batch(b);
    return VECCHIA_ECUDA;
  }
  a.fields = b->d_fields;
  a.partial = b->d_partial;
  a.counter = b->d_counter;
  a.errloc = b->d_counter + 1;
  *out = b;
  return VECCHIA_OK;
}

}  // namespace

// Drops cached batch layouts that reference `plan` (called by vecchia_plan_destroy).
void forget_plan_in_batches(const void* plan) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (size_t k = 0; k < g_batches.size();) {
    BatchState* b = g_batches[k];
    if (std::find(b->plans.begin(), b->plans.end(), plan) != b->plans.end()) {
      free_batch(b);
      g_batches.erase(g_batches.begin() + k);
    } else {
      ++k;
    }
  }
}

}  // namespace vecchia

extern "C" int vecchia_batched_prepare(const double* nus, int32_t nnu, void* stream) {
  using namespace vecchia;
  if (!nus || nnu < 1 || nnu > kMaxNu) return VECCHIA_EINVAL;
  for (int k = 0; k < nnu; ++k)
    if (!std::isfinite(nus[k]) || !(nus[k] > 0.0)) return VECCHIA_EINVAL;
  int dev = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_mu);
  PreparedNu* p = prepared_for(dev);
  if (!p) {
    g_prepared.emplace_back();
    p = &g_prepared.back();
    p->device = dev;
    if (cudaMalloc(&p->d_nus, sizeof(double) * kMaxNu) != cudaSuccess ||
        cudaMalloc(&p->d_tabs, sizeof(double*) * kMaxNu) != cudaSuccess)
      return VECCHIA_ENOMEM;
    for (int k = 0; k < kMaxNu; ++k)
      if (cudaMalloc(&p->tabs[k], kTableBytes) != cudaSuccess) return VECCHIA_ENOMEM;
  }
  VECCHIA_CUDA_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < nnu; ++k) {
    p->nus[k] = nus[k];
    int rc = launch_matern_table(nus[k], p->tabs[k], s);
    if (rc) return rc;
  }
  p->nnu = nnu;
  VECCHIA_CUDA_TRY(cudaMemcpyAsync(p->d_nus, p->nus, sizeof(double) * kMaxNu, cudaMemcpyHostToDevice, s));
  VECCHIA_CUDA_TRY(cudaMemcpyAsync(p->d_tabs, p->tabs, sizeof(double*) * kMaxNu, cudaMemcpyHostToDevice, s));
  VECCHIA_CUDA_TRY(cudaStreamSynchronize(s));
  return VECCHIA_OK;
}

extern "C" int vecchia_loglik_batched(const vecchia_plan_t* plans, const double* const* y_devs, int32_t nfields,
                                      const double* thetas_dev, int32_t ntheta, int want_grad, double* out_dev,
                                      void* stream) {
  using namespace vecchia;
  if (!plans || !y_devs || nfields < 1 || ntheta < 1 || !thetas_dev || !out_dev) return VECCHIA_EINVAL;
  for (int f = 0; f < nfields; ++f)
    if (!plans[f] || !y_devs[f] || plans[f]->family != kFamilyMatern || plans[f]->m > kMaxMWarp ||
        plans[f]->metric != 0)
      return VECCHIA_EINVAL;
  want_grad = want_grad ? 1 : 0;
  int dev = 0;
  VECCHIA_CUDA_TRY(cudaGetDevice(&dev));
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_mu);
  PreparedNu* pn = prepared_for(dev);
  if (!pn || pn->nnu == 0) return VECCHIA_EINVAL;
  BatchState* b = nullptr;
  for (BatchState* c : g_batches) {
    if (c->device != dev || c->ntheta != ntheta || c->want_grad != want_grad || (int)c->plans.size() != nfields)
      continue;
    bool same = true;
    for (int f = 0; f < nfields && same; ++f)
      same = c->plans[f] == (const void*)plans[f] && c->ys[f] == y_devs[f];
    if (same) { b = c; break; }
  }
  if (!b) {
    // First call for this set of fields: lay out the work (allocates; not capturable).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    VECCHIA_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return VECCHIA_EINVAL;
    std::vector<const Plan*> pp(nfields);
    for (int f = 0; f < nfields; ++f) pp[f] = plans[f];
    int rc = build_batch(pp.data(), y_devs, nfields, ntheta, want_grad, dev, &b);
    if (rc) return rc;
    g_batches.push_back(b);
  }
  BatchArgs a = b->args;
  a.thetas = thetas_dev;
  a.nus = pn->d_nus;
  a.tabs = pn->d_tabs;
  a.nnu = pn->nnu;
  VECCHIA_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s));
  VECCHIA_CUDA_TRY(cudaMemsetAsync(b->d_counter + 1, 0xFF, sizeof(unsigned long long), s));
  if (want_grad) vecchia_batched_kernel<true><<<b->blocks, b->W * 32, b->smem, s>>>(a);
  else vecchia_batched_kernel<false><<<b->blocks, b->W * 32, b->smem, s>>>(a);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  const int64_t pairs = (int64_t)nfields * ntheta;
  vecchia_batched_finalize<<<(unsigned)((pairs + 3) / 4), 128, 0, s>>>(b->d_fields, nfields, ntheta, thetas_dev,
                                                                           b->d_partial, want_grad, out_dev);
  VECCHIA_CUDA_TRY(cudaGetLastError());
  return VECCHIA_OK;
}

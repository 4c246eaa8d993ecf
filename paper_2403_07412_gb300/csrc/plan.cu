// Plan construction: ordering (Sec. V-A) and conditioning sets (Algorithm 1, the
// nearest-neighbour loop), plus the plan's C-ABI accessors.
//
// Orderings run on the host (both are inherently sequential):
//   random — Durstenfeld's Fisher–Yates shuffle driven by splitmix64 (Steele, Lea &
//            Flood 2014), j = next() mod (i+1) for i = n-1 .. 1;
//   maxmin — exact greedy farthest-point ordering from the point nearest the centroid,
//            ties to the lowest original index; a lazy max-heap of each point's squared
//            distance to the chosen set, updated only inside the disc that can change;
//   morton — Z-order of 16-bit cell indices over the bounding box.
// Conditioning sets are found on the GPU, one thread per ordered location, over a
// hierarchy of uniform grids: level l holds the first N_l ordered points (N_l doubling),
// bucketed by cell with each cell's points in ascending ordered index, so a query i
// scans level l(i) (the smallest with N_l >= i) ring by ring, stops reading a cell at
// the first index >= i, and stops searching once the distance from the query to the
// unscanned region exceeds the current m-th best.  Selection is exact in
// (d^2, index) with d^2 = round(round(dx*dx) + round(dy*dy)).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "common.cuh"

namespace vecchia {

// ------------------------------------------------------------------ host orderings
static uint64_t splitmix64(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static void order_random(int64_t n, uint64_t seed, int64_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  uint64_t st = seed;
  for (int64_t i = n - 1; i >= 1; --i) {
    const int64_t j = (int64_t)(splitmix64(st) % (uint64_t)(i + 1));
    std::swap(perm[i], perm[j]);
  }
}

// Morton (Z-order) ordering (Sec. V-A, Fig. 1): each coordinate is mapped to a 16-bit
// cell index over the bounding box, q = min(65535, floor((v - lo) / (hi - lo) * 65536))
// (q = 0 when hi == lo), the two indices are bit-interleaved (x in the even bits), and
// locations are sorted by (code, original index).
static uint32_t morton_cell(double v, double lo, double hi) {
  if (!(hi > lo)) return 0;
  const double t = (v - lo) / (hi - lo);
  const double q = std::floor(t * 65536.0);
  return q < 0.0 ? 0u : (q > 65535.0 ? 65535u : (uint32_t)q);
}

static void order_morton(int64_t n, const double* xy, int64_t* perm) {
  double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
  for (int64_t i = 1; i < n; ++i) {
    x0 = std::min(x0, xy[2 * i]); x1 = std::max(x1, xy[2 * i]);
    y0 = std::min(y0, xy[2 * i + 1]); y1 = std::max(y1, xy[2 * i + 1]);
  }
  std::vector<std::pair<uint32_t, int64_t>> key(n);
  for (int64_t i = 0; i < n; ++i) {
    const uint32_t qx = morton_cell(xy[2 * i], x0, x1), qy = morton_cell(xy[2 * i + 1], y0, y1);
    uint32_t code = 0;
    for (int b = 0; b < 16; ++b) code |= ((qx >> b) & 1u) << (2 * b) | ((qy >> b) & 1u) << (2 * b + 1);
    key[i] = {code, i};
  }
  std::sort(key.begin(), key.end());
  for (int64_t k = 0; k < n; ++k) perm[k] = key[k].second;
}

// Squared distance without contraction: the host compiler runs with -ffp-contract=off.
static inline double hd2(double ax, double ay, double bx, double by) {
  const double dx = ax - bx, dy = ay - by;
  const double px = dx * dx, py = dy * dy;
  return px + py;
}

struct HeapItem {
  double d;
  int64_t j;
};
struct HeapLess {  // max-heap on d, then min on index
  bool operator()(const HeapItem& a, const HeapItem& b) const {
    return a.d < b.d || (a.d == b.d && a.j > b.j);
  }
};

static void order_maxmin(int64_t n, const double* xy, int64_t* perm) {
  double sx = 0.0, sy = 0.0;
  for (int64_t i = 0; i < n; ++i) { sx += xy[2 * i]; sy += xy[2 * i + 1]; }
  const double cxm = sx / (double)n, cym = sy / (double)n;
  int64_t first = 0;
  double best = hd2(xy[0], xy[1], cxm, cym);
  for (int64_t i = 1; i < n; ++i) {
    const double d = hd2(xy[2 * i], xy[2 * i + 1], cxm, cym);
    if (d < best) { best = d; first = i; }
  }
  // fine grid, about one point per cell
  double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
  for (int64_t i = 1; i < n; ++i) {
    x0 = std::min(x0, xy[2 * i]); x1 = std::max(x1, xy[2 * i]);
    y0 = std::min(y0, xy[2 * i + 1]); y1 = std::max(y1, xy[2 * i + 1]);
  }
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t)std::sqrt((double)n)));
  const double ext = std::max(std::max(x1 - x0, y1 - y0), 1e-300);
  const double h = ext / G * (1.0 + 1e-9), ih = 1.0 / h;
  auto cell_of = [&](double v, double lo) {
    long c = (long)std::floor((v - lo) * ih);
    return (int)std::min<long>(G - 1, std::max<long>(0, c));
  };
  std::vector<int64_t> start((size_t)G * G + 1, 0), pts(n);
  std::vector<int> cid(n);
  for (int64_t i = 0; i < n; ++i) {
    cid[i] = cell_of(xy[2 * i + 1], y0) * G + cell_of(xy[2 * i], x0);
    start[cid[i] + 1]++;
  }
  for (size_t c = 0; c < (size_t)G * G; ++c) start[c + 1] += start[c];
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < n; ++i) pts[fill[cid[i]]++] = i;
  }
  std::vector<double> mind(n, INFINITY);
  std::vector<char> chosen(n, 0);
  std::vector<HeapItem> heap;
  heap.reserve((size_t)n * 2);
  perm[0] = first;
  chosen[first] = 1;
  for (int64_t j = 0; j < n; ++j) {
    if (j == first) continue;
    mind[j] = hd2(xy[2 * j], xy[2 * j + 1], xy[2 * first], xy[2 * first + 1]);
    heap.push_back({mind[j], j});
  }
  std::make_heap(heap.begin(), heap.end(), HeapLess());
  for (int64_t k = 1; k < n; ++k) {
    HeapItem top{0.0, -1};
    while (true) {
      std::pop_heap(heap.begin(), heap.end(), HeapLess());
      top = heap.back();
      heap.pop_back();
      if (!chosen[top.j] && mind[top.j] == top.d) break;
    }
    const int64_t j = top.j;
    perm[k] = j;
    chosen[j] = 1;
    const double px = xy[2 * j], py = xy[2 * j + 1];
    const double R = std::sqrt(top.d) * (1.0 + 1e-12);
    const int ax0 = std::max(0, cell_of(px - R, x0) - 1), ax1 = std::min(G - 1, cell_of(px + R, x0) + 1);
    const int ay0 = std::max(0, cell_of(py - R, y0) - 1), ay1 = std::min(G - 1, cell_of(py + R, y0) + 1);
    for (int ay = ay0; ay <= ay1; ++ay) {
      for (int ax = ax0; ax <= ax1; ++ax) {
        const size_t c = (size_t)ay * G + ax;
        for (int64_t t = start[c]; t < start[c + 1]; ++t) {
          const int64_t q = pts[t];
          if (chosen[q]) continue;
          const double d = hd2(xy[2 * q], xy[2 * q + 1], px, py);
          if (d < mind[q]) {
            mind[q] = d;
            heap.push_back({d, q});
            std::push_heap(heap.begin(), heap.end(), HeapLess());
          }
        }
      }
    }
    if (heap.size() > (size_t)n * 3) {  // drop stale entries
      heap.clear();
      for (int64_t q = 0; q < n; ++q)
        if (!chosen[q]) heap.push_back({mind[q], q});
      std::make_heap(heap.begin(), heap.end(), HeapLess());
    }
  }
}

// ------------------------------------------------------------------ GPU kNN
struct Level {
  int N;            // points [0, N) of the ordering
  int Gx, Gy;
  double x0, y0, h, ih;
  int64_t cell_off;  // into cell_start (Gx*Gy + 1 entries)
  int64_t pt_off;    // into pt_idx / pt_xy (N entries)
};

constexpr int kBrute = 1024;
constexpr int kMaxLevels = 32;

struct KnnArgs {
  const double2* __restrict__ xyo;       // ordered coordinates
  const int32_t* __restrict__ cell_start;
  const int32_t* __restrict__ pt_idx;
  const double2* __restrict__ pt_xy;
  const Level* __restrict__ levels;
  int nlev;
  int64_t n;
  int m;
  const int64_t* __restrict__ perm;      // ordered -> original
  int32_t* nbr;                          // n x m, ORIGINAL indices
};

__device__ __forceinline__ double kd2(double2 a, double2 b) {
  const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Lexicographic (d2, idx) "less than" on non-negative distances, compared as bits.
__device__ __forceinline__ bool lex_less(long long da, int ia, long long db, int ib) {
  return da < db || (da == db && ia < ib);
}

struct BestList {
  long long d[kMaxM + 1];
  int id[kMaxM + 1];
  int cnt;
  __device__ __forceinline__ void offer(long long dd, int j, int cap) {
    if (cnt == cap) {
      if (!lex_less(dd, j, d[cap - 1], id[cap - 1])) return;
      --cnt;
    }
    int p = cnt;
    while (p > 0 && lex_less(dd, j, d[p - 1], id[p - 1])) { d[p] = d[p - 1]; id[p] = id[p - 1]; --p; }
    d[p] = dd;
    id[p] = j;
    ++cnt;
  }
};

// Exact ring search of one query in one grid level: every point of the level with index
// below `limit` is a candidate (cell lists ascend in index); rings of cells are added
// until the m-th best distance is below the distance to the unscanned cells.
__device__ void ring_search(const KnnArgs& a, const Level& L, double2 q, int64_t limit, BestList& bl, int mi) {
  const int32_t* cs = a.cell_start + L.cell_off;
  const int32_t* pidx = a.pt_idx + L.pt_off;
  const double2* pxy = a.pt_xy + L.pt_off;
  const int cx = min(L.Gx - 1, max(0, (int)floor((q.x - L.x0) * L.ih)));
  const int cy = min(L.Gy - 1, max(0, (int)floor((q.y - L.y0) * L.ih)));
  const double slop = 1e-9 * L.h + 4e-16 * (fabs(L.x0) + fabs(L.y0) + L.h * (L.Gx + L.Gy));
  for (int R = 0;; ++R) {
    for (int dy = -R; dy <= R; ++dy) {
      const int ay = cy + dy;
      if (ay < 0 || ay >= L.Gy) continue;
      const bool edge = (dy == -R || dy == R);
      for (int dx = -R; dx <= R; dx += edge ? 1 : 2 * R) {
        const int ax = cx + dx;
        if (ax >= 0 && ax < L.Gx) {
          const int c = ay * L.Gx + ax;
          for (int t = cs[c]; t < cs[c + 1]; ++t) {
            const int j = pidx[t];
            if (j >= limit) break;  // cell lists ascend in index
            bl.offer(__double_as_longlong(kd2(q, pxy[t])), j, mi);
          }
        }
        if (R == 0) break;
      }
    }
    const bool all = (cx - R <= 0) && (cy - R <= 0) && (cx + R >= L.Gx - 1) && (cy + R >= L.Gy - 1);
    if (all) break;
    if (bl.cnt == mi) {
      // distance from q to the outside of the scanned square of cells
      double bd = INFINITY;
      if (cx - R > 0) bd = fmin(bd, q.x - (L.x0 + (cx - R) * L.h));
      if (cx + R < L.Gx - 1) bd = fmin(bd, (L.x0 + (cx + R + 1) * L.h) - q.x);
      if (cy - R > 0) bd = fmin(bd, q.y - (L.y0 + (cy - R) * L.h));
      if (cy + R < L.Gy - 1) bd = fmin(bd, (L.y0 + (cy + R + 1) * L.h) - q.y);
      bd -= slop;
      if (bd > 0.0 && bd * bd * (1.0 - 1e-12) > __longlong_as_double(bl.d[mi - 1])) break;
    }
  }
}

__global__ void knn_kernel(const KnnArgs a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int m = a.m;
  const int mi = (int)(i < m ? i : m);
  BestList bl;
  bl.cnt = 0;
  const double2 q = a.xyo[i];
  if (i <= kBrute) {
    for (int j = 0; j < (int)i; ++j) bl.offer(__double_as_longlong(kd2(q, a.xyo[j])), j, mi);
  } else {
    int lv = 0;
    while (lv < a.nlev - 1 && a.levels[lv].N < i) ++lv;
    ring_search(a, a.levels[lv], q, i, bl, mi);
  }
  int32_t* out = a.nbr + i * m;
  for (int p = 0; p < m; ++p) out[p] = p < bl.cnt ? (int32_t)a.perm[bl.id[p]] : -1;
}

// Prediction queries: the m nearest of ALL points of the single level (original order,
// so ties go to the lower original index) for each query point.
__global__ void knn_query_kernel(const KnnArgs a, const double2* __restrict__ queries, int64_t nq) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nq) return;
  BestList bl;
  bl.cnt = 0;
  ring_search(a, a.levels[0], queries[k], a.levels[0].N, bl, a.m);
  int32_t* out = a.nbr + k * a.m;
  for (int p = 0; p < a.m; ++p) out[p] = p < bl.cnt ? bl.id[p] : -1;
}

static void build_levels(int64_t n, const double* xyo, std::vector<Level>& lev, std::vector<int32_t>& cs,
                         std::vector<int32_t>& pidx, std::vector<double>& pxy, int64_t first_N = kBrute) {
  double x0 = xyo[0], x1 = xyo[0], y0 = xyo[1], y1 = xyo[1];
  for (int64_t i = 1; i < n; ++i) {
    x0 = std::min(x0, xyo[2 * i]); x1 = std::max(x1, xyo[2 * i]);
    y0 = std::min(y0, xyo[2 * i + 1]); y1 = std::max(y1, xyo[2 * i + 1]);
  }
  const double wx = std::max(x1 - x0, 1e-300), wy = std::max(y1 - y0, 1e-300);
  int64_t N = first_N;
  while (true) {
    const int64_t Nl = std::min<int64_t>(N, n);
    Level L;
    L.N = (int)Nl;
    const double cells = std::max(1.0, (double)Nl / 3.0);
    double h = std::sqrt(wx * wy / cells);
    if (wx < h) h = std::max(wx, wy / cells);
    if (wy < h) h = std::max(wy, wx / cells);
    L.Gx = (int)std::min<double>(8192, std::max(1.0, std::ceil(wx / h)));
    L.Gy = (int)std::min<double>(8192, std::max(1.0, std::ceil(wy / h)));
    L.h = std::max(wx / L.Gx, wy / L.Gy) * (1.0 + 1e-9);
    L.ih = 1.0 / L.h;
    L.x0 = x0;
    L.y0 = y0;
    L.cell_off = (int64_t)cs.size();
    L.pt_off = (int64_t)pidx.size();
    const int64_t nc = (int64_t)L.Gx * L.Gy;
    std::vector<int32_t> start(nc + 1, 0);
    std::vector<int32_t> cid(Nl);
    for (int64_t i = 0; i < Nl; ++i) {
      const int ax = (int)std::min<double>(L.Gx - 1, std::max(0.0, std::floor((xyo[2 * i] - L.x0) * L.ih)));
      const int ay = (int)std::min<double>(L.Gy - 1, std::max(0.0, std::floor((xyo[2 * i + 1] - L.y0) * L.ih)));
      cid[i] = ay * L.Gx + ax;
      start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) start[c + 1] += start[c];
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    const size_t base = pidx.size();
    pidx.resize(base + Nl);
    pxy.resize(2 * (base + Nl));
    for (int64_t i = 0; i < Nl; ++i) {  // ascending i keeps each cell sorted by index
      const int64_t t = base + fill[cid[i]]++;
      pidx[t] = (int32_t)i;
      pxy[2 * t] = xyo[2 * i];
      pxy[2 * t + 1] = xyo[2 * i + 1];
    }
    cs.insert(cs.end(), start.begin(), start.end());
    lev.push_back(L);
    if (Nl >= n || (int)lev.size() >= kMaxLevels) break;
    N *= 2;
  }
}

static int knn_gpu(Plan* p, const double* xy_host, cudaStream_t stream) {
  const int64_t n = p->n;
  std::vector<double> xyo(2 * n);
  for (int64_t k = 0; k < n; ++k) {
    xyo[2 * k] = xy_host[2 * p->h_perm[k]];
    xyo[2 * k + 1] = xy_host[2 * p->h_perm[k] + 1];
  }
  std::vector<Level> lev;
  std::vector<int32_t> cs, pidx;
  std::vector<double> pxy;
  build_levels(n, xyo.data(), lev, cs, pidx, pxy);
  double *d_xyo = nullptr, *d_pxy = nullptr;
  int32_t *d_cs = nullptr, *d_pidx = nullptr;
  Level* d_lev = nullptr;
  int64_t* d_perm = nullptr;
  int rc = VECCHIA_OK;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (rc) return;
    if (cudaMalloc(ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) rc = VECCHIA_ENOMEM;
  };
  alloc((void**)&d_xyo, sizeof(double) * 2 * n);
  alloc((void**)&d_pxy, sizeof(double) * pxy.size());
  alloc((void**)&d_cs, sizeof(int32_t) * cs.size());
  alloc((void**)&d_pidx, sizeof(int32_t) * pidx.size());
  alloc((void**)&d_lev, sizeof(Level) * lev.size());
  alloc((void**)&d_perm, sizeof(int64_t) * n);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (rc) return;
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  };
  up(d_xyo, xyo.data(), sizeof(double) * 2 * n);
  up(d_pxy, pxy.data(), sizeof(double) * pxy.size());
  up(d_cs, cs.data(), sizeof(int32_t) * cs.size());
  up(d_pidx, pidx.data(), sizeof(int32_t) * pidx.size());
  up(d_lev, lev.data(), sizeof(Level) * lev.size());
  up(d_perm, p->h_perm, sizeof(int64_t) * n);
  if (!rc) {
    KnnArgs a;
    a.xyo = reinterpret_cast<const double2*>(d_xyo);
    a.cell_start = d_cs;
    a.pt_idx = d_pidx;
    a.pt_xy = reinterpret_cast<const double2*>(d_pxy);
    a.levels = d_lev;
    a.nlev = (int)lev.size();
    a.n = n;
    a.m = p->m;
    a.perm = d_perm;
    a.nbr = p->d_nbr;
    const int threads = 128;
    knn_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) rc = VECCHIA_ECUDA;
  }
  if (!rc && cudaStreamSynchronize(stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  cudaFree(d_xyo);
  cudaFree(d_pxy);
  cudaFree(d_cs);
  cudaFree(d_pidx);
  cudaFree(d_lev);
  cudaFree(d_perm);
  return rc;
}

// ------------------------------------------------------------------ sphere
// Unit vectors of (longitude, latitude) points in degrees, on the host.
static void sphere_unit_vectors(int64_t n, const double* lonlat, double* xyz) {
  const double rad = 3.14159265358979323846 / 180.0;
  for (int64_t i = 0; i < n; ++i) {
    const double lam = lonlat[2 * i] * rad, phi = lonlat[2 * i + 1] * rad;
    const double cp = cos(phi);
    xyz[3 * i] = cp * cos(lam);
    xyz[3 * i + 1] = cp * sin(lam);
    xyz[3 * i + 2] = sin(phi);
  }
}

struct SphereKnnArgs {
  const double* __restrict__ xyzo;  // candidates: ordered unit vectors, n x 3
  int64_t n;
  int m;
  const int64_t* __restrict__ perm;  // ordered -> original (nullptr: candidates are in original order)
  int32_t* nbr;                      // rows x m, ORIGINAL indices
  const double* __restrict__ queries = nullptr;  // prediction: nq x 3 query unit vectors, all n candidates
  int64_t nq = 0;
};

constexpr int kSphereTile = 256;

// Brute-force search on the sphere: one thread per ordered query i scans every j < i,
// with CTA-wide tiles of candidates staged in shared memory.  Candidates whose FP32
// squared chord exceeds the current m-th best by more than its rounding bound are
// skipped; the rest are ranked by the exact FP64 key ((dx*dx + dy*dy) + dz*dz, no
// fused operations) and the index.
__global__ void __launch_bounds__(128) knn_sphere_kernel(const SphereKnnArgs a) {
  __shared__ double tx[kSphereTile], ty[kSphereTile], tz[kSphereTile];
  __shared__ float fx[kSphereTile], fy[kSphereTile], fz[kSphereTile];
  const bool query = a.queries != nullptr;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t i = i0 + threadIdx.x;
  const bool live = i < (query ? a.nq : a.n);
  const int m = a.m;
  const int mi = live ? (query ? m : (int)(i < m ? i : m)) : 0;
  const int64_t limit = query ? a.n : i;  // candidates j < limit
  BestList bl;
  bl.cnt = 0;
  double qx = 0.0, qy = 0.0, qz = 0.0;
  if (live) {
    const double* qp = query ? a.queries + 3 * i : a.xyzo + 3 * i;
    qx = qp[0];
    qy = qp[1];
    qz = qp[2];
  }
  const float gx = (float)qx, gy = (float)qy, gz = (float)qz;
  float wf = INFINITY;  // prefilter threshold (stays infinite until the list is full)
  // candidates any thread of the block needs: [0, jend)
  const int64_t jend = query ? a.n : min(a.n, i0 + (int64_t)blockDim.x) - 1;
  for (int64_t t0 = 0; t0 < jend; t0 += kSphereTile) {
    __syncthreads();
    for (int k = threadIdx.x; k < kSphereTile; k += blockDim.x) {
      const int64_t j = t0 + k;
      if (j < a.n) {
        const double x = a.xyzo[3 * j], y = a.xyzo[3 * j + 1], z = a.xyzo[3 * j + 2];
        tx[k] = x;
        ty[k] = y;
        tz[k] = z;
        fx[k] = (float)x;
        fy[k] = (float)y;
        fz[k] = (float)z;
      }
    }
    __syncthreads();
    if (!live) continue;
    const int kend = (int)min((int64_t)kSphereTile, limit - t0);
    for (int k = 0; k < kend; ++k) {
      const float ex = fx[k] - gx, ey = fy[k] - gy, ez = fz[k] - gz;
      if (ex * ex + ey * ey + ez * ez > wf) continue;
      const double dx = __dsub_rn(tx[k], qx), dy = __dsub_rn(ty[k], qy), dz = __dsub_rn(tz[k], qz);
      const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      const int cnt0 = bl.cnt;
      const long long worst0 = cnt0 == mi && mi > 0 ? bl.d[mi - 1] : -1;
      bl.offer(__double_as_longlong(d2), (int)(t0 + k), mi);
      if (bl.cnt == mi && mi > 0 && (cnt0 != mi || bl.d[mi - 1] != worst0)) {
        // FP32 chord^2 differs from the exact one by at most 6 * 2^-24 sqrt(3) |chord|
        // + 3 * 2^-24 chord^2 + 27 * 2^-48 (unit vectors): skip only beyond that.
        const double w = __longlong_as_double(bl.d[mi - 1]);
        wf = __double2float_ru(w + 1.2e-6 * sqrt(w) + 2.5e-7 * w + 3e-13);
      }
    }
  }
  if (!live) return;
  int32_t* out = a.nbr + i * m;
  for (int p = 0; p < m; ++p) out[p] = p < bl.cnt ? (int32_t)(a.perm ? a.perm[bl.id[p]] : bl.id[p]) : -1;
}

static int knn_sphere_gpu(Plan* p, const double* xyz_host, cudaStream_t stream) {
  const int64_t n = p->n;
  std::vector<double> xyzo(3 * n);
  for (int64_t k = 0; k < n; ++k)
    for (int c = 0; c < 3; ++c) xyzo[3 * k + c] = xyz_host[3 * p->h_perm[k] + c];
  double* d_xyzo = nullptr;
  int64_t* d_perm = nullptr;
  int rc = VECCHIA_OK;
  if (cudaMalloc(&d_xyzo, sizeof(double) * 3 * n) != cudaSuccess ||
      cudaMalloc(&d_perm, sizeof(int64_t) * n) != cudaSuccess)
    rc = VECCHIA_ENOMEM;
  if (!rc && (cudaMemcpyAsync(d_xyzo, xyzo.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, stream) !=
                  cudaSuccess ||
              cudaMemcpyAsync(d_perm, p->h_perm, sizeof(int64_t) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess))
    rc = VECCHIA_ECUDA;
  if (!rc) {
    SphereKnnArgs a;
    a.xyzo = d_xyzo;
    a.n = n;
    a.m = p->m;
    a.perm = d_perm;
    a.nbr = p->d_nbr;
    knn_sphere_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) rc = VECCHIA_ECUDA;
  }
  if (!rc && cudaStreamSynchronize(stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  cudaFree(d_xyzo);
  cudaFree(d_perm);
  return rc;
}

// Conditioning sets of prediction points: the m nearest OBSERVED points of the plan
// (all of them are candidates; ties to the lower original index), written to d_nbr_new
// (n_new x m, original indices) on `stream`.  xy_new_host: n_new x 2 (plane) or
// (longitude, latitude) in degrees (sphere); for the sphere, xyz_new_out receives the
// query unit vectors (n_new x 3, host).
int knn_predict(Plan* p, const double* xy_new_host, int64_t n_new, int32_t* d_nbr_new, std::vector<double>* xyz_new_out,
                cudaStream_t stream) {
  const int64_t n = p->n;
  int rc = VECCHIA_OK;
  if (p->metric == 1) {
    std::vector<double>& xyzq = *xyz_new_out;
    xyzq.resize(3 * n_new);
    sphere_unit_vectors(n_new, xy_new_host, xyzq.data());
    double* d_q = nullptr;
    if (cudaMalloc(&d_q, sizeof(double) * 3 * n_new) != cudaSuccess) return VECCHIA_ENOMEM;
    if (cudaMemcpyAsync(d_q, xyzq.data(), sizeof(double) * 3 * n_new, cudaMemcpyHostToDevice, stream) != cudaSuccess)
      rc = VECCHIA_ECUDA;
    if (!rc) {
      SphereKnnArgs a;
      a.xyzo = p->d_xyz;  // original order
      a.n = n;
      a.m = p->m;
      a.perm = nullptr;
      a.nbr = d_nbr_new;
      a.queries = d_q;
      a.nq = n_new;
      knn_sphere_kernel<<<(unsigned)((n_new + 127) / 128), 128, 0, stream>>>(a);
      if (cudaGetLastError() != cudaSuccess) rc = VECCHIA_ECUDA;
    }
    if (!rc && cudaStreamSynchronize(stream) != cudaSuccess) rc = VECCHIA_ECUDA;
    cudaFree(d_q);
    return rc;
  }
  std::vector<double> xy(2 * n);
  if (cudaMemcpy(xy.data(), p->d_xy, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return VECCHIA_ECUDA;
  std::vector<Level> lev;
  std::vector<int32_t> cs, pidx;
  std::vector<double> pxy;
  build_levels(n, xy.data(), lev, cs, pidx, pxy, n);  // one level over all points, original order
  double *d_pxy = nullptr, *d_q = nullptr;
  int32_t *d_cs = nullptr, *d_pidx = nullptr;
  Level* d_lev = nullptr;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (rc) return;
    if (cudaMalloc(ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) rc = VECCHIA_ENOMEM;
  };
  alloc((void**)&d_pxy, sizeof(double) * pxy.size());
  alloc((void**)&d_cs, sizeof(int32_t) * cs.size());
  alloc((void**)&d_pidx, sizeof(int32_t) * pidx.size());
  alloc((void**)&d_lev, sizeof(Level) * lev.size());
  alloc((void**)&d_q, sizeof(double) * 2 * n_new);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (rc) return;
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  };
  up(d_pxy, pxy.data(), sizeof(double) * pxy.size());
  up(d_cs, cs.data(), sizeof(int32_t) * cs.size());
  up(d_pidx, pidx.data(), sizeof(int32_t) * pidx.size());
  up(d_lev, lev.data(), sizeof(Level) * lev.size());
  up(d_q, xy_new_host, sizeof(double) * 2 * n_new);
  if (!rc) {
    KnnArgs a;
    a.xyo = nullptr;
    a.cell_start = d_cs;
    a.pt_idx = d_pidx;
    a.pt_xy = reinterpret_cast<const double2*>(d_pxy);
    a.levels = d_lev;
    a.nlev = (int)lev.size();
    a.n = n;
    a.m = p->m;
    a.perm = nullptr;
    a.nbr = d_nbr_new;
    knn_query_kernel<<<(unsigned)((n_new + 127) / 128), 128, 0, stream>>>(a, reinterpret_cast<const double2*>(d_q),
                                                                           n_new);
    if (cudaGetLastError() != cudaSuccess) rc = VECCHIA_ECUDA;
  }
  if (!rc && cudaStreamSynchronize(stream) != cudaSuccess) rc = VECCHIA_ECUDA;
  cudaFree(d_pxy);
  cudaFree(d_cs);
  cudaFree(d_pidx);
  cudaFree(d_lev);
  cudaFree(d_q);
  return rc;
}

static void plan_free(Plan* p) {
  if (!p) return;
  cudaFree(p->d_xyz);
  cudaFree(p->d_xy);
  cudaFree(p->d_nbr);
  cudaFree(p->d_self);
  cudaFree(p->d_inv);
  cudaFree(p->d_partial);
  cudaFree(p->d_errloc);
  delete[] p->h_perm;
  delete p;
}

int launch_loglik(Plan* p, const double* y_dev, const double* theta, bool grad, double* out_dev,
                  double* terms_dev, cudaStream_t stream, int64_t i0, int64_t i1);
int predict(Plan* p, const double* xy_new_host, int64_t n_new, const double* y_dev, const double* theta,
            double* mean_dev, double* var_dev, int32_t* nbr_host, cudaStream_t stream);
void forget_plan_in_batches(const void* plan);
int autotune(Plan* p, const double* y_dev, const double* theta, bool grad, int* G_out, int* W_out,
             cudaStream_t stream);

// Plan construction for both metrics (metric 0: plane, 1: sphere of the given radius).
static int plan_create(const double* xy_host, int64_t n, int32_t m, int order, uint64_t seed,
                       const int64_t* perm_in, int metric, double radius, void* stream, vecchia_plan_t* out) {
  if (!out) return VECCHIA_EINVAL;
  *out = nullptr;
  if (!xy_host || n < 1 || n > 2147483647LL || m < 1 || m > kMaxM) return VECCHIA_EINVAL;
  if (order != VECCHIA_ORDER_GIVEN && order != VECCHIA_ORDER_RANDOM && order != VECCHIA_ORDER_MAXMIN &&
      order != VECCHIA_ORDER_MORTON)
    return VECCHIA_EINVAL;
  for (int64_t i = 0; i < 2 * n; ++i)
    if (!std::isfinite(xy_host[i])) return VECCHIA_EINVAL;
  if (metric == 1) {
    if (!(radius > 0.0) || !std::isfinite(radius)) return VECCHIA_EINVAL;
    if (order != VECCHIA_ORDER_GIVEN && order != VECCHIA_ORDER_RANDOM) return VECCHIA_EINVAL;
    for (int64_t i = 0; i < n; ++i)
      if (!(fabs(xy_host[2 * i + 1]) <= 90.0)) return VECCHIA_EINVAL;
  }
  vecchia_plan* p = new (std::nothrow) vecchia_plan();
  if (!p) return VECCHIA_ENOMEM;
  p->n = n;
  p->m = m;
  p->metric = metric;
  p->radius = radius;
  cudaGetDevice(&p->device);
  p->h_perm = new (std::nothrow) int64_t[n];
  if (!p->h_perm) { plan_free(p); return VECCHIA_ENOMEM; }
  if (order == VECCHIA_ORDER_GIVEN) {
    if (!perm_in) { plan_free(p); return VECCHIA_EINVAL; }
    std::vector<char> seen(n, 0);
    for (int64_t k = 0; k < n; ++k) {
      const int64_t v = perm_in[k];
      if (v < 0 || v >= n || seen[v]) { plan_free(p); return VECCHIA_EINVAL; }
      seen[v] = 1;
      p->h_perm[k] = v;
    }
  } else if (order == VECCHIA_ORDER_RANDOM) {
    order_random(n, seed, p->h_perm);
  } else if (order == VECCHIA_ORDER_MAXMIN) {
    order_maxmin(n, xy_host, p->h_perm);
  } else {
    order_morton(n, xy_host, p->h_perm);
  }
  cudaStream_t s = (cudaStream_t)stream;
  int rc = VECCHIA_OK;
  if (cudaMalloc(&p->d_xy, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMalloc(&p->d_nbr, sizeof(int32_t) * n * m) != cudaSuccess ||
      cudaMalloc(&p->d_self, sizeof(int32_t) * n) != cudaSuccess ||
      cudaMalloc(&p->d_inv, sizeof(int32_t) * n) != cudaSuccess ||
      cudaMalloc(&p->d_errloc, sizeof(unsigned long long)) != cudaSuccess ||
      (metric == 1 && cudaMalloc(&p->d_xyz, sizeof(double) * 3 * n) != cudaSuccess)) {
    plan_free(p);
    return VECCHIA_ENOMEM;
  }
  std::vector<int32_t> self(n), inv(n);
  for (int64_t k = 0; k < n; ++k) {
    self[k] = (int32_t)p->h_perm[k];
    inv[p->h_perm[k]] = (int32_t)k;
  }
  std::vector<double> xyz;
  if (metric == 1) {
    xyz.resize(3 * n);
    sphere_unit_vectors(n, xy_host, xyz.data());
  }
  if (cudaMemcpyAsync(p->d_xy, xy_host, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p->d_self, self.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p->d_inv, inv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(p->d_errloc, 0xFF, sizeof(unsigned long long), s) != cudaSuccess ||
      (metric == 1 && cudaMemcpyAsync(p->d_xyz, xyz.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s) !=
                          cudaSuccess)) {
    plan_free(p);
    return VECCHIA_ECUDA;
  }
  rc = metric == 1 ? knn_sphere_gpu(p, xyz.data(), s) : knn_gpu(p, xy_host, s);
  if (rc) { plan_free(p); return rc; }
  p->last_stream = s;
  *out = p;
  return VECCHIA_OK;
}

}  // namespace vecchia

using vecchia::Plan;

extern "C" {

int vecchia_plan_create(const double* xy_host, int64_t n, int32_t m, int order, uint64_t seed,
                        const int64_t* perm_in, void* stream, vecchia_plan_t* out) {
  return vecchia::plan_create(xy_host, n, m, order, seed, perm_in, 0, 1.0, stream, out);
}

int vecchia_plan_create_sphere(const double* lonlat_host, int64_t n, int32_t m, int order, uint64_t seed,
                               const int64_t* perm_in, double radius, void* stream, vecchia_plan_t* out) {
  return vecchia::plan_create(lonlat_host, n, m, order, seed, perm_in, 1, radius, stream, out);
}

void vecchia_plan_destroy(vecchia_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  vecchia::forget_plan_in_batches(plan);
  vecchia::plan_free(plan);
}

int vecchia_plan_set_kernel(vecchia_plan_t plan, int kernel) {
  if (!plan || (kernel != VECCHIA_KERNEL_MATERN && kernel != VECCHIA_KERNEL_POWEXP)) return VECCHIA_EINVAL;
  plan->family = kernel;
  return VECCHIA_OK;
}

int vecchia_plan_size(vecchia_plan_t plan, int64_t* n, int32_t* m) {
  if (!plan) return VECCHIA_EINVAL;
  if (n) *n = plan->n;
  if (m) *m = plan->m;
  return VECCHIA_OK;
}

int vecchia_plan_perm(vecchia_plan_t plan, int64_t* perm_out) {
  if (!plan || !perm_out) return VECCHIA_EINVAL;
  std::memcpy(perm_out, plan->h_perm, sizeof(int64_t) * plan->n);
  return VECCHIA_OK;
}

int vecchia_plan_neighbors(vecchia_plan_t plan, int32_t* nbr_out) {
  if (!plan || !nbr_out) return VECCHIA_EINVAL;
  const int64_t total = plan->n * plan->m;
  VECCHIA_CUDA_TRY(cudaStreamSynchronize(plan->last_stream));
  VECCHIA_CUDA_TRY(cudaMemcpy(nbr_out, plan->d_nbr, sizeof(int32_t) * total, cudaMemcpyDeviceToHost));
  std::vector<int32_t> inv(plan->n);
  for (int64_t k = 0; k < plan->n; ++k) inv[plan->h_perm[k]] = (int32_t)k;
  for (int64_t t = 0; t < total; ++t)
    if (nbr_out[t] >= 0) nbr_out[t] = inv[nbr_out[t]];
  return VECCHIA_OK;
}

int vecchia_loglik(vecchia_plan_t plan, const double* y_dev, const double theta[4], double* out_dev,
                   void* stream) {
  if (!out_dev) return VECCHIA_EINVAL;
  return vecchia::launch_loglik(plan, y_dev, theta, false, out_dev, nullptr, (cudaStream_t)stream, 0, -1);
}

int vecchia_loglik_grad(vecchia_plan_t plan, const double* y_dev, const double theta[4], double* out_dev,
                        void* stream) {
  if (!out_dev) return VECCHIA_EINVAL;
  return vecchia::launch_loglik(plan, y_dev, theta, true, out_dev, nullptr, (cudaStream_t)stream, 0, -1);
}

int vecchia_loglik_terms(vecchia_plan_t plan, const double* y_dev, const double theta[4], int want_grad,
                         double* terms_dev, void* stream) {
  if (!terms_dev) return VECCHIA_EINVAL;
  return vecchia::launch_loglik(plan, y_dev, theta, want_grad != 0, nullptr, terms_dev, (cudaStream_t)stream, 0, -1);
}

int vecchia_loglik_range(vecchia_plan_t plan, const double* y_dev, const double theta[4], int64_t i0, int64_t i1,
                         int want_grad, double* out_dev, void* stream) {
  if (!out_dev || i0 < 0 || i1 < i0) return VECCHIA_EINVAL;
  return vecchia::launch_loglik(plan, y_dev, theta, want_grad != 0, out_dev, nullptr, (cudaStream_t)stream, i0, i1);
}

int vecchia_autotune(vecchia_plan_t plan, const double* y_dev, const double theta[4], int want_grad,
                     int32_t* lanes_out, int32_t* warps_out, void* stream) {
  int G = 0, W = 0;
  const int rc = vecchia::autotune(plan, y_dev, theta, want_grad != 0, &G, &W, (cudaStream_t)stream);
  if (rc) return rc;
  if (lanes_out) *lanes_out = G;
  if (warps_out) *warps_out = W;
  return VECCHIA_OK;
}

int vecchia_predict(vecchia_plan_t plan, const double* xy_new_host, int64_t n_new, const double* y_dev,
                    const double theta[4], double* mean_dev, double* var_dev, int32_t* nbr_host, void* stream) {
  return vecchia::predict(plan, xy_new_host, n_new, y_dev, theta, mean_dev, var_dev, nbr_host, (cudaStream_t)stream);
}

int vecchia_last_error_location(vecchia_plan_t plan, int64_t* loc) {
  if (!plan || !loc) return VECCHIA_EINVAL;
  VECCHIA_CUDA_TRY(cudaStreamSynchronize(plan->last_stream));
  unsigned long long v = 0;
  VECCHIA_CUDA_TRY(cudaMemcpy(&v, plan->d_errloc, sizeof(v), cudaMemcpyDeviceToHost));
  if (v == ~0ULL) {
    *loc = -1;
    return VECCHIA_OK;
  }
  *loc = (int64_t)(v >> 2);
  return (v & 3u) == vecchia::kErrNotPD ? VECCHIA_ENOTPD : VECCHIA_EINVAL;
}

const char* vecchia_strerror(int code) {
  switch (code) {
    case VECCHIA_OK: return "success";
    case VECCHIA_EINVAL: return "invalid argument";
    case VECCHIA_ENOTPD: return "conditional covariance block not positive definite";
    case VECCHIA_ECUDA: return "CUDA runtime error";
    case VECCHIA_ETIMEOUT: return "device-side wait timed out";
    case VECCHIA_ENOMEM: return "out of memory";
    default: return "unknown status code";
  }
}

}  // extern "C"

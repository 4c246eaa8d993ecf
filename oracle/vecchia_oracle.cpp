// Vecchia log-likelihood ORACLE — test infrastructure only.
//
// Plain, slow, obviously-correct FP64 CPU implementation of what the GPU path
// computes, written from the paper (arXiv 2403.07412).  Only tests/, the smoke
// check and bench.py's cpu_baseline / reference arm may load it.  It shares no
// code with the CUDA library: its own Cholesky, its own kNN, its own orderings,
// and the Matérn covariance through the C++17 library routine
// std::cyl_bessel_k (an independent implementation of K_nu).
//
// Every function cites the passage it follows:
//   Eq. (1)  exact Gaussian log-likelihood                       (Sec. IV-A)
//   Eq. (2)  Matérn covariance, theta = (sigma^2, beta, nu)      (Sec. IV-A)
//   Eq. (3)  power-exponential covariance (real-data model, Sec. VI-C)
//   Vecchia factorisation p(y1) prod p(y_i | y_{J_i})             (Sec. V-B)
//   Algorithm 1: permutation, m nearest previously-ordered
//   neighbours, conditional mean / variance, univariate terms     (Sec. V-B)
//   Sec. V-A: random and maxmin orderings.
//   Sec. VI-C: great-circle distance by the haversine formula (longitude/latitude
//   data), used with a sphere of given radius.
// Readings where the paper is silent (nugget, ties, maxmin start, short early
// conditioning sets, splitmix64 Fisher–Yates) are listed in the design notes and
// restated at each function below.
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC
// (-ffp-contract=off: squared distances are round(round(dx*dx)+round(dy*dy)),
//  never a fused multiply-add, so kNN selections are reproducible bit for bit.)

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kLog2Pi = 1.8378770664093454835606594728112;  // log(2*pi)
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- covariance
// Eq. (2): C(d) = sigma2 * 2^(1-nu)/Gamma(nu) * (d/beta)^nu * K_nu(d/beta),
// with the d -> 0 limit C(0) = sigma2.  No sqrt(2 nu) factor (the paper's form).
double matern(double d, double sigma2, double beta, double nu) {
  if (d == 0.0) return sigma2;
  const double x = d / beta;
  const double k = std::cyl_bessel_k(nu, x);
  if (k == 0.0) return 0.0;  // far field: K_nu underflowed
  return sigma2 * std::pow(2.0, 1.0 - nu) / std::tgamma(nu) * std::pow(x, nu) * k;
}

// dC/dbeta from Eq. (2): d/dx[x^nu K_nu(x)] = -x^nu K_{nu-1}(x) (DLMF 10.29.4)
// and dx/dbeta = -x/beta, so dC/dbeta = sigma2 c_nu x^(nu+1) K_{nu-1}(x) / beta,
// with K_{-mu} = K_mu (DLMF 10.27.3).  Zero at d = 0.
double matern_dbeta(double d, double sigma2, double beta, double nu) {
  if (d == 0.0) return 0.0;
  const double x = d / beta;
  const double k = std::cyl_bessel_k(std::fabs(nu - 1.0), x);
  if (k == 0.0) return 0.0;
  return sigma2 * std::pow(2.0, 1.0 - nu) / std::tgamma(nu) * std::pow(x, nu + 1.0) * k / beta;
}

// Eq. (3), the power-exponential covariance: C(d) = sigma2 exp(-d^nu / beta), and
// dC/dbeta = sigma2 exp(-d^nu/beta) d^nu / beta^2 (here nu is the exponent alpha).
double powexp(double d, double sigma2, double beta, double nu) {
  return sigma2 * std::exp(-std::pow(d, nu) / beta);
}

double powexp_dbeta(double d, double sigma2, double beta, double nu) {
  const double a = std::pow(d, nu);
  return sigma2 * std::exp(-a / beta) * a / (beta * beta);
}

// Covariance family 0 = Matérn (Eq. 2), 1 = power exponential (Eq. 3).
double cov(int family, double d, double sigma2, double beta, double nu) {
  return family == 1 ? powexp(d, sigma2, beta, nu) : matern(d, sigma2, beta, nu);
}

double cov_dbeta(int family, double d, double sigma2, double beta, double nu) {
  return family == 1 ? powexp_dbeta(d, sigma2, beta, nu) : matern_dbeta(d, sigma2, beta, nu);
}

// Squared Euclidean distance, evaluated as round(round(dx*dx) + round(dy*dy)).
inline double dist2(const double* a, const double* b) {
  const double dx = a[0] - b[0];
  const double dy = a[1] - b[1];
  const double px = dx * dx;
  const double py = dy * dy;
  return px + py;
}

// Great-circle distance (Sec. VI-C): with latitudes phi and longitudes lambda in
// radians, hav(d / r) = hav(phi2 - phi1) + cos(phi1) cos(phi2) hav(lambda2 - lambda1),
// hav(x) = sin^2(x / 2), so d = 2 r asin(sqrt(h)).  Points are (longitude, latitude)
// in degrees.
double gcd(const double* a, const double* b, double radius) {
  const double rad = kPi / 180.0;
  const double p1 = a[1] * rad, p2 = b[1] * rad;
  const double sp = std::sin(0.5 * (p2 - p1));
  const double sl = std::sin(0.5 * (b[0] - a[0]) * rad);
  double h = sp * sp + std::cos(p1) * std::cos(p2) * (sl * sl);
  if (h > 1.0) h = 1.0;
  return 2.0 * radius * std::asin(std::sqrt(h));
}

// Distance between points p and q: Euclidean in the plane (metric 0, pts n x 2 in the
// plane) or great-circle on a sphere of the given radius (metric 1, pts n x 2 as
// longitude/latitude in degrees).
inline double point_dist(const double* pts, int64_t p, int64_t q, int metric, double radius) {
  if (metric == 1) return gcd(pts + 2 * p, pts + 2 * q, radius);
  return std::sqrt(dist2(pts + 2 * p, pts + 2 * q));
}

// Unit vector of a (longitude, latitude) point in degrees:
// (cos(phi) cos(lambda), cos(phi) sin(lambda), sin(phi)).  The nearest-neighbour
// search on the sphere ranks candidates by the squared chord between these vectors,
// which increases with the great-circle distance (chord = 2 sin(d / 2r)).
void unit_vector(const double* lonlat, double* out) {
  const double rad = kPi / 180.0;
  const double lam = lonlat[0] * rad, phi = lonlat[1] * rad;
  const double cp = std::cos(phi);
  out[0] = cp * std::cos(lam);
  out[1] = cp * std::sin(lam);
  out[2] = std::sin(phi);
}

// Squared chord, evaluated as round(round(round(dx*dx) + round(dy*dy)) + round(dz*dz)).
inline double chord2(const double* a, const double* b) {
  const double dx = a[0] - b[0];
  const double dy = a[1] - b[1];
  const double dz = a[2] - b[2];
  const double px = dx * dx;
  const double py = dy * dy;
  const double pz = dz * dz;
  return (px + py) + pz;
}

// ---------------------------------------------------------------- dense algebra
// Textbook Cholesky (Cholesky–Banachiewicz, row by row), A = L L^T, A is k x k
// row-major, L written into a separate k x k array (upper part zero).
// Returns false if a pivot is <= 0 or not finite.
bool cholesky(int k, const double* A, double* L) {
  std::fill(L, L + (size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = A[(size_t)i * k + j];
      for (int p = 0; p < j; ++p) s -= L[(size_t)i * k + p] * L[(size_t)j * k + p];
      if (i == j) {
        if (!(s > 0.0) || !std::isfinite(s)) return false;
        L[(size_t)i * k + i] = std::sqrt(s);
      } else {
        L[(size_t)i * k + j] = s / L[(size_t)j * k + j];
      }
    }
  }
  return true;
}

// Solve A x = b with the Cholesky factor L (forward then backward substitution).
void chol_solve(int k, const double* L, const double* b, double* x) {
  std::vector<double> z(k);
  for (int i = 0; i < k; ++i) {
    double s = b[i];
    for (int p = 0; p < i; ++p) s -= L[(size_t)i * k + p] * z[p];
    z[i] = s / L[(size_t)i * k + i];
  }
  for (int i = k - 1; i >= 0; --i) {
    double s = z[i];
    for (int p = i + 1; p < k; ++p) s -= L[(size_t)p * k + i] * x[p];
    x[i] = s / L[(size_t)i * k + i];
  }
}

// A^{-1} from its Cholesky factor, column by column.
void chol_inverse(int k, const double* L, double* Ainv) {
  std::vector<double> e(k), col(k);
  for (int c = 0; c < k; ++c) {
    std::fill(e.begin(), e.end(), 0.0);
    e[c] = 1.0;
    chol_solve(k, L, e.data(), col.data());
    for (int r = 0; r < k; ++r) Ainv[(size_t)r * k + c] = col[r];
  }
}

// Neumaier's compensated summation, in index order.
struct Neumaier {
  double s = 0.0, c = 0.0;
  void add(double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// ---------------------------------------------------------------- neighbours
// Algorithm 1 (nearest-neighbour loop): J_i = the m_i = min(i, m) points among
// the previously ordered points 0..i-1 (0-based) with the smallest (d^2, index),
// lexicographically; listed in that ascending order.
void knn_row(const double* xy, int64_t i, int m, int32_t* out) {
  const int mi = (int)std::min<int64_t>(i, m);
  std::vector<double> bd(mi);
  std::vector<int64_t> bj(mi);
  int cnt = 0;
  for (int64_t j = 0; j < i; ++j) {
    const double d = dist2(xy + 2 * i, xy + 2 * j);
    if (cnt == mi) {
      // j increases, so an equal distance never beats an already-kept index.
      if (!(d < bd[mi - 1])) continue;
      --cnt;
    }
    int p = cnt;
    while (p > 0 && (d < bd[p - 1])) { bd[p] = bd[p - 1]; bj[p] = bj[p - 1]; --p; }
    bd[p] = d; bj[p] = j; ++cnt;
  }
  for (int p = 0; p < m; ++p) out[p] = p < mi ? (int32_t)bj[p] : -1;
}

// The same search on the sphere: xyz are unit vectors (n x 3), keys (chord^2, index).
void knn_row_sphere(const double* xyz, int64_t i, int m, int32_t* out) {
  const int mi = (int)std::min<int64_t>(i, m);
  std::vector<double> bd(mi);
  std::vector<int64_t> bj(mi);
  int cnt = 0;
  for (int64_t j = 0; j < i; ++j) {
    const double d = chord2(xyz + 3 * i, xyz + 3 * j);
    if (cnt == mi) {
      if (!(d < bd[mi - 1])) continue;
      --cnt;
    }
    int p = cnt;
    while (p > 0 && (d < bd[p - 1])) { bd[p] = bd[p - 1]; bj[p] = bj[p - 1]; --p; }
    bd[p] = d; bj[p] = j; ++cnt;
  }
  for (int p = 0; p < m; ++p) out[p] = p < mi ? (int32_t)bj[p] : -1;
}

// ---------------------------------------------------------------- one location
// Vecchia term for ordered location i with conditioning set J (Sec. V-B):
//   mu_i = Sigma_iJ Sigma_JJ^{-1} y_J,   s_i = Sigma_ii - Sigma_iJ Sigma_JJ^{-1} Sigma_Ji,
//   l_i  = -1/2 (y_i - mu_i)^2 / s_i - 1/2 log s_i - 1/2 log(2 pi).
// sigma^new of Algorithm 1 is read as the conditional standard deviation sqrt(s_i).
// The nugget tau2 is added to every diagonal entry (a location's own variance).
// If grad != nullptr, also d l_i / d(sigma2, beta, tau2) by the identity
//   l_i = log N(y_B; 0, Sigma_B) - log N(y_J; 0, Sigma_J),  B = J u {i},
//   d log N(y; 0, S)/d theta_p = -1/2 tr(S^{-1} S_p) + 1/2 a^T S_p a,  a = S^{-1} y,
// with S_sigma2 = (S - tau2 I)/sigma2, S_tau2 = I, S_beta = [dC/dbeta(d_pq)].
int location_term(const double* xy, const double* y, int64_t i, const int32_t* J, int mi,
                  const double* theta, int family, int metric, double radius, double* term, double* grad,
                  double* mu_out, double* s_out) {
  const double sigma2 = theta[0], beta = theta[1], nu = theta[2], tau2 = theta[3];
  const int k = mi + 1;  // block B = J followed by i
  std::vector<int64_t> idx(k);
  for (int p = 0; p < mi; ++p) idx[p] = J[p];
  idx[mi] = i;
  std::vector<double> S((size_t)k * k), D((size_t)k * k);
  for (int p = 0; p < k; ++p) {
    for (int q = 0; q < k; ++q) {
      const double d = p == q ? 0.0 : point_dist(xy, idx[p], idx[q], metric, radius);
      S[(size_t)p * k + q] = (p == q ? sigma2 + tau2 : cov(family, d, sigma2, beta, nu));
      if (grad) D[(size_t)p * k + q] = (p == q ? 0.0 : cov_dbeta(family, d, sigma2, beta, nu));
    }
  }
  const double cii = S[(size_t)mi * k + mi];
  double mu = 0.0, s = cii;
  if (mi > 0) {
    std::vector<double> SJ((size_t)mi * mi), LJ((size_t)mi * mi), v(mi), w(mi);
    for (int p = 0; p < mi; ++p) {
      for (int q = 0; q < mi; ++q) SJ[(size_t)p * mi + q] = S[(size_t)p * k + q];
      v[p] = S[(size_t)p * k + mi];
    }
    if (!cholesky(mi, SJ.data(), LJ.data())) return 2;
    chol_solve(mi, LJ.data(), v.data(), w.data());   // w = Sigma_JJ^{-1} Sigma_Ji
    double vw = 0.0;
    for (int p = 0; p < mi; ++p) { mu += w[p] * y[idx[p]]; vw += w[p] * v[p]; }
    s = cii - vw;
  }
  if (!(s > 0.0) || !std::isfinite(s)) return 2;
  const double r = y[i] - mu;
  *term = -0.5 * r * r / s - 0.5 * std::log(s) - 0.5 * kLog2Pi;
  if (mu_out) *mu_out = mu;
  if (s_out) *s_out = s;
  if (!grad) return 0;

  // Gradient by the joint-minus-marginal trace identity (explicit inverses).
  auto dlogN = [&](int kk, double out[3]) -> int {
    std::vector<double> SS((size_t)kk * kk), LL((size_t)kk * kk), Si((size_t)kk * kk), yy(kk), a(kk);
    for (int p = 0; p < kk; ++p) {
      yy[p] = y[idx[p]];
      for (int q = 0; q < kk; ++q) SS[(size_t)p * kk + q] = S[(size_t)p * k + q];
    }
    if (!cholesky(kk, SS.data(), LL.data())) return 2;
    chol_inverse(kk, LL.data(), Si.data());
    chol_solve(kk, LL.data(), yy.data(), a.data());
    for (int t = 0; t < 3; ++t) {
      double tr = 0.0, quad = 0.0;
      for (int p = 0; p < kk; ++p) {
        for (int q = 0; q < kk; ++q) {
          double Sp;
          if (t == 0) Sp = (SS[(size_t)p * kk + q] - (p == q ? tau2 : 0.0)) / sigma2;
          else if (t == 1) Sp = D[(size_t)p * k + q];
          else Sp = (p == q ? 1.0 : 0.0);
          tr += Si[(size_t)q * kk + p] * Sp;
          quad += a[p] * Sp * a[q];
        }
      }
      out[t] = -0.5 * tr + 0.5 * quad;
    }
    return 0;
  };
  double gB[3], gJ[3] = {0.0, 0.0, 0.0};
  if (dlogN(k, gB)) return 2;
  if (mi > 0 && dlogN(mi, gJ)) return 2;
  for (int t = 0; t < 3; ++t) grad[t] = gB[t] - gJ[t];
  return 0;
}

uint64_t splitmix64_next(uint64_t& state) {
  // splitmix64 (Steele, Lea, Flood, OOPSLA 2014): golden-gamma increment, then
  // two xor-shift-multiply mixing rounds.
  state += 0x9E3779B97F4A7C15ULL;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

// Eq. (2) on an array of distances.
int oracle_matern(int64_t n, const double* d, double sigma2, double beta, double nu, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = matern(d[i], sigma2, beta, nu);
  return 0;
}

int oracle_matern_dbeta(int64_t n, const double* d, double sigma2, double beta, double nu, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = matern_dbeta(d[i], sigma2, beta, nu);
  return 0;
}

int oracle_powexp(int64_t n, const double* d, double sigma2, double beta, double nu, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = powexp(d[i], sigma2, beta, nu);
  return 0;
}

int oracle_powexp_dbeta(int64_t n, const double* d, double sigma2, double beta, double nu, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = powexp_dbeta(d[i], sigma2, beta, nu);
  return 0;
}

int oracle_bessel_k(int64_t n, const double* x, double nu, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = std::cyl_bessel_k(nu, x[i]);
  return 0;
}

void oracle_splitmix64(uint64_t seed, int64_t count, uint64_t* out) {
  uint64_t s = seed;
  for (int64_t i = 0; i < count; ++i) out[i] = splitmix64_next(s);
}

// Random ordering (Sec. V-A, Algorithm 1 permutation step): Fisher–Yates
// (Durstenfeld) shuffle of the identity, i from n-1 down to 1, swap position i
// with j = splitmix64() mod (i+1); state seeded with `seed`.
// perm[k] = original index of the k-th ordered location.
int oracle_order_random(int64_t n, uint64_t seed, int64_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  uint64_t s = seed;
  for (int64_t i = n - 1; i >= 1; --i) {
    const int64_t j = (int64_t)(splitmix64_next(s) % (uint64_t)(i + 1));
    std::swap(perm[i], perm[j]);
  }
  return 0;
}

// Maxmin ordering (Sec. V-A; the paper gives no details): start at the point
// nearest the centroid (sums in index order), then repeatedly take the point
// whose minimum squared distance to the chosen set is largest; ties go to the
// lowest original index.  O(n^2), parallel over points.
// oracle_order_maxmin_prefix stops after the first `count` picks (perm holds count
// entries): the same greedy steps, so its output is a prefix of the full ordering.
int oracle_order_maxmin_prefix(int64_t n, const double* xy, int64_t count, int64_t* perm) {
  if (n <= 0 || count <= 0) return 0;
  if (count > n) return 1;
  double sx = 0.0, sy = 0.0;
  for (int64_t i = 0; i < n; ++i) { sx += xy[2 * i]; sy += xy[2 * i + 1]; }
  const double c[2] = {sx / (double)n, sy / (double)n};
  int64_t first = 0;
  double best = dist2(xy, c);
  for (int64_t i = 1; i < n; ++i) {
    const double d = dist2(xy + 2 * i, c);
    if (d < best) { best = d; first = i; }
  }
  std::vector<double> mind(n, std::numeric_limits<double>::infinity());
  std::vector<char> used(n, 0);
  perm[0] = first;
  used[first] = 1;
  int64_t last = first;
  for (int64_t k = 1; k < count; ++k) {
    double gbest = -1.0;
    int64_t gidx = -1;
#pragma omp parallel
    {
      double tb = -1.0;
      int64_t ti = -1;
#pragma omp for schedule(static)
      for (int64_t j = 0; j < n; ++j) {
        if (used[j]) continue;
        const double d = dist2(xy + 2 * j, xy + 2 * last);
        if (d < mind[j]) mind[j] = d;
        if (mind[j] > tb || (mind[j] == tb && j < ti)) { tb = mind[j]; ti = j; }
      }
#pragma omp critical
      {
        if (ti >= 0 && (tb > gbest || (tb == gbest && ti < gidx))) { gbest = tb; gidx = ti; }
      }
    }
    perm[k] = gidx;
    used[gidx] = 1;
    last = gidx;
  }
  return 0;
}

int oracle_order_maxmin(int64_t n, const double* xy, int64_t* perm) {
  return oracle_order_maxmin_prefix(n, xy, n, perm);
}

// Morton ordering (Sec. V-A and Fig. 1, the Z-order alternative to random ordering):
// a 16-bit cell index per coordinate over the bounding box,
// q = min(65535, floor((v - lo)/(hi - lo) * 65536)), q = 0 if hi == lo; the Z-order key
// takes bit b of x to position 2b and bit b of y to position 2b+1; sort by (key, index).
int oracle_order_morton(int64_t n, const double* xy, int64_t* perm) {
  if (n <= 0) return 0;
  double lo[2] = {xy[0], xy[1]}, hi[2] = {xy[0], xy[1]};
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 2; ++a) {
      lo[a] = std::min(lo[a], xy[2 * i + a]);
      hi[a] = std::max(hi[a], xy[2 * i + a]);
    }
  std::vector<uint64_t> key(n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t q[2];
    for (int a = 0; a < 2; ++a) {
      if (!(hi[a] > lo[a])) { q[a] = 0; continue; }
      const double f = std::floor((xy[2 * i + a] - lo[a]) / (hi[a] - lo[a]) * 65536.0);
      q[a] = f < 0.0 ? 0 : (f > 65535.0 ? 65535 : (uint64_t)f);
    }
    uint64_t k = 0;
    for (int bit = 15; bit >= 0; --bit) k = (k << 2) | (((q[1] >> bit) & 1) << 1) | ((q[0] >> bit) & 1);
    key[i] = (k << 32) | (uint64_t)i;  // n < 2^32 here
  }
  std::sort(key.begin(), key.end());
  for (int64_t i = 0; i < n; ++i) perm[i] = (int64_t)(key[i] & 0xFFFFFFFFULL);
  return 0;
}

// Brute-force conditioning sets for the listed ordered rows (Algorithm 1, lines
// on the nearest-neighbour loop).  xy is ordered; out is nrows x m, -1 padded.
int oracle_knn_rows(int64_t n, const double* xy, int32_t m, const int64_t* rows, int64_t nrows,
                    int32_t* out) {
  if (m < 1) return 1;
  for (int64_t r = 0; r < nrows; ++r) if (rows[r] < 0 || rows[r] >= n) return 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nrows; ++r) knn_row(xy, rows[r], m, out + (size_t)r * m);
  return 0;
}

// Unit vectors of n (longitude, latitude) points in degrees (n x 3 out).
void oracle_sphere_xyz(int64_t n, const double* lonlat, double* xyz) {
  for (int64_t i = 0; i < n; ++i) unit_vector(lonlat + 2 * i, xyz + 3 * i);
}

// Great-circle distances between n pairs of (longitude, latitude) points in degrees.
void oracle_gcd(int64_t n, const double* a, const double* b, double radius, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = gcd(a + 2 * i, b + 2 * i, radius);
}

// Brute-force conditioning sets on the sphere for the listed ordered rows; xyz is the
// ordered unit vectors (n x 3).
int oracle_knn_rows_sphere(int64_t n, const double* xyz, int32_t m, const int64_t* rows, int64_t nrows,
                           int32_t* out) {
  if (m < 1) return 1;
  for (int64_t r = 0; r < nrows; ++r) if (rows[r] < 0 || rows[r] >= n) return 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nrows; ++r) knn_row_sphere(xyz, rows[r], m, out + (size_t)r * m);
  return 0;
}

// Vecchia terms for the listed ordered rows, given their conditioning sets
// (nbr: nrows x m, -1 padded, as produced by oracle_knn_rows).
// out: nrows x (want_grad ? 4 : 1): (l_i[, dl_i/dsigma2, dl_i/dbeta, dl_i/dtau2]).
// mu_s (optional): nrows x 2 conditional means and variances.
// bad_row (optional): first failing row index on a non-PD block.
int oracle_vecchia_rows(int64_t n, const double* xy, const double* y, int32_t m, const double* theta,
                        const int64_t* rows, int64_t nrows, const int32_t* nbr, int want_grad,
                        double* out, double* mu_s, int64_t* bad_row, int family, int metric, double radius) {
  (void)n;
  const int w = want_grad ? 4 : 1;
  int64_t first_bad = -1;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t r = 0; r < nrows; ++r) {
    const int32_t* J = nbr + (size_t)r * m;
    int mi = 0;
    while (mi < m && J[mi] >= 0) ++mi;
    double g[3];
    double mu = 0.0, s = 0.0;
    const int rc = location_term(xy, y, rows[r], J, mi, theta, family, metric, radius, out + (size_t)r * w,
                                 want_grad ? g : nullptr, &mu, &s);
    if (rc) {
#pragma omp critical
      { if (first_bad < 0 || rows[r] < first_bad) first_bad = rows[r]; }
      continue;
    }
    if (want_grad) for (int t = 0; t < 3; ++t) out[(size_t)r * w + 1 + t] = g[t];
    if (mu_s) { mu_s[2 * r] = mu; mu_s[2 * r + 1] = s; }
  }
  if (bad_row) *bad_row = first_bad;
  return first_bad >= 0 ? 2 : 0;
}

// Prediction (kriging) at new locations from the m nearest OBSERVED locations (any of
// them; ties by observed index): the conditional mean and variance of y at the new
// point given y_J, by the same formulas as a Vecchia term (Sec. V-B) with y_new
// unknown.  Metric 1: points are (longitude, latitude) in degrees, neighbours ranked
// by the squared chord of unit vectors, covariance from great-circle distances.
// Outputs: mean, var (n_new each), nbr (n_new x m observed indices).
int oracle_predict(int64_t n_obs, const double* xy_obs, const double* y_obs, int64_t n_new, const double* xy_new,
                   int32_t m, const double* theta, int family, int metric, double radius, double* mean,
                   double* var, int32_t* nbr) {
  if (m < 1 || m > n_obs) return 1;
  std::vector<double> xyz_obs;
  if (metric == 1) {
    xyz_obs.resize(3 * (size_t)n_obs);
    for (int64_t j = 0; j < n_obs; ++j) unit_vector(xy_obs + 2 * j, xyz_obs.data() + 3 * j);
  }
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < n_new; ++k) {
    // m nearest observed points, lexicographic (key, index), brute force
    std::vector<double> bd(m);
    std::vector<int64_t> bj(m);
    double q3[3];
    if (metric == 1) unit_vector(xy_new + 2 * k, q3);
    int cnt = 0;
    for (int64_t j = 0; j < n_obs; ++j) {
      const double d = metric == 1 ? chord2(q3, xyz_obs.data() + 3 * j) : dist2(xy_new + 2 * k, xy_obs + 2 * j);
      if (cnt == m) {
        if (!(d < bd[m - 1])) continue;
        --cnt;
      }
      int p = cnt;
      while (p > 0 && (d < bd[p - 1])) { bd[p] = bd[p - 1]; bj[p] = bj[p - 1]; --p; }
      bd[p] = d; bj[p] = j; ++cnt;
    }
    // mu = Sigma_kJ Sigma_JJ^-1 y_J and s = Sigma_kk - Sigma_kJ Sigma_JJ^-1 Sigma_Jk on a
    // local array (the m neighbours, then the new point); s may be 0 (interpolation).
    const double sigma2 = theta[0], beta = theta[1], nu = theta[2], tau2 = theta[3];
    std::vector<double> lxy(2 * (size_t)(m + 1)), SJ((size_t)m * m), LJ((size_t)m * m), v(m), w(m);
    for (int p = 0; p < m; ++p) {
      lxy[2 * p] = xy_obs[2 * bj[p]];
      lxy[2 * p + 1] = xy_obs[2 * bj[p] + 1];
      nbr[(size_t)k * m + p] = (int32_t)bj[p];
    }
    lxy[2 * m] = xy_new[2 * k];
    lxy[2 * m + 1] = xy_new[2 * k + 1];
    for (int p = 0; p < m; ++p) {
      for (int q = 0; q < m; ++q)
        SJ[(size_t)p * m + q] = p == q ? sigma2 + tau2 : cov(family, point_dist(lxy.data(), p, q, metric, radius),
                                                              sigma2, beta, nu);
      v[p] = cov(family, point_dist(lxy.data(), p, m, metric, radius), sigma2, beta, nu);
    }
    if (!cholesky(m, SJ.data(), LJ.data())) {
#pragma omp atomic write
      bad = 1;
      mean[k] = var[k] = std::numeric_limits<double>::quiet_NaN();
      continue;
    }
    chol_solve(m, LJ.data(), v.data(), w.data());
    double mu = 0.0, vw = 0.0;
    for (int p = 0; p < m; ++p) { mu += w[p] * y_obs[bj[p]]; vw += w[p] * v[p]; }
    mean[k] = mu;
    var[k] = sigma2 + tau2 - vw;
  }
  return bad ? 2 : 0;
}

// Neumaier-compensated sum of `cols` interleaved columns, in row order.
void oracle_sum_columns(int64_t nrows, int32_t cols, const double* v, double* out) {
  for (int c = 0; c < cols; ++c) {
    Neumaier acc;
    for (int64_t r = 0; r < nrows; ++r) acc.add(v[(size_t)r * cols + c]);
    out[c] = acc.value();
  }
}

// Eq. (1): exact log-likelihood with zero mean, Sigma_pq = C(||s_p - s_q||) +
// tau2 delta_pq; O(n^3) with the oracle's own Cholesky.  grad (optional):
// d l / d(sigma2, beta, tau2) by -1/2 tr(Sigma^{-1} Sigma_p) + 1/2 a^T Sigma_p a.
int oracle_loglik_exact(int64_t n, const double* xy, const double* y, const double* theta,
                        double* out, double* grad, int family, int metric, double radius) {
  const double sigma2 = theta[0], beta = theta[1], nu = theta[2], tau2 = theta[3];
  const int k = (int)n;
  std::vector<double> S((size_t)k * k), L((size_t)k * k), a(k);
  for (int p = 0; p < k; ++p)
    for (int q = 0; q < k; ++q) {
      const double d = p == q ? 0.0 : point_dist(xy, p, q, metric, radius);
      S[(size_t)p * k + q] = p == q ? sigma2 + tau2 : cov(family, d, sigma2, beta, nu);
    }
  if (!cholesky(k, S.data(), L.data())) return 2;
  chol_solve(k, L.data(), y, a.data());
  double logdet = 0.0, quad = 0.0;
  for (int p = 0; p < k; ++p) { logdet += 2.0 * std::log(L[(size_t)p * k + p]); quad += y[p] * a[p]; }
  *out = -0.5 * (double)n * kLog2Pi - 0.5 * logdet - 0.5 * quad;
  if (!grad) return 0;
  std::vector<double> Si((size_t)k * k);
  chol_inverse(k, L.data(), Si.data());
  for (int t = 0; t < 3; ++t) {
    double tr = 0.0, qd = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q) {
        double Sp;
        if (t == 0) Sp = (S[(size_t)p * k + q] - (p == q ? tau2 : 0.0)) / sigma2;
        else if (t == 1) {
          Sp = p == q ? 0.0 : cov_dbeta(family, point_dist(xy, p, q, metric, radius), sigma2, beta, nu);
        } else Sp = p == q ? 1.0 : 0.0;
        tr += Si[(size_t)q * k + p] * Sp;
        qd += a[p] * Sp * a[q];
      }
    grad[t] = -0.5 * tr + 0.5 * qd;
  }
  return 0;
}

// One block's Gaussian log-density log N(y; 0, S) (k x k, row-major), used by
// the identity-padding invariance check.
int oracle_block_logdensity(int32_t k, const double* S, const double* y, double* out) {
  std::vector<double> L((size_t)k * k), a(k);
  if (!cholesky(k, S, L.data())) return 2;
  chol_solve(k, L.data(), y, a.data());
  double logdet = 0.0, quad = 0.0;
  for (int p = 0; p < k; ++p) { logdet += 2.0 * std::log(L[(size_t)p * k + p]); quad += y[p] * a[p]; }
  *out = -0.5 * k * kLog2Pi - 0.5 * logdet - 0.5 * quad;
  return 0;
}

}  // extern "C"

/*
 * vecchia.h — C ABI of the GB300-native Vecchia log-likelihood library (libvecchia.so).
 *
 * The library evaluates the Vecchia approximation of the zero-mean Gaussian-process
 * log-likelihood of arXiv 2403.07412 (Sec. V-B, Algorithm 1) with the Matérn
 * covariance of Eq. (2) plus a nugget:
 *
 *   l(theta) = sum_i log N(y_i | mu_i, s_i),
 *   mu_i = Sigma_iJ Sigma_JJ^{-1} y_J,  s_i = Sigma_ii - Sigma_iJ Sigma_JJ^{-1} Sigma_Ji,
 *   Sigma_pq = C(||s_p - s_q||) + tau2 [p == q],
 *   C(d) = sigma2 2^{1-nu}/Gamma(nu) (d/beta)^nu K_nu(d/beta),  C(0) = sigma2,
 *
 * where J = J_i holds the m_i = min(i, m) nearest previously ordered locations of the
 * i-th ordered location (0-based i).  theta is passed as double[4] =
 * {sigma2, beta, nu, tau2}.
 *
 * Conventions for every entry point:
 *   - Return value: a VECCHIA_* status code; nothing aborts or prints.
 *   - "_dev" pointers are CUDA device pointers on the current device; "_host" and
 *     unsuffixed array pointers are host memory.  The caller owns every buffer it
 *     passes; the library never keeps a caller pointer after a call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream only enqueue work on it and return before the GPU
 *     finishes; results are valid once that stream has been synchronised.
 *   - A plan may be used by one stream at a time: calls that share a plan must be
 *     ordered on the same stream (or externally synchronised).
 *   - Failures found on the GPU (a conditional block that is not positive
 *     definite, a non-finite value in y) cannot be returned by the asynchronous call
 *     itself: the affected outputs become NaN and vecchia_last_error_location()
 *     reports the first failing ordered location and the kind of failure.
 */
#ifndef VECCHIA_H
#define VECCHIA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vecchia_plan* vecchia_plan_t; /* opaque; immutable after create */

enum {
  VECCHIA_OK = 0,
  VECCHIA_EINVAL = 1,   /* an argument is out of range or not finite            */
  VECCHIA_ENOTPD = 2,   /* a conditional block was not positive definite        */
  VECCHIA_ECUDA = 3,    /* a CUDA runtime call failed                           */
  VECCHIA_ETIMEOUT = 4, /* reserved: no kernel of this library waits on another */
  VECCHIA_ENOMEM = 5    /* device or host allocation failed                     */
};

enum {
  VECCHIA_ORDER_GIVEN = 0,  /* use perm_in                                          */
  VECCHIA_ORDER_RANDOM = 1, /* Sec. V-A random ordering (splitmix64 Fisher–Yates)   */
  VECCHIA_ORDER_MAXMIN = 2, /* Sec. V-A maxmin ordering (exact greedy farthest point) */
  VECCHIA_ORDER_MORTON = 3  /* Sec. V-A Morton (Z-order) ordering                     */
};

enum {
  VECCHIA_KERNEL_MATERN = 0, /* Eq. (2): sigma2 2^{1-nu}/Gamma(nu) (d/beta)^nu K_nu(d/beta)       */
  VECCHIA_KERNEL_POWEXP = 1  /* Eq. (3): sigma2 exp(-d^nu / beta), 0 < nu <= 2 (nu = the exponent) */
};

/* Largest conditioning-set size m accepted by plans and the single-field likelihood
 * calls; up to VECCHIA_MAX_M_WARP a warp (or part of one) owns a location, beyond it a
 * CTA does.  The batched and allocation-free calls accept m <= VECCHIA_MAX_M_WARP. */
#define VECCHIA_MAX_M 150
#define VECCHIA_MAX_M_WARP 63

/*
 * vecchia_plan_create — ordering and conditioning sets (Algorithm 1, permutation and
 * nearest-neighbour loop; Sec. V-A for the orderings).
 *   xy_host : n x 2 doubles, row-major (x_k, y_k) in the caller's ORIGINAL order.
 *   n       : number of locations, 1 <= n <= 2^31 - 1.
 *   m       : conditioning-set size, 1 <= m <= VECCHIA_MAX_M; location i (0-based,
 *             ordered) conditions on m_i = min(i, m) points.
 *   order   : VECCHIA_ORDER_*.  RANDOM: Fisher–Yates (i from n-1 down to 1, swap with
 *             j = splitmix64() mod (i+1)), splitmix64 state initialised to `seed`.
 *             MAXMIN: first the point nearest the centroid, then repeatedly the point
 *             whose minimum squared distance to those chosen is largest; ties to the
 *             lowest original index.  MORTON: each coordinate mapped to a 16-bit cell
 *             q = min(65535, floor((v - lo)/(hi - lo) * 65536)) over the bounding box,
 *             bits interleaved (x in the even bits), sorted by (code, original index).
 *             GIVEN: perm_in.
 *   perm_in : n int64 (host), a permutation of 0..n-1, perm_in[k] = original index of
 *             the k-th ordered location; only read for ORDER_GIVEN (else may be NULL).
 *   stream  : stream for the GPU neighbour search and uploads.
 *   out     : receives the plan handle.
 * Conditioning sets: J_i = the m_i previously ordered points with the smallest
 * (d^2, ordered index), d^2 = round(round(dx*dx) + round(dy*dy)), computed on the GPU.
 * Synchronous: returns after the plan is complete.  Errors: EINVAL (n, m, order,
 * non-finite xy, perm_in not a permutation), ENOMEM, ECUDA.
 */
int vecchia_plan_create(const double* xy_host, int64_t n, int32_t m, int order, uint64_t seed,
                        const int64_t* perm_in, void* stream, vecchia_plan_t* out);

/* Frees every device and host resource of the plan (NULL is ignored). */
void vecchia_plan_destroy(vecchia_plan_t plan);

/*
 * vecchia_plan_create_sphere — a plan for (longitude, latitude) data with great-circle
 * distances (Sec. VI-C, the haversine distance of the paper's real-data study) on a
 * sphere of radius `radius` (the unit of distance, hence of beta: e.g. 6371 for km).
 *   lonlat_host : n x 2 doubles (longitude, latitude) in degrees, host memory, copied;
 *                 |latitude| <= 90.
 *   order       : VECCHIA_ORDER_GIVEN (perm_in) or VECCHIA_ORDER_RANDOM (seed); the
 *                 planar orderings (maxmin, Morton) return VECCHIA_EINVAL.
 *   Conditioning sets: the m_i nearest previously ordered points by great-circle
 *   distance, found as the smallest (squared chord of the unit vectors, index), the
 *   squared chord evaluated as ((dx*dx + dy*dy) + dz*dz) in FP64 without fused
 *   multiply-adds on unit vectors (cos(lat) cos(lon), cos(lat) sin(lon), sin(lat))
 *   computed on the host from lat, lon times (3.14159265358979323846 / 180).
 *   The search is a brute-force GPU scan (O(n^2 / 2) candidate checks).
 * The likelihood calls (vecchia_loglik, _grad, _terms, _autotune) accept the plan;
 * the batched and allocation-free calls return VECCHIA_EINVAL for it.  Matérn with
 * great-circle distance is positive definite on the whole sphere only for nu <= 1/2
 * (and the power exponential for exponent <= 1); larger values may meet
 * VECCHIA_ENOTPD on global data.  Errors as vecchia_plan_create, plus EINVAL for a
 * latitude outside [-90, 90] or a radius that is not positive and finite.
 */
int vecchia_plan_create_sphere(const double* lonlat_host, int64_t n, int32_t m, int order, uint64_t seed,
                               const int64_t* perm_in, double radius, void* stream, vecchia_plan_t* out);

/*
 * vecchia_plan_set_kernel — the covariance family used by this plan's likelihood calls:
 * VECCHIA_KERNEL_MATERN (default, Eq. (2)) or VECCHIA_KERNEL_POWEXP (the power
 * exponential of Eq. (3), used by the paper for its real data, Sec. VI-C).  With the
 * power exponential, theta = {sigma2, beta, nu, tau2} means C(d) = sigma2 exp(-d^nu/beta)
 * + tau2 [d = 0 on the diagonal] and requires 0 < nu <= 2 (EINVAL otherwise); the
 * gradient is still d/d(sigma2, beta, tau2).  Not for plans in use on a stream.  The
 * batched call accepts Matérn plans only.  Errors: EINVAL.
 */
int vecchia_plan_set_kernel(vecchia_plan_t plan, int kernel);

/* n and m of the plan. */
int vecchia_plan_size(vecchia_plan_t plan, int64_t* n, int32_t* m);

/* perm_out (host, n int64): perm_out[k] = original index of the k-th ordered location. */
int vecchia_plan_perm(vecchia_plan_t plan, int64_t* perm_out);

/*
 * nbr_out (host, n x m int32, row-major by ordered location): the conditioning set J_i
 * as ORDERED indices, ascending in (d^2, index), padded with -1 after m_i entries.
 * Synchronous (device-to-host copy).
 */
int vecchia_plan_neighbors(vecchia_plan_t plan, int32_t* nbr_out);

/*
 * vecchia_loglik — the Vecchia log-likelihood (Algorithm 1 output l).
 *   y_dev   : n doubles on the device, in the ORIGINAL location order.
 *   theta   : host double[4] {sigma2 > 0, beta > 0, nu > 0, tau2 >= 0}, all finite.
 *   out_dev : 1 double on the device: l.
 * Asynchronous on `stream`.  Errors returned: EINVAL (bad theta, NULL pointers),
 * ECUDA.  A non-positive-definite block makes out_dev NaN (see
 * vecchia_last_error_location); a block counts as such when a pivot of its elimination
 * falls outside [2^-1022, 2^1022) (see vecchia_pivot_reciprocal) or its conditional
 * variance is not positive and finite.
 */
int vecchia_loglik(vecchia_plan_t plan, const double* y_dev, const double theta[4], double* out_dev,
                   void* stream);

/*
 * vecchia_loglik_grad — l and its gradient (not in the paper: the adjoint of Algorithm 1
 * with respect to sigma2, beta and tau2, recomputing each block's factor).  l is computed
 * exactly as by vecchia_loglik (FP64 elimination); the adjoint's two backward solves and
 * its beta pair sums run in double-float arithmetic (about 2^-46 relative per operation).
 *   out_dev : 4 doubles on the device: {l, dl/dsigma2, dl/dbeta, dl/dtau2}.
 * Same arguments, asynchrony and errors as vecchia_loglik.
 */
int vecchia_loglik_grad(vecchia_plan_t plan, const double* y_dev, const double theta[4],
                        double* out_dev, void* stream);

/*
 * vecchia_loglik_terms — the per-location terms l_i (Algorithm 1, univariate Gaussian
 * terms) and, if want_grad, their gradients, indexed by ORDERED location.
 *   terms_dev : n x (want_grad ? 4 : 1) doubles on the device, row-major:
 *               {l_i[, dl_i/dsigma2, dl_i/dbeta, dl_i/dtau2]}.
 * Same arguments, asynchrony and errors as vecchia_loglik.
 */
int vecchia_loglik_terms(vecchia_plan_t plan, const double* y_dev, const double theta[4],
                         int want_grad, double* terms_dev, void* stream);

/*
 * vecchia_loglik_range — the part of l (and, if want_grad, of its gradient) contributed by
 * the ordered locations i0 <= i < i1: Algorithm 1's sum restricted to a contiguous range
 * of its n independent terms (Sec. V-B), the unit by which the likelihood is split
 * across GPUs.  For disjoint ranges covering [0, n) the outputs add up to those of
 * vecchia_loglik / vecchia_loglik_grad (every output is linear in the per-location sums).
 *   i0, i1  : 0 <= i0 <= i1 <= n; i0 == i1 writes zeros.
 *   out_dev : 1 (want_grad == 0) or 4 doubles on the device: the range's {l[, dl/dsigma2,
 *             dl/dbeta, dl/dtau2]}.
 * Same asynchrony and errors as vecchia_loglik, plus EINVAL for a range outside [0, n];
 * vecchia_last_error_location reports the first failing location within the range.
 */
int vecchia_loglik_range(vecchia_plan_t plan, const double* y_dev, const double theta[4], int64_t i0, int64_t i1,
                         int want_grad, double* out_dev, void* stream);

/*
 * vecchia_matern — the covariance of Eq. (2) and its beta-derivative, evaluated by the
 * same device code the likelihood kernels use.
 *   d_dev        : count distances (>= 0) on the device.
 *   c_dev        : count doubles on the device: C(d) (sigma2 at d = 0, without nugget).
 *   dcdbeta_dev  : count doubles on the device (may be NULL): dC/dbeta(d).
 * Asynchronous on `stream`.  Errors: EINVAL, ECUDA.
 */
int vecchia_matern(const double* d_dev, int64_t count, const double theta[4], double* c_dev,
                   double* dcdbeta_dev, void* stream);

/*
 * vecchia_covariance — vecchia_matern for either covariance family (VECCHIA_KERNEL_*):
 * C(d) of Eq. (2) or Eq. (3) and dC/dbeta, through the kernels' device code.  Same
 * arguments and errors as vecchia_matern, plus EINVAL for an unknown kernel or, for the
 * power exponential, an exponent outside (0, 2].
 */
int vecchia_covariance(int kernel, const double* d_dev, int64_t count, const double theta[4], double* c_dev,
                       double* dcdbeta_dev, void* stream);

/*
 * vecchia_pivot_reciprocal — the reciprocal the likelihood kernels take of each LDL^T pivot
 * (the 1/d_j that scales column j), exposed so its accuracy can be checked.  It uses no
 * FP64 instruction: an FP32 seed, an exact 32-bit integer residual and a second-order
 * correction in 64-bit fixed point; the result is within about half an ulp of 1/d.
 *   d_dev   : count doubles on the device.
 *   out_dev : count doubles on the device: 1/d for d in [2^-1022, 2^1022), NaN otherwise
 *             (the likelihood kernels report a pivot outside that range as a block that
 *             is not positive definite).
 * Asynchronous on `stream`.  Errors: EINVAL (count < 0, or NULL buffers), ECUDA.
 */
int vecchia_pivot_reciprocal(const double* d_dev, int64_t count, double* out_dev, void* stream);

/*
 * vecchia_mul_by_positive — the product the full-warp likelihood kernels use to scale an
 * elimination column by its pivot reciprocal (Algorithm 1's factorisation step, written
 * as L D L^T), exposed so its exactness can be checked.  It uses no FP64 instruction:
 * the 106-bit mantissa product is formed from 32-bit integer limbs and rounded to
 * nearest, ties to even.
 *   a_dev, b_dev : count doubles each on the device; b must be a positive normal double
 *                  (a pivot reciprocal), a any finite double.
 *   out_dev      : count doubles on the device: a * b, bit-identical to the FP64 product
 *                  whenever the exact product is finite with magnitude at least 2^-1022;
 *                  an exact product below 2^-1022 in magnitude (or a zero or subnormal a)
 *                  gives a zero of a's sign, one that rounds beyond the largest double an
 *                  infinity.
 * Asynchronous on `stream`.  Errors: EINVAL (count < 0, or NULL buffers), ECUDA.
 */
int vecchia_mul_by_positive(const double* a_dev, const double* b_dev, int64_t count, double* out_dev, void* stream);

/*
 * vecchia_batched_prepare — builds the covariance tables the batched call may use, one per
 * smoothness value nus[0..nnu-1] (each > 0 and finite, 1 <= nnu <= 8), on the current
 * device, replacing the previously prepared set.  Synchronises `stream` before and after
 * (tables in use by earlier batched launches on that stream are not overwritten early).
 * Must precede vecchia_loglik_batched and any graph capture of it.  Errors: EINVAL,
 * ENOMEM, ECUDA.
 */
int vecchia_batched_prepare(const double* nus, int32_t nnu, void* stream);

/*
 * vecchia_loglik_batched — many (field, theta) evaluations in one persistent launch (not
 * in the paper, which batches only over the locations of one field).
 *   plans      : nfields plan handles (host array); fields may differ in n and m (at most
 *                four distinct m per call, each m <= VECCHIA_MAX_M_WARP).
 *   y_devs     : nfields device pointers (host array), field f's n values in the ORIGINAL
 *                order of plans[f].
 *   thetas_dev : nfields x ntheta x 4 doubles on the DEVICE, row-major; each theta's nu
 *                must be one of the values given to vecchia_batched_prepare (compared bit
 *                for bit).
 *   want_grad  : 0 -> out_dev has 1 double per (field, theta): l; else 4:
 *                {l, dl/dsigma2, dl/dbeta, dl/dtau2}.
 *   out_dev    : nfields x ntheta x (1|4) doubles on the device.
 * Asynchronous on `stream`.  The first call for a given (plans, y_devs, ntheta, want_grad)
 * lays out the work and allocates for it (it must not be made during stream capture:
 * EINVAL); later calls with the same arguments reuse that layout, allocate nothing and
 * may be captured in a CUDA graph and replayed with new values in thetas_dev.  A theta
 * whose nu was not prepared, an invalid theta or a block that is not positive definite
 * makes that (field, theta)'s outputs NaN.  Destroying a plan drops the layouts that use
 * it.  Errors: EINVAL (arguments, nothing prepared, more than four distinct m), ENOMEM,
 * ECUDA.
 */
int vecchia_loglik_batched(const vecchia_plan_t* plans, const double* const* y_devs, int32_t nfields,
                           const double* thetas_dev, int32_t ntheta, int want_grad, double* out_dev,
                           void* stream);

/*
 * vecchia_loglik_noalloc — the same log-likelihood as vecchia_loglik for callers that
 * cannot allocate device memory: code running where cudaMalloc is unavailable or
 * forbidden (for example inside a host allocator's callback, a memory-capped arena
 * that owns every device byte, or a runtime that must never trigger an allocation
 * while serving).  It has no counterpart in the paper.  It calls no cudaMalloc,
 * cudaFree or other allocating routine; its scratch (partial sums for launches of at
 * most 4096 warps, an error slot and one covariance table, about 190 KB) is a
 * file-scope __device__ array that every GPU loading the library keeps until the
 * process exits.  The launch is capped at 4096 warps; the kernel strides over the
 * locations, so no n is too large for the scratch.
 *   xy_dev   : n x 2 doubles, ORIGINAL order (as passed to vecchia_plan_create).
 *   y_dev    : n doubles, ORIGINAL order.
 *   nbr_dev  : n x m int32, row i = the conditioning set of the i-th ORDERED location as
 *              ORIGINAL indices, -1 padded after m_i = min(i, m) entries; from a plan:
 *              perm[vecchia_plan_neighbors()] for entries >= 0.
 *   self_dev : n int32, ORIGINAL index of the i-th ordered location (= perm[i]).
 *   n, m     : 1 <= n <= 2^31 - 1, 1 <= m <= VECCHIA_MAX_M_WARP; otherwise EINVAL.
 *   theta    : host double[4] as for vecchia_loglik; out_dev: 1 double on the device.
 * The kernel checks every entry of self_dev and the first m_i entries of each nbr_dev
 * row against [0, n) before reading through it: an entry outside that range makes
 * out_dev NaN (it is never used as an address).
 * Asynchronous on `stream`.  The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress); with lazy module loading (the CUDA default)
 * that first call, or the first launch of this library's kernels on the device, is
 * also when the driver loads the module and its __device__ arrays, which can allocate
 * device memory.  So make the first call on each device outside any context that must
 * not allocate, and before any stream capture.  The looked-up address is kept for the
 * life of the process: a device reset (cudaDeviceReset) or a new primary context on the
 * device invalidates it, and the library must not be called on that device afterwards.
 * Every call reuses the same scratch and rebuilds the covariance table in
 * it, so calls that overlap on the GPU (different streams, or different host threads,
 * on one device) race and must be serialised by the caller.  A block that is not
 * positive definite makes out_dev NaN.  Errors: EINVAL, ECUDA.
 */
int vecchia_loglik_noalloc(const double* xy_dev, const double* y_dev, const int32_t* nbr_dev,
                           const int32_t* self_dev, int64_t n, int32_t m, const double theta[4],
                           double* out_dev, void* stream);

/*
 * vecchia_autotune — picks the launch shape of the likelihood kernels for this plan's
 * block size (m + 1) by timing: lanes per location (4, 8, 16 or 32; 32/lanes locations
 * share a warp; 4 lanes take blocks of up to 16 rows, 8 lanes up to 32) and warps per CTA.
 * Each candidate is timed on the caller's own problem (two
 * timed launches after one warm-up; the fastest wins) and recorded, process-wide, for
 * every later call with the same block size and kind (want_grad) on this device,
 * including the batched call's layouts created afterwards.  Without tuning, blocks of
 * up to 16 rows use 4 lanes, up to 32 rows 8, up to 48 rows 16 (forward) or 32
 * (gradient), larger ones a full warp; a call over fewer locations than would give
 * one group of them per SM sub-partition widens those defaults (up to 16 lanes), and
 * a call with fewer groups than the shape's resident warps spreads them over every SM
 * with fewer warps per CTA.  Results are deterministic for a given plan, range and
 * shape; a different shape changes only the order of the final additions.
 * Not in the paper (its batched kernels are library routines).
 *   y_dev, theta : as for vecchia_loglik (theta on the host).
 *   lanes_out, warps_out : host int32 (may be NULL): the chosen shape.  For m >
 *                          VECCHIA_MAX_M_WARP (one CTA per location, sized by
 *                          occupancy) nothing is timed: lanes_out = the CTA's threads,
 *                          warps_out = its warps.
 * Synchronous (waits on `stream`); must not be called during stream capture.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
int vecchia_autotune(vecchia_plan_t plan, const double* y_dev, const double theta[4], int want_grad,
                     int32_t* lanes_out, int32_t* warps_out, void* stream);

/*
 * vecchia_predict — kriging at new locations (the prediction step of the paper's
 * real-data study, Sec. VI-C / Table III) from the plan's observed data: for each new
 * point, its m nearest OBSERVED points (any of the plan's n points; ties to the lower
 * original index; Euclidean or great-circle as the plan) condition it, and
 *   mean = Sigma_kJ Sigma_JJ^{-1} y_J,   var = sigma2 + tau2 - Sigma_kJ Sigma_JJ^{-1} Sigma_Jk,
 * the Vecchia conditional of Sec. V-B with y at the new point unknown (var includes the
 * nugget: it is the predictive variance of an observation there).
 *   xy_new_host : n_new x 2 doubles, host (the plan's coordinate kind), copied.
 *   y_dev       : n doubles, device, ORIGINAL order (as for vecchia_loglik).
 *   theta       : (sigma2, beta, nu, tau2), host; the plan's covariance family.
 *   mean_dev    : n_new doubles, device, written.  var_dev: n_new doubles or NULL.
 *   nbr_host    : optional n_new x m int32, host: the conditioning sets (original
 *                 indices, nearest first).
 * Synchronises `stream` before returning (temporary buffers are freed).  m must be at
 * most VECCHIA_MAX_M_WARP and at most n.  A location whose neighbour block is not
 * positive definite gets NaN and is reported through vecchia_last_error_location, with
 * status VECCHIA_OK (the other predictions stand).  EINVAL: non-finite or (sphere)
 * out-of-range coordinates, bad theta, m > VECCHIA_MAX_M_WARP or m > n, n_new < 1.
 */
int vecchia_predict(vecchia_plan_t plan, const double* xy_new_host, int64_t n_new, const double* y_dev,
                    const double theta[4], double* mean_dev, double* var_dev, int32_t* nbr_host, void* stream);

/*
 * vecchia_last_error_location — synchronises the stream of the plan's last call and
 * reports the first ordered location whose term failed in that call (*loc = -1 if
 * none).  Returns VECCHIA_ENOTPD if that location's block was not positive definite,
 * VECCHIA_EINVAL if the block held a non-finite data value (y at the location or at one
 * of its conditioning points: y_dev is not scanned up front, since the calls are
 * asynchronous), else VECCHIA_OK.
 */
int vecchia_last_error_location(vecchia_plan_t plan, int64_t* loc);

/* Static, NUL-terminated description of a status code. */
const char* vecchia_strerror(int code);

/*
 * vecchia_fp64_peak — measures this GPU's sustained FP64 fused-multiply-add rate with a
 * register-resident DFMA chain kernel (the denominator of the library's fraction-of-
 * peak figures).  *gflops_out receives GFLOP/s (2 flops per DFMA).  Synchronous.
 */
int vecchia_fp64_peak(double* gflops_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* VECCHIA_H */

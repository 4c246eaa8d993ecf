"""Benchmark: Vecchia log-likelihood + gradient throughput on the GPU.

Workload (default): n = 1,000,000 locations from a 20-component Gaussian mixture in the
unit square, random-Fourier-feature Matérn field with nu = 1.0 (general Bessel K),
sigma2 = 1, beta = 0.02, tau2 = 0.01, maxmin ordering, m = 60.  One step = one call of
vecchia_loglik_grad over all n locations (log-likelihood and d/d(sigma2, beta, tau2)).

Prints one JSON line.  ``value`` = locations per second over the whole job, timed with
CUDA events on the launching stream with the inputs resident in HBM; ``e2e`` repeats the
measurement through the same C-ABI call with the field copied from pinned host memory
and the result copied back every step.  ``roofline`` rates the dominant kernel
(vecchia_lik_kernel, fwd+adjoint) against the FP64 FMA peak measured in the same run.
``cpu_baseline`` times the CPU oracle on a bounded sample of the same workload.

``roofline.achieved`` counts the algorithmic linear-algebra flops of the likelihood,
F(k) = k^3/3 + k^2/2 + k/6 + k^2 per location (k = m_i + 1), for the forward and the
forward + gradient step alike; ``roofline.frac_with_adjoint_solves`` adds the adjoint's
two unit triangular solves (2 m_i^2 per location).  ``configs`` times the other
workloads (2k / 100k forward, 250k forward + gradient) as lines of their own.

Multi-GPU (torchrun, N > 1), ``--shard locations`` (default): one field of n locations,
its ordered locations split into N contiguous ranges (shard.location_ranges); every rank
holds the same plan, evaluates its range with vecchia_loglik_range and the ranks sum the
four result doubles with one NCCL all-reduce per step; value = n / max step time (strong
scaling: the job's work is fixed).  ``--shard fields``: every rank evaluates its own
independent field of n locations (weak scaling; no collective on the data path); value =
N * n / max step time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "vecchia-matern-gmm1M-maxmin-m60-nu1.0-fwd+grad"
METRIC = "Vecchia loglik+grad locations/sec (n=1M, m=60) and fraction of FP64 peak"


def la_flops(n: int, m: int, grad: bool) -> float:
    """Algorithmic FP64 flops of one evaluation: per location k = m_i + 1,
    k^3/3 + k^2/2 + k/6 (Cholesky) + k^2 (two triangular solves); the adjoint adds
    two unit triangular solves of size m_i (2 m_i^2)."""
    return la_flops_range(0, n, m, grad)


def la_flops_range(i0: int, i1: int, m: int, grad: bool) -> float:
    """la_flops over the ordered locations [i0, i1)."""
    i = np.arange(i0, i1, dtype=np.float64)
    mi = np.minimum(i, m)
    k = mi + 1
    f = k ** 3 / 3 + k ** 2 / 2 + k / 6 + k ** 2
    if grad:
        f = f + 2 * mi ** 2
    return float(f.sum())


def workload_label(n: int, m: int, order: str, fwd: bool) -> str:
    """The config's workload name; the default arguments give WORKLOAD."""
    n_label = "1M" if n == 1_000_000 else str(n)
    return f"vecchia-matern-gmm{n_label}-{order}-m{m}-nu1.0-{'fwd' if fwd else 'fwd+grad'}"


def kernel_source_hash() -> str:
    """Hash of the likelihood kernel's sources (its translation unit loglik.cu, every
    header, and matern.cu, which builds the table the kernel reads) with comments and blank
    space removed, so that the DRAM counters in profiles/traffic.json stay attached to the
    code they were taken on."""
    import glob
    import hashlib
    import re

    csrc = os.path.join(ROOT, "paper_2403_07412_gb300", "csrc")
    files = [os.path.join(csrc, "loglik.cu"), os.path.join(csrc, "matern.cu")] + glob.glob(os.path.join(csrc, "*.cuh"))
    h = hashlib.sha256()
    for f in sorted(files):
        src = open(f, encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).strip().encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = dict(ln.split(":", 1) for ln in out.splitlines() if ":" in ln)
        name = fields.get("Model name", "").strip()
        vendor = fields.get("Vendor ID", "").strip()
        if name:
            return f"{vendor} {name}".strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model", "hardware")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def make_workload(n, device, rank):
    from paper_2403_07412_gb300 import datagen

    seed = datagen.BASE_SEED + 5 + 1000 * rank
    xy = datagen.gmm_locations(n, seed)
    theta = (1.0, 0.02, 1.0, 0.01)
    y = datagen.field_rff(xy, theta, seed + 1000, device=device)
    return xy, y, theta


def la_flops_fields(ns, ms, grad: bool) -> float:
    return sum(la_flops(int(n), int(m), grad) for n, m in zip(ns, ms))


def run_batched(V, dev, peak_tflops, nfields=64, ntheta=32, scale=1.0, reps=1):
    """Many-field workload: nfields uniform fields, n log-uniform in [10k, 500k] (times
    scale), m uniform on {10, 30, 60}, ntheta candidates per field with nu in
    {0.5, 1.0, 1.5}; loglik + gradient for every (field, theta) in one persistent launch,
    captured once in a CUDA graph and replayed."""
    import torch
    from paper_2403_07412_gb300 import datagen

    seed = datagen.BASE_SEED + 4
    ns, ms = datagen.batch_sizes(nfields, seed)
    ns = np.maximum((ns * scale).astype(np.int64), 100)
    thetas = datagen.theta_candidates(nfields, ntheta, seed + 1)
    plans, ys = [], []
    t0 = time.perf_counter()
    for f in range(nfields):
        xy = datagen.uniform_locations(int(ns[f]), seed + 10 + f)
        y = datagen.field_rff(xy, thetas[f, 0], seed + 1000 + f, device=dev)
        plans.append(V.Plan(xy, int(ms[f]), order=V.ORDER_RANDOM, seed=seed + 2000 + f))
        ys.append(torch.as_tensor(y, device=dev))
    setup_s = time.perf_counter() - t0
    V.vecchia_batched_prepare([0.5, 1.0, 1.5])
    b = V.Batch(plans, ys, ntheta, want_grad=True)
    th = torch.as_tensor(thetas, device=dev).contiguous()
    out = torch.empty((nfields, ntheta, 4), dtype=torch.float64, device=dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        b.run(th, out)  # lays out the work (first call), also the warm-up
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run(th, out)
    g.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms_rep = e0.elapsed_time(e1) / reps
    locs = float(ns.sum()) * ntheta
    flops = la_flops_fields(ns, ms, True) * ntheta
    achieved = flops / (ms_rep * 1e-3) / 1e12
    res = out.cpu().numpy()
    for p in plans:
        p.close()
    return {"workload": f"{nfields} fields x {ntheta} thetas, n log-uniform 10k-500k (sum {int(ns.sum())}), "
                        "m in {10,30,60}, nu in {0.5,1.0,1.5}, uniform locations, random ordering, fwd+grad",
            "value": locs / (ms_rep * 1e-3), "unit": "locations/s", "ms_per_call": ms_rep,
            "location_evaluations": int(locs), "graph_replays_timed": reps,
            "frac_of_fp64_peak": achieved / peak_tflops, "achieved_tflops": achieved,
            "result_finite": bool(np.all(np.isfinite(res))), "setup_seconds": round(setup_s, 1)}


def _time_call(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_configs(V, dev, peak_tflops):
    """The other workloads of the study as lines of their own (seeds as in the tests):
    2,000 uniform locations with an exactly drawn field (nu = 0.5, m = 10, forward);
    100,000 uniform, random-Fourier-feature field (nu = 1.5, tau2 = 0.01, m = 30,
    forward); 250,000 uniform (nu = 2.5, tau2 = 0.05, m = 60, forward + gradient).  All
    random ordering.  frac counts F(k) per location as the headline's roofline does."""
    import torch
    from paper_2403_07412_gb300 import datagen

    B = datagen.BASE_SEED
    specs = [
        ("uniform2k-exact-nu0.5-m10-fwd", 2_000, (1.0, 0.1, 0.5, 0.0), 10, B + 1, False, True, 200),
        ("uniform100k-rff-nu1.5-m30-fwd", 100_000, (1.0, 0.05, 1.5, 0.01), 30, B + 2, False, False, 20),
        ("uniform250k-rff-nu2.5-m60-fwd+grad", 250_000, (1.5, 0.03, 2.5, 0.05), 60, B + 3, True, False, 10),
    ]
    rows = []
    for name, n, theta, m, seed, grad, exact, reps in specs:
        xy = datagen.uniform_locations(n, seed)
        y = datagen.field_dense(xy, theta, seed + 1000) if exact else datagen.field_rff(xy, theta, seed + 1000,
                                                                                        device=dev)
        yd = torch.as_tensor(y, device=dev)
        plan = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=seed)
        out = torch.empty(4, dtype=torch.float64, device=dev)
        fn = V.vecchia_loglik_grad if grad else V.vecchia_loglik
        ms_call = _time_call(lambda: fn(plan, yd, theta, out=out), reps)
        tf = la_flops(n, m, False) / (ms_call * 1e-3) / 1e12
        rows.append({"workload": f"vecchia-matern-{name}", "n": n, "m": m, "theta": list(theta),
                     "ms_per_call": round(ms_call, 4), "value": n / (ms_call * 1e-3), "unit": "locations/s",
                     "frac_of_fp64_peak": round(tf / peak_tflops, 4), "result_finite": bool(
                         np.all(np.isfinite(out[: 4 if grad else 1].cpu().numpy())))})
        plan.close()
    return rows


def run_nu_steps(V, dev, n=100_000, m=30, steps=8):
    """Smoothness estimation: wall time per step of the differentiable likelihood
    (VecchiaLogLik forward + backward: the adjoint call plus two forward calls at nu +/- h
    for the nu derivative), each step at a smoothness not seen before (so two covariance
    tables are built per step), against the same steps at one cached nu; and an L-BFGS-B
    fit of (sigma2, beta, nu, tau2) on a 20k-location field, per likelihood evaluation."""
    import torch
    from paper_2403_07412_gb300 import datagen, mle

    seed = datagen.BASE_SEED + 2
    theta0 = (1.0, 0.05, 1.5, 0.01)
    xy = datagen.uniform_locations(n, seed)
    yd = torch.as_tensor(datagen.field_rff(xy, theta0, seed + 1000, device=dev), device=dev)
    plan = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=seed)

    def step(nu):
        th = torch.tensor([theta0[0], theta0[1], nu, theta0[3]], dtype=torch.float64, requires_grad=True)
        V.VecchiaLogLik.apply(th, plan, yd).backward()
        torch.cuda.synchronize()

    step(1.5)
    t0 = time.perf_counter()
    for k in range(steps):
        step(1.5 + 0.0123 * (k + 1))
    fresh = (time.perf_counter() - t0) / steps
    t0 = time.perf_counter()
    for _ in range(steps):
        step(1.5)
    cached = (time.perf_counter() - t0) / steps
    plan.close()
    n2 = 20_000
    xy2 = datagen.uniform_locations(n2, seed + 7)
    y2 = torch.as_tensor(datagen.field_rff(xy2, theta0, seed + 1007, device=dev), device=dev)
    p2 = V.Plan(xy2, m, order=V.ORDER_RANDOM, seed=seed)
    t0 = time.perf_counter()
    res = mle.fit(p2, y2, (0.8, 0.08, 1.0, 0.02), estimate_nu=True)
    fit_s = time.perf_counter() - t0
    p2.close()
    return {"workload": f"{n} uniform locations, m = {m}, Matern, autograd step at a new nu each step",
            "ms_per_step_new_nu": round(fresh * 1e3, 3), "ms_per_step_cached_nu": round(cached * 1e3, 3),
            "table_builds_per_step": 2,
            "mle_fit": {"n": n2, "m": m, "evaluations": res.evaluations, "seconds": round(fit_s, 3),
                        "ms_per_evaluation": round(fit_s / max(res.evaluations, 1) * 1e3, 3),
                        "theta_hat": [round(float(v), 5) for v in res.theta], "theta_true": list(theta0),
                        "iterations": res.iterations, "converged": res.converged, "message": res.message}}


def run_m_sweep(V, dev, peak_tflops, n=250_000, ms=(10, 30, 60, 90, 120, 150)):
    """One evaluation per conditioning size, as in the paper's performance study
    (time and flop rate of a single likelihood evaluation vs m): n uniform locations,
    random ordering, Matérn nu = 1.5."""
    import torch
    from paper_2403_07412_gb300 import datagen

    seed = datagen.BASE_SEED + 6
    xy = datagen.uniform_locations(n, seed)
    theta = (1.0, 0.03, 1.5, 0.01)
    y = torch.as_tensor(datagen.field_rff(xy, theta, seed + 1000, device=dev), device=dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    rows = []
    for m in ms:
        plan = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=seed)
        row = {"m": m, "n": n}
        for name, fn, grad in (("fwd", V.vecchia_loglik, False), ("grad", V.vecchia_loglik_grad, True)):
            fn(plan, y, theta, out=out)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                fn(plan, y, theta, out=out)
            e1.record()
            torch.cuda.synchronize()
            ms_call = e0.elapsed_time(e1) / 3
            tf = la_flops(n, m, grad) / (ms_call * 1e-3) / 1e12
            row[name] = {"ms": round(ms_call, 3), "locations_per_s": n / (ms_call * 1e-3),
                         "tflops": round(tf, 4), "frac_of_fp64_peak": round(tf / peak_tflops, 4)}
        plan.close()
        rows.append(row)
    return rows


def run_sphere(V, dev, peak_tflops, n=250_000, m=60):
    """Great-circle workload (Sec. VI-C stand-in): n (longitude, latitude) points on a
    15 x 15 degree patch, radius 6371 km, random ordering, Matérn nu = 0.5 with
    beta = 50 km and a 3-D random-Fourier-feature field in chordal distance."""
    import torch
    from paper_2403_07412_gb300 import datagen

    seed = datagen.BASE_SEED + 7
    radius = 6371.0
    ll = datagen.sphere_locations(n, seed)
    theta = (1.0, 50.0, 0.5, 0.02)
    y = torch.as_tensor(datagen.field_rff(datagen.sphere_coords(ll, radius), theta, seed + 1000, device=dev),
                        device=dev)
    t0 = time.perf_counter()
    plan = V.Plan(ll, m, order=V.ORDER_RANDOM, seed=seed, radius=radius)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    out = torch.empty(4, dtype=torch.float64, device=dev)
    row = {"workload": f"{n} lon/lat points on a 15x15-degree patch, great-circle distance (r = 6371 km), "
                       f"random ordering, m = {m}, Matern nu = 0.5, beta = 50 km",
           "plan_seconds": round(plan_s, 3)}
    for name, fn, grad in (("fwd", V.vecchia_loglik, False), ("grad", V.vecchia_loglik_grad, True)):
        fn(plan, y, theta, out=out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fn(plan, y, theta, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms_call = e0.elapsed_time(e1) / 3
        tf = la_flops(n, m, grad) / (ms_call * 1e-3) / 1e12
        row[name] = {"ms": round(ms_call, 3), "locations_per_s": n / (ms_call * 1e-3),
                     "frac_of_fp64_peak": round(tf / peak_tflops, 4)}
    plan.close()
    return row


def run_predict(V, dev, n=250_000, n_new=25_000, m=30):
    """Kriging (the paper's prediction experiment, Sec. VI-C: 250K training and 25K test
    locations) on a synthetic field: predictions per second through vecchia_predict
    (conditioning-set search included) and the mean squared prediction error against
    the held-out values."""
    import torch
    from paper_2403_07412_gb300 import datagen

    seed = datagen.BASE_SEED + 8
    theta = (1.0, 0.01, 1.5, 0.01)
    xy = datagen.uniform_locations(n + n_new, seed)
    y = datagen.field_rff(xy, theta, seed + 1000, device=dev)
    plan = V.Plan(xy[:n], m, order=V.ORDER_RANDOM, seed=seed)
    yd = torch.as_tensor(y[:n], device=dev)
    V.vecchia_predict(plan, xy[n:n + 1000], yd, theta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mean, var = V.vecchia_predict(plan, xy[n:], yd, theta)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    err = mean.cpu().numpy() - y[n:]
    plan.close()
    return {"workload": f"{n} observed / {n_new} new uniform locations, m = {m}, Matern nu = 1.5, beta = 0.01",
            "predictions_per_s": n_new / dt, "seconds": round(dt, 4),
            "mspe": float(np.mean(err ** 2)), "field_variance": float(np.var(y[n:])),
            "mean_predictive_var": float(var.mean().item())}


def cpu_baseline(xy, y, theta, m, budget_s, perm, nbr):
    """The oracle, as it stands, on a bounded random sample of the timed plan's own rows:
    the GPU plan's maxmin ordering ``perm`` and conditioning sets ``nbr`` (ordered
    indices) are handed to the oracle's per-location evaluation, so both sides compute
    the same terms.  The plan (ordering, neighbour search) is excluded from the timing;
    the oracle's own brute-force neighbour search and maxmin ordering are timed apart."""
    import oracle

    oracle.build()
    n = xy.shape[0]
    xo, yo = xy[perm], y[perm]
    rng = np.random.default_rng(0)
    probe = np.sort(rng.choice(np.arange(m + 1, n), 64, replace=False))
    nb = np.ascontiguousarray(nbr[probe])
    t0 = time.perf_counter()
    oracle.vecchia_rows(xo, yo, m, theta, rows=probe, nbr=nb, want_grad=True)
    per_row = (time.perf_counter() - t0) / probe.size
    rows_n = int(max(64, min(200_000, budget_s / max(per_row, 1e-7))))
    rows = np.sort(rng.choice(np.arange(m + 1, n), rows_n, replace=False))
    nb = np.ascontiguousarray(nbr[rows])
    knn_rows = rows[: max(64, rows_n // 8)]
    t0 = time.perf_counter()
    nb_oracle = oracle.knn_rows(xo, m, knn_rows)
    knn_s = time.perf_counter() - t0
    knn_same = bool(np.array_equal(nb_oracle, nb[: knn_rows.size]))
    t0 = time.perf_counter()
    oracle.vecchia_rows(xo, yo, m, theta, rows=rows, nbr=nb, want_grad=True)
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    # one thread on a smaller slice of the same rows
    one = rows[: max(16, rows_n // (4 * max(cores, 1)))]
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.vecchia_rows(xo, yo, m, theta, rows=one, nbr=nb[: one.size], want_grad=True)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    # the oracle's maxmin ordering on the first 100k locations of the workload
    sub = xy[: min(n, 100_000)]
    t0 = time.perf_counter()
    oracle.order_maxmin(sub)
    mm_s = time.perf_counter() - t0
    return {"value": rows_n / dt, "unit": "locations/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"{rows_n} random locations (i > m) of the timed {n}-location plan, loglik+grad, "
                      f"the plan's own maxmin ordering and conditioning sets; {dt:.1f} s wall",
            "same_config": True,
            "excludes": "the plan (ordering and neighbour search), on both sides",
            "single_thread": {"value": one.size / dt1, "unit": "locations/s", "sample": f"{one.size} of the same rows"},
            "knn_rows_per_s": knn_rows.size / knn_s,
            "knn_rows_match_plan": knn_same,
            "maxmin_100k_s": round(mm_s, 3)}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, timed per step on a bounded sample."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    n, m = args.n, args.m
    xy, y, theta = make_workload(n, None, 0)
    perm = oracle.order_random(n, 99)
    xo, yo = xy[perm], y[perm]
    rng = np.random.default_rng(0)
    probe = np.sort(rng.choice(np.arange(m + 1, n), 64, replace=False))
    nb = oracle.knn_rows(xo, m, probe)
    t0 = time.perf_counter()
    oracle.vecchia_rows(xo, yo, m, theta, rows=probe, nbr=nb, want_grad=True)
    per_row = (time.perf_counter() - t0) / probe.size
    total_steps = args.steps + args.warmup
    rows_n = int(max(32, min(100_000, args.ref_budget / total_steps / max(per_row, 1e-7))))
    rows = np.sort(rng.choice(np.arange(m + 1, n), rows_n, replace=False))
    nb = oracle.knn_rows(xo, m, rows)
    times = []
    for s in range(total_steps):
        t0 = time.perf_counter()
        oracle.vecchia_rows(xo, yo, m, theta, rows=rows, nbr=nb, want_grad=True)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_step = statistics.median(times)
    value = rows_n / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "locations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_label(n, m, args.order, False), "n": n, "m": m,
                   "ordering": "random (oracle's own)",
                   "theta": list(theta), "sample_locations_per_step": rows_n},
        "cpu_baseline": {"value": value, "unit": "locations/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                         "sample": f"{rows_n} random locations of the {n}-location workload per step "
                                   "(the oracle's own random ordering and brute-force conditioning sets)",
                         "excludes": "the ordering and neighbour search (done once, untimed)"},
        "e2e": {"value": value, "unit": "locations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--m", type=int, default=60)
    ap.add_argument("--order", default="maxmin", choices=["maxmin", "random"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle wall time")
    ap.add_argument("--ref-budget", type=float, default=90.0, help="seconds for the whole reference run")
    ap.add_argument("--fwd", action="store_true", help="time the forward-only kernel instead")
    ap.add_argument("--no-batched", action="store_true", help="skip the many-field batched measurement")
    ap.add_argument("--no-m-sweep", action="store_true", help="skip the conditioning-size sweep")
    ap.add_argument("--no-sphere", action="store_true", help="skip the great-circle workload")
    ap.add_argument("--no-predict", action="store_true", help="skip the kriging workload")
    ap.add_argument("--batched-scale", type=float, default=1.0, help="scale of the batched fields' sizes")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' lines")
    ap.add_argument("--shard", default="locations", choices=["locations", "fields"],
                    help="N > 1: split one field's locations across ranks, or one independent field per rank")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2403_07412_gb300 import build as vbuild

    if rank == 0:
        vbuild.build()
    if dist is not None:
        dist.barrier()
    from paper_2403_07412_gb300 import vecchia as V

    from paper_2403_07412_gb300 import shard

    dev = torch.device("cuda", local)
    n, m = args.n, args.m
    split = world > 1 and args.shard == "locations"
    # one field shared by all ranks (location split), or one field per rank
    xy, y, theta = make_workload(n, dev, 0 if args.shard == "locations" else rank)
    t0 = time.perf_counter()
    plan = V.Plan(xy, m, order=V.ORDER_MAXMIN if args.order == "maxmin" else V.ORDER_RANDOM, seed=5)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    yd = torch.as_tensor(y, device=dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    fn = V.vecchia_loglik if args.fwd else V.vecchia_loglik_grad
    r0, r1 = shard.location_ranges(n, world)[rank] if split else (0, n)

    def call(plan, yd, theta, out):
        if split:  # this rank's range, then one all-reduce of the result doubles
            return shard.loglik_sharded(plan, yd, theta, rank, world, want_grad=not args.fwd, out=out)
        return fn(plan, yd, theta, out=out)

    peak_gflops = V.vecchia_fp64_peak()

    for _ in range(args.warmup):
        call(plan, yd, theta, out=out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if world == 1 else str(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        time.sleep(0.3)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for s in range(args.steps):
            ev[s][0].record(stream)
            call(plan, yd, theta, out=out)
            ev[s][1].record(stream)
        g1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = g0.elapsed_time(g1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    job_locations = n if (split or world == 1) else world * n
    value = job_locations / (ms_per_step * 1e-3)
    res = out.cpu().numpy()
    ok = bool(np.all(np.isfinite(res)))

    # end to end: field from pinned host memory, result back to the host, every step
    y_host = torch.as_tensor(y).pin_memory()
    res_host = torch.empty(4, dtype=torch.float64).pin_memory()
    for _ in range(2):
        yd.copy_(y_host, non_blocking=True)
        call(plan, yd, theta, out=out)
        res_host.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        yd.copy_(y_host, non_blocking=True)
        call(plan, yd, theta, out=out)
        res_host.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    # the plain per-field forward kernel on the same plan
    fwd_ms = None
    if not args.fwd:
        for _ in range(2):
            V.vecchia_loglik(plan, yd, theta, out=out)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            V.vecchia_loglik(plan, yd, theta, out=out)
        f1.record(stream)
        torch.cuda.synchronize()
        fwd_ms = f0.elapsed_time(f1) / args.steps

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # rank 0's kernel processes its own range [r0, r1) (all n on one GPU)
    flops = la_flops_range(r0, r1, m, grad=False)
    flops_adj = la_flops_range(r0, r1, m, grad=not args.fwd)
    kern_ms = statistics.mean(step_ms)
    achieved = flops / (kern_ms * 1e-3) / 1e12
    peak = peak_gflops / 1e3
    traffic = None
    traffic_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(traffic_path):
        # DRAM bytes per launch from the last ncu capture, valid only for the kernel
        # sources it was taken on.
        try:
            tj = json.load(open(traffic_path))
            key = "fwd" if args.fwd else "grad"
            if (tj.get("n") == n and tj.get("m") == m and tj.get("order", "maxmin") == args.order
                    and tj.get("source_hash") == kernel_source_hash()):
                traffic = tj.get(key)
        except Exception:
            traffic = None
    hbm_gbs = traffic / (kern_ms * 1e-3) / 1e9 if traffic else None
    cov_evals = float(sum(min(i, m) * (min(i, m) + 1) // 2 for i in range(min(n, m + 1)))) + \
        float(max(n - (m + 1), 0)) * (m * (m + 1) // 2)
    # labels follow the arguments; the defaults give WORKLOAD and the warp kernel
    workload = workload_label(n, m, args.order, args.fwd)
    kern_name = ("vecchia_big_kernel" if m > 63 else "vecchia_lik_kernel") + ("<false>" if args.fwd else "<true>")
    step_bytes = n * (16 + 8 + 4 * m)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "locations/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "strong" if args.shard == "locations" else "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": workload,
            "n": n, "m": m, "ordering": args.order, "theta": list(theta),
            "locations": "20-component Gaussian mixture in [0,1]^2",
            "field": "random Fourier features, 4096, Matern nu=1.0",
            "l2": (f"inputs {'exceed' if step_bytes > 129e6 else 'fit in'} L2 ({step_bytes / 1e6:.0f} MB per step: "
                   f"{n * 4 * m / 1e6:.0f} MB neighbour table, {n * 16 / 1e6:.0f} MB coordinates, "
                   f"{n * 8 / 1e6:.0f} MB field)"),
            "plan_seconds": round(plan_s, 3),
            "result_finite": ok,
            "parallelism": (f"one field, ordered locations split into {world} ranges (one per GPU), "
                            "NCCL all-reduce of the 4 result doubles per step" if split else
                            "1 GPU" if world == 1 else f"{world} independent fields (one per GPU)"),
        },
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kern_name,
                     "flops_per_launch": flops,
                     "flops_count": "F(k) = k^3/3 + k^2/2 + k/6 + k^2 per location, k = m_i + 1 "
                                    "(Cholesky and two triangular solves)",
                     "frac_with_adjoint_solves": (flops_adj / (kern_ms * 1e-3) / 1e12) / peak,
                     "peak_source": "FP64 DFMA-chain kernel measured in this run (vecchia_fp64_peak)"},
        "covariance": {"entries_per_call": cov_evals, "entries_per_s": cov_evals / (kern_ms * 1e-3),
                       "note": "off-diagonal covariance entries k(k-1)/2 per location, k = m_i + 1"},
        "hbm": {"gbs": hbm_gbs, "source": "ncu dram bytes per launch (profiles/traffic.json) / CUDA-event time"},
        "e2e": {"value": job_locations / (e2e_ms * 1e-3), "unit": "locations/s",
                "h2d_bytes_per_step": int(y_host.numel() * 8), "d2h_bytes_per_step": int(res_host.numel() * 8)},
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
    }
    if fwd_ms is not None:
        ff = la_flops(n, m, grad=False)
        line["forward"] = {"kernel": "vecchia_lik_kernel<false> (plain per-field forward)",
                           "value": n / (fwd_ms * 1e-3), "unit": "locations/s", "ms_per_call": fwd_ms,
                           "frac_of_fp64_peak": ff / (fwd_ms * 1e-3) / 1e12 / peak}
    if not args.no_configs:
        line["configs"] = run_configs(V, dev, peak)
        line["nu_estimation"] = run_nu_steps(V, dev)
    if not args.no_batched:
        line["batched"] = run_batched(V, dev, peak, scale=args.batched_scale)
    if not args.no_m_sweep:
        line["m_sweep"] = run_m_sweep(V, dev, peak)
    if not args.no_sphere:
        line["sphere"] = run_sphere(V, dev, peak)
    if not args.no_predict:
        line["predict"] = run_predict(V, dev)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(xy, y, theta, m, args.cpu_budget, plan.perm(), plan.neighbors())
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""RS-S benchmark on GB300: factor + solve of the 1024 x 1024 Laplace workload.

A step is one pass of the whole hot path over one synthetic problem: every
compressed level of the factorization (leaf kernel blocks, proxy ID,
sparsification and LU, Schur updates, merge), the dense top LU, and one
1-right-hand-side solve (upward sweep, top solve, downward sweep).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead: each step is the oracle on a 128 x 128 grid of the same
workload, and the config names that size (a scaled full-size figure is reported
separately and labelled as a model).  With N > 1 under torchrun every rank
factors its own copy (replicas: the single-GPU path has no data exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD = "laplace_1024x1024_eps1e-6"
METRIC = "RS-S factor s and solve RHS/s at N=1M, rel.res<=1e-5; serve p50/p99 latency"
# FP64 roof of the FP64-bound phases: the nominal FP64 rate of a GB300, 1.25
# TFLOP/s (152 SMs x 2.07 GHz x 2 FP64 FMA per clock and SM x 2 flop = 1.26).  The
# bench also measures it with the library's DFMA probe (rss_probe_fp64) and
# reports both; FP64 tensor-core MMAs (mma.sync f64) are no faster than DFMA here.
FP64_PEAK_TFLOPS = 1.25
# DRAM bytes (read + write) of the dominant phase's kernels per factorization of
# the 1024 x 1024 Laplace workload, from an ncu capture of the same kernels on a
# smaller grid scaled by the boxes processed (source in the dict); None when the
# kernels have changed since the capture.
TRAFFIC = {"id": {"bytes_per_factor": 31.22e9 * (78.52 / 19.18),
                  "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over every k_id and k_id_cl "
                            "launch of one 512 x 512 Laplace factorization (31.2 GB), scaled to 1024 x 1024 "
                            "by the ratio of the phase's algorithmic flops (78.5 / 19.2 GFLOP), then divided "
                            "by the launches of one factorization"}}
CPU_SAMPLE_SIDES = (128, 256)   # oracle samples: the same workload on these grids


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--multi-rhs", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2100,
                    help="requests per load, the first 100 warm-up (2100: the full protocol)")
    ap.add_argument("--no-large", action="store_true", help="skip the 2048^2 Helmholtz served run")
    ap.add_argument("--solve-launch", default="tune", choices=["tune", "per_class", "persistent"],
                    help="launch form of the 1-RHS sweeps: measured once during the warm-up (tune), or "
                         "fixed (for captures under a profiler, which distorts the measurement)")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the FP64 throughput probes (the roofline then keeps the nominal peak only)")
    ap.add_argument("--serve-loads", type=float, nargs="+", default=[0.5, 0.9])
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- residual
def fft_relres(torch, pts_side, kind, h, kappa, x, b):
    """||A x - b|| / ||b|| on the GPU with a zero-padded 2D FFT (A is BTTB on the grid).

    A validation check of the result, separate from the hot path."""
    s = pts_side
    dev = x.device
    d = torch.arange(-(s - 1), s, device=dev, dtype=torch.float64)
    DY, DX = torch.meshgrid(d, d, indexing="ij")
    r2 = (DX * DX + DY * DY) * (h * h)
    r2[s - 1, s - 1] = 1.0
    if kind == W.LAPLACE:
        kv = -(h * h / (4 * math.pi)) * torch.log(r2)
    else:
        kr = kappa * torch.sqrt(r2)
        kv = (h * h) * torch.complex(-0.25 * torch.special.bessel_y0(kr), 0.25 * torch.special.bessel_j0(kr))
    kv[s - 1, s - 1] = 0
    circ = torch.zeros((2 * s, 2 * s), dtype=kv.dtype, device=dev)
    idx = torch.arange(-(s - 1), s, device=dev) % (2 * s)
    circ[idx[:, None], idx[None, :]] = kv
    kf = torch.fft.fft2(circ)
    num = den = 0.0
    for j in range(x.shape[1]):
        pad = torch.zeros((2 * s, 2 * s), dtype=torch.complex128, device=dev)
        pad[:s, :s] = x[:, j].reshape(s, s)
        y = torch.fft.ifft2(kf * torch.fft.fft2(pad))[:s, :s].reshape(-1)
        if not x.is_complex():
            y = y.real
        r = y + x[:, j] - b[:, j]            # diagonal entries are 1
        num += float(torch.linalg.vector_norm(r)) ** 2
        den += float(torch.linalg.vector_norm(b[:, j])) ** 2
    return math.sqrt(num / den)


# ----------------------------------------------------------------------------- CPU oracle
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import workloads as W
from oracle import rss
from oracle.rss import KernelSpec
kind, kappa, eps, seed = {kind}, {kappa}, {eps}, {seed}
out = []
for side, reps in {plan!r}:
    pts = W.grid_points(side)
    spec = KernelSpec("laplace" if kind == W.LAPLACE else "helmholtz", h=1.0 / side, kappa=kappa)
    b = W.gaussian_rhs(side * side, 1, kind != W.LAPLACE, seed)
    for _ in range(reps):
        t0, c0 = time.perf_counter(), time.process_time()
        fac = rss.factor(pts, spec, eps)
        x = rss.solve(fac, b)
        out.append({{"side": side, "s": time.perf_counter() - t0, "cpu_s": time.process_time() - c0}})
print(json.dumps(out))
"""


def host_info():
    """Host cores and CPU model (the oracle's timings are only meaningful with them)."""
    info = {"nproc": os.cpu_count()}
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        keep = ("Architecture", "Model name", "Socket(s)", "Core(s) per socket", "Thread(s) per core",
                "CPU(s)", "CPU max MHz")
        info["lscpu"] = {k.strip(): v.strip() for k, v in
                         (ln.split(":", 1) for ln in txt.splitlines() if ":" in ln) if k.strip() in keep}
    except (OSError, subprocess.SubprocessError):
        info["lscpu"] = None
    return info


def run_oracle(w, plan):
    """Time the oracle (factor + 1-RHS solve) as it stands, once per (side, reps)
    entry of plan, in one process, with the BLAS thread pools set to every host core."""
    nproc = str(os.cpu_count() or 1)
    env = dict(os.environ, OMP_NUM_THREADS=nproc, OPENBLAS_NUM_THREADS=nproc, MKL_NUM_THREADS=nproc)
    code = CPU_SNIPPET.format(root=ROOT, kind=w["kind"], kappa=w["kappa"], eps=w["eps"], seed=w["seed"],
                              plan=list(plan))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def sample_name(w, side):
    kind = "laplace" if w["kind"] == W.LAPLACE else f"helmholtz_k{w['kappa']:g}"
    return f"{kind}_{side}x{side}_eps" + f"{w['eps']:.0e}".replace("e-0", "e-")


def cpu_block(w, runs):
    """The oracle on two grids of the workload (the larger one is the reported
    sample); the full-size figure is a power-law model fitted to the two, kept in
    its own key."""
    by = {}
    for r in runs:
        by.setdefault(r["side"], []).append(r)
    sides = sorted(by)
    big = sides[-1]
    t = {sd: statistics.mean(r["s"] for r in by[sd]) for sd in sides}
    util = statistics.mean(r["cpu_s"] / r["s"] for r in by[big])
    out = {"value": t[big], "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": (f"oracle factor + 1-RHS solve of {sample_name(w, big)} ({big * big} points; the "
                      f"workload's kernel, eps, leaf and proxies), {len(by[big])} run(s), BLAS threads = "
                      f"{os.cpu_count()} (cores), measured CPU time / wall time {util:.2f}"),
           "n": big * big, "cpu_busy_cores": util, "host": host_info(),
           "measured_s": {str(sd * sd): t[sd] for sd in sides}}
    if len(sides) > 1 and w["side"] > big:
        a = math.log(t[big] / t[sides[0]]) / math.log((big / sides[0]) ** 2)
        out["model_full_size"] = {"s": t[big] * ((w["side"] / big) ** 2) ** a, "n": w["side"] ** 2,
                                  "exponent": a, "kind": "model, not measured: t ~ N^exponent fitted "
                                                         "to the two measured sizes"}
    return out


REF_SAMPLE_SIDE = 128   # one reference step: the oracle on a 128 x 128 grid of the workload


def reference_arm(args, w):
    """The CPU oracle as it stands, timed on the host cores.  A step is one oracle
    factor + 1-RHS solve of the workload's problem on a 128 x 128 grid (the full
    1024 x 1024 problem takes the oracle far longer than the run may last); the
    config names that size.  A linear (O(N)) model of the full size is given in
    its own key and is not a measurement."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    side = min(REF_SAMPLE_SIDE, w["side"])
    runs = run_oracle(w, [(side, args.warmup + args.steps)])
    times = [r["s"] for r in runs[args.warmup:]]
    util = statistics.mean(r["cpu_s"] / r["s"] for r in runs[args.warmup:])
    value = statistics.mean(times)
    cb = {"value": value, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": (f"oracle factor + 1-RHS solve of {sample_name(w, side)} ({side * side} points) per step, "
                     f"BLAS threads = {os.cpu_count()} (cores), measured CPU time / wall time {util:.2f}"),
          "cpu_busy_cores": util, "host": host_info()}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if not w["complex"] else "c128", "data": "synthetic",
            "config": {"workload": sample_name(w, side), "sample_of": args.workload, "n": side * side,
                       "eps": w["eps"], "leaf": W.LEAF, "proxy_n": W.PROXY_N, "rhs": 1,
                       "parallelism": "replicas" if args.gpus > 1 else "single"},
            "model_full_size": {"s": value * (w["side"] / side) ** 2, "n": w["side"] ** 2,
                                "kind": "model, not measured: the sample's time scaled by the point count "
                                        "(the method is O(N); this oracle grows faster than that, so the "
                                        "model is a lower bound)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- the paper's problems
PAPER_SET = [("laplace_quadrature_2048x2048", W.LAPLACE, 2048, 0.0),
             ("lippmann_schwinger_k25_1024x1024", W.HELMHOLTZ_LS, 1024, 25.0),
             # increasing frequency, kappa = pi sqrt(N) / 16 (32 points per wavelength)
             ("lippmann_schwinger_increasing_1024x1024", W.HELMHOLTZ_LS, 1024, math.pi * 1024 / 16),
             ("lippmann_schwinger_increasing_2048x2048", W.HELMHOLTZ_LS, 2048, math.pi * 2048 / 16)]


def proxy_count(kappa, side):
    """Proxy points for the paper's problems: at least 64, and 2 kappa R + 30 on the
    proxy circle of radius R = 2.5 L of the coarsest compressed boxes (L = 1/4), so
    that the circle resolves the kernel's oscillation at the highest frequencies."""
    return max(64, int(math.ceil(2 * kappa * 2.5 * 0.25 + 30)))


def paper_problems(P, torch):
    """The paper's own discretisations (Section 5), run as the paper runs them:
    Laplace with the self-cell quadrature diagonal (Eq. 16) and the symmetrised
    Lippmann-Schwinger system at kappa = 25 and at the increasing frequency
    kappa = pi sqrt(N) / 16 of Table "h2" (Eqs. 19-20, Gaussian bump), proxy
    radius 2.5 L (Section 2.3), eps 1e-6, leaf 64, one right-hand side of
    uniform random entries, refined to a relative residual of 1e-12 by PCG /
    GMRES(20) with the factorization as preconditioner.  Reported beside the
    paper's single-process rows (CPU, other hardware): context only."""
    out = {}
    for name, kind, side, kappa in PAPER_SET:
        n = side * side
        tree = P.rss_build_tree(W.grid_points(side), W.LEAF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            f = P.rss_factor(tree, kind=kind, eps=1e-6, h=1.0 / side, kappa=kappa, diag_rule=1,
                             proxy_radius_over_side=2.5, proxy_n=proxy_count(kappa, side))
        except P.RSSError as e:
            out[name] = {"n": n, "kappa": kappa, "error": str(e)}
            continue
        torch.cuda.synchronize()
        t_fact = time.perf_counter() - t0
        rng = np.random.default_rng(2001)
        if f.is_complex:
            bh = rng.uniform(size=n) + 1j * rng.uniform(size=n)
        else:
            bh = rng.uniform(size=n)
        b = torch.from_numpy(bh).cuda()
        x = b.clone()
        P.rss_solve(f, x)                      # warm-up (plans, workspaces)
        P.rss_matvec(f, x)
        x = b.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.rss_solve(f, x)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        r = P.rss_matvec(f, x) - b
        direct = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it, rr = P.rss_solve_iterative(f, b, tol=1e-12)
        torch.cuda.synchronize()
        t_it = time.perf_counter() - t0
        info = P.rss_info(f)
        out[name] = {"n": n, "kappa": kappa, "proxy_n": proxy_count(kappa, side),
                     "factor_s": t_fact, "solve_s": t_solve, "relres_direct": direct,
                     "iterations": it, "relres_iterative": rr, "iterative_s": t_it,
                     "method": "gmres20" if f.is_complex else "pcg",
                     "ranks": [{"side": L["side"], "k_mean": L["k_mean"], "k_max": L["k_max"]}
                               for L in info["levels"]]}
        del f, tree
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- serving
SERVE_SET = [("laplace", 128, 0.0), ("laplace", 256, 0.0), ("laplace", 512, 0.0),
             ("helmholtz", 256, 25.0)]


def _drive(P, srv, ids, pool, which, nrhs, gaps):
    """Submit request q at time sum(gaps[:q+1]) (all at once when gaps is None) from
    host buffers; a second thread waits for the tickets in order.  Returns the
    latencies (s) and the wall time from the first submission to the last result."""
    import threading
    nreq = len(which)
    tickets = [None] * nreq
    lat = [0.0] * nreq
    done = threading.Event()

    def waiter():
        for q in range(nreq):
            while tickets[q] is None:
                time.sleep(1e-5)
            _, lat[q] = P.rss_server_wait(srv, tickets[q], timeout=300.0)
        done.set()

    th = threading.Thread(target=waiter)
    th.start()
    t_start = time.perf_counter()
    t_next = t_start
    for q in range(nreq):
        if gaps is not None:
            t_next += gaps[q]
            while time.perf_counter() < t_next:
                pass
        j = int(which[q])
        tickets[q] = P.rss_server_submit(srv, ids[j], np.asfortranarray(pool[j][:, :int(nrhs[q])]))
    done.wait()
    t_total = time.perf_counter() - t_start
    th.join()
    return np.array(lat), t_total


def serve_run(P, torch, args):
    """Resident factorizations (Laplace 128^2, 256^2, 512^2 and Helmholtz kappa = 25 at
    256^2, eps 1e-6) behind the continuous-batching server; seeded Poisson arrivals of
    requests with 1-64 Gaussian right-hand sides on a uniformly drawn factorization, at
    loads of 50 % and 90 % of the solo capacity, then the same requests submitted all at
    once (saturation: the server's capacity).  The first 100 requests of each run are
    warm-up.  Latency = submit to result in host memory.  Beside it, requests of the
    saturation run solved one after another with no server (each alone, host buffers)
    give the plain throughput."""
    facs = []
    for kind, side, kappa in SERVE_SET:
        tree = P.rss_build_tree(W.grid_points(side), W.LEAF)
        facs.append(P.rss_factor(tree, kind=W.LAPLACE if kind == "laplace" else W.HELMHOLTZ,
                                 eps=1e-6, h=1.0 / side, kappa=kappa))
    # the solve's launch form for each resident factorization, tuned once (1 column)
    tuning = [P.rss_tune_solve(f, 1) for f in facs]
    pool = {}
    for j, f in enumerate(facs):
        pool[j] = W.gaussian_rhs(f.n, 64, f.is_complex, 2000 + j)
    # solo capacity: mean service time of one request alone (32-column panel, host buffers)
    solo = []
    for j, f in enumerate(facs):
        b = np.asfortranarray(pool[j][:, :32].copy())
        P.rss_solve(f, b)
        t0 = time.perf_counter()
        for _ in range(3):
            b = np.asfortranarray(pool[j][:, :32].copy())
            P.rss_solve(f, b)
        solo.append((time.perf_counter() - t0) / 3)
    srv = P.rss_server_create(24 << 30, 256)
    ids = [P.rss_server_add(srv, f) for f in facs]
    nreq = args.serve_requests
    warm = min(100, nreq // 6)
    rng = np.random.default_rng(1003)
    which = rng.integers(0, len(facs), nreq)
    nrhs = rng.integers(1, 65, nreq)
    mean_service = float(np.mean(solo)) * (np.mean(nrhs) / 32.0)
    runs = []
    for li, load in enumerate(list(args.serve_loads) + [None]):
        if load is None:
            lat, t_total = _drive(P, srv, ids, pool, which, nrhs, None)
            rate = None
        else:
            rate = load / mean_service
            gaps = np.random.default_rng(2003 + li).exponential(1.0 / rate, nreq)
            lat, t_total = _drive(P, srv, ids, pool, which, nrhs, gaps)
        l = lat[warm:] * 1e3
        runs.append({"load": "saturation (all requests submitted at once)" if load is None else load,
                     "arrival_rate_per_s": rate, "p50_ms": float(np.percentile(l, 50)),
                     "p99_ms": float(np.percentile(l, 99)), "mean_ms": float(l.mean()),
                     "rhs_per_s": float(nrhs.sum() / t_total), "wall_s": t_total})
    st = P.rss_server_stats(srv)
    # the plain form: requests one after another, each solved alone (host buffers)
    nplain = min(nreq - warm, 600)
    t0 = time.perf_counter()
    for q in range(warm, warm + nplain):
        j = int(which[q])
        b = np.asfortranarray(pool[j][:, :int(nrhs[q])].copy())
        P.rss_solve(facs[j], b)
    plain = float(nrhs[warm:warm + nplain].sum() / (time.perf_counter() - t0))
    sat = runs[-1]["rhs_per_s"]
    return {"workload": "Laplace 128^2, 256^2, 512^2 + Helmholtz k=25 256^2, eps 1e-6, 1-64 RHS",
            "requests_per_run": nreq, "warmup_requests": warm, "runs": runs,
            "plain_sequential_rhs_per_s": plain, "plain_sequential_requests": nplain,
            "served_over_plain_at_saturation": sat / plain,
            "panels": st["batches"], "max_requests_per_panel": st["max_requests_per_batch"],
            "solo_ms_32rhs": [t * 1e3 for t in solo],
            "solve_launch_1rhs": [{"launch": t["launch"], "ms": t["ms"],
                                   "per_class_ms": t["candidates"][0]["ms"]} for t in tuning]}


def served_large_run(P, torch):
    """The 2048 x 2048 Helmholtz workload (kappa = 50, complex, eps 1e-6): factored, then
    its 64 seeded complex Gaussian right-hand sides submitted to the server as 64
    one-column requests at once; the worker batches them into panels.  Relative
    residual of every column by the FFT matvec of the exact A."""
    w = W.WORKLOADS["helmholtz_k50_2048x2048_eps1e-6"]
    side, n = w["side"], w["side"] ** 2
    tree = P.rss_build_tree(W.grid_points(side), W.LEAF)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = P.rss_factor(tree, kind=W.HELMHOLTZ, eps=w["eps"], h=1.0 / side, kappa=w["kappa"])
    torch.cuda.synchronize()
    t_fact = time.perf_counter() - t0
    info = P.rss_info(f)
    b = W.gaussian_rhs(n, w["nrhs"], True, w["seed"])
    srv = P.rss_server_create(64 << 30, 64)
    fid = P.rss_server_add(srv, f)
    # warm-up request (plans, workspaces)
    P.rss_server_wait(srv, P.rss_server_submit(srv, fid, np.asfortranarray(b[:, :1])), timeout=300.0)
    t0 = time.perf_counter()
    tickets = [P.rss_server_submit(srv, fid, np.asfortranarray(b[:, j])) for j in range(w["nrhs"])]
    xs, lat = [], []
    for t in tickets:
        x, l = P.rss_server_wait(srv, t, timeout=300.0)
        xs.append(x)
        lat.append(l)
    t_all = time.perf_counter() - t0
    st = P.rss_server_stats(srv)
    X = torch.from_numpy(np.ascontiguousarray(np.stack(xs, axis=0))).cuda().T
    B = torch.from_numpy(np.ascontiguousarray(b.T)).cuda().T
    R = P.rss_matvec(f, X) - B
    relres = float(torch.linalg.vector_norm(R) / torch.linalg.vector_norm(B))
    lat = np.array(lat) * 1e3
    out = {"workload": "helmholtz_k50_2048x2048_eps1e-6", "n": n, "factor_s": t_fact,
           "factor_gpu_ms": info["gpu_ms"], "rhs": w["nrhs"], "served_rhs_per_s": w["nrhs"] / t_all,
           "served_wall_s": t_all, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "panels": st["batches"] - 1, "relres": relres,
           "ranks": [{"side": L["side"], "k_mean": L["k_mean"], "k_max": L["k_max"]} for L in info["levels"]]}
    del srv, f, tree, X, B, R
    torch.cuda.empty_cache()
    return out


def batching_run(P, torch):
    """What batching a colour class into one launch per phase gains: the 256 x 256
    Laplace workload factored batched and in the plain per-box form (one box per
    launch, same order, one-CTA ID in both so the arithmetic is identical)."""
    side = 256
    tree = P.rss_build_tree(W.grid_points(side), W.LEAF)
    b = W.gaussian_rhs(side * side, 1, False, 1003)[:, 0]
    out = {"workload": "laplace_256x256_eps1e-6"}
    xs = []
    for name, per_box in (("batched", False), ("per_box", True)):
        f = P.rss_factor(tree, kind=W.LAPLACE, eps=1e-6, h=1.0 / side, id_cluster=-1, per_box=per_box)
        del f
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = P.rss_factor(tree, kind=W.LAPLACE, eps=1e-6, h=1.0 / side, id_cluster=-1, per_box=per_box)
        torch.cuda.synchronize()
        out[name + "_factor_s"] = time.perf_counter() - t0
        x = b.copy()
        P.rss_solve(f, x)
        xs.append(x)
        out[name + "_launches"] = P.rss_info(f)["launches"]
        del f
    out["identical_solutions"] = bool(np.array_equal(xs[0], xs[1]))
    return out


# ----------------------------------------------------------------------------- replicas
def max_over_ranks(torch, ms: float, dist, device) -> float:
    """Max of the per-rank times (each rank factors its own copy: no data exchange)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_replicas(torch, step, steps: int, warmup: int, dist, device, start, stop) -> float:
    """warmup untimed steps, a barrier, `steps` timed steps, a barrier; returns the max
    over ranks of ms per step.  start/stop bracket the timed region (CUDA events on the
    GPU)."""
    for _ in range(warmup):
        step()
    if dist is not None and dist.is_initialized():
        dist.barrier()
    start()
    for _ in range(steps):
        step()
    ms = stop() / steps
    if dist is not None and dist.is_initialized():
        dist.barrier()
    return max_over_ranks(torch, ms, dist, device)


# ----------------------------------------------------------------------------- native arm
def native_arm(args, w):
    import torch

    import paper_2310_15458_gb300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    side, eps = w["side"], w["eps"]
    n = side * side
    kind = w["kind"]
    is_c = w["complex"]
    h = 1.0 / side
    pts = W.grid_points(side)
    tree = P.rss_build_tree(pts, W.LEAF)
    b_host = W.gaussian_rhs(n, 1, is_c, w["seed"])
    tdt = torch.complex128 if is_c else torch.float64
    b_dev = torch.from_numpy(np.ascontiguousarray(b_host.T)).to("cuda").T.contiguous()
    stream = torch.cuda.current_stream()
    x = torch.empty_like(b_dev)

    tune = {}   # the solve's launch schedule, measured once during the warm-up

    def factor():
        return P.rss_factor(tree, kind=kind, eps=eps, h=h, kappa=w["kappa"], tune_table=tune or None)

    def step():
        f = factor()
        x.copy_(b_dev)
        P.rss_solve(f, x.view(n, 1), stream=stream)
        return f

    if args.solve_launch == "per_class":
        tune = {"launch": "per_class"}
    elif args.solve_launch == "persistent":
        tune = {"launch": "persistent", "spread": 1, "ctas_per_sm": 0}
    for i in range(args.warmup):
        f = step()
        if i == 0 and args.solve_launch == "tune":
            tune = P.rss_tune_solve(f, 1, stream=stream)
        del f
    barrier()
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        f = step()
        infos.append(P.rss_info(f))
        if _ + 1 < args.steps:
            del f
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(torch, ms, dist, "cuda")
    info = infos[-1]
    relres = fft_relres(torch, side, kind, h, w["kappa"], x.view(n, 1), b_dev.view(n, 1))

    # solve throughput on the resident factorization (1 and multi RHS)
    def solve_rate(nrhs, reps):
        bb = torch.randn(nrhs, n, dtype=torch.float64, device="cuda", generator=None)
        if is_c:
            bb = torch.complex(bb, torch.randn_like(bb))
        xx = bb.clone().T
        P.rss_solve(f, xx, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            xx.copy_(bb.T)
            P.rss_solve(f, xx, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        return t, nrhs / (t * 1e-3)

    t1, r1 = solve_rate(1, 10)
    tm, rm = solve_rate(args.multi_rhs, 2)

    # end to end through the public API with host buffers
    pts_h = np.ascontiguousarray(pts)
    bh = np.ascontiguousarray(b_host[:, 0]).copy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr = P.rss_build_tree(pts_h, W.LEAF)
    fe = P.rss_factor(tr, kind=kind, eps=eps, h=h, kappa=w["kappa"], tune_table=tune or None)
    P.rss_solve(fe, bh)
    e2e_s = time.perf_counter() - t0
    del fe, tr
    esz = 16 if is_c else 8

    # roofline of the dominant factor kernel (device time from CUDA events on the factor's stream)
    gms = info["gpu_ms"]
    dom = max(("id", "elim", "schur"), key=lambda k: gms[k])
    launches = info["phase_launches"][dom]
    flops = info["flops"][dom]
    achieved = flops / (gms[dom] * 1e-3) / 1e12
    kern = {"id": "k_id", "elim": "k_elim", "schur": "k_schur"}[dom]
    tr = TRAFFIC.get(dom) if args.workload == WORKLOAD else None
    traffic = tr["bytes_per_factor"] / max(launches, 1) if tr else None
    if args.no_probe:
        probe_tflops = probe_ms = dmma_tflops = None
    else:
        probe_tflops, probe_ms = P.rss_probe_fp64(stream=stream)
        dmma_tflops, dmma_ms = P.rss_probe_dmma(stream=stream)
    # kernels of one 1-RHS solve: the user-order permutations, the top block's gather and
    # product, and per colour class k_up_r, k_up_c and k_down (per-class form) or the two
    # persistent sweeps (persistent form)
    if info.get("solve_launch") == "persistent":
        solve_launches = 2 + 2 + 2
    else:
        solve_launches = 2 + 2 + 3 * info["batches"]
    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128" if is_c else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "eps": eps, "leaf": W.LEAF, "proxy_n": W.PROXY_N,
                   "rhs": 1, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: the leaf stencil alone is "
                         f"{n // W.LEAF * 25 * W.LEAF * W.LEAF * esz / 1e9:.1f} GB"},
        "factor_s": info["ms"]["total"] / 1e3,
        "solve_1rhs_ms": t1,
        "solve_rhs_per_s": {"1": r1, str(args.multi_rhs): rm},
        "relres": relres,
        "phase_gpu_ms": {k: v for k, v in gms.items() if k != "span"},
        # device time from the first to the last kernel of the factor, and the part of
        # it in which no phase kernel ran (host work between launches)
        "factor_gpu_span_ms": gms.get("span"),
        "factor_gpu_idle_ms": gms["span"] - sum(v for k, v in gms.items() if k != "span")
        if gms.get("span") else None,
        "phase_tflops": {k: info["flops"][k] / (gms[k] * 1e-3) / 1e12 for k in ("id", "elim", "schur", "top")
                         if gms.get(k)},
        "ranks": [{"side": L["side"], "k_mean": L["k_mean"], "k_max": L["k_max"]} for L in info["levels"]],
        "level_gpu_ms": [{"side": L["side"], **L["gpu_ms"]} for L in info["levels"]],
        "ntop": info["ntop"],
        "solve_tuning": tune,
        "clocks": clk,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": pts_h.nbytes + bh.nbytes,
                "d2h_bytes_per_step": bh.nbytes},
        "gpu_launches": args.steps * (info["launches"] + solve_launches),
        "roofline": {"kernel": kern, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "launches": launches, "avg_launch_ms": gms[dom] / max(launches, 1),
                     "peak_source": "nominal FP64 rate (152 SMs x 2.07 GHz x 2 FMA/clk x 2); no FP64 "
                                    "figure in MEASURED_PEAKS.json",
                     "peak_probe": probe_tflops, "frac_of_probe": achieved / probe_tflops if probe_tflops else None,
                     "probe": ("rss_probe_fp64: independent DFMA chains, 8 CTAs x 256 threads per SM, "
                               "best of 5 launches of %.1f ms" % probe_ms) if probe_ms else None,
                     "fp64_mma_probe": dmma_tflops,
                     "traffic_source": tr["source"] if tr else "none for the kernels as built"},
    }
    if not args.no_serve:
        line["serve"] = serve_run(P, torch, args)
        if not args.no_large and world == 1:
            line["served_helmholtz_2048"] = served_large_run(P, torch)
    if not args.no_paper and world == 1:
        line["paper_problems"] = paper_problems(P, torch)
        line["batching"] = batching_run(P, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_block(w, run_oracle(w, [(sd, 1) for sd in CPU_SAMPLE_SIDES if sd <= side]))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    w = W.WORKLOADS[args.workload]
    if args.impl == "reference":
        reference_arm(args, w)
    else:
        native_arm(args, w)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark: ASPCG (SIPG + two-level additive Schwarz PCG) time to a 1e-8 relative residual and solves
per second on one GB300, on the 16384-cell Lloyd-Voronoi workload at p = 3 (163840 dofs, 64 RCB
subdomains, 256 agglomerates at p_c = 1, checkerboard coefficient 1e4 aligned to the subdomains).

One step = one complete solve through the C-ABI: dgasm_setup (extraction and tile Cholesky of the 64
local matrices, coarse transfer, Galerkin A_0, its factor and inverse) followed by dgasm_solve to 1e-8
(SpMV, local solves, coarse correction, fused vector updates, stop test, true residual, Lanczos
estimate).  The assembled SIPG system is resident in HBM before timing starts.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dgasm|reference]
Under torchrun each rank runs an independent replica on its own GPU (the method has no exchange step
on one GPU): weak scaling, value = solves of all ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 rel. residual & solves/s vs FP64 plain PCG; p50/p99 latency"
N_ELEM, SEED, P_DEG, NSUB, NCOARSE, P_C, CONTRAST = 16384, 2, 3, 64, 256, 1, 1e4
WORKLOAD = ("16384 Lloyd-relaxed Voronoi cells of (0,1)^2 (seed 2, 20 Lloyd steps), SIPG p=3 (163840 dofs), "
            "C_sigma=10, 64 RCB subdomains (~2560 dofs), 256 RCB agglomerates at p_c=1, rho=1e4 on a 4x4 "
            "checkerboard of subdomains; f = 2 pi^2 sin(pi x) sin(pi y); rtol 1e-8 from x0=0")
# nominal FP64 issue rate (1/64 of the FP32 rate): 2 FMA per clock per SM; the roofline uses the rate the
# library's probe measures (dgasm_probe_fp64: about 1.68 FMA per clock per SM with every sub-partition busy)
FP64_NOMINAL_FMA_PER_CLK_SM = 2.0
# DRAM bytes (read + write) per stream tile of the FP64 local-solve kernel, from one ncu capture of the
# headline workload's launch (615.8 MB for 74087 tiles); valid only for the kernel source it was taken on
LOCAL_TRAFFIC = {"sha256": "dd12d7c7069094093c9801a4ad85cb01dfb5fe167d8c84b1fbf30787c96a9b65",
                 "bytes_per_stream_tile": 8312}


def local_traffic(tiles):
    import hashlib
    path = os.path.join(ROOT, "paper_1903_11357_gb300", "csrc", "kernels_local.cu")
    with open(path, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()
    if LOCAL_TRAFFIC["sha256"] != h or not LOCAL_TRAFFIC["bytes_per_stream_tile"]:
        return None
    return LOCAL_TRAFFIC["bytes_per_stream_tile"] * tiles


def f_sin(X):
    return 2 * np.pi ** 2 * np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])


def build_problem():
    from synth.coeff import checker_per_subdomain
    from synth.voronoi import voronoi_mesh
    from paper_1903_11357_gb300 import dgasm as dg
    m = voronoi_mesh(N_ELEM, SEED)
    sub, _ = dg.Mesh.from_polymesh(m, np.ones(m.n_elem)).partition(NSUB, 0)
    rho = checker_per_subdomain(m, sub, CONTRAST)
    M = dg.Mesh.from_polymesh(m, rho)
    S = dg.System(M, P_DEG, 10.0, f=f_sin)
    return m, rho, M, S


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_iters():
    """The oracle's own PCG iteration count to 1e-8 on the headline workload, from its stored converged solve
    (tests/golden, written by a script that calls only the oracle)."""
    from tests.golden.make_oracle_solutions import load
    return int(load("p3_c1e4")["iters"])


def oracle_prep(m, rho):
    """Untimed preparation for the CPU baseline: the oracle's SIPG assembly and partitions, and the full
    coarse transfer (needed by the sampled PCG iterations)."""
    import scipy.sparse as sp

    from oracle import partition, schwarz, sipg
    A, b, g = sipg.assemble(m, rho, P_DEG, 10.0, f_sin)
    sub = partition.subdomains(g.centroid, NSUB)
    agg = partition.agglomerates(g.centroid, sub, NSUB, NCOARSE)
    nb = (P_DEG + 1) * (P_DEG + 2) // 2
    R0T = schwarz.prolongation(m, g, agg, P_DEG, P_C)
    return {"m": m, "A": sp.csr_matrix(A), "b": b, "g": g, "agg": agg, "dofs": schwarz.local_dof_sets(sub, nb),
            "R0T": R0T}


def oracle_sample(prep, iters, sample_subdomains=4, sample_elems=1024, sample_iters=10):
    """The CPU oracle timed on a bounded sample of the workload, scaled to one solve.  Setup: the dense
    Cholesky of `sample_subdomains` of the 64 subdomain matrices (x 64 / sample), the L2 prolongation on the
    first `sample_elems` elements (x ne / sample), the Galerkin product A_0 and its Cholesky (measured in
    full).  Solve: `sample_iters` PCG iterations (x iters / sample_iters, iters = the oracle's own count)."""
    from oracle import pcg, schwarz
    from synth.voronoi import PolyMesh
    A, b, m, g, agg, dofs, R0T = (prep[k] for k in ("A", "b", "m", "g", "agg", "dofs", "R0T"))
    t0 = time.perf_counter()
    chol = [np.linalg.cholesky(A[idx][:, idx].toarray()) for idx in dofs[:sample_subdomains]]
    t_local = (time.perf_counter() - t0) * NSUB / sample_subdomains
    ne = m.n_elem
    sub_mesh = PolyMesh(xy=m.xy, poly_ptr=m.poly_ptr[:sample_elems + 1], poly_vtx=m.poly_vtx)
    t0 = time.perf_counter()
    schwarz.prolongation(sub_mesh, g, agg[:sample_elems], P_DEG, P_C)
    t_r0t = (time.perf_counter() - t0) * ne / sample_elems
    t0 = time.perf_counter()
    A0 = (R0T.T @ (A @ R0T)).toarray()
    A0 = 0.5 * (A0 + A0.T)
    L0 = np.linalg.cholesky(A0)
    t_a0 = time.perf_counter() - t0
    # the iterations reuse the sampled factors cyclically: same sizes, so the same cost per apply
    S = schwarz.Schwarz(local_dofs=dofs, local_chol=[chol[i % len(chol)] for i in range(NSUB)], R0T=R0T, A0=A0,
                        A0_chol=L0)
    t0 = time.perf_counter()
    pcg.pcg(A, b, S.apply, fixed_iters=sample_iters)
    t_iter = (time.perf_counter() - t0) / sample_iters
    t_setup = t_local + t_r0t + t_a0
    t_solve = t_iter * iters
    return {"setup_s": t_setup, "solve_s": t_solve, "seconds_per_solve": t_setup + t_solve,
            "measured": f"A_0 product and Cholesky in full; {sample_subdomains}/{NSUB} subdomain Cholesky "
                        f"factorisations, {sample_elems}/{ne} elements of the prolongation, {sample_iters} PCG "
                        f"iterations",
            "extrapolated": f"subdomain factorisations x{NSUB / sample_subdomains:g}, prolongation "
                            f"x{ne / sample_elems:g}, PCG iterations x{iters / sample_iters:g} to the oracle's own "
                            f"{iters} iterations; SIPG assembly untimed"}


def cpu_worker(args):
    """Runs oracle_sample on a pickled preparation (bench.py --cpu-worker FILE) and prints its JSON; started
    as a fresh process so that the BLAS thread count set in its environment holds from the first import."""
    import pickle
    with open(args.cpu_worker, "rb") as f:
        prep, iters = pickle.load(f)
    print(json.dumps(oracle_sample(prep, iters)), flush=True)


def cpu_baseline(m, rho):
    """The oracle on this host at all cores (BLAS default) and at one thread, setup and solve separately."""
    import pickle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    iters = oracle_iters()
    prep = oracle_prep(m, rho)
    allc = oracle_sample(prep, iters)
    one = None
    with tempfile.NamedTemporaryFile(suffix=".pkl", delete=False) as f:
        pickle.dump((prep, iters), f)
        path = f.name
    try:
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", path], env=env,
                           capture_output=True, text=True, timeout=900)
        for line in r.stdout.splitlines():
            if line.startswith("{"):
                one = json.loads(line)
    finally:
        os.unlink(path)
    out = {"value": 1.0 / allc["seconds_per_solve"], "unit": "solves/s", "cores": cores, "kind": "oracle",
           "sample": ("numpy/scipy FP64 oracle on this workload, one solve (setup + solve) extrapolated from a sample: "
                      + allc["measured"] + " measured; " + allc["extrapolated"] + "; BLAS threads = all cores"),
           "setup_s": allc["setup_s"], "solve_s": allc["solve_s"], "oracle_iters": iters}
    if one:
        out["one_thread"] = {"value": 1.0 / one["seconds_per_solve"], "setup_s": one["setup_s"],
                             "solve_s": one["solve_s"], "cores": 1}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    from synth.coeff import checker_per_subdomain
    from synth.voronoi import voronoi_mesh
    from oracle import partition
    from oracle.geometry import build_geometry
    m = voronoi_mesh(N_ELEM, SEED)
    g = build_geometry(m)
    sub = partition.subdomains(g.centroid, NSUB)
    rho = checker_per_subdomain(m, sub, CONTRAST)
    prep = oracle_prep(m, rho)
    iters = oracle_iters()
    vals = []
    last = None
    for step in range(args.warmup + args.steps):
        last = oracle_sample(prep, iters, sample_subdomains=2, sample_elems=256, sample_iters=1)
        if step >= args.warmup:
            vals.append(last["seconds_per_solve"])
    t = statistics.mean(vals)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = ("numpy/scipy FP64 oracle, one solve per step extrapolated from a sample: " + last["measured"] +
              " measured; " + last["extrapolated"] + "; BLAS threads = all cores")
    out = {"impl": "reference", "metric": METRIC, "value": 1.0 / t, "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": "fp64 (plain FP64 ASPCG)", "parallelism": f"replicas x{world}",
                      "solver": "CPU oracle (numpy/scipy FP64)"},
           "cpu_baseline": {"value": 1.0 / t, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample,
                            "setup_s": last["setup_s"], "solve_s": last["solve_s"], "oracle_iters": iters},
           "e2e": {"value": 1.0 / t, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _systems(specs, meshes, dg, torch, rhs_seed_offset=1):
    """Systems of a problem mix: one coefficient per subdomain, log-uniform in [1, 1e3]; N(0,1) rhs."""
    from synth.coeff import loguniform_per_subdomain
    out = []
    for s, m in zip(specs, meshes):
        sub, _ = dg.Mesh.from_polymesh(m, np.ones(m.n_elem)).partition(s["nsub"], 0)
        rho = loguniform_per_subdomain(sub, np.random.default_rng(s["coef_seed"]))
        S = dg.System(dg.Mesh.from_polymesh(m, rho), s["p"], 10.0)
        b = torch.tensor(np.random.default_rng(s["coef_seed"] + rhs_seed_offset).standard_normal(S.ndof),
                         dtype=torch.float64, device="cuda")
        out.append((s, S, b))
    return out


def batch_measure(steps, warmup):
    """48 independent problems (element counts log-uniform in 1024..16384, p in 1..4, N/256 subdomains,
    N/64 agglomerates at p_c=1): setup of all 48 preconditioners at once (dgasm_setup_batch) and one batched
    solve of all of them (FP64 outer PCG; per iteration one launch per kernel kind for the whole batch, replayed
    from CUDA graphs), with
    FP32 / BF16 / FP64 local factors, against the plain FP64 library mode, one
    problem at a time (setup + solve each)."""
    from synth.workloads import build_meshes, problem_specs
    specs = problem_specs(48, 4)
    meshes = build_meshes(specs)
    import torch
    from paper_1903_11357_gb300 import dgasm as dg
    stream = torch.cuda.current_stream()
    probs = _systems(specs, meshes, dg, torch)
    nrhs = len(probs)

    def batched(precision):
        # all 48 set up at once (dgasm_setup_batch: host plans on the worker threads, device work on per-problem
        # streams), then one batched solve
        precs = dg.setup_batch([dict(system=S, nsub=s["nsub"], ncoarse=s["ncoarse"], p_c=1, precision=precision)
                                for s, S, _ in probs])
        xs = [torch.zeros_like(b) for _, _, b in probs]
        rc, sts = dg.solve_batch(precs, [b for _, _, b in probs], xs, rtol=1e-8, stream=stream)
        assert rc == 0, rc
        return precs, xs, sts

    def plain():
        xs, sts = [], []
        for s, S, b in probs:
            P = dg.Prec(S, s["nsub"], s["ncoarse"], 1, precision="fp64", stream=stream)
            x = torch.zeros_like(b)
            rc, st = P.solve(b, x, rtol=1e-8, stream=stream)
            assert rc == 0, rc
            xs.append(x)
            sts.append(st[0])
        return xs, sts

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = None
        e0.record(stream)
        for _ in range(steps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0 / steps, out

    t_mix, (precs_mix, x_mix, st_mix) = timed(lambda: batched("fp32"), steps, warmup)
    variants = {}
    for P in precs_mix:
        v = P.local_variant()
        variants[v] = variants.get(v, 0) + 1
    t_bf, (_, x_bf, st_bf) = timed(lambda: batched("bf16"), steps, 1)
    t_b64, (_, x_b64, st_b64) = timed(lambda: batched("fp64"), steps, 1)
    t_plain, (x_64, st_64) = timed(plain, steps, 1)
    rel = lambda xa: max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(xa, x_64))
    it = lambda sts: [int(s["iters"]) for s in sts]
    return {
        "problems": nrhs, "total_dofs": int(sum(S.ndof for _, S, _ in probs)),
        "fp32_batched": {"solves_per_s": nrhs / t_mix, "ms_per_step": 1000.0 * t_mix,
                         "max_rel_diff_vs_fp64": rel(x_mix), "iters_sum": sum(it(st_mix)),
                         "max_true_relres": max(float(s["true_relres"]) for s in st_mix)},
        "bf16_batched": {"solves_per_s": nrhs / t_bf, "ms_per_step": 1000.0 * t_bf,
                         "max_rel_diff_vs_fp64": rel(x_bf), "iters_sum": sum(it(st_bf)),
                         "max_true_relres": max(float(s["true_relres"]) for s in st_bf)},
        "fp64_batched": {"solves_per_s": nrhs / t_b64, "ms_per_step": 1000.0 * t_b64, "iters_sum": sum(it(st_b64))},
        "fp64_plain": {"solves_per_s": nrhs / t_plain, "ms_per_step": 1000.0 * t_plain, "iters_sum": sum(it(st_64)),
                       "what": "FP64 local factors, one problem at a time (setup + solve each)"},
        "speedup_mixed_batched_vs_fp64_plain": t_plain / t_mix,
        "local_variant_counts_fp32": variants,
        "iters_fp32_minus_fp64_max": max(a - c for a, c in zip(it(st_mix), it(st_64))),
    }


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    r = batch_measure(args.steps, args.warmup)
    clocks = sampler.stop()
    t_mix = r["fp32_batched"]["ms_per_step"] / 1000.0
    out = {
        "metric": METRIC, "value": r["problems"] / t_mix, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_mix, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 outer / f32 local", "data": "synthetic",
        "config": {"workload": "batch of 48 problems: Voronoi meshes (rng 4) with 1024..16384 cells log-uniform, "
                               "p in {1..4}, N/256 RCB subdomains, N/64 agglomerates at p_c=1, rho per subdomain "
                               "log-uniform in [1,1e3], rhs N(0,1) per dof, rtol 1e-8",
                   "total_dofs": r["total_dofs"], "step": "setup of 48 preconditioners + one batched solve of all 48"},
        "batch": r, "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


def serve_measure(n_req, fracs):
    """Poisson arrivals of solve requests (problem drawn from a pool of 16 problems shaped like the batch
    mix, 1..8 N(0,1) right-hand sides each) into the continuous-batching server; latency from arrival to
    completion, p50 / p99, and right-hand sides completed per second.  Per precision (FP32 local factors,
    and plain FP64): the saturation rate (all requests at once), then Poisson arrivals at each fraction
    of it; fracs: {precision: [fractions]}."""
    from synth.workloads import build_meshes, problem_specs
    specs = problem_specs(16, 5)
    meshes = build_meshes(specs)
    import torch
    from paper_1903_11357_gb300 import dgasm as dg
    pool = _systems(specs, meshes, dg, torch)
    rng = np.random.default_rng(5)

    def make_request():
        s, S, _ = pool[int(rng.integers(len(pool)))]
        k = int(rng.integers(1, 9))
        b = torch.tensor(rng.standard_normal((k, S.ndof)), dtype=torch.float64, device="cuda")
        return s, S, b, k

    def run(precision, arrivals):
        srv = dg.Server(hbm_budget=96 << 30, max_slots=24)
        reqs = [make_request() for _ in arrivals]
        t0 = time.perf_counter()
        pending, lat, rhs_done = {}, [], 0
        failed = {}   # return code -> requests that ended with it (reported, not dropped silently)
        i = 0
        t_last = t0
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and arrivals[i] <= now:
                s, S, b, k = reqs[i]
                x = torch.zeros_like(b)
                t = srv.submit(S, s["nsub"], s["ncoarse"], 1, b if k > 1 else b[0], x if k > 1 else x[0],
                               precision=precision)
                pending[t] = (arrivals[i], k, x)
                i += 1
            for t in list(pending):
                rc, st = srv.poll(t)
                if rc == 1:
                    continue
                a, k, _ = pending.pop(t)
                if rc != 0:
                    failed[str(rc)] = failed.get(str(rc), 0) + 1
                    continue
                t_done = time.perf_counter() - t0
                lat.append(t_done - a)
                rhs_done += k
                t_last = t_done
            time.sleep(0.0005)
        stats = srv.stats()
        srv.close()
        lat.sort()
        out = {"requests": len(lat), "rhs": rhs_done, "rhs_per_s": rhs_done / max(t_last - arrivals[0], 1e-9),
               "rounds": stats["rounds"], "stalls": stats["stalls"]}
        if lat:
            out.update(p50_ms=1000 * lat[len(lat) // 2], p99_ms=1000 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       mean_ms=1000 * sum(lat) / len(lat))
        if failed:
            out["failed_requests_by_code"] = failed
        return out

    res = {}
    for precision, fr in fracs.items():
        run(precision, [0.0] * 4)   # warm-up
        sat = run(precision, [0.0] * n_req)   # everything at once: saturation throughput
        rows = {"saturation_closed_batch": sat}
        for frac in fr:
            lam = frac * sat["rhs_per_s"] / 4.5   # requests/s: 4.5 right-hand sides per request on average
            gaps = np.random.default_rng(int(frac * 100)).exponential(1.0 / lam, size=n_req)
            arrivals = list(np.cumsum(gaps) - gaps[0])
            rows[f"poisson_{frac:.2f}x_saturation"] = dict(run(precision, arrivals), rate_req_per_s=lam)
        res[precision] = rows
    return res


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    n_req = max(16, args.requests)
    sampler = ClockSampler(0)
    res = serve_measure(n_req, {"fp32": (0.5, 0.9), "fp64": (0.5, 0.9)})
    clocks = sampler.stop()
    mixed = res["fp32"]["poisson_0.90x_saturation"]
    out = {
        "metric": METRIC, "value": res["fp32"]["saturation_closed_batch"]["rhs_per_s"], "unit": "solves/s",
        "n_gpus": 1, "steps": n_req, "warmup": 4, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 outer / f32 local (fp64 row: all f64)", "data": "synthetic",
        "config": {"workload": "serving: pool of 16 problems (rng 5) shaped like the batch mix, 1..8 N(0,1) rhs per "
                               "request, Poisson arrivals at 0.5x and 0.9x the saturation rate, budget 96 GiB, 24 slots",
                   "requests_per_rate": n_req},
        "p50_ms_mixed_0.9x": mixed["p50_ms"], "p99_ms_mixed_0.9x": mixed["p99_ms"],
        "saturation_speedup_mixed_vs_fp64": res["fp32"]["saturation_closed_batch"]["rhs_per_s"] /
                                            res["fp64"]["saturation_closed_batch"]["rhs_per_s"],
        "results": res, "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


SWEEP_FIXTURE = {1.0: "p4_c1", 1e2: "p4_c1e2", 1e4: "p4_c1e4", 1e6: "p4_c1e6"}


def sweep_measure(contrasts=(1.0, 1e2, 1e4, 1e6), precisions=("fp64", "fp32", "tf32", "bf16"), timed_reps=2):
    """Precision / contrast sweep: the 16384-cell mesh at p = 4 (245760 dofs, 64 subdomains, 256
    agglomerates), checkerboard contrast 1, 1e2, 1e4, 1e6; local factors in FP64, FP32, TF32, BF16 (FP64
    outer PCG, residual and coarse solve).  Per case: iterations, true relative residual, time to 1e-8
    (setup + solve; the last of timed_reps solves), relative difference to the library's FP64 solution, and,
    where the oracle's converged FP64 solve of the case is stored (tests/golden, written by a script that calls
    only the oracle), the oracle's iteration count and the error against the oracle's solution at its 1000
    sampled dofs (max |x - x_oracle| / max |x_oracle|)."""
    from synth.coeff import checker_per_subdomain
    from synth.voronoi import voronoi_mesh
    import torch
    from paper_1903_11357_gb300 import dgasm as dg
    from tests.golden.make_oracle_solutions import load as load_oracle_solve, path_of
    stream = torch.cuda.current_stream()
    m = voronoi_mesh(N_ELEM, SEED)
    sub, _ = dg.Mesh.from_polymesh(m, np.ones(m.n_elem)).partition(NSUB, 0)
    rows = []
    for contrast in contrasts:
        S = dg.System(dg.Mesh.from_polymesh(m, checker_per_subdomain(m, sub, contrast)), 4, 10.0, f=f_sin,
                      device=True, stream=stream)
        b = torch.tensor(S.rhs(), dtype=torch.float64, device="cuda")
        fx = SWEEP_FIXTURE.get(contrast)
        oref = load_oracle_solve(fx) if fx and os.path.exists(path_of(fx)) else None
        ref = None
        for precision in precisions:
            for _ in range(timed_reps):   # the last solve is timed
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                P = dg.Prec(S, NSUB, NCOARSE, P_C, precision=precision, stream=stream)
                x = torch.zeros_like(b)
                rc, st = P.solve(b, x, rtol=1e-8, maxit=20000, stream=stream)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                del P
            if precision == "fp64":
                ref = x.clone()
            row = {"contrast": contrast, "precision": precision, "rc": rc, "iters": st[0]["iters"],
                   "true_relres": st[0]["true_relres"], "kappa": st[0]["kappa"], "ms": 1000 * dt,
                   "rel_diff_vs_fp64": float(torch.linalg.norm(x - ref) / torch.linalg.norm(ref)) if ref is not None
                   else None}
            if oref is not None:
                xs = x[torch.tensor(oref["idx"], device="cuda")].cpu().numpy()
                row["oracle_iters"] = int(oref["iters"])
                row["err_vs_oracle_sampled"] = float(np.abs(xs - oref["x"]).max() / np.abs(oref["x"]).max())
            rows.append(row)
    return rows


def run_sweep(args):
    import torch
    torch.cuda.set_device(0)
    rows = sweep_measure()
    t = {r["precision"]: r["ms"] for r in rows if r["contrast"] == 1e4}
    out = {"metric": METRIC, "value": 1000.0 / t["fp32"], "unit": "solves/s", "n_gpus": 1, "steps": 1,
           "warmup": 1, "ms_per_step": t["fp32"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 outer / local per row", "data": "synthetic",
           "config": {"workload": "precision sweep: 16384-cell mesh (seed 2), p=4 (245760 dofs), 64 subdomains, "
                                  "256 agglomerates p_c=1, checkerboard contrast 1..1e6; value = FP32-local "
                                  "solves/s at contrast 1e4"},
           "rows": rows}
    print(json.dumps(out), flush=True)


# Sec. 7, Example 4 (independent Voronoi grids, rho = 1): K(P_ad) (iterations) for p = q, by fine element
# count N_h (columns) and coarse element count N_H (rows).  Context only: the paper's meshes are not published.
def paper_table(example, p):
    """The paper's printed K(P_ad) and iteration counts (Sec. 7, Example 2: nested grids, Example 4: non-nested
    grids; p = q), from the cited fixtures in tests/golden: {(N_h, N_H): (K, iterations)}."""
    out = {}
    path = os.path.join(ROOT, "tests", "golden", f"paper_example{example}_p{p}.txt")
    if not os.path.exists(path):
        return out
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            nh, nH, K, it = line.split()
            out[(int(nh), int(nH))] = (float(K), int(it))
    return out


def run_paper(args):
    """The paper's experimental setting on the GPU (Sec. 7): subdomains = fine elements (element-block
    local solves), q = p, rho = 1, C_sigma = 10, rtol 1e-8 from x0 = 0 with an N(0,1) right-hand side; K(P_ad)
    from the Lanczos estimate.  Fine meshes of 256 .. 16384 cells; coarse spaces of 16 .. 1024 cells
    (n_0 <= 3072) of two kinds: RCB agglomerates of the fine mesh (nested) and an independently generated
    Voronoi mesh (non-nested, Example 4's setting, seed 7); p = q = 1 and 3.  The paper's numbers (its own
    meshes and machine) are attached as context: Example 2 to the nested rows, Example 4 to the non-nested ones."""
    from synth.voronoi import voronoi_mesh
    import torch
    from paper_1903_11357_gb300 import dgasm as dg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    rows = []
    t_ref = None
    coarse_meshes = {}
    for nh in (256, 1024, 4096, 16384):
        m = voronoi_mesh(nh, 1)
        M = dg.Mesh.from_polymesh(m, np.ones(nh))
        for p in (1, 3):
            S = dg.System(M, p, 10.0)
            b = torch.tensor(np.random.default_rng(0).standard_normal(S.ndof), dtype=torch.float64, device="cuda")
            for nH in (16, 64, 256, 1024):
                # the coarse solve keeps A_0^{-1} dense: n_0 = N_H (q+1)(q+2)/2 up to 3072
                if nH >= nh or nH * (p + 1) * (p + 2) // 2 > 3072:
                    continue
                for kind in ("nested", "non-nested"):
                    cm = None
                    if kind == "non-nested":
                        if nH not in coarse_meshes:
                            coarse_meshes[nH] = dg.Mesh.from_polymesh(voronoi_mesh(nH, 7), np.ones(nH))
                        cm = coarse_meshes[nH]
                    for rep in range(2):   # the second solve is timed
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        P = dg.Prec(S, nh, nH if cm is None else 0, p, stream=stream, coarse_mesh=cm)
                        x = torch.zeros_like(b)
                        rc, st = P.solve(b, x, rtol=1e-8, maxit=20000, stream=stream)
                        torch.cuda.synchronize()
                        dt = time.perf_counter() - t0
                    ctx = paper_table(4 if cm is not None else 2, p).get((nh, nH))
                    rows.append({"N_h": nh, "N_H": nH, "p": p, "coarse": kind, "rc": rc, "iters": st[0]["iters"],
                                 "kappa": st[0]["kappa"], "true_relres": st[0]["true_relres"], "ms": 1000 * dt,
                                 "paper_kappa_iters": ctx,
                                 "paper_table": ("Example 4 (non-nested)" if cm is not None else "Example 2 (nested)")
                                 if ctx else None})
                    if (nh, nH, p, kind) == (16384, 256, 3, "nested"):
                        t_ref = dt
                    del P
    out = {"metric": METRIC, "value": 1.0 / t_ref, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "ms_per_step": 1000 * t_ref, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "paper setting: subdomains = elements, nested (RCB agglomerates) and non-nested "
                                  "(independent Voronoi) coarse spaces, q = p, rho = 1; value = solves/s at "
                                  "N_h = 16384, N_H = 256, p = 3, nested"},
           "rows": rows}
    print(json.dumps(out), flush=True)


def slowest_rank_seconds(elapsed, world, device="cpu"):
    """Replicas: every rank solves its own copy of the workload; the job's time is the slowest rank's
    (max over ranks, the same on every rank), and the whole-job value is world * steps / that time."""
    if world <= 1:
        return float(elapsed)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def profiled_step(dg, step, barrier, precision):
    """One untimed step with every kernel kind bracketed by CUDA events: per-kind device time."""
    barrier()
    dg.profile_read(reset=True)
    dg.profile_enable(True)
    rc, _, P, x = step(precision)
    assert rc == 0, rc
    barrier()
    dg.profile_enable(False)
    prof = dg.profile_read(reset=True)
    del P, x
    return {k: {"total_ms": v[0], "launches": v[1], "avg_ms": v[0] / max(v[1], 1)} for k, v in prof.items() if v[1]}


def main():
    global N_ELEM, NSUB, NCOARSE, P_DEG, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dgasm", choices=["dgasm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline solve only: no precision sweep, batch or serving "
                                                         "sections, no CPU baseline")
    ap.add_argument("--elems", type=int, default=N_ELEM, help="smaller workloads for profiling runs")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "bf16"],
                    help="local-factor precision of the timed step (profiling runs; the headline is fp64)")
    ap.add_argument("--nsub", type=int, default=NSUB)
    ap.add_argument("--ncoarse", type=int, default=NCOARSE)
    ap.add_argument("--degree", type=int, default=P_DEG)
    ap.add_argument("--workload", default="cfg2", choices=["cfg2", "batch", "serve", "sweep", "paper"],
                    help="cfg2: the headline solve (default, with compact sweep / batch / serving sections); batch: "
                         "48-problem batch; serve: Poisson arrivals into the server; sweep: precision / contrast "
                         "sweep at p=4; paper: the paper's setting (subdomains = elements) over fine and coarse "
                         "mesh sizes")
    ap.add_argument("--requests", type=int, default=200, help="requests per arrival rate (serving)")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args)
        return
    if args.workload != "cfg2":
        {"batch": run_batch, "serve": run_serve, "sweep": run_sweep, "paper": run_paper}[args.workload](args)
        return
    if args.precision != "fp64":
        args.quick = True
    if (args.elems, args.nsub, args.ncoarse, args.degree) != (N_ELEM, NSUB, NCOARSE, P_DEG):
        N_ELEM, NSUB, NCOARSE, P_DEG = args.elems, args.nsub, args.ncoarse, args.degree
        WORKLOAD = (f"profiling case: {N_ELEM} Lloyd-Voronoi cells, p={P_DEG}, {NSUB} subdomains, {NCOARSE} "
                    f"agglomerates at p_c=1, checkerboard 1e4 (not the headline workload)")
        args.quick = True
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_1903_11357_gb300 import dgasm as dg

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    stream = torch.cuda.current_stream()
    m, rho, M, S = build_problem()
    b_host = S.rhs()
    b = torch.tensor(b_host, dtype=torch.float64, device="cuda")
    ndof = S.ndof
    # the matrix assembly (outside the timed step: the step starts from the assembled system), on the host
    # threads and on the device, second call of each timed
    asm = {}
    for dev_asm in (False, True):
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S_tmp = dg.System(M, P_DEG, 10.0, device=dev_asm, stream=stream)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            del S_tmp
        asm["device_ms" if dev_asm else "host_ms"] = 1000.0 * dt
    asm.update({"cells": N_ELEM, "p": P_DEG, "host_threads": os.cpu_count(), "what": "block matrix only (no load vector)"})

    def step(precision=args.precision, keep=None):
        P = dg.Prec(S, NSUB, NCOARSE, P_C, precision=precision, stream=stream)
        x = torch.zeros_like(b)
        rc, st = P.solve(b, x, rtol=1e-8, stream=stream)
        if keep is not None:
            keep.append((P, x))
        return rc, st[0], P, x

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        rc, st, P, x = step()
        assert rc == 0, rc
    del P, x
    # per-kernel breakdown: one untimed step with every kind bracketed by events
    breakdown = profiled_step(dg, step, barrier, args.precision)
    dom = max(breakdown, key=lambda k: breakdown[k]["total_ms"])
    # timed region: no instrumentation; every step's preconditioner is kept until the region ends
    keep = []
    sampler = ClockSampler(local_rank)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    per_step = []
    ev0.record(stream)
    for _ in range(args.steps):
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record(stream)
        rc, st, P, x = step(keep=keep)
        e_b.record(stream)
        per_step.append((e_a, e_b, st))
        assert rc == 0, rc
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    t_max = slowest_rank_seconds(elapsed, world, device="cuda")
    lat = sorted(a.elapsed_time(bq) for a, bq, _ in per_step)
    info = keep[0][0].info()
    sts = [s for _, _, s in per_step]
    iters = sts[-1]["iters"]
    launches = sum(P_.info()["setup_launches"] for P_, _ in keep) + sum(s["launches"] for s in sts)
    x_fp64 = keep[-1][1].clone()
    del keep
    # the dominant kernel's launch times, in a separate pass of the same steps with only that kind bracketed
    dg.profile_read(reset=True)
    dg.profile_enable(True, kinds=[dom])
    barrier()
    for _ in range(min(args.steps, 3)):
        rc, _, P, x = step()
        assert rc == 0, rc
    barrier()
    dg.profile_enable(False)
    prof = dg.profile_read(reset=True)
    del P, x

    # end to end through the C-ABI with host buffers (b copied in, x copied out inside the call), both in
    # pinned host memory allocated before the timed region
    b_pin = torch.from_numpy(b_host).pin_memory().numpy()
    x_pin = torch.zeros(ndof, dtype=torch.float64).pin_memory().numpy()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Pe = dg.Prec(S, NSUB, NCOARSE, P_C, precision=args.precision, stream=stream)
        rc, _ = Pe.solve(b_pin, x_pin, rtol=1e-8, stream=stream, host_buffers=True)
        assert rc == 0
        del Pe
    barrier()
    e2e_t = time.perf_counter() - t0

    def run_mixed(precision, label):
        """The same workload with lower-precision local factors (FP64 outer PCG, residual and coarse solve)."""
        barrier()
        mx = []
        for _ in range(args.warmup):
            step(precision)
        breakdown_m = profiled_step(dg, step, barrier, precision)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            rc, stm, Pm, xm = step(precision, keep=mx)
        e1.record(stream)
        barrier()
        tm = e0.elapsed_time(e1) / 1000.0
        err = float(torch.linalg.norm(xm - x_fp64) / torch.linalg.norm(x_fp64))
        return {"precision": label, "solves_per_s": args.steps / tm, "ms_per_step": 1000.0 * tm / args.steps,
                "iters": stm["iters"], "true_relres": stm["true_relres"], "rel_diff_vs_fp64": err,
                "speedup_vs_fp64": (args.steps / tm) / (args.steps / elapsed), "kernels_one_step": breakdown_m}

    def rhs_chunk_tuning():
        """Eight right-hand sides on a problem with few subdomains (4096 cells, p = 3, 16 subdomains): the
        local-solve work split into 1 or 4 right-hand sides per CTA pair, each timed, and the tuner's pick."""
        from synth.voronoi import voronoi_mesh
        mm = voronoi_mesh(4096, SEED)
        Sx = dg.System(dg.Mesh.from_polymesh(mm, np.ones(mm.n_elem)), P_DEG, 10.0)
        Px = dg.Prec(Sx, 16, 64, P_C, stream=stream)
        Bx = torch.tensor(np.random.default_rng(3).standard_normal((8, Sx.ndof)), dtype=torch.float64, device="cuda")
        res = {"case": "4096 cells, p=3, 16 subdomains, 64 agglomerates, 8 N(0,1) right-hand sides, FP64"}
        for kc in (4, 1):
            Px.set_rhs_chunk(8, kc)
            for rep in range(2):
                Xx = torch.zeros_like(Bx)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                Px.solve(Bx, Xx, rtol=1e-8, stream=stream)
                torch.cuda.synchronize()
                res[f"solve_ms_kc{kc}"] = 1000.0 * (time.perf_counter() - t0)
        Px.set_rhs_chunk(8, 0)
        Px.solve(Bx, torch.zeros_like(Bx), rtol=1e-8, stream=stream)
        res["tuned_kc"] = Px.rhs_chunk(8)
        return res

    def local_variant_tuning():
        """The small configuration (256 cells, p = 2, 4 subdomains of ~384 dofs, 16 agglomerates): local solves
        by the envelope sweeps and by explicit subdomain inverses, each timed (setup excluded, median of 5
        solves), and the tuner's pick."""
        from synth.voronoi import voronoi_mesh
        mm = voronoi_mesh(256, 1)
        Sx = dg.System(dg.Mesh.from_polymesh(mm, np.ones(mm.n_elem)), 2, 10.0, f=f_sin)
        bx = torch.tensor(Sx.rhs(), dtype=torch.float64, device="cuda")
        res = {"case": "256 cells (seed 1), p=2, 4 subdomains, 16 agglomerates at p_c=1, FP64, rtol 1e-8"}
        for variant in ("sweeps", "inverse"):
            Px = dg.Prec(Sx, 4, 16, P_C, stream=stream)
            Px.set_local_variant(variant)
            ts = []
            for _ in range(6):
                xx = torch.zeros_like(bx)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, stx = Px.solve(bx, xx, rtol=1e-8, stream=stream)
                torch.cuda.synchronize()
                ts.append(1000.0 * (time.perf_counter() - t0))
            res[f"solve_ms_{variant}"] = statistics.median(ts[1:])
            res[f"iters_{variant}"] = stx[0]["iters"]
        Px = dg.Prec(Sx, 4, 16, P_C, stream=stream)
        Px.solve(bx, torch.zeros_like(bx), rtol=1e-8, stream=stream)
        res["tuned"] = Px.local_variant()
        return res

    tuning = rhs_chunk_tuning() if rank == 0 else None
    variant_tuning = local_variant_tuning() if rank == 0 else None

    mixed = mixed_tf32 = mixed_bf16 = None
    if not args.no_mixed:
        mixed = run_mixed("fp32", "fp32 local factors, fp64 outer")
        mixed_tf32 = run_mixed("tf32", "fp32 local factors with tensor-core (split TF32) trailing updates, fp64 outer")
        mixed_bf16 = run_mixed("bf16", "bf16 local factor streams (fp32 factorisation and accumulation), fp64 outer")

    # the precision (p = 4), batching and serving configurations, compact (rank 0 only); a section that fails
    # is recorded in the line with its error instead of ending the run before the headline is printed
    def section(fn):
        t0 = time.perf_counter()
        try:
            out = fn()
        except Exception as e:
            out = {"error": f"{type(e).__name__}: {e}"}
        out["seconds"] = time.perf_counter() - t0
        return out

    def sweep_section():
        return {"workload": "16384-cell mesh (seed 2) at p=4 (245760 dofs), 64 subdomains, 256 agglomerates p_c=1, "
                            "checkerboard contrast 1..1e6, local factors per row, fp64 outer PCG; error against the "
                            "oracle's converged FP64 solve at 1000 sampled dofs",
                "rows": sweep_measure(timed_reps=2)}

    def batch_section():
        bm = batch_measure(1, 1)
        bm["workload"] = ("48 problems: Voronoi meshes (rng 4) with 1024..16384 cells log-uniform, p in {1..4}, N/256 "
                          "subdomains, N/64 agglomerates p_c=1, rho per subdomain log-uniform in [1,1e3], N(0,1) rhs; "
                          "step = setup of all 48 + one batched solve")
        return bm

    def serving_section():
        sv = serve_measure(args.requests, {"fp32": (0.5, 0.75, 0.9), "fp64": (0.9,)})
        return {"workload": f"pool of 16 problems (rng 5) shaped like the batch mix, 1..8 N(0,1) rhs per request, "
                            f"{args.requests} requests per rate: all at once (saturation), then Poisson arrivals at "
                            f"fractions of the saturation rate; budget 96 GiB, 24 slots",
                "fp32": sv["fp32"], "fp64": sv["fp64"],
                "saturation_speedup_mixed_vs_fp64": sv["fp32"]["saturation_closed_batch"]["rhs_per_s"] /
                                                    sv["fp64"]["saturation_closed_batch"]["rhs_per_s"]}

    extras = {}
    if rank == 0 and not args.quick:
        extras["precision_sweep"] = section(sweep_section)
        extras["batch"] = section(batch_section)
        extras["serving"] = section(serving_section)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = read_peaks()
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # FP64 peak: SMs x the measured FMA issue rate per SM and clock x 2 flop x the maximum SM clock
    nsm, fma_clk_sm, probe_tflops = dg.probe_fp64()
    fp64_peak = nsm * fma_clk_sm * 2 * sm_max * 1e6 / 1e12
    fp64_nominal = nsm * FP64_NOMINAL_FMA_PER_CLK_SM * 2 * sm_max * 1e6 / 1e12
    # roofline of the dominant kernel (largest device time in the breakdown step), its launches timed in a
    # separate pass of the same steps
    dom_ms, dom_n = prof[dom]
    avg_s = dom_ms / 1000.0 / max(dom_n, 1)
    tiles = info["stream_tiles"]
    if dom == "local":
        flops = 2 * tiles * 1024 * 1.0              # stream tiles of both sweeps, 2 flop per FMA, one rhs
        bytes_ = tiles * 1024 * 8 + ndof * 8 * 3
    elif dom == "chol_update":
        total_upd_flops = info["factor_flops"]
        flops = total_upd_flops / max(prof["chol_update"][1], 1)
        bytes_ = None
    elif dom == "spmv":
        npb = (P_DEG + 1) * (P_DEG + 2) // 2
        flops = 2 * info["nnzb"] * npb * npb
        bytes_ = info["nnzb"] * npb * npb * 8
    else:
        flops, bytes_ = None, None
    roof = {"kernel": dom, "bound": "alu", "achieved": (flops / avg_s / 1e12) if flops else None,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": (flops / avg_s / 1e12 / fp64_peak) if flops else None,
            "traffic": local_traffic(tiles) if dom == "local" else None, "avg_launch_ms": avg_s * 1e3, "launches": dom_n,
            "algorithmic_bytes_per_launch": bytes_, "algorithmic_flops_per_launch": flops,
            "peak_source": (f"FP64: {nsm} SMs x {fma_clk_sm:.3f} FMA/clk/SM (dgasm_probe_fp64, measured in this run) x 2 "
                            f"flop x max SM clock {sm_max:.0f} MHz; the probe itself ran at {probe_tflops:.3f} TFLOP/s"),
            "peak_nominal_2_fma_per_clk": fp64_nominal,
            "frac_vs_nominal": (flops / avg_s / 1e12 / fp64_nominal) if flops else None}
    if dom == "local" and args.precision != "fp64":
        # lower-precision local factors: the sweeps stream 1024 entries of 4 (FP32) or 2 (BF16) bytes per tile
        eb = 2 if args.precision == "bf16" else 4
        bytes_ = tiles * 1024 * eb + ndof * 8 * 3
        hbm = peaks.get("hbm_gbs", 6800.0)
        roof = {"kernel": dom, "bound": "hbm", "achieved": bytes_ / avg_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bytes_ / avg_s / 1e9 / hbm, "traffic": None, "avg_launch_ms": avg_s * 1e3, "launches": dom_n,
                "algorithmic_bytes_per_launch": bytes_, "algorithmic_flops_per_launch": 2 * tiles * 1024,
                "peak_source": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}

    out = {
        "metric": METRIC, "value": world * args.steps / t_max, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 (plain FP64 ASPCG)" if args.precision == "fp64" else
                   f"{args.precision} local factors, fp64 outer (profiling run)", "parallelism": f"replicas x{world}",
                   "l2": "working set > L2 (matrix 92 MB + local factors + Krylov vectors per step), no flush"},
        "time_to_1e8_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "mean": sum(lat) / len(lat)},
        "iters": iters, "true_relres": sts[-1]["true_relres"], "kappa_estimate": sts[-1]["kappa"],
        "setup": {"plan_ms": info["plan_ms"], "setup_ms": info["setup_ms"], "local_tiles": info["local_tiles"],
                  "stream_tiles": tiles, "factor_flops": info["factor_flops"]},
        "gpu_launches": int(launches),
        "assembly": asm,
        "rhs_chunk_tuning": tuning,
        "local_variant_tuning": variant_tuning,
        "kernels_one_step": breakdown,
        "roofline": roof,
        "e2e": {"value": world * args.steps / e2e_t, "unit": "solves/s", "h2d_bytes_per_step": ndof * 8,
                "d2h_bytes_per_step": ndof * 8, "host_memory": "pinned"},
        "mixed_fp32": mixed,
        "mixed_tf32": mixed_tf32,
        "mixed_bf16": mixed_bf16,
        "clocks": clocks,
    }
    out.update(extras)
    if world == 1 and not args.no_cpu_baseline and not args.quick:
        out["cpu_baseline"] = cpu_baseline(m, rho)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

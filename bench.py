#!/usr/bin/env python
"""Benchmark of the pruning + domain-selection hot path on GB300.

One bench step is one full solve through the C ABI on a synthetic instance
shaped like the paper's workloads: pruning, B restarts x T steps of the fused
domain-selection step (Sec. III-B), best-of-restarts, reconstruction and the
energy of the result on the full instance.

Default workload (the largest single-GPU configuration): dense SK N = 4096,
J_ij ~ N(0, 1/N) FP32, h_i ~ N(0, 0.1), 4096 restarts x 5000 steps, lr 6.0,
on the tensor cores with J as two FP16 planes (FP32-level products, FP32
accumulate). The same JSON line also carries the other bench workloads
(ER N = 2000 max-cut, 2D torus N = 20 000, ER N = 100 000 with pendant trees)
with their own throughput and roofline figures.

Prints one JSON line (metric: relaxed spin-updates/s = N_reduced * B * T per
second of device time). ``--impl reference`` times the FP64 CPU oracle on the
same workload instead (bounded samples of the same solve).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the serving leg runs up to 32 requests' streams at once: give the CUDA
# context as many hardware work queues (read when the context is created,
# so before torch touches the GPU); it changes nothing else
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "relaxed spin-updates/s"
UNIT = "spin-updates/s"
WORKLOADS = {
    # name: (instance, restarts, steps)
    "er2000": ("er2000", 1024, 2000),
    "er800": ("er800", 1024, 2000),
    "sk100": ("sk100", 64, 1000),
    "sk4096": ("sk4096", 4096, 5000),
    "torus20k": ("torus20k", 512, 3000),
    "er100k_pendant": ("er100k_pendant", 512, 3000),
    # complete 1000-spin graphs of the solver comparison (Sec. IV-C)
    "table2_uniform": ("table2_uniform", 1024, 1000),
    "table2_gaussian": ("table2_gaussian", 1024, 1000),
}
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sk4096", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--lr", type=float, default=6.0)
    ap.add_argument("--mu", type=float, default=0.0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bounded oracle sample per CPU-baseline timing")
    ap.add_argument("--cpu-leg", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--secondary", default="er2000,torus20k,er100k_pendant",
                    help="other workloads measured into the same line ('' for none)")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="solves timed end to end with host buffers (at most --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the time-to-target and serving legs")
    ap.add_argument("--profile-steps", type=int, default=200)
    return ap.parse_args()


# ----------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- helpers

def device_instance(inst, torch):
    import dataclasses
    def t(x):
        return None if x is None else torch.from_numpy(x).cuda()
    return dataclasses.replace(inst, J=t(inst.J), indptr=t(inst.indptr),
                               indices=t(inst.indices), data=t(inst.data), h=t(inst.h))


def pinned_instance(inst, torch):
    import dataclasses
    def p(x):
        if x is None:
            return None
        return torch.from_numpy(x).pin_memory().numpy()
    return dataclasses.replace(inst, J=p(inst.J), indptr=p(inst.indptr),
                               indices=p(inst.indices), data=p(inst.data), h=p(inst.h))


def input_bytes(inst) -> int:
    arrs = [inst.J, inst.indptr, inst.indices, inst.data, inst.h]
    return int(sum(a.nbytes for a in arrs if a is not None))


def peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


def traffic_for(kernel: str, src_file: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on this workload and on the current source of the kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(kernel)
    if not d or d.get("workload") != workload:
        return None
    h = hashlib.sha256(open(os.path.join(ROOT, src_file), "rb").read()).hexdigest()[:16]
    return d["bytes_per_launch"] if d.get("source_sha") == h else None


def launches_per_solve(T: int, rounds: int, path: int, resident: bool, rowsum: bool,
                       rowscale: bool) -> int:
    """Kernels of one solve, as the ncu launch list of a solve shows them:
    instance checks (couplings twice, field once), pruning (dense->CSR 2,
    init 1, 7 per round incl. the final empty one, sum + reduced J + reduced
    field 3), session set-up (fills 2, init 1, operand 1, plus the row-sum
    bound when the tensor-core path accumulates integer energies: `rowsum`,
    plus the per-row scales of row-scaled operands: `rowscale`), the steps
    (one launch when resident; on the streaming tensor-core path one launch
    per step, each also tracking its predecessor, plus one tracking launch
    for the last step; else step + track per step, plus the copy of improved
    bit-packed spins on the sparse path), finish (energy-only step + track
    (+ copy) + argmin), reconstruction (1), full-instance energy (2)."""
    per_step = 3 if path == 2 else 2
    if resident:
        steps = 1
    elif path == 1:
        steps = T + 1
    else:
        steps = per_step * T
    setup = 4 + (1 if rowsum else 0) + (1 if rowscale else 0)
    return 3 + 3 + 7 * (rounds + 1) + 3 + setup + steps + per_step + 1 + 1 + 2


# ----------------------------------------------------------------- reference arm

def over_ranks(dist, x: float, op: str, device) -> float:
    """The max or the sum of a per-rank number over all ranks (the number
    itself without a process group); `device` is where the collective's
    tensor lives ("cuda" for NCCL, "cpu" for gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def reference_sample_steps(name: str) -> int:
    """Domain-selection steps per bounded oracle sample: one on the N = 4096
    dense workload (two FP64 products of 4096 x 4096 by 4096 x 4096 per
    sample with the final evaluation), three elsewhere."""
    return 1 if name == "sk4096" else 3


def host_info() -> dict:
    import platform
    return {"uname_m": platform.machine(), "nproc": os.cpu_count()}


def run_reference(a, rank, world):
    """The FP64 CPU oracle on the same workload: each step is one bounded
    sample of the solve (pruning, `sample` domain-selection steps over all
    restarts, reconstruction, final energy)."""
    if rank != 0:
        return
    import numpy as np
    import synth
    from oracle import domain_selection as ods
    from oracle import ising, pruning
    name, B, T = WORKLOADS[a.workload]
    inst = synth.workload(name, 0)
    sample = reference_sample_steps(name)

    def one():
        res = pruning.prune(inst)
        red = res.reduced
        r = ods.select_domain(red, ods.Params(restarts=B, steps=sample, lr=a.lr, mu=a.mu, seed=0))
        full = pruning.reconstruct(res, r["best_spins"])
        ising.energy(inst, full.astype(np.float64))
        return red.n * B * sample

    for _ in range(a.warmup):
        one()
    t0 = time.perf_counter()
    units = 0
    for _ in range(a.steps):
        units += one()
    dt = time.perf_counter() - t0
    value = units / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * dt / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{a.workload}: N={inst.n}, restarts={B}, steps={T}",
                       "sample_steps_per_bench_step": sample, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per bench step: prune + {sample} of {T} steps x {B} "
                                       "restarts (+ the final evaluation) + reconstruct + "
                                       "energy, numpy FP64, BLAS threads = all host cores",
                             **host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- CPU baseline

def cpu_leg(a):
    """Child process of the CPU baseline (BLAS threads fixed by its
    environment before numpy loads): the oracle's domain-selection step on
    the workload's instance, repeated for about `cpu_seconds`; prints one
    JSON object."""
    import numpy as np
    import synth
    from oracle import domain_selection as ods
    from oracle import ising, rng
    name, B, T = WORKLOADS[a.workload]
    inst = synth.workload(name, 0)
    cq, ch = ising.coefficients(inst.j_scale, inst.convention)
    J = ising.coupling_matrix(inst)
    h = ising.field(inst)
    p = ods.Params(restarts=B, steps=1 << 30, lr=a.lr, mu=a.mu, seed=0)
    th = rng.theta_init(0, B, inst.n)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t0 = time.perf_counter()
    steps = 0
    while True:
        r = ods.step(J, h, cq, ch, p, th, m, v, steps + 1)
        th, m, v = r.theta, r.m, r.v
        steps += 1
        if time.perf_counter() - t0 >= a.cpu_seconds:
            break
    dt = time.perf_counter() - t0
    print(json.dumps({"n": inst.n, "steps": steps, "seconds": dt,
                      "value": inst.n * B * steps / dt}), flush=True)


def cpu_baseline(a, B, T):
    """The oracle timed on the host cores twice, single-threaded and with
    BLAS on every core, each in a fresh interpreter (numpy fixes its thread
    count when it loads): relaxed spin-updates/s of its domain-selection
    step on the same instance, over a bounded sample (about `cpu_seconds`
    each); the full run's time is this rate extrapolated to N B T."""
    out = {}
    ncores = os.cpu_count() or 1
    for label, threads in [("single_thread", 1), ("all_cores", ncores)]:
        env = dict(os.environ)
        for k in ["OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"]:
            env[k] = str(threads)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", "1",
                            "--workload", a.workload, "--cpu-seconds", str(a.cpu_seconds),
                            "--lr", str(a.lr), "--mu", str(a.mu)],
                           env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            out[label] = {"error": r.stderr[-400:]}
            continue
        d = json.loads(r.stdout.strip().splitlines()[-1])
        d["threads"] = threads
        d["extrapolated_full_run_s"] = d["n"] * B * T / d["value"]
        out[label] = d
    best = out.get("all_cores", {})
    return {"value": best.get("value"), "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": f"{best.get('steps')} domain-selection steps x {B} restarts on the same "
                      f"instance (numpy FP64, BLAS threads = {ncores}, "
                      f"{best.get('seconds', 0):.1f} s); the full run "
                      f"({T} steps) extrapolated from it",
            **host_info(), "single_thread": out.get("single_thread"), "all_cores": best}


# ----------------------------------------------------------------- time to target

def run_checked(ctx, dinst, integer, B, T, seed, prec, chunk):
    """One session of T steps in chunks of `chunk` steps, the best so far
    taken after each chunk as the session reports it (ising_ds_result: exact
    for integer couplings, otherwise the near-best restarts re-evaluated in
    FP64). Returns [(cumulative wall ms of steps + checks, best)], the
    result."""
    import torch
    from paper_2312_05837_gb300 import api
    s = api.Session(ctx, dinst, restarts=B, steps=T, seed=seed, precision=prec)
    torch.cuda.synchronize()
    done, ms, h = 0, 0.0, []
    while done < T:
        k = min(chunk, T - done)
        w0 = time.perf_counter()
        s.run(k)
        done += k
        best = float(s.result()["best_energy"])
        ms += 1e3 * (time.perf_counter() - w0)
        h.append((ms, best))
    s.finish()
    res = s.result()
    s.close()
    return h, res


def precision_runs(ctx, dinst, integer, n, B, T, seed, forms, chunk):
    """Each operand form runs the same instance and seed for T steps (chunks
    of `chunk` steps, the exact best after each): spin-updates/s from the
    device time of the steps, the final exact best, its gap to the plain
    FP32 form's, and the plain form's history (its time to its own final
    best is the time-to-target reference)."""
    out, hist = {}, {}
    # first uses of a kernel (ours and torch's reductions) load it
    for prec in forms:
        run_checked(ctx, dinst, integer, B, 2, seed, prec, 2)
    for prec in forms:
        h, res = run_checked(ctx, dinst, integer, B, T, seed, prec, chunk)
        hist[prec] = h
        out[prec] = {"value": n * B * T / (res["device_ms"] / 1e3), "device_ms": res["device_ms"],
                     "best_energy": res["best_energy"], "operand_planes": res["operand_planes"]}
    ref = out["fp32"]["best_energy"]
    for prec in forms:
        out[prec]["gap_vs_fp32"] = (out[prec]["best_energy"] - ref) / abs(ref)
    return out, hist["fp32"]


def served_time_to_target(ctx, inst, B, T, seed, target, prec, chunk, batch, budget_s, pack,
                          max_rounds=1000):
    """Wall time from the first submission of (B restarts, T steps) requests
    to the server until one of them returns a result at or below `target`
    (ising_server_submit_target: the full-instance energy of the request's
    best spins is evaluated exactly after every chunk of `chunk` steps, and
    the request finishes as soon as it meets the target). `batch` requests
    with different seeds (the first `seed`) are submitted together and run
    side by side (packed when `pack`); once one meets the target the others
    are cancelled. Further batches (fresh seeds) follow until the target is
    met, `budget_s` has passed or `max_rounds` batches have run. The timed
    region holds everything a client waits for: the instance copies at
    submission, upload, pruning, set-up, steps, checks, finishing."""
    from paper_2312_05837_gb300 import api
    srv = api.Server(ctx, budget_bytes=120 << 30, max_active=max(batch, 1), chunk_steps=chunk,
                     pack=pack)
    t0 = time.perf_counter()
    hit, rounds, steps = None, 0, None
    while hit is None and rounds < max_rounds and time.perf_counter() - t0 < budget_s:
        seeds = [seed + k if rounds == 0 else seed + 1000 * rounds + k for k in range(batch)]
        pending = [srv.submit(inst, restarts=B, steps=T, seed=sd, precision=prec, target=target)
                   for sd in seeds]
        while pending:
            for rid in list(pending):
                r = srv.poll(rid)
                if not r["done"]:
                    continue
                pending.remove(rid)
                if r["status"] != 0:
                    srv.close()
                    raise RuntimeError(f"time to target: request failed: {r['error']}")
                if r["reached"] and hit is None:
                    hit = time.perf_counter() - t0
                    steps = r["steps_done"]
                    for other in pending:
                        srv.cancel(other)
            time.sleep(2e-4)
        rounds += 1
    srv.close()
    return {"time_ms": 1e3 * hit if hit is not None else None, "rounds": rounds, "batch": batch,
            "steps_to_target": steps}


def time_to_target(ctx, inst, integer, B, T, seed, plain_hist, fast_forms, chunk, budget_s=20.0):
    """Time to the plain FP32 form's best energy E* (its final best over the
    configuration's run with seed `seed`), measured on the served form
    against the plain form served the same way (served_time_to_target):
    (1) within the tolerance the reduced-precision forms are held to, E* +
    0.005 |E*| (one request each, seed `seed`); (2) E* itself. The plain
    form reaches E* in its own run by construction; the served mixed-
    precision forms follow other trajectories (other operand roundings), so
    for (2) they submit batches of 4 seeds at once until one meets it. With
    integer couplings the exact fast form computes the plain arithmetic, so
    one request each suffices."""
    E = plain_hist[-1][1]
    tol = 0.005
    out = {"target_energy": E, "tolerance": tol, "tolerance_target": E + tol * abs(E),
           "restarts": B, "steps": T, "chunk_steps": chunk,
           "plain_fp32_session_ms_to_E": next(ms for ms, e in plain_hist if e <= E),
           "plain_fp32_full_run_ms": plain_hist[-1][0],
           "timing": ("wall time from submission to the returned result through the server "
                      "(ising_server_submit_target), exact energy checks every chunk_steps "
                      "steps; plain FP32 served alone (CUDA-core SGEMM / sparse kernel), fast "
                      "forms packed")}
    # untimed: first launches of each form's kernels and its tile autotuning
    for prec in ["fp32"] + list(fast_forms):
        served_time_to_target(ctx, inst, B, 2 * chunk, seed, -math.inf, prec, chunk, 1,
                              budget_s=1e9, pack=prec != "fp32", max_rounds=1)
    for label, tgt, batch in [("within_tolerance", out["tolerance_target"], 1), ("exact", E, 4)]:
        b = 1 if integer else batch
        plain = served_time_to_target(ctx, inst, B, T, seed, tgt, "fp32", chunk, 1,
                                      budget_s=1e9, pack=False, max_rounds=1)
        row = {"plain_fp32": plain, "forms": {}}
        for prec in fast_forms:
            f = served_time_to_target(ctx, inst, B, T, seed, tgt, prec, chunk, b, budget_s, True)
            if plain["time_ms"] and f["time_ms"]:
                f["speedup"] = plain["time_ms"] / f["time_ms"]
            row["forms"][prec] = f
        out[label] = row
    return out


# ----------------------------------------------------------------- serving

def serve_stream(ctx, reqs, B, T, precision_dense, pack, max_active, budget, chunk=250):
    """Submits the requests at their arrival times to a server and waits for
    all; returns per-request results (latency = done - submit) and the
    server's host-time stats."""
    from paper_2312_05837_gb300 import api
    srv = api.Server(ctx, budget_bytes=budget, max_active=max_active, chunk_steps=chunk, pack=pack)
    t0 = time.perf_counter()
    ids = []
    for k, (ta, inst) in enumerate(reqs):
        wait = t0 + ta - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        prec = precision_dense if inst.layout == "dense" else "auto"
        ids.append(srv.submit(inst, restarts=B, steps=T, seed=k, precision=prec))
    res = [srv.wait(r, timeout=3600) for r in ids]
    st = srv.stats()
    srv.close()
    return res, st


def latency_summary(res, rate):
    import numpy as np
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in res])
    adm = np.array([r["t_admit_ms"] - r["t_submit_ms"] for r in res])
    span = (max(r["t_done_ms"] for r in res) - min(r["t_submit_ms"] for r in res)) / 1e3
    thr = len(res) / span
    return {"requests": len(res), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "admission_wait_p50_ms": float(np.percentile(adm, 50)),
            "admission_wait_p99_ms": float(np.percentile(adm, 99)),
            "instances_per_s": thr, "offered_per_s": rate,
            "sustains_offered_load": bool(thr >= 0.95 * rate),
            "all_ok": all(r["status"] == 0 for r in res)}


def serving_capacity(reqs, B, T, pk):
    """Requests per second the GPU could complete at its measured peaks for
    this stream's mix, from the sizes alone (before pruning): a dense
    request needs 2 N^2 B T flop at the E4M3 rate (2 x the sustained BF16
    figure) and moves at least 24 B of state per update plus its E4M3 J once
    per step; a sparse one moves 24.25 B per update (restarts padded to 128);
    each takes the longer of its compute and memory times."""
    fp8 = 2.0 * pk["bf16_tflops_sustained"] * 1e12
    hbm = pk["hbm_gbs"] * 1e9
    total = 0.0
    for _, inst in reqs:
        n = float(inst.n)
        if inst.layout == "dense":
            total += max(2.0 * n * n * B * T / fp8, (24.0 * n * B + n * n) * T / hbm)
        else:
            total += 24.25 * n * ((B + 127) // 128 * 128) * T / hbm
    return len(reqs) / total


def serving(ctx, pk, count=1000, rate=200.0, n_max=8192, B=256, T=2000, seed=5, plain_count=200):
    """The serving stream (Poisson arrivals at `rate`, N log-uniform in
    [64, n_max] over pooled instances, half dense SK J ~ N(0, 1/N) with
    h ~ N(0, 0.1), half sparse ER degree 8 +-1; B restarts x T steps each,
    120 GB admission budget) through the server in its served form: dense
    requests in row-scaled E4M3 (mixed precision: FP32 accumulate, the
    result's energy re-evaluated in FP64), packed launches, 32 requests
    admitted at once. Baseline: the plain per-request FP32 form served live,
    one request at a time in arrival order (the CUDA-core SGEMM for dense
    requests), on the first `plain_count` requests of the same stream; the
    served form's figures on those same requests come from its full run."""
    import synth
    from paper_2312_05837_gb300 import api
    reqs = synth.serving_stream_pooled(count, seed, rate=rate, n_max=n_max)
    budget = 120 << 30
    # first launches of a kernel load it: warm both forms on small requests
    small = [(0.0, inst) for _, inst in sorted(reqs, key=lambda r: r[1].n)[:4]]
    serve_stream(ctx, small, B, 4, "fp8", True, 4, budget)
    serve_stream(ctx, small, B, 4, "fp32", False, 1, budget)
    served, st = serve_stream(ctx, reqs, B, T, "fp8", True, 32, budget)
    plain, _ = serve_stream(ctx, reqs[:plain_count], B, T, "fp32", False, 1, budget)
    out = {"requests": count, "rate_per_s": rate, "n_range": [64, n_max], "restarts": B,
           "steps": T, "budget_gb": 120,
           "capacity_at_roofline_per_s": serving_capacity(reqs, B, T, pk),
           "mix": "50% dense SK J~N(0,1/N) h~N(0,0.1), 50% sparse ER deg 8 +-1 (24 pooled sizes "
                  "per kind, N drawn log-uniformly, nearest pooled size)",
           "served": {**latency_summary(served, rate), "form": "packed launches, dense in "
                      "row-scaled E4M3 + FP64 final energy, max_active 32, chunk 250, 2 helper "
                      "threads", "server_host_ms": {k: round(v, 1) for k, v in st.items()}},
           "served_first_%d" % plain_count: latency_summary(served[:plain_count], rate),
           "plain_fp32_per_request_live": {**latency_summary(plain, rate),
                                           "form": "one request at a time, dense on the "
                                                   "CUDA-core FP32 SGEMM"}}
    import numpy as np
    # the served answers against the plain ones on the same requests (energies
    # of the full instances, exact)
    gaps = [(a["best_energy"] - b["best_energy"]) / abs(b["best_energy"])
            for a, b in zip(served[:plain_count], plain) if b["best_energy"] != 0]
    out["served_vs_plain_energy_gap"] = {"mean": float(np.mean(gaps)), "max": float(np.max(gaps))}
    return out


# ----------------------------------------------------------------- early retirement

def early_retirement(ctx, B=1024, T=1000, families=("uniform", "gaussian", "binary")):
    """The Sec. IV-B convergence rule on one 1000-spin 6-regular instance of
    each Table 1 family, B restarts, at most T steps: the restart-steps the
    kernels computed (tiles whose restarts have all stopped are skipped) and
    the device time, against the same run without the rule."""
    import synth
    from paper_2312_05837_gb300 import api
    out = {}
    for fam in families:
        inst = synth.table1_instance(fam, 0)
        row = {}
        for conv in (False, True):
            s = api.Session(ctx, inst, restarts=B, steps=T, seed=1, converge=conv)
            s.run(T)
            r = s.result()
            row["converge" if conv else "fixed"] = {
                "steps_run": r["steps_done"], "restart_steps": s.work(), "device_ms": r["device_ms"],
                "best_energy": r["best_energy"]}
            if conv:
                c = s.convergence()
                row["stopped_fraction"] = float((c > 0).mean())
            s.close()
        row["work_saved"] = 1.0 - row["converge"]["restart_steps"] / (B * T)
        row["time_saved"] = 1.0 - row["converge"]["device_ms"] / row["fixed"]["device_ms"]
        out[fam] = row
    out["config"] = {"restarts": B, "max_steps": T, "lr": 6.0, "n": 1000}
    return out


# ----------------------------------------------------------------- roofline

def roofline(ctx, inst, dinst, name, B, kw, steps, pk, sessions=1):
    """The dominant step kernel, timed launch by launch with CUDA events on
    the context's stream (ISING_DS_PROFILE) over `steps` steps of a session
    on the full instance; with several sessions, the median of their average
    launch times (all kept). Algorithmic work per launch: 2 N^2 B flop on
    the dense paths, 24.25 B per update (theta, m, v read + write, spin bits)
    on the sparse path."""
    from paper_2312_05837_gb300 import api
    per = []
    st = None
    for k in range(sessions):
        prof = api.Session(ctx, dinst, restarts=B, steps=steps, seed=7 + k, profile=True, **kw)
        prof.run(steps)
        st = prof.result()
        prof.close()
        per.append(st["kernel_ms"] / max(st["kernel_launches"], 1))
    avg_ms = statistics.median(per)
    path = st["path"]
    n = inst.n
    if path == 2:  # sparse: HBM bound
        alg = n * ((B + 127) // 128 * 128) * (24 + 0.25)
        roof = {"bound": "hbm", "achieved": alg / (avg_ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "peak_note": "measured copy bandwidth"}
        kname, ksrc = "sparse_step_kernel", "paper_2312_05837_gb300/csrc/ds_sparse.cu"
    elif path == 1:  # tensor cores: 2 N^2 B flop per step
        alg = 2.0 * n * n * B
        fp8 = st["precision"] == 4
        peak = pk["bf16_tflops_sustained"] * (2.0 if fp8 else 1.0)
        roof = {"bound": "tensor", "achieved": alg / (avg_ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s",
                "peak_note": ("E4M3: 2 x measured BF16 sustained (nominal FP8/BF16 ratio)" if fp8
                              else "measured BF16 sustained (FP16 runs at the BF16 rate)")}
        planes = st["operand_planes"]
        if planes > 1:
            # J as hi + lo planes: the tensor cores execute `planes` products
            roof["operand_planes"] = planes
            roof["executed_frac"] = planes * roof["achieved"] / peak
        kname = {0: "tc_step_kernel", 1: "tc_resident_kernel", 2: "tc_small_kernel"}[st["resident"]]
        if st["resident"] == 0:
            # the streaming form's kernel for the chosen tile shape
            kname = ("tc_step_kernel", "tc_step_pair_kernel",
                     "tc_step_split_kernel")[st.get("tile_pair", 0)]
            roof["tile"] = {"restarts": st.get("tile_restarts", 0), "pair": st.get("tile_pair", 0)}
        ksrc = "paper_2312_05837_gb300/csrc/ds_tc.cu"
    else:  # plain FP32 FMA on the CUDA cores
        import torch
        alg = 2.0 * n * n * B
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        fp32_peak = sms * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": alg / (avg_ms / 1e3) / 1e12, "peak": fp32_peak,
                "unit": "TFLOP/s", "peak_note": "152 SMs x 128 FP32 lanes x 2 flop x max clock"}
        kname, ksrc = "plain_step_kernel", "paper_2312_05837_gb300/csrc/ds_plain.cu"
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_for(kname, ksrc, name)
    roof["kernel"] = kname
    roof["peak_source"] = pk["source"]
    roof["avg_launch_ms"] = avg_ms
    roof["algorithmic_per_launch"] = alg
    if sessions > 1:
        roof["sessions_avg_launch_ms"] = per
    return roof, st


def timed_solves(ctx, dinst, B, T, kw, K, flush, stream, seed0=0):
    """K solves, each bracketed by CUDA events on the launching stream, the
    L2 flushed (a 512 MB write) before each one outside the timed region.
    Returns the summed device milliseconds and the last result."""
    import torch
    from paper_2312_05837_gb300 import api
    total_ms, last = 0.0, None
    for k in range(K):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = api.solve(ctx, dinst, restarts=B, steps=T, seed=seed0 + k, **kw)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    return total_ms, last


def secondary(ctx, name, a, pk, flush, stream, solves=3, warm=2):
    """Another bench workload measured into the same line: its own
    throughput over `solves` timed solves (clocks sampled meanwhile) and its
    dominant kernel's roofline (sparse: median of 5 profiled sessions)."""
    import torch
    import synth
    from paper_2312_05837_gb300 import api
    inst_name, B, T = WORKLOADS[name]
    inst = synth.workload(inst_name, 0)
    dinst = device_instance(inst, torch)
    kw = dict(lr=a.lr, mu=a.mu, precision="auto")
    for w in range(warm):
        api.solve(ctx, dinst, restarts=B, steps=T, seed=1000 + w, **kw)
    torch.cuda.synchronize()
    pr = api.prune(ctx, inst)
    n_red = pr.n_reduced
    pr.close()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms, last = timed_solves(ctx, dinst, B, T, kw, solves, flush, stream)
    clk = clocks.stop()
    roof, st = roofline(ctx, inst, dinst, name, B, kw, a.profile_steps, pk,
                        sessions=5 if last["path"] == 2 else 1)
    out = {"workload": f"{name}: N={inst.n} (N_reduced={n_red}), restarts={B}, steps={T}",
           "value": n_red * B * T * solves / (ms / 1e3), "unit": UNIT, "solves": solves,
           "ms_per_solve": ms / solves, "path": {0: "plain", 1: "tc", 2: "sparse"}[last["path"]],
           "precision": last["precision"], "kernel_us": roof["avg_launch_ms"] * 1e3,
           "roofline": roof, "clocks": clk, "best_energy": float(last["best_energy"].item())}
    del dinst
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------- main

def main():
    a = args_()
    if a.cpu_leg:
        cpu_leg(a)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    import numpy as np
    import torch
    import synth
    from paper_2312_05837_gb300 import api

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    name, B, T = WORKLOADS[a.workload]
    inst = synth.workload(name, seed=rank)
    dinst = device_instance(inst, torch)
    hinst = pinned_instance(inst, torch)
    ctx = api.Context(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    kw = dict(lr=a.lr, mu=a.mu, precision=a.precision)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for w in range(a.warmup):
        api.solve(ctx, dinst, restarts=B, steps=T, seed=1000 + w, **kw)
    torch.cuda.synchronize()
    pr = api.prune(ctx, inst)
    n_red, rounds = pr.n_reduced, pr.rounds
    pr.close()

    clocks = Clocks(local)
    clocks.start()
    barrier()
    total_ms, last = timed_solves(ctx, dinst, B, T, kw, a.steps, flush, stream)
    barrier()
    clk = clocks.stop()
    max_ms = over_ranks(dist, total_ms, "max", "cuda")
    units = n_red * B * T
    # each rank solves its own instance (seeded by its rank), so the reduced
    # sizes differ: the job's units are the sum over ranks
    job_units = over_ranks(dist, float(units), "sum", "cuda")
    value = job_units * a.steps / (max_ms / 1e3)

    # end to end: host (pinned) inputs, host outputs, copies inside the timed region
    e2e_k = max(1, min(a.steps, a.e2e_steps))
    barrier()
    w0 = time.perf_counter()
    for k in range(e2e_k):
        api.solve(ctx, hinst, restarts=B, steps=T, seed=k, **kw)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    e2e_value = job_units * e2e_k / over_ranks(dist, e2e_s, "max", "cuda")

    pk = peaks()
    roof, st = roofline(ctx, inst, dinst, name, B, kw, a.profile_steps, pk,
                        sessions=5 if last["path"] == 2 else 1)
    path = last["path"]
    prec = st["precision"]
    dtype = {0: "f32", 2: "f32"}.get(path)
    if path == 1:
        dtype = {4: "e4m3", 3: "bf16"}.get(prec, "f16x2" if st["operand_planes"] == 2 else "f16/bf16")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": max_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": f"{name}: N={inst.n} (N_reduced={n_red}), restarts={B}, "
                                   f"steps={T}, lr={a.lr}, mu={a.mu}",
                       "precision": a.precision,
                       "operands": ("J as two FP16 planes hi + lo of J / 2^e_i (power-of-two "
                                    "row scales, about 22 significant bits), spins FP16 +-1, "
                                    "FP32 accumulate" if dtype == "f16x2" else dtype),
                       "path": {0: "plain", 1: "tc", 2: "sparse"}[path],
                       "l2": "flushed (512 MB write) before each timed solve",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": input_bytes(inst),
                    "d2h_bytes_per_step": int(inst.n) + 8, "solves": e2e_k},
            "gpu_launches": launches_per_solve(
                T, rounds, path, bool(last["resident"]), path == 1 and bool(inst.integer),
                path == 1 and not inst.integer and prec in (2, 4)) * a.steps,
            "roofline": roof, "clocks": clk,
            "best_energy": float(last["best_energy"].item())}
    if name.startswith("table2"):
        from paper_2312_05837_gb300.metrics import paper_metrics
        line["paper_metrics"] = paper_metrics(inst, line["best_energy"], max_ms / a.steps / 1e3)
    del dinst
    torch.cuda.empty_cache()
    if rank == 0 and a.secondary:
        line["workloads"] = {w: secondary(ctx, w, a, pk, flush, stream)
                             for w in a.secondary.split(",") if w and w != name}
    if rank == 0 and not a.no_extras:
        forms = ["fp32", "tc", "bf16", "fp8"] if not inst.integer else ["fp32", "auto"]
        dinst = device_instance(inst, torch)
        chunk = 100 if T >= 4000 else 50
        sweep, plain_hist = precision_runs(ctx, dinst, bool(inst.integer), inst.n, B, T, seed=3,
                                           forms=forms, chunk=chunk)
        line["precision_sweep"] = sweep
        del dinst
        torch.cuda.empty_cache()
        line["time_to_target"] = {name: time_to_target(
            ctx, hinst, bool(inst.integer), B, T, 3, plain_hist,
            ["fp8", "tc"] if not inst.integer else ["auto"], chunk)}
        if name != "er2000":
            # the integer max-cut workload: exact E4M3 against plain FP32
            w_name, wB, wT = WORKLOADS["er2000"]
            winst = synth.workload(w_name, 0)
            wd = device_instance(winst, torch)
            _, w_hist = precision_runs(ctx, wd, True, winst.n, wB, wT, seed=3, forms=["fp32"],
                                       chunk=50)
            del wd
            torch.cuda.empty_cache()
            line["time_to_target"]["er2000"] = time_to_target(
                ctx, pinned_instance(winst, torch), True, wB, wT, 3, w_hist, ["auto"], 50)
        line["early_retirement"] = early_retirement(ctx)
        line["serving"] = serving(ctx, pk)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, B, T)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

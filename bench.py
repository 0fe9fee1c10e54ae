#!/usr/bin/env python3
"""Throughput of the GB300 norm-1 ADMM on the 8192 x 131072 mixed-precision workload.

Headline workload: H 8192 x 131072 complex64, i.i.d. CN(0, 1/8192) drawn on the
host in seeded row chunks (synth.chunked_gaussian_problem, seed 3), 400 planted
nonzeros, 30 dB, lambda = 0.05 max|H^H g|, rho = 1, consensus over 16 row blocks
of 512 rows.  One step = one ADMM iteration with the complex64 H; the timed
region runs the K steps as one launch of the persistent iteration kernel
(admm_iterate(h, K)).  H (8.6 GB) is far larger than L2, so no flush is needed.
Beside it: the FP16-H mode, the 280 FP16 + 20 complex64 schedule against 300
complex64 iterations and the time to 1e-4 relative error of both, each with its
error against the stored FP64 oracle solution of this exact problem; then the
CRA-shaped 1440 x 32768 workload in the paper's three splits, the 256 x 4096
workload, and the batched, differentiable, uneven-problem and direct-form legs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank solves its own scene (weak scaling, no
collective on the data path; a barrier and a max-reduction of the timings
only).  Rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ADMM iters/s & HBM GB/s vs roofline; time to 1e-4 rel. err, chosen vs plain"
UNIT = "iters/s"
SPLITS = ((8, 1), (1, 8), (4, 4))
M_ROWS, N_COLS = 1440, 32768
C3_M, C3_N, C3_NNZ, C3_SEED, C3_BLOCKS = 8192, 131072, 400, 3, 16
C3_FP16, C3_POLISH = 280, 20
C3_VSTAR = os.path.join(ROOT, "tests", "golden", "vstar_gaussian_8192x131072_c16.txt")
WORKLOAD = ("Gaussian 8192x131072 complex64 CN(0,1/8192), 400 nonzeros, 30 dB, consensus 16x1 "
            "(512-row blocks), lambda 0.05 max|H^H g|, rho 1; one complex64 iteration per step")
CONFIG = {"workload": WORKLOAD, "m": C3_M, "n": C3_N, "row_blocks": C3_BLOCKS, "col_blocks": 1,
          "inputs": "host generator synth.chunked_gaussian_problem(8192, 131072, 400, seed 3)",
          "l2": "inputs larger than L2 (H 8.6 GB vs 129 MB L2), no flush"}
# the CPU oracle sample: the same recipe at a quarter of the rows
CPU_M, CPU_NNZ = 2048, 100


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-iters", type=int, default=30,
                    help="iterations per split in the bounded CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-direct", action="store_true",
                    help="skip the direct-factor-form leg (overdetermined 32768 x 2048)")
    ap.add_argument("--no-uneven", action="store_true",
                    help="skip the 48 uneven problems workload")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the differentiable workload (forward with recording + reverse sweep)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched shared-H workload (tensor-core GEMMs)")
    ap.add_argument("--batch", type=int, default=256, help="scenes of the batched workload")
    ap.add_argument("--no-cra", action="store_true",
                    help="skip the CRA-shaped 1440x32768 workload in the three splits")
    ap.add_argument("--no-small", action="store_true", help="skip the 256x4096 workload")
    ap.add_argument("--no-sharded", action="store_true",
                    help="skip the sharded iteration of the headline problem on one GPU")
    ap.add_argument("--no-time-to-tol", action="store_true",
                    help="skip the time-to-1e-4 comparison of FP16+polish against plain complex64")
    ap.add_argument("--l2-keep-mb", type=float, default=None,
                    help="MiB of H per pass kept in L2 for the reversed next pass "
                         "(ADMM_OPT_L2_KEEP_BYTES; default: the library's)")
    ap.add_argument("--cpu-sample-worker", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d.get("bf16_tflops", 1900.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


TRAFFIC_FILES = ("iterate_kernel_gaussian8192x131072_dram.txt", "iterate_kernel_cra1440x32768_dram.txt")


def load_traffic() -> dict | None:
    """DRAM bytes per iteration of the iteration kernel from the committed ncu
    summaries (keys: workload or split names), each file used only while the
    kernel's source hash matches the one it was captured with."""
    import hashlib
    src = os.path.join(ROOT, "paper_1811_05571_gb300", "csrc", "admm_iterate.cu")
    have = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    out = {}
    for name in TRAFFIC_FILES:
        path = os.path.join(ROOT, "profiles", name)
        if not os.path.exists(path):
            continue
        want, vals = None, {}
        for line in open(path):
            parts = line.split()
            if len(parts) == 2 and parts[0] == "source_sha256":
                want = parts[1]
            elif len(parts) == 3 and parts[0] == "traffic_bytes":
                vals[parts[1]] = float(parts[2])
        if want == have:
            out.update(vals)
    return out or None


def make_problem(rank: int):
    """Rank r's replica: the shared CRA-shaped matrix with its own scene (seed 2 + r)."""
    import synth
    H = synth.cra_matrix(seed=1)
    return synth.cra_problem(H=H, scene_seed=2 + rank)


def max_over_ranks(seconds: float, world: int, device=None) -> float:
    """The largest of the ranks' timings (the whole job lasts as long as the
    slowest rank).  The tensor lives on `device` for NCCL, on the host for gloo."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    on = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], device=on, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, splits: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: iterations of every split on every rank per second."""
    return world * splits * steps / seconds


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.file.read())) if len(r) >= 9]
        self.file.close()
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def quarter_problem():
    """The CPU-oracle sample: the headline recipe at a quarter of the rows
    (2048 x 131072, 100 nonzeros), as complex128 for the oracle."""
    import numpy as np
    import synth
    H, g, _, lam = synth.chunked_gaussian_problem(CPU_M, C3_N, CPU_NNZ, C3_SEED)
    return H.astype(np.complex128), g, lam


def oracle_seconds_per_iteration(H, g, lam, k: int, warmup: int) -> float:
    """Seconds per iteration of the oracle as it stands (consensus, 16 row
    blocks): one run of warmup + k iterations, timed from the end of the last
    warm-up iteration to the end of the last one (at least one warm-up
    iteration, so the one-time factorisation is excluded)."""
    import oracle
    k, warmup = max(int(k), 1), max(int(warmup), 1)
    stamps = []
    oracle.run_split(H, g, C3_BLOCKS, 1, lam, 1.0, warmup + k,
                     on_iter=lambda it: stamps.append(time.perf_counter()))
    return (stamps[warmup + k - 1] - stamps[warmup - 1]) / k


# per-iteration cost of the oracle is two passes over H: proportional to the rows at fixed n
CPU_SCALE = C3_M / CPU_M


def cpu_sample_text(iters: int, warmup: int, cores: int) -> str:
    return (f"FP64 oracle (numpy/OpenBLAS, {cores} threads) on the headline recipe at a quarter of the "
            f"rows (2048x131072, 100 nonzeros, 16 row blocks of 128): {iters} iterations after "
            f"{max(warmup, 1)} warm-up, factorisation excluded; seconds per iteration x4 for "
            f"8192 rows (two passes over H per iteration)")


def cpu_sample_worker(args) -> None:
    H, g, lam = quarter_problem()
    per = oracle_seconds_per_iteration(H, g, lam, args.cpu_iters, 2)
    print(json.dumps({"per_iter_s": per, "cores": int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))}))


def cpu_baseline(iters: int) -> dict:
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for key in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[key] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample-worker",
                          "--cpu-iters", str(iters)], env=env, capture_output=True, text=True,
                         timeout=900)
    if res.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"failed: {res.stderr.strip()[-200:]}"}
    d = json.loads(res.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / (d["per_iter_s"] * CPU_SCALE), "unit": UNIT, "cores": d["cores"],
            "kind": "oracle", "sample": cpu_sample_text(iters, 2, d["cores"]),
            "quarter_scale_s_per_iter": d["per_iter_s"]}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    H, g, lam = quarter_problem()
    k = max(args.steps, 1)
    per = oracle_seconds_per_iteration(H, g, lam, k, max(args.warmup, 0)) * CPU_SCALE
    value = 1.0 / per
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": cpu_sample_text(k, max(args.warmup, 0), cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

TT_TOL, TT_MAX = 1e-4, 600


def load_vstar_file(path: str, n: int):
    """(header, v*) of a stored FP64 oracle solution (nonzeros only)."""
    import numpy as np
    head, v = {}, np.zeros(n, dtype=np.complex128)
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                parts = line[1:].split()
                if len(parts) >= 2 and parts[0] in ("lambda", "rho", "iterations", "nonzeros", "norm"):
                    head[parts[0]] = float(parts[1])
                continue
            k, re, im = line.split()
            v[int(k)] = float(re) + 1j * float(im)
    return head, v


def config3_solver(pkg, stream, dev, rank: int):
    """The headline problem on the device.  Rank 0 draws the host recipe whose
    FP64 oracle solution is stored (so its error can be stated); further ranks
    solve a device-generated instance of the same shape (seed 3 + rank).
    Returns (solver, g, v* or None, timings)."""
    import numpy as np
    import torch
    import synth
    t0 = time.perf_counter()
    vstar = None
    if rank == 0 and os.path.exists(C3_VSTAR):
        head, vstar = load_vstar_file(C3_VSTAR, C3_N)
        lam = head["lambda"]
        H_d = torch.empty((C3_M, C3_N), dtype=torch.complex64, device=dev)

        def sink(r0, rows):
            with torch.cuda.device(dev):
                H_d[r0:r0 + rows.shape[0]].copy_(torch.from_numpy(rows))

        _, g, _, _ = synth.chunked_gaussian_problem(C3_M, C3_N, C3_NNZ, C3_SEED, sink=sink, lam=lam)
        g_d = torch.from_numpy(g.astype(np.complex64)).to(dev)
    else:
        H_d, g_d, _, lam = synth.gaussian_problem_device(C3_M, C3_N, C3_NNZ, C3_SEED + rank, device=dev)
        g = g_d.cpu().numpy().astype(np.complex128)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        s = pkg.Solver(H_d, g_d, C3_BLOCKS, 1, lam, 1.0, stream=stream)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    del H_d, g_d
    torch.cuda.empty_cache()
    return s, g, lam, vstar, {"inputs_s": gen_s, "setup_ms": setup_ms}


def rel_err(s, vstar) -> float:
    import numpy as np
    v = s.v().cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(v - vstar) / np.linalg.norm(vstar))


def config3_schedules(s, stream, barrier, vstar) -> dict:
    """The workload's 300-iteration schedules from the zero state: 280 FP16-H
    iterations then 20 complex64 polish iterations ("chosen") against 300
    complex64 iterations ("plain"); CUDA events on the launching stream, and
    each result's relative error against the FP64 oracle solution."""
    import torch

    def schedule(k16: int, k32: int):
        s.reset()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if k16:
            s.use_fp16(True)
            s.iterate(k16)
            s.use_fp16(False)
        s.iterate(k32)
        b.record(stream)
        barrier()
        rec = s.residuals(1)[0].tolist()
        out = {"ms": a.elapsed_time(b), "final_rp2_rd2": rec[:2]}
        if vstar is not None:
            out["rel_err_vs_fp64_oracle"] = rel_err(s, vstar)
        return out

    chosen = schedule(C3_FP16, C3_POLISH)
    chosen.update({"fp16_iters": C3_FP16, "polish_iters": C3_POLISH})
    plain = schedule(0, C3_FP16 + C3_POLISH)
    plain.update({"iters": C3_FP16 + C3_POLISH})
    if s.status() != 0:
        raise RuntimeError("device status after the schedules")
    return {"chosen": chosen, "plain": plain, "speedup": plain["ms"] / chosen["ms"]}


def config3_time_to_tol(s, stream, barrier, vstar, setup_ms: float, setup16_ms: float) -> dict:
    """Time to ||v - v*|| / ||v*|| <= 1e-4 on the headline problem, v* the stored
    FP64 oracle solution: plain complex64 iterations against the chosen schedule
    (FP16-H iterations, then 20 complex64 polish iterations).

    Calibration (untimed) finds the fewest iterations, in steps of 5, that meet
    the tolerance: for plain by reading v every 5 iterations; for chosen by
    checkpointing the FP16 run every 5 iterations, polishing a copy and
    restoring the checkpoint.  The timed runs then execute exactly those
    iterations from the zero state (CUDA events on the launching stream, median
    of 3).  "with setup" adds the handle creation (Gram products and FP64
    factorisation) and, for chosen, building the FP16 copy and its factors."""
    import torch
    out = {"tol": TT_TOL, "vstar": "FP64 oracle (stored), residuals at the Boyd tolerances 1e-14 / 1e-12"}
    s.reset()
    k_plain = None
    for k in range(5, TT_MAX + 1, 5):
        s.iterate(5)
        if rel_err(s, vstar) <= TT_TOL:
            k_plain = k
            break
    s.reset()
    s.use_fp16(True)
    k16 = None
    for k in range(0, TT_MAX + 1, 5):
        if k:
            s.iterate(5)
        ck = s.state()
        s.use_fp16(False)
        s.iterate(C3_POLISH)
        e = rel_err(s, vstar)
        if e <= TT_TOL:
            k16 = k
            break
        s.set_state(*ck)
        s.use_fp16(True)
    s.use_fp16(False)
    if k_plain is None or k16 is None:
        out["unavailable"] = f"a schedule did not reach the tolerance within {TT_MAX} iterations"
        return out

    def timed(fp16_iters: int, plain_iters: int):
        ts = []
        for _ in range(3):
            s.reset()
            barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if fp16_iters:
                s.use_fp16(True)
                s.iterate(fp16_iters)
                s.use_fp16(False)
            s.iterate(plain_iters)
            b.record(stream)
            barrier()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), rel_err(s, vstar)

    ms_plain, e_plain = timed(0, k_plain)
    ms_chosen, e_chosen = timed(k16, C3_POLISH)
    if s.status() != 0:
        raise RuntimeError("device status after the time-to-tolerance runs")
    out.update({
        "plain": {"iters": k_plain, "ms": ms_plain, "setup_ms": setup_ms,
                  "ms_with_setup": ms_plain + setup_ms, "rel_err": e_plain},
        "chosen": {"fp16_iters": k16, "polish_iters": C3_POLISH, "ms": ms_chosen,
                   "setup_ms": setup_ms + setup16_ms, "ms_with_setup": ms_chosen + setup_ms + setup16_ms,
                   "rel_err": e_chosen},
        "speedup": ms_plain / ms_chosen,
        "speedup_with_setup": (ms_plain + setup_ms) / (ms_chosen + setup_ms + setup16_ms),
    })
    return out


def batched_shared_h(pkg, stream, dev, barrier, p, peaks, batch: int = 256, steps: int = 10) -> dict:
    """B three-plate scenes (seeds 100 ...) on the CRA matrix, iterated together by
    the tensor-core path in each split; per split the time of one iteration of
    all scenes (CUDA events around `steps` graph launches), the tensor-core
    FLOP rate issued, and the state bytes moved per second."""
    import numpy as np
    import torch
    import synth
    G, _, lam = synth.shared_h_scenes(p.H, batch, seed0=100, kind="plates")
    H_d = torch.from_numpy(p.H_c64()).to(dev)
    G_d = torch.from_numpy(G.astype(np.complex64)).to(dev)
    out = {"workload": f"CRA-shaped 1440x32768, {batch} three-plate scenes (seeds 100-{99 + batch}), "
                       f"30 dB, lambda_b = 0.05 max|H^H g_b|, rho {p.rho:.1f}, FP16 H",
           "batch": batch, "splits": {}}
    for M, N in SPLITS:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            bs = pkg.BatchSolver(H_d, M, N, lam, p.rho, stream=stream)
            bs.set_g(G_d)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        bs.iterate(3)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bs.iterate(steps)
        b.record(stream)
        barrier()
        us = a.elapsed_time(b) / steps * 1e3
        if bs.status() != 0:
            raise RuntimeError("device status after the batched runs")
        info = bs.info()
        bs.close()
        out["splits"][f"{M}x{N}"] = {
            "us_per_iteration": us, "scene_iterations_per_s": batch / us * 1e6,
            "tensor_tflops": info["tensor_flops"] / us / 1e6,
            "tensor_frac": info["tensor_flops"] / us / 1e6 / peaks["bf16_tflops"],
            "method_tflops": info["method_flops"] / us / 1e6,
            "state_gbs": info["state_bytes"] / us / 1e3,
            "state_frac": info["state_bytes"] / us / 1e3 / peaks["hbm_gbs"],
            "tensor_flops_per_iter": info["tensor_flops"], "state_bytes_per_iter": info["state_bytes"],
            "forward_k_splits": info["splits"], "setup_ms": setup_ms}
    return out


def uneven_problems(pkg, stream, dev, barrier, peaks, iters: int = 300) -> dict:
    """48 Gaussian problems of uneven sizes (synth.uneven_problem_sizes), each
    with its own handle (consensus over ceil(m/256) row blocks, lambda 0.05
    max|H^H g|, rho 1), run for `iters` iterations (a) as one persistent launch
    per problem, all on one stream, and (b) grouped (admm_group_*: the problems
    of a wave share one persistent launch, each on its share of the SMs):
    total time with CUDA events, problem-iterations per second and the
    algorithmic bytes moved per second."""
    import torch
    import synth
    sizes = synth.uneven_problem_sizes()
    solvers, alg = [], 0.0
    with torch.cuda.stream(stream):
        for m, n, nnz, M, seed in sizes:
            H, g, _, lam = synth.gaussian_problem_device(m, n, nnz, seed, device=dev)
            s = pkg.Solver(H, g, M, 1, lam, 1.0, stream=stream)
            info = s.info()
            alg += 2 * info["h_bytes"] + info["factor_bytes"] + state_bytes(M, n)
            solvers.append(s)
            del H, g
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    for s in solvers:
        s.iterate(3)
    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for s in solvers:
        s.iterate(iters)
    b.record(stream)
    barrier()
    ms = a.elapsed_time(b)
    for s in solvers:
        if s.status() != 0:
            raise RuntimeError("device status after the uneven problems")
    # the same problems in one persistent launch per wave (admm_group_*)
    grp = pkg.Group(solvers, stream=stream)
    ginfo = grp.info()
    grp.iterate(3)
    barrier()
    a.record(stream)
    grp.iterate(iters)
    b.record(stream)
    barrier()
    ms_group = a.elapsed_time(b)
    grp.close()
    for s in solvers:
        if s.status() != 0:
            raise RuntimeError("device status after the grouped uneven problems")
        s.close()
    elems = sum(m * n for m, n, _, _, _ in sizes)
    return {"workload": f"{len(sizes)} Gaussian problems, m in [256, 4096], n in [4096, 32768] "
                        f"(log-uniform, seeds 1000-{999 + len(sizes)}), consensus ceil(m/256)x1, "
                        f"{iters} iterations each, one launch per problem",
            "problems": len(sizes), "elements": elems, "ms": ms,
            "problem_iterations_per_s": len(sizes) * iters / (ms / 1e3),
            "alg_gbs": alg * iters / (ms / 1e3) / 1e9, "frac": alg * iters / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "group": {"waves": ginfo["waves"], "ms": ms_group,
                      "problem_iterations_per_s": len(sizes) * iters / (ms_group / 1e3),
                      "alg_gbs": alg * iters / (ms_group / 1e3) / 1e9,
                      "frac": alg * iters / (ms_group / 1e3) / 1e9 / peaks["hbm_gbs"]}}


def differentiable(pkg, stream, dev, barrier, K: int = 100) -> dict:
    """The differentiable workload: H 2048 x 16384, 16 scenes of 64 nonzeros
    (seeds 500-515), consensus over 8 row blocks, loss sum_b ||v_K - u_b||^2.
    (a) complex64 H: UnrolledADMM over 16 single-scene handles (K recorded
    iterations each, then each handle's reverse sweep) -- gradients in G,
    lambda and rho through loss.backward(); (b) the FP16-encoded H: all 16
    scenes together on the tensor cores (BatchSolver).  Forward and reverse
    times with CUDA events on the launching stream (median of 3)."""
    import numpy as np
    import torch
    import synth
    p = synth.gaussian_problem(2048, 16384, 64, seed=5)
    G, U, lam = synth.shared_h_scenes(p.H, 16, seed0=500, nnz=64)
    Hd = torch.from_numpy(p.H_c64()).to(dev)
    G_d = torch.from_numpy(G.astype(np.complex64)).to(dev)
    U_d = torch.from_numpy(U.astype(np.complex64)).to(dev)
    out = {"workload": "gaussian 2048x16384 CN(0,1/2048), 16 scenes x 64 nonzeros (seeds 500-515), "
                       "consensus 8x1, K = 100, loss sum ||v_K - u||^2"}

    # (a) complex64, one handle per scene, through torch.autograd
    with torch.cuda.stream(stream):
        solvers = [pkg.Solver(Hd, G_d[b], 8, 1, lam[b], 1.0, stream=stream) for b in range(16)]
    torch.cuda.synchronize()

    def once_c64():
        Gt = G_d.clone().requires_grad_(True)
        lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
        rho_t = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        barrier()
        a.record(stream)
        with torch.cuda.stream(stream):
            V = pkg.UnrolledADMM.apply(Gt, lam_t, rho_t, solvers, K)
            loss = ((V - U_d).abs() ** 2).sum()
        b.record(stream)
        with torch.cuda.stream(stream):
            loss.backward()
        c.record(stream)
        barrier()
        return a.elapsed_time(b), b.elapsed_time(c)

    once_c64()
    fw, bw = zip(*[once_c64() for _ in range(3)])
    for sv in solvers:
        if sv.status() != 0:
            raise RuntimeError("device status after the complex64 differentiable workload")
        sv.close()
    fwd, bwd = statistics.median(fw), statistics.median(bw)
    out["complex64_per_scene"] = {"forward_ms": fwd, "backward_ms": bwd,
                                  "gradients_per_s": 16 / ((fwd + bwd) / 1e3),
                                  "backward_over_forward": bwd / fwd,
                                  "path": "UnrolledADMM over 16 Solver handles (admm_backward)"}

    # (b) FP16-encoded H, all scenes on the tensor cores
    with torch.cuda.stream(stream):
        bs = pkg.BatchSolver(Hd, 8, 1, lam, 1.0, stream=stream)

    def once():
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        bs.record(K)
        bs.set_g(G_d)
        barrier()
        a.record(stream)
        bs.iterate(K)
        b.record(stream)
        with torch.cuda.stream(stream):
            dV = (2.0 * (bs.v() - U_d)).contiguous()
        bs.backward(dV)
        c.record(stream)
        barrier()
        return a.elapsed_time(b), b.elapsed_time(c)

    once()
    fw, bw = zip(*[once() for _ in range(3)])
    if bs.status() != 0:
        raise RuntimeError("device status after the differentiable workload")
    info = bs.info()
    bs.close()
    fwd, bwd = statistics.median(fw), statistics.median(bw)
    out["fp16_batched"] = {"forward_ms": fwd, "backward_ms": bwd, "gradients_per_s": 16 / ((fwd + bwd) / 1e3),
                           "backward_over_forward": bwd / fwd, "tensor_flops_per_iter": info["tensor_flops"]}
    return out


def direct_form(pkg, stream, dev, barrier, peaks, iters: int = 64) -> dict:
    """The direct factor form on an overdetermined 32768 x 2048 Gaussian
    problem in three splits (every block has m_b >= n_b), and the lemma form on
    the consensus split for comparison.  Per split: one call of `iters`
    iterations timed with CUDA events on the launching stream, after 19
    warm-up iterations (which capture both iteration graphs).  Algorithmic
    bytes per iteration: the passes over H (none with one column block:
    H_i^H g_i is cached, two otherwise), every factor once (the tile pass: its
    lower-triangle tiles), the state v, s read and written, and with one
    column block the cached H_i^H g_i.  The consensus split also runs with the
    full-factor-row pass (`rows_pass_8x1`)."""
    import torch
    import synth
    c = synth.TALL
    H, g, _, lam = synth.gaussian_problem_device(c["m"], c["n"], c["nnz"], c["seed"], device=dev)
    torch.cuda.synchronize()
    out = {"workload": f"gaussian {c['m']}x{c['n']} CN(0,1/{c['m']}), {c['nnz']} nonzeros, 30 dB, "
                       f"seed {c['seed']} (device generator), lambda 0.05 max|H^H g|, rho {c['rho']}",
           "iters_per_call": iters, "splits": {}}

    def measure(M, N, form, factor_pass=0):
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            s = pkg.Solver(H, g, M, N, lam, c["rho"], stream=stream, form=form)
            if factor_pass:
                s.set_option(pkg.ADMM_OPT_DIR_FACTOR_PASS, factor_pass)
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t0) * 1e3
        info = s.info()
        s.iterate(19)   # both iteration graphs (16 and 1) captured before the timed call
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.iterate(iters)
        b.record(stream)
        barrier()
        if s.status() != 0:
            raise RuntimeError(f"device status after the {form} {M}x{N} run")
        us = a.elapsed_time(b) / iters * 1e3
        state = state_bytes(M, c["n"])
        if form == "direct":
            passes = 0 if N == 1 else 2
            alg = passes * info["h_bytes"] + info["factor_bytes"] + state + (M * c["n"] * 8 if N == 1 else 0)
        else:
            alg = 2 * info["h_bytes"] + info["factor_bytes"] + state
        s.close()
        return {"factor_form": form, "factor_pass": ("tiles" if info["rows_per_stage"] == 64 else "rows")
                if form == "direct" else None,
                "us_per_iter": us, "iters_per_s": 1e6 / us, "alg_bytes_per_iter": alg,
                "gbs": alg / us / 1e3, "frac": alg / us / 1e3 / peaks["hbm_gbs"],
                "factor_bytes": info["factor_bytes"], "setup_ms": setup_ms,
                "setup_gram_ms": info["setup_gram_ms"], "setup_factor_ms": info["setup_factor_ms"]}

    for M, N in c["splits"]:
        out["splits"][f"{M}x{N}"] = measure(M, N, "direct")
    # the full-factor-row pass beside the lower-triangle tiles
    out["rows_pass_8x1"] = measure(8, 1, "direct", factor_pass=1)
    lem = measure(8, 1, "lemma")
    out["lemma_8x1"] = lem
    out["speedup_8x1"] = lem["us_per_iter"] / out["splits"]["8x1"]["us_per_iter"]
    del H, g
    torch.cuda.empty_cache()
    return out


def state_bytes(M: int, n: int) -> int:
    """Algorithmic state bytes of one iteration: v and the M duals read by the
    first product and again by the update, and written once, complex64."""
    return (3 * M + 3) * n * 8


def cra_three_splits(pkg, stream, dev, barrier, peaks, K: int, warmup: int, rank: int) -> dict:
    """The CRA-shaped 1440 x 32768 workload in the paper's three splits (8x1,
    1x8, 4x4), K iterations per split as one persistent launch, complex64 and
    FP16 H, with each split's algorithmic bytes per iteration."""
    import torch
    p = make_problem(rank)
    H_d = torch.from_numpy(p.H_c64()).to(dev)
    g_d = torch.from_numpy(p.g_c64()).to(dev)
    torch.cuda.synchronize()
    solvers = []
    with torch.cuda.stream(stream):
        for M, N in SPLITS:
            solvers.append(pkg.Solver(H_d, g_d, M, N, p.lam, p.rho, stream=stream))
    del H_d, g_d
    torch.cuda.synchronize()
    out = {"workload": ("CRA-shaped imaging, H 1440x32768 complex64 (40 freqs x 36 rx, 32^3 voxels), "
                        "three-plate scene, 30 dB"), "lambda": p.lam, "rho": p.rho, "splits": {}}

    def timed(s, fp16: bool):
        s.use_fp16(fp16)
        for _ in range(max(warmup, 0)):
            s.iterate(1)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.iterate(K)
        b.record(stream)
        barrier()
        info = s.info()
        hb = info["h16_bytes"] if fp16 else info["h_bytes"]
        alg = 2 * hb + info["factor_bytes"] + state_bytes(s.M, s.n)
        us = a.elapsed_time(b) / K * 1e3
        return {"us_per_iter": us, "iters_per_s": 1e6 / us, "alg_bytes_per_iter": alg,
                "gbs": alg / us / 1e3, "frac": alg / us / 1e3 / peaks["hbm_gbs"]}, info

    traffic = load_traffic()
    for (M, N), s in zip(SPLITS, solvers):
        c64, info = timed(s, False)
        f16, _ = timed(s, True)
        s.use_fp16(False)
        name = f"{M}x{N}"
        c64.update({"ctas": info["ctas"], "rows_per_stage": info["rows_per_stage"], "stages": info["stages"],
                    "setup_ms": {"gram": info["setup_gram_ms"], "cholesky_inverse": info["setup_factor_ms"]},
                    "fp16_h": f16})
        if traffic:
            c64["dram_bytes_per_launch"] = traffic.get(name)
            f16["dram_bytes_per_launch"] = traffic.get(name + "_fp16")
            if traffic.get(name):
                # DRAM bytes actually moved (ncu) over the same time: the reversed
                # second pass finds the first pass's last 52 MiB in L2
                c64["dram_frac"] = traffic[name] / c64["us_per_iter"] / 1e3 / peaks["hbm_gbs"]
        out["splits"][name] = c64
        if s.status() != 0:
            raise RuntimeError(f"device status after the CRA {name} runs")
        s.close()
    tot_us = sum(v["us_per_iter"] for v in out["splits"].values())
    out["iters_per_s_all_splits"] = len(SPLITS) / tot_us * 1e6
    out["note"] = ("frac counts algorithmic bytes; where it exceeds the DRAM-based dram_frac the "
                   "difference is the L2 reuse between the two passes, not a faster memory")
    return out


def small_workload(pkg, stream, dev, barrier, iters: int = 300, reps: int = 5) -> dict:
    """The 256 x 4096 workload (consensus over 4 row blocks of 64, rho 1, 300
    iterations): H (8.4 MB) stays in L2, so the iteration is latency bound;
    iterations per second of one 300-iteration launch (median of `reps`)."""
    import torch
    import synth
    c = synth.CONFIG1
    p = synth.gaussian_problem(c["m"], c["n"], c["nnz"], seed=c["seed"])
    with torch.cuda.stream(stream):
        s = pkg.Solver(torch.from_numpy(p.H_c64()).to(dev), torch.from_numpy(p.g_c64()).to(dev),
                       c["row_blocks"], 1, p.lam, c["rho"], stream=stream)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps + 1):
        s.reset()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.iterate(iters)
        b.record(stream)
        barrier()
        ts.append(a.elapsed_time(b))
    if s.status() != 0:
        raise RuntimeError("device status after the 256x4096 runs")
    info = s.info()
    s.close()
    ms = statistics.median(ts[1:])
    alg = 2 * info["h_bytes"] + info["factor_bytes"] + state_bytes(c["row_blocks"], c["n"])
    return {"workload": "Gaussian 256x4096 CN(0,1/256), 16 nonzeros, 30 dB, seed 0, consensus 4x1, rho 1",
            "iters": iters, "ms": ms, "iters_per_s": iters / ms * 1e3, "us_per_iter": ms / iters * 1e3,
            "l2_gbs": alg * iters / ms / 1e6, "ctas": info["ctas"],
            "note": "H is L2-resident: latency bound, HBM fraction not meaningful"}


def sharded_one_gpu(pkg, stream, dev, barrier, peaks, ranks: int = 2, iters: int = 10) -> dict:
    """The sharded iteration (Section IV) of the headline workload's consensus
    split with its 16 row blocks on `ranks` ranks, every rank a handle of its
    8192/ranks rows on this one GPU and the consensus sums exchanged in this
    process (sharded.LocalComm).  Per iteration: each rank's u-step launch over
    its rows, the n-value sums, each rank's v/s update; CUDA events on the
    stream.  The exchange a multi-GPU run would do over NCCL is a host-side
    sum here, so the time is the ranks' kernels one after the other plus the
    exchange: a check of the sharded path at full size, not a multi-GPU
    timing."""
    import torch
    import synth
    from paper_1811_05571_gb300 import sharded as SH
    H, g, _, lam = synth.gaussian_problem_device(C3_M, C3_N, C3_NNZ, C3_SEED, device=dev)
    lays = [SH.ShardLayout(C3_M, C3_N, C3_BLOCKS, 1, ranks, 1, r) for r in range(ranks)]
    engines = [SH.CudaShardEngine(H, g, lay, lam, 1.0) for lay in lays]
    del H, g
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    sol = SH.ShardedSolver(list(zip(lays, engines)), SH.LocalComm(lays), 1.0)
    sol.iterate(2)
    barrier()
    t0 = time.perf_counter()
    sol.iterate(iters)
    barrier()
    ms = (time.perf_counter() - t0) / iters * 1e3
    for e in engines:
        e.close()
    alg = 2 * C3_M * C3_N * 8 + state_bytes(C3_BLOCKS, C3_N)
    return {"workload": f"headline problem shape (device generator), consensus 16x1 over {ranks} ranks on one GPU",
            "ranks": ranks, "ms_per_iter": ms, "alg_gbs": alg / ms / 1e6,
            "timing": "host clock around synchronised iterations (the exchange runs on the host)"}


def run_ours(args) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()

    # CPU baseline first (spawned before any CUDA work of this process)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_iters)

    import paper_1811_05571_gb300 as pkg
    pkg.load()
    peaks = load_peaks()
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    s, g_np, lam, vstar, prep = config3_solver(pkg, stream, dev, rank)
    info = s.info()
    if args.l2_keep_mb is not None:
        s.set_option(pkg.ADMM_OPT_L2_KEEP_BYTES, int(args.l2_keep_mb * (1 << 20)))
    alg = 2 * info["h_bytes"] + info["factor_bytes"] + state_bytes(C3_BLOCKS, C3_N)

    # warm-up, then K steps as one persistent launch of K iterations
    for _ in range(max(args.warmup, 0)):
        s.iterate(1)
    barrier()
    K = args.steps
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev)
    clocks.start()
    barrier()
    t0.record(stream)
    s.iterate(K)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    if s.status() != 0:
        raise RuntimeError("device status after the timed region")
    timed_s = t0.elapsed_time(t1) / 1e3
    total_s = max_over_ranks(timed_s, world, dev)

    # for reference: K single-iteration launches
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    barrier()
    for e0, e1 in ev:
        e0.record(stream)
        s.iterate(1)
        e1.record(stream)
    barrier()
    single_us = sum(e0.elapsed_time(e1) for e0, e1 in ev) / K * 1e3

    # end to end through the public API with host buffers: per step, the data
    # vector from pinned host memory, one iteration, the image back to pinned memory
    g_host = torch.from_numpy(g_np.astype(np.complex64)).pin_memory()
    v_host = torch.empty(C3_N, dtype=torch.complex64).pin_memory()
    barrier()
    t0.record(stream)
    for _ in range(K):
        s.set_g(g_host)
        s.iterate(1)
        s.v(out=v_host)
    t1.record(stream)
    barrier()
    e2e_s = max_over_ranks(t0.elapsed_time(t1) / 1e3, world, dev)

    # FP16 H: build the copy and its factors (timed), then K iterations in one launch
    t_f = time.perf_counter()
    s.use_fp16(True)
    torch.cuda.synchronize()
    setup16_ms = (time.perf_counter() - t_f) * 1e3
    info16 = s.info()
    alg16 = 2 * info16["h16_bytes"] + info16["factor_bytes"] + state_bytes(C3_BLOCKS, C3_N)
    for _ in range(max(args.warmup, 0)):
        s.iterate(1)
    barrier()
    t0.record(stream)
    s.iterate(K)
    t1.record(stream)
    barrier()
    us16 = t0.elapsed_time(t1) / K * 1e3
    s.use_fp16(False)
    if s.status() != 0:
        raise RuntimeError("device status after the FP16 timed region")

    us = timed_s / K * 1e6
    headline = {
        "complex64": {"us_per_iter": us, "iters_per_s": 1e6 / us, "alg_bytes_per_iter": alg,
                      "gbs": alg / us / 1e3, "frac": alg / us / 1e3 / peaks["hbm_gbs"],
                      "us_per_single_iteration_launch": single_us},
        "fp16_h": {"us_per_iter": us16, "iters_per_s": 1e6 / us16, "alg_bytes_per_iter": alg16,
                   "gbs": alg16 / us16 / 1e3, "frac": alg16 / us16 / 1e3 / peaks["hbm_gbs"],
                   "setup_ms": setup16_ms},
        "ctas": info["ctas"], "rows_per_stage": info["rows_per_stage"], "stages": info["stages"],
        "inputs_s": prep["inputs_s"], "setup_ms": prep["setup_ms"],
        "setup_gram_ms": info["setup_gram_ms"], "setup_factor_ms": info["setup_factor_ms"],
    }
    if vstar is not None:
        headline["schedules"] = config3_schedules(s, stream, barrier, vstar)
        if not args.no_time_to_tol:
            headline["time_to_tol"] = config3_time_to_tol(s, stream, barrier, vstar, prep["setup_ms"],
                                                          setup16_ms)
    s.close()
    torch.cuda.empty_cache()

    extra = {}
    if not args.no_cra:
        extra["cra_three_splits"] = cra_three_splits(pkg, stream, dev, barrier, peaks, K, args.warmup, rank)
    if not args.no_small:
        extra["small_256x4096"] = small_workload(pkg, stream, dev, barrier)
    if not args.no_batch:
        extra["batched_shared_h"] = batched_shared_h(pkg, stream, dev, barrier, make_problem(rank),
                                                     peaks=peaks, batch=args.batch)
    if not args.no_adjoint:
        extra["differentiable"] = differentiable(pkg, stream, dev, barrier)
    if not args.no_uneven:
        extra["uneven_problems"] = uneven_problems(pkg, stream, dev, barrier, peaks=peaks)
    if not args.no_direct:
        extra["direct_form"] = direct_form(pkg, stream, dev, barrier, peaks=peaks)
    if not args.no_sharded:
        extra["sharded_one_gpu"] = sharded_one_gpu(pkg, stream, dev, barrier, peaks)

    traffic = load_traffic()
    tr = traffic.get("c3") if traffic else None
    value = job_value(world, 1, K, total_s)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_s / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": CONFIG,
        "roofline": {"bound": "hbm", "achieved": alg / us / 1e3, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": alg / us / 1e3 / peaks["hbm_gbs"], "traffic": tr,
                     "peak_source": peaks["source"], "kernel": "admm::iterate_kernel",
                     "per": "iteration (achieved and traffic per iteration; one launch runs K iterations)",
                     "dram_frac": (tr / us / 1e3 / peaks["hbm_gbs"]) if tr else None},
        "e2e": {"value": job_value(world, 1, K, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": C3_M * 8, "d2h_bytes_per_step": C3_N * 8},
        "gpu_launches": 1,
        "clocks": clk,
        "headline": headline,
        "parallelism": "replicas" if world > 1 else "single GPU",
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main(argv=None) -> int:
    args = parse_args(argv)
    if args.cpu_sample_worker:
        cpu_sample_worker(args)
        return 0
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark: evolution steps/s of rho <- U rho U^dag for a Tavis-Cummings
system (arXiv 2403.06937, Eq. 6) on one GB300, through libtc's C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision bf16x3|tf32x3|tf32|fp64|ozaki]
                    [--workload n14|n15|n16|n12|n8|batch|grad|open14|open12]

One "step" is one pass of the step loop: X = U rho, rho' = X U^dag (Hermitian
half) and the observable row (populations, photon-number probabilities,
trace, purity, energy), plus the FP64 renormalisation when due.  H and U are
built once before timing (U in FP64, as every precision form requires).

Prints ONE JSON line on rank 0.  With N > 1 GPUs (torchrun) every rank runs
its own independent replica of the workload (the step does not shard);
value = all ranks' steps / max-over-ranks time.

--impl reference times the CPU oracle (test infrastructure, plain C) on the
host cores for the same workload, on a bounded sample of rows of the dense
step, extrapolated to steps/s.

Every line states its error against the oracle (the O-psi trajectory of the
workload; for the batch, every system's; for the gradient, the oracle's
forward-mode tangent and central differences).  n16 runs through the
host-buffer call with rho in page-locked host memory (U and the workspace
fill HBM), so its value is an end-to-end figure.
"""
from __future__ import annotations

import argparse
import math
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "evolution steps/s and complex-GEMM TFLOP/s at n=14 (FP64 vs split-BF16) at stated error"

# DRAM bytes (read + write) per launch of the dominant kernel, keyed by
# (precision, n): dram__bytes_read.sum + dram__bytes_write.sum averaged over
# the four launches (two of each product) of a one-pass ncu capture at
# n = 12 (1.484 GB), scaled to n = 14 by the N^3 units a launch processes;
# null for any other key.
NCU_TRAFFIC = {("bf16x3", 14): 1.484e9 * 64}


def _args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16x3", "tf32x3", "tf32", "fp64", "ozaki"], default="bf16x3")
    ap.add_argument("--workload", choices=["n14", "n15", "n16", "n12", "n8", "batch", "grad", "open14", "open12"],
                    default="n14",
                    help="n14 (default, the metric's workload), n12, n8; batch: 64 systems n=6..12 "
                         "(aggregate system-steps/s vs per-system sequential calls); grad: n=11 gradient")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the TF32 / TF32x3 / FP64 comparison forms")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--full", action="store_true",
                    help="also run the workload's whole run (500 steps at n=14) and state its error vs the oracle")
    ap.add_argument("--shapes", action="store_true",
                    help="batch workload: also time the batch in each tile shape, pinned")
    ap.add_argument("--batch-systems", type=int, default=64,
                    help="batch workload: the first K systems of the 64 (a smaller case for profiling)")
    ap.add_argument("--batch-steps", type=int, default=200, help="batch workload: steps")
    ap.add_argument("--no-tune", action="store_true", help="batch workload: no autotuning (default shapes)")
    ap.add_argument("--no-seq", action="store_true", help="batch workload: skip the per-system comparison")
    return ap.parse_args()


def _workload(name: str):
    return {"n14": W.config_n14, "n15": W.config_n15, "n12": W.config_n12, "n8": W.config_n8}[name]()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi sampled every 200 ms during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,clocks.mem")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, power, mem = [], [], set(), [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                    power.append(float(parts[2]))
                except ValueError:
                    continue
                try:
                    mem.append(float(parts[8]))
                except (ValueError, IndexError):
                    pass
                for nm, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_mhz_min": float(min(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": float(max(power)) if power else None,
                "mem_mhz_min": float(min(mem)) if mem else None, "mem_mhz_max": float(max(mem)) if mem else None}


# ------------------------------------------------------------------ peaks
def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "MEASURED_PEAKS.json"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _fp64_peak_live(torch):
    """cuBLAS DGEMM (torch.matmul float64, 4096^3) best of 3: the FP64 pipe's measured rate."""
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * 4096 ** 3 / (best * 1e-3) / 1e12


def _tf32_peak_live(torch, seconds: float = 2.0):
    """cuBLAS TF32 GEMM (torch.matmul float32 with TF32 allowed, 8192^3): the
    TF32 tensor pipe's measured rate, as a burst (best of 5) and sustained
    (back to back for `seconds`, as the kernels run inside a long step)."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        m = 8192
        a = torch.randn(m, m, dtype=torch.float32, device="cuda")
        b = torch.randn(m, m, dtype=torch.float32, device="cuda")
        c = torch.matmul(a, b)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        per = best * 1e-3
        reps = max(4, int(seconds / per))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        flop = 2.0 * m ** 3
        burst = flop / per / 1e12
        sustained = flop * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del a, b, c
        return burst, sustained
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


# ------------------------------------------------------------------ CPU oracle
def _cpu_sample(cfg, target_s: float, reps: int = 1):
    """Time the oracle's dense step (rows of rho' = U rho U^dag) on host cores.

    Returns (steps_per_s, cores, sample description).  U and rho are dense
    seeded synthetic matrices of the workload's size (the oracle's loops do
    the same work for any dense operands).
    """
    import oracle
    oracle.build()
    N = cfg.N
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    rng = np.random.default_rng(1234)
    U = (rng.random((N, N)) - 0.5) + 1j * (rng.random((N, N)) - 0.5)
    rho = (rng.random((N, N)) - 0.5) + 1j * (rng.random((N, N)) - 0.5)
    # calibrate: one row per core
    rows = cores
    t0 = time.perf_counter()
    oracle.dense_step(U, rho, rows=(0, rows))
    t1 = time.perf_counter() - t0
    per_row = t1 / rows
    rows = max(cores, int(target_s / max(per_row, 1e-9)) // cores * cores)
    rows = min(rows, N)
    times = []
    for r in range(reps):
        t0 = time.perf_counter()
        oracle.dense_step(U, rho, rows=(0, rows))
        times.append(time.perf_counter() - t0)
    t = float(np.median(times))
    steps_per_s = rows / (t * N)
    sample = ("oracle dense step (plain C loops, OpenMP over rows): rows 0..%d of rho' = U rho U^dag at N=%d, "
              "%.2f s per sample, extrapolated to whole steps (x %d/%d)" % (rows - 1, N, t, N, rows))
    return steps_per_s, cores, sample, t


# ------------------------------------------------------------------ reference arm
def run_reference(a, cfg, metric=METRIC, scale=1.0, scale_note="", workload=None):
    """The reference arm: the CPU oracle's dense step (the paper ships no code).

    Each of the W + K "steps" of this arm is one bounded sample of the
    workload's dense step: a block of rows of rho' = U rho U^dag, sized so the
    whole run ends within a few minutes.  `ms_per_step` is the wall time of
    one such sample, `steps` the number of samples timed, and `value` the
    whole dense steps per second they extrapolate to (`scale` converts a
    dense N x N step into the workload's step)."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    vals, secs, rows_list = [], [], []
    per_step_target = max(1.0, min(a.cpu_seconds, 150.0 / max(1, a.steps + a.warmup)))
    sample = cores = None
    for i in range(a.warmup + a.steps):
        v, cores, sample, t = _cpu_sample(cfg, per_step_target)
        if i >= a.warmup:
            vals.append(v * scale)
            secs.append(t)
    value = float(np.median(vals))
    t_sample = float(np.median(secs))
    frac = value / scale * t_sample       # fraction of one dense step a sample computes
    sample = sample + scale_note
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": "steps/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_sample, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "step_kind": ("each step of this arm is one bounded row sample of the dense step (%.4f of a whole "
                      "step, %.2f s); ms_per_step is a sample's wall time and value the whole steps/s "
                      "they extrapolate to" % (frac, t_sample)),
        "config": {"workload": workload or cfg.description, "dim": cfg.N,
                   "reference": "CPU oracle (no code ships with the paper)"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ replicas
def max_over_ranks(x: float, world: int) -> float:
    """Max of a per-rank float over all ranks (the one collective of the
    benchmark: the step itself is not sharded, every rank runs a replica)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(steps: int, world: int, max_ms: float) -> float:
    """Whole-job steps/s: every rank ran `steps` steps of its own replica."""
    return world * steps / (max_ms * 1e-3)


# ------------------------------------------------------------------ our arm
def _compulsory_bytes(prec, N):
    """Bytes one complex product Y = A B^H must move at least once: the A and B
    operand planes, and for the split forms the FP32 increment term read and
    the FP32 result plus its split planes written."""
    if prec == "fp64":
        return 3 * 16 * N * N
    if prec == "ozaki":
        # nine BF16 digit planes of U and of P read, the FP64 result written
        return (2 * 2 * 9 * 2 + 16) * N * N
    parts, pbytes = {"bf16x3": (3, 2), "tf32": (1, 4), "tf32x3": (2, 4)}[prec]
    planes = 2 * parts * pbytes
    return (3 * planes + 8 + 8) * N * N


def oz_pairs(N):
    """Digit-slice pairs per complex product of the FP64-emulated form: the
    library takes 8-bit digits for inner dimension K <= 1024, 7-bit for
    K <= 4096, else 6-bit (TC_OZ_BITS=6 forces 6-bit)."""
    K = max(N, 128)
    if os.environ.get("TC_OZ_BITS") == "6" or K > 4096:
        return 45
    return 28 if K <= 1024 else 36


def _sample_entries(torch, rho, count=20000, top=48, seed=5):
    """Indices (i, j) of a seeded random sample of rho's entries plus the
    top x top block on the largest diagonal entries, and rho's values there
    (gathered on the device, copied to the host)."""
    N = rho.shape[0]
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, N, size=(count, 2))
    big = torch.argsort(rho.diagonal().real.abs(), descending=True)[:min(top, N)].cpu().numpy()
    ii = np.concatenate([idx[:, 0], np.repeat(big, len(big))])
    jj = np.concatenate([idx[:, 1], np.tile(big, len(big))])
    vals = rho[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].cpu().numpy()
    return ii, jj, vals


def _drift(o, n, steps_done):
    return {"kind": "conserved quantities after %d steps" % steps_done,
            "trace": float(abs(o[-1, 2 * n + 2] - 1.0)),
            "purity": float(abs(o[-1, 2 * n + 3] - 1.0)),
            "energy_rel": float(abs(o[-1, 2 * n + 4] - o[0, 2 * n + 4]) / abs(o[0, 2 * n + 4]))}


def _time_form(tc, torch, U, n, params, prec, steps, warmup, renorm, stream, with_clocks=None):
    """W untimed steps, then K steps of one tc_evolve call timed with CUDA events.

    Also returns what the oracle comparison needs: the observable rows of the
    timed call (steps W..W+K) and a sample of rho's entries after step W+K."""
    N = 1 << n
    rho = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    rho[N - 1, N - 1] = 1.0
    work = torch.empty(tc.workspace_size(n, tc.PRECISIONS[prec], tc.TC_OP_EVOLVE), dtype=torch.uint8, device="cuda")
    if warmup:
        rho, _ = tc.evolve(U, rho, n, warmup, prec, renorm_every=renorm, params=params, inplace=True, work=work)
        tc.sync_status()
    torch.cuda.synchronize()
    # the timed region: one tc_evolve call of K steps (steps 2..K as one CUDA
    # graph); with K <= 2 there is no graph and the product launches are
    # bracketed by events in the same run
    inline = steps <= 2
    if inline:
        tc.timing_read()
        tc.timing_enable(True)
    launches0 = tc.launch_count()
    if with_clocks is not None:
        with_clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rho, obs = tc.evolve(U, rho, n, steps, prec, renorm_every=renorm, params=params, inplace=True, work=work)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = with_clocks.stop() if with_clocks is not None else None
    launches = tc.launch_count() - launches0
    tc.sync_status()
    ms = e0.elapsed_time(e1)
    o = obs.cpu().numpy()
    sample = _sample_entries(torch, rho)
    # the roofline of the product kernels: the same K steps again with an event
    # pair around every product launch (direct launches, no graph)
    if not inline:
        tc.timing_read()
        tc.timing_enable(True)
        tc.evolve(U, rho, n, steps, prec, renorm_every=renorm, params=params, inplace=True, work=work)
        torch.cuda.synchronize()
    tc.timing_enable(False)
    klaunch, kms, kflops = tc.timing_read()
    del work, rho
    return {"ms": ms, "launches": launches, "klaunch": klaunch, "kms": kms, "kflops": kflops, "clocks": ck,
            "drift": _drift(o, n, warmup + steps), "obs": o, "sample": sample, "first": warmup,
            "steps": steps}


def _full_run(tc, torch, U, n, params, prec, steps, renorm):
    """The workload's whole run (all its steps, renormalised as it states) in
    one tc_evolve call, for the error of the final result against the oracle."""
    N = 1 << n
    rho = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    rho[N - 1, N - 1] = 1.0
    t0 = time.perf_counter()
    rho, obs = tc.evolve(U, rho, n, steps, prec, renorm_every=renorm, params=params, inplace=True)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    tc.sync_status()
    o = obs.cpu().numpy()
    res = {"seconds": t, "drift": _drift(o, n, steps), "obs": o, "sample": _sample_entries(torch, rho),
           "first": 0, "steps": steps}
    del rho
    return res


def _oracle_trajectories(cfg, upto):
    """O-psi: the oracle's pure-state propagation of the workload from the
    all-excited state, the observable rows of every step up to max(upto) and
    psi after each step count in `upto`.  Returns (rows, {steps: psi}, s/step)."""
    import oracle
    oracle.build()
    marks = sorted(set(int(u) for u in upto))
    psi = W.all_excited_state(cfg.n)
    rows = [oracle.observables_pure(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, psi)]
    psis = {0: psi.copy()}
    done = 0
    t0 = time.perf_counter()
    for m in marks:
        if m > done:
            psi, ob = oracle.propagate(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, m - done, psi)
            rows.extend(ob[1:])
            done = m
        psis[m] = psi.copy()
    t = time.perf_counter() - t0
    return np.array(rows), psis, t / max(done, 1)


def _dicke_pm(cfg, steps):
    """Equal couplings only: P(m) of every step up to `steps` by the oracle's
    second route, the (n+1) x (n+1) Dicke tridiagonal of the symmetric
    subspace diagonalised (Jacobi) and evolved exactly; else None."""
    if not np.all(np.asarray(cfg.g) == cfg.g[0]):
        return None
    import oracle
    oracle.build()
    n = cfg.n
    w, V = oracle.jacobi_eig(oracle.dicke_matrix(n, float(cfg.g[0]), cfg.omega_a, cfg.omega_c))
    e0 = np.zeros(n + 1)
    e0[0] = 1.0
    c = V.T @ e0
    return np.array([np.abs(V @ (np.exp(-1j * w * cfg.dt * k) * c)) ** 2 for k in range(steps + 1)])


def _error_vs_oracle(r, n, rows, psis, dicke=None):
    """Max-abs error of a form's results against the oracle over the steps it
    ran: populations P_i, mean photon number <p>, photon-number
    probabilities P(m) (Eq. 13) and the sampled rho entries; with equal
    couplings also P(m) against the Dicke route."""
    o = r["obs"]
    first, k = r["first"], r["steps"]
    ref = rows[first:first + k + 1]
    ii, jj, vals = r["sample"]
    psi = psis[first + k]
    want = psi[ii] * psi[jj].conj()
    out = {"steps": "%d..%d" % (first, first + k),
           "populations": float(np.max(np.abs(o[:, :n] - ref[:, :n]))),
           "mean_photons": float(np.max(np.abs(o[:, n] - ref[:, n]))),
           "photon_number_probabilities": float(np.max(np.abs(o[:, n + 1:2 * n + 2] - ref[:, n + 1:2 * n + 2]))),
           "rho_sampled": float(np.max(np.abs(vals - want))),
           "rho_entries_sampled": int(len(ii))}
    if dicke is not None:
        out["photon_number_probabilities_vs_dicke"] = float(
            np.max(np.abs(o[:, n + 1:2 * n + 2] - dicke[first:first + k + 1])))
    return out


def run_ours(a, cfg):
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()

    n, N = cfg.n, cfg.N
    prec = a.precision
    params = tc.Params(n, list(map(float, cfg.g)), cfg.omega_a, cfg.omega_c)
    t_setup = time.perf_counter()
    U = tc.expm_model(params, cfg.dt)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    renorm = cfg.renorm_every
    stream = torch.cuda.current_stream()
    credited = 12.0 * N ** 3
    peaks, peak_src = _measured_peaks()

    def peak_of(p, fp64_peak=None, tf32_peak=None):
        if p == "fp64":
            return fp64_peak, "FP64: cuBLAS DGEMM 4096^3 measured live in this run (torch.matmul float64)"
        if p in ("tf32", "tf32x3"):
            if tf32_peak is not None:
                return tf32_peak[1], ("TF32: cuBLAS TF32 GEMM 8192^3 measured live in this run, sustained "
                                      "(back to back for 2 s; burst %.0f TFLOP/s)" % tf32_peak[0])
            return peaks["bf16_tflops_sustained"] / 2.0, \
                "TF32: %s bf16_tflops_sustained x 1/2 (nominal tf32:bf16 ratio)" % peak_src
        return peaks["bf16_tflops_sustained"], "BF16: %s bf16_tflops_sustained (kernel timed inside a long step)" % peak_src

    fp64_peak = _fp64_peak_live(torch) if (prec == "fp64" or not a.no_compare) else None
    tf32_peak = _tf32_peak_live(torch) if (prec in ("tf32", "tf32x3") or not a.no_compare) else None
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    r = _time_form(tc, torch, U, n, params, prec, a.steps, a.warmup, renorm if prec != "fp64" else 0, stream,
                   with_clocks=clocks)
    ms = max_over_ranks(r["ms"], world)
    value = replica_value(a.steps, world, ms)
    peak, peak_note = peak_of(prec, fp64_peak, tf32_peak)
    achieved = r["kflops"] / (r["kms"] * 1e-3) / 1e12 if r["kms"] > 0 else 0.0
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None, "traffic": NCU_TRAFFIC.get((prec, n)),
            "traffic_unit": "DRAM bytes per launch (ncu one-pass capture at n=12, scaled by N^3); compulsory "
                            "operand bytes per launch %.2e" % (_compulsory_bytes(prec, N)),
            "kernel": "complex GEMM (%s), %d launches timed, %.3f ms avg" % (prec, r["klaunch"],
                                                                             r["kms"] / max(r["klaunch"], 1)),
            "peak_source": peak_note,
            "algorithmic_flops_per_launch_avg": r["kflops"] / max(r["klaunch"], 1)}
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "bf16x3": "bf16", "tf32": "tf32", "tf32x3": "tf32", "ozaki": "bf16"}[prec],
        "data": "synthetic",
        "config": {"workload": cfg.description, "precision": prec, "dim": N,
                   "products_per_complex_product": {"fp64": 1, "bf16x3": 6, "tf32": 1, "tf32x3": 3, "ozaki": oz_pairs(N)}[prec],
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (U and rho are %d MiB each in complex128)" % (16 * N * N >> 20),
                   "setup_s": t_setup},
        "credited_tflops": credited * value / world / 1e12,
        "credited_flops_per_step": credited,
        "roofline": roof,
        "clocks": r["clocks"],
        "gpu_launches": r["launches"],
        "error": {"vs_oracle": None, "drift": r["drift"]},
    }
    forms = {prec: r}      # every timed form's results, for the oracle comparison

    if not a.no_e2e:
        # end to end through the public C ABI call with host buffers: every step copies
        # rho (pinned host) in, runs one step, copies rho and the observable rows back.
        rho_h = torch.zeros((N, N), dtype=torch.complex128, pin_memory=True)
        rho_h[N - 1, N - 1] = 1.0
        obs_h = torch.empty((2, 2 * n + 5), dtype=torch.float64, pin_memory=True)
        hw = torch.empty(tc.workspace_size(n, tc.PRECISIONS[prec], 16, 1), dtype=torch.uint8, device="cuda")
        tc.evolve_host(U, rho_h, n, 1, prec, params=params, obs_host=obs_h, work=hw)   # warm
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        calls, phases = [], []
        tc.phases_enable(True)     # event marks at the phase boundaries of each call (no extra sync)
        tc.phases_read()
        eclk = Clocks(local)
        eclk.start()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            tc0 = time.perf_counter()
            tc.evolve_host(U, rho_h, n, 1, prec, params=params, obs_host=obs_h, work=hw)
            calls.append(1e3 * (time.perf_counter() - tc0))
            phases.append(tc.phases_read())
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world)
        eck = eclk.stop()
        tc.phases_enable(False)
        marks = [m for m, _ in phases[0]] if phases and phases[0] else []
        line["e2e"] = {"value": world * a.steps / te, "unit": "steps/s", "h2d_bytes_per_step": 16 * N * N,
                       "d2h_bytes_per_step": 16 * N * N + 2 * (2 * n + 5) * 8,
                       "api": "tc_evolve_host (C ABI, pinned host rho, one step per call)",
                       "call_ms": [round(c, 1) for c in calls], "clocks": eck,
                       "phases": {"marks": marks,
                                  "ms_after_start": [[round(t, 1) for _, t in p] for p in phases]}}
        del rho_h, hw

    if not a.no_compare:
        # the other forms on the same workload: split-TF32, TF32 and one FP64 step
        others = {}
        for p2, k2, w2 in (("tf32x3", a.steps, a.warmup), ("tf32", a.steps, a.warmup), ("ozaki", 2, 1),
                           ("fp64", 1, 0)):
            if p2 == prec:
                continue
            if p2 == "fp64" and n >= 15:
                others["fp64"] = {"omitted": "one FP64 step takes about %.0f s at n=%d" % (credited / 1.1e12, n)}
                continue
            r2 = _time_form(tc, torch, U, n, params, p2, k2, w2, renorm if p2 != "fp64" else 0, stream)
            forms[p2] = r2
            v2 = k2 / (r2["ms"] * 1e-3)
            pk, pk_note = peak_of(p2, fp64_peak, tf32_peak)
            ach = r2["kflops"] / (r2["kms"] * 1e-3) / 1e12 if r2["kms"] > 0 else 0.0
            others[p2] = {"value": v2, "unit": "steps/s", "steps": k2, "warmup": w2,
                          "credited_tflops": credited * v2 / 1e12, "achieved_tflops": ach, "peak": pk,
                          "frac": ach / pk if pk else None, "peak_source": pk_note,
                          "error": {"vs_oracle": None, "drift": r2["drift"]}}
            if p2 == "ozaki":
                others[p2]["digit_pairs"] = oz_pairs(1 << n)
        line["other_forms"] = others
        if "value" in others.get("fp64", {}):
            line["speedup_vs_fp64"] = (value / world) / others["fp64"]["value"]
            if "value" in others.get("ozaki", {}):
                others["ozaki"]["speedup_vs_fp64"] = others["ozaki"]["value"] / others["fp64"]["value"]

    full = None
    if a.full:
        # the headline's whole run (all the workload's steps) for the error of its final result
        full = _full_run(tc, torch, U, n, params, prec, cfg.steps, renorm if prec != "fp64" else 0)
        line["full_run"] = {"steps": cfg.steps, "seconds": full["seconds"], "drift": full["drift"],
                            "error": {"vs_oracle": None}}

    if rank == 0 and not a.no_cpu:
        # CPU leg (rank 0, host cores): the like-for-like dense-step sample, then the
        # oracle's pure-state propagation (O-psi) of this workload, timed per step;
        # its trajectory is the reference every timed form's result is compared with.
        v, cores, sample, _ = _cpu_sample(cfg, a.cpu_seconds)
        upto = [f["first"] + f["steps"] for f in forms.values()]
        if full is not None:
            upto.append(full["steps"])
        rows, psis, per_step = _oracle_trajectories(cfg, upto)
        line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle", "sample": sample,
                                "oracle_pure_state": {"seconds_per_step": per_step,
                                                      "seconds_for_%d_steps" % cfg.steps: per_step * cfg.steps,
                                                      "threads": 1,
                                                      "what": "O-psi: psi <- e^{-iH dt} psi by the Taylor series to "
                                                              "convergence with the sparse H, plus one observable "
                                                              "row per step"}}
        dicke = _dicke_pm(cfg, max(upto))
        line["error"]["vs_oracle"] = _error_vs_oracle(forms[prec], n, rows, psis, dicke)
        for p2, f in forms.items():
            if p2 != prec and p2 in line.get("other_forms", {}):
                line["other_forms"][p2]["error"]["vs_oracle"] = _error_vs_oracle(f, n, rows, psis, dicke)
        if full is not None:
            line["full_run"]["error"]["vs_oracle"] = _error_vs_oracle(full, n, rows, psis, dicke)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def run_batch(a):
    """64 systems, n ~ U{6..12} (seed 2), 200 steps: one tc_batch_evolve vs per-system tc_evolve
    (--batch-systems / --batch-steps: the first K systems, S steps)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    prec = a.precision
    cfgs = W.config_batch(steps=a.batch_steps if prec != "fp64" else 2)[:max(1, min(64, a.batch_systems))]
    steps = cfgs[0].steps
    Us, rhos, ps = [], [], []
    for c in cfgs:
        p = tc.Params(c.n, list(map(float, c.g)), c.omega_a, c.omega_c)
        Us.append(tc.expm(tc.build_hamiltonian(p), c.n, c.dt))
        r = torch.zeros((c.N, c.N), dtype=torch.complex128, device="cuda")
        r[-1, -1] = 1.0
        rhos.append(r)
        ps.append(p)
    # the autotuner picks tile shape, raster group and ring depth for every n of the batch (the
    # per-system calls use them), and the batch's own shape and group (tc_batch_autotune)
    nmax = max(c.n for c in cfgs)
    tuned, batch_choice = {}, None
    if prec not in ("fp64", "ozaki") and not a.no_tune:
        for n in sorted({c.n for c in cfgs}):
            tuned[n] = tc.autotune(n, prec)
        batch_choice = tc.batch_autotune([c.n for c in cfgs], prec)
    tc.batch_evolve(Us, rhos, 1, prec, params=ps)          # warm (attributes, modules)
    torch.cuda.synchronize()
    l0 = tc.launch_count()
    t0 = time.perf_counter()
    out, obs = tc.batch_evolve(Us, rhos, steps, prec, params=ps)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    launches = tc.launch_count() - l0
    # the same batch in each tile shape, pinned (the speed the tuner chose from)
    shapes = {}
    if batch_choice and a.shapes:
        # every shape pinned for this batch (the tuner's group), then the tuned choice put back
        for name, code in (("single", 1), ("pair32", 2), ("pair_wide", 3)):
            tc.batch_autotune_set([c.n for c in cfgs], prec, batch_choice["tc_group"], code)
            tc.batch_evolve(Us, rhos, 1, prec, params=ps)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tc.batch_evolve(Us, rhos, steps, prec, params=ps)
            torch.cuda.synchronize()
            shapes[name] = len(cfgs) * steps / (time.perf_counter() - t0)
        tc.batch_autotune_set([c.n for c in cfgs], prec, batch_choice["tc_group"], batch_choice["tc_shape"])
    ts = None
    if not a.no_seq:
        t0 = time.perf_counter()
        for U, r, p in zip(Us, rhos, ps):
            tc.evolve(U, r, p.n, steps, prec, params=p)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
    credited = sum(12.0 * c.N ** 3 for c in cfgs) * steps
    value = len(cfgs) * steps / tb
    line = {"metric": "batched evolution: aggregate system-steps/s (%d systems, n=6..12)" % len(cfgs), "value": value,
            "unit": "system-steps/s", "n_gpus": 1, "steps": steps, "warmup": 1, "ms_per_step": 1e3 * tb / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x3": "bf16", "tf32": "tf32", "tf32x3": "tf32", "ozaki": "bf16"}[prec],
            "data": "synthetic",
            "config": {"workload": "%d systems, n ~ U{6..12} seed 2, own g_i ~ U[0.005,0.015], dt=0.05, %d steps"
                       % (len(cfgs), steps), "precision": prec, "ns": [c.n for c in cfgs]},
            "credited_tflops": credited / tb / 1e12,
            "sequential": None if ts is None else {"value": len(cfgs) * steps / ts, "unit": "system-steps/s",
                                                   "api": "tc_evolve per system, one after another"},
            "speedup_vs_sequential": None if ts is None else ts / tb, "gpu_launches": launches}
    if batch_choice:
        names = {0: "auto", 1: "single", 2: "pair32", 3: "pair_wide"}
        line["config"]["tile_shape"] = names[batch_choice["tc_shape"]]
        line["config"]["raster_group"] = batch_choice["tc_group"]
        line["config"]["tuning"] = "tc_batch_autotune (batch); tc_autotune per n (the per-system calls)"
        line["tuned_per_n"] = {str(n): names[t["tc_shape"]] for n, t in tuned.items()}
    if shapes:
        line["by_shape"] = shapes
    if not a.no_cpu and obs is not None:
        # the stated error: every system's observable rows (all steps) against the oracle's
        # pure-state propagation of that system (O-psi)
        import oracle
        oracle.build()
        worst = {"populations": 0.0, "mean_photons": 0.0, "photon_number_probabilities": 0.0}
        t0 = time.perf_counter()
        for c, ob in zip(cfgs, obs):
            n = c.n
            _, ref = oracle.propagate(n, c.g, c.omega_a, c.omega_c, c.dt, steps, W.all_excited_state(n))
            o = ob.cpu().numpy()
            worst["populations"] = max(worst["populations"], float(np.max(np.abs(o[:, :n] - ref[:, :n]))))
            worst["mean_photons"] = max(worst["mean_photons"], float(np.max(np.abs(o[:, n] - ref[:, n]))))
            worst["photon_number_probabilities"] = max(
                worst["photon_number_probabilities"],
                float(np.max(np.abs(o[:, n + 1:2 * n + 2] - ref[:, n + 1:2 * n + 2]))))
        line["error"] = {"vs_oracle": dict(worst, systems=len(cfgs), steps="0..%d" % steps,
                                           oracle_seconds=time.perf_counter() - t0)}
    print(json.dumps(line), flush=True)
    return 0


def run_grad(a):
    """n = 11, 400 steps, checkpoints every 20: wall time of tc_evolve_backward (FP64)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    cfg = W.config_n11_grad()
    n, N = cfg.n, cfg.N
    p = tc.Params(n, list(map(float, cfg.g)), cfg.omega_a, cfg.omega_c)
    U = tc.expm(tc.build_hamiltonian(p), n, cfg.dt)
    rho0 = torch.zeros((N, N), dtype=torch.complex128, device="cuda")
    rho0[-1, -1] = 1.0
    s = torch.arange(N, device="cuda")
    O = ((s >> (n - cfg.loss_atom)) & 1).to(torch.float64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grad, loss = tc.evolve_backward(p, cfg.dt, cfg.steps, rho0, U, O, ckpt_every=cfg.ckpt_every,
                                    precision="ozaki" if a.precision == "ozaki" else "fp64")
    t = time.perf_counter() - t0
    # FP64 products: forward 12N^3 + recompute 12N^3 + Lambda 12N^3 + W 8N^3 per step
    flops = cfg.steps * 44.0 * N ** 3
    gprec = a.precision if a.precision in ("fp64", "ozaki") else "fp64"
    line = {"metric": "gradient wall time, n=11, 400 steps (FP64 adjoint + Frechet)", "value": t, "unit": "s",
            "n_gpus": 1, "steps": cfg.steps, "warmup": 0, "ms_per_step": 1e3 * t / cfg.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.description,
                       "products": "FP64 DMMA" if gprec == "fp64" else "FP64 emulated on the BF16 tensor cores"},
            "loss": loss, "grad": grad.tolist(), "fp64_tflops": flops / t / 1e12}
    if not a.no_cpu:
        # the stated errors: against the oracle's forward-mode tangent (all 13 components) and
        # central differences of the oracle's forward run (h = 1e-6; g_1, g_6 and omega_a)
        import oracle
        oracle.build()
        Od = O.cpu().numpy()
        psi0 = W.all_excited_state(n)
        t0 = time.perf_counter()
        ref = oracle.grad_forward(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, cfg.steps, psi0, Od)
        t_tan = time.perf_counter() - t0
        g_np = np.asarray(grad.tolist())
        h = 1e-6

        def L(g_, wa_, wc_):
            q, _ = oracle.propagate(n, g_, wa_, wc_, cfg.dt, cfg.steps, psi0, observe=False)
            return float(np.real(np.vdot(q, Od * q)))

        fd = {}
        for j in (0, 5):
            gp, gm = np.array(cfg.g, dtype=float), np.array(cfg.g, dtype=float)
            gp[j] += h
            gm[j] -= h
            fd[j] = (L(gp, cfg.omega_a, cfg.omega_c) - L(gm, cfg.omega_a, cfg.omega_c)) / (2 * h)
        fd[n] = (L(cfg.g, cfg.omega_a + h, cfg.omega_c) - L(cfg.g, cfg.omega_a - h, cfg.omega_c)) / (2 * h)
        scale = max(abs(v) for v in fd.values())
        line["error"] = {
            "vs_oracle_tangent": float(np.max(np.abs(g_np - ref)) / np.max(np.abs(ref))),
            "vs_central_differences": float(max(abs(g_np[j] - v) / max(abs(v), scale) for j, v in fd.items())),
            "fd": {"h": h, "components": ["g_1", "g_6", "omega_a"]},
            "oracle_tangent_seconds": t_tan}
    print(json.dumps(line), flush=True)
    return 0


def run_open(a):
    """Open system (Eq. 5 with photon leakage): split steps of tc_lindblad_evolve on the excitation blocks."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    n = int(a.workload[4:])
    cfg = W.config_open(n)
    prec = a.precision
    p = tc.Params(n, list(map(float, cfg.g)), cfg.omega_a, cfg.omega_c)
    lay = tc.lindblad_layout(n)
    work = torch.empty(tc.workspace_size(n, tc.PRECISIONS[prec], tc._abi.TC_OP_LINDBLAD), dtype=torch.uint8,
                       device="cuda")
    t_setup = time.perf_counter()
    U = tc.lindblad_propagators(p, cfg.dt, work=work)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    rho = torch.zeros(lay.total, dtype=torch.complex128, device="cuda")
    j = lay.basis.index((1 << n) - 1)
    lay.blocks(rho)[n][j, j] = 1.0
    stream = torch.cuda.current_stream()
    renorm = cfg.renorm_every if prec != "fp64" else 0
    if a.warmup:
        tc.lindblad_evolve(p, cfg.kappa, cfg.dt, U, rho, a.warmup, prec, renorm_every=renorm, inplace=True, work=work)
    torch.cuda.synchronize()
    l0 = tc.launch_count()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rho, obs = tc.lindblad_evolve(p, cfg.kappa, cfg.dt, U, rho, a.steps, prec, renorm_every=renorm, inplace=True,
                                  work=work)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    launches = tc.launch_count() - l0
    tc.sync_status()
    ms = e0.elapsed_time(e1)
    # roofline of the block GEMM: the same steps again with event pairs around each product launch
    tc.timing_read()
    tc.timing_enable(True)
    tc.lindblad_evolve(p, cfg.kappa, cfg.dt, U, rho, a.steps, prec, renorm_every=renorm, inplace=True, work=work,
                       observe=False)
    torch.cuda.synchronize()
    tc.timing_enable(False)
    klaunch, kms, kflops = tc.timing_read()
    o = obs.cpu().numpy()
    credited = sum(12.0 * d ** 3 for d in lay.dims)
    peaks, peak_src = _measured_peaks()
    peak = peaks["bf16_tflops_sustained"] if prec in ("bf16x3", "ozaki") else (
        _tf32_peak_live(torch)[1] if prec in ("tf32", "tf32x3") else _fp64_peak_live(torch))
    achieved = kflops / (kms * 1e-3) / 1e12 if kms > 0 else 0.0
    value = a.steps / (ms * 1e-3)
    line = {"metric": "open-system split steps/s (Eq. 5 with photon leakage)", "value": value, "unit": "steps/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "bf16x3": "bf16", "tf32": "tf32", "tf32x3": "tf32", "ozaki": "bf16"}[prec],
            "data": "synthetic",
            "config": {"workload": cfg.description, "precision": prec, "blocks": lay.dims,
                       "state_elements": lay.total, "setup_s": t_setup,
                       "l2": "inputs larger than L2 (packed state %d MiB in complex128)" % (16 * lay.total >> 20)},
            "credited_flops_per_step": credited, "credited_tflops": credited * value / 1e12,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if peak else None, "traffic": None,
                         "kernel": "batched complex GEMM over the excitation blocks (%s), %d launches, %.3f ms avg"
                                   % (prec, klaunch, kms / max(klaunch, 1)),
                         "peak_source": peak_src if prec in ("bf16x3", "ozaki") else (
                             "TF32: cuBLAS TF32 GEMM 8192^3 measured live in this run, sustained"
                             if prec in ("tf32", "tf32x3") else "FP64: cuBLAS DGEMM 4096^3 measured live")},
            "clocks": ck, "gpu_launches": launches,
            "error": {"kind": "conserved total trace after %d steps (oracle-free)" % (a.warmup + a.steps),
                      "trace": float(abs(o[-1, 2 * n + 2] - 1.0)),
                      "mean_photons": float(o[-1, n]), "excitation": float(o[-1, :n].sum() + o[-1, n])}}
    if not a.no_e2e:
        # end to end: the packed state from pinned host memory, one split step, the state and its row back
        rho_h = torch.empty(lay.total, dtype=torch.complex128, pin_memory=True)
        rho_h.copy_(rho)
        obs_h = torch.empty((2, 2 * n + 5), dtype=torch.float64, pin_memory=True)
        k = max(1, min(a.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            rho.copy_(rho_h, non_blocking=True)
            rho, ob = tc.lindblad_evolve(p, cfg.kappa, cfg.dt, U, rho, 1, prec, inplace=True, work=work)
            rho_h.copy_(rho, non_blocking=True)
            obs_h.copy_(ob, non_blocking=True)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        line["e2e"] = {"value": k / te, "unit": "steps/s", "h2d_bytes_per_step": 16 * lay.total,
                       "d2h_bytes_per_step": 16 * lay.total + obs_h.numel() * 8,
                       "api": "tc_lindblad_evolve (C ABI) with the packed state copied from and to pinned host memory"}
    if not a.no_cpu:
        v, cores, sample, _ = _cpu_sample(W.config_n14() if n == 14 else W.config_n12(), a.cpu_seconds)
        scale = (1 << n) ** 3 / sum(d ** 3 for d in lay.dims)
        line["cpu_baseline"] = {"value": v * scale, "unit": "steps/s", "cores": cores, "kind": "oracle",
                                "sample": sample + "; scaled by N^3 / sum_k d_k^3 = %.3f to the block products "
                                                   "(the damping pass is O(sum d_k^2))" % scale}
    print(json.dumps(line), flush=True)
    return 0


def run_n16(a):
    """n = 16 (dim 65536): split-BF16 steps through the host-buffer call with rho in
    page-locked host memory (the only arrangement in which U and the workspace fit
    in HBM), so `value` and `e2e` are the same measurement; the product launches
    are timed with events for the roofline; the error is against O-psi."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2403_06937_gb300 as tc
    tc.device_check()
    cfg = W.config_n16()
    n, N = cfg.n, cfg.N
    steps = max(1, min(a.steps, 4))
    prec = a.precision if a.precision in ("bf16x3", "tf32x3", "tf32") else "bf16x3"
    p = tc.Params(n, list(map(float, cfg.g)), cfg.omega_a, cfg.omega_c)
    t0 = time.perf_counter()
    U = tc.expm_model(p, cfg.dt)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    torch.cuda.empty_cache()
    rho = torch.empty((N, N), dtype=torch.complex128, pin_memory=True)
    rho.zero_()
    rho[-1, -1] = 1.0
    obs = torch.empty((steps + 1, tc.obs_stride(n)), dtype=torch.float64, pin_memory=True)
    work = torch.empty(tc.workspace_size(n, tc.PRECISIONS[prec], tc._abi.TC_OP_EVOLVE_HOST_PINNED, steps),
                       dtype=torch.uint8, device="cuda")
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    tc.timing_read()
    tc.timing_enable(True)
    t0 = time.perf_counter()
    tc.evolve_host(U, rho, n, steps, prec, renorm_every=cfg.renorm_every, params=p, obs_host=obs, work=work)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    tc.timing_enable(False)
    ck = clocks.stop()
    klaunch, kms, kflops = tc.timing_read()
    del U, work
    torch.cuda.empty_cache()
    peaks, peak_src = _measured_peaks()
    peak = peaks["bf16_tflops_sustained"] if prec == "bf16x3" else _tf32_peak_live(torch)[1]
    achieved = kflops / (kms * 1e-3) / 1e12 if kms > 0 else 0.0
    value = steps / sec
    h2d = d2h = 16 * N * N
    line = {"metric": "evolution steps/s at n=16 through the host-buffer call (rho in page-locked host memory)",
            "value": value, "unit": "steps/s", "n_gpus": 1, "steps": steps, "warmup": 0,
            "ms_per_step": 1e3 * sec / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16x3": "bf16", "tf32": "tf32", "tf32x3": "tf32"}[prec], "data": "synthetic",
            "config": {"workload": cfg.description, "precision": prec, "dim": N,
                       "rho": "page-locked host memory, read and written by the SMs (no device copy)",
                       "setup_s": t_setup},
            "credited_tflops": 12.0 * N ** 3 * steps / sec / 1e12,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if peak else None, "traffic": None,
                         "kernel": "complex GEMM (%s), %d launches, %.1f ms avg" % (prec, klaunch,
                                                                                   kms / max(klaunch, 1)),
                         "peak_source": peak_src if prec == "bf16x3" else "TF32: cuBLAS TF32 GEMM measured live",
                         "note": "the peak is cuBLAS on random operands under the power cap; the sparse early "
                                 "steps of this workload draw less power, so the clock can hold its maximum "
                                 "(see clocks) and the fraction exceed 1"},
            "clocks": ck,
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": h2d // steps,
                    "d2h_bytes_per_step": d2h // steps,
                    "api": "tc_evolve_host (C ABI, page-locked host rho); the same measurement as value"}}
    if not a.no_cpu:
        import oracle
        oracle.build()
        psi, oobs = oracle.propagate(n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, steps, W.all_excited_state(n))
        o = obs.numpy()
        rng = np.random.default_rng(16)
        top = np.argsort(-np.abs(psi))[:48]
        ii = np.concatenate([rng.integers(0, N, 20000), np.repeat(top, len(top))])
        jj = np.concatenate([rng.integers(0, N, 20000), np.tile(top, len(top))])
        got = rho[torch.from_numpy(ii), torch.from_numpy(jj)].numpy()
        line["error"] = {"vs_oracle": {
            "steps": "0..%d" % steps,
            "populations": float(np.max(np.abs(o[:, :n] - oobs[:, :n]))),
            "mean_photons": float(np.max(np.abs(o[:, n] - oobs[:, n]))),
            "photon_number_probabilities": float(np.max(np.abs(o[:, n + 1:2 * n + 2] - oobs[:, n + 1:2 * n + 2]))),
            "rho_sampled": float(np.max(np.abs(got - psi[ii] * psi[jj].conj()))),
            "rho_entries_sampled": int(len(ii))}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = _args()
    if a.workload == "n16":
        if a.impl == "reference":
            if _dist()[0] == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the n16 workload has no CPU-oracle arm (one "
                                  "dense oracle step at dim 65536 would take hours); O-psi states its error"}),
                      flush=True)
            return 0
        return run_n16(a)
    if a.impl == "reference" and a.workload in ("batch", "grad"):
        if _dist()[0] == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the %s workload has no CPU-oracle arm; the oracle "
                              "is timed on the n8/n12/n14/n15 and open workloads" % a.workload}), flush=True)
        return 0
    if a.impl == "reference" and a.workload.startswith("open"):
        n = int(a.workload[4:])
        dims = [sum(math.comb(n, j) for j in range(k + 1)) for k in range(n + 1)]
        scale = (1 << n) ** 3 / sum(d ** 3 for d in dims)
        return run_reference(a, W.config_n14() if n == 14 else W.config_n12(),
                             metric="open-system split steps/s (Eq. 5 with photon leakage)", scale=scale,
                             scale_note="; scaled by N^3 / sum_k d_k^3 = %.3f to the block products of the "
                                        "open-system step" % scale, workload=W.config_open(n).description)
    if a.workload == "batch":
        return run_batch(a)
    if a.workload.startswith("open"):
        return run_open(a)
    if a.workload == "grad":
        return run_grad(a)
    cfg = _workload(a.workload)
    if a.impl == "reference":
        return run_reference(a, cfg)
    return run_ours(a, cfg)


if __name__ == "__main__":
    sys.exit(main())

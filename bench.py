"""Benchmark: QAOA adjoint-gradient evaluations per second on GB300.

Default workload (one unit = one gradient of <C> with respect to all 2p
angles, forward + adjoint sweep): Sherrington-Kirkpatrick cost on n = 28
qubits (2^28 complex64 amplitudes, 2 GiB state), transverse-field mixer,
p = 8 rounds, per-round state checkpoints, J_ij ~ N(0,1) from the seeded
generator.  The state (2 GiB) is larger than L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is measured on the device with CUDA
events around K steps of the batched entry point (device-resident angles and
results).  `e2e` times the host-pointer entry point qaoa_gradient (angles
uploaded from pinned host memory, <C> and the gradient read back every step).
`roofline` divides the dominant kernel's algorithmic bytes by its CUDA-event
time inside the timed region.  `cpu_baseline` times the CPU oracle on the host
cores on one round of the same workload (scaled to the p-round unit).
With --impl reference the CPU oracle is the timed arm.  Under torchrun each
rank runs its own replica of the workload (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = 2  # index into qaoa_inputs.WORKLOADS: SK n=28, p=8, gradient
METRIC = "QAOA grad evals/s (fwd+adjoint) n=28 p=8 & batched n=20; HBM GB/s vs peak"
UNIT = "grad/s"


# ------------------------------------------------------------------ helpers

def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def aggregate(local_seconds: float, local_units: int, world: int, reduce_max=None, reduce_sum=None):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    t = reduce_max(local_seconds) if reduce_max else local_seconds
    u = reduce_sum(local_units) if reduce_sum else local_units
    return u / t, t, u


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(family: str):
    """ncu DRAM bytes per launch of a kernel family, if the committed capture
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(family)
    if not ent:
        return None
    import hashlib

    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != ent.get("source_sha"):
        return None
    return ent.get("dram_bytes_per_launch_full_size")


# ------------------------------------------------------------- CPU oracle

def oracle_sample(threads: int | None = None):
    """Time the CPU oracle on one round (p=1) of the workload at full n and
    scale to the p-round unit.  Returns (grad/s, seconds of the sample, cores)."""
    import oracle
    from qaoa_inputs import workload_instance

    oracle.build()
    if threads:
        oracle.set_threads(threads)
    w = workload_instance(WORKLOAD)
    n, p = w["spec"]["n"], w["spec"]["p"]
    cost = oracle.cost_sk(n, w["J"].astype(np.float64))
    a = w["angles"][0]
    one_round = np.array([a[0], a[p]])

    def run():
        t = time.perf_counter()
        oracle.qaoa_gradient(n, cost, one_round)
        return time.perf_counter() - t

    return run, p, oracle.get_threads(), n


# ---------------------------------------------------------------- GPU arm

def gpu_arm(args, ws, rank, local):
    import torch

    import paper_2312_06451_gb300 as qg
    from qaoa_inputs import workload_instance

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod

        dist_mod.init_process_group("nccl")
        dist = dist_mod
    w = workload_instance(WORKLOAD, n_sets=args.steps + args.warmup)
    if args.n:
        from qaoa_inputs import BASE_SEED, sk_couplings

        w["spec"]["n"] = args.n
        w["spec"]["name"] = f"sk{args.n}_p8_grad"
        w["J"] = sk_couplings(args.n, BASE_SEED + WORKLOAD)
    n, p = w["spec"]["n"], w["spec"]["p"]
    ctx = qg.Context(local)
    cost = ctx.cost_precompute("sk", n, J=w["J"], dtype=torch.float32)
    mixer = qg.XMixer(n)
    dev = f"cuda:{local}"
    angles_all = torch.from_numpy(w["angles"]).to(dev)
    ang = angles_all[0:1].clone()
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    G = torch.zeros(1, 2 * p, dtype=torch.float64, device=dev)
    job = [{"cost": cost, "mixer": mixer, "angles": ang, "E": E, "grad": G}]
    stream = torch.cuda.current_stream(local)

    def step(i):
        ang.copy_(angles_all[i:i + 1], non_blocking=True)
        ctx.expectation_batched(job, want_grad=True)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ctx.reset_stats()
    ctx.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    ctx.set_profiling(False)
    stats = ctx.kernel_stats()
    clk = clocks.stop()

    def rmax(v):
        if not dist:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()

    def rsum(v):
        if not dist:
            return v
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return int(t.item())

    value, tmax, units = aggregate(ms / 1e3, args.steps, ws, rmax, rsum)
    grad_last = G.cpu().numpy()[0]

    # end to end through the host-pointer API: angles from pinned host memory,
    # results read back, every step
    pinned = torch.from_numpy(w["angles"]).pin_memory()
    for i in range(2):
        ctx.gradient(cost, mixer, pinned[i].numpy())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        Eh, gh = ctx.gradient(cost, mixer, pinned[args.warmup + i].numpy())
    torch.cuda.synchronize()
    e2e_s = rmax(time.perf_counter() - t0)
    e2e_value = rsum(args.steps) / e2e_s

    # dominant kernel family by time inside the timed region
    fam = max((k for k in stats if stats[k]["launches"]), key=lambda k: stats[k]["total_ms"])
    st = stats[fam]
    peaks = measured_peaks()
    per_launch_bytes = st["algo_bytes"] / st["launches"]
    per_launch_ms = st["total_ms"] / st["launches"]
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["spec"]["name"], "problem": "SK, J_ij~N(0,1) on 2^-20 grid",
                       "n": n, "p": p, "mixer": "X (transverse field)", "state": "complex64",
                       "ckpt": "per-round state checkpoints", "angle_sets_per_step": 1,
                       "units_per_rank": args.steps,
                       "l2": f"state {2 ** n * 8 / 2 ** 30:.2f} GiB vs 129 MB L2; no flush",
                       "parallelism": f"replicas x{ws}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * 2 * p,
                    "d2h_bytes_per_step": 8 * (2 * p + 1)},
            "roofline": {"bound": "hbm", "kernel": fam, "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                         "peak_source": peaks["source"], "traffic": traffic_for(fam),
                         "algo_bytes_per_launch": per_launch_bytes, "launch_ms": per_launch_ms},
            "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4),
                            "GBps": round(v["algo_bytes"] / v["total_ms"] / 1e6, 1) if v["total_ms"] else None}
                        for k, v in stats.items() if v["launches"]},
            "gpu_launches": launches,
            "clocks": clk,
            "result_check": {"E_last": float(E.item()), "grad_norm_last": float(np.linalg.norm(grad_last)),
                             "e2e_E_last": Eh},
        }
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None,
                    help="override the qubit count (small cases for profiler captures)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        # The reference arm is the CPU oracle on the host cores (rank 0 only).
        if rank != 0:
            return
        run, p, cores, n = oracle_sample()
        for _ in range(args.warmup):
            run()
        ts = [run() for _ in range(args.steps)]
        t_round = sum(ts) / len(ts)
        value = 1.0 / (t_round * p)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_round * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "sk28_p8_grad", "n": n, "p": p, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: oracle gradient of one round (p=1) at n={n}, "
                                       f"scaled x{p} to the p={p} unit"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return

    out = gpu_arm(args, ws, rank, local)
    if rank == 0 and out is not None:
        if ws == 1 and not args.no_cpu_baseline:
            run, p, cores, n = oracle_sample()
            ts = [run()]
            if ts[0] < 8.0:
                ts.append(run())
            t_round = min(ts)
            out["cpu_baseline"] = {"value": 1.0 / (t_round * p), "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": f"oracle gradient of one round (p=1) at n={n}, best of "
                                             f"{len(ts)}, scaled x{p} to the p={p} unit"}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

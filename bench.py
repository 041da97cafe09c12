"""Benchmark: QAOA adjoint-gradient evaluations per second on GB300.

Default workload (one unit = one gradient of <C> with respect to all 2p
angles, forward + adjoint sweep): Sherrington-Kirkpatrick cost on n = 28
qubits (2^28 complex64 amplitudes, 2 GiB state), transverse-field mixer,
p = 8 rounds, per-pass state checkpoints, J_ij ~ N(0,1) from the seeded
generator.  The state (2 GiB) is larger than L2, so no flush is needed
between steps.  Two sub-records ride on the default line: `batched`, the
uneven 512-instance batch (n = 14..22, p = 6, 4 angle sets each) replayed from
a captured CUDA graph, and `grover`, the same n = 28 workload with the Grover
mixer applied as a rank-one update.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is measured on the device with CUDA
events around K steps of the batched entry point (device-resident angles and
results).  `e2e` times the same evaluation end to end through the host-buffer
batched entry point (qaoa_expectation_batched_host): angles copied in from
pinned host memory and <C> and the gradients read back to the host, every step.
`roofline` divides the dominant kernel's algorithmic bytes by its CUDA-event
time inside the timed region.  `cpu_baseline` times the CPU oracle on the host
cores on one round of the same workload (scaled to the p-round unit).
With --impl reference the CPU oracle is the timed arm.  Under torchrun each
rank runs its own replica of the workload (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import math
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


def gemm_peak(gemm: str):
    """Denominator of a contraction's roofline.  CUDA-core fp32: 152 SMs x 128
    FP32 lanes x 2 flop x 2070 MHz (unit counts and maximum clock).  TF32 /
    split-precision tensor paths: the measured bf16 dense peak x the nominal
    tf32 / bf16 ratio (1.1 / 2.25)."""
    if gemm == "fp32":
        return {"bound": "alu", "peak": 152 * 128 * 2 * 2.070e9 / 1e12, "source": "derived: 152 SM x 128 lanes x 2 x 2.07 GHz"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16 = 1901.6
    src = "fallback"
    if os.path.exists(path):
        with open(path) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        src = "measured"
    return {"bound": "tensor", "peak": bf16 * 1.1 / 2.25, "source": f"{src} bf16 burst x 1.1/2.25 (tf32)"}


def reducers(dist, device):
    """Max and sum over ranks of a host scalar (identity without a process
    group).  `device` is where the one-element tensor lives: the rank's GPU
    under NCCL, "cpu" under gloo."""
    import torch

    def rmax(v):
        if not dist:
            return v
        t = torch.tensor([float(v)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()

    def rsum(v):
        if not dist:
            return v
        t = torch.tensor([float(v)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return int(round(t.item()))

    return rmax, rsum


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


def traffic_for(family: str, workload: str):
    """ncu DRAM bytes per launch of a kernel family on this workload, if the
    committed capture was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ent = d.get(family)
    if not isinstance(ent, dict) or ent.get("workload") != workload:
        return None
    import hashlib

    src = os.path.join(ROOT, ent["source"])
    if not os.path.exists(src):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != ent.get("source_sha"):
        return None
    return ent.get("dram_bytes_per_launch_full_size")


def headline_config(n, p):
    """Workload description of the headline line (the same for both arms)."""
    return {"workload": "sk28_p8_grad", "problem": "SK, J_ij~N(0,1) on 2^-20 grid", "n": n, "p": p,
            "mixer": "X (transverse field)", "angle_sets_per_step": 1, "cost_dtype": "f32",
            "l2": f"state {2 ** n * 8 / 2 ** 30:.2f} GiB per set vs 129 MB L2; no flush"}


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


# ------------------------------------------------------------ workloads

class Workload:
    """Device-resident inputs of one benchmark workload and how to step it.

    A step evaluates `units` angle sets (gradients, or expectations when
    `grad` is False) through the batched entry point; angles for each step are
    copied into the job buffers from a device pool first (a 2p-double copy per
    set, so every step evaluates fresh angles)."""

    def __init__(self, qg, ctx, idx, dev, pool_steps, n_override=None, gemm="fp32", mixer="x", eig_cache=None,
                 eig_form="blocks"):
        import torch

        from qaoa_inputs import BASE_SEED, sk_couplings, uneven_batch_recipe, uniform_angles, workload_instance

        self.idx = idx
        self.ctx = ctx
        self.qg = qg
        self.dev = dev
        from qaoa_inputs import WORKLOADS

        spec = dict(WORKLOADS[idx])
        self.p = p = spec["p"]
        self.jobs = []
        self.pools = []
        if idx == 4:
            w = workload_instance(4, n_sets=spec["n_sets"] * pool_steps)
            n, k = spec["n"], spec["k"]
            self.grad = True
            cost = ctx.cost_precompute("dks", n, edges=w["edges"], k=k, dtype=torch.uint8)
            t0 = time.perf_counter()
            xy = "clique" if mixer == "clique" else "ring"
            self.eig_form = eig_form
            if eig_form == "blocks":
                mixer = qg.xy_sym_mixer(ctx, xy, n, k, precision=gemm, cache_file=eig_cache)
            else:
                mixer = qg.xy_eigen_mixer(ctx, xy, n, k, precision=gemm, cache_file=eig_cache)
            torch.cuda.synchronize()
            self.precompute_s = time.perf_counter() - t0
            self.eig_mixer = mixer
            self.xy = xy
            self._add_job(cost, n, w["angles"], spec["n_sets"])
            self.name = spec["name"] if xy == "ring" else spec["name"].replace("_ring_", "_clique_")
            self.units = spec["n_sets"]
            self.config = {"workload": self.name, "problem": "densest k-subgraph, G(16,0.5)", "n": n, "k": k,
                           "feasible_states": int(mixer.dim), "p": p, "mixer": f"{xy} XY",
                           "angle_sets_per_step": spec["n_sets"], "cost_dtype": "u8",
                           "l2": "per step 24 products over 256 sets; operands ~0.36 GB (blocks) / 2.7 GB "
                                 "(dense) vs 129 MB L2; no flush"}
            self.run_info_eig = {
                "gemm": gemm, "eig_precompute_s": round(self.precompute_s, 2),
                "mixer_form": ("cyclic-shift momentum blocks V_b diag(e^-ib lambda) V_b^T, block sizes "
                               f"{mixer.block_dims}" if eig_form == "blocks" else "dense V diag(e^-ib lambda) V^T")}
        elif idx == 5:
            inst = uneven_batch_recipe(spec["n_instances"], BASE_SEED + 5)
            self.grad = True
            for i, it in enumerate(inst):
                n = it["n"]
                cost = ctx.cost_precompute("maxcut", n, edges=it["edges"], dtype=torch.uint8)
                A = uniform_angles(p, BASE_SEED + 5 + 1000 + i, spec["n_sets"] * pool_steps)
                self._add_job(cost, n, A, spec["n_sets"])
            self.name = spec["name"]
            self.inst = inst
            self.config = {"workload": spec["name"], "problem": "MaxCut, 3-regular (even i) / G(n,0.3) (odd i)",
                           "instances": len(inst), "n_range": [14, 22], "p": p, "angle_sets_per_instance":
                           spec["n_sets"], "mixer": "X", "cost_dtype": "u8",
                           "amplitudes_per_step": int(sum(spec["n_sets"] << it["n"] for it in inst)),
                           "l2": "each step evaluates all 2048 angle sets, states of 15 GB in all vs 129 MB "
                                 "L2; no flush"}
            self.units = len(inst) * spec["n_sets"]
        else:
            w = workload_instance(idx, n_sets=spec["n_sets"] * pool_steps)
            n = n_override or spec["n"]
            self.grad = bool(spec["grad"])
            # mixer variant: transverse field, multi-angle, sum of X and XX
            # terms (mixer_X([1, 2])), or the Grover mixer on all 2^n states
            # (as the rank-one update, or through the general X-mixer passes)
            self.mixer_variant = mixer
            if mixer == "ma":
                from qaoa_inputs import uniform_angles_ma

                w["angles"] = uniform_angles_ma(p, n, BASE_SEED + idx + 1000, spec["n_sets"] * pool_steps)
                self.x_mixer = qg.XMixer(n, multi_angle=True)
            elif mixer == "terms":
                self.x_mixer = qg.x_terms_mixer(n, {1: 1.0, 2: 1.0})
            elif mixer == "grover":
                self.x_mixer = qg.GroverMixer.full(n)
            elif mixer == "grover_x":
                self.x_mixer = qg.grover_x_mixer(n)
            if spec["problem"] == "sk":
                J = w["J"] if n == spec["n"] else sk_couplings(n, BASE_SEED + idx)
                cost = ctx.cost_precompute("sk", n, J=J, dtype=torch.float32)
                prob = "SK, J_ij~N(0,1) on 2^-20 grid"
            else:
                cost = ctx.cost_precompute("maxcut", n, edges=w["edges"], dtype=torch.uint8)
                prob = "MaxCut " + ("G(12,0.5)" if idx == 1 else "random 3-regular")
            self._add_job(cost, n, w["angles"], spec["n_sets"])
            self.name = spec["name"] if n == spec["n"] else f"{spec['name']}_n{n}"
            if mixer != "x":
                self.name += f"_{mixer}"
            self.units = spec["n_sets"]
            mix_desc = {"x": "X (transverse field)", "ma": "multi-angle X (one angle per qubit and round)",
                        "terms": "sum_i X_i + sum_{i<j} X_i X_j (half rounds around a weight diagonal)",
                        "grover": "Grover |+><+| on all 2^n states (rank-one update, one pass per round)",
                        "grover_x": "Grover |+><+| on all 2^n states (half rounds around a weight diagonal)"}[mixer]
            self.config = {"workload": self.name, "problem": prob, "n": n, "p": p, "mixer": mix_desc,
                           "angle_sets_per_step": spec["n_sets"],
                           "cost_dtype": "f32" if spec["problem"] == "sk" else "u8"}
            self.config["l2"] = (f"state {2 ** n * 8 / 2 ** 30:.2f} GiB per set vs 129 MB L2; no flush"
                                 if n >= 24 else "on-chip state (whole state in shared memory)")
        # how this implementation runs the workload (not part of the workload)
        self.run_info = {"state": "complex64"}
        self.run_info.update(getattr(self, "run_info_eig", {}))
        if not self.grad:
            self.run_info["ckpt"] = "none (forward only)"
        elif getattr(self, "mixer_variant", "x") == "grover":
            self.run_info["ckpt"] = "every round's phase-separated state phi_r (p + 1 vectors)"
        elif idx == 4:
            self.run_info["ckpt"] = "per-round state checkpoints"
        else:
            self.run_info["ckpt"] = "per-pass state checkpoints (the adjoint writes lambda only)"

    def autotune(self):
        """Pick the pass schedule of every X-mixer problem size in the workload
        (untimed, before the warm-up); returns {n: schedule}."""
        out = {}
        for job in self.jobs:
            n = job["mixer"].n
            if not isinstance(job["mixer"], self.qg.XMixer) or n <= 12 or n in out:
                continue
            t = self.ctx.autotune(job["cost"], n, p=2, want_grad=self.grad)
            out[n] = {k: t[k] for k in ("cmin", "split", "nbuf_bwd_contig", "nbuf_bwd_gather")}
        return out

    def pin_schedule(self, split):
        """Install the pass schedule (cmin 4, the given split) for every
        X-mixer problem size in the workload; returns {n: schedule}."""
        import torch

        out = {}
        for job in self.jobs:
            n = job["mixer"].n
            if not isinstance(job["mixer"], self.qg.XMixer) or n <= 12 or n in out:
                continue
            t = {"n": n, "cost_dtype": 0 if job["cost"].dtype == torch.float32 else 1, "cmin": 4, "split": split,
                 "nbuf_bwd_contig": 1, "nbuf_bwd_gather": 1}
            self.ctx.set_tuning(t)
            out[n] = {k: t[k] for k in ("cmin", "split", "nbuf_bwd_contig", "nbuf_bwd_gather")}
        return out

    def _add_job(self, cost, n, A, n_sets):
        import torch

        pool = torch.from_numpy(np.ascontiguousarray(A)).to(self.dev)
        ang = pool[:n_sets].clone()
        E = torch.zeros(n_sets, dtype=torch.float64, device=self.dev)
        G = torch.zeros(n_sets, 2 * self.p, dtype=torch.float64, device=self.dev)
        mixer = getattr(self, "eig_mixer", None) or getattr(self, "x_mixer", None) or self.qg.XMixer(n)
        self.jobs.append({"cost": cost, "mixer": mixer, "angles": ang, "E": E, "grad": G})
        self.pools.append((pool, n_sets, n, np.ascontiguousarray(A)))

    def load_angles(self, step):
        for job, (pool, k, _, _) in zip(self.jobs, self.pools):
            s = (step * k) % pool.shape[0]
            job["angles"].copy_(pool[s:s + k], non_blocking=True)

    def run(self):
        # the job list is marshalled once; every step re-issues the same call
        if getattr(self, "_call", None) is None:
            self._call = self.ctx.batched_call(self.jobs, want_grad=self.grad)
        self._call.run()

    def e2e_step(self, step, pinned):
        """This step's angles from the pinned host pool into the call's pinned
        angle buffers, then the host-buffer batched call
        (qaoa_expectation_batched_host: angles copied in, launches, <C> and the
        gradients copied back, synchronised); returns the host results."""
        import torch

        if getattr(self, "_hcall", None) is None:
            self._h_ang, self._h_out, hjobs = [], [], []
            for job, (_, k, _, A) in zip(self.jobs, self.pools):
                na = A.shape[1]
                ha = torch.empty(k, na, dtype=torch.float64).pin_memory()
                hE = torch.empty(k, dtype=torch.float64).pin_memory()
                hG = torch.empty(k, na, dtype=torch.float64).pin_memory() if self.grad else None
                hjobs.append({"cost": job["cost"], "mixer": job["mixer"], "angles": ha, "E": hE, "grad": hG,
                              "init": job.get("init")})
                self._h_ang.append(ha)
                self._h_out.append((hE, hG))
            self._hcall = self.ctx.batched_call_host(hjobs, want_grad=self.grad)
        for ha, hp, (pool, k, _, _) in zip(self._h_ang, pinned, self.pools):
            s = (step * k) % pool.shape[0]
            ha.copy_(hp[s:s + k])
        self._hcall.run()
        outs = [e for e, _ in self._h_out]
        if self.grad:
            outs += [g for _, g in self._h_out]
        return outs

    def h2d_bytes(self):
        return sum(8 * 2 * self.p * k for (_, k, _, _) in self.pools)

    def d2h_bytes(self):
        return sum(8 * k * ((2 * self.p + 1) if self.grad else 1) for (_, k, _, _) in self.pools)

    def oracle_baseline(self):
        """Time the CPU oracle on a bounded sample of this workload; returns
        (units/s, cores, description, extra).  extra may carry more baseline
        fields ("baseline") and, where the sample's results can be compared
        with the GPU's, the error record ("oracle_error")."""
        import oracle
        from qaoa_inputs import BASE_SEED, sk_couplings, workload_instance

        oracle.build()
        p = self.p
        if self.idx == 2:
            w = workload_instance(2)
            n = self.pools[0][2]
            J = w["J"] if n == 28 else sk_couplings(n, BASE_SEED + 2)
            cost = oracle.cost_sk(n, J.astype(np.float64))
            a = self.pools[0][3][0]
            var = getattr(self, "mixer_variant", "x")

            def one_round(nn, cc):
                if var == "ma":
                    oracle.qaoa_gradient_ma(nn, cc, np.concatenate([a[:nn], a[p * nn:p * nn + 1]]))
                elif var == "grover":
                    oracle.qaoa_gradient(nn, cc, np.array([a[0], a[p]]), "grover")
                elif var in ("terms", "grover_x"):
                    w_ = self.x_mixer.weights.cpu().numpy() if nn == n else None
                    if w_ is None:
                        return None
                    oracle.qaoa_gradient_general(nn, w_, cc, np.array([a[0], a[p]]))
                else:
                    oracle.qaoa_gradient(nn, cc, np.array([a[0], a[p]]))
                return True

            t = time.perf_counter()
            one_round(n, cost)
            dt = (time.perf_counter() - t) * p
            cores = oracle.get_threads()
            del cost
            extra = {}
            if var == "x" and n >= 25:
                # one thread, on one round at n - 3 (an eighth of the state),
                # scaled by the mixer's n 2^n work to the full unit
                n1 = n - 3
                c1 = oracle.cost_sk(n1, sk_couplings(n1, BASE_SEED + 2).astype(np.float64))
                oracle.set_threads(1)
                try:
                    t = time.perf_counter()
                    one_round(n1, c1)
                    dt1 = (time.perf_counter() - t) * p * (n * 2.0 ** n) / (n1 * 2.0 ** n1)
                finally:
                    oracle.set_threads(cores)
                extra["baseline"] = {"single_thread": {
                    "value": 1.0 / dt1, "unit": UNIT, "cores": 1,
                    "sample": f"oracle gradient of one round (p=1) at n={n1} on one thread, scaled x{p} rounds "
                              f"and x{(n * 2.0 ** n) / (n1 * 2.0 ** n1):.2f} (n 2^n work) to the n={n}, p={p} unit"}}
            return 1.0 / dt, cores, (f"oracle gradient of one round (p=1) at n={n}, scaled x{p} to the p={p} "
                                     f"unit"), extra
        if self.idx == 4:
            w = workload_instance(4, n_sets=1)
            n, k = 16, 8
            st = oracle.dicke_states(n, k)
            cost = oracle.cost_dks(n, w["edges"], st)
            a = w["angles"][0]
            t = time.perf_counter()
            oracle.qaoa_gradient(n, cost, np.array([a[0], a[p]]), self.xy, st)
            dt = (time.perf_counter() - t) * p
            return 1.0 / dt, oracle.get_threads(), (f"oracle gradient of one round (p=1) of one angle set, "
                                                     f"power-series {self.xy} mixer on D={len(st)}, scaled x{p}"), {}
        if self.idx in (1, 3):
            w = workload_instance(self.idx, n_sets=2)
            n = self.pools[0][2]
            cost = oracle.cost_maxcut(n, w["edges"])
            k = 1 if self.idx == 3 else 20
            t = time.perf_counter()
            for s in range(k):
                a = w["angles"][s % 2]
                if self.grad:
                    oracle.qaoa_gradient(n, cost, a)
                else:
                    oracle.qaoa_expectation(n, cost, a)
            return k / (time.perf_counter() - t), oracle.get_threads(), (
                f"oracle on {k} of the workload's angle sets at n={n}, scaled per set"), {}
        # uneven batch: the first angle set of 16 of the 512 instances, timed;
        # their results are compared with the GPU's for the same angles
        import torch

        n_s = 16
        res, t_tot = [], 0.0
        for i in range(n_s):
            it = self.inst[i]
            c = oracle.cost_maxcut(it["n"], it["edges"])
            a = self.pools[i][3][0]
            t = time.perf_counter()
            E, g = oracle.qaoa_gradient(it["n"], c, a)
            t_tot += time.perf_counter() - t
            res.append((E, g, float(np.sqrt(np.mean(c ** 2)))))
        self.load_angles(0)
        self.run()
        torch.cuda.synchronize()
        worst_E, worst_g = 0.0, 0.0
        for i, (E, g, sig) in enumerate(res):
            Eg = float(self.jobs[i]["E"][0].item())
            gg = self.jobs[i]["grad"][0].cpu().numpy()
            worst_E = max(worst_E, abs(Eg - E) / max(abs(E), sig))
            worst_g = max(worst_g, float(np.max(np.abs(gg - g)) / np.max(np.abs(g))))
        err = {"reference": "CPU oracle (complex128, exact reverse mode), run here",
               "sets": f"first angle set of instances 0..{n_s - 1} (n = "
                       f"{sorted({self.inst[i]['n'] for i in range(n_s)})})",
               "max_abs_dE_over_max_absE_sigmaC": worst_E, "max_abs_dg_over_max_abs_g": worst_g}
        return n_s / t_tot, oracle.get_threads(), (
            f"oracle gradient of the first angle set of {n_s} of the 512 instances, per set"), {"oracle_error": err}


class GroverWorkload:
    """Grover-mixer QAOA on cost degeneracies: one step counts every weight-k
    subset of the 100-vertex graph by cost (the unit: feasible states counted)
    and evaluates <C> and the gradient of 1024 angle sets on the distinct
    values."""

    def __init__(self, qg, ctx, dev, pool_steps):
        import torch

        from qaoa_inputs import WORKLOADS, workload_instance

        self.idx, self.qg, self.ctx, self.dev = 6, qg, ctx, dev
        spec = dict(WORKLOADS[6])
        w = workload_instance(6, n_sets=spec["n_sets"] * pool_steps)
        self.n, self.k, self.p, self.S = spec["n"], spec["k"], spec["p"], spec["n_sets"]
        self.edges = w["edges"]
        self.grad = True
        self.name = spec["name"]
        self.units = math.comb(self.n, self.k)
        A = np.ascontiguousarray(w["angles"])
        pool = torch.from_numpy(A).to(dev)
        self.angles = pool[:self.S].clone()
        self.pools = [(pool, self.S, self.n, A)]
        self.counts = ctx.cost_degeneracy("dks", self.n, edges=self.edges, k=self.k)
        self.E, self.G = ctx.grover_batched(self.counts, self.angles)
        self.jobs = [{"E": self.E}]
        self.deg_ms = []
        self.run_info = {}
        self.config = {"workload": self.name, "problem": "densest k-subgraph, G(100,0.5), weight-6 subsets",
                       "n": self.n, "k": self.k, "feasible_states": self.units, "p": self.p,
                       "mixer": "Grover, on cost degeneracies", "angle_sets_per_step": self.S,
                       "unit_note": "value counts feasible states enumerated per second",
                       "state": "float64 reduced vector (one amplitude per cost value)",
                       "l2": "no state in memory: integer enumeration"}

    def autotune(self):
        return {}

    def load_angles(self, step):
        s = (step * self.S) % self.pools[0][0].shape[0]
        self.angles.copy_(self.pools[0][0][s:s + self.S], non_blocking=True)

    def run(self):
        import torch

        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st = torch.cuda.current_stream()
        a.record(st)
        self.counts = self.ctx.cost_degeneracy("dks", self.n, edges=self.edges, k=self.k)
        b.record(st)
        self.E, self.G = self.ctx.grover_batched(self.counts, self.angles)
        self.jobs[0]["E"] = self.E
        self.deg_ms.append((a, b))

    def e2e_step(self, step, pinned):
        s = (step * self.S) % pinned[0].shape[0]
        self.angles.copy_(pinned[0][s:s + self.S], non_blocking=True)
        self.run()
        outs = [self.E.to("cpu", non_blocking=True), self.G.to("cpu", non_blocking=True)]
        import torch

        torch.cuda.current_stream().synchronize()
        return outs

    def h2d_bytes(self):
        return 8 * 2 * self.p * self.S

    def d2h_bytes(self):
        return 8 * self.S * (2 * self.p + 1)

    def degeneracy_ms(self, last):
        ev = self.deg_ms[-last:]
        return sum(a.elapsed_time(b) for a, b in ev) / len(ev)

    def oracle_baseline(self):
        """The oracle's brute-force count on the weight-3 subsets of the same
        graph, per state, scaled to states/s."""
        import oracle

        oracle.build()
        t = time.perf_counter()
        oracle.cost_degeneracy(self.n, self.edges, "dks", 3, method="subsets")
        dt = time.perf_counter() - t
        return math.comb(self.n, 3) / dt, 1, (f"oracle brute-force degeneracy count of all weight-3 subsets "
                                              f"of the same graph ({math.comb(self.n, 3)} states, numpy on one "
                                              f"core), per state"), {}


# ---------------------------------------------------------------- GPU arm

def gpu_arm(args, ws, rank, local):
    import torch

    import paper_2312_06451_gb300 as qg

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod

        dist_mod.init_process_group("nccl")
        dist = dist_mod
    dev = f"cuda:{local}"
    stream = torch.cuda.Stream(device=local)
    with torch.cuda.stream(stream):
        return _gpu_arm_on_stream(args, ws, rank, local, dist, dev, stream, qg)


def _gpu_arm_on_stream(args, ws, rank, local, dist, dev, stream, qg):
    import torch

    ctx = qg.Context(local, stream)
    if args.workload == 6:
        W = GroverWorkload(qg, ctx, dev, args.steps + args.warmup)
    else:
        W = Workload(qg, ctx, args.workload, dev, args.steps + args.warmup, args.n, args.gemm, args.mixer,
                     args.eig_cache, args.eig)
    out = measure(args, W, qg, ctx, stream, dist, ws, rank, local, dev, graph_mode=args.graph,
                  steps=args.steps, warmup=args.warmup)
    headline = args.workload == WORKLOAD and not args.n and args.mixer == "x"
    if rank == 0 and out is not None:
        out["metric"] = METRIC if headline else f"QAOA {out['unit']} ({W.name})"
        if headline:
            err = oracle_error_golden(W)
            if err is not None:
                out["oracle_error"] = err
    del W
    ctx.close()
    if headline and not args.no_batched:
        # the batched half of the metric: the uneven angle-finding batch
        # (512 instances, n = 14..22, 4 angle sets each, p = 6), every step
        # replayed from one captured CUDA graph, in a context of its own
        torch.cuda.empty_cache()
        ctx5 = qg.Context(local, stream)
        W5 = Workload(qg, ctx5, 5, dev, args.steps + args.warmup)
        b = measure(args, W5, qg, ctx5, stream, dist, ws, rank, local, dev, graph_mode=True,
                    steps=args.steps, warmup=args.warmup)
        if rank == 0 and b is not None:
            b["metric"] = f"QAOA {b['unit']} ({W5.name})"
            out["batched"] = b
        del W5
        ctx5.close()
    if headline and not args.no_grover:
        # the same workload with the Grover mixer of Sec. 2.4 as the rank-one
        # update (one streaming pass per round and direction), direct launches
        torch.cuda.empty_cache()
        ctxg = qg.Context(local, stream)
        Wg = Workload(qg, ctxg, WORKLOAD, dev, args.steps + args.warmup, mixer="grover")
        gargs = argparse.Namespace(**vars(args))
        gargs.no_cpu_baseline = True
        g = measure(gargs, Wg, qg, ctxg, stream, dist, ws, rank, local, dev, graph_mode=False,
                    steps=args.steps, warmup=args.warmup)
        if rank == 0 and g is not None:
            g["metric"] = f"QAOA {g['unit']} ({Wg.name})"
            out["grover"] = g
        del Wg
        ctxg.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def measure(args, W, qg, ctx, stream, dist, ws, rank, local, dev, graph_mode, steps, warmup):
    """Time `steps` steps of workload W after `warmup` untimed ones.

    value: CUDA events on the library's stream around the steps, with no
    per-kernel events inside (graph replay when graph_mode).  Per-kernel
    family times for the roofline come from a separate repeat of the same
    steps as direct launches, each bracketed by CUDA events.  e2e: the same
    steps end to end from pinned host angles to host results."""
    import torch

    if args.split is not None:
        sched = W.pin_schedule(args.split)
        if sched:
            W.run_info["schedule"] = sched if len(sched) > 1 else next(iter(sched.values()))
    elif not args.no_autotune:
        sched = W.autotune()
        if sched:
            W.run_info["schedule"] = sched if len(sched) > 1 else next(iter(sched.values()))

    graph, launches_per_step = None, None
    if graph_mode:
        # capture one step (angle copies + batched call) after a plan-building call
        W.load_angles(0)
        W.run()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        l0 = ctx.launch_count()
        with torch.cuda.graph(graph, stream=stream):
            W.run()
        launches_per_step = ctx.launch_count() - l0

    def step(i, replay=True):
        W.load_angles(i)
        if graph is not None and replay:
            graph.replay()
        else:
            W.run()

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ctx.set_profiling(False)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launch_count()
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(steps):
        step(warmup + i)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = launches_per_step * steps if graph is not None else ctx.launch_count() - l0
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()

    # per-family kernel times: the same steps again, direct launches, each
    # launch bracketed by CUDA events on the library's stream
    ctx.reset_stats()
    ctx.set_profiling(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for i in range(steps):
        step(warmup + i, replay=False)
    p1.record(stream)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    prof_ms = p0.elapsed_time(p1)
    stats = ctx.kernel_stats()

    rmax, rsum = reducers(dist, dev)
    value, tmax, units = aggregate(ms / 1e3, steps * W.units, ws, rmax, rsum)
    E_last = float(W.jobs[0]["E"][0].item())

    # end to end through the public API: host angles from pinned memory copied
    # in, batched call, <C> (and gradients) read back, every step
    pinned = [torch.from_numpy(pl[3]).pin_memory() for pl in W.pools]
    for i in range(2):
        W.e2e_step(i, pinned)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(steps):
        outs = W.e2e_step(warmup + i, pinned)
    torch.cuda.synchronize()
    e2e_s = rmax(time.perf_counter() - t0)
    e2e_value = rsum(steps * W.units) / e2e_s

    fd = None
    if W.grad and ws == 1 and not args.no_fd and W.idx != 6 and getattr(W, "mixer_variant", "x") in ("x", "clique"):
        fd = fd_compare(W, stream, value)

    roof = roofline(W, stats, args.gemm if W.idx == 4 else None, steps)
    unit = UNIT if W.grad else "evals/s"
    if W.idx == 6:
        unit = "states/s"
    out = None
    if rank == 0:
        cfg = dict(W.config)
        cfg.update({"units_per_step_per_rank": W.units, "parallelism": f"replicas x{ws}"})
        run = dict(W.run_info)
        run.update({"timing": "CUDA graph replay" if graph is not None else "direct launches",
                    "kernel_times": "a second run of the same steps, direct launches, one CUDA event pair "
                                    "per launch on the library's stream",
                    "profiled_ms_per_step": prof_ms / steps})
        out = {
            "metric": None, "value": value, "unit": unit, "n_gpus": ws, "steps": steps,
            "warmup": warmup, "ms_per_step": tmax * 1e3 / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg, "run": run,
            "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": W.h2d_bytes(),
                    "d2h_bytes_per_step": W.d2h_bytes(),
                    "api": ("qaoa_expectation_batched_host" if getattr(W, "_hcall", None) is not None
                            else "device-buffer call with pinned torch copies")},
            "roofline": roof,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4),
                            "GBps": round(v["algo_bytes"] / v["total_ms"] / 1e6, 1) if v["total_ms"] else None}
                        for k, v in stats.items() if v["launches"]},
            "gpu_launches": launches,
            "clocks": clk,
            "result_check": {"E_first_set_last_step": E_last, "e2e_E0": float(outs[0][0])},
        }
        if fd is not None:
            out["fd_baseline"] = fd
        if ws == 1 and not args.no_cpu_baseline:
            v, cores, desc, extra = W.oracle_baseline()
            out["cpu_baseline"] = {"value": v, "unit": unit, "cores": cores, "kind": "oracle", "sample": desc}
            out["cpu_baseline"].update(extra.get("baseline", {}))
            if "oracle_error" in extra:
                out["oracle_error"] = extra["oracle_error"]
    return out


def roofline(W, stats, gemm, steps):
    """Roofline of the dominant kernel family (most device time): its
    algorithmic bytes (or useful flops) per launch over its average launch
    time from the profiled steps."""
    peaks = measured_peaks()
    fams = [k for k in stats if stats[k]["launches"] and stats[k]["total_ms"] > 0]
    roof = None
    if W.idx == 6:
        # integer enumeration: the bound is the SM's bit-count unit (16
        # 32-bit population counts a clock per SM).  The bit-sliced count
        # takes, per (k-1)-set T, one 64-bit population count (2 x 32-bit)
        # per plane combination 1..k-1 (the swept vertices v < w lie in the
        # low word for all but 0.5% of the T), and T covers (n-k+1)/k
        # states on average: 2k(k-1)/(n-k+1) counts per state.
        dms = W.degeneracy_ms(steps)
        ops = 2 * W.k * (W.k - 1) / (W.n - W.k + 1)
        achieved = W.units / (dms * 1e-3) / 1e9
        peak = 152 * 16 * 2.07e9 / ops / 1e9
        return {"bound": "alu", "kernel": "degeneracy_sliced_kernel", "achieved": achieved, "peak": peak,
                "unit": "Gstates/s", "frac": achieved / peak,
                "peak_source": f"derived: 152 SM x 16 bit-count ops/clk x 2.07 GHz / {ops:.3f} counts per state",
                "traffic": None, "launch_ms": dms}
    if not fams:
        return None
    fam = max(fams, key=lambda k: stats[k]["total_ms"])
    st = stats[fam]
    if st["algo_flops"] > 0:
        achieved = st["algo_flops"] / (st["total_ms"] * 1e-3) / 1e12
        pk = gemm_peak(gemm or "3xtf32")
        roof = {"bound": pk["bound"], "kernel": fam, "achieved": achieved, "peak": pk["peak"], "unit": "TFLOP/s",
                "frac": achieved / pk["peak"], "peak_source": pk["source"], "traffic": traffic_for(fam, W.name),
                "algo_flops_per_launch": st["algo_flops"] / st["launches"],
                "launch_ms": st["total_ms"] / st["launches"]}
    else:
        per_launch_bytes = st["algo_bytes"] / st["launches"]
        per_launch_ms = st["total_ms"] / st["launches"]
        achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": fam, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"],
                "traffic": traffic_for(fam, W.name), "algo_bytes_per_launch": per_launch_bytes,
                "launch_ms": per_launch_ms}
    tot = sum(stats[k]["total_ms"] for k in fams)
    roof["share_of_kernel_time"] = st["total_ms"] / tot if tot else None
    if roof["bound"] == "hbm":
        # the whole step: every kernel's algorithmic bytes over the profiled
        # step time (kernel times summed; launch gaps excluded)
        step_bytes = sum(stats[k]["algo_bytes"] for k in fams) / steps
        step_ms = tot / steps
        roof["step"] = {"algo_bytes": step_bytes, "kernel_ms": step_ms,
                        "achieved": step_bytes / (step_ms * 1e-3) / 1e9,
                        "frac": step_bytes / (step_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    return roof


def oracle_error_golden(W):
    """Error of the timed path against the CPU oracle (complex128) on the
    stored oracle values of the headline workload: the first angle set of the
    timed pool and a linear-ramp schedule where |<C>| is several sigma_C.
    Runs the same batched call as the timed steps, outside the timed region."""
    import torch

    path = os.path.join(ROOT, "tests", "golden", "oracle_fullsize.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)["workloads"]
    job = W.jobs[0]
    rows = []
    for key, label in (("2", "first angle set of the timed pool (U[0, pi))"),
                       ("2ramp", "linear ramp beta_k = 0.6 (1 - t_k), gamma_k = -0.12 t_k")):
        g = gold.get(key)
        if g is None:
            continue
        job["angles"][0].copy_(torch.tensor(g["angles"], dtype=torch.float64))
        W.run()
        torch.cuda.synchronize()
        E = float(job["E"][0].item())
        G = job["grad"][0].cpu().numpy()
        gref = np.array(g["grad"])
        sig = g["cost_rms"]
        rows.append({"set": label, "E_oracle": g["E"], "E_gpu": E, "abs_dE": abs(E - g["E"]),
                     "abs_dE_over_sigma_C": abs(E - g["E"]) / sig,
                     "rel_dE": abs(E - g["E"]) / abs(g["E"]) if g["E"] else None,
                     "max_abs_dg_over_max_abs_g": float(np.max(np.abs(G - gref)) / np.max(np.abs(gref))),
                     "max_rel_dg_per_component": float(np.max(np.abs(G - gref) / np.abs(gref)))})
    return {"reference": "tests/golden/oracle_fullsize.json (CPU oracle, complex128, exact reverse mode)",
            "sets": rows, "sigma_C": gold["2"]["cost_rms"]}


def fd_compare(W, stream, adjoint_value, h=1e-3, reps=3, max_jobs=8):
    """The plain finite-difference gradient on the same GPU, for comparison
    with the adjoint: per angle set, 4p forward <C> evaluations at
    theta +- h e_j (central differences), issued as one batched forward call
    per sampled set (the fastest way to run them).  Returns its throughput,
    the adjoint/FD ratio and the largest difference from the adjoint gradient
    of the same angles (relative to the gradient's largest component)."""
    import torch

    jobs, ref = [], []
    for job in W.jobs[:max_jobs]:
        a = job["angles"][0].detach().cpu().numpy().astype(np.float64)
        g = job["grad"][0].detach().cpu().numpy().astype(np.float64)
        m = a.shape[0]
        A = np.repeat(a[None, :], 2 * m, axis=0)
        for j in range(m):
            A[2 * j, j] += h
            A[2 * j + 1, j] -= h
        jobs.append({"cost": job["cost"], "mixer": job["mixer"], "angles": torch.from_numpy(A).to(W.dev),
                     "E": torch.zeros(2 * m, dtype=torch.float64, device=W.dev)})
        ref.append(g)
    W.ctx.expectation_batched(jobs, want_grad=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        W.ctx.expectation_batched(jobs, want_grad=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    rate = len(jobs) / t
    err = 0.0
    for jb, g in zip(jobs, ref):
        E = jb["E"].cpu().numpy()
        gfd = (E[0::2] - E[1::2]) / (2 * h)
        err = max(err, float(np.max(np.abs(gfd - g)) / max(np.max(np.abs(g)), 1e-300)))
    return {"value": rate, "unit": "grad/s", "adjoint_over_fd": adjoint_value / rate,
            "method": f"central differences h={h}: 4p forward <C> per gradient, complex64 state",
            "sample": f"{len(jobs)} angle set(s) (first set of the first {len(jobs)} job(s)), {reps} timed calls",
            "max_abs_diff_vs_adjoint_rel": err}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None,
                    help="override the qubit count (small cases for profiler captures)")
    ap.add_argument("--workload", type=int, default=WORKLOAD, choices=[1, 2, 3, 4, 5, 6],
                    help="1: MaxCut n=12 p=3 forward; 2: SK n=28 p=8 gradient (default); "
                         "3: 3-regular n=24 p=10, 1024 angle sets; 4: densest 8-subgraph n=16 ring mixer "
                         "(D=12870), 256 angle sets; 5: 512 uneven instances x 4 sets; "
                         "6: Grover mixer on cost degeneracies, densest 6-subgraph n=100")
    ap.add_argument("--eig-cache", default=None,
                    help="workload 4: load the mixer's eigendecomposition (dense V or its blocks) from this file, "
                         "or save it there")
    ap.add_argument("--gemm", default="3xtf32", choices=["fp32", "3xtf32"],
                    help="eigenbasis product precision (workload 4): tcgen05 3xTF32 or CUDA-core float32")
    ap.add_argument("--eig", default="blocks", choices=["blocks", "dense"],
                    help="workload 4: the mixer through its cyclic-shift momentum blocks (default) or one dense "
                         "eigendecomposition")
    ap.add_argument("--graph", action="store_true", help="replay each step from a captured CUDA graph")
    ap.add_argument("--mixer", default="x", choices=["x", "ma", "terms", "grover", "grover_x", "clique"],
                    help="X-mixer workloads (1-3): transverse field, multi-angle, X + XX terms, Grover (rank-one "
                         "update) or Grover through the general X-mixer passes; "
                         "workload 4: clique instead of ring XY mixer")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default X-mixer pass schedule instead of tuning it before the warm-up")
    ap.add_argument("--split", type=int, default=None, choices=[0, 1, 2],
                    help="pin the X-mixer pass schedule's chunk order (0 equal chunks, 1 full chunks first, "
                         "2 remainder first) at the minimum contiguous run of 4, instead of tuning it")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload only: skip the batched sub-record (uneven 512-instance batch)")
    ap.add_argument("--no-grover", action="store_true",
                    help="default workload only: skip the sub-record of the same workload with the Grover mixer "
                         "(rank-one update)")
    ap.add_argument("--no-fd", action="store_true",
                    help="skip the central finite-difference comparison on the same GPU")
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
        t_unit = sum(ts) / len(ts) * p  # one round timed, p rounds per gradient
        value = 1.0 / t_unit
        cfg = headline_config(n, p)
        cfg.update({"units_per_step_per_rank": 1, "parallelism": f"replicas x{ws}"})
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_unit * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "run": {"state": "complex128", "timing": "host wall clock per step",
                    "step": f"one round (p=1) of the n={n} gradient, timed; ms_per_step and value are per "
                            f"p={p} gradient (x{p})"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: oracle gradient of one round (p=1) at n={n}, "
                                       f"scaled x{p} to the p={p} unit"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return

    out = gpu_arm(args, ws, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

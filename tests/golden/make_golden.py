"""Write oracle results for the full-size workloads to oracle_fullsize.json.

Calls only the CPU oracle (oracle/) and the seeded generators (qaoa_inputs/);
nothing here touches the CUDA library.  The GPU tests compare against these
stored values at sizes where running the oracle inside the test would take
minutes.  Re-run after any change to the oracle's arithmetic:

    python tests/golden/make_golden.py
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from qaoa_inputs import ramp_angles, workload_instance  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_fullsize.json")


def main():
    oracle.build()
    res = {"generated_by": "tests/golden/make_golden.py (CPU oracle, complex128)", "workloads": {}}
    if os.path.exists(OUT) and "--all" not in sys.argv:
        with open(OUT) as f:
            res = json.load(f)
    if "4" not in res["workloads"]:
        workload4(res)
        with open(OUT, "w") as f:
            json.dump(res, f, indent=1)
    if "2ramp" not in res["workloads"]:
        workload2_ramp(res)
        with open(OUT, "w") as f:
            json.dump(res, f, indent=1)
    if "2" in res["workloads"] and "3" in res["workloads"]:
        return
    rng = np.random.default_rng(7)

    # Workload 2: SK n=28, p=8, one angle set, E and gradient.
    w = workload_instance(2)
    n, p = w["spec"]["n"], w["spec"]["p"]
    t = time.time()
    cost = oracle.cost_sk(n, w["J"].astype(np.float64))
    idx = np.sort(rng.choice(1 << n, size=64, replace=False))
    E, g = oracle.qaoa_gradient(n, cost, w["angles"][0])
    res["workloads"]["2"] = {
        "name": w["spec"]["name"], "n": n, "p": p, "angles": w["angles"][0].tolist(),
        "E": E, "grad": g.tolist(), "cost_mean": float(cost.mean()),
        "cost_rms": float(np.sqrt(np.mean(cost ** 2))),
        "cost_sample_idx": idx.tolist(), "cost_sample": cost[idx].tolist(),
        "oracle_seconds": time.time() - t, "oracle_threads": oracle.get_threads(),
    }
    del cost
    print("workload 2 done", res["workloads"]["2"]["oracle_seconds"])

    # Workload 3: 3-regular n=24, p=10: the first two angle sets.
    w = workload_instance(3, n_sets=2)
    n, p = w["spec"]["n"], w["spec"]["p"]
    t = time.time()
    cost = oracle.cost_maxcut(n, w["edges"])
    sets = []
    for s in range(2):
        E, g = oracle.qaoa_gradient(n, cost, w["angles"][s])
        sets.append({"angles": w["angles"][s].tolist(), "E": E, "grad": g.tolist()})
    res["workloads"]["3"] = {"name": w["spec"]["name"], "n": n, "p": p, "sets": sets,
                             "cost_rms": float(np.sqrt(np.mean(cost ** 2))),
                             "oracle_seconds": time.time() - t}
    print("workload 3 done", res["workloads"]["3"]["oracle_seconds"])
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)


def workload2_ramp(res):
    """SK n=28, p=8 on a linear-ramp schedule (ramp_angles), where <C> sits
    several sigma_C from the mean: E and the gradient."""
    w = workload_instance(2)
    n, p = w["spec"]["n"], w["spec"]["p"]
    a = ramp_angles(p)[0]
    t = time.time()
    cost = oracle.cost_sk(n, w["J"].astype(np.float64))
    E, g = oracle.qaoa_gradient(n, cost, a)
    res["workloads"]["2ramp"] = {
        "name": w["spec"]["name"] + "_ramp", "n": n, "p": p, "angles": a.tolist(), "E": E, "grad": g.tolist(),
        "cost_rms": float(np.sqrt(np.mean(cost ** 2))), "oracle_seconds": time.time() - t,
        "oracle_threads": oracle.get_threads(),
    }
    print("workload 2 ramp done", res["workloads"]["2ramp"]["oracle_seconds"], E)


def workload4(res, mixer="ring"):
    """Densest 8-subgraph on G(16, 0.5), ring (or clique) mixer on the 12870
    weight-8 states, p=6: two angle sets, <C> and gradient."""
    w = workload_instance(4, n_sets=2)
    n, k, p = w["spec"]["n"], w["spec"]["k"], w["spec"]["p"]
    t = time.time()
    st = oracle.dicke_states(n, k)
    cost = oracle.cost_dks(n, w["edges"], st)
    sets = []
    for s in range(2):
        E, g = oracle.qaoa_gradient(n, cost, w["angles"][s], mixer, st)
        sets.append({"angles": w["angles"][s].tolist(), "E": E, "grad": g.tolist()})
    key = "4" if mixer == "ring" else "4" + mixer
    name = w["spec"]["name"] if mixer == "ring" else w["spec"]["name"].replace("_ring_", f"_{mixer}_")
    res["workloads"][key] = {"name": name, "n": n, "k": k, "p": p, "sets": sets, "mixer": mixer,
                             "cost_rms": float(np.sqrt(np.mean(cost ** 2))),
                             "oracle_seconds": time.time() - t}
    print("workload 4 done", mixer, res["workloads"][key]["oracle_seconds"])


if __name__ == "__main__":
    main()

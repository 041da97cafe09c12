"""Seeded generators for the synthetic QAOA workloads.

The paper evaluates QAOA on random graph instances it draws itself: MaxCut on
Erdos-Renyi G(n, 0.5) graphs (Section 3, Listing 1; Section 4, Fig. 4), Densest
k-Subgraph on G(n, 0.5) (Listing 2), all with uniformly random angles
(Listing 1 draws ``rand(2p)``; Listing 3 draws ``2*pi*rand(2p)``).  Graphs.jl's
random streams cannot be reproduced here, so every instance below comes from
numpy's PCG64 with a stated seed.  Nothing in this module evaluates a cost, a
state or a mixer.

Angle layout everywhere: ``[beta_1 .. beta_p, gamma_1 .. gamma_p]`` (the
comment in Listing 1: betas first, then gammas).
"""

from __future__ import annotations

import numpy as np

#: Base seed of the five workloads; workload i (1-based) uses BASE_SEED + i
#: for its instance and BASE_SEED + i + 1000 for its angles.
BASE_SEED = 2312064510

#: J couplings are quantised to multiples of this step (see sk_couplings).
SK_GRID = 2.0 ** -20


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def erdos_renyi(n: int, p_edge: float, seed: int) -> np.ndarray:
    """G(n, p_edge): every unordered pair (u < v), visited in lexicographic
    order, is an edge independently with probability p_edge.

    Returns an int32 array of shape (m, 2) with u < v in each row.
    """
    rng = _rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p_edge
    return np.stack([iu[keep], ju[keep]], axis=1).astype(np.int32)


def random_regular3(n: int, seed: int, max_tries: int = 100000) -> np.ndarray:
    """Uniform-ish random 3-regular simple graph by the configuration model.

    Each vertex gets three half-edges; a random perfect matching of the 3n
    half-edges is drawn and rejected if it makes a self-loop or a repeated
    edge.  n must be even (3n half-edges must pair up).  Returns int32 (m, 2),
    rows sorted with u < v, m = 3n/2.
    """
    if n % 2 or n < 4:
        raise ValueError("a 3-regular graph needs an even n >= 4")
    rng = _rng(seed)
    stubs = np.repeat(np.arange(n), 3)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        u, v = np.minimum(a, b), np.maximum(a, b)
        key = u * n + v
        if np.unique(key).shape[0] != key.shape[0]:
            continue
        order = np.argsort(key)
        return np.stack([u[order], v[order]], axis=1).astype(np.int32)
    raise RuntimeError("configuration model did not produce a simple graph")


def sk_couplings(n: int, seed: int) -> np.ndarray:
    """Sherrington-Kirkpatrick couplings J_ij ~ N(0, 1) for i < j.

    Each draw is rounded to the nearest multiple of 2**-20 and clipped to
    |J| < 8, so it is exactly representable in float32 and every partial sum of
    up to 2**12 signed couplings is exact in float64.  Returned as a
    symmetric float32 (n, n) matrix with a zero diagonal.
    """
    rng = _rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    g = rng.standard_normal(iu.shape[0])
    g = np.clip(np.rint(g / SK_GRID) * SK_GRID, -8.0 + SK_GRID, 8.0 - SK_GRID)
    J = np.zeros((n, n), dtype=np.float64)
    J[iu, ju] = g
    J[ju, iu] = g
    return J.astype(np.float32)


def uniform_angles(p: int, seed: int, n_sets: int = 1, high: float = np.pi) -> np.ndarray:
    """n_sets angle vectors of length 2p, each entry ~ U[0, high), float64."""
    rng = _rng(seed)
    return rng.random((n_sets, 2 * p)) * high


def ramp_angles(p: int, beta0: float = 0.6, gamma1: float = -0.12) -> np.ndarray:
    """One deterministic annealing-like schedule (the kind of smooth angle
    pattern the paper's angle-finding discussion starts from, Sec. 2.3):
    beta_k = beta0 (1 - t_k), gamma_k = gamma1 t_k with t_k = (k - 1/2) / p.
    Unlike uniform random angles it drives <C> far from the uniform mean, so
    a relative error bound on <C> is tested at |<C>| of several sigma_C.
    Returns float64 (1, 2p)."""
    t = (np.arange(p) + 0.5) / p
    return np.concatenate([beta0 * (1.0 - t), gamma1 * t])[None, :].astype(np.float64)


def uniform_angles_ma(p: int, n: int, seed: int, n_sets: int = 1, high: float = np.pi) -> np.ndarray:
    """Multi-angle sets: n_sets vectors of p (n + 1) entries ~ U[0, high)
    (p rounds of n per-qubit betas, then p gammas), float64."""
    rng = _rng(seed)
    return rng.random((n_sets, p * (n + 1))) * high


def uneven_batch_recipe(n_instances: int, seed: int, n_lo: int = 14, n_hi: int = 22):
    """Instances of the uneven angle-finding batch.

    Even index -> MaxCut on a random 3-regular graph with n drawn uniformly
    from the even values in [n_lo, n_hi] (a 3-regular graph needs 3n even).
    Odd index -> MaxCut on G(n, 0.3) with n drawn uniformly from [n_lo, n_hi].
    Returns a list of dicts {"kind", "n", "edges", "seed"}.
    """
    rng = _rng(seed)
    evens = np.arange(n_lo + (n_lo % 2), n_hi + 1, 2)
    out = []
    for i in range(n_instances):
        s = int(rng.integers(0, 2**62))
        if i % 2 == 0:
            n = int(rng.choice(evens))
            edges = random_regular3(n, s)
            kind = "3reg"
        else:
            n = int(rng.integers(n_lo, n_hi + 1))
            edges = erdos_renyi(n, 0.3, s)
            kind = "er0.3"
        out.append({"kind": kind, "n": n, "edges": edges, "seed": s})
    return out


#: The five synthetic workloads, shaped like the paper's (Section 2.1
#: feasible sets, Section 3 listings, Section 4 figures).
WORKLOADS = {
    1: dict(name="maxcut_er12_p3", problem="maxcut", graph="er", n=12, p_edge=0.5,
            mixer="x", p=3, n_sets=1, grad=False),
    2: dict(name="sk28_p8_grad", problem="sk", n=28, mixer="x", p=8, n_sets=1, grad=True),
    3: dict(name="maxcut_3reg24_p10_b1024", problem="maxcut", graph="3reg", n=24,
            mixer="x", p=10, n_sets=1024, grad=True),
    4: dict(name="dks_er16_k8_ring_p6_b256", problem="dks", graph="er", n=16, k=8,
            p_edge=0.5, mixer="ring", p=6, n_sets=256, grad=True),
    5: dict(name="uneven512_p6_s4", problem="maxcut", graph="uneven", n_instances=512,
            mixer="x", p=6, n_sets=4, grad=True),
    # Grover mixer on cost degeneracies (Section 2.4: up to n = 100): all
    # weight-6 subsets of 100 vertices counted by cost, then 1024 angle sets
    6: dict(name="grover_dks_er100_k6_p10_b1024", problem="dks", graph="er", n=100, k=6,
            p_edge=0.5, mixer="grover", p=10, n_sets=1024, grad=True),
}


def workload_instance(i: int, n_sets: int | None = None):
    """Instance data for workload i (1..5): graph/couplings and angle sets."""
    w = dict(WORKLOADS[i])
    seed = BASE_SEED + i
    if n_sets is not None:
        w["n_sets"] = n_sets
    out = {"spec": w, "seed": seed}
    if w["problem"] == "sk":
        out["J"] = sk_couplings(w["n"], seed)
    elif w.get("graph") == "er":
        out["edges"] = erdos_renyi(w["n"], w["p_edge"], seed)
    elif w.get("graph") == "3reg":
        out["edges"] = random_regular3(w["n"], seed)
    elif w.get("graph") == "uneven":
        out["instances"] = uneven_batch_recipe(w["n_instances"], seed)
    if w.get("graph") == "uneven":
        out["angles"] = uniform_angles(w["p"], seed + 1000, w["n_instances"] * w["n_sets"])
    else:
        out["angles"] = uniform_angles(w["p"], seed + 1000, w["n_sets"])
    return out

"""Grover-mixer QAOA on cost degeneracies (Sec. 2.4) against the oracle.

The library counts the states of every cost value on the GPU (all 2^n states
for MaxCut, the weight-k states for densest k-subgraph and k-vertex cover up
to n = 128) and runs the QAOA on the distinct values; the oracle counts by
brute force and simulates either the full state vector (small n) or the
reduced vector (n = 100).  Counts are integers: compared exactly.
"""

import math

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, random_regular3, uniform_angles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2312_06451_gb300 as qg

    ctx = qg.Context(0)
    yield qg, ctx
    ctx.close()


@pytest.mark.parametrize("prob,n,k,p_edge", [
    ("maxcut", 12, -1, 0.5), ("maxcut", 20, -1, 0.3), ("maxcut", 5, -1, 1.0),
    ("dks", 20, 7, 0.5), ("dks", 20, 13, 0.5), ("dks", 16, 0, 0.5), ("dks", 16, 16, 0.5),
    ("kvc", 16, 5, 0.4), ("kvc", 18, 12, 0.3),
    ("dks", 100, 3, 0.5), ("kvc", 128, 2, 0.1), ("dks", 70, 67, 0.2),
    # bit-sliced count (cost a function of the inside edges, set size 2..8):
    # one and two 64-bit words, set sizes 2 and 8, the complement form
    ("dks", 28, 8, 0.4), ("dks", 90, 2, 0.5), ("dks", 64, 4, 0.3), ("dks", 66, 4, 0.3),
    ("dks", 128, 3, 0.3), ("kvc", 24, 22, 0.3), ("kvc", 26, 19, 0.3),
])
def test_degeneracies_match_brute_force(Q, oracle_mod, prob, n, k, p_edge):
    qg, ctx = Q
    e = erdos_renyi(n, p_edge, 1000 + n + max(k, 0))
    m = len(e)
    got = ctx.cost_degeneracy(prob, n, edges=e, k=k, n_bins=m + 1).cpu().numpy()
    ref = oracle_mod.cost_degeneracy(n, e, prob, None if k < 0 else k, n_bins=m + 1)
    np.testing.assert_array_equal(got, ref)


def test_degeneracies_two_slabs(Q):
    """2^37 states (two enumeration slabs): the count, the MaxCut mean |E|/2
    and the complement symmetry (every count even) hold exactly."""
    qg, ctx = Q
    n = 37
    e = random_regular3(36, 5)
    got = ctx.cost_degeneracy("maxcut", n, edges=e, k=-1).cpu().numpy().astype(object)
    assert sum(got) == 1 << n
    assert sum(c * v for c, v in enumerate(got)) * 2 == len(e) * (1 << n)
    assert all(v % 2 == 0 for v in got)


def test_degeneracies_full_size_moments(Q):
    """All weight-6 subsets of the 100-vertex benchmark graph (1.19e9 states):
    the count and the first two moments of the inside-edge count are fixed by
    the graph alone, exactly.  sum_S I(S)^2 counts ordered edge pairs inside S:
    equal pairs C(n-2, k-2) times, pairs sharing one vertex C(n-3, k-3) times,
    disjoint pairs C(n-4, k-4) times."""
    from qaoa_inputs import WORKLOADS, workload_instance

    qg, ctx = Q
    spec = WORKLOADS[6]
    n, k = spec["n"], spec["k"]
    e = np.asarray(workload_instance(6, n_sets=1)["edges"]).reshape(-1, 2)
    m = len(e)
    deg = np.bincount(e.ravel(), minlength=n).astype(object)
    share = sum(d * (d - 1) for d in deg)
    got = [int(v) for v in ctx.cost_degeneracy("dks", n, edges=e, k=k).cpu().numpy()]
    assert sum(got) == math.comb(n, k)
    assert sum(c * v for c, v in enumerate(got)) == m * math.comb(n - 2, k - 2)
    second = m * math.comb(n - 2, k - 2) + share * math.comb(n - 3, k - 3) + \
        (m * (m - 1) - share) * math.comb(n - 4, k - 4)
    assert sum(c * c * v for c, v in enumerate(got)) == second


def test_kvc_cost_vector(Q, oracle_mod):
    qg, ctx = Q
    n, k = 14, 5
    e = erdos_renyi(n, 0.4, 31)
    c = ctx.cost_precompute("kvc", n, edges=e, k=k, dtype=torch.uint8).cpu().numpy()
    ref = oracle_mod.cost_kvc(n, e, oracle_mod.dicke_states(n, k))
    np.testing.assert_array_equal(c.astype(np.float64), ref)


@pytest.mark.parametrize("case", ["maxcut12", "dks10_4", "kvc11_8"])
def test_grover_qaoa_matches_full_state_oracle(Q, oracle_mod, case):
    qg, ctx = Q
    if case == "maxcut12":
        n, k, prob = 12, -1, "maxcut"
        e = erdos_renyi(n, 0.5, 41)
        cost, st = oracle_mod.cost_maxcut(n, e), None
    elif case == "dks10_4":
        n, k, prob = 10, 4, "dks"
        e = erdos_renyi(n, 0.5, 42)
        st = oracle_mod.dicke_states(n, k)
        cost = oracle_mod.cost_dks(n, e, st)
    else:
        n, k, prob = 11, 8, "kvc"
        e = erdos_renyi(n, 0.4, 43)
        st = oracle_mod.dicke_states(n, k)
        cost = oracle_mod.cost_kvc(n, e, st)
    counts = ctx.cost_degeneracy(prob, n, edges=e, k=k)
    A = uniform_angles(3, 44, 5)
    E, G = ctx.grover_batched(counts, torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    for s in range(5):
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, cost, A[s], "grover", st)
        assert E[s].item() == pytest.approx(E_ref, abs=1e-10 * max(1.0, abs(E_ref)))
        np.testing.assert_allclose(G[s].cpu().numpy(), g_ref, rtol=0, atol=1e-9 * max(1.0, np.abs(g_ref).max()))


def test_grover_qaoa_n100(Q, oracle_mod):
    """Densest 4-subgraph on G(100, 0.5): 3,921,225 states counted on the
    GPU, p = 5; against the oracle's reduced simulation on its own counts."""
    qg, ctx = Q
    n, k = 100, 4
    e = erdos_renyi(n, 0.5, 45)
    counts = ctx.cost_degeneracy("dks", n, edges=e, k=k)
    ref_counts = oracle_mod.cost_degeneracy(n, e, "dks", k, n_bins=counts.shape[0])
    np.testing.assert_array_equal(counts.cpu().numpy(), ref_counts)
    assert int(counts.sum()) == math.comb(n, k)
    A = uniform_angles(5, 46, 3)
    E, G = ctx.grover_batched(counts, torch.from_numpy(A).cuda())
    E2, G2 = ctx.grover_batched(counts, torch.from_numpy(A).cuda(), want_grad=False)
    torch.cuda.synchronize()
    assert G2 is None and torch.equal(E, E2)
    for s in range(3):
        E_ref, g_ref = oracle_mod.grover_reduced_gradient(ref_counts, A[s])
        assert E[s].item() == pytest.approx(E_ref, abs=1e-10 * max(1.0, abs(E_ref)))
        np.testing.assert_allclose(G[s].cpu().numpy(), g_ref, rtol=0, atol=1e-9 * max(1.0, np.abs(g_ref).max()))


def test_degeneracy_argument_checks(Q):
    qg, ctx = Q
    e = erdos_renyi(10, 0.5, 47)
    with pytest.raises(qg.QAOAError):
        ctx.cost_degeneracy("dks", 10, edges=e, k=4, n_bins=6)  # a 4-subset can hold 6 edges: no bin for 6
    with pytest.raises(qg.QAOAError):
        ctx.cost_degeneracy("sk", 10, edges=e)
    with pytest.raises(qg.QAOAError):
        ctx.cost_degeneracy("dks", 129, edges=e, k=3)
    with pytest.raises(qg.QAOAError):
        ctx.cost_degeneracy("dks", 100, edges=e, k=50)  # C(100, 50) states: over the enumeration cap

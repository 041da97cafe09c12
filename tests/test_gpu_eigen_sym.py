"""Parity of the block-diagonal XY mixers (cyclic-shift momentum blocks,
QAOA_MIXER_EIGEN_SYM) with the CPU oracle, which applies e^{-i b H_M} by its
power series on the full Dicke subspace and never forms blocks, a momentum
basis or eigenvectors.  Densest k-subgraph costs, uniform Dicke initial state
unless stated.  Tolerances: |dE| <= 1e-5 max(|E|, sigma_C), |dg_i| <= 1e-4 max|g|.
"""

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, uniform_angles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2312_06451_gb300 as qg

    ctx = qg.Context(0)
    yield qg, ctx
    ctx.close()


def sigma(c):
    return float(np.sqrt(np.mean(np.asarray(c, dtype=np.float64) ** 2)))


def check(E, g, E_ref, g_ref, c):
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c)), (E, E_ref)
    if g is not None:
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


def problem(qg, ctx, oracle_mod, n, k, seed, precision, kind):
    e = erdos_renyi(n, 0.5, seed)
    st = oracle_mod.dicke_states(n, k)
    c = oracle_mod.cost_dks(n, e, st)
    dc = ctx.cost_precompute("dks", n, edges=e, k=k, dtype=torch.uint8)
    return st, c, dc, qg.xy_sym_mixer(ctx, kind, n, k, precision=precision)


@pytest.mark.parametrize("kind", ["ring", "clique"])
@pytest.mark.parametrize("precision", ["fp32", "3xtf32"])
@pytest.mark.parametrize("n,k,p", [(8, 4, 3), (9, 3, 2), (12, 4, 3), (12, 6, 4), (18, 2, 2), (20, 3, 2)])
def test_sym_mixer_expectation_and_gradient(Q, oracle_mod, kind, precision, n, k, p):
    """Even and odd n, orbits shorter than n (n = 12: periods 3, 4, 6), and
    n > 16 (orbits of up to 32 members in the orbit kernel)."""
    qg, ctx = Q
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 300 + n + k, precision, kind)
    assert sum(mixer.block_dims) == len(st)
    ang = uniform_angles(p, 310 + n + k)[0]
    E = ctx.expectation(dc, mixer, ang)
    check(E, None, oracle_mod.qaoa_expectation(n, c, ang, kind, st), None, c)
    E2, g = ctx.gradient(dc, mixer, ang)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, kind, st)
    check(E2, g, E_ref, g_ref, c)


@pytest.mark.parametrize("precision", ["fp32", "3xtf32"])
def test_sym_mixer_batched_ragged_sets(Q, oracle_mod, precision):
    """67 angle sets: two 64-set column tiles, the last ragged."""
    qg, ctx = Q
    n, k, p = 10, 4, 3
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 7, precision, "ring")
    S = 67
    A = uniform_angles(p, 8, S)
    E = torch.zeros(S, dtype=torch.float64, device="cuda")
    G = torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")
    ctx.expectation_batched([{"cost": dc, "mixer": mixer, "angles": torch.from_numpy(A).cuda(), "E": E, "grad": G}],
                            want_grad=True)
    torch.cuda.synchronize()
    for s in (0, 1, 63, 64, 66):
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A[s], "ring", st)
        check(E[s].item(), G[s].cpu().numpy(), E_ref, g_ref, c)


def test_sym_mixer_custom_initial_state_and_dense_path(Q, oracle_mod):
    """A user initial state, and the same numbers as the dense eigenbasis path."""
    qg, ctx = Q
    n, k, p = 9, 4, 2
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 11, "3xtf32", "clique")
    rng = np.random.default_rng(5)
    psi0 = rng.standard_normal(len(st)) + 1j * rng.standard_normal(len(st))
    psi0 /= np.linalg.norm(psi0)
    init = torch.view_as_real(torch.from_numpy(psi0.astype(np.complex64)).cuda()).contiguous()
    ang = uniform_angles(p, 12)[0]
    E, g = ctx.gradient(dc, mixer, ang, init=init)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "clique", st, psi0=psi0)
    check(E, g, E_ref, g_ref, c)
    dense = qg.xy_eigen_mixer(ctx, "clique", n, k, precision="3xtf32")
    E_d, g_d = ctx.gradient(dc, dense, ang, init=init)
    check(E_d, g_d, E_ref, g_ref, c)


def test_sym_mixer_graph_replay(Q, oracle_mod):
    """The batched block-mixer call captured in a CUDA graph after a warm-up
    call, replayed with new angles in the same buffers."""
    qg, ctx = Q
    n, k, p, S = 10, 5, 2, 5
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 21, "3xtf32", "ring")
    A1, A2 = uniform_angles(p, 22, S), uniform_angles(p, 23, S)
    ang = torch.from_numpy(A1).cuda()
    E = torch.zeros(S, dtype=torch.float64, device="cuda")
    G = torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")
    job = [{"cost": dc, "mixer": mixer, "angles": ang, "E": E, "grad": G}]
    s = torch.cuda.Stream()
    qctx = qg.Context(0, s)
    try:
        with torch.cuda.stream(s):
            qctx.expectation_batched(job, want_grad=True)
            s.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                qctx.expectation_batched(job, want_grad=True)
            ang.copy_(torch.from_numpy(A2))
            graph.replay()
        s.synchronize()
        for i in (0, S - 1):
            E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A2[i], "ring", st)
            check(E[i].item(), G[i].cpu().numpy(), E_ref, g_ref, c)
    finally:
        qctx.close()


def test_prepared_operands_follow_the_mixer_not_its_address(Q, oracle_mod):
    """The library keeps padded copies of V per mixer id, not per device
    address: a clique mixer built where a freed ring mixer lived gets its own
    operands; with id 0, V changed in place between calls is picked up."""
    qg, ctx = Q
    n, k, p = 8, 4, 2
    e = erdos_renyi(n, 0.5, 41)
    st = oracle_mod.dicke_states(n, k)
    c = oracle_mod.cost_dks(n, e, st)
    dc = ctx.cost_precompute("dks", n, edges=e, k=k, dtype=torch.uint8)
    ang = uniform_angles(p, 42)[0]
    for precision in ("fp32", "3xtf32"):
        ring = qg.xy_sym_mixer(ctx, "ring", n, k, precision=precision)
        check(*ctx.gradient(dc, ring, ang), *oracle_mod.qaoa_gradient(n, c, ang, "ring", st), c)
        del ring
        clique = qg.xy_sym_mixer(ctx, "clique", n, k, precision=precision)
        check(*ctx.gradient(dc, clique, ang), *oracle_mod.qaoa_gradient(n, c, ang, "clique", st), c)
        # id 0: the operands are rebuilt from V and lambda by every call
        other = qg.xy_sym_mixer(ctx, "ring", n, k, precision=precision)
        clique.struct.id = 0
        check(*ctx.gradient(dc, clique, ang), *oracle_mod.qaoa_gradient(n, c, ang, "clique", st), c)
        clique.V.copy_(other.V)
        clique.lam.copy_(other.lam)
        check(*ctx.gradient(dc, clique, ang), *oracle_mod.qaoa_gradient(n, c, ang, "ring", st), c)
        # the dense path keys its operands the same way
        dense = qg.xy_eigen_mixer(ctx, "clique", n, k, precision=precision)
        dense.struct.id = 0
        check(*ctx.gradient(dc, dense, ang), *oracle_mod.qaoa_gradient(n, c, ang, "clique", st), c)
        dense_ring = qg.xy_eigen_mixer(ctx, "ring", n, k, precision=precision)
        dense.V.copy_(dense_ring.V)
        dense.lam.copy_(dense_ring.lam)
        check(*ctx.gradient(dc, dense, ang), *oracle_mod.qaoa_gradient(n, c, ang, "ring", st), c)


def test_sym_mixer_cache_file_round_trip(Q, oracle_mod, tmp_path):
    """The block eigendecomposition written to a cache file and read back
    gives the same operands and the oracle's numbers; a file for another
    shape or for the dense form is refused."""
    qg, ctx = Q
    n, k, p = 10, 4, 3
    st, c, dc, _ = problem(qg, ctx, oracle_mod, n, k, 21, "3xtf32", "ring")
    path = str(tmp_path / "ring10_4.blocks")
    m1 = qg.xy_sym_mixer(ctx, "ring", n, k, precision="3xtf32", cache_file=path)
    m2 = qg.xy_sym_mixer(ctx, "ring", n, k, precision="3xtf32", cache_file=path)
    assert torch.equal(m1.V, m2.V) and torch.equal(m1.lam, m2.lam) and m1.block_dims == m2.block_dims
    ang = uniform_angles(p, 22)[0]
    E1, g1 = ctx.gradient(dc, m1, ang)
    E2, g2 = ctx.gradient(dc, m2, ang)
    assert E1 == E2 and np.array_equal(g1, g2)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "ring", st)
    check(E2, g2, E_ref, g_ref, c)
    with pytest.raises(ValueError):
        qg.xy_sym_mixer(ctx, "clique", n, k, cache_file=path)
    with pytest.raises(ValueError):
        qg.xy_sym_mixer(ctx, "ring", n, k + 1, cache_file=path)
    dense_path = str(tmp_path / "ring10_4.dense")
    qg.xy_eigen_mixer(ctx, "ring", n, k, cache_file=dense_path)
    with pytest.raises(ValueError):
        qg.xy_sym_mixer(ctx, "ring", n, k, cache_file=dense_path)

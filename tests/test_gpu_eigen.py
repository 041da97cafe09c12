"""Parity of the eigenbasis (constrained) mixer path with the CPU oracle.

The GPU path applies e^{-i b H_M} as V e^{-i b lambda} V^T with V from a
float64 eigendecomposition of the ring or clique Hamiltonian (Sec. 2.1, 2.2); the oracle
applies the same exponential by its power series, never forming V.  Densest
k-subgraph costs on the Dicke subspace, uniform Dicke initial state.
Tolerances as everywhere: |dE| <= 1e-5 max(|E|, sigma_C), |dg| <= 1e-4 max(|g|, sigma_C).
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


def problem(qg, ctx, oracle_mod, n, k, seed, precision="fp32", kind="ring"):
    e = erdos_renyi(n, 0.5, seed)
    st = oracle_mod.dicke_states(n, k)
    c = oracle_mod.cost_dks(n, e, st)
    dc = ctx.cost_precompute("dks", n, edges=e, k=k, dtype=torch.uint8)
    mixer = qg.xy_eigen_mixer(ctx, kind, n, k, precision=precision)
    return st, c, dc, mixer


@pytest.mark.parametrize("kind", ["ring", "clique"])
@pytest.mark.parametrize("n,k", [(5, 2), (8, 4), (9, 3)])
def test_xy_hamiltonian_matches_oracle(Q, oracle_mod, kind, n, k):
    """The library's dense mixer equals the oracle's H_M applied to basis vectors."""
    qg, ctx = Q
    H = (ctx.ring_hamiltonian(n, k) if kind == "ring" else ctx.clique_hamiltonian(n, k)).cpu().numpy()
    st = oracle_mod.dicke_states(n, k)
    D = len(st)
    ref = np.stack([oracle_mod.hm_apply(n, np.eye(D)[i], kind, st) for i in range(D)], axis=1).real
    np.testing.assert_array_equal(H, ref)


@pytest.mark.parametrize("precision", ["fp32", "3xtf32"])
@pytest.mark.parametrize("n,k,p", [(8, 4, 3), (10, 3, 2)])
def test_clique_mixer_expectation_and_gradient(Q, oracle_mod, n, k, p, precision):
    qg, ctx = Q
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 90 + n, precision, "clique")
    ang = uniform_angles(p, 91 + n)[0]
    E, g = ctx.gradient(dc, mixer, ang)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "clique", st)
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c)), (E, E_ref)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


PRECISIONS = ["fp32", "3xtf32"]


@pytest.mark.parametrize("n,k", [(8, 4), (10, 5), (12, 6)])
def test_eigen_decomposition_is_an_eigenbasis(Q, n, k):
    qg, ctx = Q
    mixer = qg.ring_eigen_mixer(ctx, n, k)
    H = ctx.ring_hamiltonian(n, k)
    V = mixer.V.double()
    res = (H @ V - V * mixer.lam[None, :]).abs().max().item()
    orth = (V.T @ V - torch.eye(V.shape[0], device=V.device, dtype=V.dtype)).abs().max().item()
    assert res < 1e-5 and orth < 1e-5, (res, orth)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n,k,p", [(8, 4, 3), (10, 5, 2), (12, 6, 4)])
def test_eigen_expectation_and_gradient(Q, oracle_mod, n, k, p, precision):
    qg, ctx = Q
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 50 + n, precision)
    ang = uniform_angles(p, 60 + n)[0]
    E = ctx.expectation(dc, mixer, ang)
    E_ref = oracle_mod.qaoa_expectation(n, c, ang, "ring", st)
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c)), (E, E_ref)
    E2, g = ctx.gradient(dc, mixer, ang)
    E_ref2, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "ring", st)
    assert abs(E2 - E_ref2) <= 1e-5 * max(abs(E_ref2), sigma(c))
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


@pytest.mark.parametrize("precision", PRECISIONS)
def test_eigen_batched_ragged_sets(Q, oracle_mod, precision):
    """67 angle sets: more than one 64-set column tile, the last one ragged."""
    qg, ctx = Q
    n, k, p = 10, 4, 3
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 7, precision)
    S = 67
    A = uniform_angles(p, 8, S)
    E = torch.zeros(S, dtype=torch.float64, device="cuda")
    G = torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")
    ctx.expectation_batched([{"cost": dc, "mixer": mixer, "angles": torch.from_numpy(A).cuda(), "E": E, "grad": G}],
                            want_grad=True)
    torch.cuda.synchronize()
    for s in (0, 1, 63, 64, 66):
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A[s], "ring", st)
        assert abs(E[s].item() - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c))
        np.testing.assert_allclose(G[s].cpu().numpy(), g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


@pytest.mark.parametrize("precision", PRECISIONS)
def test_eigen_custom_initial_state(Q, oracle_mod, precision):
    qg, ctx = Q
    n, k, p = 8, 3, 2
    st, c, dc, mixer = problem(qg, ctx, oracle_mod, n, k, 9, precision)
    rng = np.random.default_rng(4)
    psi0 = rng.standard_normal(len(st)) + 1j * rng.standard_normal(len(st))
    psi0 /= np.linalg.norm(psi0)
    init = torch.view_as_real(torch.from_numpy(psi0.astype(np.complex64)).cuda()).contiguous()
    ang = uniform_angles(p, 10)[0]
    E, g = ctx.gradient(dc, mixer, ang, init=init)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "ring", st, psi0=psi0)
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c))
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


def test_eigen_mixer_file_cache(Q, tmp_path):
    qg, ctx = Q
    path = str(tmp_path / "ring_8_4.npz")
    m1 = qg.ring_eigen_mixer(ctx, 8, 4, cache_file=path)
    m2 = qg.ring_eigen_mixer(ctx, 8, 4, cache_file=path)
    assert torch.equal(m1.V, m2.V) and torch.equal(m1.lam, m2.lam)
    with pytest.raises(ValueError):
        qg.load_eigen_mixer(path, 8, 5)          # wrong shape
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0xFF                   # damage the file
    open(path, "wb").write(bytes(raw))
    with pytest.raises(ValueError):
        qg.load_eigen_mixer(path, 8, 4)

"""Parity of the CUDA path with the CPU oracle, element by element, through
the C ABI.

Tolerances (complex64 state, float64 reductions):
  cost vectors   bit-exact for integer costs; SK on the 2^-20 coupling grid is
                 bit-exact to float32(round-to-nearest(exact sum))
  <C>            |dE| <= 1e-5 * max(|E|, sigma_C)
  gradient       |dg_i| <= 1e-4 * max|g|   (relative to the largest component)
with sigma_C the RMS of C over the feasible set.
"""

import math

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, random_regular3, sk_couplings, uniform_angles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2312_06451_gb300 as qg

    ctx = qg.Context(0)
    yield ctx
    ctx.close()


def sigma(cost):
    return float(np.sqrt(np.mean(np.asarray(cost, dtype=np.float64) ** 2)))


def assert_E(E, E_ref, cost):
    tol = 1e-5 * max(abs(E_ref), sigma(cost))
    assert abs(E - E_ref) <= tol, (E, E_ref, tol)


def assert_grad(g, g_ref, cost):
    tol = 1e-4 * np.abs(g_ref).max()
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=tol)


def maxcut_instance(n, seed):
    return random_regular3(n, seed) if n % 2 == 0 and n >= 6 and seed % 2 else erdos_renyi(n, 0.5, seed)


# ------------------------------------------------------------ cost vectors

@pytest.mark.parametrize("n,seed", [(3, 1), (12, 2), (16, 3), (20, 5), (21, 4)])
def test_cost_maxcut_bit_exact(Q, oracle_mod, n, seed):
    e = maxcut_instance(n, seed)
    ref = oracle_mod.cost_maxcut(n, e)
    got8 = Q.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8).cpu().numpy()
    np.testing.assert_array_equal(got8.astype(np.float64), ref)
    got32 = Q.cost_precompute("maxcut", n, edges=e, dtype=torch.float32).cpu().numpy()
    np.testing.assert_array_equal(got32.astype(np.float64), ref)


def test_cost_weighted_maxcut(Q, oracle_mod):
    n = 14
    e = erdos_renyi(n, 0.4, 8)
    w = np.random.default_rng(1).random(len(e)).astype(np.float32) * 3
    ref = oracle_mod.cost_maxcut(n, e, weights=w.astype(np.float64))
    got = Q.cost_precompute("wmaxcut", n, edges=e, weights=w, dtype=torch.float32).cpu().numpy()
    np.testing.assert_array_equal(got, ref.astype(np.float32))


@pytest.mark.parametrize("n,seed", [(2, 1), (9, 2), (16, 3), (22, 4)])
def test_cost_sk_exact(Q, oracle_mod, n, seed):
    J = sk_couplings(n, seed)
    ref = oracle_mod.cost_sk(n, J.astype(np.float64))
    got = Q.cost_precompute("sk", n, J=J, dtype=torch.float32).cpu().numpy()
    np.testing.assert_array_equal(got, ref.astype(np.float32))


def test_cost_sk_off_grid_within_one_ulp(Q, oracle_mod):
    n = 12
    J = np.random.default_rng(3).standard_normal((n, n)).astype(np.float32)
    J = np.triu(J, 1) + np.triu(J, 1).T
    ref = oracle_mod.cost_sk(n, J.astype(np.float64)).astype(np.float32)
    got = Q.cost_precompute("sk", n, J=J, dtype=torch.float32).cpu().numpy()
    ulp = np.spacing(np.abs(ref))
    assert np.all(np.abs(got - ref) <= ulp)


@pytest.mark.parametrize("n,k", [(6, 3), (10, 1), (16, 8), (20, 10)])
def test_dicke_and_dks_cost_bit_exact(Q, oracle_mod, n, k):
    st = oracle_mod.dicke_states(n, k)
    np.testing.assert_array_equal(Q.dicke_states(n, k).cpu().numpy().astype(np.uint64), st)
    e = erdos_renyi(n, 0.5, n + k)
    ref = oracle_mod.cost_dks(n, e, st)
    got = Q.cost_precompute("dks", n, edges=e, k=k, dtype=torch.uint8).cpu().numpy()
    np.testing.assert_array_equal(got.astype(np.float64), ref)


@pytest.mark.parametrize("n,k", [(5, 2), (8, 4), (9, 3)])
def test_ring_hamiltonian_matches_oracle(Q, oracle_mod, n, k):
    st = oracle_mod.dicke_states(n, k)
    D = len(st)
    ref = np.stack([oracle_mod.hm_apply(n, np.eye(D)[i], "ring", st) for i in range(D)], axis=1).real
    got = Q.ring_hamiltonian(n, k).cpu().numpy()
    np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------- <C> and gradient

# sizes cover: whole state on chip (n <= 12), one tile (n = 13), two passes
# per round (14..22), three passes (>= 23)
SIZES = [2, 5, 12, 13, 14, 17, 22, 23]


def problem(Q, oracle_mod, n, kind, seed):
    if kind == "maxcut_u8":
        e = maxcut_instance(n, seed) if n > 1 else np.zeros((0, 2), np.int32)
        return Q.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8), oracle_mod.cost_maxcut(n, e)
    J = sk_couplings(n, seed)
    return Q.cost_precompute("sk", n, J=J, dtype=torch.float32), oracle_mod.cost_sk(n, J.astype(np.float64))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind", ["maxcut_u8", "sk_f32"])
def test_expectation_matches_oracle(Q, oracle_mod, n, kind):
    import paper_2312_06451_gb300 as qg

    p = 3
    dc, c = problem(Q, oracle_mod, n, kind, 100 + n)
    for s, ang in enumerate(uniform_angles(p, 7 * n, 2)):
        E = Q.expectation(dc, qg.XMixer(n), ang)
        assert_E(E, oracle_mod.qaoa_expectation(n, c, ang), c)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("kind,ckpt", [("maxcut_u8", True), ("sk_f32", True), ("sk_f32", False)])
def test_gradient_matches_oracle(Q, oracle_mod, n, kind, ckpt):
    import paper_2312_06451_gb300 as qg

    p = 3
    dc, c = problem(Q, oracle_mod, n, kind, 200 + n)
    ang = uniform_angles(p, 11 * n)[0]
    E, g = Q.gradient(dc, qg.XMixer(n), ang, ckpt=ckpt)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang)
    assert_E(E, E_ref, c)
    assert_grad(g, g_ref, c)


@pytest.mark.parametrize("n", [4, 12, 13, 16])
def test_custom_initial_state(Q, oracle_mod, n):
    """Warm start (initial_state of Sec. 3): a normalised complex psi_0."""
    import paper_2312_06451_gb300 as qg

    p = 2
    J = sk_couplings(n, 5)
    c = oracle_mod.cost_sk(n, J.astype(np.float64))
    dc = Q.cost_precompute("sk", n, J=J, dtype=torch.float32)
    rng = np.random.default_rng(n)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    init = torch.from_numpy(psi0.astype(np.complex64)).cuda()
    ang = uniform_angles(p, 3)[0]
    E, g = Q.gradient(dc, qg.XMixer(n), ang, init=torch.view_as_real(init).contiguous())
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, psi0=psi0)
    assert_E(E, E_ref, c)
    assert_grad(g, g_ref, c)


@pytest.mark.parametrize("kind", ["maxcut_u8", "sk_f32"])
def test_n12_rotation_regimes(Q, oracle_mod, kind):
    """n = 12 runs as one register-staged tile; betas in every rotation form:
    tan form (beta = 0.1, 2.9), tan form with per-stage rescaling
    (|cos beta| < 1/4 at beta = 1.4) and the direct form (beta = pi / 2)."""
    import paper_2312_06451_gb300 as qg

    n = 12
    if kind == "maxcut_u8":
        e = erdos_renyi(n, 0.5, 31)
        c = oracle_mod.cost_maxcut(n, e)
        dc = Q.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
    else:
        J = sk_couplings(n, 32)
        c = oracle_mod.cost_sk(n, J.astype(np.float64))
        dc = Q.cost_precompute("sk", n, J=J, dtype=torch.float32)
    ang = np.array([0.1, 1.4, np.pi / 2, 2.9, 0.7, 1.9, 0.3, 2.5])
    E, g = Q.gradient(dc, qg.XMixer(n), ang)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang)
    assert_E(E, E_ref, c)
    assert_grad(g, g_ref, c)
    assert_E(Q.expectation(dc, qg.XMixer(n), ang), E_ref, c)


@pytest.mark.parametrize("n,kind", [(18, "maxcut_u8"), (22, "sk_f32")])
def test_pass_rotation_regimes(Q, oracle_mod, n, kind):
    """The pass kernels with fused round boundaries in every combination of
    rotation forms: betas 0.1 (tan form), pi/2 (direct form: |cos b| tiny),
    pi/2, 1.4 (tan form with per-stage rescaling), 2.9, so the boundaries
    see tan-direct, direct-direct, direct-tan and tan-tan."""
    import paper_2312_06451_gb300 as qg

    if kind == "maxcut_u8":
        e = erdos_renyi(n, 0.4, 41)
        c = oracle_mod.cost_maxcut(n, e)
        dc = Q.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
    else:
        J = sk_couplings(n, 42)
        c = oracle_mod.cost_sk(n, J.astype(np.float64))
        dc = Q.cost_precompute("sk", n, J=J, dtype=torch.float32)
    ang = np.array([0.1, np.pi / 2, np.pi / 2, 1.4, 2.9, 0.7, 1.9, 0.3, 2.5, 1.1])
    E, g = Q.gradient(dc, qg.XMixer(n), ang, ckpt="pass")
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang)
    assert_E(E, E_ref, c)
    assert_grad(g, g_ref, c)
    assert_E(Q.expectation(dc, qg.XMixer(n), ang), E_ref, c)


def test_many_rounds(Q, oracle_mod):
    import paper_2312_06451_gb300 as qg

    n, p = 15, 12
    e = erdos_renyi(n, 0.5, 3)
    c = oracle_mod.cost_maxcut(n, e)
    dc = Q.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
    ang = uniform_angles(p, 4)[0]
    E, g = Q.gradient(dc, qg.XMixer(n), ang)
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang)
    assert_E(E, E_ref, c)
    assert_grad(g, g_ref, c)


def test_batched_uneven_jobs(Q, oracle_mod):
    """Many instances of uneven n, several angle sets each, one batched call."""
    import paper_2312_06451_gb300 as qg

    p = 3
    jobs, refs = [], []
    for i, n in enumerate([10, 14, 17, 13, 21, 14]):
        e = maxcut_instance(n, 30 + i)
        c = oracle_mod.cost_maxcut(n, e)
        dc = Q.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
        A = uniform_angles(p, 40 + i, 3)
        jobs.append({"cost": dc, "mixer": qg.XMixer(n), "angles": torch.from_numpy(A).cuda(),
                     "E": torch.zeros(3, dtype=torch.float64, device="cuda"),
                     "grad": torch.zeros(3, 2 * p, dtype=torch.float64, device="cuda")})
        refs.append((n, c, A))
    Q.expectation_batched(jobs, want_grad=True)
    torch.cuda.synchronize()
    for j, (n, c, A) in zip(jobs, refs):
        for s in range(3):
            E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A[s])
            assert_E(j["E"][s].item(), E_ref, c)
            assert_grad(j["grad"][s].cpu().numpy(), g_ref, c)


def test_batched_uneven_sk_gradients_repeat_bitwise(Q, oracle_mod):
    """Float costs in one batched call over uneven n (13..21 qubits): a step
    launch mixes descriptors that read the cost (the first adjoint pass of one
    job, the phase pass of another) with ones that do not, and tiles are
    claimed dynamically.  Gradients match the oracle, and a repeat of the call
    gives bitwise the same E and gradients (every partial sum has its slot)."""
    import paper_2312_06451_gb300 as qg

    p, S = 3, 2
    jobs, refs = [], []
    for i, n in enumerate([13, 21, 16, 19, 14]):
        J = sk_couplings(n, 60 + i)
        c = oracle_mod.cost_sk(n, J.astype(np.float64))
        dc = Q.cost_precompute("sk", n, J=J, dtype=torch.float32)
        A = uniform_angles(p, 70 + i, S)
        jobs.append({"cost": dc, "mixer": qg.XMixer(n), "angles": torch.from_numpy(A).cuda(),
                     "E": torch.zeros(S, dtype=torch.float64, device="cuda"),
                     "grad": torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")})
        refs.append((n, c, A))
    Q.expectation_batched(jobs, want_grad=True)
    torch.cuda.synchronize()
    first = [(j["E"].clone(), j["grad"].clone()) for j in jobs]
    for j, (n, c, A) in zip(jobs, refs):
        for s in range(S):
            E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A[s])
            assert_E(j["E"][s].item(), E_ref, c)
            assert_grad(j["grad"][s].cpu().numpy(), g_ref, c)
    Q.expectation_batched(jobs, want_grad=True)
    torch.cuda.synchronize()
    for j, (E0, g0) in zip(jobs, first):
        assert torch.equal(j["E"], E0) and torch.equal(j["grad"], g0)


def test_batched_expectation_only_and_replay(Q, oracle_mod):
    """A repeated identical batched call reuses its plan and gives bitwise
    identical results; new angles in the same buffers are picked up."""
    import paper_2312_06451_gb300 as qg

    n, p = 16, 2
    J = sk_couplings(n, 9)
    c = oracle_mod.cost_sk(n, J.astype(np.float64))
    dc = Q.cost_precompute("sk", n, J=J, dtype=torch.float32)
    A = torch.from_numpy(uniform_angles(p, 1, 5)).cuda()
    E = torch.zeros(5, dtype=torch.float64, device="cuda")
    job = [{"cost": dc, "mixer": qg.XMixer(n), "angles": A, "E": E}]
    Q.expectation_batched(job)
    torch.cuda.synchronize()
    first = E.clone()
    Q.expectation_batched(job)
    torch.cuda.synchronize()
    assert torch.equal(first, E)
    A.copy_(torch.from_numpy(uniform_angles(p, 2, 5)))
    Q.expectation_batched(job)
    torch.cuda.synchronize()
    for s in range(5):
        assert_E(E[s].item(), oracle_mod.qaoa_expectation(n, c, A[s].cpu().numpy()), c)


def test_autograd_function(Q, oracle_mod):
    import paper_2312_06451_gb300 as qg

    n, p = 14, 2
    e = erdos_renyi(n, 0.5, 2)
    c = oracle_mod.cost_maxcut(n, e)
    dc = Q.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
    ang = torch.tensor(uniform_angles(p, 5)[0], requires_grad=True)
    E = qg.QAOAExpectation.apply(ang, Q, dc, qg.XMixer(n))
    (3.0 * E).backward()
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang.detach().numpy())
    assert_E(E.item(), E_ref, c)
    assert_grad(ang.grad.numpy() / 3.0, g_ref, c)


def test_deterministic(Q):
    import paper_2312_06451_gb300 as qg

    n = 18
    dc = Q.cost_precompute("sk", n, J=sk_couplings(n, 1), dtype=torch.float32)
    ang = uniform_angles(4, 3)[0]
    r1 = Q.gradient(dc, qg.XMixer(n), ang)
    r2 = Q.gradient(dc, qg.XMixer(n), ang)
    assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1])


def test_invalid_arguments_raise(Q):
    import paper_2312_06451_gb300 as qg
    from paper_2312_06451_gb300 import QAOAError

    n = 10
    dc = Q.cost_precompute("maxcut", n, edges=erdos_renyi(n, 0.5, 1), dtype=torch.uint8)
    with pytest.raises(QAOAError):
        Q.expectation(dc, qg.XMixer(n), [])            # p = 0
    with pytest.raises(QAOAError):
        Q.expectation(dc, qg.XMixer(n), [0.1, float("nan")])
    bad = qg.XMixer(n)
    bad.struct.dim = 5
    with pytest.raises(QAOAError):
        Q.expectation(dc, bad, [0.1, 0.2])
    with pytest.raises(QAOAError):
        Q.cost_precompute("maxcut", n, edges=[[0, 0]])   # self loop
    with pytest.raises(QAOAError):
        Q.cost_precompute("maxcut", 4, edges=[[0, 9]])   # vertex out of range
    # the context stays usable
    assert math.isfinite(Q.expectation(dc, qg.XMixer(n), [0.1, 0.2]))

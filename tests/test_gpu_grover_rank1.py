"""Grover mixer as a rank-one update on the stored state (QAOA_MIXER_GROVER,
Sec. 2.4) against the CPU oracle, which applies e^{-i b |u><u|} to the full
complex128 vector of whatever feasible set the cost vector covers.

Cases: all 2^n states and the Hamming-weight-k subspace (odd dimension, so the
last amplitude pair of a tile is ragged), uint8 and float32 costs, a warm
start, both checkpoint modes (p + 1 vectors, or two vectors with each round
undone on the state), batches mixing dimensions and round counts down to a
single feasible state, CUDA-graph replay, and at full size the reduction to
cost degeneracies (the Grover-mixer QAOA depends on the cost histogram only).
Tolerances: |dE| <= 1e-5 max(|E|, sigma_C), |dg_i| <= 1e-4 max|g|, at angles
where the mixer acts: gamma up to about 1/std(C) (beyond that the phases
decorrelate, e^{-i g C} averages out over the feasible set, the overlap <u|phi>
and with it the whole gradient drop towards zero).  With gamma over [0, pi)
the gradient can sit 1e-6 below its natural scale Var(C), and complex64 states
cannot resolve it to 1e-4 of itself: the Grover-mixer state is a function of
the cost value alone, so every state of one cost class carries the same
float32 rounding of e^{-i g c} and the roundings add up instead of averaging
out.  That case is checked against a floor of 1e-7 Var(C) (test_wide_angles).
"""

import math

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, ramp_angles, sk_couplings, uniform_angles

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


def check(E, g, E_ref, g_ref, c, floor=0.0):
    sig = sigma(c)
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sig), (E, E_ref)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=max(1e-4 * np.abs(g_ref).max(), floor))


def full_problem(ctx, oracle_mod, n, seed, f32):
    if f32:
        J = sk_couplings(n, seed)
        return ctx.cost_precompute("sk", n, J=J, dtype=torch.float32), oracle_mod.cost_sk(n, J.astype(np.float64))
    e = erdos_renyi(n, 0.4, seed)
    return ctx.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8), oracle_mod.cost_maxcut(n, e)


def dicke_problem(ctx, oracle_mod, n, k, seed, f32=False):
    e = erdos_renyi(n, 0.5, seed)
    st = oracle_mod.dicke_states(n, k)
    c = oracle_mod.cost_dks(n, e, st)
    dc = ctx.cost_precompute("dks", n, edges=e, k=k, dtype=torch.uint8)
    if f32:
        dc = dc.to(torch.float32).contiguous()
    return dc, c


def scaled_angles(p, seed, c, n_sets=1):
    """beta ~ U[0, pi), gamma ~ U[0, 1 / std(C)): the range where the Grover
    mixer changes the state (see the module docstring)."""
    A = uniform_angles(p, seed, n_sets)
    A[:, p:] /= np.pi * max(float(np.std(c)), 1e-3)
    return A


def angle_sets(p, seed, c):
    """A random set in the acting range and the smooth ramp schedule."""
    return [scaled_angles(p, seed, c)[0], ramp_angles(p)[0]]


@pytest.mark.parametrize("n,p,f32", [(3, 2, True), (10, 3, False), (16, 2, True), (21, 4, False), (22, 3, True)])
def test_full_space(Q, oracle_mod, n, p, f32):
    qg, ctx = Q
    cost, c = full_problem(ctx, oracle_mod, n, 700 + n, f32)
    mixer = qg.GroverMixer.full(n)
    for ang in angle_sets(p, 710 + n, c):
        E, g = ctx.gradient(cost, mixer, ang)
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover")
        check(E, g, E_ref, g_ref, c)
        assert ctx.expectation(cost, mixer, ang) == pytest.approx(E_ref, abs=1e-5 * max(abs(E_ref), sigma(c)))


@pytest.mark.parametrize("n,p,f32", [(21, 4, False), (22, 3, True)])
def test_wide_angles(Q, oracle_mod, n, p, f32):
    """gamma over [0, pi): <C> to 1e-5; the gradient to 1e-4 of itself or
    1e-7 Var(C), whichever is larger (the complex64 resolution for a state
    that is a function of the cost value; see the module docstring)."""
    qg, ctx = Q
    cost, c = full_problem(ctx, oracle_mod, n, 700 + n, f32)
    mixer = qg.GroverMixer.full(n)
    for s in range(3):
        ang = uniform_angles(p, 715 + n + s)[0]
        E, g = ctx.gradient(cost, mixer, ang)
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover")
        check(E, g, E_ref, g_ref, c, floor=1e-7 * float(np.var(c)))


@pytest.mark.parametrize("n,k,p,f32", [(15, 7, 3, False), (16, 6, 2, True), (20, 9, 3, False), (9, 0, 2, False),
                                       (12, 2, 3, True)])
def test_dicke_subspace(Q, oracle_mod, n, k, p, f32):
    """u is the Dicke state; C(15, 7) = 6435 and C(20, 9) = 167960 leave a
    ragged last tile (6435 is odd: a lone last amplitude)."""
    qg, ctx = Q
    cost, c = dicke_problem(ctx, oracle_mod, n, k, 720 + n + k, f32)
    mixer = qg.GroverMixer.dicke(n, k)
    assert mixer.dim == math.comb(n, k) == c.shape[0]
    for ang in angle_sets(p, 730 + n, c):
        E, g = ctx.gradient(cost, mixer, ang)
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover")
        if k == 0:  # one feasible state: <C> is its cost and nothing moves
            assert E == pytest.approx(c[0], abs=1e-5 * max(abs(c[0]), 1.0)) and np.abs(g).max() < 1e-6
            continue
        check(E, g, E_ref, g_ref, c)


@pytest.mark.parametrize("space", ["full", "dicke"])
def test_warm_start(Q, oracle_mod, space):
    """A user initial state (Sec. 3, initial_state); the oracle gets the same
    complex64 values widened to complex128."""
    qg, ctx = Q
    p = 3
    if space == "full":
        n = 14
        cost, c = full_problem(ctx, oracle_mod, n, 740, True)
        mixer = qg.GroverMixer.full(n)
    else:
        n, k = 14, 5
        cost, c = dicke_problem(ctx, oracle_mod, n, k, 741)
        mixer = qg.GroverMixer.dicke(n, k)
    rng = np.random.default_rng(742)
    psi0 = rng.standard_normal(mixer.dim) + 1j * rng.standard_normal(mixer.dim)
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex64)
    init = torch.view_as_real(torch.from_numpy(psi0).cuda()).contiguous()
    for ang in angle_sets(p, 743, c):
        E, g = ctx.gradient(cost, mixer, ang, init=init)
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover", psi0=psi0.astype(np.complex128))
        check(E, g, E_ref, g_ref, c)


def test_checkpoint_modes_agree(Q, oracle_mod):
    """p + 1 stored vectors (round checkpoints) and two vectors with the
    forward round undone on the state: both match the oracle."""
    qg, ctx = Q
    n, p = 19, 6
    cost, c = full_problem(ctx, oracle_mod, n, 750, False)
    mixer = qg.GroverMixer.full(n)
    ang = ramp_angles(p)[0]
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover")
    for mode in ("round", "pass", "none"):
        E, g = ctx.gradient(cost, mixer, ang, ckpt=mode)
        check(E, g, E_ref, g_ref, c)


def test_batched_mixed(Q, oracle_mod):
    """One batched call: full-space and Dicke jobs, two round counts (so two
    launch groups), a three-state and a one-state feasible set, uint8 and
    float32 costs, several angle sets each."""
    qg, ctx = Q
    S = 3
    specs = []
    cost, c = full_problem(ctx, oracle_mod, 17, 760, False)
    specs.append((17, cost, c, qg.GroverMixer.full(17), 3))
    cost, c = dicke_problem(ctx, oracle_mod, 13, 6, 761, f32=True)
    specs.append((13, cost, c, qg.GroverMixer.dicke(13, 6), 3))
    cost, c = full_problem(ctx, oracle_mod, 11, 762, True)
    specs.append((11, cost, c, qg.GroverMixer.full(11), 2))
    c3 = np.array([2.0, 5.0, 1.0])
    specs.append((2, torch.tensor(c3, dtype=torch.float32, device="cuda"), c3, qg.GroverMixer(3, 2), 2))
    c1 = np.array([4.0])
    specs.append((1, torch.tensor(c1, dtype=torch.float32, device="cuda"), c1, qg.GroverMixer(1, 1), 3))
    jobs = []
    for j, (n, cost, c, mixer, p) in enumerate(specs):
        A = scaled_angles(p, 770 + j, c, S)
        jobs.append({"cost": cost, "mixer": mixer, "angles": torch.from_numpy(A).cuda(),
                     "E": torch.zeros(S, dtype=torch.float64, device="cuda"),
                     "grad": torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda"), "A": A})
    ctx.expectation_batched(jobs, want_grad=True)
    torch.cuda.synchronize()
    for (n, cost, c, mixer, p), jb in zip(specs, jobs):
        for s in range(S):
            E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, jb["A"][s], "grover")
            E, g = jb["E"][s].item(), jb["grad"][s].cpu().numpy()
            if c.shape[0] == 1:
                assert E == pytest.approx(c[0], abs=1e-5 * abs(c[0])) and np.abs(g).max() < 1e-6
            else:
                check(E, g, E_ref, g_ref, c)


def test_graph_replay(Q, oracle_mod):
    """The batched call captured in a CUDA graph after one warm-up call and
    replayed with new angles in the same buffers."""
    qg, ctx = Q
    n, k, p, S = 16, 7, 3, 4
    cost, c = dicke_problem(ctx, oracle_mod, n, k, 780)
    mixer = qg.GroverMixer.dicke(n, k)
    A1, A2 = scaled_angles(p, 781, c, S), scaled_angles(p, 782, c, S)
    ang = torch.from_numpy(A1).cuda()
    E = torch.zeros(S, dtype=torch.float64, device="cuda")
    G = torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")
    job = [{"cost": cost, "mixer": mixer, "angles": ang, "E": E, "grad": G}]
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
        for i in range(S):
            E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A2[i], "grover")
            check(E[i].item(), G[i].cpu().numpy(), E_ref, g_ref, c)
    finally:
        qctx.close()


def test_matches_general_x_path(Q, oracle_mod):
    """The same full-space Grover mixer through the general X-mixer passes
    (Hadamard-basis weights [1, 0, ..., 0]): both paths agree with the oracle."""
    qg, ctx = Q
    n, p = 18, 3
    cost, c = full_problem(ctx, oracle_mod, n, 790, True)
    ang = ramp_angles(p)[0]
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover")
    E1, g1 = ctx.gradient(cost, qg.GroverMixer.full(n), ang)
    check(E1, g1, E_ref, g_ref, c)
    E2, g2 = ctx.gradient(cost, qg.grover_x_mixer(n), ang, ckpt="pass")
    assert abs(E2 - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c))


def test_invalid_arguments(Q):
    qg, ctx = Q
    cost = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        qg.GroverMixer(0)
    bad = qg.GroverMixer(64, 6)
    bad.struct.dim = 0
    with pytest.raises(qg.QAOAError):
        ctx.expectation(cost, bad, [0.1, 0.2])
    init = torch.zeros(2 * 65, dtype=torch.float32, device="cuda")[2:]  # 8-byte, not 16-byte aligned
    with pytest.raises(qg.QAOAError):
        ctx.expectation(cost, qg.GroverMixer(64, 6), [0.1, 0.2], init=init)


def test_full_size_against_degeneracies(Q, oracle_mod):
    """3-regular MaxCut at n = 28, p = 8 (2^28 amplitudes, 2 GiB a vector):
    the Grover-mixer QAOA depends on the costs only through their histogram,
    so the oracle's brute-force count and its reduced-vector reverse mode give
    <C> and the gradient exactly.  Batched sets with round checkpoints, and the
    host-pointer call with two vectors."""
    from qaoa_inputs import random_regular3

    qg, ctx = Q
    n, p, S = 28, 8, 2
    e = random_regular3(n, 5)
    counts = oracle_mod.cost_degeneracy(n, e, "maxcut")
    cost = ctx.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
    sig = float(np.sqrt((counts * np.arange(counts.shape[0]) ** 2.0).sum() / counts.sum()))
    vals = np.arange(counts.shape[0], dtype=np.float64)
    mean = (counts * vals).sum() / counts.sum()
    std = float(np.sqrt((counts * (vals - mean) ** 2).sum() / counts.sum()))
    A = np.stack([ramp_angles(p)[0], uniform_angles(p, 800)[0]])
    A[1, p:] /= np.pi * std
    mixer = qg.GroverMixer.full(n)
    E = torch.zeros(S, dtype=torch.float64, device="cuda")
    G = torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")
    ctx.expectation_batched([{"cost": cost, "mixer": mixer, "angles": torch.from_numpy(A).cuda(), "E": E,
                              "grad": G}], want_grad=True)
    torch.cuda.synchronize()
    for s in range(S):
        E_ref, g_ref = oracle_mod.grover_reduced_gradient(counts, A[s])
        assert abs(E[s].item() - E_ref) <= 1e-5 * max(abs(E_ref), sig), (E[s].item(), E_ref)
        np.testing.assert_allclose(G[s].cpu().numpy(), g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())
    E2, g2 = ctx.gradient(cost, mixer, A[0], ckpt="none")
    E_ref, g_ref = oracle_mod.grover_reduced_gradient(counts, A[0])
    assert abs(E2 - E_ref) <= 1e-5 * max(abs(E_ref), sig)
    np.testing.assert_allclose(g2, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


def test_state_limit_steps_down_then_refuses(Q, oracle_mod):
    """Under a state cap the rank-one path keeps two vectors instead of p + 1
    (each adjoint pass then undoes its round on the state) and still matches
    the oracle; below two vectors the call fails with QAOA_ERR_OOM before any
    launch, and the context works again once the cap is lifted."""
    qg, ctx = Q
    n, p = 20, 4
    cost, c = full_problem(ctx, oracle_mod, n, 810, False)
    mixer = qg.GroverMixer.full(n)
    ang = ramp_angles(p)[0]
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover")
    vec = (1 << n) * 8
    with qg.Context(0) as cx:
        cx.set_state_limit(int(2.5 * vec))  # two vectors fit, p + 1 = 5 do not
        E, g = cx.gradient(cost, mixer, ang, ckpt="round")
        check(E, g, E_ref, g_ref, c)
        cx.set_state_limit(vec)  # not even two
        with pytest.raises(qg.QAOAError) as ei:
            cx.gradient(cost, mixer, ang, ckpt="round")
        from paper_2312_06451_gb300 import _binding as B

        assert ei.value.status == B.QAOA_ERR_OOM
        cx.set_state_limit(None)
        E, g = cx.gradient(cost, mixer, ang, ckpt="round")
        check(E, g, E_ref, g_ref, c)


def test_autograd_with_grover_mixer(Q, oracle_mod):
    """QAOAExpectation (the torch.autograd.Function) over the rank-one Grover
    path: backward gives the oracle's gradient, and a few plain gradient-ascent
    steps raise <C> (the angle-finding use of Sec. 2.3)."""
    qg, ctx = Q
    n, p = 14, 3
    cost, c = full_problem(ctx, oracle_mod, n, 820, False)
    mixer = qg.GroverMixer.full(n)
    a0 = ramp_angles(p)[0]
    ang = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    E = qg.QAOAExpectation.apply(ang, ctx, cost, mixer)
    E.backward()
    E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, a0, "grover")
    check(E.item(), ang.grad.numpy(), E_ref, g_ref, c)
    x = torch.tensor(a0, dtype=torch.float64, requires_grad=True)
    E_first = None
    for _ in range(5):
        x.grad = None
        Ex = qg.QAOAExpectation.apply(x, ctx, cost, mixer)
        E_first = Ex.item() if E_first is None else E_first
        Ex.backward()
        with torch.no_grad():
            x += 0.01 * x.grad / max(1.0, float(x.grad.abs().max()))
    assert qg.QAOAExpectation.apply(x.detach(), ctx, cost, mixer).item() > E_first


def test_mixed_batch_with_x_mixer_graph_replay(Q, oracle_mod):
    """One batched call holding an X-mixer job and Grover-mixer jobs (full
    space and Dicke), captured in a CUDA graph and replayed with new angles."""
    qg, ctx = Q
    S, p = 2, 3
    cx, c = full_problem(ctx, oracle_mod, 16, 830, True)
    cd, cdk = dicke_problem(ctx, oracle_mod, 14, 6, 831)
    specs = [(16, cx, c, qg.XMixer(16), None), (16, cx, c, qg.GroverMixer.full(16), "grover"),
             (14, cd, cdk, qg.GroverMixer.dicke(14, 6), "grover")]
    jobs = []
    for j, (n, cost, cc, mixer, kind) in enumerate(specs):
        A = scaled_angles(p, 840 + j, cc, S) if kind else uniform_angles(p, 840 + j, S)
        jobs.append({"cost": cost, "mixer": mixer, "angles": torch.from_numpy(A).cuda(),
                     "E": torch.zeros(S, dtype=torch.float64, device="cuda"),
                     "grad": torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")})
    s = torch.cuda.Stream()
    qctx = qg.Context(0, s)
    try:
        with torch.cuda.stream(s):
            qctx.expectation_batched(jobs, want_grad=True)
            s.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                qctx.expectation_batched(jobs, want_grad=True)
            new = []
            for j, (n, cost, cc, mixer, kind) in enumerate(specs):
                A = scaled_angles(p, 850 + j, cc, S) if kind else uniform_angles(p, 850 + j, S)
                jobs[j]["angles"].copy_(torch.from_numpy(A))
                new.append(A)
            graph.replay()
        s.synchronize()
        for (n, cost, cc, mixer, kind), jb, A in zip(specs, jobs, new):
            for i in range(S):
                E_ref, g_ref = (oracle_mod.qaoa_gradient(n, cc, A[i], kind) if kind
                                else oracle_mod.qaoa_gradient(n, cc, A[i]))
                check(jb["E"][i].item(), jb["grad"][i].cpu().numpy(), E_ref, g_ref, cc)
    finally:
        qctx.close()


@pytest.mark.parametrize("n,k,p,mode", [(15, 7, 3, "none"), (15, 7, 1, "round"), (15, 7, 1, "none"),
                                        (13, 6, 4, "none")])
def test_uncompute_and_single_round(Q, oracle_mod, n, k, p, mode):
    """Odd Dicke dimensions (C(15, 7) = 6435, C(13, 6) = 1716: a lone last
    amplitude in the last tile) with a warm start, without checkpoints (the
    adjoint undoes each round on the state in place) and at p = 1 (the
    adjoint writes no lambda)."""
    qg, ctx = Q
    cost, c = dicke_problem(ctx, oracle_mod, n, k, 860 + n + p)
    mixer = qg.GroverMixer.dicke(n, k)
    rng = np.random.default_rng(861 + p)
    psi0 = rng.standard_normal(mixer.dim) + 1j * rng.standard_normal(mixer.dim)
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex64)
    init = torch.view_as_real(torch.from_numpy(psi0).cuda()).contiguous()
    for ang in angle_sets(p, 862 + n, c):
        E, g = ctx.gradient(cost, mixer, ang, init=init, ckpt=mode)
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang, "grover", psi0=psi0.astype(np.complex128))
        check(E, g, E_ref, g_ref, c)


def test_tiny_set_without_checkpoints(Q, oracle_mod):
    """Five feasible states (less than one tile, an odd count) without
    checkpoints, float32 costs, several rounds."""
    qg, ctx = Q
    c = np.array([3.0, -1.0, 4.0, 1.5, -2.5])
    cost = torch.tensor(c, dtype=torch.float32, device="cuda")
    mixer = qg.GroverMixer(5, 3)
    for ang in angle_sets(4, 870, c):
        E, g = ctx.gradient(cost, mixer, ang, ckpt="none")
        E_ref, g_ref = oracle_mod.qaoa_gradient(3, c, ang, "grover")
        check(E, g, E_ref, g_ref, c)

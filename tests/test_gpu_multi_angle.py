"""Multi-angle QAOA (Sec. 3: one mixer per qubit and layer, each with its own
angle) against the oracle: the whole state on chip (n <= 12) and the pass
kernels (contiguous and gathered passes), every checkpoint mode, float32 and
uint8 costs, batched next to standard X-mixer jobs, and through autograd.
"""

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, sk_couplings, uniform_angles

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
    sig = sigma(c)
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sig), (E, E_ref)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


def problem(ctx, oracle_mod, kind, n, seed):
    if kind == "maxcut_u8":
        e = erdos_renyi(n, 0.4, seed)
        return ctx.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8), oracle_mod.cost_maxcut(n, e)
    J = sk_couplings(n, seed)
    return ctx.cost_precompute("sk", n, J=J, dtype=torch.float32), oracle_mod.cost_sk(n, J.astype(np.float64))


@pytest.mark.parametrize("kind", ["maxcut_u8", "sk_f32"])
@pytest.mark.parametrize("n,p", [(8, 3), (14, 2), (20, 2)])
@pytest.mark.parametrize("ckpt", ["none", "round", "pass"])
def test_multi_angle_gradient(Q, oracle_mod, kind, n, p, ckpt):
    qg, ctx = Q
    cost, c = problem(ctx, oracle_mod, kind, n, 200 + n)
    a = np.random.default_rng(300 + n).random(p * (n + 1)) * np.pi
    E, g = ctx.gradient(cost, qg.XMixer(n, multi_angle=True), a, ckpt=ckpt)
    E_ref, g_ref = oracle_mod.qaoa_gradient_ma(n, c, a)
    check(E, g, E_ref, g_ref, c)
    assert ctx.expectation(cost, qg.XMixer(n, multi_angle=True), a) == pytest.approx(E, abs=1e-9 * max(1, abs(E)))


def test_equal_angles_match_standard_path(Q, oracle_mod):
    qg, ctx = Q
    n, p = 17, 3
    cost, c = problem(ctx, oracle_mod, "sk_f32", n, 7)
    ang = uniform_angles(p, 8)[0]
    a = np.concatenate([np.repeat(ang[:p], n), ang[p:]])
    E, g = ctx.gradient(cost, qg.XMixer(n, multi_angle=True), a)
    E0, g0 = ctx.gradient(cost, qg.XMixer(n), ang)
    assert abs(E - E0) <= 1e-5 * max(abs(E0), sigma(c))
    np.testing.assert_allclose(g[:p * n].reshape(p, n).sum(axis=1), g0[:p], rtol=0,
                               atol=1e-4 * np.abs(g0).max())


def test_batched_next_to_standard_jobs(Q, oracle_mod):
    qg, ctx = Q
    n, p, S = 16, 2, 5
    cost, c = problem(ctx, oracle_mod, "maxcut_u8", n, 9)
    A_ma = np.random.default_rng(10).random((S, p * (n + 1))) * np.pi
    A_x = uniform_angles(p, 11, S)
    jobs = []
    for mx, A in ((qg.XMixer(n, multi_angle=True), A_ma), (qg.XMixer(n), A_x)):
        jobs.append({"cost": cost, "mixer": mx, "angles": torch.from_numpy(A).cuda(),
                     "E": torch.zeros(S, dtype=torch.float64, device="cuda"),
                     "grad": torch.zeros(A.shape, dtype=torch.float64, device="cuda")})
    ctx.expectation_batched(jobs, want_grad=True)
    torch.cuda.synchronize()
    for s in (0, S - 1):
        E_ref, g_ref = oracle_mod.qaoa_gradient_ma(n, c, A_ma[s])
        check(jobs[0]["E"][s].item(), jobs[0]["grad"][s].cpu().numpy(), E_ref, g_ref, c)
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A_x[s])
        check(jobs[1]["E"][s].item(), jobs[1]["grad"][s].cpu().numpy(), E_ref, g_ref, c)


def test_autograd(Q, oracle_mod):
    qg, ctx = Q
    n, p = 13, 2
    cost, c = problem(ctx, oracle_mod, "sk_f32", n, 12)
    a = torch.tensor(np.random.default_rng(13).random(p * (n + 1)) * np.pi, dtype=torch.float64,
                     requires_grad=True)
    E = qg.QAOAExpectation.apply(a, ctx, cost, qg.XMixer(n, multi_angle=True))
    (2.0 * E).backward()
    E_ref, g_ref = oracle_mod.qaoa_gradient_ma(n, c, a.detach().numpy())
    check(E.item(), a.grad.numpy() / 2.0, E_ref, g_ref, c)


def test_bad_angle_count(Q):
    qg, ctx = Q
    with pytest.raises(ValueError):
        qg.XMixer(10, multi_angle=True).rounds(21)

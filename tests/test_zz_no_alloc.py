"""qaoa_gradient_small_noalloc: the entry point for callers that cannot
allocate device memory (it keeps its scratch in a fixed device array inside
the library).  Checked through the C ABI against the CPU oracle's complex128
result and against the context-based qaoa_gradient / qaoa_expectation, on two
calls in a row, so that whatever the first call leaves in the shared array
cannot leak into the second.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""

import numpy as np
import pytest
import torch

import oracle
from qaoa_inputs import erdos_renyi, sk_couplings, uniform_angles

pytestmark = pytest.mark.gpu


def _close(E, E_ref, g, g_ref, cost):
    sig = float(np.sqrt(np.mean(np.asarray(cost, dtype=np.float64) ** 2)))
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sig), (E, E_ref)
    if g_ref is not None:
        tol = 1e-4 * np.abs(g_ref).max()
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=tol)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2312_06451_gb300 as qg

    ctx = qg.Context(0)
    yield qg, ctx
    ctx.close()


@pytest.mark.parametrize("kind,n", [("maxcut_u8", 12), ("sk_f32", 7)])
def test_noalloc_matches_context_path_twice(setup, kind, n):
    qg, ctx = setup
    if kind == "maxcut_u8":
        cost = ctx.cost_precompute("maxcut", n, edges=erdos_renyi(n, 0.5, 3), dtype=torch.uint8)
    else:
        cost = ctx.cost_precompute("sk", n, J=sk_couplings(n, 4), dtype=torch.float32)
    host_cost = cost.cpu().numpy()
    # call 1: gradient, p = 5; call 2: expectation only, p = 3, new angles
    for call, (p, seed, want_grad) in enumerate([(5, 11, True), (3, 12, False)]):
        ang = uniform_angles(p, seed)[0]
        d_ang = torch.from_numpy(ang).cuda()
        E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        G = torch.full((2 * p,), float("nan"), dtype=torch.float64, device="cuda") if want_grad else None
        qg.qaoa_gradient_small_noalloc(cost, n, d_ang, E, G)
        c64 = host_cost.astype(np.float64)
        if want_grad:
            E_or, g_or = oracle.qaoa_gradient(n, c64, ang)
            _close(E.item(), E_or, G.cpu().numpy(), g_or, host_cost)
            E_ref, g_ref = ctx.gradient(cost, qg.XMixer(n), ang)
            _close(E.item(), E_ref, G.cpu().numpy(), g_ref, host_cost)
        else:
            _close(E.item(), oracle.qaoa_expectation(n, c64, ang), None, None, host_cost)
            E_ref = ctx.expectation(cost, qg.XMixer(n), ang)
            _close(E.item(), E_ref, None, None, host_cost)


def test_noalloc_repeated_calls_are_identical(setup):
    qg, ctx = setup
    n, p = 10, 96
    cost = ctx.cost_precompute("maxcut", n, edges=erdos_renyi(n, 0.6, 5), dtype=torch.uint8)
    d_ang = torch.from_numpy(uniform_angles(p, 3)[0]).cuda()
    out = []
    for _ in range(2):
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        G = torch.zeros(2 * p, dtype=torch.float64, device="cuda")
        qg.qaoa_gradient_small_noalloc(cost, n, d_ang, E, G)
        out.append((E.clone(), G.clone()))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    E_or, g_or = oracle.qaoa_gradient(n, cost.cpu().numpy().astype(np.float64), d_ang.cpu().numpy())
    _close(out[1][0].item(), E_or, out[1][1].cpu().numpy(), g_or, cost.cpu().numpy())
    E_ref, g_ref = ctx.gradient(cost, qg.XMixer(n), d_ang.cpu().numpy())
    _close(out[1][0].item(), E_ref, out[1][1].cpu().numpy(), g_ref, cost.cpu().numpy())


def test_noalloc_rejects_sizes_beyond_its_limit(setup):
    qg, ctx = setup
    from paper_2312_06451_gb300 import QAOAError

    cost = ctx.cost_precompute("maxcut", 13, edges=erdos_renyi(13, 0.5, 1), dtype=torch.uint8)
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(QAOAError):  # n = 13 > 12
        qg.qaoa_gradient_small_noalloc(cost, 13, torch.zeros(4, dtype=torch.float64, device="cuda"), E)
    small = ctx.cost_precompute("maxcut", 6, edges=erdos_renyi(6, 0.5, 1), dtype=torch.uint8)
    with pytest.raises(QAOAError):  # p = 97 > 96
        qg.qaoa_gradient_small_noalloc(small, 6, torch.zeros(194, dtype=torch.float64, device="cuda"), E)

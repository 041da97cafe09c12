"""qaoa_expectation_batched_host: the batched evaluation with angles and
results in host memory (the angle-finding loop of Sec. 2.3).  Its numbers
must be the device-buffer batched call's, bit for bit (same plan, same
kernels), and the oracle's within the usual tolerances:
|dE| <= 1e-5 max(|E|, sigma_C), |dg_i| <= 1e-4 max|g|.
"""

import ctypes

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, sk_couplings, uniform_angles, uniform_angles_ma

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


def instances(qg, ctx, oracle_mod):
    """(device cost, mixer, host angles, oracle cost, n, multi-angle) of three
    uneven jobs: n = 10 uint8 MaxCut, n = 14 float32 SK, n = 9 multi-angle."""
    out = []
    e = erdos_renyi(10, 0.4, 41)
    out.append((ctx.cost_precompute("maxcut", 10, edges=e, dtype=torch.uint8), qg.XMixer(10),
                uniform_angles(3, 42, 5), oracle_mod.cost_maxcut(10, e), 10, False))
    J = sk_couplings(14, 43)
    out.append((ctx.cost_precompute("sk", 14, J=J, dtype=torch.float32), qg.XMixer(14),
                uniform_angles(4, 44, 3), oracle_mod.cost_sk(14, J.astype(np.float64)), 14, False))
    e9 = erdos_renyi(9, 0.5, 45)
    out.append((ctx.cost_precompute("maxcut", 9, edges=e9, dtype=torch.uint8), qg.XMixer(9, multi_angle=True),
                uniform_angles_ma(2, 9, 46, 4), oracle_mod.cost_maxcut(9, e9), 9, True))
    return out


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("want_grad", [True, False])
def test_host_batched_matches_device_call_and_oracle(Q, oracle_mod, pinned, want_grad):
    qg, ctx = Q
    inst = instances(qg, ctx, oracle_mod)
    host, dev = [], []
    for cost, mx, A, _, _, _ in inst:
        S, na = A.shape

        def h(t):
            return t.pin_memory() if pinned else t

        host.append({"cost": cost, "mixer": mx, "angles": h(torch.from_numpy(A.copy())),
                     "E": h(torch.zeros(S, dtype=torch.float64)),
                     "grad": h(torch.zeros(S, na, dtype=torch.float64)) if want_grad else None})
        dev.append({"cost": cost, "mixer": mx, "angles": torch.from_numpy(A).cuda(),
                    "E": torch.zeros(S, dtype=torch.float64, device="cuda"),
                    "grad": torch.zeros(S, na, dtype=torch.float64, device="cuda") if want_grad else None})
    ctx.expectation_batched_host(host, want_grad=want_grad)
    ctx.expectation_batched(dev, want_grad=want_grad)
    torch.cuda.synchronize()
    for hj, dj, (_, _, A, c, n, ma) in zip(host, dev, inst):
        assert torch.equal(hj["E"], dj["E"].cpu())
        if want_grad:
            assert torch.equal(hj["grad"], dj["grad"].cpu())
        for s in (0, A.shape[0] - 1):
            if ma:
                E_ref, g_ref = oracle_mod.qaoa_gradient_ma(n, c, A[s])
            else:
                E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A[s])
            assert abs(hj["E"][s].item() - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c))
            if want_grad:
                np.testing.assert_allclose(hj["grad"][s].numpy(), g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


def test_host_batched_call_reuse_with_new_angles(Q, oracle_mod):
    """A prepared call re-run after the angles were overwritten in place gives
    the new angles' results (the loop of an optimiser)."""
    qg, ctx = Q
    n, p, S = 12, 3, 4
    e = erdos_renyi(n, 0.5, 51)
    cost = ctx.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
    c = oracle_mod.cost_maxcut(n, e)
    A = torch.from_numpy(uniform_angles(p, 52, S)).pin_memory()
    E = torch.zeros(S, dtype=torch.float64).pin_memory()
    G = torch.zeros(S, 2 * p, dtype=torch.float64).pin_memory()
    call = ctx.batched_call_host([{"cost": cost, "mixer": qg.XMixer(n), "angles": A, "E": E, "grad": G}],
                                 want_grad=True)
    for it in range(3):
        A.copy_(torch.from_numpy(uniform_angles(p, 60 + it, S)))
        call.run()
        for s in (0, S - 1):
            E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A[s].numpy())
            assert abs(E[s].item() - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c))
            np.testing.assert_allclose(G[s].numpy(), g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


def test_host_batched_errors_leave_the_context_usable(Q, oracle_mod):
    """NULL host pointers and a non-finite angle are refused with
    QAOA_ERR_INVALID; the next call on the same context still works."""
    qg, ctx = Q
    from paper_2312_06451_gb300 import _binding as B

    n, p = 10, 2
    e = erdos_renyi(n, 0.5, 71)
    cost = ctx.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
    mx = qg.XMixer(n)
    A = np.ascontiguousarray(uniform_angles(p, 72, 2))
    E = np.zeros(2)
    arr = (B.QaoaHostJob * 1)()
    arr[0] = B.QaoaHostJob(cost.data_ptr(), B.QAOA_COST_U8, ctypes.pointer(mx.struct), p, 2,
                           A.ctypes.data, None, None, None)
    assert ctx._lib.qaoa_expectation_batched_host(ctx._h, 1, arr, 0) == B.QAOA_ERR_INVALID
    arr[0] = B.QaoaHostJob(cost.data_ptr(), B.QAOA_COST_U8, ctypes.pointer(mx.struct), p, 2,
                           A.ctypes.data, E.ctypes.data, None, None)
    assert ctx._lib.qaoa_expectation_batched_host(ctx._h, 1, arr, 1) == B.QAOA_ERR_INVALID  # no grad buffer
    bad = A.copy()
    bad[1, 0] = np.nan
    with pytest.raises(qg.QAOAError) as ei:
        ctx.expectation_batched_host([{"cost": cost, "mixer": mx, "angles": bad, "E": E}])
    assert ei.value.status == B.QAOA_ERR_INVALID
    ctx.expectation_batched_host([{"cost": cost, "mixer": mx, "angles": A, "E": E}])
    c = oracle_mod.cost_maxcut(n, e)
    for s in range(2):
        E_ref = oracle_mod.qaoa_expectation(n, c, A[s])
        assert abs(E[s] - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c))


def test_host_batched_other_mixers(Q, oracle_mod):
    """A Grover job (rank-one passes, float32 SK cost) and a block-diagonal
    ring XY job (tensor-core products, DkS cost on the weight-4 states) in one
    host-buffer call: the device-buffer call's numbers bit for bit, and the
    oracle's."""
    qg, ctx = Q
    n1, p1 = 16, 3
    J = sk_couplings(n1, 81)
    cost1 = ctx.cost_precompute("sk", n1, J=J, dtype=torch.float32)
    c1 = oracle_mod.cost_sk(n1, J.astype(np.float64))
    A1 = uniform_angles(p1, 82, 3)
    n2, k2, p2 = 10, 4, 2
    e2 = erdos_renyi(n2, 0.5, 83)
    st2 = oracle_mod.dicke_states(n2, k2)
    c2 = oracle_mod.cost_dks(n2, e2, st2)
    cost2 = ctx.cost_precompute("dks", n2, edges=e2, k=k2, dtype=torch.uint8)
    A2 = uniform_angles(p2, 84, 4)
    specs = [(cost1, qg.GroverMixer.full(n1), A1), (cost2, qg.xy_sym_mixer(ctx, "ring", n2, k2), A2)]
    host = [{"cost": c, "mixer": m, "angles": torch.from_numpy(A.copy()).pin_memory(),
             "E": torch.zeros(A.shape[0], dtype=torch.float64).pin_memory(),
             "grad": torch.zeros(A.shape, dtype=torch.float64).pin_memory()} for c, m, A in specs]
    dev = [{"cost": c, "mixer": m, "angles": torch.from_numpy(A).cuda(),
            "E": torch.zeros(A.shape[0], dtype=torch.float64, device="cuda"),
            "grad": torch.zeros(A.shape, dtype=torch.float64, device="cuda")} for c, m, A in specs]
    ctx.expectation_batched_host(host, want_grad=True)
    ctx.expectation_batched(dev, want_grad=True)
    torch.cuda.synchronize()
    for hj, dj in zip(host, dev):
        assert torch.equal(hj["E"], dj["E"].cpu()) and torch.equal(hj["grad"], dj["grad"].cpu())
    for s in range(A1.shape[0]):
        E_ref, g_ref = oracle_mod.qaoa_gradient(n1, c1, A1[s], "grover")
        assert abs(host[0]["E"][s].item() - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c1))
        np.testing.assert_allclose(host[0]["grad"][s].numpy(), g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())
    for s in range(A2.shape[0]):
        E_ref, g_ref = oracle_mod.qaoa_gradient(n2, c2, A2[s], "ring", st2)
        assert abs(host[1]["E"][s].item() - E_ref) <= 1e-5 * max(abs(E_ref), sigma(c2))
        np.testing.assert_allclose(host[1]["grad"][s].numpy(), g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())

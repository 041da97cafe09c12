"""Failure path and graph capture.

* Every device-side wait of the kernels is bounded.  A wait on a barrier that
  nothing completes must give up, surface as QAOA_ERR_TIMEOUT and leave the
  context usable: no fault, no trap, no hang.
* The batched entry point can be captured in a CUDA graph after one warm-up
  call has sized the scratch; replaying the graph with new angles in the same
  buffers gives the oracle's results for the new angles.
"""

import time

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, sk_couplings, uniform_angles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2312_06451_gb300

    return paper_2312_06451_gb300


def sigma(c):
    return float(np.sqrt(np.mean(np.asarray(c, dtype=np.float64) ** 2)))


def check(E, g, E_ref, g_ref, c):
    sig = sigma(c)
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sig), (E, E_ref)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


def test_bounded_wait_gives_up_and_context_stays_usable(qg, oracle_mod):
    from paper_2312_06451_gb300 import _binding as B

    ctx = qg.Context(0)
    try:
        t = time.time()
        with pytest.raises(qg.QAOAError) as ei:
            ctx.check_bounded_wait()
        assert ei.value.status == B.QAOA_ERR_TIMEOUT
        assert time.time() - t < 10  # the wait limit is one second of GPU time
        # the same context still computes correctly
        n, p = 15, 2
        e = erdos_renyi(n, 0.5, 71)
        cost = ctx.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
        c = oracle_mod.cost_maxcut(n, e)
        ang = uniform_angles(p, 72)[0]
        E, g = ctx.gradient(cost, qg.XMixer(n), ang)
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang)
        check(E, g, E_ref, g_ref, c)
    finally:
        ctx.close()


def test_cuda_graph_replay_of_batched_call(qg, oracle_mod):
    stream = torch.cuda.Stream()
    ctx = qg.Context(0, stream)
    try:
        with torch.cuda.stream(stream):
            n1, n2, p, S = 17, 10, 2, 3
            J = sk_couplings(n1, 73)
            cost1 = ctx.cost_precompute("sk", n1, J=J, dtype=torch.float32)
            e2 = erdos_renyi(n2, 0.5, 74)
            cost2 = ctx.cost_precompute("maxcut", n2, edges=e2, dtype=torch.uint8)
            jobs = []
            for cost, n in ((cost1, n1), (cost2, n2)):
                jobs.append({"cost": cost, "mixer": qg.XMixer(n),
                             "angles": torch.from_numpy(uniform_angles(p, 75, S)).cuda(),
                             "E": torch.zeros(S, dtype=torch.float64, device="cuda"),
                             "grad": torch.zeros(S, 2 * p, dtype=torch.float64, device="cuda")})
            ctx.expectation_batched(jobs, want_grad=True)  # sizes scratch, builds the plan
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ctx.expectation_batched(jobs, want_grad=True)
        A_new = uniform_angles(p, 76, S)
        for j in jobs:
            j["angles"].copy_(torch.from_numpy(A_new))
            j["E"].zero_()
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        refs = [(n1, oracle_mod.cost_sk(n1, J.astype(np.float64))), (n2, oracle_mod.cost_maxcut(n2, e2))]
        for j, (n, c) in zip(jobs, refs):
            for s in range(S):
                E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, A_new[s])
                check(j["E"][s].item(), j["grad"][s].cpu().numpy(), E_ref, g_ref, c)
    finally:
        ctx.close()


def test_state_limit_refuses_before_launch_and_context_recovers(qg, oracle_mod):
    """A cap on state scratch below what one angle set needs (even without
    checkpoints) makes the planner refuse with QAOA_ERR_OOM before anything is
    launched; lifting the cap, the same context computes the oracle's result."""
    from paper_2312_06451_gb300 import _binding as B

    n, p = 20, 3
    e = erdos_renyi(n, 0.3, 81)
    ang = uniform_angles(p, 82, 2)
    ctx = qg.Context(0)
    try:
        cost = ctx.cost_precompute("maxcut", n, edges=e, dtype=torch.uint8)
        job = {"cost": cost, "mixer": qg.XMixer(n), "angles": torch.from_numpy(ang).cuda(),
               "E": torch.full((2,), float("nan"), dtype=torch.float64, device="cuda"),
               "grad": torch.full((2, 2 * p), float("nan"), dtype=torch.float64, device="cuda")}
        ctx.set_state_limit((2 << n) * 8 - 1)  # one byte short of W and lambda
        launches = ctx.launch_count()
        with pytest.raises(qg.QAOAError) as ei:
            ctx.expectation_batched([job], want_grad=True)
        assert ei.value.status == B.QAOA_ERR_OOM
        assert ctx.launch_count() == launches
        torch.cuda.synchronize()
        assert torch.isnan(job["E"]).all()
        # a cap that admits one set at a time without checkpoints still works
        ctx.set_state_limit((2 << n) * 8)
        ctx.expectation_batched([job], want_grad=True)
        torch.cuda.synchronize()
        c = oracle_mod.cost_maxcut(n, e)
        for s in range(2):
            E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang[s])
            check(job["E"][s].item(), job["grad"][s].cpu().numpy(), E_ref, g_ref, c)
        ctx.set_state_limit(None)
        ctx.expectation_batched([job], want_grad=True)
        torch.cuda.synchronize()
        E_ref, g_ref = oracle_mod.qaoa_gradient(n, c, ang[1])
        check(job["E"][1].item(), job["grad"][1].cpu().numpy(), E_ref, g_ref, c)
    finally:
        ctx.close()

"""Every X-mixer pass schedule, adjoint buffer choice and checkpoint mode
gives the oracle's <C> and gradient (the schedule only regroups commuting
rotations, Sec. 2.2), and the autotuner leaves a working schedule behind.
"""

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, uniform_angles

pytestmark = pytest.mark.gpu

N = 20  # 8 qubits above the contiguous tile: one, two or three gathered passes


@pytest.fixture(scope="module")
def setup(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2312_06451_gb300 as qg

    ctx = qg.Context(0)
    edges = erdos_renyi(N, 0.3, 77)
    cost = ctx.cost_precompute("maxcut", N, edges=edges, dtype=torch.uint8)
    c = oracle_mod.cost_maxcut(N, edges)
    ang = uniform_angles(3, 78)[0]
    E_ref, g_ref = oracle_mod.qaoa_gradient(N, c, ang)
    sig = float(np.sqrt(np.mean(c ** 2)))
    yield qg, ctx, cost, ang, E_ref, g_ref, sig
    ctx.close()


def _check(E, g, E_ref, g_ref, sig):
    assert abs(E - E_ref) <= 1e-5 * max(abs(E_ref), sig), (E, E_ref)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())


SCHEDULES = sorted({tuple(s) for s in [(cm, sp) for cm in range(4, 9) for sp in range(3)]})


@pytest.mark.parametrize("cmin,split", SCHEDULES)
@pytest.mark.parametrize("ckpt", ["none", "round", "pass"])
def test_every_schedule_and_checkpoint_mode(setup, cmin, split, ckpt):
    qg, ctx, cost, ang, E_ref, g_ref, sig = setup
    ctx.set_tuning({"n": N, "cost_dtype": 1, "cmin": cmin, "split": split, "nbuf_bwd_contig": 1,
                    "nbuf_bwd_gather": 1})
    E, g = ctx.gradient(cost, qg.XMixer(N), ang, ckpt=ckpt)
    _check(E, g, E_ref, g_ref, sig)


@pytest.mark.parametrize("bc,bg", [(1, 2), (2, 1), (2, 2)])
def test_adjoint_buffer_choices(setup, bc, bg):
    qg, ctx, cost, ang, E_ref, g_ref, sig = setup
    ctx.set_tuning({"n": N, "cost_dtype": 1, "cmin": 5, "split": 0, "nbuf_bwd_contig": bc, "nbuf_bwd_gather": bg})
    for ckpt in ("round", "pass"):
        E, g = ctx.gradient(cost, qg.XMixer(N), ang, ckpt=ckpt)
        _check(E, g, E_ref, g_ref, sig)


def test_autotune_then_batched_gradient(setup):
    qg, ctx, cost, ang, E_ref, g_ref, sig = setup
    t = ctx.autotune(cost, N, p=2, want_grad=True)
    assert t["n"] == N and t["cost_dtype"] == 1 and 4 <= t["cmin"] <= 8 and t["ms"] > 0
    assert ctx.get_tuning(N, 1) == t
    A = torch.from_numpy(np.stack([ang, ang])).cuda()
    E = torch.zeros(2, dtype=torch.float64, device="cuda")
    G = torch.zeros(2, 6, dtype=torch.float64, device="cuda")
    ctx.set_checkpointing("pass")
    ctx.expectation_batched([{"cost": cost, "mixer": qg.XMixer(N), "angles": A, "E": E, "grad": G}],
                            want_grad=True)
    torch.cuda.synchronize()
    for s in range(2):
        _check(E[s].item(), G[s].cpu().numpy(), E_ref, g_ref, sig)


def test_tuning_saved_and_restored(setup, tmp_path):
    """A tuned schedule written to a file (the autotuner's cache) and loaded
    into a fresh context is the schedule the fresh context uses."""
    qg, ctx, cost, *_ = setup
    t = ctx.autotune(cost, N, p=2, want_grad=True)
    path = str(tmp_path / "xtune.json")
    ctx.save_tuning(path)
    with qg.Context(0) as fresh:
        assert fresh.load_tuning(path) >= 1
        got = fresh.get_tuning(N, 1)
        assert {k: got[k] for k in ("cmin", "split", "nbuf_bwd_contig", "nbuf_bwd_gather")} == \
            {k: t[k] for k in ("cmin", "split", "nbuf_bwd_contig", "nbuf_bwd_gather")}


def test_bad_tuning_and_mode_are_rejected(setup):
    qg, ctx, *_ = setup
    with pytest.raises(qg.QAOAError):
        ctx.set_tuning({"n": N, "cost_dtype": 1, "cmin": 3, "split": 0, "nbuf_bwd_contig": 1, "nbuf_bwd_gather": 1})
    with pytest.raises(qg.QAOAError):
        ctx.set_checkpointing(3)

"""Round-boundary fusion of the X-mixer passes in every mode, each in a process
of its own (the mode is read once per process from QAOA_FUSE): none, all
boundaries, only those on the contiguous group, only those on a gathered
group.  With partial fusion, rounds that follow an unfused boundary start on
a gathered group, so the phase separator, the gamma partial and the phase undo
run in gathered passes.  Every mode must give the oracle's <C> and gradient.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from qaoa_inputs import erdos_renyi, sk_couplings, uniform_angles

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
import paper_2312_06451_gb300 as qg
from qaoa_inputs import erdos_renyi, sk_couplings, uniform_angles
out = []
with qg.Context(0) as ctx:
    for n, p, f32 in ((20, 3, False), (20, 4, True), (25, 5, True)):
        if f32:
            cost = ctx.cost_precompute("sk", n, J=sk_couplings(n, 900 + n), dtype=torch.float32)
        else:
            cost = ctx.cost_precompute("maxcut", n, edges=erdos_renyi(n, 0.4, 900 + n), dtype=torch.uint8)
        a = uniform_angles(p, 910 + n + p)[0]
        A = torch.from_numpy(np.stack([a, a])).cuda()
        E = torch.zeros(2, dtype=torch.float64, device="cuda")
        G = torch.zeros(2, 2 * p, dtype=torch.float64, device="cuda")
        ctx.expectation_batched([{"cost": cost, "mixer": qg.XMixer(n), "angles": A, "E": E, "grad": G}],
                                want_grad=True)
        torch.cuda.synchronize()
        Ef = ctx.expectation(cost, qg.XMixer(n), a)
        out.append({"n": n, "p": p, "f32": f32, "E": E[1].item(), "g": G[1].cpu().tolist(), "Ef": Ef})
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def oracle_refs(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    refs = {}
    for n, p, f32 in ((20, 3, False), (20, 4, True), (25, 5, True)):
        if f32:
            c = oracle_mod.cost_sk(n, sk_couplings(n, 900 + n).astype(np.float64))
        else:
            c = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.4, 900 + n))
        a = uniform_angles(p, 910 + n + p)[0]
        E, g = oracle_mod.qaoa_gradient(n, c, a)
        refs[(n, p)] = (E, g, float(np.sqrt(np.mean(c ** 2))))
    return refs


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_fusion_mode_matches_oracle(oracle_refs, mode):
    env = dict(os.environ, QAOA_FUSE=str(mode), PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    for rec in json.loads(r.stdout.strip().splitlines()[-1]):
        E_ref, g_ref, sig = oracle_refs[(rec["n"], rec["p"])]
        assert abs(rec["E"] - E_ref) <= 1e-5 * max(abs(E_ref), sig), (mode, rec["n"], rec["E"], E_ref)
        assert abs(rec["Ef"] - E_ref) <= 1e-5 * max(abs(E_ref), sig), (mode, rec["n"], rec["Ef"], E_ref)
        np.testing.assert_allclose(rec["g"], g_ref, rtol=0, atol=1e-4 * np.abs(g_ref).max())

"""Host-side argument checks of the Python binding (no GPU needed): every
malformed call is refused before anything reaches the device, where a short
or mistyped buffer would become an out-of-bounds access."""

import pytest
import torch

import paper_2312_06451_gb300 as qg
from paper_2312_06451_gb300 import _check_noalloc_args


def _good(n=6, p=3):
    return (torch.zeros(1 << n, dtype=torch.uint8), n, torch.zeros(2 * p, dtype=torch.float64),
            torch.zeros(1, dtype=torch.float64), torch.zeros(2 * p, dtype=torch.float64))


@pytest.mark.parametrize("bad,msg", [
    (lambda a: (a[0].float().double(), *a[1:]), "uint8 or float32"),
    (lambda a: (a[0], a[1], a[2].float(), *a[3:]), "angles must be float64"),
    (lambda a: (*a[:3], a[3].float(), a[4]), "E must be float64"),
    (lambda a: (*a[:4], a[4].float()), "grad must be float64"),
    (lambda a: (a[0][:-1], *a[1:]), r"2\^n"),
    (lambda a: (a[0], 7, *a[2:]), r"2\^n"),
    (lambda a: (a[0], a[1], a[2][:-1], a[3], a[4][:-1]), "2p values"),
    (lambda a: (a[0], a[1], a[2][:0], a[3], None), "2p values"),
    (lambda a: (*a[:3], a[3][:0], a[4]), "at least one"),
    (lambda a: (*a[:4], a[4][:-2]), "grad must hold"),
    (lambda a: (a[0], a[1], [0.0] * 6, *a[3:]), "torch tensor"),
])
def test_noalloc_rejects_malformed_arguments(bad, msg):
    with pytest.raises(ValueError, match=msg):
        _check_noalloc_args(*bad(_good()))


def test_noalloc_rejects_host_tensors_before_any_call():
    # well-formed shapes and dtypes, but host memory: refused on the host
    with pytest.raises(ValueError, match="CUDA tensor"):
        qg.qaoa_gradient_small_noalloc(*_good())


@pytest.mark.parametrize("n,coeffs", [(1, {1: 1.0}), (8, {1: 1.0, 2: 1.0}), (21, {1: 1.0, 2: 1.0}),
                                      (13, {0: 0.5, 1: -1.0, 3: 2.5}), (34, {2: 1.0, 17: 1e-3})])
def test_x_mixer_weights_match_the_oracle(oracle_mod, n, coeffs):
    """qaoa_x_mixer_weights (host-only library call) against the oracle's
    Krawtchouk sums, which the oracle pins check against dense Pauli
    products."""
    import numpy as np

    d = qg.krawtchouk_weights(n, coeffs)
    ref = oracle_mod.krawtchouk_weights(n, coeffs)
    np.testing.assert_allclose(d, ref, rtol=1e-13, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_x_mixer_weights_grover_sum_is_exact():
    """Sum over every order k of K_k(w) is 2^n [w = 0]: with all c_k = 2^-n
    the weights are exactly the Grover mixer's [1, 0, ..., 0]."""
    import numpy as np

    n = 30
    d = qg.krawtchouk_weights(n, {k: 2.0 ** -n for k in range(n + 1)})
    np.testing.assert_array_equal(d, [1.0] + [0.0] * n)


def test_x_mixer_weights_rejects_bad_sizes():
    import ctypes

    import numpy as np

    from paper_2312_06451_gb300 import _binding as B

    c = np.ones(3)
    d = np.zeros(3)
    lib = B.load()
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    assert lib.qaoa_x_mixer_weights(0, 1, P(c), P(d)) == B.QAOA_ERR_INVALID
    assert lib.qaoa_x_mixer_weights(2, 3, P(c), P(d)) == B.QAOA_ERR_INVALID
    assert lib.qaoa_x_mixer_weights(2, 1, None, P(d)) == B.QAOA_ERR_INVALID


def test_grover_mixer_struct():
    """GroverMixer: dimensions of the full space and the weight-k subspace,
    the mixer kind the library sees, and no empty feasible set."""
    import math

    import pytest

    import paper_2312_06451_gb300 as qg
    from paper_2312_06451_gb300 import _binding as B

    m = qg.GroverMixer.full(10)
    assert (m.dim, m.n, m.struct.kind, m.struct.dim) == (1024, 10, B.QAOA_MIXER_GROVER, 1024)
    d = qg.GroverMixer.dicke(20, 9)
    assert d.dim == math.comb(20, 9) == d.struct.dim
    assert qg.GroverMixer(3).dim == 3
    with pytest.raises(ValueError):
        qg.GroverMixer(0)


def test_tuning_file_round_trip_and_damage(tmp_path):
    """The pass-schedule tuning file: what is written reads back; a changed
    value, a truncated file, another version or another GPU are refused."""
    import json

    import pytest

    import paper_2312_06451_gb300 as qg

    ents = [{"n": 24, "cost_dtype": 1, "cmin": 5, "split": 1, "nbuf_bwd_contig": 2, "nbuf_bwd_gather": 1,
             "ms": 3.25},
            {"n": 28, "cost_dtype": 0, "cmin": 4, "split": 0, "nbuf_bwd_contig": 1, "nbuf_bwd_gather": 1,
             "ms": 48.0}]
    path = str(tmp_path / "tune.json")
    qg.write_tuning_file(path, ents, "GPU A")
    assert qg.read_tuning_file(path, "GPU A") == ents
    assert qg.read_tuning_file(path) == ents
    with pytest.raises(ValueError, match="tuned on"):
        qg.read_tuning_file(path, "GPU B")
    doc = json.load(open(path))
    doc["entries"][0]["cmin"] = 6  # altered without a new checksum
    json.dump(doc, open(path, "w"))
    with pytest.raises(ValueError, match="checksum"):
        qg.read_tuning_file(path)
    qg.write_tuning_file(path, ents)
    text = open(path).read()
    open(path, "w").write(text[: len(text) // 2])
    with pytest.raises(ValueError, match="unreadable"):
        qg.read_tuning_file(path)
    qg.write_tuning_file(path, ents)
    doc = json.load(open(path))
    doc["version"] = 99
    json.dump(doc, open(path, "w"))
    with pytest.raises(ValueError, match="version"):
        qg.read_tuning_file(path)


def test_host_buffers_of_the_host_batched_call():
    """The host-buffer batched call takes contiguous float64 host tensors or
    arrays (wrapped, not copied) and refuses anything else before marshalling."""
    import numpy as np

    from paper_2312_06451_gb300 import _host_tensor

    a = np.arange(12, dtype=np.float64).reshape(3, 4)
    t = _host_tensor(a, "angles")
    assert t.data_ptr() == a.ctypes.data  # the caller's memory, no copy
    assert _host_tensor(None, "grad") is None
    assert _host_tensor(torch.zeros(5, dtype=torch.float64), "E").numel() == 5
    for bad in (a.astype(np.float32), a[:, ::2], torch.zeros(4, dtype=torch.float32),
                torch.zeros(4, 4, dtype=torch.float64).t(), [0.0, 1.0]):
        with pytest.raises(ValueError):
            _host_tensor(bad, "angles")

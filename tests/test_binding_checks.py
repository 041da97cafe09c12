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

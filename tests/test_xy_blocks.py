"""Cyclic-shift blocks of the XY mixers (host-side library call, no GPU):
the block matrices are symmetric, their sizes add up to C(n, k), and together
they carry exactly the spectrum of the full mixer, which the oracle applies
by its own definition (the oracle pins fix that spectrum to the free-fermion
and total-spin formulas)."""

import numpy as np
import pytest

import paper_2312_06451_gb300 as qg


def dense_from_oracle(oracle_mod, kind, n, k):
    st = oracle_mod.dicke_states(n, k)
    D = len(st)
    return np.stack([oracle_mod.hm_apply(n, np.eye(D)[i].astype(complex), kind, st) for i in range(D)], axis=1).real


@pytest.mark.parametrize("kind", ["ring", "clique"])
@pytest.mark.parametrize("n,k", [(3, 1), (4, 2), (6, 3), (8, 4), (9, 3), (10, 5), (12, 4), (7, 0), (7, 7)])
def test_blocks_carry_the_full_spectrum(oracle_mod, kind, n, k):
    dims, Hs = qg.xy_block_hamiltonians(kind, n, k)
    H = dense_from_oracle(oracle_mod, kind, n, k)
    assert sum(dims) == H.shape[0]
    assert len(dims) <= n // 2 + 1
    for d, Hb in zip(dims, Hs):
        assert Hb.shape == (d, d)
        np.testing.assert_allclose(Hb, Hb.T, rtol=0, atol=1e-13)
    ev = np.sort(np.concatenate([np.linalg.eigvalsh(Hb) for Hb in Hs]))
    np.testing.assert_allclose(ev, np.sort(np.linalg.eigvalsh(H)), rtol=0, atol=1e-11)
    # the traces of H and H^2 are sums over the blocks too
    assert sum(np.trace(Hb) for Hb in Hs) == pytest.approx(np.trace(H), abs=1e-10)
    assert sum(np.sum(Hb * Hb) for Hb in Hs) == pytest.approx(np.sum(H * H), rel=1e-12)


def test_block_sizes_follow_the_orbits():
    """n = 16, k = 8 (12870 states): 9 momentum blocks; momentum 0 holds one
    vector per orbit, the paired momenta two per orbit that allows them."""
    import ctypes

    from paper_2312_06451_gb300 import _binding as B

    lib = B.load()
    nb = ctypes.c_int(0)
    assert lib.qaoa_xy_block_hamiltonians(B.QAOA_XY_RING, 16, 8, ctypes.byref(nb), None, None) == B.QAOA_OK
    d = np.zeros(nb.value, dtype=np.int64)
    assert lib.qaoa_xy_block_hamiltonians(B.QAOA_XY_RING, 16, 8, ctypes.byref(nb),
                                          d.ctypes.data_as(ctypes.c_void_p), None) == B.QAOA_OK
    assert nb.value == 9 and d.sum() == 12870
    # orbits under the 16-cycle: Burnside count of weight-8 necklaces
    from math import comb, gcd

    def phi(m):
        return sum(1 for i in range(1, m + 1) if gcd(i, m) == 1)

    orbits = sum(phi(dd) * comb(16 // dd, 8 // dd) for dd in (1, 2, 4, 8) if 16 % dd == 0) // 16
    assert d[0] == orbits
    # too small a capacity and bad arguments are refused
    nb2 = ctypes.c_int(3)
    assert lib.qaoa_xy_block_hamiltonians(B.QAOA_XY_RING, 16, 8, ctypes.byref(nb2),
                                          d.ctypes.data_as(ctypes.c_void_p), None) == B.QAOA_ERR_INVALID
    assert lib.qaoa_xy_block_hamiltonians(7, 16, 8, ctypes.byref(nb), None, None) == B.QAOA_ERR_INVALID
    assert lib.qaoa_xy_block_hamiltonians(B.QAOA_XY_RING, 33, 2, ctypes.byref(nb), None, None) == B.QAOA_ERR_INVALID

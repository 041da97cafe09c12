"""Host logic of the X-mixer pass schedule (qaoa_pass_schedule; no GPU).

A round's mixer is n commuting single-qubit rotations (Sec. 2.2), so any
grouping of the qubits into passes gives the same state; the schedule must
cover every qubit exactly once, keep each gathered run at least 2^cmin
amplitudes long and use the fewest passes.
"""

import pytest


@pytest.fixture(scope="module")
def sched():
    import paper_2312_06451_gb300 as qg

    return qg.pass_schedule


@pytest.mark.parametrize("n", list(range(13, 33)))
@pytest.mark.parametrize("cmin", [4, 5, 6, 7, 8])
@pytest.mark.parametrize("split", [0, 1, 2])
def test_schedule_covers_every_qubit_once(sched, n, cmin, split):
    T = 12
    g = sched(n, cmin, split)
    assert g[0] == (T, T)  # qubits 0..11, contiguous tiles
    covered = list(range(T))
    nxt = T
    for c, lo in g[1:]:
        assert cmin <= c < T
        assert lo == nxt  # chunks in increasing qubit order
        covered += list(range(lo, lo + T - c))
        nxt = lo + T - c
    assert covered == list(range(n))
    hmax = T - cmin
    assert len(g) == 1 + -(-(n - T) // hmax)  # fewest passes


def test_split_modes(sched):
    # n = 20: 8 high qubits, chunks of at most 12 - 5 = 7
    assert sched(20, 5, 0) == [(12, 12), (8, 12), (8, 16)]   # 4 + 4
    assert sched(20, 5, 1) == [(12, 12), (5, 12), (11, 19)]  # 7 + 1
    assert sched(20, 5, 2) == [(12, 12), (11, 12), (5, 13)]  # 1 + 7
    # n = 28: two gathered passes of 8 qubits from 128-byte runs
    assert sched(28, 4, 0) == [(12, 12), (4, 12), (4, 20)]


@pytest.mark.parametrize("args", [(12, 4, 0), (33, 4, 0), (20, 3, 0), (20, 9, 0), (20, 4, 3)])
def test_schedule_rejects_bad_arguments(sched, args):
    with pytest.raises(ValueError):
        sched(*args)

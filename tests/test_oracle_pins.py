"""Pins of the CPU oracle against facts that do not reuse its arithmetic.

Each test names what fixes the expected value: a dense matrix exponential
built from Pauli matrices, the Hadamard-diagonal identity of Eq. 2, the p=1
MaxCut closed form, sum rules of the cost functions, symmetries of Eq. 1,
the free-fermion spectrum of the ring mixer, or finite differences.  The
paper prints no numerical value for any worked example, so there is no
printed number to pin against.
"""

import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla

from qaoa_inputs import erdos_renyi, random_regular3, sk_couplings

# ----------------------------------------------------------------- helpers

PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
P1 = np.eye(2, dtype=np.complex128)


def pauli_op(n, ops):
    """Dense 2^n x 2^n tensor product; ops maps qubit -> 2x2; qubit i is bit i
    of the basis index (the kron's last factor is qubit 0)."""
    out = np.array([[1.0 + 0j]])
    for q in reversed(range(n)):
        out = np.kron(out, ops.get(q, P1))
    return out


def dense_x_mixer(n):
    return sum(pauli_op(n, {i: PX}) for i in range(n))


def dense_ring_mixer(n):
    H = 0
    for i in range(n):
        j = (i + 1) % n
        H = H + pauli_op(n, {i: PX, j: PX}) + pauli_op(n, {i: PY, j: PY})
    return H


def dense_clique_mixer(n):
    H = 0
    for i in range(n):
        for j in range(i + 1, n):
            H = H + pauli_op(n, {i: PX, j: PX}) + pauli_op(n, {i: PY, j: PY})
    return H


def bits_matrix(n, xs=None):
    xs = np.arange(1 << n, dtype=np.int64) if xs is None else np.asarray(xs, dtype=np.int64)
    return ((xs[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)


def dense_qaoa_state(H_M, cost, angles, psi0):
    p = len(angles) // 2
    v = psi0.astype(np.complex128)
    for k in range(p):
        v = np.exp(-1j * angles[p + k] * cost) * v
        v = sla.expm(-1j * angles[k] * H_M) @ v
    return v


# --------------------------------------------------------- feasible states

@pytest.mark.parametrize("n,k", [(1, 0), (4, 2), (6, 3), (8, 4), (10, 1), (12, 12)])
def test_dicke_states(oracle_mod, n, k):
    s = oracle_mod.dicke_states(n, k)
    assert s.shape[0] == math.comb(n, k)
    assert np.all(np.diff(s.astype(np.int64)) > 0)
    assert all(bin(int(x)).count("1") == k for x in s)
    assert np.all(s < (1 << n))


# ------------------------------------------------------------ cost vectors

@pytest.mark.parametrize("n,seed", [(3, 1), (7, 2), (10, 3), (12, 4)])
def test_maxcut_cost_matrix_form(oracle_mod, n, seed):
    """Cut size = sum over edges of (1 - z_u z_v)/2 with z = 1 - 2x; checked
    as a matrix expression and against the sum rule mean = |E|/2."""
    e = erdos_renyi(n, 0.5, seed)
    c = oracle_mod.cost_maxcut(n, e)
    z = 1 - 2 * bits_matrix(n)
    A = np.zeros((n, n))
    A[e[:, 0], e[:, 1]] = 1
    ref = 0.5 * (A.sum() - np.einsum("xi,ij,xj->x", z, A, z))
    np.testing.assert_array_equal(c, ref)
    assert c.mean() == pytest.approx(len(e) / 2, abs=1e-12)
    # complement symmetry: flipping every bit keeps the cut
    np.testing.assert_array_equal(c, c[::-1])


def test_weighted_maxcut(oracle_mod):
    n = 6
    e = erdos_renyi(n, 0.6, 9)
    w = np.linspace(0.5, 2.0, len(e))
    c = oracle_mod.cost_maxcut(n, e, weights=w)
    assert c.mean() == pytest.approx(w.sum() / 2, abs=1e-12)
    assert c.max() <= w.sum() + 1e-12


@pytest.mark.parametrize("n,seed", [(5, 21), (9, 22), (12, 23)])
def test_weighted_maxcut_laplacian_form(oracle_mod, n, seed):
    """Weighted cut = x^T L x with the weighted graph Laplacian L = D - W
    (each edge adds w_uv (x_u - x_v)^2), and = (1/2) sum_uv w_uv (1 - z_u z_v)
    over edges with z = 1 - 2x.  Distinct random weights make any mix-up of
    weights and edges (a permutation, a transposed pair) change the values;
    a single set bit cuts exactly the edges at that vertex, its weighted
    degree."""
    e = erdos_renyi(n, 0.5, seed)
    w = np.random.default_rng(seed).uniform(0.1, 3.0, len(e))
    c = oracle_mod.cost_maxcut(n, e, weights=w)
    W = np.zeros((n, n))
    np.add.at(W, (e[:, 0], e[:, 1]), w)
    np.add.at(W, (e[:, 1], e[:, 0]), w)
    L = np.diag(W.sum(1)) - W
    x = bits_matrix(n).astype(np.float64)
    np.testing.assert_allclose(c, np.einsum("xi,ij,xj->x", x, L, x), rtol=0, atol=1e-12)
    z = 1 - 2 * x
    zz = z[:, e[:, 0]] * z[:, e[:, 1]]
    np.testing.assert_allclose(c, 0.5 * ((1 - zz) @ w), rtol=0, atol=1e-12)
    for v in range(n):
        assert c[1 << v] == pytest.approx(W[v].sum(), abs=1e-12)
    # a permutation of the weights over the edges gives another cost vector
    perm = np.roll(np.arange(len(e)), 1)
    assert not np.allclose(oracle_mod.cost_maxcut(n, e, weights=w[perm]), c)


@pytest.mark.parametrize("n,seed", [(2, 5), (6, 6), (11, 7)])
def test_sk_cost_quadratic_form(oracle_mod, n, seed):
    """C = z^T J z / 2 for symmetric zero-diagonal J; mean over all x is 0,
    global spin flip leaves C unchanged."""
    J = sk_couplings(n, seed).astype(np.float64)
    c = oracle_mod.cost_sk(n, J)
    z = (1 - 2 * bits_matrix(n)).astype(np.float64)
    ref = 0.5 * np.einsum("xi,ij,xj->x", z, J, z)
    np.testing.assert_allclose(c, ref, rtol=0, atol=1e-12)
    assert abs(c.mean()) < 1e-12
    np.testing.assert_allclose(c, c[::-1], atol=1e-12)


def test_sk_cost_exact_in_float64(oracle_mod):
    """Couplings on the 2^-20 grid make every C(x) a multiple of 2^-20, so
    the float64 sums carry no rounding at all."""
    n = 14
    J = sk_couplings(n, 11).astype(np.float64)
    assert np.all(J * 2**20 == np.rint(J * 2**20))
    c = oracle_mod.cost_sk(n, J)
    assert np.all(c * 2**20 == np.rint(c * 2**20))


@pytest.mark.parametrize("n,k,seed", [(6, 3, 1), (8, 4, 2), (10, 5, 3)])
def test_dks_cost(oracle_mod, n, k, seed):
    """Induced edge count = x^T A x on Dicke states; mean over the weight-k
    set is |E| k(k-1) / (n(n-1))."""
    e = erdos_renyi(n, 0.5, seed)
    s = oracle_mod.dicke_states(n, k)
    c = oracle_mod.cost_dks(n, e, s)
    x = bits_matrix(n, s.astype(np.int64))
    A = np.zeros((n, n))
    A[e[:, 0], e[:, 1]] = 1
    np.testing.assert_array_equal(c, np.einsum("xi,ij,xj->x", x, A, x))
    assert c.mean() == pytest.approx(len(e) * k * (k - 1) / (n * (n - 1)), abs=1e-12)


# ------------------------------------------------- mixer operators, Eq. 2

@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_x_mixer_hadamard_form(oracle_mod, n):
    """Eq. 2: e^{-i b sum X_i} = H^n diag(e^{-i b (n - 2|x|)}) H^n."""
    rng = np.random.default_rng(n)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    beta = 0.731
    Hn = sla.hadamard(1 << n) / math.sqrt(1 << n)
    w = bits_matrix(n).sum(axis=1)
    ref = Hn @ (np.exp(-1j * beta * (n - 2 * w)) * (Hn @ v))
    np.testing.assert_allclose(oracle_mod.mixer_apply(n, v, beta), ref, atol=1e-12)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_x_hm_matches_pauli_sum(oracle_mod, n):
    rng = np.random.default_rng(10 + n)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    np.testing.assert_allclose(oracle_mod.hm_apply(n, v), dense_x_mixer(n) @ v, atol=1e-12)


@pytest.mark.parametrize("n,k", [(3, 1), (4, 2), (6, 3), (7, 2), (8, 4)])
def test_ring_hm_matches_pauli_sum(oracle_mod, n, k):
    """Ring H_M built from Pauli X, Y on the full 2^n space, restricted to the
    weight-k states, equals the oracle's bit-swap form, and the full operator
    does not leak out of the weight-k subspace."""
    s = oracle_mod.dicke_states(n, k).astype(np.int64)
    Hf = dense_ring_mixer(n)
    mask = np.zeros(1 << n, bool)
    mask[s] = True
    assert np.abs(Hf[np.ix_(~mask, mask)]).max() == 0
    D = len(s)
    Hs = np.stack([oracle_mod.hm_apply(n, np.eye(D)[i], "ring", s) for i in range(D)], axis=1)
    np.testing.assert_allclose(Hs, Hf[np.ix_(s, s)], atol=1e-12)


def free_fermion_ring_spectrum(n, k):
    """Jordan-Wigner: the XY ring is free hopping with amplitude 2, single
    particle energies 4 cos(2 pi (m + s)/n), s = 0 for odd k (periodic),
    s = 1/2 for even k (antiperiodic); many-body levels sum k distinct modes."""
    s = 0.0 if k % 2 else 0.5
    eps = [4 * math.cos(2 * math.pi * (m + s) / n) for m in range(n)]
    return np.sort([sum(c) for c in itertools.combinations(eps, k)])


@pytest.mark.parametrize("n,k", [(4, 2), (5, 2), (6, 3), (7, 3), (8, 4), (9, 4)])
def test_ring_spectrum_free_fermions(oracle_mod, n, k):
    s = oracle_mod.dicke_states(n, k)
    D = len(s)
    Hs = np.stack([oracle_mod.hm_apply(n, np.eye(D)[i], "ring", s) for i in range(D)], axis=1)
    np.testing.assert_allclose(Hs, Hs.conj().T, atol=0)
    ev = np.linalg.eigvalsh(Hs)
    np.testing.assert_allclose(ev, free_fermion_ring_spectrum(n, k), atol=1e-10)
    assert np.trace(Hs).real == pytest.approx(0, abs=1e-12)
    assert np.trace(Hs @ Hs).real == pytest.approx(8 * n * math.comb(n - 2, k - 1), rel=1e-12)


@pytest.mark.parametrize("n,k,beta", [(6, 3, 0.4), (8, 4, 2.9), (7, 3, -1.3)])
def test_ring_mixer_exponential(oracle_mod, n, k, beta):
    """The oracle's series for e^{-i beta H} equals scipy's expm of the
    Pauli-built, restricted ring Hamiltonian."""
    s = oracle_mod.dicke_states(n, k).astype(np.int64)
    Hs = dense_ring_mixer(n)[np.ix_(s, s)]
    rng = np.random.default_rng(3)
    v = rng.standard_normal(len(s)) + 1j * rng.standard_normal(len(s))
    ref = sla.expm(-1j * beta * Hs) @ v
    got = oracle_mod.mixer_apply(n, v, beta, "ring", s)
    np.testing.assert_allclose(got, ref, atol=1e-11 * np.abs(v).max())


def total_spin_clique_spectrum(n, k):
    """sum_{i<j} (X_i X_j + Y_i Y_j) = 2 (S_x^2 + S_y^2) - n = 2 (S^2 - S_z^2) - n
    with S = (1/2) sum of the Pauli vectors.  On weight k, S_z = m = n/2 - k;
    spin s (|m| <= s <= n/2) occurs C(n, n/2 - s) - C(n, n/2 - s - 1) times
    among n spins 1/2, each contributing one state with S_z = m."""
    m = n / 2 - k
    levels = []
    s = abs(m)
    while s <= n / 2 + 1e-9:
        j = round(n / 2 - s)
        mult = math.comb(n, j) - (math.comb(n, j - 1) if j >= 1 else 0)
        levels += [2 * (s * (s + 1) - m * m) - n] * mult
        s += 1
    return np.sort(levels)


@pytest.mark.parametrize("n,k", [(2, 1), (4, 2), (5, 2), (6, 3), (7, 1)])
def test_clique_hm_matches_pauli_sum(oracle_mod, n, k):
    s = oracle_mod.dicke_states(n, k).astype(np.int64)
    Hf = dense_clique_mixer(n)
    mask = np.zeros(1 << n, bool)
    mask[s] = True
    assert np.abs(Hf[np.ix_(~mask, mask)]).max() == 0
    D = len(s)
    Hs = np.stack([oracle_mod.hm_apply(n, np.eye(D)[i], "clique", s) for i in range(D)], axis=1)
    np.testing.assert_allclose(Hs, Hf[np.ix_(s, s)], atol=1e-12)


@pytest.mark.parametrize("n,k", [(4, 2), (6, 2), (7, 3), (8, 4), (9, 4), (10, 3)])
def test_clique_spectrum_total_spin(oracle_mod, n, k):
    s = oracle_mod.dicke_states(n, k)
    D = len(s)
    Hs = np.stack([oracle_mod.hm_apply(n, np.eye(D)[i], "clique", s) for i in range(D)], axis=1)
    np.testing.assert_allclose(Hs, Hs.conj().T, atol=0)
    np.testing.assert_allclose(np.linalg.eigvalsh(Hs), total_spin_clique_spectrum(n, k), atol=1e-9)
    assert np.trace(Hs).real == pytest.approx(0, abs=1e-12)
    # every weight-k state has k (n - k) swap partners, each with element 2
    assert np.trace(Hs @ Hs).real == pytest.approx(4 * k * (n - k) * D, rel=1e-12)


@pytest.mark.parametrize("n,k,beta", [(6, 3, 0.4), (7, 2, -1.1), (8, 4, 2.2)])
def test_clique_mixer_exponential(oracle_mod, n, k, beta):
    s = oracle_mod.dicke_states(n, k).astype(np.int64)
    Hs = dense_clique_mixer(n)[np.ix_(s, s)]
    rng = np.random.default_rng(5)
    v = rng.standard_normal(len(s)) + 1j * rng.standard_normal(len(s))
    ref = sla.expm(-1j * beta * Hs) @ v
    got = oracle_mod.mixer_apply(n, v, beta, "clique", s)
    np.testing.assert_allclose(got, ref, atol=1e-11 * np.abs(v).max())


# ------------------------------------------------ Grover mixer (Sec. 2.4)

@pytest.mark.parametrize("space", ["full6", "dicke8_3"])
def test_grover_mixer_is_projector_exponential(oracle_mod, space):
    if space == "full6":
        n, dim, st = 6, 64, None
    else:
        st = oracle_mod.dicke_states(8, 3)
        n, dim = 8, len(st)
    u = np.full(dim, 1 / math.sqrt(dim))
    H = np.outer(u, u)
    rng = np.random.default_rng(8)
    v = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    np.testing.assert_allclose(oracle_mod.hm_apply(n, v, "grover", st), H @ v, atol=1e-13)
    for beta in (0.3, -2.1):
        np.testing.assert_allclose(oracle_mod.mixer_apply(n, v, beta, "grover", st),
                                   sla.expm(-1j * beta * H) @ v, atol=1e-12)


def _grover_cases(oracle_mod):
    e10 = erdos_renyi(10, 0.5, 21)
    st4 = oracle_mod.dicke_states(10, 4)
    e9 = erdos_renyi(9, 0.4, 22)
    st3 = oracle_mod.dicke_states(9, 3)
    return {
        "maxcut10": (10, oracle_mod.cost_maxcut(10, e10), None, ("maxcut", e10, None)),
        "dks10_4": (10, oracle_mod.cost_dks(10, e10, st4), st4, ("dks", e10, 4)),
        "kvc9_3": (9, oracle_mod.cost_kvc(9, e9, st3), st3, ("kvc", e9, 3)),
    }


@pytest.mark.parametrize("case", ["maxcut10", "dks10_4", "kvc9_3"])
def test_grover_reduced_equals_full_state(oracle_mod, case):
    """Fair sampling (Sec. 2.4): the reduced simulation on (value, degeneracy)
    pairs gives the full-state <C> and gradient."""
    n, cost, st, (prob, e, k) = _grover_cases(oracle_mod)[case]
    counts = oracle_mod.cost_degeneracy(n, e, prob, k)
    assert counts.sum() == len(cost)
    ang = np.random.default_rng(9).random(6) * np.pi
    E_full, g_full = oracle_mod.qaoa_gradient(n, cost, ang, "grover", st)
    E_red, g_red = oracle_mod.grover_reduced_gradient(counts, ang)
    assert E_red == pytest.approx(E_full, abs=1e-11)
    np.testing.assert_allclose(g_red, g_full, atol=1e-10)


def test_grover_p1_closed_form(oracle_mod):
    """p = 1 by hand: after the phase, s = sum_j w_j e^{-i g c_j} (w_j = d_j / N)
    is the overlap with the uniform state, and every state of value c_j has
    amplitude (e^{-i g c_j} + (e^{-i b} - 1) s) / sqrt(N)."""
    n, cost, st, (prob, e, k) = _grover_cases(oracle_mod)["maxcut10"]
    counts = oracle_mod.cost_degeneracy(n, e, prob, k)
    w = counts / counts.sum()
    c = np.arange(len(counts))
    for b, g in [(0.7, 0.4), (2.0, -1.3)]:
        s = np.sum(w * np.exp(-1j * g * c))
        ref = np.sum(w * np.abs(np.exp(-1j * g * c) + (np.exp(-1j * b) - 1) * s) ** 2 * c)
        assert oracle_mod.qaoa_expectation(n, cost, [b, g], "grover") == pytest.approx(ref, abs=1e-11)
        assert oracle_mod.grover_reduced_gradient(counts, [b, g])[0] == pytest.approx(ref, abs=1e-11)


def test_kvc_cost_definition(oracle_mod):
    n, k = 7, 3
    e = erdos_renyi(n, 0.5, 23)
    st = oracle_mod.dicke_states(n, k)
    got = oracle_mod.cost_kvc(n, e, st)
    for a, x in enumerate(st):
        chosen = {i for i in range(n) if (int(x) >> i) & 1}
        assert got[a] == sum(1 for u, v in e if u in chosen or v in chosen)


@pytest.mark.parametrize("prob,n,k", [("dks", 12, 4), ("kvc", 11, 3), ("dks", 9, 9), ("kvc", 10, 1)])
def test_degeneracy_two_enumerations_and_sum_rules(oracle_mod, prob, n, k):
    e = erdos_renyi(n, 0.5, 24)
    m = len(e)
    a = oracle_mod.cost_degeneracy(n, e, prob, k, n_bins=m + 1, method="states")
    b = oracle_mod.cost_degeneracy(n, e, prob, k, n_bins=m + 1, method="subsets")
    np.testing.assert_array_equal(a, b)
    N = math.comb(n, k)
    assert a.sum() == N
    mean = np.dot(np.arange(m + 1), a) / N
    if prob == "dks":  # each edge lies inside a random k-set with prob C(n-2,k-2)/C(n,k)
        ref = m * (math.comb(n - 2, k - 2) if k >= 2 else 0) / N
    else:  # each edge is missed with prob C(n-2,k)/C(n,k)
        ref = m * (1 - math.comb(n - 2, k) / N)
    assert mean == pytest.approx(ref, rel=1e-12)


def test_maxcut_degeneracy_sum_rule(oracle_mod):
    n = 12
    e = erdos_renyi(n, 0.5, 25)
    d = oracle_mod.cost_degeneracy(n, e, "maxcut")
    assert d.sum() == 1 << n
    assert np.dot(np.arange(len(d)), d) / (1 << n) == pytest.approx(len(e) / 2, rel=1e-12)
    # a cut and its complement have the same value: every count is even
    assert np.all(d % 2 == 0)


# ------------------------------------------------- multi-angle QAOA (Sec. 3)

@pytest.mark.parametrize("n,p", [(3, 1), (5, 2), (6, 3)])
def test_multi_angle_vs_dense_expm(oracle_mod, n, p):
    """Round k applies e^{-i g_k C}, then e^{-i sum_q b_{kq} X_q} (the X_q
    commute): a dense expm of the weighted Pauli sum."""
    rng = np.random.default_rng(30 + n)
    cost = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.6, 31 + n))
    a = rng.random(p * (n + 1)) * np.pi
    v = np.full(1 << n, 2 ** (-n / 2), dtype=np.complex128)
    for k in range(p):
        v = np.exp(-1j * a[p * n + k] * cost) * v
        Hk = sum(a[k * n + q] * pauli_op(n, {q: PX}) for q in range(n))
        v = sla.expm(-1j * Hk) @ v
    E_ref = float(np.real(np.vdot(v, cost * v)))
    E, _ = oracle_mod.qaoa_gradient_ma(n, cost, a)
    assert E == pytest.approx(E_ref, abs=1e-12)


def test_multi_angle_reduces_to_standard(oracle_mod):
    """Equal angles on every qubit give the standard QAOA, and by the chain
    rule the per-qubit beta partials of a round sum to dE/dbeta_k."""
    n, p = 7, 3
    cost = oracle_mod.cost_sk(n, sk_couplings(n, 32).astype(np.float64))
    ang = np.random.default_rng(33).random(2 * p) * np.pi
    a = np.concatenate([np.repeat(ang[:p], n), ang[p:]])
    E, g = oracle_mod.qaoa_gradient_ma(n, cost, a)
    E0, g0 = oracle_mod.qaoa_gradient(n, cost, ang)
    assert E == pytest.approx(E0, abs=1e-12)
    np.testing.assert_allclose(g[:p * n].reshape(p, n).sum(axis=1), g0[:p], atol=1e-10)
    np.testing.assert_allclose(g[p * n:], g0[p:], atol=1e-10)


def test_multi_angle_gradient_vs_finite_differences(oracle_mod):
    n, p = 6, 2
    cost = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.5, 34))
    a = np.random.default_rng(35).random(p * (n + 1)) * np.pi
    E, g = oracle_mod.qaoa_gradient_ma(n, cost, a)
    fd = richardson_fd(lambda x: oracle_mod.qaoa_gradient_ma(n, cost, x)[0], a)
    np.testing.assert_allclose(g, fd, atol=1e-8 * max(1.0, np.abs(g).max()))


# ---------------------------------------------- general X mixers (Sec. 2.1)

def dense_x_products(n, coeffs):
    H = 0
    for k, ck in coeffs.items():
        for S in itertools.combinations(range(n), k):
            H = H + ck * pauli_op(n, {q: PX for q in S})
    return H


@pytest.mark.parametrize("coeffs", [{1: 1.0}, {2: 1.0}, {1: 1.0, 2: 0.5}, {3: -0.7, 1: 0.2}, {0: 0.3, 4: 1.0}])
def test_general_mixer_vs_dense_pauli_products(oracle_mod, coeffs):
    n = 5
    d = oracle_mod.krawtchouk_weights(n, coeffs)
    H = dense_x_products(n, coeffs)
    rng = np.random.default_rng(40)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    for beta in (0.6, -1.9):
        np.testing.assert_allclose(oracle_mod.general_mixer_apply(n, d, v, beta), sla.expm(-1j * beta * H) @ v,
                                   atol=1e-11 * np.abs(v).max())


def test_grover_mixer_weights(oracle_mod):
    """|+><+| = prod (1 + X_i)/2: c_k = 2^-n for every k, so d_w = [w = 0]."""
    n = 6
    d = oracle_mod.krawtchouk_weights(n, {k: 2.0 ** -n for k in range(n + 1)})
    np.testing.assert_allclose(d, [1.0] + [0.0] * n, atol=1e-14)
    cost = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.5, 41))
    ang = np.random.default_rng(42).random(4) * np.pi
    E, g = oracle_mod.qaoa_gradient_general(n, d, cost, ang)
    E2, g2 = oracle_mod.qaoa_gradient(n, cost, ang, "grover")
    assert E == pytest.approx(E2, abs=1e-12)
    np.testing.assert_allclose(g, g2, atol=1e-10)


def test_general_mixer_single_x_is_transverse_field(oracle_mod):
    n, p = 7, 3
    cost = oracle_mod.cost_sk(n, sk_couplings(n, 43).astype(np.float64))
    ang = np.random.default_rng(44).random(2 * p) * np.pi
    d = oracle_mod.krawtchouk_weights(n, {1: 1.0})
    np.testing.assert_allclose(d, n - 2 * np.arange(n + 1), atol=1e-14)
    E, g = oracle_mod.qaoa_gradient_general(n, d, cost, ang)
    E0, g0 = oracle_mod.qaoa_gradient(n, cost, ang)
    assert E == pytest.approx(E0, abs=1e-12)
    np.testing.assert_allclose(g, g0, atol=1e-10)


def test_general_mixer_gradient_vs_finite_differences(oracle_mod):
    n, p = 6, 2
    cost = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.5, 45))
    d = oracle_mod.krawtchouk_weights(n, {1: 0.4, 2: 1.0, 3: -0.3})
    ang = np.random.default_rng(46).random(2 * p) * np.pi
    E, g = oracle_mod.qaoa_gradient_general(n, d, cost, ang)
    fd = richardson_fd(lambda x: oracle_mod.qaoa_gradient_general(n, d, cost, x)[0], ang)
    np.testing.assert_allclose(g, fd, atol=1e-8 * max(1.0, np.abs(g).max()))


# -------------------------------------------------------- QAOA state, Eq. 1

@pytest.mark.parametrize("n,p,seed", [(1, 1, 1), (3, 2, 2), (5, 3, 3), (8, 2, 4)])
def test_x_state_vs_dense_expm(oracle_mod, n, p, seed):
    e = erdos_renyi(n, 0.5, seed) if n > 1 else np.zeros((0, 2), np.int32)
    cost = oracle_mod.cost_maxcut(n, e)
    ang = np.random.default_rng(seed).random(2 * p) * np.pi
    psi0 = np.full(1 << n, 2 ** (-n / 2), dtype=np.complex128)
    ref = dense_qaoa_state(dense_x_mixer(n), cost, ang, psi0)
    got = oracle_mod.qaoa_state(n, cost, ang)
    np.testing.assert_allclose(got, ref, atol=1e-12)
    E = oracle_mod.qaoa_expectation(n, cost, ang)
    assert E == pytest.approx(float(np.real(ref.conj() @ (cost * ref))), abs=1e-12)


def test_x_state_custom_initial_state(oracle_mod):
    """Warm start (Sec. 3, initial_state): an arbitrary normalised psi_0."""
    n, p = 6, 3
    J = sk_couplings(n, 21).astype(np.float64)
    cost = oracle_mod.cost_sk(n, J)
    rng = np.random.default_rng(22)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    ang = rng.random(2 * p) * np.pi
    ref = dense_qaoa_state(dense_x_mixer(n), cost, ang, psi0)
    np.testing.assert_allclose(oracle_mod.qaoa_state(n, cost, ang, psi0=psi0), ref, atol=1e-12)


@pytest.mark.parametrize("n,k,p", [(6, 3, 3), (8, 4, 2), (7, 2, 2)])
def test_ring_state_vs_dense_expm(oracle_mod, n, k, p):
    """Densest k-subgraph with the ring mixer from the uniform Dicke state
    (Sec. 2.1, Listing 2, default initial state of Sec. 3)."""
    e = erdos_renyi(n, 0.5, 40 + n)
    s = oracle_mod.dicke_states(n, k)
    cost = oracle_mod.cost_dks(n, e, s)
    Hs = dense_ring_mixer(n)[np.ix_(s.astype(np.int64), s.astype(np.int64))]
    ang = np.random.default_rng(n + k).random(2 * p) * np.pi
    psi0 = np.full(len(s), 1 / math.sqrt(len(s)), dtype=np.complex128)
    ref = dense_qaoa_state(Hs, cost, ang, psi0)
    got = oracle_mod.qaoa_state(n, cost, ang, "ring", s)
    np.testing.assert_allclose(got, ref, atol=1e-11)


def maxcut_p1_closed_form(n, edges, beta, gamma):
    """p=1 MaxCut expectation for any graph (Wang, Hadfield, Jiang, Rieffel,
    PRA 97, 022304 (2018), Theorem 1), phase e^{-i gamma C} then mixer
    e^{-i beta sum X}: per edge (u,v) with d = deg u - 1, e = deg v - 1 and
    f triangles through (u,v),
    <C_uv> = 1/2 + 1/4 sin 4b sin g (cos^d g + cos^e g)
                 - 1/4 sin^2 2b cos^(d+e-2f) g (1 - cos^f 2g)."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    tot = 0.0
    for u, v in edges:
        d, e = len(adj[u]) - 1, len(adj[v]) - 1
        f = len(adj[u] & adj[v])
        cg = math.cos(gamma)
        tot += (0.5 + 0.25 * math.sin(4 * beta) * math.sin(gamma) * (cg**d + cg**e)
                - 0.25 * math.sin(2 * beta) ** 2 * cg ** (d + e - 2 * f)
                * (1 - math.cos(2 * gamma) ** f))
    return tot


@pytest.mark.parametrize("graph", ["er7", "er10", "3reg12", "k5", "er12"])
def test_p1_maxcut_closed_form(oracle_mod, graph):
    if graph == "er7":
        n, e = 7, erdos_renyi(7, 0.5, 1)
    elif graph == "er10":
        n, e = 10, erdos_renyi(10, 0.4, 2)
    elif graph == "er12":
        n, e = 12, erdos_renyi(12, 0.5, 3)
    elif graph == "3reg12":
        n, e = 12, random_regular3(12, 4)
    else:
        n = 5
        e = np.array(list(itertools.combinations(range(5), 2)), dtype=np.int32)
    cost = oracle_mod.cost_maxcut(n, e)
    for beta, gamma in [(0.37, 0.81), (1.1, -0.4), (2.5, 2.0), (0.0, 1.3)]:
        E = oracle_mod.qaoa_expectation(n, cost, [beta, gamma])
        assert E == pytest.approx(maxcut_p1_closed_form(n, e, beta, gamma), abs=1e-12)


# ------------------------------------------------------------- invariants

def test_invariants_x_mixer(oracle_mod):
    n, p = 9, 4
    e = erdos_renyi(n, 0.5, 77)
    cost = oracle_mod.cost_maxcut(n, e)
    rng = np.random.default_rng(5)
    ang = rng.random(2 * p) * np.pi
    psi = oracle_mod.qaoa_state(n, cost, ang)
    assert np.linalg.norm(psi) == pytest.approx(1, abs=1e-13)
    E = oracle_mod.qaoa_expectation(n, cost, ang)
    mean = len(e) / 2
    assert oracle_mod.qaoa_expectation(n, cost, np.zeros(2 * p)) == pytest.approx(mean, abs=1e-12)
    # beta = 0: phases alone leave |psi|^2 uniform; gamma = 0: |+> is an X eigenstate
    a = ang.copy(); a[:p] = 0
    assert oracle_mod.qaoa_expectation(n, cost, a) == pytest.approx(mean, abs=1e-12)
    a = ang.copy(); a[p:] = 0
    assert oracle_mod.qaoa_expectation(n, cost, a) == pytest.approx(mean, abs=1e-12)
    # real C, real H_M, real psi_0: E(-b,-g) = E(b,g) but E(b,-g) differs
    assert oracle_mod.qaoa_expectation(n, cost, -ang) == pytest.approx(E, abs=1e-12)
    a = ang.copy(); a[p:] *= -1
    assert abs(oracle_mod.qaoa_expectation(n, cost, a) - E) > 1e-3
    # e^{-i pi X} = -I: beta period pi; integer C: gamma period 2 pi
    a = ang.copy(); a[1] += np.pi
    assert oracle_mod.qaoa_expectation(n, cost, a) == pytest.approx(E, abs=1e-12)
    a = ang.copy(); a[p + 2] += 2 * np.pi
    assert oracle_mod.qaoa_expectation(n, cost, a) == pytest.approx(E, abs=1e-12)
    # the round order matters: swapping two rounds changes E
    a = ang.copy(); a[[0, 1]] = a[[1, 0]]; a[[p, p + 1]] = a[[p + 1, p]]
    assert abs(oracle_mod.qaoa_expectation(n, cost, a) - E) > 1e-6


def test_invariants_ring_mixer(oracle_mod):
    n, k, p = 8, 4, 3
    e = erdos_renyi(n, 0.5, 8)
    s = oracle_mod.dicke_states(n, k)
    cost = oracle_mod.cost_dks(n, e, s)
    ang = np.random.default_rng(9).random(2 * p) * np.pi
    psi = oracle_mod.qaoa_state(n, cost, ang, "ring", s)
    assert np.linalg.norm(psi) == pytest.approx(1, abs=1e-12)
    mean = cost.mean()
    assert oracle_mod.qaoa_expectation(n, cost, np.zeros(2 * p), "ring", s) == pytest.approx(mean, abs=1e-12)
    E = oracle_mod.qaoa_expectation(n, cost, ang, "ring", s)
    assert oracle_mod.qaoa_expectation(n, cost, -ang, "ring", s) == pytest.approx(E, abs=1e-11)


# --------------------------------------------------------------- gradient

def richardson_fd(f, x, h=1e-3):
    """Central differences at h and h/2 combined to cancel the h^2 term."""
    g = np.zeros_like(x)
    for i in range(len(x)):
        def d(hh):
            ep = np.zeros_like(x); ep[i] = hh
            return (f(x + ep) - f(x - ep)) / (2 * hh)
        g[i] = (4 * d(h / 2) - d(h)) / 3
    return g


@pytest.mark.parametrize("case", ["maxcut_x", "sk_x", "dks_ring", "warm_x", "dks_clique", "maxcut_grover",
                                  "dks_grover_warm", "grover_small_set"])
def test_gradient_vs_finite_differences(oracle_mod, case):
    rng = np.random.default_rng({"maxcut_x": 1, "sk_x": 2, "dks_ring": 3, "warm_x": 4, "dks_clique": 5,
                                 "maxcut_grover": 6, "dks_grover_warm": 7, "grover_small_set": 8}[case])
    psi0 = None
    if case == "maxcut_x":
        n, p, mix, st = 7, 3, "x", None
        cost = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.5, 3))
    elif case == "sk_x":
        n, p, mix, st = 6, 4, "x", None
        cost = oracle_mod.cost_sk(n, sk_couplings(n, 4).astype(np.float64))
    elif case == "warm_x":
        n, p, mix, st = 5, 2, "x", None
        cost = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.7, 5))
        psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
        psi0 /= np.linalg.norm(psi0)
    elif case == "maxcut_grover":
        n, p, mix, st = 7, 3, "grover", None
        cost = oracle_mod.cost_maxcut(n, erdos_renyi(n, 0.5, 7))
    elif case == "dks_grover_warm":
        # the Grover mixer on the weight-3 states (u = the Dicke state), warm start
        n, p, mix, st = 8, 3, "grover", None
        cost = oracle_mod.cost_dks(n, erdos_renyi(n, 0.5, 9), oracle_mod.dicke_states(n, 3))
        psi0 = rng.standard_normal(len(cost)) + 1j * rng.standard_normal(len(cost))
        psi0 /= np.linalg.norm(psi0)
    elif case == "grover_small_set":
        # any listed feasible set: five states with real costs
        n, p, mix, st = 3, 4, "grover", None
        cost = np.array([3.0, -1.0, 4.0, 1.5, -2.5])
    elif case == "dks_clique":
        n, k, p, mix = 7, 3, 2, "clique"
        st = oracle_mod.dicke_states(n, k)
        cost = oracle_mod.cost_dks(n, erdos_renyi(n, 0.5, 8), st)
    else:
        n, k, p, mix = 7, 3, 2, "ring"
        st = oracle_mod.dicke_states(n, k)
        cost = oracle_mod.cost_dks(n, erdos_renyi(n, 0.5, 6), st)
    ang = rng.random(2 * p) * np.pi
    E, g = oracle_mod.qaoa_gradient(n, cost, ang, mix, st, psi0)
    assert E == pytest.approx(oracle_mod.qaoa_expectation(n, cost, ang, mix, st, psi0), abs=1e-12)
    fd = richardson_fd(lambda a: oracle_mod.qaoa_expectation(n, cost, a, mix, st, psi0), ang)
    np.testing.assert_allclose(g, fd, atol=1e-8 * max(1.0, np.abs(g).max()))
    if psi0 is None:
        # real C, H_M and psi_0: E is even in the angles, the gradient odd
        _, gm = oracle_mod.qaoa_gradient(n, cost, -ang, mix, st, psi0)
        np.testing.assert_allclose(gm, -g, atol=1e-10)


def test_gradient_zero_at_zero_angles(oracle_mod):
    """At zero angles psi_0 = |+>^n is an eigenvector of sum X_i and of no
    phase, so both partial derivatives vanish."""
    n, p = 8, 3
    cost = oracle_mod.cost_sk(n, sk_couplings(n, 31).astype(np.float64))
    E, g = oracle_mod.qaoa_gradient(n, cost, np.zeros(2 * p))
    assert E == pytest.approx(cost.mean(), abs=1e-12)
    np.testing.assert_allclose(g, 0, atol=1e-12)


def test_gradient_p1_closed_form(oracle_mod):
    """d<C>/d(beta, gamma) of the p=1 closed form, by central differences of
    the closed form itself."""
    n = 8
    e = erdos_renyi(n, 0.5, 12)
    cost = oracle_mod.cost_maxcut(n, e)
    b, gm = 0.61, 1.27
    _, g = oracle_mod.qaoa_gradient(n, cost, [b, gm])
    h = 1e-5
    db = (maxcut_p1_closed_form(n, e, b + h, gm) - maxcut_p1_closed_form(n, e, b - h, gm)) / (2 * h)
    dg = (maxcut_p1_closed_form(n, e, b, gm + h) - maxcut_p1_closed_form(n, e, b, gm - h)) / (2 * h)
    np.testing.assert_allclose(g, [db, dg], atol=1e-8)


# ------------------------------------------------------- input generators

def test_generators():
    e = random_regular3(20, 3)
    deg = np.bincount(e.ravel(), minlength=20)
    assert np.all(deg == 3) and len({tuple(r) for r in e}) == 30
    assert np.all(e[:, 0] < e[:, 1])
    e2 = erdos_renyi(30, 0.3, 1)
    assert 0.2 < len(e2) / (30 * 29 / 2) < 0.4
    np.testing.assert_array_equal(erdos_renyi(12, 0.5, 7), erdos_renyi(12, 0.5, 7))
    J = sk_couplings(10, 2)
    assert J.dtype == np.float32 and np.all(J == J.T) and np.all(np.diag(J) == 0)
    assert np.all(J.astype(np.float64) * 2**20 == np.rint(J.astype(np.float64) * 2**20))

"""ctypes wrapper of the C oracle (``qaoa_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports
it.  ``build()`` compiles the C file with gcc (OpenMP when available) into
``oracle/_build/liboracle.so``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qaoa_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

MIXER_X = 0
MIXER_RING = 1
MIXER_CLIQUE = 2
MIXER_GROVER = 3
_MIXERS = {"x": MIXER_X, "ring": MIXER_RING, "clique": MIXER_CLIQUE, "grover": MIXER_GROVER}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle; returns the path of the shared library."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "oracle_set_threads": (None, [i32]),
            "oracle_get_threads": (i32, []),
            "oracle_dicke_states": (i64, [i32, i32, P]),
            "oracle_cost_maxcut": (None, [i32, i32, P, P, i64, P, P]),
            "oracle_cost_sk": (None, [i32, P, i64, P, P]),
            "oracle_cost_dks": (None, [i32, i32, P, i64, P, P]),
            "oracle_cost_kvc": (None, [i32, i32, P, i64, P, P]),
            "oracle_qaoa_state": (i32, [i32, i32, i64, P, P, i32, P, P, P]),
            "oracle_qaoa_expectation": (f64, [i32, i32, i64, P, P, i32, P, P]),
            "oracle_qaoa_gradient": (i32, [i32, i32, i64, P, P, i32, P, P, P, P]),
            "oracle_mixer_apply": (i32, [i32, i32, i64, P, f64, P]),
            "oracle_hm_apply": (i32, [i32, i32, i64, P, P, P]),
            "oracle_qaoa_gradient_ma": (i32, [i32, P, i32, P, P, P, P]),
            "oracle_qaoa_gradient_general": (i32, [i32, P, P, i32, P, P, P, P]),
            "oracle_general_mixer_apply": (i32, [i32, P, f64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.complex128)


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def dicke_states(n: int, k: int) -> np.ndarray:
    lib = _load()
    cnt = lib.oracle_dicke_states(n, k, None)
    out = np.empty(cnt, dtype=np.uint64)
    lib.oracle_dicke_states(n, k, _ptr(out))
    return out


def _states_dim(n, states):
    if states is None:
        return 1 << n, None
    states = np.ascontiguousarray(states, dtype=np.uint64)
    return states.shape[0], states


def cost_maxcut(n, edges, weights=None, states=None) -> np.ndarray:
    dim, states = _states_dim(n, states)
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    w = _f64(weights)
    out = np.empty(dim, dtype=np.float64)
    _load().oracle_cost_maxcut(n, e.shape[0], _ptr(e), _ptr(w), dim, _ptr(states), _ptr(out))
    return out


def cost_sk(n, J, states=None) -> np.ndarray:
    dim, states = _states_dim(n, states)
    Jd = _f64(np.asarray(J)).reshape(n, n)
    out = np.empty(dim, dtype=np.float64)
    _load().oracle_cost_sk(n, _ptr(Jd), dim, _ptr(states), _ptr(out))
    return out


def cost_dks(n, edges, states) -> np.ndarray:
    dim, states = _states_dim(n, states)
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    out = np.empty(dim, dtype=np.float64)
    _load().oracle_cost_dks(n, e.shape[0], _ptr(e), dim, _ptr(states), _ptr(out))
    return out


def cost_kvc(n, edges, states) -> np.ndarray:
    dim, states = _states_dim(n, states)
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    out = np.empty(dim, dtype=np.float64)
    _load().oracle_cost_kvc(n, e.shape[0], _ptr(e), dim, _ptr(states), _ptr(out))
    return out


def cost_degeneracy(n, edges, problem, k=None, n_bins=None, method=None) -> np.ndarray:
    """Number of feasible states with each integer cost value 0..n_bins-1, by
    brute force over every feasible state (Sec. 2.4: Grover-QAOA needs only
    the distinct values and their degeneracies).  problem: "maxcut" (all 2^n
    states), "dks" or "kvc" (the C(n, k) weight-k states).  Up to 64 qubits
    from the oracle's cost vectors; above that (weight-k only) from all
    k-subsets drawn with itertools, the cost counted from an adjacency matrix."""
    import itertools

    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if method is None:
        method = "states" if (problem == "maxcut" or n <= 40) else "subsets"
    if method == "states":
        if problem == "maxcut":
            c = cost_maxcut(n, e)
        else:
            st = dicke_states(n, k)
            c = cost_dks(n, e, st) if problem == "dks" else cost_kvc(n, e, st)
    else:
        if problem == "maxcut":
            raise ValueError("brute force over 2^n states needs n <= 64")
        A = np.zeros((n, n), dtype=np.int64)
        A[e[:, 0], e[:, 1]] = 1
        A[e[:, 1], e[:, 0]] = 1
        deg = A.sum(axis=1)
        chunks = []
        it = itertools.combinations(range(n), k)
        while True:
            block = np.array(list(itertools.islice(it, 1 << 18)), dtype=np.int64).reshape(-1, k)
            if block.shape[0] == 0:
                break
            inside = np.zeros(block.shape[0], dtype=np.int64)
            for a in range(k):
                for b in range(a + 1, k):
                    inside += A[block[:, a], block[:, b]]
            if problem == "dks":
                chunks.append(inside)
            else:  # covered edges = sum of degrees - edges counted twice
                chunks.append(deg[block].sum(axis=1) - inside)
        c = np.concatenate(chunks)
    c = np.rint(c).astype(np.int64)
    nb = int(c.max()) + 1 if n_bins is None else n_bins
    return np.bincount(c, minlength=nb)[:nb].astype(np.int64)


def grover_reduced_gradient(counts, angles, values=None):
    """<C> and its 2p derivatives for QAOA with the Grover mixer and the
    uniform initial state, on the distinct cost values (Sec. 2.4).

    Fair sampling: every state of cost c_j keeps one amplitude, so the
    weighted vector b_j = sqrt(d_j) a_j (d_j = degeneracy, N = sum d) evolves
    as a QAOA on len(counts) states with cost diag(c_j), initial state
    u_j = sqrt(d_j / N) and mixer H_G = u u^T.  Plain complex128 reverse mode,
    the same recurrences as the full-state oracle."""
    d = np.asarray(counts, dtype=np.float64)
    c = np.arange(d.shape[0], dtype=np.float64) if values is None else np.asarray(values, dtype=np.float64)
    a = np.asarray(angles, dtype=np.float64)
    p = a.shape[0] // 2
    u = np.sqrt(d / d.sum())

    def mix(v, beta):
        return v + (np.exp(-1j * beta) - 1.0) * np.dot(u, v) * u

    psi = u.astype(np.complex128)
    for k in range(p):
        psi = np.exp(-1j * a[p + k] * c) * psi
        psi = mix(psi, a[k])
    E = float(np.sum(c * np.abs(psi) ** 2))
    lam = c * psi
    g = np.zeros(2 * p)
    for k in range(p - 1, -1, -1):
        g[k] = 2.0 * np.imag(np.conj(np.dot(u, lam)) * np.dot(u, psi))
        lam, psi = mix(lam, -a[k]), mix(psi, -a[k])
        g[p + k] = 2.0 * np.imag(np.sum(np.conj(lam) * c * psi))
        ph = np.exp(1j * a[p + k] * c)
        lam, psi = ph * lam, ph * psi
    return E, g


def _problem(mixer, n, cost, states):
    kind = _MIXERS[mixer]
    cost = _f64(cost)
    if kind in (MIXER_RING, MIXER_CLIQUE):
        if states is None:
            raise ValueError(f"the {mixer} mixer needs the feasible states")
        states = np.ascontiguousarray(states, dtype=np.uint64)
    else:
        states = None  # X: all 2^n states; Grover: whatever set the cost vector covers
    return kind, cost, states, cost.shape[0]


def qaoa_state(n, cost, angles, mixer="x", states=None, psi0=None) -> np.ndarray:
    kind, cost, states, dim = _problem(mixer, n, cost, states)
    a = _f64(angles)
    p = a.shape[0] // 2
    out = np.empty(dim, dtype=np.complex128)
    r = _load().oracle_qaoa_state(kind, n, dim, _ptr(states), _ptr(cost), p, _ptr(a),
                                  _ptr(_c128(psi0)), _ptr(out))
    if r:
        raise RuntimeError(f"oracle_qaoa_state failed ({r})")
    return out


def qaoa_expectation(n, cost, angles, mixer="x", states=None, psi0=None) -> float:
    kind, cost, states, dim = _problem(mixer, n, cost, states)
    a = _f64(angles)
    p = a.shape[0] // 2
    e = _load().oracle_qaoa_expectation(kind, n, dim, _ptr(states), _ptr(cost), p, _ptr(a),
                                        _ptr(_c128(psi0)))
    if not np.isfinite(e):
        raise RuntimeError("oracle_qaoa_expectation failed")
    return float(e)


def qaoa_gradient(n, cost, angles, mixer="x", states=None, psi0=None):
    """Returns (E, grad[2p]) by exact reverse mode in complex128."""
    kind, cost, states, dim = _problem(mixer, n, cost, states)
    a = _f64(angles)
    p = a.shape[0] // 2
    E = np.zeros(1)
    g = np.zeros(2 * p)
    r = _load().oracle_qaoa_gradient(kind, n, dim, _ptr(states), _ptr(cost), p, _ptr(a),
                                     _ptr(_c128(psi0)), _ptr(E), _ptr(g))
    if r:
        raise RuntimeError(f"oracle_qaoa_gradient failed ({r})")
    return float(E[0]), g


def qaoa_gradient_ma(n, cost, angles, psi0=None):
    """Multi-angle QAOA with one X angle per (round, qubit): angles =
    [beta_{1,0..n-1}, ..., beta_{p,0..n-1}, gamma_1..gamma_p]; returns
    (E, grad) in the same layout, exact reverse mode in complex128."""
    cost = _f64(cost)
    a = _f64(angles)
    p = a.shape[0] // (n + 1)
    if p * (n + 1) != a.shape[0]:
        raise ValueError("multi-angle QAOA needs p (n + 1) angles")
    E = np.zeros(1)
    g = np.zeros(a.shape[0])
    r = _load().oracle_qaoa_gradient_ma(n, _ptr(cost), p, _ptr(a), _ptr(_c128(psi0)), _ptr(E), _ptr(g))
    if r:
        raise RuntimeError(f"oracle_qaoa_gradient_ma failed ({r})")
    return float(E[0]), g


def krawtchouk_weights(n, coeffs) -> np.ndarray:
    """d_w = sum_k c_k K_k(w) for w = 0..n: the Hadamard-basis eigenvalues of
    f(X) = sum_S c_{|S|} prod_{i in S} X_i (Sec. 2.1); coeffs maps the term
    order k to c_k."""
    import math

    d = np.zeros(n + 1)
    for w in range(n + 1):
        for k, ck in coeffs.items():
            d[w] += ck * sum((-1) ** j * math.comb(w, j) * math.comb(n - w, k - j) for j in range(0, k + 1))
    return d


def qaoa_gradient_general(n, d, cost, angles, psi0=None):
    """(E, grad) of QAOA with the general X mixer H^n diag(d_|z|) H^n."""
    dd = _f64(d)
    if dd.shape[0] != n + 1:
        raise ValueError("d needs n + 1 entries")
    cost = _f64(cost)
    a = _f64(angles)
    p = a.shape[0] // 2
    E = np.zeros(1)
    g = np.zeros(2 * p)
    r = _load().oracle_qaoa_gradient_general(n, _ptr(dd), _ptr(cost), p, _ptr(a), _ptr(_c128(psi0)), _ptr(E),
                                             _ptr(g))
    if r:
        raise RuntimeError(f"oracle_qaoa_gradient_general failed ({r})")
    return float(E[0]), g


def general_mixer_apply(n, d, psi, beta) -> np.ndarray:
    v = _c128(psi).copy()
    r = _load().oracle_general_mixer_apply(n, _ptr(_f64(d)), float(beta), _ptr(v))
    if r:
        raise RuntimeError(f"oracle_general_mixer_apply failed ({r})")
    return v


def mixer_apply(n, psi, beta, mixer="x", states=None) -> np.ndarray:
    kind = _MIXERS[mixer]
    v = _c128(psi).copy()
    st = None if states is None else np.ascontiguousarray(states, dtype=np.uint64)
    r = _load().oracle_mixer_apply(kind, n, v.shape[0], _ptr(st), float(beta), _ptr(v))
    if r:
        raise RuntimeError(f"oracle_mixer_apply failed ({r})")
    return v


def hm_apply(n, psi, mixer="x", states=None) -> np.ndarray:
    kind = _MIXERS[mixer]
    v = _c128(psi)
    st = None if states is None else np.ascontiguousarray(states, dtype=np.uint64)
    out = np.empty_like(v)
    r = _load().oracle_hm_apply(kind, n, v.shape[0], _ptr(st), _ptr(v), _ptr(out))
    if r:
        raise RuntimeError(f"oracle_hm_apply failed ({r})")
    return out

"""GB300 (sm_103a) QAOA statevector simulation: Python binding of the C ABI.

Every method below marshals arguments into one call of the C library declared
in ``include/qaoa.h`` (same names without the ``qaoa_`` prefix on the context
methods); all computation happens in the CUDA kernels.  PyTorch provides device
memory and streams only.  There is no CPU fallback: without the built library
or a CUDA device the calls raise.

Conventions (arXiv 2312.06451, Eq. 1 and Listing 1): qubit i is bit i of the
basis index, angles are ``[beta_1..beta_p, gamma_1..gamma_p]``, round k applies
``e^{-i gamma_k C}`` then ``e^{-i beta_k H_M}``, the default initial state is the
uniform superposition over the feasible set.
"""

from __future__ import annotations

import ctypes
import math
import itertools

import numpy as np
import torch

from . import _binding as B
from ._binding import QAOAError  # noqa: F401

__all__ = ["Context", "XMixer", "EigenMixer", "QAOAExpectation", "QAOAError", "pass_schedule",
           "qaoa_cost_precompute", "qaoa_expectation", "qaoa_gradient", "qaoa_expectation_batched",
           "qaoa_gradient_small_noalloc", "ring_eigen_mixer", "clique_eigen_mixer", "xy_eigen_mixer",
           "save_eigen_mixer", "load_eigen_mixer", "GeneralXMixer", "x_terms_mixer", "grover_x_mixer", "GroverMixer",
           "write_tuning_file", "read_tuning_file", "krawtchouk_weights", "EigenSymMixer", "xy_block_hamiltonians", "xy_sym_mixer", "BatchedCall",
           "HostBatchedCall", "qaoa_expectation_batched_host"]

_MIXER_IDS = itertools.count(1)

_PROBLEMS = {"maxcut": B.QAOA_PROBLEM_MAXCUT, "wmaxcut": B.QAOA_PROBLEM_WMAXCUT,
             "sk": B.QAOA_PROBLEM_SK, "dks": B.QAOA_PROBLEM_DKS, "kvc": B.QAOA_PROBLEM_KVC}
_GEMM = {"fp32": B.QAOA_GEMM_FP32_SIMT, "3xtf32": B.QAOA_GEMM_3XTF32, "bf16x3": B.QAOA_GEMM_BF16X3}


def _cost_dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.uint8:
        return B.QAOA_COST_U8
    if t.dtype == torch.float32:
        return B.QAOA_COST_F32
    raise TypeError(f"cost vector must be uint8 or float32, got {t.dtype}")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_tensor(t, name):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return t


def _host_tensor(t, name):
    """A contiguous float64 host tensor (numpy arrays are wrapped, not copied)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(t)
    if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.is_contiguous()
            and t.dtype == torch.float64):
        raise ValueError(f"{name} must be a contiguous float64 host tensor or array")
    return t


class XMixer:
    """Transverse-field mixer H_M = sum_i X_i on all 2^n states (Eq. 2).

    multi_angle=True: one angle per qubit and round (multi-angle QAOA, Sec. 3);
    an angle set is then [beta_{1,0..n-1}, ..., beta_{p,0..n-1}, gamma_1..gamma_p]."""

    def __init__(self, n: int, multi_angle: bool = False):
        self.n = int(n)
        self.dim = 1 << self.n
        self.multi_angle = bool(multi_angle)
        kind = B.QAOA_MIXER_X_MA if self.multi_angle else B.QAOA_MIXER_X
        self.struct = B.QaoaMixer(kind, self.n, self.dim, None, None, 0)

    def rounds(self, n_angles: int) -> int:
        per = self.n + 1 if self.multi_angle else 2
        if n_angles % per:
            raise ValueError(f"{n_angles} angles do not make whole rounds of {per}")
        return n_angles // per


class GeneralXMixer:
    """A sum of products of Pauli X, f(X) = sum_S c_|S| prod_{i in S} X_i, on
    all 2^n states (Sec. 2.1), given by its Hadamard-basis eigenvalues d_w for
    w = 0..n (e^{-i b f(X)} = H^n e^{-i b f(Z)} H^n, f(Z) = d_|z|)."""

    def __init__(self, n: int, weights, device: int = 0):
        w = torch.as_tensor(np.asarray(weights, dtype=np.float64))
        if w.shape != (n + 1,):
            raise ValueError(f"need n + 1 = {n + 1} weights")
        self.n = int(n)
        self.dim = 1 << self.n
        self.weights = w.to(f"cuda:{device}").contiguous()
        self.struct = B.QaoaMixer(B.QAOA_MIXER_X_GENERAL, self.n, self.dim, None, self.weights.data_ptr(), 0)


def krawtchouk_weights(n: int, coeffs: dict) -> np.ndarray:
    """Hadamard-basis eigenvalues d_w, w = 0..n, of f(X) = sum_S c_|S| prod X_i
    (qaoa_x_mixer_weights); coeffs maps the term order k to c_k."""
    kmax = max(coeffs) if coeffs else 0
    c = np.zeros(kmax + 1, dtype=np.float64)
    for k, ck in coeffs.items():
        c[int(k)] = float(ck)
    d = np.zeros(n + 1, dtype=np.float64)
    st = B.load().qaoa_x_mixer_weights(int(n), kmax, c.ctypes.data_as(ctypes.c_void_p),
                                       d.ctypes.data_as(ctypes.c_void_p))
    if st != B.QAOA_OK:
        raise QAOAError(st, f"qaoa_x_mixer_weights(n={n}, kmax={kmax}) failed")
    return d


def x_terms_mixer(n: int, coeffs: dict, device: int = 0) -> GeneralXMixer:
    """mixer_X-style sums (Sec. 3): coeffs maps the term order k to c_k, e.g.
    {1: 1, 2: 1} for sum_i X_i + sum_{i<j} X_i X_j."""
    return GeneralXMixer(n, krawtchouk_weights(n, coeffs), device)


def grover_x_mixer(n: int, device: int = 0) -> GeneralXMixer:
    """Grover mixer |+><+| on all 2^n states (Sec. 2.4): d_w = [w = 0]."""
    return GeneralXMixer(n, [1.0] + [0.0] * n, device)


class GroverMixer:
    """Grover mixer |u><u| (Sec. 2.4), u the uniform superposition over the dim
    states a cost vector lists: all 2^n states, the binom(n, k) weight-k states,
    or any other feasible set.  Applied as the rank-one update
    phi + (e^{-i b} - 1) <u|phi> u, one streaming pass per round
    (QAOA_MIXER_GROVER); n only labels the problem."""

    def __init__(self, dim: int, n: int = 0):
        self.dim = int(dim)
        if self.dim < 1:
            raise ValueError("a Grover mixer needs at least one feasible state")
        self.n = int(n)
        self.struct = B.QaoaMixer(B.QAOA_MIXER_GROVER, self.n, self.dim, None, None, 0)

    @classmethod
    def full(cls, n: int) -> "GroverMixer":
        """On all 2^n states (u = |+>^n)."""
        return cls(1 << int(n), n)

    @classmethod
    def dicke(cls, n: int, k: int) -> "GroverMixer":
        """On the binom(n, k) Hamming-weight-k states (u = the Dicke state)."""
        return cls(math.comb(int(n), int(k)), n)


class EigenMixer:
    """Constrained mixer through its stored eigendecomposition H_M V = V diag(lam)
    on the D feasible states (Sec. 2.1); V: D x D float32 CUDA tensor (columns
    are eigenvectors), lam: D float64 CUDA tensor."""

    def __init__(self, n: int, V: torch.Tensor, lam: torch.Tensor, precision: str = "3xtf32"):
        V = _dev_tensor(V, "V")
        lam = _dev_tensor(lam, "lam")
        if V.dtype != torch.float32 or lam.dtype != torch.float64:
            raise TypeError("V must be float32 and lam float64")
        self.n = int(n)
        self.dim = int(lam.shape[0])
        self.V, self.lam = V, lam
        # a fresh id per mixer object: the library keeps its prepared copies
        # of V under it (addresses alone are reused once tensors are freed)
        self.struct = B.QaoaMixer(B.QAOA_MIXER_EIGEN, self.n, self.dim, V.data_ptr(), lam.data_ptr(),
                                  _GEMM[precision], 0, next(_MIXER_IDS))


MIXER_FILE_VERSION = 1


def save_eigen_mixer(path: str, n: int, k: int, V: torch.Tensor, lam: torch.Tensor, kind: str = "ring"):
    """Store a mixer's eigendecomposition for re-use (the paper saves the costly
    constrained-mixer decomposition to a user file, Sec. 3, Listing 2).  The file
    carries a format version, the problem shape and a SHA-256 of the arrays."""
    import hashlib

    Vh = V.detach().to("cpu", torch.float32).contiguous().numpy()
    lh = lam.detach().to("cpu", torch.float64).contiguous().numpy()
    digest = hashlib.sha256(Vh.tobytes() + lh.tobytes()).hexdigest()
    with open(path, "wb") as f:
        np.savez(f, V=Vh, lam=lh, meta=np.array([MIXER_FILE_VERSION, n, k], dtype=np.int64),
                 kind=np.array(kind), sha256=np.array(digest))


def load_eigen_mixer(path: str, n: int, k: int, kind: str = "ring", device: int = 0):
    """Read a file written by save_eigen_mixer; raises ValueError when the
    version, shape or checksum does not match (a truncated or altered file)."""
    import hashlib

    try:
        with np.load(path, allow_pickle=False) as z:
            meta, V, lam = z["meta"], z["V"], z["lam"]
            fkind, digest = str(z["kind"]), str(z["sha256"])
    except Exception as e:  # zipfile / npy errors of a damaged file
        raise ValueError(f"unreadable mixer file {path}: {e}") from e
    if meta.tolist() != [MIXER_FILE_VERSION, n, k] or fkind != kind:
        raise ValueError(f"mixer file {path} is for {fkind} {meta.tolist()}, wanted {kind} [{MIXER_FILE_VERSION}, {n}, {k}]")
    if hashlib.sha256(np.ascontiguousarray(V).tobytes() + np.ascontiguousarray(lam).tobytes()).hexdigest() != digest:
        raise ValueError(f"mixer file {path} fails its checksum")
    dev = f"cuda:{device}"
    return torch.from_numpy(V).to(dev), torch.from_numpy(lam).to(dev)


def xy_eigen_mixer(ctx: "Context", kind: str, n: int, k: int, precision: str = "fp32",
                   cache_file: str | None = None):
    """EigenMixer of the ring or clique XY mixer on the Hamming-weight-k states.

    Pre-computation (Sec. 2.1, done once): the dense Hamiltonian is built by
    the library (qaoa_ring_hamiltonian / qaoa_clique_hamiltonian) and
    diagonalised in float64 with torch.linalg.eigh; V is kept in float32, the
    eigenvalues in float64.  With cache_file the decomposition is loaded from /
    saved to that file (Sec. 3: mixer_clique(...; file))."""
    import os

    if kind not in ("ring", "clique"):
        raise ValueError(f"unknown XY mixer {kind!r}")
    if cache_file and os.path.exists(cache_file):
        V, lam = load_eigen_mixer(cache_file, n, k, kind, ctx.device)
    else:
        H = ctx.ring_hamiltonian(n, k) if kind == "ring" else ctx.clique_hamiltonian(n, k)
        lam, V64 = torch.linalg.eigh(H)
        V = V64.to(torch.float32).contiguous()
        del V64, H
        if cache_file:
            save_eigen_mixer(cache_file, n, k, V, lam, kind)
    return EigenMixer(n, V.contiguous(), lam.contiguous(), precision)


class EigenSymMixer:
    """Ring or clique XY mixer on the weight-k states through the
    eigendecompositions of its cyclic-shift blocks (QAOA_MIXER_EIGEN_SYM):
    V holds the block eigenvector matrices back to back (float32), lam the
    eigenvalues block after block (float64)."""

    def __init__(self, n: int, k: int, V: torch.Tensor, lam: torch.Tensor, block_dims, precision: str = "3xtf32"):
        V = _dev_tensor(V, "V")
        lam = _dev_tensor(lam, "lam")
        if V.dtype != torch.float32 or lam.dtype != torch.float64:
            raise TypeError("V must be float32 and lam float64")
        dims = [int(d) for d in block_dims]
        if V.numel() != sum(d * d for d in dims) or lam.numel() != sum(dims):
            raise ValueError("V and lam do not match the block sizes")
        self.n, self.k = int(n), int(k)
        self.dim = int(lam.numel())
        self.block_dims = dims
        self.V, self.lam = V, lam
        self.struct = B.QaoaMixer(B.QAOA_MIXER_EIGEN_SYM, self.n, self.dim, V.data_ptr(), lam.data_ptr(),
                                  _GEMM[precision], self.k, next(_MIXER_IDS))


def xy_block_hamiltonians(kind: str, n: int, k: int):
    """(block sizes, [H_b as float64 numpy arrays]) of the ring or clique XY
    mixer in the real momentum basis of the cyclic qubit shift
    (qaoa_xy_block_hamiltonians; host-only)."""
    lib = B.load()
    mk = {"ring": B.QAOA_XY_RING, "clique": B.QAOA_XY_CLIQUE}[kind]
    nb = ctypes.c_int(0)
    st = lib.qaoa_xy_block_hamiltonians(mk, int(n), int(k), ctypes.byref(nb), None, None)
    if st != B.QAOA_OK:
        raise QAOAError(st, f"qaoa_xy_block_hamiltonians({kind}, n={n}, k={k}) failed")
    dims = np.zeros(nb.value, dtype=np.int64)
    dims_only = nb.value
    st = lib.qaoa_xy_block_hamiltonians(mk, int(n), int(k), ctypes.byref(nb), dims.ctypes.data_as(ctypes.c_void_p),
                                        None)
    if st != B.QAOA_OK or nb.value != dims_only:
        raise QAOAError(st, "qaoa_xy_block_hamiltonians failed")
    H = np.zeros(int(np.sum(dims * dims)), dtype=np.float64)
    st = lib.qaoa_xy_block_hamiltonians(mk, int(n), int(k), ctypes.byref(nb), dims.ctypes.data_as(ctypes.c_void_p),
                                        H.ctypes.data_as(ctypes.c_void_p))
    if st != B.QAOA_OK:
        raise QAOAError(st, "qaoa_xy_block_hamiltonians failed")
    out, o = [], 0
    for d in dims.tolist():
        out.append(H[o:o + d * d].reshape(d, d))
        o += d * d
    return dims.tolist(), out


def xy_sym_mixer(ctx: "Context", kind: str, n: int, k: int, precision: str = "3xtf32",
                 cache_file: str | None = None) -> EigenSymMixer:
    """EigenSymMixer of the ring or clique XY mixer: the block matrices come
    from the library, each is diagonalised once in float64 with
    torch.linalg.eigh (the pre-computation the paper does for the dense
    mixer, Sec. 2.1, now on blocks of about 2D/n states).  With cache_file the
    block eigenvectors and eigenvalues are loaded from / saved to that file
    (save_eigen_mixer's format, kind "<kind>-blocks")."""
    import os

    dims, Hs = xy_block_hamiltonians(kind, n, k)
    tag = f"{kind}-blocks"
    if cache_file and os.path.exists(cache_file):
        V, lam = load_eigen_mixer(cache_file, n, k, tag, ctx.device)
        if V.numel() != sum(d * d for d in dims) or lam.numel() != sum(dims):
            raise ValueError(f"mixer file {cache_file} does not match the {kind} blocks of n={n}, k={k}")
        return EigenSymMixer(n, k, V.to(torch.float32), lam.to(torch.float64), dims, precision)
    dev = f"cuda:{ctx.device}"
    Vs, lams = [], []
    for H in Hs:
        lam, V = torch.linalg.eigh(torch.from_numpy(H).to(dev))
        Vs.append(V.to(torch.float32).reshape(-1))
        lams.append(lam)
    V = torch.cat(Vs).contiguous()
    lam = torch.cat(lams).contiguous()
    if cache_file:
        save_eigen_mixer(cache_file, n, k, V, lam, tag)
    return EigenSymMixer(n, k, V, lam, dims, precision)


def ring_eigen_mixer(ctx: "Context", n: int, k: int, precision: str = "fp32", cache_file: str | None = None):
    """EigenMixer of the ring mixer (see xy_eigen_mixer)."""
    return xy_eigen_mixer(ctx, "ring", n, k, precision, cache_file)


def clique_eigen_mixer(ctx: "Context", n: int, k: int, precision: str = "fp32", cache_file: str | None = None):
    """EigenMixer of the clique mixer (see xy_eigen_mixer)."""
    return xy_eigen_mixer(ctx, "clique", n, k, precision, cache_file)


TUNING_FILE_FORMAT = "qaoa-gb300-xtune"
TUNING_FILE_VERSION = 1
_XTUNE_KEYS = ("n", "cost_dtype", "cmin", "split", "nbuf_bwd_contig", "nbuf_bwd_gather")


def _tuning_digest(entries) -> str:
    import hashlib
    import json

    return hashlib.sha256(json.dumps(entries, sort_keys=True).encode()).hexdigest()


def write_tuning_file(path: str, entries, gpu: str = "") -> None:
    """Store X-mixer pass schedules (autotune() results) for re-use: a JSON
    file with a format tag and version, the GPU they were tuned on and a
    SHA-256 of the entries.  Written to a temporary name and renamed, so a
    crash never leaves a half-written file under `path`."""
    import json
    import os

    ents = [dict({k: int(e[k]) for k in _XTUNE_KEYS}, ms=float(e.get("ms", 0.0))) for e in entries]
    doc = {"format": TUNING_FILE_FORMAT, "version": TUNING_FILE_VERSION, "gpu": gpu, "entries": ents,
           "sha256": _tuning_digest(ents)}
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1)
    os.replace(tmp, path)


def read_tuning_file(path: str, gpu: str | None = None) -> list:
    """Entries of a file written by write_tuning_file.  Raises ValueError for a
    damaged or altered file, another format or version, or (gpu given) a file
    tuned on another GPU.  The values are checked again by the library when
    installed (qaoa_set_xtune)."""
    import json

    try:
        with open(path) as f:
            doc = json.load(f)
    except (OSError, ValueError) as e:
        raise ValueError(f"unreadable tuning file {path}: {e}") from e
    if not isinstance(doc, dict) or doc.get("format") != TUNING_FILE_FORMAT:
        raise ValueError(f"{path} is not a pass-schedule tuning file")
    if doc.get("version") != TUNING_FILE_VERSION:
        raise ValueError(f"tuning file {path} has version {doc.get('version')}, wanted {TUNING_FILE_VERSION}")
    ents = doc.get("entries")
    if not isinstance(ents, list) or _tuning_digest(ents) != doc.get("sha256"):
        raise ValueError(f"tuning file {path} fails its checksum")
    for e in ents:
        if not isinstance(e, dict) or any(not isinstance(e.get(k), int) for k in _XTUNE_KEYS):
            raise ValueError(f"tuning file {path} holds a malformed entry")
    if gpu is not None and doc.get("gpu") != gpu:
        raise ValueError(f"tuning file {path} was tuned on {doc.get('gpu')!r}, this is {gpu!r}")
    return ents


class Context:
    """A library context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self._lib = B.load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        st = self._lib.qaoa_create(ctypes.byref(h), self.device, ctypes.c_void_p(self.stream.cuda_stream))
        if st != B.QAOA_OK:
            raise QAOAError(st, "qaoa_create failed")
        self._h = h
        self._tuned = {}  # (n, cost dtype) -> schedule installed by autotune() / set_tuning()

    # ------------------------------------------------------------ plumbing
    def close(self):
        if getattr(self, "_h", None):
            self._lib.qaoa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int):
        if st != B.QAOA_OK:
            msg = self._lib.qaoa_last_error(self._h)
            raise QAOAError(st, msg.decode() if msg else "")

    # ----------------------------------------------------- pre-computation
    def cost_precompute(self, problem: str, n: int, *, edges=None, weights=None, J=None, k: int = -1,
                        dtype: torch.dtype = torch.uint8) -> torch.Tensor:
        """Cost vector over the feasible set as a new CUDA tensor (qaoa_cost_precompute)."""
        kind = _PROBLEMS[problem]
        e = None if edges is None else np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        Jh = None if J is None else np.ascontiguousarray(J, dtype=np.float32).reshape(n, n)
        m = 0 if e is None else e.shape[0]
        if kind in (B.QAOA_PROBLEM_DKS, B.QAOA_PROBLEM_KVC):
            dim = int(np.round(np.prod([(n - i) / (i + 1) for i in range(k)]))) if k > 0 else 1
        else:
            dim = 1 << n
        out = torch.empty(dim, dtype=dtype, device=f"cuda:{self.device}")
        prob = B.QaoaProblem(kind, n, k, m,
                             None if e is None else e.ctypes.data_as(ctypes.c_void_p),
                             None if w is None else w.ctypes.data_as(ctypes.c_void_p),
                             None if Jh is None else Jh.ctypes.data_as(ctypes.c_void_p))
        self._check(self._lib.qaoa_cost_precompute(self._h, ctypes.byref(prob), _ptr(out),
                                                   _cost_dtype(out), dim))
        return out

    def cost_degeneracy(self, problem: str, n: int, *, edges, k: int = -1, n_bins: int | None = None) -> torch.Tensor:
        """Number of feasible states with each cost value 0..n_bins-1 as an
        int64 CUDA tensor (qaoa_cost_degeneracy): "maxcut" over all 2^n states
        (k = -1), "dks" / "kvc" over the weight-k states (n <= 128)."""
        kind = _PROBLEMS[problem]
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        m = e.shape[0]
        top = min(m, k * (k - 1) // 2) if problem == "dks" else m  # the largest possible cost
        nb = top + 1 if n_bins is None else int(n_bins)
        out = torch.empty(nb, dtype=torch.int64, device=f"cuda:{self.device}")
        prob = B.QaoaProblem(kind, n, k, m, e.ctypes.data_as(ctypes.c_void_p), None, None)
        self._check(self._lib.qaoa_cost_degeneracy(self._h, ctypes.byref(prob), _ptr(out), nb))
        return out

    def grover_batched(self, counts: torch.Tensor, angles: torch.Tensor, want_grad: bool = True):
        """(E, grad) CUDA float64 tensors for QAOA with the Grover mixer on the
        degeneracies `counts` (qaoa_grover_batched); angles: n_sets x 2p
        float64 CUDA tensor.  Asynchronous on the context stream."""
        counts = _dev_tensor(counts, "counts")
        A = _dev_tensor(angles, "angles")
        if counts.dtype != torch.int64 or A.dtype != torch.float64:
            raise TypeError("counts must be int64 and angles float64")
        A = A.reshape(-1, A.shape[-1]).contiguous()
        S, p2 = A.shape
        E = torch.empty(S, dtype=torch.float64, device=A.device)
        G = torch.empty(S, p2, dtype=torch.float64, device=A.device) if want_grad else None
        self._check(self._lib.qaoa_grover_batched(self._h, _ptr(counts), counts.shape[0], p2 // 2, S, _ptr(A),
                                                  _ptr(E), _ptr(G)))
        return E, G

    def dicke_states(self, n: int, k: int) -> torch.Tensor:
        """Hamming-weight-k states in increasing order (int64 CUDA tensor)."""
        dim = int(round(np.prod([(n - i) / (i + 1) for i in range(k)]))) if k > 0 else 1
        out = torch.empty(dim, dtype=torch.int64, device=f"cuda:{self.device}")
        self._check(self._lib.qaoa_dicke_states(self._h, n, k, _ptr(out), dim))
        return out

    def ring_hamiltonian(self, n: int, k: int) -> torch.Tensor:
        """Dense ring mixer on the weight-k states (float64 CUDA tensor)."""
        dim = int(round(np.prod([(n - i) / (i + 1) for i in range(k)]))) if k > 0 else 1
        out = torch.empty((dim, dim), dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self._lib.qaoa_ring_hamiltonian(self._h, n, k, _ptr(out), dim))
        return out

    def clique_hamiltonian(self, n: int, k: int) -> torch.Tensor:
        """Dense clique mixer on the weight-k states (float64 CUDA tensor)."""
        dim = int(round(np.prod([(n - i) / (i + 1) for i in range(k)]))) if k > 0 else 1
        out = torch.empty((dim, dim), dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self._lib.qaoa_clique_hamiltonian(self._h, n, k, _ptr(out), dim))
        return out

    # ---------------------------------------------------------- simulation
    def expectation(self, cost: torch.Tensor, mixer, angles, init: torch.Tensor | None = None) -> float:
        """<C> for one angle set (qaoa_expectation); angles: 2p host values."""
        cost = _dev_tensor(cost, "cost")
        init = _dev_tensor(init, "init")
        a = np.ascontiguousarray(np.asarray(angles, dtype=np.float64).ravel())
        E = ctypes.c_double()
        self._check(self._lib.qaoa_expectation(self._h, _ptr(cost), _cost_dtype(cost),
                                               ctypes.byref(mixer.struct), _ptr(init), _rounds(mixer, a.shape[0]),
                                               a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(E)))
        return E.value

    def gradient(self, cost: torch.Tensor, mixer, angles, init: torch.Tensor | None = None,
                 ckpt=True):
        """(<C>, d<C>/d angles) for one angle set (qaoa_gradient).  ckpt:
        False / "none", True / "round" or "pass" (QAOA_CKPT_*)."""
        cost = _dev_tensor(cost, "cost")
        init = _dev_tensor(init, "init")
        a = np.ascontiguousarray(np.asarray(angles, dtype=np.float64).ravel())
        E = ctypes.c_double()
        g = np.zeros(a.shape[0], dtype=np.float64)
        self._check(self._lib.qaoa_gradient(self._h, _ptr(cost), _cost_dtype(cost), ctypes.byref(mixer.struct),
                                            _ptr(init), _rounds(mixer, a.shape[0]), a.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(E), g.ctypes.data_as(ctypes.c_void_p),
                                            _ckpt_mode(ckpt)))
        return E.value, g

    def set_state_limit(self, nbytes: int | None):
        """Cap the state scratch a call may plan (qaoa_set_state_limit); None
        removes the cap."""
        self._check(self._lib.qaoa_set_state_limit(self._h, -1 if nbytes is None else int(nbytes)))

    def set_checkpointing(self, mode):
        """Checkpointing of batched gradients: "none", "round" or "pass" (default)."""
        self._check(self._lib.qaoa_set_checkpointing(self._h, _ckpt_mode(mode)))

    # ------------------------------------------------ pass-schedule tuning
    def autotune(self, cost: torch.Tensor, n: int, p: int = 2, want_grad: bool = True) -> dict:
        """Time every X-mixer pass schedule for (n, cost dtype) on this cost
        vector and keep the fastest in the context (qaoa_autotune_x)."""
        cost = _dev_tensor(cost, "cost")
        t = B.QaoaXTune()
        self._check(self._lib.qaoa_autotune_x(self._h, _ptr(cost), _cost_dtype(cost), n, p, 1 if want_grad else 0,
                                              ctypes.byref(t)))
        d = _xtune_dict(t)
        self._tuned[(d["n"], d["cost_dtype"])] = d
        return d

    def set_tuning(self, t: dict):
        """Install a schedule (e.g. one saved from autotune())."""
        st = B.QaoaXTune(*(int(t[k]) for k in ("n", "cost_dtype", "cmin", "split", "nbuf_bwd_contig",
                                               "nbuf_bwd_gather")), float(t.get("ms", 0.0)))
        self._check(self._lib.qaoa_set_xtune(self._h, ctypes.byref(st)))
        self._tuned[(int(t["n"]), int(t["cost_dtype"]))] = dict(t)

    def save_tuning(self, path: str) -> None:
        """Write every schedule this context tuned or was given to `path`
        (write_tuning_file), for a later run to load instead of re-tuning."""
        write_tuning_file(path, list(self._tuned.values()), torch.cuda.get_device_name(self.device))

    def load_tuning(self, path: str) -> int:
        """Install the schedules of a tuning file written on the same GPU model;
        returns how many.  A damaged, altered or foreign file raises
        ValueError and installs nothing."""
        ents = read_tuning_file(path, torch.cuda.get_device_name(self.device))
        for e in ents:
            self.set_tuning(e)
        return len(ents)

    def get_tuning(self, n: int, cost_dtype: int) -> dict:
        t = B.QaoaXTune()
        self._check(self._lib.qaoa_get_xtune(self._h, n, cost_dtype, ctypes.byref(t)))
        return _xtune_dict(t)

    def expectation_batched(self, jobs, want_grad: bool = False):
        """Enqueue many angle sets / instances (qaoa_expectation_batched).

        jobs: list of dicts with keys cost, mixer, angles (n_sets x 2p float64
        CUDA tensor), E (n_sets float64 CUDA tensor), grad (n_sets x 2p, when
        want_grad) and optionally init.  Asynchronous on the context stream."""
        self.batched_call(jobs, want_grad).run()

    def batched_call(self, jobs, want_grad: bool = False) -> "BatchedCall":
        """The same call with its job list marshalled once: run() re-issues it
        on the same tensors (new angles copied into them in place), which
        takes the per-call argument handling off small problems."""
        return BatchedCall(self, jobs, want_grad)

    def batched_call_host(self, jobs, want_grad: bool = False) -> "HostBatchedCall":
        """qaoa_expectation_batched_host prepared once: jobs as for
        batched_call, but angles, E and grad are host tensors (pinned ones give
        asynchronous copies).  run() copies the angles in, evaluates, copies
        <C> (and the gradients) back into the same host tensors and returns
        when they are there."""
        return HostBatchedCall(self, jobs, want_grad)

    def expectation_batched_host(self, jobs, want_grad: bool = False):
        """One synchronous host-buffer batched call (see batched_call_host)."""
        self.batched_call_host(jobs, want_grad).run()

    def _host_job_array(self, jobs, want_grad):
        arr = (B.QaoaHostJob * len(jobs))()
        keep = []
        for i, j in enumerate(jobs):
            ang = _host_tensor(j["angles"], "angles")
            E = _host_tensor(j["E"], "E")
            G = _host_tensor(j.get("grad"), "grad")
            cost = _dev_tensor(j["cost"], "cost")
            init = _dev_tensor(j.get("init"), "init")
            n_sets = ang.shape[0] if ang.dim() == 2 else 1
            mx = j["mixer"]
            na = ang.shape[-1]
            p = _rounds(mx, na)
            if E.numel() < n_sets or (want_grad and (G is None or G.numel() < n_sets * na)):
                raise ValueError("E (and grad) must hold a result per angle set")
            keep.append(mx)
            arr[i] = B.QaoaHostJob(cost.data_ptr(), _cost_dtype(cost), ctypes.pointer(mx.struct), p, n_sets,
                                   ang.data_ptr(), E.data_ptr(), None if G is None else G.data_ptr(),
                                   None if init is None else init.data_ptr())
            keep.extend([ang, E, G, cost, init])
        return arr, keep

    def _job_array(self, jobs):
        arr = (B.QaoaJob * len(jobs))()
        keep = []
        for i, j in enumerate(jobs):
            ang = _dev_tensor(j["angles"], "angles")
            E = _dev_tensor(j["E"], "E")
            G = _dev_tensor(j.get("grad"), "grad")
            cost = _dev_tensor(j["cost"], "cost")
            init = _dev_tensor(j.get("init"), "init")
            if ang.dtype != torch.float64 or E.dtype != torch.float64 or (G is not None and G.dtype != torch.float64):
                raise TypeError("angles, E and grad must be float64")
            n_sets = ang.shape[0] if ang.dim() == 2 else 1
            mx = j["mixer"]
            p = _rounds(mx, ang.shape[-1])
            keep.append(mx)
            arr[i] = B.QaoaJob(cost.data_ptr(), _cost_dtype(cost), ctypes.pointer(mx.struct), p, n_sets,
                               ang.data_ptr(), E.data_ptr(), None if G is None else G.data_ptr(),
                               None if init is None else init.data_ptr())
            keep.extend([ang, E, G, cost, init])
        return arr, keep

    def check_bounded_wait(self):
        """qaoa_check_bounded_wait: raises QAOAError with status
        QAOA_ERR_TIMEOUT when the device-side wait gave up as designed."""
        self._check(self._lib.qaoa_check_bounded_wait(self._h))

    # --------------------------------------------------------- measurement
    def set_profiling(self, on: bool = True):
        self._check(self._lib.qaoa_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self):
        """{family: {launches, total_ms, algo_bytes}} of the profiled launches."""
        n = self._lib.qaoa_kernel_stats(self._h, None, 0)
        arr = (B.QaoaKernelStat * max(n, 1))()
        n = self._lib.qaoa_kernel_stats(self._h, arr, n)
        return {arr[i].name.decode(): {"launches": arr[i].launches, "total_ms": arr[i].total_ms,
                                       "algo_bytes": arr[i].algo_bytes, "algo_flops": arr[i].algo_flops}
                for i in range(n)}

    def reset_stats(self):
        self._lib.qaoa_reset_stats(self._h)

    def launch_count(self) -> int:
        return int(self._lib.qaoa_launch_count(self._h))

    def scratch_bytes(self) -> int:
        return int(self._lib.qaoa_scratch_bytes(self._h))


class BatchedCall:
    """A qaoa_expectation_batched call prepared once (Context.batched_call):
    the job structs point at the given tensors, which it keeps alive; run()
    enqueues the call again.  Asynchronous on the context stream."""

    def __init__(self, ctx: Context, jobs, want_grad: bool = False):
        self._ctx = ctx
        self._arr, self._keep = ctx._job_array(jobs)
        self._n = len(jobs)
        self._grad = 1 if want_grad else 0

    def run(self):
        c = self._ctx
        c._check(c._lib.qaoa_expectation_batched(c._h, self._n, self._arr, self._grad))


class HostBatchedCall:
    """A qaoa_expectation_batched_host call prepared once
    (Context.batched_call_host): the job structs point at the given host and
    device tensors, which it keeps alive; run() copies the current contents of
    the angle tensors in and the results back, synchronously."""

    def __init__(self, ctx: Context, jobs, want_grad: bool = False):
        self._ctx = ctx
        self._grad = 1 if want_grad else 0
        self._arr, self._keep = ctx._host_job_array(jobs, want_grad)
        self._n = len(jobs)

    def run(self):
        c = self._ctx
        c._check(c._lib.qaoa_expectation_batched_host(c._h, self._n, self._arr, self._grad))


def _rounds(mixer, n_angles: int) -> int:
    """p from the length of one angle set."""
    if hasattr(mixer, "rounds"):
        return mixer.rounds(n_angles)
    return n_angles // 2


def _ckpt_mode(m) -> int:
    names = {"none": B.QAOA_CKPT_NONE, "round": B.QAOA_CKPT_ROUND, "pass": B.QAOA_CKPT_PASS}
    if isinstance(m, str):
        return names[m]
    if isinstance(m, bool):
        return B.QAOA_CKPT_ROUND if m else B.QAOA_CKPT_NONE
    return int(m)


def _xtune_dict(t) -> dict:
    return {k: getattr(t, k) for k in ("n", "cost_dtype", "cmin", "split", "nbuf_bwd_contig", "nbuf_bwd_gather",
                                       "ms")}


def pass_schedule(n: int, cmin: int = 4, split: int = 0):
    """[(c, lo), ...]: the X-mixer passes of one round (qaoa_pass_schedule;
    host only, needs no GPU)."""
    lib = B.load()
    c = (ctypes.c_int * 16)()
    lo = (ctypes.c_int * 16)()
    k = lib.qaoa_pass_schedule(n, cmin, split, c, lo, 16)
    if k < 0:
        raise ValueError(f"no schedule for n={n}, cmin={cmin}, split={split}")
    return [(c[j], lo[j]) for j in range(k)]


# Module-level aliases with the C names.
def qaoa_cost_precompute(ctx: Context, *args, **kw):
    return ctx.cost_precompute(*args, **kw)


def qaoa_expectation(ctx: Context, *args, **kw):
    return ctx.expectation(*args, **kw)


def qaoa_gradient(ctx: Context, *args, **kw):
    return ctx.gradient(*args, **kw)


def qaoa_expectation_batched(ctx: Context, *args, **kw):
    return ctx.expectation_batched(*args, **kw)


def qaoa_expectation_batched_host(ctx: Context, *args, **kw):
    return ctx.expectation_batched_host(*args, **kw)


def qaoa_gradient_small_noalloc(cost: torch.Tensor, n: int, angles: torch.Tensor, E: torch.Tensor,
                                grad: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None):
    """<C> (and the gradient) for n <= 12, p <= 96 through the C entry point
    that allocates no device memory (for callers that cannot allocate: the
    library keeps a fixed device array instead).  angles, E, grad: float64 CUDA
    tensors (2p, 1, 2p); results land in E and grad.  Synchronous."""
    n, p = _check_noalloc_args(cost, n, angles, E, grad)
    lib = B.load()
    with torch.cuda.device(cost.device):
        s = stream if stream is not None else torch.cuda.current_stream(cost.device)
        st = lib.qaoa_gradient_small_noalloc(_ptr(cost), _cost_dtype(cost), n, p, _ptr(angles), _ptr(E),
                                             _ptr(grad), ctypes.c_void_p(s.cuda_stream))
    if st != B.QAOA_OK:
        raise QAOAError(st, "qaoa_gradient_small_noalloc failed")


def _check_noalloc_args(cost, n, angles, E, grad):
    """Shapes, dtypes and devices of a qaoa_gradient_small_noalloc call,
    checked on the host before anything reaches the device: the C entry point
    trusts the sizes it is given, so a short or mistyped buffer here would
    turn into an out-of-bounds device access.  Returns (n, p)."""
    n = int(n)
    for name, t in (("cost", cost), ("angles", angles), ("E", E)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
    if grad is not None and not isinstance(grad, torch.Tensor):
        raise ValueError("grad must be a torch tensor or None")
    if cost.dtype not in (torch.uint8, torch.float32):
        raise ValueError(f"cost must be uint8 or float32, got {cost.dtype}")
    for name, t in (("angles", angles), ("E", E), ("grad", grad)):
        if t is not None and t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, got {t.dtype}")
    if not 1 <= n <= 62 or cost.numel() != 1 << n:
        raise ValueError(f"cost must hold 2^n = 2^{n} values, has {cost.numel()}")
    if angles.numel() < 2 or angles.numel() % 2:
        raise ValueError(f"angles must hold 2p values (p >= 1), has {angles.numel()}")
    if E.numel() < 1:
        raise ValueError("E must hold at least one value")
    if grad is not None and grad.numel() != angles.numel():
        raise ValueError(f"grad must hold {angles.numel()} values like angles, has {grad.numel()}")
    for name, t in (("cost", cost), ("angles", angles), ("E", E), ("grad", grad)):
        if t is not None and not (t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t is not None and t.device != cost.device:
            raise ValueError(f"{name} is on {t.device}, cost on {cost.device}")
    return n, angles.numel() // 2


class QAOAExpectation(torch.autograd.Function):
    """E = <C>(angles) with the adjoint gradient (Sec. 2.3).

    Usage: ``E = QAOAExpectation.apply(angles, ctx, cost, mixer)`` with angles a
    float64 tensor of length 2p.  When angles requires grad, the forward runs
    qaoa_gradient (one forward and one adjoint sweep) and keeps the gradient;
    backward returns grad_out * dE/dangles."""

    @staticmethod
    def forward(fctx, angles, qctx, cost, mixer, init=None, ckpt=True):
        a = angles.detach().to("cpu", torch.float64).contiguous().numpy()
        if angles.requires_grad:
            E, g = qctx.gradient(cost, mixer, a, init, ckpt)
            fctx.save_for_backward(torch.from_numpy(g).to(angles.device))
        else:
            E = qctx.expectation(cost, mixer, a, init)
            fctx.save_for_backward(torch.zeros_like(angles, dtype=torch.float64))
        return torch.tensor(E, dtype=torch.float64, device=angles.device)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return grad_out * g, None, None, None, None, None

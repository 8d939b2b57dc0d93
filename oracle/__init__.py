"""FP64 CPU oracle for the even-odd Wilson matrix (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package. The CUDA product path never calls
it; the two share no code.

The arithmetic lives in ``wilson_oracle.c`` (plain C99 complex FP64, optional
OpenMP over output sites); this module only compiles it with gcc and marshals
numpy ``complex128`` arrays in the canonical layouts:

* gauge ``U``: ``(4, V, 3, 3)``, lexicographic sites ``((t*Lz+z)*Ly+y)*Lx+x``;
* single-parity spinor: ``(V/2, 4, 3)`` or batched ``(nrhs, V/2, 4, 3)``,
  parity index ``lex // 2`` (compacted in x, Sec. 3.3 of the paper).

Every function cites the passage of arXiv:2303.08609 it follows; see the C
file's header for the readings of points the paper leaves open.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``wilson_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _bind(lib):
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    Lg = ctypes.c_long
    sig = {
        "oracle_gamma": (None, [I, P]),
        "oracle_hop": (None, [P, P, I, I, P, P]),
        "oracle_hop_adj": (None, [P, P, I, I, P, P]),
        "oracle_meo": (None, [P, P, D, P, P]),
        "oracle_meo_dag": (None, [P, P, D, P, P]),
        "oracle_meo_sign": (None, [P, P, D, I, P, P]),
        "oracle_meo_sites": (None, [P, P, D, I, P, Lg, P, P]),
        "oracle_link_grad": (None, [P, P, D, P, P, P]),
        "oracle_force": (None, [P, P, D, P, P, P]),
        "oracle_cg": (I, [P, P, D, P, P, D, I, P, P]),
        "oracle_set_threads": (None, [I]),
        "oracle_get_threads": (I, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


class use_library:
    """Context manager: route every oracle call through another build of
    ``wilson_oracle.c`` (the tests use it to check that planted mistakes are
    caught by the pins)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = _bind(ctypes.CDLL(_LIB))
    _lib = lib
    return lib


def _dims(dims) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    if d.shape != (4,) or np.any(d < 2) or np.any(d % 2):
        raise ValueError(f"lattice dims must be 4 even extents >= 2, got {dims}")
    return d


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _batched(fn, psi, *args):
    psi = _c128(psi)
    if psi.ndim == 4:
        return np.stack([fn(p, *args) for p in psi])
    return fn(psi, *args)


def set_threads(n: int) -> None:
    """OpenMP threads used by the site loops."""
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def gamma(mu: int) -> np.ndarray:
    """The oracle's 4x4 gamma_mu (mu = 0..3 for x, y, z, t), chiral basis."""
    out = np.zeros((4, 4), dtype=np.complex128)
    _load().oracle_gamma(int(mu), _ptr(out))
    return out


def hop(U, psi, dims, out_parity: int, sign: int = 1) -> np.ndarray:
    """Hopping term of Eq. 1 (without -kappa) onto sites of ``out_parity``.

    ``sign=+1``: (1 - gamma) forward / (1 + gamma) backward, as in Eq. 1;
    ``sign=-1``: the projectors swapped (the pairing drawn in Fig. 2).
    """
    d, U = _dims(dims), _c128(U)

    def one(p):
        out = np.empty_like(p)
        _load().oracle_hop(_ptr(d), _ptr(U), int(sign), int(out_parity), _ptr(out), _ptr(p))
        return out

    return _batched(one, psi)


def hop_adj(U, psi, dims, out_parity: int, sign: int = 1) -> np.ndarray:
    """Adjoint of the hopping term, built from the conjugate-transposed blocks."""
    d, U = _dims(dims), _c128(U)

    def one(p):
        out = np.empty_like(p)
        _load().oracle_hop_adj(_ptr(d), _ptr(U), int(sign), int(out_parity), _ptr(out), _ptr(p))
        return out

    return _batched(one, psi)


def meo(U, kappa: float, psi, dims) -> np.ndarray:
    """M_eo psi = psi - kappa^2 H_eo H_oe psi (Eq. 4, Wilson: D_ee = D_oo = 1)."""
    d, U = _dims(dims), _c128(U)

    def one(p):
        out = np.empty_like(p)
        _load().oracle_meo(_ptr(d), _ptr(U), float(kappa), _ptr(out), _ptr(p))
        return out

    return _batched(one, psi)


def meo_dag(U, kappa: float, psi, dims) -> np.ndarray:
    """M_eo^dag psi, from the explicit adjoint of every hopping block."""
    d, U = _dims(dims), _c128(U)

    def one(p):
        out = np.empty_like(p)
        _load().oracle_meo_dag(_ptr(d), _ptr(U), float(kappa), _ptr(out), _ptr(p))
        return out

    return _batched(one, psi)


def meo_sign(U, kappa: float, psi, dims, sign: int) -> np.ndarray:
    """M_eo built with projector sign ``sign`` (see :func:`hop`)."""
    d, U = _dims(dims), _c128(U)

    def one(p):
        out = np.empty_like(p)
        _load().oracle_meo_sign(_ptr(d), _ptr(U), float(kappa), int(sign), _ptr(out), _ptr(p))
        return out

    return _batched(one, psi)


def meo_sites(U, kappa: float, psi, dims, sites, dag: bool = False) -> np.ndarray:
    """(M_eo psi) or (M_eo^dag psi) at the listed even parity indices only.

    Returns ``(len(sites), 4, 3)``. Cost is independent of the lattice volume,
    so it checks full-size outputs site by site.
    """
    d, U, p = _dims(dims), _c128(U), _c128(psi)
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.empty((len(s), 4, 3), dtype=np.complex128)
    _load().oracle_meo_sites(_ptr(d), _ptr(U), float(kappa), int(bool(dag)), _ptr(p),
                             ctypes.c_long(len(s)), _ptr(s), _ptr(out))
    return out


def link_grad(U, kappa: float, g, phi, dims) -> np.ndarray:
    """Gradient of Re<g, M_eo phi> with respect to every link, ``(4, V, 3, 3)``.

    Convention of a real loss of complex inputs: G = dL/dRe U + i dL/dIm U.
    """
    d, U, g, phi = _dims(dims), _c128(U), _c128(g), _c128(phi)
    G = np.empty_like(U)
    _load().oracle_link_grad(_ptr(d), _ptr(U), float(kappa), _ptr(g), _ptr(phi), _ptr(G))
    return G


def force(U, kappa: float, phi, dims):
    """Force of S = |M_eo phi|^2: ``(F, dS/dphi)``.

    ``F[mu, x]`` is the traceless anti-Hermitian matrix with
    dS/d eps = Re tr(X^dag F) under U_mu(x) -> exp(eps X) U_mu(x);
    ``dS/dphi = 2 M^dag M phi``.
    """
    d, U, phi = _dims(dims), _c128(U), _c128(phi)
    F = np.empty_like(U)
    dphi = np.empty_like(phi)
    _load().oracle_force(_ptr(d), _ptr(U), float(kappa), _ptr(phi), _ptr(F), _ptr(dphi))
    return F, dphi


def cg(U, kappa: float, b, dims, tol: float = 1e-10, maxiter: int = 10000, x0=None):
    """CG on M_eo^dag M_eo x = b in FP64. Returns ``(x, iters, true_relres, converged)``."""
    d, U, b = _dims(dims), _c128(U), _c128(b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = _load().oracle_cg(_ptr(d), _ptr(U), float(kappa), _ptr(b), _ptr(x), float(tol),
                           int(maxiter), ctypes.byref(it), ctypes.byref(rr))
    if rc < 0:
        raise MemoryError("oracle_cg: out of memory")
    return x, int(it.value), float(rr.value), rc == 0

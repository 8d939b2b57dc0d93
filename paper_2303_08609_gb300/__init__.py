"""Even-odd Wilson fermion matrix on GB300 -- Python binding of ``libwilson_eo.so``.

The C ABI (``include/wilson_eo.h``) is the product; this module only marshals
arguments to it through ``ctypes``: torch tensors (CUDA or CPU) and numpy
arrays are passed as raw pointers, torch's current CUDA stream is passed as the
stream. Every step of the computation runs in the library's CUDA kernels. If
the library is missing, every call raises: there is no CPU fallback.

Function names match the C ABI (``wilson_eo_create``, ``wilson_eo_apply`` ...);
:class:`WilsonEO` wraps a handle for convenience.

Canonical layouts (see the header for details):

* gauge ``(4, V, 3, 3)`` complex128 or complex64, sites lexicographic
  ``((t*Lz+z)*Ly+y)*Lx+x``;
* even/odd spinors, planar: ``(nrhs, 4, 3, V/2)`` complex128 (FP64 handles) or
  complex64 (FP32 / FP16 / BF16 handles), site index ``lex // 2``.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwilson_eo.so")

WEO_OK = 0
STATUS = {
    0: "WEO_OK", -1: "WEO_ERR_ARG", -2: "WEO_ERR_DIMS", -3: "WEO_ERR_UNSUPPORTED",
    -4: "WEO_ERR_CUDA", -5: "WEO_ERR_NOT_CONVERGED", -6: "WEO_ERR_NONFINITE",
    -7: "WEO_ERR_TIMEOUT", -8: "WEO_ERR_OOM",
}
PREC = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
LINKFMT = {18: 0, 12: 1}

_lib = None


class WilsonEOError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2303_08609_gb300.build` "
            "(nvcc for sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, LL, SZ = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                       ctypes.c_size_t)
    IP = ctypes.POINTER(ctypes.c_int)
    sig = {
        "wilson_eo_create": (I, [ctypes.POINTER(P), IP, D, I, I, P, I, P]),
        "wilson_eo_set_gauge": (I, [P, P, I, P]),
        "wilson_eo_set_kappa": (I, [P, D]),
        "wilson_eo_info": (I, [P, IP, ctypes.POINTER(LL), IP, IP, ctypes.POINTER(D),
                               ctypes.POINTER(SZ)]),
        "wilson_eo_apply": (I, [P, P, P, I, P]),
        "wilson_eo_apply_dag": (I, [P, P, P, I, P]),
        "wilson_eo_hop": (I, [P, I, I, P, P, I, P]),
        "wilson_eo_set_launch": (I, [P, I, I, I]),
        "wilson_eo_profile": (I, [P, I]),
        "wilson_eo_profile_read": (I, [P, I, ctypes.c_char_p, I, ctypes.POINTER(D),
                                       ctypes.POINTER(LL), IP, I]),
        "wilson_eo_destroy": (None, [P]),
        "wilson_eo_strerror": (ctypes.c_char_p, [I]),
        "wilson_eo_last_error": (ctypes.c_char_p, []),
    }
    optional = {
        "wilson_eo_force": (I, [P, P, P, P, P]),
        "wilson_eo_link_grad": (I, [P, P, P, P, P]),
        "wilson_eo_solve": (I, [P, P, P, D, I, I, IP, ctypes.POINTER(D), P]),
        "wilson_eo_solver_config": (I, [P, D, I, I]),
        "wilson_eo_solve_multi": (I, [P, P, P, I, D, I, I, IP, ctypes.POINTER(D), P]),
        "wilson_eo_prepare_source": (I, [P, P, P, P, P]),
        "wilson_eo_reconstruct": (I, [P, P, P, P, P]),
        "wilson_eo_solve_full": (I, [P, P, P, P, P, D, I, I, IP, ctypes.POINTER(D), P]),
        "wilson_eo_solve_stats": (I, [P, IP, IP, IP, IP, ctypes.POINTER(D)]),
        "wilson_eo_solver_residual": (I, [P, I]),
        "wilson_eo_solver_restart": (I, [P, I]),
        "wilson_eo_l2_peak": (I, [ctypes.POINTER(D), P]),
        "wilson_eo_set_tile_links": (I, [P, I, I]),
        "wilson_eo_set_site_blocks": (I, [P, I]),
        "wilson_eo_get_tile_links": (I, [P, P, P]),
        "wilson_eo_spinor_layout": (I, [ctypes.c_longlong, I, I, I, P, P, P]),
        "wilson_eo_apply_ff64": (I, [P, P, P, I, I, P]),
        "wilson_eo_apply_batch": (I, [I, ctypes.POINTER(P), ctypes.POINTER(P),
                                      ctypes.POINTER(P), I, P]),
        "wilson_eo_apply_batch_rhs": (I, [I, ctypes.POINTER(P), ctypes.POINTER(P),
                                          ctypes.POINTER(P), IP, I, P]),
        "wilson_eo_tune": (I, [P, I, IP, IP, ctypes.POINTER(D), P]),
        "wilson_eo_get_launch": (I, [P, IP, IP, IP]),
        "wilson_eo_set_algorithm": (I, [P, I, I, I]),
        "wilson_eo_check": (I, [P, P]),
        "wilson_eo_hop_split": (I, [P, I, I, I, P, P, P]),
        "wilson_eo_inject_fused_timeout": (I, [P, P, P, P]),
        "wilson_eo_set_staging": (I, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "wilson_eo_get_staging": (I, [P, IP, IP, IP]),
        "wilson_eo_inject_staged_timeout": (I, [P, P, P, P]),
        "wilson_eo_get_algorithm": (I, [P, IP, IP, IP]),
        "wilson_eo_apply_noalloc": (I, [IP, D, P, P, P, I, P]),
        "wilson_eo_alu_peak": (I, [I, ctypes.POINTER(D), P]),
        "wilson_eo_set_rhs_lanes": (I, [P, I]),
    }
    for name, (res, args) in list(sig.items()) + list(optional.items()):
        f = getattr(lib, name, None)
        if f is None:
            if name in sig:
                raise RuntimeError(f"{LIB_PATH} does not export {name}")
            continue
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def library():
    """The loaded ``ctypes.CDLL`` (raises if the library was not built)."""
    return _load()


def _check(status: int, where: str):
    if status != WEO_OK:
        msg = _load().wilson_eo_last_error().decode(errors="replace")
        raise WilsonEOError(status, where, msg)


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError(f"cannot pass {type(a)} to the C ABI")


def _nbytes(a):
    if isinstance(a, np.ndarray):
        return a.nbytes
    if hasattr(a, "element_size"):
        return a.numel() * a.element_size()
    return None


def _dtype_name(a):
    return str(getattr(a, "dtype", "")).replace("torch.", "")


def _expect(h, arrays, nrhs=1, kind="spinor", where=""):
    """Refuse arrays whose dtype or size does not match what the library will
    read or write for handle ``h`` -- the C ABI cannot check sizes itself.
    kind: "spinor" (handle's spinor dtype), "spinor64" (complex128 spinors),
    "gauge" (handle's spinor dtype, 4*V*9 complex)."""
    info = wilson_eo_info(h)
    vh = info["half_volume"]
    f64 = info["prec"] == PREC["f64"] or kind == "spinor64"
    want_dtype = "complex128" if f64 else "complex64"
    elt = 16 if f64 else 8
    need = (4 * 2 * vh * 9 * elt) if kind == "gauge" else 12 * vh * nrhs * elt
    for a in arrays:
        if a is None or isinstance(a, int):
            continue
        dt = _dtype_name(a)
        if dt and dt != want_dtype:
            raise TypeError(f"{where}: expected {want_dtype} arrays for this handle, got {dt}")
        nb = _nbytes(a)
        if nb is not None and nb < need:
            raise ValueError(f"{where}: array of {nb} bytes, the call touches {need}")


def _stream(stream):
    """cudaStream_t of ``stream``: a torch.cuda.Stream, an int handle, or None
    for torch's current stream (the legacy default stream without torch CUDA)."""
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------- C ABI, by name --


def wilson_eo_create(dims, kappa, prec, linkfmt, gauge, gauge_is_f64=None, stream=None):
    """Create a handle; ``prec`` in PREC names or ints, ``linkfmt`` 18/12 or 0/1."""
    lib = _load()
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    f = {18: 0, 12: 1, 0: 0, 1: 1}[int(linkfmt)]
    if gauge_is_f64 is None:
        gauge_is_f64 = _is_f64(gauge)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    h = ctypes.c_void_p()
    _check(lib.wilson_eo_create(ctypes.byref(h), d, float(kappa), p, f, _ptr(gauge),
                                int(bool(gauge_is_f64)), _stream(stream)), "wilson_eo_create")
    return h


def wilson_eo_set_gauge(h, gauge, gauge_is_f64=None, stream=None):
    if gauge_is_f64 is None:
        gauge_is_f64 = _is_f64(gauge)
    _check(_load().wilson_eo_set_gauge(h, _ptr(gauge), int(bool(gauge_is_f64)), _stream(stream)),
           "wilson_eo_set_gauge")


def wilson_eo_set_kappa(h, kappa):
    _check(_load().wilson_eo_set_kappa(h, float(kappa)), "wilson_eo_set_kappa")


def wilson_eo_info(h):
    d = (ctypes.c_int * 4)()
    vh = ctypes.c_longlong()
    p = ctypes.c_int()
    f = ctypes.c_int()
    k = ctypes.c_double()
    b = ctypes.c_size_t()
    _check(_load().wilson_eo_info(h, d, ctypes.byref(vh), ctypes.byref(p), ctypes.byref(f),
                                  ctypes.byref(k), ctypes.byref(b)), "wilson_eo_info")
    return {"dims": tuple(d), "half_volume": vh.value, "prec": p.value, "linkfmt": f.value,
            "kappa": k.value, "device_bytes": b.value}


def wilson_eo_apply(h, out_e, in_e, nrhs=1, stream=None):
    _expect(h, (out_e, in_e), nrhs, where="wilson_eo_apply")
    _check(_load().wilson_eo_apply(h, _ptr(out_e), _ptr(in_e), int(nrhs), _stream(stream)),
           "wilson_eo_apply")


def wilson_eo_apply_dag(h, out_e, in_e, nrhs=1, stream=None):
    _expect(h, (out_e, in_e), nrhs, where="wilson_eo_apply_dag")
    _check(_load().wilson_eo_apply_dag(h, _ptr(out_e), _ptr(in_e), int(nrhs), _stream(stream)),
           "wilson_eo_apply_dag")


def wilson_eo_hop(h, out_parity, dag, out, inp, nrhs=1, stream=None):
    _expect(h, (out, inp), nrhs, where="wilson_eo_hop")
    _check(_load().wilson_eo_hop(h, int(out_parity), int(bool(dag)), _ptr(out), _ptr(inp),
                                 int(nrhs), _stream(stream)), "wilson_eo_hop")


def wilson_eo_set_launch(h, threads, rhs_block=1, order=1):
    _check(_load().wilson_eo_set_launch(h, int(threads), int(rhs_block), int(order)),
           "wilson_eo_set_launch")


def wilson_eo_profile(h, enable=True):
    _check(_load().wilson_eo_profile(h, int(bool(enable))), "wilson_eo_profile")


def wilson_eo_profile_read(h, reset=True, max_kernels=64):
    """{kernel label: (total_ms, launches)} since the last reset."""
    name_len = 96
    names = ctypes.create_string_buffer(max_kernels * name_len)
    ms = (ctypes.c_double * max_kernels)()
    cnt = (ctypes.c_longlong * max_kernels)()
    n = ctypes.c_int()
    _check(_load().wilson_eo_profile_read(h, max_kernels, names, name_len, ms, cnt,
                                          ctypes.byref(n), int(bool(reset))),
           "wilson_eo_profile_read")
    out = {}
    for k in range(n.value):
        label = names.raw[k * name_len:(k + 1) * name_len].split(b"\0", 1)[0].decode()
        out[label] = (ms[k], cnt[k])
    return out


def wilson_eo_link_grad(h, grad, g_e, phi_e, stream=None):
    _expect(h, (g_e, phi_e), 1, where="wilson_eo_link_grad")
    _expect(h, (grad,), kind="gauge", where="wilson_eo_link_grad")
    _check(_load().wilson_eo_link_grad(h, _ptr(grad), _ptr(g_e), _ptr(phi_e), _stream(stream)),
           "wilson_eo_link_grad")


def wilson_eo_force(h, force, dS_dphi_e, phi_e, stream=None):
    _expect(h, (dS_dphi_e, phi_e), 1, where="wilson_eo_force")
    _expect(h, (force,), kind="gauge", where="wilson_eo_force")
    _check(_load().wilson_eo_force(h, _ptr(force), _ptr(dS_dphi_e), _ptr(phi_e), _stream(stream)),
           "wilson_eo_force")


def _noalloc_device(arrays):
    """CUDA device index shared by the torch tensors among ``arrays`` (None if
    there are none). Tensors that are not on a CUDA device, or on different
    devices, are refused here, before the library is called."""
    devs = set()
    for a in arrays:
        if not hasattr(a, "data_ptr") or not hasattr(a, "is_cuda"):
            continue  # numpy arrays and raw pointers: the library checks those
        d = a.device
        if d.type != "cuda":
            raise ValueError(f"wilson_eo_apply_noalloc takes CUDA device arrays only, got {d}")
        devs.add(d.index)
    if len(devs) > 1:
        raise ValueError(f"wilson_eo_apply_noalloc: arrays on different devices {sorted(devs)}")
    return devs.pop() if devs else None


def wilson_eo_apply_noalloc(dims, kappa, gauge, out_e, in_e, dag=False, stream=None):
    """FP32 M_eo (or M_eo^dag) on caller-owned device arrays; the library
    allocates nothing for it (see the header for the scratch-array rules).
    The call runs with the arrays' device current."""
    dev = _noalloc_device((gauge, out_e, in_e))
    V = int(np.prod([int(x) for x in dims]))
    for a, need, what in ((gauge, 4 * V * 9 * 8, "gauge"), (out_e, 6 * V * 8, "out_e"),
                          (in_e, 6 * V * 8, "in_e")):
        dt = _dtype_name(a)
        if dt and dt != "complex64":
            raise TypeError(f"wilson_eo_apply_noalloc: {what} must be complex64, got {dt}")
        nb = _nbytes(a)
        valid_dims = all(int(x) >= 2 and int(x) % 2 == 0 for x in dims)
        if nb is not None and nb < need and valid_dims and V // 2 <= 349525:
            raise ValueError(f"wilson_eo_apply_noalloc: {what} has {nb} bytes, needs {need}")
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])

    def call():
        return _load().wilson_eo_apply_noalloc(d, float(kappa), _ptr(gauge), _ptr(out_e),
                                               _ptr(in_e), int(bool(dag)), _stream(stream))

    if dev is None:
        st = call()
    else:
        import torch

        with torch.cuda.device(dev):
            st = call()
    _check(st, "wilson_eo_apply_noalloc")


def wilson_eo_set_rhs_lanes(h, lanes):
    """Right-hand sides of a multi-RHS apply on ``lanes`` neighbouring threads per
    site (1, 2, 4 or 8), sharing each link load."""
    _check(_load().wilson_eo_set_rhs_lanes(h, int(lanes)), "wilson_eo_set_rhs_lanes")


def wilson_eo_alu_peak(prec="f64", stream=None):
    """Measured FMA peak of the current GPU in flop/s, for prec "f64" or "f32"."""
    out = ctypes.c_double(0.0)
    _check(_load().wilson_eo_alu_peak(PREC.get(prec, -1), ctypes.byref(out), _stream(stream)),
           "wilson_eo_alu_peak")
    return out.value


def wilson_eo_l2_peak(stream=None):
    """Measured L2 -> SM read bandwidth of the current GPU in bytes/s."""
    out = ctypes.c_double(0.0)
    _check(_load().wilson_eo_l2_peak(ctypes.byref(out), _stream(stream)), "wilson_eo_l2_peak")
    return out.value


def wilson_eo_solve(h, x_e, b_e, tol=1e-10, maxiter=10000, mixed=True, stream=None,
                    raise_on_error=True):
    """Solve M^dag M x = b in place on ``x_e`` (complex128). Returns
    ``(status, iterations, true_relres)``."""
    _expect(h, (x_e, b_e), 1, kind="spinor64", where="wilson_eo_solve")
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = _load().wilson_eo_solve(h, _ptr(x_e), _ptr(b_e), float(tol), int(maxiter),
                                 int(bool(mixed)), ctypes.byref(it), ctypes.byref(rr),
                                 _stream(stream))
    if raise_on_error and st not in (WEO_OK, -5):
        _check(st, "wilson_eo_solve")
    return st, it.value, rr.value


def wilson_eo_prepare_source(h, rhs_e, eta_e, eta_o, stream=None):
    _expect(h, (rhs_e, eta_e, eta_o), 1, where="wilson_eo_prepare_source")
    _check(_load().wilson_eo_prepare_source(h, _ptr(rhs_e), _ptr(eta_e), _ptr(eta_o),
                                            _stream(stream)), "wilson_eo_prepare_source")


def wilson_eo_reconstruct(h, xi_o, eta_o, xi_e, stream=None):
    _expect(h, (xi_o, eta_o, xi_e), 1, where="wilson_eo_reconstruct")
    _check(_load().wilson_eo_reconstruct(h, _ptr(xi_o), _ptr(eta_o), _ptr(xi_e), _stream(stream)),
           "wilson_eo_reconstruct")


def wilson_eo_solve_full(h, xi_e, xi_o, eta_e, eta_o, tol=1e-10, maxiter=10000, mixed=True,
                         stream=None, raise_on_error=True):
    """D_W xi = eta (complex128 planar even/odd parts); xi_e holds the guess.
    Returns (status, iterations, even-system relres)."""
    _expect(h, (xi_e, xi_o, eta_e, eta_o), 1, kind="spinor64", where="wilson_eo_solve_full")
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = _load().wilson_eo_solve_full(h, _ptr(xi_e), _ptr(xi_o), _ptr(eta_e), _ptr(eta_o),
                                      float(tol), int(maxiter), int(bool(mixed)), ctypes.byref(it),
                                      ctypes.byref(rr), _stream(stream))
    if raise_on_error and st not in (WEO_OK, -5):
        _check(st, "wilson_eo_solve_full")
    return st, it.value, rr.value


def wilson_eo_solve_multi(h, x_e, b_e, nrhs, tol=1e-10, maxiter=10000, mixed=True, stream=None,
                          raise_on_error=True):
    """Solve nrhs systems M^dag M x_r = b_r in lockstep (complex128 planar, in place
    on ``x_e``). Returns ``(status, iterations[nrhs], true_relres[nrhs])``."""
    _expect(h, (x_e, b_e), nrhs, kind="spinor64", where="wilson_eo_solve_multi")
    it = (ctypes.c_int * nrhs)()
    rr = (ctypes.c_double * nrhs)()
    st = _load().wilson_eo_solve_multi(h, _ptr(x_e), _ptr(b_e), int(nrhs), float(tol), int(maxiter),
                                       int(bool(mixed)), it, rr, _stream(stream))
    if raise_on_error and st not in (WEO_OK, -5):
        _check(st, "wilson_eo_solve_multi")
    return st, list(it), list(rr)


def wilson_eo_solver_config(h, delta=-1.0, chunk=0, use_graphs=-1):
    _check(_load().wilson_eo_solver_config(h, float(delta), int(chunk), int(use_graphs)),
           "wilson_eo_solver_config")


def wilson_eo_solve_stats(h):
    it, ru, hi, fa = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    sec = ctypes.c_double()
    _check(_load().wilson_eo_solve_stats(h, ctypes.byref(it), ctypes.byref(ru), ctypes.byref(hi),
                                         ctypes.byref(fa), ctypes.byref(sec)), "wilson_eo_solve_stats")
    return {"iterations": it.value, "reliable_updates": ru.value, "fp64_applies": hi.value,
            "ff_applies": fa.value, "seconds": sec.value}


def wilson_eo_solver_residual(h, mode):
    """True residuals of reliable updates: 1 float-float (FP64 confirms
    convergence), 0 native FP64."""
    _check(_load().wilson_eo_solver_residual(h, int(mode)), "wilson_eo_solver_residual")


def wilson_eo_set_site_blocks(h, blocked=True):
    """One-site-per-thread hops: CTAs take 2x2x2 blocks of rows in (y, z, t)."""
    _check(_load().wilson_eo_set_site_blocks(h, int(bool(blocked))), "wilson_eo_set_site_blocks")


def wilson_eo_set_tile_links(h, groups, rhs_per_thread=1):
    """Multi-RHS hops over tiles whose links sit in shared memory: ``groups``
    (2, 4, 8) thread groups per tile, each taking ``rhs_per_thread`` (1, 2)
    right-hand sides per pass; groups = 0 turns it off."""
    _check(_load().wilson_eo_set_tile_links(h, int(groups), int(rhs_per_thread)),
           "wilson_eo_set_tile_links")


def wilson_eo_get_tile_links(h):
    """(groups, rhs_per_thread) of the handle's tile-shared-link hops."""
    n, r = ctypes.c_int(0), ctypes.c_int(0)
    _check(_load().wilson_eo_get_tile_links(h, ctypes.byref(n), ctypes.byref(r)),
           "wilson_eo_get_tile_links")
    return n.value, r.value


def wilson_eo_spinor_layout(dst, src, to_planar=True, stream=None):
    """Reorder device spinors between site-major (..., V/2, 4, 3) and planar
    (..., 4, 3, V/2): ``to_planar`` reads site-major ``src`` into planar ``dst``,
    otherwise the reverse. Both complex64 or both complex128, same size."""
    shape = tuple(src.shape)
    if len(shape) < 3:
        raise ValueError("spinor arrays need at least 3 dimensions")
    if to_planar and shape[-2:] != (4, 3):
        raise ValueError(f"site-major src must end in (4, 3), got {shape}")
    if not to_planar and shape[-3:-1] != (4, 3):
        raise ValueError(f"planar src must end in (4, 3, V/2), got {shape}")
    vh = shape[-3] if to_planar else shape[-1]
    nrhs = int(np.prod(shape[:-3])) if len(shape) > 3 else 1
    dt = _dtype_name(src)
    if dt not in ("complex64", "complex128") or _dtype_name(dst) != dt:
        raise TypeError(f"wilson_eo_spinor_layout: complex64 or complex128 arrays of one dtype, "
                        f"got {dt} and {_dtype_name(dst)}")
    if _nbytes(dst) != _nbytes(src):
        raise ValueError("wilson_eo_spinor_layout: dst and src differ in size")
    elem = 8 if dt == "complex64" else 16
    _check(_load().wilson_eo_spinor_layout(int(vh), int(nrhs), elem, int(bool(to_planar)), _ptr(dst),
                                           _ptr(src), _stream(stream)),
           "wilson_eo_spinor_layout")


def wilson_eo_solver_restart(h, restart):
    """Mixed solver, search direction at a reliable update: 1 restart (defect
    correction), 0 keep, 2 (default) restart for BF16 inner operators only."""
    _check(_load().wilson_eo_solver_restart(h, int(restart)), "wilson_eo_solver_restart")


def wilson_eo_apply_ff64(h, out_e, in_e, nrhs=1, dag=False, stream=None):
    """M_eo (or M_eo^dag) in float-float arithmetic on complex128 spinors."""
    _expect(h, (out_e, in_e), nrhs, kind="spinor64", where="wilson_eo_apply_ff64")
    _check(_load().wilson_eo_apply_ff64(h, _ptr(out_e), _ptr(in_e), int(nrhs), int(bool(dag)),
                                        _stream(stream)), "wilson_eo_apply_ff64")


def wilson_eo_apply_batch(handles, outs, ins, dag=False, stream=None):
    """M_eo (or M_eo^dag) on several lattices in one persistent launch."""
    n = len(handles)
    if not (len(outs) == len(ins) == n):
        raise ValueError("handles, outs and ins must have the same length")
    for h, o, i in zip(handles, outs, ins):
        _expect(h, (o, i), 1, where="wilson_eo_apply_batch")
    P = ctypes.c_void_p
    hs = (P * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    os_ = (P * n)(*[_ptr(o).value for o in outs])
    is_ = (P * n)(*[_ptr(i).value for i in ins])
    _check(_load().wilson_eo_apply_batch(n, hs, os_, is_, int(bool(dag)), _stream(stream)),
           "wilson_eo_apply_batch")


def wilson_eo_apply_batch_rhs(handles, outs, ins, nrhs, dag=False, stream=None):
    """Several lattices with nrhs[k] right-hand sides each, in one persistent launch."""
    n = len(handles)
    if not (len(outs) == len(ins) == len(nrhs) == n):
        raise ValueError("handles, outs, ins and nrhs must have the same length")
    for h, o, i, r in zip(handles, outs, ins, nrhs):
        _expect(h, (o, i), int(r), where="wilson_eo_apply_batch_rhs")
    P = ctypes.c_void_p
    hs = (P * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    os_ = (P * n)(*[_ptr(o).value for o in outs])
    is_ = (P * n)(*[_ptr(i).value for i in ins])
    rs = (ctypes.c_int * n)(*[int(r) for r in nrhs])
    _check(_load().wilson_eo_apply_batch_rhs(n, hs, os_, is_, rs, int(bool(dag)), _stream(stream)),
           "wilson_eo_apply_batch_rhs")


def wilson_eo_tune(h, nrhs=1, stream=None):
    """Autotune; returns (threads, rhs_block, ms per M_eo)."""
    t, r = ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check(_load().wilson_eo_tune(h, int(nrhs), ctypes.byref(t), ctypes.byref(r), ctypes.byref(ms),
                                  _stream(stream)), "wilson_eo_tune")
    return t.value, r.value, ms.value


def wilson_eo_set_algorithm(h, algo, lookahead=0, threads=0):
    """algo 0: two hop launches; 1: fused single launch, the first hop running
    ``lookahead`` t-slices ahead of the second; 2 ("fused_staged"): the same
    wavefront through the TMA-staged pipeline (FP32 18-real handles)."""
    a = {"two_pass": 0, "fused": 1, "fused_staged": 2}.get(algo, algo)
    _check(_load().wilson_eo_set_algorithm(h, int(a), int(lookahead), int(threads)),
           "wilson_eo_set_algorithm")


def wilson_eo_get_algorithm(h):
    a, r, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_load().wilson_eo_get_algorithm(h, ctypes.byref(a), ctypes.byref(r), ctypes.byref(t)),
           "wilson_eo_get_algorithm")
    return {"algo": a.value, "lookahead": r.value, "threads": t.value}


def wilson_eo_hop_split(h, ranks, out_parity, dag, out, inp, stream=None):
    """Hopping term with the lattice split along t into `ranks` sub-domains and
    every crossing hop exchanged through face buffers (forced self-exchange)."""
    _expect(h, (out, inp), 1, where="wilson_eo_hop_split")
    _check(_load().wilson_eo_hop_split(h, int(ranks), int(out_parity), int(bool(dag)), _ptr(out),
                                       _ptr(inp), _stream(stream)), "wilson_eo_hop_split")


def wilson_eo_inject_fused_timeout(h, out_e, in_e, stream=None):
    _expect(h, (out_e, in_e), 1, where="wilson_eo_inject_fused_timeout")
    _check(_load().wilson_eo_inject_fused_timeout(h, _ptr(out_e), _ptr(in_e), _stream(stream)),
           "wilson_eo_inject_fused_timeout")


def wilson_eo_set_staging(h, staged=True, rows=0, depth=0):
    """Hops of FP32 18-real operators fed by TMA through a shared-memory ring
    (True or 1: single-RHS hops; 2: multi-RHS hops too) or the default
    one-site-per-thread kernel (False); rows per tile and ring depth, 0 for
    automatic."""
    _check(_load().wilson_eo_set_staging(h, int(staged), int(rows), int(depth)),
           "wilson_eo_set_staging")


def wilson_eo_get_staging(h):
    """{"staged": bool, "rows": R, "depth": stages} (rows = depth = 0 when the
    lattice cannot use the staged hop)."""
    v, r, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_load().wilson_eo_get_staging(h, ctypes.byref(v), ctypes.byref(r), ctypes.byref(d)),
           "wilson_eo_get_staging")
    return {"staged": v.value, "rows": r.value, "depth": d.value}


def wilson_eo_inject_staged_timeout(h, out_o, in_e, stream=None):
    _expect(h, (out_o, in_e), 1, where="wilson_eo_inject_staged_timeout")
    _check(_load().wilson_eo_inject_staged_timeout(h, _ptr(out_o), _ptr(in_e), _stream(stream)),
           "wilson_eo_inject_staged_timeout")


def wilson_eo_check(h, stream=None):
    _check(_load().wilson_eo_check(h, _stream(stream)), "wilson_eo_check")


def wilson_eo_get_launch(h):
    """(threads per CTA, right-hand sides per thread, right-hand-side lanes)."""
    t, r, l = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_load().wilson_eo_get_launch(h, ctypes.byref(t), ctypes.byref(r), ctypes.byref(l)),
           "wilson_eo_get_launch")
    return t.value, r.value, l.value


def wilson_eo_destroy(h):
    if h:
        _load().wilson_eo_destroy(h)


def wilson_eo_strerror(status):
    return _load().wilson_eo_strerror(int(status)).decode()


def wilson_eo_last_error():
    return _load().wilson_eo_last_error().decode(errors="replace")


def _is_f64(a) -> bool:
    dt = getattr(a, "dtype", None)
    s = str(dt)
    return "complex128" in s or "float64" in s


# ------------------------------------------------------------ convenience --


class WilsonEO:
    """One lattice: gauge field, kappa, storage precision and link format.

    ``gauge``: canonical ``(4, V, 3, 3)`` complex tensor/array (device or host).
    Spinor arguments are planar ``(nrhs, 4, 3, V/2)`` or ``(4, 3, V/2)`` tensors.
    """

    def __init__(self, dims, kappa, gauge, prec="f32", linkfmt=18, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.kappa = float(kappa)
        self.prec = prec
        self.linkfmt = linkfmt
        self.vh = int(np.prod(self.dims)) // 2
        self._h = wilson_eo_create(self.dims, kappa, prec, linkfmt, gauge, stream=stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            wilson_eo_destroy(self._h)
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

    def spinor_dtype(self):
        import torch

        return torch.complex128 if self.prec == "f64" else torch.complex64

    def _nrhs(self, psi):
        if tuple(psi.shape[-3:]) != (4, 3, self.vh):
            raise ValueError(f"spinor shape must end in (4, 3, {self.vh}), got {tuple(psi.shape)}")
        return 1 if psi.dim() == 3 else int(np.prod(psi.shape[:-3]))

    def apply(self, psi, dag=False, out=None, stream=None):
        """M_eo psi (or M_eo^dag psi)."""
        import torch

        nrhs = self._nrhs(psi)
        out = torch.empty_like(psi) if out is None else out
        (wilson_eo_apply_dag if dag else wilson_eo_apply)(self._h, out, psi, nrhs, stream)
        return out

    def apply_ff64(self, psi, dag=False, out=None, stream=None):
        """M_eo psi (or M_eo^dag psi) in float-float arithmetic (FP64-class
        accuracy on the FP32 pipes); psi and the result are complex128."""
        import torch

        nrhs = self._nrhs(psi)
        out = torch.empty_like(psi) if out is None else out
        wilson_eo_apply_ff64(self._h, out, psi, nrhs, dag, stream)
        return out

    def hop(self, psi, out_parity, dag=False, out=None, stream=None):
        import torch

        nrhs = self._nrhs(psi)
        out = torch.empty_like(psi) if out is None else out
        wilson_eo_hop(self._h, out_parity, dag, out, psi, nrhs, stream)
        return out

    def link_grad(self, g, phi, out=None, stream=None):
        """Gradient of Re<g, M_eo phi> with respect to the links, (4, V, 3, 3)."""
        import torch

        V = 2 * self.vh
        out = torch.empty((4, V, 3, 3), dtype=self.spinor_dtype(), device=phi.device) \
            if out is None else out
        wilson_eo_link_grad(self._h, out, g, phi, stream)
        return out

    def force(self, phi, want_dphi=False, stream=None):
        """(F, dS/dphi or None) for S = |M_eo phi|^2."""
        import torch

        V = 2 * self.vh
        F = torch.empty((4, V, 3, 3), dtype=self.spinor_dtype(), device=phi.device)
        d = torch.empty_like(phi) if want_dphi else None
        wilson_eo_force(self._h, F, d, phi, stream)
        return F, d

    def solve(self, b, x0=None, tol=1e-10, maxiter=10000, mixed=True, stream=None):
        """x with M^dag M x = b (complex128 planar; a leading batch dimension
        solves several systems in lockstep). Returns (x, info dict)."""
        import torch

        x = torch.zeros_like(b) if x0 is None else x0.clone()
        if b.dim() == 3:
            st, it, rr = wilson_eo_solve(self._h, x, b, tol, maxiter, mixed, stream)
        else:
            nrhs = int(np.prod(b.shape[:-3]))
            st, it, rr = wilson_eo_solve_multi(self._h, x, b, nrhs, tol, maxiter, mixed, stream)
        info = wilson_eo_solve_stats(self._h)
        info.update({"status": STATUS.get(st, st), "true_relres": rr, "rhs_iterations": it,
                     "converged": st == WEO_OK})
        return x, info

    def set_gauge(self, gauge, stream=None):
        wilson_eo_set_gauge(self._h, gauge, stream=stream)

    def set_kappa(self, kappa):
        self.kappa = float(kappa)
        wilson_eo_set_kappa(self._h, kappa)

    def info(self):
        return wilson_eo_info(self._h)

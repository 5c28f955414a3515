"""Python binding of the libsyk_gb300 C ABI (include/syk.h): argument marshalling only.

Functions carry the C names.  Device vectors are torch CUDA tensors of shape
(D, B) (compact sector index x batch column, row-major = state-interleaved)
with dtype complex64 (SYK_C64) or complex128 (SYK_C128).  Every computation
runs in the CUDA library; if it is not built, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SYK_OK = 0
SYK_EINVAL, SYK_ENOMEM, SYK_ECUDA, SYK_ENUMERIC, SYK_ETIMEOUT = -1, -2, -3, -4, -5  # include/syk.h
SYK_C64 = 1
SYK_C128 = 2
MAX_KRYLOV = 64


class SykError(RuntimeError):
    pass


_lib = None


def library_path() -> str:
    """The library to load: $SYK_LIBRARY if set (a variant build), else the in-tree build."""
    return os.environ.get("SYK_LIBRARY", _build.LIB)


def load(build_if_missing: bool = False):
    """Loads the shared library (building it first only if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing or path != _build.LIB:
            raise SykError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                           "or python -m paper_2002_05725_gb300.build")
        _build.build()
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "syk_build_terms": (i32, [i32, vp, ctypes.POINTER(vp)]),
        "syk_free_terms": (None, [vp]),
        "syk_terms_info": (i32, [vp, vp, vp, vp, vp]),
        "syk_term_table": (i32, [vp, vp, vp, vp]),
        "syk_apply_H": (i32, [vp, i32, i32, vp, vp, i64, vp]),
        "syk_apply_chi": (i32, [i32, i32, i32, i32, vp, vp, i64, vp]),
        "syk_tridiag_expm": (i32, [i32, i64, vp, vp, vp, dbl, dbl, vp, vp]),
        "syk_workspace_bytes": (sz, [i32, i32, i32, i64, i32]),
        "syk_expmv": (i32, [vp, i32, i32, dbl, dbl, vp, vp, i64, i32, dbl, vp, sz, vp, vp]),
        "syk_expmv_static": (i32, [vp, i32, i32, dbl, dbl, vp, vp, i64, i32, dbl, vp, vp]),
        "syk_correlator_G": (i32, [vp, dbl, i32, vp, i32, vp, i64, i32, i32, dbl, vp, vp, vp]),
        "syk_otoc": (i32, [vp, dbl, i32, i32, vp, i32, vp, i64, i32, i32, dbl, vp, vp]),
        "syk_last_error": (ctypes.c_char_p, []),
        "syk_counters": (i32, [vp, vp, vp, i32]),
        "syk_profile_enable": (i32, [i32]),
        "syk_use_graphs": (i32, [i32]),
        "syk_profile_read": (i32, [vp, vp, i32]),
        "syk_autotune_apply": (i32, [vp, i32, i32, i64, i32, vp, vp]),
        "syk_otoc_split": (i32, [vp, dbl, vp, i32, i32, vp, i32, vp, i64, i32, i32, dbl, vp, vp]),
        "syk_correlator_G_imag": (i32, [vp, dbl, i32, vp, i32, vp, i64, i32, i32, dbl, vp, vp, vp]),
        "syk_otoc_batch": (i32, [vp, i32, i32, i32, vp, i32, i32, i32, dbl, i32, vp]),
        "syk_otoc_grad": (i32, [vp, dbl, i32, i32, dbl, vp, i64, i32, i32, dbl, dbl, vp, vp, vp, vp]),
        "syk_correlator_G_grad": (i32, [vp, dbl, i32, dbl, vp, i64, i32, i32, dbl, dbl, vp, vp, vp, vp]),
        "syk_autotune_export": (i32, [ctypes.c_char_p, sz]),
        "syk_autotune_import": (i32, [ctypes.c_char_p]),
        "syk_autotune_reset": (i32, []),
        "syk_lowest_eigenvalues": (i32, [vp, i32, i32, vp, i32, i32, dbl, vp, vp, vp, vp]),
        "syk_fma_peak": (i32, [i32, i32, vp, vp, vp, vp]),
        "syk_matvec_launches": (i32, [vp, vp, vp, i32]),
        "syk_c128_arith": (i32, [i32]),
        "syk_status": (i32, [vp, i32, vp]),
        "syk_lanczos_orth": (i32, [i32, i32]),
        "syk_batch_persistent": (i32, [i32]),
        "syk_batch_report": (i32, [vp, i32]),
        "syk_batch_plan": (i32, [i32, i64, i32, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/syk.h that the loaded library must export."""
    return ["syk_build_terms", "syk_free_terms", "syk_terms_info", "syk_term_table", "syk_apply_H",
            "syk_apply_chi", "syk_tridiag_expm", "syk_workspace_bytes", "syk_expmv", "syk_expmv_static", "syk_correlator_G",
            "syk_otoc", "syk_last_error", "syk_counters", "syk_profile_enable", "syk_profile_read",
            "syk_autotune_apply", "syk_autotune_export", "syk_autotune_import", "syk_otoc_grad",
            "syk_correlator_G_grad", "syk_otoc_batch", "syk_use_graphs", "syk_otoc_split",
            "syk_correlator_G_imag", "syk_autotune_reset", "syk_lowest_eigenvalues", "syk_fma_peak",
            "syk_matvec_launches", "syk_c128_arith", "syk_status", "syk_lanczos_orth", "syk_batch_persistent",
            "syk_batch_report", "syk_batch_plan"]


def _check(rc: int, what: str):
    if rc != SYK_OK:
        msg = load().syk_last_error().decode(errors="replace")
        raise SykError(f"{what} failed with code {rc}: {msg}")


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return SYK_C64
    if t.dtype == torch.complex128:
        return SYK_C128
    raise SykError(f"unsupported dtype {t.dtype}")


def _as_cols(t):
    if t.dim() == 1:
        return t.reshape(-1, 1)
    if t.dim() != 2:
        raise SykError("vectors must have shape (D,) or (D, B)")
    return t


class Terms:
    """Owns a syk_terms* (freed with syk_free_terms)."""

    def __init__(self, ptr: int, N: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.N = N
        info = syk_terms_info(self)
        self.nterms, self.nmasks, self.D = info["nterms"], info["nmasks"], info["dim"]

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.syk_free_terms(self.ptr)
            self.ptr = ctypes.c_void_p(None)


def syk_build_terms(N: int, J) -> Terms:
    L = load()
    J = np.ascontiguousarray(J, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(L.syk_build_terms(int(N), J.ctypes.data, ctypes.byref(out)), "syk_build_terms")
    return Terms(out.value, int(N))


def syk_terms_info(terms: Terms) -> dict:
    N = ctypes.c_int()
    nt, nm, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().syk_terms_info(terms.ptr, ctypes.byref(N), ctypes.byref(nt), ctypes.byref(nm), ctypes.byref(d)),
           "syk_terms_info")
    return {"N": N.value, "nterms": nt.value, "nmasks": nm.value, "dim": d.value}


def syk_term_table(terms: Terms):
    xm = np.zeros(terms.nterms, dtype=np.uint64)
    zm = np.zeros(terms.nterms, dtype=np.uint64)
    ph = np.zeros(terms.nterms, dtype=np.uint8)
    _check(load().syk_term_table(terms.ptr, xm.ctypes.data, zm.ctypes.data, ph.ctypes.data), "syk_term_table")
    return xm, zm, ph


def syk_apply_H(terms: Terms, parity: int, psi, out=None, stream=None):
    import torch
    p = _as_cols(psi)
    y = torch.empty_like(p) if out is None else _as_cols(out)
    _check(load().syk_apply_H(terms.ptr, int(parity), _dtype_code(p), p.data_ptr(), y.data_ptr(), p.shape[1],
                              _stream(stream)), "syk_apply_H")
    return y.reshape(psi.shape)


def syk_apply_chi(N: int, i: int, parity_in: int, psi, out=None, stream=None):
    import torch
    p = _as_cols(psi)
    y = torch.empty_like(p) if out is None else _as_cols(out)
    _check(load().syk_apply_chi(int(N), int(i), int(parity_in), _dtype_code(p), p.data_ptr(), y.data_ptr(),
                                p.shape[1], _stream(stream)), "syk_apply_chi")
    return y.reshape(psi.shape)


def syk_tridiag_expm(alpha, beta, beta0, z: complex, stream=None):
    """alpha (m, B), beta (m-1, B), beta0 (B,) float64 CUDA tensors -> (m, B) complex128."""
    import torch
    m, B = alpha.shape
    out = torch.empty((m, B), dtype=torch.complex128, device=alpha.device)
    bptr = beta.data_ptr() if beta.numel() else alpha.data_ptr()
    _check(load().syk_tridiag_expm(m, B, alpha.data_ptr(), bptr, beta0.data_ptr(), float(z.real), float(z.imag),
                                   out.data_ptr(), _stream(stream)), "syk_tridiag_expm")
    return out


def syk_workspace_bytes(N: int, dtype: int, krylov_dim: int, batch: int, kind: int = 0) -> int:
    return int(load().syk_workspace_bytes(int(N), int(dtype), int(krylov_dim), int(batch), int(kind)))


def syk_expmv(terms: Terms, parity: int, z: complex, psi, krylov_dim: int = 40, tol: float = 1e-12, out=None,
              workspace=None, stream=None):
    """Returns (e^{zH} psi, number of Krylov bases)."""
    import torch
    p = _as_cols(psi)
    y = torch.empty_like(p) if out is None else _as_cols(out)
    ns = ctypes.c_int(0)
    wptr, wbytes = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (None, 0)
    z = complex(z)
    _check(load().syk_expmv(terms.ptr, int(parity), _dtype_code(p), z.real, z.imag, p.data_ptr(), y.data_ptr(),
                            p.shape[1], int(krylov_dim), float(tol), wptr, wbytes, _stream(stream),
                            ctypes.byref(ns)), "syk_expmv")
    return y.reshape(psi.shape), ns.value


def syk_expmv_static(terms: Terms, parity: int, z: complex, psi, krylov_dim: int = 40, tol: float = 1e-12,
                     out=None, stream=None):
    """syk_expmv with the library's fixed device scratch (no allocation by the call).

    The term set must already be on the device (any earlier call uploads it).
    Returns (e^{zH} psi, number of Krylov bases).
    """
    import torch
    p = _as_cols(psi)
    y = torch.empty_like(p) if out is None else _as_cols(out)
    ns = ctypes.c_int(0)
    z = complex(z)
    _check(load().syk_expmv_static(terms.ptr, int(parity), _dtype_code(p), z.real, z.imag, p.data_ptr(),
                                   y.data_ptr(), p.shape[1], int(krylov_dim), float(tol), _stream(stream),
                                   ctypes.byref(ns)), "syk_expmv_static")
    return y.reshape(psi.shape), ns.value


def _input_ptr(psi0):
    """(pointer, B, dtype code, keep-alive) for a CUDA tensor, a host tensor or a numpy array."""
    if isinstance(psi0, np.ndarray):
        a = np.ascontiguousarray(psi0)
        a2 = a.reshape(a.shape[0], -1)
        code = SYK_C64 if a.dtype == np.complex64 else SYK_C128 if a.dtype == np.complex128 else None
        if code is None:
            raise SykError("numpy input must be complex64 or complex128")
        return a.ctypes.data, a2.shape[1], code, a
    t = _as_cols(psi0)
    if not t.is_contiguous():
        raise SykError("input tensor must be contiguous")
    return t.data_ptr(), t.shape[1], _dtype_code(t), t


def syk_correlator_G(terms: Terms, beta: float, i: int, times, psi0, krylov_dim: int = 30, tol: float = 1e-12,
                     stream=None):
    """Returns (G complex (nt, B), Z (B,)) for G(t) = <phi|chi_i(t) chi_i|phi>/<phi|phi>."""
    t = np.ascontiguousarray(times, dtype=np.float64)
    ptr, B, code, keep = _input_ptr(psi0)
    G = np.zeros((len(t), B, 2))
    Z = np.zeros(B)
    _check(load().syk_correlator_G(terms.ptr, float(beta), int(i), t.ctypes.data, len(t), ptr, B, code,
                                   int(krylov_dim), float(tol), G.ctypes.data, Z.ctypes.data, _stream(stream)),
           "syk_correlator_G")
    del keep
    return G[..., 0] + 1j * G[..., 1], Z


def syk_otoc(terms: Terms, beta: float, i: int, j: int, times, psi0, krylov_dim: int = 40, tol: float = 1e-12,
             stream=None):
    """Returns the unnormalised regularized OTOC F (nt, B) complex; F~ = F / F[t=0]."""
    t = np.ascontiguousarray(times, dtype=np.float64)
    ptr, B, code, keep = _input_ptr(psi0)
    F = np.zeros((len(t), B, 2))
    _check(load().syk_otoc(terms.ptr, float(beta), int(i), int(j), t.ctypes.data, len(t), ptr, B, code,
                           int(krylov_dim), float(tol), F.ctypes.data, _stream(stream)), "syk_otoc")
    del keep
    return F[..., 0] + 1j * F[..., 1]


def syk_counters(reset: bool = False):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().syk_counters(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), int(reset)), "syk_counters")
    return {"h_applies": a.value, "krylov_bases": b.value, "launches": c.value}


def syk_profile_enable(on: bool = True):
    _check(load().syk_profile_enable(int(on)), "syk_profile_enable")


def syk_profile_read(reset: bool = False):
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(load().syk_profile_read(ctypes.byref(n), ctypes.byref(ms), int(reset)), "syk_profile_read")
    return {"launches": n.value, "total_ms": ms.value}


def syk_autotune_apply(terms: Terms, dtype: int, batch: int, parity: int = 0, reps: int = 2, stream=None) -> float:
    """Tunes the matvec launch shape for (N, dtype, batch); returns the best ms per apply."""
    best = ctypes.c_double(0.0)
    _check(load().syk_autotune_apply(terms.ptr, int(parity), int(dtype), int(batch), int(reps), _stream(stream),
                                     ctypes.byref(best)), "syk_autotune_apply")
    return best.value


def syk_autotune_export() -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().syk_autotune_export(buf, len(buf)), "syk_autotune_export")
    return buf.value.decode()


def syk_autotune_import(text: str):
    _check(load().syk_autotune_import(text.encode()), "syk_autotune_import")


def syk_autotune_reset():
    """Forgets every tuned launch shape (the built-in heuristic applies again)."""
    _check(load().syk_autotune_reset(), "syk_autotune_reset")


def syk_otoc_grad(terms: Terms, beta: float, i: int, j: int, t: float, psi0, krylov_dim: int = 40,
                  tol: float = 1e-12, quad_dz: float = 0.25, stream=None):
    """Returns (F~(t) (B,), dF~/dJ (C(N,4), B), dF~/dbeta (B,)) as complex numpy arrays."""
    ptr, B, code, keep = _input_ptr(psi0)
    F = np.zeros((B, 2))
    dJ = np.zeros((terms.nterms, B, 2))
    db = np.zeros((B, 2))
    _check(load().syk_otoc_grad(terms.ptr, float(beta), int(i), int(j), float(t), ptr, B, code, int(krylov_dim),
                                float(tol), float(quad_dz), F.ctypes.data, dJ.ctypes.data, db.ctypes.data,
                                _stream(stream)), "syk_otoc_grad")
    del keep
    c = lambda a: a[..., 0] + 1j * a[..., 1]
    return c(F), c(dJ), c(db)


def syk_correlator_G_grad(terms: Terms, beta: float, i: int, t: float, psi0, krylov_dim: int = 30,
                          tol: float = 1e-12, quad_dz: float = 0.25, stream=None):
    """Returns (G(t) (B,), dG/dJ (C(N,4), B), dG/dbeta (B,)) as complex numpy arrays."""
    ptr, B, code, keep = _input_ptr(psi0)
    G = np.zeros((B, 2))
    dJ = np.zeros((terms.nterms, B, 2))
    db = np.zeros((B, 2))
    _check(load().syk_correlator_G_grad(terms.ptr, float(beta), int(i), float(t), ptr, B, code, int(krylov_dim),
                                        float(tol), float(quad_dz), G.ctypes.data, dJ.ctypes.data, db.ctypes.data,
                                        _stream(stream)), "syk_correlator_G_grad")
    del keep
    c = lambda a: a[..., 0] + 1j * a[..., 1]
    return c(G), c(dJ), c(db)


class _OtocItem(ctypes.Structure):
    _fields_ = [("terms", ctypes.c_void_p), ("beta", ctypes.c_double), ("psi0", ctypes.c_void_p),
                ("nstates", ctypes.c_int64), ("F_re_im", ctypes.c_void_p)]


def syk_otoc_batch(items, i: int, j: int, times, dtype: int = SYK_C64, krylov_dim: int = 40, tol: float = 1e-7,
                   nworkers: int = 4):
    """items: list of (Terms, beta, psi0) with psi0 a (D, B) CUDA tensor, host tensor or numpy array.

    Returns a list of complex arrays F (nt, B), one per item.
    """
    t = np.ascontiguousarray(times, dtype=np.float64)
    keep, outs = [], []
    arr = (_OtocItem * len(items))()
    for k, (terms, beta, psi0) in enumerate(items):
        ptr, B, code, kp = _input_ptr(psi0)
        if code != dtype:
            raise SykError("every item must use the batch dtype")
        F = np.zeros((len(t), B, 2))
        keep.append((kp, terms))
        outs.append(F)
        arr[k] = _OtocItem(terms.ptr.value, float(beta), ptr, B, F.ctypes.data)
    status = np.zeros(len(items), dtype=np.int32)
    _check(load().syk_otoc_batch(ctypes.cast(arr, ctypes.c_void_p), len(items), int(i), int(j), t.ctypes.data,
                                 len(t), int(dtype), int(krylov_dim), float(tol), int(nworkers),
                                 status.ctypes.data), "syk_otoc_batch")
    del keep
    return [F[..., 0] + 1j * F[..., 1] for F in outs]


BATCH_STREAMS, BATCH_PERSISTENT, BATCH_PERSISTENT_SPLIT_ALWAYS = 0, 1, 2


def syk_batch_persistent(mode=True) -> int:
    """0 / False: every syk_otoc_batch item on the per-item streams; 1 / True: items that fit
    run in the persistent launch (split items only in large batches); 2: split items always
    go there too.  Returns the previous mode."""
    rc = load().syk_batch_persistent(int(mode))
    if rc < 0:
        _check(rc, "syk_batch_persistent")
    return rc


def syk_batch_plan(N: int, nstates: int, krylov_dim: int = 40, smem_limit: int = 0):
    """(states per CTA, shared memory per CTA) of the persistent launch for a complex64 item;
    states per CTA 0 means the per-item path.  smem_limit <= 0: the current device's limit."""
    bs, sm = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().syk_batch_plan(int(N), int(nstates), int(krylov_dim), int(smem_limit), ctypes.byref(bs),
                                 ctypes.byref(sm)), "syk_batch_plan")
    return bs.value, sm.value


BATCH_REPORT_KEYS = ("persistent_items", "stream_items", "persistent_ctas", "cycles_matvec", "cycles_check",
                     "cycles_eig", "cycles_items", "h_applies", "checks", "full_eigs", "persistent_subitems",
                     "matvec_flops")


def syk_batch_report() -> dict:
    """Counters of the last syk_otoc_batch call (see include/syk.h)."""
    out = np.zeros(len(BATCH_REPORT_KEYS), dtype=np.int64)
    _check(load().syk_batch_report(out.ctypes.data, len(out)), "syk_batch_report")
    return {k: int(v) for k, v in zip(BATCH_REPORT_KEYS, out)}


def syk_lowest_eigenvalues(terms: Terms, k: int, psi0, parity: int = 0, max_steps: int = 1024, tol: float = 1e-8,
                           stream=None, check: bool = True):
    """k lowest eigenvalues of H in one sector by Lanczos from psi0 (a (D,) or (D, 1) vector).

    Returns (evals (k,), residual bounds (k,), Lanczos steps). With check=False a run that did
    not converge returns its current Ritz values instead of raising."""
    ptr, B, code, keep = _input_ptr(psi0)
    if B != 1:
        raise SykError("syk_lowest_eigenvalues takes one start vector")
    ev = np.zeros(int(k))
    rs = np.zeros(int(k))
    n = ctypes.c_int(0)
    rc = load().syk_lowest_eigenvalues(terms.ptr, int(parity), code, ptr, int(k), int(max_steps), float(tol),
                                       ev.ctypes.data, rs.ctypes.data, ctypes.byref(n), _stream(stream))
    if check or rc != SYK_ENUMERIC:
        _check(rc, "syk_lowest_eigenvalues")
    del keep
    return ev, rs, n.value


GRAPHS_OFF, GRAPHS_SEGMENTS, GRAPHS_DEVICE = 0, 1, 2


def syk_use_graphs(mode=True):
    """0 / False: direct launches; 1 / True: segment graphs (default); 2: device-driven evolutions."""
    _check(load().syk_use_graphs(int(mode)), "syk_use_graphs")


def syk_otoc_split(terms: Terms, beta: float, x, i: int, j: int, times, psi0, krylov_dim: int = 40,
                   tol: float = 1e-12, stream=None):
    """OTOC with rho split as Tr[W rho^x1 V rho^x2 W rho^x3 V rho^x4]; returns F (nt, B) complex."""
    t = np.ascontiguousarray(times, dtype=np.float64)
    xs = np.ascontiguousarray(x, dtype=np.float64)
    if xs.shape != (4,):
        raise SykError("the split needs four fractions")
    ptr, B, code, keep = _input_ptr(psi0)
    F = np.zeros((len(t), B, 2))
    _check(load().syk_otoc_split(terms.ptr, float(beta), xs.ctypes.data, int(i), int(j), t.ctypes.data, len(t), ptr,
                                 B, code, int(krylov_dim), float(tol), F.ctypes.data, _stream(stream)),
           "syk_otoc_split")
    del keep
    return F[..., 0] + 1j * F[..., 1]


def syk_correlator_G_imag(terms: Terms, beta: float, i: int, taus, psi0, krylov_dim: int = 30, tol: float = 1e-12,
                          stream=None):
    """Imaginary-time G(tau) (ntau, B) complex and Z (B,)."""
    t = np.ascontiguousarray(taus, dtype=np.float64)
    ptr, B, code, keep = _input_ptr(psi0)
    G = np.zeros((len(t), B, 2))
    Z = np.zeros(B)
    _check(load().syk_correlator_G_imag(terms.ptr, float(beta), int(i), t.ctypes.data, len(t), ptr, B, code,
                                        int(krylov_dim), float(tol), G.ctypes.data, Z.ctypes.data, _stream(stream)),
           "syk_correlator_G_imag")
    del keep
    return G[..., 0] + 1j * G[..., 1], Z


def syk_fma_peak(bits: int = 32, iters: int = 4096, stream=None):
    """Measured FMA throughput of the current device: {"tflops", "sms", "ms"} (2 flop per FMA)."""
    L = load()
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    sms = ctypes.c_int(0)
    _check(L.syk_fma_peak(int(bits), int(iters), ctypes.byref(tf), ctypes.byref(sms), ctypes.byref(ms),
                          _stream(stream)), "syk_fma_peak")
    return {"tflops": tf.value, "sms": sms.value, "ms": ms.value}


def syk_matvec_launches(reset: bool = False):
    """Matvec launches by kernel family since the last reset: {"rows", "tiled", "coset"}."""
    L = load()
    v = [ctypes.c_int64(0) for _ in range(3)]
    _check(L.syk_matvec_launches(*(ctypes.byref(x) for x in v), int(bool(reset))), "syk_matvec_launches")
    return {"rows": v[0].value, "tiled": v[1].value, "coset": v[2].value}


C128_DOUBLE_FLOAT, C128_FP64 = 0, 1


def syk_c128_arith(mode: int = -1) -> int:
    """Sets the complex128 matvec arithmetic (0: double-float, 1: FP64; < 0 only queries) and
    returns the previous mode."""
    rc = load().syk_c128_arith(int(mode))
    if rc < 0:
        _check(rc, "syk_c128_arith")
    return rc


def syk_status(terms: Terms, reset: bool = False, stream=None) -> int:
    """Status word of the term set's matvecs (synchronising): SYK_OK or SYK_ETIMEOUT."""
    return int(load().syk_status(terms.ptr, int(bool(reset)), _stream(stream)))


ORTH_FULL, ORTH_LOCAL = 0, 1


def syk_lanczos_orth(dtype: int, mode: int = -1) -> int:
    """Sets expmv's Lanczos orthogonalisation for dtype (0: full Gram-Schmidt, 1: three-term
    recurrence; < 0 only queries) and returns the previous mode."""
    rc = load().syk_lanczos_orth(int(dtype), int(mode))
    if rc < 0:
        _check(rc, "syk_lanczos_orth")
    return rc

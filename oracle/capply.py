"""ctypes wrapper of the oracle's plain-C term-at-a-time H|psi> (c/apply_terms.c).

TEST INFRASTRUCTURE (CPU oracle).  ``build()`` compiles the C file with gcc
and OpenMP into oracle/c/_build/; ``apply_H`` evaluates (H psi) for all or a
sample of compact rows, using the term table of ``hamiltonian.term_table``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .hamiltonian import term_table

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "apply_terms.c")
_OUT = os.path.join(_HERE, "c", "_build", "liboracle_apply.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", _OUT])
    return _OUT


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        f = _lib.oracle_apply_terms
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return _lib


class TermList:
    """Pauli-string terms w_T X^m Z^z of one coupling draw (w_T = J_T i^p / 4)."""

    def __init__(self, N: int, J: np.ndarray):
        m, z, p = term_table(N)
        self.N = N
        self.m = np.ascontiguousarray(m, dtype=np.uint64)
        self.z = np.ascontiguousarray(z, dtype=np.uint64)
        w = np.asarray(J, dtype=np.float64) * (1j ** p.astype(np.int64)) / 4.0
        self.w_re = np.ascontiguousarray(w.real)
        self.w_im = np.ascontiguousarray(w.imag)


def apply_H(terms: TermList, sector: int, psi: np.ndarray, rows=None, nthreads: int | None = None):
    """(H psi) at compact ``rows`` (all rows if None); psi has shape (D,) or (D, B)."""
    lib = _load()
    psi2 = np.ascontiguousarray(psi.reshape(psi.shape[0], -1), dtype=np.complex128)
    D, B = psi2.shape
    if D != 1 << (terms.N // 2 - 1):
        raise ValueError("psi has the wrong sector dimension")
    if rows is None:
        nrows, rows_arr, rows_ptr = D, None, None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nrows, rows_ptr = len(rows_arr), rows_arr.ctypes.data
    y = np.zeros((nrows, B), dtype=np.complex128)
    nt = nthreads or os.cpu_count() or 1
    rc = lib.oracle_apply_terms(terms.N, sector, len(terms.m), terms.m.ctypes.data, terms.z.ctypes.data,
                                terms.w_re.ctypes.data, terms.w_im.ctypes.data, nrows, rows_ptr, B,
                                psi2.ctypes.data, y.ctypes.data, nt)
    if rc != 0:
        raise RuntimeError("oracle_apply_terms failed")
    return y.reshape((nrows,) + psi.shape[1:])

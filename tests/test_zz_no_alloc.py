"""syk_expmv_static: the expmv variant that allocates nothing.

Some callers cannot allocate device memory when they call (services whose
device memory is budgeted up front, hosts that route every allocation through
their own pool, latency-critical loops where cudaMalloc/cudaFree would stall
the device).  For them syk_expmv_static keeps its Krylov workspace in a fixed
array of device memory inside the library.  This file runs last so that a
failure here cannot hide any other test; it passes alone in a fresh process
and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from helpers import TOL, rel, to_dev, torch_or_skip
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_expmv_static_matches_expmv_repeatedly(dt):
    """Three calls in a row agree with syk_expmv, and calls after the first take no device
    memory: the first call may still load the library's device code (lazy module loading)
    and look up the array's address, later ones must not capture or instantiate graphs."""
    torch = torch_or_skip()
    lib = syk.load(build_if_missing=True)
    N, B, m = 20, 4, 30
    tol = 1e-12 if dt == "c128" else 1e-7
    code = syk.SYK_C128 if dt == "c128" else syk.SYK_C64
    terms = syk.syk_build_terms(N, inputs.couplings(N, 17))
    psi = to_dev(torch, inputs.random_states(N, B, 23), dt)
    z = complex(-0.3, -4.0)
    # the allocating entry point: reference result, and it uploads the term set to this device
    ref, _ = syk.syk_expmv(terms, 1, z, psi, krylov_dim=m, tol=tol)
    ref = ref.cpu().numpy()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [torch.empty_like(psi) for _ in range(3)]
    torch.cuda.synchronize()
    free = []
    for call, out in enumerate(outs):
        out.fill_(complex(float("nan"), float("nan")))
        nsteps = ctypes.c_int(0)
        rc = lib.syk_expmv_static(terms.ptr, 1, code, z.real, z.imag, psi.data_ptr(), out.data_ptr(), B, m, tol,
                                  stream, ctypes.byref(nsteps))
        assert rc == syk.SYK_OK, lib.syk_last_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert nsteps.value >= 1
        assert rel(out.cpu().numpy(), ref) < TOL[dt], (call, rel(out.cpu().numpy(), ref))
    assert free[1] == free[2], free


def test_expmv_static_rejects_oversize_and_unuploaded_terms():
    torch = torch_or_skip()
    lib = syk.load(build_if_missing=True)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # N=32 with 16 states and Krylov dimension 40 needs ~700 MB: far above the 16 MiB limit
    big = syk.syk_build_terms(32, inputs.couplings(32, 0))
    psi = torch.zeros((1 << 15, 16), dtype=torch.complex64, device="cuda")
    syk.syk_apply_H(big, 0, psi)
    rc = lib.syk_expmv_static(big.ptr, 0, syk.SYK_C64, 0.0, -1.0, psi.data_ptr(), psi.data_ptr(), 16, 40, 1e-7,
                              stream, None)
    assert rc == -2 and b"static scratch" in lib.syk_last_error()
    # a term set never used on this device is refused rather than uploaded
    fresh = syk.syk_build_terms(12, inputs.couplings(12, 0))
    small = torch.zeros((32, 1), dtype=torch.complex128, device="cuda")
    rc = lib.syk_expmv_static(fresh.ptr, 0, syk.SYK_C128, 0.0, -1.0, small.data_ptr(), small.data_ptr(), 1, 8,
                              1e-12, stream, None)
    assert rc == -1 and b"not on device" in lib.syk_last_error()
    assert np.isfinite(syk.syk_workspace_bytes(12, syk.SYK_C128, 8, 1))

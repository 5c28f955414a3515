"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

The matvec kernels wait on mbarriers for the bulk copies that stage partner tiles.  Each wait
has a poll budget; a CTA whose wait runs out sets the term set's status word (SYK_ETIMEOUT),
lets every copy it has started land (the drain keeps the full budget), and exits, so the
context stays usable.  A variant build with a main-loop budget of zero polls
(-DSYK_WAIT_POLLS=0) makes every such wait give up at once.  In a child process loading that
variant: syk_expmv returns SYK_ETIMEOUT, the status query reports the bare syk_apply_H's
timeout and clears it, and a matvec on the row kernel (no waits) is still correct.  A fresh
process with the normal build then computes the same matvec correctly.
"""
import os
import subprocess
import sys
import textwrap

import pytest

from helpers import torch_or_skip

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import torch
    from oracle import hamiltonian as hm
    from paper_2002_05725_gb300 import inputs, syk
    syk.load()
    expect_timeout = {expect_timeout}
    N = 20
    J = inputs.couplings(N, 3)
    terms = syk.syk_build_terms(N, J)
    H = hm.H_sector_sparse(N, J, 0)
    def dev(B, seed):
        psi = inputs.random_states(N, B, seed)
        return psi, torch.from_numpy(np.ascontiguousarray(psi.T)).to(torch.complex64).cuda()
    # tiled / coset kernels (4 states): the waits for staged tiles
    psi, x = dev(4, 1)
    y = syk.syk_apply_H(terms, 0, x)
    st = syk.syk_status(terms, reset=True)
    err = float(np.abs(y.cpu().numpy() - H @ psi.T).max() / np.abs(H @ psi.T).max())
    if expect_timeout:
        assert st == syk.SYK_ETIMEOUT, st
        assert syk.syk_status(terms) == syk.SYK_OK  # cleared by the reset
        try:
            syk.syk_expmv(terms, 0, complex(0.0, -1.0), x, krylov_dim=20, tol=1e-7)
            raise AssertionError("syk_expmv did not report the timeout")
        except syk.SykError as e:
            assert "code -5" in str(e), str(e)
        syk.syk_status(terms, reset=True)
        # a correlator chain, host-driven and with the step control on the device (the timeout
        # then surfaces when the chain ends)
        for mode in (syk.GRAPHS_SEGMENTS, syk.GRAPHS_DEVICE):
            syk.syk_use_graphs(mode)
            try:
                syk.syk_otoc(terms, 1.0, 0, 1, [0.0, 0.5], x, krylov_dim=20, tol=1e-7)
                raise AssertionError("syk_otoc did not report the timeout")
            except syk.SykError as e:
                assert "code -5" in str(e), str(e)
            syk.syk_status(terms, reset=True)
        syk.syk_use_graphs(syk.GRAPHS_SEGMENTS)
    else:
        assert st == syk.SYK_OK, st
        assert err < 1e-5, err
        out, _ = syk.syk_expmv(terms, 0, complex(0.0, -1.0), x, krylov_dim=20, tol=1e-7)
        assert syk.syk_status(terms) == syk.SYK_OK
    # the row kernel (3 states) has no waits: correct in both builds, context still usable
    psi3, x3 = dev(3, 2)
    y3 = syk.syk_apply_H(terms, 0, x3).cpu().numpy()
    ref3 = H @ psi3.T
    assert np.abs(y3 - ref3).max() / np.abs(ref3).max() < 1e-5
    assert syk.syk_status(terms) == syk.SYK_OK
    torch.cuda.synchronize()
    print("child ok", st, err)
""")


def _run_child(expect_timeout, lib=None):
    env = dict(os.environ)
    if lib:
        env["SYK_LIBRARY"] = lib
    else:
        env.pop("SYK_LIBRARY", None)
    code = CHILD.format(root=ROOT, expect_timeout=expect_timeout)
    return subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                          timeout=900)


def test_bounded_wait_gives_up_with_status_and_context_survives(tmp_path):
    torch_or_skip()
    out = tmp_path / "wait0"
    b = subprocess.run([sys.executable, "-m", "paper_2002_05725_gb300.build", "--out-dir", str(out),
                        "-D", "SYK_WAIT_POLLS=0"], cwd=ROOT, capture_output=True, text=True, timeout=1200)
    assert b.returncode == 0, b.stdout[-2000:] + b.stderr[-2000:]
    r = _run_child(True, str(out / "libsyk_gb300.so"))
    assert r.returncode == 0 and "child ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
    r = _run_child(False)
    assert r.returncode == 0 and "child ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]

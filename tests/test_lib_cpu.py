"""Host-only checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host-built term table is bit-exact against the
oracle's.  No GPU call is made here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import hamiltonian as hm
from paper_2002_05725_gb300 import build, inputs, syk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return syk.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "syk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(syk_[A-Za-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/syk.h but not exported"
    assert sorted(syk.exported_symbols()) == names


@pytest.mark.parametrize("N", [4, 8, 12, 20, 28])
def test_term_table_bit_exact_vs_oracle(lib, N):
    J = inputs.couplings(N, 3)
    t = syk.syk_build_terms(N, J)
    xm, zm, ph = syk.syk_term_table(t)
    m, z, p = hm.term_table(N)
    assert np.array_equal(xm, m) and np.array_equal(zm, z) and np.array_equal(ph, p)
    n = N // 2
    masks = math.comb(n, 4) + (math.comb(n, 2) if n >= 3 else 0) + 1  # popcount-2 masks need a third spin
    assert t.nterms == math.comb(N, 4) and t.nmasks == masks and t.D == 1 << (n - 1)


def test_term_table_sampled_N60(lib):
    """N=60: every flip mask, plus the full (m, z, p) of sampled terms against the oracle."""
    N = 60
    J = inputs.couplings(N, 1)
    t = syk.syk_build_terms(N, J)
    xm, zm, ph = syk.syk_term_table(t)
    q = hm.quadruples(N)
    assert np.array_equal(xm, hm.flip_mask(q).astype(np.uint64))
    rng = np.random.default_rng(0)
    idx = rng.choice(len(q), 300, replace=False)
    amp0, x0 = hm.term_action(q[idx], 0)
    assert np.array_equal(x0.astype(np.uint64), xm[idx])
    assert np.allclose(4 * amp0, 1j ** ph[idx].astype(np.int64), atol=1e-12)
    for k in range(N // 2):
        ak, _ = hm.term_action(q[idx], np.int64(1) << k)
        sgn = np.real(4 * ak / (1j ** ph[idx].astype(np.int64)))
        assert np.array_equal(sgn < 0, ((zm[idx] >> np.uint64(k)) & np.uint64(1)).astype(bool))


def test_invalid_arguments(lib):
    out = ctypes.c_void_p()
    J = np.zeros(10)
    for N in (3, 5, 2, 66):
        assert lib.syk_build_terms(N, J.ctypes.data, ctypes.byref(out)) == -1
        assert b"N=" in lib.syk_last_error()
    with pytest.raises(syk.SykError):
        syk.syk_build_terms(8, np.full(70, np.nan))
    assert lib.syk_apply_chi(7, 0, 0, 1, None, None, 1, None) == -1
    assert syk.syk_workspace_bytes(12, syk.SYK_C64, 0, 1) == 0
    assert syk.syk_workspace_bytes(12, 3, 8, 1) == 0


def test_workspace_formula(lib):
    b1 = syk.syk_workspace_bytes(40, syk.SYK_C64, 40, 16)
    vec = (1 << 19) * 16 * 8
    assert 42 * vec <= b1 < 42 * vec + (64 << 20)
    assert syk.syk_workspace_bytes(40, syk.SYK_C128, 40, 16) > b1


def test_autotune_table_json(lib):
    """The launch-shape table (host only): kernel variant round trip, invalid entries refused."""
    syk.syk_autotune_import('{"apply_tiles": [{"N": 36, "dtype": 1, "batch": 16, "ntb": 6, "cluster": 2,'
                            ' "variant": 2, "ms": 1.5}, {"N": 36, "dtype": 2, "batch": 4, "ntb": 7, "cluster": 1}]}')
    js = syk.syk_autotune_export()
    assert '"N": 36, "dtype": 1, "batch": 16, "ntb": 6, "cluster": 2, "variant": 2' in js
    assert '"N": 36, "dtype": 2, "batch": 4, "ntb": 7, "cluster": 1, "variant": 0' in js
    for bad in ('{"N": 36, "dtype": 2, "batch": 16, "ntb": 6, "cluster": 1, "variant": 2}',  # c128 has no cosets
                '{"N": 36, "dtype": 1, "batch": 16, "ntb": 6, "cluster": 1, "variant": 3}',  # 8 rows x 16 columns
                '{"N": 36, "dtype": 1, "batch": 2, "ntb": 6, "cluster": 1, "variant": 1}',
                '{"N": 36, "dtype": 1, "batch": 8, "ntb": 9, "cluster": 1}',
                '{"N": 36, "dtype": 1, "batch": 8, "ntb": 6, "cluster": 3}'):
        with pytest.raises(syk.SykError):
            syk.syk_autotune_import('{"apply_tiles": [%s]}' % bad)
    syk.syk_autotune_reset()
    assert syk.syk_autotune_export() == '{"apply_tiles": []}'


def test_return_codes_match_header(lib):
    """The binding's return-code constants are the header's."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "syk.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (SYK_E[A-Z]+) \((-?\d+)\)", hdr)}
    assert codes and all(getattr(syk, k) == v for k, v in codes.items())

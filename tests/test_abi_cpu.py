"""The C-ABI library builds, loads and exports every symbol include/tm.h
declares; host-side argument checks work without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tm():
    from paper_2212_06635_gb300 import build
    build.build()
    from paper_2212_06635_gb300 import tm as _tm
    return _tm


def _declared():
    src = open(os.path.join(ROOT, "include", "tm.h")).read()
    return sorted(set(re.findall(r"\b(tm_[a-zA-Z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(tm):
    names = _declared()
    assert "tm_solve_cg" in names and "tm_apply_Mhat" in names
    for n in names:
        assert hasattr(tm.lib, n), n
    assert set(names) <= set(tm.EXPORTED)


def test_bad_dims_rejected_on_host(tm):
    for dims in [(3, 4, 4, 4), (4, 4, 0, 4), (4, 4, 4, 1)]:
        with pytest.raises(tm.TMError) as e:
            tm.tm_create(dims)
        assert e.value.status == tm.TM_ERR_ARG
        assert "even" in tm.tm_last_error()


def test_null_arguments_rejected(tm):
    import ctypes as ct
    assert tm.lib.tm_create(None, None, 0) == tm.TM_ERR_ARG
    assert tm.lib.tm_solve_cg(None, 2, None, None, None, None, None) == tm.TM_ERR_ARG
    assert tm.lib.tm_destroy(None) == tm.TM_OK
    v = ct.c_double()
    assert tm.lib.tm_gauge_id(None, ct.byref(v)) == tm.TM_ERR_ARG
    assert tm.lib.tm_apply_Mhat_dw(None, 2, None, None, None) == tm.TM_ERR_ARG
    assert "bad pointers" in tm.tm_last_error()


def test_force_outer_host_checks(tm):
    """Argument checks of tm_force_outer that run before any CUDA call."""
    assert tm.lib.tm_force_outer(None, 1, 2, 0, None, None, None, 0, None, None) == tm.TM_ERR_ARG
    assert "bad pointers" in tm.tm_last_error()
    with pytest.raises(ValueError):
        tm.tm_force_outer(None, 1, 2, [1.0, 2.0], [(0, 0)], [(0, 0)], 0)


def test_rational_coefficients_match_oracle(tm):
    """tm_rational_inv_sqrt (host code of the library: theta-function poles,
    extrema located by root finding) against the oracle's Zolotarev coefficients
    (AGM poles, constant centred on a fixed grid), which are pinned by Chebyshev
    alternation.  Poles and residues agree to 1e-9; the constant and delta to
    the resolution of the oracle's 200001-point grid (delta within 3e-3 relative
    at 16 poles, where it is 1.2e-8)."""
    import numpy as np
    from oracle import rational as RA
    for n, lo, hi in ((4, 1e-3, 2.0), (8, 2.7e-5, 2.7), (12, 2.7e-5, 2.7), (16, 1e-6, 1.0)):
        a0, a, s, d = tm.tm_rational_inv_sqrt(n, lo, hi)
        b0, b, t, e = RA.zolotarev_inv_sqrt(n, lo, hi)
        assert abs(a0 - b0) <= 1e-8 * b0
        assert np.allclose(a, b, rtol=1e-8) and np.allclose(s, t, rtol=1e-9)
        assert abs(d - e) <= 3e-3 * e
    for bad in ((0, 1e-3, 1.0), (17, 1e-3, 1.0), (4, 0.0, 1.0), (4, 1.0, 0.5)):
        with pytest.raises(tm.TMError):
            tm.tm_rational_inv_sqrt(*bad)


@pytest.mark.parametrize("n,lo,hi", [(1, 0.1, 1.0), (3, 1e-2, 1.0), (4, 1e-3, 2.0), (8, 2.7e-5, 2.7),
                                     (12, 1e-5, 1.0), (16, 1e-6, 1.0)])
def test_library_rational_equioscillates(tm, n, lo, hi):
    """The library's own coefficients, independently of the oracle: the relative
    error sqrt(x) r(x) - 1 of the partial fractions it returns equioscillates at
    2n + 2 points of [lo, hi] (Chebyshev's alternation theorem for the best
    type-(n, n) approximation), its peak is the returned delta, and delta is
    Zolotarev's error 4 q^(2n+1), q = exp(-pi K'/K) the nome of k = sqrt(1 - lo/hi)
    (K from scipy, not from the library)."""
    import numpy as np
    from scipy.special import ellipk
    a0, a, sigma, delta = tm.tm_rational_inv_sqrt(n, lo, hi)
    assert a0 > 0 and np.all(np.asarray(a) > 0) and np.all(np.asarray(sigma) > 0)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 400001))
    r = a0 + np.sum(np.asarray(a)[:, None] / (x[None, :] + np.asarray(sigma)[:, None]), axis=0)
    err = np.sqrt(x) * r - 1.0
    peak = np.abs(err).max()
    near = np.nonzero(np.abs(err) >= 0.98 * peak)[0]
    runs = 1 + int(np.count_nonzero(np.diff(np.sign(err[near])) != 0))
    assert runs == 2 * n + 2, runs
    assert abs(peak - delta) <= 1e-3 * delta
    eps = lo / hi
    q = np.exp(-np.pi * ellipk(eps) / ellipk(1.0 - eps))
    assert abs(delta - 4 * q ** (2 * n + 1)) <= 1e-4 * delta


def test_rational_coefficients_match_golden(tm):
    import os
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "zolotarev_n12_1e-5.txt")
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    a0, a, s, d = tm.tm_rational_inv_sqrt(12, 1e-5, 1.0)
    assert abs(a0 - float(rows[0][0])) <= 1e-9 * a0
    assert np.allclose(a, [float(r[0]) for r in rows[1:13]], rtol=1e-9)
    assert np.allclose(s, [float(r[1]) for r in rows[1:13]], rtol=1e-9)
    assert abs(d - float(rows[13][0])) <= 1e-3 * d

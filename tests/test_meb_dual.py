"""The host solver of the SES core-set certificates (pdscp_meb_dual: the
minimum enclosing ball's dual by Frank-Wolfe steps with away steps) against
exact solvers: Welzl's algorithm in the plane, support-set enumeration in
d = 3, the closed forms of one point, two points and a regular simplex, and
the oracle's own implementation of the bounds. CPU only (host code of the
library, no GPU)."""

import ctypes
import math

import numpy as np
import pytest

from oracle import exact, ses as oses
from paper_2405_09157_gb300 import _ffi, api


@pytest.mark.parametrize("seed", range(5))
def test_bracket_welzl_in_the_plane(seed):
    rng = np.random.default_rng(seed)
    V = rng.random((400, 2)) - 0.5
    opt = exact.mec_2d(V)[1]
    for tol in (1e-3, 1e-6, 1e-10):
        lb, far, mu, c = api.meb_dual(V, tol=tol)
        assert lb <= opt * (1 + 1e-12) and far >= opt * (1 - 1e-12), (tol, lb, opt, far)
        assert far <= (1 + tol) * lb * (1 + 1e-12), (tol, far, lb)
        assert math.isclose(mu.sum(), 1.0, rel_tol=1e-12) and np.all(mu >= 0.0)
        assert np.allclose(c, mu @ V, rtol=0, atol=1e-12)
        assert math.isclose(far, float(np.linalg.norm(V - c, axis=1).max()), rel_tol=1e-12)


def test_bracket_support_enumeration_in_3d():
    rng = np.random.default_rng(11)
    for _ in range(5):
        V = rng.normal(size=(10, 3))
        opt = exact.meb_bruteforce(V)[1]
        lb, far, _, _ = api.meb_dual(V, tol=1e-12)
        assert lb <= opt * (1 + 1e-9) and far >= opt * (1 - 1e-9)
        assert math.isclose(lb, opt, rel_tol=1e-9) and math.isclose(far, opt, rel_tol=1e-9)


def test_closed_forms():
    lb, far, mu, c = api.meb_dual([[1.0, -2.0, 3.0]])
    assert lb == 0.0 and far == 0.0 and mu[0] == 1.0 and np.allclose(c, [1.0, -2.0, 3.0])
    lb, far, mu, c = api.meb_dual([[0.0, 0.0], [2.0, 0.0]], tol=1e-14)
    assert math.isclose(lb, 1.0, rel_tol=1e-12) and math.isclose(far, 1.0, rel_tol=1e-12)
    assert np.allclose(c, [1.0, 0.0]) and np.allclose(mu, [0.5, 0.5])
    d = 6
    V = np.eye(d + 1) - 1.0 / (d + 1)  # the regular simplex centred at the origin
    lb, far, _, c = api.meb_dual(V, tol=1e-13)
    r = math.sqrt(d / (d + 1))
    assert math.isclose(lb, r, rel_tol=1e-10) and math.isclose(far, r, rel_tol=1e-10)
    assert np.allclose(c, 0.0, atol=1e-10)


def test_translation_and_the_oracle():
    rng = np.random.default_rng(5)
    V = rng.normal(size=(300, 8))
    lb, far, _, c = api.meb_dual(V, tol=1e-9)
    shift = rng.normal(size=8) * 3.0
    lb2, far2, _, c2 = api.meb_dual(V + shift, tol=1e-9)
    assert math.isclose(lb2, lb, rel_tol=1e-7) and math.isclose(far2, far, rel_tol=1e-7)
    assert np.allclose(c2, c + shift, atol=1e-6)
    # the oracle's independent implementation of the same bounds
    _, c_o, lb_o, far_o = oses.meb_dual_fw(V, 1e-9)
    assert lb <= far_o * (1 + 1e-12) and lb_o <= far * (1 + 1e-12)
    assert math.isclose(lb, lb_o, rel_tol=2e-9) and math.isclose(far, far_o, rel_tol=2e-9)


def test_argument_errors():
    lib = _ffi.load()
    p = (ctypes.c_double * 4)()
    out = ctypes.c_double()
    assert lib.pdscp_meb_dual(None, 1, 1, 0.0, 10, p, p, ctypes.byref(out), ctypes.byref(out)) == 1
    assert lib.pdscp_meb_dual(p, 0, 1, 0.0, 10, p, p, ctypes.byref(out), ctypes.byref(out)) == 1
    assert lib.pdscp_meb_dual(p, 1, 0, 0.0, 10, p, p, ctypes.byref(out), ctypes.byref(out)) == 1
    assert lib.pdscp_meb_dual(p, 1, 1, -1.0, 10, p, p, ctypes.byref(out), ctypes.byref(out)) == 1
    assert lib.pdscp_meb_dual(p, 1, 1, 0.0, 0, p, p, ctypes.byref(out), ctypes.byref(out)) == 1
    with pytest.raises(ValueError):
        api.meb_dual(np.ones(3))

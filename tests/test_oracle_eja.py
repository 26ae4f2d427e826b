"""Pins for the oracle's Jordan-algebra primitives (Sec. 2.1, 2.3).

The closed-form SOC exponential is checked against the power series built
from the Jordan product alone; the spectral decomposition against the
defining identities of a Jordan frame; the d = 1 cone against its
isomorphism with R^2_+; the orthant SCMWU against scipy's softmax.
"""

import math

import numpy as np
import pytest
from scipy.special import softmax

from oracle import eja


def _rand_soc(rng, m, d, scale=1.0):
    return scale * rng.standard_normal((m, d + 1))


def _power_series_exp(x, terms=80):
    """sum_k x^{ok}/k! with x^{o0} = e and x^{ok} = x o x^{o(k-1)} (Jordan product)."""
    d = x.shape[-1] - 1
    term = np.tile(eja.soc_identity(d), (x.shape[0], 1))
    acc = term.copy()
    for k in range(1, terms):
        term = eja.soc_product(x, term) / k
        acc = acc + term
    return acc


def test_exp_closed_form_matches_jordan_power_series():
    rng = np.random.default_rng(1)
    for d in (1, 2, 5, 17):
        x = _rand_soc(rng, 20, d, scale=1.5)
        closed = eja.soc_exp(x)
        series = _power_series_exp(x)
        assert np.allclose(closed, series, rtol=1e-12, atol=1e-12)


def test_spectral_frame_identities():
    rng = np.random.default_rng(2)
    x = _rand_soc(rng, 30, 6)
    lam1, lam2, q1, q2 = eja.soc_spectral(x)
    e = eja.soc_identity(6)
    assert np.allclose(lam1[:, None] * q1 + lam2[:, None] * q2, x, atol=1e-13)
    assert np.allclose(eja.soc_product(q1, q1), q1, atol=1e-13)
    assert np.allclose(eja.soc_product(q2, q2), q2, atol=1e-13)
    assert np.allclose(eja.soc_product(q1, q2), 0.0, atol=1e-13)
    assert np.allclose(q1 + q2, e[None, :], atol=1e-13)
    assert np.allclose(eja.soc_trace(q1), 1.0) and np.allclose(eja.soc_trace(q2), 1.0)
    assert np.allclose(eja.soc_trace(x), lam1 + lam2)
    assert np.all(lam1 >= lam2)


def test_identity_and_exp_of_zero():
    e = eja.soc_identity(4)
    rng = np.random.default_rng(3)
    x = _rand_soc(rng, 5, 4)
    assert np.allclose(eja.soc_product(e[None, :], x), x)
    assert np.allclose(eja.soc_exp(np.zeros((3, 5))), np.tile(e, (3, 1)))
    assert math.isclose(float(eja.soc_trace(e)), 2.0)  # rank 2


def test_jordan_axioms_and_associative_inner_product():
    rng = np.random.default_rng(4)
    x, y, z = (_rand_soc(rng, 10, 3) for _ in range(3))
    x2 = eja.soc_product(x, x)
    lhs = eja.soc_product(x2, eja.soc_product(x, y))
    rhs = eja.soc_product(x, eja.soc_product(x2, y))
    assert np.allclose(lhs, rhs, atol=1e-12)
    assert np.allclose(eja.soc_product(x, y), eja.soc_product(y, x))
    assert np.allclose(eja.soc_inner(eja.soc_product(x, y), z), eja.soc_inner(x, eja.soc_product(y, z)))
    # Tr(x o y) is the plain dot product of R^{d+1}
    assert np.allclose(eja.soc_inner(x, y), np.sum(x * y, axis=1))


def test_exp_and_squares_lie_in_the_cone():
    rng = np.random.default_rng(5)
    x = _rand_soc(rng, 50, 8, scale=3.0)
    assert np.all(eja.soc_in_cone(eja.soc_exp(x)))
    assert np.all(eja.soc_in_cone(eja.soc_product(x, x), tol=1e-12))
    assert np.allclose(eja.soc_trace(eja.soc_exp(x)),
                       np.exp(eja.soc_spectral(x)[0]) + np.exp(eja.soc_spectral(x)[1]))


def test_q2_reduces_to_orthant_r2():
    # Q^2 = {(u; u0): |u| <= u0} is R^2_+ in the eigen-coordinates
    # ((u0+u)/sqrt2, (u0-u)/sqrt2); exp must act componentwise there.
    rng = np.random.default_rng(6)
    x = _rand_soc(rng, 40, 1, scale=2.0)
    a = (x[:, 1] + x[:, 0]) / math.sqrt(2)
    b = (x[:, 1] - x[:, 0]) / math.sqrt(2)
    ex = eja.soc_exp(x)
    assert np.allclose((ex[:, 1] + ex[:, 0]) / math.sqrt(2), np.exp(a))
    assert np.allclose((ex[:, 1] - ex[:, 0]) / math.sqrt(2), np.exp(b))


def test_scmwu_orthant_is_softmax_and_shift_invariant():
    rng = np.random.default_rng(7)
    x = 50.0 * rng.standard_normal(1000)
    p, _, _ = eja.scmwu_orthant(x)
    assert np.allclose(p, softmax(x), rtol=1e-12, atol=1e-300)
    p2, _, _ = eja.scmwu_orthant(x + 1234.5)
    assert np.allclose(p, p2, rtol=1e-12)


def test_scmwu_soc_trace_one_cone_and_init():
    rng = np.random.default_rng(8)
    X = _rand_soc(rng, 25, 4, scale=20.0)
    P, _, _ = eja.scmwu_soc(X)
    assert math.isclose(float(np.sum(eja.soc_trace(P))), 1.0, rel_tol=1e-13)
    # on the boundary when e^{lambda_2} underflows: allow rounding
    assert np.all(np.linalg.norm(P[:, :-1], axis=1) <= P[:, -1] * (1 + 1e-12))
    # unshifted definition exp(X)/Tr(exp(X)) on a range where nothing overflows
    Xs = X / 20.0
    E = eja.soc_exp(Xs)
    assert np.allclose(eja.scmwu_soc(Xs)[0], E / np.sum(eja.soc_trace(E)), rtol=1e-12)
    # p^1 = e/r: zero exponent on m cones of rank 2
    P0, _, _ = eja.scmwu_soc(np.zeros((7, 4)))
    assert np.allclose(P0, np.tile(eja.soc_identity(3) / 14.0, (7, 1)))


@pytest.mark.parametrize("d", [1, 3])
def test_inf_norm_and_lambda_min(d):
    rng = np.random.default_rng(9)
    x = _rand_soc(rng, 6, d)
    lam1, lam2, _, _ = eja.soc_spectral(x)
    assert math.isclose(eja.soc_inf_norm(x), float(np.max(np.maximum(abs(lam1), abs(lam2)))))
    assert np.allclose(eja.soc_lambda_min(x), lam2)

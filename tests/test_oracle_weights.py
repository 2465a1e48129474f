"""Pins of the oracle's finite-difference operators (CPU only).

The paper uses first derivatives ``u.dx`` of order ``space_order`` (Sec. II-A,
Function/TimeFunction listings) and their transposes ``.T`` (Sec. III-A,
rotated finite-difference listing); staggered derivatives for the elastic
system (Sec. IV-A).  The weights are not printed in the paper; they are pinned
here by what mathematics fixes: Taylor moment conditions, exactness on
polynomials, the textbook rational values, and the antisymmetry of the
assembled matrices (D^T = -D, (D+)^T = -D-).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

SOS = [2, 4, 6, 8, 10, 12, 14, 16]


@pytest.mark.parametrize("so", SOS)
def test_centred_moment_conditions(so):
    c = oracle.weights_centred(so)
    M = so // 2
    k = np.arange(1, M + 1, dtype=np.float64)
    # D x = 1  :  sum_k c_k (k - (-k)) = 1
    assert abs(np.sum(c * 2 * k) - 1.0) < 1e-13
    # odd powers 3..2M-1 are annihilated
    for p in range(3, 2 * M, 2):
        assert abs(np.sum(c * 2 * k ** p)) < 1e-9 * max(1.0, np.sum(np.abs(c) * 2 * k ** p))


@pytest.mark.parametrize("so", SOS)
def test_centred_equals_fornberg(so):
    M = so // 2
    x = np.array([j for j in range(-M, M + 1)], dtype=np.float64)
    w = oracle.fornberg(1, 0.0, x)
    c = oracle.weights_centred(so)
    for k in range(1, M + 1):
        assert abs(w[M + k] - c[k - 1]) < 1e-13
        assert abs(w[M - k] + c[k - 1]) < 1e-13
    assert abs(w[M]) < 1e-13


@pytest.mark.parametrize("so", SOS)
def test_staggered_moment_conditions(so):
    b = oracle.weights_staggered(so)
    M = so // 2
    s = np.arange(1, M + 1) - 0.5
    assert abs(np.sum(b * 2 * s) - 1.0) < 1e-12
    for p in range(3, 2 * M, 2):
        assert abs(np.sum(b * 2 * s ** p)) < 1e-9 * max(1.0, np.sum(np.abs(b) * 2 * s ** p))


def test_textbook_values():
    # Closed-form centred and staggered weights (textbook values)
    exp_c = {2: [Fraction(1, 2)], 4: [Fraction(2, 3), Fraction(-1, 12)],
             8: [Fraction(4, 5), Fraction(-1, 5), Fraction(4, 105), Fraction(-1, 280)],
             12: [Fraction(6, 7), Fraction(-15, 56), Fraction(5, 63), Fraction(-1, 56),
                  Fraction(1, 385), Fraction(-1, 5544)]}
    exp_b = {2: [Fraction(1)], 4: [Fraction(9, 8), Fraction(-1, 24)],
             8: [Fraction(1225, 1024), Fraction(-245, 3072), Fraction(49, 5120),
                 Fraction(-5, 7168)]}
    for so, v in exp_c.items():
        np.testing.assert_allclose(oracle.weights_centred(so), [float(f) for f in v],
                                   rtol=1e-13, atol=1e-15)
    for so, v in exp_b.items():
        np.testing.assert_allclose(oracle.weights_staggered(so), [float(f) for f in v],
                                   rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("so", [2, 4, 8, 12])
def test_exact_on_polynomials(so):
    """Interior exactness: D x^p = p x^(p-1) for p <= so (centred), and the
    staggered pair differentiates polynomials of degree <= so exactly."""
    n, h = 40, 0.7
    M = so // 2
    x = np.arange(n) * h
    for p in range(0, so + 1):
        f = (x / 10.0) ** p
        d = oracle.line_op("D", so, h, f)
        exact = p * (x / 10.0) ** max(p - 1, 0) / 10.0 if p else 0 * x
        sl = slice(M, n - M)
        np.testing.assert_allclose(d[sl], exact[sl], rtol=1e-9, atol=1e-11)
        # node -> half: derivative at x + h/2
        dp = oracle.line_op("Dp", so, h, f)
        xh = x + 0.5 * h
        exh = p * (xh / 10.0) ** max(p - 1, 0) / 10.0 if p else 0 * x
        slp = slice(M - 1, n - M)
        np.testing.assert_allclose(dp[slp], exh[slp], rtol=1e-9, atol=1e-11)
        # half -> node: values at x + h/2 stored at index i
        g = (xh / 10.0) ** p
        dm = oracle.line_op("Dm", so, h, g)
        slm = slice(M, n - M + 1)
        np.testing.assert_allclose(dm[slm], exact[slm], rtol=1e-9, atol=1e-11)


def _matrix(name, so, n, h=1.3):
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = oracle.line_op(name, so, h, e)
    return A


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
def test_antisymmetry_and_literal_transposes(so):
    n = 23
    D = _matrix("D", so, n)
    DT = _matrix("DT", so, n)
    Dp = _matrix("Dp", so, n)
    Dm = _matrix("Dm", so, n)
    DpT = _matrix("DpT", so, n)
    DmT = _matrix("DmT", so, n)
    np.testing.assert_allclose(DT, D.T, atol=1e-15)
    np.testing.assert_allclose(D.T, -D, atol=1e-15)          # zero extension => D^T = -D
    np.testing.assert_allclose(DpT, Dp.T, atol=1e-15)
    np.testing.assert_allclose(DmT, Dm.T, atol=1e-15)
    np.testing.assert_allclose(Dp.T, -Dm, atol=1e-15)        # (D+)^T = -D-


def _golden_weights():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "fd_weights.txt")
    rows = []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            kind, so, *w = line.split()
            rows.append((kind, int(so), [Fraction(v) for v in w]))
    return rows


@pytest.mark.parametrize("row", _golden_weights(), ids=lambda r: f"{r[0]}{r[1]}")
def test_golden_weights(row):
    """The oracle's weights equal the published rational values
    (tests/golden/fd_weights.txt, sources cited there) to FP64 rounding."""
    kind, so, w = row
    got = oracle.weights_centred(so) if kind == "centred" else oracle.weights_staggered(so)
    assert len(got) == len(w)
    for a, b in zip(got, w):
        assert abs(a - float(b)) <= 2e-16 * max(1.0, abs(float(b))) * 8, (kind, so, a, b)

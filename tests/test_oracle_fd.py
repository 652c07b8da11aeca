"""Pins for the oracle's finite-difference operator (Section 3.1, Eq. FD:Laplacian).

Independent references: the textbook table of centred FD coefficients
(tests/golden/fd_weights_order12.txt), exactness on polynomials, and the
Fourier symbol of the stencil."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd_weights_order12.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        d, num, den = (int(t) for t in line.split())
        out[d] = Fraction(num, den)
    return out


@pytest.mark.parametrize("h", [1.0, 0.478125, 0.3])
def test_weights_match_textbook_table(h):
    g = _golden()
    w = oracle.fd_weights(6, h)
    assert abs(2 * w[0] * h * h - float(g[0])) < 1e-14
    for d in range(1, 7):
        assert abs(w[d] * h * h - float(g[d])) < 1e-14 * max(1.0, abs(float(g[d])))


@pytest.mark.parametrize("no", [1, 2, 4, 6])
def test_1d_stencil_exact_on_polynomials(no):
    """A 2n_o-order central second difference is exact for degree <= 2n_o+1."""
    h = 0.37
    w = oracle.fd_weights(no, h)
    x0 = 0.81
    for k in range(0, 2 * no + 2):
        f = lambda x: x ** k
        approx = 2 * w[0] * f(x0) + sum(w[d] * (f(x0 + d * h) + f(x0 - d * h)) for d in range(1, no + 1))
        exact = k * (k - 1) * x0 ** (k - 2) if k >= 2 else 0.0
        scale = max(1.0, abs(exact), sum(abs(w[d]) * (abs(x0) + no * h) ** k for d in range(no + 1)))
        assert abs(approx - exact) < 1e-11 * scale, (k, approx, exact)
    # degree 2n_o+2 is NOT exact: the order is exactly 2n_o
    k = 2 * no + 2
    f = lambda x: x ** k
    approx = 2 * w[0] * f(x0) + sum(w[d] * (f(x0 + d * h) + f(x0 - d * h)) for d in range(1, no + 1))
    assert abs(approx - k * (k - 1) * x0 ** (k - 2)) > 1e-9


def test_symbol_small_theta():
    """-sum_d w_d 2cos(d theta) h^2 - 2 w_0 h^2 = theta^2 + O(theta^14)."""
    h = 0.478125
    w = oracle.fd_weights(6, h)
    for th in [1e-2, 0.1, 0.3]:
        s = -(2 * w[0] + 2 * sum(w[d] * math.cos(d * th) for d in range(1, 7))) * h * h
        assert abs(s - th * th) < 1e-12 + 10 * th ** 14
    s_pi = -(2 * w[0] + 2 * sum(w[d] * math.cos(d * math.pi) for d in range(1, 7)))
    assert 30.9 < s_pi < 31.0   # top of the 1-D symbol at h = 0.478125, bohr^-2


def test_3d_kinetic_exact_on_polynomial():
    """H_q with V = 0 and no projectors equals -1/2 Lap on a cubic polynomial
    at every region point at least n_o away from the Dirichlet faces."""
    n, m, h = 32, 9, 0.41
    V = np.zeros((n, n, n))
    osys = oracle.OracleSystem(V, h, m)
    S = 2 * m + 1
    c = np.arange(S) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = X ** 3 * Y - 2 * Y ** 2 * Z ** 2 + X * Y * Z + 5 * Z ** 4
    lap = 6 * X * Y - 4 * Z ** 2 - 4 * Y ** 2 + 60 * Z ** 2
    y = osys.apply_H(0, f.ravel()).reshape(S, S, S)
    inner = (slice(6, S - 6),) * 3
    np.testing.assert_allclose(y[inner], -0.5 * lap[inner], rtol=0, atol=1e-9 * np.abs(f).max() / h ** 2)
    # at the faces the stencil is truncated (zero Dirichlet): not equal there
    assert np.abs(y[0] - (-0.5 * lap[0])).max() > 1e-3


@pytest.mark.parametrize("no", [1, 2, 4, 6])
def test_gradient_weights_exact_on_polynomials(no):
    """The central difference of order 2 n_o (Eq. FD:Gradient) differentiates
    every polynomial of degree <= 2 n_o exactly, and misses x^(2 n_o + 1)."""
    h, x0 = 0.37, 0.8
    wt = oracle.grad_weights(no, h)
    assert wt[0] == 0.0
    for k in range(2 * no + 2):
        f = lambda x: x ** k
        approx = sum(wt[d] * (f(x0 + d * h) - f(x0 - d * h)) for d in range(1, no + 1))
        exact = k * x0 ** (k - 1) if k else 0.0
        if k <= 2 * no:
            assert abs(approx - exact) <= 1e-10 * max(1.0, abs(exact))
        else:
            assert abs(approx - exact) > 1e-8


def test_gradient_weights_converge_at_order_2no():
    """On sin(x) the error falls as h^(2 n_o): halving h divides it by ~2^12 for n_o = 6."""
    x0 = 0.3
    errs = []
    for h in (0.4, 0.2):
        wt = oracle.grad_weights(6, h)
        approx = sum(wt[d] * (np.sin(x0 + d * h) - np.sin(x0 - d * h)) for d in range(1, 7))
        errs.append(abs(approx - np.cos(x0)))
    assert 2 ** 11 < errs[0] / errs[1] < 2 ** 13

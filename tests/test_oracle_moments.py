"""Pins for the oracle's Chebyshev moments (Section 3.2, Eqs. Rec:FD, rhoqj)
and Lanczos bounds (Section 3.2).

Independent references: dense eigendecomposition of H_q, closed forms for
rho^0..rho^2, the infinite-lattice (Brillouin-zone) value of the free-electron
moments, and numpy's tridiagonal eigenvalues."""

import numpy as np
import pytest

import oracle
import synth


def _sys(n=16, m=4, nonlocal_=False, cells=1, seed=11, sigma=0.15):
    pos = synth.fcc_positions(cells, sigma, seed)
    L = synth.LATTICE_A * cells
    V = synth.local_potential(n, L, pos)
    return oracle.OracleSystem(V, L / n, m, pos, synth.projector_types(nonlocal_))


def _cheb_T(j, x):
    return np.cos(j * np.arccos(np.clip(x, -1, 1)))


@pytest.mark.parametrize("nonlocal_", [False, True])
def test_moments_match_dense_eigendecomposition(nonlocal_):
    osys = _sys(m=4, nonlocal_=nonlocal_)
    q = 1234
    H = osys.dense_H(q)
    lam, vec = np.linalg.eigh(H)
    chi = 0.5 * (lam[-1] + lam[0]) + 0.3
    zeta = 0.5 * (lam[-1] - lam[0]) * 1.05
    S = 2 * osys.m + 1
    c = osys.m + S * (osys.m + S * osys.m)
    w2 = vec[c, :] ** 2
    lh = (lam - chi) / zeta
    npl = 40
    expect = np.array([np.sum(w2 * _cheb_T(j, lh)) for j in range(npl + 1)])
    for pr in (False, True):
        mom = osys.moments([q], [chi], [zeta], npl, product_rule=pr)[0]
        np.testing.assert_allclose(mom, expect, rtol=0, atol=1e-12)


def test_product_rule_equals_direct_recurrence():
    osys = _sys(m=5, nonlocal_=True, n=16)
    nodes = [0, 77, 4095]
    chi, zeta = osys.bounds(nodes, 40, 0.01)
    a = osys.moments(nodes, chi, zeta, 48, product_rule=False)
    b = osys.moments(nodes, chi, zeta, 48, product_rule=True)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_low_moments_closed_form():
    """rho^0 = 1, rho^1 = (H_cc - chi)/zeta, rho^2 = 2 |Hhat e_c|^2 - 1."""
    osys = _sys(m=4, nonlocal_=True)
    q = 999
    H = osys.dense_H(q)
    S = 9
    c = 4 + S * (4 + S * 4)
    chi, zeta = 21.7, 24.9
    mom = osys.moments([q], [chi], [zeta], 8)[0]
    col = H[:, c].copy()
    col[c] -= chi
    col /= zeta
    assert mom[0] == 1.0
    assert abs(mom[1] - (H[c, c] - chi) / zeta) < 1e-14
    assert abs(mom[2] - (2 * col @ col - 1)) < 1e-13


def test_moments_bounded_by_one_with_lanczos_bounds(synth_cache):
    s = synth_cache("al4_16")
    osys = oracle.OracleSystem.from_synth(s)
    nodes = synth.sample_nodes(s.wl.n_nodes, 6)
    chi, zeta = osys.bounds(nodes, s.wl.n_lanczos, s.wl.margin)
    mom = osys.moments(nodes, chi, zeta, s.wl.npl)
    assert np.all(np.abs(mom) <= 1 + 1e-12)
    assert np.all(mom[:, 0] == 1.0)


def test_free_electron_moments_equal_brillouin_zone_integral():
    """V = 0 with n_o = 1 (second-order stencil): while t^a never reaches the
    Dirichlet faces (a <= m), rho^j for j <= 2m equals the infinite-lattice
    value (2pi)^-3 int T_j((sum_i s(theta_i)/2 - chi)/zeta) d^3theta, with
    s(theta) = (2 - 2cos theta)/h^2; the trapezoidal rule with more than
    j points per axis integrates this trigonometric polynomial exactly."""
    h, m, n = 0.5, 8, 20
    osys = oracle.OracleSystem(np.zeros((n, n, n)), h, m, fd_half_order=1)
    chi, zeta = 6.0 / h ** 2 * 0.5 + 0.1, 6.0 / h ** 2 * 0.5 + 0.2
    npl = 2 * m
    mom = osys.moments([0], [chi], [zeta], npl)[0]
    P = 4 * npl + 4
    th = 2 * np.pi * np.arange(P) / P
    s = (2 - 2 * np.cos(th)) / h ** 2
    E = 0.5 * (s[:, None, None] + s[None, :, None] + s[None, None, :])
    x = (E - chi) / zeta
    bz = np.array([_cheb_T(j, x).mean() for j in range(npl + 1)])
    np.testing.assert_allclose(mom, bz, rtol=0, atol=1e-12)
    # with one more moment the boundary is felt and agreement breaks
    mom2 = osys.moments([0], [chi], [zeta], npl + 4)[0]
    bz2 = np.array([_cheb_T(j, x).mean() for j in range(npl + 5)])
    assert abs(mom2[-1] - bz2[-1]) > 1e-8


def test_tridiag_extremes_match_numpy():
    rng = np.random.default_rng(5)
    for k in [1, 2, 7, 40]:
        a = rng.normal(size=k) * 10
        b = np.abs(rng.normal(size=max(k - 1, 0))) + 0.1
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        ev = np.linalg.eigvalsh(T)
        lo, hi = oracle.tridiag_extremes(a, b)
        assert abs(lo - ev[0]) < 1e-12 * max(1, abs(ev[0]))
        assert abs(hi - ev[-1]) < 1e-12 * max(1, abs(ev[-1]))


def test_lanczos_ritz_values_converge_to_spectrum_edges():
    osys = _sys(m=6, nonlocal_=True)
    q = 321
    lam = np.linalg.eigvalsh(osys.dense_H(q))
    a, b = osys.lanczos_tridiag(q, 90)
    assert len(a) == 90
    lo, hi = oracle.tridiag_extremes(a, b)
    assert lo >= lam[0] - 1e-9 and hi <= lam[-1] + 1e-9      # Ritz values lie inside
    assert abs(lo - lam[0]) < 1e-8 and abs(hi - lam[-1]) < 1e-8
    # the default 40 steps + 1% margin enclose the spectrum
    chi, zeta = osys.bounds([q], 40, 0.01)
    assert chi[0] - zeta[0] < lam[0] and chi[0] + zeta[0] > lam[-1]


def test_lanczos_breakdown_on_one_point_region():
    """m = 0: H_q is 1x1; Lanczos stops after one step and the width floor of
    1 Ha keeps zeta > 0."""
    osys = oracle.OracleSystem(np.full((4, 4, 4), -0.7), 0.5, 0)
    a, b = osys.lanczos_tridiag(3, 10)
    assert len(a) == 1
    chi, zeta = osys.bounds([3], 10, 0.01)
    w = oracle.fd_weights(6, 0.5)
    d = -3 * w[0] - 0.7
    assert abs(chi[0] - d) < 1e-12 and abs(zeta[0] - 0.01) < 1e-12
    mom = osys.moments([3], chi, zeta, 8)[0]
    np.testing.assert_allclose(mom, [_cheb_T(j, 0.0) for j in range(9)], atol=1e-11)

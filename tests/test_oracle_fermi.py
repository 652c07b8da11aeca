"""Pins for the oracle's quadrature weights, Fermi level, density, band
energy and entropy (Section 3.2 Eqs. ElectronDensity, cqj; Section 3.3 Eqs.
Eband, d_q, Entropy, e_q).

Independent references: discrete orthogonality of Chebyshev polynomials,
dense diagonalisation of the periodic finite-difference Hamiltonian (the
periodic-region mode reduces SQ to e_q^T g(H) e_q), the free-electron
Brillouin-zone integral, and exact invariants."""

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
import synth


def _T(j, x):
    return np.cos(j * np.arccos(np.clip(x, -1, 1)))


def test_weights_reproduce_all_moments():
    """sum_k W_k T_j(x_k) = rho^j for every j <= npl (so sum_k W_k = rho^0)."""
    rng = np.random.default_rng(1)
    npl = 24
    mom = rng.uniform(-1, 1, size=(3, npl + 1))
    mom[:, 0] = 1.0
    W = oracle.cc_weights(mom)
    x = oracle.cheb_nodes(npl)
    np.testing.assert_allclose(x, np.cos(np.pi * (np.arange(npl + 1) + 0.5) / (npl + 1)), atol=1e-15)
    for j in range(npl + 1):
        np.testing.assert_allclose(W @ _T(j, x), mom[:, j], atol=1e-13)
    np.testing.assert_allclose(W.sum(axis=1), 1.0, atol=1e-13)


def _fd_periodic_dense(osys):
    N = osys.region_size
    return osys.dense_H(0)   # periodic mode: the region is the whole cell for every node


def _periodic_reference(osys, Ne, kT):
    """Exact finite-temperature answers from dense diagonalisation of H_per."""
    H = _fd_periodic_dense(osys)
    lam, vec = np.linalg.eigh(H)
    g = lambda mu: 1.0 / (1.0 + np.exp((lam - mu) / kT))
    mu = brentq(lambda mu: 2 * g(mu).sum() - Ne, lam[0] - 50 * kT, lam[-1] + 50 * kT, xtol=1e-14)
    gv = g(mu)
    h3 = osys.h ** 3
    rho = 2.0 / h3 * (vec ** 2 @ gv)
    eb = 2 * np.sum(lam * gv)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(gv > 0, gv * np.log(gv), 0) + np.where(gv < 1, (1 - gv) * np.log1p(-gv), 0)
    es = 2 * kT * np.sum(s)
    return mu, rho, eb, es


def test_periodic_mode_converges_to_dense_diagonalisation():
    """With the region = the periodic cell, SQ is e_q^T p(H) e_q with p the
    Chebyshev interpolant of g; at high degree it must agree with the exact
    diagonalisation (density, Fermi level, band energy, entropy)."""
    n, cells = 10, 1
    pos = synth.fcc_positions(cells, 0.1, 4)
    L = synth.LATTICE_A
    V = synth.local_potential(n, L, pos)
    osys = oracle.OracleSystem(V, L / n, 0, pos, synth.projector_types(True), periodic=True)
    Ne, kT = 12.0, 0.5
    mu_ex, rho_ex, eb_ex, es_ex = _periodic_reference(osys, Ne, kT)
    errs = []
    for npl in (40, 80, 160):
        r = oracle.solve(osys, npl, kT, Ne, n_lanczos=60, margin=0.01)
        errs.append(np.abs(r["rho"] - rho_ex).max() / rho_ex.max())
    assert errs[0] > errs[1] > errs[2]                 # exponential convergence in npl
    assert errs[2] < 1e-8
    assert abs(r["mu"] - mu_ex) < 1e-7
    assert abs(r["e_band"] - eb_ex) < 1e-6 * abs(eb_ex)
    assert abs(r["e_ent"] - es_ex) < 1e-6 * abs(es_ex)
    assert abs(r["n_elec"] - Ne) < 1e-9 * Ne


def test_periodic_mode_matches_dense_diagonalisation_at_16_cubed():
    """al4_16's grid and potential (16^3, the 4096 x 4096 periodic H, kT 0.1,
    12 electrons, no projectors).  mu from the dense spectrum; the periodic-
    region SQ density at seeded nodes tends to (2/h^3) sum_n |psi_n(q)|^2
    g(lambda_n) as the degree grows: the Chebyshev interpolant of g converges
    geometrically, to rounding at n_pl = 800 on a spectrum ~47 Ha wide."""
    s = synth.make_system("al4_16")
    wl = s.wl
    osys = oracle.OracleSystem(s.V, wl.h, 0, s.positions, (), periodic=True)
    lam, vec = np.linalg.eigh(osys.dense_H(0))
    assert lam.size == 4096
    kT, Ne = wl.kT, wl.n_electrons
    g = lambda mu: 1.0 / (1.0 + np.exp((lam - mu) / kT))  # noqa: E731
    mu = brentq(lambda mu: 2 * g(mu).sum() - Ne, lam[0] - 50 * kT, lam[-1] + 50 * kT, xtol=1e-14)
    nodes = synth.sample_nodes(wl.n_nodes, 6, seed=11)
    exact = 2.0 / wl.h ** 3 * (vec[nodes] ** 2 @ g(mu))
    chi, zeta = osys.bounds(nodes, 80, 0.01)
    assert np.all(chi - zeta < lam[0]) and np.all(chi + zeta > lam[-1])       # the bounds enclose the spectrum
    errs = []
    for npl in (200, 400, 800):
        W = oracle.cc_weights(osys.moments(nodes, chi, zeta, npl))
        rho, *_ = oracle.density_energy(W, chi, zeta, mu, kT, wl.h)
        errs.append(np.abs(rho - exact).max() / exact.max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-6 and errs[2] < 1e-11


def test_infinite_cell_density_matches_dense_nodal_matrix():
    """e_q^T g(H_q) e_q from the dense nodal matrix (same chi, zeta, mu)."""
    n = 16
    pos = synth.fcc_positions(1, 0.1, 1708)
    V = synth.local_potential(n, synth.LATTICE_A, pos)
    h = synth.LATTICE_A / n
    osys = oracle.OracleSystem(V, h, 5, pos, synth.projector_types(True))
    q, kT, mu = 100, 0.2, 0.3
    chi, zeta = osys.bounds([q], 60, 0.01)
    lam, vec = np.linalg.eigh(osys.dense_H(q))
    c = 5 + 11 * (5 + 11 * 5)
    exact = 2.0 / h ** 3 * np.sum(vec[c] ** 2 / (1 + np.exp((lam - mu) / kT)))
    prev = None
    for npl in (60, 120, 240):
        mom = osys.moments([q], chi, zeta, npl)
        W = oracle.cc_weights(mom)
        rho, *_ = oracle.density_energy(W, chi, zeta, mu, kT, h)
        err = abs(rho[0] - exact) / exact
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-7


def test_free_electron_fermi_level_matches_bz_integral():
    """V = 0: every node is equivalent, N(mu) = N_d * (one node's count); as
    R_cut and npl grow the SQ Fermi level tends to the root of the
    Brillouin-zone integral N_e/N_d = 2 (2pi)^-3 int g(sum s(theta_i)/2) d^3theta."""
    h, kT = 0.5, 0.3
    w = oracle.fd_weights(6, h)
    n_nodes = 1000
    Ne = 0.02 * n_nodes * h ** 3 * 2 / 2      # electrons per node volume
    P = 96
    th = 2 * np.pi * (np.arange(P) + 0.5) / P
    s = -(2 * w[0] + 2 * sum(w[d] * np.cos(d * th) for d in range(1, 7)))
    E = 0.5 * (s[:, None, None] + s[None, :, None] + s[None, None, :]).ravel()
    count = lambda mu: 2 * np.mean(1 / (1 + np.exp((E - mu) / kT))) * n_nodes
    mu_bz = brentq(lambda mu: count(mu) - Ne, -5, 50, xtol=1e-14)
    errs = []
    for m, npl in [(6, 40), (12, 80), (18, 120)]:
        osys = oracle.OracleSystem(np.zeros((4, 4, 4)), h, m)
        chi, zeta = osys.bounds([0], 60, 0.01)
        mom = osys.moments([0], chi, zeta, npl)
        W = np.repeat(oracle.cc_weights(mom), n_nodes, axis=0)
        mu, _ = oracle.fermi_level(W, np.repeat(chi, n_nodes), np.repeat(zeta, n_nodes), Ne, kT)
        errs.append(abs(mu - mu_bz))
    assert errs[0] > errs[2]
    assert errs[2] < 2e-3


def test_shift_invariance_of_density_and_energies():
    """V -> V + c: chi -> chi + c, moments unchanged, mu -> mu + c, rho and
    E_ent unchanged, E_band -> E_band + c N_e."""
    n = 12
    pos = synth.fcc_positions(1, 0.1, 9)
    V = synth.local_potential(n, synth.LATTICE_A, pos)
    h = synth.LATTICE_A / n
    c, Ne, kT, npl = 0.625, 12.0, 0.1, 24
    pt = synth.projector_types(True)
    a = oracle.solve(oracle.OracleSystem(V, h, 3, pos, pt), npl, kT, Ne, 30, 0.01)
    b = oracle.solve(oracle.OracleSystem(V + c, h, 3, pos, pt), npl, kT, Ne, 30, 0.01)
    np.testing.assert_allclose(b["chi"], a["chi"] + c, atol=1e-10)
    np.testing.assert_allclose(b["zeta"], a["zeta"], atol=1e-10)
    np.testing.assert_allclose(b["moments"], a["moments"], atol=1e-10)
    assert abs(b["mu"] - (a["mu"] + c)) < 1e-9
    np.testing.assert_allclose(b["rho"], a["rho"], rtol=1e-8)
    assert abs(b["e_band"] - (a["e_band"] + c * Ne)) < 1e-8
    assert abs(b["e_ent"] - a["e_ent"]) < 1e-8


def test_electron_count_limits_and_conservation():
    n = 8
    pos = synth.fcc_positions(1, 0.1, 2)
    V = synth.local_potential(n, synth.LATTICE_A, pos)
    h = synth.LATTICE_A / n
    osys = oracle.OracleSystem(V, h, 2)
    r = oracle.solve(osys, 16, 0.1, 12.0, 20, 0.01)
    W, chi, zeta = r["W"], r["chi"], r["zeta"]
    # g = 1 everywhere (mu far above the spectrum) gives 2 N_d
    assert abs(oracle.electron_count(W, chi, zeta, 1e6, 0.1) - 2 * n ** 3) < 1e-9 * n ** 3
    assert abs(oracle.electron_count(W, chi, zeta, -1e6, 0.1)) < 1e-12
    assert abs(r["n_elec"] - 12.0) < 1e-10
    assert abs(h ** 3 * r["rho"].sum() - 12.0) < 1e-10
    assert r["e_ent"] <= 0.0


def test_fermi_level_rejects_unreachable_electron_count():
    mom = np.zeros((2, 9)); mom[:, 0] = 1
    W = oracle.cc_weights(mom)
    with pytest.raises(ValueError):
        oracle.fermi_level(W, np.zeros(2), np.ones(2), 4.5, 0.1)   # > 2 N_d

"""Pins of the SCF-loop oracle (oracle/scf_oracle.c): the periodic
finite-difference Laplacian and Poisson solve of Eq. (PoissonEqn), Slater
X-alpha exchange, Anderson mixing, and the SCF loop around the SQ path.

Independent references: the discrete Fourier symbol of the FD operator (the
exact solution of the periodic Poisson problem is a division in Fourier
space), the continuum derivative of a smooth periodic function, the
derivative of the exchange energy, the finite termination of Anderson mixing
on linear fixed-point maps (its equivalence to GMRES), and an SCF built on
dense diagonalisation with plain linear mixing (a fixed point does not depend
on how it is reached)."""
import numpy as np
from scipy.optimize import brentq

import oracle
import synth


def _symbol(n, h, no=6):
    """Discrete Fourier symbol of -lap_h on a periodic n^3 grid (3-D array)."""
    w = oracle.fd_weights(no, h)
    th = 2 * np.pi * np.fft.fftfreq(n)
    s1 = -(2 * w[0] + 2 * sum(w[d] * np.cos(d * th) for d in range(1, no + 1)))
    return s1[:, None, None] + s1[None, :, None] + s1[None, None, :]


def test_laplacian_is_the_fd_stencil_in_fourier_space():
    rng = np.random.default_rng(0)
    n, h = 11, 0.55
    x = rng.standard_normal((n, n, n))
    y = oracle.laplacian_periodic(x, h)
    y_ref = np.real(np.fft.ifftn(np.fft.fftn(x) * _symbol(n, h)))
    np.testing.assert_allclose(y, y_ref, atol=1e-11)


def test_laplacian_of_a_smooth_periodic_function():
    """12th-order accuracy on sin(2 pi x/L) sin(4 pi y/L) cos(2 pi z/L)."""
    n, L = 24, 7.65
    h = L / n
    g = np.arange(n) * h
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    k1, k2, k3 = 2 * np.pi / L, 4 * np.pi / L, 2 * np.pi / L
    f = np.sin(k1 * x) * np.sin(k2 * y) * np.cos(k3 * z)
    np.testing.assert_allclose(oracle.laplacian_periodic(f, h), (k1 ** 2 + k2 ** 2 + k3 ** 2) * f, atol=2e-9)


def test_poisson_is_the_exact_discrete_solve():
    """CG reaches the Fourier-space solution of -(1/4pi) lap_h phi = rho - mean(rho);
    phi has zero mean and does not see a constant added to rho."""
    rng = np.random.default_rng(1)
    n, h = 10, 0.7
    rho = rng.uniform(0.0, 0.1, size=(n, n, n))
    phi, it, res = oracle.poisson(rho, h, tol=1e-13)
    S = _symbol(n, h)
    S[0, 0, 0] = 1.0
    P = 4 * np.pi * np.fft.fftn(rho - rho.mean()) / S
    P[0, 0, 0] = 0.0
    np.testing.assert_allclose(phi, np.real(np.fft.ifftn(P)), atol=1e-11)
    assert res <= 1e-13 and 0 < it < n ** 3
    assert abs(phi.mean()) < 1e-13
    phi2, _, _ = oracle.poisson(rho + 0.37, h, tol=1e-13)
    np.testing.assert_allclose(phi2, phi, atol=1e-11)
    zero, _, _ = oracle.poisson(np.full((4, 4, 4), 0.2), h)      # neutral: phi = 0 up to rounding
    assert np.abs(zero).max() < 1e-14


def test_kerker_is_its_fourier_symbol():
    """(-lap_h + a k0^2)(-lap_h + k0^2)^-1 is the multiplier (S + a k0^2)/(S + k0^2)
    in Fourier space; the mean is scaled by exactly a."""
    rng = np.random.default_rng(11)
    n, h = 9, 0.6
    f = rng.standard_normal((n, n, n)) + 0.4
    for k0, a in ((1.0, 0.1), (0.5, 1.0), (2.0, 0.3)):
        y, it = oracle.kerker(f, h, k0, a, tol=1e-13)
        S = _symbol(n, h)
        ref = np.real(np.fft.ifftn(np.fft.fftn(f) * (S + a * k0 ** 2) / (S + k0 ** 2)))
        np.testing.assert_allclose(y, ref, atol=1e-11 * np.abs(f).max())
        assert abs(y.mean() - a * f.mean()) < 1e-12 and 0 < it < n ** 3
    np.testing.assert_allclose(oracle.kerker(f, h, 1.0, 1.0)[0], f, atol=1e-11)      # a = 1: identity


def test_xalpha_is_the_derivative_of_the_exchange_energy():
    """v_x = d e_x / d rho with e_x = -(9 alpha/8)(3/pi)^(1/3) rho^(4/3);
    alpha = 2/3 gives the uniform-gas exchange -(3 rho/pi)^(1/3)."""
    rho = np.array([1e-4, 0.003, 0.02, 0.1, 0.7])
    for alpha in (2.0 / 3.0, 0.7):
        e = lambda r: -(9 * alpha / 8) * (3 / np.pi) ** (1 / 3) * r ** (4 / 3)
        d = 1e-6 * rho
        np.testing.assert_allclose(oracle.xalpha(rho, alpha), (e(rho + d) - e(rho - d)) / (2 * d), rtol=1e-8)
    np.testing.assert_allclose(oracle.xalpha(rho), -(3 * rho / np.pi) ** (1 / 3), rtol=1e-14)
    assert np.all(oracle.xalpha(np.array([0.0, -1e-3])) == 0.0)


def test_anderson_without_history_is_simple_mixing():
    rng = np.random.default_rng(2)
    x, f = rng.standard_normal((1, 9)), rng.standard_normal((1, 9))
    np.testing.assert_allclose(oracle.anderson_step(x, f, 0.3), x[0] + 0.3 * f[0], atol=1e-15)


def test_anderson_terminates_on_a_linear_map():
    """For g(x) = G x + c in n dimensions, Anderson mixing with the whole
    history is GMRES on (I - G) x = c: the residual vanishes within n + 1
    steps, while simple mixing has barely started."""
    rng = np.random.default_rng(3)
    n = 6
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    G = Q @ np.diag(np.linspace(-0.9, 0.95, n)) @ Q.T
    c = rng.standard_normal(n)
    x_star = np.linalg.solve(np.eye(n) - G, c)
    Xs, Fs = [], []
    x = np.zeros(n)
    for k in range(n + 2):
        f = G @ x + c - x
        Xs.append(x.copy())
        Fs.append(f)
        x = oracle.anderson_step(np.array(Xs), np.array(Fs), 0.5)
    assert np.linalg.norm(x - x_star) < 1e-9 * np.linalg.norm(x_star)
    y = np.zeros(n)
    for k in range(n + 2):
        y = y + 0.5 * (G @ y + c - y)
    assert np.linalg.norm(y - x_star) > 1e-3 * np.linalg.norm(x_star)


def _dense_scf(V_loc, h, Ne, kT, tol=1e-11, beta=0.4, max_iter=400):
    """Reference SCF: dense diagonalisation of the periodic H, FFT Poisson
    solve, exchange formula, plain linear mixing."""
    n = V_loc.shape[0]
    S = _symbol(n, h)
    S[0, 0, 0] = 1.0
    V = V_loc.copy()
    for _ in range(max_iter):
        H = oracle.OracleSystem(V, h, 0, periodic=True).dense_H(0)
        lam, vec = np.linalg.eigh(H)
        g = lambda mu: 1.0 / (1.0 + np.exp((lam - mu) / kT))
        mu = brentq(lambda mu: 2 * g(mu).sum() - Ne, lam[0] - 50 * kT, lam[-1] + 50 * kT, xtol=1e-14)
        rho = (2.0 / h ** 3 * (vec ** 2 @ g(mu))).reshape(V.shape)
        P = 4 * np.pi * np.fft.fftn(rho - rho.mean()) / S
        P[0, 0, 0] = 0.0
        V_out = V_loc + np.real(np.fft.ifftn(P)) - (3 * np.maximum(rho, 0) / np.pi) ** (1 / 3)
        if np.linalg.norm(V_out - V) <= tol * np.linalg.norm(V_out):
            return V, rho, mu
        V = V + beta * (V_out - V)
    raise AssertionError("reference SCF did not converge")


def test_scf_reaches_the_dense_diagonalisation_fixed_point():
    """Periodic-region SQ (region = cell) at high degree, CG Poisson,
    X-alpha and Anderson mixing converge to the fixed point of the dense
    reference SCF (6^3 grid, one FCC cell, local potential, kT = 0.5; both
    sides use the same discretisation, so a coarse grid pins the loop)."""
    n = 6
    L = synth.LATTICE_A
    h = L / n
    pos = synth.fcc_positions(1, 0.1, 5)
    V_loc = synth.local_potential(n, L, pos)
    Ne, kT = 12.0, 0.5
    V_ref, rho_ref, mu_ref = _dense_scf(V_loc, h, Ne, kT)
    # the fixed point depends neither on the preconditioner nor on the mixing schedule
    for kerker, period in ((None, 1), ((1.0, 0.2), 1), (None, 3)):
        r = oracle.scf(V_loc, h, 0, pos, (), Ne, kT, npl=100, tol=1e-8, periodic=True, n_lanczos=60, kerker=kerker,
                       period=period)
        assert r["converged"] and r["iterations"] < 40
        assert r["residuals"][-1] <= 1e-8 < r["residuals"][0]
        np.testing.assert_allclose(r["V"], V_ref, atol=1e-6 * np.abs(V_ref).max())
        np.testing.assert_allclose(r["rho"], rho_ref, atol=1e-6 * rho_ref.max())
        assert abs(r["mu"] - mu_ref) < 1e-6
        assert abs(r["n_elec"] - Ne) < 1e-9 * Ne

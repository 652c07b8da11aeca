"""Pins of the oracle's nonlocal atomic force (Eq. Discrete:NLforce with the
recurrence of Eq. Rec:FD1 to n_pl): in periodic-region mode at high degree
SQ is exact diagonalisation, and the Hellmann-Feynman force at fixed mu is
-dOmega/dR_I of the grand potential Omega = -2 kT sum ln(1 + e^{-(e - mu)/kT})
of the discrete Hamiltonian, differentiated here by central differences of
dense eigenvalues while only the projectors move.  The projectors are made
wide and their support large (cut where they are 1e-8 of their peak) so that
neither the finite-difference gradient of the formula nor the moving
support boundary matters at the tested level.  A symmetric atom feels no
force."""
import numpy as np
from scipy.optimize import brentq

import oracle
import synth


def test_nl_force_is_the_derivative_of_the_grand_potential():
    n = 9
    L = synth.LATTICE_A
    h = L / n
    pos = synth.fcc_positions(1, 0.12, 11)[:2]
    V = synth.local_potential(n, L, pos)
    pt = [(0, 0.5, 2.5, 15.0), (1, -0.3, 2.5, 15.0)]
    kT, Ne = 0.4, 8.0

    def eig(R):
        return np.linalg.eigvalsh(oracle.OracleSystem(V, h, 0, R, pt, periodic=True).dense_H(0))

    lam = eig(pos)
    g = lambda mu: 1.0 / (1.0 + np.exp((lam - mu) / kT))
    mu = brentq(lambda m: 2 * g(m).sum() - Ne, lam[0] - 50 * kT, lam[-1] + 50 * kT, xtol=1e-14)
    omega = lambda R: -2 * kT * np.sum(np.logaddexp(0.0, -(eig(R) - mu) / kT))
    d = 1e-3
    fd = np.zeros((2, 3))
    for I in range(2):
        for a in range(3):
            Rp, Rm = pos.copy(), pos.copy()
            Rp[I, a] += d
            Rm[I, a] -= d
            fd[I, a] = -(omega(Rp) - omega(Rm)) / (2 * d)
    o = oracle.OracleSystem(V, h, 0, pos, pt, periodic=True)
    nodes = np.arange(n ** 3)
    chi, zeta = o.bounds(nodes, 80, 0.01)
    F = o.nl_force(nodes, chi, zeta, 100, mu, kT)
    assert np.abs(fd).max() > 1e-3                       # a force worth checking
    np.testing.assert_allclose(F, fd, atol=2e-4 * np.abs(fd).max())


def test_nl_force_vanishes_for_a_symmetric_atom():
    """One atom at the centre of a cubic cell, V = 0: inversion symmetry."""
    n = 8
    L = synth.LATTICE_A
    h = L / n
    pos = np.array([[L / 2, L / 2, L / 2]])
    o = oracle.OracleSystem(np.zeros((n, n, n)), h, 3, pos, synth.projector_types(True))
    nodes = np.arange(n ** 3)
    chi, zeta = o.bounds(nodes, 40, 0.01)
    F = o.nl_force(nodes, chi, zeta, 24, -0.5, 0.1)
    assert np.abs(F).max() < 1e-12

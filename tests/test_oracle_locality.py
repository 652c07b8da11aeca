"""Locality of the SQ density (the paper's convergence claim for the region
of influence: nodal quantities converge exponentially with R_cut, and
faster at higher temperature, because the density matrix decays
exponentially in real space at finite temperature).  The oracle's nodal
density at a fixed chemical potential, computed on regions of growing
half-width m, must settle geometrically, and faster at the higher kT."""
import numpy as np

import oracle
import synth


def _density_by_region(V, h, pos, nodes, kT, npl, ms):
    rhos = []
    for m in ms:
        o = oracle.OracleSystem(V, h, m, pos, ())
        chi, zeta = o.bounds(nodes, 60, 0.01)
        W = oracle.cc_weights(o.moments(nodes, chi, zeta, npl))
        rho, _, _, _ = oracle.density_energy(W, chi, zeta, 0.0, kT, h)   # same mu for every region
        rhos.append(rho)
    return np.array(rhos)


def test_density_converges_exponentially_with_region_size():
    n = 12
    L = synth.LATTICE_A
    h = L / n
    pos = synth.fcc_positions(1, 0.1, 6)
    V = synth.local_potential(n, L, pos)
    nodes = np.array([0, 100, 777], dtype=np.int64)
    ms = range(1, 8)                               # regions 3^3 .. 15^3
    d_hot = np.abs(np.diff(_density_by_region(V, h, pos, nodes, 1.0, 120, ms), axis=0)).max(axis=1)
    d_warm = np.abs(np.diff(_density_by_region(V, h, pos, nodes, 0.5, 200, ms), axis=0)).max(axis=1)
    assert np.all(np.diff(d_hot) < 0)              # every larger region changes the density less
    assert d_hot[-1] < 1e-5 * d_hot[0]             # ~ geometric: five orders over six steps
    assert d_hot[-1] < 1e-2 * d_warm[-1]           # the hotter system is the more local one
    assert d_warm[-1] < 1e-3 * d_warm[0]

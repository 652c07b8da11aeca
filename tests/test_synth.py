"""The seeded synthetic inputs shared by the oracle and the GPU path: the
named workloads have the stated sizes, the positions lie in the cell, the
local potential has the stated range and periodicity, and the seeds make
every system reproducible and the batch systems distinct."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("name,cells,n,atoms,m", [("al4_16", 1, 16, 4, 6), ("al108_48", 3, 48, 108, 12),
                                                  ("al32_32", 2, 32, 32, 12), ("al256_64", 4, 64, 256, 12),
                                                  ("al32_32_r7", 2, 32, 32, 14), ("al2048_128", 8, 128, 2048, 14)])
def test_named_workloads(name, cells, n, atoms, m):
    wl = synth.WORKLOADS[name]
    assert (wl.cells, wl.n, wl.n_atoms, wl.m) == (cells, n, atoms, m)
    assert abs(wl.h - 0.478125) < 1e-12 and wl.n_electrons == 3 * atoms
    s = synth.make_system(name)
    assert s.V.shape == (n, n, n) and s.positions.shape == (atoms, 3)
    assert np.all(s.positions >= 0) and np.all(s.positions < wl.L)
    assert -3.2 < s.V.min() < -2.5 and s.V.max() <= 0.0
    again = synth.make_system(name)
    assert np.array_equal(again.V, s.V) and np.array_equal(again.positions, s.positions)


def test_local_potential_is_periodic_and_translation_covariant():
    """Moving every atom by one grid step along x moves V by one node."""
    wl = synth.custom_workload("t", cells=1, n=12, sigma_disp=0.1, seed=3)
    pos = synth.fcc_positions(1, 0.1, 3)
    V = synth.local_potential(wl.n, wl.L, pos)
    V2 = synth.local_potential(wl.n, wl.L, np.mod(pos + [wl.h, 0, 0], wl.L))
    np.testing.assert_allclose(V2, np.roll(V, 1, axis=2), atol=1e-12)


def test_batch_systems_are_distinct_and_reproducible():
    a, b = synth.batch_workloads(), synth.batch_workloads()
    assert a == b and len(a) == 16 and len({w.seed for w in a}) == 16

"""The work counts bench.py divides by (no GPU): the nodes the force visits
and the mean number of projector supports covering a grid point, checked
against brute-force counts over every grid point and atom image."""
import itertools
import math
import os
import sys

import numpy as np

import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _cover_counts(wl, positions):
    """Number of (atom image) supports |x - R - L e| < r_nl covering each grid point."""
    n, h, L, rnl = wl.n, wl.h, wl.L, synth.PROJ_RNL
    g = np.arange(n) * h
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    cnt = np.zeros((n, n, n), dtype=int)
    reach = int(math.ceil(rnl / L)) + 1
    for R in positions:
        for e in itertools.product(range(-reach, reach + 1), repeat=3):
            d2 = (x - R[0] - e[0] * L) ** 2 + (y - R[1] - e[1] * L) ** 2 + (z - R[2] - e[2] * L) ** 2
            cnt += d2 < rnl * rnl
    return cnt


def test_touched_nodes_is_the_brute_force_count():
    for cells, n, seed in ((1, 10, 3), (2, 13, 4)):
        wl = synth.custom_workload("acc", cells=cells, n=n, r_cut=2.0, npl=8, kT=0.1, sigma_disp=0.3,
                                   nonlocal_=True, seed=seed)
        s = synth.make_system(wl)
        assert bench.touched_nodes(wl, s.positions) == int((_cover_counts(wl, s.positions) > 0).sum())


def test_supports_per_point_match_the_grid_count():
    """The continuum estimate n_atoms (4/3) pi r_nl^3 / L^3 used in the flop
    model is within 3 % of the exact grid average."""
    wl = synth.custom_workload("acc2", cells=2, n=32, r_cut=2.0, npl=8, kT=0.1, sigma_disp=0.15,
                               nonlocal_=True, seed=5)
    s = synth.make_system(wl)
    exact = _cover_counts(wl, s.positions).mean()
    assert abs(bench.nl_pairs_per_point(wl) - exact) <= 0.03 * exact

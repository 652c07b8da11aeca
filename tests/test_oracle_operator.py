"""Pins for the oracle's nodal Hamiltonian H_q (Section 3.1, region of
influence; Eq. Hamiltonian) including the Kleinman-Bylander projectors.

Independent references: symmetry, exact spectral shift, closed-form Gaussian
normalisation integrals (erf), parity of the p projectors, rank and inertia of
the nonlocal term, and translation covariance."""
import math

import numpy as np
from scipy.special import erf

import oracle
import synth


def _small_system(n=12, m=3, cells=1, nonlocal_=True, seed=3):
    pos = synth.fcc_positions(cells, 0.2, seed)
    L = synth.LATTICE_A * cells
    V = synth.local_potential(n, L, pos)
    pt = synth.projector_types(nonlocal_)
    return oracle.OracleSystem(V, L / n, m, pos, pt), pos, V, L / n


def test_dense_H_symmetric_with_projectors():
    osys, *_ = _small_system()
    H = osys.dense_H(17)
    assert osys.num_projectors(17) > 0
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-13 * np.abs(H).max())


def test_potential_shift_is_identity_shift():
    osys, pos, V, h = _small_system()
    c = 0.731
    o2 = oracle.OracleSystem(V + c, h, osys.m, pos, synth.projector_types(True))
    H1, H2 = osys.dense_H(5), o2.dense_H(5)
    np.testing.assert_allclose(H2 - H1, c * np.eye(H1.shape[0]), atol=1e-12)


def test_potential_change_moves_spectrum_within_its_max():
    """Weyl's inequality for the nodal Hamiltonian: changing V by dV moves
    every eigenvalue of H_q by at most max|dV| over the region, so bounds
    widened by max|dV| still enclose the spectrum (the reading behind reusing
    spectral bounds between SCF iterations).  Checked on dense H_q with
    projectors for a smooth and a rough change."""
    osys, pos, V, h = _small_system()
    rng = np.random.default_rng(17)
    for dV in (0.05 * np.sin(np.arange(V.size) * 0.37).reshape(V.shape), 0.2 * rng.standard_normal(V.shape)):
        o2 = oracle.OracleSystem(V + dV, h, osys.m, pos, synth.projector_types(True))
        for q in (0, 5, 17, 200):
            e1 = np.linalg.eigvalsh(osys.dense_H(q))
            e2 = np.linalg.eigvalsh(o2.dense_H(q))
            assert np.abs(e2 - e1).max() <= np.abs(dV).max() * (1 + 1e-12) + 1e-12
            assert e2.min() >= e1.min() - np.abs(dV).max() - 1e-12 and e2.max() <= e1.max() + np.abs(dV).max() + 1e-12


def _nonlocal_spectrum(h, R, pt, m, n):
    """Non-zero eigenvalues of the region-restricted V_nl = H - H(no projectors)
    at the node (m+1, m+1, m+1).  V_nl has rank <= 4 per atom, so a random
    block of 8 probes spans its range exactly: eig(Q^T V_nl Q) with
    Q = orth(V_nl Y) gives its non-zero spectrum without a dense matrix."""
    V = np.zeros((n, n, n))
    o1 = oracle.OracleSystem(V, h, m, np.atleast_2d(R), pt)
    o0 = oracle.OracleSystem(V, h, m)
    node = int((m + 1) + n * ((m + 1) + n * (m + 1)))
    Ns = o1.region_size
    vnl = lambda x: o1.apply_H(node, x) - o0.apply_H(node, x)
    Y = np.random.default_rng(0).normal(size=(Ns, 8))
    Z = np.stack([vnl(Y[:, i]) for i in range(8)], axis=1)
    U, s, _ = np.linalg.svd(Z, full_matrices=False)
    Q = U[:, s > 1e-10 * s[0]]
    T = Q.T @ np.stack([vnl(Q[:, i]) for i in range(Q.shape[1])], axis=1)
    return np.sort(np.linalg.eigvalsh(0.5 * (T + T.T))), o1.num_projectors(node)


def _one_atom(h, rnl=4.5, offset=(0.123, -0.071, 0.2)):
    m = int(math.ceil(rnl / h)) + 2
    n = 2 * m + 5
    R = (m + 1) * h * np.ones(3) + np.array(offset) * h
    return R, m, n


def test_projector_normalisation_matches_erf_closed_form():
    """With gamma = 1, trace(V_nl) = sum_p h^3 |chi_p|^2 ~ integral of chi_p^2
    over the support ball, which has a closed form through erf."""
    h, rc, rnl = 0.25, 1.5, 4.5
    R, m, n = _one_atom(h, rnl)
    ev, nproj = _nonlocal_spectrum(h, R, [(0, 1.0, rc, rnl), (1, 1.0, rc, rnl)], m, n)
    assert nproj == 4 and len(ev) == 4
    U = rnl / rc
    frac_s = erf(U) - 2.0 / math.sqrt(math.pi) * U * math.exp(-U * U)
    frac_p = (8.0 / (3.0 * math.sqrt(math.pi))) * (
        3.0 / 8.0 * math.sqrt(math.pi) * erf(U) - math.exp(-U * U) * (U ** 3 / 2.0 + 3.0 * U / 4.0))
    expected = frac_s + 3 * frac_p
    assert abs(ev.sum() - expected) < 2e-3 * expected, (ev.sum(), expected)


def test_nonlocal_rank_and_inertia():
    """V_nl = sum_p gamma_p h^3 chi_p chi_p^T: rank = #projectors, with as many
    positive eigenvalues as s channels (gamma_s > 0) and negative as p."""
    h = 0.45
    R, m, n = _one_atom(h, offset=(0.1, 0.05, -0.12))
    ev, nproj = _nonlocal_spectrum(h, R, synth.projector_types(True), m, n)
    assert nproj == 4 and len(ev) == 4
    assert (ev > 0).sum() == 1 and (ev < 0).sum() == 3


def test_p_projector_odd_and_orthogonal_to_s_on_grid():
    """Atom on a grid point: the support is symmetric, so <chi_s, chi_pa> = 0
    and <chi_pa, chi_pb> = 0 for a != b, and the three p eigenvalues of V_nl
    (gamma = 1) are exactly degenerate."""
    h = 0.5
    R, m, n = _one_atom(h, offset=(0.0, 0.0, 0.0))
    ev, nproj = _nonlocal_spectrum(h, R, [(0, 1.0, 1.5, 4.5), (1, 1.0, 1.5, 4.5)], m, n)
    assert len(ev) == 4
    gaps = np.diff(ev)
    # three equal p eigenvalues and one distinct s eigenvalue
    assert np.sum(gaps < 1e-10 * ev.max()) == 2


def test_translation_covariance():
    """Shifting V and the atoms by one grid vector maps H_q to H_{q+e}."""
    osys, pos, V, h = _small_system(n=12, m=3)
    n = 12
    Vs = np.roll(V, shift=(1, 2, 3), axis=(0, 1, 2))          # (z, y, x) rolls
    pos_s = np.mod(pos + h * np.array([3, 2, 1]), synth.LATTICE_A)
    o2 = oracle.OracleSystem(Vs, h, 3, pos_s, synth.projector_types(True))
    i, j, k = 4, 7, 9
    q = i + n * (j + n * k)
    q2 = (i + 3) % n + n * ((j + 2) % n + n * ((k + 1) % n))
    np.testing.assert_allclose(o2.dense_H(q2), osys.dense_H(q), atol=1e-11)


def test_region_larger_than_cell_uses_periodic_potential():
    """Infinite-cell mode: a region wider than the cell sees V periodically."""
    n, m = 6, 4
    rng = np.random.default_rng(0)
    V = rng.normal(size=(n, n, n))
    osys = oracle.OracleSystem(V, 0.5, m)
    H = osys.dense_H(0)
    S = 2 * m + 1
    diag = np.diag(H).reshape(S, S, S) - np.diag(H)[0]
    c = np.arange(-m, m + 1) % n
    Vr = V[np.ix_(c, c, c)]
    np.testing.assert_allclose(diag, Vr - Vr[0, 0, 0], atol=1e-12)


def test_projector_images_brute_force():
    """The nonlocal block of H_q equals a brute-force sum over every atom and
    every periodic image in a wide shell (region wider than the cell, so each
    atom contributes several images)."""
    n, cells, m = 8, 1, 6
    pos = synth.fcc_positions(cells, 0.2, 21)
    L = synth.LATTICE_A * cells
    h = L / n
    pt = synth.projector_types(True)
    V = np.zeros((n, n, n))
    o1 = oracle.OracleSystem(V, h, m, pos, pt)
    o0 = oracle.OracleSystem(V, h, m)
    q = 3 + n * (0 + n * 7)                    # a node next to two cell faces
    S = 2 * m + 1
    Ns = S ** 3
    rng = np.random.default_rng(2)
    x = rng.normal(size=Ns)
    got = o1.apply_H(q, x) - o0.apply_H(q, x)
    qi, qj, qk = 3, 0, 7
    a = np.arange(S) - m
    gx = (qi + a) * h
    gy = (qj + a) * h
    gz = (qk + a) * h
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    want = np.zeros(Ns)
    rc, rnl = synth.PROJ_RC, synth.PROJ_RNL
    As = (np.pi * rc * rc) ** -0.75
    Ap = np.sqrt(2.0) / rc * As
    for R in pos:
        for e in np.ndindex(7, 7, 7):
            Rs = R + L * (np.array(e) - 3)
            d = pts - Rs
            r2 = (d ** 2).sum(axis=1)
            inside = r2 < rnl * rnl
            if not inside.any():
                continue
            g = np.where(inside, np.exp(-r2 / (2 * rc * rc)), 0.0)
            chis = [(synth.GAMMA_S, As * g)] + [(synth.GAMMA_P, Ap * d[:, k] * g) for k in range(3)]
            for gam, chi in chis:
                want += gam * h ** 3 * chi * (chi @ x)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())

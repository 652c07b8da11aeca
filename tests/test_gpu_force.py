"""Nonlocal atomic forces on the GPU (sq_nl_forces) against the oracle's
or_nl_force (Eq. Discrete:NLforce with the recurrence of Eq. Rec:FD1 to
n_pl), which tests/test_oracle_force.py pins to the derivative of the grand
potential.

Tolerance: FP64, the same arithmetic in another summation order over a
recurrence of n_pl steps: 1e-10 of the largest force component, absolute.
Three kernel forms are run: the region form (the region kernels'
recurrence, the default; in FP32 its projector update adds with shared-
memory atomics, so its repeats agree to rounding rather than bit for bit)
and the first form with its vectors in global scratch or in shared memory.
FP32 context (recurrence, D and projector sums in FP32; coefficients and
contraction in FP64): 1e-4 of the largest component.  The rounding error of
the FP32 recurrence grows with the degree; the same arithmetic run on the
host gave at most 6e-6 at n_pl <= 12 and 2.3e-5 at n_pl = 260 on these
cases, and 1e-4 leaves a factor 4.
The spectral bounds and the Fermi level come from the oracle and are copied
to the GPU (never the reverse), so the comparison isolates the force path.
The whole GPU pipeline (its own bounds, moments and Fermi level) is compared
at 1e-6: the Lanczos bounds of the two sides agree to 1e-9 relative, and the
interpolation coefficients move with the interval."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQSolver, build, sq  # noqa: E402

build()
DEV = "cuda:0"
FP64_FORCE = 1e-10
FP32_FORCE = 1e-4


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(DEV)


def _system(n, r_cut, npl, kT, proj_types, seed, cells=1):
    wl = synth.custom_workload("force", cells=cells, n=n, r_cut=r_cut, npl=npl, kT=kT, sigma_disp=0.2,
                               nonlocal_=True, seed=seed)
    s = synth.make_system(wl)
    return wl, s, list(proj_types)


CASES = {
    # one FCC cell, 10^3 grid (a ragged 8^3 tile), m = 3, s + 3p projectors
    "sp_n10_m3": dict(n=10, r_cut=2.5, npl=12, kT=0.2, proj_types=synth.projector_types(True), seed=21),
    # s only / p only, 9^3 grid, m = 2
    "s_n9_m2": dict(n=9, r_cut=2.0, npl=8, kT=0.2, proj_types=synth.projector_types(True)[:1], seed=22),
    "p_n9_m2": dict(n=9, r_cut=2.0, npl=8, kT=0.2, proj_types=synth.projector_types(True)[1:], seed=23),
    # region (7^3) larger than the cell (6^3): several images of one atom per region
    "sp_n6_m3": dict(n=6, r_cut=4.0, npl=8, kT=0.2, proj_types=synth.projector_types(True), seed=24),
    # narrow supports: most nodes touch no projector; degree above the CTA width
    "narrow_n8_npl260": dict(n=8, r_cut=2.0, npl=260, kT=0.05,
                             proj_types=[(0, 0.5, 0.6, 1.3), (1, -0.3, 0.6, 1.3)], seed=25),
    # two cells per axis (32 atoms), 12^3 grid: tile lists longer than one chunk
    "sp_2cells_n12": dict(n=12, r_cut=4.0, npl=8, kT=0.2, proj_types=synth.projector_types(True), seed=26,
                          cells=2),
    # 108 atoms on a 10^3 grid: tile lists of up to 365 entries (more than one 256-entry chunk)
    "sp_3cells_n10": dict(n=10, r_cut=4.7, npl=8, kT=0.2, proj_types=synth.projector_types(True), seed=27,
                          cells=3),
}


def _form(monkeypatch, form):
    """The force kernel the library uses for the next call: the region form
    (the default), or the first form with every vector in global scratch
    (SQ_FORCE_KERNEL=legacy) or with the current vector in shared memory
    (and SQ_FORCE_SMEM=1); both variables are read at each call."""
    monkeypatch.delenv("SQ_FORCE_KERNEL", raising=False)
    monkeypatch.delenv("SQ_FORCE_SMEM", raising=False)
    if form != "region":
        monkeypatch.setenv("SQ_FORCE_KERNEL", "legacy")
    if form == "legacy_smem":
        monkeypatch.setenv("SQ_FORCE_SMEM", "1")


@pytest.mark.parametrize("form", ["region", "legacy_global", "legacy_smem"])
@pytest.mark.parametrize("precision", [SQ_FP64, SQ_FP32])
@pytest.mark.parametrize("name", list(CASES))
def test_nl_forces_match_oracle(name, precision, form, monkeypatch):
    _form(monkeypatch, form)
    wl, s, pt = _system(**CASES[name])
    osys = oracle.OracleSystem(s.V, wl.h, wl.m, s.positions, pt)
    nodes = np.arange(wl.n_nodes)
    chi, zeta = osys.bounds(nodes, 40, 0.02)
    mu = float(np.median(chi))
    F_ref = osys.nl_force(nodes, chi, zeta, wl.npl, mu, wl.kT)
    solver = SQSolver((wl.n,) * 3, wl.h, wl.r_cut, wl.npl, precision, s.positions, pt, device=DEV)
    F = solver.nl_forces(_dev(s.V), mu, wl.kT, chi=_dev(chi), zeta=_dev(zeta)).cpu().numpy()
    scale = np.abs(F_ref).max()
    assert scale > 1e-4
    tol = FP64_FORCE if precision == SQ_FP64 else FP32_FORCE
    np.testing.assert_allclose(F, F_ref, rtol=0, atol=tol * scale)
    F2 = solver.nl_forces(_dev(s.V), mu, wl.kT, chi=_dev(chi), zeta=_dev(zeta)).cpu().numpy()
    if precision == SQ_FP64 or form != "region":
        assert np.array_equal(F, F2)                               # fixed-order sums: repeats bit for bit
    else:                                                          # FP32 shared-memory atomics in the update
        assert np.abs(F - F2).max() <= 1e-5 * scale
    solver.close()


@pytest.mark.parametrize("name,precision,count,form", [("al108_48", SQ_FP64, 16, "region"),
                                                       ("al108_48", SQ_FP32, 16, "region"),
                                                       ("al108_48", SQ_FP32, 16, "legacy_global"),
                                                       ("al2048_128", SQ_FP32, 6, "region")])
def test_nl_forces_full_size_sampled_nodes(name, precision, count, form, monkeypatch):
    """Full-size workloads: al108_48 (the benchmark workload: 25^3 regions,
    n_pl 48, 108 atoms) and al2048_128 (the scale workload: 128^3 grid, 29^3
    regions, n_pl 64, 2048 atoms; FP32, as FP64 regions stop at 25^3), s + 3p.
    The force contributions of seeded nodes on the benchmark's launch
    configuration, against the oracle on the same nodes (the oracle's bounds
    and Fermi level on the GPU side)."""
    _form(monkeypatch, form)
    s = synth.make_system(name)
    wl = s.wl
    nodes = synth.sample_nodes(wl.n_nodes, count, seed=31)
    osys = oracle.OracleSystem.from_synth(s)
    chi, zeta = osys.bounds(nodes, wl.n_lanczos, wl.margin)
    mu = float(np.median(chi))
    F_ref = osys.nl_force(nodes, chi, zeta, wl.npl, mu, wl.kT)
    solver = SQSolver.from_workload(wl, s.positions, precision=precision, device=DEV)
    chi_all = torch.zeros(wl.n_nodes, dtype=torch.float64, device=DEV)
    zeta_all = torch.ones(wl.n_nodes, dtype=torch.float64, device=DEV)
    chi_all[torch.from_numpy(nodes).to(DEV)] = _dev(chi)
    zeta_all[torch.from_numpy(nodes).to(DEV)] = _dev(zeta)
    F = solver.nl_forces(_dev(s.V), mu, wl.kT, chi=chi_all, zeta=zeta_all,
                         nodes=torch.from_numpy(nodes).to(DEV)).cpu().numpy()
    scale = np.abs(F_ref).max()
    assert scale > 1e-5
    tol = FP64_FORCE if precision == SQ_FP64 else FP32_FORCE
    np.testing.assert_allclose(F, F_ref, rtol=0, atol=tol * scale)
    with pytest.raises(sq.SQError) as e:                                    # an index outside the grid
        bad = torch.tensor([0, wl.n_nodes], dtype=torch.int64, device=DEV)
        solver.nl_forces(_dev(s.V), mu, wl.kT, chi=chi_all, zeta=zeta_all, nodes=bad)
    assert e.value.code == sq.SQ_EINVAL
    solver.close()


def test_nl_forces_whole_pipeline():
    """GPU bounds, moments, Fermi level and forces vs the oracle's."""
    wl, s, pt = _system(**CASES["sp_n10_m3"])
    osys = oracle.OracleSystem(s.V, wl.h, wl.m, s.positions, pt)
    ref = oracle.solve(osys, wl.npl, wl.kT, wl.n_electrons, 40, 0.02)
    nodes = np.arange(wl.n_nodes)
    F_ref = osys.nl_force(nodes, ref["chi"], ref["zeta"], wl.npl, ref["mu"], wl.kT)
    solver = SQSolver((wl.n,) * 3, wl.h, wl.r_cut, wl.npl, SQ_FP64, s.positions, pt, device=DEV)
    V = _dev(s.V)
    out = solver.solve(V, wl.n_electrons, wl.kT, 40, 0.02)
    F = solver.nl_forces(V, out["mu"], wl.kT).cpu().numpy()
    np.testing.assert_allclose(F, F_ref, rtol=0, atol=1e-6 * np.abs(F_ref).max())
    solver.close()


def test_nl_forces_vanish_for_a_symmetric_atom():
    n = 8
    L = synth.LATTICE_A
    h = L / n
    pos = np.array([[L / 2, L / 2, L / 2]])
    solver = SQSolver((n,) * 3, h, 3 * h + 1e-9, 24, SQ_FP64, pos, synth.projector_types(True), device=DEV)
    V = torch.zeros(n ** 3, dtype=torch.float64, device=DEV)
    solver.bounds(V, 40, 0.01)
    F = solver.nl_forces(V, -0.5, 0.1).cpu().numpy()
    assert F.shape == (1, 3) and np.abs(F).max() < 1e-12
    solver.close()


def test_nl_forces_arguments():
    wl, s, pt = _system(**CASES["s_n9_m2"])
    V = _dev(s.V)
    solver = SQSolver((wl.n,) * 3, wl.h, wl.r_cut, wl.npl, SQ_FP64, s.positions, pt, device=DEV)
    solver.bounds(V, 40, 0.02)
    F = torch.zeros(3 * len(s.positions), dtype=torch.float64, device=DEV)
    with pytest.raises(sq.SQError) as e:                                       # kT <= 0
        sq.sq_nl_forces(solver.ctx, V, solver.chi, solver.zeta, 0.0, 0.0, F)
    assert e.value.code == sq.SQ_EINVAL
    with pytest.raises(sq.SQError) as e:                                       # forces missing
        sq.sq_nl_forces(solver.ctx, V, solver.chi, solver.zeta, 0.0, 0.1, None)
    assert e.value.code == sq.SQ_EINVAL
    solver.close()
    local = SQSolver((wl.n,) * 3, wl.h, wl.r_cut, wl.npl, SQ_FP64, s.positions, (), device=DEV)
    local.bounds(V, 40, 0.02)
    assert local.nl_forces(V, 0.0, 0.1).shape == (0, 3)                        # no projectors: no force
    local.close()

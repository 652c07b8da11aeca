"""The SCF loop's device pieces (sq_poisson, sq_effective_potential,
sq_mixer_*) against the oracle (oracle/scf_oracle.c, pinned by
tests/test_oracle_scf.py), and the whole loop (SQSCF) against oracle.scf on
a small infinite-cell system."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQSCF, SQSolver, build, sq  # noqa: E402

build()
DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(DEV)


@pytest.fixture(scope="module")
def small():
    s = synth.make_system("al4_16")
    solver = SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP64, device=DEV)
    yield s, solver
    solver.close()


def test_poisson_matches_oracle(small):
    s, solver = small
    n = s.wl.n
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.0, 0.05, size=(n, n, n)) + 0.02 * np.exp(-((np.arange(n) - n / 2) ** 2) / 8)[None, None, :]
    phi_ref, _, _ = oracle.poisson(rho, s.wl.h, tol=1e-13)
    phi = torch.empty(n ** 3, dtype=torch.float64, device=DEV)
    sq.sq_set_stream(solver.ctx)
    it, res = sq.sq_poisson(solver.ctx, _dev(rho), phi, 1e-13)
    assert res <= 1e-13 and it > 0
    np.testing.assert_allclose(phi.cpu().numpy(), phi_ref.ravel(), atol=1e-10 * np.abs(phi_ref).max())
    assert abs(phi.cpu().numpy().mean()) < 1e-13 * np.abs(phi_ref).max()
    it0, _ = sq.sq_poisson(solver.ctx, _dev(np.full(n ** 3, 0.013)), phi, 1e-12)   # neutral density
    assert it0 == 0 and np.all(phi.cpu().numpy() == 0.0)
    with pytest.raises(sq.SQError) as e:                                            # too few iterations
        sq.sq_poisson(solver.ctx, _dev(rho), phi, 1e-13, max_iter=3)
    assert e.value.code == sq.SQ_ENOCONV


def test_effective_potential_matches_oracle(small):
    s, solver = small
    N = s.wl.n_nodes
    rng = np.random.default_rng(8)
    rho = rng.uniform(-1e-3, 0.2, size=N)
    phi = rng.standard_normal(N)
    V_out = torch.empty(N, dtype=torch.float64, device=DEV)
    for alpha in (2.0 / 3.0, 0.7):
        sq.sq_effective_potential(solver.ctx, _dev(s.V), _dev(phi), _dev(rho), alpha, V_out)
        ref = s.V.ravel() + phi + oracle.xalpha(rho, alpha)
        np.testing.assert_allclose(V_out.cpu().numpy(), ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("period", [1, 3])
def test_mixer_matches_oracle(period):
    """Anderson mixing (period 1) and Periodic Pulay (period 3: the
    extrapolation on steps 2, 5, 8, simple mixing on the others)."""
    rng = np.random.default_rng(9)
    n, hist, beta = 777, 4, 0.35
    mixer = sq.sq_mixer_create(n, hist, beta)
    sq.sq_mixer_set_period(mixer, period, 0)
    Xs, Fs = [], []
    v_next = torch.empty(n, dtype=torch.float64, device=DEV)
    x = rng.standard_normal(n)
    for k in range(9):
        v_out = 0.6 * np.tanh(x) + rng.standard_normal(n) * 0.1 + 1.0
        res = sq.sq_mixer_step(mixer, _dev(x), _dev(v_out), v_next)
        f = v_out - x
        assert abs(res - np.linalg.norm(f) / np.linalg.norm(v_out)) < 1e-13 * res
        Xs.append(x.copy())
        Fs.append(f)
        Xs, Fs = Xs[-(hist + 1):], Fs[-(hist + 1):]
        use = len(Xs) if (k + 1) % period == 0 else 1
        ref = oracle.anderson_step(np.array(Xs[-use:]), np.array(Fs[-use:]), beta)
        np.testing.assert_allclose(v_next.cpu().numpy(), ref, rtol=0, atol=1e-11 * np.abs(ref).max())
        x = v_next.cpu().numpy().copy()
    sq.sq_mixer_destroy(mixer)


def test_scf_matches_oracle_scf():
    """One FCC cell, 8^3 grid (h = 0.956), R_cut = 2.5 (5^3 regions), s + 3p
    projectors, kT = 0.1: the device SCF follows the oracle's SCF (same
    iteration count) and reaches the same fixed point."""
    wl = synth.custom_workload("scf8", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1741)
    s = synth.make_system(wl)
    pt = synth.projector_types(True)
    ref = oracle.scf(s.V, wl.h, wl.m, s.positions, pt, wl.n_electrons, wl.kT, wl.npl, tol=1e-9, max_iter=60)
    assert ref["converged"]
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    scf = SQSCF(solver, _dev(s.V), wl.n_electrons, wl.kT)
    out = scf.run(tol=1e-9, max_iter=60)
    assert out["converged"] and abs(out["iterations"] - ref["iterations"]) <= 1
    np.testing.assert_allclose(out["residuals"][:5], ref["residuals"][:5], rtol=1e-6)
    np.testing.assert_allclose(out["V"].cpu().numpy(), ref["V"].ravel(), atol=1e-7 * np.abs(ref["V"]).max())
    np.testing.assert_allclose(out["rho"].cpu().numpy(), ref["rho"].ravel(), atol=1e-7 * ref["rho"].max())
    assert abs(out["mu"] - ref["mu"]) < 1e-7
    assert abs(out["n_elec"] - wl.n_electrons) < 1e-8 * wl.n_electrons
    scf.close()
    solver.close()


def test_widen_bounds_and_scf_that_reuses_them():
    """sq_widen_bounds: zeta grows by exactly max|V - V_ref| (chi unchanged),
    and the widened bounds of a changed potential still enclose every nodal
    spectrum (all moments in [-1, 1]).  An SCF that reuses widened bounds
    (refreshed when the widening would pass 0.05 Ha) runs fewer Lanczos
    steps, converges, and lands within the effect of that widening of the
    plain SCF's fixed point (a wider interval changes the SQ approximation,
    not its correctness)."""
    wl = synth.custom_workload("scf8r", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1742)
    s = synth.make_system(wl)
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    V = _dev(s.V)
    chi0, zeta0 = (t.clone() for t in solver.bounds(V, wl.n_lanczos, wl.margin))
    dV = 0.03 * np.cos(np.arange(wl.n_nodes) * 0.21)
    V2 = V + _dev(dV)
    w = solver.widen_bounds(V2, V, chi0, zeta0)
    assert w == np.abs(V2.cpu().numpy() - V.cpu().numpy()).max()
    assert torch.equal(solver.chi, chi0)
    np.testing.assert_array_equal(solver.zeta.cpu().numpy(), zeta0.cpu().numpy() + w)
    mom = solver.compute_moments(V2).cpu().numpy()
    assert np.abs(mom).max() <= 1 + 1e-9
    V_loc = _dev(s.V)
    plain = SQSCF(solver, V_loc, wl.n_electrons, wl.kT).run(tol=1e-8, max_iter=60)
    rho_plain = plain["rho"].cpu().numpy().copy()            # the solver's buffer, reused by the next run
    reuse = SQSCF(solver, V_loc, wl.n_electrons, wl.kT, reuse_bounds=0.05).run(tol=1e-8, max_iter=60)
    assert plain["converged"] and reuse["converged"]
    assert plain["lanczos_runs"] == plain["iterations"] and reuse["lanczos_runs"] < reuse["iterations"]
    np.testing.assert_allclose(reuse["rho"].cpu().numpy(), rho_plain, atol=2e-3 * np.abs(rho_plain).max())
    assert abs(reuse["mu"] - plain["mu"]) < 2e-3
    print(f"SCF to 1e-8: plain {plain['iterations']} iterations ({plain['lanczos_runs']} Lanczos runs), "
          f"reusing bounds {reuse['iterations']} ({reuse['lanczos_runs']} Lanczos runs)")
    solver.close()


def test_scf_that_stops_reusing_bounds_reaches_the_fresh_fixed_point():
    """Bounds reused (widened by the potential change, up to 0.05 Ha) while
    the residual is above 1e-4, fresh from then on, with the mixing history
    dropped at the switch: the loop converges to 1e-9 and lands on the fixed
    point of the SCF that takes fresh bounds every iteration (FP64: to the
    residual left), not on the one of the reused bounds."""
    wl = synth.custom_workload("scf8s", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1744)
    s = synth.make_system(wl)
    V_loc = _dev(s.V)
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    fresh = SQSCF(solver, V_loc, wl.n_electrons, wl.kT).run(tol=1e-9, max_iter=80)
    rho_fresh, mu_fresh = fresh["rho"].cpu().numpy().copy(), fresh["mu"]
    mixed = SQSCF(solver, V_loc, wl.n_electrons, wl.kT, reuse_bounds=0.05, fresh_below=1e-4).run(tol=1e-9,
                                                                                                 max_iter=80)
    assert fresh["converged"] and mixed["converged"]
    assert mixed["lanczos_runs"] < mixed["iterations"]
    np.testing.assert_allclose(mixed["rho"].cpu().numpy(), rho_fresh, rtol=0, atol=1e-6 * np.abs(rho_fresh).max())
    assert abs(mixed["mu"] - mu_fresh) < 1e-7
    print(f"SCF to 1e-9: fresh bounds {fresh['iterations']} iterations; reuse until 1e-4, then fresh: "
          f"{mixed['iterations']} ({mixed['lanczos_runs']} Lanczos runs)")
    solver.close()


def test_fp32_scf_refined_in_fp64_reaches_the_fp64_fixed_point():
    """FP32 iterations until the residual is 1e-5, then an FP64 context of
    the same grid and atoms takes over with the mixing history: the loop
    converges to 1e-10, far below what FP32 rounding allows, and its density
    is the FP64 SCF's fixed point (both end on FP64 solves with the same
    enclosing-bound policy, up to the residual left)."""
    wl = synth.custom_workload("scf8f", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1743)
    s = synth.make_system(wl)
    V_loc = _dev(s.V)
    coarse = SQSolver.from_workload(wl, s.positions, precision=SQ_FP32, device=DEV)
    fine = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    mixed = SQSCF(coarse, V_loc, wl.n_electrons, wl.kT, reuse_bounds=0.05, refine=(fine, 1e-5))
    out = mixed.run(tol=1e-10, max_iter=80)
    assert out["converged"] and out["refined_at"] is not None
    assert out["residuals"][out["refined_at"] - 1] <= 1e-5 < out["residuals"][out["refined_at"] - 2]
    rho_mixed = out["rho"].cpu().numpy().copy()
    ref = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    plain = SQSCF(ref, V_loc, wl.n_electrons, wl.kT, reuse_bounds=0.05).run(tol=1e-10, max_iter=80)
    assert plain["converged"]
    # both fixed points use bounds widened from some earlier Lanczos run, so they agree to the effect of
    # the bounds on the SQ approximation (cf. the bound-reuse test), not to rounding
    np.testing.assert_allclose(rho_mixed, plain["rho"].cpu().numpy(), atol=2e-3 * np.abs(rho_mixed).max())
    print(f"FP32 -> FP64 at iteration {out['refined_at']}: converged to 1e-10 in {out['iterations']} iterations "
          f"(FP64 throughout: {plain['iterations']})")
    mixed.close()
    for x in (coarse, fine, ref):
        x.close()


def test_scf_checkpoint_and_resume(tmp_path):
    """An SCF stopped after 4 iterations and resumed from its checkpoint (the
    next input potential and the mixing history) takes the same iterations
    as one that ran through, and reaches the same fixed point."""
    wl = synth.custom_workload("scf8r", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1742)
    s = synth.make_system(wl)
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    scf = SQSCF(solver, _dev(s.V), wl.n_electrons, wl.kT)
    full = scf.run(tol=1e-9, max_iter=60)
    V_full = full["V"].cpu().numpy().copy()
    ck = str(tmp_path / "scf.npz")
    part = scf.run(tol=1e-9, max_iter=4, checkpoint=ck)
    assert not part["converged"] and len(part["residuals"]) == 4
    rest = scf.run(tol=1e-9, max_iter=60, resume=ck)
    assert rest["converged"] and rest["iterations"] == full["iterations"]
    np.testing.assert_allclose(rest["residuals"], full["residuals"], rtol=1e-9)
    np.testing.assert_allclose(rest["V"].cpu().numpy(), V_full, atol=1e-12 * np.abs(V_full).max())
    scf.close()
    solver.close()


def test_kerker_matches_oracle(small):
    s, solver = small
    n = s.wl.n
    rng = np.random.default_rng(12)
    v_in = rng.standard_normal((n, n, n))
    v_out = v_in + rng.standard_normal((n, n, n)) * 0.1 + 0.05
    v_pre = torch.empty(n ** 3, dtype=torch.float64, device=DEV)
    sq.sq_set_stream(solver.ctx)
    for k0, amin in ((1.0, 0.2), (0.6, 1.0)):
        res, it = sq.sq_kerker(solver.ctx, _dev(v_in), _dev(v_out), k0, amin, v_pre, tol=1e-13)
        y, _ = oracle.kerker(v_out - v_in, s.wl.h, k0, amin, tol=1e-13)
        ref = v_in + y
        np.testing.assert_allclose(v_pre.cpu().numpy(), ref.ravel(), atol=1e-10 * np.abs(ref).max())
        assert abs(res - np.linalg.norm(v_out - v_in) / np.linalg.norm(v_out)) < 1e-13 and it > 0
    with pytest.raises(sq.SQError) as e:                           # output aliases an input
        x = _dev(v_in)
        sq.sq_kerker(solver.ctx, x, _dev(v_out), 1.0, 0.2, x)
    assert e.value.code == sq.SQ_EINVAL


def test_scf_with_kerker_matches_oracle_scf():
    """The SCF of test_scf_matches_oracle_scf with the Kerker-preconditioned
    residual mixed: same iterations as the oracle's preconditioned SCF and
    the same fixed point as without the preconditioner."""
    wl = synth.custom_workload("scf8k", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1741)
    s = synth.make_system(wl)
    pt = synth.projector_types(True)
    kk = (1.0, 0.2)
    ref = oracle.scf(s.V, wl.h, wl.m, s.positions, pt, wl.n_electrons, wl.kT, wl.npl, tol=1e-9, max_iter=60,
                     kerker=kk)
    assert ref["converged"]
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    scf = SQSCF(solver, _dev(s.V), wl.n_electrons, wl.kT, kerker=kk)
    out = scf.run(tol=1e-9, max_iter=60)
    assert out["converged"] and abs(out["iterations"] - ref["iterations"]) <= 1
    np.testing.assert_allclose(out["residuals"][:5], ref["residuals"][:5], rtol=1e-6)
    np.testing.assert_allclose(out["V"].cpu().numpy(), ref["V"].ravel(), atol=1e-7 * np.abs(ref["V"]).max())
    scf.close()
    solver.close()


def _symbol(n, h, no=6):
    """Discrete Fourier symbol of -lap_h on a periodic n^3 grid."""
    w = oracle.fd_weights(no, h)
    th = 2 * np.pi * np.fft.fftfreq(n)
    s1 = -(2 * w[0] + 2 * sum(w[d] * np.cos(d * th) for d in range(1, no + 1)))
    return s1[:, None, None] + s1[None, :, None] + s1[None, None, :]


def test_poisson_and_kerker_full_size_match_their_fourier_symbols():
    """On the 64^3 grid of the 4x4x4-cell system: phi is the spectral solution
    4 pi (rho - mean)/S, and the preconditioned residual is (S + a k0^2)/(S +
    k0^2) times f, both checked by FFT (properties that hold at any size)."""
    s = synth.make_system("al256_64")
    wl = s.wl
    n = wl.n
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    sq.sq_set_stream(solver.ctx)
    S = _symbol(n, wl.h)
    rng = np.random.default_rng(44)
    rho = 0.02 + 0.01 * np.sin(2 * np.pi * np.arange(n) / n)[None, None, :] + rng.uniform(0, 0.005, (n, n, n))
    phi = torch.empty(n ** 3, dtype=torch.float64, device=DEV)
    it, res = sq.sq_poisson(solver.ctx, _dev(rho), phi, 1e-12)
    S0 = S.copy()
    S0[0, 0, 0] = 1.0
    P = 4 * np.pi * np.fft.fftn(rho - rho.mean()) / S0
    P[0, 0, 0] = 0.0
    ref = np.real(np.fft.ifftn(P))
    np.testing.assert_allclose(phi.cpu().numpy().reshape(n, n, n), ref, atol=1e-9 * np.abs(ref).max())
    v_in = rng.standard_normal((n, n, n))
    v_out = v_in + 0.1 * rng.standard_normal((n, n, n)) + 0.05
    v_pre = torch.empty(n ** 3, dtype=torch.float64, device=DEV)
    k0, a = 0.8, 0.2
    r, _ = sq.sq_kerker(solver.ctx, _dev(v_in), _dev(v_out), k0, a, v_pre, tol=1e-12)
    y = np.real(np.fft.ifftn(np.fft.fftn(v_out - v_in) * (S + a * k0 ** 2) / (S + k0 ** 2)))
    np.testing.assert_allclose(v_pre.cpu().numpy().reshape(n, n, n) - v_in, y, atol=1e-9 * np.abs(y).max())
    solver.close()

"""The learned warm start end to end on a small system: SCF iterations of
the SQ path supply (V_in, rho) training pairs, the network trains on them
with its own kernels, and the surrogate SCF (the network in place of the SQ
solve) gives a starting potential from which the real SCF converges.  The
parity of the network's kernels is in tests/test_gpu_cnn.py."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_07913_gb300 import SQ_FP64, SQCNN, SQSCF, SQSolver, build, warm_start_potential  # noqa: E402

build()
DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(DEV)


def test_train_then_warm_start(tmp_path):
    wl = synth.custom_workload("ws8", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1750)
    s = synth.make_system(wl)
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    V_loc = _dev(s.V)
    shape = (wl.n,) * 3
    pairs = []
    scf = SQSCF(solver, V_loc, wl.n_electrons, wl.kT)
    plain = scf.run(tol=1e-6, max_iter=60,
                    on_step=lambda V, rho, mu: pairs.append((shape, V.clone(), rho.clone(), float(mu))))
    assert plain["converged"] and len(pairs) == plain["iterations"]
    rho_plain = plain["rho"].cpu().numpy().copy()

    net = SQCNN(bf16=True, seed=3, v_shift=float(s.V.mean()), v_scale=float(s.V.std()),
                rho_scale=float(pairs[-1][2].mean().item()))
    first = net.train_step([p[:3] for p in pairs[:3]], lr=3e-3)
    rng = np.random.default_rng(0)
    for _ in range(60):
        idx = rng.choice(len(pairs), size=min(3, len(pairs)), replace=False)
        last = net.train_step([pairs[i][:3] for i in idx], lr=3e-3)
    assert np.isfinite(last) and last < 0.5 * first

    path = str(tmp_path / "net.npz")
    net.save(path)
    again = SQCNN.load(path, device=DEV)
    assert np.array_equal(again.params(), net.params())
    r1, r2 = net.predict(shape, V_loc), again.predict(shape, V_loc)
    assert torch.equal(r1, r2)
    again.close()

    V0, res, used = warm_start_potential(net, solver, V_loc, iters=20)
    assert len(res) >= 1 and np.all(np.isfinite(res)) and used
    warm = scf.run(V0=V0, tol=1e-6, max_iter=60)
    assert warm["converged"]
    np.testing.assert_allclose(warm["rho"].cpu().numpy(), rho_plain, atol=1e-5 * np.abs(rho_plain).max())
    print(f"SCF iterations: plain {plain['iterations']}, warm start {warm['iterations']}")
    net.close()
    scf.close()
    solver.close()


def test_fermi_referenced_warm_start():
    """The network trained on V - mu; each surrogate step finds mu so that
    the predicted density holds N_e electrons; the SCF from that start
    reaches the same fixed point.  Every SQ solve also gives the densities
    at Fermi levels 0.05 and 0.1 Ha either side of its own (same moments),
    so the network sees how the density moves with mu and its electron
    count N(mu) rises through N_e near the training Fermi levels."""
    from paper_1708_07913_gb300 import warmstart as wsm
    wl = synth.custom_workload("ws8m", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1, sigma_disp=0.1, nonlocal_=True,
                               seed=1751)
    s = synth.make_system(wl)
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    V_loc = _dev(s.V)
    shape = (wl.n,) * 3
    pairs = []
    scf = SQSCF(solver, V_loc, wl.n_electrons, wl.kT)
    plain = scf.run(tol=1e-6, max_iter=60,
                    on_step=wsm.pair_collector(solver, wl.kT, pairs, (-0.1, -0.05, 0.0, 0.05, 0.1)))
    assert plain["converged"] and len(pairs) == 5 * plain["iterations"]
    rho_plain = plain["rho"].cpu().numpy().copy()
    scf_only = wsm.scf_pairs(pairs)
    assert len(scf_only) == plain["iterations"]
    # the collector restores the SCF's own density: the last SCF pair is the converged density
    np.testing.assert_array_equal(scf_only[-1][2].cpu().numpy(), rho_plain)
    mus = np.array([p[3] for p in scf_only])
    Vm = np.concatenate([p[1].cpu().numpy() - p[3] for p in pairs])
    net = SQCNN(bf16=True, seed=4, v_shift=float(Vm.mean()), v_scale=float(Vm.std()),
                rho_scale=float(np.mean([p[2].mean().item() for p in pairs])))
    first = net.train_step(pairs[:3], lr=3e-3)
    rng = np.random.default_rng(1)
    for _ in range(60):
        idx = rng.choice(len(pairs), size=3, replace=False)
        last = net.train_step([pairs[i] for i in idx], lr=3e-3)
    assert np.isfinite(last) and last < 0.5 * first
    rho, mu = net.predict_electrons(shape, scf_only[-1][1], wl.n_electrons, wl.h)
    assert rho is not None, f"no crossing of N_e on the scan: {net.last_scan}"
    assert mus.min() - 1.0 < mu < mus.max() + 1.0
    # bfloat16 storage rounds the shifted input, so N(mu) is a fine staircase: the
    # bisection lands on a step, within one step of N_e
    assert abs(wl.h ** 3 * rho.sum().item() - wl.n_electrons) < 1e-3 * wl.n_electrons
    V0, res, used = warm_start_potential(net, solver, V_loc, iters=20, n_electrons=wl.n_electrons)
    assert np.all(np.isfinite(res))
    warm = scf.run(V0=V0, tol=1e-6, max_iter=60)
    assert warm["converged"]
    np.testing.assert_allclose(warm["rho"].cpu().numpy(), rho_plain, atol=1e-5 * np.abs(rho_plain).max())
    print(f"SCF iterations: plain {plain['iterations']}, Fermi-referenced warm start {warm['iterations']} "
          f"(network used: {used})")
    net.close()
    scf.close()
    solver.close()


def test_warm_start_gain_on_held_out_geometry():
    """What the trained network gains, judged by plain SQ on a geometry it
    never saw: trained (V - mu form, densities at the SCF's Fermi level and
    0.05, 0.1 Ha either side) on the SCF pairs of four seeded one-cell
    geometries, its surrogate SCF gives a starting potential from which the
    SQ SCF of a fifth geometry starts with a residual at least five times
    smaller than from V_loc and needs no more iterations.  (CPU oracle
    rehearsal of this setting: first residual 0.011 against 0.59, 11 against
    13 iterations.)"""
    from paper_1708_07913_gb300 import warmstart as wsm
    mk = lambda seed: synth.custom_workload(f"ho{seed}", cells=1, n=8, r_cut=2.5, npl=24, kT=0.1,  # noqa: E731
                                            sigma_disp=0.1, nonlocal_=True, seed=seed)
    pairs = []
    for seed in (1800, 1801, 1802, 1803):
        wl = mk(seed)
        s = synth.make_system(wl)
        solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
        scf = SQSCF(solver, _dev(s.V), wl.n_electrons, wl.kT)
        out = scf.run(tol=1e-6, max_iter=60, on_step=wsm.pair_collector(solver, wl.kT, pairs,
                                                                        (-0.1, -0.05, 0.0, 0.05, 0.1)))
        assert out["converged"]
        scf.close()
        solver.close()
    Vm = np.concatenate([p[1].cpu().numpy() - p[3] for p in pairs])
    net = SQCNN(bf16=True, seed=4, v_shift=float(Vm.mean()), v_scale=float(Vm.std()),
                rho_scale=float(np.mean([p[2].mean().item() for p in pairs])))
    rng = np.random.default_rng(2)
    for _ in range(150):
        idx = rng.choice(len(pairs), size=4, replace=False)
        net.train_step([pairs[i] for i in idx], lr=3e-3)
    wl = mk(1900)
    s = synth.make_system(wl)
    solver = SQSolver.from_workload(wl, s.positions, precision=SQ_FP64, device=DEV)
    V_loc = _dev(s.V)
    scf = SQSCF(solver, V_loc, wl.n_electrons, wl.kT)
    plain = scf.run(tol=1e-6, max_iter=60)
    rho_plain = plain["rho"].cpu().numpy().copy()
    V0, surrogate, used = warm_start_potential(net, solver, V_loc, iters=30, n_electrons=wl.n_electrons)
    assert used, f"surrogate SCF rejected: residuals {surrogate}"
    warm = scf.run(V0=V0, tol=1e-6, max_iter=60)
    assert plain["converged"] and warm["converged"]
    print(f"held-out geometry: first residual {warm['residuals'][0]:.3e} (warm) vs {plain['residuals'][0]:.3e} "
          f"(V_loc); SCF iterations {warm['iterations']} vs {plain['iterations']}")
    assert warm["residuals"][0] < 0.2 * plain["residuals"][0]
    assert warm["iterations"] <= plain["iterations"]
    np.testing.assert_allclose(warm["rho"].cpu().numpy(), rho_plain, atol=1e-5 * np.abs(rho_plain).max())
    net.close()
    scf.close()
    solver.close()

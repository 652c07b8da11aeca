"""Batched launch (sq_batch_*): the whole step of several uneven systems as
one CUDA graph must give what the single-system calls give for each system
-- bit for bit in FP64 (every sum there has a fixed order and a node's result
does not depend on the grid it runs in), and to FP32 rounding in FP32 (the
projector update adds with shared-memory atomics).  The single-system calls
are themselves pinned to the oracle by test_gpu_parity.py; one system here
is also checked against the oracle on sampled nodes."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQBatch, SQError, SQSolver, build, sq  # noqa: E402

build()
DEV = "cuda:0"

# uneven grids, regions (m = 6, 6, 7, 4, 11), degrees and temperatures; FP64 fits all of them.  The
# first two share a region size but not the size of their projector tables (the larger first), so
# one region kernel launches from the graph with two shared-memory sizes.
SYSTEMS = [
    dict(cells=1, n=16, r_cut=3.0, npl=24, kT=0.12, nonlocal_=True, seed=1730),
    dict(cells=1, n=16, r_cut=3.0, npl=24, kT=0.10, nonlocal_=False, seed=1731),
    dict(cells=1, n=15, r_cut=4.0, npl=32, kT=0.07, nonlocal_=True, seed=1732),
    dict(cells=2, n=30, r_cut=2.5, npl=16, kT=0.15, nonlocal_=True, seed=1733),
    dict(cells=1, n=17, r_cut=5.0, npl=24, kT=0.05, nonlocal_=True, seed=1734),
]


@pytest.fixture(scope="module")
def systems():
    return [synth.make_system(synth.custom_workload(f"b{i}", sigma_disp=0.15, **kw)) for i, kw in enumerate(SYSTEMS)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(DEV)


def _snapshot(solver, scal):
    return dict(moments=solver.moments.cpu().numpy().copy(), rho=solver.rho.cpu().numpy().copy(),
                chi=solver.chi.cpu().numpy().copy(), **scal)


@pytest.mark.parametrize("precision", [SQ_FP64, SQ_FP32])
def test_batch_matches_single_system_calls(systems, precision):
    Vs = [_dev(s.V) for s in systems]
    single = []
    for s, V in zip(systems, Vs):
        solver = SQSolver.from_workload(s.wl, s.positions, precision=precision, device=DEV)
        out = solver.solve(V, s.wl.n_electrons, s.wl.kT, s.wl.n_lanczos, s.wl.margin)
        single.append(_snapshot(solver, dict(mu=out["mu"], e_band=out["e_band"], e_ent=out["e_ent"],
                                             n_elec=out["n_elec"])))
        solver.close()
    solvers = [SQSolver.from_workload(s.wl, s.positions, precision=precision, device=DEV) for s in systems]
    batch = SQBatch(solvers)
    args = ([s.wl.n_electrons for s in systems], [s.wl.kT for s in systems])
    runs = []
    for _ in range(2):                      # the second run replays the instantiated graph
        batch.run(Vs, *args)
        res = batch.results()
        runs.append([_snapshot(sv, r) for sv, r in zip(solvers, res)])
    blocks = batch.blocks()
    assert len(blocks) == len(systems) and all(b >= 0 for b in blocks)
    for one, b1, b2 in zip(single, runs[0], runs[1]):
        if precision == SQ_FP64:
            for k in ("moments", "rho", "chi"):
                assert np.array_equal(b1[k], one[k]) and np.array_equal(b2[k], one[k])
            for k in ("mu", "e_band", "e_ent", "n_elec"):
                assert b1[k] == one[k] and b2[k] == one[k]
        else:
            for b in (b1, b2):
                assert np.abs(b["moments"] - one["moments"]).max() < 2e-5   # the FP32 moment tolerance
                np.testing.assert_allclose(b["chi"], one["chi"], rtol=5e-5)
                assert np.linalg.norm(b["rho"] - one["rho"]) < 1e-5 * np.linalg.norm(one["rho"])
                assert abs(b["mu"] - one["mu"]) < 1e-5
                assert abs(b["e_band"] - one["e_band"]) < 1e-5 * max(1.0, abs(one["e_band"]))
                assert abs(b["n_elec"] - one["n_elec"]) < 1e-8 * one["n_elec"]
    batch.close()
    for sv in solvers:
        sv.close()


def test_batch_against_oracle_sampled(systems):
    """System 4 (m = 11, projectors) of an FP64 batch on sampled nodes."""
    solvers = [SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP64, device=DEV) for s in systems]
    batch = SQBatch(solvers)
    batch.run([_dev(s.V) for s in systems], [s.wl.n_electrons for s in systems], [s.wl.kT for s in systems])
    batch.results()
    s, sv = systems[4], solvers[4]
    nodes = synth.sample_nodes(s.wl.n_nodes, 6, seed=4)
    osys = oracle.OracleSystem.from_synth(s)
    ochi, ozeta = osys.bounds(nodes, s.wl.n_lanczos, s.wl.margin)
    np.testing.assert_allclose(sv.chi.cpu().numpy()[nodes], ochi, rtol=1e-9)
    np.testing.assert_allclose(sv.zeta.cpu().numpy()[nodes], ozeta, rtol=1e-9)
    omom = osys.moments(nodes, ochi, ozeta, s.wl.npl)
    np.testing.assert_allclose(sv.moments.cpu().numpy()[nodes], omom, rtol=0, atol=1e-10)
    batch.close()
    for x in solvers:
        x.close()


def test_batch_rejects_bad_arguments(systems):
    solvers = [SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP32, device=DEV) for s in systems[:2]]
    batch = SQBatch(solvers)
    Vs = [_dev(s.V) for s in systems[:2]]
    with pytest.raises(SQError) as e:              # N_e outside (0, 2 N_d)
        batch.run(Vs, [0.0, systems[1].wl.n_electrons], [0.1, 0.1])
    assert e.value.code == sq.SQ_EINVAL
    with pytest.raises(SQError) as e:              # kT <= 0
        batch.run(Vs, [s.wl.n_electrons for s in systems[:2]], [0.1, -1.0])
    assert e.value.code == sq.SQ_EINVAL
    with pytest.raises(SQError) as e:              # no Lanczos step
        batch.run(Vs, [s.wl.n_electrons for s in systems[:2]], [0.1, 0.1], n_lanczos=0)
    assert e.value.code == sq.SQ_EINVAL
    with pytest.raises(SQError) as e:              # the C entry point itself, a NULL batch
        sq._check(sq.load().sq_batch_run(None, None, None, None, None, None, None, None, 40, 0.01), "sq_batch_run")
    assert e.value.code == sq.SQ_EINVAL
    batch.close()
    for x in solvers:
        x.close()

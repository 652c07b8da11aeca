"""Batched launch (sq_batch_*): the whole step of several uneven systems as
one CUDA graph must give what the single-system calls give for each system,
in every launch plan (per-system streams, or persistent queue kernels per
group of systems with one region size) -- bit for bit in FP64 (every sum
there has a fixed order and a node's result does not depend on the CTA or
grid it runs in), and to FP32 rounding in FP32 (the projector update adds
with shared-memory atomics).  The single-system calls are themselves pinned
to the oracle by test_gpu_parity.py; here one system of an FP64 batch and
every system of the 16-system FP32 benchmark batch are also checked against
the oracle on sampled nodes.  The queue plan's bounded waits are made to run
out (a count that nothing completes) and must end the run with SQ_ETIMEOUT,
leaving the batch usable."""
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


PLANS = {"streams": (sq.SQ_BATCH_STREAMS, 1), "queue1": (sq.SQ_BATCH_QUEUE, 1), "queue5": (sq.SQ_BATCH_QUEUE, 5)}


@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("precision", [SQ_FP64, SQ_FP32])
def test_batch_matches_single_system_calls(systems, precision, plan):
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
    batch.set_plan(*PLANS[plan])
    args = ([s.wl.n_electrons for s in systems], [s.wl.kT for s in systems])
    runs = []
    for _ in range(2):                      # the second run replays the instantiated graph
        batch.run(Vs, *args)
        res = batch.results()
        runs.append([_snapshot(sv, r) for sv, r in zip(solvers, res)])
    blocks = batch.blocks()
    assert len(blocks) == len(systems) and all(b >= 0 for b in blocks)
    kind, npi = batch.plan()
    assert kind == PLANS[plan][0] and npi == (PLANS[plan][1] if kind == sq.SQ_BATCH_QUEUE else 0)
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


def test_batch_autotuner_picks_a_plan(systems):
    solvers = [SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP32, device=DEV) for s in systems]
    batch = SQBatch(solvers)
    batch.run([_dev(s.V) for s in systems], [s.wl.n_electrons for s in systems], [s.wl.kT for s in systems])
    res = batch.results()
    kind, npi = batch.plan()
    assert kind in (sq.SQ_BATCH_STREAMS, sq.SQ_BATCH_STREAMS_SHARE, sq.SQ_BATCH_QUEUE)
    assert (npi in (1, 4)) if kind == sq.SQ_BATCH_QUEUE else npi == 0
    for s, r in zip(systems, res):
        assert abs(r["n_elec"] - s.wl.n_electrons) < 1e-8 * s.wl.n_electrons
    batch.close()
    for x in solvers:
        x.close()


def test_queue_wait_runs_out_then_batch_recovers(systems):
    """Every Lanczos item waits for one potential slab more than exist: each
    wait ends after its budget (2e6 SM cycles, ~1 ms) and the run reports
    SQ_ETIMEOUT; with normal waits the same batch then gives the single-system
    results again."""
    sub = systems[:3]
    Vs = [_dev(s.V) for s in sub]
    args = ([s.wl.n_electrons for s in sub], [s.wl.kT for s in sub])
    solvers = [SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP64, device=DEV) for s in sub]
    batch = SQBatch(solvers)
    batch.set_plan(sq.SQ_BATCH_QUEUE, 64)
    batch.set_wait(2_000_000, wait_on_unset=True)
    batch.run(Vs, *args)
    with pytest.raises(SQError) as e:
        batch.results()
    assert e.value.code == sq.SQ_ETIMEOUT
    batch.set_wait(2_000_000_000, wait_on_unset=False)
    batch.run(Vs, *args)
    res = batch.results()
    for s, sv, V, r in zip(sub, solvers, Vs, res):
        one = SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP64, device=DEV)
        out = one.solve(V, s.wl.n_electrons, s.wl.kT, s.wl.n_lanczos, s.wl.margin)
        assert np.array_equal(sv.rho.cpu().numpy(), one.rho.cpu().numpy())
        assert r["mu"] == out["mu"]
        one.close()
    with pytest.raises(SQError) as e:
        batch.set_wait(0)
    assert e.value.code == sq.SQ_EINVAL
    with pytest.raises(SQError) as e:
        batch.set_plan(sq.SQ_BATCH_QUEUE, 0)
    assert e.value.code == sq.SQ_EINVAL
    batch.close()
    for x in solvers:
        x.close()


def test_batch16_fp32_every_system_against_oracle():
    """The 16 systems of the batch benchmark (regions 15^3 to 31^3, n_pl 24
    to 64), FP32, queue plan: on 3 seeded nodes of every system the bounds
    and moments against the oracle's (tolerances of the FP32 context: bounds
    2e-4 relative, moments 2e-5), and every system's electron count.  The
    density step itself is pinned to the oracle by the single-system tests
    (with the oracle's bounds injected and a test-chosen Fermi level, which a
    batch run cannot take); here the batch must conserve the electrons."""
    wls = synth.batch_workloads()
    systems = [synth.make_system(w) for w in wls]
    solvers = [SQSolver.from_workload(s.wl, s.positions, precision=SQ_FP32, device=DEV) for s in systems]
    batch = SQBatch(solvers)
    batch.set_plan(sq.SQ_BATCH_QUEUE, 1)
    margin, n_lz = wls[0].margin, wls[0].n_lanczos
    batch.run([_dev(s.V) for s in systems], [w.n_electrons for w in wls], [w.kT for w in wls], n_lz, margin)
    res = batch.results()
    for i, (s, sv, r) in enumerate(zip(systems, solvers, res)):
        nodes = synth.sample_nodes(s.wl.n_nodes, 3, seed=100 + i)
        osys = oracle.OracleSystem.from_synth(s)
        ochi, ozeta = osys.bounds(nodes, n_lz, margin)
        np.testing.assert_allclose(sv.chi.cpu().numpy()[nodes], ochi, rtol=2e-4, err_msg=f"system {i}")
        np.testing.assert_allclose(sv.zeta.cpu().numpy()[nodes], ozeta, rtol=2e-4, err_msg=f"system {i}")
        omom = osys.moments(nodes, ochi, ozeta, s.wl.npl)
        np.testing.assert_allclose(sv.moments.cpu().numpy()[nodes], omom, rtol=0, atol=2e-5, err_msg=f"system {i}")
        assert abs(r["n_elec"] - s.wl.n_electrons) < 1e-8 * s.wl.n_electrons
        rho = sv.rho.cpu().numpy()
        assert rho.min() > 0 and abs(rho.sum() * s.wl.h ** 3 - s.wl.n_electrons) < 1e-8 * s.wl.n_electrons
    batch.close()
    for x in solvers:
        x.close()

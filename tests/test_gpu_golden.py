"""Full-size end-to-end parity on the benchmark workload (3x3x3 FCC cells,
48^3 grid, 25^3 regions, n_pl = 48, s + 3p projectors), in the launch
configuration bench.py times, against whole-grid oracle results written by
tests/golden/make_golden.py (which calls only oracle/)."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_07913_gb300 import SQ_FP32, SQ_FP64, SQSolver, build  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "al108_48_oracle.json")


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))


@pytest.mark.parametrize("precision,tol_rho,tol_e_atom,tol_mu", [
    (SQ_FP64, 1e-10, 1e-10, 1e-10),
    (SQ_FP32, 1e-5, 1e-5, 1e-5),
])
def test_al108_48_full_grid(golden, precision, tol_rho, tol_e_atom, tol_mu):
    build()
    s = synth.make_system("al108_48")
    wl = s.wl
    solver = SQSolver.from_workload(wl, s.positions, precision=precision)
    V = torch.from_numpy(s.V.ravel().copy()).cuda()
    out = solver.solve(V, wl.n_electrons, wl.kT, wl.n_lanczos, wl.margin)
    torch.cuda.synchronize()
    rho = out["rho"].cpu().numpy()
    nodes = np.array(golden["sample_nodes"])
    # Fermi level, energies per atom, electron count
    assert abs(out["mu"] - golden["mu"]) < tol_mu * max(1.0, abs(golden["mu"]))
    assert abs(out["e_band"] - golden["e_band"]) / wl.n_atoms < max(tol_e_atom, 1e-10 * abs(golden["e_band"]))
    assert abs(out["e_ent"] - golden["e_ent"]) / wl.n_atoms < max(tol_e_atom, 1e-10 * abs(golden["e_ent"]))
    assert abs(out["n_elec"] - wl.n_electrons) < 1e-8 * wl.n_electrons
    # density: global norms and the sampled nodes
    assert abs(np.linalg.norm(rho) - golden["rho_norm2"]) < tol_rho * golden["rho_norm2"]
    assert abs(rho.sum() - golden["rho_sum"]) < tol_rho * golden["rho_sum"]
    d = rho[nodes] - np.array(golden["sample_rho"])
    assert np.abs(d).max() < tol_rho * golden["rho_max"]
    assert np.linalg.norm(d) < tol_rho * np.linalg.norm(golden["sample_rho"])
    # spectral bounds and moments of the sampled nodes; FP32 Lanczos vectors
    # leave unconverged Ritz values a few 1e-5 away from the FP64 ones (the
    # density targets above are what the FP32 form must meet)
    tol_b = 1e-9 if precision == SQ_FP64 else 2e-4
    np.testing.assert_allclose(out["chi"].cpu().numpy()[nodes], golden["sample_chi"], rtol=tol_b)
    np.testing.assert_allclose(out["zeta"].cpu().numpy()[nodes], golden["sample_zeta"], rtol=tol_b)
    if precision == SQ_FP64:
        # (FP32 moments depend on the FP32 bounds; moment-level FP32 parity with
        # the oracle's bounds injected is checked in test_full_size_sampled_nodes)
        np.testing.assert_allclose(out["moments"].cpu().numpy()[nodes], golden["sample_moments"], rtol=0,
                                   atol=1e-9)
    solver.close()

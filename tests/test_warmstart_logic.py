"""Control flow of warm_start_potential (no GPU): the libsq calls are
replaced by stand-ins that script the surrogate's residuals, so the three
outcomes are checked on the host: converged (the network's potential is
kept), a rejected state (plain SQ's V_loc is returned), and a residual
above the acceptance threshold (V_loc as well)."""
import contextlib
import types

import pytest

torch = pytest.importorskip("torch")

import paper_1708_07913_gb300 as pkg  # noqa: E402
from paper_1708_07913_gb300 import sq  # noqa: E402


class _Net:
    def predict(self, shape, V, out=None):
        return out


def _solver(n=8):
    return types.SimpleNamespace(torch=torch, device=torch.device("cpu"), shape=(2, 2, 2), n_nodes=n, ctx=1)


def _script(monkeypatch, residuals, fail_at=None):
    it = {"k": 0}

    def mixer_step(m, v_in, v_out, v_next):
        v_next.copy_(v_in + 1.0)
        r = residuals[it["k"]]
        it["k"] += 1
        return r

    def poisson(ctx, rho, phi, tol):
        if fail_at is not None and it["k"] == fail_at:
            raise sq.SQError(sq.SQ_ENOCONV, "sq_poisson")
        return 1, 0.0

    monkeypatch.setattr(torch.cuda, "device", lambda d: contextlib.nullcontext())   # host tensors here
    monkeypatch.setattr(sq, "sq_mixer_create", lambda n, h, b: 7)
    monkeypatch.setattr(sq, "sq_mixer_destroy", lambda m: None)
    monkeypatch.setattr(sq, "sq_set_stream", lambda ctx: None)
    monkeypatch.setattr(sq, "sq_poisson", poisson)
    monkeypatch.setattr(sq, "sq_effective_potential", lambda *a: None)
    monkeypatch.setattr(sq, "sq_mixer_step", mixer_step)
    return it


def test_converged_surrogate_is_used(monkeypatch):
    it = _script(monkeypatch, [0.6, 0.1, 0.01, 5e-5, 1.0])
    V_loc = torch.zeros(8, dtype=torch.float64)
    V, res, used = pkg.warm_start_potential(_Net(), _solver(), V_loc, iters=10, tol=1e-4)
    assert used and res == [0.6, 0.1, 0.01, 5e-5] and it["k"] == 4
    assert torch.all(V == 4.0)                      # four mixing steps from V_loc = 0


def test_rejected_state_falls_back_to_plain_sq(monkeypatch):
    _script(monkeypatch, [0.6, 0.2, 0.1], fail_at=2)
    V_loc = torch.full((8,), 3.0, dtype=torch.float64)
    V, res, used = pkg.warm_start_potential(_Net(), _solver(), V_loc, iters=10)
    assert not used and len(res) == 3 and res[-1] != res[-1]      # NaN recorded
    assert torch.equal(V, V_loc) and V.data_ptr() != V_loc.data_ptr()


def test_unconverged_surrogate_above_threshold_falls_back(monkeypatch):
    _script(monkeypatch, [0.6, 0.5, 0.4])
    V_loc = torch.full((8,), -1.0, dtype=torch.float64)
    V, res, used = pkg.warm_start_potential(_Net(), _solver(), V_loc, iters=3, accept=0.1)
    assert not used and res == [0.6, 0.5, 0.4] and torch.equal(V, V_loc)


def _scripted_net(monkeypatch, count):
    """An SQCNN whose electron count per h^3 is count(mu) (no GPU)."""
    state = {"mu": 0.0}
    monkeypatch.setattr(sq, "sq_cnn_set_shift", lambda net, mu: state.__setitem__("mu", mu))
    monkeypatch.setattr(sq, "sq_cnn_forward_sum", lambda net, shape, V, rho: count(state["mu"]))
    monkeypatch.setattr(sq, "sq_cnn_destroy", lambda net: None)        # the handle below is a stand-in
    net = pkg.SQCNN.__new__(pkg.SQCNN)
    net.torch, net.device, net.net = torch, torch.device("cpu"), 1
    net.scales = (0.0, 1.0, 1.0)              # v_scale 1: the scan spans at least +-2 about its centre
    net.mu_seen = (0.0, 0.6)                  # training Fermi levels: the scan is centred on 0.3
    return net, state


def test_predict_electrons_bisects_the_shift(monkeypatch):
    """SQCNN.predict_electrons with a scripted count N(mu) = 10 + 4 tanh(mu - 0.3):
    the shift found puts N_e electrons in the density; a count that never
    reaches N_e gives (None, None) and leaves the scan for diagnosis."""
    import math
    net, state = _scripted_net(monkeypatch, lambda mu: 10.0 + 4.0 * math.tanh(mu - 0.3))
    V = torch.zeros(8, dtype=torch.float64)
    rho, mu = net.predict_electrons((2, 2, 2), V, n_electrons=12.0, h=1.0)
    assert abs(mu - (0.3 + math.atanh(0.5))) < 1e-12 and state["mu"] == 0.0     # shift reset afterwards
    rho, mu = net.predict_electrons((2, 2, 2), V, n_electrons=20.0, h=1.0)     # unreachable: 10 + 4 tanh < 14
    assert rho is None and mu is None
    shifts, counts = net.last_scan
    assert len(shifts) == 33 and abs(shifts[0] + 1.7) < 1e-12 and abs(shifts[-1] - 2.3) < 1e-12
    assert max(counts) < 14.0
    net.net = None


def test_predict_electrons_without_assumed_direction(monkeypatch):
    """A count that falls with mu, and one that rises and falls again (what a
    network does far outside its training range): the crossing nearest the
    centre of the training Fermi levels is the one kept."""
    import math
    net, _ = _scripted_net(monkeypatch, lambda mu: 10.0 - 4.0 * math.tanh(mu - 0.3))
    V = torch.zeros(8, dtype=torch.float64)
    rho, mu = net.predict_electrons((2, 2, 2), V, n_electrons=8.0, h=1.0)
    assert abs(mu - (0.3 + math.atanh(0.5))) < 1e-12
    net.net = None
    net, _ = _scripted_net(monkeypatch, lambda mu: 13.0 * math.exp(-(mu - 0.2) ** 2))
    rho, mu = net.predict_electrons((2, 2, 2), V, n_electrons=12.0, h=1.0)
    assert abs(mu - (0.2 + math.sqrt(math.log(13.0 / 12.0)))) < 1e-12          # 0.483, not -0.083
    net.net = None
    # rises to 11.9, then falls to a plateau of 8.4 (the shape seen with an
    # undertrained network): N_e = 12 is never reached
    net, _ = _scripted_net(monkeypatch, lambda mu: 8.4 + 3.5 * math.exp(-(mu - 0.3) ** 2 / 0.02)
                           if mu > 0.3 else 11.9 * math.exp(-(mu - 0.3) ** 2))
    rho, mu = net.predict_electrons((2, 2, 2), V, n_electrons=12.0, h=1.0)
    assert rho is None and mu is None
    net.net = None

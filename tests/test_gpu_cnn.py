"""The warm-start network on the GPU (sq_cnn_*) against the FP64 oracle
(oracle/cnn_oracle.py, pinned by tests/test_oracle_cnn.py), on the same
seeded weights and inputs.

Tolerances.  FP32 storage: every sum of at most 864 products accumulates in
FP32 (relative rounding ~1e-7 per term), so the density and every gradient
tensor agree to 1e-5 relative to their largest entry.  bfloat16 storage: the
oracle rounds the weights and activations at the same points, but an
activation whose FP32 and FP64 values straddle a rounding boundary comes
out one bfloat16 step (2^-8 relative) apart; a few such flips per output
bound the density at 2e-3 of its largest value and the gradients at 1e-3
(2-norm).  The Adam step is compared in 2-norm at 1e-3 of its length: where
a gradient entry is near zero its normalised step is sensitive to the
rounding of that entry."""
import numpy as np
import pytest

from oracle import cnn_oracle as cnn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1708_07913_gb300 import build, sq  # noqa: E402

build()
DEV = "cuda:0"


def _flat(p):
    return np.concatenate([p[k].ravel() for k in cnn.TRAINED])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(DEV)


def _problem(shape, seed):
    rng = np.random.default_rng(seed)
    p = cnn.init_params(seed, v_shift=-1.0, v_scale=1.2, rho_scale=0.03)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.2 * rng.standard_normal(p[k].shape)
    for k in cnn.TRAINED:                                  # the library keeps FP32 master weights
        p[k] = p[k].astype(np.float32).astype(np.float64)
    V = rng.uniform(-3.0, 0.5, size=shape[::-1])
    ref = rng.uniform(0.0, 0.08, size=V.shape)
    return p, V, ref


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("shape", [(6, 5, 7), (9, 8, 10), (1, 1, 1), (16, 16, 16)])
def test_forward_backward_adam_match_oracle(shape, bf16):
    p, V, ref = _problem(shape, seed=sum(shape))
    net = sq.sq_cnn_create(32, bf16)
    sq.sq_cnn_set_params(net, _flat(p), p["v_shift"], p["v_scale"], p["rho_scale"])
    np.testing.assert_array_equal(sq.sq_cnn_get_params(net), _flat(p))
    N = V.size
    rho = torch.empty(N, dtype=torch.float64, device=DEV)
    sq.sq_cnn_forward(net, shape, _dev(V), rho)
    rho_o, _ = cnn.forward(p, V, bf16=bf16)
    tol_rho = 2e-3 if bf16 else 1e-5
    np.testing.assert_allclose(rho.cpu().numpy(), rho_o.ravel(), rtol=0, atol=tol_rho * np.abs(rho_o).max())

    L = sq.sq_cnn_backward(net, shape, _dev(V), _dev(ref), rho)
    L_o, g_o = cnn.backward(p, V, ref, bf16=bf16)
    assert abs(L - L_o) <= (1e-3 if bf16 else 1e-6) * L_o
    g = sq.sq_cnn_get_grads(net)
    off = 0
    for k in cnn.TRAINED:
        n = g_o[k].size
        a, b = g[off:off + n], g_o[k].ravel()
        off += n
        if bf16:
            assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), k
        else:
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * np.abs(b).max(), err_msg=k)

    lr = 1e-3
    sq.sq_cnn_adam_step(net, lr)
    st = cnn.adam_init(p)
    p1 = cnn.adam_step(dict(p), g_o, st, lr=lr)
    step_dev = sq.sq_cnn_get_params(net) - _flat(p)
    step_or = _flat(p1) - _flat(p)
    assert np.linalg.norm(step_dev - step_or) <= 1e-3 * np.linalg.norm(step_or)
    sq.sq_cnn_destroy(net)


def test_backward_repeats_and_accumulates():
    shape = (9, 8, 10)
    p, V, ref = _problem(shape, seed=5)
    net = sq.sq_cnn_create(32, True)
    sq.sq_cnn_set_params(net, _flat(p), p["v_shift"], p["v_scale"], p["rho_scale"])
    rho = torch.empty(V.size, dtype=torch.float64, device=DEV)
    L1 = sq.sq_cnn_backward(net, shape, _dev(V), _dev(ref), rho)
    g1 = sq.sq_cnn_get_grads(net)
    L2 = sq.sq_cnn_backward(net, shape, _dev(V), _dev(ref), rho)
    assert L1 == L2 and np.array_equal(g1, sq.sq_cnn_get_grads(net))          # fixed-order sums
    sq.sq_cnn_backward(net, shape, _dev(V), _dev(ref), rho, accumulate=True)
    np.testing.assert_allclose(sq.sq_cnn_get_grads(net), 2 * g1, rtol=1e-6, atol=0)
    with pytest.raises(sq.SQError) as e:
        sq.sq_cnn_forward(net, (0, 4, 4), _dev(V), rho)
    assert e.value.code == sq.SQ_EINVAL
    sq.sq_cnn_destroy(net)
    fresh = sq.sq_cnn_create(32, True)
    with pytest.raises(sq.SQError):                       # no parameters yet
        sq.sq_cnn_forward(fresh, shape, _dev(V), rho)
    with pytest.raises(sq.SQError):                       # no gradient yet
        sq.sq_cnn_adam_step(fresh, 1e-3)
    sq.sq_cnn_destroy(fresh)


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_full_size_sampled_nodes(bf16):
    """The 64^3 grid of the warm-start target (al256_64's local potential):
    the output at 48 seeded nodes against the oracle evaluated on the 9^3 box
    around each node (an output depends on exactly that patch, so the box's
    centre never sees the box's own wrap-around)."""
    import synth
    s = synth.make_system("al256_64")
    V = s.V                                             # (64, 64, 64), x fastest
    n = V.shape[0]
    p, _, _ = _problem((4, 4, 4), seed=17)
    p["v_shift"], p["v_scale"] = float(V.mean()), float(V.std())
    net = sq.sq_cnn_create(32, bf16)
    sq.sq_cnn_set_params(net, _flat(p), p["v_shift"], p["v_scale"], p["rho_scale"])
    rho = torch.empty(V.size, dtype=torch.float64, device=DEV)
    sq.sq_cnn_forward(net, (n, n, n), _dev(V), rho)
    rho = rho.cpu().numpy().reshape(V.shape)
    nodes = synth.sample_nodes(V.size, 48, seed=23)
    ref, got = [], []
    for q in nodes:
        i, j, k = q % n, (q // n) % n, q // (n * n)
        idx = [np.arange(c - 4, c + 5) % n for c in (k, j, i)]
        patch = V[np.ix_(*idx)]
        r, _ = cnn.forward(p, patch, bf16=bf16)
        ref.append(r[4, 4, 4])
        got.append(rho[k, j, i])
    ref, got = np.array(ref), np.array(got)
    tol = 2e-3 if bf16 else 1e-5
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol * np.abs(ref).max())
    sq.sq_cnn_destroy(net)


@pytest.mark.parametrize("bf16", [False, True])
def test_input_shift_and_density_sum(bf16):
    """sq_cnn_set_shift(s) makes the network see V - s; sq_cnn_forward_sum
    returns sum rho.  Against the oracle on V - s."""
    shape = (9, 8, 10)
    p, V, _ = _problem(shape, seed=41)
    net = sq.sq_cnn_create(32, bf16)
    sq.sq_cnn_set_params(net, _flat(p), p["v_shift"], p["v_scale"], p["rho_scale"])
    rho = torch.empty(V.size, dtype=torch.float64, device=DEV)
    for s in (0.0, 0.37, -1.25):
        sq.sq_cnn_set_shift(net, s)
        tot = sq.sq_cnn_forward_sum(net, shape, _dev(V), rho)
        ref, _ = cnn.forward(p, V - s, bf16=bf16)
        tol = 2e-3 if bf16 else 1e-5
        np.testing.assert_allclose(rho.cpu().numpy(), ref.ravel(), rtol=0, atol=tol * np.abs(ref).max())
        assert abs(tot - rho.cpu().numpy().sum()) <= 1e-12 * abs(tot)
    sq.sq_cnn_destroy(net)


def test_full_size_gradient_is_the_derivative_of_the_loss():
    """At 64^3 (the warm-start target's grid; FP32 storage, so the loss is
    smooth in the weights) the stored gradient is the derivative of the
    device's own loss: g . (theta+ - theta-) equals L(theta+) - L(theta-)
    for theta +- eps d along a seeded direction, to the FD truncation and
    FP32 rounding (1e-2 relative)."""
    import synth
    s = synth.make_system("al256_64")
    V = s.V
    n = V.shape[0]
    p, _, _ = _problem((4, 4, 4), seed=29)
    p["v_shift"], p["v_scale"] = float(V.mean()), float(V.std())
    rng = np.random.default_rng(30)
    ref = _dev(rng.uniform(0.0, 0.06, size=V.size))
    Vd = _dev(V)
    rho = torch.empty(V.size, dtype=torch.float64, device=DEV)
    net = sq.sq_cnn_create(32, False)
    theta = _flat(p)
    sq.sq_cnn_set_params(net, theta, p["v_shift"], p["v_scale"], p["rho_scale"])
    sq.sq_cnn_backward(net, (n, n, n), Vd, ref, rho)
    g = sq.sq_cnn_get_grads(net)
    d = rng.standard_normal(theta.size)
    d /= np.linalg.norm(d)
    eps = 2e-3 * np.linalg.norm(theta)
    losses, thetas = [], []
    for sgn in (1.0, -1.0):
        sq.sq_cnn_set_params(net, theta + sgn * eps * d, p["v_shift"], p["v_scale"], p["rho_scale"])
        thetas.append(sq.sq_cnn_get_params(net))                 # as rounded to FP32
        losses.append(sq.sq_cnn_backward(net, (n, n, n), Vd, ref, rho))
    fd = losses[0] - losses[1]
    an = float(g @ (thetas[0] - thetas[1]))
    assert abs(fd) > 1e-6 and abs(an - fd) <= 1e-2 * abs(fd)
    sq.sq_cnn_destroy(net)


@pytest.mark.parametrize("shape", [(16, 16, 16), (21, 20, 19)])
def test_tensor_core_middle_layer(shape, monkeypatch):
    """The bfloat16 network's 32 -> 32 layer on the tensor cores (tcgen05
    implicit GEMM, FP32 accumulation in TMEM; the default) against the same
    layer on CUDA cores (SQ_CNN_TENSOR=0) and against the oracle.  The two
    GPU forms differ only in the order of the FP32 sums, so apart from
    activations that round to a neighbouring bfloat16 value they agree; both
    meet the oracle tolerance of the bfloat16 network.  Grids with a ragged
    last 128-node tile (21 x 20 x 19 = 7980 nodes)."""
    p, V, _ = _problem(shape, seed=7 + sum(shape))
    rho = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("SQ_CNN_TENSOR", mode)
        net = sq.sq_cnn_create(32, True)
        sq.sq_cnn_set_params(net, _flat(p), p["v_shift"], p["v_scale"], p["rho_scale"])
        out = torch.empty(V.size, dtype=torch.float64, device=DEV)
        total = sq.sq_cnn_forward_sum(net, shape, _dev(V), out)       # synchronises and reports wait expiry
        rho[mode] = out.cpu().numpy()
        assert abs(total - rho[mode].sum()) < 1e-9 * abs(total)
        sq.sq_cnn_destroy(net)
    rho_o, _ = cnn.forward(p, V, bf16=True)
    rho_o = rho_o.ravel()
    for mode in ("1", "0"):
        np.testing.assert_allclose(rho[mode], rho_o, rtol=0, atol=2e-3 * np.abs(rho_o).max())
    d = rho["1"] - rho["0"]
    assert np.abs(d).max() <= 2e-3 * np.abs(rho["0"]).max()
    assert np.linalg.norm(d) <= 2e-4 * np.linalg.norm(rho["0"])

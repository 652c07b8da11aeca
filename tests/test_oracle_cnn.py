"""Pins of the learned-warm-start oracle (oracle/cnn_oracle.py) against
references that share nothing with it: scipy's wrapped correlation, the
convolution theorem (FFT), central finite differences of the loss, exact
translation equivariance and the 9^3 receptive field, torch's bfloat16
conversion, and the closed form of Adam's first steps."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import cnn_oracle as cnn


def test_single_channel_conv_is_scipy_wrapped_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((7, 6, 8))
    for k in (3, 5):
        W = rng.standard_normal((k, k, k))
        got = cnn.conv(x[None], W[None, None])[0]
        np.testing.assert_allclose(got, ndimage.correlate(x, W, mode="wrap"), atol=1e-12)


def test_multichannel_conv_by_the_convolution_theorem():
    """out[o] = sum_i IFFT(FFT(x_i) conj(FFT(w_oi))) with w_oi the kernel
    placed at offsets d (wrapped) on the grid, plus the bias."""
    rng = np.random.default_rng(1)
    shape = (6, 7, 5)
    Ci, Co, k = 3, 4, 3
    x = rng.standard_normal((Ci,) + shape)
    W = rng.standard_normal((Co, Ci, k, k, k))
    b = rng.standard_normal(Co)
    r = (k - 1) // 2
    ref = np.zeros((Co,) + shape)
    for o in range(Co):
        acc = np.zeros(shape, dtype=complex)
        for i in range(Ci):
            w = np.zeros(shape)
            for dz in range(-r, r + 1):
                for dy in range(-r, r + 1):
                    for dx in range(-r, r + 1):
                        w[dz % shape[0], dy % shape[1], dx % shape[2]] += W[o, i, dz + r, dy + r, dx + r]
            acc += np.fft.fftn(x[i]) * np.conj(np.fft.fftn(w))
        ref[o] = np.real(np.fft.ifftn(acc)) + b[o]
    np.testing.assert_allclose(cnn.conv(x, W, b), ref, atol=1e-12)


def test_conv_adjoints():
    """<conv(x), g> = <x, conv_input_grad(g)> = <W, conv_weight_grad(g, x)>."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 5, 6, 7))
    g = rng.standard_normal((2, 5, 6, 7))
    for k in (3, 5):
        W = rng.standard_normal((2, 3, k, k, k))
        lhs = np.sum(cnn.conv(x, W) * g)
        assert abs(lhs - np.sum(x * cnn.conv_input_grad(g, W))) < 1e-10 * abs(lhs)
        assert abs(lhs - np.sum(W * cnn.conv_weight_grad(g, x, k))) < 1e-10 * abs(lhs)


def _small_params(seed=3, C=3):
    p = cnn.init_params(seed, channels=C, v_shift=-1.0, v_scale=1.5, rho_scale=0.05)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.3 * rng.standard_normal(p[k].shape)
    return p


def test_gradients_match_central_differences():
    rng = np.random.default_rng(4)
    p = _small_params()
    V = rng.uniform(-3.0, 0.5, size=(6, 5, 7))
    rho_ref = rng.uniform(0.0, 0.1, size=V.shape)
    L, g = cnn.backward(p, V, rho_ref)
    assert abs(L - cnn.loss(p, V, rho_ref)) < 1e-15 * max(L, 1.0)
    h = 1e-6
    for name in cnn.TRAINED:
        flat = p[name].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            Lp = cnn.loss(p, V, rho_ref)
            flat[idx] = old - h
            Lm = cnn.loss(p, V, rho_ref)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[name].ravel()[idx]
            assert abs(an - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g[name]).max()), (name, idx, an, fd)


def test_translation_equivariance_and_receptive_field():
    rng = np.random.default_rng(5)
    p = _small_params(C=4)
    V = rng.uniform(-3.0, 0.5, size=(12, 12, 12))
    rho, _ = cnn.forward(p, V)
    shifted, _ = cnn.forward(p, np.roll(V, (2, -3, 5), axis=(0, 1, 2)))
    np.testing.assert_allclose(shifted, np.roll(rho, (2, -3, 5), axis=(0, 1, 2)), atol=1e-14)
    q = (6, 6, 6)
    for dist, changes in ((4, True), (5, False)):
        W = V.copy()
        W[q[0] + dist, q[1] - 1, q[2] + 2] += 0.7                   # Chebyshev distance `dist` from q
        r2, _ = cnn.forward(p, W)
        assert (r2[q] != rho[q]) == changes


def test_bf16_rounding_is_torch_bfloat16():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    a = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.4e38, -3.4e38, 1e-40, np.inf, -np.inf]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.to_bf16(a), ref)
    assert np.isnan(cnn.to_bf16(np.array([np.nan]))[0])
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert cnn.to_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert cnn.to_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_adam_first_steps_closed_form():
    """Step 1 moves each parameter by lr sign(g) (up to eps); with a constant
    gradient every step does, since m/(1-b1^t) = g and v/(1-b2^t) = g^2."""
    p = {k: np.ones(3) for k in cnn.TRAINED}
    st = cnn.adam_init(p)
    g = {k: np.array([2.0, -0.5, 1e-3]) for k in cnn.TRAINED}
    for t in range(1, 4):
        cnn.adam_step(p, g, st, lr=0.01, eps=0.0)
        np.testing.assert_allclose(p["W1"], 1.0 - 0.01 * t * np.sign(g["W1"]), atol=1e-14)
    g2 = {k: np.array([4.0, 4.0, 4.0]) for k in cnn.TRAINED}
    cnn.adam_step(p, g2, st, lr=0.01, eps=0.0)
    m = 0.9 ** 4 * 0 + (0.9 ** 3 * 0.1 + 0.9 ** 2 * 0.1 + 0.9 * 0.1) * g["W1"] + 0.1 * 4.0
    v = (0.999 ** 2 * 0.001 + 0.999 * 0.001 + 0.001) * g["W1"] ** 2 * 0.999 + 0.001 * 16.0
    step = 0.01 * (m / (1 - 0.9 ** 4)) / np.sqrt(v / (1 - 0.999 ** 4))
    np.testing.assert_allclose(p["W1"], 1.0 - 0.03 * np.sign(g["W1"]) - step, atol=1e-13)

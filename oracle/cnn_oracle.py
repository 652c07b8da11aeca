"""Plain FP64 numpy oracle of the learned SCF warm start: a small 3-D
convolutional network that maps the 9^3 patch of the effective potential
around a node to the node's SQ electron density, its gradients, and the
optimiser step that trains it.

TEST INFRASTRUCTURE ONLY, like the C oracle: tests, the package's smoke
check and the benchmark's CPU leg are the only callers; it shares no code
with the CUDA library and imports nothing from it.

The paper has no network; the architecture is this library's reading
(fully convolutional on the periodic grid, so every node's output sees
exactly the 9^3 patch around it):

    x0 = (V - v_shift) / v_scale                       (1 channel)
    a1 = silu(conv5(x0; W1) + b1)                      (C channels, 5^3 kernel)
    a2 = silu(conv3(a1; W2) + b2)                      (C channels, 3^3 kernel)
    y  = conv3(a2; W3) + b3                            (1 channel, 3^3 kernel)
    rho = rho_scale * softplus(y)

conv_k is a periodic cross-correlation with a centred k^3 kernel:
    out[o](p) = sum_i sum_{d in [-r, r]^3} W[o, i, d + r] x[i](p + d),  r = (k - 1)/2,
indices wrapped on the periodic grid (arrays are (z, y, x), x fastest).
silu(z) = z sigmoid(z), softplus(y) = log(1 + e^y).  Receptive field
5 + 2 + 2 = 9 points per axis.

Loss: mean over nodes of (rho - rho_ref)^2 / rho_scale^2.  Optimiser: Adam
(Kingma and Ba, 2015) with bias correction.

Parity status: conv, its adjoints, the loss gradients, bf16 rounding and the
Adam step are pinned by tests/test_oracle_cnn.py (scipy's wrapped
correlation, the convolution theorem, central finite differences of the
loss, exact translation equivariance and receptive field, torch's bfloat16
conversion, closed forms of the first Adam steps).
"""
from __future__ import annotations

import numpy as np

KERNELS = (5, 3, 3)       # kernel edge of the three layers
CHANNELS = 32             # hidden channels


# ---------------------------------------------------------------------------
# bfloat16 rounding (round to nearest, ties to even, on the FP32 bit pattern)
# ---------------------------------------------------------------------------
def to_bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) via FP32; returns float64.
    NaN stays NaN; values beyond the bfloat16 range round to +-inf."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


# ---------------------------------------------------------------------------
# periodic cross-correlation and its two adjoints
# ---------------------------------------------------------------------------
def _offsets(k):
    r = (k - 1) // 2
    return [(dz, dy, dx) for dz in range(-r, r + 1) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]


def _shift(x, d):
    """s(p) = x(p + d) on the periodic grid (last three axes are z, y, x)."""
    return np.roll(x, shift=(-d[0], -d[1], -d[2]), axis=(-3, -2, -1))


def conv(x, W, b=None):
    """out[o](p) = sum_i sum_d W[o, i, d+r] x[i](p + d) (+ b[o]).
    x: (Ci, n3, n2, n1); W: (Co, Ci, k, k, k)."""
    Co, Ci, k = W.shape[0], W.shape[1], W.shape[2]
    r = (k - 1) // 2
    out = np.zeros((Co,) + x.shape[1:])
    for d in _offsets(k):
        Wd = W[:, :, d[0] + r, d[1] + r, d[2] + r]                 # (Co, Ci)
        out += np.einsum("oi,izyx->ozyx", Wd, _shift(x, d))
    if b is not None:
        out += b[:, None, None, None]
    return out


def conv_input_grad(g, W):
    """Adjoint in x: dx[i](p) = sum_o sum_d W[o, i, d+r] g[o](p - d)."""
    Co, Ci, k = W.shape[0], W.shape[1], W.shape[2]
    r = (k - 1) // 2
    dx = np.zeros((Ci,) + g.shape[1:])
    for d in _offsets(k):
        Wd = W[:, :, d[0] + r, d[1] + r, d[2] + r]
        dx += np.einsum("oi,ozyx->izyx", Wd, _shift(g, (-d[0], -d[1], -d[2])))
    return dx


def conv_weight_grad(g, x, k):
    """Adjoint in W: dW[o, i, d+r] = sum_p g[o](p) x[i](p + d)."""
    r = (k - 1) // 2
    dW = np.zeros((g.shape[0], x.shape[0], k, k, k))
    for d in _offsets(k):
        dW[:, :, d[0] + r, d[1] + r, d[2] + r] = np.einsum("ozyx,izyx->oi", g, _shift(x, d))
    return dW


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------
def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def softplus(y):
    return np.logaddexp(0.0, y)


def init_params(seed: int, channels: int = CHANNELS, v_shift: float = 0.0, v_scale: float = 1.0,
                rho_scale: float = 0.03) -> dict:
    """Seeded initial weights: normal with variance 1/fan_in, zero biases."""
    rng = np.random.default_rng(seed)
    k1, k2, k3 = KERNELS
    C = channels
    return dict(
        W1=rng.standard_normal((C, 1, k1, k1, k1)) / np.sqrt(k1 ** 3),
        b1=np.zeros(C),
        W2=rng.standard_normal((C, C, k2, k2, k2)) / np.sqrt(C * k2 ** 3),
        b2=np.zeros(C),
        W3=rng.standard_normal((1, C, k3, k3, k3)) / np.sqrt(C * k3 ** 3),
        b3=np.zeros(1),
        v_shift=float(v_shift), v_scale=float(v_scale), rho_scale=float(rho_scale))


TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3")


def _stored(params, bf16):
    """The weights as the network applies them: bf16-rounded when the
    weights and activations are stored in bfloat16."""
    if not bf16:
        return params
    q = dict(params)
    for k in ("W1", "W2", "W3"):
        q[k] = to_bf16(params[k])
    return q


def forward(params, V, bf16=False):
    """rho (n3, n2, n1) and the activations the backward pass needs.  With
    bf16=True, the weights, x0, a1 and a2 are rounded to bfloat16 where they
    are stored (everything else stays FP64)."""
    rnd = to_bf16 if bf16 else (lambda a: a)
    p = _stored(params, bf16)
    x0 = rnd(((np.asarray(V, dtype=np.float64) - p["v_shift"]) / p["v_scale"])[None])
    z1 = conv(x0, p["W1"], p["b1"])
    a1 = rnd(silu(z1))
    z2 = conv(a1, p["W2"], p["b2"])
    a2 = rnd(silu(z2))
    y = conv(a2, p["W3"], p["b3"])
    rho = p["rho_scale"] * softplus(y[0])
    return rho, dict(x0=x0, z1=z1, a1=a1, z2=z2, a2=a2, y=y)


def loss(params, V, rho_ref):
    rho, _ = forward(params, V)
    return float(np.mean((rho - rho_ref) ** 2) / params["rho_scale"] ** 2)


def backward(params, V, rho_ref, bf16=False):
    """Loss and its gradient with respect to every trained parameter.  With
    bf16=True the backward pass of the rounded network takes the stored
    (rounded) weights and activations and treats the rounding as the
    identity."""
    rho, c = forward(params, V, bf16)
    params = _stored(params, bf16)
    N = rho.size
    rs = params["rho_scale"]
    L = float(np.mean((rho - rho_ref) ** 2) / rs ** 2)
    g_rho = 2.0 * (rho - rho_ref) / (N * rs ** 2)
    g_y = (g_rho * rs * sigmoid(c["y"][0]))[None]
    k1, k2, k3 = KERNELS
    grads = {}
    grads["W3"] = conv_weight_grad(g_y, c["a2"], k3)
    grads["b3"] = g_y.sum(axis=(1, 2, 3))
    g_z2 = conv_input_grad(g_y, params["W3"]) * silu_grad(c["z2"])
    grads["W2"] = conv_weight_grad(g_z2, c["a1"], k2)
    grads["b2"] = g_z2.sum(axis=(1, 2, 3))
    g_z1 = conv_input_grad(g_z2, params["W2"]) * silu_grad(c["z1"])
    grads["W1"] = conv_weight_grad(g_z1, c["x0"], k1)
    grads["b1"] = g_z1.sum(axis=(1, 2, 3))
    return L, grads


def adam_init(params) -> dict:
    return dict(t=0, m={k: np.zeros_like(params[k]) for k in TRAINED}, v={k: np.zeros_like(params[k]) for k in TRAINED})


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    state["t"] += 1
    t = state["t"]
    for k in TRAINED:
        g = grads[k]
        state["m"][k] = beta1 * state["m"][k] + (1.0 - beta1) * g
        state["v"][k] = beta2 * state["v"][k] + (1.0 - beta2) * g * g
        mh = state["m"][k] / (1.0 - beta1 ** t)
        vh = state["v"][k] / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params

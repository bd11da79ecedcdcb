"""Learned Davidson preconditioner: features, MLP forward / backward and Adam (oracle; test
infrastructure only).

The paper does not have this component; it is the learned correction the library adds beside
the diagonal preconditioner of the generalised Davidson solver.  Per element i of the two-site
vector the network sees

    f = ( sqrt(n) r_i / |r|,  sqrt(n) d_i / |d|,  dn_i,  tanh(delta_i / (1 + |theta|)) ),
    delta_i = dh_i - theta dn_i,   d_i = -r_i / delta_i  (|delta_i| clamped to >= 1e-4),

with r the residual, dh / dn the diagonals of H_eff / N_eff and theta the current Ritz value,
and predicts one number, the correction t_i (in units where the target error vector has
norm sqrt(n)).  The network is a 3-layer perceptron: 4 -> 256 -> 256 -> 1 with ReLU.  The loss of
a batch is the mean squared error.  Plain float64 NumPy, written out step by step.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 4
HIDDEN = 256
CLAMP = 1e-4


def features(r, dh, dn, theta):
    """(n, 4) feature matrix of one residual."""
    n = r.shape[0]
    delta = dh - theta * dn
    den = np.where(np.abs(delta) < CLAMP, np.where(delta < 0, -CLAMP, CLAMP), delta)
    d = -r / den
    rn = np.linalg.norm(r)
    dnrm = np.linalg.norm(d)
    s = np.sqrt(n)
    f = np.empty((n, N_FEATURES))
    f[:, 0] = s * r / rn if rn > 0 else 0.0
    f[:, 1] = s * d / dnrm if dnrm > 0 else 0.0
    f[:, 2] = dn
    f[:, 3] = np.tanh(delta / (1.0 + abs(theta)))
    return f


def init_params(seed: int):
    """He-normal weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((N_FEATURES, HIDDEN)) * np.sqrt(2.0 / N_FEATURES),
        "b1": np.zeros(HIDDEN),
        "W2": rng.standard_normal((HIDDEN, HIDDEN)) * np.sqrt(2.0 / HIDDEN),
        "b2": np.zeros(HIDDEN),
        "w3": rng.standard_normal(HIDDEN) * np.sqrt(1.0 / HIDDEN),
        "b3": np.zeros(1),
    }


def forward(p, X):
    """Returns the prediction (B,) and the cache of activations."""
    Z1 = X @ p["W1"] + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"] + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, (X, Z1, H1, Z2, H2)


def loss_and_grads(p, X, t):
    """Mean squared error of a batch and its gradients with respect to every parameter."""
    y, (X, Z1, H1, Z2, H2) = forward(p, X)
    B = X.shape[0]
    diff = y - t
    loss = float(np.mean(diff * diff))
    dy = 2.0 * diff / B                      # dL/dy
    g = {}
    g["w3"] = H2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dH2 = np.outer(dy, p["w3"])
    dZ2 = dH2 * (Z2 > 0.0)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ p["W2"].T
    dZ1 = dH1 * (Z1 > 0.0)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; state holds m, v and the step."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


def to_bf16(a):
    """Round float32 values to bfloat16 (round to nearest, ties to even) and back to float64:
    the 16 low bits of the float32 pattern are rounded away."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16_layer2(p, X):
    """The forward pass with the operands of the 256 x 256 layer (H1 and W2) rounded to bfloat16
    and everything else in float64: the arithmetic of a BF16 tensor-core layer with exact
    accumulation."""
    Z1 = X @ p["W1"] + p["b1"]
    H1 = to_bf16(np.maximum(Z1, 0.0))
    Z2 = H1 @ to_bf16(p["W2"]) + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    return H2 @ p["w3"] + p["b3"][0]


def flatten(p):
    """The parameter vector layout of the library: W1, b1, W2, b2, w3, b3."""
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["w3"], p["b3"]])


def unflatten(v):
    v = np.asarray(v, dtype=np.float64)
    o = 0
    out = {}
    for k, shape in (("W1", (N_FEATURES, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
                     ("w3", (HIDDEN,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[k] = v[o:o + size].reshape(shape)
        o += size
    return out

"""FP64 reference of the warm-start network (test infrastructure only).

A per-node multilayer perceptron 14 -> 256 -> 256 -> 256 -> 3 with ReLU
activations and mean-squared-error loss, written from the definitions: the
forward pass is a chain of affine maps and ReLUs, and the backward pass is the
chain rule applied to it (dL/dZ = dL/dH * [Z > 0], dL/dW = dZ^T H_prev,
dL/db = column sums of dZ, dL/dH_prev = dZ W).  Pinned by finite differences.
"""
import numpy as np

SIZES = [(256, 14), (256, 256), (256, 256), (3, 256)]
NPARAMS = sum(n * k + n for n, k in SIZES)


def unpack(params):
    """Logical parameter vector -> [(W [n,k], b [n])]."""
    out, q = [], 0
    p = np.asarray(params, dtype=np.float64)
    for n, k in SIZES:
        W = p[q:q + n * k].reshape(n, k); q += n * k
        b = p[q:q + n]; q += n
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def init_params(seed):
    """He-normal weights, zero biases (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = []
    for n, k in SIZES:
        layers.append((rng.normal(0.0, np.sqrt(2.0 / k), size=(n, k)), np.zeros(n)))
    return pack(layers)


def _identity(x):
    return x


def forward(params, X, store=_identity):
    """Returns (prediction [B,3], list of activations).  `store` is applied to
    each hidden activation as it is kept for the next layer (the identity in
    FP64; bf16_round for a network that stores its activations in BF16)."""
    layers = unpack(params)
    H = [np.asarray(X, dtype=np.float64)]
    Z = []
    for i, (W, b) in enumerate(layers):
        z = H[-1] @ W.T + b
        Z.append(z)
        H.append(store(np.maximum(z, 0.0)) if i < len(layers) - 1 else z)
    return H[-1], (H, Z)


def loss_grad(params, X, T, store=_identity):
    """Mean-squared error over all B*3 outputs and its gradient (logical
    layout).  `store` is applied wherever an intermediate is kept for a later
    product: the hidden activations and the back-propagated dL/dZ of every
    layer (the identity gives the plain FP64 chain rule)."""
    layers = unpack(params)
    pred, (H, Z) = forward(params, X, store)
    B = len(X)
    r = pred - T
    loss = float(np.sum(r * r) / (3 * B))
    dZ = store(2.0 * r / (3 * B))
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        grads[i] = (dZ.T @ H[i], dZ.sum(axis=0))
        if i > 0:
            dZ = store((dZ @ W) * (Z[i - 1] > 0))
    return loss, pack(grads)


def bf16_round(x):
    """Round float64 values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)

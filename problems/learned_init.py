"""Seeded initial parameters of the learned preconditioner M_theta.

Only random numbers: the network's arithmetic lives in the oracle and in the
CUDA library.  Both are handed the same initial parameters from here.

Layout (width W = 32, L = 3 message-passing layers):
  e, b0        (W,)       embedding of the normalised residual value
  Ws, Wm       (L, W, W)  self and neighbour-message weights
  b            (L, W)     layer biases
  wo           (W,)       read-out weights
  omega_j      scalar     weight of the Jacobi skip term (starts at 1)
"""
import numpy as np

from . import rng

WIDTH = 32
LAYERS = 3


def init_params(seed: int = 2505_20719 + 50, width: int = WIDTH, layers: int = LAYERS, readout_scale: float = 0.0):
    """He-style normal initialisation; the read-out starts at readout_scale
    (0 makes the untrained net exactly the Jacobi skip term)."""
    W, L = width, layers
    g = rng.normal(seed, 51, W * 2 + L * (2 * W * W + W) + W)
    k = 0

    def take(cnt):
        nonlocal k
        out = g[k:k + cnt]
        k += cnt
        return out

    p = {}
    p["e"] = take(W) * 1.0
    p["b0"] = take(W) * 0.1
    p["Ws"] = take(L * W * W).reshape(L, W, W) * np.sqrt(2.0 / (2 * W))
    p["Wm"] = take(L * W * W).reshape(L, W, W) * np.sqrt(2.0 / (2 * W)) * 0.25
    p["b"] = take(L * W).reshape(L, W) * 0.01
    p["wo"] = take(W) * readout_scale
    p["omega_j"] = np.array(1.0)
    return p


PARAM_ORDER = ("e", "b0", "Ws", "Wm", "b", "wo", "omega_j")


def flatten(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def unflatten(v, width: int = WIDTH, layers: int = LAYERS):
    W, L = width, layers
    shapes = {"e": (W,), "b0": (W,), "Ws": (L, W, W), "Wm": (L, W, W), "b": (L, W), "wo": (W,), "omega_j": ()}
    out, k = {}, 0
    for name in PARAM_ORDER:
        cnt = int(np.prod(shapes[name])) if shapes[name] else 1
        out[name] = np.asarray(v[k:k + cnt], dtype=np.float64).reshape(shapes[name])
        k += cnt
    return out

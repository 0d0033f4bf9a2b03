"""Oracle of the learned preconditioner M_theta (test infrastructure only).

A small message-passing network over the graph of the scaled matrix A^ that
stands in for the primary preconditioner M inside the fp16 Richardson level
(a project addition: the paper's M is an algebraic preconditioner, Sec. 3;
the flexible outer FGMRES levels admit a nonlinear preconditioner, Sec. 4.2).

For a residual r (n values), with s = 2^ceil(log2 max|r|) and r~ = r / s:
    h0_i = relu(e r~_i + b0)
    g_i  = sum_{j != i} A^_ij h_j                        (message aggregation)
    h_i  = relu(Ws_l h_i + Wm_l g_i + b_l),  l = 1..3
    z_i  = s (omega_j r~_i + wo . h_i)
The s-normalisation makes M_theta(a r) = a M_theta(r) for every power of two
a > 0, and with wo = 0, omega_j = 1 it is the Jacobi preconditioner of A^
(diag A^ = 1).

Two training losses over samples p = 1..P (means over p):
    error     ||M_theta(r_p) - e_p||^2 / ||e_p||^2        (e_p = A^-1 r_p)
    residual  ||A M_theta(r_p) - r_p||^2 / ||r_p||^2      (A the matrix the
              preconditioned level applies, here the fp16 copy of A^)

forward() / backward() are plain fp64 numpy; with bf16=True they round the
values the network stores between its steps to bfloat16 and nothing else:
forward -- the weights e, Ws, Wm, wo, the activations h and the aggregated
messages g; backward -- the weights it multiplies by, the masked output
gradients dP = bf16(dh * [h > 0]) of every layer and the messages
u = bf16(dP Wm) it aggregates (dh itself, the weight gradients and all sums
stay in full precision).  That is the reference the GPU is compared with.
The fp64 gradient is checked against central finite differences.
"""
import numpy as np
import scipy.sparse as sp

from . import BF16, round_to

WIDTH = 32


def scale_of(r) -> float:
    """s = 2^ceil(log2 max|r|) (1 for r = 0)."""
    mx = float(np.max(np.abs(r))) if r.size else 0.0
    if not (mx > 0.0) or not np.isfinite(mx):
        return 1.0
    f, e = np.frexp(mx)  # mx = f 2^e, f in [0.5, 1)
    return float(np.ldexp(1.0, e - 1 if f == 0.5 else e))


def offdiag(ahat_vals, rowptr, colidx, n):
    """A^ without its diagonal as a scipy CSR matrix."""
    A = sp.csr_matrix((np.asarray(ahat_vals, dtype=np.float64), colidx, rowptr), shape=(n, n))
    A = A.tolil()
    A.setdiag(0.0)
    A = A.tocsr()
    A.eliminate_zeros()
    return A


def _bf(x):
    return round_to(BF16, x).reshape(np.shape(x))


def forward(A_off, r, p, bf16: bool = False):
    """z = M_theta(r) and the cache backward() needs."""
    r = np.asarray(r, dtype=np.float64)
    s = scale_of(r)
    rt = r / s
    e, b0, Ws, Wm, b, wo = p["e"], p["b0"], p["Ws"], p["Wm"], p["b"], p["wo"]
    if bf16:
        e, Ws, Wm, wo = _bf(e), _bf(Ws), _bf(Wm), _bf(wo)
    p0 = np.outer(rt, e) + b0
    h = np.maximum(p0, 0.0)
    if bf16:
        h = _bf(h)
    cache = {"s": s, "rt": rt, "p": [p0], "h": [h], "g": []}
    for l in range(Ws.shape[0]):
        g = A_off @ h
        if bf16:
            g = _bf(g)
        pl = h @ Ws[l].T + g @ Wm[l].T + b[l]
        h = np.maximum(pl, 0.0)
        if bf16:
            h = _bf(h)
        cache["g"].append(g)
        cache["p"].append(pl)
        cache["h"].append(h)
    y = float(p["omega_j"]) * rt + h @ wo
    return s * y, cache


def backward(A_off, p, cache, dz, bf16: bool = False):
    """Gradient of sum(dz * z) with respect to every parameter (chain rule
    through forward(); bf16=True rounds the stored values named above)."""
    rnd = _bf if bf16 else (lambda x: x)
    s, rt = cache["s"], cache["rt"]
    dy = s * np.asarray(dz, dtype=np.float64)
    L = p["Ws"].shape[0]
    Ws, Wm, wo = rnd(p["Ws"]), rnd(p["Wm"]), rnd(p["wo"])
    hL = cache["h"][L]
    grads = {"omega_j": np.array(rt @ dy), "wo": hL.T @ dy}
    dh = np.outer(dy, wo)
    dWs = np.zeros_like(p["Ws"])
    dWm = np.zeros_like(p["Wm"])
    db = np.zeros_like(p["b"])
    for l in range(L - 1, -1, -1):
        dp = rnd(dh * (cache["p"][l + 1] > 0))
        h_prev, g = cache["h"][l], cache["g"][l]
        dWs[l] = dp.T @ h_prev
        dWm[l] = dp.T @ g
        db[l] = dp.sum(axis=0)
        dh = dp @ Ws[l] + A_off.T @ rnd(dp @ Wm[l])
    dp0 = rnd(dh * (cache["p"][0] > 0))
    grads["e"] = dp0.T @ rt
    grads["b0"] = dp0.sum(axis=0)
    grads["Ws"], grads["Wm"], grads["b"] = dWs, dWm, db
    return grads


def loss_and_grad(A_off, p, R, E, bf16: bool = False):
    """Mean over samples of ||M_theta(r) - e||^2 / ||e||^2 and its gradient.
    R, E: (samples, n) residuals and corrections e = A^-1 r."""
    P = R.shape[0]
    total = 0.0
    grads = None
    for k in range(P):
        z, cache = forward(A_off, R[k], p, bf16=bf16)
        den = float(E[k] @ E[k])
        d = z - E[k]
        total += float(d @ d) / den / P
        gk = backward(A_off, p, cache, 2.0 * d / den / P, bf16=bf16)
        grads = gk if grads is None else {key: grads[key] + gk[key] for key in grads}
    return total, grads


def loss_and_grad_residual(A, A_off, p, R, bf16: bool = False):
    """Mean over samples of ||A M_theta(r) - r||^2 / ||r||^2 and its gradient
    (A: the full matrix, A_off: its off-diagonal graph for the net)."""
    P = R.shape[0]
    total = 0.0
    grads = None
    for k in range(P):
        z, cache = forward(A_off, R[k], p, bf16=bf16)
        den = float(R[k] @ R[k])
        t = A @ z - R[k]
        total += float(t @ t) / den / P
        gk = backward(A_off, p, cache, 2.0 * (A.T @ t) / den / P, bf16=bf16)
        grads = gk if grads is None else {key: grads[key] + gk[key] for key in grads}
    return total, grads

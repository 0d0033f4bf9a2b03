"""Pins of the learned-preconditioner oracle (oracle/learned.py)."""
import numpy as np

import oracle as O
from oracle import learned as LM
from problems import generators as G
from problems import learned_init as LI
from problems import rng


def _graph(N=4, seed=601):
    prob = G.diffusion27_nodal(dims=(N, N, N), seed=seed)
    P = O.Problem(prob, diag_scale=1)
    return prob, LM.offdiag(P.get("ahat"), prob.rowptr, prob.colidx, prob.n)


def test_gradient_matches_central_differences():
    prob, A = _graph()
    p = LI.init_params(readout_scale=0.3)
    R = rng.normal(1, 1, 2 * prob.n).reshape(2, prob.n)
    E = rng.normal(2, 1, 2 * prob.n).reshape(2, prob.n)
    f0, g = LM.loss_and_grad(A, p, R, E)
    flat = LI.flatten(p)
    gflat = LI.flatten(g)
    h = 1e-6
    idx = np.concatenate([np.arange(0, 64), rng.integers(3, 1, 200, 64, flat.size - 1)])
    for k in idx:
        fp = flat.copy()
        fp[k] += h
        fm = flat.copy()
        fm[k] -= h
        lp, _ = LM.loss_and_grad(A, LI.unflatten(fp), R, E)
        lm, _ = LM.loss_and_grad(A, LI.unflatten(fm), R, E)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, gflat[k])


def test_residual_loss_gradient_matches_central_differences():
    """The residual loss ||A M(r) - r||^2 / ||r||^2: analytic gradient
    against central differences, and its value by a direct evaluation."""
    prob = G.diffusion27_nodal(dims=(4, 4, 4), seed=603)
    P = O.Problem(prob, diag_scale=1)
    import scipy.sparse as sp
    Afull = sp.csr_matrix((P.get("ahat"), prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    A = LM.offdiag(P.get("ahat"), prob.rowptr, prob.colidx, prob.n)
    p = LI.init_params(readout_scale=0.3)
    R = rng.normal(6, 1, 2 * prob.n).reshape(2, prob.n)
    f0, g = LM.loss_and_grad_residual(Afull, A, p, R)
    want = np.mean([np.sum((Afull @ LM.forward(A, R[k], p)[0] - R[k]) ** 2) / np.sum(R[k] ** 2) for k in range(2)])
    assert abs(f0 - want) <= 1e-12 * want
    flat = LI.flatten(p)
    gflat = LI.flatten(g)
    h = 1e-6
    idx = np.concatenate([np.arange(0, 64), rng.integers(7, 1, 150, 64, flat.size - 1)])
    for k in idx:
        fp = flat.copy()
        fp[k] += h
        fm = flat.copy()
        fm[k] -= h
        lp, _ = LM.loss_and_grad_residual(Afull, A, LI.unflatten(fp), R)
        lm, _ = LM.loss_and_grad_residual(Afull, A, LI.unflatten(fm), R)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, gflat[k])


def test_untrained_net_is_jacobi_and_scale_homogeneous():
    prob, A = _graph()
    p = LI.init_params(readout_scale=0.0)
    r = rng.normal(4, 1, prob.n)
    z, _ = LM.forward(A, r, p)
    assert np.array_equal(z, r)  # diag A^ = 1: Jacobi is the identity
    p = LI.init_params(readout_scale=0.5)
    z1, _ = LM.forward(A, r, p)
    for k in (-7, 3, 11):
        zk, _ = LM.forward(A, np.ldexp(r, k), p)
        assert np.array_equal(zk, np.ldexp(z1, k))


def test_message_passing_by_explicit_loops():
    prob, A = _graph(N=3, seed=602)
    p = LI.init_params(readout_scale=0.7)
    r = rng.normal(5, 1, prob.n)
    z, _ = LM.forward(A, r, p)
    s = LM.scale_of(r)
    rt = r / s
    h = [[max(0.0, p["e"][c] * rt[i] + p["b0"][c]) for c in range(32)] for i in range(prob.n)]
    Ad = A.toarray()
    for l in range(3):
        g = [[sum(Ad[i, j] * h[j][c] for j in range(prob.n) if Ad[i, j] != 0) for c in range(32)]
             for i in range(prob.n)]
        h = [[max(0.0, sum(p["Ws"][l][a][c] * h[i][c] for c in range(32))
                  + sum(p["Wm"][l][a][c] * g[i][c] for c in range(32)) + p["b"][l][a])
              for a in range(32)] for i in range(prob.n)]
    want = [s * (float(p["omega_j"]) * rt[i] + sum(p["wo"][c] * h[i][c] for c in range(32))) for i in range(prob.n)]
    assert np.allclose(z, want, rtol=1e-12, atol=1e-12)


def test_bf16_forward_close_to_fp64():
    prob, A = _graph(N=6, seed=603)
    p = LI.init_params(readout_scale=0.3)
    r = rng.normal(6, 1, prob.n)
    z, _ = LM.forward(A, r, p)
    zb, _ = LM.forward(A, r, p, bf16=True)
    assert np.linalg.norm(zb - z) <= 3e-2 * np.linalg.norm(z)


def test_bf16_gradient_close_to_exact():
    """The bf16-storage backward (the reference the GPU gradients are compared
    with) stays within bf16 rounding of the exact gradient, per tensor."""
    prob, A = _graph(N=6, seed=604)
    p = LI.init_params(readout_scale=0.5)
    R = rng.normal(8, 1, 2 * prob.n).reshape(2, prob.n)
    E = rng.normal(9, 1, 2 * prob.n).reshape(2, prob.n)
    _, g = LM.loss_and_grad(A, p, R, E)
    _, gb = LM.loss_and_grad(A, p, R, E, bf16=True)
    for k in LI.PARAM_ORDER:
        a, b = np.ravel(gb[k]), np.ravel(g[k])
        assert a @ b >= 0.99 * np.linalg.norm(a) * np.linalg.norm(b), k
        assert np.linalg.norm(a - b) <= 0.1 * np.linalg.norm(b) + 1e-12, k
        assert not np.array_equal(a, b) or np.linalg.norm(b) == 0, k

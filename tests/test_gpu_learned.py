"""Learned preconditioner M_theta on the GPU against the CPU oracle
(oracle/learned.py): forward in bf16 storage, gradients (against the oracle's
backward with the same bf16 storage points: cosine >= 0.999 and 2e-2 relative
per tensor), training and use as M inside the fp16 Richardson level."""
import numpy as np
import pytest

import oracle as O
from oracle import learned as LM
from problems import generators as G
from problems import learned_init as LI
from problems import rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_20719_gb300 import f3r  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def setup():
    prob = G.diffusion27_nodal(dims=(13, 12, 11), seed=701)  # n = 1716: ragged 16-node groups and slices
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.default_params())
    P = O.Problem(prob, diag_scale=1)
    # the fp16 copy of A^ the net aggregates over
    A16 = LM.offdiag(P.get("a16"), prob.rowptr, prob.colidx, prob.n)
    return prob, s, A16


def _cos(a, b):
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def test_forward_matches_oracle_bf16(setup):
    prob, s, A16 = setup
    p = LI.init_params(readout_scale=0.5)
    s.learned_load(LI.flatten(p).astype(np.float32))
    for seed in (1, 2):
        r = rng.normal(seed, 7, prob.n).astype(np.float32)
        z = torch.empty(prob.n, dtype=torch.float32, device="cuda")
        s.learned_apply(dev(r), z)
        torch.cuda.synchronize()
        pf = LI.unflatten(LI.flatten(p).astype(np.float32).astype(np.float64))
        want, _ = LM.forward(A16, r.astype(np.float64), pf, bf16=True)
        got = z.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - want) <= 1e-2 * np.linalg.norm(want)
    # an untrained read-out (wo = 0, omega_j = 1) is Jacobi on A^ (diag = 1): z = r exactly
    s.learned_load(LI.flatten(LI.init_params(readout_scale=0.0)).astype(np.float32))
    r = rng.normal(3, 7, prob.n).astype(np.float32)
    z = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.learned_apply(dev(r), z)
    torch.cuda.synchronize()
    assert np.array_equal(z.cpu().numpy(), r)


def test_gradient_matches_oracle(setup):
    prob, s, A16 = setup
    p = LI.init_params(readout_scale=0.5)
    flat = LI.flatten(p).astype(np.float32)
    s.learned_load(flat, train=True)
    R = rng.normal(11, 7, 2 * prob.n).reshape(2, prob.n).astype(np.float32)
    E = rng.normal(12, 7, 2 * prob.n).reshape(2, prob.n).astype(np.float32)
    loss, grad = s.learned_loss_grad(dev(R), dev(E))
    pf = LI.unflatten(flat.astype(np.float64))
    want_loss, want = LM.loss_and_grad(A16, pf, R.astype(np.float64), E.astype(np.float64), bf16=True)
    assert abs(loss - want_loss) <= 2e-2 * want_loss
    g = LI.unflatten(grad.astype(np.float64))
    for k in LI.PARAM_ORDER:
        a, b = np.ravel(g[k]), np.ravel(want[k])
        print(f"{k}: cos {_cos(a, b):.6f}, rel {np.linalg.norm(a - b) / np.linalg.norm(b):.2e}")
        assert _cos(a, b) >= 0.999, k
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-6, k


def test_residual_loss_gradient_matches_oracle(setup):
    """Residual loss ||A16 M(r) - r||^2 / ||r||^2 (no error vectors needed)."""
    prob, s, A16 = setup
    import scipy.sparse as sp
    P = O.Problem(prob, diag_scale=1)
    A16full = sp.csr_matrix((P.get("a16"), prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    p = LI.init_params(readout_scale=0.5)
    flat = LI.flatten(p).astype(np.float32)
    s.learned_load(flat, train=True)
    s.learned_set_loss(1)
    try:
        R = rng.normal(13, 7, 2 * prob.n).reshape(2, prob.n).astype(np.float32)
        loss, grad = s.learned_loss_grad(dev(R), None)
    finally:
        s.learned_set_loss(0)
    pf = LI.unflatten(flat.astype(np.float64))
    want_loss, want = LM.loss_and_grad_residual(A16full, A16, pf, R.astype(np.float64), bf16=True)
    assert abs(loss - want_loss) <= 2e-2 * want_loss
    g = LI.unflatten(grad.astype(np.float64))
    for k in LI.PARAM_ORDER:
        a, b = np.ravel(g[k]), np.ravel(want[k])
        print(f"{k}: cos {_cos(a, b):.6f}, rel {np.linalg.norm(a - b) / np.linalg.norm(b):.2e}")
        assert _cos(a, b) >= 0.999, k
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-6, k


def test_arnoldi_training_pairs(setup):
    """Pairs from the fp64 solver's own Arnoldi vectors: r_k = D^-1/2 v_k with
    v_k orthonormal, and e_k solving A^ e_k = r_k."""
    prob, s, A16 = setup
    import scipy.sparse as sp
    rp, ci, va, b = dev(prob.rowptr), dev(prob.colidx), dev(prob.val), dev(prob.b)
    R, E = f3r.arnoldi_training_pairs(rp, ci, va, b, 6, tol=1e-11)
    P = O.Problem(prob, diag_scale=1)
    d = P.get("d")
    Ah = sp.csr_matrix((P.get("ahat"), prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    Rh, Eh = R.double().cpu().numpy(), E.double().cpu().numpy()
    Vh = Rh / d  # back to the original space: v_k = D^1/2 r_k
    G = Vh @ Vh.T
    assert np.abs(G - np.eye(6)).max() < 1e-5  # orthonormal up to the fp32 storage of r
    for k in range(6):
        assert np.linalg.norm(Ah @ Eh[k] - Rh[k]) <= 1e-6 * np.linalg.norm(Rh[k])


def test_training_reduces_loss_and_solves(setup):
    prob, s, A16 = setup
    n = prob.n
    # (residual, correction) pairs from the fp64 solver's Arnoldi vectors
    R, E = f3r.arnoldi_training_pairs(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), dev(prob.b), 8,
                                      tol=1e-11)
    R, E = R.cpu().numpy(), E.cpu().numpy()
    s.learned_load(LI.flatten(LI.init_params(readout_scale=0.0)).astype(np.float32), train=True)
    l0, _ = s.learned_loss_grad(dev(R), dev(E))
    hist = s.learned_train(dev(R), dev(E), steps=150, batch=4, lr=3e-3)
    l1, _ = s.learned_loss_grad(dev(R), dev(E))
    assert np.all(np.isfinite(hist)) and l1 < 0.9 * l0
    # the trained net as M inside the fp16 Richardson level: the fp64 outer level judges
    theta = s.learned_get()
    sl = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.default_params(precond=f3r.PC_LEARNED))
    sl.learned_load(theta)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = sl.solve(dev(prob.b), x)
    A = prob.to_scipy()
    rel = np.linalg.norm(prob.b - A @ x.cpu().numpy()) / np.linalg.norm(prob.b)
    assert res.status == f3r.OK and rel < 1e-9
    assert res.m_applies == 64 * res.outer_iters


def test_learned_against_jacobi_reported(setup):
    """What the trained net gains (or loses) against Jacobi-F3R on the same
    system and tolerance: outer iterations and solve time of both, printed.
    Asserted: both reach 1e-9 on the true residual (the fp64 outer level
    judges), and the net was trained (its training loss fell)."""
    prob, s, A16 = setup
    n = prob.n
    rp, ci, va, b = dev(prob.rowptr), dev(prob.colidx), dev(prob.val), dev(prob.b)
    R, E = f3r.arnoldi_training_pairs(rp, ci, va, b, 8, tol=1e-11)
    st = f3r.Solver(rp, ci, va, f3r.default_params(precond=f3r.PC_LEARNED))
    st.learned_load(LI.flatten(LI.init_params(readout_scale=0.0)).astype(np.float32), train=True)
    st.learned_set_loss(1)
    l0, _ = st.learned_loss_grad(R, None)
    st.learned_train(R, E, steps=200, batch=4, lr=3e-3)
    l1, _ = st.learned_loss_grad(R, None)
    theta = st.learned_get()
    st.close()
    assert l1 < l0
    A = prob.to_scipy()
    out = {}
    for name, prm in (("jacobi", f3r.default_params()), ("learned", f3r.default_params(precond=f3r.PC_LEARNED))):
        sv = f3r.Solver(rp, ci, va, prm)
        if name == "learned":
            sv.learned_load(theta)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        sv.solve(b, x)  # warm-up
        x.zero_()
        r = sv.solve(b, x)
        rel = np.linalg.norm(prob.b - A @ x.cpu().numpy()) / np.linalg.norm(prob.b)
        out[name] = (r.outer_iters, r.t_solve_ms, rel, r.status)
        sv.close()
    print(f"learned M: {out['learned'][0]} outer iterations, {out['learned'][1]:.2f} ms; "
          f"Jacobi: {out['jacobi'][0]} outer iterations, {out['jacobi'][1]:.2f} ms; "
          f"time ratio learned/Jacobi {out['learned'][1] / out['jacobi'][1]:.2f}")
    for name in out:
        assert out[name][3] == f3r.OK and out[name][2] < 1e-9, (name, out[name])

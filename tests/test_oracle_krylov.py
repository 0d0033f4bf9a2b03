"""Pins of the Krylov-comparator oracle (oracle/krylov.py): preconditioned CG
and BiCGStab in fp64 (Sec. 5's comparators)."""
import numpy as np
import scipy.sparse as sp

import oracle as O
from oracle import krylov as K
from problems import generators as G
from problems import rng


def _setup(prob, ds=1):
    P = O.Problem(prob, diag_scale=ds)
    d, m = K.preconditioner(P)
    return prob.to_scipy(), d, m


def test_cg_matches_dense_solution():
    prob = G.diffusion3d_7pt(dims=(7, 6, 5), seed=31)
    A, d, m = _setup(prob)
    res = K.solve("cg", A, prob.b, d, m, tol=1e-12)
    x = np.linalg.solve(A.toarray(), prob.b)
    kappa = np.linalg.cond(A.toarray())
    assert res["rel"] < 1e-12
    assert np.linalg.norm(res["x"] - x) <= kappa * 1e-12 * np.linalg.norm(x)


def test_cg_iterate_minimises_energy_error_over_krylov_space():
    """x_k minimises ||x - x*||_A over x0 + K_k(PA, P r0) (brute force by the
    normal equations of a dense Krylov basis)."""
    prob = G.diffusion3d_7pt(dims=(5, 5, 4), seed=32)
    A, d, m = _setup(prob)
    Ad = A.toarray()
    b = prob.b
    xs = np.linalg.solve(Ad, b)
    Pm = np.diag(d * m * d)
    z0 = Pm @ b
    for k in range(1, 5):
        xk = K.solve("cg", A, b, d, m, tol=1e-300, max_iters=k)["x"]
        Kb = np.column_stack([np.linalg.matrix_power(Pm @ Ad, q) @ z0 for q in range(k)])
        c = np.linalg.solve(Kb.T @ Ad @ Kb, Kb.T @ (Ad @ xs))
        xb = Kb @ c
        assert np.linalg.norm(xk - xb) <= 1e-9 * np.linalg.norm(xb), k


def test_bicgstab_matches_dense_solution_nonsymmetric():
    prob = G.convdiff3d_27pt(dims=(6, 6, 5), seed=33)
    A, d, m = _setup(prob)
    res = K.solve("bicgstab", A, prob.b, d, m, tol=1e-12)
    x = np.linalg.solve(A.toarray(), prob.b)
    assert res["rel"] < 1e-12 and not res["breakdown"]
    assert np.linalg.norm(res["x"] - x) <= 1e-9 * np.linalg.norm(x)


def test_exact_preconditioner_converges_in_one_iteration():
    """On a diagonal A the Jacobi preconditioner is A^-1 (P A = I up to
    rounding): both methods finish in one iteration."""
    n = 50
    a = 1.0 + 9.0 * rng.uniform01(34, 1, n)
    prob = G.Problem("diag", n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), a.copy(),
                     rng.uniform01(34, 2, n))
    A, d, m = _setup(prob)
    for method in ("cg", "bicgstab"):
        res = K.solve(method, A, prob.b, d, m, tol=1e-12)
        assert res["iters"] == 1 and res["rel"] < 1e-14, method


def test_restart_from_true_residual_and_iteration_cap():
    prob = G.diffusion3d_7pt(dims=(8, 8, 8), seed=35)
    A, d, m = _setup(prob)
    res = K.solve("cg", A, prob.b, d, m, tol=1e-9, max_iters=5)
    assert res["iters"] == 5 and res["rel"] > 1e-9
    full = K.solve("cg", A, prob.b, d, m, tol=1e-9)
    assert full["rel"] < 1e-9 and full["iters"] <= prob.n
    assert np.all(np.diff(np.log(full["hist"][:5])) < 0.5)
    assert sp.issparse(A)

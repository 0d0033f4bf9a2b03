"""Pins of the approximate-inverse preconditioner in the oracle:
M = (I - Dt^-1 U) Dt^-1 (I - L Dt^-1), Dt = alpha diag(A^), A^ = L + D + U."""
import numpy as np
import scipy.sparse as sp

import oracle as O
from problems import generators as G
from problems import rng


def _dense_m(P, n, rowptr, colidx, alpha):
    A = sp.csr_matrix((P.get("ahat"), colidx, rowptr), shape=(n, n)).toarray()
    L = np.tril(A, -1)
    U = np.triu(A, 1)
    Dt = alpha * np.diag(A)
    Dti = np.diag(1.0 / Dt)
    I = np.eye(n)
    return (I - Dti @ U) @ Dti @ (I - L @ Dti)


def test_application_is_the_dense_product():
    """m4 = 1 with unit weight is the bare preconditioner (Sec. 6.1): with fp64
    factors and vectors it equals the dense (I - Dt^-1 U) Dt^-1 (I - L Dt^-1)."""
    prob = G.convdiff3d_27pt(dims=(5, 4, 4), seed=41)
    n = prob.n
    for alpha in (1.0, 1.5):
        P = O.Problem(prob, diag_scale=1, precond=O.PC_AINV, ainv_alpha=alpha)
        prm = O.preset("fp64-F3R", precond=O.PC_AINV, rich_m=1, omega_fixed=1.0)
        v = rng.normal(42, 1, n)
        z = P.apply(prm, O.rich_state(), 3, v)
        want = _dense_m(P, n, prob.rowptr, prob.colidx, alpha) @ v
        assert np.linalg.norm(z - want) <= 1e-14 * np.linalg.norm(want), alpha


def test_factors_sit_on_their_triangles():
    prob = G.diffusion3d_7pt(dims=(5, 5, 5), seed=43)
    P = O.Problem(prob, diag_scale=1, precond=O.PC_AINV, ainv_alpha=1.2)
    rows = np.repeat(np.arange(prob.n), np.diff(prob.rowptr))
    lo, up = P.get("ainv_l"), P.get("ainv_u")
    assert np.all(lo[prob.colidx >= rows] == 0) and np.all(up[prob.colidx <= rows] == 0)
    assert np.all(lo[prob.colidx < rows] != 0) and np.all(up[prob.colidx > rows] != 0)
    ah = P.get("ahat")
    diag = ah[prob.colidx == rows]
    assert np.allclose(P.get("ainv_dinv"), 1.0 / (np.float64(np.float32(1.2)) * diag), rtol=0, atol=0)


def test_diagonal_matrix_solves_in_one_outer_iteration():
    """L = U = 0: M = Dt^-1 = A^-1 for alpha = 1, so R(v) = z exact to fp16."""
    n = 40
    a = 1.0 + 3.0 * rng.uniform01(44, 1, n)
    prob = G.Problem("diag", n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), a.copy(),
                     rng.uniform01(44, 2, n))
    P = O.Problem(prob, diag_scale=1, precond=O.PC_AINV)
    res = P.solve(O.params(precond=O.PC_AINV), prob.b)
    assert res.status == O.OK and res.outer_iters <= 2


def test_solve_with_ainv_converges_and_counts():
    prob = G.diffusion3d_7pt(dims=(12, 12, 12), seed=45)
    P = O.Problem(prob, diag_scale=1, precond=O.PC_AINV)
    res = P.solve(O.params(precond=O.PC_AINV), prob.b)
    assert res.status == O.OK and res.rel_res_true < 1e-9
    assert res.m_applies == 64 * res.outer_iters

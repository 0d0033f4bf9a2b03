"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: dense LU,
the Arnoldi relation, the Givens residual identity, finite termination, the
Krylov minimal-residual property, closed forms of Algorithm 1 on a diagonal
matrix, the special cases Sec. 4.3 and Sec. 6.1 name, the counting
invariant of Sec. 4.2 / Table 3, and the precision robustness of Sec. 5.1.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from problems import generators as G
from problems import rng

U16 = 2.0 ** -11
UBF = 2.0 ** -8
HERE = os.path.dirname(os.path.abspath(__file__))


def _diag_problem(n=64, seed=3, lo=1.0, hi=10.0):
    a = lo + (hi - lo) * rng.uniform01(seed, 1, n)
    rowptr = np.arange(n + 1, dtype=np.int32)
    colidx = np.arange(n, dtype=np.int32)
    return G.Problem("diag", n, rowptr, colidx, a.copy(), np.ones(n)), a


def _lu_pp_solve(A, b):
    """Textbook Gaussian elimination with partial pivoting."""
    A = A.astype(np.float64).copy()
    b = b.astype(np.float64).copy()
    n = len(b)
    for k in range(n - 1):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p]] = A[[p, k]]
            b[[k, p]] = b[[p, k]]
        l = A[k + 1:, k] / A[k, k]
        A[k + 1:, k + 1:] -= np.outer(l, A[k, k + 1:])
        b[k + 1:] -= l * b[k]
    x = np.zeros(n)
    for k in range(n - 1, -1, -1):
        x[k] = (b[k] - A[k, k + 1:] @ x[k + 1:]) / A[k, k]
    return x


# ------------------------------------------------------------------ set-up
def test_golden_defaults_match_paper(orc):
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "f3r_defaults.txt"))
            if l.strip() and not l.startswith("#")]
    tab = {r[0]: r[1:] for r in rows}
    p = O.params()
    assert [p.m[0], p.m[1], p.m[2], p.rich_m] == [int(tab[k][0]) for k in ("F1", "F2", "F3", "R")]
    names = {"fp64": O.F64, "fp32": O.F32, "fp16": O.F16}
    assert [p.a_prec[0], p.a_prec[1], p.a_prec[2], p.rich_a_prec] == \
        [names[tab[k][1]] for k in ("F1", "F2", "F3", "R")]
    assert [p.v_prec[0], p.v_prec[1], p.v_prec[2], p.rich_v_prec] == \
        [names[tab[k][2]] for k in ("F1", "F2", "F3", "R")]
    assert p.m_prec == names[tab["R"][3]]
    assert p.c == int(tab["c"][0]) and p.max_outer == int(tab["max_outer"][0])


def test_scaling_and_rounded_copies(orc):
    prob = G.convdiff3d_27pt(dims=(7, 6, 5), seed=9)
    A = prob.to_scipy()
    P = O.Problem(prob, diag_scale=1, row_scale=1)
    dinv = 1.0 / np.sqrt(np.abs(A.diagonal()))
    Ah = (sp.diags(dinv) @ A @ sp.diags(dinv)).tocsr()
    Ah.sort_indices()
    ah = P.get("ahat")
    assert np.allclose(ah, Ah.data, rtol=4e-16, atol=0)
    assert np.allclose(np.abs(Ah.diagonal()), 1.0, rtol=4e-16)
    assert np.array_equal(P.get("a32"), ah.astype(np.float32).astype(np.float64))
    rs = P.get("rs16")
    assert np.all(np.log2(rs) == np.round(np.log2(rs)))
    rowmax = np.maximum.reduceat(np.abs(ah), prob.rowptr[:-1])
    assert np.all((rowmax / rs > 0.5) & (rowmax / rs <= 1.0))
    s_nz = np.repeat(rs, np.diff(prob.rowptr))
    assert np.array_equal(P.get("a16"), (ah / s_nz).astype(np.float16).astype(np.float64))
    m = P.get("m64")
    assert np.allclose(m * Ah.diagonal(), 1.0, rtol=1e-15)
    assert np.array_equal(P.get("m16"), m.astype(np.float16).astype(np.float64))


def test_spmv_f64_matches_scipy(orc):
    prob = G.diffusion3d_7pt(dims=(9, 8, 7), seed=4)
    P = O.Problem(prob, diag_scale=0)
    x = rng.normal(1, 1, prob.n)
    assert np.allclose(P.spmv_orig(x), prob.to_scipy() @ x, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prec,u", [(O.F16, U16), (O.BF16, UBF)])
def test_spmv_16bit_elementwise_bound(orc, prec, u):
    """|y - A^ x| <= 2 u |A^||x| elementwise for a 16-bit copy of A^ (fp32 x)."""
    prob = G.convdiff3d_27pt(dims=(10, 9, 8), seed=5)
    P = O.Problem(prob, diag_scale=1, row_scale=1)
    x = rng.normal(2, 1, prob.n).astype(np.float32).astype(np.float64)
    Ah = sp.csr_matrix((P.get("ahat"), prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    exact = Ah @ x
    bound = 2 * u * (abs(Ah) @ np.abs(x))
    y = P.spmv(prec, O.F32, x)
    assert np.all(np.abs(y - exact) <= bound)


def test_spmv_f32_is_sequential_fused_multiply_add(orc):
    """Each row sum is fl32(a_k x_k + acc) in CSR order, checked with exact rationals."""
    prob = G.random_dd_sparse(60, per_row=5, seed=11)
    P = O.Problem(prob, diag_scale=1)
    x = rng.normal(3, 1, prob.n).astype(np.float32).astype(np.float64)
    y = P.spmv(O.F32, O.F32, x)
    a32 = P.get("a32")
    for i in range(prob.n):
        acc = np.float32(0.0)
        for k in range(prob.rowptr[i], prob.rowptr[i + 1]):
            exact = Fraction(float(a32[k])) * Fraction(float(x[prob.colidx[k]])) + Fraction(float(acc))
            acc = np.float32(float(exact))  # Fraction -> double is correctly rounded ...
            # ... and double -> float32 can double-round only on exact double ties; recheck
            lo, hi = np.nextafter(acc, np.float32(-np.inf)), np.nextafter(acc, np.float32(np.inf))
            d0 = abs(Fraction(float(acc)) - exact)
            assert d0 <= abs(Fraction(float(lo)) - exact) and d0 <= abs(Fraction(float(hi)) - exact)
        assert float(acc) == y[i]


# --------------------------------------------------------------- solver pins
@pytest.mark.parametrize("kind", ["poisson20", "random_nonsym"])
@pytest.mark.parametrize("preset", ["fp16-F3R", "fp32-F3R", "bf16-F3R"])
def test_solution_matches_dense_lu(orc, kind, preset):
    if kind == "poisson20":
        prob = G.poisson2d_5pt(20)
        ds = 0
    else:
        prob = G.random_dd_sparse(300, per_row=6, seed=12, dominance=1.1)
        ds = 1
    P = O.Problem(prob, diag_scale=ds, row_scale=1 if preset == "bf16-F3R" else 0)
    res = P.solve(O.preset(preset, diag_scale=ds), prob.b)
    A = prob.to_scipy().toarray()
    x_lu = _lu_pp_solve(A, prob.b)
    assert np.allclose(x_lu, np.linalg.solve(A, prob.b), rtol=1e-11, atol=1e-12)
    assert res.status == O.OK
    rel = np.linalg.norm(prob.b - A @ res.x) / np.linalg.norm(prob.b)
    assert rel < 1e-9 and abs(rel - res.rel_res_true) <= 1e-12
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(res.x - x_lu) / np.linalg.norm(x_lu) <= kappa * 1e-9


def test_outer_arnoldi_relation_fp64(orc):
    """A Z_m = V_{m+1} H_m and ||V^T V - I|| <= 1e-12 for the fp64 outer level,
    with the whole mixed-precision nest as its (flexible) preconditioner."""
    prob = G.convdiff3d_27pt(dims=(8, 8, 8), seed=13)
    P = O.Problem(prob)
    steps = 20
    V, Z, H = P.outer_arnoldi(O.params(), prob.b, steps)
    A = prob.to_scipy()
    lhs = (A @ Z.T)
    rhs = V.T @ H
    assert np.linalg.norm(lhs - rhs) / sp.linalg.norm(A) <= 1e-12
    assert np.abs(V @ V.T - np.eye(steps + 1)).max() <= 1e-12
    assert np.allclose(np.triu(H, -1), H)  # upper Hessenberg


def test_givens_estimate_equals_true_residual(orc):
    prob = G.diffusion3d_7pt(dims=(10, 10, 10), seed=14)
    P = O.Problem(prob)
    nb = np.linalg.norm(prob.b)
    A = prob.to_scipy()
    for k in range(1, 6):
        res = P.solve(O.params(max_outer=k, tol=0.0), prob.b)
        assert res.outer_iters == k
        true = np.linalg.norm(prob.b - A @ res.x) / nb
        assert abs(res.hist[-1] - true) <= 1e-6 * true + 1e-13


def test_finite_termination_identity(orc):
    n = 40
    prob = G.random_dd_sparse(n, per_row=4, seed=15, dominance=0.3)
    P = O.Problem(prob, diag_scale=0, precond=O.PC_IDENTITY)
    prm = O.params(nlevels=1, m=[n, 0, 0, 0], rich_m=0, m_prec=O.F64, tol=1e-13, max_outer=n,
                   diag_scale=0, precond=O.PC_IDENTITY)
    res = P.solve(prm, prob.b)
    A = prob.to_scipy()
    assert res.outer_iters <= n
    assert np.linalg.norm(prob.b - A @ res.x) / np.linalg.norm(prob.b) <= 1e-12


def test_minimal_residual_over_krylov_space(orc):
    n, m = 50, 10
    prob = G.random_dd_sparse(n, per_row=4, seed=16, dominance=0.5)
    A = prob.to_scipy().toarray()
    b = prob.b
    P = O.Problem(prob, diag_scale=0, precond=O.PC_IDENTITY)
    prm = O.params(nlevels=1, m=[m, 0, 0, 0], rich_m=0, m_prec=O.F64, tol=0.0, max_outer=m,
                   diag_scale=0, precond=O.PC_IDENTITY)
    res = P.solve(prm, b)
    # brute force: orthonormal basis of K_m(A, b) by Householder QR, then least squares
    K = np.empty((n, m))
    v = b.copy()
    for j in range(m):
        K[:, j] = v / np.linalg.norm(v)
        v = A @ K[:, j]
    Q, _ = np.linalg.qr(K)
    c, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    best = np.linalg.norm(b - A @ Q @ c)
    got = np.linalg.norm(b - A @ res.x)
    assert abs(got - best) <= 1e-9 * np.linalg.norm(b)


# ------------------------------------------------------------- Algorithm 1
def _rich_params(prec=O.F64, **kw):
    base = dict(nlevels=1, m=[10, 0, 0, 0], rich_m=2, rich_a_prec=prec, rich_v_prec=prec, m_prec=prec,
                diag_scale=0, precond=O.PC_IDENTITY)
    base.update(kw)
    return O.params(**base)


def test_richardson_closed_form_plain_call(orc):
    prob, a = _diag_problem()
    P = O.Problem(prob, diag_scale=0, precond=O.PC_IDENTITY)
    v = rng.normal(4, 1, prob.n)
    w1, w2 = 0.7, 0.35
    st = O.rich_state(c_ntr=5, omega=[w1, w2])
    z = P.apply(_rich_params(), st, 1, v)
    want = (1 - (1 - w1 * a) * (1 - w2 * a)) * v / a
    assert np.allclose(z, want, rtol=1e-14, atol=1e-15)
    assert st.c_ntr == 6 and st.omega[0] == w1 and st.omega[1] == w2


def test_richardson_closed_form_update_call(orc):
    prob, a = _diag_problem()
    P = O.Problem(prob, diag_scale=0, precond=O.PC_IDENTITY)
    v = rng.normal(5, 1, prob.n)
    st = O.rich_state(c_ntr=64, omega=[0.9, 1.2])
    z = P.apply(_rich_params(), st, 1, v)
    wp1 = np.sum(a * v * v) / np.sum((a * v) ** 2)       # (r, AMr)/(AMr, AMr), M = I
    r1 = v - a * (wp1 * v)
    wp2 = np.sum(a * r1 * r1) / np.sum((a * r1) ** 2)
    want = wp1 * v + wp2 * r1
    assert np.allclose(z, want, rtol=1e-13, atol=1e-14)
    # Eq. 5 with l = c_ntr / c = 1
    assert np.isclose(st.omega[0], (0.9 + wp1) / 2, rtol=1e-14)
    assert np.isclose(st.omega[1], (1.2 + wp2) / 2, rtol=1e-14)


def test_richardson_weight_sequence_is_cumulative_average(orc):
    """With the same v on every call, w'_k is the same on every update call, so
    after L updates w_k = (1 + L w'_k)/(L + 1) (initial weight 1, Eq. 5)."""
    prob, a = _diag_problem()
    P = O.Problem(prob, diag_scale=0, precond=O.PC_IDENTITY)
    v = rng.normal(6, 1, prob.n)
    c = 4
    prm = _rich_params(c=c)
    st = O.rich_state(c_ntr=1)
    wp1 = np.sum(a * v * v) / np.sum((a * v) ** 2)
    r1 = v - a * (wp1 * v)
    wp2 = np.sum(a * r1 * r1) / np.sum((a * r1) ** 2)
    for call in range(1, 4 * 64 + 1):
        P.apply(prm, st, 1, v)
        L = call // c
        assert np.isclose(st.omega[0], (1 + L * wp1) / (L + 1), rtol=1e-13)
        assert np.isclose(st.omega[1], (1 + L * wp2) / (L + 1), rtol=1e-13)


def test_richardson_fp16_within_rounding_of_closed_form(orc):
    prob, a = _diag_problem(lo=0.5, hi=1.0)
    P = O.Problem(prob, diag_scale=0, precond=O.PC_IDENTITY)
    v = rng.normal(7, 1, prob.n).astype(np.float32).astype(np.float64)
    w1, w2 = 0.8, 1.1
    st = O.rich_state(c_ntr=3, omega=[w1, w2])
    z = P.apply(_rich_params(O.F16, scale_cast=1), st, 1, v)
    want = (1 - (1 - w1 * a) * (1 - w2 * a)) * v / a
    # v, z1, r1, z2 and A each carry one fp16 rounding; |z1|, |r1| <= |v|
    assert np.all(np.abs(z - want) <= 12 * U16 * np.abs(v) / a + 1e-30)


def test_m4_1_with_unit_weight_is_the_bare_preconditioner(orc):
    """Sec. 6.1: with m4 = 1 and the weight left out, (R_m4, M) is M."""
    prob = G.convdiff3d_27pt(dims=(6, 6, 6), seed=17)
    P = O.Problem(prob, diag_scale=1)
    v = rng.normal(8, 1, prob.n)
    prm = O.params(nlevels=1, m=[10, 0, 0, 0], rich_m=1, omega_fixed=1.0, rich_a_prec=O.F64,
                   rich_v_prec=O.F64, m_prec=O.F64)
    z = P.apply(prm, O.rich_state(), 1, v)
    assert np.array_equal(z, P.get("m64") * v)


def test_update_every_call_is_gmres1(orc):
    """Sec. 4.3: computing w' on every call (c = 1) is GMRES(1) on A M."""
    prob = G.convdiff3d_27pt(dims=(6, 6, 6), seed=18)
    P = O.Problem(prob, diag_scale=1)
    Ah = sp.csr_matrix((P.get("ahat"), prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    m = P.get("m64")
    v = rng.normal(9, 1, prob.n)
    prm = O.params(nlevels=1, m=[10, 0, 0, 0], rich_m=1, c=1, rich_a_prec=O.F64, rich_v_prec=O.F64,
                   m_prec=O.F64)
    z = P.apply(prm, O.rich_state(c_ntr=7), 1, v)
    d = Ah @ (m * v)
    alpha = (v @ d) / (d @ d)
    assert np.allclose(z, alpha * m * v, rtol=1e-13)
    best = np.linalg.norm(v - Ah @ z)
    for t in np.linspace(0.5, 1.5, 21):
        assert best <= np.linalg.norm(v - t * alpha * d) + 1e-12


def test_structural_reduction_to_fgmres(orc):
    """(F_100, F_1, F_1, R_1 with w = 1, M = I) spans the same outer Krylov space
    as FGMRES(100) with M = I, so the residual histories coincide (fp64)."""
    prob = G.poisson2d_5pt(16)
    P = O.Problem(prob, diag_scale=0, precond=O.PC_IDENTITY)
    nest = O.preset("fp64-F3R", m=[100, 1, 1, 0], rich_m=1, omega_fixed=1.0, diag_scale=0,
                    precond=O.PC_IDENTITY, tol=1e-10)
    plain = O.params(nlevels=1, m=[100, 0, 0, 0], rich_m=0, m_prec=O.F64, diag_scale=0,
                     precond=O.PC_IDENTITY, tol=1e-10)
    h1 = P.solve(nest, prob.b).hist
    h2 = P.solve(plain, prob.b).hist
    k = min(len(h1), len(h2))
    assert abs(len(h1) - len(h2)) <= 1
    assert np.allclose(h1[:k], h2[:k], rtol=1e-6)


def test_counting_invariant(orc):
    """Sec. 4.2: the innermost level runs m2*m3*m4 = 64 M applications and
    m2*m3 = 32 Richardson calls per outer iteration (Table 3: multiples of 64)."""
    prob = G.poisson2d_5pt(32)
    P = O.Problem(prob, diag_scale=0)
    res = P.solve(O.params(diag_scale=0), prob.b)
    assert res.status == O.OK
    assert res.m_applies == 64 * res.outer_iters
    assert res.r_calls == 32 * res.outer_iters
    assert res.r_update_calls == (32 * res.outer_iters) // 64


def test_adaptive_inner_level_reductions(orc):
    """Adaptive m3 (Sec. 6 / Sec. 7, stop the innermost FGMRES level once
    |g_{j+1}| <= rtol * beta): a threshold no estimate reaches is the fixed-m
    solver exactly; a threshold every first step meets (|g_1| = |s_0| beta <
    beta) is m3 = 1 exactly when the weights are fixed (the weight counter
    then plays no part)."""
    prob = G.diffusion3d_7pt(dims=(12, 11, 10), seed=23)
    P = O.Problem(prob, diag_scale=1)
    a = P.solve(O.params(inner_rtol=1e-300), prob.b)
    b = P.solve(O.params(), prob.b)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.hist, b.hist) and a.r_calls == b.r_calls
    c = P.solve(O.params(inner_rtol=1.0 - 2.0 ** -20, omega_fixed=1.0), prob.b)
    d = P.solve(O.params(m=[100, 8, 1, 0], omega_fixed=1.0), prob.b)
    assert np.array_equal(c.x, d.x) and np.array_equal(c.hist, d.hist)
    assert c.r_calls == d.r_calls == 8 * c.outer_iters


def test_adaptive_inner_level_counts(orc):
    """With a moderate threshold the level runs fewer Richardson calls than it
    schedules; every executed call still applies M m4 times, and the solve
    converges."""
    prob = G.diffusion3d_7pt(dims=(14, 14, 14), seed=24)
    P = O.Problem(prob, diag_scale=1)
    res = P.solve(O.params(m=[100, 8, 8, 0], inner_rtol=0.2), prob.b)
    assert res.status == O.OK and res.rel_res_true < 1e-9
    assert 8 * res.outer_iters <= res.r_calls < 64 * res.outer_iters
    assert res.m_applies == 2 * res.r_calls


def test_fp16_iterations_close_to_fp64(orc):
    """Sec. 5.1: fp16-F3R needs at most ~9 % more iterations than fp64-F3R."""
    for prob, ds in [(G.poisson2d_5pt(64), 0), (G.diffusion3d_7pt(dims=(20, 20, 20), seed=19), 1)]:
        P = O.Problem(prob, diag_scale=ds)
        i16 = P.solve(O.preset("fp16-F3R", diag_scale=ds), prob.b).outer_iters
        i64 = P.solve(O.preset("fp64-F3R", diag_scale=ds), prob.b).outer_iters
        assert i16 <= 1.1 * i64 + 1


def test_restart_after_m1(orc):
    """Sec. 4.2: if m1 outer iterations are not enough the nest is run again
    from the current x (restart); the count of outer iterations continues."""
    prob = G.diffusion3d_7pt(dims=(16, 16, 16), seed=20)
    P = O.Problem(prob)
    res = P.solve(O.params(m=[3, 8, 4, 0]), prob.b)
    assert res.status == O.OK
    assert res.restarts == (res.outer_iters - 1) // 3
    assert len(res.true_hist) == res.restarts + 2


def test_not_converged_status(orc):
    prob = G.diffusion3d_7pt(dims=(16, 16, 16), seed=21)
    P = O.Problem(prob)
    res = P.solve(O.params(max_outer=2), prob.b)
    assert res.status == O.NOT_CONVERGED and res.outer_iters == 2
    assert res.rel_res_true > 1e-9

"""Pins of the oracle's inner levels: the fp32 FGMRES levels F_{m2}, F_{m3},
the D^{-1/2} map that enters the scaled system, and the rounding points of
Algorithm 1.

Each pin checks the oracle against something other than itself:
* the Arnoldi relation A Z_k = V_{k+1} H_k and the orthonormality of V at
  the fp32 levels (Sec. 4.2: each inner level is FGMRES in its own
  precision), to 50 m u32 (u32 = 2^-24);
* the Givens least-squares state against numpy's dense least squares on the
  recorded Hessenberg matrix, and the level's true residual ||v - A z||;
* the map P(v) = D^{-1/2} F(D^{-1/2} v) against A^{-1} v when the inner level
  solves exactly (fp64, m >= n);
* Richardson calls (Algorithm 1, Table 1) on a diagonal matrix worked by hand
  in exact rational arithmetic with a float16 rounding at each declared store
  and nowhere else.
Where a pin could pass by accident, the test also shows that the plausible
mistake (one Gram-Schmidt pass, one D^{-1/2}, a dropped or extra fp16 store)
fails it.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from problems import generators as G
from problems import rng

U32 = 2.0 ** -24


def _level_matrix(P, prob, prec):
    """The level's copy of A^ (values as the level stores them, row scale applied)."""
    if prec == O.F32:
        vals = P.get("a32")
    elif prec == O.F16:
        vals = P.get("a16") * np.repeat(P.get("rs16"), np.diff(prob.rowptr))
    elif prec == O.BF16:
        vals = P.get("abf16") * np.repeat(P.get("rsbf16"), np.diff(prob.rowptr))
    else:
        vals = P.get("ahat")
    return sp.csr_matrix((vals, prob.colidx, prob.rowptr), shape=(prob.n, prob.n))


_CASES = [
    ("diffusion7", lambda: G.diffusion3d_7pt(dims=(12, 11, 10), seed=31)),
    ("convdiff27", lambda: G.convdiff3d_27pt(dims=(9, 8, 7), seed=32)),
]
_LEVELS = [(1, O.F32), (2, O.F16)]  # F_{m2}: fp32 A; F_{m3}: fp16 A, fp32 vectors (Table 1)


def _inner_call(prob, level, **kw):
    P = O.Problem(prob)
    prm = O.params(**kw)
    v = rng.normal(40 + level, 1, prob.n).astype(np.float32).astype(np.float64)
    z, V, Z, H, g, k = P.inner_arnoldi(prm, O.rich_state(), level, v)
    return P, prm, v, z, V, Z, H, g, k


@pytest.mark.parametrize("case", _CASES, ids=[c[0] for c in _CASES])
@pytest.mark.parametrize("level,aprec", _LEVELS, ids=["F2", "F3"])
def test_inner_arnoldi_relation_fp32(orc, case, level, aprec):
    """Per column: ||A z_j - V h_j|| <= 50 m u32 ||A||_F ||z_j||, and
    ||V^T V - I||_max <= 50 m u32 for the k+1 basis vectors (CGS2)."""
    prob = case[1]()
    P, prm, v, z, V, Z, H, g, k = _inner_call(prob, level)
    m = prm.m[level]
    assert k == m
    A = _level_matrix(P, prob, aprec)
    R = A @ Z[:k].T - V[:k + 1].T @ H[:k + 1, :k]
    col = np.linalg.norm(R, axis=0) / (sp.linalg.norm(A) * np.linalg.norm(Z[:k], axis=1))
    assert col.max() <= 50 * m * U32
    assert np.abs(V[:k + 1] @ V[:k + 1].T - np.eye(k + 1)).max() <= 50 * m * U32
    assert np.allclose(np.triu(H, -1), H)  # upper Hessenberg
    assert np.all(np.diag(H, -1)[:k] > 0)   # h_{j+1,j} = ||w|| > 0


@pytest.mark.parametrize("case", _CASES, ids=[c[0] for c in _CASES])
def test_long_inner_level_arnoldi_relation(orc, case):
    """Table 4's F2: an inner fp32 FGMRES(64) keeps the Arnoldi relation and
    an orthonormal basis to 50 m u32, and its output is Z y for the numpy
    least-squares y of the recorded Hessenberg matrix."""
    prob = case[1]()
    P = O.Problem(prob)
    prm = O.preset("F2")
    v = rng.normal(45, 1, prob.n).astype(np.float32).astype(np.float64)
    z, V, Z, H, g, k = P.inner_arnoldi(prm, O.rich_state(), 1, v)
    m = prm.m[1]
    assert m == 64 and k == m
    A = _level_matrix(P, prob, O.F32)
    R = A @ Z[:k].T - V[:k + 1].T @ H[:k + 1, :k]
    col = np.linalg.norm(R, axis=0) / (sp.linalg.norm(A) * np.linalg.norm(Z[:k], axis=1))
    assert col.max() <= 50 * m * U32
    assert np.abs(V[:k + 1] @ V[:k + 1].T - np.eye(k + 1)).max() <= 50 * m * U32
    e1 = np.zeros(k + 1)
    e1[0] = np.linalg.norm(v)
    y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
    assert np.linalg.norm(z - Z[:k].T @ y) <= 1e-4 * np.linalg.norm(z)


def test_inner_orthogonality_pin_rejects_single_pass(orc):
    """The orthogonality bound separates CGS2 from one classical pass: with one
    pass the fp32 F_{m2} basis loses orthogonality by orders of magnitude."""
    prob = _CASES[0][1]()
    lvl = 1
    *_, V2, _, _, _, k2 = _inner_call(prob, lvl)
    *_, V1, _, _, _, k1 = _inner_call(prob, lvl, cgs_passes=1)
    m = O.params().m[lvl]
    e2 = np.abs(V2[:k2 + 1] @ V2[:k2 + 1].T - np.eye(k2 + 1)).max()
    e1 = np.abs(V1[:k1 + 1] @ V1[:k1 + 1].T - np.eye(k1 + 1)).max()
    assert e2 <= 50 * m * U32 < e1


@pytest.mark.parametrize("case", _CASES, ids=[c[0] for c in _CASES])
@pytest.mark.parametrize("level,aprec", _LEVELS, ids=["F2", "F3"])
def test_inner_givens_least_squares(orc, case, level, aprec):
    """The rotated right-hand side and the level output solve the level's small
    least-squares problem min_y ||beta e1 - H y|| (numpy, fp64, on the recorded
    H): |g_k| equals its minimum to 1e-4 relative (plus 10 m u32 beta), z equals
    Z y to 1e-4, and the true residual ||v - A z|| equals |g_k| to 100 m u32 beta."""
    prob = case[1]()
    P, prm, v, z, V, Z, H, g, k = _inner_call(prob, level)
    m = prm.m[level]
    A = _level_matrix(P, prob, aprec)
    beta = np.linalg.norm(v)
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
    ls = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
    assert abs(abs(g[k]) - ls) <= 1e-4 * ls + 10 * m * U32 * beta
    zy = Z[:k].T @ y
    assert np.linalg.norm(z - zy) <= 1e-4 * np.linalg.norm(zy)
    assert abs(np.linalg.norm(v - A @ z) - abs(g[k])) <= 100 * m * U32 * beta
    # g_0 = beta before rotation; every rotation preserves the norm of g
    assert abs(np.linalg.norm(g[:k + 1]) - beta) <= 10 * m * U32 * beta


@pytest.mark.parametrize("seed", [41, 42])
def test_scaled_inner_map_is_exact_inverse(orc, seed):
    """Reading of Sec. 5's diagonal scaling: the outer level runs on A and the
    nest is P(v) = D^{-1/2} F(D^{-1/2} v) with F solving A^ = D^{-1/2} A D^{-1/2}.
    With an exact inner solve (fp64 FGMRES(n), M = I) P(v) = A^{-1} v; applying
    D^{-1/2} once instead of twice would give D^{-1/2} A^{-1} v-like vectors far
    from it."""
    n = 40
    prob = G.random_dd_sparse(n, per_row=5, seed=seed, dominance=1.2)
    A = prob.to_scipy().toarray()
    assert np.ptp(np.abs(np.diag(A))) > 1.0  # D is far from a multiple of I
    P = O.Problem(prob, diag_scale=1, precond=O.PC_IDENTITY)
    f64 = [O.F64] * 4
    prm = O.params(nlevels=2, m=[1, n, 0, 0], a_prec=f64, v_prec=f64, rich_m=0, m_prec=O.F64,
                   precond=O.PC_IDENTITY, diag_scale=1, tol=0.0)
    V, Z, H = P.outer_arnoldi(prm, prob.b, 1)
    want = np.linalg.solve(A, V[0])
    assert np.linalg.norm(Z[0] - want) <= 1e-12 * np.linalg.norm(want)
    d = P.get("d")
    Ah = _level_matrix(P, prob, O.F64).toarray()
    once = d * np.linalg.solve(Ah, V[0])
    assert np.linalg.norm(once - want) > 0.1 * np.linalg.norm(want)


# ------------------------------------------------- Algorithm 1 rounding points
def _round_exact(x: Fraction, p: int, emin: int) -> Fraction:
    """Round a rational to p significand bits, ties to even, gradual underflow
    below 2^emin (IEEE 754 roundTiesToEven; no overflow in these pins)."""
    if x == 0:
        return Fraction(0)
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()  # floor(log2 a) or one more
    if Fraction(2) ** e > a:
        e -= 1
    spacing = Fraction(2) ** (max(e, emin) - (p - 1))
    q = round(a / spacing)  # Fraction.__round__: nearest integer, ties to even
    return (q * spacing) if x > 0 else -(q * spacing)


def _f16(x: Fraction) -> Fraction:
    return _round_exact(x, 11, -14)


def _f32(x: Fraction) -> Fraction:
    return _round_exact(x, 24, -126)


def test_exact_rounding_helper_matches_numpy(orc):
    """The rational rounding used below agrees with numpy's float16 / float32
    casts on values exact in double, including ties."""
    xs = rng.normal(70, 1, 4000) * 2.0 ** np.round(rng.normal(71, 1, 4000) * 5)
    xs = xs[np.abs(xs) < 65504]  # inside the binary16 range
    ties = [1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -24 * 1.5, 2.0 ** -25]
    for x in list(xs) + ties:
        assert float(_f16(Fraction(x))) == float(np.float16(x))
        assert float(_f32(Fraction(x))) == float(np.float32(x))


def _rich_by_hand(a, v, omegas, store16=True, round_r=True, round_u=False):
    """One plain call of Algorithm 1 (z_0 = 0, fixed weights) on A = diag(a),
    M = diag(fl16(1/a)), written out entry by entry in exact rationals.

    The rounding points (Table 1; 16-bit storage, fp32 arithmetic):
      v16 = fl16(sigma v), sigma = 2^-floor(log2 max|v|)
      r_k = fl16(fl32(v16 - a z_k))        (r_0 = v16)
      u_k = fl32(m r_k)                    (exact: two 11-bit factors)
      z_{k+1} = fl16(fl32(omega_k u_k + z_k))
      out = z_m4 / sigma
    The flags plant the mistakes the pin has to catch."""
    vmax = max(abs(x) for x in v)
    e = int(np.floor(np.log2(vmax)))
    sigma = Fraction(2) ** (-e)
    out = []
    for ai, vi in zip(a, v):
        ai = Fraction(ai)
        mi = _f16(Fraction(1) / ai)
        v16 = _f16(sigma * Fraction(vi))
        z = Fraction(0)
        for k, w in enumerate(omegas):
            if k == 0:
                r = v16
            else:
                r = _f32(v16 - _f32(ai * z))
                if round_r:
                    r = _f16(r)
            u = _f32(mi * r)
            if round_u:
                u = _f16(u)
            z = _f32(Fraction(w) * u + z)
            if store16:
                z = _f16(z)
        out.append(float(z / sigma))
    return np.array(out)


def _one_over_fp16(a):
    """1 / a rounded once to fp16 from the exact quotient."""
    return np.array([float(_f16(Fraction(1) / Fraction(x))) for x in a])


@pytest.mark.parametrize("m4", [2, 3])
def test_richardson_rounding_points_by_hand(orc, m4):
    """A plain Richardson call equals the hand-worked rounding points bit for bit,
    and each planted mistake (r kept in fp32, u rounded to fp16, z kept in fp32)
    changes some entries, so the pin would catch it."""
    n = 256
    base = np.array([3.0, 5.0, 6.0, 7.0, 1.5, 2.5, 0.75, 9.0])  # exact in fp16; 1/a is not
    a = base[np.arange(n) % base.size]
    prob = G.Problem("diag", n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                     a.copy(), np.ones(n))
    P = O.Problem(prob, diag_scale=0, precond=O.PC_JACOBI)
    assert np.array_equal(P.get("m16"), _one_over_fp16(a))
    # fp32 inputs with more than 11 significant bits, a range of binades
    v = (rng.normal(50 + m4, 1, n) * 2.0 ** rng.uniform01(60 + m4, 1, n) * 3).astype(np.float32).astype(np.float64)
    # dyadic weights, exact in fp32, below 1 so the residuals stay comparable to
    # z and their fp16 rounding shows in the result
    omegas = [0.375, 0.5, 0.625][:m4]
    prm = O.params(nlevels=1, m=[10, 0, 0, 0], rich_m=m4, rich_a_prec=O.F16, rich_v_prec=O.F16,
                   m_prec=O.F16, diag_scale=0, precond=O.PC_JACOBI, scale_cast=1)
    st = O.rich_state(c_ntr=5, omega=omegas)
    z = P.apply(prm, st, 1, v)
    want = _rich_by_hand(a, v, omegas)
    assert np.array_equal(z, want)
    assert st.c_ntr == 6
    for planted in (dict(round_r=False), dict(round_u=True), dict(store16=False)):
        assert not np.array_equal(_rich_by_hand(a, v, omegas, **planted), want), planted


def test_richardson_update_call_by_hand(orc):
    """An update call (c_ntr = c) on a 2 x 2 diagonal system, worked by hand:
    u stays fp32, w = A u in fp32, w' = fl32(fl32(r.w) / fl32(w.w)) with the dot
    products as two fused multiply-adds, z_1 = fl16(fl32(w' u)), and the weight
    becomes (l w + w') / (l + 1) with l = c_ntr / c = 1 (Eq. 5)."""
    a = [3.0, 5.0]
    v = [0.8125 + 2.0 ** -14, -0.37109375]  # v[0] needs rounding to fp16
    n = 2
    prob = G.Problem("diag2", n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                     np.array(a), np.ones(n))
    P = O.Problem(prob, diag_scale=0, precond=O.PC_JACOBI)
    prm = O.params(nlevels=1, m=[10, 0, 0, 0], rich_m=1, rich_a_prec=O.F16, rich_v_prec=O.F16,
                   m_prec=O.F16, diag_scale=0, precond=O.PC_JACOBI, scale_cast=1, c=64)
    st = O.rich_state(c_ntr=64, omega=[0.5])
    z = P.apply(prm, st, 1, np.array(v))

    F = Fraction
    sigma = F(2)  # max|v| lies in [1/2, 1), so sigma = 2^-floor(log2 max|v|) = 2
    v16 = [_f16(sigma * F(x)) for x in v]
    m16 = [_f16(F(1) / F(x)) for x in a]
    u = [_f32(mi * ri) for mi, ri in zip(m16, v16)]
    w = [_f32(F(ai) * ui) for ai, ui in zip(a, u)]
    num = _f32(v16[0] * w[0])
    num = _f32(v16[1] * w[1] + num)
    den = _f32(w[0] * w[0])
    den = _f32(w[1] * w[1] + den)
    wp = _f32(num / den)
    z1 = [_f16(_f32(wp * ui)) for ui in u]
    want = [float(zz / sigma) for zz in z1]
    assert list(z) == want
    # Eq. 5 with l = 1, in fp32
    lw = np.float32(1.0) * np.float32(0.5) + np.float32(float(wp))
    assert st.omega[0] == float(lw / np.float32(2.0))
    assert st.c_ntr == 65

"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bit-exact where the method's arithmetic is elementwise or a row sum in a fixed
order (set-up conversions, SpMV, a plain Richardson call); within stated
tolerances where reductions enter (dot products are summed in a tree on the
GPU and sequentially in the oracle).
"""
import numpy as np
import pytest

import oracle as O
from problems import generators as G
from problems import rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_20719_gb300 import f3r  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solver(prob, prm, on_device=True):
    if on_device:
        return f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), prm)
    return f3r.Solver.from_problem(prob, prm)


def f16_bits(vals):
    return vals.astype(np.float16).view(np.uint16)


def bf16_bits(vals):
    return (vals.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


@pytest.fixture(scope="module")
def convdiff():
    return G.convdiff3d_27pt(dims=(21, 19, 17), seed=101)


# ---------------------------------------------------------------- set-up
@pytest.mark.parametrize("row_scale", [0, 1])
def test_setup_copies_bit_exact(convdiff, row_scale):
    prob = convdiff
    P = O.Problem(prob, diag_scale=1, row_scale=row_scale)
    s16 = solver(prob, f3r.default_params(row_scale=row_scale))
    assert np.array_equal(s16.export(0), P.get("d"))
    assert np.array_equal(s16.export(2, prob.nnz), P.get("a32").astype(np.float32))
    assert np.array_equal(s16.export(3, prob.nnz), f16_bits(P.get("a16")))
    assert np.array_equal(s16.export(6), f16_bits(P.get("m16")))
    if row_scale:
        assert np.array_equal(s16.export(5).astype(np.float64), P.get("rs16"))
    sbf = solver(prob, f3r.preset("bf16-F3R", row_scale=row_scale))
    assert np.array_equal(sbf.export(4, prob.nnz), bf16_bits(P.get("abf16")))
    assert np.array_equal(sbf.export(6), bf16_bits(P.get("mbf16")))
    s64 = solver(prob, f3r.preset("fp64-F3R"))
    assert np.array_equal(s64.export(1, prob.nnz), P.get("ahat"))
    assert np.array_equal(s64.export(6).view(np.float64), P.get("m64"))


# ------------------------------------------------------------------ SpMV
def _spmv_cases():
    return [("orig", f3r.F64, f3r.F64), ("f32", f3r.F32, f3r.F32), ("f16", f3r.F16, f3r.F32),
            ("f16x16", f3r.F16, f3r.F16), ("bf16", f3r.BF16, f3r.F32)]


@pytest.mark.parametrize("name,p,vp", _spmv_cases())
@pytest.mark.parametrize("row_scale", [0, 1])
def test_spmv_bit_exact(convdiff, name, p, vp, row_scale):
    prob = convdiff
    n = prob.n
    if p == f3r.BF16:
        prm = f3r.preset("bf16-F3R", row_scale=row_scale)
    elif p == f3r.F32:
        prm = f3r.preset("fp32-F3R", row_scale=row_scale)
    else:
        prm = f3r.default_params(row_scale=row_scale)
    s = solver(prob, prm)
    P = O.Problem(prob, diag_scale=1, row_scale=row_scale)
    x = rng.normal(7, 1, n)
    if p == f3r.F64:
        xd = dev(x)
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        want = P.spmv_orig(x)
    else:
        if vp == f3r.F16:
            x = x.astype(np.float16).astype(np.float64)
            xd = dev(x.astype(np.float16))
        else:
            x = x.astype(np.float32).astype(np.float64)
            xd = dev(x.astype(np.float32))
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        want = P.spmv({f3r.F32: O.F32, f3r.F16: O.F16, f3r.BF16: O.BF16}[p], O.F32, x)
    s.spmv(p, vp, xd, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("which", ["diffusion7_128", "convdiff27_160"])
def test_spmv_full_size_bit_exact(which):
    """Full workload sizes, in the solver's launch configuration: every row."""
    prob = G.by_name(which)
    s = solver(prob, f3r.default_params())
    P = O.Problem(prob, diag_scale=1)
    x = rng.normal(8, 1, prob.n).astype(np.float32)
    y = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.spmv(f3r.F16, f3r.F32, dev(x), y)
    torch.cuda.synchronize()
    want = P.spmv(O.F16, O.F32, x.astype(np.float64))
    assert np.array_equal(y.cpu().numpy().astype(np.float64), want)


def test_spmv_and_solve_random_far_columns():
    """A random sparse pattern (columns up to n away from their row, no
    locality for the x gathers): SpMV bit-exact and the solve converges."""
    prob = G.random_dd_sparse(70000, per_row=5, seed=109, dominance=1.5)
    rows = np.repeat(np.arange(prob.n), np.diff(prob.rowptr))
    assert np.max(np.abs(prob.colidx.astype(np.int64) - rows)) > 32767
    s = solver(prob, f3r.default_params())
    P = O.Problem(prob, diag_scale=1)
    x = rng.normal(10, 1, prob.n).astype(np.float32)
    y = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.spmv(f3r.F16, f3r.F32, dev(x), y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy().astype(np.float64), P.spmv(O.F16, O.F32, x.astype(np.float64)))
    xs = np.zeros(prob.n)
    res = s.solve(np.ascontiguousarray(prob.b), xs)
    A = prob.to_scipy()
    assert res.status == f3r.OK and np.linalg.norm(prob.b - A @ xs) / np.linalg.norm(prob.b) < 1e-9


# ------------------------------------------------------------- Richardson
def _rich_prm(kind, **kw):
    if kind == "fp16":
        return f3r.default_params(**kw)
    if kind == "bf16":
        return f3r.preset("bf16-F3R", **kw)
    if kind == "fp32":
        return f3r.preset("fp32-F3R", **kw)
    return f3r.preset("fp64-F3R", **kw)


def _orc_prm(kind, **kw):
    name = {"fp16": "fp16-F3R", "bf16": "bf16-F3R", "fp32": "fp32-F3R", "fp64": "fp64-F3R"}[kind]
    return O.preset(name, **kw)


@pytest.mark.parametrize("kind", ["fp16", "bf16", "fp32", "fp64"])
@pytest.mark.parametrize("m4", [1, 2, 3])
def test_richardson_plain_call_bit_exact(convdiff, kind, m4):
    prob = convdiff
    n = prob.n
    rs = 1 if kind == "bf16" else 0
    s = solver(prob, _rich_prm(kind, rich_m=m4))
    P = O.Problem(prob, diag_scale=1, row_scale=rs)
    v = rng.normal(9, 1, n) * 1e-3
    omega = [0.83, 1.07, 0.91][:m4]
    s.set_rich_state(omega, 5)
    is64 = kind == "fp64"
    vt = v if is64 else v.astype(np.float32)
    z = torch.empty(n, dtype=torch.float64 if is64 else torch.float32, device="cuda")
    s.apply(3, dev(vt), z)
    torch.cuda.synchronize()
    st = O.rich_state(c_ntr=5, omega=omega)
    want = P.apply(_orc_prm(kind, rich_m=m4), st, 3, vt.astype(np.float64))
    assert np.array_equal(z.cpu().numpy().astype(np.float64), want)
    om, cn = s.rich_state()
    assert cn == 6 and om[:m4] == pytest.approx(omega)


@pytest.mark.parametrize("kind", ["fp16", "bf16", "fp32"])
def test_richardson_update_call(convdiff, kind):
    """Every c-th call computes w' = (r, AMr)/(AMr, AMr) in fp32 (Algorithm 1);
    the dot products are reductions, so w' agrees to fp32 rounding."""
    prob = convdiff
    n = prob.n
    rs = 1 if kind == "bf16" else 0
    s = solver(prob, _rich_prm(kind))
    P = O.Problem(prob, diag_scale=1, row_scale=rs)
    v = (rng.normal(10, 1, n) * 1e-3).astype(np.float32)
    s.set_rich_state([0.9, 1.1], 128)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    s.apply(3, dev(v), z)
    torch.cuda.synchronize()
    st = O.rich_state(c_ntr=128, omega=[0.9, 1.1])
    want = P.apply(_orc_prm(kind), st, 3, v.astype(np.float64))
    got = z.cpu().numpy().astype(np.float64)
    om, cn = s.rich_state()
    assert cn == 129
    assert np.allclose(om[:2], list(st.omega)[:2], rtol=2e-5, atol=0)
    assert np.linalg.norm(got - want) <= 2e-3 * np.linalg.norm(want)


# ------------------------------------------------------------ inner levels
@pytest.mark.parametrize("fuse", [1, 0])
@pytest.mark.parametrize("kind", ["fp16", "bf16", "fp32", "fp64"])
@pytest.mark.parametrize("level", [1, 2])
def test_inner_level_call(convdiff, kind, level, fuse):
    """One call of F_{m2} (level 1) or F_{m3} (level 2) against the oracle,
    with the fused cooperative CGS2 / normalisation kernel and without."""
    prob = convdiff
    n = prob.n
    rs = 1 if kind == "bf16" else 0
    s = solver(prob, _rich_prm(kind, fuse_cgs=fuse))
    P = O.Problem(prob, diag_scale=1, row_scale=rs)
    is64 = kind == "fp64"
    v = rng.normal(11, 1, n)
    v = v / np.linalg.norm(v)
    vt = v if is64 else v.astype(np.float32)
    z = torch.empty(n, dtype=torch.float64 if is64 else torch.float32, device="cuda")
    s.set_rich_state([1.0, 1.0], 2)
    s.apply(level, dev(vt), z)
    torch.cuda.synchronize()
    want = P.apply(_orc_prm(kind), O.rich_state(c_ntr=2), level, vt.astype(np.float64))
    got = z.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    # GPU and oracle differ only in the summation order of dot products (tree
    # vs sequential: ~sqrt(n) u32 relative), amplified by the level's small
    # least-squares solve; at the 16-bit levels that perturbation moves a
    # fraction ~ (perturbation / u) of the entries cast to 16 bits by one ulp
    # each (u16 = 2^-11, u_bf = 2^-8), a level-output change of order 1e-4.
    # Bounds: fp16 10 u16, bf16 2.5 u_bf.
    tol = {"fp64": 1e-12, "fp32": 1e-4, "fp16": 10 * 2.0 ** -11, "bf16": 2.5 * 2.0 ** -8}[kind]
    print(f"level {level} {kind}: rel diff {err:.3e}")
    assert err <= tol


# ------------------------------------------------------------- full solves
def _solve_both(prob, kind, ds=1, **kw):
    rs = 1 if kind == "bf16" else 0
    prm = _rich_prm(kind, diag_scale=ds, **kw) if kind != "fgmres64" else f3r.preset("fgmres64", diag_scale=ds, **kw)
    s = solver(prob, prm)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    res = s.solve(dev(prob.b), x)
    torch.cuda.synchronize()
    P = O.Problem(prob, diag_scale=ds, row_scale=rs)
    oprm = _orc_prm(kind, diag_scale=ds, **kw) if kind != "fgmres64" else O.preset("fgmres64", diag_scale=ds, **kw)
    ref = P.solve(oprm, prob.b)
    return res, ref, x.cpu().numpy()


def _check_history(res, ref, prob, xg, tol=1e-9):
    A = prob.to_scipy()
    rel = np.linalg.norm(prob.b - A @ xg) / np.linalg.norm(prob.b)
    assert res.status == f3r.OK and ref.status == O.OK
    assert rel < tol and res.rel_res_true < tol
    assert abs(rel - res.rel_res_true) <= 1e-3 * tol
    assert abs(res.outer_iters - ref.outer_iters) <= max(1, int(0.1 * ref.outer_iters))
    k = min(len(res.hist), len(ref.hist))
    mask = ref.hist[:k] > 1e-8
    ratio = np.abs(np.log10(res.hist[:k][mask] / ref.hist[:k][mask]))
    assert np.all(ratio <= 0.5), ratio


@pytest.mark.parametrize("kind", ["fp16", "fp32", "fp64", "bf16"])
def test_solve_poisson64_matches_oracle(kind):
    """2-D Poisson 64x64, Jacobi, unscaled (the small F3R workload)."""
    prob = G.poisson2d_5pt(64)
    res, ref, xg = _solve_both(prob, kind, ds=0)
    _check_history(res, ref, prob, xg)
    assert np.linalg.norm(xg - prob.x_true) / np.linalg.norm(prob.x_true) < 1e-6
    assert res.m_applies == 64 * res.outer_iters and res.r_calls == 32 * res.outer_iters
    assert res.r_update_calls == (32 * res.outer_iters) // 64


@pytest.mark.parametrize("kind", ["fp16", "bf16", "fp32"])
def test_solve_diffusion_matches_oracle(kind):
    prob = G.diffusion3d_7pt(dims=(24, 24, 24), seed=102)
    res, ref, xg = _solve_both(prob, kind)
    _check_history(res, ref, prob, xg)


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_solve_convdiff_matches_oracle(kind):
    prob = G.convdiff3d_27pt(dims=(20, 20, 20), seed=103)
    res, ref, xg = _solve_both(prob, kind)
    _check_history(res, ref, prob, xg)


@pytest.mark.parametrize("name", ["F2", "fp16-F2", "F3", "fp16-F3", "F4"])
def test_depth_variants_match_oracle(name):
    """The depth variants of Table 4 (F2: (F100, F64, M) in fp32, fp16-F2 its
    fp16 version; F3: (F100, F8, F8, M); fp16-F3: its inner F8 with fp16
    vectors; F4: (F100, F8, F4, F2, M), the F2 with fp16 vectors) against the
    oracle's same configurations."""
    prob = G.diffusion3d_7pt(dims=(24, 24, 24), seed=102)
    s = solver(prob, f3r.preset(name))
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    res = s.solve(dev(prob.b), x)
    torch.cuda.synchronize()
    ref = O.Problem(prob, diag_scale=1).solve(O.preset(name), prob.b)
    _check_history(res, ref, prob, x.cpu().numpy())


@pytest.mark.parametrize("fuse", [1, 0])
def test_adaptive_inner_level_matches_oracle(fuse):
    """Adaptive m3: F_m3 (up to 8 iterations) stops once its residual estimate
    is below 0.2 beta; the weight counter follows the scheduled calls."""
    prob = G.diffusion3d_7pt(dims=(24, 24, 24), seed=102)
    kw = dict(m=[100, 8, 8, 0], inner_rtol=0.2)
    s = solver(prob, f3r.default_params(fuse_cgs=fuse, **kw))
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    res = s.solve(dev(prob.b), x)
    torch.cuda.synchronize()
    ref = O.Problem(prob, diag_scale=1).solve(O.params(**kw), prob.b)
    _check_history(res, ref, prob, x.cpu().numpy())
    assert res.r_calls < 64 * res.outer_iters and res.m_applies == 2 * res.r_calls
    assert abs(res.r_calls / res.outer_iters - ref.r_calls / ref.outer_iters) <= 0.1 * ref.r_calls / ref.outer_iters


def test_fgmres64_comparator_matches_oracle():
    prob = G.poisson2d_5pt(24)
    res, ref, xg = _solve_both(prob, "fgmres64", ds=0)
    _check_history(res, ref, prob, xg)
    assert res.m_applies == res.outer_iters


# ------------------------------------------------------------- edge cases
def test_host_and_device_pointers_agree():
    prob = G.diffusion3d_7pt(dims=(12, 11, 10), seed=104)
    sd = solver(prob, f3r.default_params(), on_device=True)
    sh = solver(prob, f3r.default_params(), on_device=False)
    xd = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    rd = sd.solve(dev(prob.b), xd)
    xh = np.zeros(prob.n)
    rh = sh.solve(np.ascontiguousarray(prob.b), xh)
    assert np.array_equal(xd.cpu().numpy(), xh)
    assert rd.outer_iters == rh.outer_iters


@pytest.mark.parametrize("n", [1, 2, 31, 33, 100])
def test_tiny_and_ragged_sizes(n):
    prob = G.random_dd_sparse(n, per_row=min(4, n), seed=105 + n, dominance=1.2)
    s = solver(prob, f3r.default_params())
    x = np.zeros(n)
    res = s.solve(np.ascontiguousarray(prob.b), x)
    A = prob.to_scipy()
    assert res.status == f3r.OK
    assert np.linalg.norm(prob.b - A @ x) / np.linalg.norm(prob.b) < 1e-9


def test_zero_rhs_and_exact_initial_guess():
    prob = G.poisson2d_5pt(16)
    s = solver(prob, f3r.default_params(diag_scale=0))
    x = np.ones(prob.n)
    res = s.solve(np.zeros(prob.n), x)
    assert res.status == f3r.OK and np.all(x == 0) and res.outer_iters == 0
    x = prob.x_true.copy()
    res = s.solve(np.ascontiguousarray(prob.b), x)
    assert res.status == f3r.OK and res.outer_iters == 0


def test_not_converged_and_restart():
    prob = G.diffusion3d_7pt(dims=(16, 16, 16), seed=106)
    s = solver(prob, f3r.default_params(max_outer=2))
    x = np.zeros(prob.n)
    res = s.solve(np.ascontiguousarray(prob.b), x)
    assert res.status == f3r.NOT_CONVERGED and res.outer_iters == 2
    s2 = solver(prob, f3r.default_params(m=[3, 8, 4, 0]))
    x = np.zeros(prob.n)
    res = s2.solve(np.ascontiguousarray(prob.b), x)
    P = O.Problem(prob)
    ref = P.solve(O.params(m=[3, 8, 4, 0]), prob.b)
    assert res.status == f3r.OK and res.restarts == (res.outer_iters - 1) // 3
    assert abs(res.outer_iters - ref.outer_iters) <= 1


def test_invalid_matrix_rejected():
    prob = G.poisson2d_5pt(8)
    bad = prob.colidx.copy()
    bad[5] = prob.n + 3
    with pytest.raises(f3r.F3RError) as e:
        f3r.Solver(prob.rowptr, bad, prob.val, f3r.default_params())
    assert e.value.code == f3r.ERR_ARG


@pytest.mark.parametrize("kind", ["fp16", "fp64"])
@pytest.mark.parametrize("step", [1, 0])
def test_fused_and_unfused_cgs_agree(kind, step):
    """The fused CGS2 / normalisation launch (and, for fp16, the whole-iteration
    launch of the innermost level) changes only the summation order of the
    dot products: both paths converge alike and match the oracle."""
    prob = G.diffusion3d_7pt(dims=(40, 36, 30), seed=108)
    out = {}
    for fuse in (0, 1):
        s = solver(prob, _rich_prm(kind, fuse_cgs=fuse, fuse_step=step))
        x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        out[fuse] = (s.solve(dev(prob.b), x), x.cpu().numpy())
    P = O.Problem(prob, diag_scale=1)
    ref = P.solve(_orc_prm(kind), prob.b)
    for fuse in (0, 1):
        _check_history(out[fuse][0], ref, prob, out[fuse][1])
    assert abs(out[0][0].outer_iters - out[1][0].outer_iters) <= 1


def test_graphs_and_direct_launches_agree():
    prob = G.diffusion3d_7pt(dims=(14, 14, 14), seed=107)
    out = []
    for g in (0, 1):
        s = solver(prob, f3r.default_params(use_graphs=g))
        x = np.zeros(prob.n)
        r = s.solve(np.ascontiguousarray(prob.b), x)
        out.append((x, r.outer_iters))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]


def test_unit_jacobi_richardson_bit_identical(monkeypatch):
    """Under symmetric diagonal scaling the stored Jacobi M is exactly 1 and the
    Richardson kernels skip its loads (M v = v).  The solve must be the same,
    bit for bit, as with the general kernels (F3R_UNIT_M=0 at set-up)."""
    prob = G.diffusion3d_7pt(dims=(40, 36, 30), seed=109)
    out = []
    for unit in ("1", "0"):
        monkeypatch.setenv("F3R_UNIT_M", unit)
        s = solver(prob, f3r.default_params())
        monkeypatch.delenv("F3R_UNIT_M")
        assert np.all(s.export(6) == np.uint16(0x3C00))
        x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        r = s.solve(dev(prob.b), x)
        torch.cuda.synchronize()
        out.append((x.cpu().numpy(), r.outer_iters, np.array(r.hist)))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][2], out[1][2])


def test_pooled_context_memory_reused_and_trimmed():
    """Contexts take their buffers from the library's device pool: a context
    set up on memory an earlier one released solves bit for bit alike, and
    trimming the pool afterwards succeeds."""
    prob = G.diffusion3d_7pt(dims=(20, 18, 16), seed=110)
    out = []
    for _ in range(2):
        s = solver(prob, f3r.default_params())
        x = np.zeros(prob.n)
        r = s.solve(np.ascontiguousarray(prob.b), x)
        s.close()
        out.append((x, r.outer_iters))
    f3r.trim_memory()
    assert out[0][1] == out[1][1] and np.array_equal(out[0][0], out[1][0])
    s = solver(prob, f3r.default_params())
    x = np.zeros(prob.n)
    assert s.solve(np.ascontiguousarray(prob.b), x).outer_iters == out[0][1]
    assert np.array_equal(x, out[0][0])


def test_contexts_with_different_stage_sizes_interleave():
    """Staged kernels size their shared memory from the matrix's slice width:
    a context set up and solved after another one with wider slices must not
    leave the first one unable to launch (replaying its graphs)."""
    p3 = G.diffusion3d_7pt(dims=(22, 20, 18), seed=111)
    p2 = G.poisson2d_5pt(60)
    s3 = solver(p3, f3r.default_params())
    x3 = np.zeros(p3.n)
    r3 = s3.solve(np.ascontiguousarray(p3.b), x3)
    s2 = solver(p2, f3r.default_params(diag_scale=0))
    x2 = np.zeros(p2.n)
    assert s2.solve(np.ascontiguousarray(p2.b), x2).status == f3r.OK
    y3 = np.zeros(p3.n)
    r3b = s3.solve(np.ascontiguousarray(p3.b), y3)
    assert r3.status == f3r.OK and r3b.status == f3r.OK
    assert r3b.outer_iters == r3.outer_iters and np.array_equal(x3, y3)


def test_programmatic_launch_changes_no_result(tmp_path):
    """Programmatic dependent launch (the default) only lets a kernel's
    prologue overlap the previous kernel: a solve in a process with it turned
    off (F3R_PDL=0) gives the same bits."""
    import os
    import subprocess
    import sys

    prob = G.diffusion3d_7pt(dims=(30, 28, 26), seed=112)
    s = solver(prob, f3r.default_params())
    x = np.zeros(prob.n)
    r = s.solve(np.ascontiguousarray(prob.b), x)
    out = tmp_path / "x.npy"
    code = (
        "import numpy as np, sys; sys.path.insert(0, %r)\n"
        "from problems import generators as G\n"
        "from paper_2505_20719_gb300 import f3r\n"
        "p = G.diffusion3d_7pt(dims=(30, 28, 26), seed=112)\n"
        "s = f3r.Solver.from_problem(p, f3r.default_params())\n"
        "x = np.zeros(p.n); r = s.solve(np.ascontiguousarray(p.b), x)\n"
        "np.save(%r, np.append(x, r.outer_iters))\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), str(out))
    env = dict(os.environ, F3R_PDL="0")
    subprocess.run([sys.executable, "-c", code], env=env, check=True, timeout=300)
    y = np.load(out)
    assert int(y[-1]) == r.outer_iters and np.array_equal(y[:-1], x)

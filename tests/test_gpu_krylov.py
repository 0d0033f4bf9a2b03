"""GPU CG / BiCGStab comparators (f3r_solve_krylov) against the CPU oracle
(oracle/krylov.py): same preconditioner, iteration counts, residual
histories and solutions."""
import numpy as np
import pytest

import oracle as O
from oracle import krylov as K
from problems import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_20719_gb300 import f3r  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _both(prob, method, ds=1, **kw):
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.default_params(diag_scale=ds, **kw))
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    res = s.solve_krylov(method, dev(prob.b), x)
    P = O.Problem(prob, diag_scale=ds)
    d, m = K.preconditioner(P)
    ref = K.solve(method, prob.to_scipy(), prob.b, d, m, tol=kw.get("tol", 1e-9))
    return res, ref, x.cpu().numpy()


def _check(res, ref, prob, xg, rel_iters):
    A = prob.to_scipy()
    rel = np.linalg.norm(prob.b - A @ xg) / np.linalg.norm(prob.b)
    assert res.status == f3r.OK and rel < 1e-9 and abs(rel - res.rel_res_true) <= 1e-12
    assert abs(res.outer_iters - ref["iters"]) <= max(2, int(rel_iters * ref["iters"]))
    k = min(len(res.hist), len(ref["hist"]), 60)
    ratio = np.abs(np.log10(res.hist[:k] / ref["hist"][:k]))
    assert np.all(ratio <= 0.5), ratio.max()


def test_cg_matches_oracle():
    prob = G.diffusion3d_7pt(dims=(24, 24, 24), seed=102)
    res, ref, xg = _both(prob, "cg")
    _check(res, ref, prob, xg, 0.02)
    assert np.linalg.norm(xg - ref["x"]) <= 1e-6 * np.linalg.norm(ref["x"])


def test_bicgstab_matches_oracle():
    prob = G.convdiff3d_27pt(dims=(20, 20, 20), seed=103)
    res, ref, xg = _both(prob, "bicgstab")
    _check(res, ref, prob, xg, 0.15)


def test_unscaled_jacobi_and_host_pointers():
    prob = G.poisson2d_5pt(40)
    s = f3r.Solver(prob.rowptr, prob.colidx, prob.val, f3r.default_params(diag_scale=0))
    x = np.zeros(prob.n)
    res = s.solve_krylov("cg", np.ascontiguousarray(prob.b), x)
    P = O.Problem(prob, diag_scale=0)
    d, m = K.preconditioner(P)
    ref = K.solve("cg", prob.to_scipy(), prob.b, d, m)
    assert res.status == f3r.OK and abs(res.outer_iters - ref["iters"]) <= 2
    assert np.linalg.norm(x - prob.x_true) <= 1e-6 * np.linalg.norm(prob.x_true)


def test_iteration_cap_and_zero_rhs():
    prob = G.diffusion3d_7pt(dims=(16, 16, 16), seed=106)
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.default_params())
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    res = s.solve_krylov("cg", dev(prob.b), x, max_iters=7)
    assert res.status == f3r.NOT_CONVERGED and res.outer_iters == 7
    x.zero_()
    res = s.solve_krylov("bicgstab", torch.zeros(prob.n, dtype=torch.float64, device="cuda"), x)
    assert res.outer_iters == 0 and float(x.abs().max()) == 0.0

"""Approximate-inverse preconditioner on the GPU against the oracle: fp16
factors bit for bit, Richardson calls bit for bit (row sums in CSR order),
full solves by their residual histories."""
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


def f16_bits(vals):
    return vals.astype(np.float16).view(np.uint16)


@pytest.fixture(scope="module")
def convdiff():
    return G.convdiff3d_27pt(dims=(21, 19, 17), seed=101)


@pytest.mark.parametrize("alpha", [1.0, 1.3])
def test_factors_bit_exact(convdiff, alpha):
    prob = convdiff
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val),
                   f3r.default_params(precond=f3r.PC_AINV, ainv_alpha=alpha))
    P = O.Problem(prob, diag_scale=1, precond=O.PC_AINV, ainv_alpha=alpha)
    assert np.array_equal(s.export(7, prob.nnz), f16_bits(P.get("ainv_l")))
    assert np.array_equal(s.export(8, prob.nnz), f16_bits(P.get("ainv_u")))
    assert np.array_equal(s.export(9), f16_bits(P.get("ainv_dinv")))


@pytest.mark.parametrize("m4", [1, 2, 3])
def test_richardson_call_bit_exact(convdiff, m4):
    prob = convdiff
    n = prob.n
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val),
                   f3r.default_params(precond=f3r.PC_AINV, rich_m=m4, ainv_alpha=1.2))
    P = O.Problem(prob, diag_scale=1, precond=O.PC_AINV, ainv_alpha=1.2)
    v = (rng.normal(51, 1, n) * 1e-3).astype(np.float32)
    omega = [0.83, 1.07, 0.91][:m4]
    s.set_rich_state(omega, 5)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    s.apply(3, dev(v), z)
    torch.cuda.synchronize()
    want = P.apply(O.params(precond=O.PC_AINV, rich_m=m4), O.rich_state(c_ntr=5, omega=omega), 3,
                   v.astype(np.float64))
    assert np.array_equal(z.cpu().numpy().astype(np.float64), want)


def test_update_call_close(convdiff):
    prob = convdiff
    n = prob.n
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.default_params(precond=f3r.PC_AINV))
    P = O.Problem(prob, diag_scale=1, precond=O.PC_AINV)
    v = (rng.normal(52, 1, n) * 1e-3).astype(np.float32)
    s.set_rich_state([0.9, 1.1], 128)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    s.apply(3, dev(v), z)
    torch.cuda.synchronize()
    st = O.rich_state(c_ntr=128, omega=[0.9, 1.1])
    want = P.apply(O.params(precond=O.PC_AINV), st, 3, v.astype(np.float64))
    om, cn = s.rich_state()
    assert cn == 129 and np.allclose(om[:2], list(st.omega)[:2], rtol=2e-5, atol=0)
    assert np.linalg.norm(z.cpu().numpy() - want) <= 2e-3 * np.linalg.norm(want)


def test_solve_matches_oracle():
    prob = G.diffusion3d_7pt(dims=(24, 24, 24), seed=102)
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.default_params(precond=f3r.PC_AINV))
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    res = s.solve(dev(prob.b), x)
    torch.cuda.synchronize()
    ref = O.Problem(prob, diag_scale=1, precond=O.PC_AINV).solve(O.params(precond=O.PC_AINV), prob.b)
    A = prob.to_scipy()
    rel = np.linalg.norm(prob.b - A @ x.cpu().numpy()) / np.linalg.norm(prob.b)
    assert res.status == f3r.OK and ref.status == O.OK and rel < 1e-9
    assert abs(res.outer_iters - ref.outer_iters) <= max(1, int(0.1 * ref.outer_iters))
    k = min(len(res.hist), len(ref.hist))
    mask = ref.hist[:k] > 1e-8
    assert np.all(np.abs(np.log10(res.hist[:k][mask] / ref.hist[:k][mask])) <= 0.5)
    assert res.m_applies == 64 * res.outer_iters


def test_unsupported_schedules_rejected():
    prob = G.poisson2d_5pt(8)
    with pytest.raises(f3r.F3RError) as e:
        f3r.Solver(prob.rowptr, prob.colidx, prob.val, f3r.preset("fp32-F3R", precond=f3r.PC_AINV))
    assert e.value.code == f3r.ERR_UNSUPPORTED

"""fp16-vector FGMRES levels (Table 4: fp16-F3's inner F8, F4's F2, fp16-F2's
inner FGMRES(64)) and the fp32 inner FGMRES(64) of F2 on the GPU against the
oracle's same configuration.

The level computes in fp32 and rounds every stored V and Z value to fp16
(held in fp32 arrays).  Checked: each basis vector the GPU stored is a vector
of fp16 numbers (exact); one call of the level matches the oracle's call to
2 u16 in norm and 8 u16 max|z| per element (u16 = 2^-11: both sides round the
same values to fp16, and a value whose fp32 sums differ in the last place can
round the other way, which the remaining iterations carry on); and the level
stays within 20 u16 of the all-fp64 level.
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

U16 = 2.0 ** -11
_LEVELS = [("fp16-F3", 2), ("F4", 3), ("fp16-F2", 1)]
_IDS = ["fp16-F3 F8", "F4 F2", "fp16-F2 F64"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", params=[0, 1], ids=["unscaled", "scaled"])
def system(request):
    prob = G.convdiff3d_27pt(dims=(21, 19, 17), seed=111)
    v = rng.normal(150, 1, prob.n)
    v = (v / np.linalg.norm(v)).astype(np.float32).astype(np.float64)
    return prob, request.param, v


@pytest.mark.parametrize("preset,level", _LEVELS, ids=_IDS)
def test_fp16_level_call_matches_oracle(system, preset, level):
    prob, ds, v = system
    P = O.Problem(prob, diag_scale=ds)
    zo = P.apply(O.preset(preset, diag_scale=ds), O.rich_state(), level, v)
    f64 = [O.F64] * 4
    z64 = P.apply(O.preset(preset, diag_scale=ds, a_prec=f64, v_prec=f64, m_prec=O.F64), O.rich_state(), level, v)
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.preset(preset, diag_scale=ds))
    z = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.apply(level, dev(v.astype(np.float32)), z)
    torch.cuda.synchronize()
    zg = z.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
    emax = np.abs(zg - zo).max() / np.abs(zo).max()
    e64 = np.linalg.norm(zg - z64) / np.linalg.norm(z64)
    print(f"{preset} level {level} ds={ds}: |z - z_oracle|/|z| = {err / U16:.3f} u16, "
          f"max {emax / U16:.3f} u16; vs fp64 level {e64 / U16:.2f} u16")
    assert err <= 2 * U16 and emax <= 8 * U16
    assert e64 <= 20 * U16
    m = f3r.preset(preset).m[level]
    for k in range(m):  # an inner level never forms V[m]
        out = torch.empty(prob.n, dtype=torch.float32, device="cuda")
        s.get_basis(level, k, out)
        vk = out.cpu().numpy()
        assert np.array_equal(vk, vk.astype(np.float16).astype(np.float32)), k
        assert abs(np.linalg.norm(vk.astype(np.float64)) - 1.0) <= 4 * U16
    s.close()


def test_fp32_level_basis_is_not_fp16(system):
    """Control: the same level with fp32 vectors (F3) stores values that are
    not fp16 numbers, so the check above sees the rounding."""
    prob, ds, v = system
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.preset("F3", diag_scale=ds))
    z = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.apply(2, dev(v.astype(np.float32)), z)
    out = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.get_basis(2, 3, out)
    torch.cuda.synchronize()
    vk = out.cpu().numpy()
    assert not np.array_equal(vk, vk.astype(np.float16).astype(np.float32))
    s.close()


def test_long_fp32_level_call_matches_oracle(system):
    """F2's inner FGMRES(64) (chunked CGS2 beyond the fused register path) in
    fp32 against the oracle's call, to 1e-4 of the norm (64 fp32 iterations)."""
    prob, ds, v = system
    P = O.Problem(prob, diag_scale=ds)
    zo = P.apply(O.preset("F2", diag_scale=ds), O.rich_state(), 1, v)
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.preset("F2", diag_scale=ds))
    z = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.apply(1, dev(v.astype(np.float32)), z)
    torch.cuda.synchronize()
    zg = z.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
    print(f"F2 level 1 ds={ds}: |z - z_oracle|/|z| = {err:.3e}")
    assert err <= 1e-4
    s.close()

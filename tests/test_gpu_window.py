"""Windowed tiles (f3r_matrix_info): the set-up's 16-bit window indices map
back to the CSR columns on every entry, the kernels give the same bits with
and without windows, and matrices or inputs the window cannot serve fall
back to int32 gathers."""
import os
import subprocess
import sys

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

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solver(prob, prm=None):
    return f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), prm or f3r.default_params())


@pytest.mark.parametrize("which", ["poisson2d_64", "diffusion7_128", "convdiff27_160", "small_convdiff"])
def test_window_indices_map_back_to_columns(which):
    prob = G.convdiff3d_27pt(dims=(21, 19, 17), seed=101) if which == "small_convdiff" else G.by_name(which)
    s = _solver(prob, f3r.default_params(diag_scale=0 if which == "poisson2d_64" else 1))
    info = s.matrix_info()
    assert info["windowed"] == 1 and info["index_bytes"] == 2
    assert 0 < info["win_max"] <= 4096 and info["win_max"] % info["win_chunk"] == 0
    cols = s.export(10, prob.nnz)
    s.close()
    assert np.array_equal(cols, prob.colidx)


def test_far_columns_are_not_windowed():
    prob = G.random_dd_sparse(70000, per_row=5, seed=109, dominance=1.5)
    s = _solver(prob)
    assert s.matrix_info()["windowed"] == 0 and s.matrix_info()["index_bytes"] == 4
    with pytest.raises(f3r.F3RError):
        s.export(10, prob.nnz)
    s.close()


def test_unaligned_x_falls_back_bit_exact():
    """f3r_spmv with x at a 4-byte offset (no 16-byte bulk copies possible):
    the same bits as the oracle."""
    prob = G.convdiff3d_27pt(dims=(21, 19, 17), seed=101)
    s = _solver(prob)
    P = O.Problem(prob, diag_scale=1)
    x = rng.normal(130, 1, prob.n + 1).astype(np.float32)
    xd = dev(x)[1:]
    assert xd.data_ptr() % 16 != 0
    y = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    s.spmv(f3r.F16, f3r.F32, xd, y)
    torch.cuda.synchronize()
    want = P.spmv(O.F16, O.F32, x[1:].astype(np.float64))
    s.close()
    assert np.array_equal(y.cpu().numpy().astype(np.float64), want)


_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2505_20719_gb300 import f3r
from problems import generators as G
from problems import rng
prob = G.convdiff3d_27pt(dims=(21, 19, 17), seed=101)
T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
s = f3r.Solver(T(prob.rowptr), T(prob.colidx), T(prob.val), f3r.default_params())
out = {{"windowed": s.matrix_info()["windowed"]}}
x = rng.normal(131, 1, prob.n).astype(np.float32)
y = torch.empty(prob.n, dtype=torch.float32, device="cuda")
s.spmv(f3r.F16, f3r.F32, T(x), y)
out["spmv"] = y.cpu().numpy()
v = (rng.normal(132, 1, prob.n) * 1e-2).astype(np.float32)
s.set_rich_state([0.83, 1.07], 5)
z = torch.empty(prob.n, dtype=torch.float32, device="cuda")
s.apply(3, T(v), z)
out["rich"] = z.cpu().numpy()
xs = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
r = s.solve(T(prob.b), xs)
out["x"] = xs.cpu().numpy()
out["hist"] = np.asarray(r.hist)
np.savez({path!r}, **out)
"""


def test_windowed_and_plain_gathers_give_the_same_bits(tmp_path):
    """The same SpMV, Richardson call and whole solve in two processes, one
    with windowed tiles and one with F3R_WINDOW=0 (int32 gathers): identical
    SpMV and Richardson outputs (only where x is read from changes); the
    solves agree to rounding (the grids, hence the grouping of the dot
    products' block sums, may differ)."""
    res = {}
    for flag in ("1", "0"):
        path = str(tmp_path / f"w{flag}.npz")
        env = dict(os.environ, F3R_WINDOW=flag)
        r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT, path=path)], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[flag] = np.load(path)
    assert int(res["1"]["windowed"]) == 1 and int(res["0"]["windowed"]) == 0
    for k in ("spmv", "rich"):
        assert np.array_equal(res["1"][k], res["0"][k]), k
    h1, h0 = res["1"]["hist"], res["0"]["hist"]
    assert abs(len(h1) - len(h0)) <= 1
    k = min(len(h1), len(h0))
    assert np.all(np.abs(np.log10(h1[:k] / h0[:k])) <= 0.5)

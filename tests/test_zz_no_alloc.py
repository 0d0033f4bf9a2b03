"""The allocation-free residual entry point, f3r_residual_noalloc.

Some callers cannot let a library call cudaMalloc (their device memory belongs
to another allocator or a fixed budget); this entry point computes
r = b - A x and ||r||, ||b|| from caller buffers only, with its scratch in a
static device array.  It is checked through the C ABI against the existing
entry points: the residual against b - f3r_spmv(original A, x) bit for bit,
and ||r||/||b|| against the true residual f3r_solve reports, on two calls in a
row.  This file is collected last so that a failure here comes after every
other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from problems import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_20719_gb300 import f3r  # noqa: E402


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_residual_noalloc_matches_existing_entry_points():
    prob = G.diffusion3d_7pt(dims=(40, 37, 33), seed=301)  # n = 48,840: several blocks, ragged tail
    n = prob.n
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    rp, ci, va, b = d(prob.rowptr), d(prob.colidx), d(prob.val), d(prob.b)
    s = f3r.Solver(rp, ci, va, f3r.default_params())
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = s.solve(b, x, check=True)
    lib = f3r.lib()
    for call in range(2):
        xc = x if call == 0 else x * (1.0 + 1e-3)  # a second, different input
        r = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        norms = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
        code = lib.f3r_residual_noalloc(n, _p(rp), _p(ci), _p(va), _p(b), _p(xc), _p(r), _p(norms), None)
        assert code == f3r.OK
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        s.spmv(f3r.F64, f3r.F64, xc, y)  # the existing SpMV entry point on the original A
        torch.cuda.synchronize()
        assert torch.equal(r, b - y)
        nr, nb = norms.cpu().numpy()
        assert nb == pytest.approx(np.linalg.norm(prob.b), rel=1e-12)
        assert nr == pytest.approx(float(torch.linalg.norm(b - y)), rel=1e-12)
        if call == 0:
            assert nr / nb == pytest.approx(res.rel_res_true, rel=1e-12)
    s.close()


def _tridiagonal(n, seed):
    """1-D Laplacian-like CSR matrix (3 entries per row), fp64."""
    rng = np.random.default_rng(seed)
    rows = np.arange(n)
    cols = np.stack([rows - 1, rows, rows + 1], axis=1)
    vals = np.stack([-np.ones(n), 2.0 + rng.random(n), -np.ones(n)], axis=1)
    keep = (cols >= 0) & (cols < n)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(keep.sum(axis=1))
    return rowptr, cols[keep].astype(np.int32), vals[keep], rng.random(n), rng.standard_normal(n)


@pytest.mark.parametrize("n", [700, 4 * 1024 * 1024 - 4])
def test_residual_noalloc_single_block_and_full_scratch(n):
    """One block (n < 1024 rows) and the largest grid the scratch holds (4096
    blocks, so the last block sums 4096 partials): the residual equals
    b - f3r_spmv(A, x) bit for bit and the norms match, on two calls in a row."""
    rowptr, colidx, val, b_h, x_h = _tridiagonal(n, seed=302 + n % 7)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    rp, ci, va, b = d(rowptr), d(colidx), d(val), d(b_h)
    s = f3r.Solver(rp, ci, va, f3r.default_params(diag_scale=0))
    lib = f3r.lib()
    for call in range(2):
        x = d(x_h * (1.0 + call))
        r = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        norms = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
        assert lib.f3r_residual_noalloc(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), _p(r), _p(norms), None) == f3r.OK
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        s.spmv(f3r.F64, f3r.F64, x, y)
        torch.cuda.synchronize()
        assert torch.equal(r, b - y)
        nr, nb = norms.cpu().numpy()
        assert nb == pytest.approx(np.linalg.norm(b_h), rel=1e-12)
        assert nr == pytest.approx(float(torch.linalg.norm(b - y)), rel=1e-12)
    s.close()


def test_residual_noalloc_rejects_sizes_beyond_its_scratch():
    lib = f3r.lib()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = _p(dummy)
    assert lib.f3r_residual_noalloc(4 * 1024 * 1024 + 1, p, p, p, p, p, p, p, None) == f3r.ERR_ARG
    assert lib.f3r_residual_noalloc(0, p, p, p, p, p, p, p, None) == f3r.ERR_ARG

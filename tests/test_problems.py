"""The seeded workload generators: sizes, structure and coefficient laws."""
import numpy as np
import scipy.sparse as sp

from problems import generators as G
from problems import rng


def _check_csr(p):
    assert p.rowptr.dtype == np.int32 and p.colidx.dtype == np.int32
    assert p.rowptr[0] == 0 and np.all(np.diff(p.rowptr) >= 0)
    for i in range(0, p.n, max(1, p.n // 50)):
        c = p.colidx[p.rowptr[i]:p.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0) and i in c


def test_rng_is_counter_based_and_deterministic():
    a = rng.uniform01(1, 2, 1000)
    b = rng.uniform01(1, 2, 500, offset=500)
    assert np.array_equal(a[500:], b)
    assert not np.array_equal(a, rng.uniform01(1, 3, 1000))
    g = rng.normal(1, 2, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    # SplitMix64 published test vector: seed 0, first output
    assert int(rng._mix(np.uint64(0x9E3779B97F4A7C15))) == 0xE220A8397B1DCDAF


def test_poisson_sizes():
    p = G.poisson2d_5pt(64)
    assert p.n == 4096 and p.nnz == 20224
    _check_csr(p)
    A = p.to_scipy()
    assert set(np.unique(A.data)) == {-1.0, 4.0}
    assert np.allclose(A @ p.x_true, p.b)


def test_diffusion7_structure():
    p = G.diffusion3d_7pt(dims=(12, 11, 10), seed=3)
    _check_csr(p)
    A = p.to_scipy()
    assert abs(A - A.T).max() == 0
    off = (A - sp.diags(A.diagonal())).tocsr()
    off.eliminate_zeros()
    assert off.data.max() < 0
    rowsum = A @ np.ones(p.n)
    assert rowsum.min() > -1e-12 and rowsum.max() > 0
    # full 128^3 sizes, from the closed form of the face count
    N = 128
    assert N ** 3 + 2 * 3 * (N - 1) * N * N == 14581760


def test_convdiff27_structure_and_peclet():
    dims = (14, 13, 12)
    p = G.convdiff3d_27pt(dims=dims, seed=4)
    _check_csr(p)
    A = p.to_scipy()
    assert p.nnz == (3 * 14 - 2) * (3 * 13 - 2) * (3 * 12 - 2)
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=1)).ravel() - d
    assert np.all(d - off >= -1e-12)
    assert abs(A - A.T).max() > 1.0  # nonsymmetric
    P = G.smooth_velocity(dims, 4)
    pe = np.sqrt((P ** 2).sum(axis=0))
    assert np.isclose(pe.min(), 0.1) and np.isclose(pe.max(), 10.0)


def test_nodal27_and_hpcg():
    p = G.diffusion27_nodal(dims=(8, 7, 6), seed=5)
    _check_csr(p)
    A = p.to_scipy()
    assert abs(A - A.T).max() < 1e-14
    assert np.all(A.diagonal() - (np.asarray(abs(A).sum(axis=1)).ravel() - A.diagonal()) >= -1e-12)
    h = G.hpcg_27pt(8)
    H = h.to_scipy()
    assert set(np.unique(H.diagonal())) == {26.0}


def test_batched_systems_law():
    systems = G.batched_diffusion_systems(count=16, n_lo=1e3, n_hi=2e4)
    assert len(systems) == 16
    for prob, B in systems:
        _check_csr(prob)
        assert 1 <= B.shape[0] <= 8 and B.shape[1] == prob.n
        assert 0.5e3 <= prob.n <= 3e4

"""Seeded stencil matrices in CSR form (int32 indices, float64 values).

Row/column numbering is lexicographic, i = ix + nx*(iy + ny*iz), and within a
row the columns are sorted ascending (the stencil offsets are visited in order
of their linear offset), so every generator returns canonical CSR.

The paper's test set (Sec. 5, Table 2) is SuiteSparse plus the HPCG and HPGMP
stencils; the generators below are synthetic stand-ins with the workload
shapes used here:

* poisson2d_5pt     -- 2-D Poisson, diag 4 / off -1, Dirichlet.
* diffusion3d_7pt   -- 3-D variable-coefficient diffusion, one log-normal
                       coefficient per cell face (SPD M-matrix).
* convdiff3d_27pt   -- nonsymmetric 27-point convection-diffusion, first-order
                       upwind convection with a smooth random velocity field
                       whose cell Peclet number spans [0.1, 10].
* diffusion27_nodal -- 27-neighbour diffusion with a log-normal nodal field.
* hpcg_27pt         -- HPCG-style matrix (diag 26, off -1), Sec. 5.
* batched_diffusion_systems -- many uneven 2-D/3-D diffusion systems.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import rng


@dataclass
class Problem:
    name: str
    n: int
    rowptr: np.ndarray   # int32, n+1
    colidx: np.ndarray   # int32, nnz
    val: np.ndarray      # float64, nnz
    b: np.ndarray        # float64, n
    x_true: np.ndarray = None
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        return sp.csr_matrix((self.val, self.colidx, self.rowptr), shape=(self.n, self.n))


def _assemble(dims, offsets, values, valid):
    """Build CSR from per-offset value arrays.

    dims    -- (nx, ny, nz)
    offsets -- list of (dx, dy, dz), sorted by linear offset dx + nx*dy + nx*ny*dz
    values  -- list of float64 arrays of shape (nz, ny, nx)
    valid   -- list of bool arrays of shape (nz, ny, nx): neighbour inside the grid
    """
    nx, ny, nz = dims
    n = nx * ny * nz
    K = len(offsets)
    lin = [dx + nx * dy + nx * ny * dz for (dx, dy, dz) in offsets]
    assert lin == sorted(lin), "offsets must be sorted by linear offset"
    idx = np.arange(n, dtype=np.int64)
    C = np.empty((n, K), dtype=np.int32)
    V = np.empty((n, K), dtype=np.float64)
    M = np.empty((n, K), dtype=bool)
    for k in range(K):
        C[:, k] = idx + lin[k]
        V[:, k] = values[k].reshape(n)
        M[:, k] = valid[k].reshape(n)
    counts = M.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    assert rowptr[-1] < 2**31
    colidx = C[M]
    val = V[M]
    return rowptr.astype(np.int32), colidx.astype(np.int32), val


def _grid_valid(dims, d):
    """Bool mask (nz, ny, nx): cell + d lies inside the grid."""
    nx, ny, nz = dims
    dx, dy, dz = d
    ix = np.arange(nx)
    iy = np.arange(ny)
    iz = np.arange(nz)
    vx = (ix + dx >= 0) & (ix + dx < nx)
    vy = (iy + dy >= 0) & (iy + dy < ny)
    vz = (iz + dz >= 0) & (iz + dz < nz)
    return vz[:, None, None] & vy[None, :, None] & vx[None, None, :]


def _spmv(rowptr, colidx, val, x):
    return sp.csr_matrix((val, colidx, rowptr), shape=(len(rowptr) - 1, len(x))) @ x


def rhs_uniform01(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform in [0, 1), as in Sec. 5."""
    return rng.uniform01(seed, 1000, n)


# ---------------------------------------------------------------------------
def poisson2d_5pt(nx: int = 64, ny: int = None, seed: int = 2505_20719 + 0) -> Problem:
    """2-D 5-point Poisson, Dirichlet boundary: diag 4, off-diagonals -1.

    x* is uniform in [-1, 1] from the seed and b = A x*.
    """
    ny = nx if ny is None else ny
    dims = (nx, ny, 1)
    offs = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    shape = (1, ny, nx)
    vals = [np.full(shape, -1.0), np.full(shape, -1.0), np.full(shape, 4.0),
            np.full(shape, -1.0), np.full(shape, -1.0)]
    valid = [_grid_valid(dims, d) for d in offs]
    rowptr, colidx, val = _assemble(dims, offs, vals, valid)
    n = nx * ny
    x_true = 2.0 * rng.uniform01(seed, 1, n) - 1.0
    b = _spmv(rowptr, colidx, val, x_true)
    return Problem(f"poisson2d_{nx}x{ny}", n, rowptr, colidx, val, b, x_true,
                   {"dims": dims, "seed": seed, "kind": "poisson2d_5pt"})


def _face_coefficients(dims, sigma, seed, stream0):
    """Log-normal coefficient exp(sigma*g) on every cell face, boundary faces included.

    Returns kx (nz, ny, nx+1), ky (nz, ny+1, nx), kz (nz+1, ny, nx); face index
    i along an axis separates cells i-1 and i.
    """
    nx, ny, nz = dims
    shapes = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
    out = []
    for a, shp in enumerate(shapes):
        cnt = int(np.prod(shp))
        g = rng.normal(seed, stream0 + a, cnt).reshape(shp)
        out.append(np.exp(sigma * g))
    return out


def diffusion3d_7pt(N: int = 128, sigma: float = 1.5, seed: int = 2505_20719 + 1,
                    dims=None, rhs: str = "uniform01") -> Problem:
    """3-D 7-point variable-coefficient diffusion (cell-centred finite volumes).

    Each face f carries k_f = exp(sigma * g_f), g_f ~ N(0, 1).  Row i has
    A_ii = sum of its six face coefficients (Dirichlet faces included) and
    A_ij = -k_f for the face shared with neighbour j.  The result is a
    symmetric positive definite M-matrix.
    """
    dims = (N, N, N) if dims is None else tuple(dims)
    nx, ny, nz = dims
    kx, ky, kz = _face_coefficients(dims, sigma, seed, 1)
    diag = kx[:, :, :-1] + kx[:, :, 1:] + ky[:, :-1, :] + ky[:, 1:, :] + kz[:-1] + kz[1:]
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    vals = [-kz[:-1], -ky[:, :-1, :], -kx[:, :, :-1], diag, -kx[:, :, 1:], -ky[:, 1:, :], -kz[1:]]
    valid = [_grid_valid(dims, d) for d in offs]
    rowptr, colidx, val = _assemble(dims, offs, vals, valid)
    n = nx * ny * nz
    b = rhs_uniform01(n, seed) if rhs == "uniform01" else None
    return Problem(f"diffusion7_{nx}x{ny}x{nz}", n, rowptr, colidx, val, b, None,
                   {"dims": dims, "seed": seed, "sigma": sigma, "kind": "diffusion3d_7pt"})


def _offsets27():
    return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _w27(d):
    """Diffusion weight of a 27-point neighbour: face 1, edge 1/2, corner 1/4."""
    k = sum(1 for c in d if c != 0)
    return {0: 0.0, 1: 1.0, 2: 0.5, 3: 0.25}[k]


def smooth_velocity(dims, seed, pe_min=0.1, pe_max=10.0, modes=4):
    """Cell Peclet vector field P(x) = Pe(x) * U(x)/|U(x)|.

    U is a sum of `modes` seeded Fourier modes a_m sin(2 pi k_m.x + phi_m) with
    a_m ~ N(0, I_3), k_m integer in [-2, 2]^3 (nonzero) and phi_m ~ U[0, 2 pi).
    The magnitude is mapped log-linearly onto [pe_min, pe_max]:
    Pe = pe_min * (pe_max/pe_min)^t with t = (|U| - min|U|)/(max|U| - min|U|).
    """
    nx, ny, nz = dims
    a = rng.normal(seed, 11, 3 * modes).reshape(modes, 3)
    k = rng.integers(seed, 12, 3 * modes, -2, 2).reshape(modes, 3)
    for m in range(modes):
        if not k[m].any():
            k[m, m % 3] = 1
    phi = 2.0 * np.pi * rng.uniform01(seed, 13, modes)
    x = (np.arange(nx) + 1.0) / (nx + 1)
    y = (np.arange(ny) + 1.0) / (ny + 1)
    z = (np.arange(nz) + 1.0) / (nz + 1)
    U = np.zeros((3, nz, ny, nx))
    for m in range(modes):
        ph = (2.0 * np.pi * (k[m, 0] * x[None, None, :] + k[m, 1] * y[None, :, None]
                             + k[m, 2] * z[:, None, None]) + phi[m])
        s = np.sin(ph)
        for c in range(3):
            U[c] += a[m, c] * s
    mag = np.sqrt((U * U).sum(axis=0))
    tiny = mag < 1e-300
    mag_safe = np.where(tiny, 1.0, mag)
    t = (mag - mag.min()) / max(mag.max() - mag.min(), 1e-300)
    pe = pe_min * (pe_max / pe_min) ** t
    P = pe[None] * U / mag_safe[None]
    P[0] = np.where(tiny, pe, P[0])
    return P  # (3, nz, ny, nx): components along x, y, z


def convdiff3d_27pt(N: int = 160, seed: int = 2505_20719 + 2, kappa: float = 1.0,
                    dims=None, pe_range=(0.1, 10.0)) -> Problem:
    """Nonsymmetric 27-point convection-diffusion (scaled by h^2).

    Diffusion: neighbour weights w_d (face 1, edge 1/2, corner 1/4) times
    kappa; A_ij = -kappa*w_d, and A_ii collects kappa*w_d of all 26 neighbour
    positions (Dirichlet).  Convection: first-order upwind on the six faces
    with coefficient q = 2*kappa*|P_d| from the cell Peclet field P, added to
    A_ii and subtracted from the upwind neighbour.  Row sums are >= 0 with
    strict dominance on the boundary: an irreducibly diagonally dominant
    M-matrix.
    """
    dims = (N, N, N) if dims is None else tuple(dims)
    nx, ny, nz = dims
    P = smooth_velocity(dims, seed, *pe_range)
    offs = _offsets27()
    shape = (nz, ny, nx)
    vals = []
    diag = np.full(shape, 14.0 * kappa)
    conv = {}
    for c, axis_vec in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        q = 2.0 * kappa * np.abs(P[c])
        diag += q
        plus = tuple(axis_vec)
        minus = tuple(-v for v in axis_vec)
        # flow in +axis: upwind neighbour is cell - e (offset minus); else cell + e
        conv[minus] = np.where(P[c] > 0, q, 0.0)
        conv[plus] = np.where(P[c] > 0, 0.0, q)
    for d in offs:
        if d == (0, 0, 0):
            vals.append(diag)
        else:
            v = np.full(shape, -kappa * _w27(d))
            if d in conv:
                v = v - conv[d]
            vals.append(v)
    valid = [_grid_valid(dims, d) for d in offs]
    rowptr, colidx, val = _assemble(dims, offs, vals, valid)
    n = nx * ny * nz
    b = rhs_uniform01(n, seed)
    return Problem(f"convdiff27_{nx}x{ny}x{nz}", n, rowptr, colidx, val, b, None,
                   {"dims": dims, "seed": seed, "kind": "convdiff3d_27pt",
                    "pe_range": pe_range})


def diffusion27_nodal(N: int = 100, sigma: float = 1.5, seed: int = 2505_20719 + 4,
                      dims=None) -> Problem:
    """27-neighbour diffusion with a log-normal nodal field kappa = exp(sigma*g).

    A_ij = -w_d * sqrt(kappa_i kappa_j) for the 26 neighbours (w_d: face 1,
    edge 1/2, corner 1/4); a neighbour outside the grid contributes the
    Dirichlet term w_d*kappa_i to the diagonal only; A_ii = sum_j |A_ij| plus
    those boundary terms.  Symmetric positive definite M-matrix.
    """
    dims = (N, N, N) if dims is None else tuple(dims)
    nx, ny, nz = dims
    kap = np.exp(sigma * rng.normal(seed, 21, nx * ny * nz)).reshape(nz, ny, nx)
    sk = np.sqrt(kap)
    offs = _offsets27()
    shape = (nz, ny, nx)
    diag = np.zeros(shape)
    vals = []
    for d in offs:
        if d == (0, 0, 0):
            vals.append(None)
            continue
        dx, dy, dz = d
        nb = np.roll(sk, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        valid = _grid_valid(dims, d)
        w = _w27(d) * sk * nb
        diag += np.where(valid, w, _w27(d) * kap)
        vals.append(-w)
    vals[offs.index((0, 0, 0))] = diag
    valid = [_grid_valid(dims, d) for d in offs]
    rowptr, colidx, val = _assemble(dims, offs, vals, valid)
    n = nx * ny * nz
    b = rhs_uniform01(n, seed)
    return Problem(f"diffusion27_{nx}x{ny}x{nz}", n, rowptr, colidx, val, b, None,
                   {"dims": dims, "seed": seed, "sigma": sigma, "kind": "diffusion27_nodal"})


def hpcg_27pt(N: int = 32, seed: int = 2505_20719 + 5, beta: float = 0.0) -> Problem:
    """HPCG-style 27-point matrix (diag 26, off -1), Sec. 5.

    beta != 0 gives the HPGMP variant: the +z neighbour becomes -1+beta and
    the -z neighbour -1-beta (reading: '+z' is the forward direction).
    """
    dims = (N, N, N)
    offs = _offsets27()
    shape = (N, N, N)
    vals = []
    for d in offs:
        if d == (0, 0, 0):
            vals.append(np.full(shape, 26.0))
        elif d == (0, 0, 1):
            vals.append(np.full(shape, -1.0 + beta))
        elif d == (0, 0, -1):
            vals.append(np.full(shape, -1.0 - beta))
        else:
            vals.append(np.full(shape, -1.0))
    valid = [_grid_valid(dims, d) for d in offs]
    rowptr, colidx, val = _assemble(dims, offs, vals, valid)
    n = N ** 3
    b = rhs_uniform01(n, seed)
    kind = "hpgmp_27pt" if beta else "hpcg_27pt"
    return Problem(f"{kind}_{N}", n, rowptr, colidx, val, b, None,
                   {"dims": dims, "seed": seed, "beta": beta, "kind": kind})


def random_dd_sparse(n: int, per_row: int = 6, seed: int = 7, symmetric: bool = False,
                     dominance: float = 1.5) -> Problem:
    """Random sparse, strictly diagonally dominant matrix (small-n test cases).

    Off-diagonal pattern: `per_row` random distinct columns per row, values
    N(0, 1); diagonal = dominance * (sum of |off-diagonals| in the row) + 1 with
    a random sign.  Symmetric variant: A + A^T pattern and values.
    """
    cols = rng.integers(seed, 31, n * per_row, 0, n - 1).reshape(n, per_row)
    vals = rng.normal(seed, 32, n * per_row).reshape(n, per_row)
    rows = np.repeat(np.arange(n), per_row)
    A = sp.coo_matrix((vals.ravel(), (rows, cols.ravel())), shape=(n, n)).tocsr()
    A.setdiag(0.0)
    A.eliminate_zeros()
    if symmetric:
        A = (A + A.T).tocsr()
    A.sum_duplicates()
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    sign = np.where(rng.uniform01(seed, 33, n) < 0.5, -1.0, 1.0)
    if symmetric:
        sign = np.ones(n)
    A = (A + sp.diags(sign * (dominance * absrow + 1.0))).tocsr()
    A.sort_indices()
    x_true = 2.0 * rng.uniform01(seed, 34, n) - 1.0
    b = A @ x_true
    return Problem(f"random_dd_{n}", n, A.indptr.astype(np.int32), A.indices.astype(np.int32),
                   A.data.astype(np.float64), b, x_true, {"seed": seed, "kind": "random_dd"})


def _diffusion2d_5pt(dims2, sigma, seed):
    nx, ny = dims2
    dims = (nx, ny, 1)
    kx, ky, _ = _face_coefficients(dims, sigma, seed, 1)
    diag = kx[:, :, :-1] + kx[:, :, 1:] + ky[:, :-1, :] + ky[:, 1:, :]
    offs = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    vals = [-ky[:, :-1, :], -kx[:, :, :-1], diag, -kx[:, :, 1:], -ky[:, 1:, :]]
    valid = [_grid_valid(dims, d) for d in offs]
    return _assemble(dims, offs, vals, valid)


def batched_diffusion_systems(count: int = 64, n_lo: float = 1e4, n_hi: float = 5e5,
                              sigma: float = 1.5, seed: int = 2505_20719 + 3,
                              max_rhs: int = 8):
    """Many uneven diffusion systems: n log-uniform in [n_lo, n_hi], 2-D
    5-point or 3-D 7-point by a seeded coin, face coefficients as in
    diffusion3d_7pt, and 1..max_rhs right-hand sides each.

    2-D: nx = floor(sqrt(n)), ny = ceil(n/nx).  3-D: nx = ny = round(n^(1/3)),
    nz = ceil(n/(nx*ny)).  Returns a list of (Problem, B) with B of shape
    (nrhs, n) holding uniform [0, 1) right-hand sides.
    """
    u = rng.uniform01(seed, 41, count)
    coin = rng.uniform01(seed, 42, count)
    nrhs = rng.integers(seed, 43, count, 1, max_rhs)
    out = []
    for s in range(count):
        target = float(np.exp(np.log(n_lo) + u[s] * (np.log(n_hi) - np.log(n_lo))))
        sub_seed = seed * 1000 + s
        if coin[s] < 0.5:
            nx = int(np.floor(np.sqrt(target)))
            ny = int(np.ceil(target / nx))
            rowptr, colidx, val = _diffusion2d_5pt((nx, ny), sigma, sub_seed)
            dims = (nx, ny, 1)
        else:
            nx = max(2, int(round(target ** (1.0 / 3.0))))
            nz = int(np.ceil(target / (nx * nx)))
            dims = (nx, nx, nz)
            p = diffusion3d_7pt(dims=dims, sigma=sigma, seed=sub_seed, rhs="none")
            rowptr, colidx, val = p.rowptr, p.colidx, p.val
        n = dims[0] * dims[1] * dims[2]
        B = rng.uniform01(sub_seed, 44, int(nrhs[s]) * n).reshape(int(nrhs[s]), n)
        prob = Problem(f"batch{s}_{'x'.join(map(str, dims))}", n, rowptr, colidx, val,
                       B[0].copy(), None, {"dims": dims, "seed": sub_seed, "kind": "batched"})
        out.append((prob, B))
    return out


def by_name(name: str) -> Problem:
    """The named workloads of the benchmark and tests, at their full sizes."""
    if name == "poisson2d_64":
        return poisson2d_5pt(64)
    if name == "diffusion7_128":
        return diffusion3d_7pt(128)
    if name == "convdiff27_160":
        return convdiff3d_27pt(160)
    if name == "diffusion27_100":
        return diffusion27_nodal(100)
    if name == "diffusion27_160":
        return diffusion27_nodal(160, seed=2505_20719 + 14)
    raise KeyError(name)

"""Pins of the oracle's fp16-vector FGMRES levels (Table 4: the inner F8 of
fp16-F3, the F2 of F4 and the inner FGMRES(64) of fp16-F2 keep their
vectors in fp16).

Reading: such a level computes in fp32 and rounds what it stores -- V[0],
each normalised V[j+1] and each Z[j] = M V[j] -- to fp16.  The pins check
that reading against facts that do not come from the oracle's own code path:
* every stored value is an fp16 number (exact);
* Z[j] is the fp16 rounding of M V[j], whose product of two fp16 numbers is
  exact in fp64 (bit-exact);
* V[0] and V[j+1] are the NEAREST fp16 numbers to v / beta and to
  (A^ z_j - sum_i h_ij v_i) / h_{j+1,j}, recomputed in fp64 from the
  recorded basis and Hessenberg matrix (the Arnoldi relation of Sec. 4.2),
  up to the fp32 arithmetic the level runs in;
* the Givens least-squares solution against numpy's on the recorded H.
The plausible mistakes -- storing fp32 values, or rounding to bf16 -- fail
these checks, which the last tests show on the oracle itself.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from problems import generators as G
from problems import rng

U32 = 2.0 ** -24

_LEVELS = [("fp16-F3", 2), ("F4", 3), ("fp16-F2", 1)]
_IDS = ["fp16-F3 F8", "F4 F2", "fp16-F2 F64"]


def _call(preset, level, v_prec=None, seed=61):
    prob = G.diffusion3d_7pt(dims=(12, 11, 10), seed=seed)
    P = O.Problem(prob, diag_scale=0)  # unscaled: M = diag(A)^-1 is not the identity
    prm = O.preset(preset)
    if v_prec is not None:
        prm.v_prec[level] = v_prec
    v = rng.normal(60 + level, 1, prob.n).astype(np.float32).astype(np.float64)
    z, V, Z, H, g, k = P.inner_arnoldi(prm, O.rich_state(), level, v)
    A16 = sp.csr_matrix((P.get("a16") * np.repeat(P.get("rs16"), np.diff(prob.rowptr)), prob.colidx,
                         prob.rowptr), shape=(prob.n, prob.n))
    return P, prm, v, z, V, Z, H, g, k, A16


def _nearest_excess(exact, stored):
    """max over elements of (|exact - stored| - half the fp16 gap on exact's
    side of stored), relative to max |exact|; <= 0 when stored is the nearest
    fp16 number to exact."""
    r16 = stored.astype(np.float16)
    up = np.nextafter(r16, np.float16(np.inf)).astype(np.float64)
    dn = np.nextafter(r16, np.float16(-np.inf)).astype(np.float64)
    gap = np.where(exact > stored, up - stored, stored - dn)
    return float(np.max(np.abs(exact - stored) - 0.5 * gap) / np.max(np.abs(exact)))


def _arnoldi_targets(v, V, Z, H, k, A16):
    """v / beta, then (A^ z_j - V h_j) / h_{j+1,j} for each kept column."""
    out = [v / np.linalg.norm(v)]
    for j in range(k):
        w = A16 @ Z[j] - V[:j + 1].T @ H[:j + 1, j]
        out.append(w / H[j + 1, j])
    return out


@pytest.mark.parametrize("preset,level", _LEVELS, ids=_IDS)
def test_fp16_level_stores_fp16_numbers(orc, preset, level):
    P, prm, v, z, V, Z, H, g, k, A16 = _call(preset, level)
    assert k == prm.m[level]
    assert np.array_equal(V[:k + 1], V[:k + 1].astype(np.float16).astype(np.float64))
    assert np.array_equal(Z[:k], Z[:k].astype(np.float16).astype(np.float64))
    m16 = P.get("m16")
    assert not np.allclose(m16, 1.0)
    for j in range(k):
        assert np.array_equal(Z[j], (m16 * V[j]).astype(np.float16).astype(np.float64)), j


@pytest.mark.parametrize("preset,level", _LEVELS, ids=_IDS)
def test_fp16_level_basis_is_nearest_rounding_of_arnoldi(orc, preset, level):
    """Each stored basis vector is the nearest fp16 vector to the exact
    Arnoldi update, up to 64 u32 max|.| of fp32 arithmetic."""
    P, prm, v, z, V, Z, H, g, k, A16 = _call(preset, level)
    for j, t in enumerate(_arnoldi_targets(v, V, Z, H, k, A16)):
        assert _nearest_excess(t, V[j]) <= 64 * U32, j
    # the fp16 basis is orthonormal to O(u16), not to fp32 accuracy
    e = np.abs(V[:k + 1] @ V[:k + 1].T - np.eye(k + 1)).max()
    assert e <= 20 * k * 2.0 ** -11


@pytest.mark.parametrize("preset,level", _LEVELS, ids=_IDS)
def test_fp16_level_least_squares(orc, preset, level):
    P, prm, v, z, V, Z, H, g, k, A16 = _call(preset, level)
    beta = np.linalg.norm(v)
    e1 = np.zeros(k + 1)
    e1[0] = beta
    y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
    ls = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
    assert abs(abs(g[k]) - ls) <= 1e-4 * ls + 10 * k * U32 * beta
    zy = Z[:k].T @ y
    assert np.linalg.norm(z - zy) <= 1e-4 * np.linalg.norm(zy)
    # the level still reduces its residual (8, 2 or 64 iterations on a diffusion matrix)
    assert np.linalg.norm(v - A16 @ z) < 0.9 * beta


def test_fp16_pins_reject_fp32_storage(orc):
    """The same level with fp32 vectors stores values that are not fp16 numbers."""
    P, prm, v, z, V, Z, H, g, k, A16 = _call("fp16-F3", 2, v_prec=O.F32)
    assert not np.array_equal(V[1:k + 1], V[1:k + 1].astype(np.float16).astype(np.float64))


def test_fp16_pins_reject_bf16_rounding(orc):
    """Rounding to bf16 instead (8-bit significand) misses the nearest-fp16 pin
    by far more than the fp32 allowance."""
    P, prm, v, z, V, Z, H, g, k, A16 = _call("fp16-F3", 2, v_prec=O.BF16)
    excess = max(_nearest_excess(t, V[j]) for j, t in enumerate(_arnoldi_targets(v, V, Z, H, k, A16)))
    assert excess > 1000 * U32

"""Per-level error of the low-precision levels against the all-fp64 oracle.

For one input v (unit norm, fp32) the GPU runs one call of F_m2 (level 1),
F_m3 (level 2) and R_m4 (level 3) with fp16, bf16 (row-scaled) and fp32
storage; the oracle runs the same calls with every level in fp64 (Table 1
with all precisions raised to fp64).  Reported per level: the relative
difference of the outputs, ||z - z64|| / ||z64||, and each level's own
residual reduction ||v - A^ z|| / ||v|| next to the fp64 one.  Asserted: the
difference stays within a small multiple of the storage precision's unit
roundoff (the 16-bit levels round every stored vector, so a level output
carries O(u) relative error; 20 u leaves room for the m-step recurrences;
fp32 within 200 u32), and the low-precision level reduces the residual as
well as the fp64 level up to that error.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from problems import generators as G
from problems import rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_20719_gb300 import f3r  # noqa: E402

U = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8, "fp32": 2.0 ** -24}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def system():
    prob = G.convdiff3d_27pt(dims=(21, 19, 17), seed=101)
    P = O.Problem(prob, diag_scale=1)
    Ah = sp.csr_matrix((P.get("ahat"), prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    v = rng.normal(140, 1, prob.n)
    v = (v / np.linalg.norm(v)).astype(np.float32).astype(np.float64)
    z64 = {lvl: P.apply(O.preset("fp64-F3R"), O.rich_state(c_ntr=2), lvl, v) for lvl in (1, 2, 3)}
    return prob, Ah, v, z64


@pytest.mark.parametrize("kind", ["fp16", "bf16", "fp32"])
def test_level_error_against_fp64_oracle(system, kind):
    prob, Ah, v, z64 = system
    prm = {"fp16": f3r.default_params(), "bf16": f3r.preset("bf16-F3R"), "fp32": f3r.preset("fp32-F3R")}[kind]
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), prm)
    vd = dev(v.astype(np.float32))
    bound = 20 * U[kind] if kind != "fp32" else 200 * U[kind]
    # ||A^||_2 <= sqrt(||A^||_1 ||A^||_inf)
    norm_a = float(np.sqrt(abs(Ah).sum(axis=0).max() * abs(Ah).sum(axis=1).max()))
    for level, name in ((1, "F_m2"), (2, "F_m3"), (3, "R_m4")):
        s.set_rich_state([1.0, 1.0], 2)
        z = torch.empty(prob.n, dtype=torch.float32, device="cuda")
        s.apply(level, vd, z)
        torch.cuda.synchronize()
        zg = z.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(zg - z64[level]) / np.linalg.norm(z64[level])
        res = np.linalg.norm(v - Ah @ zg) / np.linalg.norm(v)
        res64 = np.linalg.norm(v - Ah @ z64[level]) / np.linalg.norm(v)
        print(f"{kind} {name}: |z - z64|/|z64| = {err:.3e} ({err / U[kind]:.1f} u), "
              f"level residual {res:.4e} (fp64 {res64:.4e})")
        assert err <= bound, (name, err)
        # ||v - A z|| <= ||v - A z64|| + ||A|| ||z - z64||  (||v|| = 1)
        assert res <= res64 + norm_a * err * np.linalg.norm(z64[level]) * (1 + 1e-6), (name, res, res64)
    s.close()

"""GPU parity at the benchmark's full size (128^3 7-point diffusion, n =
2,097,152), in the launch configuration bench.py times.

* Whole solves against the oracle's own full solves, stored by
  tests/golden/make_oracle_solves.py (oracle only): outer iterations within
  +-1, true residual below 1e-9, and the per-iteration residual estimate
  within |log10 ratio| <= 0.5 while it is above 1e-8 (dot products are tree
  reductions on the GPU and sequential in the oracle, so the histories agree
  to rounding, not bit for bit).
* One fused Richardson call (Algorithm 1, m4 = 2) on every row, bit for bit.
"""
import json
import os

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

HERE = os.path.dirname(os.path.abspath(__file__))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def diffusion128():
    return G.by_name("diffusion7_128")


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "oracle_solves.json")) as f:
        return json.load(f)["diffusion7_128"]


@pytest.mark.parametrize("kind", ["fp16-F3R", "fp32-F3R", "fp64-F3R"])
def test_full_size_solve_matches_oracle_history(diffusion128, golden, kind):
    prob = diffusion128
    ref = golden[kind]
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.preset(kind))
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    res = s.solve(dev(prob.b), x)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    s.close()
    A = prob.to_scipy()
    rel = np.linalg.norm(prob.b - A @ xh) / np.linalg.norm(prob.b)
    print(f"{kind}: {res.outer_iters} outer iterations (oracle {ref['outer_iters']}), rel {rel:.3e} "
          f"(oracle {ref['rel_res_true']:.3e})")
    assert res.status == f3r.OK and ref["status"] == O.OK
    assert rel < 1e-9 and res.rel_res_true < 1e-9
    assert abs(rel - res.rel_res_true) <= 1e-12
    assert abs(res.outer_iters - ref["outer_iters"]) <= 1
    assert res.m_applies == 64 * res.outer_iters
    hg, ho = np.asarray(res.hist), np.asarray(ref["hist"])
    k = min(len(hg), len(ho))
    mask = ho[:k] > 1e-8
    ratio = np.abs(np.log10(hg[:k][mask] / ho[:k][mask]))
    print(f"  max |log10 ratio| of the history: {ratio.max():.3f}")
    assert np.all(ratio <= 0.5), ratio


def test_full_size_richardson_call_bit_exact(diffusion128):
    """The fused m4 = 2 Richardson call of the fp16 level on all 2,097,152 rows."""
    prob = diffusion128
    n = prob.n
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), f3r.default_params())
    P = O.Problem(prob, diag_scale=1)
    v = (rng.normal(120, 1, n) * 1e-2).astype(np.float32)
    omega = [0.83, 1.07]
    s.set_rich_state(omega, 5)
    z = torch.empty(n, dtype=torch.float32, device="cuda")
    s.apply(3, dev(v), z)
    torch.cuda.synchronize()
    want = P.apply(O.params(), O.rich_state(c_ntr=5, omega=omega), 3, v.astype(np.float64))
    got = z.cpu().numpy().astype(np.float64)
    s.close()
    assert np.array_equal(got, want), int(np.sum(got != want))

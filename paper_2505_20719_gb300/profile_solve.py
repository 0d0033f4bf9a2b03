"""Run a few F3R solves of a generated system, for kernel profilers.

    python -m paper_2505_20719_gb300.profile_solve --workload diffusion7_128 --max-outer 2
    python -m paper_2505_20719_gb300.profile_solve --workload diffusion7_160 --m1 8 --max-outer 1

Workloads: the named ones of ``problems.generators.by_name`` plus
``diffusion7_<N>`` (7-point diffusion on an N^3 grid) and ``convdiff27_<N>``
(27-point convection-diffusion on an N^3 grid), so a capture can use a case
whose matrix exceeds the L2 cache but whose fp64 outer basis (``--m1``) stays
small.  Every solve starts from x0 = 0; the solves run back to back on the
current device and the script prints the outer iterations and kernel launches
of the last one.
"""
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2505_20719_gb300 import f3r  # noqa: E402
from problems import generators as G  # noqa: E402


def make_problem(name: str):
    if name.startswith("diffusion7_") and name != "diffusion7_128":
        return G.diffusion3d_7pt(int(name.split("_")[1]))
    if name.startswith("convdiff27_") and name != "convdiff27_160":
        return G.convdiff3d_27pt(int(name.split("_")[1]))
    return G.by_name(name)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="diffusion7_128")
    ap.add_argument("--preset", default="fp16-F3R")
    ap.add_argument("--max-outer", type=int, default=2)
    ap.add_argument("--m1", type=int, default=0, help="outer restart length (0: the preset's)")
    ap.add_argument("--solves", type=int, default=1)
    a = ap.parse_args(argv)
    prob = make_problem(a.workload)
    kw = {"max_outer": a.max_outer}
    params = f3r.preset(a.preset, **kw)
    if a.m1 > 0:
        params.m[0] = a.m1
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    s = f3r.Solver(dev(prob.rowptr), dev(prob.colidx), dev(prob.val), params)
    b = dev(prob.b)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    r = None
    for _ in range(a.solves):
        x.zero_()
        r = s.solve(b, x)
    torch.cuda.synchronize()
    print(f"workload {a.workload} n {prob.n} nnz {prob.nnz} outer {r.outer_iters} "
          f"rel_res {r.rel_res_true:.3e} launches {r.kernel_launches}")


if __name__ == "__main__":
    main()

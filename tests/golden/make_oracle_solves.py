"""Write tests/golden/oracle_solves.json: the CPU oracle's full solves of the
benchmark workloads (outer iterations, final true residual, the estimated
relative residual after every outer iteration and the true one at each cycle
start).  Calls only oracle/ and problems/; the full-size GPU parity test
compares its residual history with these, and the benchmark's reference arm
scales its per-iteration timing by the counts."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from problems import generators as G  # noqa: E402


def main():
    out = {}
    for wl, ds in (("poisson2d_64", 0), ("diffusion7_128", 1)):
        prob = G.by_name(wl)
        P = O.Problem(prob, diag_scale=ds)
        out[wl] = {}
        for kind in ("fp16-F3R", "fp32-F3R", "fp64-F3R"):
            t0 = time.time()
            r = P.solve(O.preset(kind, diag_scale=ds), prob.b)
            out[wl][kind] = {"outer_iters": r.outer_iters, "rel_res_true": r.rel_res_true, "status": r.status,
                             "m_applies": r.m_applies, "seconds": round(time.time() - t0, 1),
                             "threads": O.num_threads(), "hist": [float(h) for h in r.hist],
                             "true_hist": [float(h) for h in r.true_hist]}
            print(wl, kind, {k: v for k, v in out[wl][kind].items() if "hist" not in k}, flush=True)
    with open(os.path.join(HERE, "oracle_solves.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()

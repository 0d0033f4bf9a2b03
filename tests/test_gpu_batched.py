"""Batched F3R (many systems and right-hand sides in one persistent launch)
against the single-system CUDA path and the CPU oracle."""
import numpy as np
import pytest

import oracle as O
from problems import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_20719_gb300 import f3r  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def batch():
    return G.batched_diffusion_systems(count=6, n_lo=500, n_hi=20000, max_rhs=3, seed=401)


@pytest.mark.parametrize("cluster", [1, 2, 8])
def test_batched_matches_single_system_solves(batch, cluster):
    systems = [(dev(p.rowptr), dev(p.colidx), dev(p.val), B.shape[0]) for p, B in batch]
    bs = f3r.BatchedSolver(systems, f3r.default_params())
    bs.set_cluster(cluster)
    Bs, Xs, meta = [], [], []
    for k, (p, B) in enumerate(batch):
        for r in range(B.shape[0]):
            Bs.append(dev(B[r]))
            Xs.append(torch.zeros(p.n, dtype=torch.float64, device="cuda"))
            meta.append((k, r))
    code, res = bs.solve(Bs, Xs)
    torch.cuda.synchronize()
    assert code == f3r.OK
    for q, (k, r) in enumerate(meta):
        p, B = batch[k]
        A = p.to_scipy()
        x = Xs[q].cpu().numpy()
        rel = np.linalg.norm(B[r] - A @ x) / np.linalg.norm(B[r])
        assert res[q].status == f3r.OK and res[q].system == k and res[q].rhs == r
        assert rel < 1e-9 and abs(rel - res[q].rel_res_true) <= 1e-12
        assert res[q].m_applies == 64 * res[q].outer_iters
        s = f3r.Solver(dev(p.rowptr), dev(p.colidx), dev(p.val), f3r.default_params())
        xs = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        rs = s.solve(dev(B[r]), xs)
        assert abs(rs.outer_iters - res[q].outer_iters) <= 1
        s.close()
    bs.close()


def test_batched_instance_matches_oracle(batch):
    p, B = batch[0]
    bs = f3r.BatchedSolver([(dev(p.rowptr), dev(p.colidx), dev(p.val), 1)], f3r.default_params())
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    code, res = bs.solve([dev(B[0])], [x])
    ref = O.Problem(p).solve(O.params(), B[0])
    assert code == f3r.OK and ref.status == O.OK
    assert abs(res[0].outer_iters - ref.outer_iters) <= max(1, ref.outer_iters // 10)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


def test_batched_split_large_systems_to_single_path(batch):
    """With batch_wide < 0, systems of at least batch_split rows are solved one
    after another by the single-system path: their results are bit for bit
    those of a separate f3r_solve; the rest still go through the persistent
    launch and converge."""
    split = 5000
    assert any(p.n >= split for p, _ in batch) and any(p.n < split for p, _ in batch)
    systems = [(dev(p.rowptr), dev(p.colidx), dev(p.val), B.shape[0]) for p, B in batch]
    bs = f3r.BatchedSolver(systems, f3r.default_params(batch_split=split, batch_wide=-1))
    Bs, Xs, meta = [], [], []
    for k, (p, B) in enumerate(batch):
        for r in range(B.shape[0]):
            Bs.append(dev(B[r]))
            Xs.append(torch.zeros(p.n, dtype=torch.float64, device="cuda"))
            meta.append((k, r))
    bs.autotune(Bs, Xs)
    code, res = bs.solve(Bs, Xs)
    torch.cuda.synchronize()
    assert code == f3r.OK
    for q, (k, r) in enumerate(meta):
        p, B = batch[k]
        x = Xs[q].cpu().numpy()
        rel = np.linalg.norm(B[r] - p.to_scipy() @ x) / np.linalg.norm(B[r])
        assert res[q].status == f3r.OK and res[q].system == k and res[q].rhs == r and rel < 1e-9
        if p.n >= split:
            s = f3r.Solver(dev(p.rowptr), dev(p.colidx), dev(p.val), f3r.default_params(batch_split=split))
            xs = torch.zeros(p.n, dtype=torch.float64, device="cuda")
            rs = s.solve(dev(B[r]), xs)
            assert rs.outer_iters == res[q].outer_iters
            assert torch.equal(xs, Xs[q])
            s.close()
    bs.close()


def _instances(batch):
    Bs, Xs, meta = [], [], []
    for k, (p, B) in enumerate(batch):
        for r in range(B.shape[0]):
            Bs.append(dev(B[r]))
            Xs.append(torch.zeros(p.n, dtype=torch.float64, device="cuda"))
            meta.append((k, r))
    return Bs, Xs, meta


def _check(batch, Xs, meta, res):
    for q, (k, r) in enumerate(meta):
        p, B = batch[k]
        rel = np.linalg.norm(B[r] - p.to_scipy() @ Xs[q].cpu().numpy()) / np.linalg.norm(B[r])
        assert res[q].status == f3r.OK and rel < 1e-9, (q, rel)
        assert res[q].path == 0  # every system here is below batch_split: the persistent launch


@pytest.mark.parametrize("cluster,threads", [(2, 256), (4, 512), (1, 256)])
def test_batched_team_shapes_and_graph_replay(batch, cluster, threads):
    """Every team shape solves every instance; the second solve replays the
    captured graph with other x buffers (the pinned table carries them)."""
    systems = [(dev(p.rowptr), dev(p.colidx), dev(p.val), B.shape[0]) for p, B in batch]
    bs = f3r.BatchedSolver(systems, f3r.default_params())
    bs.set_shape(cluster, threads)
    for rep in range(2):
        Bs, Xs, meta = _instances(batch)
        code, res = bs.solve(Bs, Xs)
        torch.cuda.synchronize()
        assert code == f3r.OK
        _check(batch, Xs, meta, res)
    info = bs.info()
    assert (info["cluster"], info["threads"]) == (cluster, threads)
    assert info["graph_launches"] == 2 and info["instances_launch"] == len(meta) and info["instances_single"] == 0
    assert info["grid"] % cluster == 0 and info["grid"] > 0
    bs.close()


def test_batched_autotune_picks_a_shape(batch):
    systems = [(dev(p.rowptr), dev(p.colidx), dev(p.val), B.shape[0]) for p, B in batch]
    bs = f3r.BatchedSolver(systems, f3r.default_params())
    Bs, Xs, meta = _instances(batch)
    chosen = bs.autotune(Bs, Xs)
    info = bs.info()
    assert chosen == info["cluster"] and info["cluster"] in (1, 2, 4, 8) and info["threads"] in (256, 512)
    assert all(float(x.abs().max()) == 0.0 for x in Xs)  # X zeroed again
    code, res = bs.solve(Bs, Xs)
    torch.cuda.synchronize()
    assert code == f3r.OK
    _check(batch, Xs, meta, res)
    bs.close()


def test_batched_large_systems_next_to_the_launch(batch):
    """With batch_split below some systems' size and batch_wide < 0, those
    instances run on the single-system path beside the persistent launch:
    every instance is still solved, each path reports itself."""
    systems = [(dev(p.rowptr), dev(p.colidx), dev(p.val), B.shape[0]) for p, B in batch]
    ns = sorted(p.n for p, _ in batch)
    split = ns[len(ns) // 2]
    bs = f3r.BatchedSolver(systems, f3r.default_params(batch_split=split, batch_wide=-1))
    Bs, Xs, meta = _instances(batch)
    code, res = bs.solve(Bs, Xs)
    torch.cuda.synchronize()
    assert code == f3r.OK
    info = bs.info()
    assert info["instances_single"] > 0 and info["instances_launch"] > 0
    for q, (k, r) in enumerate(meta):
        p, B = batch[k]
        rel = np.linalg.norm(B[r] - p.to_scipy() @ Xs[q].cpu().numpy()) / np.linalg.norm(B[r])
        assert res[q].status == f3r.OK and rel < 1e-9, (q, rel)
        assert res[q].path == (1 if p.n >= split else 0)
    bs.close()


@pytest.mark.parametrize("cluster,wide", [(1, 2), (2, 3), (1, 0)])
def test_batched_wide_teams_all_in_one_launch(batch, cluster, wide):
    """Every instance in the one persistent launch: the large systems' on wide
    teams of several clusters (global-memory barriers, cluster sums added in
    cluster order), the others on one cluster each.  Each instance converges
    to 1e-9 within one outer iteration of its single-system solve, reports its
    path, and a solve is one graph replay with no single-system work."""
    systems = [(dev(p.rowptr), dev(p.colidx), dev(p.val), B.shape[0]) for p, B in batch]
    ns = sorted(p.n for p, _ in batch)
    split = ns[len(ns) // 2]
    bs = f3r.BatchedSolver(systems, f3r.default_params(batch_split=split, batch_wide=wide))
    bs.set_shape(cluster, 512)
    Bs, Xs, meta = _instances(batch)
    if wide == 0:  # automatic: the autotuner also picks the clusters per wide team
        bs.autotune(Bs, Xs)
    g0 = bs.info()["graph_launches"]
    code, res = bs.solve(Bs, Xs)
    torch.cuda.synchronize()
    assert code == f3r.OK
    info, wi = bs.info(), bs.wide_info()
    assert info["instances_single"] == 0 and info["instances_launch"] == len(meta)
    assert info["graph_launches"] == g0 + 1
    assert wi["teams"] >= 1 and wi["instances"] == sum(B.shape[0] for p, B in batch if p.n >= split)
    if wide > 0:
        assert wi["clusters_per_team"] == wide
    else:
        assert wi["clusters_per_team"] in (2, 4, 8)
    for q, (k, r) in enumerate(meta):
        p, B = batch[k]
        rel = np.linalg.norm(B[r] - p.to_scipy() @ Xs[q].cpu().numpy()) / np.linalg.norm(B[r])
        assert res[q].status == f3r.OK and rel < 1e-9, (q, rel)
        assert abs(rel - res[q].rel_res_true) <= 1e-12
        assert res[q].path == (2 if p.n >= split else 0)
        assert res[q].m_applies == 64 * res[q].outer_iters
        if p.n >= split:
            s = f3r.Solver(dev(p.rowptr), dev(p.colidx), dev(p.val), f3r.default_params())
            xs = torch.zeros(p.n, dtype=torch.float64, device="cuda")
            rs = s.solve(dev(B[r]), xs)
            assert abs(rs.outer_iters - res[q].outer_iters) <= 1
            s.close()
    bs.close()

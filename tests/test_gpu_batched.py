"""Batched form: systems of uneven size solved together with grouped kernels and one V-cycle graph,
against the same systems solved one by one and against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2408_08262_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2408_08262_gb300 import airg  # noqa: E402


def dev(p):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (p.rowptr, p.col, p.val))


def systems():
    spec = [(16, 0.3, 0.0), (24, 2.0, 1.5), (32, 4.0, 0.5), (20, 5.5, 3.0), (40, 1.0, 0.0), (12, 3.0, 4.9)]
    return [P.p1_dg_2d(m, th, sigma=sg, seed=1000 + k) for k, (m, th, sg) in enumerate(spec)]


def test_batched_matches_individual_solves_and_oracle():
    ps = systems()
    par = airg.Params(coarse_size=64)
    Hs = [airg.Hierarchy(*dev(p), par) for p in ps]
    assert len({H.num_levels for H in Hs}) > 1  # uneven depths
    bs = [torch.from_numpy(p.b).cuda() for p in ps]
    B = airg.Batch(Hs)
    xs, infos = B.solve(bs, rtol=1e-12)
    for p, H, b, x, info in zip(ps, Hs, bs, xs, infos):
        xi, ii = H.solve(b, rtol=1e-12)
        assert info["status"] == 0 and info["relres"] <= 1e-12
        assert abs(info["iters"] - ii["iters"]) <= 1
        assert (torch.linalg.norm(x - xi) / torch.linalg.norm(xi)).item() <= 1e-10
    Ho = O.Hierarchy(ps[2].rowptr, ps[2].col, ps[2].val, O.Params(coarse_size=64))
    xo, io = Ho.solve(ps[2].b, rtol=1e-12)
    assert np.linalg.norm(xs[2].cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-10
    B.close()


def test_batched_restarts_and_per_system_status():
    ps = systems()[:4]
    Hs = [airg.Hierarchy(*dev(p), airg.Params(coarse_size=64)) for p in ps]
    bs = [torch.from_numpy(p.b).cuda() for p in ps]
    B = airg.Batch(Hs)
    xs, infos = B.solve(bs, rtol=1e-12, restart=3, max_it=200)  # several restart cycles
    for p, x, info in zip(ps, xs, infos):
        assert info["status"] == 0
        r = p.b - p.scipy() @ x.cpu().numpy()
        assert np.linalg.norm(r) / np.linalg.norm(p.b) <= 1e-12
    xs, infos = B.solve(bs, rtol=1e-30, max_it=4)
    assert all(i["status"] == 1 and i["iters"] == 4 for i in infos)
    zero = [torch.zeros_like(b) for b in bs]
    xs, infos = B.solve(zero, rtol=1e-10)
    assert all(i["iters"] == 0 for i in infos) and all(torch.count_nonzero(x) == 0 for x in xs)


def test_batched_autotuner_picks_lanes_and_keeps_the_solution(monkeypatch):
    # the autotuner times every lanes-per-row variant of the large grouped operators; the chosen
    # variants change only the rounding of the row sums
    ps = systems()
    par = airg.Params(coarse_size=64)
    Hs = [airg.Hierarchy(*dev(p), par) for p in ps]
    bs = [torch.from_numpy(p.b).cuda() for p in ps]
    B = airg.Batch(Hs)
    tuned = B.tuned()
    assert tuned and all(r in (1, 2, 4, 8, 16, 32) and c in (1, 2, 4, 8, 16, 32) for r, c in tuned)
    xs, infos = B.solve(bs, rtol=1e-12)
    B.close()
    monkeypatch.setenv("AIRG_NO_AUTOTUNE", "1")
    Br = airg.Batch(Hs)
    assert Br.tuned() == []
    xr, ir = Br.solve(bs, rtol=1e-12)
    Br.close()
    for x, i, y, j in zip(xs, infos, xr, ir):
        assert i["status"] == 0 and j["status"] == 0 and abs(i["iters"] - j["iters"]) <= 1
        assert (torch.linalg.norm(x - y) / torch.linalg.norm(y)).item() <= 1e-10


def test_batched_at_the_full_system_sizes():
    # the largest and smallest member sizes of the 64-system batch (512^2: 1,572,864 DOFs; 64^2:
    # 24,576 DOFs) in one batch, with the default parameters (automatic truncation): each against
    # its individual solve, the small one also against the oracle
    ps = [P.p1_dg_2d(512, 2.2, sigma=1.7, seed=2001), P.p1_dg_2d(64, 4.1, sigma=0.4, seed=2002)]
    par = airg.Params()
    Hs = [airg.Hierarchy(*dev(p), par) for p in ps]
    bs = [torch.from_numpy(p.b).cuda() for p in ps]
    B = airg.Batch(Hs)
    xs, infos = B.solve(bs, rtol=1e-12, max_it=300)
    for p, H, b, x, info in zip(ps, Hs, bs, xs, infos):
        xi, ii = H.solve(b, rtol=1e-12, max_it=300)
        assert info["status"] == 0 and ii["status"] == 0 and info["relres"] <= 1e-12
        assert abs(info["iters"] - ii["iters"]) <= 1
        assert (torch.linalg.norm(x - xi) / torch.linalg.norm(xi)).item() <= 1e-10
    q = ps[1]
    Ho = O.Hierarchy(q.rowptr, q.col, q.val, O.Params(coarse_size=max(64, min(60000, q.n // 16))))
    xo, io = Ho.solve(q.b, rtol=1e-12, max_it=300)
    assert io["status"] == 0
    assert np.linalg.norm(xs[1].cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-10
    B.close()


def test_concurrent_setups_equal_the_individual_setups():
    # airg_setup_many builds the hierarchies of many systems on several host threads and streams at
    # once; every hierarchy must be bitwise the one airg_setup builds, and they batch as usual
    ps = systems() + [P.p1_dg_2d(128, 0.7, sigma=2.0, seed=1010), P.p1_dg_2d(96, 5.1, sigma=0.0, seed=1011)]
    par = airg.Params(coarse_size=64, keep_setup=1)
    mats = [dev(p) for p in ps]
    Hm = airg.setup_many(mats, par, nthreads=4)
    Hs = [airg.Hierarchy(*m, par) for m in mats]
    for Ha, Hb in zip(Hm, Hs):
        assert Ha.num_levels == Hb.num_levels
        for l in range(Ha.num_levels):
            names = ["A", "Ainv"] if Ha.level_info(l)["coarsest"] else ["A", "Ainv", "Z", "AF_solve", "Z_solve"]
            for which in names:
                for a, b in zip(Ha.export(l, which), Hb.export(l, which)):
                    assert np.array_equal(a, b), (l, which)
    bs = [torch.from_numpy(p.b).cuda() for p in ps]
    for Ha, Hb, b in zip(Hm, Hs, bs):
        xa, ia = Ha.solve(b, rtol=1e-12)
        xb, ib = Hb.solve(b, rtol=1e-12)
        assert ia == ib and torch.equal(xa, xb)
    B = airg.Batch(Hm)
    xs, infos = B.solve(bs, rtol=1e-12)
    assert all(i["status"] == 0 for i in infos)
    B.close()
    for H in Hm + Hs:
        H.close()

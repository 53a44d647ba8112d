"""Adjoint form: A^T hierarchy, SDDMM and the differentiable solve, against independent routes.

* transpose and SDDMM against scipy / numpy;
* the A^T hierarchy's solve and CF splitting against the oracle run on the transposed matrix;
* gradients of J = sum_i w_i u_i (u = A(sigma)^-1 b(q), upwind P1 DG, per-element sigma) against
  central finite differences with h = 1e-6 on 20 seeded entries, and against the oracle's
  dense-solve gradient on a 16 x 16 mesh.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2408_08262_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2408_08262_gb300 import airg  # noqa: E402


def dev(rp, ci, v):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rp, ci, v))


def sp_t(p):
    T = p.scipy().T.tocsr()
    T.sort_indices()
    return T.indptr.astype(np.int32), T.indices.astype(np.int32), T.data.astype(np.float64)


def test_transpose_matches_scipy():
    p = P.adjoint_2d(40)
    rp, ci, v = airg.transpose(*dev(p.rowptr, p.col, p.val))
    trp, tci, tv = sp_t(p)
    assert np.array_equal(rp.cpu().numpy(), trp)
    assert np.array_equal(ci.cpu().numpy(), tci)
    assert np.array_equal(v.cpu().numpy(), tv)


def test_sddmm_is_the_sampled_outer_product():
    p = P.adjoint_2d(24)
    rng = np.random.default_rng(5)
    lam, x = rng.standard_normal(p.n), rng.standard_normal(p.n)
    rp, ci, _ = dev(p.rowptr, p.col, p.val)
    out = airg.sddmm(rp, ci, torch.from_numpy(lam).cuda(), torch.from_numpy(x).cuda(), -1.0).cpu().numpy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    assert np.array_equal(out, (-1.0 * lam[rows]) * x[p.col])


def test_transpose_hierarchy_matches_oracle():
    p = P.adjoint_2d(48)
    trp, tci, tv = sp_t(p)
    op = O.Params(coarse_size=64)
    c = np.random.default_rng(2).standard_normal(p.n)
    Ho = O.Hierarchy(trp, tci, tv, op)
    yo, io = Ho.solve(c, rtol=1e-12)
    HT = airg.Hierarchy(*dev(p.rowptr, p.col, p.val), airg.Params(coarse_size=64, keep_setup=1), transpose=True)
    yg, ig = HT.solve(torch.from_numpy(c).cuda(), rtol=1e-12)
    assert ig["status"] == 0
    assert np.linalg.norm(yg.cpu().numpy() - yo) / np.linalg.norm(yo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1
    # level 0 of the transposed hierarchy is the oracle's splitting of A^T, bit for bit
    assert np.array_equal(HT.vectors(0)["cf"], Ho.vectors(0)["cf"])


class Model:
    """J(sigma, q) = w . u with A(sigma) u = b(q) on the upwind P1 DG discretisation."""

    def __init__(self, p, params):
        self.p = p
        self.val0, self.pos, self.coef, self.area = P.sigma_q_maps(p)
        self.params = params
        self.rp, self.ci, _ = dev(p.rowptr, p.col, p.val)
        self.pos_t = torch.from_numpy(self.pos.ravel()).cuda()
        self.coef_t = torch.from_numpy(self.coef).cuda()
        self.val0_t = torch.from_numpy(self.val0).cuda()
        self.area_t = torch.from_numpy(self.area).cuda()

    def values(self, sigma):
        return self.val0_t.index_add(0, self.pos_t, (sigma[:, None] * self.coef_t).reshape(-1))

    def load(self, q):
        return torch.repeat_interleave(q * self.area_t / 3.0, 3)

    def J_and_grads(self, sigma, q, w):
        sigma = sigma.clone().requires_grad_(True)
        q = q.clone().requires_grad_(True)
        x = airg.solve_fn().apply(self.rp, self.ci, self.values(sigma), self.load(q), self.params, 1e-12)
        J = (w * x).sum()
        J.backward()
        return J.item(), sigma.grad.cpu().numpy(), q.grad.cpu().numpy(), x.detach()

    def solve(self, val, b):
        H = airg.Hierarchy(self.rp, self.ci, val, self.params)
        x, info = H.solve(b, rtol=1e-12, max_it=500)
        assert info["status"] == 0
        return x


def central_difference(model, sigma, q, w, which, e, h):
    """(J(+h) - J(-h)) / 2h, evaluated with the exact identity
    J(+h) - J(-h) = w . A_+^{-1} (b_+ - b_- - (A_+ - A_-) u_-), so that two nearly equal values of J
    are never subtracted (the gradient of one element is ~1e-6 of J)."""
    s_p, s_m, q_p, q_m = sigma.clone(), sigma.clone(), q.clone(), q.clone()
    if which == "sigma":
        s_p[e] += h
        s_m[e] -= h
    else:
        q_p[e] += h
        q_m[e] -= h
    vp, vm = model.values(s_p), model.values(s_m)
    bp, bm = model.load(q_p), model.load(q_m)
    um = model.solve(vm, bm)
    dA_um = torch.zeros_like(um)
    rows = torch.repeat_interleave(torch.arange(model.p.n, device="cuda"), torch.from_numpy(np.diff(model.p.rowptr)).cuda())
    dA_um.index_add_(0, rows, (vp - vm) * um[torch.from_numpy(model.p.col.astype(np.int64)).cuda()])
    du = model.solve(vp, (bp - bm) - dA_um)
    return (w * du).sum().item() / (2 * h)


def test_adjoint_gradients_match_central_differences():
    p = P.adjoint_2d(256)  # 393,216 DOFs, per-element sigma ~ U[0, 2], theta = 1.1
    model = Model(p, airg.Params())
    w = torch.from_numpy(np.random.default_rng(240808266).standard_normal(p.n)).cuda()
    sigma = torch.from_numpy(p.meta["sigma_e"].copy()).cuda()
    q = torch.ones(p.meta["n_tri"], dtype=torch.float64, device="cuda")
    J, gs, gq, _ = model.J_and_grads(sigma, q, w)
    rng = np.random.default_rng(7)
    ne = p.meta["n_tri"]
    for which, g in (("sigma", gs), ("q", gq)):
        for e in rng.choice(ne, 10, replace=False):
            fd = central_difference(model, sigma, q, w, which, int(e), 1e-6)
            assert fd == pytest.approx(g[e], rel=1e-5, abs=1e-9 * np.abs(g).max()), (which, e)


def test_adjoint_gradients_match_oracle_dense_solve():
    p = P.adjoint_2d(16)
    model = Model(p, airg.Params(coarse_size=64))
    w_np = np.random.default_rng(11).standard_normal(p.n)
    w = torch.from_numpy(w_np).cuda()
    sigma = torch.from_numpy(p.meta["sigma_e"].copy()).cuda()
    q = torch.ones(p.meta["n_tri"], dtype=torch.float64, device="cuda")
    J, gs, gq, x = model.J_and_grads(sigma, q, w)
    # dense route: u = A^-1 b, lambda = A^-T w, dJ/dA = -lambda u^T, chained through the maps
    u = O.dense_solve(p.rowptr, p.col, p.val, p.b)
    trp, tci, tv = sp_t(p)
    lam = O.dense_solve(trp, tci, tv, w_np)
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    G = -lam[rows] * u[p.col]
    gs_ref = (G[model.pos] * model.coef).sum(axis=1)
    gq_ref = (lam.reshape(-1, 3) * (model.area / 3.0)[:, None]).sum(axis=1)
    assert J == pytest.approx(w_np @ u, rel=1e-10)
    np.testing.assert_allclose(gs, gs_ref, rtol=1e-8, atol=1e-12 * np.abs(gs_ref).max())
    np.testing.assert_allclose(gq, gq_ref, rtol=1e-8, atol=1e-12 * np.abs(gq_ref).max())


def test_cached_hierarchies_are_reused_while_the_matrix_is_unchanged():
    # the adjoint form's cache keeps the hierarchies of A and A^T: right-hand sides that change
    # (the source q) re-use them, and the gradients are bitwise those of fresh setups; writing to
    # the matrix's values builds new ones
    p = P.adjoint_2d(32)
    rp, ci, v = dev(p.rowptr, p.col, p.val)
    w = torch.from_numpy(np.random.default_rng(7).standard_normal(p.n)).cuda()
    cache = airg.HierarchyCache()
    Fc, Fn = airg.solve_fn(cache), airg.solve_fn()
    grads, held = [], []
    for q in (1.0, 2.0, 0.5):
        out = []
        for F in (Fc, Fn):
            vv = v.detach().clone().requires_grad_(True) if F is Fn else v.requires_grad_(True)
            bb = (q * torch.from_numpy(p.b).cuda()).requires_grad_(True)
            x = F.apply(rp, ci, vv, bb, airg.Params(), 1e-10)
            (w * x).sum().backward()
            out.append((vv.grad.clone(), bb.grad.clone()))
            vv.grad = None
        grads.append(out)
        held.append((cache.entries[False][1], cache.entries[True][1]))
    for (gc, gn) in grads:
        assert torch.equal(gc[0], gn[0]) and torch.equal(gc[1], gn[1])
    assert all(h[0] is held[0][0] and h[1] is held[0][1] for h in held)  # built once, re-used twice
    with torch.no_grad():
        v.mul_(1.0)  # a write: the version counter moves, so the next call sets up again
    x = Fc.apply(rp, ci, v, torch.from_numpy(p.b).cuda(), airg.Params(), 1e-10)
    assert cache.entries[False][1] is not held[0][0]
    cache.clear()

"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on identical seeded inputs.

Bars (from the method's statement of parity):
  * CF splittings: bit-exact (integer output of FP64 decisions taken in the same order).
  * Extracted blocks A_ff / A_fc / A_cf: bit-exact (pure data movement).
  * Polynomial coefficients: relative 1e-10 (power basis and TSQR reduce in a different order).
  * Ainv, Z, coarse matrices: identical patterns, values within 1e-10 relative to the row scale.
  * Solutions: relative error <= 1e-10 against the oracle at rtol 1e-12; iterations within +-1.
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


def dev(p_or_tuple):
    if hasattr(p_or_tuple, "rowptr"):
        rp, ci, v = p_or_tuple.rowptr, p_or_tuple.col, p_or_tuple.val
    else:
        rp, ci, v = p_or_tuple
    return (torch.from_numpy(np.ascontiguousarray(rp, dtype=np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(ci, dtype=np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda())


def gpu_params(op: O.Params, keep=1) -> airg.Params:
    return airg.Params(strong_threshold=op.strong_threshold, ddc_fraction=op.ddc_fraction,
                       pmisr_max_loops=op.pmisr_max_loops, poly_order=op.poly_order,
                       coarse_poly_order=op.coarse_poly_order, coarse_iters=op.coarse_iters,
                       coarse_size=op.coarse_size, max_levels=op.max_levels, drop_R=op.drop_R, drop_Ac=op.drop_Ac,
                       n_smooth_up=op.n_smooth_up, keep_setup=keep, seed=op.seed, sparsity_order=op.sparsity_order,
                       matrix_free=op.matrix_free, ideal_prolong=op.ideal_prolong)


def assert_csr_close(a, b, rtol=1e-10, what=""):
    (r1, c1, v1), (r2, c2, v2) = a, b
    assert np.array_equal(r1, r2), f"{what}: row pointers differ"
    assert np.array_equal(c1, c2), f"{what}: columns differ"
    if len(v1) == 0:
        return
    n = len(r1) - 1
    rows = np.repeat(np.arange(n), np.diff(r1))
    scale = np.zeros(n)
    np.maximum.at(scale, rows, np.abs(v1))
    err = np.abs(v1 - v2) / np.maximum(scale[rows], 1e-300)
    assert err.max() <= rtol, f"{what}: max rel err {err.max():.3e}"


# ---------------------------------------------------------------------------------------------
# CF splitting: bit-exact
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mesh,theta,alpha,loops", [(64, 0.3, 0.5, 3), (64, 0.3, 0.0, 3), (64, 0.3, 0.99, 3),
                                                     (37, 2.0, 0.5, 0), (64, 5.1, 0.25, 1)])
def test_cf_split_bitexact_top_level(mesh, theta, alpha, loops):
    p = P.p1_dg_2d(mesh, theta, seed=mesh * 7 + 1)
    op = O.Params(strong_threshold=alpha, pmisr_max_loops=loops)
    ref = O.cf_split(p.rowptr, p.col, p.val, op)["cf"]
    got = airg.cf_split(*dev(p), gpu_params(op), level=0).cpu().numpy()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mesh", [64, 33])
def test_ddc_theta_matches_oracle_bitexact(mesh):
    # airg_ddc_theta on the PMISR splitting (DDC fraction 0) is the oracle's theta bit for bit; on
    # the final splitting every F-point is below the oracle's threshold tau
    p = P.p1_dg_2d(mesh, 0.3, seed=mesh + 11, sigma_uniform=(0.0, 2.0))
    d = O.cf_split(p.rowptr, p.col, p.val, O.Params())
    rp, ci, v = dev(p)
    cf0 = airg.cf_split(rp, ci, v, airg.Params(ddc_fraction=0.0))
    assert np.array_equal(cf0.cpu().numpy(), d["cf_pmisr"])
    th0 = airg.ddc_theta(rp, ci, v, cf0).cpu().numpy()
    assert np.array_equal(th0, d["theta"])
    cf1 = airg.cf_split(rp, ci, v, airg.Params())
    th1 = airg.ddc_theta(rp, ci, v, cf1).cpu().numpy()
    F = cf1.cpu().numpy() == 1
    assert np.all(th1[F] < d["tau"]) and np.all(th1[~F] == 0)
    assert th0[d["cf_pmisr"] == 1].max() > th1[F].max()


def test_cf_split_bitexact_3d():
    p = P.kuhn_3d(10)
    op = O.Params()
    ref = O.cf_split(p.rowptr, p.col, p.val, op, level=2)["cf"]
    got = airg.cf_split(*dev(p), gpu_params(op), level=2).cpu().numpy()
    assert np.array_equal(got, ref)


def test_cf_split_bitexact_on_oracle_coarse_levels():
    p = P.streaming_2d(64)
    op = O.Params()
    H = O.Hierarchy(p.rowptr, p.col, p.val, op)
    checked = 0
    for l in range(1, H.num_levels):
        if H.level_info(l)["coarsest"]:
            break
        A = H.export(l, "A")
        ref = H.vectors(l)["cf"]
        got = airg.cf_split(*dev(A), gpu_params(op), level=l).cpu().numpy()
        assert np.array_equal(got, ref), f"level {l}"
        checked += 1
    assert checked >= 5


# ---------------------------------------------------------------------------------------------
# One level of setup on identical input
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mesh,order,sparsity,ideal", [(64, 2, 1, 0), (48, 6, 1, 0), (20, 3, 1, 0), (48, 6, 2, 0),
                                                      (40, 3, 2, 0), (48, 6, 1, 1), (40, 3, 2, 1)])
def test_level_operators_match_oracle(mesh, order, sparsity, ideal):
    p = P.p1_dg_2d(mesh, 0.3, seed=3 + mesh, sigma_uniform=(0.0, 2.0))
    op = O.Params(poly_order=order, max_levels=2, coarse_size=0, sparsity_order=sparsity, ideal_prolong=ideal)
    Ho = O.Hierarchy(p.rowptr, p.col, p.val, op)
    Hg = airg.Hierarchy(*dev(p), gpu_params(op))
    assert Hg.num_levels == Ho.num_levels == 2
    io, ig = Ho.level_info(0), Hg.level_info(0)
    for k in ("n", "nnz", "nf", "nc", "nnz_aff", "nnz_afc", "nnz_ainv", "nnz_z", "nnz_acf"):
        assert io[k] == ig[k], k
    vo, vg = Ho.vectors(0), Hg.vectors(0)
    assert np.array_equal(vo["cf"], vg["cf"])
    assert np.array_equal(vo["w"], vg["w"])
    np.testing.assert_allclose(vg["alpha"], vo["alpha"], rtol=1e-10, atol=1e-12 * np.abs(vo["alpha"]).max())
    for which in ("Aff", "Afc", "Acf"):
        a, b = Ho.export(0, which), Hg.export(0, which)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), which
    assert_csr_close(Ho.export(0, "Ainv"), Hg.export(0, "Ainv"), what="Ainv")
    assert_csr_close(Ho.export(0, "Z"), Hg.export(0, "Z"), what="Z")
    if ideal:
        assert io["nnz_w"] == ig["nnz_w"] > io["nf"]
        assert_csr_close(Ho.export(0, "W"), Hg.export(0, "W"), what="W")
    else:
        assert ig["nnz_w"] == 0
    assert_csr_close(Ho.export(1, "A"), Hg.export(1, "A"), what="A_c")
    # coarsest-level polynomial on the same coarse matrix
    np.testing.assert_allclose(Hg.vectors(1)["alpha"], Ho.vectors(1)["alpha"], rtol=1e-8)
    assert_csr_close(Ho.export(1, "Ainv"), Hg.export(1, "Ainv"), rtol=1e-8, what="coarsest Ainv")


def test_full_hierarchy_structure_matches_oracle():
    # Level 0 is bit-exact end to end.  Deeper levels depend on polynomial coefficients that the
    # GPU reduces in a different order (differences ~1e-15), which can move a strength or PMISR
    # tie on a coarse matrix; there the structure is compared loosely and the coarse-level CF
    # splittings are checked bit-exactly on identical inputs by
    # test_cf_split_bitexact_on_oracle_coarse_levels.
    p = P.streaming_2d(64)
    op = O.Params()
    Ho = O.Hierarchy(p.rowptr, p.col, p.val, op)
    Hg = airg.Hierarchy(*dev(p), gpu_params(op))
    io, ig = Ho.level_info(0), Hg.level_info(0)
    assert (io["n"], io["nf"], io["nnz_z"]) == (ig["n"], ig["nf"], ig["nnz_z"])
    assert Ho.level_info(1)["n"] == Hg.level_info(1)["n"]
    assert abs(Hg.num_levels - Ho.num_levels) <= 2
    c = Hg.level_info(-1)
    co = Ho.complexities()
    assert c["grid"] == pytest.approx(co["grid"], rel=0.02)
    assert c["operator"] == pytest.approx(co["operator"], rel=0.03)


def natural_vcycle(H, b):
    """The paper's V-cycle evaluated in numpy, in each level's natural numbering, on the operators
    the GPU setup exported: checks the solve kernels and their nested F-then-C layout exactly."""
    L = H.num_levels
    par = H.params

    def rec(l, bl):
        inf = H.level_info(l)
        n = inf["n"]
        if inf["coarsest"]:
            rp, ci, v = H.export(l, "A")
            A = sp.csr_matrix((v, ci, rp), shape=(n, n))
            rp, ci, v = H.export(l, "Ainv")
            Ai = sp.csr_matrix((v, ci, rp), shape=(n, n))
            x = Ai @ bl
            for _ in range(par.coarse_iters - 1):
                x = x + Ai @ (bl - A @ x)
            return x
        nf, nc = inf["nf"], inf["nc"]
        vec = H.vectors(l)
        F, Cn = np.nonzero(vec["cf"] == 1)[0], np.nonzero(vec["cf"] == 2)[0]
        mk = lambda w, nr, ncl: sp.csr_matrix(tuple(H.export(l, w)[::-1]), shape=(nr, ncl))
        Z, Aff, Afc, Ai = mk("Z", nc, nf), mk("Aff", nf, nf), mk("Afc", nf, nc), mk("Ainv", nf, nf)
        xC = rec(l + 1, bl[Cn] + Z @ bl[F])
        w = vec["w"]
        xF = np.where(w >= 0, xC[np.maximum(w, 0)], 0.0)
        for _ in range(par.n_smooth_up):
            xF = xF + Ai @ (bl[F] - Aff @ xF - Afc @ xC)
        x = np.zeros(n)
        x[F], x[Cn] = xF, xC
        return x

    return rec(0, b)


def test_vcycle_matches_oracle_two_levels():
    # with two levels both hierarchies are identical (level 0 bit-exact, level 1 the coarsest);
    # a 3rd-order coarsest polynomial keeps its coefficient fit well conditioned (at 12th order the
    # fit amplifies reduction-order rounding to ~1e-10)
    p = P.streaming_2d(40)
    op = O.Params(max_levels=2, coarse_poly_order=3)
    Ho = O.Hierarchy(p.rowptr, p.col, p.val, op)
    Hg = airg.Hierarchy(*dev(p), gpu_params(op))
    b = np.random.default_rng(1).standard_normal(p.n)
    xo = Ho.vcycle(b)
    xg = Hg.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-12


def test_ideal_operators_two_level_exact_on_gpu():
    """Section "Reduction multigrid", eq. prolong: with exact A_ff^-1 (unit diagonal and strength 0
    make A_ff = I, so the degree-0 polynomial is exact), no drops and a converged coarse solve,
    R A P is the Schur complement and one V-cycle solves exactly."""
    import scipy.sparse as sps
    p = P.streaming_2d(4)
    A = p.scipy()
    d = 1.0 / A.diagonal()
    As = sps.csr_matrix(sps.diags(d) @ A)
    As.sort_indices()
    b = d * p.b
    op = O.Params(strong_threshold=0.0, ddc_fraction=0.0, drop_R=0.0, drop_Ac=0.0, poly_order=0,
                  max_levels=2, coarse_size=1, coarse_poly_order=8, coarse_iters=200, n_smooth_up=1)
    H = airg.Hierarchy(*dev((As.indptr.astype(np.int32), As.indices.astype(np.int32), As.data)), gpu_params(op))
    assert H.num_levels == 2
    x = H.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    xs = np.linalg.solve(As.toarray(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-12


@pytest.mark.parametrize("mesh,gen", [(40, "2d"), (64, "2d"), (12, "3d")])
def test_deep_vcycle_applies_its_operators_exactly(mesh, gen):
    p = P.streaming_2d(mesh) if gen == "2d" else P.kuhn_3d(mesh)
    Hg = airg.Hierarchy(*dev(p), airg.Params(keep_setup=1, coarse_size=32))
    assert Hg.num_levels >= 5
    b = np.random.default_rng(2).standard_normal(p.n)
    xg = Hg.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    xr = natural_vcycle(Hg, b)
    assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-13


# ---------------------------------------------------------------------------------------------
# Solve
# ---------------------------------------------------------------------------------------------

def solve_both(p, op, outer="fgmres", rtol=1e-12, max_it=300):
    Ho = O.Hierarchy(p.rowptr, p.col, p.val, op)
    xo, io = Ho.solve(p.b, outer=outer, rtol=rtol, max_it=max_it)
    Hg = airg.Hierarchy(*dev(p), gpu_params(op, keep=0))
    b = torch.from_numpy(p.b).cuda()
    xg, ig = Hg.solve(b, outer=outer, rtol=rtol, max_it=max_it)
    return xo, io, xg.cpu().numpy(), ig, Hg


@pytest.mark.parametrize("mesh,degree", [(64, 2), (64, 6), (33, 6), (128, 6), (48, 1), (48, 3), (48, 4), (48, 5)])
def test_solution_matches_oracle(mesh, degree):
    # (64, 2) is the 24,576-DOF pure-streaming configuration with a degree-2 polynomial
    p = P.streaming_2d(mesh)
    xo, io, xg, ig, _ = solve_both(p, O.Params(poly_order=degree))
    assert ig["status"] == 0 and io["status"] == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert ig["relres"] <= 1e-12


@pytest.mark.parametrize("mesh,degree", [(48, 2), (48, 6)])
def test_second_order_sparsity_solution_matches_oracle(mesh, degree):
    p = P.streaming_2d(mesh)
    xo, io, xg, ig, _ = solve_both(p, O.Params(poly_order=degree, sparsity_order=2))
    assert ig["status"] == 0 and io["status"] == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1


def test_matrix_free_vcycle_matches_oracle_two_levels():
    # the polynomials applied matrix-free (Horner's rule on the GPU, the power series in the oracle)
    p = P.streaming_2d(40)
    op = O.Params(max_levels=2, coarse_poly_order=3, matrix_free=1)
    Ho = O.Hierarchy(p.rowptr, p.col, p.val, op)
    Hg = airg.Hierarchy(*dev(p), gpu_params(op))
    b = np.random.default_rng(1).standard_normal(p.n)
    xo = Ho.vcycle(b)
    xg = Hg.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-11
    # and it is a different operator from the assembled fixed-sparsity inverse
    Ha = airg.Hierarchy(*dev(p), gpu_params(O.Params(max_levels=2, coarse_poly_order=3)))
    xa = Ha.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.linalg.norm(xa - xo) / np.linalg.norm(xo) > 1e-6


@pytest.mark.parametrize("mesh,degree,sparsity", [(64, 2, 1), (48, 6, 1), (33, 1, 1), (48, 3, 2)])
def test_matrix_free_solution_matches_oracle(mesh, degree, sparsity):
    p = P.streaming_2d(mesh)
    xo, io, xg, ig, Hg = solve_both(p, O.Params(poly_order=degree, sparsity_order=sparsity, matrix_free=1))
    assert Hg.num_levels > 2
    assert ig["status"] == 0 and io["status"] == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1


@pytest.mark.parametrize("flag", ["matrix_free", "ideal_prolong"])
def test_variants_are_fp64_and_unbatched(flag):
    p = P.streaming_2d(16)
    with pytest.raises(airg.AirgError):
        airg.Hierarchy(*dev(p), airg.Params(precision=1, **{flag: 1}))
    H = airg.Hierarchy(*dev(p), airg.Params(**{flag: 1}))
    with pytest.raises(airg.AirgError):
        airg.Batch([H])


@pytest.mark.parametrize("mesh,degree,mf", [(64, 2, 0), (48, 6, 0), (33, 3, 1)])
def test_ideal_prolongator_solution_matches_oracle(mesh, degree, mf):
    p = P.streaming_2d(mesh)
    xo, io, xg, ig, Hg = solve_both(p, O.Params(poly_order=degree, ideal_prolong=1, matrix_free=mf))
    assert Hg.num_levels > 2 and Hg.level_info(0)["nnz_w"] > Hg.level_info(0)["nf"]
    assert ig["status"] == 0 and io["status"] == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1


def test_ideal_prolongator_interpolates_the_exact_f_values_on_gpu():
    """eq. prolong with exact A_ff^-1 (unit diagonal, strength 0: A_ff = I), no drops, a converged
    coarse solve and no smoothing: x_C is exact and x_F = W x_C = x*_F - b_F with the ideal W."""
    import scipy.sparse as sps
    p = P.streaming_2d(4)
    A = p.scipy()
    d = 1.0 / A.diagonal()
    As = sps.csr_matrix(sps.diags(d) @ A)
    As.sort_indices()
    b = d * p.b
    xs = np.linalg.solve(As.toarray(), b)
    op = O.Params(strong_threshold=0.0, ddc_fraction=0.0, drop_R=0.0, drop_Ac=0.0, poly_order=0,
                  max_levels=2, coarse_size=0, coarse_poly_order=8, coarse_iters=200, n_smooth_up=0,
                  ideal_prolong=1)
    H = airg.Hierarchy(*dev((As.indptr.astype(np.int32), As.indices.astype(np.int32), As.data)), gpu_params(op))
    assert H.num_levels == 2
    v = H.vectors(0)
    F, Cp = np.flatnonzero(v["cf"] == 1), np.flatnonzero(v["cf"] == 2)
    x = H.vcycle(torch.from_numpy(b).cuda()).cpu().numpy()
    sc = np.abs(xs).max()
    assert np.abs(x[Cp] - xs[Cp]).max() <= 1e-12 * sc
    assert np.abs(x[F] - (xs[F] - b[F])).max() <= 1e-12 * sc


def test_setup_reuse_matches_the_oracle_with_the_same_splittings():
    # another energy group set up with the template group's splittings on every level
    gs = P.groups_2d(64, ngroups=4)
    op = O.Params()
    T = airg.Hierarchy(*dev(gs[0]), gpu_params(op))
    cf = [T.vectors(l)["cf"] for l in range(T.num_levels - 1)]
    g = gs[3]
    Hr = airg.Hierarchy(*dev(g), gpu_params(op), reuse=T)
    assert Hr.num_levels == T.num_levels
    Ho = O.Hierarchy(g.rowptr, g.col, g.val, op, cf=cf)
    for l in range(Hr.num_levels - 1):
        assert np.array_equal(Hr.vectors(l)["cf"], cf[l])
    assert_csr_close(Ho.export(0, "Z"), Hr.export(0, "Z"), what="Z")
    assert_csr_close(Ho.export(1, "A"), Hr.export(1, "A"), what="A_c")
    xo, io = Ho.solve(g.b, rtol=1e-12, max_it=300)
    xg, ig = Hr.solve(torch.from_numpy(g.b).cuda(), rtol=1e-12, max_it=300)
    assert ig["status"] == 0 and io["status"] == 0
    xg = xg.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1
    # a matrix of another size is refused
    q = P.groups_2d(32, ngroups=1)[0]
    with pytest.raises(airg.AirgError):
        airg.Hierarchy(*dev(q), gpu_params(op), reuse=T)


def test_setup_reuse_with_strength_zero_is_a_fresh_setup():
    # strength 0: the level-0 splitting depends on the pattern only, so re-using it is exact
    gs = P.groups_2d(64, ngroups=3)
    par = airg.Params(strong_threshold=0.0)
    T = airg.Hierarchy(*dev(gs[0]), par)
    g = gs[2]
    b = torch.from_numpy(g.b).cuda()
    Hf = airg.Hierarchy(*dev(g), par)
    Hr = airg.Hierarchy(*dev(g), par, reuse=T, reuse_levels=1)
    xf, i_f = Hf.solve(b, rtol=1e-10)
    xr, i_r = Hr.solve(b, rtol=1e-10)
    assert i_f["status"] == 0 and i_f["iters"] == i_r["iters"]
    assert torch.equal(xf, xr)


def test_host_buffer_setup_and_solve_equal_the_device_ones():
    # airg_setup_host copies the CSR arrays in itself; with airg_solve_host a caller with host data
    # goes through the C ABI alone, and the solution is bitwise the device path's
    p = P.blocked_sigma_2d(96)
    host = [torch.from_numpy(a).pin_memory() for a in (p.rowptr, p.col, p.val)]
    Hh = airg.Hierarchy(*host, airg.Params(), host=True)
    Hd = airg.Hierarchy(*dev(p), airg.Params())
    bh = torch.from_numpy(p.b).pin_memory()
    xh = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    _, ih = Hh.solve_host(bh, xh, rtol=1e-10)
    xd, i_d = Hd.solve(torch.from_numpy(p.b).cuda(), rtol=1e-10)
    assert ih["status"] == 0 and ih["iters"] == i_d["iters"]
    assert torch.equal(xh, xd.cpu())
    with pytest.raises(TypeError):
        airg.Hierarchy(*dev(p), airg.Params(), host=True)


def test_setup_reuse_across_directions():
    # directions of one mesh that share the upwind pattern (unjittered cells, angles inside one
    # 45-degree sector): with strength 0 the re-used level-0 splitting of another direction is the
    # one a fresh setup computes, so the solve is bitwise the fresh one; with the default strength
    # the template direction's splittings on every level give the oracle's hierarchy with the same
    # forced splittings
    ds = P.directions_2d(64)
    b = torch.from_numpy(ds[3].b).cuda()
    par0 = airg.Params(strong_threshold=0.0)
    T0 = airg.Hierarchy(*dev(ds[0]), par0)
    Hf = airg.Hierarchy(*dev(ds[3]), par0)
    Hr = airg.Hierarchy(*dev(ds[3]), par0, reuse=T0, reuse_levels=1)
    xf, i_f = Hf.solve(b, rtol=1e-10)
    xr, i_r = Hr.solve(b, rtol=1e-10)
    assert i_f["status"] == 0 and i_f["iters"] == i_r["iters"]
    assert torch.equal(xf, xr)
    op = O.Params()
    T = airg.Hierarchy(*dev(ds[0]), gpu_params(op))
    cf = [T.vectors(l)["cf"] for l in range(T.num_levels - 1)]
    g = ds[2]
    Hd = airg.Hierarchy(*dev(g), gpu_params(op), reuse=T)
    Ho = O.Hierarchy(g.rowptr, g.col, g.val, op, cf=cf)
    assert_csr_close(Ho.export(0, "Z"), Hd.export(0, "Z"), what="Z")
    assert_csr_close(Ho.export(1, "A"), Hd.export(1, "A"), what="A_c")
    xo, io = Ho.solve(g.b, rtol=1e-12, max_it=300)
    xg, ig = Hd.solve(torch.from_numpy(g.b).cuda(), rtol=1e-12, max_it=300)
    assert ig["status"] == 0 and io["status"] == 0
    xg = xg.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1


def test_polynomial_order_trend():
    """Section "GMRES polynomial order" (table of orders 1-6): with first-order fixed sparsity the
    iteration count falls steeply from order 1 and flattens by order 4-6."""
    p = P.blocked_sigma_2d(256)
    b = torch.from_numpy(p.b).cuda()
    its = []
    for d in range(1, 7):
        H = airg.Hierarchy(*dev(p), airg.Params(poly_order=d))
        x, info = H.solve(b, rtol=1e-10, max_it=2000)
        assert info["status"] == 0, (d, info)
        its.append(info["iters"])
        H.close()
    assert its[0] >= 2 * its[5], its
    assert all(its[k + 1] <= its[k] + 1 for k in range(5)), its


def test_richardson_matches_oracle():
    # the paper's outer iteration.  With two levels the hierarchies are identical and so are the
    # iteration counts; on deep hierarchies coarse-level tie-breaks may differ, so only the
    # solution is compared there.
    p = P.streaming_2d(48)
    xo, io, xg, ig, _ = solve_both(p, O.Params(max_levels=2, coarse_poly_order=3, coarse_iters=4),
                                   outer="richardson", max_it=500)
    assert ig["status"] == 0 and io["status"] == 0
    assert abs(ig["iters"] - io["iters"]) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    xo, io, xg, ig, _ = solve_both(P.streaming_2d(64), O.Params(), outer="richardson")
    assert ig["status"] == 0 and io["status"] == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10


def test_solution_matches_dense_lu():
    for mesh in (8, 16):
        p = P.adjoint_2d(mesh)
        xs = O.dense_solve(p.rowptr, p.col, p.val, p.b)
        Hg = airg.Hierarchy(*dev(p), airg.Params(coarse_size=16))
        xg, ig = Hg.solve(torch.from_numpy(p.b).cuda(), rtol=1e-12)
        assert np.linalg.norm(xg.cpu().numpy() - xs) / np.linalg.norm(xs) <= 1e-10


def test_3d_p0_solution_matches_oracle():
    p = P.kuhn_3d(12)
    xo, io, xg, ig, _ = solve_both(p, O.Params())
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    assert abs(ig["iters"] - io["iters"]) <= 1


def test_solve_is_deterministic():
    p = P.blocked_sigma_2d(96)
    Hg = airg.Hierarchy(*dev(p), airg.Params())
    b = torch.from_numpy(p.b).cuda()
    x1, i1 = Hg.solve(b, rtol=1e-10)
    x2, i2 = Hg.solve(b, rtol=1e-10)
    assert i1 == i2
    assert torch.equal(x1, x2)


def test_setup_is_deterministic_run_to_run():
    """Two independent setups of one matrix give bitwise-identical hierarchies: the TSQR combine
    order, the SpGEMM accumulation order and every reduction are fixed, whatever order the warps,
    the atomics and the two streams run in."""
    p = P.blocked_sigma_2d(256)
    par = airg.Params(keep_setup=1)
    H1 = airg.Hierarchy(*dev(p), par)
    H2 = airg.Hierarchy(*dev(p), par)
    assert H1.num_levels == H2.num_levels
    for l in range(H1.num_levels):
        v1, v2 = H1.vectors(l), H2.vectors(l)
        assert np.array_equal(v1["alpha"], v2["alpha"]), l
        assert np.array_equal(v1["cf"], v2["cf"]) and np.array_equal(v1["w"], v2["w"]), l
        names = ["A", "Ainv"] if H1.level_info(l)["coarsest"] else ["A", "Ainv", "Z", "AF_solve", "Z_solve"]
        for which in names:
            for a, b in zip(H1.export(l, which), H2.export(l, which)):
                assert np.array_equal(a, b), (l, which)
    b = torch.from_numpy(p.b).cuda()
    x1, i1 = H1.solve(b, rtol=1e-10)
    x2, i2 = H2.solve(b, rtol=1e-10)
    assert i1 == i2 and torch.equal(x1, x2)


def test_expand_sort_products_equal_the_per_column_products(monkeypatch):
    # product rows of more than 1024 candidates (the coarse 3D levels) are formed by expand - sort -
    # compress in one CTA; each output keeps the ascending-l fma chain, so every level's operators
    # are bitwise those of the per-column block kernel
    p = P.kuhn_3d(48)
    par = airg.Params(keep_setup=1)
    He = airg.Hierarchy(*dev(p), par)
    monkeypatch.setenv("AIRG_SPGEMM_NO_ESC", "1")
    Hb = airg.Hierarchy(*dev(p), par)
    assert He.num_levels == Hb.num_levels
    for l in range(He.num_levels):
        names = ["A", "Ainv"] if He.level_info(l)["coarsest"] else ["A", "Ainv", "Z"]
        for which in names:
            for a, b in zip(He.export(l, which), Hb.export(l, which)):
                assert np.array_equal(a, b), (l, which)


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_sliced_ell_and_csr_agree_bitwise(monkeypatch, prec):
    # the float / bf16-value V-cycle reads the large residual operators from their sliced ELL copy
    # (values cast element by element, as for the CSR copy) and sums each row in CSR order with
    # fmaf from zero: V-cycles and solves are bitwise those of the CSR kernels
    p = P.blocked_sigma_2d(150)
    b = torch.from_numpy(p.b).cuda()
    par = airg.Params(precision=prec)
    Hs = airg.Hierarchy(*dev(p), par)
    assert Hs.level_info(0)["sell_mask"] & 1
    ys = Hs.vcycle(b)
    xs, is_ = Hs.solve(b, rtol=1e-10)
    monkeypatch.setenv("AIRG_NO_SELL", "1")
    Hc = airg.Hierarchy(*dev(p), par)
    assert Hc.level_info(0)["sell_mask"] == 0
    yc = Hc.vcycle(b)
    xc, ic = Hc.solve(b, rtol=1e-10)
    assert torch.equal(ys, yc)
    assert is_["iters"] == ic["iters"] and torch.equal(xs, xc)


@pytest.mark.parametrize("mesh,variant", [(160, {}), (160, {"matrix_free": 1}), (160, {"ideal_prolong": 1}),
                                          (150, {})])
def test_sliced_ell_and_csr_solves_agree_bitwise(monkeypatch, mesh, variant):
    # the sliced ELL SpMV keeps each row's CSR entry order and accumulates from zero with one FMA
    # per entry, as the CSR row kernel does: the solves are bitwise identical.  160^2 gives 153,600
    # rows (150 full 1024-row windows); 150^2 gives 135,000 (a ragged last window and slice)
    p = P.blocked_sigma_2d(mesh)
    b = torch.from_numpy(p.b).cuda()
    Hs = airg.Hierarchy(*dev(p), airg.Params(**variant))
    assert Hs.level_info(-1)["top_sell"] == 1
    assert Hs.level_info(0)["sell_mask"] & 1  # [A_ff A_fc]
    xs, is_ = Hs.solve(b, rtol=1e-10)
    monkeypatch.setenv("AIRG_NO_SELL", "1")
    Hc = airg.Hierarchy(*dev(p), airg.Params(**variant))
    assert Hc.level_info(-1)["top_sell"] == 0 and Hc.level_info(0)["sell_mask"] == 0
    xc, ic = Hc.solve(b, rtol=1e-10)
    assert is_["status"] == ic["status"] == 0
    assert is_["iters"] == ic["iters"]
    assert torch.equal(xs, xc)


def test_graph_and_eager_vcycles_agree_bitwise(monkeypatch):
    p = P.blocked_sigma_2d(80)
    b = torch.from_numpy(p.b).cuda()
    Hg = airg.Hierarchy(*dev(p), airg.Params())
    xg, ig = Hg.solve(b, rtol=1e-10)
    monkeypatch.setenv("AIRG_NO_GRAPH", "1")
    He = airg.Hierarchy(*dev(p), airg.Params())
    xe, ie = He.solve(b, rtol=1e-10)
    assert ig["iters"] == ie["iters"]
    assert torch.equal(xg, xe)


def test_host_buffer_solve_matches_device_solve():
    p = P.streaming_2d(32)
    Hg = airg.Hierarchy(*dev(p), airg.Params())
    b = torch.from_numpy(p.b)
    xd, _ = Hg.solve(b.cuda(), rtol=1e-10)
    xh = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    xh, info = Hg.solve_host(b.pin_memory(), xh, rtol=1e-10)
    assert torch.equal(xd.cpu(), xh)


# ---------------------------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------------------------

def test_edge_cases():
    # 1 x 1
    H = airg.Hierarchy(*dev((np.array([0, 1]), np.array([0]), np.array([4.0]))), airg.Params())
    x, info = H.solve(torch.tensor([2.0], dtype=torch.float64, device="cuda"), rtol=1e-14)
    assert x.item() == pytest.approx(0.5, rel=1e-14)
    # diagonal: every node isolated -> single level
    n = 1000
    d = np.linspace(1, 2, n)
    H = airg.Hierarchy(*dev((np.arange(n + 1), np.arange(n), d)), airg.Params(coarse_size=4))
    assert H.num_levels == 1
    x, info = H.solve(torch.ones(n, dtype=torch.float64, device="cuda"), rtol=1e-12)
    np.testing.assert_allclose(x.cpu().numpy(), 1 / d, rtol=1e-10)
    # zero rhs
    p = P.streaming_2d(16)
    H = airg.Hierarchy(*dev(p), airg.Params())
    x, info = H.solve(torch.zeros(p.n, dtype=torch.float64, device="cuda"))
    assert info["iters"] == 0 and torch.count_nonzero(x) == 0
    # max_levels = 1: the whole-matrix polynomial alone preconditions GMRES
    H = airg.Hierarchy(*dev(p), airg.Params(max_levels=1))
    assert H.num_levels == 1
    x, info = H.solve(torch.from_numpy(p.b).cuda(), rtol=1e-10, max_it=500)
    assert info["status"] == 0
    # not converged is reported, not raised
    H = airg.Hierarchy(*dev(p), airg.Params())
    x, info = H.solve(torch.from_numpy(p.b).cuda(), rtol=1e-30, max_it=3)
    assert info["status"] == 1 and info["iters"] == 3


def test_invalid_inputs_are_rejected():
    p = P.streaming_2d(8)
    col = p.col.copy()
    col[5], col[6] = col[6], col[5]  # unsorted row
    with pytest.raises(airg.AirgError) as e:
        airg.Hierarchy(*dev((p.rowptr, col, p.val)), airg.Params())
    assert e.value.code == -2
    val = p.val.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    val[np.nonzero((p.col == rows))[0][3]] = 0.0
    with pytest.raises(airg.AirgError) as e:
        airg.Hierarchy(*dev((p.rowptr, p.col, val)), airg.Params())
    assert e.value.code == -3
    with pytest.raises(airg.AirgError):
        airg.Hierarchy(*dev(p), airg.Params(poly_order=-1))


# ---------------------------------------------------------------------------------------------
# Full size (the benchmarked workload): properties the oracle can check at any size
# ---------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    return P.blocked_sigma_2d(1024)


def test_full_size_cf_split_bitexact(big):
    op = O.Params()
    ref = O.cf_split(big.rowptr, big.col, big.val, op)["cf"]
    got = airg.cf_split(*dev(big), gpu_params(op), level=0).cpu().numpy()
    assert np.array_equal(got, ref)


def test_full_size_setup_is_deterministic(big):
    b = torch.from_numpy(big.b).cuda()
    xs = []
    for _ in range(2):
        H = airg.Hierarchy(*dev(big), airg.Params())
        x, info = H.solve(b, rtol=1e-8)
        xs.append((x, info["iters"], H.num_levels))
        H.close()
    assert xs[0][1:] == xs[1][1:]
    assert torch.equal(xs[0][0], xs[1][0])


def test_full_size_solve_reaches_tolerance(big):
    H = airg.Hierarchy(*dev(big), airg.Params())
    x, info = H.solve(torch.from_numpy(big.b).cuda(), rtol=1e-8)
    assert info["status"] == 0
    xh = x.cpu().numpy()
    r = big.b - big.scipy() @ xh
    assert np.linalg.norm(r) / np.linalg.norm(big.b) <= 1e-8
    # sampled rows of the residual through the oracle's own SpMV
    rng = np.random.default_rng(0)
    rows = rng.choice(big.n, 2000, replace=False)
    sub = big.scipy()[rows]
    sub.sort_indices()
    Ax = sub @ xh
    assert np.all(np.abs(big.b[rows] - Ax) <= 1e-6 * np.abs(big.b).max())


# ---------------------------------------------------------------------------------------------
# Mixed-precision form: V-cycle operators and vectors in FP32 (or bf16 values), FP64 outer loop
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("gen", ["2d", "3d"])
@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_reaches_fp64_tolerance(gen, prec):
    p = P.blocked_sigma_2d(128) if gen == "2d" else P.kuhn_3d(32)
    b = torch.from_numpy(p.b).cuda()
    H64 = airg.Hierarchy(*dev(p), airg.Params(coarse_size=2000))
    x64, i64 = H64.solve(b, rtol=1e-10)
    Hlo = airg.Hierarchy(*dev(p), airg.Params(coarse_size=2000, precision=prec))
    xlo, ilo = Hlo.solve(b, rtol=1e-10)
    assert ilo["status"] == 0 and ilo["relres"] <= 1e-10  # true FP64 residual
    assert ilo["iters"] <= i64["iters"] + (2 if prec == 1 else 4)
    x64, xlo = x64.cpu().numpy(), xlo.cpu().numpy()
    assert np.linalg.norm(xlo - x64) / np.linalg.norm(x64) <= 1e-8
    if gen == "3d":  # the 32^3 instance against the oracle
        Ho = O.Hierarchy(p.rowptr, p.col, p.val, O.Params(coarse_size=2000))
        xo, io = Ho.solve(p.b, rtol=1e-10)
        assert np.linalg.norm(xlo - xo) / np.linalg.norm(xo) <= 1e-8


def test_mixed_precision_vcycle_is_close_to_fp64_vcycle():
    p = P.streaming_2d(64)
    b = torch.from_numpy(np.random.default_rng(3).standard_normal(p.n)).cuda()
    y64 = airg.Hierarchy(*dev(p), airg.Params(coarse_size=500)).vcycle(b)
    y32 = airg.Hierarchy(*dev(p), airg.Params(coarse_size=500, precision=1)).vcycle(b)
    ybf = airg.Hierarchy(*dev(p), airg.Params(coarse_size=500, precision=2)).vcycle(b)
    r32 = (torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64)).item()
    rbf = (torch.linalg.norm(ybf - y64) / torch.linalg.norm(y64)).item()
    assert r32 < 1e-4   # single-precision rounding through the cycle
    assert rbf < 5e-2   # bf16 values carry 8 bits of mantissa
    assert r32 < rbf

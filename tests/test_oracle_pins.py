"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test ties an oracle function to the paper's statement through an independent route: a
textbook/library routine (dense LU, dense matmul), a closed form, a theorem (greedy-MIS
equivalence, Cayley-Hamilton, exactness of ideal reduction operators), or a hand-worked fixture
under tests/golden/.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.stats

from oracle import oracle as O
from paper_2408_08262_gb300 import problems as P

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def dense(rp, ci, v, ncols=None):
    n = len(rp) - 1
    return sp.csr_matrix((v, ci, rp), shape=(n, ncols if ncols is not None else n)).toarray()


def to_csr(M):
    m = sp.csr_matrix(M)
    m.sort_indices()
    return m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64)


# ---------------------------------------------------------------------------------------------
# Plain definitions: dense LU and the generator
# ---------------------------------------------------------------------------------------------

def test_dense_lu_matches_numpy():
    rng = np.random.default_rng(1)
    for n in (1, 2, 7, 40):
        M = rng.standard_normal((n, n)) + n * np.eye(n)
        b = rng.standard_normal(n)
        x = O.dense_solve(*to_csr(M), b)
        np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-12, atol=1e-12)


def test_generator_reproduces_linear_solution():
    # Omega = (1, 0), sigma = 0, q = 1, u = 0 at x = 0: the exact solution u = x is linear, so
    # upwind P1 DG reproduces it at every node.
    p = P.p1_dg_2d(6, 0.0, seed=11)
    xy, tris = P.tri_mesh(6, np.random.default_rng(11), 0.2)
    u = O.dense_solve(p.rowptr, p.col, p.val, p.b)
    np.testing.assert_allclose(u, xy[tris].reshape(-1, 2)[:, 0], atol=1e-12)


def test_generator_matrix_structure():
    p = P.streaming_2d(8)
    A = p.scipy()
    assert p.n == 3 * 2 * 64
    assert np.all(A.diagonal() > 0)
    assert np.all(np.diff(p.rowptr) > 0)
    for i in range(p.n):
        c = p.col[p.rowptr[i]:p.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    assert np.count_nonzero(p.val == 0) == 0
    q = P.kuhn_3d(3)
    assert q.n == 6 * 27
    assert np.all(q.scipy().diagonal() > 0)


def test_energy_groups_share_the_pattern():
    # the setup re-use workload: groups of one mesh and direction differ in values only, and the
    # removal term only adds to each element's own block (the sigma-free part is the same)
    gs = P.groups_2d(8, ngroups=3)
    for g in gs[1:]:
        assert np.array_equal(g.rowptr, gs[0].rowptr) and np.array_equal(g.col, gs[0].col)
        assert not np.array_equal(g.val, gs[0].val)
    d = [g.scipy() - gs[0].scipy() for g in gs[1:]]
    elem = np.arange(gs[0].n) // 3
    for D in d:
        D = D.tocoo()
        nz = D.data != 0
        assert nz.any() and np.all(elem[D.row[nz]] == elem[D.col[nz]])


# ---------------------------------------------------------------------------------------------
# Strength of connection (eq. soc)
# ---------------------------------------------------------------------------------------------

def test_strength_hand_example():
    g = gold("strength_example.json")
    d = O.cf_split(g["rowptr"], g["col"], g["val"], O.Params(strong_threshold=g["alpha"]))
    assert d["strong"].tolist() == g["strong"]


def test_strength_zero_threshold_is_adjacency():
    p = P.streaming_2d(6)
    d = O.cf_split(p.rowptr, p.col, p.val, O.Params(strong_threshold=0.0))
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    offdiag = (p.col != rows)
    assert np.array_equal(d["strong"].astype(bool), offdiag)


# ---------------------------------------------------------------------------------------------
# PMISR (Algorithm 1)
# ---------------------------------------------------------------------------------------------

def sym_adj(rp, ci, strong):
    n = len(rp) - 1
    nb = [set() for _ in range(n)]
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            if strong[k]:
                nb[i].add(int(ci[k]))
                nb[int(ci[k])].add(i)
    return nb


def greedy_mis(nb, w):
    """Sequential greedy MIS visiting nodes in increasing (w_i, i).  With fixed priorities the
    round-based parallel selection yields exactly this set (the lexicographically-first MIS;
    Blelloch, Fineman & Shun 2012)."""
    order = sorted(range(len(w)), key=lambda i: (w[i], i))
    sel = np.zeros(len(w), dtype=bool)
    for i in order:
        if not any(sel[j] for j in nb[i]):
            sel[i] = True
    return sel


def random_graph(n, deg, rng):
    rows, cols = [], []
    for i in range(n):
        for j in rng.choice(n, size=deg, replace=False):
            if j != i:
                rows.append(i)
                cols.append(j)
        rows.append(i)
        cols.append(i)
    M = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    M.sum_duplicates()
    M.sort_indices()
    rp, ci = M.indptr.astype(np.int32), M.indices.astype(np.int32)
    rowid = np.repeat(np.arange(n), np.diff(rp))
    strong = ((ci != rowid) & (rng.random(len(ci)) < 0.7)).astype(np.int8)
    return rp, ci, strong


@pytest.mark.parametrize("seed", range(6))
def test_pmisr_uncapped_equals_greedy_mis(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 13)) if seed < 3 else 400
    rp, ci, strong = random_graph(n, 3, rng)
    nb = sym_adj(rp, ci, strong)
    deg = np.array([len(x) for x in nb])
    # weights as in Algorithm 1: |S_i| + |S_i^T| + r_i
    rowid = np.repeat(np.arange(n), np.diff(rp))
    nS = np.bincount(rowid, weights=strong, minlength=n)
    nST = np.bincount(ci, weights=strong, minlength=n)
    w = nS + nST + rng.random(n)
    cf, rounds = O.pmisr(rp, ci, strong, w, max_loops=0)
    sel = greedy_mis(nb, w)
    assert np.array_equal(cf == 1, sel)
    assert np.all((cf == 1) | (cf == 2))
    # isolated nodes are F (w < 1)
    assert np.all(cf[deg == 0] == 1)


def test_pmisr_invariants_on_mesh():
    p = P.streaming_2d(16)
    par = O.Params(pmisr_max_loops=0, ddc_fraction=0.0)
    d = O.cf_split(p.rowptr, p.col, p.val, par)
    nb = sym_adj(p.rowptr, p.col, d["strong"])
    cf = d["cf_pmisr"]
    Fs = np.nonzero(cf == 1)[0]
    for i in Fs:  # independence (H1R)
        assert all(cf[j] != 1 for j in nb[i])
    for i in np.nonzero(cf == 2)[0]:  # maximality
        assert any(cf[j] == 1 for j in nb[i])
    # capped at 3 rounds: F is the prefix of the uncapped run, still independent
    d3 = O.cf_split(p.rowptr, p.col, p.val, O.Params(pmisr_max_loops=3, ddc_fraction=0.0))
    F3 = d3["cf_pmisr"] == 1
    assert np.all(cf[F3] == 1)
    assert d3["rounds"] <= 3


# ---------------------------------------------------------------------------------------------
# DDC (Algorithm 2)
# ---------------------------------------------------------------------------------------------

def test_ddc_hand_example():
    g = gold("ddc_example.json")
    for case in g["cases"]:
        cf, th, tau = O.ddc(g["rowptr"], g["col"], g["val"], g["cf_in"], case["fraction"])
        np.testing.assert_allclose(th, g["theta"], rtol=0, atol=0)
        assert cf.tolist() == case["cf_out"]
        if case["tau"] is None:
            assert np.isinf(tau)
        else:
            assert tau == case["tau"]


def test_ddc_threshold_property():
    p = P.streaming_2d(24)
    d = O.cf_split(p.rowptr, p.col, p.val, O.Params())
    before, after, th, tau = d["cf_pmisr"], d["cf"], d["theta"], d["tau"]
    nF = int(np.sum(before == 1))
    cand = (before == 1) & (th != 0)
    k = min(int(np.floor(0.1 * nF)), int(cand.sum()))
    converted = (before == 1) & (after == 2)
    assert converted.sum() >= k
    assert np.all(th[converted] >= tau)
    remaining = (after == 1) & (th > 0)
    assert np.all(th[remaining] < tau)
    # the k-th largest candidate value is tau
    assert np.sort(th[cand])[::-1][k - 1] == tau
    # removing F-points only drops terms: theta on the post-DDC F set is not larger
    cf2, th2, _ = O.ddc(p.rowptr, p.col, p.val, after, 0.0)
    assert np.all(th2[after == 1] <= th[after == 1])


@pytest.mark.parametrize("mk", [lambda: P.streaming_2d(16), lambda: P.blocked_sigma_2d(16), lambda: P.streaming_2d(24)])
def test_ddc_diagnostics_theta_and_aff_condition(mk):
    # Section "CF splitting" reports that DDC brings the largest theta over the F-points from about
    # 1 down to about 0.6 (PMISR alone leaves rows with F-F coupling as large as the diagonal), and
    # Table cond_aff relates that to the conditioning of A_ff: both, on the top level
    p = mk()
    A = p.scipy().toarray()
    d = O.cf_split(p.rowptr, p.col, p.val, O.Params())
    th_max, kappa = [], []
    for cf in (d["cf_pmisr"], d["cf"]):
        _, th, _ = O.ddc(p.rowptr, p.col, p.val, cf, 0.0)
        F = np.flatnonzero(cf == 1)
        th_max.append(th[F].max())
        s = np.linalg.svd(A[np.ix_(F, F)], compute_uv=False)
        kappa.append(s[0] / s[-1])
    assert th_max[0] > 0.9 and th_max[1] < 0.7
    assert kappa[1] <= kappa[0] * (1 + 1e-12)


def test_zero_strength_gives_diagonal_aff_and_ddc_noop():
    # Section "Strong tolerances": strength 0.0 gives an independent set in the adjacency graph,
    # a diagonal A_ff, and DDC ignores diagonal rows.
    p = P.streaming_2d(12)
    par = O.Params(strong_threshold=0.0, max_levels=2)
    H = O.Hierarchy(p.rowptr, p.col, p.val, par)
    v = H.vectors(0)
    assert np.array_equal(v["cf"], v["cf_pmisr"])
    rp, ci, _ = H.export(0, "Aff")
    rowid = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    assert np.array_equal(ci, rowid)


# ---------------------------------------------------------------------------------------------
# GMRES polynomial (eq. gmres_poly, setup steps 3-8)
# ---------------------------------------------------------------------------------------------

def test_random_streams_are_uniform_and_normal():
    r = O.unif01(240808262, 3, 0, 200000)
    assert r.min() >= 0 and r.max() < 1
    assert scipy.stats.kstest(r, "uniform").pvalue > 1e-4
    z = O.box_muller(240808262, 0, 200000)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5 / np.sqrt(z.size)


def test_box_muller_matches_the_transform_in_double():
    """The single-precision ln/cos sequences of the Box-Muller rhs agree with libm's double
    transform of the same 24-bit draws to float accuracy (a wrong quadrant, sign or coefficient
    would be off by O(1) or O(1e-3))."""
    n = 100000
    k = O.unif24(240808262, 2, 1, 2 * n).astype(np.float64)
    u1 = 1.0 - k[0::2] * 2.0**-24
    u2 = k[1::2] * 2.0**-24
    ref = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    z = O.box_muller(240808262, 2, n)
    err = np.abs(z - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < 2e-6
    # the quadrant boundaries and the extreme draws are covered
    assert (u2 < 1e-4).any() and (np.abs(u2 - 0.25) < 1e-4).any() and (np.abs(u2 - 0.75) < 1e-4).any()


def test_poly_degree0_closed_form():
    rng = np.random.default_rng(3)
    M = sp.random(30, 30, density=0.2, random_state=4) + 3 * sp.eye(30)
    rp, ci, v = to_csr(M.toarray())
    b = rng.standard_normal(30)
    alpha, mf = O.poly_fit(rp, ci, v, 1, b)
    Ab = M @ b
    assert mf == 1
    assert alpha[0] == pytest.approx(b @ Ab / (Ab @ Ab), rel=1e-13)


def test_poly_degree1_normal_equations():
    rng = np.random.default_rng(5)
    M = sp.random(25, 25, density=0.3, random_state=6) + 2 * sp.eye(25)
    rp, ci, v = to_csr(M.toarray())
    b = rng.standard_normal(25)
    alpha, _ = O.poly_fit(rp, ci, v, 2, b)
    K = np.stack([M @ b, M @ (M @ b)], 1)
    ref = np.linalg.lstsq(K, b, rcond=None)[0]
    np.testing.assert_allclose(alpha, ref, rtol=1e-10)


@pytest.mark.parametrize("m", [3, 5, 7])
def test_poly_minimises_the_residual_like_lstsq(m):
    # eq. gmres_poly: the coefficients minimise ||b - A q(A) b|| over polynomials q of degree m-1,
    # a least-squares problem on [A b, ..., A^m b] that numpy solves by SVD (not by the oracle's
    # Householder TSQR and Givens solve)
    rng = np.random.default_rng(40 + m)
    n = 60
    M = sp.random(n, n, density=0.1, random_state=50 + m) * 0.5 + sp.diags(1.0 + rng.random(n))
    rp, ci, v = to_csr(M.toarray())
    b = rng.standard_normal(n)
    alpha, mf = O.poly_fit(rp, ci, v, m, b)
    assert mf == m
    K = np.empty((n, m))
    w = b.copy()
    for k in range(m):
        w = M @ w
        K[:, k] = w
    ref = np.linalg.lstsq(K, b, rcond=None)[0]
    res, res_ref = np.linalg.norm(b - K @ alpha), np.linalg.norm(b - K @ ref)
    assert res <= res_ref * (1 + 1e-10) + 1e-14
    assert res < 0.9 * np.linalg.norm(b)
    np.testing.assert_allclose(alpha, ref, rtol=1e-6, atol=1e-8 * np.abs(ref).max())


@pytest.mark.parametrize("n", [2, 3, 5, 6])
def test_poly_degree_n_minus_1_is_exact_inverse(n):
    # Cayley-Hamilton: for a dense n x n matrix (fixed sparsity = full pattern, closed under
    # powers) the degree n-1 GMRES polynomial annihilates the residual and q(A) = A^-1.
    rng = np.random.default_rng(10 + n)
    M = rng.standard_normal((n, n)) * 0.3 + np.diag(1.0 + np.arange(n))
    rp, ci, v = to_csr(M)
    alpha, mf = O.poly_fit(rp, ci, v, n, seed=99, level=0)
    r2, c2, v2 = O.fixed_sparsity_inverse(rp, ci, v, alpha)
    Ainv = dense(r2, c2, v2)
    np.testing.assert_allclose(Ainv @ M, np.eye(n), atol=1e-9)


def test_poly_block_diagonal_identical_blocks_exact():
    n, nb = 4, 5
    rng = np.random.default_rng(7)
    B = rng.standard_normal((n, n)) * 0.4 + np.diag([1.0, 2.0, 3.0, 4.5])
    M = np.kron(np.eye(nb), B)
    rp, ci, v = to_csr(M)
    alpha, mf = O.poly_fit(rp, ci, v, n, seed=5, level=1)
    r2, c2, v2 = O.fixed_sparsity_inverse(rp, ci, v, alpha)
    np.testing.assert_allclose(dense(r2, c2, v2) @ M, np.eye(n * nb), atol=1e-9)


def test_poly_breakdown_truncates():
    # identity: the Krylov space has dimension 1, alpha = (1, 0, 0, ...)
    n = 10
    rp, ci, v = to_csr(np.eye(n))
    alpha, mf = O.poly_fit(rp, ci, v, 5, seed=1)
    assert mf == 1
    np.testing.assert_allclose(alpha, [1, 0, 0, 0, 0], atol=1e-15)


def test_fixed_sparsity_hand_example():
    g = gold("fixed_sparsity_tridiag.json")
    r, c, v = O.fixed_sparsity_inverse(g["rowptr"], g["col"], g["val"], g["alpha"])
    assert r.tolist() == g["rowptr"] and c.tolist() == g["col"]
    np.testing.assert_allclose(v, g["ainv"], rtol=0, atol=1e-15)
    # the individual powers through unit coefficient vectors
    r, c, v = O.fixed_sparsity_inverse(g["rowptr"], g["col"], g["val"], [0, 0, 1.0])
    assert v.tolist() == g["power2"]
    r, c, v = O.fixed_sparsity_inverse(g["rowptr"], g["col"], g["val"], [0, 0, 0, 1.0])
    assert v.tolist() == g["power3"]


def test_fixed_sparsity_closed_pattern_equals_true_powers():
    rng = np.random.default_rng(8)
    B = rng.standard_normal((3, 3))
    M = np.kron(np.eye(6), B)
    alpha = rng.standard_normal(5)
    r, c, v = O.fixed_sparsity_inverse(*to_csr(M), alpha)
    ref = sum(a * np.linalg.matrix_power(M, k) for k, a in enumerate(alpha))
    np.testing.assert_allclose(dense(r, c, v), ref, rtol=1e-12, atol=1e-12)


def test_second_order_sparsity_is_exact_for_degree_two_on_a_tridiagonal_matrix():
    # Section "AIRG": second-order fixed sparsity enforces the pattern of A_ff^2.  For a tridiagonal
    # A that pattern is pentadiagonal and holds A^2 exactly, so the degree-2 polynomial is exact,
    # while first order (tridiagonal) truncates A^2.
    n = 14
    rng = np.random.default_rng(12)
    M = np.diag(4 + rng.random(n)) + np.diag(rng.standard_normal(n - 1), -1) + np.diag(rng.standard_normal(n - 1), 1)
    alpha = np.array([0.7, -0.2, 0.05])
    ref = alpha[0] * np.eye(n) + alpha[1] * M + alpha[2] * M @ M
    r, c, v = O.fixed_sparsity_inverse(*to_csr(M), alpha, order=2)
    assert np.diff(r).max() == 5  # pentadiagonal
    np.testing.assert_allclose(dense(r, c, v), ref, rtol=1e-14, atol=1e-14)
    r1, c1, v1 = O.fixed_sparsity_inverse(*to_csr(M), alpha, order=1)
    assert np.abs(dense(r1, c1, v1) - ref).max() > 1e-3


def test_second_order_sparsity_matches_a_dense_masked_recursion():
    # tilde(A^k) = mask(tilde(A^{k-1}) A) with mask = pattern(A^2), computed densely
    A = sp.random(30, 30, density=0.08, random_state=21, format="csr") + 3 * sp.eye(30)
    A = sp.csr_matrix(A)
    A.sort_indices()
    D = A.toarray()
    mask = (np.abs((A != 0).astype(float) @ (A != 0).astype(float)).toarray() > 0)
    alpha = np.array([0.5, -0.3, 0.2, -0.1, 0.05])
    P = D * mask
    ref = alpha[0] * np.eye(30) + alpha[1] * P
    for k in range(2, len(alpha)):
        P = (P @ D) * mask
        ref = ref + alpha[k] * P
    r, c, v = O.fixed_sparsity_inverse(A.indptr, A.indices, A.data, alpha, order=2)
    got = dense(r, c, v)
    assert np.array_equal(got != 0, (ref != 0) | (got != 0))  # pattern contains every nonzero
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------------------------------------
# Products, coarse matrix, operators
# ---------------------------------------------------------------------------------------------

def test_spgemm_matches_dense_product():
    for seed in range(3):
        A = sp.random(40, 30, density=0.15, random_state=seed, format="csr")
        B = sp.random(30, 35, density=0.15, random_state=seed + 10, format="csr")
        A.sort_indices()
        B.sort_indices()
        r, c, v = O.spgemm((A.indptr, A.indices, A.data), (B.indptr, B.indices, B.data), 35, scale=-1.0)
        np.testing.assert_allclose(dense(r, c, v, 35), -(A @ B).toarray(), rtol=1e-13, atol=1e-15)


def test_spgemm_drop_hand_example():
    # rows: [1, 0.5, 0.01] -> tol 0.05 drops 0.01; row 1 diagonal 0.001 kept with keep_diag.
    A = (np.array([0, 1, 2], dtype=np.int32), np.array([0, 1], dtype=np.int32), np.array([1.0, 1.0]))
    B = (np.array([0, 3, 6], dtype=np.int32), np.array([0, 1, 2, 0, 1, 2], dtype=np.int32),
         np.array([1.0, 0.5, 0.01, 5.0, 0.001, -4.0]))
    r, c, v = O.spgemm(A, B, 3, tol=0.05, keep_diag=True)
    assert r.tolist() == [0, 2, 5]
    assert c.tolist() == [0, 1, 0, 1, 2]
    assert v.tolist() == [1.0, 0.5, 5.0, 0.001, -4.0]
    r, c, v = O.spgemm(A, B, 3, tol=0.05, keep_diag=False)
    assert c.tolist() == [0, 1, 0, 2]


def test_coarse_matrix_is_RAP():
    p = P.streaming_2d(10)
    par = O.Params(drop_Ac=0.0, max_levels=3)
    H = O.Hierarchy(p.rowptr, p.col, p.val, par)
    info = H.level_info(0)
    v = H.vectors(0)
    n, nf, nc = info["n"], info["nf"], info["nc"]
    A = p.scipy().toarray()
    F = np.nonzero(v["cf"] == 1)[0]
    Cn = np.nonzero(v["cf"] == 2)[0]
    Z = dense(*H.export(0, "Z"), nf)
    R = np.zeros((nc, n))
    R[:, F] = Z
    R[np.arange(nc), Cn] = 1.0
    Pm = np.zeros((n, nc))
    Pm[Cn, np.arange(nc)] = 1.0
    has = v["w"] >= 0
    Pm[F[has], v["w"][has]] = 1.0
    Ac = dense(*H.export(1, "A"))
    np.testing.assert_allclose(Ac, R @ A @ Pm, rtol=1e-12, atol=1e-14)
    # Z = -A_cf Ainv (drop 0.01 relative row-wise): kept entries equal the product
    Acf = A[np.ix_(Cn, F)]
    Ainv = dense(*H.export(0, "Ainv"))
    Zfull = -Acf @ Ainv
    kept = Z != 0
    np.testing.assert_allclose(Z[kept], Zfull[kept], rtol=1e-12)
    rowmax = np.abs(Zfull).max(axis=1, keepdims=True)
    dropped = np.abs(Zfull) * (~kept)
    assert np.all((dropped < 0.01 * rowmax) | (dropped == 0))


def test_one_point_prolongation_hand_worked_fixture():
    # Setup step 10 (classical one-point operator, Section "Results"): the choice of every F-row of
    # a hand-worked 10-point example with a given splitting, covering a tie (smaller index, by
    # magnitude), the fallback to weak C entries, a transpose-only strong dependency (not used),
    # a stored zero (never chosen) and a strong F neighbour larger than every C entry.
    g = gold("one_point_example.json")
    rp, ci, v = (np.array(g[k], dtype=t) for k, t in (("rowptr", np.int32), ("col", np.int32), ("val", np.float64)))
    cf = np.array(g["cf"], dtype=np.int8)
    F = np.flatnonzero(cf == 1)
    Cn = np.flatnonzero(cf == 2)
    # the strength flags the choice is made from
    st = O.cf_split(rp, ci, v, O.Params(strong_threshold=g["alpha"]))["strong"]
    for f, i in enumerate(F):
        assert st[rp[i]:rp[i + 1]].tolist() == g["strong_F_rows"][f], i
    par = O.Params(strong_threshold=g["alpha"], max_levels=2, coarse_size=1, poly_order=2, coarse_poly_order=3)
    H = O.Hierarchy(rp, ci, v, par, cf=[cf])
    vec = H.vectors(0)
    assert np.array_equal(vec["cf"], cf)
    expect = [-1 if j < 0 else int(np.flatnonzero(Cn == j)[0]) for j in g["w_natural"]]
    assert vec["w"].tolist() == expect


def test_one_point_prolongation_picks_strongest_C():
    p = P.streaming_2d(8)
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params(max_levels=2))
    v = H.vectors(0)
    d = O.cf_split(p.rowptr, p.col, p.val, O.Params())
    assert np.array_equal(d["cf"], v["cf"])
    F = np.nonzero(v["cf"] == 1)[0]
    Cn = np.nonzero(v["cf"] == 2)[0]
    cpos = {int(c): k for k, c in enumerate(Cn)}
    for f, i in enumerate(F):
        lo, hi = p.rowptr[i], p.rowptr[i + 1]
        cols, vals, st = p.col[lo:hi], p.val[lo:hi], d["strong"][lo:hi]
        cand = [(abs(a), -int(j)) for j, a, s in zip(cols, vals, st) if s and v["cf"][j] == 2]
        if not cand:
            cand = [(abs(a), -int(j)) for j, a in zip(cols, vals) if j != i and v["cf"][j] == 2 and a != 0]
        if not cand:
            assert v["w"][f] == -1
            continue
        best = -max(cand)[1]
        assert v["w"][f] == cpos[best]


# ---------------------------------------------------------------------------------------------
# Solve phase
# ---------------------------------------------------------------------------------------------

def test_ideal_operators_two_level_exact():
    # Section "Reduction multigrid", eq. prolong: with exact A_ff^-1, no drops and an exact coarse
    # solve, R A P is the Schur complement and one V-cycle solves exactly for any W.
    # Unit diagonal + strength 0 makes A_ff = I, so the degree-0 polynomial is exact.
    p = P.streaming_2d(4)
    A = p.scipy()
    d = 1.0 / A.diagonal()
    As = sp.diags(d) @ A
    As = sp.csr_matrix(As)
    As.sort_indices()
    b = d * p.b
    par = O.Params(strong_threshold=0.0, ddc_fraction=0.0, drop_R=0.0, drop_Ac=0.0, poly_order=0,
                   max_levels=2, coarse_size=0, coarse_poly_order=8, coarse_iters=200, n_smooth_up=1)
    H = O.Hierarchy(As.indptr, As.indices, As.data, par)
    assert H.num_levels == 2
    x = H.vcycle(b)
    xs = np.linalg.solve(As.toarray(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-12


def _dense_poly(M, alpha):
    Q = np.zeros_like(M)
    Pk = np.eye(M.shape[0])
    for a in alpha:
        Q = Q + a * Pk
        Pk = Pk @ M
    return Q


@pytest.mark.parametrize("iters", [1, 2])
def test_matrix_free_coarse_solve_is_the_matrix_polynomial(iters):
    # Section "AIRG": the stationary polynomial q(A) = sum_k alpha_k A^k applied without assembling
    # it.  A single-level hierarchy is its coarse solve: one iteration gives q(A) b, two give
    # q b + q (b - A q b), with q built here from dense matrix powers.
    p = P.streaming_2d(6)
    A = p.scipy().toarray()
    par = O.Params(max_levels=1, coarse_poly_order=5, coarse_iters=iters, matrix_free=1)
    H = O.Hierarchy(p.rowptr, p.col, p.val, par)
    alpha = H.vectors(0)["alpha"]
    assert alpha.size == 6 and np.all(alpha[:2] != 0)
    Q = _dense_poly(A, alpha)
    b = np.random.default_rng(3).standard_normal(p.n)
    x = Q @ b
    if iters == 2:
        x = x + Q @ (b - A @ x)
    got = H.vcycle(b)
    np.testing.assert_allclose(got, x, rtol=1e-11, atol=1e-12 * np.abs(x).max())
    # the assembled first-order fixed-sparsity inverse truncates the powers: a different operator
    Ha = O.Hierarchy(p.rowptr, p.col, p.val, O.Params(max_levels=1, coarse_poly_order=5, coarse_iters=iters))
    assert np.abs(Ha.vcycle(b) - x).max() > 1e-6 * np.abs(x).max()


@pytest.mark.parametrize("matrix_free,ideal", [(0, 0), (1, 0), (0, 1)])
def test_two_level_vcycle_matches_a_dense_restatement(matrix_free, ideal):
    # Section "Results" V-cycle on two levels, rebuilt densely from the exported operators:
    # b_c = b_C + Z b_F; coarse iterations x += M_c (b_c - A_c x); prolongation x_F = W x_C (one-point
    # or approximate ideal W); then n_smooth_up smooths x_F += M_f (b_F - A_ff x_F - A_fc x_C), with
    # M the assembled inverse or, matrix-free, the dense polynomial in A_ff (A_c on the coarse
    # level).  With no drop on A_c, the coarse matrix is the dense triple product R A P.
    p = P.streaming_2d(8)
    par = O.Params(max_levels=2, coarse_size=0, poly_order=3, coarse_poly_order=4, coarse_iters=2,
                   drop_Ac=0.0, matrix_free=matrix_free, ideal_prolong=ideal)
    H = O.Hierarchy(p.rowptr, p.col, p.val, par)
    assert H.num_levels == 2
    i0, i1 = H.level_info(0), H.level_info(1)
    v0, v1 = H.vectors(0), H.vectors(1)
    F, Cp = np.flatnonzero(v0["cf"] == 1), np.flatnonzero(v0["cf"] == 2)
    nf, nc = i0["nf"], i0["nc"]
    Aff = dense(*H.export(0, "Aff"), nf)
    Afc = dense(*H.export(0, "Afc"), nc)
    Z = dense(*H.export(0, "Z"), nf)
    Ac = dense(*H.export(1, "A"), nc)
    w = v0["w"]
    if ideal:
        W = dense(*H.export(0, "W"), nc)
        assert i0["nnz_w"] > nf  # more than one entry per F row on average
    else:
        W = np.zeros((nf, nc))
        W[np.flatnonzero(w >= 0), w[w >= 0]] = 1.0
    Pm = np.zeros((p.n, nc))
    Pm[F], Pm[Cp] = W, np.eye(nc)
    Rm = np.zeros((nc, p.n))
    Rm[:, F], Rm[:, Cp] = Z, np.eye(nc)
    np.testing.assert_allclose(Ac, Rm @ p.scipy().toarray() @ Pm, rtol=0, atol=1e-13 * np.abs(Ac).max())
    if matrix_free:
        Mf, Mc = _dense_poly(Aff, v0["alpha"]), _dense_poly(Ac, v1["alpha"])
    else:
        Mf, Mc = dense(*H.export(0, "Ainv"), nf), dense(*H.export(1, "Ainv"), nc)
    b = np.random.default_rng(5).standard_normal(p.n)
    bF, bC = b[F], b[Cp]
    bc = bC + Z @ bF
    xc = np.zeros(nc)
    for _ in range(par.coarse_iters):
        xc = xc + Mc @ (bc - Ac @ xc)
    xF = W @ xc
    for _ in range(par.n_smooth_up):
        xF = xF + Mf @ (bF - Aff @ xF - Afc @ xc)
    x = np.zeros(p.n)
    x[F], x[Cp] = xF, xc
    got = H.vcycle(b)
    np.testing.assert_allclose(got, x, rtol=1e-10, atol=1e-11 * np.abs(x).max())


def test_ideal_prolongator_is_minus_ainv_afc_with_the_restrictor_drop():
    # eq. prolong: W = -A_ff^-1 A_fc with the assembled Ainv, the counterpart of Z = -A_cf Ainv,
    # sparsified with the same relative row-wise inf-norm drop (entries below drop_R x row max go)
    p = P.streaming_2d(12)
    par = O.Params(max_levels=2, coarse_size=0, ideal_prolong=1)
    H = O.Hierarchy(p.rowptr, p.col, p.val, par)
    i0 = H.level_info(0)
    nf, nc = i0["nf"], i0["nc"]
    ref = -dense(*H.export(0, "Ainv"), nf) @ dense(*H.export(0, "Afc"), nc)
    thr = par.drop_R * np.abs(ref).max(axis=1, keepdims=True)
    near = np.abs(np.abs(ref) - thr) <= 1e-9 * thr
    assert not near[ref != 0].any()  # no entry within rounding of the threshold
    ref = np.where(np.abs(ref) >= thr, ref, 0.0)
    got = dense(*H.export(0, "W"), nc)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * np.abs(ref).max())
    assert (ref != 0).sum() < (np.abs(-dense(*H.export(0, "Ainv"), nf) @ dense(*H.export(0, "Afc"), nc)) > 0).sum()


def test_ideal_prolongator_interpolates_the_exact_f_values():
    # eq. prolong with an exact A_ff^-1 (unit diagonal and strength 0 make A_ff = I, so degree 0 is
    # exact), no drops and a converged coarse solve: the coarse correction is exact on the C-points
    # for any P, and with no smoothing the ideal W gives x_F = W x_C = x*_F - A_ff^-1 b_F, where the
    # one-point operator does not.
    p = P.streaming_2d(4)
    A = p.scipy()
    d = 1.0 / A.diagonal()
    As = sp.csr_matrix(sp.diags(d) @ A)
    As.sort_indices()
    b = d * p.b
    xs = np.linalg.solve(As.toarray(), b)
    out = {}
    for ideal in (0, 1):
        par = O.Params(strong_threshold=0.0, ddc_fraction=0.0, drop_R=0.0, drop_Ac=0.0, poly_order=0,
                       max_levels=2, coarse_size=0, coarse_poly_order=8, coarse_iters=200, n_smooth_up=0,
                       ideal_prolong=ideal)
        H = O.Hierarchy(As.indptr, As.indices, As.data, par)
        v = H.vectors(0)
        F, Cp = np.flatnonzero(v["cf"] == 1), np.flatnonzero(v["cf"] == 2)
        x = H.vcycle(b)
        np.testing.assert_allclose(x[Cp], xs[Cp], rtol=1e-12, atol=1e-12 * np.abs(xs).max())
        out[ideal] = np.abs(x[F] - (xs[F] - b[F])).max() / np.abs(xs).max()
    assert out[1] < 1e-12
    assert out[0] > 1e-3


def test_ideal_prolongator_solution_matches_dense_lu():
    p = P.streaming_2d(16)
    xs = O.dense_solve(p.rowptr, p.col, p.val, p.b)
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params(coarse_size=16, ideal_prolong=1))
    assert H.num_levels > 2
    x, info = H.solve(p.b, rtol=1e-12, max_it=300)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-10


def test_strength_zero_splitting_depends_on_the_pattern_only():
    # Sections "Strong tolerances" and "Conclusions": with strength threshold 0 every connection is
    # strong, PMISR picks an independent set of the matrix graph and A_ff is diagonal, so DDC
    # (theta = 0 everywhere) converts nothing: the splitting is a function of the pattern alone and
    # is the same for every energy group of a mesh and direction
    gs = P.groups_2d(24, ngroups=3)
    par = O.Params(strong_threshold=0.0)
    cfs = [O.cf_split(g.rowptr, g.col, g.val, par) for g in gs]
    for d in cfs:
        assert np.array_equal(d["cf"], cfs[0]["cf"])
        assert np.array_equal(d["cf"], d["cf_pmisr"])
    # with the default strength 0.5 the splittings of the groups differ
    c5 = [O.cf_split(g.rowptr, g.col, g.val, O.Params())["cf"] for g in gs]
    assert not np.array_equal(c5[0], c5[2])


def test_forced_splittings_reproduce_the_computed_hierarchy():
    # the setup with every level's splitting given is the setup that computed them
    p = P.groups_2d(24, ngroups=1)[0]
    par = O.Params(coarse_size=32)
    H = O.Hierarchy(p.rowptr, p.col, p.val, par)
    L = H.num_levels
    assert L > 3
    cf = [H.vectors(l)["cf"] for l in range(L - 1)]
    Hf = O.Hierarchy(p.rowptr, p.col, p.val, par, cf=cf)
    assert Hf.num_levels == L
    for l in range(L):
        for which in ("A", "Ainv") + (("Z", "Aff") if l < L - 1 else ()):
            for x, y in zip(H.export(l, which), Hf.export(l, which)):
                assert np.array_equal(x, y), (l, which)
    b = np.random.default_rng(0).standard_normal(p.n)
    assert np.array_equal(H.vcycle(b), Hf.vcycle(b))
    with pytest.raises(ValueError):
        O.Hierarchy(p.rowptr, p.col, p.val, par, cf=[cf[0][:-1]])


def test_reused_splittings_give_a_convergent_solver():
    # another group's splittings on every level: a valid splitting (diagonals kept), so AIRG still
    # solves to the dense LU solution
    gs = P.groups_2d(16, ngroups=4)
    par = O.Params(coarse_size=16)
    T = O.Hierarchy(gs[0].rowptr, gs[0].col, gs[0].val, par)
    cf = [T.vectors(l)["cf"] for l in range(T.num_levels - 1)]
    g = gs[3]
    H = O.Hierarchy(g.rowptr, g.col, g.val, par, cf=cf)
    assert H.num_levels == T.num_levels
    xs = O.dense_solve(g.rowptr, g.col, g.val, g.b)
    x, info = H.solve(g.b, rtol=1e-12, max_it=300)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-10


def test_directions_of_one_sector_share_the_pattern_and_the_strength_zero_splitting():
    # directions across a mesh (Sections "Strong tolerances" and "Conclusions": the splitting at
    # strength 0 does not depend on the angle): on the unjittered mesh every edge is horizontal,
    # vertical or diagonal, so directions inside (0, pi/4) see the same inflow edges.  The patterns
    # coincide (a direction in another sector has another pattern), the values differ, the strength-0
    # splittings are identical, and another direction's splittings on every level still solve to the
    # dense LU solution
    ds = P.directions_2d(12, thetas=(0.1, 0.4, 0.7))
    for d in ds[1:]:
        assert np.array_equal(d.rowptr, ds[0].rowptr) and np.array_equal(d.col, ds[0].col)
        assert not np.array_equal(d.val, ds[0].val)
    other = P.p1_dg_2d(12, 1.2, sigma=1.0, q=1.0, seed=ds[0].meta["seed"], jitter=0.0)
    assert not (np.array_equal(other.rowptr, ds[0].rowptr) and np.array_equal(other.col, ds[0].col))
    par0 = O.Params(strong_threshold=0.0)
    cfs = [O.cf_split(d.rowptr, d.col, d.val, par0)["cf"] for d in ds]
    assert all(np.array_equal(c, cfs[0]) for c in cfs)
    par = O.Params(coarse_size=16)
    T = O.Hierarchy(ds[0].rowptr, ds[0].col, ds[0].val, par)
    cf = [T.vectors(l)["cf"] for l in range(T.num_levels - 1)]
    g = ds[2]
    H = O.Hierarchy(g.rowptr, g.col, g.val, par, cf=cf)
    xs = O.dense_solve(g.rowptr, g.col, g.val, g.b)
    x, info = H.solve(g.b, rtol=1e-12, max_it=300)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-10


def test_matrix_free_airg_solution_matches_dense_lu():
    p = P.streaming_2d(16)
    xs = O.dense_solve(p.rowptr, p.col, p.val, p.b)
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params(coarse_size=16, matrix_free=1))
    assert H.num_levels > 2
    x, info = H.solve(p.b, rtol=1e-12, max_it=300)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-10


def test_vcycle_is_linear():
    p = P.streaming_2d(8)
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params())
    rng = np.random.default_rng(0)
    b1, b2 = rng.standard_normal(p.n), rng.standard_normal(p.n)
    lhs = H.vcycle(2.5 * b1 + b2)
    rhs = 2.5 * H.vcycle(b1) + H.vcycle(b2)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-11, atol=1e-12 * np.abs(rhs).max())


def test_unpreconditioned_gmres_finite_termination():
    rng = np.random.default_rng(4)
    n = 12
    M = rng.standard_normal((n, n)) + 4 * np.eye(n)
    rp, ci, v = to_csr(M)
    H = O.Hierarchy(rp, ci, v, O.Params(max_levels=1))
    b = rng.standard_normal(n)
    x, info = H.solve(b, outer="gmres", restart=n, max_it=n, rtol=1e-12)
    assert info["iters"] <= n
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-9)


@pytest.mark.parametrize("mesh,outer", [(8, "fgmres"), (16, "fgmres"), (16, "richardson")])
def test_airg_solution_matches_dense_lu(mesh, outer):
    p = P.streaming_2d(mesh)
    xs = O.dense_solve(p.rowptr, p.col, p.val, p.b)
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params(coarse_size=16))
    assert H.num_levels > 2
    x, info = H.solve(p.b, outer=outer, rtol=1e-12, max_it=300)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-10


def test_adjoint_size_problem_matches_dense_lu():
    p = P.adjoint_2d(16)
    xs = O.dense_solve(p.rowptr, p.col, p.val, p.b)
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params(coarse_size=16))
    x, info = H.solve(p.b, rtol=1e-12)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-10


def test_zero_rhs_and_degenerate_sizes():
    p = P.streaming_2d(4)
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params())
    x, info = H.solve(np.zeros(p.n))
    assert info["iters"] == 0 and np.all(x == 0)
    # 1 x 1 system
    H1 = O.Hierarchy(np.array([0, 1]), np.array([0]), np.array([4.0]), O.Params())
    x, info = H1.solve(np.array([2.0]), rtol=1e-14)
    assert x[0] == pytest.approx(0.5, rel=1e-14)
    # diagonal matrix: every node isolated -> all F, hierarchy is a single level
    n = 50
    Hd = O.Hierarchy(np.arange(n + 1), np.arange(n), np.linspace(1, 2, n), O.Params(coarse_size=4))
    assert Hd.num_levels == 1
    x, info = Hd.solve(np.ones(n), rtol=1e-12)
    np.testing.assert_allclose(x, 1 / np.linspace(1, 2, n), rtol=1e-10)


def test_oracle_spmv_threads_give_bitwise_the_same_solve():
    # the all-cores CPU baseline runs the oracle's SpMV row loop on several threads: rows are
    # independent and keep their summation order, so hierarchy and solution must not change a bit
    p = P.blocked_sigma_2d(48)
    out = []
    for t in (1, 3):
        prev = O.set_threads(t)
        try:
            H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params())
            x, info = H.solve(p.b, rtol=1e-10)
            out.append((x, info["iters"], H.export(1, "A")))
        finally:
            O.set_threads(prev)
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    for a, b in zip(out[0][2], out[1][2]):
        assert np.array_equal(a, b)

"""Seeded synthetic transport systems (the inputs both the CUDA path and the oracle consume).

This module only *generates inputs*: jittered meshes and an upwind discontinuous Galerkin
discretisation of the steady transport equation  Omega . grad(u) + sigma u = q  with u = 0 on
the inflow boundary.  It holds none of the reduction-multigrid arithmetic (strength, splitting,
polynomials, products, cycles, Krylov): those live in the CUDA library and, independently, in
the oracle.

The paper (Section "Discretisation", eq. bte) solves the streaming limit of the Boltzmann
transport equation on unstructured triangles with a sub-grid-scale CG/DG scheme whose Schur
complement is a non-symmetric, non-normal advection operator.  That FEM infrastructure is not
available, so two stand-ins with the same character are generated here:

* 2D: n x n unit-square cells, each split into two triangles along a diagonal chosen by a seeded
  coin; interior vertices jittered uniformly by +-0.2h per coordinate; linear DG (P1, three DOFs
  per triangle) with full upwinding.  Element integrals (|K| area, |e| edge length):
      int_K (Omega.grad phi_j) phi_i = (Omega.grad phi_j) |K| / 3
      int_K sigma phi_i phi_j        = sigma |K| (1 + delta_ij) / 12
      int_e phi_i phi_j              = |e| (1 + delta_ij) / 6      (i, j the two edge nodes)
  and on every inflow edge (Omega.n_e < 0) the term |Omega.n_e| int_e (u_K - u_up) v, with
  u_up = 0 on the domain boundary.  Source q is integrated as q |K| / 3.
* 3D: n^3 cubes, six Kuhn tetrahedra each, vertices jittered by +-0.15h; piecewise-constant DG
  (P0, one DOF per tet): diagonal sigma|K| + sum over inflow faces |Omega.n||f|, and
  -|Omega.n||f| to the upwind neighbour across each interior inflow face.

All matrices are CSR with int32 indices, sorted unique columns, a stored (positive) diagonal and
no stored zeros.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

BASE_SEED = 240808262


def _mix64(z: int) -> int:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) used only to derive numpy seeds."""
    m = (1 << 64) - 1
    z &= m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def derive_seed(config_index: int, stream: int, base: int = BASE_SEED) -> int:
    """Independent numpy seed for (config, stream); stream 0 = mesh, 1 = coefficients, 2 = extra."""
    return _mix64(base + 0x9E3779B97F4A7C15 * (1 + 16 * config_index + stream)) >> 1


@dataclass
class Problem:
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]
    b: np.ndarray  # float64 [n]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _to_csr(rows, cols, vals, n) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    m = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    m.sum_duplicates()
    m.eliminate_zeros()
    m.sort_indices()
    rowptr = m.indptr.astype(np.int32)
    col = m.indices.astype(np.int32)
    val = m.data.astype(np.float64)
    return rowptr, col, val


# ----------------------------------------------------------------------------------------------
# 2D jittered triangle mesh, P1 upwind DG
# ----------------------------------------------------------------------------------------------

def tri_mesh(n: int, rng: np.random.Generator, jitter: float = 0.2):
    """Vertices (n+1)^2 on [0,1]^2 (row-major, x fastest) and 2 n^2 CCW triangles."""
    h = 1.0 / n
    iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    xy = np.stack([ix.ravel() * h, iy.ravel() * h], axis=1)
    interior = ((ix > 0) & (ix < n) & (iy > 0) & (iy < n)).ravel()
    d = rng.uniform(-jitter * h, jitter * h, size=(interior.sum(), 2))
    xy[interior] += d
    cy, cx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cx = cx.ravel()
    cy = cy.ravel()
    v00 = cy * (n + 1) + cx
    v10 = v00 + 1
    v01 = v00 + (n + 1)
    v11 = v01 + 1
    flip = rng.integers(0, 2, size=cx.size).astype(bool)
    # diagonal v00-v11 (flip False) or v10-v01 (flip True); both triangles counter-clockwise
    t0 = np.where(flip[:, None], np.stack([v00, v10, v01], 1), np.stack([v00, v10, v11], 1))
    t1 = np.where(flip[:, None], np.stack([v10, v11, v01], 1), np.stack([v00, v11, v01], 1))
    tris = np.empty((2 * cx.size, 3), dtype=np.int64)
    tris[0::2] = t0
    tris[1::2] = t1
    return xy, tris


def _tri_neighbours(tris: np.ndarray):
    """For local edge k (opposite vertex k) of every triangle: neighbour triangle and its edge."""
    nt = tris.shape[0]
    a = tris[:, [1, 2, 0]]  # edge k = (v[k+1], v[k+2])
    bb = tris[:, [2, 0, 1]]
    lo = np.minimum(a, bb).ravel()
    hi = np.maximum(a, bb).ravel()
    key = lo * (tris.max() + 1) + hi
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = ks[1:] == ks[:-1]
    nb = np.full(3 * nt, -1, dtype=np.int64)
    i0 = order[:-1][same]
    i1 = order[1:][same]
    nb[i0] = i1
    nb[i1] = i0
    nb = nb.reshape(nt, 3)
    nbt = np.where(nb >= 0, nb // 3, -1)
    nbe = np.where(nb >= 0, nb % 3, -1)
    return nbt, nbe


def assemble_p1_dg(xy, tris, omega, sigma_e, q_e=1.0):
    """Upwind P1 DG operator and load vector on a CCW triangle mesh."""
    nt = tris.shape[0]
    p = xy[tris]  # [nt,3,2]
    x, y = p[..., 0], p[..., 1]
    area = 0.5 * ((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    if not np.all(area > 0):
        raise ValueError("non-positive triangle area after jitter")
    # grad of barycentric phi_k = (y_{k+1} - y_{k+2}, x_{k+2} - x_{k+1}) / (2|K|)
    k1 = [1, 2, 0]
    k2 = [2, 0, 1]
    gx = (y[:, k1] - y[:, k2]) / (2 * area[:, None])
    gy = (x[:, k2] - x[:, k1]) / (2 * area[:, None])
    og = omega[0] * gx + omega[1] * gy  # [nt,3]  Omega.grad phi_j
    sigma_e = np.broadcast_to(np.asarray(sigma_e, dtype=np.float64), (nt,))
    q_e = np.broadcast_to(np.asarray(q_e, dtype=np.float64), (nt,))
    dof = 3 * np.arange(nt)[:, None] + np.arange(3)[None, :]
    rows, cols, vals = [], [], []
    # element block: advection + mass
    I, J = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    blk = og[:, None, :] * (area[:, None, None] / 3.0)
    blk = blk + sigma_e[:, None, None] * area[:, None, None] * (1.0 + (I == J)) / 12.0
    rows.append(np.repeat(dof[:, :, None], 3, axis=2).ravel())
    cols.append(np.repeat(dof[:, None, :], 3, axis=1).ravel())
    vals.append(blk.ravel())
    # inflow edges
    nbt, nbe = _tri_neighbours(tris)
    for k in range(3):
        a, c = k1[k], k2[k]  # local node indices on edge k (tail a -> head c, CCW)
        ex = x[:, c] - x[:, a]
        ey = y[:, c] - y[:, a]
        elen = np.hypot(ex, ey)
        # outward normal of a CCW edge: tangent rotated clockwise
        on = (omega[0] * ey - omega[1] * ex) / elen  # Omega . n_e
        inflow = on < 0
        w = np.abs(on) * elen / 6.0  # |Omega.n| |e| / 6
        t = np.nonzero(inflow)[0]
        wt = w[t]
        for (li, lj, f) in ((a, a, 2.0), (a, c, 1.0), (c, a, 1.0), (c, c, 2.0)):
            rows.append(dof[t, li])
            cols.append(dof[t, lj])
            vals.append(f * wt)
        # coupling to the upwind neighbour's trace (same physical vertices)
        tt = t[nbt[t, k] >= 0]
        if tt.size:
            nt2 = nbt[tt, k]
            wt2 = w[tt]
            va = tris[tt, a]
            vc = tris[tt, c]
            tri2 = tris[nt2]
            la = np.argmax(tri2 == va[:, None], axis=1)
            lc = np.argmax(tri2 == vc[:, None], axis=1)
            d2a = 3 * nt2 + la
            d2c = 3 * nt2 + lc
            for (li, dj, f) in ((a, d2a, 2.0), (a, d2c, 1.0), (c, d2a, 1.0), (c, d2c, 2.0)):
                rows.append(dof[tt, li])
                cols.append(dj)
                vals.append(-f * wt2)
    n = 3 * nt
    rowptr, col, val = _to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
    b = np.repeat(q_e * area / 3.0, 3)
    return rowptr, col, val, b, area


def csr_positions(rowptr: np.ndarray, col: np.ndarray, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Positions of the entries (rows[k], cols[k]) in a CSR with sorted columns (all must exist)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    lo = rowptr[rows].astype(np.int64)
    hi = rowptr[rows + 1].astype(np.int64)
    # vectorised binary search inside each row
    while True:
        active = lo < hi
        if not active.any():
            break
        mid = (lo + hi) // 2
        c = col[np.minimum(mid, len(col) - 1)]
        go_right = active & (c < cols)
        lo = np.where(go_right, mid + 1, lo)
        hi = np.where(active & ~go_right, mid, hi)
    if not np.all(col[lo] == cols):
        raise ValueError("entry not in pattern")
    return lo


def sigma_q_maps(p: Problem):
    """Element maps of a P1 DG problem for the adjoint form: the matrix values are
    val = val0 + sum_e sigma_e * (mass coefficient at 9 positions of element e), and the load is
    b = sum_e q_e * |K_e| / 3 on the element's 3 DOFs.  Returns (val0, mass_pos [ne,9], mass_coef
    [ne,9], area [ne])."""
    m = p.meta
    if m.get("kind") != "p1dg2d":
        raise ValueError("P1 DG problems only")
    area, sig = m["area"], m["sigma_e"]
    ne = area.size
    I, J = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    rows = (3 * np.arange(ne)[:, None] + I.ravel()[None, :])
    cols = (3 * np.arange(ne)[:, None] + J.ravel()[None, :])
    pos = csr_positions(p.rowptr, p.col, rows.ravel(), cols.ravel()).reshape(ne, 9)
    coef = area[:, None] * (1.0 + (I == J).ravel()[None, :]) / 12.0
    val0 = p.val.copy()
    np.subtract.at(val0, pos.ravel(), (sig[:, None] * coef).ravel())
    return val0, pos, coef, area


def p1_dg_2d(n: int, theta: float, sigma=0.0, q=1.0, seed: int = BASE_SEED, jitter: float = 0.2,
             sigma_blocks: tuple | None = None, sigma_uniform: tuple | None = None) -> Problem:
    """2D upwind P1 DG system on an n x n jittered triangle mesh (3 * 2 n^2 DOFs).

    sigma: scalar removal coefficient, or
    sigma_blocks=(nb, values): piecewise constant on an nb x nb block pattern with each block's
        value drawn by seed from `values`, or
    sigma_uniform=(lo, hi): per-element uniform draw.
    """
    rng = np.random.default_rng(seed)
    xy, tris = tri_mesh(n, rng, jitter)
    nt = tris.shape[0]
    srng = np.random.default_rng(_mix64(seed + 1) >> 1)
    if sigma_blocks is not None:
        nb, values = sigma_blocks
        bv = srng.choice(np.asarray(values, dtype=np.float64), size=(nb, nb))
        cell = np.arange(nt) // 2
        cx = cell % n
        cy = cell // n
        sig = bv[(cy * nb) // n, (cx * nb) // n]
    elif sigma_uniform is not None:
        sig = srng.uniform(sigma_uniform[0], sigma_uniform[1], size=nt)
    else:
        sig = np.full(nt, float(sigma))
    omega = np.array([math.cos(theta), math.sin(theta)])
    rowptr, col, val, b, area = assemble_p1_dg(xy, tris, omega, sig, q)
    meta = dict(kind="p1dg2d", mesh_n=n, theta=theta, seed=seed, jitter=jitter, n_tri=nt, area=area,
                sigma_e=np.asarray(sig, dtype=np.float64))
    return Problem(3 * nt, rowptr, col, val, b, meta)


# ----------------------------------------------------------------------------------------------
# 3D Kuhn tetrahedra, P0 upwind DG
# ----------------------------------------------------------------------------------------------

_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def kuhn_mesh(n: int, rng: np.random.Generator, jitter: float = 0.15):
    h = 1.0 / n
    iz, iy, ix = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    xyz = np.stack([ix.ravel() * h, iy.ravel() * h, iz.ravel() * h], axis=1)
    interior = ((ix > 0) & (ix < n) & (iy > 0) & (iy < n) & (iz > 0) & (iz < n)).ravel()
    xyz[interior] += rng.uniform(-jitter * h, jitter * h, size=(interior.sum(), 3))
    cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], 1)
    N1 = n + 1

    def vid(c):
        return (c[:, 2] * N1 + c[:, 1]) * N1 + c[:, 0]

    tets = np.empty((base.shape[0], 6, 4), dtype=np.int64)
    eye = np.eye(3, dtype=np.int64)
    for t, perm in enumerate(_KUHN):
        c0 = base
        c1 = c0 + eye[perm[0]]
        c2 = c1 + eye[perm[1]]
        c3 = c2 + eye[perm[2]]
        tets[:, t] = np.stack([vid(c0), vid(c1), vid(c2), vid(c3)], 1)
    return xyz, tets.reshape(-1, 4)


def assemble_p0_dg_3d(xyz, tets, omega, sigma_e):
    nt = tets.shape[0]
    p = xyz[tets]  # [nt,4,3]
    vol = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0]) / 6.0
    # orient positively
    neg = vol < 0
    if np.any(neg):
        tets = tets.copy()
        tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
        p = xyz[tets]
        vol = np.abs(vol)
    if not np.all(vol > 0):
        raise ValueError("non-positive tet volume after jitter")
    sigma_e = np.broadcast_to(np.asarray(sigma_e, dtype=np.float64), (nt,))
    faces = [(1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)]  # face k opposite vertex k, outward
    keys = []
    for k, f in enumerate(faces):
        s = np.sort(tets[:, list(f)], axis=1)
        keys.append((s[:, 0] * (xyz.shape[0]) + s[:, 1]) * (xyz.shape[0]) + s[:, 2])
    key = np.stack(keys, 1).ravel()
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = ks[1:] == ks[:-1]
    nb = np.full(4 * nt, -1, dtype=np.int64)
    nb[order[:-1][same]] = order[1:][same]
    nb[order[1:][same]] = order[:-1][same]
    nb = nb.reshape(nt, 4)
    diag = sigma_e * vol
    rows, cols, vals = [], [], []
    for k, f in enumerate(faces):
        a, b_, c = p[:, f[0]], p[:, f[1]], p[:, f[2]]
        nvec = 0.5 * np.cross(b_ - a, c - a)  # area-weighted normal
        # make it outward: points away from the opposite vertex
        sgn = np.sign(np.einsum("ij,ij->i", nvec, a - p[:, k]))
        nvec = nvec * sgn[:, None]
        flux = nvec @ omega  # Omega . n |f|
        inflow = flux < 0
        diag = diag + np.where(inflow, -flux, 0.0)
        t = np.nonzero(inflow & (nb[:, k] >= 0))[0]
        rows.append(t)
        cols.append(nb[t, k] // 4)
        vals.append(flux[t])  # = -|Omega.n||f|
    rows.append(np.arange(nt))
    cols.append(np.arange(nt))
    vals.append(diag)
    rowptr, col, val = _to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), nt)
    return rowptr, col, val, vol


def p0_dg_3d(n: int, omega=(0.48, 0.60, 0.64), sigma_pair=(0.0, 0.01), seed: int = BASE_SEED,
             jitter: float = 0.15, q=1.0) -> Problem:
    """3D upwind P0 DG system on n^3 cubes x 6 jittered Kuhn tets; sigma split by a seeded plane."""
    rng = np.random.default_rng(seed)
    xyz, tets = kuhn_mesh(n, rng, jitter)
    om = np.asarray(omega, dtype=np.float64)
    om = om / np.linalg.norm(om)
    srng = np.random.default_rng(_mix64(seed + 1) >> 1)
    nrm = srng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    cen = xyz[tets].mean(axis=1)
    side = (cen - 0.5) @ nrm > 0
    sig = np.where(side, sigma_pair[1], sigma_pair[0])
    rowptr, col, val, vol = assemble_p0_dg_3d(xyz, tets, om, sig)
    b = q * vol
    meta = dict(kind="p0dg3d", mesh_n=n, omega=tuple(om), seed=seed, jitter=jitter)
    return Problem(tets.shape[0], rowptr, col, val, b.astype(np.float64), meta)


# ----------------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------------

def streaming_2d(mesh_n: int = 64, theta: float = 0.3, config_index: int = 0) -> Problem:
    """Pure streaming (sigma = 0, q = 1) P1 DG on a jittered mesh; 64 x 64 gives 24,576 DOFs."""
    return p1_dg_2d(mesh_n, theta, sigma=0.0, q=1.0, seed=derive_seed(config_index, 0))


def blocked_sigma_2d(mesh_n: int = 1024, theta: float = 0.3, config_index: int = 1) -> Problem:
    """sigma piecewise constant on a seeded 8 x 8 block pattern with values in {0, 1, 10}, q = 1;
    1024 x 1024 gives 6,291,456 DOFs."""
    return p1_dg_2d(mesh_n, theta, q=1.0, seed=derive_seed(config_index, 0),
                    sigma_blocks=(8, (0.0, 1.0, 10.0)))


def kuhn_3d(mesh_n: int = 128, config_index: int = 2) -> Problem:
    """P0 DG on jittered Kuhn tets, Omega = (0.48, 0.60, 0.64), sigma in {0, 0.01} by half-space."""
    return p0_dg_3d(mesh_n, seed=derive_seed(config_index, 0))


def batched_2d(nsys: int = 64, sizes=(64, 128, 256, 512), config_index: int = 3) -> list[Problem]:
    """Independent systems: mesh size drawn from `sizes`, theta ~ U[0, 2 pi), sigma ~ U[0, 5]."""
    rng = np.random.default_rng(derive_seed(config_index, 1))
    out = []
    for s in range(nsys):
        m = int(rng.choice(np.asarray(sizes)))
        th = float(rng.uniform(0.0, 2 * math.pi))
        sg = float(rng.uniform(0.0, 5.0))
        out.append(p1_dg_2d(m, th, sigma=sg, q=1.0, seed=derive_seed(config_index, 2 + s)))
    return out


def adjoint_2d(mesh_n: int = 256, theta: float = 1.1, config_index: int = 4) -> Problem:
    """Per-element sigma ~ U[0, 2], theta = 1.1; 256 x 256 gives 393,216 DOFs."""
    return p1_dg_2d(mesh_n, theta, q=1.0, seed=derive_seed(config_index, 0), sigma_uniform=(0.0, 2.0))


def groups_2d(mesh_n: int = 512, ngroups: int = 4, theta: float = 0.3, config_index: int = 5) -> list[Problem]:
    """Energy groups of one mesh and direction: the blocked sigma pattern of blocked_sigma_2d with
    its values {0, 1, 10} scaled by 0.1 * 4^g for group g; every group has the same sparsity
    pattern (the setup re-use workload)."""
    seed = derive_seed(config_index, 0)
    return [p1_dg_2d(mesh_n, theta, q=1.0, seed=seed, sigma_blocks=(8, tuple(v * 0.1 * 4.0 ** g for v in (0.0, 1.0, 10.0))))
            for g in range(ngroups)]


def directions_2d(mesh_n: int = 512, thetas=(0.15, 0.35, 0.55, 0.75), config_index: int = 6) -> list[Problem]:
    """Directions of one mesh whose upwind couplings coincide: the square cells are not jittered, so
    every edge is horizontal, vertical or on a +-45 degree diagonal, and any two directions strictly
    inside one 45-degree sector (here (0, pi/4)) see the same inflow edges; the matrices share their
    sparsity pattern and differ in values.  sigma = 1, q = 1 (the setup re-use workload across
    directions)."""
    seed = derive_seed(config_index, 0)
    for th in thetas:
        if not 0.0 < th < math.pi / 4:
            raise ValueError("directions must lie strictly inside (0, pi/4)")
    return [p1_dg_2d(mesh_n, float(th), sigma=1.0, q=1.0, seed=seed, jitter=0.0) for th in thetas]


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)

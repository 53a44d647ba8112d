"""ctypes wrapper of the AIRG oracle (liboracle.so).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the CPU-baseline
leg of bench.py.  The CUDA library and its Python binding never import this module.

The oracle is a plain single-thread FP64 C++ restatement of the paper's method; see the header
of airg_oracle.cpp for the passages each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "airg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
I8P = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain g++, -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _lib.oracle_setup.restype = C.c_int
        _lib.oracle_setup_forced.restype = C.c_int
        _lib.oracle_num_levels.restype = C.c_int
        _lib.oracle_free.restype = None
        _lib.oracle_set_threads.restype = C.c_int
        _lib.oracle_set_threads.argtypes = [C.c_int]
    return _lib


@dataclass
class Params:
    """AIRG parameters; defaults follow the paper's parallel settings (Section "Parallel
    results"): strength 0.5, 3 PMISR loops, 10 % DDC, drops 0.01 (R) / 0.001 (A_c), 6th-order
    polynomials with first-order fixed sparsity (Section "GMRES polynomial order"), 2 up smooths,
    coarse solve 3 iterations of a 12th-order polynomial."""
    strong_threshold: float = 0.5
    ddc_fraction: float = 0.1
    drop_R: float = 0.01
    drop_Ac: float = 0.001
    pmisr_max_loops: int = 3
    poly_order: int = 6
    coarse_poly_order: int = 12
    coarse_iters: int = 3
    coarse_size: int = 64
    max_levels: int = 64
    n_smooth_up: int = 2
    one_point_weighted: int = 0
    seed: int = 240808262
    sparsity_order: int = 1
    matrix_free: int = 0
    ideal_prolong: int = 0

    def arrays(self):
        dp = np.array([self.strong_threshold, self.ddc_fraction, self.drop_R, self.drop_Ac], dtype=np.float64)
        ip = np.array([self.pmisr_max_loops, self.poly_order, self.coarse_poly_order, self.coarse_iters,
                       self.coarse_size, self.max_levels, self.n_smooth_up, self.one_point_weighted,
                       self.seed & 0x7FFFFFFFFFFFFFFF, self.sparsity_order, self.matrix_free, self.ideal_prolong], dtype=np.int64)
        return dp, ip


def _csr(rowptr, col, val):
    return (np.ascontiguousarray(rowptr, dtype=np.int32), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


class Hierarchy:
    def __init__(self, rowptr, col, val, params: Params | None = None, cf=None):
        """cf: optional list of CF splittings (int8 arrays, 1 = F, 2 = C) taken as given for the
        first len(cf) levels (setup re-use)."""
        self.params = params or Params()
        rp, ci, v = _csr(rowptr, col, val)
        self.n = len(rp) - 1
        dp, ip = self.params.arrays()
        h = C.c_void_p()
        if cf:
            arrs = [np.ascontiguousarray(c, dtype=np.int8) for c in cf]
            ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
            lens = np.array([a.size for a in arrs], dtype=np.int32)
            rc = lib().oracle_setup_forced(C.c_int(self.n), rp.ctypes.data_as(C.c_void_p),
                                           ci.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p),
                                           dp.ctypes.data_as(C.c_void_p), ip.ctypes.data_as(C.c_void_p),
                                           C.c_int(len(arrs)), ptrs, lens.ctypes.data_as(C.c_void_p), C.byref(h))
        else:
            rc = lib().oracle_setup(C.c_int(self.n), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                                    v.ctypes.data_as(C.c_void_p), dp.ctypes.data_as(C.c_void_p),
                                    ip.ctypes.data_as(C.c_void_p), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle_setup failed ({rc})")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_free(self._h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return lib().oracle_num_levels(self._h)

    def level_info(self, l: int) -> dict:
        info = np.zeros(13, dtype=np.int64)
        tau = C.c_double()
        rc = lib().oracle_level_info(self._h, C.c_int(l), info.ctypes.data_as(C.c_void_p), C.byref(tau))
        if rc:
            raise IndexError(l)
        keys = ["n", "nnz", "nf", "nc", "nnz_aff", "nnz_afc", "nnz_ainv", "nnz_z", "coarsest", "rounds",
                "alpha_fitted", "nnz_acf", "nnz_w"]
        d = {k: int(x) for k, x in zip(keys, info)}
        d["tau"] = tau.value
        return d

    def export(self, l: int, which: str):
        """CSR export of a level operator: A, Aff, Afc, Acf, Acc, Ainv, Z, W (ideal prolongator)."""
        code = {"A": 0, "Aff": 1, "Afc": 2, "Acf": 3, "Acc": 4, "Ainv": 5, "Z": 6, "W": 7}[which]
        info = self.level_info(l)
        rows = {"A": info["n"], "Aff": info["nf"], "Afc": info["nf"], "Acf": info["nc"], "Acc": info["nc"],
                "Ainv": info["nf"] if not info["coarsest"] else info["n"], "Z": info["nc"],
                "W": info["nf"] if info["nnz_w"] or self.params.ideal_prolong else 0}[which]
        nnz = {"A": info["nnz"], "Aff": info["nnz_aff"], "Afc": info["nnz_afc"], "Acf": info["nnz_acf"],
               "Ainv": info["nnz_ainv"], "Z": info["nnz_z"], "W": info["nnz_w"], "Acc": None}[which]
        if nnz is None:
            rp = np.zeros(rows + 1, dtype=np.int32)
            lib().oracle_export_csr(self._h, C.c_int(l), C.c_int(code), rp.ctypes.data_as(C.c_void_p), None, None)
            nnz = int(rp[-1])
        rp = np.zeros(rows + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        v = np.zeros(nnz, dtype=np.float64)
        lib().oracle_export_csr(self._h, C.c_int(l), C.c_int(code), rp.ctypes.data_as(C.c_void_p),
                                ci.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p))
        return rp, ci, v

    def vectors(self, l: int):
        info = self.level_info(l)
        n, nf = info["n"], info["nf"]
        m = (self.params.coarse_poly_order if info["coarsest"] else self.params.poly_order) + 1
        cf = np.zeros(0 if info["coarsest"] else n, dtype=np.int8)
        cfp = np.zeros_like(cf)
        w = np.zeros(nf, dtype=np.int32)
        alpha = np.zeros(m, dtype=np.float64)
        lib().oracle_export_vectors(self._h, C.c_int(l), cf.ctypes.data_as(C.c_void_p),
                                    cfp.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p),
                                    alpha.ctypes.data_as(C.c_void_p))
        return dict(cf=cf, cf_pmisr=cfp, w=w, alpha=alpha)

    def solve(self, b, x0=None, outer: str = "fgmres", restart: int = 30, max_it: int = 200, rtol: float = 1e-10):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        it = C.c_int()
        rr = C.c_double()
        hist = np.zeros(max_it + 2 + max_it // max(restart, 1) + 2, dtype=np.float64)
        code = {"fgmres": 0, "richardson": 1, "gmres": 2}[outer]
        st = lib().oracle_solve(self._h, b.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p), C.c_int(code),
                                C.c_int(restart), C.c_int(max_it), C.c_double(rtol), C.byref(it), C.byref(rr),
                                hist.ctypes.data_as(C.c_void_p), C.c_int(hist.size))
        return x, dict(iters=it.value, relres=rr.value, status=st)

    def vcycle(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        lib().oracle_vcycle(self._h, b.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p))
        return x

    def complexities(self) -> dict:
        out = np.zeros(3)
        lib().oracle_complexities(self._h, out.ctypes.data_as(C.c_void_p))
        return dict(grid=out[0], operator=out[1], storage=out[2])


def set_threads(t: int) -> int:
    """Threads of the oracle's SpMV row loop (1 by default); returns the previous count.  Results are
    bitwise the same for any count: rows are independent and keep their summation order."""
    return int(lib().oracle_set_threads(int(t)))


def cf_split(rowptr, col, val, params: Params | None = None, level: int = 0) -> dict:
    p = params or Params()
    rp, ci, v = _csr(rowptr, col, val)
    n = len(rp) - 1
    dp, ip = p.arrays()
    strong = np.zeros(len(ci), dtype=np.int8)
    w = np.zeros(n)
    cfp = np.zeros(n, dtype=np.int8)
    th = np.zeros(n)
    cf = np.zeros(n, dtype=np.int8)
    tau = C.c_double()
    rounds = C.c_int()
    rc = lib().oracle_cf_split(C.c_int(n), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                               v.ctypes.data_as(C.c_void_p), dp.ctypes.data_as(C.c_void_p),
                               ip.ctypes.data_as(C.c_void_p), C.c_int(level), strong.ctypes.data_as(C.c_void_p),
                               w.ctypes.data_as(C.c_void_p), cfp.ctypes.data_as(C.c_void_p),
                               th.ctypes.data_as(C.c_void_p), cf.ctypes.data_as(C.c_void_p), C.byref(tau),
                               C.byref(rounds))
    if rc:
        raise ValueError("oracle_cf_split: invalid CSR")
    return dict(strong=strong, w=w, cf_pmisr=cfp, theta=th, cf=cf, tau=tau.value, rounds=rounds.value)


def pmisr(rowptr, col, strong, w, max_loops: int = 0):
    rp, ci, _ = _csr(rowptr, col, np.zeros(len(col)))
    n = len(rp) - 1
    s = np.ascontiguousarray(strong, dtype=np.int8)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    cf = np.zeros(n, dtype=np.int8)
    rounds = C.c_int()
    lib().oracle_pmisr(C.c_int(n), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                       s.ctypes.data_as(C.c_void_p), ww.ctypes.data_as(C.c_void_p), C.c_int(max_loops),
                       cf.ctypes.data_as(C.c_void_p), C.byref(rounds))
    return cf, rounds.value


def ddc(rowptr, col, val, cf_in, fraction: float = 0.1):
    rp, ci, v = _csr(rowptr, col, val)
    n = len(rp) - 1
    cin = np.ascontiguousarray(cf_in, dtype=np.int8)
    cout = np.zeros(n, dtype=np.int8)
    th = np.zeros(n)
    tau = C.c_double()
    lib().oracle_ddc(C.c_int(n), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                     v.ctypes.data_as(C.c_void_p), cin.ctypes.data_as(C.c_void_p), C.c_double(fraction),
                     cout.ctypes.data_as(C.c_void_p), th.ctypes.data_as(C.c_void_p), C.byref(tau))
    return cout, th, tau.value


def poly_fit(rowptr, col, val, m: int, b=None, seed: int = 240808262, level: int = 0):
    rp, ci, v = _csr(rowptr, col, val)
    n = len(rp) - 1
    alpha = np.zeros(m)
    bp = None
    if b is not None:
        bb = np.ascontiguousarray(b, dtype=np.float64)
        bp = bb.ctypes.data_as(C.c_void_p)
    mf = lib().oracle_poly_fit(C.c_int(n), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                               v.ctypes.data_as(C.c_void_p), C.c_int(m), bp, C.c_ulonglong(seed), C.c_int(level),
                               alpha.ctypes.data_as(C.c_void_p))
    return alpha, mf


def box_muller(seed: int, level: int, n: int):
    z = np.zeros(n)
    lib().oracle_box_muller(C.c_ulonglong(seed), C.c_int(level), C.c_int(n), z.ctypes.data_as(C.c_void_p))
    return z


def unif24(seed: int, level: int, stream: int, n: int):
    """Top 24 bits of the first n outputs of a SplitMix64 stream (the Box-Muller draws)."""
    r = np.zeros(n, dtype=np.uint32)
    lib().oracle_unif24(C.c_ulonglong(seed), C.c_int(level), C.c_int(stream), C.c_int(n), r.ctypes.data_as(C.c_void_p))
    return r


def unif01(seed: int, level: int, stream: int, n: int):
    r = np.zeros(n)
    lib().oracle_unif01(C.c_ulonglong(seed), C.c_int(level), C.c_int(stream), C.c_int(n), r.ctypes.data_as(C.c_void_p))
    return r


def fixed_sparsity_inverse(rowptr, col, val, alpha, order: int = 1):
    rp, ci, v = _csr(rowptr, col, val)
    n = len(rp) - 1
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    orp = np.zeros(n + 1, dtype=np.int32)
    args = (C.c_int(n), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p), v.ctypes.data_as(C.c_void_p),
            C.c_int(len(al)), al.ctypes.data_as(C.c_void_p), C.c_int(order))
    lib().oracle_fixed_sparsity_inverse(*args, orp.ctypes.data_as(C.c_void_p), None, None)
    nz = int(orp[-1])
    oci = np.zeros(nz, dtype=np.int32)
    ov = np.zeros(nz)
    lib().oracle_fixed_sparsity_inverse(*args, orp.ctypes.data_as(C.c_void_p), oci.ctypes.data_as(C.c_void_p),
                                        ov.ctypes.data_as(C.c_void_p))
    return orp, oci, ov


def spgemm(A, B, ncols_b: int, scale=1.0, tol=0.0, keep_diag=False):
    """A, B: (rowptr, col, val) tuples.  A is (len(A.rowptr)-1) x (len(B.rowptr)-1)."""
    arp, aci, av = _csr(*A)
    brp, bci, bv = _csr(*B)
    ar, ac = len(arp) - 1, len(brp) - 1
    args = [C.c_int(ar), C.c_int(ac), arp.ctypes.data_as(C.c_void_p), aci.ctypes.data_as(C.c_void_p),
            av.ctypes.data_as(C.c_void_p), C.c_int(ncols_b), brp.ctypes.data_as(C.c_void_p),
            bci.ctypes.data_as(C.c_void_p), bv.ctypes.data_as(C.c_void_p), C.c_double(scale), C.c_double(tol),
            C.c_int(int(keep_diag))]
    orp = np.zeros(ar + 1, dtype=np.int32)
    lib().oracle_spgemm(*args, orp.ctypes.data_as(C.c_void_p), None, None)
    nz = int(orp[-1])
    oci = np.zeros(nz, dtype=np.int32)
    ov = np.zeros(nz)
    lib().oracle_spgemm(*args, orp.ctypes.data_as(C.c_void_p), oci.ctypes.data_as(C.c_void_p),
                        ov.ctypes.data_as(C.c_void_p))
    return orp, oci, ov


def spmv(rowptr, col, val, x):
    rp, ci, v = _csr(rowptr, col, val)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(len(rp) - 1)
    lib().oracle_spmv(C.c_int(len(rp) - 1), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                      v.ctypes.data_as(C.c_void_p), xx.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p))
    return y


def dense_solve(rowptr, col, val, b):
    rp, ci, v = _csr(rowptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(len(rp) - 1)
    rc = lib().oracle_dense_solve(C.c_int(len(rp) - 1), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                                  v.ctypes.data_as(C.c_void_p), bb.ctypes.data_as(C.c_void_p),
                                  x.ctypes.data_as(C.c_void_p))
    if rc:
        raise np.linalg.LinAlgError("singular")
    return x

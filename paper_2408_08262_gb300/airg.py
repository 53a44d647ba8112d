"""Thin Python binding of libairg.so (the C ABI in include/airg.h).

Argument marshalling only: every step of setup and solve runs in the library's CUDA kernels.
PyTorch provides device memory and the current stream.  There is no CPU fallback: if the
compiled library is missing, importing the functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libairg.so")
_lib = None

AIRG_OK, AIRG_NOT_CONVERGED = 0, 1
STATUS = {0: "ok", 1: "not converged", -1: "invalid argument", -2: "invalid CSR", -3: "zero diagonal",
          -4: "NaN", -5: "out of memory", -6: "CUDA error", -7: "unsupported",
          -8: "input larger than the no-allocation scratch array"}
PROFILE_CLASSES = ["smooth_resid", "smooth_update", "restrict", "top_op", "coarsest", "prolong", "gram_schmidt",
                   "vcycle"]


class AirgError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("strong_threshold", C.c_double), ("ddc_fraction", C.c_double), ("pmisr_max_loops", C.c_int),
                ("poly_order", C.c_int), ("coarse_poly_order", C.c_int), ("coarse_iters", C.c_int),
                ("coarse_size", C.c_int), ("max_levels", C.c_int), ("drop_R", C.c_double), ("drop_Ac", C.c_double),
                ("n_smooth_up", C.c_int), ("precision", C.c_int), ("keep_setup", C.c_int), ("seed", C.c_uint64),
                ("sparsity_order", C.c_int), ("matrix_free", C.c_int),
                ("ideal_prolong", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("outer", C.c_int), ("restart", C.c_int), ("max_it", C.c_int), ("rtol", C.c_double),
                ("x0_zero", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres", C.c_double), ("status", C.c_int), ("levels", C.c_int)]


def lib():
    """Loads libairg.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libairg.so not built ({LIB_PATH}); run paper_2408_08262_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.airg_setup.argtypes = [C.POINTER(_Csr), C.POINTER(_Params), C.c_void_p, C.POINTER(C.c_void_p)]
        L.airg_setup_host.argtypes = [C.POINTER(_Csr), C.POINTER(_Params), C.c_void_p, C.POINTER(C.c_void_p)]
        L.airg_setup_many.argtypes = [C.POINTER(_Csr), C.c_int, C.POINTER(_Params), C.c_int, C.c_void_p,
                                      C.POINTER(C.c_void_p)]
        L.airg_setup_reuse.argtypes = [C.POINTER(_Csr), C.POINTER(_Params), C.c_void_p, C.c_int, C.c_void_p,
                                       C.POINTER(C.c_void_p)]
        L.airg_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Opts), C.POINTER(_Info), C.c_void_p]
        L.airg_solve_host.argtypes = L.airg_solve.argtypes
        L.airg_vcycle.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.airg_cf_split.argtypes = [C.POINTER(_Csr), C.POINTER(_Params), C.c_int, C.c_void_p, C.c_void_p]
        L.airg_ddc_theta.argtypes = [C.POINTER(_Csr), C.c_void_p, C.c_void_p, C.c_void_p]
        L.airg_cf_split_noalloc.argtypes = [C.POINTER(_Csr), C.POINTER(_Params), C.c_int, C.c_void_p, C.c_void_p]
        L.airg_setup_transpose.argtypes = [C.POINTER(_Csr), C.POINTER(_Params), C.c_void_p, C.POINTER(C.c_void_p)]
        L.airg_transpose.argtypes = [C.POINTER(_Csr), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.airg_sddmm.argtypes = [C.POINTER(_Csr), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
        L.airg_batch_create.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
        L.airg_solve_batched.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Opts), C.c_void_p, C.c_void_p]
        L.airg_batch_free.argtypes = [C.c_void_p]
        L.airg_batch_tuned.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.airg_batch_free.restype = None
        L.airg_free.argtypes = [C.c_void_p]
        L.airg_free.restype = None
        L.airg_num_levels.argtypes = [C.c_void_p]
        L.airg_level_info.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.airg_export_csr.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.airg_export_vectors.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.airg_export_layout.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.airg_profile_enable.argtypes = [C.c_void_p, C.c_int]
        L.airg_kernel_times.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.airg_kernel_times_level.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.airg_status_string.restype = C.c_char_p
        L.airg_launch_count.restype = C.c_int64
        L.airg_params_default.argtypes = [C.POINTER(_Params)]
        L.airg_params_default.restype = None
        _lib = L
    return _lib


EXPORTED = ["airg_params_default", "airg_setup", "airg_setup_host", "airg_setup_many", "airg_setup_reuse", "airg_setup_transpose", "airg_ddc_theta", "airg_transpose", "airg_sddmm",
            "airg_solve", "airg_solve_host", "airg_vcycle", "airg_cf_split", "airg_batch_create",
            "airg_solve_batched", "airg_batch_free", "airg_batch_tuned",
            "airg_cf_split_noalloc",
            "airg_free", "airg_num_levels", "airg_level_info", "airg_export_csr", "airg_export_vectors", "airg_export_layout",
            "airg_profile_enable", "airg_kernel_times", "airg_kernel_times_level", "airg_launch_count",
            "airg_status_string"]


def launch_count() -> int:
    """Kernel launches issued by libairg.so so far in this process."""
    return int(lib().airg_launch_count())


@dataclass
class Params:
    strong_threshold: float = 0.5
    ddc_fraction: float = 0.1
    pmisr_max_loops: int = 3
    poly_order: int = 6
    coarse_poly_order: int = 12
    coarse_iters: int = 3
    coarse_size: int = 0
    max_levels: int = 64
    drop_R: float = 0.01
    drop_Ac: float = 0.001
    n_smooth_up: int = 2
    precision: int = 0
    keep_setup: int = 0
    seed: int = 240808262
    sparsity_order: int = 1
    matrix_free: int = 0
    ideal_prolong: int = 0

    def c(self) -> _Params:
        return _Params(**{k: getattr(self, k) for k, _ in _Params._fields_})


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(code: int, what: str, allow_not_converged: bool = False):
    if code == AIRG_OK or (allow_not_converged and code == AIRG_NOT_CONVERGED):
        return
    raise AirgError(code, what)


def _csr(rowptr, col, val, host: bool = False) -> _Csr:
    import torch
    for t, dt in ((rowptr, torch.int32), (col, torch.int32), (val, torch.float64)):
        if not (t.is_cuda != host and t.dtype == dt and t.is_contiguous()):
            where = "CPU" if host else "CUDA"
            raise TypeError(f"CSR arrays must be contiguous {where} tensors (int32, int32, float64)")
    return _Csr(rowptr.numel() - 1, col.numel(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())


class Hierarchy:
    """An AIRG hierarchy built on the GPU (airg_setup)."""

    def __init__(self, rowptr, col, val, params: Params | None = None, stream=None, transpose: bool = False,
                 reuse: "Hierarchy | None" = None, reuse_levels: int = 0, host: bool = False):
        """transpose=True builds the hierarchy of A^T (airg_setup_transpose), for adjoint solves.
        reuse=T takes the CF splittings of T's first reuse_levels levels (0: all) instead of computing
        them (airg_setup_reuse); the matrix should share T's sparsity pattern.  host=True takes CPU
        tensors (pinned ones copy fastest) and lets the library copy them in (airg_setup_host)."""
        self.params = params or Params()
        self._keep = (rowptr, col, val)
        A = _csr(rowptr, col, val, host=host)
        self.n = A.n
        h = C.c_void_p()
        if host:
            if transpose or reuse is not None:
                raise TypeError("host=True builds a plain hierarchy (no transpose or re-use)")
            _check(lib().airg_setup_host(C.byref(A), C.byref(self.params.c()), _stream(stream), C.byref(h)),
                   "airg_setup_host")
        elif reuse is not None:
            _check(lib().airg_setup_reuse(C.byref(A), C.byref(self.params.c()), reuse._h, reuse_levels,
                                          _stream(stream), C.byref(h)), "airg_setup_reuse")
        else:
            fn = lib().airg_setup_transpose if transpose else lib().airg_setup
            _check(fn(C.byref(A), C.byref(self.params.c()), _stream(stream), C.byref(h)),
                   "airg_setup_transpose" if transpose else "airg_setup")
        self._h = h

    @classmethod
    def _adopt(cls, handle, n, params, keep):
        """A Hierarchy object around a handle the library built (airg_setup_many)."""
        H = cls.__new__(cls)
        H.params, H._keep, H.n, H._h = params, keep, n, handle
        return H

    def close(self):
        if getattr(self, "_h", None):
            lib().airg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self) -> int:
        return lib().airg_num_levels(self._h)

    def level_info(self, level: int) -> dict:
        info = np.zeros(18, dtype=np.int64)
        _check(lib().airg_level_info(self._h, level, info.ctypes.data), "airg_level_info")
        if level == -1:
            return dict(levels=int(info[0]), grid=info[1] / 1e6, operator=info[2] / 1e6, storage=info[3] / 1e6,
                        setup_ms=info[4] / 1e3,
                        phase_ms=dict(cf_split=info[5] / 1e3, extract=info[6] / 1e3, polynomial=info[7] / 1e3,
                                      restrictor=info[8] / 1e3, coarse=info[9] / 1e3, layout=info[10] / 1e3),
                        top_sell=int(info[11]))
        keys = ["n", "nnz", "nf", "nc", "nnz_aff", "nnz_afc", "nnz_ainv", "nnz_z", "coarsest", "nnz_acf",
                "alpha_fitted", "nnz_af", "us_cf", "us_poly", "us_z", "us_coarse", "nnz_w", "sell_mask"]
        return {k: int(v) for k, v in zip(keys, info)}

    def solve(self, b, x=None, outer: str = "fgmres", restart: int = 30, max_it: int = 200, rtol: float = 1e-10,
              stream=None):
        import torch
        if x is None:
            x = torch.zeros_like(b)
            x0_zero = 1
        else:
            x0_zero = 0
        opts = _Opts({"fgmres": 0, "richardson": 1}[outer], restart, max_it, rtol, x0_zero)
        info = _Info()
        rc = lib().airg_solve(self._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(opts),
                              C.byref(info), _stream(stream))
        _check(rc, "airg_solve", allow_not_converged=True)
        return x, dict(iters=info.iters, relres=info.relres, status=info.status, levels=info.levels)

    def solve_host(self, b_host, x_host, outer="fgmres", restart=30, max_it=200, rtol=1e-10, x0_zero=True,
                   stream=None):
        """b_host, x_host: CPU tensors (ideally pinned), float64; copies run inside the call."""
        opts = _Opts({"fgmres": 0, "richardson": 1}[outer], restart, max_it, rtol, int(x0_zero))
        info = _Info()
        rc = lib().airg_solve_host(self._h, C.c_void_p(b_host.data_ptr()), C.c_void_p(x_host.data_ptr()),
                                   C.byref(opts), C.byref(info), _stream(stream))
        _check(rc, "airg_solve_host", allow_not_converged=True)
        return x_host, dict(iters=info.iters, relres=info.relres, status=info.status, levels=info.levels)

    def vcycle(self, b, stream=None):
        import torch
        x = torch.empty_like(b)
        _check(lib().airg_vcycle(self._h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), _stream(stream)),
               "airg_vcycle")
        return x

    def export(self, level: int, which: str):
        """which: A, Aff, Afc, Acf, Ainv, Z (natural numbering, needs keep_setup) or the solve layout
        AF_solve, Z_solve, A0_solve, Ainv_solve, A_coarsest; W (natural, keep_setup) and W_solve with
        ideal_prolong."""
        code = {"A": 0, "Aff": 1, "Afc": 2, "Acf": 3, "Ainv": 5, "Z": 6, "AF_solve": 7, "Z_solve": 8,
                "A0_solve": 9, "Ainv_solve": 10, "A_coarsest": 11, "W": 12, "W_solve": 13}[which]
        inf = self.level_info(level)
        top = self.level_info(0)
        rows = {"A": inf["n"], "Aff": inf["nf"], "Afc": inf["nf"], "Acf": inf["nc"], "Z": inf["nc"],
                "Ainv": inf["n"] if inf["coarsest"] else inf["nf"], "AF_solve": inf["nf"], "Z_solve": inf["nc"],
                "A0_solve": top["n"], "Ainv_solve": inf["n"] if inf["coarsest"] else inf["nf"],
                "A_coarsest": inf["n"], "W": inf["nf"], "W_solve": inf["nf"]}[which]
        nnz = {"A": inf["nnz"], "Aff": inf["nnz_aff"], "Afc": inf["nnz_afc"], "Acf": inf["nnz_acf"],
               "Z": inf["nnz_z"], "Ainv": inf["nnz_ainv"], "AF_solve": inf["nnz_af"], "Z_solve": inf["nnz_z"],
               "A0_solve": top["nnz"], "Ainv_solve": inf["nnz_ainv"], "A_coarsest": inf["nnz"],
               "W": inf["nnz_w"], "W_solve": inf["nnz_w"]}[which]
        rp = np.zeros(rows + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        v = np.zeros(nnz, dtype=np.float64)
        _check(lib().airg_export_csr(self._h, level, code, rp.ctypes.data, ci.ctypes.data, v.ctypes.data),
               "airg_export_csr")
        return rp, ci, v

    def vectors(self, level: int) -> dict:
        inf = self.level_info(level)
        m = (self.params.coarse_poly_order if inf["coarsest"] else self.params.poly_order) + 1
        cf = np.zeros(0 if inf["coarsest"] else inf["n"], dtype=np.int8)
        w = np.zeros(inf["nf"], dtype=np.int32)
        alpha = np.zeros(m, dtype=np.float64)
        keep = bool(self.params.keep_setup)
        _check(lib().airg_export_vectors(self._h, level, cf.ctypes.data if keep else None,
                                         w.ctypes.data if keep else None, alpha.ctypes.data), "airg_export_vectors")
        return dict(cf=cf, w=w, alpha=alpha)

    def layout(self, level: int) -> dict:
        inf = self.level_info(level)
        pos = np.zeros(inf["n"], dtype=np.int32)
        ws = np.zeros(inf["nf"], dtype=np.int32)
        _check(lib().airg_export_layout(self._h, level, pos.ctypes.data, ws.ctypes.data), "airg_export_layout")
        return dict(pos=pos, w_solve=ws)

    def profile(self, classes=None):
        """Times kernel classes with CUDA events: None = all, [] = off, or a list of class names."""
        if classes is None:
            mask = -1
        else:
            mask = 0
            for c in classes:
                mask |= 1 << PROFILE_CLASSES.index(c)
        _check(lib().airg_profile_enable(self._h, mask), "airg_profile_enable")

    def kernel_times(self) -> dict:
        n = len(PROFILE_CLASSES)
        la = np.zeros(n, dtype=np.int64)
        ms = np.zeros(n)
        by = np.zeros(n)
        _check(lib().airg_kernel_times(self._h, la.ctypes.data, ms.ctypes.data, by.ctypes.data, n), "airg_kernel_times")
        return {c: dict(launches=int(la[i]), ms=float(ms[i]), bytes=float(by[i])) for i, c in enumerate(PROFILE_CLASSES)}

    def kernel_times_level(self, level: int) -> dict:
        n = len(PROFILE_CLASSES)
        la = np.zeros(n, dtype=np.int64)
        ms = np.zeros(n)
        by = np.zeros(n)
        _check(lib().airg_kernel_times_level(self._h, level, la.ctypes.data, ms.ctypes.data, by.ctypes.data, n),
               "airg_kernel_times_level")
        return {c: dict(launches=int(la[i]), ms=float(ms[i]), bytes=float(by[i])) for i, c in enumerate(PROFILE_CLASSES)}


def setup_many(mats, params: Params | None = None, nthreads: int = 8, stream=None) -> list:
    """Hierarchies of many independent systems built concurrently (airg_setup_many): mats is a list
    of (rowptr, col, val) CUDA tensor triples; returns one Hierarchy per system."""
    p = params or Params()
    arr = (_Csr * len(mats))(*[_csr(*m) for m in mats])
    hs = (C.c_void_p * len(mats))()
    _check(lib().airg_setup_many(arr, len(mats), C.byref(p.c()), nthreads, _stream(stream), hs), "airg_setup_many")
    return [Hierarchy._adopt(C.c_void_p(h), m[0].numel() - 1, p, m) for h, m in zip(hs, mats)]


def cf_split(rowptr, col, val, params: Params | None = None, level: int = 0, stream=None):
    """Two-pass CF splitting on the GPU; returns a CUDA int8 tensor (1 = F, 2 = C)."""
    import torch
    A = _csr(rowptr, col, val)
    cf = torch.empty(A.n, dtype=torch.int8, device=rowptr.device)
    p = params or Params()
    _check(lib().airg_cf_split(C.byref(A), C.byref(p.c()), level, C.c_void_p(cf.data_ptr()), _stream(stream)),
           "airg_cf_split")
    return cf


def ddc_theta(rowptr, col, val, cf, stream=None):
    """airg_ddc_theta: theta_i = sum_{j in F, j != i} |a_ij| / |a_ii| for the F-points of the
    splitting cf (CUDA int8, 1 = F, 2 = C); a CUDA float64 tensor, 0 on C-points."""
    import torch
    A = _csr(rowptr, col, val)
    if not (cf.is_cuda and cf.dtype == torch.int8 and cf.numel() == A.n):
        raise TypeError("cf must be a CUDA int8 tensor with one entry per row")
    theta = torch.empty(A.n, dtype=torch.float64, device=rowptr.device)
    _check(lib().airg_ddc_theta(C.byref(A), C.c_void_p(cf.data_ptr()), C.c_void_p(theta.data_ptr()),
                                _stream(stream)), "airg_ddc_theta")
    return theta


def cf_split_noalloc(rowptr, col, val, cf_out, params: Params | None = None, level: int = 0, stream=None):
    """airg_cf_split_noalloc: the CF splitting written into the caller's int8 CUDA tensor cf_out,
    with no device allocation inside the library (for callers that cannot allocate at that point;
    see include/airg.h for the capacity and the sharing rules)."""
    A = _csr(rowptr, col, val)
    import torch
    if not (cf_out.is_cuda and cf_out.dtype == torch.int8 and cf_out.is_contiguous() and cf_out.numel() == A.n
            and cf_out.device == rowptr.device):
        raise TypeError("cf_out must be a contiguous int8 CUDA tensor on the matrix's device, one entry per row")
    p = params or Params()
    _check(lib().airg_cf_split_noalloc(C.byref(A), C.byref(p.c()), level, C.c_void_p(cf_out.data_ptr()),
                                       _stream(stream)), "airg_cf_split_noalloc")
    return cf_out


class Batch:
    """Many systems solved together (airg_batch_create / airg_solve_batched); keeps the
    hierarchies alive."""

    def __init__(self, hierarchies, stream=None):
        self.H = list(hierarchies)
        arr = (C.c_void_p * len(self.H))(*[h._h.value for h in self.H])
        b = C.c_void_p()
        _check(lib().airg_batch_create(arr, len(self.H), _stream(stream), C.byref(b)), "airg_batch_create")
        self._b = b

    def tuned(self) -> list:
        """(rule lanes, chosen lanes) of every group the SpMV autotuner timed (airg_batch_tuned)."""
        n = lib().airg_batch_tuned(self._b, None, None, 0)
        rule = (C.c_int * max(n, 1))()
        chosen = (C.c_int * max(n, 1))()
        lib().airg_batch_tuned(self._b, rule, chosen, n)
        return [(rule[k], chosen[k]) for k in range(n)]

    def close(self):
        if getattr(self, "_b", None):
            lib().airg_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, bs, restart: int = 30, max_it: int = 200, rtol: float = 1e-10, stream=None):
        import torch
        xs = [torch.zeros_like(b) for b in bs]
        bp = (C.c_void_p * len(bs))(*[b.data_ptr() for b in bs])
        xp = (C.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        infos = (_Info * len(bs))()
        opts = _Opts(0, restart, max_it, rtol, 1)
        rc = lib().airg_solve_batched(self._b, bp, xp, C.byref(opts), infos, _stream(stream))
        _check(rc, "airg_solve_batched", allow_not_converged=True)
        return xs, [dict(iters=i.iters, relres=i.relres, status=i.status, levels=i.levels) for i in infos]


def transpose(rowptr, col, val, stream=None):
    """A^T on the device (airg_transpose); returns (rowptr, col, val) CUDA tensors."""
    import torch
    A = _csr(rowptr, col, val)
    rp = torch.empty_like(rowptr)
    ci = torch.empty_like(col)
    v = torch.empty_like(val)
    _check(lib().airg_transpose(C.byref(A), C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()),
                                C.c_void_p(v.data_ptr()), _stream(stream)), "airg_transpose")
    return rp, ci, v


def sddmm(rowptr, col, lam, x, scale: float = 1.0, stream=None):
    """out[k] = scale * lam[i] * x[col[k]] on the pattern (airg_sddmm)."""
    import torch
    A = _Csr(rowptr.numel() - 1, col.numel(), rowptr.data_ptr(), col.data_ptr(), 0)
    out = torch.empty(col.numel(), dtype=torch.float64, device=col.device)
    _check(lib().airg_sddmm(C.byref(A), C.c_void_p(lam.data_ptr()), C.c_void_p(x.data_ptr()), C.c_double(scale),
                            C.c_void_p(out.data_ptr()), _stream(stream)), "airg_sddmm")
    return out


class HierarchyCache:
    """Hierarchies of the adjoint form kept for re-use: one for A (forward solves) and one for A^T
    (backward solves), each for the most recent matrix.  A matrix is the same one when it is given by
    the same three tensors (storage, offset, size, device) and none of them has been written since
    (torch's version counter of each tensor); anything else builds a new hierarchy.  Only a
    bookkeeping layer: the hierarchies and solves are the library's."""

    def __init__(self):
        self.entries = {}

    @staticmethod
    def key(rowptr, col, val, params, transpose):
        def tk(t):
            return (t.data_ptr(), t.numel(), t.dtype, str(t.device), t._version)
        return (tk(rowptr), tk(col), tk(val), tuple(sorted(vars(params).items())), bool(transpose))

    def get(self, rowptr, col, val, params, transpose=False):
        k = self.key(rowptr, col, val, params, transpose)
        ent = self.entries.get(transpose)
        if ent is not None and ent[0] == k:
            return ent[1]
        if ent is not None:
            ent[1].close()
        H = Hierarchy(rowptr, col, val, params, transpose=transpose)
        self.entries[transpose] = (k, H, (rowptr, col, val))  # the tensors stay alive with the entry
        return H

    def clear(self):
        for ent in self.entries.values():
            ent[1].close()
        self.entries.clear()


def _solve_fn(cache: "HierarchyCache | None"):
    import torch

    class SolveFn(torch.autograd.Function):
        """x = A^-1 b with AIRG-preconditioned FGMRES; differentiable in A's values and b.

        backward: lambda = A^-T g by an AIRG solve with the hierarchy of A^T (airg_setup_transpose);
        dL/db = lambda and dL/dA = -lambda x^T on A's pattern (airg_sddmm).  With a cache, the
        hierarchies of A and A^T are kept and re-used while the matrix tensors are unchanged."""

        @staticmethod
        def forward(ctx, rowptr, col, val, b, params=None, rtol=1e-12):
            par = params or Params()
            if cache is not None:
                H = cache.get(rowptr, col, val, par)
            else:
                H = Hierarchy(rowptr, col, val, par)
            x, info = H.solve(b.contiguous(), rtol=rtol, max_it=500)
            if cache is None:
                H.close()
            if info["status"] != 0:
                raise AirgError(info["status"], "SolveFn forward")
            ctx.save_for_backward(rowptr, col, val, x)
            ctx.params, ctx.rtol = par, rtol
            return x

        @staticmethod
        def backward(ctx, gx):
            rowptr, col, val, x = ctx.saved_tensors
            if cache is not None:
                HT = cache.get(rowptr, col, val, ctx.params, transpose=True)
            else:
                HT = Hierarchy(rowptr, col, val, ctx.params, transpose=True)
            lam, info = HT.solve(gx.contiguous(), rtol=ctx.rtol, max_it=500)
            if cache is None:
                HT.close()
            if info["status"] != 0:
                raise AirgError(info["status"], "SolveFn backward")
            gval = sddmm(rowptr, col, lam, x, -1.0) if ctx.needs_input_grad[2] else None
            gb = lam if ctx.needs_input_grad[3] else None
            return None, None, gval, gb, None, None

    return SolveFn


_SolveFn = None


def solve_fn(cache: "HierarchyCache | None" = None):
    """The torch.autograd.Function of the adjoint form (SolveFn.apply(rowptr, col, val, b, params, rtol)).
    With a HierarchyCache, forward and backward re-use the hierarchies of A and A^T while the matrix
    tensors are unchanged (several right-hand sides, or an optimisation over the source only)."""
    global _SolveFn
    if cache is not None:
        return _solve_fn(cache)
    if _SolveFn is None:
        _SolveFn = _solve_fn(None)
    return _SolveFn


def setup(rowptr, col, val, params: Params | None = None, stream=None) -> Hierarchy:
    return Hierarchy(rowptr, col, val, params, stream)


def solve(H: Hierarchy, b, **kw):
    return H.solve(b, **kw)

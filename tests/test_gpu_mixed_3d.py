"""The mixed-precision form on its own configuration, at full size: 3D upwind P0 DG on 128^3 cubes
of six jittered Kuhn tetrahedra each (12,582,912 DOFs), Omega = (0.48, 0.60, 0.64), sigma in
{0, 0.01} split by a seeded half-space.  The V-cycle runs with FP32 values (or bf16 value storage)
and FP32 vectors; the outer FGMRES, its residuals and the coefficient fits stay FP64.

Bars:
  * every form reaches the FP64 true residual ||b - A x|| / ||b|| <= 1e-8, checked on the host;
  * the mixed solutions agree with the FP64 GPU solution to a relative 1e-8, the bar of the 32^3
    instance (the outer FP64 FGMRES takes the same number of iterations, so the two solutions
    differ by far less than what two residuals of 1e-8 would allow; measured 1e-13 with FP32
    values and 5e-12 with bf16 values);
  * iterations within +2 (FP32) / +4 (bf16) of FP64, as on the 32^3 instance, whose oracle
    comparison is in test_gpu_parity.py.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2408_08262_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2408_08262_gb300 import airg  # noqa: E402


@pytest.fixture(scope="module")
def c3():
    p = P.kuhn_3d(128)
    assert p.n == 12_582_912
    d = tuple(torch.from_numpy(a).cuda() for a in (p.rowptr, p.col, p.val, p.b))
    return p, d


def test_full_size_3d_forms_reach_rtol_and_agree_with_fp64(c3):
    p, (rp, ci, v, b) = c3
    A = sp.csr_matrix((p.val, p.col, p.rowptr), shape=(p.n, p.n))
    bn = np.linalg.norm(p.b)
    out = {}
    for prec in (0, 1, 2):
        H = airg.Hierarchy(rp, ci, v, airg.Params(precision=prec))
        x, info = H.solve(b, rtol=1e-8)
        H.close()
        assert info["status"] == 0 and info["relres"] <= 1e-8, (prec, info)
        xh = x.cpu().numpy()
        rel = np.linalg.norm(p.b - A @ xh) / bn
        assert rel <= 1.0001e-8, (prec, rel)
        out[prec] = (xh, info)
    x64, i64 = out[0]
    bar = 1e-8
    for prec, extra in ((1, 2), (2, 4)):
        xlo, ilo = out[prec]
        err = np.linalg.norm(xlo - x64) / np.linalg.norm(x64)
        print(f"precision {prec}: iters {ilo['iters']} (FP64 {i64['iters']}), rel err vs FP64 {err:.3e}, "
              f"bar {bar:.3e}")
        assert err <= bar, (prec, err, bar)
        assert ilo["iters"] <= i64["iters"] + extra

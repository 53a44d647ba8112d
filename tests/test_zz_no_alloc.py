"""airg_cf_split_noalloc: the CF splitting for callers that cannot allocate device memory at the
point they need it (a program that reserved all GPU memory at start-up, or a latency-critical loop
where an allocation is not acceptable).  It must give exactly what airg_cf_split gives while using
only the library's fixed scratch array.

This file is collected last, so a run that stops at the first failure has already run every other
test; it also passes when run on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2408_08262_gb300 import airg  # noqa: E402
from paper_2408_08262_gb300 import problems as P  # noqa: E402


def dev(p):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (p.rowptr, p.col, p.val))


def test_noalloc_first_and_then_without_any_device_allocation():
    # In a fresh process this is the library's first call on the device: it loads the kernels and
    # the array (CUDA loads modules on first use), so only the calls after it are checked for
    # allocations.  Free device memory and torch's reserved pool must not move across them, and
    # every result must equal the allocating entry point's, computed afterwards.
    p = P.blocked_sigma_2d(96)
    rp, ci, v = dev(p)
    params = airg.Params()
    outs = [torch.full((p.n,), -1, dtype=torch.int8, device="cuda") for _ in range(3)]
    airg.cf_split_noalloc(rp, ci, v, outs[0], params)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for out in outs[1:]:
        airg.cf_split_noalloc(rp, ci, v, out, params)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_reserved() == reserved0
    ref = airg.cf_split(rp, ci, v, params)
    for out in outs:
        assert torch.equal(out, ref)


@pytest.mark.parametrize("mesh,level", [(64, 0), (128, 3)])
def test_noalloc_matches_the_allocating_entry_point_on_two_calls(mesh, level):
    p = P.blocked_sigma_2d(mesh)
    rp, ci, v = dev(p)
    params = airg.Params()
    ref = airg.cf_split(rp, ci, v, params, level=level)  # the existing entry point
    for _ in range(2):  # the second call reuses the array the first one left behind
        out = torch.full((p.n,), -1, dtype=torch.int8, device="cuda")
        airg.cf_split_noalloc(rp, ci, v, out, params, level=level)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_rejects_inputs_beyond_its_capacity():
    p = P.streaming_2d(8)
    rp, ci, v = dev(p)
    # sizes far beyond the fixed array: rejected before any GPU work touches the pointers
    A = airg._Csr(10_000_000, 100_000_000, rp.data_ptr(), ci.data_ptr(), v.data_ptr())
    out = torch.empty(p.n, dtype=torch.int8, device="cuda")
    rc = airg.lib().airg_cf_split_noalloc(ctypes.byref(A), ctypes.byref(airg.Params().c()), 0,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert rc == -8
    assert b"scratch" in airg.lib().airg_status_string(rc)

"""cp_resid_noalloc: the direct residual for callers that cannot allocate device memory.

Programs whose own pool has reserved the GPU, or latency-critical loops where
cudaMalloc would synchronise the device, call this variant; its scratch is a
fixed device array inside the library.  Checked against cp_fit(exact = 1) on two
calls in a row (the array keeps the previous call's contents, which must not
leak into the next result).  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2010_12056_gb300 as p
    return p


@pytest.mark.parametrize("dims,R", [((64, 64, 64), 16), ((33, 40, 29, 7), 5)])
def test_resid_noalloc_matches_cp_fit_twice(pkg, dims, R):
    T64, _, A0 = synth.make_problem(90, dims, R, eta=1e-2)
    Td = torch.from_numpy(np.ascontiguousarray(T64.astype(np.float32))).cuda()
    ctx = pkg.CPContext(Td, R, A0=A0, prec="fp32")
    ctx.sweep_dt(2)
    _, r_ref = ctx.fit(exact=True)
    A32 = [torch.from_numpy(np.ascontiguousarray(ctx.get_factor(n).astype(np.float32))).cuda()
           for n in range(len(dims))]
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        pkg.resid_noalloc(Td, A32, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        r = math.sqrt(o[0] / o[1])
        assert abs(r - r_ref) <= 1e-6, (call, r, r_ref)
    # a different problem right after: nothing of the previous call may remain
    A_other = [torch.rand(d, R, dtype=torch.float32, device="cuda") for d in dims]
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    pkg.resid_noalloc(Td, A_other, out)
    ctx2 = pkg.CPContext(Td, R, A0=[a.double().cpu().numpy() for a in A_other], prec="fp32")
    _, r2 = ctx2.fit(exact=True)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert abs(math.sqrt(o[0] / o[1]) - r2) <= 1e-6
    ctx.close()
    ctx2.close()


def test_resid_noalloc_rejects_oversized(pkg):
    L = pkg.lib()
    dims = (ctypes.c_int64 * 3)(1024, 1024, 1024)      # 262144 tiles > 65536
    fake = ctypes.c_void_p(256)
    ptrs = (ctypes.c_void_p * 3)(256, 256, 256)
    assert L.cp_resid_noalloc(3, dims, 8, fake, ptrs, fake, None) == 1
    # a last mode so large that (row tiles x column tiles) would wrap int64
    huge = (ctypes.c_int64 * 3)(1 << 20, 1 << 20, (1 << 62) + 1)
    assert L.cp_resid_noalloc(3, huge, 8, fake, ptrs, fake, None) == 1
    wide = (ctypes.c_int64 * 3)(1, 1, 64 * 65536 + 1)     # one row tile, 65537 column tiles
    assert L.cp_resid_noalloc(3, wide, 8, fake, ptrs, fake, None) == 1

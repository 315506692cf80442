"""gbem_solve_noalloc against gbem_solve, through the C ABI.

gbem_solve_noalloc exists for callers that may not allocate device memory at
solve time (a serving worker with a fixed HBM reservation, a host program
whose arena owns all device memory, a latency-critical loop that must avoid
the device synchronisation of cudaMalloc/cudaFree).  It keeps its work
buffers in a fixed static device array, shared by all calls, so this test
runs it twice in a row -- the second call starts from the first call's
leftovers -- and checks both results against the allocating gbem_solve.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10   # relative, the tolerance of the FP64 entry parity tests


def _noalloc(lib):
    f = lib.gbem_solve_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
    return f


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_noalloc_matches_solve(prec):
    import torch
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    B.build()
    lib = gbem.load()
    solve_noalloc = _noalloc(lib)
    ctx = gbem.Context(0)
    mesh = ctx.mesh(*W.two_bars())
    mat = gbem.gbem_assemble(mesh, prec)
    mat.factor()
    n = mesh.n
    gen = torch.Generator("cuda").manual_seed(11)
    stream = torch.cuda.current_stream()
    for call in range(2):
        nrhs = 3 + call                      # different shapes on the two calls
        Bm = torch.randn(nrhs, n, dtype=torch.float64, device="cuda", generator=gen)   # column-major N x nrhs
        X_ref, _ = mat.solve(Bm.t())
        X_ref = X_ref.contiguous().cpu().numpy()
        Xn = torch.full((nrhs, n), float("nan"), dtype=torch.float64, device="cuda")
        it = ctypes.c_int(-1)
        st = solve_noalloc(mat.h, ctypes.c_void_p(Bm.data_ptr()), nrhs, n, ctypes.c_void_p(Xn.data_ptr()), n,
                           ctypes.byref(it), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.gbem_last_error(ctx.h)
        torch.cuda.synchronize()
        Xh = Xn.t().cpu().numpy()
        assert np.all(np.isfinite(Xh))
        err = np.max(np.abs(Xh - X_ref)) / np.max(np.abs(X_ref))
        assert err <= TOL, (prec, call, err)
        if prec == 1:
            assert it.value >= 1
    mat.close()
    mesh.close()
    ctx.close()


def test_solve_noalloc_rejects_oversize():
    import torch
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    torch.cuda.set_device(0)
    B.build()
    lib = gbem.load()
    solve_noalloc = _noalloc(lib)
    ctx = gbem.Context(0)
    mesh = ctx.mesh(*W.two_bars())
    mat = gbem.gbem_assemble(mesh, 0)
    mat.factor()
    nrhs = 2000   # 640 x 2000 x 40 bytes > 16 MiB
    Bm = torch.zeros(nrhs, mesh.n, dtype=torch.float64, device="cuda")
    st = solve_noalloc(mat.h, ctypes.c_void_p(Bm.data_ptr()), nrhs, mesh.n, ctypes.c_void_p(Bm.data_ptr()),
                       mesh.n, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1
    assert b"limit" in lib.gbem_last_error(ctx.h)
    mat.close()
    mesh.close()
    ctx.close()

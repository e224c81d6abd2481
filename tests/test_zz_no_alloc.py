"""The allocation-free local-solve entry point (msp_sample_patch_static).

It serves callers that cannot allocate device memory during the call (a memory
pool they do not own, a hot path where allocation is forbidden, an allocator
at its limit).  Its scratch is a static device array shared by all calls, so
this file also checks that a second call in a row, which starts from the first
call's leftovers, gives the same result.  The reference is the allocating
entry point (msp_sample_patches) on the same medium, patch and seed, compared
at the FP64 parity tolerance of the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")

FP64_TOL = 1e-8
MIXED_TOL = 1e-6


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol,check", [("fp64", 1e-12, FP64_TOL), ("mixed", 1e-10, MIXED_TOL)])
def test_static_scratch_matches_allocating_path(precision, tol, check):
    from paper_1807_08848_gb300 import _native as N
    lib = N.load()
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    med.sample(w["seed"], precision, tol=tol, max_iter=20000)
    m = 5                                   # an interior patch: Gaussian columns only
    info = med.patch(m)
    assert info.n_b == 0
    ref = med.snapshots(m).cpu().numpy()
    aE, aN = med.coefficients()
    boxes = (C.c_int * 8)(info.x0, info.x1, info.y0, info.y1, info.X0, info.X1, info.Y0, info.Y1)
    stream = torch.cuda.current_stream()
    outs = []
    for _ in range(2):                      # two calls in a row share the static scratch
        out = torch.full((info.samples, info.n_k), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.msp_sample_patch_static(C.c_void_p(aE.data_ptr()), C.c_void_p(aN.data_ptr()), med.n_cells, boxes, m,
                                         info.samples, C.c_uint64(w["seed"]), msp.precision_code(precision), tol,
                                         20000, C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        N.check(st)
        torch.cuda.synchronize()
        outs.append(out.T.cpu().numpy())
    for o in outs:
        assert np.all(np.isfinite(o))
        assert rel(o, ref[:, :info.samples]) <= check


def test_static_scratch_rejects_oversized_requests():
    from paper_1807_08848_gb300 import _native as N
    lib = N.load()
    aE = torch.ones((257, 256), dtype=torch.float64, device="cuda")
    aN = torch.ones((256, 257), dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    big = (C.c_int * 8)(50, 200, 50, 100, 0, 256, 0, 150)    # interior far wider than the tile
    st = lib.msp_sample_patch_static(C.c_void_p(aE.data_ptr()), C.c_void_p(aN.data_ptr()), 256, big, 0, 4,
                                     C.c_uint64(1), 0, 1e-10, 100, C.c_void_p(out.data_ptr()), None)
    assert st == N.MSP_ERR_INVALID_ARG and b"tile" in lib.msp_last_error()
    ok = (C.c_int * 8)(64, 128, 64, 128, 48, 144, 48, 144)
    st = lib.msp_sample_patch_static(C.c_void_p(aE.data_ptr()), C.c_void_p(aN.data_ptr()), 256, ok, 0, 5000,
                                     C.c_uint64(1), 0, 1e-10, 100, C.c_void_p(out.data_ptr()), None)
    assert st == N.MSP_ERR_INVALID_ARG

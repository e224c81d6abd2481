"""The allocation-free local-solve entry point (msp_sample_patch_static).

It serves callers that cannot allocate device memory during the call (a memory
pool they do not own, a hot path where allocation is forbidden, an allocator
at its limit).  Its scratch is a static device array shared by all calls, so
this file also checks that a second call in a row, which starts from the first
call's leftovers, gives the same result.  The reference is the allocating
entry point (msp_sample_patches) on the same medium, patch and seed, compared
at the parity tolerances of the other GPU tests (FP64 path 1e-8, mixed 1e-6).
Cases: an interior patch of the small workload, a corner patch whose buffered
box is clipped by the domain (compared with the Gaussian columns of the
allocating path, which adds boundary-delta columns after them), and a patch
whose 95 x 95 interior needs the 12-row instance of the tile kernel.  The file
is collected last, so a run that stops at the first failure has run every other
test before it.
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


def _workload(name):
    if name == "small":
        w = synth.workload_small()
        return w["medium"], w["patches"], w["seed"]
    # 256 cells, middle patch of 64 cells with a 16-cell buffer: 95 x 95 interior
    br = np.array([0, 96, 160, 256])
    ps = synth.PatchSpec(br, br, np.full(9, 16), np.full(9, 24))
    return synth.lognormal(256, 2.0 ** -4, 64, 1), ps, 7


def _static_call(lib, med, info, m, seed, precision, tol, max_iter, out, stream, count=None):
    aE, aN = med.coefficients()
    boxes = (C.c_int * 8)(info.x0, info.x1, info.y0, info.y1, info.X0, info.X1, info.Y0, info.Y1)
    return lib.msp_sample_patch_static(C.c_void_p(aE.data_ptr()), C.c_void_p(aN.data_ptr()), med.n_cells, boxes, m,
                                       info.samples, C.c_uint64(seed), msp.precision_code(precision), tol, max_iter,
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream),
                                       C.byref(count) if count is not None else None)


@pytest.mark.parametrize("case,m", [("small", 5), ("small", 0), ("r12", 4)], ids=["interior", "corner", "rows12"])
@pytest.mark.parametrize("precision,tol,check", [("fp64", 1e-12, FP64_TOL), ("mixed", 1e-10, MIXED_TOL)])
def test_static_scratch_matches_allocating_path(case, m, precision, tol, check):
    from paper_1807_08848_gb300 import _native as N
    lib = N.load()
    medium, patches, seed = _workload(case)
    med = msp.Medium(medium, patches)
    med.sample(seed, precision, tol=tol, max_iter=20000)
    info = med.patch(m)
    if case == "corner":
        assert info.n_b > 0                 # the allocating path adds delta columns after the Gaussian ones
    if case == "rows12":
        assert info.X1 - info.X0 - 1 == 95 and info.Y1 - info.Y0 - 1 == 95
    ref = med.snapshots(m).cpu().numpy()[:, :info.samples]
    stream = torch.cuda.current_stream()
    outs = []
    for call in range(2):                   # two calls in a row share the static scratch
        out = torch.full((info.samples, info.n_k), float("nan"), dtype=torch.float64, device="cuda")
        count = C.c_int(-1)
        st = _static_call(lib, med, info, m, seed, precision, tol, 20000, out, stream,
                          count if call == 1 else None)
        N.check(st)
        if call == 1:
            assert count.value == 0
        torch.cuda.synchronize()
        outs.append(out.T.cpu().numpy())
    for o in outs:
        assert np.all(np.isfinite(o))
        assert rel(o, ref) <= check


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_scratch_reports_unconverged_columns(precision):
    """max_iter = 1 stops every column's CG before the tolerance: the count comes
    back from the static array's statistics and the call says NOT_CONVERGED; a
    following call with a normal max_iter converges again."""
    from paper_1807_08848_gb300 import _native as N
    lib = N.load()
    medium, patches, seed = _workload("small")
    med = msp.Medium(medium, patches)
    m = 5
    info = med.patch(m)
    stream = torch.cuda.current_stream()
    out = torch.empty((info.samples, info.n_k), dtype=torch.float64, device="cuda")
    count = C.c_int(-1)
    st = _static_call(lib, med, info, m, seed, precision, 1e-12, 1, out, stream, count)
    assert st == N.MSP_ERR_NOT_CONVERGED
    assert count.value == info.samples
    assert b"max_iter" in lib.msp_last_error()
    st = _static_call(lib, med, info, m, seed, precision, 1e-10, 20000, out, stream, count)
    assert st == N.MSP_OK and count.value == 0


def test_static_scratch_rejects_oversized_requests():
    from paper_1807_08848_gb300 import _native as N
    lib = N.load()
    aE = torch.ones((257, 256), dtype=torch.float64, device="cuda")
    aN = torch.ones((256, 257), dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    big = (C.c_int * 8)(50, 200, 50, 100, 0, 256, 0, 150)    # interior far wider than the tile
    st = lib.msp_sample_patch_static(C.c_void_p(aE.data_ptr()), C.c_void_p(aN.data_ptr()), 256, big, 0, 4,
                                     C.c_uint64(1), 0, 1e-10, 100, C.c_void_p(out.data_ptr()), None, None)
    assert st == N.MSP_ERR_INVALID_ARG and b"tile" in lib.msp_last_error()
    ok = (C.c_int * 8)(64, 128, 64, 128, 48, 144, 48, 144)
    st = lib.msp_sample_patch_static(C.c_void_p(aE.data_ptr()), C.c_void_p(aN.data_ptr()), 256, ok, 0, 5000,
                                     C.c_uint64(1), 0, 1e-10, 100, C.c_void_p(out.data_ptr()), None, None)
    assert st == N.MSP_ERR_INVALID_ARG

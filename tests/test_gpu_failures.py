"""Failure detection through the C ABI, with no GPU fault.

Every failure here is made on the host or by a bound the test sets: an
iteration cap that stops the solves early, a device-side grid barrier whose
poll bound is lowered until it gives up, boundary data with a NaN, and a
device allocation too large for the GPU.  Each call must return its status
code (not trap, hang or poison the context), and a following call with normal
arguments must give the correct result again.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")
from paper_1807_08848_gb300 import _native as N  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small():
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    med.sample(w["seed"], "fp64", tol=1e-12, max_iter=20000)
    basis = med.extract(w["tau"], "fp64")
    phi = torch.tensor(w["phi"], device="cuda")
    u_ok, _ = basis.solve(phi, tol=1e-10, max_iter=2000)
    return w, med, basis, phi, u_ok.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_local_solves_capped_report_not_converged(precision):
    """max_iter = 1 caps every CG before tol (Algorithm alg:summary, the local
    solver): msp_sample_patches reports NOT_CONVERGED and counts every solve."""
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    with pytest.raises(msp.MspError) as ei:
        med.sample(w["seed"], precision, tol=1e-12, max_iter=1)
    assert ei.value.status == N.MSP_ERR_NOT_CONVERGED
    st = med.sample(w["seed"], precision, tol=1e-10, max_iter=20000)     # same medium: converges again
    assert st.n_not_converged == 0


def test_online_capped_reports_not_converged(small):
    """The online CGLS (Eq. elliptic_cond_reduced) capped at one iteration with an
    unreachable tolerance: NOT_CONVERGED, with or without the iteration counts."""
    w, med, basis, phi, u_ok = small
    with pytest.raises(msp.MspError) as ei:
        basis.solve(phi, tol=1e-15, max_iter=1)
    assert ei.value.status == N.MSP_ERR_NOT_CONVERGED
    with pytest.raises(msp.MspError) as ei:
        basis.solve(phi, tol=1e-15, max_iter=1, want_iters=False)
    assert ei.value.status == N.MSP_ERR_NOT_CONVERGED
    u, _ = basis.solve(phi, tol=1e-10, max_iter=2000)
    assert rel(u.cpu().numpy(), u_ok) <= 1e-12


def test_grid_barrier_gives_up_and_context_survives(small):
    """The cooperative sweeps of the online factor synchronise the grid with a
    bounded barrier.  With the poll bound lowered to one poll, the first CTA to
    arrive gives up long before the rest of the grid comes: the launch ends, the
    call returns TIMEOUT, and after the default bound is restored the same solve
    gives the same field."""
    w, med, basis, phi, u_ok = small
    assert basis.stats()["online_blocks"] > 1          # the block-row factor (and its sweeps) is in use
    msp.set_wait_limit(1)
    try:
        with pytest.raises(msp.MspError) as ei:
            basis.solve(phi, tol=1e-10, max_iter=2000)
        assert ei.value.status == N.MSP_ERR_TIMEOUT
    finally:
        msp.set_wait_limit(0)
    u, _ = basis.solve(phi, tol=1e-10, max_iter=2000)
    assert rel(u.cpu().numpy(), u_ok) <= 1e-12
    with pytest.raises(msp.MspError):
        msp.set_wait_limit(-1)


def test_nan_boundary_data_stops_that_data_set(small):
    """A NaN in one data set's boundary values makes its residual non-finite: that
    data set stops at once (NOT_CONVERGED for the call), the other data set of the
    batch still reaches its solution."""
    w, med, basis, phi, u_ok = small
    bad = phi.clone()
    bad[7] = float("nan")
    both = torch.stack([bad, phi])
    u = torch.empty((2, 129, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(msp.MspError) as ei:
        basis.solve(both, tol=1e-10, max_iter=2000, u=u)
    assert ei.value.status == N.MSP_ERR_NOT_CONVERGED
    assert b"not finite" in N.load().msp_last_error()
    assert rel(u[1].cpu().numpy(), u_ok) <= 1e-12
    u1, it = basis.solve(phi, tol=1e-10, max_iter=2000)
    assert rel(u1.cpu().numpy(), u_ok) <= 1e-12


def test_allocation_failure_reports_oom():
    """A medium whose snapshot storage (2049^2 nodes x 2^20 columns, tens of terabytes)
    cannot be allocated: msp_build_medium returns OOM, keeps no handle, and the
    next medium builds and samples normally."""
    ps = synth.uniform_patches(2048, 1, 1, 0, 1 << 20)
    with pytest.raises(msp.MspError) as ei:
        msp.Medium(synth.periodic_sin(2048, 1 / 16), ps)
    assert ei.value.status == N.MSP_ERR_OOM
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    st = med.sample(w["seed"], "fp64", tol=1e-12, max_iter=20000)
    assert st.n_not_converged == 0
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"], patch_subset=[3])
    assert rel(med.snapshots(3).cpu().numpy(), off.R[0]) <= 1e-8

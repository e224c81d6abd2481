"""GPU tests of the direct local solver (launch mode "direct": a block LDL^T
factorisation over the grid rows of every buffered patch, FP32 inverses of the
Schur complements shared by all columns of the patch, FP64 iterative refinement;
the local solver of Algorithm alg:summary).

Snapshots against the oracle's sparse direct solves (Sec. 5.2, Eq.
elliptic_random), relative L2 <= 1e-6 (the mixed-path bound; the refinement
stops at |r| <= tol |b| with tol far below it), on: the small periodic workload,
a ragged uneven partition with a zero buffer and odd tile shapes, and the uneven
high-contrast channel medium whose buffered tiles reach 143 x 143 interior nodes.
The direct solver and the CG launches agree to the solver tolerance, a CUDA-graph
replay repeats the direct run bit for bit, and the online solution built on
direct-solver bases matches the oracle.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")

MIXED_TOL = 1e-6


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def direct_medium(ms, ps):
    med = msp.Medium(ms, ps)
    med.set_launch("mixed", "direct")
    return med


def test_small_workload_snapshots_and_online():
    w = synth.workload_small()
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
    u_ref, *_ = E.online(off, w["patches"], 128, w["phi"])
    med = direct_medium(w["medium"], w["patches"])
    st = med.sample(w["seed"], "mixed", tol=1e-11, max_iter=20000)
    assert st.n_not_converged == 0 and st.max_iters <= 8
    for m in range(16):
        assert rel(med.snapshots(m).cpu().numpy(), off.R[m]) <= 1e-9, m
    basis = med.extract(w["tau"], "mixed")
    for m in range(16):
        assert np.max(np.abs(basis.sigma(m) - off.sigma[m])) <= 1e-6 * off.sigma[m][0]
    u, _ = basis.solve(torch.tensor(w["phi"], device="cuda"), tol=1e-12, max_iter=20000)
    assert rel(u.cpu().numpy(), u_ref) <= MIXED_TOL


def test_ragged_partition_with_zero_buffer():
    N = 60
    ps = synth.PatchSpec(np.array([0, 13, 37, 60]), np.array([0, 22, 41, 60]),
                         np.array([3, 0, 5, 2, 4, 1, 6, 3, 2]), np.array([9, 17, 5, 12, 30, 7, 11, 8, 20]))
    ms = synth.hou_wu(N, 1 / 6)
    off = E.offline(ms, ps, 21, 1e-6)
    med = direct_medium(ms, ps)
    st = med.sample(21, "mixed", tol=1e-12, max_iter=20000)
    assert st.n_not_converged == 0
    for m in range(ps.n_patches):
        assert rel(med.snapshots(m).cpu().numpy(), off.R[m]) <= 1e-9, m


def test_uneven_channel_medium_large_tiles():
    """The uneven high-contrast workload (1025^2, contrast 1e3, patches of 16-96
    cells, buffers 4-24): sampled patches, the widest tiles first, against the
    oracle; every column converges within the pass limit."""
    w = synth.workload_uneven()
    ps = w["patches"]
    med = direct_medium(w["medium"], ps)
    st = med.sample(w["seed"], "mixed", tol=1e-10, max_iter=40000)
    assert st.n_not_converged == 0
    aE, aN = E.face_coefficients(w["medium"])
    patches = E.patch_boxes(1024, ps)
    order = sorted(range(len(patches)), key=lambda m: -(patches[m].X1 - patches[m].X0) * (patches[m].Y1 - patches[m].Y0))
    assert patches[order[0]].X1 - patches[order[0]].X0 - 1 > 128
    for m in order[:2] + [order[len(order) // 2], order[-1]]:
        R = E.snapshots(aE, aN, patches[m], w["seed"], 1024)
        assert rel(med.snapshots(m).cpu().numpy(), R) <= MIXED_TOL, m


def test_direct_agrees_with_cg_and_graph_replay():
    ms, ps = synth.lognormal(256, 1 / 16, 32, 3), synth.uniform_patches(256, 4, 4, 16, 48)
    cg = msp.Medium(ms, ps)
    cg.sample(5, "mixed", tol=1e-11, max_iter=20000)
    d = direct_medium(ms, ps)
    d.sample(5, "mixed", tol=1e-11, max_iter=20000)
    for m in range(ps.n_patches):
        assert rel(d.snapshots(m).cpu().numpy(), cg.snapshots(m).cpu().numpy()) <= 1e-9, m
    g = direct_medium(ms, ps)
    g.set_graph(True)
    for rep in range(3):   # direct run + capture, then replays
        st = g.sample(5, "mixed", tol=1e-11, max_iter=20000)
        assert st.n_not_converged == 0
        for m in range(ps.n_patches):
            assert np.array_equal(g.snapshots(m).cpu().numpy(), d.snapshots(m).cpu().numpy()), (rep, m)


def test_direct_mode_is_mixed_only():
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    with pytest.raises(msp.MspError):
        med.set_launch("fp64", "direct")

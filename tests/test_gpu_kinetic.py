"""GPU parity of the kinetic (discrete-ordinates) path against the CPU oracle.

Tolerances: relative L2 <= 1e-8 for the FP64 path; singular values within
1e-6 sigma_1; the exactness case (full-rank local spaces) within 1e-9 of the
global direct solve.
"""
import numpy as np
import pytest
import torch

from oracle import kinetic as K

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


SMALL = dict(n_cells=128, eps=1 / 32, n_v=8, n_patches=4, buffer=8, samples=12)


@pytest.fixture(scope="module")
def small():
    c = SMALL
    off = K.offline(c["n_cells"], c["eps"], c["n_v"], c["n_patches"], c["buffer"], c["samples"], 7, 1e-10)
    km = msp.KineticMedium(**c)
    st = km.sample(7, tol=1e-14, max_iter=200000)
    kb = km.extract(1e-10)
    return off, km, kb, st


def test_velocities(small):
    _, km, _, _ = small
    v, w = km.velocities()
    vo, wo = K.velocities(SMALL["n_v"])
    np.testing.assert_allclose(v, vo, atol=1e-15)
    np.testing.assert_allclose(w, wo, atol=1e-15)


def test_snapshots(small):
    off, km, _, st = small
    assert st.n_not_converged == 0
    for m in range(SMALL["n_patches"]):
        assert rel(km.snapshots(m).cpu().numpy(), off.R[m]) <= 1e-8, m


def test_singular_values_and_rank(small):
    off, _, kb, _ = small
    for m in range(SMALL["n_patches"]):
        s = kb.sigma(m)
        assert np.max(np.abs(s - off.sigma[m])) <= 1e-6 * off.sigma[m][0]
        assert kb.k(m) == off.Q[m].shape[1] == SMALL["n_v"]


def test_online_matches_oracle_and_global_solve(small):
    off, _, kb, _ = small
    c = SMALL
    v, _ = K.velocities(c["n_v"])
    left, right = 3 + np.sin(2 * np.pi * v), 2 + np.sin(2 * np.pi * v)
    f_ref, _ = K.online(off, c["n_cells"], c["n_v"], left, right)
    f = kb.solve(torch.tensor(np.stack([left, right]), device="cuda")).cpu().numpy()
    assert rel(f, f_ref) <= 1e-8
    g = K.global_reference(c["n_cells"], c["eps"], c["n_v"], left, right)
    assert rel(f, g) <= 1e-9


def test_batch_of_inflows(small):
    _, _, kb, _ = small
    rng = np.random.default_rng(0)
    data = rng.standard_normal((5, 2, SMALL["n_v"]))
    fb = kb.solve(torch.tensor(data, device="cuda"))
    for b in (0, 4):
        fa = kb.solve(torch.tensor(data[b], device="cuda"))
        assert torch.equal(fa, fb[b])


def test_slab_workload_sampled_patches():
    """The 8192-cell, 64-velocity workload: snapshots of sampled patches (first,
    interior, last) against the oracle."""
    c = dict(n_cells=8192, eps=2.0 ** -8, n_v=64, n_patches=64, buffer=32, samples=96)
    km = msp.KineticMedium(**c)
    st = km.sample(4, tol=1e-13, max_iter=200000)
    assert st.n_not_converged == 0 and st.n_solves == 64 * 96
    pts = K.patches(c["n_cells"], c["n_patches"], c["buffer"], c["samples"])
    for m in (0, 31, 63):
        R = K.snapshots(c["n_cells"], c["eps"], c["n_v"], pts[m], 4)
        assert rel(km.snapshots(m).cpu().numpy(), R) <= 1e-8, m
    kb = km.extract(1e-6)
    v, _ = K.velocities(c["n_v"])
    f = kb.solve(torch.tensor(np.stack([3 + np.sin(2 * np.pi * v), 2 + np.sin(2 * np.pi * v)]), device="cuda"))
    f = f.cpu().numpy()
    assert np.all(np.isfinite(f))
    # incoming data carried exactly at the ends; density between the two boundary values
    np.testing.assert_array_equal(f[0, v > 0], 3 + np.sin(2 * np.pi * v[v > 0]))
    rho = 0.5 * (f * K.velocities(64)[1]).sum(1)
    assert 1.0 < rho[4096] < 4.0


def test_mixed_precision_sweeps_match_the_oracle():
    """FP32 source-iteration corrections inside FP64 residual iteration reach the
    FP64 path's accuracy (relative L2 <= 1e-8 against the direct oracle)."""
    c = SMALL
    off = K.offline(c["n_cells"], c["eps"], c["n_v"], c["n_patches"], c["buffer"], c["samples"], 7, 1e-10)
    km = msp.KineticMedium(**c)
    st = km.sample(7, tol=1e-14, max_iter=200000, precision="mixed")
    assert st.n_not_converged == 0
    for m in range(c["n_patches"]):
        assert rel(km.snapshots(m).cpu().numpy(), off.R[m]) <= 1e-8, m


def test_mixed_precision_slab_workload():
    """The 8192-cell workload: mixed and FP64 snapshots agree to 1e-8."""
    c = dict(n_cells=8192, eps=2.0 ** -8, n_v=64, n_patches=64, buffer=32, samples=96)
    km64 = msp.KineticMedium(**c)
    km64.sample(4, tol=1e-13, max_iter=200000)
    kmx = msp.KineticMedium(**c)
    st = kmx.sample(4, tol=1e-13, max_iter=200000, precision="mixed")
    assert st.n_not_converged == 0
    for m in (0, 31, 63):
        assert rel(kmx.snapshots(m).cpu().numpy(), km64.snapshots(m).cpu().numpy()) <= 1e-8, m

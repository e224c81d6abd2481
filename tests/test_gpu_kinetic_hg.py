"""GPU parity of the anisotropic (Henyey-Greenstein, Eq. HG) kinetic path and of
the direct block-tridiagonal local solver against the CPU oracle.

Tolerances: snapshots relative L2 <= 1e-9 for both the FP64 and the FP32-factor
(mixed) direct solver, refined in FP64 to a scaled residual of 1e-13; the
exactness case of Sec. 4.3 (M = 10 patches, dx = 0.01, buffered patches twice
as long, full-rank random local spaces) within 1e-8 of the global solve.
"""
import numpy as np
import pytest
import torch

from oracle import kinetic as K

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# 40 samples: one full group of 32 lanes and a ragged group of 8
RAGGED = dict(n_cells=128, eps=1 / 16, n_v=16, n_patches=4, buffer=8, samples=40)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("g", [0.5, -0.3])
def test_hg_snapshots_match_the_oracle(precision, g):
    c = RAGGED
    km = msp.KineticMedium(**c, g=g)
    st = km.sample(11, tol=1e-13, max_iter=16, precision=precision)
    assert st.n_not_converged == 0 and st.n_solves == c["n_patches"] * c["samples"]
    assert st.max_iters <= (2 if precision == "fp64" else 5)
    pts = K.patches(c["n_cells"], c["n_patches"], c["buffer"], c["samples"])
    for m in range(c["n_patches"]):
        R = K.snapshots(c["n_cells"], c["eps"], c["n_v"], pts[m], 11, g)
        assert rel(km.snapshots(m).cpu().numpy(), R) <= 1e-9, (m, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_direct_solver_isotropic_matches_source_iteration(precision):
    """At g = 0 the direct solver and the source iteration solve the same
    system: both agree with the oracle and with each other."""
    c = dict(n_cells=128, eps=1 / 32, n_v=8, n_patches=4, buffer=8, samples=12)
    off = K.offline(c["n_cells"], c["eps"], c["n_v"], c["n_patches"], c["buffer"], c["samples"], 7, 1e-10)
    a = msp.KineticMedium(**c)
    a.sample(7, tol=1e-14, max_iter=200000, precision=precision)
    b = msp.KineticMedium(**c)
    b.set_solver("direct")
    st = b.sample(7, tol=1e-13, max_iter=16, precision=precision)
    assert st.n_not_converged == 0
    for m in range(c["n_patches"]):
        Rb = b.snapshots(m).cpu().numpy()
        assert rel(Rb, off.R[m]) <= 1e-9, m
        assert rel(Rb, a.snapshots(m).cpu().numpy()) <= 1e-9, m


@pytest.mark.parametrize("eps", [1.0, 2.0 ** -6])
def test_paper_global_test_exactness(eps):
    """Sec. 4.3 set-up: g = 1/2, M = 10 patches, dx = 0.01, buffered patches twice
    as long as the patches (5-cell margins), 120 velocities (Gauss-Legendre,
    reading of the velocity grid).  With S = 128 > 120 = n_v random data sets the
    local spaces are full and the least-squares glue reproduces the global
    solve; the GPU bases and online field match the oracle's."""
    c = dict(n_cells=100, eps=eps, n_v=120, n_patches=10, buffer=5, samples=128)
    g = 0.5
    km = msp.KineticMedium(**c, g=g)
    st = km.sample(3, tol=1e-13, max_iter=16, precision="mixed")
    assert st.n_not_converged == 0
    off = K.offline(c["n_cells"], eps, c["n_v"], c["n_patches"], c["buffer"], c["samples"], 3, 1e-12, g)
    for m in (0, 4, 9):
        assert rel(km.snapshots(m).cpu().numpy(), off.R[m]) <= 1e-9, m
    kb = km.extract(1e-12)
    v, _ = K.velocities(c["n_v"])
    left, right = 1 + 0.5 * np.sin(np.pi * v), 0.5 + v ** 2
    f = kb.solve(torch.tensor(np.stack([left, right]), device="cuda")).cpu().numpy()
    ref = K.global_reference(c["n_cells"], eps, c["n_v"], left, right, g)
    assert rel(f, ref) <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hg_slab_workload_sampled_patches(precision):
    """The 8192-cell, 64-velocity slab with g = 1/2: snapshots of the first, an
    interior and the last patch against the oracle."""
    c = dict(n_cells=8192, eps=2.0 ** -8, n_v=64, n_patches=64, buffer=32, samples=96)
    km = msp.KineticMedium(**c, g=0.5)
    st = km.sample(4, tol=1e-13, max_iter=16, precision=precision)
    assert st.n_not_converged == 0 and st.n_solves == 64 * 96
    pts = K.patches(c["n_cells"], c["n_patches"], c["buffer"], c["samples"])
    for m in (0, 31, 63):
        R = K.snapshots(c["n_cells"], c["eps"], c["n_v"], pts[m], 4, 0.5)
        assert rel(km.snapshots(m).cpu().numpy(), R) <= 1e-9, m
    # a second call reuses the factor and gives the same snapshots for the same seed
    before = km.snapshots(31).clone()
    km.sample(4, tol=1e-13, max_iter=16, precision=precision)
    assert torch.equal(before, km.snapshots(31))


def test_solver_arguments():
    from paper_1807_08848_gb300 import _native as N
    km = msp.KineticMedium(64, 0.1, 8, 2, 4, 4, g=0.5)
    with pytest.raises(N.MspError) as e:
        km.set_solver("source_iteration")
    assert e.value.status == N.MSP_ERR_INVALID_ARG
    km.set_solver("direct")
    iso = msp.KineticMedium(64, 0.1, 8, 2, 4, 4)
    iso.set_solver("direct")
    iso.set_solver("source_iteration")

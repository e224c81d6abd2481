"""GPU parity of the overlapping Schwarz variant of the online step (restricted
additive Schwarz on the buffered patches, reduced to the bases) against the CPU
oracle's direct fixed-point solve.

Tolerances: online fields within 1e-8 of the oracle on the FP64 path (GMRES to
1e-12) and 1e-6 on the mixed path; with full local spaces the fine-grid solution
to 1e-9; a data set's result is bitwise the same alone and inside a batch.
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


RAGGED = (60, synth.PatchSpec(np.array([0, 13, 37, 60]), np.array([0, 22, 41, 60]),
                              np.array([3, 1, 5, 2, 4, 1, 6, 3, 2]), np.full(9, 60)), synth.hou_wu(60, 1 / 6))
# buffers wider than the neighbouring patch: rings reach two patches away
WIDE = (72, synth.PatchSpec(np.array([0, 12, 52, 72]), np.array([0, 20, 44, 72]), np.full(9, 14), np.full(9, 80)),
        synth.lognormal(72, 1 / 6, 16, 4))


def _case(name):
    if name == "small":
        w = synth.workload_small()
        return 128, w["patches"], w["medium"], w["seed"], w["tau"], w["phi"]
    N, ps, ms = RAGGED if name == "ragged" else WIDE
    return N, ps, ms, 21, 1e-6, synth.phi_fourier(N, 6, 9, kmax=3)[0]


def _full(ms, ps):
    full = msp.Medium(ms, ps, full_basis=True)
    st = full.sample(0, "fp64", tol=1e-13, max_iter=20000)
    assert st.n_not_converged == 0
    return full


@pytest.mark.parametrize("name", ["small", "ragged", "wide"])
@pytest.mark.parametrize("coarse", [True, False], ids=["two-level", "one-level"])
def test_schwarz_matches_the_oracle(name, coarse):
    N, ps, ms, seed, tau, phi = _case(name)
    med = msp.Medium(ms, ps)
    med.sample(seed, "fp64", tol=1e-13, max_iter=20000)
    basis = med.extract(tau, "fp64")
    basis.setup_schwarz(_full(ms, ps), coarse=coarse)
    off = E.offline(ms, ps, seed, tau)
    assert [q.shape[1] for q in off.Q] == [basis.k(m) for m in range(len(off.Q))]
    u_ref, *_ = E.online_ras(off, N, phi)
    u, it = basis.solve(torch.tensor(phi, device="cuda"), tol=1e-12, max_iter=2000, schwarz=True)
    assert rel(u.cpu().numpy(), u_ref) <= 1e-8
    assert 0 < it[0] < 2000


def test_two_level_needs_fewer_iterations():
    """The coarse space leaves the answer alone and cuts the GMRES iterations on
    8 x 8 patches."""
    N = 256
    ms = synth.lognormal(N, 1 / 16, 64, 1)
    ps = synth.uniform_patches(N, 8, 8, 8, 64)
    med = msp.Medium(ms, ps)
    med.sample(0, "fp64", tol=1e-13, max_iter=20000)
    basis = med.extract(1e-6, "fp64")
    full = _full(ms, ps)
    phi = torch.tensor(synth.phi_fourier(N, 16, 3)[0], device="cuda")
    basis.setup_schwarz(full, coarse=False)
    u1, it1 = basis.solve(phi, tol=1e-12, max_iter=5000, schwarz=True)
    basis.setup_schwarz(full, coarse=True)
    u2, it2 = basis.solve(phi, tol=1e-12, max_iter=5000, schwarz=True)
    assert rel(u2.cpu().numpy(), u1.cpu().numpy()) <= 1e-9
    assert it2[0] < it1[0]


def test_schwarz_full_basis_exactness():
    """Full local spaces: the Schwarz fixed point is the fine-grid solution."""
    N = 40
    ms = synth.periodic_sin(N, 1 / 5)
    ps = synth.PatchSpec(np.array([0, 12, 28, 40]), np.array([0, 20, 40]), np.array([3, 4, 2, 5, 4, 3]),
                         np.full(6, 1))
    full = _full(ms, ps)
    basis = full.extract(1e-13, "fp64")
    basis.setup_schwarz(full, coarse=True)
    phi = synth.phi_fourier(N, 6, 9, kmax=3)[0]
    u, _ = basis.solve(torch.tensor(phi, device="cuda"), tol=1e-14, max_iter=2000, schwarz=True)
    aE, aN = E.face_coefficients(ms)
    assert rel(u.cpu().numpy(), E.global_reference(aE, aN, N, phi)) <= 1e-9


def test_schwarz_batch_alone_and_mixed_basis():
    """A data set gives the same bits alone and inside a batch (also across the
    passes of 16), and the variant runs on a basis extracted on the mixed path to
    1e-6 of the oracle."""
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    med.sample(w["seed"], "mixed", tol=1e-10, max_iter=20000)
    basis = med.extract(w["tau"], "mixed")
    basis.setup_schwarz(_full(w["medium"], w["patches"]))
    phis = synth.phi_fourier(128, 6, 5, kmax=4, batch=19)
    ub, itb = basis.solve(torch.tensor(phis, device="cuda"), tol=1e-10, max_iter=2000, schwarz=True)
    for b in (0, 7, 18):
        u1, it1 = basis.solve(torch.tensor(phis[b], device="cuda"), tol=1e-10, max_iter=2000, schwarz=True)
        assert torch.equal(u1, ub[b]) and it1[0] == itb[b]
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
    u_ref, *_ = E.online_ras(off, 128, phis[7])
    assert rel(ub[7].cpu().numpy(), u_ref) <= 1e-6


def test_schwarz_failures_are_reported():
    """Before set-up, with a medium that is not a full-basis one, at max_iter and
    for non-finite data: the status says so and the other data sets finish."""
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    med.sample(w["seed"], "fp64", tol=1e-12, max_iter=20000)
    basis = med.extract(w["tau"], "fp64")
    phi = torch.tensor(np.stack([w["phi"], w["phi"]]), device="cuda")
    with pytest.raises(N.MspError) as e:
        basis.solve(phi, schwarz=True)
    assert e.value.status == N.MSP_ERR_INVALID_ARG
    with pytest.raises(N.MspError) as e:
        basis.setup_schwarz(med)
    assert e.value.status == N.MSP_ERR_INVALID_ARG
    basis.setup_schwarz(_full(w["medium"], w["patches"]))
    with pytest.raises(N.MspError) as e:
        basis.solve(phi, tol=1e-12, max_iter=1, schwarz=True)
    assert e.value.status == N.MSP_ERR_NOT_CONVERGED
    bad = phi.clone()
    bad[1, 3] = float("nan")
    u = torch.zeros((2, 129, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(N.MspError) as e:
        basis.solve(bad, tol=1e-12, max_iter=2000, schwarz=True, u=u)
    assert e.value.status == N.MSP_ERR_NOT_CONVERGED
    good, _ = basis.solve(phi[0], tol=1e-12, max_iter=2000, schwarz=True)
    assert torch.equal(u[0], good)

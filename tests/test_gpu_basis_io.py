"""GPU checks of basis persistence and of the exported online system: a basis
written and read back gives bit-identical online results; P~ and d exported by
the library agree with the oracle's assembly (Eq. elliptic_cond_reduced, readings
R6-R8) from the same bases, compared through the row-order and row-sign
invariant P~^T P~ and P~^T d (relative 1e-12)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")


@pytest.fixture(scope="module")
def basis():
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    med.sample(w["seed"], "fp64", tol=1e-13, max_iter=20000)
    return w, med, med.extract(w["tau"], "fp64")


def test_saved_and_loaded_basis_solves_identically(basis, tmp_path):
    w, _, b = basis
    path = tmp_path / "small.mspb"
    b.save(path)
    b2 = msp.Basis.load(path)
    assert (b2.n_cells, b2.n_patches, b2.n_unknowns, b2.n_rows) == (b.n_cells, b.n_patches, b.n_unknowns, b.n_rows)
    for m in (0, 5, 15):
        assert b2.k(m) == b.k(m)
        assert np.array_equal(b2.sigma(m), b.sigma(m))
        assert torch.equal(b2.Q(m), b.Q(m))
    phi = torch.tensor(synth.phi_fourier(128, 16, 3, batch=3), device="cuda")
    u1, _ = b.solve(phi, tol=1e-12, max_iter=5000)
    u2, _ = b2.solve(phi, tol=1e-12, max_iter=5000)
    assert torch.equal(u1, u2)


def test_exported_online_system_matches_the_oracle(basis):
    w, med, b = basis
    N = 128
    aE, aN = E.face_coefficients(w["medium"])
    patches = E.patch_boxes(N, w["patches"])
    Qs = [b.Q(m).cpu().numpy() for m in range(b.n_patches)]
    Pm, d, _ = E.online_system(aE, aN, patches, Qs, N, w["patches"], w["phi"])
    r, c, v, dg = b.online_system(w["phi"])
    Pg = sp.csr_matrix((v, (r, c)), shape=(b.n_rows, b.n_unknowns))
    assert Pg.shape == Pm.shape
    H, Hg = (Pm.T @ Pm).toarray(), (Pg.T @ Pg).toarray()
    assert np.abs(Hg - H).max() <= 1e-12 * np.abs(H).max()
    g, gg = Pm.T @ d, Pg.T @ dg
    assert np.linalg.norm(gg - g) <= 1e-12 * np.linalg.norm(g)
    assert np.sort(np.abs(dg)).tolist() == pytest.approx(np.sort(np.abs(d)).tolist(), abs=0)

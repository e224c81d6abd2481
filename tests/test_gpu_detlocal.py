"""DetLocalSolu on the GPU and the paper's local and global experiments of
Sec. 5.3 as regression checks, against the oracle.

Setup of the paper's elliptic test: [0,1]^2, the two-scale medium with
eps = 2^-4, 5 x 5 patches of 20 x 20 fine cells (h = 1/100), buffered patches
twice as long (a buffer of 10 cells on every side); the (2,2) patch is read as
the centre patch (zero-based (2,2), m = 12), which has the whole buffer.

* The full Green's matrices (DetLocalSolu: one delta per ring node) of the
  buffered patch, G~ (Eq. lr2), and of the patch itself, G (Eq. lr3, buffer 0),
  against the oracle's sparse direct solves; the sampled snapshots equal
  G~ Omega (Sec. 3.3) on the GPU's own data.
* Singular values of G~ and G against the oracle (within 1e-6 sigma_1), with the
  decay the paper reports: fast with the buffer, slow without.
* The range error |G~ - Q Q^T G~|_2 / |G~|_2 with Q from the QR of the first k
  sampled columns, k = 1..50: the GPU's curve against the oracle's, never below
  the optimal sigma_{k+1} / sigma_1, decaying exponentially.
* The global test: with the full basis the online least-squares solution is the
  fine-grid solution (the full-basis exactness of Eq. elliptic_cond); with k_m
  random samples the GPU's global error matches the oracle's and falls quickly.
Each figure of the paper is only plotted, so no value of the paper is stored:
the oracle gives the numbers and the paper the shape of the curves.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")

N = 100
PATCH = 12
SEED = 3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def faces():
    return E.face_coefficients(synth.hou_wu(N, 2.0 ** -4))


def full_medium(buffer, precision="fp64", tol=1e-13):
    med = msp.Medium(synth.hou_wu(N, 2.0 ** -4), synth.uniform_patches(N, 5, 5, buffer, 1), full_basis=True)
    st = med.sample(0, precision, tol=tol, max_iter=20000)
    assert st.n_not_converged == 0
    return med


@pytest.mark.parametrize("precision,tol,check", [("fp64", 1e-13, 1e-8), ("mixed", 1e-12, 1e-6)])
@pytest.mark.parametrize("buffer", [10, 0])
def test_full_green_matrices(faces, buffer, precision, tol, check):
    aE, aN = faces
    med = full_medium(buffer, precision, tol)
    info = med.patch(PATCH)
    assert info.samples == 0 and info.cols == info.n_ring == info.n_b
    P = E.patch_boxes(N, synth.uniform_patches(N, 5, 5, buffer, 1))[PATCH]
    G = E.full_green(aE, aN, P)
    assert rel(med.snapshots(PATCH).cpu().numpy(), G) <= check
    # a boundary patch as well: its ring reaches the domain boundary
    P0 = E.patch_boxes(N, synth.uniform_patches(N, 5, 5, buffer, 1))[0]
    assert rel(med.snapshots(0).cpu().numpy(), E.full_green(aE, aN, P0)) <= check


def test_sampled_snapshots_are_green_times_samples():
    """G^r = G~ Omega (Sec. 3.3) on the GPU's own data: the Gaussian snapshots of
    the centre patch against its full Green's matrix times its ring samples."""
    ps = synth.uniform_patches(N, 5, 5, 10, 30)
    med = msp.Medium(synth.hou_wu(N, 2.0 ** -4), ps)
    med.sample(SEED, "fp64", tol=1e-13, max_iter=20000)
    full = full_medium(10)
    Gt = full.snapshots(PATCH).cpu().numpy()
    Om = med.samples(PATCH, SEED).cpu().numpy()
    Gr = med.snapshots(PATCH).cpu().numpy()
    assert rel(Gr, Gt @ Om) <= 1e-10


def test_singular_value_decay_with_and_without_buffer(faces):
    aE, aN = faces
    out = {}
    for buffer in (10, 0):
        med = full_medium(buffer)
        basis = med.extract(1e-8, "fp64")       # sigma() returns every singular value, kept or not
        s = basis.sigma(PATCH)
        P = E.patch_boxes(N, synth.uniform_patches(N, 5, 5, buffer, 1))[PATCH]
        so = np.linalg.svd(E.full_green(aE, aN, P), compute_uv=False)
        assert s.shape == so.shape
        assert np.max(np.abs(s - so)) <= 1e-6 * so[0]
        out[buffer] = s / s[0]
    # the buffer makes G~ nearly low rank; without it the spectrum stays flat
    assert out[10][20] < 1e-3 and out[10][40] < 1e-5
    assert out[0][20] > 0.1 and out[0][40] > 0.1
    assert out[10][20] < 1e-2 * out[0][20]


def test_range_error_of_the_random_basis(faces):
    aE, aN = faces
    ps = synth.uniform_patches(N, 5, 5, 10, 50)
    med = msp.Medium(synth.hou_wu(N, 2.0 ** -4), ps)
    med.sample(SEED, "fp64", tol=1e-13, max_iter=20000)
    Gr = med.snapshots(PATCH).cpu().numpy()
    Gt = full_medium(10).snapshots(PATCH).cpu().numpy()
    P = E.patch_boxes(N, ps)[PATCH]
    Gt_o = E.full_green(aE, aN, P)
    Gr_o = E.snapshots(aE, aN, P, SEED, N)
    s = np.linalg.svd(Gt_o, compute_uv=False)

    def curve(Gr_, Gt_):
        out = []
        for k in range(1, 51):
            Q, _ = np.linalg.qr(Gr_[:, :k])
            out.append(np.linalg.norm(Gt_ - Q @ (Q.T @ Gt_), 2) / np.linalg.norm(Gt_, 2))
        return np.array(out)

    e_gpu, e_or = curve(Gr, Gt), curve(Gr_o, Gt_o)
    assert np.max(np.abs(e_gpu - e_or)) <= 1e-6
    ks = np.arange(1, 51)
    assert np.all(e_gpu >= s[ks] / s[0] * (1 - 1e-6))       # no basis of k columns does better
    assert e_gpu[9] < 0.1 and e_gpu[29] < 1e-3 and e_gpu[49] < 1e-5
    assert e_gpu[49] < 1e-4 * e_gpu[9]


def test_global_full_basis_is_the_fine_solution_and_random_error_curve(faces):
    aE, aN = faces
    phi = synth.phi_sin_cos(N)
    u_ref = E.global_reference(aE, aN, N, phi)
    full = full_medium(10)
    # the full basis truncated at 1e-10: the directions below it are numerically
    # null and would leave the normal matrix of the online system singular
    basis = full.extract(1e-10, "fp64")
    u, _ = basis.solve(torch.tensor(phi, device="cuda"), tol=1e-12, max_iter=20000)
    assert rel(u.cpu().numpy(), u_ref) <= 1e-8
    errs = []
    # the online least squares with k_m random columns has a large residual at
    # k_m = 10 (error 0.3 against the fine grid): CGLS stopped at a normal-equation
    # residual of 1e-12 leaves about cond(P)^2 1e-12 in the solution there, so the
    # GPU and the oracle's direct solve agree to 1e-5; at k_m = 50 to 1e-7
    for km, bound in ((10, 1e-5), (50, 1e-7)):
        ps = synth.uniform_patches(N, 5, 5, 10, km)
        med = msp.Medium(synth.hou_wu(N, 2.0 ** -4), ps)
        med.sample(SEED, "fp64", tol=1e-13, max_iter=20000)
        b = med.extract(1e-10, "fp64")
        u, _ = b.solve(torch.tensor(phi, device="cuda"), tol=1e-12, max_iter=20000)
        off = E.offline(synth.hou_wu(N, 2.0 ** -4), ps, SEED, 1e-10)
        assert all(b.k(m) == off.Q[m].shape[1] for m in range(25)), km
        u_or, *_ = E.online(off, ps, N, phi)
        assert rel(u.cpu().numpy(), u_or) <= bound, km
        errs.append(rel(u.cpu().numpy(), u_ref))
    assert errs[0] > 0.1 and errs[1] < 1e-4

"""GPU parity at the sizes of the measured workloads, against the CPU oracle.

* The 513^2 log-normal medium (eps = 2^-5, 8 x 8 patches of 64 cells, 16-cell
  buffers, 128 samples: the same buffered tiles, 97 x 97 nodes, as the 2049^2
  workload the benchmark times, and the smallest medium of the serving
  workload): the whole pipeline -- local solves, bases, online least squares
  (Eq. elliptic_cond_reduced), reconstruction -- against the oracle's direct
  solves, for the plain FP64 path (relative L2 <= 1e-8) and the mixed path
  (<= 1e-6), with principal angles of the mixed bases; the serving form (the
  FP32 boundary-to-coefficient map on the tensor cores, alone and through the
  request loop) against the oracle's FP64 online solution (<= 1e-6); the
  overlapping Schwarz variant of the online step against the oracle's direct
  fixed-point solve (<= 1e-6, mixed-path basis).
* The 8192-cell slab transport workload (64 Gauss-Legendre velocities, 64
  patches, 96 samples): the online field of Eq. rte_cond_reduced against the
  oracle (FP64 path <= 1e-8, mixed sweeps <= 1e-6).

The oracle runs on the host (about a minute each for the two workloads); the
truncation margins were checked: no sigma_i / sigma_1 of either workload lies
within 0.05% of tau = 1e-6, far outside the GPU's sigma error at these
tolerances, so both sides keep the same k_m.
"""
import time

import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E
from oracle import kinetic as K

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")

FP64_TOL = 1e-8
MIXED_TOL = 1e-6


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_principal_angle(Qa, Qb):
    s = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0))) if s.size else 0.0


def wedin_dims(sig, err, bound=1e-6):
    return [j for j in range(1, len(sig)) if sig[j - 1] > sig[j] and err / (sig[j - 1] - sig[j]) <= bound]


N513 = 512
SEED513 = 1


@pytest.fixture(scope="module")
def oracle513():
    ms = synth.lognormal(N513, 2.0 ** -5, 64, 11)
    ps = synth.uniform_patches(N513, 8, 8, 16, 128)
    off = E.offline(ms, ps, SEED513, 1e-6)
    phis = np.concatenate([synth.phi_sin_cos(N513)[None], synth.phi_fourier(N513, 16, 77, batch=2)])
    refs = [E.online(off, ps, N513, phi)[0] for phi in phis]
    return ms, ps, off, phis, refs


@pytest.mark.parametrize("precision,local_tol,check", [("fp64", 1e-12, FP64_TOL), ("mixed", 1e-11, MIXED_TOL)])
def test_513_pipeline(oracle513, precision, local_tol, check):
    ms, ps, off, phis, refs = oracle513
    med = msp.Medium(ms, ps)
    st = med.sample(SEED513, precision, tol=local_tol, max_iter=20000)
    assert st.n_not_converged == 0
    for m in (0, 3, 27, 63):                      # corner, edge and interior patches
        assert rel(med.snapshots(m).cpu().numpy(), off.R[m]) <= check, m
    basis = med.extract(1e-6, precision)
    for m in range(64):
        assert basis.k(m) == off.Q[m].shape[1], m
        assert np.max(np.abs(basis.sigma(m) - off.sigma[m])) <= 1e-6 * off.sigma[m][0], m
    if precision == "mixed":
        for m in (0, 9, 36, 63):
            Qg = basis.Q(m).cpu().numpy()
            err = float(np.linalg.norm(med.snapshots(m).cpu().numpy() - off.R[m]))
            dims = [j for j in wedin_dims(off.sigma[m], err) if j <= Qg.shape[1]]
            assert dims, m
            for j in dims:
                assert max_principal_angle(Qg[:, :j], off.Q[m][:, :j]) <= 1e-5, (m, j)
    u, it = basis.solve(torch.tensor(phis, device="cuda"), tol=1e-12, max_iter=5000)
    u = u.cpu().numpy()
    for b in range(len(phis)):
        assert rel(u[b], refs[b]) <= check, b


def test_513_serving_against_the_oracle(oracle513):
    """The map (FP32, tensor-core GEMM) built on the mixed-path basis: single and
    batched map solves and results that came through the request loop, each
    against the oracle's FP64 online solution of the same data."""
    ms, ps, off, phis, refs = oracle513
    med = msp.Medium(ms, ps)
    med.sample(SEED513, "mixed", tol=1e-11, max_iter=20000)
    basis = med.extract(1e-6, "mixed")
    basis.build_map(tol=1e-11, max_iter=5000)
    ub = basis.solve_map(torch.tensor(phis, device="cuda")).cpu().numpy()
    for b in range(len(phis)):
        assert rel(ub[b], refs[b]) <= MIXED_TOL, b
    srv = msp.Server([basis], mem_budget_bytes=1 << 30, max_slots=16, max_batch=4, n_workers=1)
    try:
        ids = [srv.submit(0, p) for p in phis]
        got = []
        for rid in ids:
            t0 = time.time()
            while srv.poll(rid)[0] == 0:
                assert time.time() - t0 < 60
                time.sleep(0.001)
            got.append(srv.fetch(rid, 0))
    finally:
        srv.close()
    for b in range(len(phis)):
        assert rel(got[b], refs[b]) <= MIXED_TOL, b


def test_513_schwarz_against_the_oracle(oracle513):
    """The overlapping Schwarz variant of the online step at 513^2 (the bench's
    tiles), two-level GMRES on the mixed-path basis, against the oracle's direct
    fixed-point solve of the same data on its FP64 bases (<= 1e-6)."""
    ms, ps, off, phis, refs = oracle513
    med = msp.Medium(ms, ps)
    med.set_launch("mixed", "direct")
    med.sample(SEED513, "mixed", tol=1e-11, max_iter=20000)
    basis = med.extract(1e-6, "mixed")
    full = msp.Medium(ms, ps, full_basis=True)
    full.set_launch("mixed", "direct")
    st = full.sample(0, "mixed", tol=1e-11, max_iter=20000)
    assert st.n_not_converged == 0
    basis.setup_schwarz(full, coarse=True)
    del full
    u, it = basis.solve(torch.tensor(phis, device="cuda"), tol=1e-12, max_iter=2000, schwarz=True)
    u = u.cpu().numpy()
    T, F, o = E.ras_operators(off.aE, off.aN, off.patches, off.Q, N513)
    for b in (0, 2):
        u_ref = E.reconstruct(off.patches, off.Q, E.ras_solve(T, F, phis[b]), o, N513, phis[b])
        assert rel(u[b], u_ref) <= MIXED_TOL, b
        # a different reading of the online step than the least-squares glue
        assert rel(u[b], refs[b]) <= 1e-2, b


KIN = dict(n_cells=8192, eps=2.0 ** -8, n_v=64, n_patches=64, buffer=32, samples=96)


@pytest.fixture(scope="module")
def oracle_slab():
    c = KIN
    off = K.offline(c["n_cells"], c["eps"], c["n_v"], c["n_patches"], c["buffer"], c["samples"], 4, 1e-6)
    v, _ = K.velocities(c["n_v"])
    left, right = 3 + np.sin(2 * np.pi * v), 2 + np.sin(2 * np.pi * v)
    f_ref, _ = K.online(off, c["n_cells"], c["n_v"], left, right)
    return off, left, right, f_ref


@pytest.mark.parametrize("precision,check", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_slab_online_field(oracle_slab, precision, check):
    off, left, right, f_ref = oracle_slab
    km = msp.KineticMedium(**KIN)
    st = km.sample(4, tol=1e-13, max_iter=200000, precision=precision)
    assert st.n_not_converged == 0
    kb = km.extract(1e-6)
    for m in range(KIN["n_patches"]):
        assert kb.k(m) == off.Q[m].shape[1], m
    f = kb.solve(torch.tensor(np.stack([left, right]), device="cuda")).cpu().numpy()
    assert rel(f, f_ref) <= check

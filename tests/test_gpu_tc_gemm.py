"""The FP64 products of the extraction on the tensor cores (error-free BF16
slicing, tcgen05 kind::f16) against the same extraction on the CUDA cores' FP64
FMA kernels, and both against the oracle; likewise the Jacobi SVD started by
FP32 sweeps (re-orthogonalised in FP64), or by a pivoted QR, against plain FP64
sweeps.

The Gram and triangular products of Cholesky-QR and the projection onto the
singular vectors (Sec. 3.2, Eq. svd; the QR remark of Sec. 3.3) are FP64-accurate
either way, so the bases agree far inside the parity bounds: singular values to
1e-10 sigma_1 (the shifted Cholesky-QR leaves the smallest, near 1e-10 sigma_1, that sensitive), bases as orthonormal as the CUDA-core engine's, principal angles of the leading
subspaces to 1e-11 sigma_1 / gap (sine of the largest principal angle), online fields (Eq. elliptic_cond_reduced) to 1e-9 (the CGLS stopping error); against
the oracle the usual bounds hold (sigma 1e-6 sigma_1, online field 1e-8 for the
plain FP64 path)."""
import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def sin_angle(Qa, Qb):
    """Sine of the largest principal angle, |(I - Qa Qa^T) Qb|_2: unlike the arccos
    of the smallest singular value of Qa^T Qb it stays accurate for tiny angles
    (a basis orthonormal to 1e-12 puts that cosine 1e-12 below 1, whose arccos
    reads 1.5e-6)."""
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2)) if Qb.size else 0.0


def extract_both(med, tau, precision, switch="engine"):
    """Two extractions of the same snapshots: (reference setting, setting under
    test) -- CUDA-core vs tensor-core products, or FP64 vs FP32-started Jacobi."""
    set_, ref, new, default = {"engine": (msp.set_gemm_engine, "cuda_cores", "tensor_cores", "tensor_cores"),
                               "svd": (msp.set_svd_mode, "fp64", "fp32_preconditioned", "qr_preconditioned"),
                               "svd_qr": (msp.set_svd_mode, "fp64", "qr_preconditioned", "qr_preconditioned")}[switch]
    try:
        set_(ref)
        b_cc = med.extract(tau, precision)
        set_(new)
        b_tc = med.extract(tau, precision)
    finally:
        set_(default)
    return b_cc, b_tc


@pytest.mark.parametrize("switch", ["engine", "svd", "svd_qr"])
@pytest.mark.parametrize("case", ["small", "lognormal-256", "ragged"])
def test_engines_agree_and_match_the_oracle(case, switch):
    if case == "small":
        w = synth.workload_small()
        ms, ps, seed, tau, N = w["medium"], w["patches"], w["seed"], w["tau"], 128
    elif case == "lognormal-256":
        ms, ps, seed, tau, N = synth.lognormal(256, 1 / 16, 32, 3), synth.uniform_patches(256, 4, 4, 16, 64), 5, 1e-6, 256
    else:
        N = 60
        ps = synth.PatchSpec(np.array([0, 13, 37, 60]), np.array([0, 22, 41, 60]),
                             np.array([3, 0, 5, 2, 4, 1, 6, 3, 2]), np.array([9, 17, 5, 12, 30, 7, 11, 8, 20]))
        ms, seed, tau = synth.hou_wu(N, 1 / 6), 21, 1e-6
    med = msp.Medium(ms, ps)
    med.sample(seed, "fp64", tol=1e-13, max_iter=20000)
    b_cc, b_tc = extract_both(med, tau, "fp64", switch)
    off = E.offline(ms, ps, seed, tau)
    for m in range(ps.n_patches):
        s_cc, s_tc = b_cc.sigma(m), b_tc.sigma(m)
        # singular values resolved by the sweeps: pairs of columns both below
        # 1e-3 tau |T|_F / sqrt(c) (<= 1e-3 tau sigma_1) are left unrotated by design,
        # so values 1e5 below the truncation level depend on the starting basis; at
        # 0.1 tau sigma_1 and above they agree to 1e-10 sigma_1, and the rest stay
        # below the truncation level in both
        res = s_cc >= 0.1 * tau * s_cc[0]
        assert np.max(np.abs(s_tc - s_cc)[res]) <= 1e-10 * s_cc[0], m
        assert np.all(s_tc[~res] < tau * s_cc[0]), m
        assert np.max(np.abs(s_tc - off.sigma[m])) <= 1e-6 * off.sigma[m][0], m
        assert b_tc.k(m) == b_cc.k(m) == off.Q[m].shape[1], m
        Qt, Qc = b_tc.Q(m).cpu().numpy(), b_cc.Q(m).cpu().numpy()
        # orthonormality as good as the CUDA-core engine's (blocks with boundary-delta
        # columns keep about 1e-11 in either engine)
        o_tc = float(np.abs(Qt.T @ Qt - np.eye(Qt.shape[1])).max())
        o_cc = float(np.abs(Qc.T @ Qc - np.eye(Qc.shape[1])).max())
        assert o_tc <= 10.0 * o_cc + 1e-13, (m, o_tc, o_cc)
        # leading subspaces separated from the rest by a relative gap of 1e-3: both
        # engines are backward stable to about 1e-12 sigma_1 (shifted Cholesky-QR on
        # the rank-deficient corner blocks), so by Wedin's bound the subspaces agree
        # to 1e-11 sigma_1 / gap
        s = off.sigma[m]
        for j in range(1, Qt.shape[1]):
            gap = s[j - 1] - s[j]
            if gap > 1e-3 * s[0]:
                assert sin_angle(Qt[:, :j], Qc[:, :j]) <= 1e-11 * s[0] / gap, (m, j)
    phi = torch.tensor(synth.phi_sin_cos(N), device="cuda")
    u_cc, _ = b_cc.solve(phi, tol=1e-12, max_iter=20000)
    u_tc, _ = b_tc.solve(phi, tol=1e-12, max_iter=20000)
    assert rel(u_tc.cpu().numpy(), u_cc.cpu().numpy()) <= 1e-9     # each within the CGLS stopping error of the LS solution
    u_ref, *_ = E.online(off, ps, N, synth.phi_sin_cos(N))
    assert rel(u_tc.cpu().numpy(), u_ref) <= 1e-8


def test_engine_argument():
    with pytest.raises(KeyError):
        msp.set_gemm_engine("other")
    from paper_1807_08848_gb300 import _native as N
    assert N.load().msp_set_gemm_engine(7) == N.MSP_ERR_INVALID_ARG
    assert N.load().msp_set_svd_mode(7) == N.MSP_ERR_INVALID_ARG


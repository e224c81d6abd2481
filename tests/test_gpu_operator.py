"""GPU checks of the streaming matrix-free operator against the oracle's sparse
operator blocks (A_II x_I + A_IB x_B on every buffered box).

Tolerances: FP64 tiles to 1e-13 relative (rounding of a 5-term sum); FP32
tiles to 1e-5 relative to the norm of the terms (single-precision faces and
data)."""
import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")


def oracle_apply(aE, aN, P, tile):
    A_II, A_IB = E.box_operator(aE, aN, P.X0, P.X1, P.Y0, P.Y1)
    ring = E.ring_nodes(P.X0, P.X1, P.Y0, P.Y1)
    xI = tile[1:-1, 1:-1].reshape(-1)
    xB = tile[ring[:, 1] - P.Y0, ring[:, 0] - P.X0]
    return (A_II @ xI + A_IB @ xB).reshape(P.Y1 - P.Y0 - 1, P.X1 - P.X0 - 1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("uneven", [False, True])
def test_operator_matches_oracle(precision, uneven):
    if uneven:
        ms = synth.channels(128, 1 / 16, 4, 2)
        ps = synth.uneven_patches(128, 2)
    else:
        ms = synth.lognormal(128, 1 / 16, 32, 3)
        ps = synth.uniform_patches(128, 4, 4, 8, 8)
    med = msp.Medium(ms, ps)
    rows, cols = med.tile_shape()
    pitch = (cols + 3) // 4 * 4 + 4
    S = 5
    dt = torch.float64 if precision == "fp64" else torch.float32
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((med.n_patches, S, rows, pitch), generator=g, dtype=torch.float64).to(dt).cuda()
    y = med.apply_operator(x, precision).cpu().double().numpy()
    xs = x.cpu().double().numpy()
    aE, aN = E.face_coefficients(ms)
    patches = E.patch_boxes(128, ps)
    tol = 1e-13 if precision == "fp64" else 1e-5
    for m in range(med.n_patches):
        P = patches[m]
        h, w = P.Y1 - P.Y0 + 1, P.X1 - P.X0 + 1
        for s in (0, S - 1):
            ref = oracle_apply(aE, aN, P, xs[m, s, :h, :w])
            got = y[m, s]
            scale = np.abs(xs[m, s, :h, :w]).max() * max(aE.max(), aN.max()) * 8
            assert np.max(np.abs(got[1:h - 1, 1:w - 1] - ref)) <= tol * scale, (m, s)
            # ring and padding are zero
            mask = np.ones_like(got, dtype=bool)
            mask[1:h - 1, 1:w - 1] = False
            assert np.all(got[mask] == 0.0)


def test_operator_rejects_bad_pitch():
    med = msp.Medium(synth.lognormal(64, 1 / 8, 8, 1), synth.uniform_patches(64, 2, 2, 4, 4))
    rows, cols = med.tile_shape()
    x = torch.zeros((4, 2, rows, cols + 1 if (cols + 1) % 4 else cols + 2), dtype=torch.float32, device="cuda")
    with pytest.raises(msp.MspError):
        med.apply_operator(x, "mixed")

"""CPU checks of the seeded synthetic inputs: every workload has the sizes,
partitions, sample counts and value distributions its recipe states, the draws
are reproducible from their seeds, and the shared layout conventions (the
counter-clockwise boundary ring, patch numbering with p fastest) hold.  The
Gaussian boundary samples of the local solves are not drawn here (each side
implements the counter-based generator itself); their tests are in
test_oracle_philox.py."""
import math

import numpy as np
import pytest

import synth
from oracle import elliptic as E


def test_batched_workload_sizes():
    w = synth.workload_batched()
    m, p = w["medium"], w["patches"]
    assert m.kind == synth.MEDIUM_LOGNORMAL and m.n_cells == 2048 and m.eps == 2.0 ** -7
    assert m.modes.shape == (64, 4) and m.norm == pytest.approx(1 / 8)
    assert np.array_equal(p.x_breaks, np.arange(33) * 64) and np.array_equal(p.y_breaks, np.arange(33) * 64)
    assert np.all(p.buffers == 16) and np.all(p.samples == 128)
    # 131072 Gaussian columns plus one delta column per buffered-ring node on the domain boundary
    boxes = E.patch_boxes(2048, p)
    deltas = sum(len(E.domain_boundary_ring_positions(b, 2048)) for b in boxes)
    assert int(p.samples.sum()) == 131072 and deltas == 12284


def test_lognormal_wave_vectors_in_the_annulus():
    m = synth.lognormal(2048, 2.0 ** -7, 64, 1)
    r = np.hypot(m.modes[:, 0], m.modes[:, 1])
    assert np.all(r >= 1.0) and np.all(r <= 128.0 + 1e-12)
    assert np.all(m.modes[:, :2] == np.rint(m.modes[:, :2]))       # integer lattice points
    a = m.modes[:, 2:].ravel()                                      # N(0,1) amplitudes
    assert abs(a.mean()) < 0.4 and 0.6 < a.std() < 1.4


def test_small_and_kinetic_workloads():
    w = synth.workload_small()
    assert w["medium"].kind == synth.MEDIUM_PERIODIC_SIN and w["medium"].n_cells == 128
    p = w["patches"]
    assert p.nx == 4 and p.ny == 4 and np.all(p.buffers == 8) and np.all(p.samples == 40)
    k = synth.workload_kinetic()
    assert (k["n_cells"], k["n_v"], k["n_patches"], k["buffer"], k["samples"]) == (8192, 64, 64, 32, 96)
    assert k["eps"] == 2.0 ** -8


def test_uneven_partition_recipe():
    p = synth.uneven_patches(1024, 2)
    for br in (p.x_breaks, p.y_breaks):
        assert br[0] == 0 and br[-1] == 1024 and np.all(np.diff(br) > 0)
        w = np.diff(br)
        assert np.all(w >= 16)
        assert np.all(np.isin(w[:-2], (16, 32, 48, 64, 80, 96)))   # the last two may be clipped or merged
    for q in range(p.ny):
        for pp in range(p.nx):
            wx = p.x_breaks[pp + 1] - p.x_breaks[pp]
            wy = p.y_breaks[q + 1] - p.y_breaks[q]
            assert p.buffers[pp + q * p.nx] == min(wx, wy) // 4
    assert np.all(np.isin(p.samples, (64, 128, 192, 256)))


def test_draws_are_reproducible_from_seeds():
    a, b = synth.lognormal(512, 2.0 ** -5, 64, 11), synth.lognormal(512, 2.0 ** -5, 64, 11)
    assert np.array_equal(a.modes, b.modes)
    assert not np.array_equal(a.modes, synth.lognormal(512, 2.0 ** -5, 64, 12).modes)
    u1, u2 = synth.uneven_patches(1024, 2), synth.uneven_patches(1024, 2)
    assert np.array_equal(u1.x_breaks, u2.x_breaks) and np.array_equal(u1.samples, u2.samples)
    assert np.array_equal(synth.phi_fourier(64, 16, 3, batch=4), synth.phi_fourier(64, 16, 3, batch=4))


def test_domain_ring_is_counter_clockwise_and_complete():
    N = 16
    x, y = synth.domain_ring_xy(N)
    assert x.size == 4 * N and (x[0], y[0]) == (0.0, 0.0)
    pts = {(round(a * N), round(b * N)) for a, b in zip(x, y)}
    assert len(pts) == 4 * N
    assert pts == {(i, j) for i in range(N + 1) for j in range(N + 1) if i in (0, N) or j in (0, N)}
    # consecutive nodes are grid neighbours, and the signed area is positive (counter-clockwise)
    steps = np.abs(np.diff(np.r_[x, x[0]])) + np.abs(np.diff(np.r_[y, y[0]]))
    assert np.allclose(steps, 1.0 / N)
    area = 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    assert area == pytest.approx(1.0)
    # the oracle's ring of the whole domain lists the same nodes in the same order
    ring = E.ring_nodes(0, N, 0, N)
    assert np.array_equal(ring[:, 0], np.rint(x * N)) and np.array_equal(ring[:, 1], np.rint(y * N))


def test_boundary_data():
    N = 64
    x, y = synth.domain_ring_xy(N)
    assert np.allclose(synth.phi_sin_cos(N), np.sin(2 * np.pi * x) + np.cos(2 * np.pi * y))
    phi = synth.phi_fourier(N, 16, 3, batch=256)
    assert phi.shape == (256, 4 * N)
    # each data set is a sum of 16 unit-variance modes scaled by 1/4: unit variance on average
    assert 0.7 < phi.var() < 1.3 and abs(phi.mean()) < 0.15


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(2000.0, 20000, 3)
    assert np.all(np.diff(t) > 0)
    assert t[-1] / t.size == pytest.approx(1 / 2000.0, rel=0.03)
    gaps = np.diff(t)
    assert gaps.std() / gaps.mean() == pytest.approx(1.0, rel=0.05)   # exponential gaps


def test_serving_media():
    w = synth.workload_serving()
    assert w["rate_hz"] == 2000.0 and len(w["media"]) == 3
    for med, (N, eps) in zip(w["media"], ((512, 2.0 ** -5), (1024, 2.0 ** -6), (2048, 2.0 ** -7))):
        assert med["medium"].n_cells == N and med["medium"].eps == eps
        p = med["patches"]
        assert p.nx == N // 64 and np.all(np.diff(p.x_breaks) == 64)
        assert np.all(p.buffers == 16) and np.all(p.samples == 128)


def test_kinetic_paper_inflow():
    v = np.linspace(-1, 1, 9)
    left, right = synth.kinetic_inflow_paper(v)
    assert np.allclose(left, 3 + np.sin(2 * math.pi * v)) and np.allclose(right, 2 + np.sin(2 * math.pi * v))

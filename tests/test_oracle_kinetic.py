"""Pins of the kinetic (discrete-ordinates) oracle against facts the transport
equation and the quadrature fix."""
import numpy as np
import pytest

from oracle import kinetic as K


def test_gauss_legendre_quadrature():
    """Weights sum to 2, first moment vanishes, second moment is 2/3 (exact for
    polynomials of degree < 2 n_v)."""
    v, w = K.velocities(64)
    assert abs(w.sum() - 2.0) < 1e-13
    assert abs((w * v).sum()) < 1e-14
    assert abs((w * v ** 2).sum() - 2.0 / 3.0) < 1e-14
    assert abs((w * v ** 10).sum() - 2.0 / 11.0) < 1e-13
    assert np.all(np.diff(v) > 0) and np.all(v != 0)


def test_constant_inflow_is_equilibrium():
    """f = 1 everywhere is the solution for unit incoming data (rho = f)."""
    n_v = 8
    F = K.range_solve(64, 1 / 16, n_v, 0, 64, np.ones(n_v))
    np.testing.assert_allclose(F, 1.0, atol=1e-12)


def test_free_streaming_limit():
    """Without collisions (1/eps = 0) the upwind scheme carries the incoming
    data unchanged along each characteristic."""
    n_v = 8
    g = np.arange(1, n_v + 1, dtype=float)
    F = K.range_solve(32, 1e300, n_v, 3, 20, g)
    v, _ = K.velocities(n_v)
    pos, neg = np.nonzero(v > 0)[0], np.nonzero(v < 0)[0]
    for t, l in enumerate(pos):
        np.testing.assert_allclose(F[:, l], g[t], rtol=1e-12)
    for t, l in enumerate(neg):
        np.testing.assert_allclose(F[:, l], g[len(pos) + t], rtol=1e-12)


def test_discrete_flux_is_conserved():
    """Pure scattering conserves particles: summing the upwind equations with
    the weights w_l gives J_{i+1/2} = sum_{v>0} w v f_i + sum_{v<0} w v f_{i+1}
    constant in i (the collision terms cancel since sum_l w_l = 2 and
    rho = sum w f / 2)."""
    n_v = 16
    rng = np.random.default_rng(2)
    g = rng.uniform(0.0, 3.0, n_v)
    F = K.range_solve(128, 1 / 32, n_v, 0, 128, g)
    v, w = K.velocities(n_v)
    p, n = v > 0, v < 0
    J = (F[:-1][:, p] * (w * v)[p]).sum(1) + (F[1:][:, n] * (w * v)[n]).sum(1)
    np.testing.assert_allclose(J, J[0], rtol=1e-11, atol=1e-12)


def test_positivity():
    """Positive incoming data gives a positive solution (M-matrix)."""
    n_v = 8
    rng = np.random.default_rng(3)
    F = K.range_solve(64, 1 / 64, n_v, 0, 64, rng.uniform(0.1, 1.0, n_v))
    assert F.min() > 0


def test_diffusive_limit_density_is_nearly_linear():
    """Small eps: rho solves a diffusion problem away from thin boundary layers,
    so it is close to linear in the interior (Sec. 2.1, diffusion limit)."""
    n_v = 16
    v, w = K.velocities(n_v)
    g = np.where(v > 0, 3.0, 1.0)      # 3 enters on the left, 1 on the right
    F = K.range_solve(512, 1 / 256, n_v, 0, 512, g)
    rho = 0.5 * (F * w).sum(1)
    x = np.arange(513) / 512
    mid = (x > 0.1) & (x < 0.9)
    coef = np.polyfit(x[mid], rho[mid], 1)
    assert np.max(np.abs(np.polyval(coef, x[mid]) - rho[mid])) < 1e-3 * np.ptp(rho)
    assert 1.0 < rho[256] < 3.0


def test_random_snapshots_span_full_space():
    """With S >= n_v samples the random snapshots have rank n_v (the full local
    solution space of the buffered patch restricted to K_m)."""
    pts = K.patches(64, 4, 4, 12)
    R = K.snapshots(64, 1 / 16, 8, pts[1], 5)
    s = np.linalg.svd(R, compute_uv=False)
    assert s[7] > 1e-10 * s[0] and s[8] < 1e-12 * s[0]


@pytest.mark.parametrize("eps", [1.0, 1 / 64])
def test_full_basis_reproduces_global_solve(eps):
    """Exactness (Sec. 4.2): full-rank local spaces and no truncation make the
    least-squares glue reproduce the global discrete-ordinates solution."""
    n_cells, n_v = 128, 8
    off = K.offline(n_cells, eps, n_v, 4, 8, 12, 7, 1e-13)
    v, _ = K.velocities(n_v)
    left, right = 3 + np.sin(2 * np.pi * v), 2 + np.sin(2 * np.pi * v)
    f, c = K.online(off, n_cells, n_v, left, right)
    ref = K.global_reference(n_cells, eps, n_v, left, right)
    assert np.linalg.norm(f - ref) < 1e-10 * np.linalg.norm(ref)

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


@pytest.mark.parametrize("g", [0.0, 0.5, -0.7])
def test_constant_inflow_is_equilibrium(g):
    """f = 1 everywhere is the solution for unit incoming data: the collision
    annihilates constants because k is symmetric, so the gain sum_l' w_l' k(v, v')
    equals the loss rate sigma(v)."""
    n_v = 8
    F = K.range_solve(64, 1 / 16, n_v, 0, 64, np.ones(n_v), g)
    np.testing.assert_allclose(F, 1.0, atol=1e-12)


@pytest.mark.parametrize("gHG", [0.0, 0.5])
def test_free_streaming_limit(gHG):
    """Without collisions (1/eps = 0) the upwind scheme carries the incoming
    data unchanged along each characteristic."""
    n_v = 8
    g = np.arange(1, n_v + 1, dtype=float)
    F = K.range_solve(32, 1e300, n_v, 3, 20, g, gHG)
    v, _ = K.velocities(n_v)
    pos, neg = np.nonzero(v > 0)[0], np.nonzero(v < 0)[0]
    for t, l in enumerate(pos):
        np.testing.assert_allclose(F[:, l], g[t], rtol=1e-12)
    for t, l in enumerate(neg):
        np.testing.assert_allclose(F[:, l], g[len(pos) + t], rtol=1e-12)


@pytest.mark.parametrize("gHG", [0.0, 0.5, -0.3])
def test_discrete_flux_is_conserved(gHG):
    """Pure scattering conserves particles: summing the upwind equations with
    the weights w_l gives J_{i+1/2} = sum_{v>0} w v f_i + sum_{v<0} w v f_{i+1}
    constant in i (the collision terms cancel: sum_l w_l w_l' k(v_l, v_l') =
    w_l' sigma_l' by the symmetry of k)."""
    n_v = 16
    rng = np.random.default_rng(2)
    g = rng.uniform(0.0, 3.0, n_v)
    F = K.range_solve(128, 1 / 32, n_v, 0, 128, g, gHG)
    v, w = K.velocities(n_v)
    p, n = v > 0, v < 0
    J = (F[:-1][:, p] * (w * v)[p]).sum(1) + (F[1:][:, n] * (w * v)[n]).sum(1)
    np.testing.assert_allclose(J, J[0], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("g", [0.0, 0.9])
def test_positivity(g):
    """Positive incoming data gives a positive solution (M-matrix: k > 0)."""
    n_v = 8
    rng = np.random.default_rng(3)
    F = K.range_solve(64, 1 / 64, n_v, 0, 64, rng.uniform(0.1, 1.0, n_v), g)
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


@pytest.mark.parametrize("eps,g", [(1.0, 0.0), (1 / 64, 0.0), (1 / 16, 0.5)])
def test_full_basis_reproduces_global_solve(eps, g):
    """Exactness (Sec. 4.2): full-rank local spaces and no truncation make the
    least-squares glue reproduce the global discrete-ordinates solution."""
    n_cells, n_v = 128, 8
    off = K.offline(n_cells, eps, n_v, 4, 8, 12, 7, 1e-13, g)
    v, _ = K.velocities(n_v)
    left, right = 3 + np.sin(2 * np.pi * v), 2 + np.sin(2 * np.pi * v)
    f, c = K.online(off, n_cells, n_v, left, right)
    ref = K.global_reference(n_cells, eps, n_v, left, right, g)
    assert np.linalg.norm(f - ref) < 1e-10 * np.linalg.norm(ref)


def test_hg_isotropic_special_case():
    """At g = 0 the Henyey-Greenstein kernel is the constant 1/2: the gain is
    rho = (1/2) sum w f and every loss rate is 1."""
    v, w = K.velocities(12)
    Kw, sigma = K.scattering(12, 0.0)
    np.testing.assert_allclose(Kw, np.tile(0.5 * w, (12, 1)), rtol=0, atol=1e-16)
    np.testing.assert_allclose(sigma, 1.0, rtol=1e-14)


@pytest.mark.parametrize("g", [0.5, -0.3, 0.8])
def test_hg_loss_rate_closed_form(g):
    """sigma(v) = int_{-1}^{1} k(v', v) dv' has the closed form
    (1 - g^2) / (4 g v) ln((1 + g^2 + 2 g v) / (1 + g^2 - 2 g v)) (an elementary
    integral of 1/(a + b v')); the Gauss-Legendre sum converges to it
    exponentially since the pole -(1 + g^2)/(2 g v) stays off [-1, 1]."""
    n_v = 96 if abs(g) > 0.6 else 48
    v, _ = K.velocities(n_v)
    _, sigma = K.scattering(n_v, g)
    a = 1 + g * g
    exact = (1 - g * g) / (4 * g * v) * np.log((a + 2 * g * v) / (a - 2 * g * v))
    np.testing.assert_allclose(sigma, exact, rtol=1e-12)


def test_hg_two_velocity_hand_solution():
    """Brute force on the smallest slab: one cell, two ordinates v = +-1/sqrt(3)
    (weights 1).  The unknowns are f(x_1, v+) and f(x_0, v-); each satisfies one
    scalar upwind equation, solved here by hand:
        v (f1+ - a)/dx = (k(+,+) f1+ + k(+,-) b - sigma f1+)/eps
        |v| (f0- - b)/dx = (k(-,+) a + k(-,-) f0- - sigma f0-)/eps
    with k(+,+) = k(-,-) = (1/2)(1-g^2)/(1+g^2+2g/3), k(+,-) = (1/2)(1-g^2)/(1+g^2-2g/3),
    sigma = k(+,+) + k(+,-).  A wrong sign of g v v' swaps forward and backward
    scattering and fails here."""
    g, eps, a, b = 0.6, 0.3, 2.0, 0.5
    dx = 1.0
    vp = 1 / np.sqrt(3)
    kf = 0.5 * (1 - g * g) / (1 + g * g + 2 * g / 3)
    kb = 0.5 * (1 - g * g) / (1 + g * g - 2 * g / 3)
    sig = kf + kb
    f1p = (vp * a / dx + kb * b / eps) / (vp / dx + (sig - kf) / eps)
    f0m = (vp * b / dx + kb * a / eps) / (vp / dx + (sig - kf) / eps)
    F = K.range_solve(1, eps, 2, 0, 1, np.array([a, b]), g)
    assert abs(F[1, 1] - f1p) < 1e-14 and abs(F[0, 0] - f0m) < 1e-14
    assert F[0, 1] == a and F[1, 0] == b

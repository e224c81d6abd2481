"""Pins of the elliptic oracle against facts the paper and the mathematics fix.

Each test names what it pins; a dropped term, a sign, an index or a transposed
operand in the oracle breaks at least one of them.
"""
import math

import numpy as np
import pytest

import synth
from oracle import elliptic as E


def _ones(N):
    return np.ones((N + 1, N)), np.ones((N, N + 1))


# --------------------------------------------------------------- medium

def test_face_coefficients_periodic_closed_form():
    """aE[j,i] = a((i+1/2)h, jh), aN[j,i] = a(ih, (j+1/2)h) for
    a = 2 + sin(2 pi x/eps) sin(2 pi y/eps): with N = 16, eps = 1/4,
    2 pi x/eps = pi (i+1/2)/2 on x-faces, so on row j = 1 (sin(pi/2) = 1)
    aE = 2 + sin(pi (i + 1/2) / 2); the medium is symmetric so aN = aE^T."""
    aE, aN = E.face_coefficients(synth.periodic_sin(16, 0.25))
    assert aE.shape == (17, 16) and aN.shape == (16, 17)
    want = 2 + np.sin(np.pi * (np.arange(16) + 0.5) / 2)
    np.testing.assert_allclose(aE[1], want, atol=1e-14)
    np.testing.assert_allclose(aE[0], 2.0, atol=1e-14)          # sin(0) = 0 on row 0
    np.testing.assert_allclose(aN, aE.T, atol=1e-14)


def test_lognormal_medium_statistics():
    """a = exp(0.5 g) with Var g ~ 1 for the normalised medium: log a has
    mean ~0 and std ~0.5 over the grid; all coefficients positive."""
    aE, aN = E.face_coefficients(synth.lognormal(128, 2.0 ** -4, 64, 1))
    la = np.log(aE)
    assert np.all(aE > 0) and np.all(aN > 0)
    assert abs(la.mean()) < 0.2 and 0.25 < la.std() < 0.8


def test_channels_medium_two_values():
    aE, _ = E.face_coefficients(synth.channels(256, 2.0 ** -4, 4, 2, contrast=1e3))
    vals = np.unique(aE)
    assert set(vals.tolist()) <= {1.0, 1e3} and len(vals) == 2


def test_hou_wu_medium_hand_values():
    """The two-scale medium of Sec. 5.3,
    a = 2 + sin(2 pi x) cos(2 pi y) + (2 + 1.8 sin(2 pi x/eps)) / (2 + 1.8 cos(2 pi y/eps))
          + (2 + sin(2 pi y/eps)) / (2 + 1.8 cos(2 pi x/eps)),
    at points where the sines and cosines are 0, +-1, sqrt(2)/2 or sin(pi/8), worked by hand.
    The points are chosen so that exchanging x and y, dropping eps from one
    argument or exchanging sin and cos changes the value."""
    r2 = math.sqrt(0.5)
    cases = [
        # (eps, x, y, value)
        (1.0, 0.0, 0.0, 2.0 + 0.0 + 2.0 / 3.8 + 2.0 / 3.8),
        (1.0, 0.25, 0.0, 2.0 + 1.0 + 3.8 / 3.8 + 2.0 / 2.0),        # sin(pi/2) cos 0; cos(pi/2) = 0 below
        (0.5, 0.0, 0.125, 2.0 + 0.0 + 2.0 / 2.0 + 3.0 / 3.8),       # y/eps = 1/4: sin = 1, cos = 0
        (0.5, 0.125, 0.0, 2.0 + r2 + 3.8 / 3.8 + 2.0 / 2.0),        # x/eps = 1/4; sin(2 pi x) = sqrt(2)/2
        (0.25, 0.0625, 0.125, 2.0 + math.sin(math.pi / 8) * r2 + 3.8 / 0.2 + 2.0 / 2.0),   # x/eps = 1/4, y/eps = 1/2
    ]
    spec = synth.hou_wu(8, 1.0)
    for eps, x, y, want in cases:
        spec.eps = eps
        got = float(E.medium_value(spec, np.array(x), np.array(y)))
        assert abs(got - want) <= 1e-13 * abs(want), (eps, x, y, got, want)


def test_lognormal_medium_hand_values():
    """a = exp(amp * norm * sum_q [A_q cos(2 pi k_q.x) + B_q sin(2 pi k_q.x)])
    with two hand-set modes, k = (1, 0) and k = (0, 2): at (1/4, 0) the first
    phase is pi/2 (its sine term counts), at (0, 1/4) the second phase is pi
    (its cosine term counts, negated), so a transposed k, a swapped cos/sin
    or a dropped norm or amp all change the values."""
    modes = np.array([[1.0, 0.0, 0.3, -0.7],
                      [0.0, 2.0, 0.5, 0.9]])
    spec = synth.MediumSpec(synth.MEDIUM_LOGNORMAL, 8, 0.5, modes=modes, amp=0.5, norm=1.0 / math.sqrt(2.0))
    s = 0.5 / math.sqrt(2.0)
    cases = [
        (0.0, 0.0, s * (0.3 + 0.5)),                 # both phases 0: A_1 + A_2
        (0.25, 0.0, s * (-0.7 + 0.5)),               # phase_1 = pi/2 -> B_1; phase_2 = 0 -> A_2
        (0.0, 0.25, s * (0.3 - 0.5)),                # phase_1 = 0 -> A_1; phase_2 = pi -> -A_2
        (0.5, 0.125, s * (-0.3 + 0.9)),              # phase_1 = pi -> -A_1; phase_2 = pi/2 -> B_2
    ]
    for x, y, g in cases:
        got = float(E.medium_value(spec, np.array(x), np.array(y)))
        assert abs(got - math.exp(g)) <= 1e-14 * math.exp(g), (x, y, got, math.exp(g))


def test_channels_medium_hand_strips():
    """Strips of width w through (px, py) at angle theta: a = contrast where the
    distance |-(x - px) sin theta + (y - py) cos theta| <= w/2, else 1.  A
    horizontal strip (theta = 0) measures the distance in y, a vertical one
    (theta = pi/2) in x, an oblique one (theta = pi/4) |y - x| / sqrt 2; nodes
    just inside and just outside w/2 = 0.05 decide each case."""
    def value(px, py, th, x, y):
        spec = synth.MediumSpec(synth.MEDIUM_CHANNELS, 8, 0.1, channels=np.array([[px, py, th]]),
                                width=0.1, contrast=1e3)
        return float(E.medium_value(spec, np.array(x), np.array(y)))

    assert value(0.5, 0.5, 0.0, 0.9, 0.549) == 1e3
    assert value(0.5, 0.5, 0.0, 0.1, 0.451) == 1e3
    assert value(0.5, 0.5, 0.0, 0.5, 0.551) == 1.0
    assert value(0.5, 0.5, 0.0, 0.549, 0.7) == 1.0           # x distance does not count
    assert value(0.5, 0.5, math.pi / 2, 0.549, 0.9) == 1e3
    assert value(0.5, 0.5, math.pi / 2, 0.551, 0.5) == 1.0
    assert value(0.5, 0.5, math.pi / 2, 0.5, 0.9) == 1e3
    assert value(0.3, 0.3, math.pi / 4, 0.6, 0.6 + 0.07) == 1e3      # distance 0.07 / sqrt 2 = 0.0495
    assert value(0.3, 0.3, math.pi / 4, 0.6, 0.6 + 0.072) == 1.0     # 0.0509
    assert value(0.3, 0.3, math.pi / 4, 0.6 + 0.072, 0.6) == 1.0
    # the union of two strips
    spec = synth.MediumSpec(synth.MEDIUM_CHANNELS, 8, 0.1,
                            channels=np.array([[0.5, 0.2, 0.0], [0.2, 0.5, math.pi / 2]]), width=0.1, contrast=7.0)
    got = E.medium_value(spec, np.array([0.9, 0.22, 0.9, 0.5]), np.array([0.21, 0.9, 0.9, 0.5]))
    np.testing.assert_array_equal(got, [7.0, 7.0, 1.0, 1.0])


# --------------------------------------------------------------- local solver

@pytest.mark.parametrize("poly", [
    lambda x, y: x * x - y * y,
    lambda x, y: x * y,
    lambda x, y: x ** 3 - 3 * x * y * y,
    lambda x, y: 1.0 + 2.0 * x - 3.0 * y,
])
def test_harmonic_polynomials_exact(poly):
    """a = 1: the 5-point truncation error is a sum of 4th derivatives, which
    vanish for harmonic polynomials of degree <= 3, so the discrete solution
    equals the polynomial at the nodes up to rounding."""
    N = 24
    aE, aN = _ones(N)
    X0, X1, Y0, Y1 = 3, 16, 5, 21
    ring = E.ring_nodes(X0, X1, Y0, Y1)
    h = 1.0 / N
    U = E.box_solve(aE, aN, X0, X1, Y0, Y1, poly(ring[:, 0] * h, ring[:, 1] * h))
    jj, ii = np.meshgrid(np.arange(Y0, Y1 + 1), np.arange(X0, X1 + 1), indexing="ij")
    np.testing.assert_allclose(U, poly(ii * h, jj * h), atol=1e-12)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_layered_medium_closed_form(axis):
    """A medium that varies along one axis only: the discrete flux is constant,
    so u_i = sum_{i' < i} 1/a_{i'+1/2} exactly (and constant along the other
    axis).  Pins which face array couples which neighbours and the half-index
    offset of the face coefficients."""
    N = 20
    rng = np.random.default_rng(5)
    lay = rng.uniform(0.2, 5.0, size=N)
    if axis == "x":
        aE = np.tile(lay, (N + 1, 1))
        aN = rng.uniform(0.2, 5.0, size=(N, N + 1))   # arbitrary: no flux across
    else:
        aN = np.tile(lay[:, None], (1, N + 1))
        aE = rng.uniform(0.2, 5.0, size=(N + 1, N))
    prof = np.concatenate([[0.0], np.cumsum(1.0 / lay)])
    X0, X1, Y0, Y1 = 2, 17, 1, 19
    ring = E.ring_nodes(X0, X1, Y0, Y1)
    if axis == "x":
        data = prof[ring[:, 0]]
    else:
        data = prof[ring[:, 1]]
    U = E.box_solve(aE, aN, X0, X1, Y0, Y1, data)
    jj, ii = np.meshgrid(np.arange(Y0, Y1 + 1), np.arange(X0, X1 + 1), indexing="ij")
    want = prof[ii] if axis == "x" else prof[jj]
    np.testing.assert_allclose(U, want, rtol=1e-12, atol=1e-12)


def test_solution_minimises_dirichlet_energy():
    """The 5-point equations are the stationarity conditions of the discrete
    energy 1/2 sum_faces a_f (u_a - u_b)^2 (summed face by face here), so the
    solution is its minimiser: every interior perturbation raises it, to
    second order."""
    N = 12
    rng = np.random.default_rng(1)
    aE = rng.uniform(0.5, 3.0, size=(N + 1, N))
    aN = rng.uniform(0.5, 3.0, size=(N, N + 1))
    ring = E.ring_nodes(0, N, 0, N)
    U = E.box_solve(aE, aN, 0, N, 0, N, rng.standard_normal(len(ring)))

    def energy(u):
        e = 0.0
        for j in range(N + 1):
            for i in range(N):
                e += aE[j, i] * (u[j, i + 1] - u[j, i]) ** 2
        for j in range(N):
            for i in range(N + 1):
                e += aN[j, i] * (u[j + 1, i] - u[j, i]) ** 2
        return 0.5 * e

    e0 = energy(U)
    for (j, i) in [(1, 1), (5, 7), (N - 1, N - 1), (3, 10)]:
        for d in (1e-3, -1e-3):
            V = U.copy(); V[j, i] += d
            de = energy(V) - e0
            # first-order term vanishes: de equals its quadratic part
            quad = 0.5 * d * d * (aE[j, i] + aE[j, i - 1] + aN[j, i] + aN[j - 1, i])
            assert de > 0
            assert abs(de - quad) < 1e-12


def test_second_order_convergence():
    """a = 1 and the harmonic function e^{pi x} sin(pi y): the 5-point error
    falls like h^2 (discretisation accuracy)."""
    errs = []
    for N in (8, 16, 32):
        aE, aN = _ones(N)
        f = lambda x, y: np.exp(np.pi * x) * np.sin(np.pi * y)
        ring = E.ring_nodes(0, N, 0, N)
        U = E.box_solve(aE, aN, 0, N, 0, N, f(ring[:, 0] / N, ring[:, 1] / N))
        jj, ii = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
        errs.append(np.abs(U - f(ii / N, jj / N)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.8 < r2 < 4.2


def test_maximum_principle_on_snapshots():
    """Discrete maximum principle (M-matrix): each restricted snapshot stays
    within the range of its ring data."""
    w = synth.workload_small()
    aE, aN = E.face_coefficients(w["medium"])
    P = E.patch_boxes(128, w["patches"])[5]
    om = E.sample_matrix(0, P, 128)
    R = E.snapshots(aE, aN, P, 0, 128)
    assert np.all(R <= om.max(axis=0) + 1e-12) and np.all(R >= om.min(axis=0) - 1e-12)


def test_dense_brute_force_tiny():
    """Tiny box: assemble the dense matrix node by node through the energy's
    Hessian (finite differences of the energy gradient) and compare with the
    sparse solve."""
    N = 7
    rng = np.random.default_rng(3)
    aE = rng.uniform(0.3, 2.0, size=(N + 1, N))
    aN = rng.uniform(0.3, 2.0, size=(N, N + 1))
    ring = E.ring_nodes(0, N, 0, N)
    g = rng.standard_normal(len(ring))
    U = E.box_solve(aE, aN, 0, N, 0, N, g)
    # energy gradient w.r.t. interior nodes via central differences of the energy
    def energy(u):
        return 0.5 * (np.sum(aE * np.diff(u, axis=1) ** 2) + np.sum(aN * np.diff(u, axis=0) ** 2))
    ints = [(j, i) for j in range(1, N) for i in range(1, N)]
    base = np.zeros((N + 1, N + 1)); base[ring[:, 1], ring[:, 0]] = g
    n = len(ints)
    H = np.zeros((n, n)); b = np.zeros(n)
    for a, (j, i) in enumerate(ints):
        e1 = np.zeros_like(base); e1[j, i] = 1.0
        b[a] = -(energy(base + e1) - energy(base - e1)) / 2.0
        for c, (jj, ii) in enumerate(ints):
            e2 = np.zeros_like(base); e2[jj, ii] = 1.0
            H[a, c] = (energy(e1 + e2) - energy(e1 - e2)) / 2.0
    x = np.linalg.solve(H, b)
    got = np.array([U[j, i] for (j, i) in ints])
    np.testing.assert_allclose(got, x, atol=1e-12)


# --------------------------------------------------------------- offline stage

def test_random_snapshots_are_green_times_omega():
    """G^r = G~ Omega (Sec. 3.3): random-data snapshots equal the full
    (delta-data) Green's matrix times the sample matrix."""
    N = 32
    ms = synth.periodic_sin(N, 1 / 4)
    ps = synth.uniform_patches(N, 2, 2, 4, 12)
    aE, aN = E.face_coefficients(ms)
    for P in E.patch_boxes(N, ps):
        G = E.full_green(aE, aN, P)
        om = E.sample_matrix(11, P, N)
        np.testing.assert_allclose(E.snapshots(aE, aN, P, 11, N), G @ om, atol=1e-12)


def test_boundary_delta_columns_only_on_domain_boundary():
    N = 64
    ps = synth.uniform_patches(N, 4, 4, 4, 10)
    for P in E.patch_boxes(N, ps):
        pos = E.domain_boundary_ring_positions(P, N)
        interior = 0 < P.p < 3 and 0 < P.q < 3
        assert (len(pos) == 0) == interior
        om = E.sample_matrix(0, P, N)
        assert om.shape == (P.n_ring, 10 + len(pos))


def test_basis_orthonormal_and_range_error_bound():
    """Q^T Q = I and |R - Q Q^T R|_2 = sigma_{k+1} <= tau sigma_1 (Sec. 3.2,
    best rank-k approximation)."""
    w = synth.workload_small()
    off = E.offline(w["medium"], w["patches"], 0, 1e-3, patch_subset=[0, 5])
    for R, Q, s in zip(off.R, off.Q, off.sigma):
        np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
        err = np.linalg.norm(R - Q @ (Q.T @ R), 2)
        assert err <= 1e-3 * s[0] * (1 + 1e-10)
        assert s[Q.shape[1] - 1] > 1e-3 * s[0]


def test_buffer_speeds_singular_value_decay():
    """Sec. 5.3: the buffered Green's matrix has faster singular value decay
    than the unbuffered one (the singularity at the patch ring stays outside
    K_m)."""
    N = 64
    ms = synth.periodic_sin(N, 1 / 8)
    aE, aN = E.face_coefficients(ms)
    P0 = E.patch_boxes(N, synth.uniform_patches(N, 4, 4, 0, 1))[5]
    P1 = E.patch_boxes(N, synth.uniform_patches(N, 4, 4, 8, 1))[5]
    s0 = np.linalg.svd(E.full_green(aE, aN, P0), compute_uv=False)
    s1 = np.linalg.svd(E.full_green(aE, aN, P1), compute_uv=False)
    assert s1[10] / s1[0] < 0.1 * s0[10] / s0[0]


# --------------------------------------------------------------- online stage

@pytest.mark.parametrize("grid", [(32, 2, 2, 4, synth.periodic_sin(32, 1 / 4)),
                                  (36, 3, 3, 3, synth.hou_wu(36, 1 / 4)),
                                  (48, 3, 2, 6, synth.lognormal(48, 1 / 6, 16, 4))])
def test_full_basis_reproduces_global_solve(grid):
    """Full-basis exactness (Sec. 4.2 / 5.2: the global solution restricted to
    K_m lies in span G~_m): with enough samples and no truncation the
    least-squares glue reproduces the global fine-mesh solution to rounding.
    Pins the value, flux (with its face multiplicities) and boundary rows and
    the partition of unity."""
    N, mx, my, b, ms = grid
    ring = max(2 * (N // mx + 2 * b) + 2 * (N // my + 2 * b), 1)
    ps = synth.uniform_patches(N, mx, my, b, ring + 8)
    off = E.offline(ms, ps, 3, 1e-13)
    phi = synth.phi_fourier(N, 6, 9, kmax=3)[0]
    u, c, Pm, d = E.online(off, ps, N, phi)
    uref = E.global_reference(off.aE, off.aN, N, phi)
    assert E.rel_l2(u, uref) < 1e-10
    assert np.linalg.norm(Pm @ c - d) < 1e-9 * np.linalg.norm(d)


def test_full_basis_uneven_patches():
    """Exactness on an uneven partition with different buffers per patch."""
    N = 40
    ps = synth.PatchSpec(np.array([0, 12, 28, 40]), np.array([0, 20, 40]),
                         np.array([3, 4, 2, 5, 4, 3]), np.full(6, 150))
    ms = synth.periodic_sin(N, 1 / 5)
    off = E.offline(ms, ps, 2, 1e-13)
    phi = synth.phi_sin_cos(N)
    u, *_ = E.online(off, ps, N, phi)
    assert E.rel_l2(u, E.global_reference(off.aE, off.aN, N, phi)) < 1e-10


def test_flux_rows_sum_to_residual():
    """For any nodal field, the flux rows of the patches sharing a skeleton
    node add up to (A u)(x)/h -- the 5-point residual -- by construction of
    the face multiplicities (reading of the flux continuity a d_n u_m =
    -a d_n u_n, Eq. elliptic_cont_cond)."""
    N = 24
    rng = np.random.default_rng(0)
    aE = rng.uniform(0.5, 2.0, size=(N + 1, N)); aN = rng.uniform(0.5, 2.0, size=(N, N + 1))
    ps = synth.uniform_patches(N, 3, 2, 2, 1)
    patches = E.patch_boxes(N, ps)
    U = rng.standard_normal((N + 1, N + 1))
    tot = {}
    for P in patches:
        Q = U[P.y0:P.y1 + 1, P.x0:P.x1 + 1].reshape(-1, 1)
        nodes, V, F = E.edge_rows(aE, aN, P, Q, N, list(ps.x_breaks), list(ps.y_breaks))
        for t, (i, j) in enumerate(nodes):
            tot[(int(i), int(j))] = tot.get((int(i), int(j)), 0.0) + F[t, 0]
    for (i, j), f in tot.items():
        if 0 < i < N and 0 < j < N and (i in ps.x_breaks or j in ps.y_breaks):
            res = (aE[j, i] * (U[j, i] - U[j, i + 1]) + aE[j, i - 1] * (U[j, i] - U[j, i - 1])
                   + aN[j, i] * (U[j, i] - U[j + 1, i]) + aN[j - 1, i] * (U[j, i] - U[j - 1, i]))
            assert abs(f - res * N) < 1e-10 * max(1.0, abs(res * N))


def test_direct_ls_paths_agree():
    """Dense SVD least squares and the corrected semi-normal equations give
    the same minimiser, and it satisfies the normal equations."""
    w = synth.workload_small()
    off = E.offline(w["medium"], synth.uniform_patches(128, 4, 4, 8, 40), 0, 1e-6)
    Pm, d, o = E.online_system(off.aE, off.aN, off.patches, off.Q, 128, w["patches"], w["phi"])
    c1 = E.online_solve(Pm, d, dense_limit=1e12)
    c2 = E.online_solve(Pm, d, dense_limit=0)
    np.testing.assert_allclose(c2, c1, rtol=1e-9, atol=1e-9 * np.abs(c1).max())
    # normal-equation residual at the level of a backward-stable solve:
    # |P^T r| <~ u |P| (|P| |c| + |r|)
    r = d - Pm @ c1
    g = Pm.T @ r
    nP = math.sqrt(Pm.multiply(Pm).sum())
    assert np.linalg.norm(g) < 1e-12 * nP * (nP * np.linalg.norm(c1) + np.linalg.norm(r))


def test_small_workload_method_accuracy():
    """The small workload (129^2, 4x4 patches, 40 samples, tau 1e-6) solves
    the global problem to about 1e-3 relative L2 (a method check, not a
    parity value)."""
    w = synth.workload_small()
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
    u, *_ = E.online(off, w["patches"], 128, w["phi"])
    err = E.rel_l2(u, E.global_reference(off.aE, off.aN, 128, w["phi"]))
    assert err < 5e-3


# ------------------------------------------ constrained least-squares variant

@pytest.mark.parametrize("grid", [(32, 2, 2, 4, synth.periodic_sin(32, 1 / 4)),
                                  (36, 3, 3, 3, synth.hou_wu(36, 1 / 4))])
def test_constrained_full_basis_reproduces_global_solve(grid):
    """With full local spaces the global solution meets every boundary row and
    every continuity row, so it is the constrained minimiser too: the
    constrained variant reproduces the fine-mesh solution."""
    N, mx, my, b, ms = grid
    ring = max(2 * (N // mx + 2 * b) + 2 * (N // my + 2 * b), 1)
    ps = synth.uniform_patches(N, mx, my, b, ring + 8)
    off = E.offline(ms, ps, 3, 1e-13)
    phi = synth.phi_fourier(N, 6, 9, kmax=3)[0]
    u, c, Pm, d, bnd = E.online_constrained(off, ps, N, phi)
    assert E.rel_l2(u, E.global_reference(off.aE, off.aN, N, phi)) < 1e-10


def test_constrained_solution_is_the_weighted_limit():
    """An independent route to the same point: the weighted least squares
    min |C c|^2 + w^2 |B c - phi|^2 tends to the constrained solution as w grows
    (the method of weighting; the gap shrinks like 1/w^2).  On the small
    workload's truncated bases: the boundary rows hold to rounding, the weighted
    solutions approach the constrained one, and the continuity residual is no
    larger than that of any weighted solution (it is the least among the
    solutions that meet the boundary rows)."""
    w = synth.workload_small()
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
    Pm, d, o, bnd = E.online_system_rows(off.aE, off.aN, off.patches, off.Q, 128, w["patches"], w["phi"])
    c = E.constrained_solve(Pm, d, bnd)
    B, C, f = Pm[bnd].toarray(), Pm[~bnd].toarray(), d[bnd]
    assert np.linalg.norm(B @ c - f) <= 1e-10 * np.linalg.norm(f)
    gaps = []
    for wt in (1e2, 1e3, 1e4):
        cw, *_ = np.linalg.lstsq(np.vstack([C, wt * B]), np.concatenate([np.zeros(C.shape[0]), wt * f]), rcond=None)
        gaps.append(np.linalg.norm(cw - c) / np.linalg.norm(c))
    assert gaps[2] < 1e-5 and gaps[1] < gaps[0] and gaps[2] < gaps[1]
    # the unconstrained LS trades boundary error for continuity: its continuity
    # residual is smaller, its boundary residual larger
    cu = E.online_solve(Pm, d)
    assert np.linalg.norm(C @ cu) <= np.linalg.norm(C @ c) + 1e-12
    assert np.linalg.norm(B @ cu - f) >= np.linalg.norm(B @ c - f)


def test_constrained_small_workload_accuracy():
    """The constrained variant on the small workload solves the global problem
    to the same order as the least-squares glue (a method check)."""
    w = synth.workload_small()
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
    u, *_ = E.online_constrained(off, w["patches"], 128, w["phi"])
    assert E.rel_l2(u, E.global_reference(off.aE, off.aN, 128, w["phi"])) < 5e-3

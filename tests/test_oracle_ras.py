"""Pins of the oracle's overlapping-Schwarz online variant (`ras_*`).

The reduced restricted additive Schwarz step c <- T c + F phi is pinned against
things fixed outside its own algebra:

* the classical restricted additive Schwarz step, computed here from its
  definition with fine-grid local solves (`box_solve` on every buffered patch,
  ring data read off the current field, solutions kept on K_m and averaged
  with chi_m = 1/#patches at shared nodes, phi on the domain boundary): with the
  full basis the reduced iterates reconstruct to the classical ones, and with a
  truncated basis each reduced step is the projection Q_m^T of the classical
  local solve;
* full-basis exactness: the global fine-grid solution is the fixed point;
* the plain iteration converges to the direct fixed-point solve.

A wrong partition-of-unity weight, a transposed B_m, a ring read in the wrong
order or phi placed at the wrong boundary node breaks the classical comparison.
"""
import numpy as np
import pytest

import synth
from oracle import elliptic as E


def _full_offline(ms, ps):
    """Bases spanning the whole range of every G~_m (DetLocalSolu, no truncation)."""
    aE, aN = E.face_coefficients(ms)
    patches = E.patch_boxes(ms.n_cells, ps)
    Qs = []
    for P_ in patches:
        U, s, _ = np.linalg.svd(E.full_green(aE, aN, P_), full_matrices=False)
        Qs.append(U[:, s > 1e-13 * s[0]])
    return E.Offline(aE, aN, patches, [None] * len(patches), Qs, [None] * len(patches))


def _classical_step(aE, aN, patches, N, u, phi):
    """One restricted additive Schwarz step on the fine grid, from its definition."""
    ring = E.ring_nodes(0, N, 0, N)
    acc = np.zeros((N + 1, N + 1))
    cnt = np.zeros((N + 1, N + 1))
    for P_ in patches:
        rn = E.ring_nodes(P_.X0, P_.X1, P_.Y0, P_.Y1)
        U = E.box_solve(aE, aN, P_.X0, P_.X1, P_.Y0, P_.Y1, u[rn[:, 1], rn[:, 0]])
        acc[P_.y0:P_.y1 + 1, P_.x0:P_.x1 + 1] += U[P_.y0 - P_.Y0:P_.y1 - P_.Y0 + 1, P_.x0 - P_.X0:P_.x1 - P_.X0 + 1]
        cnt[P_.y0:P_.y1 + 1, P_.x0:P_.x1 + 1] += 1
    out = acc / cnt
    out[ring[:, 1], ring[:, 0]] = phi
    return out


CASES = [
    ("uniform", 32, synth.PatchSpec(np.array([0, 16, 32]), np.array([0, 16, 32]), np.full(4, 4), np.full(4, 1)),
     synth.periodic_sin(32, 1 / 4)),
    ("uneven", 40, synth.PatchSpec(np.array([0, 12, 28, 40]), np.array([0, 20, 40]), np.array([3, 4, 2, 5, 4, 3]),
                                   np.full(6, 1)), synth.lognormal(40, 1 / 5, 16, 4)),
    # buffers wider than the neighbouring patch: rings reach two patches away
    ("wide", 36, synth.PatchSpec(np.array([0, 8, 28, 36]), np.array([0, 12, 24, 36]), np.full(9, 10),
                                 np.full(9, 1)), synth.hou_wu(36, 1 / 4)),
]


@pytest.mark.parametrize("name,N,ps,ms", CASES, ids=[c[0] for c in CASES])
def test_full_basis_iterates_are_classical_schwarz(name, N, ps, ms):
    """With the full basis, three reduced steps from c = 0 reconstruct to three
    classical restricted additive Schwarz steps from the field that is 0 inside
    and phi on the boundary."""
    off = _full_offline(ms, ps)
    phi = synth.phi_fourier(N, 6, 5, kmax=3)[0]
    T, F, o = E.ras_operators(off.aE, off.aN, off.patches, off.Q, N)
    u = E.reconstruct(off.patches, off.Q, np.zeros(o[-1]), o, N, phi)
    c = np.zeros(o[-1])
    for _ in range(3):
        u = _classical_step(off.aE, off.aN, off.patches, N, u, phi)
        c = E.ras_iterate(T, F, phi, c, 1)
        ur = E.reconstruct(off.patches, off.Q, c, o, N, phi)
        assert E.rel_l2(ur, u) < 1e-11


def test_truncated_step_is_projected_classical_step():
    """With truncated bases one reduced step from any c is, per patch, Q_m^T times
    the classical local solve on K~_m with the ring values of u(c), restricted
    to K_m."""
    N = 48
    ps = synth.uniform_patches(N, 3, 3, 6, 40)
    ms = synth.lognormal(N, 1 / 6, 16, 2)
    off = E.offline(ms, ps, 11, 1e-4)
    assert all(q.shape[1] < q.shape[0] for q in off.Q)
    phi = synth.phi_fourier(N, 6, 7, kmax=3)[0]
    T, F, o = E.ras_operators(off.aE, off.aN, off.patches, off.Q, N)
    c = np.random.default_rng(5).standard_normal(o[-1])
    u = E.reconstruct(off.patches, off.Q, c, o, N, phi)
    c1 = E.ras_iterate(T, F, phi, c, 1)
    for P_, Q in zip(off.patches, off.Q):
        rn = E.ring_nodes(P_.X0, P_.X1, P_.Y0, P_.Y1)
        U = E.box_solve(off.aE, off.aN, P_.X0, P_.X1, P_.Y0, P_.Y1, u[rn[:, 1], rn[:, 0]])
        want = Q.T @ E.restrict(U, P_)[:, 0]
        got = c1[o[P_.m]:o[P_.m + 1]]
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


@pytest.mark.parametrize("name,N,ps,ms", CASES, ids=[c[0] for c in CASES])
def test_full_basis_fixed_point_is_the_global_solve(name, N, ps, ms):
    """Full-basis exactness: the restriction of the global fine-grid solution is
    the fixed point, so the reconstruction reproduces the global solve."""
    off = _full_offline(ms, ps)
    phi = synth.phi_fourier(N, 6, 9, kmax=3)[0]
    u, c, T, F = E.online_ras(off, N, phi)
    assert E.rel_l2(u, E.global_reference(off.aE, off.aN, N, phi)) < 1e-10


def test_plain_iteration_converges_to_the_fixed_point():
    """The Schwarz step contracts (spectral radius below 1 on the small
    workload), and its plain iterates converge to the direct fixed-point solve."""
    w = synth.workload_small()
    N = w["medium"].n_cells
    off = E.offline(w["medium"], w["patches"], w["seed"], 1e-6)
    phi = synth.phi_sin_cos(N)
    T, F, o = E.ras_operators(off.aE, off.aN, off.patches, off.Q, N)
    c = E.ras_solve(T, F, phi)
    rho = max(abs(np.linalg.eigvals(T.toarray())))
    assert rho < 0.95
    ci = E.ras_iterate(T, F, phi, np.zeros(o[-1]), 300)
    assert np.linalg.norm(ci - c) <= 1e-9 * np.linalg.norm(c)


def test_small_workload_accuracy():
    """Method check on the small workload (40 samples, tau = 1e-6): the Schwarz
    fixed point is within 1e-3 of the global solve, and no worse than the
    least-squares glue on the same bases."""
    w = synth.workload_small()
    N = w["medium"].n_cells
    off = E.offline(w["medium"], w["patches"], w["seed"], 1e-6)
    phi = synth.phi_sin_cos(N)
    uref = E.global_reference(off.aE, off.aN, N, phi)
    u_ras, *_ = E.online_ras(off, N, phi)
    u_ls, *_ = E.online(off, w["patches"], N, phi)
    e_ras, e_ls = E.rel_l2(u_ras, uref), E.rel_l2(u_ls, uref)
    assert e_ras < 1e-3 and e_ras <= e_ls

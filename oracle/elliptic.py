"""Elliptic example (Sec. 5): plain FP64 restatement of the whole method.

Problem (Eq. Elliptic, Eq. elliptic_bdy):  div(a grad u) = 0 in [0,1]^2,
u = phi on the boundary.  Discretisation (reading R1; the paper's own test
uses P1/Q1 finite elements, Sec. 5.3): the conservative 5-point scheme on
the fine grid h = 1/N,

    (A u)_{ij} = sum over the four faces f of node (i,j) of a_f (u_ij - u_nbr(f)),

with a_f the coefficient evaluated at the face midpoint:
aE[j, i] = a((i+1/2) h, j h) on the face between (i,j) and (i+1,j), and
aN[j, i] = a(i h, (j+1/2) h) on the face between (i,j) and (i,j+1).
A is symmetric positive definite on the interior unknowns of any node box
with Dirichlet data on the box's ring.

Pipeline, in the order of Algorithm alg:summary:
  medium -> face coefficients                         `face_coefficients`
  domain decomposition, buffered patches              `patch_boxes`
  RanLocalSolu: Gaussian ring data, local solves on
    the buffered patch, restriction (Sec. 3.3, Eq.
    elliptic_random)                                  `snapshots`
  DetLocalSolu (delta data, Eq. ux7 / lr2)            `full_green`
  orthonormal basis from the SVD, truncated at
    sigma_i > tau sigma_1 (Sec. 3.2, Eq. svd)         `basis`
  value / flux / boundary rows (Eq. elliptic_cond_tilde)
    and c = argmin |P c - d| (Eq. elliptic_cond_reduced)  `online_system`, `online_solve`
  the constrained variant: boundary rows exact, continuity
    rows in the least-squares sense                   `constrained_solve`
  the overlapping variant: restricted additive Schwarz
    on the buffered patches, reduced to the bases      `ras_operators`, `ras_solve`
  u = sum_m G_m c_m with a partition of unity          `reconstruct`
Direct solvers replace every iteration of the GPU path.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import philox

MEDIUM_PERIODIC_SIN, MEDIUM_LOGNORMAL, MEDIUM_CHANNELS, MEDIUM_HOU_WU, MEDIUM_USER = range(5)


# ---------------------------------------------------------------------------
# medium (Sec. 5, a(x, x/eps); Sec. 5.3 for the two-scale example)
# ---------------------------------------------------------------------------

def medium_value(spec, x, y):
    """a(x, y) of a medium description at points (x, y) (numpy arrays)."""
    k = spec.kind
    if k == MEDIUM_PERIODIC_SIN:
        e = spec.eps
        return 2.0 + np.sin(2 * np.pi * x / e) * np.sin(2 * np.pi * y / e)
    if k == MEDIUM_HOU_WU:
        e = spec.eps
        return (2.0 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
                + (2.0 + 1.8 * np.sin(2 * np.pi * x / e)) / (2.0 + 1.8 * np.cos(2 * np.pi * y / e))
                + (2.0 + np.sin(2 * np.pi * y / e)) / (2.0 + 1.8 * np.cos(2 * np.pi * x / e)))
    if k == MEDIUM_LOGNORMAL:
        g = np.zeros(np.broadcast(x, y).shape)
        for kx, ky, A, B in spec.modes:
            ph = 2 * np.pi * (kx * x + ky * y)
            g = g + A * np.cos(ph) + B * np.sin(ph)
        return np.exp(spec.amp * spec.norm * g)
    if k == MEDIUM_CHANNELS:
        inside = np.zeros(np.broadcast(x, y).shape, dtype=bool)
        for px, py, th in spec.channels:
            dist = np.abs(-(x - px) * np.sin(th) + (y - py) * np.cos(th))
            inside |= dist <= 0.5 * spec.width
        return np.where(inside, spec.contrast, 1.0)
    raise ValueError(f"medium kind {k} has no analytic form")


def face_coefficients(spec):
    """Face coefficients (aE, aN): aE[j, i] = a((i+1/2)h, jh), shape (N+1, N);
    aN[j, i] = a(ih, (j+1/2)h), shape (N, N+1) (reading R1)."""
    N = spec.n_cells
    if spec.kind == MEDIUM_USER:
        return np.array(spec.user_aE, dtype=np.float64), np.array(spec.user_aN, dtype=np.float64)
    h = 1.0 / N
    jE, iE = np.meshgrid(np.arange(N + 1), np.arange(N), indexing="ij")
    aE = medium_value(spec, (iE + 0.5) * h, jE * h)
    jN, iN = np.meshgrid(np.arange(N), np.arange(N + 1), indexing="ij")
    aN = medium_value(spec, iN * h, (jN + 0.5) * h)
    return np.asarray(aE, dtype=np.float64), np.asarray(aN, dtype=np.float64)


# ---------------------------------------------------------------------------
# domain decomposition (Sec. 5: K = union of K_m; buffered patches Sec. 3.3)
# ---------------------------------------------------------------------------

@dataclass
class Patch:
    m: int
    p: int
    q: int
    x0: int   # closed node box of K_m
    x1: int
    y0: int
    y1: int
    X0: int   # closed node box of the buffered patch (clipped to the domain, reading R3)
    X1: int
    Y0: int
    Y1: int
    S: int

    @property
    def n_k(self):
        return (self.x1 - self.x0 + 1) * (self.y1 - self.y0 + 1)

    @property
    def n_ring(self):
        return 2 * (self.X1 - self.X0) + 2 * (self.Y1 - self.Y0)


def patch_boxes(N, pspec):
    """Patches K_m (p fastest) and their buffered boxes, clipped to [0, N]^2."""
    xb, yb = list(map(int, pspec.x_breaks)), list(map(int, pspec.y_breaks))
    assert xb[0] == 0 and xb[-1] == N and yb[0] == 0 and yb[-1] == N
    mx, my = len(xb) - 1, len(yb) - 1
    out = []
    for q in range(my):
        for p in range(mx):
            m = p + q * mx
            b = int(pspec.buffers[m])
            x0, x1, y0, y1 = xb[p], xb[p + 1], yb[q], yb[q + 1]
            out.append(Patch(m, p, q, x0, x1, y0, y1,
                             max(0, x0 - b), min(N, x1 + b), max(0, y0 - b), min(N, y1 + b),
                             int(pspec.samples[m])))
    return out


def ring_nodes(X0, X1, Y0, Y1):
    """Nodes (i, j) of the ring of a node box, counter-clockwise from (X0, Y0)."""
    pts = [(i, Y0) for i in range(X0, X1)]
    pts += [(X1, j) for j in range(Y0, Y1)]
    pts += [(i, Y1) for i in range(X1, X0, -1)]
    pts += [(X0, j) for j in range(Y1, Y0, -1)]
    return np.array(pts, dtype=np.int64)


# ---------------------------------------------------------------------------
# LocalPDESolver (Algorithm alg:summary) for the 5-point operator
# ---------------------------------------------------------------------------

def box_operator(aE, aN, X0, X1, Y0, Y1):
    """Sparse blocks of A on a node box: A_II (interior x interior) and A_IB
    (interior x ring), interior unknowns row-major (i fastest), ring in the
    counter-clockwise order of `ring_nodes`."""
    nx, ny = X1 - X0 - 1, Y1 - Y0 - 1
    ring = ring_nodes(X0, X1, Y0, Y1)
    ring_id = {(int(i), int(j)): t for t, (i, j) in enumerate(ring)}

    def interior_id(i, j):
        return (i - X0 - 1) + (j - Y0 - 1) * nx

    rI, cI, vI, rB, cB, vB = [], [], [], [], [], []
    for j in range(Y0 + 1, Y1):
        for i in range(X0 + 1, X1):
            r = interior_id(i, j)
            faces = ((aE[j, i], i + 1, j), (aE[j, i - 1], i - 1, j),
                     (aN[j, i], i, j + 1), (aN[j - 1, i], i, j - 1))
            diag = 0.0
            for a, ii, jj in faces:
                diag += a
                if X0 < ii < X1 and Y0 < jj < Y1:
                    rI.append(r); cI.append(interior_id(ii, jj)); vI.append(-a)
                else:
                    rB.append(r); cB.append(ring_id[(ii, jj)]); vB.append(-a)
            rI.append(r); cI.append(r); vI.append(diag)
    n = nx * ny
    A_II = sp.csc_matrix((vI, (rI, cI)), shape=(n, n))
    A_IB = sp.csc_matrix((vB, (rB, cB)), shape=(n, len(ring)))
    return A_II, A_IB


def box_solve(aE, aN, X0, X1, Y0, Y1, ring_values):
    """Solve A u = 0 in the interior of the box with u = ring_values on its
    ring, by sparse LU (LocalPDESolver with a direct method).

    ring_values: (n_ring,) or (n_ring, S).  Returns the full nodal field(s),
    shape (Y1-Y0+1, X1-X0+1[, S]), ring nodes included."""
    rv = np.asarray(ring_values, dtype=np.float64)
    vec = rv.ndim == 1
    if vec:
        rv = rv[:, None]
    A_II, A_IB = box_operator(aE, aN, X0, X1, Y0, Y1)
    nx, ny = X1 - X0 - 1, Y1 - Y0 - 1
    S = rv.shape[1]
    U = np.zeros((Y1 - Y0 + 1, X1 - X0 + 1, S))
    if nx > 0 and ny > 0:
        lu = spla.splu(A_II)
        ui = lu.solve(np.ascontiguousarray(-(A_IB @ rv)))
        U[1:-1, 1:-1, :] = ui.reshape(ny, nx, S)
    ring = ring_nodes(X0, X1, Y0, Y1)
    U[ring[:, 1] - Y0, ring[:, 0] - X0, :] = rv
    return U[..., 0] if vec else U


def restrict(U, patch):
    """Restriction of buffered-box fields to the closed K_m box, as a matrix of
    shape (n_k, S) with K_m nodes row-major (Sec. 3.3, r = r~|_{K_m})."""
    P = patch
    sub = U[P.y0 - P.Y0:P.y1 - P.Y0 + 1, P.x0 - P.X0:P.x1 - P.X0 + 1]
    return sub.reshape(P.n_k, -1)


def domain_boundary_ring_positions(patch, N):
    """Positions, in ring order, of the buffered patch's ring nodes that lie on
    the domain boundary."""
    ring = ring_nodes(patch.X0, patch.X1, patch.Y0, patch.Y1)
    on = (ring[:, 0] == 0) | (ring[:, 0] == N) | (ring[:, 1] == 0) | (ring[:, 1] == N)
    return np.nonzero(on)[0]


def sample_matrix(seed, patch, N):
    """Ring data of the local solves of one patch, shape (n_ring, S_m + n_b).

    Columns 0..S_m-1: i.i.d. N(0,1) values on every ring node (Omega_m of Eq.
    elliptic_random, drawn by Philox).  Columns S_m..: one delta per ring node
    lying on the domain boundary (n_b of them, none for interior patches).
    Reading: the paper gives patches at the domain boundary the full basis
    so that they can carry the global boundary data (Sec. 4.2, boundary
    patches of the transport example); for the elliptic problem the same rule
    is applied to the ring nodes on the domain boundary, whose data is not
    low rank (it is phi itself)."""
    om = philox.normals(seed, patch.m, patch.n_ring, patch.S, philox.TAG_ELLIPTIC)
    pos = domain_boundary_ring_positions(patch, N)
    de = np.zeros((patch.n_ring, len(pos)))
    de[pos, np.arange(len(pos))] = 1.0
    return np.concatenate([om, de], axis=1)


def snapshots(aE, aN, patch, seed, N):
    """G_m^{eps,r} = [r_{m,1} ... r_{m,S}]: RanLocalSolu on the buffered patch,
    restricted to K_m (Sec. 5.2), plus the boundary-delta columns of
    `sample_matrix`."""
    om = sample_matrix(seed, patch, N)
    U = box_solve(aE, aN, patch.X0, patch.X1, patch.Y0, patch.Y1, om)
    return restrict(U, patch)


def full_green(aE, aN, patch):
    """G~_m of Eq. lr2: DetLocalSolu on the buffered patch (one delta per ring
    node), restricted to K_m; shape (n_k, n_ring)."""
    U = box_solve(aE, aN, patch.X0, patch.X1, patch.Y0, patch.Y1, np.eye(patch.n_ring))
    return restrict(U, patch)


# ---------------------------------------------------------------------------
# basis: SVD of the snapshots, truncated (Sec. 3.2, Eq. svd; QR remark Sec. 3.3)
# ---------------------------------------------------------------------------

def basis(R, tau):
    """Left singular vectors U_k and all singular values of R, with
    k = #{sigma_i > tau sigma_1} (reading R5)."""
    U, s, _ = np.linalg.svd(R, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return U[:, :0], s
    k = int(np.count_nonzero(s > tau * s[0]))
    return U[:, :k], s


# ---------------------------------------------------------------------------
# online stage (Sec. 5.2, Eq. elliptic_cond_tilde, Eq. elliptic_cond_reduced)
# ---------------------------------------------------------------------------

def _face_multiplicity(breaks, idx):
    """How many patches' closed boxes contain a face lying on grid line `idx`
    along the other axis: 2 on an interior patch break, else 1."""
    return 2 if idx in breaks[1:-1] else 1


def edge_rows(aE, aN, patch, Q, N, xb, yb):
    """Value and flux rows of basis Q on every node of the ring of K_m.

    Value row at node x: Q[x] (the map c -> u_m(x), M~ of Eq. elliptic_cond_tilde).
    Flux row (reading R7): F_m(x) = (1/h) sum over faces f at x inside the
    closed K_m of (a_f / nu_f)(Q[x] - Q[nbr_f]), nu_f the number of patches
    whose closed box holds f.  Summed over the patches sharing x it is the
    5-point residual at x over h, so sum_j F_{m_j}(x) = 0 is the discrete form
    of the flux continuity a d_n u_m = -a d_n u_n (W~ of Eq. elliptic_cond_tilde).

    Returns (nodes (n_e, 2), V (n_e, k), F (n_e, k))."""
    P = patch
    h = 1.0 / N
    nodes = ring_nodes(P.x0, P.x1, P.y0, P.y1)
    wx = P.x1 - P.x0 + 1

    def loc(i, j):
        return (i - P.x0) + (j - P.y0) * wx

    V = np.empty((len(nodes), Q.shape[1]))
    F = np.zeros_like(V)
    for t, (i, j) in enumerate(nodes):
        i = int(i); j = int(j)
        V[t] = Q[loc(i, j)]
        faces = []
        if i + 1 <= P.x1:
            faces.append((aE[j, i] / _face_multiplicity(yb, j), i + 1, j))
        if i - 1 >= P.x0:
            faces.append((aE[j, i - 1] / _face_multiplicity(yb, j), i - 1, j))
        if j + 1 <= P.y1:
            faces.append((aN[j, i] / _face_multiplicity(xb, i), i, j + 1))
        if j - 1 >= P.y0:
            faces.append((aN[j - 1, i] / _face_multiplicity(xb, i), i, j - 1))
        for a, ii, jj in faces:
            F[t] += (a / h) * (Q[loc(i, j)] - Q[loc(ii, jj)])
    return nodes, V, F


def domain_ring_index(N):
    """Map global boundary node (i, j) -> position in the global ring
    (counter-clockwise from (0,0))."""
    return {(int(i), int(j)): t for t, (i, j) in enumerate(ring_nodes(0, N, 0, N))}


def online_system(aE, aN, patches, Qs, N, pspec, phi):
    """P~, d and the coefficient offsets of Eq. elliptic_cond_reduced (see
    `online_system_rows`, which also marks the boundary rows)."""
    Pm, d, off, _ = online_system_rows(aE, aN, patches, Qs, N, pspec, phi)
    return Pm, d, off


def online_system_rows(aE, aN, patches, Qs, N, pspec, phi):
    """Assemble P~ (sparse, rows x N_p) and d for Eq. elliptic_cond_reduced.

    Rows, node by node over the patch skeleton (readings R6-R8):
      * x on the domain boundary: one row u_m(x) = phi(x) per patch m holding x;
      * otherwise, with m_1 < ... < m_r the patches holding x:
        value rows u_{m_1}(x) - u_{m_j}(x) = 0 (j = 2..r) and one flux row
        sum_j F_{m_j}(x) = 0.
    Returns (P, d, offsets, is_boundary_row) with offsets[m] the first column
    of c_m."""
    xb, yb = list(map(int, pspec.x_breaks)), list(map(int, pspec.y_breaks))
    ks = [Q.shape[1] for Q in Qs]
    off = np.concatenate([[0], np.cumsum(ks)]).astype(int)
    rows = {}   # (m, i, j) -> (value row, flux row)
    for P_, Q in zip(patches, Qs):
        nodes, V, F = edge_rows(aE, aN, P_, Q, N, xb, yb)
        for t, (i, j) in enumerate(nodes):
            rows[(P_.m, int(i), int(j))] = (V[t], F[t])
    ring_id = domain_ring_index(N)
    mx = len(xb) - 1
    # skeleton nodes in row-major order
    skel = sorted({(i, j) for (_, i, j) in rows}, key=lambda ij: (ij[1], ij[0]))
    r_i, c_i, v_i, d, bnd = [], [], [], [], []
    nrow = 0

    def put(m, vec, sign):
        cols = np.arange(off[m], off[m] + ks[m])
        r_i.extend([nrow] * ks[m]); c_i.extend(cols); v_i.extend(sign * vec)

    for (i, j) in skel:
        ps = [p for p in range(mx) if xb[p] <= i <= xb[p + 1]]
        qs = [q for q in range(len(yb) - 1) if yb[q] <= j <= yb[q + 1]]
        ms = sorted(p + q * mx for q in qs for p in ps)
        if i in (0, N) or j in (0, N):
            for m in ms:
                put(m, rows[(m, i, j)][0], 1.0)
                d.append(phi[ring_id[(i, j)]]); bnd.append(True); nrow += 1
        else:
            for m in ms[1:]:
                put(ms[0], rows[(ms[0], i, j)][0], 1.0)
                put(m, rows[(m, i, j)][0], -1.0)
                d.append(0.0); bnd.append(False); nrow += 1
            for m in ms:
                put(m, rows[(m, i, j)][1], 1.0)
            d.append(0.0); bnd.append(False); nrow += 1
    Pm = sp.csr_matrix((v_i, (r_i, c_i)), shape=(nrow, off[-1]))
    return Pm, np.array(d), off, np.array(bnd, dtype=bool)


def online_solve(Pm, d, dense_limit=4e7):
    """c~ = argmin_e |P~ e - d|_2 (Eq. elliptic_cond_reduced) by a direct
    method: dense SVD least squares when small, else the corrected
    semi-normal equations (normal equations by sparse LU plus one
    correction step, Bjorck)."""
    if Pm.shape[0] * Pm.shape[1] <= dense_limit:
        c, *_ = np.linalg.lstsq(Pm.toarray(), d, rcond=None)
        return c
    PtP = (Pm.T @ Pm).tocsc()
    lu = spla.splu(PtP)
    c = lu.solve(Pm.T @ d)
    r = d - Pm @ c
    return c + lu.solve(Pm.T @ r)


def constrained_solve(Pm, d, is_bnd, rank_tol=1e-12):
    """The constrained least-squares variant of the online step (the remark
    after Eq. elliptic_cond_reduced): minimise the continuity rows |C c|_2 subject
    to the boundary rows B c = phi exactly, by the null-space method (Golub and
    Van Loan, Sec. 6.2): with the SVD B = U S V^T of rank r (singular values above
    rank_tol s_1), c = c_p + N z where c_p = V_r S_r^{-1} U_r^T phi is the
    minimum-norm solution of the constraints, N = V[:, r:] spans null(B), and
    z = argmin |C N z + C c_p|_2.  Dense; for the sizes the tests use."""
    B = Pm[is_bnd].toarray()
    C = Pm[~is_bnd].toarray()
    f = d[is_bnd]
    U, s, Vt = np.linalg.svd(B, full_matrices=True)
    r = int(np.sum(s > rank_tol * s[0])) if s.size else 0
    c_p = Vt[:r].T @ ((U[:, :r].T @ f) / s[:r])
    Nn = Vt[r:].T
    z, *_ = np.linalg.lstsq(C @ Nn, -(C @ c_p), rcond=None)
    return c_p + Nn @ z


def reconstruct(patches, Qs, c, off, N, phi):
    """u = sum_m chi_m G_m c_m on the fine grid (Algorithm alg:summary, return
    line) with the partition of unity chi_m = 1 / #{patches holding x}
    (reading R10); boundary nodes take phi."""
    u = np.zeros((N + 1, N + 1))
    cnt = np.zeros((N + 1, N + 1))
    for P_, Q in zip(patches, Qs):
        v = (Q @ c[off[P_.m]:off[P_.m + 1]]).reshape(P_.y1 - P_.y0 + 1, P_.x1 - P_.x0 + 1)
        u[P_.y0:P_.y1 + 1, P_.x0:P_.x1 + 1] += v
        cnt[P_.y0:P_.y1 + 1, P_.x0:P_.x1 + 1] += 1
    u /= cnt
    ring = ring_nodes(0, N, 0, N)
    u[ring[:, 1], ring[:, 0]] = phi
    return u


def global_reference(aE, aN, N, phi):
    """Fine-mesh solution of the global problem by one sparse direct solve."""
    return box_solve(aE, aN, 0, N, 0, N, phi)


def rel_l2(a, b):
    """|a - b|_2 / |b|_2 over all nodes (reading R13)."""
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# ---------------------------------------------------------------------------
# the whole method
# ---------------------------------------------------------------------------

@dataclass
class Offline:
    aE: np.ndarray
    aN: np.ndarray
    patches: list
    R: list        # snapshots per patch (n_k, S)
    Q: list        # truncated bases
    sigma: list    # singular values per patch


def offline(mspec, pspec, seed, tau, patch_subset=None):
    """Offline stage of Algorithm alg:summary with RanLocalSolu."""
    aE, aN = face_coefficients(mspec)
    patches = patch_boxes(mspec.n_cells, pspec)
    sel = patches if patch_subset is None else [patches[i] for i in patch_subset]
    R, Q, S = [], [], []
    for P_ in sel:
        r = snapshots(aE, aN, P_, seed, mspec.n_cells)
        q, s = basis(r, tau)
        R.append(r); Q.append(q); S.append(s)
    return Offline(aE, aN, sel, R, Q, S)


def online(off: Offline, pspec, N, phi):
    """Online stage: assemble, solve the least-squares glue, reconstruct."""
    Pm, d, o = online_system(off.aE, off.aN, off.patches, off.Q, N, pspec, phi)
    c = online_solve(Pm, d)
    return reconstruct(off.patches, off.Q, c, o, N, phi), c, Pm, d


def online_constrained(off: Offline, pspec, N, phi):
    """Online stage with the boundary data imposed exactly and only the
    continuity conditions relaxed (the constrained least-squares variant)."""
    Pm, d, o, is_bnd = online_system_rows(off.aE, off.aN, off.patches, off.Q, N, pspec, phi)
    c = constrained_solve(Pm, d, is_bnd)
    return reconstruct(off.patches, off.Q, c, o, N, phi), c, Pm, d, is_bnd


# ---------------------------------------------------------------------------
# online stage by overlapping Schwarz on the reduced bases
# ---------------------------------------------------------------------------
#
# The paper leaves the online step to "a standard step in domain decomposition"
# (Sec. 3, before Algorithm alg:summary).  Besides the least-squares glue of Eq.
# elliptic_cond_reduced, the buffered patches K~_m give the classical overlapping
# choice: restricted additive Schwarz (Cai and Sarkis, 1999).  One step solves the
# local problem on every K~_m with the current field's values on its ring,
# keeps each solution on K_m only and averages shared nodes with the partition
# of unity chi_m of reading R10; domain-boundary ring nodes take phi.  On the
# reduced bases the local solve with ring data g is G~_m g restricted to K_m,
# replaced by its projection onto span Q_m, Q_m Q_m^T G~_m g, so each step is
#     c_m <- B_m g_m(c),   B_m = Q_m^T G~_m (k_m x n_ring),
# with g_m(c) the ring values of the reconstruction u(c) = sum_n chi_n Q_n c_n.
# The fixed point solves (I - T) c = F phi.  With the full basis (Q_m spanning
# the range of G~_m) the restriction of the global fine-grid solution is a fixed
# point, so the reconstruction reproduces it exactly.

def ras_ring_table(patches, N):
    """For every patch m, one entry per ring node of its buffered box, in ring
    order: ('phi', global ring position) for a node on the domain boundary,
    else ('u', [(n, local index of the node in K_n, chi_n)]) over the patches n
    whose closed box K_n holds the node (chi_n = 1 / their number, reading R10)."""
    ring_id = domain_ring_index(N)
    table = []
    for P_ in patches:
        ents = []
        for (i, j) in ring_nodes(P_.X0, P_.X1, P_.Y0, P_.Y1):
            i = int(i); j = int(j)
            if i in (0, N) or j in (0, N):
                ents.append(("phi", ring_id[(i, j)]))
                continue
            own = [Pn for Pn in patches if Pn.x0 <= i <= Pn.x1 and Pn.y0 <= j <= Pn.y1]
            ents.append(("u", [(Pn.m, (i - Pn.x0) + (j - Pn.y0) * (Pn.x1 - Pn.x0 + 1), 1.0 / len(own))
                               for Pn in own]))
        table.append(ents)
    return table


def ras_operators(aE, aN, patches, Qs, N):
    """T (N_p x N_p) and F (N_p x 4N), both sparse, of the reduced restricted
    additive Schwarz step c <- T c + F phi, and the coefficient offsets.
    B_m = Q_m^T G~_m with G~_m from DetLocalSolu (`full_green`)."""
    ks = [Q.shape[1] for Q in Qs]
    off = np.concatenate([[0], np.cumsum(ks)]).astype(int)
    table = ras_ring_table(patches, N)
    Tb = sp.lil_matrix((off[-1], off[-1]))
    Fb = sp.lil_matrix((off[-1], 4 * N))
    for P_, Q in zip(patches, Qs):
        m = P_.m
        Bm = Q.T @ full_green(aE, aN, P_)
        rows = slice(off[m], off[m + 1])
        Tm = np.zeros((ks[m], off[-1]))
        Fm = np.zeros((ks[m], 4 * N))
        for r, (kind, val) in enumerate(table[m]):
            if kind == "phi":
                Fm[:, val] += Bm[:, r]
            else:
                for (n, loc, chi) in val:
                    Tm[:, off[n]:off[n + 1]] += chi * np.outer(Bm[:, r], Qs[n][loc])
        Tb[rows] = Tm
        Fb[rows] = Fm
    return Tb.tocsr(), Fb.tocsr(), off


def ras_solve(T, F, phi):
    """The fixed point of the reduced Schwarz step: (I - T) c = F phi, by one
    sparse LU (the GPU iterates to it)."""
    A = (sp.identity(T.shape[0], format="csc") - T.tocsc()).tocsc()
    return spla.splu(A).solve(F @ np.asarray(phi, dtype=np.float64))


def ras_iterate(T, F, phi, c0, steps):
    """`steps` plain Schwarz steps c <- T c + F phi from c0."""
    c = np.array(c0, dtype=np.float64)
    f = F @ np.asarray(phi, dtype=np.float64)
    for _ in range(steps):
        c = T @ c + f
    return c


def online_ras(off: Offline, N, phi):
    """Online stage by the reduced overlapping Schwarz fixed point, then the
    reconstruction with the partition of unity."""
    T, F, o = ras_operators(off.aE, off.aN, off.patches, off.Q, N)
    c = ras_solve(T, F, phi)
    return reconstruct(off.patches, off.Q, c, o, N, phi), c, T, F

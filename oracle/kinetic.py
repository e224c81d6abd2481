"""Kinetic example (Sec. 4): plain FP64 restatement, discrete ordinates.

Problem (Eq. RTE with the Henyey-Greenstein kernel of Eq. HG):

    v d_x f(x, v) = (1/eps) L f,
    L f(v) = int k(v, v') f(v') dv' - (int k(v', v) dv') f(v),
    k(v, v') = (1/2) (1 - g^2) / (1 + g^2 + 2 g v v'),
    x in [0, 1], incoming data on Gamma_-: f(0, v>0) and f(1, v<0).
At g = 0, k = 1/2 and L f = rho - f with rho = (1/2) int f dv' (isotropic
scattering, the default throughout).

Discretisation (reading R11; the paper's own test uses a uniform velocity grid,
Sec. 4.3): nodes x_i = i dx, dx = 1/N; n_v Gauss-Legendre velocities v_l with
weights w_l (sum w = 2); the collision by the same quadrature,
    (L f)_l = sum_l' w_l' k(v_l, v_l') f_l' - sigma_l f_l,  sigma_l = sum_l' w_l' k(v_l', v_l),
(at g = 0: rho - f with rho = (1/2) sum_l w_l f_l); implicit upwind
    v_l > 0:  v_l (f_i - f_{i-1}) / dx = (L f_i)_l / eps,  i = X0+1 .. X1
    v_l < 0:  v_l (f_{i+1} - f_i) / dx = (L f_i)_l / eps,  i = X0 .. X1-1
on a node range [X0, X1] with f_{X0, v>0} and f_{X1, v<0} given.

Method (Algorithm alg:summary with RanLocalSolu, Sec. 4.2):
  * patches K_m = [x_{m}, x_{m+1}] (equal cells), buffered by b cells, clipped;
  * random incoming data on the buffered patch (n_v/2 values at each end,
    i.i.d. N(0,1), Philox stream TAG_KINETIC), local solve, restriction to
    K_m -> snapshots (n_k = (cells+1) n_v rows, node-major, velocity fastest);
  * SVD basis truncated at tau (as for the elliptic example);
  * online: all n_v velocity components continuous at every interface, plus the
    incoming boundary data (Eq. rte_cond_reduced), least squares;
  * reconstruction: patch values inside, average of the two patches at an
    interface, incoming components at x = 0, 1 set to the data.
Direct sparse solves replace the GPU's source iteration.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import philox


def velocities(n_v):
    """Gauss-Legendre nodes and weights on [-1, 1] (weights sum to 2), ascending."""
    v, w = np.polynomial.legendre.leggauss(n_v)
    return v, w


@dataclass
class KPatch:
    m: int
    x0: int
    x1: int
    X0: int
    X1: int
    S: int

    @property
    def n_nodes(self):
        return self.x1 - self.x0 + 1


def patches(n_cells, n_patches, buffer, samples):
    assert n_cells % n_patches == 0
    W = n_cells // n_patches
    out = []
    for m in range(n_patches):
        x0, x1 = m * W, (m + 1) * W
        out.append(KPatch(m, x0, x1, max(0, x0 - buffer), min(n_cells, x1 + buffer), samples))
    return out


def scattering(n_v, g=0.0):
    """Quadrature form of the Henyey-Greenstein collision (Eq. HG): the matrix
    Kw[l, l'] = w_l' k(v_l, v_l') and the loss rates sigma_l = sum_l' w_l' k(v_l', v_l),
    with k(v, v') = (1/2)(1 - g^2) / (1 + g^2 + 2 g v v')."""
    v, w = velocities(n_v)
    k = 0.5 * (1.0 - g * g) / (1.0 + g * g + 2.0 * g * np.outer(v, v))
    Kw = k * w[None, :]
    sigma = (w[:, None] * k).sum(axis=0)
    return Kw, sigma


def range_operator(n_cells, eps, n_v, X0, X1, g=0.0):
    """Sparse system for the unknowns of node range [X0, X1] and the map from the
    incoming data.  Unknown ordering: node-major, velocity fastest, over the
    (node, velocity) pairs that are not incoming data; incoming data ordering:
    the n_v/2 positive velocities at X0 (ascending v), then the n_v/2 negative
    velocities at X1 (ascending v).  Returns (A, Bin, unknown_index, data_index)
    with A u = Bin g, and the (node, velocity) -> index tables."""
    v, w = velocities(n_v)
    Kw, sigma = scattering(n_v, g)
    dx = 1.0 / n_cells
    pos = np.nonzero(v > 0)[0]
    neg = np.nonzero(v < 0)[0]
    nodes = range(X0, X1 + 1)
    uidx, didx = {}, {}
    for t, l in enumerate(pos):
        didx[(X0, l)] = t
    for t, l in enumerate(neg):
        didx[(X1, l)] = len(pos) + t
    for i in nodes:
        for l in range(n_v):
            if (i, l) not in didx:
                uidx[(i, l)] = len(uidx)
    rows, cols, vals = [], [], []
    brows, bcols, bvals = [], [], []

    def add(r, key, val):
        if key in uidx:
            rows.append(r); cols.append(uidx[key]); vals.append(val)
        else:   # incoming datum moves to the right-hand side
            brows.append(r); bcols.append(didx[key]); bvals.append(-val)

    for (i, l), r in uidx.items():
        # v_l (f_i - f_nbr)/dx + sigma_l f_i/eps - sum_l' Kw[l, l'] f_{i,l'}/eps = 0 with the
        # upwind neighbour
        nb = i - 1 if v[l] > 0 else i + 1
        a = abs(v[l]) / dx
        add(r, (i, l), a + sigma[l] / eps)
        add(r, (nb, l), -a)
        for ll in range(n_v):
            add(r, (i, ll), -Kw[l, ll] / eps)
    n = len(uidx)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(n, n))
    Bin = sp.csc_matrix((bvals, (brows, bcols)), shape=(n, len(didx)))
    return A, Bin, uidx, didx


def range_solve(n_cells, eps, n_v, X0, X1, data, g=0.0):
    """Solve on [X0, X1] for incoming data (n_v,) or (n_v, S); returns the full
    field, shape (X1-X0+1, n_v[, S]).  g: anisotropy of Eq. HG."""
    d = np.asarray(data, dtype=np.float64)
    vec = d.ndim == 1
    if vec:
        d = d[:, None]
    A, Bin, uidx, didx = range_operator(n_cells, eps, n_v, X0, X1, g)
    sol = spla.splu(A).solve(np.ascontiguousarray((Bin @ d)))
    F = np.zeros((X1 - X0 + 1, n_v, d.shape[1]))
    for (i, l), r in uidx.items():
        F[i - X0, l] = sol[r]
    for (i, l), t in didx.items():
        F[i - X0, l] = d[t]
    return F[..., 0] if vec else F


def sample_matrix(seed, patch, n_v):
    """Random incoming data of the buffered patch, (n_v, S) (Eq. rte_random)."""
    return philox.normals(seed, patch.m, n_v, patch.S, philox.TAG_KINETIC)


def snapshots(n_cells, eps, n_v, patch, seed, g=0.0):
    """Restricted local solutions: (n_nodes n_v, S), node-major, velocity fastest."""
    F = range_solve(n_cells, eps, n_v, patch.X0, patch.X1, sample_matrix(seed, patch, n_v), g)
    sub = F[patch.x0 - patch.X0:patch.x1 - patch.X0 + 1]
    return sub.reshape(patch.n_nodes * n_v, -1)


def basis(R, tau):
    U, s, _ = np.linalg.svd(R, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return U[:, :0], s
    k = int(np.count_nonzero(s > tau * s[0]))
    return U[:, :k], s


def online_system(pts, Qs, n_v, inflow_left, inflow_right):
    """Rows of Eq. rte_cond_reduced: at every interface x_m all n_v components of
    u_m and u_{m+1} agree; at x = 0 the positive-velocity components of u_0, at
    x = 1 the negative ones of u_{M-1}, equal the incoming data (given as full
    n_v-vectors; only the incoming half is used)."""
    v, _ = velocities(n_v)
    ks = [Q.shape[1] for Q in Qs]
    off = np.concatenate([[0], np.cumsum(ks)]).astype(int)
    M = len(pts)
    rows = []
    d = []
    for m in range(M - 1):
        Qa, Qb = Qs[m], Qs[m + 1]
        na = pts[m].n_nodes
        for l in range(n_v):
            r = np.zeros(off[-1])
            r[off[m]:off[m + 1]] = Qa[(na - 1) * n_v + l]
            r[off[m + 1]:off[m + 2]] = -Qb[0 * n_v + l]
            rows.append(r); d.append(0.0)
    for l in np.nonzero(v > 0)[0]:
        r = np.zeros(off[-1]); r[off[0]:off[1]] = Qs[0][l]; rows.append(r); d.append(inflow_left[l])
    nl = pts[-1].n_nodes
    for l in np.nonzero(v < 0)[0]:
        r = np.zeros(off[-1]); r[off[M - 1]:off[M]] = Qs[M - 1][(nl - 1) * n_v + l]; rows.append(r)
        d.append(inflow_right[l])
    return np.array(rows), np.array(d), off


def reconstruct(pts, Qs, c, off, n_cells, n_v, inflow_left, inflow_right):
    v, _ = velocities(n_v)
    f = np.zeros((n_cells + 1, n_v))
    cnt = np.zeros(n_cells + 1)
    for P, Q in zip(pts, Qs):
        vals = (Q @ c[off[P.m]:off[P.m + 1]]).reshape(P.n_nodes, n_v)
        f[P.x0:P.x1 + 1] += vals
        cnt[P.x0:P.x1 + 1] += 1
    f /= cnt[:, None]
    f[0, v > 0] = inflow_left[v > 0]
    f[n_cells, v < 0] = inflow_right[v < 0]
    return f


@dataclass
class KOffline:
    patches: list
    R: list
    Q: list
    sigma: list


def offline(n_cells, eps, n_v, n_patches, buffer, samples, seed, tau, g=0.0):
    pts = patches(n_cells, n_patches, buffer, samples)
    R, Q, S = [], [], []
    for P in pts:
        r = snapshots(n_cells, eps, n_v, P, seed, g)
        q, s = basis(r, tau)
        R.append(r); Q.append(q); S.append(s)
    return KOffline(pts, R, Q, S)


def online(off: KOffline, n_cells, n_v, inflow_left, inflow_right):
    Pm, d, o = online_system(off.patches, off.Q, n_v, inflow_left, inflow_right)
    c, *_ = np.linalg.lstsq(Pm, d, rcond=None)
    return reconstruct(off.patches, off.Q, c, o, n_cells, n_v, inflow_left, inflow_right), c


def global_reference(n_cells, eps, n_v, inflow_left, inflow_right, g=0.0):
    """Direct solve of the whole slab with the incoming data."""
    v, _ = velocities(n_v)
    d = np.concatenate([inflow_left[v > 0], inflow_right[v < 0]])
    return range_solve(n_cells, eps, n_v, 0, n_cells, d, g)


def full_green(n_cells, eps, n_v, patch, g=0.0):
    """Restricted Green's matrix of the buffered patch (DetLocalSolu for the slab:
    one unit datum per incoming component), (n_nodes n_v, n_v)."""
    F = range_solve(n_cells, eps, n_v, patch.X0, patch.X1, np.eye(n_v), g)
    sub = F[patch.x0 - patch.X0:patch.x1 - patch.X0 + 1]
    return sub.reshape(patch.n_nodes * n_v, -1)

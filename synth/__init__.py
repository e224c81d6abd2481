"""Seeded synthetic workloads for the random-sampling multiscale solver.

This module only *draws and lays out inputs*: media descriptions (the random
Fourier modes or channel geometry a medium is built from), patch partitions,
per-patch sample counts, global Dirichlet data on the boundary ring, kinetic
inflow data and request arrival times.  It holds none of the method's
arithmetic: it never evaluates a coefficient field on the mesh, never forms an
operator, never draws the Gaussian boundary samples of the local solves (those
come from a counter-based generator that each implementation writes itself)
and never solves anything.  Both the CPU oracle and the CUDA library consume
what it returns; neither imports the other.

Workloads are shaped like the paper's examples: the elliptic problem of
Sec. 5 (Eq. 5.1-5.2 on [0,1]^2, Dirichlet data on the boundary) and the
slab radiative transfer problem of Sec. 4 (Eq. 4.1 with incoming data on
Gamma_-).  There is no public dataset behind the paper; every input here is
synthetic.

Layout conventions shared by every consumer (each consumer implements them on
its own):

* Fine grid: N cells per side, n = N + 1 nodes, h = 1/N; node (i, j) sits at
  (i h, j h); grids are stored row-major with i (x) fastest.
* Boundary ring of a node box [X0, X1] x [Y0, Y1]: counter-clockwise from the
  bottom-left corner, every node once -- bottom edge i = X0..X1-1 at j = Y0,
  right edge j = Y0..Y1-1 at i = X1, top edge i = X1..X0+1 at j = Y1, left
  edge j = Y1..Y0+1 at i = X0.  2 (X1-X0) + 2 (Y1-Y0) nodes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# medium kinds (same integer codes as the C header)
MEDIUM_PERIODIC_SIN = 0
MEDIUM_LOGNORMAL = 1
MEDIUM_CHANNELS = 2
MEDIUM_HOU_WU = 3
MEDIUM_USER = 4


@dataclass
class MediumSpec:
    """Description of a coefficient field a(x) on [0,1]^2.

    kind:   one of the MEDIUM_* codes.
    n_cells: N, cells per side of the fine grid.
    eps:    oscillation scale epsilon.
    modes:  (Q, 4) float64 rows (kx, ky, A, B) for the log-normal medium
            a = exp(amp * g), g = sum_q [A cos(2 pi k.x) + B sin(2 pi k.x)] * norm.
    amp, norm: log-normal amplitude and per-mode normalisation.
    channels: (C, 3) float64 rows (px, py, theta) for the channel medium:
            a = contrast inside a strip of width `width` through (px, py) at
            angle theta, background 1 elsewhere.
    user_aE, user_aN: explicit face coefficients for MEDIUM_USER, shapes
            (N+1, N) and (N, N+1) (row j, column i).
    """
    kind: int
    n_cells: int
    eps: float
    modes: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))
    amp: float = 0.5
    norm: float = 1.0
    channels: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    width: float = 0.0
    contrast: float = 1.0
    user_aE: np.ndarray | None = None
    user_aN: np.ndarray | None = None


def periodic_sin(n_cells: int, eps: float) -> MediumSpec:
    """a(x, y) = 2 + sin(2 pi x/eps) sin(2 pi y/eps) (the small elliptic workload)."""
    return MediumSpec(MEDIUM_PERIODIC_SIN, n_cells, eps)


def hou_wu(n_cells: int, eps: float) -> MediumSpec:
    """The two-scale medium of the paper's elliptic numerical test (Sec. 5.3)."""
    return MediumSpec(MEDIUM_HOU_WU, n_cells, eps)


def lognormal(n_cells: int, eps: float, n_modes: int, seed: int,
              amp: float = 0.5, normalised: bool = True) -> MediumSpec:
    """Log-normal medium a = exp(amp * g) from `n_modes` random Fourier modes.

    Wave vectors k in Z^2 are drawn uniformly from the lattice points with
    1 <= |k| <= 1/eps; the cosine and sine amplitudes are i.i.d. N(0,1).
    With `normalised` the sum is scaled by 1/sqrt(n_modes) so Var g ~ 1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    kmax = 1.0 / eps
    r = int(math.floor(kmax))
    kx, ky = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), indexing="ij")
    kx = kx.ravel(); ky = ky.ravel()
    rad = np.hypot(kx, ky)
    keep = (rad >= 1.0) & (rad <= kmax + 1e-12)
    lattice = np.stack([kx[keep], ky[keep]], axis=1).astype(np.float64)
    pick = rng.integers(0, lattice.shape[0], size=n_modes)
    ab = rng.standard_normal((n_modes, 2))
    modes = np.concatenate([lattice[pick], ab], axis=1)
    norm = 1.0 / math.sqrt(n_modes) if normalised else 1.0
    return MediumSpec(MEDIUM_LOGNORMAL, n_cells, eps, modes=modes, amp=amp, norm=norm)


def channels(n_cells: int, eps: float, n_channels: int, seed: int,
             contrast: float = 1e3) -> MediumSpec:
    """High-contrast medium: background 1, `contrast` inside straight strips of
    width eps through a seeded random point at a seeded random angle."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.uniform(0.0, 1.0, size=(n_channels, 2))
    th = rng.uniform(0.0, math.pi, size=(n_channels, 1))
    return MediumSpec(MEDIUM_CHANNELS, n_cells, eps, channels=np.concatenate([pts, th], axis=1),
                      width=eps, contrast=contrast)


def user_medium(aE: np.ndarray, aN: np.ndarray) -> MediumSpec:
    """Explicit face coefficients: aE shape (N+1, N), aN shape (N, N+1)."""
    aE = np.ascontiguousarray(aE, dtype=np.float64)
    aN = np.ascontiguousarray(aN, dtype=np.float64)
    n_cells = aE.shape[1]
    assert aE.shape == (n_cells + 1, n_cells) and aN.shape == (n_cells, n_cells + 1)
    return MediumSpec(MEDIUM_USER, n_cells, 1.0, user_aE=aE, user_aN=aN)


@dataclass
class PatchSpec:
    """Non-overlapping tensor partition of the N x N cells into patches.

    x_breaks, y_breaks: increasing cell indices starting at 0 and ending at N;
    patch (p, q) covers cells [x_breaks[p], x_breaks[p+1]] x [y_breaks[q], y_breaks[q+1]].
    Patch index m = p + q * (len(x_breaks) - 1) (p fastest).
    buffers: per-patch buffer width in cells.
    samples: per-patch sample count S_m.
    """
    x_breaks: np.ndarray
    y_breaks: np.ndarray
    buffers: np.ndarray
    samples: np.ndarray

    @property
    def nx(self) -> int:
        return len(self.x_breaks) - 1

    @property
    def ny(self) -> int:
        return len(self.y_breaks) - 1

    @property
    def n_patches(self) -> int:
        return self.nx * self.ny


def uniform_patches(n_cells: int, mx: int, my: int, buffer: int, samples: int) -> PatchSpec:
    assert n_cells % mx == 0 and n_cells % my == 0
    xb = np.arange(mx + 1, dtype=np.int32) * (n_cells // mx)
    yb = np.arange(my + 1, dtype=np.int32) * (n_cells // my)
    m = mx * my
    return PatchSpec(xb, yb, np.full(m, buffer, np.int32), np.full(m, samples, np.int32))


def uneven_patches(n_cells: int, seed: int, widths=(16, 32, 48, 64, 80, 96),
                   sample_choices=(64, 128, 192, 256)) -> PatchSpec:
    """Uneven tensor partition: widths drawn from `widths` until they fill N per
    axis (the last one clipped to fit), buffer = min(width_x, width_y) // 4,
    samples per patch drawn from `sample_choices`."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def axis():
        br = [0]
        while br[-1] < n_cells:
            w = int(rng.choice(widths))
            br.append(min(n_cells, br[-1] + w))
        if br[-1] - br[-2] < min(widths):      # merge a sliver into its neighbour
            br.pop(-2)
        return np.array(br, dtype=np.int32)

    xb = axis(); yb = axis()
    mx, my = len(xb) - 1, len(yb) - 1
    buf = np.empty(mx * my, np.int32)
    for q in range(my):
        for p in range(mx):
            buf[p + q * mx] = min(xb[p + 1] - xb[p], yb[q + 1] - yb[q]) // 4
    samples = rng.choice(np.asarray(sample_choices), size=mx * my).astype(np.int32)
    return PatchSpec(xb, yb, buf, samples)


def domain_ring_xy(n_cells: int):
    """Coordinates (x, y) of the global boundary ring nodes, counter-clockwise
    from (0, 0); 4N nodes."""
    N = n_cells
    i = np.concatenate([np.arange(0, N), np.full(N, N), np.arange(N, 0, -1), np.zeros(N, int)])
    j = np.concatenate([np.zeros(N, int), np.arange(0, N), np.full(N, N), np.arange(N, 0, -1)])
    return i / N, j / N


def phi_sin_cos(n_cells: int) -> np.ndarray:
    """Dirichlet data phi = sin(2 pi x) + cos(2 pi y) on the boundary ring."""
    x, y = domain_ring_xy(n_cells)
    return np.sin(2 * np.pi * x) + np.cos(2 * np.pi * y)


def phi_fourier(n_cells: int, n_modes: int, seed: int, kmax: int = 8, batch: int = 1) -> np.ndarray:
    """`batch` Dirichlet data sets, each a sum of `n_modes` random Fourier modes
    with integer wave vectors |k| <= kmax and N(0,1) amplitudes, on the ring.
    Returns shape (batch, 4N)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y = domain_ring_xy(n_cells)
    out = np.empty((batch, x.size))
    for b in range(batch):
        k = rng.integers(-kmax, kmax + 1, size=(n_modes, 2))
        a = rng.standard_normal((n_modes, 2))
        ph = 2 * np.pi * (np.outer(k[:, 0], x) + np.outer(k[:, 1], y))
        out[b] = (a[:, :1] * np.cos(ph) + a[:, 1:] * np.sin(ph)).sum(0) / math.sqrt(n_modes)
    return out


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given mean rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def kinetic_inflow_paper(v: np.ndarray):
    """Incoming data of the paper's global RTE test (Sec. 4.3):
    3 + sin(2 pi v) at x = 0 for v > 0, 2 + sin(2 pi v) at x = 1 for v < 0.
    Returns the values at the given velocity nodes (caller keeps the half that
    is incoming on each side)."""
    v = np.asarray(v, dtype=np.float64)
    return 3.0 + np.sin(2 * np.pi * v), 2.0 + np.sin(2 * np.pi * v)


# ---------------------------------------------------------------------------
# the five synthetic workloads
# ---------------------------------------------------------------------------

def workload_small():
    """129 x 129 nodes, a = 2 + sin sin, eps = 1/16, 4 x 4 patches, 8-cell buffer,
    40 samples per patch (seed 0), truncation 1e-6, online tolerance 1e-8."""
    N = 128
    return dict(name="elliptic-129-periodic", medium=periodic_sin(N, 1.0 / 16),
                patches=uniform_patches(N, 4, 4, 8, 40), seed=0, tau=1e-6,
                online_tol=1e-8, phi=phi_sin_cos(N))


def workload_batched(normalised: bool = True):
    """2049 x 2049 nodes, log-normal medium eps = 2^-7 (64 modes, seed 1),
    32 x 32 patches, 16-cell buffer, 128 samples per patch (131072 solves)."""
    N = 2048
    return dict(name="elliptic-2049-lognormal", medium=lognormal(N, 2.0 ** -7, 64, 1, normalised=normalised),
                patches=uniform_patches(N, 32, 32, 16, 128), seed=1, tau=1e-6,
                online_tol=1e-8, phi=phi_sin_cos(N))


def workload_uneven():
    """1025 x 1025 nodes, eps = 2^-6, 8 channels of contrast 1e3 (seed 2), uneven
    patches 16-96 cells, buffers 4-24, 64-256 samples per patch."""
    N = 1024
    return dict(name="elliptic-1025-channels-uneven", medium=channels(N, 2.0 ** -6, 8, 2),
                patches=uneven_patches(N, 2), seed=2, tau=1e-6, online_tol=1e-8,
                phi=phi_sin_cos(N))


def workload_serving():
    """Three prebuilt log-normal media 513^2, 1025^2, 2049^2 (eps 2^-5..2^-7), 64-cell
    patches with 16-cell buffers, 128 samples; Poisson arrivals at 2000 req/s (seed 3)."""
    media = []
    for N, e, sd in ((512, 2.0 ** -5, 11), (1024, 2.0 ** -6, 12), (2048, 2.0 ** -7, 13)):
        media.append(dict(medium=lognormal(N, e, 64, sd), patches=uniform_patches(N, N // 64, N // 64, 16, 128)))
    return dict(name="serving-lognormal-3media", media=media, rate_hz=2000.0, seed=3)


def workload_kinetic():
    """Slab RTE, eps = 2^-8, 8192 cells, 64 Gauss-Legendre velocities, 64 patches,
    32-cell buffer, 96 random inflow samples per patch (seed 4)."""
    return dict(name="kinetic-8192-gl64", n_cells=8192, eps=2.0 ** -8, n_v=64, n_patches=64,
                buffer=32, samples=96, seed=4)

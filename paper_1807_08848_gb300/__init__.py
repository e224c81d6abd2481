"""GB300 random-sampling multiscale solver (arXiv:1807.08848) -- Python binding.

Thin wrapper over the C ABI of libmsp.so (include/msp.h).  PyTorch supplies
device memory and streams; every step of the method runs in the library's
CUDA kernels.  There is no CPU fallback: without the built library or a CUDA
device the calls raise.

    med = Medium(medium_spec, patch_spec)          # msp_build_medium
    stats = med.sample(seed, "mixed", 1e-10)       # msp_sample_patches
    basis = med.extract(1e-6)                      # msp_extract_basis
    u, iters = basis.solve(phi)                    # msp_online_solve
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N
from ._native import MspError, MSP_FP64, MSP_MIXED

__all__ = ["Medium", "Basis", "Server", "KineticMedium", "KineticBasis", "MspError", "MSP_FP64", "MSP_MIXED", "load_library",
           "precision_code", "set_wait_limit", "set_gemm_engine", "set_extract_timing", "set_svd_mode"]


def load_library():
    return N.load()


def set_wait_limit(polls: int = 0):
    """Poll bound of the device-side grid barriers (msp_set_wait_limit); 0 restores
    the default."""
    N.check(N.load().msp_set_wait_limit(int(polls)))


def set_extract_timing(enable: bool = True):
    """CUDA-event timing of the extraction's phases (msp_set_extract_timing)."""
    N.check(N.load().msp_set_extract_timing(1 if enable else 0))


def set_gemm_engine(engine: str = "tensor_cores"):
    """FP64 products of the extraction and the online factorisation on the tensor
    cores (error-free BF16 slicing, the default) or on the CUDA cores."""
    N.check(N.load().msp_set_gemm_engine({"tensor_cores": 0, "cuda_cores": 1}[engine]))


def set_svd_mode(mode: str = "qr_preconditioned"):
    """Jacobi SVD of the extraction: a pivoted QR first and the FP64 sweeps on R^T
    (the default), FP64 sweeps from the identity, or FP32 sweeps re-orthogonalised
    then FP64 sweeps (msp_set_svd_mode)."""
    N.check(N.load().msp_set_svd_mode({"fp64": 0, "fp32_preconditioned": 1, "qr_preconditioned": 2}[mode]))


def precision_code(p) -> int:
    if isinstance(p, int):
        return p
    return {"fp64": MSP_FP64, "mixed": MSP_MIXED}[str(p).lower()]


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _f64p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class Medium:
    """Medium, patch decomposition and snapshot storage on the device.

    medium: object with kind, n_cells, eps, modes, amp, norm, channels, width,
            contrast, user_aE, user_aN (e.g. synth.MediumSpec).
    patches: object with x_breaks, y_breaks, buffers, samples (e.g. synth.PatchSpec).
    full_basis: DetLocalSolu -- one delta column per ring node of every buffered
            patch and no Gaussian columns (msp_build_medium_full; samples ignored).
    """

    def __init__(self, medium, patches, stream=None, full_basis: bool = False):
        lib = N.load()
        self._keep = []
        d = N.MediumDesc()
        d.kind = int(medium.kind)
        d.n_cells = int(medium.n_cells)
        d.eps = float(medium.eps)
        modes = np.ascontiguousarray(np.asarray(medium.modes, dtype=np.float64).reshape(-1, 4))
        chans = np.ascontiguousarray(np.asarray(medium.channels, dtype=np.float64).reshape(-1, 3))
        self._keep += [modes, chans]
        d.n_modes = modes.shape[0]
        d.modes_host = _f64p(modes)
        d.amp = float(medium.amp)
        d.norm = float(medium.norm)
        d.n_channels = chans.shape[0]
        d.channels_host = _f64p(chans)
        d.width = float(medium.width)
        d.contrast = float(medium.contrast)
        if medium.user_aE is not None:
            aE = np.ascontiguousarray(medium.user_aE, dtype=np.float64)
            aN = np.ascontiguousarray(medium.user_aN, dtype=np.float64)
            self._keep += [aE, aN]
            d.user_aE_host = _f64p(aE)
            d.user_aN_host = _f64p(aN)
        xb = np.ascontiguousarray(patches.x_breaks, dtype=np.int32)
        yb = np.ascontiguousarray(patches.y_breaks, dtype=np.int32)
        bu = np.ascontiguousarray(patches.buffers, dtype=np.int32)
        sa = np.ascontiguousarray(patches.samples, dtype=np.int32)
        self._keep += [xb, yb, bu, sa]
        p = N.PatchDesc(len(xb) - 1, len(yb) - 1, _i32p(xb), _i32p(yb), _i32p(bu), _i32p(sa))
        h = C.c_void_p()
        build = lib.msp_build_medium_full if full_basis else lib.msp_build_medium
        N.check(build(C.byref(d), C.byref(p), _stream_ptr(stream), C.byref(h)))
        self._h = h
        self._keep = []
        npch, ne, nc = C.c_int(), C.c_int64(), C.c_int()
        N.check(lib.msp_medium_counts(h, C.byref(npch), C.byref(ne), C.byref(nc)))
        self.n_patches, self.snapshot_elems, self.n_cells = npch.value, ne.value, nc.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            N.load().msp_medium_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def patch(self, m: int) -> N.PatchInfo:
        info = N.PatchInfo()
        N.check(N.load().msp_medium_patch(self._h, m, C.byref(info)))
        return info

    def set_launch(self, precision="mixed", mode="split", rows: int = 0):
        """Launch of the local solves: 'split' (tile kernel + global kernel) or 'fused'
        (one persistent launch); rows per thread segment 4/8/12 (0: smallest that fits)."""
        N.check(N.load().msp_medium_set_launch(self._h, precision_code(precision), {"split": 0, "fused": 1, "direct": 2}[mode],
                                               rows))

    def set_timing(self, enable: bool = True):
        """CUDA-event timing of the direct solver's phases (msp_medium_set_timing)."""
        N.check(N.load().msp_medium_set_timing(self._h, 1 if enable else 0))

    def direct_timing(self) -> dict:
        """Milliseconds and launches per phase of the last direct-solver call."""
        ms = (C.c_double * 5)()
        nl = (C.c_int * 5)()
        N.check(N.load().msp_medium_direct_timing(self._h, ms, nl))
        names = ("factor", "init", "residual", "solve", "finish")
        return {n: {"ms": ms[i], "launches": nl[i]} for i, n in enumerate(names)}

    def set_graph(self, enable: bool = True):
        """Replay the local-solve launches from a CUDA graph (captured on first use)."""
        N.check(N.load().msp_medium_set_graph(self._h, 1 if enable else 0))

    def autotune(self, seed: int, precision="mixed", tol: float = 1e-10, max_iter: int = 20000,
                 max_probe_items: int = 2048, stream=None) -> dict:
        """Time every launch configuration (CG on a subset of the columns, the direct
        solver on the whole medium) and keep the fastest."""
        r = N.TuneReport()
        N.check(N.load().msp_medium_autotune(self._h, precision_code(precision), C.c_uint64(seed), tol, max_iter,
                                             max_probe_items, _stream_ptr(stream), C.byref(r)))
        names = ["split", "fused", "direct"]
        return {"probe_items": r.probe_items, "best_mode": names[r.best_mode],
                "best_rows": r.best_rows, "best_ms": r.best_ms,
                "candidates": [{"mode": names[c.mode], "rows": c.rows, "ms": c.ms}
                               for c in r.candidates[:r.n_candidates]]}

    def tile_shape(self):
        """(rows, cols) of the largest buffered box."""
        r, c = C.c_int(), C.c_int()
        N.check(N.load().msp_operator_tile_shape(self._h, C.byref(r), C.byref(c)))
        return r.value, c.value

    def apply_operator(self, x: torch.Tensor, precision="mixed", y: torch.Tensor | None = None, stream=None,
                       timed: bool = False):
        """y = A x on every tile of x, shape (n_patches, S, rows, pitch); float32 for
        'mixed', float64 for 'fp64'.  With timed, returns (y, device ms)."""
        dt = torch.float32 if precision_code(precision) == MSP_MIXED else torch.float64
        assert x.dtype == dt and x.is_cuda and x.is_contiguous() and x.dim() == 4
        if y is None:
            y = torch.empty_like(x)
        ms = C.c_double(0.0)
        N.check(N.load().msp_apply_operator(self._h, x.shape[1], precision_code(precision), _dptr(x), _dptr(y),
                                            x.shape[3], x.shape[2], C.byref(ms) if timed else None,
                                            _stream_ptr(stream)))
        return (y, ms.value) if timed else y

    def coefficients(self, stream=None):
        n = self.n_cells
        aE = torch.empty((n + 1, n), dtype=torch.float64, device="cuda")
        aN = torch.empty((n, n + 1), dtype=torch.float64, device="cuda")
        N.check(N.load().msp_get_coefficients(self._h, _dptr(aE), _dptr(aN), _stream_ptr(stream)))
        return aE, aN

    def sample(self, seed: int, precision="fp64", tol: float = 1e-12, max_iter: int = 20000, stream=None,
               stats: bool = True):
        st = N.SolveStats()
        code = N.load().msp_sample_patches(self._h, C.c_uint64(seed), precision_code(precision), tol, max_iter,
                                           _stream_ptr(stream), C.byref(st) if stats else None)
        N.check(code)
        return st if stats else None

    def sample_patches(self, patches, seed: int, precision="fp64", tol: float = 1e-12, max_iter: int = 20000,
                       stream=None):
        """Local solves of the listed patches only (msp_sample_patch_list)."""
        lst = np.ascontiguousarray(np.asarray(patches, dtype=np.int32).ravel())
        st = N.SolveStats()
        N.check(N.load().msp_sample_patch_list(self._h, _i32p(lst), int(lst.size), C.c_uint64(seed),
                                               precision_code(precision), tol, max_iter, _stream_ptr(stream),
                                               C.byref(st)))
        return st

    def set_snapshots(self, m: int, block: torch.Tensor, stream=None):
        """Write patch m's snapshot block, an (n_k, cols) tensor as snapshots()
        returns it (stored column-major)."""
        info = self.patch(m)
        assert tuple(block.shape) == (info.n_k, info.cols)
        t = block.to(dtype=torch.float64, device="cuda").T.contiguous()     # (cols, n_k) row-major
        N.check(N.load().msp_set_snapshots(self._h, m, _dptr(t), _stream_ptr(stream)))
        (stream or torch.cuda.current_stream()).synchronize()

    def snapshots(self, m: int, stream=None) -> torch.Tensor:
        """Snapshot block of patch m as an (n_k, cols) tensor (column-major storage)."""
        info = self.patch(m)
        t = torch.empty((info.cols, info.n_k), dtype=torch.float64, device="cuda")
        N.check(N.load().msp_get_snapshots(self._h, m, _dptr(t), _stream_ptr(stream)))
        return t.T

    def samples(self, m: int, seed: int, stream=None) -> torch.Tensor:
        """Ring data of patch m, (n_ring, cols)."""
        info = self.patch(m)
        t = torch.empty((info.cols, info.n_ring), dtype=torch.float64, device="cuda")
        N.check(N.load().msp_get_samples(self._h, m, C.c_uint64(seed), _dptr(t), _stream_ptr(stream)))
        return t.T

    def extract(self, tau: float = 1e-6, precision="fp64", stream=None) -> "Basis":
        h = C.c_void_p()
        N.check(N.load().msp_extract_basis(self._h, tau, precision_code(precision), _stream_ptr(stream), C.byref(h)))
        return Basis(h, self)


class Basis:
    """Reduced bases Q_m and the online operators of one medium."""

    def __init__(self, handle, medium: Medium | None = None):
        self._h = handle
        nc, npt = C.c_int(), C.c_int()
        N.check(N.load().msp_basis_patch(handle, 0, C.byref(nc), C.byref(npt), None))
        self.n_cells, self.n_patches = nc.value, npt.value
        infos = []
        for m in range(self.n_patches):
            info = N.PatchInfo()
            N.check(N.load().msp_basis_patch(handle, m, None, None, C.byref(info)))
            infos.append(info)
        self._cols = [i.cols for i in infos]
        self._nk = [i.n_k for i in infos]
        nu, nr = C.c_int(), C.c_int()
        N.check(N.load().msp_online_counts(handle, C.byref(nu), C.byref(nr)))
        self.n_unknowns, self.n_rows = nu.value, nr.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            N.load().msp_basis_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def extract_timing(self) -> dict:
        """Milliseconds per phase of the extraction that built this basis (timing on
        through set_extract_timing) and the Jacobi SVD's algorithmic FP64 flop."""
        ms = (C.c_double * 6)()
        jf = C.c_double()
        N.check(N.load().msp_basis_extract_timing(self._h, ms, C.byref(jf)))
        names = ("cholqr", "jacobi_start", "jacobi", "projection", "online_operators", "online_factor")
        return {**{n: ms[i] for i, n in enumerate(names)}, "jacobi_flop": jf.value}

    def stats(self) -> dict:
        st = N.BasisStats()
        N.check(N.load().msp_basis_get_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def set_preconditioner(self, kind: str):
        """'block_rows' (block-tridiagonal factor, default), 'patch_blocks',
        'block_rows_fp64' (an FP64 factor always applied in FP64) or
        'block_rows_fp32' (an FP64 factor always applied through its FP32 copy)."""
        code = {"block_rows": 0, "patch_blocks": 1, "block_rows_fp64": 2, "block_rows_fp32": 3}[kind]
        N.check(N.load().msp_basis_set_preconditioner(self._h, code))

    def k(self, m: int) -> int:
        k = C.c_int()
        N.check(N.load().msp_basis_info(self._h, m, C.byref(k), None))
        return k.value

    def sigma(self, m: int) -> np.ndarray:
        out = np.zeros(self._cols[m])
        k = C.c_int()
        N.check(N.load().msp_basis_info(self._h, m, C.byref(k), _f64p(out)))
        return out

    def Q(self, m: int, stream=None) -> torch.Tensor:
        k = self.k(m)
        t = torch.empty((k, self._nk[m]), dtype=torch.float64, device="cuda")
        if k:
            N.check(N.load().msp_get_basis(self._h, m, _dptr(t), _stream_ptr(stream)))
        return t.T

    def solve(self, phi: torch.Tensor, tol: float = 1e-10, max_iter: int = 5000, stream=None,
              want_c: bool = False, want_iters: bool = True, u: torch.Tensor | None = None,
              constrained: bool = False, schwarz: bool = False):
        """Online solve for phi of shape (B, 4N) (or (4N,)) on the device: the
        least-squares glue (msp_online_solve), with constrained=True the
        variant that imposes the boundary data exactly
        (msp_online_solve_constrained), or with schwarz=True the overlapping
        Schwarz variant (msp_online_solve_ras; after setup_schwarz)."""
        squeeze = phi.dim() == 1
        phi = phi.reshape(-1, 4 * self.n_cells).to(dtype=torch.float64, device="cuda").contiguous()
        B = phi.shape[0]
        n = self.n_cells + 1
        if u is None:
            u = torch.empty((B, n, n), dtype=torch.float64, device="cuda")
        c = torch.empty((B, self.n_unknowns), dtype=torch.float64, device="cuda") if want_c else None
        iters = (C.c_int * B)() if want_iters else None
        lib = N.load()
        fn = lib.msp_online_solve_ras if schwarz else (
            lib.msp_online_solve_constrained if constrained else lib.msp_online_solve)
        code = fn(self._h, _dptr(phi), B, tol, max_iter, _dptr(u), _dptr(c) if c is not None else None, iters,
                  _stream_ptr(stream))
        N.check(code)
        it = np.array(list(iters), dtype=np.int64) if want_iters else None
        if squeeze:
            u = u[0]
            c = c[0] if c is not None else None
        return (u, it, c) if want_c else (u, it)


    def setup_schwarz(self, full: "Medium", coarse: bool = True, stream=None):
        """Operators of the overlapping Schwarz online variant (msp_ras_setup) from
        a sampled full-basis medium of the same grid and partition."""
        N.check(N.load().msp_ras_setup(self._h, full.handle, 1 if coarse else 0, _stream_ptr(stream)))

    def save(self, path: str):
        """Write the bases, singular values, geometry and face coefficients to a file."""
        N.check(N.load().msp_save_basis(self._h, str(path).encode()))

    @classmethod
    def load(cls, path: str) -> "Basis":
        """Read a basis file on the current device (the online operators are rebuilt)."""
        h = C.c_void_p()
        N.check(N.load().msp_load_basis(str(path).encode(), C.byref(h)))
        return cls(h)

    def online_system(self, phi):
        """(rows, cols, vals, d) of P~ (COO) and d for ring data phi (host arrays)."""
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        nnz = C.c_int64()
        d = np.empty(self.n_rows, dtype=np.float64)
        pd = phi.ctypes.data_as(C.POINTER(C.c_double))
        N.check(N.load().msp_get_online_system(self._h, pd, 0, C.byref(nnz), None, None, None,
                                               d.ctypes.data_as(C.POINTER(C.c_double))))
        r = np.empty(nnz.value, dtype=np.int32)
        c = np.empty(nnz.value, dtype=np.int32)
        v = np.empty(nnz.value, dtype=np.float64)
        N.check(N.load().msp_get_online_system(self._h, pd, nnz.value, C.byref(nnz),
                                               r.ctypes.data_as(C.POINTER(C.c_int)), c.ctypes.data_as(C.POINTER(C.c_int)),
                                               v.ctypes.data_as(C.POINTER(C.c_double)), None))
        return r, c, v, d

    def build_map(self, tol: float = 1e-10, max_iter: int = 5000, stream=None):
        """Boundary-to-coefficient map c = G phi (FP32 on the device) for serving."""
        N.check(N.load().msp_basis_build_map(self._h, tol, max_iter, _stream_ptr(stream)))

    def set_map_engine(self, engine: str):
        """'tensor_cores' (tcgen05, default) or 'cuda_cores' for the map GEMM."""
        N.check(N.load().msp_basis_set_map_engine(self._h, {"tensor_cores": 0, "cuda_cores": 1}[engine]))

    def solve_map(self, phi: torch.Tensor, stream=None, u: torch.Tensor | None = None) -> torch.Tensor:
        """u for phi of shape (B, 4N) (or (4N,)) through the map."""
        squeeze = phi.dim() == 1
        phi = phi.reshape(-1, 4 * self.n_cells).to(dtype=torch.float64, device="cuda").contiguous()
        B = phi.shape[0]
        n = self.n_cells + 1
        if u is None:
            u = torch.empty((B, n, n), dtype=torch.float64, device="cuda")
        N.check(N.load().msp_online_solve_map(self._h, _dptr(phi), B, _dptr(u), _stream_ptr(stream)))
        return u[0] if squeeze else u


class Server:
    """Request loop over prebuilt media (bases with maps): submit boundary data,
    poll, fetch.  Worker threads batch requests of one medium under slot and
    device-memory limits; n_workers = 0 runs batches only on step()."""

    def __init__(self, media: list, mem_budget_bytes: int, max_slots: int = 256, max_batch: int = 32,
                 n_workers: int = 2):
        arr = (C.c_void_p * len(media))(*[b._h.value if isinstance(b._h, C.c_void_p) else b._h for b in media])
        h = C.c_void_p()
        N.check(N.load().msp_server_create(arr, len(media), int(mem_budget_bytes), max_slots, max_batch, n_workers,
                                           C.byref(h)))
        self._h = h
        self._media = list(media)   # keep the bases alive
        self._n = [b.n_cells for b in media]

    def submit(self, medium: int, phi) -> int:
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
        if phi.size != 4 * self._n[medium]:
            raise ValueError("phi must hold the 4N ring values of the medium")
        rid = C.c_uint64()
        N.check(N.load().msp_server_submit(self._h, medium, phi.ctypes.data_as(C.POINTER(C.c_double)),
                                           C.byref(rid)))
        return rid.value

    def poll(self, rid: int):
        """(done, latency_ms): done = 1 finished, 0 pending."""
        d, lat = C.c_int(), C.c_double()
        N.check(N.load().msp_server_poll(self._h, rid, C.byref(d), C.byref(lat)))
        return d.value, lat.value

    def fetch(self, rid: int, medium: int) -> np.ndarray:
        n = self._n[medium] + 1
        u = np.empty((n, n), dtype=np.float64)
        N.check(N.load().msp_server_fetch(self._h, rid, u.ctypes.data_as(C.POINTER(C.c_double))))
        return u

    def release(self, rid: int):
        N.check(N.load().msp_server_release(self._h, rid))

    def step(self, stream=None) -> int:
        n = C.c_int()
        N.check(N.load().msp_server_step(self._h, _stream_ptr(stream), C.byref(n)))
        return n.value

    def set_engine(self, engine: str = "map", tol: float = 1e-8, max_iter: int = 1000):
        """Batch solves by the map ("map") or by the plain FP64 iteration
        ("iterative_fp64", to tol / max_iter)."""
        code = {"map": 0, "iterative_fp64": 1}[engine]
        N.check(N.load().msp_server_set_engine(self._h, code, tol, max_iter))

    def stats(self) -> dict:
        st = N.ServerStats()
        N.check(N.load().msp_server_get_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self._h:
            N.load().msp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


KINETIC_SOLVERS = {"source_iteration": 0, "direct": 1}


class KineticMedium:
    """Slab radiative transfer, discrete ordinates, with the Henyey-Greenstein
    collision of anisotropy g (g = 0: isotropic scattering)."""

    def __init__(self, n_cells: int, eps: float, n_v: int, n_patches: int, buffer: int, samples: int, stream=None,
                 g: float = 0.0):
        h = C.c_void_p()
        N.check(N.load().msp_kinetic_build_hg(n_cells, eps, float(g), n_v, n_patches, buffer, samples,
                                              _stream_ptr(stream), C.byref(h)))
        self._h = h
        self.n_cells, self.eps, self.n_v, self.n_patches, self.buffer, self.samples = (
            n_cells, eps, n_v, n_patches, buffer, samples)
        self.g = float(g)
        self.n_k = (n_cells // n_patches + 1) * n_v

    def set_solver(self, solver: str):
        """"source_iteration" (isotropic only) or "direct" (msp_kinetic_set_solver)."""
        N.check(N.load().msp_kinetic_set_solver(self._h, KINETIC_SOLVERS[solver]))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            N.load().msp_kinetic_destroy(h)
            self._h = None

    def velocities(self):
        v = np.zeros(self.n_v); w = np.zeros(self.n_v)
        N.check(N.load().msp_kinetic_velocities(self._h, _f64p(v), _f64p(w)))
        return v, w

    def sample(self, seed: int, tol: float = 1e-12, max_iter: int = 100000, stream=None, stats: bool = True,
               precision="fp64"):
        st = N.SolveStats()
        N.check(N.load().msp_kinetic_sample(self._h, C.c_uint64(seed), precision_code(precision), tol, max_iter,
                                            _stream_ptr(stream), C.byref(st) if stats else None))
        return st if stats else None

    def snapshots(self, m: int, stream=None) -> torch.Tensor:
        t = torch.empty((self.samples, self.n_k), dtype=torch.float64, device="cuda")
        N.check(N.load().msp_kinetic_get_snapshots(self._h, m, _dptr(t), _stream_ptr(stream)))
        return t.T

    def extract(self, tau: float = 1e-6, stream=None) -> "KineticBasis":
        h = C.c_void_p()
        N.check(N.load().msp_kinetic_extract(self._h, tau, _stream_ptr(stream), C.byref(h)))
        return KineticBasis(h, self)


class KineticBasis:
    def __init__(self, handle, medium: KineticMedium):
        self._h = handle
        self.n_cells, self.n_v, self.n_patches, self.samples = medium.n_cells, medium.n_v, medium.n_patches, medium.samples

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            N.load().msp_kinetic_basis_destroy(h)
            self._h = None

    def k(self, m: int) -> int:
        k = C.c_int()
        N.check(N.load().msp_kinetic_basis_info(self._h, m, C.byref(k), None))
        return k.value

    def sigma(self, m: int) -> np.ndarray:
        out = np.zeros(self.samples)
        k = C.c_int()
        N.check(N.load().msp_kinetic_basis_info(self._h, m, C.byref(k), _f64p(out)))
        return out

    def solve(self, inflow: torch.Tensor, stream=None) -> torch.Tensor:
        """inflow: (B, 2, n_v) or (2, n_v) -- values at x = 0 then at x = 1."""
        squeeze = inflow.dim() == 2
        inflow = inflow.reshape(-1, 2, self.n_v).to(dtype=torch.float64, device="cuda").contiguous()
        B = inflow.shape[0]
        f = torch.empty((B, self.n_cells + 1, self.n_v), dtype=torch.float64, device="cuda")
        N.check(N.load().msp_kinetic_online_solve(self._h, _dptr(inflow), B, _dptr(f), None, _stream_ptr(stream)))
        return f[0] if squeeze else f

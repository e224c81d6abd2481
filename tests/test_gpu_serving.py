"""GPU tests of the serving form: the boundary-to-coefficient map against the
iterative online solve and the CPU oracle, and the request loop (continuous
batching under slot and memory limits; each result the same alone and inside
a mix of requests).

Tolerances: the map is stored and applied in FP32, so its results are held to
the mixed-path bound, relative L2 <= 1e-6 against FP64 references; a request's
result inside a batch equals its result alone to the last bit (every data set
of a batch is computed independently, in a fixed order).
"""
import time

import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu

msp = pytest.importorskip("paper_1807_08848_gb300")

MIXED_TOL = 1e-6


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def wait_done(server, rid, timeout_s=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout_s:
        d, lat = server.poll(rid)
        if d != 0:
            return d, lat
        time.sleep(0.0005)
    raise TimeoutError(f"request {rid} not done after {timeout_s} s")


@pytest.fixture(scope="module")
def media():
    """Two small media of different grid sizes with their maps: the 129^2
    periodic workload (4 x 4 patches) and a 65^2 log-normal one (2 x 2)."""
    out = []
    w = synth.workload_small()
    m1 = msp.Medium(w["medium"], w["patches"])
    m1.sample(w["seed"], "fp64", tol=1e-13, max_iter=20000)
    b1 = m1.extract(w["tau"], "fp64")
    b1.build_map(tol=1e-12, max_iter=5000)
    out.append((w, m1, b1))
    ms = synth.lognormal(64, 1 / 8, 16, 5)
    ps = synth.uniform_patches(64, 2, 2, 8, 48)
    w2 = dict(medium=ms, patches=ps, seed=5, tau=1e-6, phi=synth.phi_sin_cos(64))
    m2 = msp.Medium(ms, ps)
    m2.sample(5, "fp64", tol=1e-13, max_iter=20000)
    b2 = m2.extract(1e-6, "fp64")
    b2.build_map(tol=1e-12, max_iter=5000)
    out.append((w2, m2, b2))
    return out


def test_map_matches_the_iterative_solve(media):
    for w, _, b in media:
        N = b.n_cells
        phis = torch.tensor(synth.phi_fourier(N, 16, 7, batch=6), device="cuda")
        u_map = b.solve_map(phis).cpu().numpy()
        b.set_preconditioner("block_rows_fp64")
        u_it, _ = b.solve(phis, tol=1e-13, max_iter=5000)
        b.set_preconditioner("block_rows")
        u_it = u_it.cpu().numpy()
        for k in range(phis.shape[0]):
            assert rel(u_map[k], u_it[k]) <= MIXED_TOL, k


def test_tensor_core_and_cuda_core_map_engines_agree(media):
    """The tcgen05 split-TF32 GEMM and the FP32 FMA GEMM give the same map solve
    to FP32 level, and both meet the mixed-path bound against the FP64 solve."""
    for w, _, b in media:
        N = b.n_cells
        phis = torch.tensor(synth.phi_fourier(N, 16, 13, batch=37), device="cuda")   # two N tiles, ragged
        b.set_map_engine("cuda_cores")
        u_cc = b.solve_map(phis).cpu().numpy()
        b.set_map_engine("tensor_cores")
        u_tc = b.solve_map(phis).cpu().numpy()
        b.set_preconditioner("block_rows_fp64")
        u_it, _ = b.solve(phis, tol=1e-13, max_iter=5000)
        b.set_preconditioner("block_rows")
        u_it = u_it.cpu().numpy()
        for k in (0, 17, 31, 32, 36):
            assert rel(u_tc[k], u_cc[k]) <= 1e-6, k
            assert rel(u_tc[k], u_it[k]) <= MIXED_TOL, k


def test_map_matches_the_oracle(media):
    w, _, b = media[0]
    off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
    u_ref, _, _, _ = E.online(off, w["patches"], 128, w["phi"])
    u = b.solve_map(torch.tensor(w["phi"], device="cuda")).cpu().numpy()
    assert rel(u, u_ref) <= MIXED_TOL


def test_map_result_does_not_depend_on_the_batch(media):
    _, _, b = media[1]
    phis = torch.tensor(synth.phi_fourier(64, 16, 9, batch=9), device="cuda")
    ub = b.solve_map(phis)
    for k in (0, 4, 8):
        assert torch.equal(b.solve_map(phis[k]), ub[k])


def test_server_alone_and_in_a_mix(media):
    bases = [m[2] for m in media]
    srv = msp.Server(bases, mem_budget_bytes=2 << 30, max_slots=64, max_batch=8, n_workers=2)
    try:
        probe = [synth.phi_fourier(b.n_cells, 16, 100 + i, batch=1)[0] for i, b in enumerate(bases)]
        alone = []
        for i in range(len(bases)):
            rid = srv.submit(i, probe[i])
            d, lat = wait_done(srv, rid)
            assert d == 1 and lat >= 0
            alone.append(srv.fetch(rid, i))
        # a mix: random requests on both media around the probes, submitted back to back
        rng = np.random.default_rng(11)
        plan = []
        for j in range(40):
            i = int(rng.integers(0, len(bases)))
            plan.append((i, synth.phi_fourier(bases[i].n_cells, 16, 1000 + j, batch=1)[0]))
            if j in (5, 17, 30):
                for i2 in range(len(bases)):
                    plan.append((i2, probe[i2]))
        ids = [(srv.submit(i, phi), i, phi) for i, phi in plan]
        results = []
        for rid, i, phi in ids:
            d, _ = wait_done(srv, rid)
            assert d == 1
            results.append((i, phi, srv.fetch(rid, i)))
        st = srv.stats()
        assert st["completed"] == st["submitted"] == len(ids) + len(bases)
        assert st["held"] == 0 and st["mem_in_use"] == 0
        for i, phi, u in results:
            if phi is probe[i]:
                assert np.array_equal(u, alone[i])
        # every mixed result equals the direct map solve of its own data
        for i, phi, u in results[::7]:
            ref = bases[i].solve_map(torch.tensor(phi, device="cuda")).cpu().numpy()
            assert np.array_equal(u, ref)
    finally:
        srv.close()


def test_server_admits_by_memory(media):
    w, _, b = media[0]
    per = 8 * ((b.n_cells + 1) ** 2 + 4 * b.n_cells)
    srv = msp.Server([b], mem_budget_bytes=3 * per, max_slots=100, max_batch=8, n_workers=1)
    try:
        phis = synth.phi_fourier(b.n_cells, 16, 21, batch=7)
        ids = [srv.submit(0, p) for p in phis]
        wait_done(srv, ids[0])
        time.sleep(0.2)
        st = srv.stats()
        assert st["completed"] == 3 and st["held"] == 3 and st["queued"] == 4
        assert st["mem_peak"] <= 3 * per
        srv.release(ids[0])
        wait_done(srv, ids[3])
        time.sleep(0.1)
        assert srv.stats()["completed"] == 4
        for rid in ids[1:]:
            wait_done(srv, rid)
            srv.release(rid)
        st = srv.stats()
        assert st["completed"] == 7 and st["mem_in_use"] == 0 and st["held"] == 0
    finally:
        srv.close()


def test_server_manual_steps(media):
    _, _, b = media[1]
    srv = msp.Server([b], mem_budget_bytes=1 << 30, max_slots=16, max_batch=4, n_workers=0)
    try:
        phis = synth.phi_fourier(64, 16, 31, batch=6)
        ids = [srv.submit(0, p) for p in phis]
        done = 0
        for _ in range(10):
            done += srv.step()
            if done == 6:
                break
        assert done == 6
        st = srv.stats()
        assert st["batches"] == 2 and st["max_batch_seen"] == 4   # queued requests go out in batches
        torch.cuda.synchronize()
        for rid, p in zip(ids, phis):
            u = srv.fetch(rid, 0)
            ref = b.solve_map(torch.tensor(p, device="cuda")).cpu().numpy()
            assert np.array_equal(u, ref)
    finally:
        srv.close()


def test_server_iterative_fp64_engine(media):
    """The plain FP64 engine of the request loop: every batch is the FP64 CGLS
    iteration of msp_online_solve (factor applied in FP64), so each result
    matches the direct FP64 online solve of its own data to the iteration's
    tolerance and the oracle's least-squares solution to the FP64 bound; the map
    engine gives the same fields within the mixed bound.  Switching to the map
    engine needs every medium's map."""
    w, _, b = media[0]
    srv = msp.Server([b], mem_budget_bytes=1 << 30, max_slots=16, max_batch=4, n_workers=0)
    try:
        srv.set_engine("iterative_fp64", tol=1e-12, max_iter=2000)
        phis = synth.phi_fourier(b.n_cells, 16, 41, batch=6)
        ids = [srv.submit(0, p) for p in phis]
        done = 0
        for _ in range(10):
            done += srv.step()
            if done == 6:
                break
        assert done == 6
        off = E.offline(w["medium"], w["patches"], w["seed"], w["tau"])
        b.set_preconditioner("block_rows_fp64")
        try:
            for rid, p in zip(ids, phis):
                u = srv.fetch(rid, 0)
                ref, _ = b.solve(torch.tensor(p, device="cuda"), tol=1e-12, max_iter=2000)
                assert rel(u, ref.cpu().numpy()) <= 1e-10
                u_or, *_ = E.online(off, w["patches"], b.n_cells, p)
                assert rel(u, u_or) <= 1e-8
                assert rel(b.solve_map(torch.tensor(p, device="cuda")).cpu().numpy(), u) <= MIXED_TOL
        finally:
            b.set_preconditioner("block_rows")
        srv.set_engine("map")
    finally:
        srv.close()
    ms = synth.periodic_sin(32, 1 / 4)
    med = msp.Medium(ms, synth.uniform_patches(32, 2, 2, 4, 12))
    med.sample(3, "fp64", tol=1e-12, max_iter=5000)
    nomap = med.extract(1e-8, "fp64")
    srv = msp.Server([nomap], mem_budget_bytes=1 << 30, max_slots=8, max_batch=4, n_workers=0)
    try:
        with pytest.raises(msp.MspError):
            srv.set_engine("map")
        srv.set_engine("iterative_fp64", tol=1e-10, max_iter=500)
        rid = srv.submit(0, synth.phi_sin_cos(32))
        assert srv.step() == 1
        assert np.all(np.isfinite(srv.fetch(rid, 0)))
    finally:
        srv.close()


def test_server_iterative_fp64_engine_several_workers(media):
    """Three workers, each with its own stream, serve batches of the same medium
    with the FP64 engine: the batches share the basis's buffers and run one after
    another; every result still equals the direct FP64 solve of its own data."""
    _, _, b = media[1]
    srv = msp.Server([b], mem_budget_bytes=1 << 30, max_slots=64, max_batch=2, n_workers=3)
    try:
        srv.set_engine("iterative_fp64", tol=1e-12, max_iter=2000)
        phis = synth.phi_fourier(64, 16, 51, batch=9)
        ids = [srv.submit(0, p) for p in phis]
        got = []
        for rid in ids:
            wait_done(srv, rid)
            got.append(srv.fetch(rid, 0))
        assert srv.stats()["batches"] >= 5
    finally:
        srv.close()
    b.set_preconditioner("block_rows_fp64")
    try:
        for u, p in zip(got, phis):
            ref, _ = b.solve(torch.tensor(p, device="cuda"), tol=1e-12, max_iter=2000)
            assert rel(u, ref.cpu().numpy()) <= 1e-10
    finally:
        b.set_preconditioner("block_rows")

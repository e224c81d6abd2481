"""GPU tests of the launch forms of the local solves on an uneven partition where
some buffered patches exceed the on-chip tile limit: one fused persistent launch,
the split launch, CUDA-graph replay and the autotuned choice.  Columns of patches
that fit on chip run the same code with the same block size in every form and are
bit-identical; columns of the patches beyond the on-chip limit run the global-scratch
code with 768 threads inside the fused launch and 512 in the split one, so their dot products
are summed in another order and they agree to the solver tolerance; the large
tiles solved inside the fused launch match the oracle.

Tolerances: relative L2 <= 1e-8 (plain FP64 path) and <= 1e-6 (mixed path)
against the oracle's sparse direct solves."""
import numpy as np
import pytest
import torch

import synth
from oracle import elliptic as E

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")

N = 256
TOL = {"fp64": 1e-8, "mixed": 1e-6}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def spec():
    return synth.channels(N, 1 / 16, 4, 2), synth.uneven_patches(N, 2)


def snapshots(med):
    return [med.snapshots(m).cpu().numpy() for m in range(med.n_patches)]


def assert_same(a, b, ps, close):
    """Every patch within `close` (relative L2); the patches that fit on chip (most of
    them here) bit-identical, so at least one patch must be."""
    identical = 0
    for m, (x, y) in enumerate(zip(snapshots(a), snapshots(b))):
        assert rel(y, x) <= close, m
        identical += int(np.array_equal(x, y))
    assert identical > 0


def big_patches(ps):
    """Patches whose buffered box is wider or taller than the on-chip tile limit (98 nodes)."""
    out = []
    for m, P in enumerate(E.patch_boxes(N, ps)):
        if P.X1 - P.X0 - 1 > 96 or P.Y1 - P.Y0 - 1 > 96:
            out.append(m)
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fused_launch_equals_split_launch(precision):
    ms, ps = spec()
    assert big_patches(ps), "the partition must have tiles beyond the on-chip limit"
    tol = 1e-13 if precision == "fp64" else 1e-11
    a = msp.Medium(ms, ps)
    a.sample(2, precision, tol=tol, max_iter=40000)
    b = msp.Medium(ms, ps)
    b.set_launch(precision, "fused")
    st = b.sample(2, precision, tol=tol, max_iter=40000)
    assert st.n_not_converged == 0
    assert_same(a, b, ps, 1e-10 if precision == "fp64" else 1e-8)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_large_tiles_in_the_fused_launch_match_the_oracle(precision):
    ms, ps = spec()
    med = msp.Medium(ms, ps)
    med.set_launch(precision, "fused")
    med.sample(2, precision, tol=1e-13 if precision == "fp64" else 1e-11, max_iter=40000)
    aE, aN = E.face_coefficients(ms)
    patches = E.patch_boxes(N, ps)
    big = big_patches(ps)
    for m in big[:2] + [0 if 0 not in big else len(patches) - 1]:
        R = E.snapshots(aE, aN, patches[m], 2, N)
        assert rel(med.snapshots(m).cpu().numpy(), R) <= TOL[precision], m


def test_graph_replay_equals_direct_launch():
    ms, ps = spec()
    ref = msp.Medium(ms, ps)
    ref.sample(3, "mixed", tol=1e-10, max_iter=40000)
    g = msp.Medium(ms, ps)
    g.set_graph(True)
    for rep in range(3):   # direct + capture, then two replays
        st = g.sample(3, "mixed", tol=1e-10, max_iter=40000)
        assert st.n_not_converged == 0
        for m, (x, y) in enumerate(zip(snapshots(ref), snapshots(g))):
            assert np.array_equal(x, y), (rep, m)
    # a new configuration is captured again, and its replay equals its direct run
    f = msp.Medium(ms, ps)
    f.set_launch("mixed", "fused")
    f.sample(3, "mixed", tol=1e-10, max_iter=40000)
    g.set_launch("mixed", "fused")
    g.sample(3, "mixed", tol=1e-10, max_iter=40000)
    g.sample(3, "mixed", tol=1e-10, max_iter=40000)
    for m, (x, y) in enumerate(zip(snapshots(f), snapshots(g))):
        assert np.array_equal(x, y), m


def test_autotune_reports_and_keeps_the_fastest():
    """Every launch form is timed (the CG forms on the probe, the direct solver on
    the whole medium), the fastest is kept, and a later sample gives what that form
    gives when set by hand (bitwise on the patches that fit on chip) and agrees with
    the CG split launch to the solver tolerance."""
    ms, ps = spec()
    med = msp.Medium(ms, ps)
    rep = med.autotune(4, "mixed", tol=1e-10, max_iter=40000, max_probe_items=400)
    ran = [c for c in rep["candidates"] if c["ms"] > 0]
    assert {c["mode"] for c in ran} == {"split", "fused", "direct"}
    assert rep["best_ms"] == min(c["ms"] for c in ran)
    assert 0 < rep["probe_items"] <= 400
    ref = msp.Medium(ms, ps)
    ref.set_launch("mixed", rep["best_mode"], rep["best_rows"])
    ref.sample(4, "mixed", tol=1e-10, max_iter=40000)
    med.sample(4, "mixed", tol=1e-10, max_iter=40000)
    assert_same(ref, med, ps, 1e-7)
    split = msp.Medium(ms, ps)
    split.sample(4, "mixed", tol=1e-10, max_iter=40000)
    for m, (x, y) in enumerate(zip(snapshots(split), snapshots(med))):
        assert rel(y, x) <= TOL["mixed"], m

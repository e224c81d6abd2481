"""The device half of the offline stage split by patches, on one GPU: the local
solves of a list of patches (msp_sample_patch_list) and the upload of snapshot
blocks computed elsewhere (msp_set_snapshots).  Two media each solve one share
of the patches of the same workload, one takes the other's blocks, and the
result must equal the whole-medium run bit for bit (every column's arithmetic
is independent of the other columns in its launch), and so must the bases."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
msp = pytest.importorskip("paper_1807_08848_gb300")
from paper_1807_08848_gb300 import sharding  # noqa: E402


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_patch_shares_and_block_exchange_equal_the_whole_run(precision):
    w = synth.workload_small()
    ref = msp.Medium(w["medium"], w["patches"])
    ref.sample(w["seed"], precision, tol=1e-11, max_iter=20000)
    costs = sharding.patch_costs([ref.patch(m) for m in range(ref.n_patches)])
    parts = sharding.lpt_partition(costs, 2)
    a = msp.Medium(w["medium"], w["patches"])
    b = msp.Medium(w["medium"], w["patches"])
    sa = a.sample_patches(parts[0], w["seed"], precision, tol=1e-11, max_iter=20000)
    b.sample_patches(parts[1], w["seed"], precision, tol=1e-11, max_iter=20000)
    assert sa.n_solves == sum(ref.patch(m).cols for m in parts[0]) and sa.n_not_converged == 0
    for m in parts[1]:
        a.set_snapshots(m, b.snapshots(m))
    for m in range(ref.n_patches):
        assert np.array_equal(a.snapshots(m).cpu().numpy(), ref.snapshots(m).cpu().numpy()), m
    ba, br = a.extract(w["tau"], precision), ref.extract(w["tau"], precision)
    for m in range(ref.n_patches):
        assert np.array_equal(ba.sigma(m), br.sigma(m)), m
    phi = torch.tensor(w["phi"], device="cuda")
    ua, _ = ba.solve(phi, tol=1e-12, max_iter=5000)
    ur, _ = br.solve(phi, tol=1e-12, max_iter=5000)
    assert torch.equal(ua, ur)


def test_patch_list_arguments():
    w = synth.workload_small()
    med = msp.Medium(w["medium"], w["patches"])
    with pytest.raises(msp.MspError):
        med.sample_patches([0, 16], w["seed"], "fp64")
    st = med.sample_patches([], w["seed"], "fp64")
    assert st.n_solves == 0

"""Pins of the oracle's random-number stage (Philox4x32-10 + Box-Muller)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(t, 16) for t in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat())
def test_known_answer_vectors(row):
    c0, c1, c2, c3, k0, k1, *want = row
    got = philox.philox4x32_10(c0, c1, c2, c3, k0, k1)
    assert [int(g) for g in got] == want


def test_uniform_ranges_and_counter_independence():
    q = np.arange(4096, dtype=np.uint64)
    u1, u2 = philox.uniforms(12345, q, 0, 7, philox.TAG_ELLIPTIC)
    assert np.all(u1 > 0) and np.all(u1 <= 1) and np.all(u2 >= 0) and np.all(u2 < 1)
    v1, _ = philox.uniforms(12345, q, 1, 7, philox.TAG_ELLIPTIC)
    assert not np.any(u1 == v1)                 # another sample -> another stream
    w1, _ = philox.uniforms(12346, q, 0, 7, philox.TAG_ELLIPTIC)
    assert not np.any(u1 == w1)                 # another seed -> another stream


def test_normals_are_standard_gaussian():
    z = philox.normals(3, 5, 2000, 500)        # 1e6 draws
    assert z.shape == (2000, 500)
    assert abs(z.mean()) < 5e-3
    assert abs(z.var() - 1.0) < 5e-3
    assert stats.kstest(z.ravel()[:200000], "norm").pvalue > 1e-3
    # odd node count: the last pair is cut, the rest is unchanged
    z_odd = philox.normals(3, 5, 1999, 500)
    np.testing.assert_array_equal(z_odd, z[:1999])


def test_box_muller_pairs():
    """Nodes 2q and 2q+1 share u1: z0^2 + z1^2 = -2 ln u1."""
    z = philox.normals(9, 0, 64, 8)
    q = np.arange(32, dtype=np.uint64)[:, None]
    s = np.arange(8, dtype=np.uint64)[None, :]
    u1, _ = philox.uniforms(9, q, s, 0, philox.TAG_ELLIPTIC)
    np.testing.assert_allclose(z[0::2] ** 2 + z[1::2] ** 2, -2 * np.log(u1), rtol=1e-13)

"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle side).

The paper draws the boundary data of every local solve i.i.d. from N(0,1)
(Sec. 3.3; Eq. rte_random for transport, Eq. elliptic_random for the
elliptic problem).  So that
the CPU oracle and the GPU path draw the *same* numbers without sharing code,
both implement Philox4x32-10 from its published definition (Salmon, Moraes,
Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the
Box-Muller transform.

Stream layout (the reading used for parity): key = (seed mod 2^32,
seed div 2^32); counter = (pair index q, sample s, patch m, tag).  One
generator call gives two uniforms and hence two normals, for boundary nodes
2q and 2q+1 of the patch's ring.

    u1 = (bits53(x1:x0) + 1) * 2^-53  in (0, 1]
    u2 =  bits53(x3:x2)      * 2^-53  in [0, 1)
    z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2)

where bits53(hi:lo) keeps the top 53 bits of the 64-bit word hi*2^32 + lo.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

TAG_ELLIPTIC = 0x4D535045   # stream tag of the elliptic boundary samples
TAG_KINETIC = 0x4D53504B    # stream tag of the kinetic inflow samples


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on uint32 counters (numpy arrays, broadcast together).

    One round: multiply c0 and c2 by the two round constants into 64-bit
    products, swap and xor the high halves with c1, c3 and the key; the key
    is advanced by the Weyl constants between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def uniforms(seed: int, c0, c1, c2, c3):
    """The two uniforms (u1 in (0,1], u2 in [0,1)) of each generator call."""
    x0, x1, x2, x3 = philox4x32_10(c0, c1, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    a = ((x1 << np.uint64(32)) | x0) >> np.uint64(11)
    b = ((x3 << np.uint64(32)) | x2) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    return u1, u2


def normals(seed: int, patch: int, n_nodes: int, n_samples: int, tag: int = TAG_ELLIPTIC) -> np.ndarray:
    """Boundary-sample matrix Omega_m of shape (n_nodes, n_samples): entry
    (t, s) is the N(0,1) value at ring node t of sample s of this patch."""
    q = np.arange((n_nodes + 1) // 2, dtype=np.uint64)[:, None]
    s = np.arange(n_samples, dtype=np.uint64)[None, :]
    u1, u2 = uniforms(seed, q, s, np.uint64(patch), np.uint64(tag))
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((2 * q.shape[0], n_samples))
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:n_nodes]

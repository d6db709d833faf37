"""Philox4x64-10 and the Rademacher probe rule (oracle side; test infrastructure).

Philox4x64-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
    (hi0, lo0) = M0 * c0      (full 128-bit product)
    (hi1, lo1) = M1 * c2
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
with the key bumped by the Weyl constants (W0, W1) between rounds.

Probe rule (the paper draws p_1..p_K Rademacher and fresh at every EM
iteration, Alg. 1 "Draw p_1 ... p_K"; the generator is not specified, so this is
this project's reading): for EM iteration t (1-based), probe k (1-based) and
coordinate j (0-based), take the 256-bit Philox4x64-10 output at
    key = (seed, 0),  counter = (j >> 8, k, t, 0)
and its bit b = j & 255 (word b >> 6, bit b & 63).  p_{t,k,j} = +1 if that bit
is 0 and -1 if it is 1.  With L tasks (multi-task CoFEM) task l draws its own
probes from counter (j >> 8, k, t, l); task 0 is the single-task rule.

Pinned against numpy's own Philox bit generator (a library implementation of
the same published algorithm) in tests/test_oracle_philox.py.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
MASK64 = (1 << 64) - 1
_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: int, b: np.ndarray):
    """(hi, lo) of the 128-bit product a*b, for a Python int constant a and a
    uint64 array b, by 32-bit limbs."""
    a_lo = np.uint64(a & 0xFFFFFFFF)
    a_hi = np.uint64(a >> 32)
    b_lo = b & _M32
    b_hi = b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _M32) + (hl & _M32)
    lo = (ll & _M32) | ((mid & _M32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(ctr, key):
    """Philox4x64-10 block function.

    ctr: array-like (..., 4) of uint64 counters; key: (k0, k1) Python ints.
    Returns a (..., 4) uint64 array.
    """
    c = np.array(ctr, dtype=np.uint64)
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = int(key[0]) & MASK64, int(key[1]) & MASK64
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = (k0 + W0) & MASK64
                k1 = (k1 + W1) & MASK64
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                              hi0 ^ c3 ^ np.uint64(k1), lo0)
    return np.stack([c0, c1, c2, c3], axis=-1)


def probe_bits(seed: int, t: int, k: int, D: int, task: int = 0) -> np.ndarray:
    """The D bits behind probe k at EM iteration t (uint8 array of 0/1)."""
    nblk = (D + 255) // 256
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
    ctr[:, 1] = np.uint64(k)
    ctr[:, 2] = np.uint64(t)
    ctr[:, 3] = np.uint64(task)
    words = philox4x64_10(ctr, (seed, 0))            # (nblk, 4) uint64
    j = np.arange(D)
    b = j & 255
    w = words[j >> 8, b >> 6]
    return ((w >> (b & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)


def rademacher_probes(seed: int, t: int, K: int, D: int, task: int = 0) -> np.ndarray:
    """Probe block for EM iteration t: a (K, D) float64 array of +-1 whose row
    k-1 is p_k (Alg. 1, fresh probes each EM iteration)."""
    out = np.empty((K, D), dtype=np.float64)
    for k in range(1, K + 1):
        out[k - 1] = 1.0 - 2.0 * probe_bits(seed, t, k, D, task).astype(np.float64)
    return out

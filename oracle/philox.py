"""Philox4x32-10 counter-based generator and the Gaussian test matrix Omega (oracle side).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package; only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter, a 2 x 32-bit key, ten rounds of
two 32x32->64 multiplications with multipliers 0xD2511F53 and 0xCD9E8D57, the key bumped
between rounds by the Weyl constants 0x9E3779B9 and 0xBB67AE85.

The paper draws Omega = randn(n, b) (Alg. 2) and randn(n, l~) (Alg. 4) with Matlab/MKL.  Our
reading makes Omega a pure function of (seed, row j, global column c):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (j, c div 2, 0, 0)
  words   = (w0, w1, w2, w3) = Philox4x32-10(counter, key)
  u1 = (((w0 * 2^32 + w1) >> 11) + 1/2) 2^-53,  u2 = (((w2 * 2^32 + w3) >> 11) + 1/2) 2^-53
  Box-Muller: rho = sqrt(-2 ln u1), theta = 2 pi u2;  Omega(j, c) = rho cos theta (c even),
                                                                    rho sin theta (c odd).
Block i of randQB_EI takes global columns [(i-1) b, i b); batch q of randQB_FP takes
[q l~, (q+1) l~), so EI and FP draw the same Omega.

The reduced-precision generator used by the mixed-precision path takes 24-bit uniforms
u1 = ((w0 >> 8) + 1/2) 2^-24, u2 = ((w2 >> 8) + 1/2) 2^-24 and evaluates Box-Muller in float32.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on (broadcastable) uint32 arrays; returns four uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64)
    c1 = np.asarray(c1, dtype=np.uint64)
    c2 = np.asarray(c2, dtype=np.uint64)
    c3 = np.asarray(c3, dtype=np.uint64)
    k0 = np.uint64(int(k0) & MASK32)
    k1 = np.uint64(int(k1) & MASK32)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    mask = np.uint64(MASK32)
    s32 = np.uint64(32)
    for rnd in range(10):
        if rnd > 0:  # key schedule: bump before every round but the first
            k0 = np.uint64((int(k0) + W0) & MASK32)
            k1 = np.uint64((int(k1) + W1) & MASK32)
        p0 = m0 * c0  # exact: both factors < 2^32
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def _words(n: int, col0: int, w: int, seed: int):
    j = np.arange(n, dtype=np.uint64)[:, None]
    c = (np.uint64(col0) + np.arange(w, dtype=np.uint64))[None, :]
    zero = np.zeros((1, 1), dtype=np.uint64)
    k0 = int(seed) & MASK32
    k1 = (int(seed) >> 32) & MASK32
    w0, w1, w2, w3 = philox4x32_10(j + zero * c, (c >> np.uint64(1)) + zero * j, zero, zero, k0, k1)
    return c, w0, w1, w2, w3


def omega(n: int, col0: int, w: int, seed: int) -> np.ndarray:
    """float64 Omega rows 0..n-1, global columns col0..col0+w-1 (an n x w array)."""
    if n == 0 or w == 0:
        return np.zeros((n, w))
    c, w0, w1, w2, w3 = _words(n, col0, w, seed)
    s32 = np.uint64(32)
    s11 = np.uint64(11)
    k1 = ((w0.astype(np.uint64) << s32) | w1.astype(np.uint64)) >> s11
    k2 = ((w2.astype(np.uint64) << s32) | w3.astype(np.uint64)) >> s11
    u1 = (k1.astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = (k2.astype(np.float64) + 0.5) * 2.0 ** -53
    rho = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    even = (c & np.uint64(1)) == 0
    return np.where(even, rho * np.cos(theta), rho * np.sin(theta))


def omega_f32(n: int, col0: int, w: int, seed: int) -> np.ndarray:
    """float32 variant (24-bit uniforms, float32 Box-Muller) used by the mixed-precision path."""
    if n == 0 or w == 0:
        return np.zeros((n, w), dtype=np.float32)
    c, w0, w1, w2, w3 = _words(n, col0, w, seed)
    s8 = np.uint32(8)
    u1 = ((w0 >> s8).astype(np.float32) + np.float32(0.5)) * np.float32(2.0 ** -24)
    u2 = ((w2 >> s8).astype(np.float32) + np.float32(0.5)) * np.float32(2.0 ** -24)
    rho = np.sqrt(np.float32(-2.0) * np.log(u1))
    theta = np.float32(2.0 * np.pi) * u2
    even = (c & np.uint64(1)) == 0
    return np.where(even, rho * np.cos(theta), rho * np.sin(theta)).astype(np.float32)

"""Philox counter-based generator for the oracle -- TEST INFRASTRUCTURE ONLY.

Written from the definition in J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.3: the Philox-4xW-R bijection
applies R rounds of

    (x0, x1, x2, x3) <- (hi(M1*x2) ^ x1 ^ k0,  lo(M1*x2),  hi(M0*x0) ^ x3 ^ k1,  lo(M0*x0))

with the key bumped by the Weyl constants (W0, W1) after every round.

``philox4_reference`` is the plain big-integer form for any word width; with the 64-bit
constants it is checked against numpy's own Philox4x64-10 bit generator, which pins the round
structure, and the 32-bit form used for the quantisation noise runs through the same code.
``philox4x32_10`` is the vectorised 32-bit form the oracle draws its noise with.

Quantisation noise (the reading the paper leaves open, Sec. II "Encoding"): the uniform
noise u of latent i of level l at iteration t is word (i mod 4) of
Philox4x32-10(counter = (i div 4, l, t, 0), key = (seed mod 2^32, seed div 2^32)), mapped to
u = (word >> 8) * 2^-24 - 1/2, so u lies on a 2^-24 grid in [-1/2, 1/2).
"""
from __future__ import annotations

import numpy as np

# Multipliers and Weyl constants of Salmon et al., Table 2 / Sec. 3.3.
PHILOX_CONSTANTS = {
    32: dict(M0=0xD2511F53, M1=0xCD9E8D57, W0=0x9E3779B9, W1=0xBB67AE85),
    64: dict(M0=0xD2E7470EE14C6C93, M1=0xCA5A826395121157,
             W0=0x9E3779B97F4A7C15, W1=0xBB67AE8584CAA73B),
}


def philox4_reference(ctr, key, width=32, rounds=10):
    """Philox-4xW-R on Python integers: ctr is 4 words, key is 2 words."""
    c = PHILOX_CONSTANTS[width]
    mask = (1 << width) - 1
    x0, x1, x2, x3 = (int(v) & mask for v in ctr)
    k0, k1 = (int(v) & mask for v in key)
    for _ in range(rounds):
        p0 = c["M0"] * x0
        p1 = c["M1"] * x2
        x0, x1, x2, x3 = ((p1 >> width) ^ x1 ^ k0, p1 & mask,
                          (p0 >> width) ^ x3 ^ k1, p0 & mask)
        k0 = (k0 + c["W0"]) & mask
        k1 = (k1 + c["W1"]) & mask
    return [x0, x1, x2, x3]


def philox4x32_10(ctr: np.ndarray, key) -> np.ndarray:
    """Vectorised Philox4x32-10.  ctr: (..., 4) integer array; returns (..., 4) uint32."""
    c = PHILOX_CONSTANTS[32]
    ctr = np.asarray(ctr, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    x0, x1, x2, x3 = (ctr[..., i].copy() for i in range(4))
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    m0, m1 = np.uint64(c["M0"]), np.uint64(c["M1"])
    lo_mask, s32 = np.uint64(0xFFFFFFFF), np.uint64(32)
    for _ in range(10):
        p0 = m0 * x0  # < 2^64: no overflow in uint64
        p1 = m1 * x2
        x0, x1, x2, x3 = ((p1 >> s32) ^ x1 ^ k0, p1 & lo_mask,
                          (p0 >> s32) ^ x3 ^ k1, p0 & lo_mask)
        k0 = (k0 + np.uint64(c["W0"])) & lo_mask
        k1 = (k1 + np.uint64(c["W1"])) & lo_mask
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def seed_key(seed: int):
    seed = int(seed) & ((1 << 64) - 1)
    return (seed & 0xFFFFFFFF, seed >> 32)


def latent_noise(seed: int, t: int, shapes):
    """Quantisation noise u for every latent of every level at iteration t (float64 arrays)."""
    key = seed_key(seed)
    out = []
    for l, (h, w) in enumerate(shapes):
        n = h * w
        i = np.arange(n, dtype=np.uint64)
        ctr = np.zeros((n, 4), dtype=np.uint64)
        ctr[:, 0] = i >> np.uint64(2)
        ctr[:, 1] = l
        ctr[:, 2] = t
        words = philox4x32_10(ctr, key)
        word = words[np.arange(n), (i & np.uint64(3)).astype(np.int64)]
        u = (word >> np.uint32(8)).astype(np.float64) * 2.0 ** -24 - 0.5
        out.append(u.reshape(h, w))
    return out

"""Oracle: Philox4x32-10 counter-based random numbers (FP64 uniforms).

Test infrastructure only (see ``oracle/__init__.py``).

The paper samples inducing columns at random (Sec. 3, "Column selection
strategies") but names no generator.  Both the oracle and the GPU path draw
from Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel
random numbers: as easy as 1, 2, 3" (SC'11), each side implementing it from
that definition:

  round:  (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
                                hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
  with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by
  (0x9E3779B9, 0xBB67AE85); 10 rounds.

Stream convention (shared by both sides as a stated interface, not code):
counter = (index lo32, index hi32, stream, 0), key = (seed lo32, seed hi32);
uniform u = (((o0 >> 5) << 26) + (o1 >> 6) + 1) * 2^-53, in (0, 1].
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF

STREAM_UNIFORM = 0  # uniform column selection
STREAM_RLS_PILOT = 1  # pilot columns of the leverage-score estimate
STREAM_RLS_SAMPLE = 2  # weighted sampling by leverage score


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10.  ctr: (..., 4) uint32-valued, key: (..., 2)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = np.uint64(M0) * c[0]
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1).astype(np.uint32)


def uniforms(n: int, seed: int, stream: int) -> np.ndarray:
    """u_i in (0, 1] for i = 0..n-1 from counter (i, stream): the random draws of the column
    sampling of Sec. 3, from Philox4x32-10 (Salmon et al., SC'11)."""
    idx = np.arange(n, dtype=np.uint64)
    ctr = np.stack([idx & np.uint64(MASK), idx >> np.uint64(32),
                    np.full(n, stream, dtype=np.uint64), np.zeros(n, dtype=np.uint64)], axis=-1)
    key = np.array([seed & MASK, (seed >> 32) & MASK], dtype=np.uint64)
    out = philox4x32_10(ctr, np.broadcast_to(key, (n, 2))).astype(np.uint64)
    mant = ((out[:, 0] >> np.uint64(5)) << np.uint64(26)) + (out[:, 1] >> np.uint64(6)) + np.uint64(1)
    return mant.astype(np.float64) * 2.0 ** -53

"""Philox4x64-10 counter-based generator, plain numpy, for the FP64 oracle.

TEST INFRASTRUCTURE ONLY.  This module belongs to the CPU oracle.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg may import it; the
CUDA product path never does, and it shares no code with it.

The random choices of the method (the hash h and signs of the sparse embedding
matrix of Sec. 2.2, the random signs D and the column subsample of the SRFT of
Sec. 2.1, drawn in step 1 of Algorithm 1) are fixed by one counter-based
generator that both the oracle and the CUDA path implement independently from
its published definition: Philox4x64 with 10 rounds (Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).

One Philox round maps a 4-word counter (c0, c1, c2, c3) under a 2-word key
(k0, k1) to

    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

with 64x64->128-bit products; between rounds the key is bumped by two Weyl
constants.  Ten rounds make one output block of four 64-bit words.
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def mulhilo64(a, b):
    """Return (hi, lo) of the exact 128-bit product of uint64 arrays a and b.

    Schoolbook multiplication on 32-bit halves; every partial product fits in
    64 bits, and the carries are propagated explicitly.
    """
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _MASK32, a >> _S32
    b_lo, b_hi = b & _MASK32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)  # < 3 * 2^32
    lo = (ll & _MASK32) | ((mid & _MASK32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64_10(counters, key):
    """Philox4x64-10 blocks.

    counters: uint64 array of shape (N, 4); key: two uint64 words.
    Returns a uint64 array of shape (N, 4): the output block of each counter.
    """
    with np.errstate(over="ignore"):
        c = np.array(counters, dtype=np.uint64).reshape(-1, 4).copy()
        k0 = np.uint64(key[0])
        k1 = np.uint64(key[1])
        for r in range(10):
            if r > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = mulhilo64(M0, c[:, 0])
            hi1, lo1 = mulhilo64(M1, c[:, 2])
            c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
    return c


def stream_blocks(key, stream, count):
    """Blocks at counters (i, stream, 0, 0) for i = 0 .. count-1."""
    ctr = np.zeros((count, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(count, dtype=np.uint64)
    ctr[:, 1] = np.uint64(stream)
    return philox4x64_10(ctr, key)

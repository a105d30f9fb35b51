"""Philox-4xW-10 counter-based generator (oracle copy; test infrastructure only).

Written from the generator's published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
    (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
with the key bumped by the Weyl constants between rounds. The 4x64 instance is checked
against numpy's Philox bit generator and the 4x32 instance (the one the chain uses)
against the published known-answer vectors.

The paper does not say how its local proposals draw random numbers; this layout is a
reading chosen so that the CPU chain and the GPU chain consume identical streams:
  * one 4x32 block per (site, sweep) with counter (i*L + l, sweep, chain, 0):
    words (0,1) give the proposal uniform, words (2,3) the Metropolis uniform;
  * one block per (cumulative update) with counter (update, 0, chain, 1):
    word 0 bit 0 is the starting colour, words (2,3) the acceptance uniform;
  * key = (seed & 0xffffffff, seed >> 32).
"""
import numpy as np

M4x32 = (0xD2511F53, 0xCD9E8D57)
W4x32 = (0x9E3779B9, 0xBB67AE85)
M4x64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
W4x64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)


def _mulhilo32(m, c):
    p = np.uint64(m) * c.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def philox4x32_10(ctr, key):
    """ctr: four uint32 arrays (broadcastable), key: two uint32 scalars/arrays.
    Returns four uint32 arrays."""
    c = [np.asarray(v, dtype=np.uint32) for v in ctr]
    c = list(np.broadcast_arrays(*c))
    k0 = np.asarray(key[0], dtype=np.uint32)
    k1 = np.asarray(key[1], dtype=np.uint32)
    for r in range(10):
        if r > 0:
            k0 = ((k0.astype(np.uint64) + np.uint64(W4x32[0])) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            k1 = ((k1.astype(np.uint64) + np.uint64(W4x32[1])) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        hi0, lo0 = _mulhilo32(M4x32[0], c[0])
        hi1, lo1 = _mulhilo32(M4x32[1], c[2])
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def philox4x64_10_scalar(ctr, key):
    """Scalar 4x64 instance in Python integers (used only to pin the round structure
    against numpy's implementation)."""
    mask = (1 << 64) - 1
    c = [int(v) & mask for v in ctr]
    k0, k1 = int(key[0]) & mask, int(key[1]) & mask
    for r in range(10):
        if r > 0:
            k0 = (k0 + W4x64[0]) & mask
            k1 = (k1 + W4x64[1]) & mask
        p0 = M4x64[0] * c[0]
        p1 = M4x64[1] * c[2]
        hi0, lo0 = p0 >> 64, p0 & mask
        hi1, lo1 = p1 >> 64, p1 & mask
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def uniform53(w_hi, w_lo):
    """Double in [0, 1) from two 32-bit words: the top 27 bits of w_hi and the top 26
    bits of w_lo form a 53-bit integer, scaled by 2^-53 (exact in FP64)."""
    a = (np.asarray(w_hi, dtype=np.uint32) >> np.uint32(5)).astype(np.float64)
    b = (np.asarray(w_lo, dtype=np.uint32) >> np.uint32(6)).astype(np.float64)
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0)


def seed_key(seed):
    seed = int(seed) & ((1 << 64) - 1)
    return (seed & 0xFFFFFFFF, seed >> 32)

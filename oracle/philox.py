"""Philox4x32-10, written from its published definition (test infrastructure).

Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
(SC'11), section on the Philox family: a 4-word counter is pushed through ten
rounds of a bijection built from two 32x32->64-bit multiplications; the two
key words are bumped by the Weyl constants between rounds.

Stream layout used by the method (the counter's last word names the stream):
  draws      counter (site // 2, sample_lo, sample_hi, 0); site parity picks
             words (0, 1) or (2, 3) as one 64-bit value  x = lo | hi << 32.
  MH         counter (t_lo, t_hi, chain, 1); words (0, 1) -> u = (x >> 11) 2^-53
  init       counter (site // 128, chain_lo, chain_hi, 2); bit (site % 128).
  sweep      counter (site, chain, sweep, 5); words (0, 1) -> u = (x >> 11) 2^-53
             (single-spin-flip Metropolis sweeps between proposals)
The key is the 64-bit seed, (seed_lo, seed_hi).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

TAG_DRAW = 0
TAG_MH = 1
TAG_INIT = 2
TAG_SWEEP = 5


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on broadcastable uint32-valued arrays.

    Returns four uint64 arrays holding 32-bit words.
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0           # < 2^64: exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def _key(seed):
    s = np.uint64(seed)
    return s & _MASK, s >> _S32


def draw_words(seed, site, sample):
    """64-bit draw for (site, sample); `sample` may be an array (uint64)."""
    k0, k1 = _key(seed)
    sample = np.asarray(sample, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(np.uint64(site // 2), sample & _MASK, sample >> _S32,
                                   np.uint64(TAG_DRAW), k0, k1)
    if site % 2 == 0:
        return w0 | (w1 << _S32)
    return w2 | (w3 << _S32)


def mh_uniform(seed, t, chain):
    """Uniform in [0, 1) with 53 random bits for proposal step t of `chain`."""
    k0, k1 = _key(seed)
    t = np.asarray(t, dtype=np.uint64)
    chain = np.asarray(chain, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(t & _MASK, t >> _S32, chain, np.uint64(TAG_MH), k0, k1)
    x = w0 | (w1 << _S32)
    return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def init_bits(seed, n_sites, chains):
    """Random +-1 start: spin = +1 iff bit (site % 128) of block site // 128 is set."""
    k0, k1 = _key(seed)
    chains = np.asarray(chains, dtype=np.uint64)
    out = np.empty((chains.size, n_sites), dtype=np.int8)
    for blk in range((n_sites + 127) // 128):
        words = philox4x32_10(np.uint64(blk), chains & _MASK, chains >> _S32,
                              np.uint64(TAG_INIT), k0, k1)
        for s in range(blk * 128, min(n_sites, blk * 128 + 128)):
            j = s - blk * 128
            bit = (words[j // 32] >> np.uint64(j % 32)) & np.uint64(1)
            out[:, s] = np.where(bit == 1, 1, -1)
    return out


def sweep_uniform(seed, site, chain, sweep):
    """Uniform in [0, 1) with 53 random bits for the Metropolis update of `site` in
    sweep `sweep` of chain `chain` (each a 32-bit counter word; arrays broadcast)."""
    k0, k1 = _key(seed)
    w0, w1, _, _ = philox4x32_10(np.asarray(site, dtype=np.uint64), np.asarray(chain, dtype=np.uint64),
                                 np.asarray(sweep, dtype=np.uint64), np.uint64(TAG_SWEEP), k0, k1)
    x = w0 | (w1 << _S32)
    return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53

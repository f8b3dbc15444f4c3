"""Philox4x64-10 counter-based generator and the draws HMC takes from it.

Test infrastructure only (see ``oracle/__init__.py``).

Philox4x64 is the counter-based generator of Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4-word counter and a
2-word key, ten rounds of two 64x64->128-bit multiplies with the key bumped by
the Weyl constants between rounds.  Written here from that definition with
plain numpy uint64 arithmetic (the 128-bit product is built from 32-bit
halves).  Pinned against ``numpy.random.Philox``, an independent library
implementation of the same generator.

Stream layout used by the sampler (the paper does not say how momenta or the
accept uniform are drawn; this layout is this project's reading):

* key     = (seed, 0)
* counter = (block, iteration, chain, tag), tag 0 = momentum, 1 = accept.
* momentum coordinate q of chain c at iteration t (q = k*p + j over the
  p x (K-1) free coefficients, class-major): block q // 4, the block's four
  words form two Box-Muller pairs (w0, w1) and (w2, w3); q even takes the
  cosine branch of its pair, q odd the sine branch.
* accept uniform of chain c at iteration t: word 0 of block 0, tag 1.
* 64-bit word -> uniform in (0, 1): ((w >> 11) + 0.5) * 2**-53 (never 0 or 1).
* Box-Muller: r = sqrt(-2 log u1), z0 = r cos(2 pi u2), z1 = r sin(2 pi u2).
"""
import numpy as np

# Multipliers and Weyl key increments of Philox4x64 (Salmon et al. 2011).
_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

TAG_MOMENTUM = 0
TAG_ACCEPT = 1


def _mulhilo(a, b):
    """Full 128-bit product of uint64 arrays: returns (high word, low word)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _LO32, a >> _S32
    b_lo, b_hi = b & _LO32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _LO32) + (hl & _LO32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    lo = a * b
    return hi, lo


def philox4x64_10(counter, key):
    """Ten Philox4x64 rounds.

    counter: sequence of 4 uint64 arrays (broadcastable), key: 2 uint64 values.
    Returns a list of 4 uint64 arrays.
    """
    c = [np.asarray(w, dtype=np.uint64) for w in counter]
    k0 = np.uint64(key[0])
    k1 = np.uint64(key[1])
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = k0 + _W0
                k1 = k1 + _W1
            hi0, lo0 = _mulhilo(_M0, c[0])
            hi1, lo1 = _mulhilo(_M1, c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def word_to_uniform(w):
    """Map a uint64 word to a double in (0, 1): ((w >> 11) + 0.5) / 2**53."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def momentum_normals(seed, iteration, chain, count):
    """The `count` standard normals of the momentum draw of one chain/iteration."""
    if count == 0:
        return np.zeros(0)
    nblk = (count + 3) // 4
    blk = np.arange(nblk, dtype=np.uint64)
    w = philox4x64_10(
        [blk, np.uint64(iteration), np.uint64(chain), np.uint64(TAG_MOMENTUM)],
        (seed, 0),
    )
    out = np.empty((nblk, 4))
    for pair in range(2):
        u1 = word_to_uniform(w[2 * pair])
        u2 = word_to_uniform(w[2 * pair + 1])
        r = np.sqrt(-2.0 * np.log(u1))
        out[:, 2 * pair] = r * np.cos(2.0 * np.pi * u2)
        out[:, 2 * pair + 1] = r * np.sin(2.0 * np.pi * u2)
    return out.reshape(-1)[:count]


def accept_uniform(seed, iteration, chain):
    """The uniform of the Metropolis test of one chain/iteration."""
    w = philox4x64_10(
        [np.uint64(0), np.uint64(iteration), np.uint64(chain), np.uint64(TAG_ACCEPT)],
        (seed, 0),
    )
    return float(word_to_uniform(w[0]))

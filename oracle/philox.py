"""Philox4x32-10 and Box-Muller normals of the oracle (test infrastructure only).

Eq. 8 needs a random variable N of zero mean and unit variance per
non-conserved moment, site and step.  The method draws it from a counter-based
generator so that every draw is a pure function of (seed, step, site, stream):

* Philox4x32 with 10 rounds, written from the description in J. K. Salmon,
  M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel Random Numbers: As Easy as
  1, 2, 3" (SC'11): a 128-bit counter and a 64-bit key; each round multiplies
  counter words 0 and 2 by two fixed odd constants, and recombines the high and
  low product halves with words 1 and 3 and the round key by XOR; the key is
  advanced by two Weyl constants between rounds.
* Counter layout: word 0 = site index y*nx + x, word 1 = step index (mod 2^32),
  word 2 = call | tag << 8 (tag 0 = dynamics, tag 1 = thermal initial state),
  word 3 = stream id of the replica.  Key = (seed mod 2^32, seed >> 32).
* D2Q9 dynamics (``pair_normals``): the six normals of a site need six words, so
  the two sites 2q and 2q + 1 (the same row, nx even) share word 0 = q: calls 0, 1
  and 2 give twelve words W0..W11, site 2q + h takes W_{6h} .. W_{6h+5}.  (A reading
  of Eq. 8, whose N only needs zero mean and unit variance: every word is used once.)
* Uniform: u = (w + 1/2) 2^-32 in FP64 (never 0 or 1).  Box-Muller on the pair
  (u_a, u_b): r = sqrt(-2 ln u_a), N = (r cos 2 pi u_b, r sin 2 pi u_b).

Parity: Philox words pinned bit-exactly against an installed independent
implementation (Triton's interpreter, run on the CPU) and statistically; the
Box-Muller normals pinned statistically (moments, Kolmogorov-Smirnov) and
against the closed form on constructed words.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)   # round multipliers (SC'11, Philox4x32)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)   # key schedule Weyl increments
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_SH = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, seed):
    """Ten Philox4x32 rounds on arrays of 32-bit counter words; returns 4 uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in np.broadcast_arrays(c0, c1, c2, c3)]
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64(seed >> 32)
    x0, x1, x2, x3 = c
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * x0                      # exact: both factors < 2^32
        p1 = _M1 * x2
        hi0, lo0 = p0 >> _SH, p0 & _MASK
        hi1, lo1 = p1 >> _SH, p1 & _MASK
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return tuple(x.astype(np.uint32) for x in (x0, x1, x2, x3))


def uniform_fp64(words):
    """u = (w + 1/2) / 2^32, exact in FP64 and strictly inside (0, 1)."""
    return (np.asarray(words, dtype=np.float64) + 0.5) * 2.0**-32


def box_muller(ua, ub):
    """Two independent unit normals from two uniforms (Box-Muller)."""
    r = np.sqrt(-2.0 * np.log(ua))
    ang = 2.0 * np.pi * ub
    return r * np.cos(ang), r * np.sin(ang)


def site_normals(n_normals, site, step, tag, stream, seed):
    """n_normals unit normals per site, array (n_normals,) + site.shape.

    Calls 0, 1, ... of the generator give words w0..w3, w4..w7, ...; the pair
    (w_{2p}, w_{2p+1}) gives normals 2p and 2p+1.
    """
    site = np.asarray(site)
    n_calls = (n_normals + 3) // 4
    words = []
    for call in range(n_calls):
        words.extend(philox4x32_10(site, step, call | (tag << 8), stream, seed))
    out = []
    for p in range((n_normals + 1) // 2):
        a, b = box_muller(uniform_fp64(words[2 * p]), uniform_fp64(words[2 * p + 1]))
        out.extend([a, b])
    return np.stack(out[:n_normals])


def pair_normals(site, step, tag, stream, seed):
    """The six unit normals of each D2Q9 site, array (6,) + site.shape.

    Sites 2q and 2q + 1 share the counter index q; calls 0, 1, 2 give words
    W0..W11 and site 2q + h takes W_{6h} .. W_{6h+5}; normals 2m and 2m + 1 of the
    site come from the pair (W_{6h+2m}, W_{6h+2m+1}).
    """
    site = np.asarray(site, dtype=np.uint64)
    q = site >> np.uint64(1)
    h = (site & np.uint64(1)).astype(bool)
    W = []
    for call in range(3):
        W.extend(philox4x32_10(q, step, call | (tag << 8), stream, seed))
    out = []
    for m in range(3):
        wa = np.where(h, W[6 + 2 * m], W[2 * m])
        wb = np.where(h, W[7 + 2 * m], W[2 * m + 1])
        a, b = box_muller(uniform_fp64(wa), uniform_fp64(wb))
        out.extend([a, b])
    return np.stack(out)

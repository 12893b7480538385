"""Oracle: Gaussian test matrix Omega (Algorithm 1, first step; Sec. II.B.2).

Test infrastructure only.  Entries come from the counter-based generator
Philox-4x32-10 of Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
easy as 1, 2, 3" (SC'11), written here from its published definition, and a
Box-Muller transform in FP64:

* key = (seed mod 2^32, seed div 2^32); counter = (n, j, 0, 0) for entry
  (row n, column j); ten rounds, the key bumped by the Weyl constants between
  rounds;
* u1 = (m1 + 1) 2^-53 in (0, 1], u2 = m2 2^-53 in [0, 1), where m1, m2 are
  the 53-bit integers (w0 >> 5) * 2^26 + (w1 >> 6) and likewise from
  (w2, w3);
* g = sqrt(-2 ln u1) cos(2 pi u2).

Omega itself is real N(0, 1) (stored complex with zero imaginary part), or
diag(Phi) times it for the physics-informed test matrix of Eq. (9).

The other test matrices Sec. II.B.2 names take their entries from the same
Philox words (counter (n, j, 0, 0)):

* Rademacher (Clarkson & Woodruff 2009): +1 if bit 0 of w0 is 0, else -1;
* sparse Rademacher with density d in (0, 1] (Achlioptas 2003 for d = 1/3):
  the entry is nonzero iff w1 < floor(d 2^32), and then +-1/sqrt(d) with the
  sign of the Rademacher rule, so that every entry has mean 0, variance 1;
* orthonormal: the Q factor of the Gaussian matrix (built in resolvent.py).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def _mulhilo(a: np.uint64, b: np.ndarray):
    p = a * b.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & MASK32).astype(np.uint32)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Vectorised Philox-4x32-10 over arrays of counters; returns 4 uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = np.uint32(k0 + W0)
                k1 = np.uint32(k1 + W1)
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def raw_words(seed: int, n_rows: int, k: int):
    """Philox words for every (n, j): four uint32 arrays of shape [n_rows, k]."""
    n = np.repeat(np.arange(n_rows, dtype=np.uint64), k).astype(np.uint32)
    j = np.tile(np.arange(k, dtype=np.uint32), n_rows)
    z = np.zeros_like(n)
    ws = philox4x32_10(n, j, z, z, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return [w.reshape(n_rows, k) for w in ws]


def gaussian(seed: int, n_rows: int, k: int) -> np.ndarray:
    """Real N(0,1) matrix [n_rows, k] (float64) from Philox + Box-Muller."""
    w0, w1, w2, w3 = (w.astype(np.uint64) for w in raw_words(seed, n_rows, k))
    m1 = (w0 >> np.uint64(5)) * np.uint64(1 << 26) + (w1 >> np.uint64(6))
    m2 = (w2 >> np.uint64(5)) * np.uint64(1 << 26) + (w3 >> np.uint64(6))
    u1 = (m1.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = m2.astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def rademacher(seed: int, n_rows: int, k: int) -> np.ndarray:
    """+-1 matrix [n_rows, k] (float64): -1 where bit 0 of the first word is set."""
    w0 = raw_words(seed, n_rows, k)[0]
    return np.where((w0 & np.uint32(1)) != 0, -1.0, 1.0)


def sparse_threshold(density: float) -> int:
    """Integer cut of the sparse Rademacher rule: entry kept iff w1 < this."""
    if not (0.0 < density <= 1.0):
        raise ValueError("density must be in (0, 1]")
    return int(np.floor(density * 2.0 ** 32))


def sparse_rademacher(seed: int, n_rows: int, k: int, density: float) -> np.ndarray:
    """Sparse sign matrix: +-1/sqrt(d) with probability d, else 0."""
    w0, w1 = raw_words(seed, n_rows, k)[:2]
    keep = w1.astype(np.uint64) < np.uint64(sparse_threshold(density))
    mag = 1.0 / np.sqrt(density)
    sign = np.where((w0 & np.uint32(1)) != 0, -mag, mag)
    return np.where(keep, sign, 0.0)


KINDS = ("gaussian", "rademacher", "sparse_rademacher", "orthonormal")


def test_matrix(seed: int, n_rows: int, k: int, phi=None, kind: str = "gaussian",
                density: float = 1.0 / 3.0) -> np.ndarray:
    """Omega (complex128, [N, k]); with phi (length N) Omega_p = diag(phi) Omega.

    kind "orthonormal" returns diag(phi) G before its QR; resolvent.py takes
    the QR (the orthonormalised test matrix of Sec. II.B.2)."""
    if kind in ("gaussian", "orthonormal"):
        g = gaussian(seed, n_rows, k)
    elif kind == "rademacher":
        g = rademacher(seed, n_rows, k)
    elif kind == "sparse_rademacher":
        g = sparse_rademacher(seed, n_rows, k, density)
    else:
        raise ValueError(f"unknown test matrix kind {kind!r}")
    if phi is not None:
        g = np.asarray(phi, dtype=np.float64)[:, None] * g
    return g.astype(np.complex128)

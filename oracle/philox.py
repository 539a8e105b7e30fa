"""Philox4x32-10 and Z4 noise for the oracle.

Z4 noise (Sec. 2, Eqs. 1-2): every component of a source eta_r is drawn
independently and uniformly from {1, i, -1, -i}.  The paper does not say how the
random numbers are produced; this library uses the counter-based generator
Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11), so that a source depends only on (seed, source
index, site) and can be regenerated anywhere.

Mapping (one Philox block per site and source):
    counter = (site_lex, r, 0, 0),  key = (seed mod 2^32, seed >> 32)
    k_{alpha,c} = bits [2(3 alpha + c), 2(3 alpha + c) + 1] of output word 0
    eta_r(x)_{alpha c} = i ** k_{alpha,c}
"""
import numpy as np

# Round multipliers and key increments of Philox4x32 (SC'11 paper).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Apply the 10-round Philox4x32 bijection.

    ctr: integer array (..., 4) of 32-bit words; key: (..., 2) of 32-bit words,
    broadcast against ctr.  Returns uint32 array (..., 4).

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
        (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
    where hi/lo are the upper/lower 32 bits of the 64-bit product; the key is
    advanced by the Weyl increments (W0, W1) between rounds.
    """
    c = np.asarray(ctr, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK32
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def z4_noise(L, seed, first_src, nsrc):
    """Z4 sources eta_r, r = first_src .. first_src + nsrc - 1.

    L = (X, Y, Z, T).  Returns complex128 array (nsrc, T, Z, Y, X, 4, 3).
    """
    X, Y, Z, T = (int(v) for v in L)
    V = X * Y * Z * T
    site = np.arange(V, dtype=np.uint64)
    out = np.empty((nsrc, V, 4, 3), dtype=np.complex128)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    phases = np.array([1, 1j, -1, -1j], dtype=np.complex128)
    for j in range(nsrc):
        r = first_src + j
        ctr = np.zeros((V, 4), dtype=np.uint64)
        ctr[:, 0] = site
        ctr[:, 1] = r
        w0 = philox4x32_10(ctr, key)[:, 0].astype(np.uint64)
        for alpha in range(4):
            for c in range(3):
                sh = np.uint64(2 * (3 * alpha + c))
                k = ((w0 >> sh) & np.uint64(3)).astype(np.int64)
                out[j, :, alpha, c] = phases[k]
    return out.reshape(nsrc, T, Z, Y, X, 4, 3)


def z4_noise_diluted(L, seed, first_src, nsrc, t0, dt):
    """Time dilution with coherent sources (Sec. 2.3): the Z4 source on the time
    slices t = t0 (mod dt), zero elsewhere."""
    eta = z4_noise(L, seed, first_src, nsrc)
    T = int(L[3])
    mask = ((np.arange(T) - t0) % dt == 0).astype(np.float64)
    return eta * mask[None, :, None, None, None, None, None]

"""Dirac matrices for the oracle.

The paper (Sec. 2.2, Eqs. 5-6, Table 2) uses the complete set of 16 Dirac
structures but does not fix a basis.  This module fixes the DeGrand-Rossi chiral
basis in Euclidean space, with mu = 0..3 for the x, y, z, t directions, and the
ordering Gamma_n = g1^n0 g2^n1 g3^n2 g4^n3 with n = n0 + 2 n1 + 4 n2 + 8 n3, so
Gamma_0 = 1 and Gamma_15 = g1 g2 g3 g4 = gamma_5 = diag(1, 1, -1, -1).
"""
import numpy as np

_i = 1j

# gamma_1 .. gamma_4 written out entry by entry (rows, columns = Dirac index).
GAMMA = np.array([
    [[0, 0, 0, _i], [0, 0, _i, 0], [0, -_i, 0, 0], [-_i, 0, 0, 0]],   # x
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],       # y
    [[0, 0, _i, 0], [0, 0, 0, -_i], [-_i, 0, 0, 0], [0, _i, 0, 0]],   # z
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],         # t
], dtype=np.complex128)

GAMMA5 = np.diag([1, 1, -1, -1]).astype(np.complex128)

ID4 = np.eye(4, dtype=np.complex128)


def gamma_basis():
    """The 16 products Gamma_n, n = 0..15, as a (16, 4, 4) array."""
    out = np.empty((16, 4, 4), dtype=np.complex128)
    for n in range(16):
        g = ID4.copy()
        for k in range(4):
            if (n >> k) & 1:
                g = g @ GAMMA[k]
        out[n] = g
    return out


GAMMA_LABELS = [
    "1", "g1", "g2", "g1g2", "g3", "g1g3", "g2g3", "g1g2g3",
    "g4", "g1g4", "g2g4", "g1g2g4", "g3g4", "g1g3g4", "g2g3g4", "g5",
]

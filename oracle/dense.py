"""Exact (dense) traces for tiny lattices (oracle).

For 12V small enough to store M, the quantities the stochastic method estimates
(Eq. 3 and the identities of Sec. 2.2) are computed exactly:

    Tr_t[Gamma M^{-1}] = sum_{x: x_t = t} Tr_{Dirac, colour}[Gamma M^{-1}(x, x)].

Used only as the exact answer in tests; numpy.linalg.inv is the inversion.
"""
import numpy as np

from .gamma import gamma_basis
from .operator import dense_matrix


def inverse(U, kappa, mu, antiperiodic=True):
    return np.linalg.inv(dense_matrix(U, kappa, mu, antiperiodic))


def diagonal_blocks(A, site_shape):
    """Site-diagonal 12x12 blocks of a (12V, 12V) matrix -> (T, Z, Y, X, 4, 3, 4, 3)."""
    V = int(np.prod(site_shape))
    B = A.reshape(V, 12, V, 12)
    d = B[np.arange(V), :, np.arange(V), :]          # (V, 12, 12)
    return d.reshape(tuple(site_shape) + (4, 3, 4, 3))


def slice_traces(A, site_shape, left=None):
    """sum_{x in slice t} Tr[left Gamma_g A(x, x)] for g = 0..15 -> complex (16, T).

    ``left`` is an optional Dirac matrix multiplying Gamma_g from the left.
    """
    G = gamma_basis()
    if left is not None:
        G = np.einsum("ab,gbc->gac", left, G)
    d = diagonal_blocks(A, site_shape)
    # Tr[G A(x,x)] = sum_{a,b,c} G_{ab} A(x,x)_{(b c),(a c)}
    per_site = np.einsum("gab,tzyxbcac->gtzyx", G, d)
    return per_site.sum(axis=(2, 3, 4))

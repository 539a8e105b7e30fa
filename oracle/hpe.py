"""Hopping Parameter Expansion (oracle), Sec. 2.4, Eqs. 7-8.

Write the operator as M = B^{-1} + H with B = (1 + 2 i kappa mu gamma_5)^{-1}
(site-local) and H = M - B^{-1}, the hopping term (-kappa times the nearest-neighbour
hops of M).  Then, exactly,

    M^{-1} = B - B H B + (BH)^2 B - (BH)^3 B + (BH)^4 M^{-1}       (Eq. 7)

and for a local insertion X the first four terms are computed exactly while
the last is estimated stochastically (Eq. 8):

    Tr[X (BH)^4 M^{-1}] ~ (1/N) sum_r eta_r^dag X (BH)^4 s_r.

This module applies B and H through the oracle operator and evaluates the exact
terms by dense matrices on small lattices.
"""
import numpy as np

from .dense import slice_traces
from .gamma import GAMMA5
from .operator import apply_DW, dense_matrix


def apply_B(psi, kappa, mu):
    """B psi = (1 - i nu g5) psi / (1 + nu^2), nu = 2 kappa mu."""
    nu = 2.0 * kappa * mu
    g5psi = np.einsum("ab,...bc->...ac", GAMMA5, psi)
    return (psi - 1j * nu * g5psi) / (1.0 + nu * nu)


def apply_H(U, psi, kappa, antiperiodic=True):
    """H psi = (M - B^{-1}) psi = D_W psi - psi (the hops of M, times -kappa)."""
    return apply_DW(U, psi, kappa, antiperiodic) - psi


def apply_BH_power(U, psi, kappa, mu, n, antiperiodic=True):
    """(BH)^n psi."""
    out = np.asarray(psi, dtype=np.complex128)
    for _ in range(n):
        out = apply_B(apply_H(U, out, kappa, antiperiodic), kappa, mu)
    return out


def exact_terms_dense(U, kappa, mu, antiperiodic=True):
    """Tr_t[Gamma_g (B - BHB + (BH)^2 B - (BH)^3 B)] per slice -> complex (16, T),
    from dense matrices (small lattices only)."""
    site_shape = U.shape[1:5]
    V = int(np.prod(site_shape))
    M = dense_matrix(U, kappa, mu, antiperiodic)
    nu = 2.0 * kappa * mu
    Ainv = np.kron(np.eye(V), np.kron((np.eye(4) - 1j * nu * GAMMA5) / (1 + nu * nu), np.eye(3)))
    A = np.kron(np.eye(V), np.kron(np.eye(4) + 1j * nu * GAMMA5, np.eye(3)))
    BH = Ainv @ (M - A)
    P1 = BH @ Ainv
    P2 = BH @ P1
    P3 = BH @ P2
    return slice_traces(Ainv - P1 + P2 - P3, site_shape)

"""Twisted-mass Wilson operator for the oracle.

Definition (twisted-mass formulation used throughout the paper, Secs. 2.2 and
2.4; kappa normalisation, nu = 2 kappa mu):

    (M psi)(x) = psi(x) + i nu gamma_5 psi(x)
                 - kappa sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu_hat)
                                + (1 + gamma_mu) U_mu(x - mu_hat)^dag psi(x - mu_hat) ]

with psi antiperiodic in time.  D_W is M at mu = 0 (the Wilson operator, used by
the generalised one-end trick, Eq. 6); M_d, the other flavour, is M with mu -> -mu
(Sec. 2.2, identity below Eq. 5).

The adjoint is the conjugate transpose of the kernel M(x, y):

    (M^dag psi)(x) = psi(x) - i nu gamma_5 psi(x)
                 - kappa sum_mu [ (1 + gamma_mu) U_mu(x) psi(x + mu_hat)
                                + (1 - gamma_mu) U_mu(x - mu_hat)^dag psi(x - mu_hat) ]

Everything is done with full 4x4 Dirac matrices and full 3x3 links; no spin
projection, no link compression.
"""
import numpy as np

from .gamma import GAMMA, GAMMA5, ID4
from .lattice import shift


def _spin(mat, chi):
    """Apply a 4x4 Dirac matrix to a spinor field (..., 4, 3)."""
    return np.einsum("st,...tc->...sc", mat, chi)


def _colour(link, chi):
    """Apply a 3x3 colour matrix field (..., 3, 3) to a spinor field (..., 4, 3)."""
    return np.einsum("...ab,...sb->...sa", link, chi)


def _colour_dag(link, chi):
    """Apply the adjoint of a 3x3 colour matrix field."""
    return np.einsum("...ba,...sb->...sa", link.conj(), chi)


def apply_M(U, psi, kappa, mu, antiperiodic=True, dagger=False):
    """M psi (or M^dag psi) for spinor field(s) psi (..., T, Z, Y, X, 4, 3)."""
    psi = np.asarray(psi, dtype=np.complex128)
    nu = 2.0 * kappa * mu
    sgn = -1.0 if dagger else 1.0
    out = psi + sgn * 1j * nu * _spin(GAMMA5, psi)
    for m in range(4):
        fwd = _colour(U[m], shift(psi, m, +1, antiperiodic))
        Ub = shift(U[m], m, -1)  # U_mu(x - mu_hat), links are periodic
        bwd = _colour_dag(Ub, shift(psi, m, -1, antiperiodic))
        p_minus = ID4 - GAMMA[m]
        p_plus = ID4 + GAMMA[m]
        if not dagger:
            out = out - kappa * (_spin(p_minus, fwd) + _spin(p_plus, bwd))
        else:
            out = out - kappa * (_spin(p_plus, fwd) + _spin(p_minus, bwd))
    return out


def apply_DW(U, psi, kappa, antiperiodic=True):
    """Wilson operator D_W = M at mu = 0."""
    return apply_M(U, psi, kappa, 0.0, antiperiodic)


def apply_MdagM(U, psi, kappa, mu, antiperiodic=True):
    return apply_M(U, apply_M(U, psi, kappa, mu, antiperiodic), kappa, mu,
                   antiperiodic, dagger=True)


def dense_matrix(U, kappa, mu, antiperiodic=True, dagger=False):
    """M as a dense (12V, 12V) matrix, built column by column from unit vectors.

    Row/column index = (site_lex * 4 + alpha) * 3 + colour.
    """
    site_shape = U.shape[1:5]
    V = int(np.prod(site_shape))
    n = 12 * V
    basis = np.eye(n, dtype=np.complex128).reshape((n,) + tuple(site_shape) + (4, 3))
    cols = apply_M(U, basis, kappa, mu, antiperiodic, dagger)
    return cols.reshape(n, n).T.copy()


def apply_M_sites(U, psi, kappa, mu, sites, antiperiodic=True, dagger=False):
    """(M psi) evaluated only at the given sites, by the same formula as apply_M.

    sites: integer array (n, 4) of (x, y, z, t); psi (..., T, Z, Y, X, 4, 3).
    Returns (..., n, 4, 3).  For checks of full-size results at sampled sites.
    """
    psi = np.asarray(psi, dtype=np.complex128)
    sites = np.asarray(sites, dtype=np.int64)
    T, Z, Y, X = psi.shape[-6:-2]
    ext = np.array([X, Y, Z, T])
    nu = 2.0 * kappa * mu
    sgn = -1.0 if dagger else 1.0

    def at(field, c):  # field value at coordinates c (n, 4)
        return field[..., c[:, 3], c[:, 2], c[:, 1], c[:, 0], :, :]

    centre = at(psi, sites)
    out = centre + sgn * 1j * nu * np.einsum("ab,...bc->...ac", GAMMA5, centre)
    for m in range(4):
        fwd = sites.copy()
        fwd[:, m] = (fwd[:, m] + 1) % ext[m]
        bwd = sites.copy()
        bwd[:, m] = (bwd[:, m] - 1) % ext[m]
        bc_f = np.ones(len(sites))
        bc_b = np.ones(len(sites))
        if antiperiodic and m == 3:
            bc_f[sites[:, 3] == T - 1] = -1.0
            bc_b[sites[:, 3] == 0] = -1.0
        Uf = U[m][sites[:, 3], sites[:, 2], sites[:, 1], sites[:, 0]]        # U_mu(x)
        Ub = U[m][bwd[:, 3], bwd[:, 2], bwd[:, 1], bwd[:, 0]]                # U_mu(x - mu)
        f = np.einsum("nab,...nsb->...nsa", Uf, at(psi, fwd)) * bc_f[:, None, None]
        b = np.einsum("nba,...nsb->...nsa", Ub.conj(), at(psi, bwd)) * bc_b[:, None, None]
        p_minus, p_plus = ID4 - GAMMA[m], ID4 + GAMMA[m]
        if not dagger:
            out = out - kappa * (_spin(p_minus, f) + _spin(p_plus, b))
        else:
            out = out - kappa * (_spin(p_plus, f) + _spin(p_minus, b))
    return out

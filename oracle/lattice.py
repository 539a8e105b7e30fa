"""Lattice shifts for the oracle.

Fields are numpy arrays whose site axes are (T, Z, Y, X) followed by a fixed
number of internal axes (two for a spinor: Dirac, colour; two for a link:
colour, colour).  Direction mu = 0, 1, 2, 3 is x, y, z, t.

Fermion fields obey periodic boundary conditions in space and, when
``antiperiodic`` is set, antiperiodic ones in time: psi(t + T) = -psi(t).  Gauge
links are always periodic.  This is the boundary condition stated with the
operator in the twisted-mass formulation used by the paper (Sec. 3, "antiperiodic
in time").
"""
import numpy as np


def site_axis(mu, n_internal=2):
    """Array axis of direction mu for a field with ``n_internal`` trailing axes."""
    return -(n_internal + 1) - mu


def shift(field, mu, step, antiperiodic=False, n_internal=2):
    """Return g with g(x) = field(x + step * mu_hat), step = +1 or -1.

    With ``antiperiodic`` and mu = 3, the value that wrapped around the time
    boundary is multiplied by -1 (fermion boundary condition).
    """
    ax = site_axis(mu, n_internal)
    g = np.roll(field, -step, axis=ax)
    if antiperiodic and mu == 3:
        T = field.shape[ax]
        idx = [slice(None)] * field.ndim
        # x + mu_hat wraps for x_t = T - 1; x - mu_hat wraps for x_t = 0.
        idx[ax] = T - 1 if step == +1 else 0
        g[tuple(idx)] *= -1
    return g


def dims_of_spinor(psi):
    """(X, Y, Z, T) extents of a spinor array (..., T, Z, Y, X, 4, 3)."""
    T, Z, Y, X = psi.shape[-6:-2]
    return X, Y, Z, T


def volume(L):
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])

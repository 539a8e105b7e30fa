"""Disconnected-loop contractions (oracle).

A loop is the trace of an insertion X against the quark propagator.  With the
stochastic inverse of Eq. 3, M^{-1} ~ (1/N) sum_r s_r eta_r^dag, every estimator
the paper uses is a bilinear  L_r^dag (P X) R_r  summed over the lattice, with
the per-source pair (L, R) and the Dirac matrix P given by the method:

  mode "std"  L = eta_r, R = s_r,            P = 1      -> Tr[X M^{-1}]            (Eq. 3)
  mode "vv"   L = s_r,   R = s_r,            P = gamma5 -> one-end trick, Eq. 5;
              -2 i nu <.> estimates Tr[M_u^{-1} X] - Tr[M_d^{-1} X]
  mode "gen"  L = s_r,   R = gamma5 D_W s_r, P = gamma5 -> generalised one-end
              trick, Eq. 6; 2 <.> estimates Tr[M_u^{-1} X] + Tr[M_d^{-1} X]

This module only evaluates L^dag P X R; building R for "gen" (one D_W
application) and the prefactors belong to the caller.  Loops are resolved in
the insertion time t: the paper computes "the fermion loop at all insertion
times simultaneously" (Sec. 2.2, end).  The overall fermion-loop sign is left
out.

Local insertions (X = Gamma_g, Sec. 1 and Table 2, "ultra-local"):
    l[g, t] = sum_{x: x_t = t} sum_{alpha beta c} conj(L(x)_{alpha c}) (P Gamma_g)_{alpha beta} R(x)_{beta c}

One-derivative insertions (X = Gamma_g D_mu, "one-derivative" operators of
Sec. 1, Fig. 1 left and Table 2): the symmetric covariant derivative
    psibar Gamma <->D_mu psi,  <->D = (->D - <-D) / 2,
    ->D_mu psi(x)    = [U_mu(x) psi(x + mu) - U_mu(x - mu)^dag psi(x - mu)] / 2,
    psibar <-D_mu(x) = [psibar(x + mu) U_mu(x)^dag - psibar(x - mu) U_mu(x - mu)] / 2,
so the contribution of site x (assigned to its own time slice) is
    1/4 [ Lb(x) G U_mu(x) R(x+mu)   - Lb(x) G U_mu(x-mu)^dag R(x-mu)
        - Lb(x+mu) G U_mu(x)^dag R(x) + Lb(x-mu) G U_mu(x-mu) R(x) ],
with Lb = L^dag, G = P Gamma_g acting on Dirac indices and the links on colour.
Fermion fields are antiperiodic in time, so the hops that wrap around the time
boundary carry a factor -1.
"""
import numpy as np

from .gamma import GAMMA5, ID4, gamma_basis
from .lattice import shift

MODES = ("std", "vv", "gen")


def mode_matrix(mode):
    if mode == "std":
        return ID4
    if mode in ("vv", "gen"):
        return GAMMA5
    raise ValueError(mode)


def _bilinear_per_site(Lf, G16, Rf):
    """conj(Lf)_{alpha c} G16[g]_{alpha beta} Rf_{beta c}, per site -> (g, ..., T, Z, Y, X)."""
    return np.einsum("...ac,gab,...bc->g...", Lf.conj(), G16, Rf)


def _slice_sum(per_site):
    """Sum (g, ..., T, Z, Y, X) over the spatial axes -> (..., g, T)."""
    s = per_site.sum(axis=(-3, -2, -1))
    return np.moveaxis(s, 0, -2)


def local_loops(L, R, mode):
    """Local loops for one source or a batch: returns complex128 (..., 16, T)."""
    G16 = np.einsum("ab,gbc->gac", mode_matrix(mode), gamma_basis())
    return _slice_sum(_bilinear_per_site(np.asarray(L), G16, np.asarray(R)))


def _colour(link, chi):
    return np.einsum("...ab,...sb->...sa", link, chi)


def _colour_dag(link, chi):
    return np.einsum("...ba,...sb->...sa", link.conj(), chi)


def oneD_loops(U, L, R, mode, antiperiodic=True):
    """One-derivative loops: returns complex128 (..., 4, 16, T), axis -3 = mu."""
    G16 = np.einsum("ab,gbc->gac", mode_matrix(mode), gamma_basis())
    L = np.asarray(L, dtype=np.complex128)
    R = np.asarray(R, dtype=np.complex128)
    out = []
    for m in range(4):
        U_x = U[m]
        U_xm = shift(U[m], m, -1)                       # U_mu(x - mu)
        R_p = shift(R, m, +1, antiperiodic)             # R(x + mu)
        R_m = shift(R, m, -1, antiperiodic)             # R(x - mu)
        L_p = shift(L, m, +1, antiperiodic)             # L(x + mu)
        L_m = shift(L, m, -1, antiperiodic)             # L(x - mu)
        site = (_bilinear_per_site(L, G16, _colour(U_x, R_p))
                - _bilinear_per_site(L, G16, _colour_dag(U_xm, R_m))
                - _bilinear_per_site(L_p, G16, _colour_dag(U_x, R))
                + _bilinear_per_site(L_m, G16, _colour(U_xm, R)))
        out.append(0.25 * _slice_sum(site))
    return np.stack(out, axis=-3)


def local_loops_mom(L, R, mode, momenta):
    """Momentum-projected local loops: sum_{x in t} exp(-i p.x) L^dag (P Gamma) R(x),
    p = 2 pi (n_x/X, n_y/Y, n_z/Z); returns (..., n_mom, 16, T)."""
    L = np.asarray(L)
    R = np.asarray(R)
    T, Z, Y, X = L.shape[-6:-2]
    G16 = np.einsum("ab,gbc->gac", mode_matrix(mode), gamma_basis())
    site = _bilinear_per_site(L, G16, R)          # (g, ..., T, Z, Y, X)
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    out = []
    for n in momenta:
        ph = np.exp(-2j * np.pi * (n[0] * x / X + n[1] * y / Y + n[2] * z / Z))
        out.append(_slice_sum(site * ph))
    return np.stack(out, axis=-3)

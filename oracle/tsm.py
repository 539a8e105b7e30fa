"""Truncated Solver Method estimator (oracle), Eq. 4 of Sec. 2.1.

With N_HP high-precision solves and N_HP + N_LP low-precision solves,

    X_TSM = (1/N_HP) sum_{j=1}^{N_HP} [ f(s_j^HP) - f(s_j^LP) ]        (correction)
          + (1/N_LP) sum_{j=N_HP+1}^{N_HP+N_LP} f(s_j^LP)              (biased estimate)

Eq. 4 is written for the inverse itself; it is applied here per source to the
loop values f(s_j) (they are linear in M_E^{-1} for the standard estimator, and
the same argument of unbiasedness holds source by source for the one-end
estimators).  The statistical error follows from the independence of the
sources:

    err^2 = Var_j(f_HP - f_LP) / N_HP + Var_j(f_LP) / N_LP,

with unbiased (n - 1) sample variances, taken separately for the real and the
imaginary part.  A complex prefactor ``scale`` (e.g. -2 i nu for the one-end
trick, 2 for its generalisation) multiplies every per-source value first.
A variance over fewer than two sources is undefined and yields NaN; with
N_HP = 0 the correction term is absent.
"""
import numpy as np


def _var(a):
    """Unbiased sample variance along axis 0, NaN for fewer than two samples."""
    n = a.shape[0]
    if n < 2:
        return np.full(a.shape[1:], np.nan)
    mean = a.sum(axis=0) / n
    return ((a - mean) ** 2).sum(axis=0) / (n - 1)


def tsm_combine(l_hp, l_lp_on_hp, l_lp, scale=1.0):
    """Return (mean complex, err_re, err_im) for arrays (N, ...) of per-source loops."""
    l_hp = np.asarray(l_hp, dtype=np.complex128) * scale
    l_lp_on_hp = np.asarray(l_lp_on_hp, dtype=np.complex128) * scale
    l_lp = np.asarray(l_lp, dtype=np.complex128) * scale
    n_hp, n_lp = l_hp.shape[0], l_lp.shape[0]
    if n_lp < 1:
        raise ValueError("the TSM estimator needs at least one low-precision-only source")
    biased = l_lp.sum(axis=0) / n_lp
    err2_re = _var(l_lp.real) / n_lp
    err2_im = _var(l_lp.imag) / n_lp
    if n_hp > 0:
        diff = l_hp - l_lp_on_hp
        mean = diff.sum(axis=0) / n_hp + biased
        err2_re = err2_re + _var(diff.real) / n_hp
        err2_im = err2_im + _var(diff.imag) / n_hp
    else:
        mean = biased
    return mean, np.sqrt(err2_re), np.sqrt(err2_im)

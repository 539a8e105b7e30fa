"""Conjugate gradient on the normal equations (oracle).

The paper inverts with "a CG solver" (Sec. 2.1) and truncates the low-precision
solves at a residual |r_hat| ~ 1e-2 (Sec. 2.1, tuning paragraph).  The residual
is read here as the recursive residual of the normal equations relative to the
right-hand side:

    solve  A x = b,  A = M^dag M,  b = M^dag eta,  x_0 = 0,
    stop when |r_k| <= tol * |b|,

so that x = M^{-1} eta = s (Eq. 3).  This is the textbook Hestenes-Stiefel
iteration, in complex128, one source at a time.
"""
import numpy as np

from .operator import apply_M


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def cg_normal(U, eta, kappa, mu, tol, max_iter=100000, antiperiodic=True):
    """Solve M s = eta through M^dag M s = M^dag eta for one source.

    Returns (s, info) with info = dict(iters, rel_res, true_res_normal, true_res_M).
    """
    eta = np.asarray(eta, dtype=np.complex128)
    b = apply_M(U, eta, kappa, mu, antiperiodic, dagger=True)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    bb = _dot(b, b).real
    rr = bb
    k = 0
    while k < max_iter and rr > tol * tol * bb:
        t = apply_M(U, p, kappa, mu, antiperiodic)
        q = apply_M(U, t, kappa, mu, antiperiodic, dagger=True)
        alpha = rr / _dot(t, t).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = _dot(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
    mx = apply_M(U, x, kappa, mu, antiperiodic)
    ax = apply_M(U, mx, kappa, mu, antiperiodic, dagger=True)
    info = dict(
        iters=k,
        rel_res=float(np.sqrt(rr / bb)) if bb > 0 else 0.0,
        true_res_normal=float(np.linalg.norm((b - ax).ravel()) / max(np.sqrt(bb), 1e-300)),
        true_res_M=float(np.linalg.norm((eta - mx).ravel())
                         / max(np.linalg.norm(eta.ravel()), 1e-300)),
    )
    return x, info


def solve_many(U, etas, kappa, mu, tol, max_iter=100000, antiperiodic=True):
    """cg_normal for each source of a batch (nsrc, T, Z, Y, X, 4, 3)."""
    sols = np.empty_like(np.asarray(etas, dtype=np.complex128))
    infos = []
    for j in range(etas.shape[0]):
        sols[j], info = cg_normal(U, etas[j], kappa, mu, tol, max_iter, antiperiodic)
        infos.append(info)
    return sols, infos

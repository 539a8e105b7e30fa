"""Pins of the oracle's Hopping Parameter Expansion (Sec. 2.4, Eqs. 7-8)."""
import numpy as np

from oracle import dense, hpe, loops
from oracle.gamma import GAMMA, GAMMA5, gamma_basis
from oracle.operator import apply_M, dense_matrix
from oracle.philox import z4_noise
from paper_1401_6749_gb300 import synth


def test_expansion_identity_by_dense_matrices():
    """Eq. 7 holds exactly with B = (1 + i nu g5)^-1, H = M - B^-1 (read: H = -kappa hops)."""
    L = (2, 2, 2, 4)
    U = synth.gauge_field(L, 3, eps=0.6)
    kappa, mu = 0.16, 0.05
    V = 32
    M = dense_matrix(U, kappa, mu)
    nu = 2 * kappa * mu
    Binv = np.kron(np.eye(V), np.kron(np.eye(4) + 1j * nu * GAMMA5, np.eye(3)))
    B = np.linalg.inv(Binv)
    BH = B @ (M - Binv)
    Minv = np.linalg.inv(M)
    rhs = B - BH @ B + BH @ BH @ B - BH @ BH @ BH @ B + np.linalg.matrix_power(BH, 4) @ Minv
    np.testing.assert_allclose(rhs, Minv, atol=1e-13)


def test_operator_pieces():
    L = (4, 2, 2, 4)
    U = synth.gauge_field(L, 5)
    psi = synth.random_spinor(L, 1, 6)[0]
    kappa, mu = 0.15, 0.03
    # B^-1 B = 1 and B^-1 + H = M
    binv_b = apply_M(U, hpe.apply_B(psi, kappa, mu), kappa, mu) - hpe.apply_H(U, hpe.apply_B(psi, kappa, mu), kappa)
    np.testing.assert_allclose(binv_b, psi, atol=1e-13)
    # (BH)^2 = BH applied twice
    np.testing.assert_allclose(hpe.apply_BH_power(U, psi, kappa, mu, 2),
                               hpe.apply_B(hpe.apply_H(U, hpe.apply_BH_power(U, psi, kappa, mu, 1), kappa),
                                           kappa, mu), atol=1e-14)


def test_exact_terms_closed_form_and_gauge_independence():
    """On L >= 4 the odd orders vanish on the diagonal and, per site,
    B + (BH)^2 B = B + kappa^2 sum_mu [B(1-g)B(1+g)B + B(1+g)B(1-g)B] (x colour identity),
    independent of the links."""
    L = (4, 4, 4, 4)
    kappa, mu = 0.16, 0.04
    nu = 2 * kappa * mu
    Bs = (np.eye(4) - 1j * nu * GAMMA5) / (1 + nu * nu)
    D = kappa ** 2 * sum(Bs @ (np.eye(4) - g) @ Bs @ (np.eye(4) + g) @ Bs
                         + Bs @ (np.eye(4) + g) @ Bs @ (np.eye(4) - g) @ Bs for g in GAMMA)
    per_site = 3 * np.einsum("gab,ba->g", gamma_basis(), Bs + D)
    expect = np.repeat(64 * per_site[:, None], 4, axis=1)          # 64 sites per slice
    for seed in (1,):
        got = hpe.exact_terms_dense(synth.gauge_field(L, seed, eps=0.8), kappa, mu)
        np.testing.assert_allclose(got, expect, atol=1e-10)


def test_stochastic_remainder_is_unbiased():
    """exact terms + (1/N) sum eta^dag X (BH)^4 s estimates Tr_t[X M^-1]."""
    L = (4, 4, 2, 4)
    site = (4, 2, 4, 4)
    U = synth.gauge_field(L, 9, eps=0.5)
    kappa, mu = 0.14, 0.05
    Minv = np.linalg.inv(dense_matrix(U, kappa, mu))
    exact = dense.slice_traces(Minv, site)
    # exact terms on this lattice (a direction of extent 2 keeps them gauge dependent,
    # but they are still exact matrix terms)
    ex = hpe.exact_terms_dense(U, kappa, mu)
    N = 48
    eta = z4_noise(L, 31, 0, N)
    s = np.stack([(Minv @ e.ravel()).reshape(e.shape) for e in eta])
    rem = loops.local_loops(eta, hpe.apply_BH_power(U, s, kappa, mu, 4), "std")
    est = ex + rem.mean(axis=0)
    err = np.sqrt(rem.real.var(axis=0, ddof=1) / N) + 1e-15
    assert np.max(np.abs(est.real - exact.real) / err) < 5
    # the remainder has a much smaller variance than the plain estimator
    plain = loops.local_loops(eta, s, "std")
    assert rem.real.var(axis=0).sum() < 0.5 * plain.real.var(axis=0).sum()

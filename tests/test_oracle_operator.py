"""Pins of the oracle's twisted-mass Wilson operator.

The operator is fixed by its definition (twisted-mass Wilson M with
nu = 2 kappa mu, antiperiodic in time); these tests check it against
consequences of that definition that do not reuse the oracle's code:
the free-field momentum-space form, gauge covariance, gamma_5-hermiticity,
adjointness, and the normal-operator identity M^dag M = D_W^dag D_W + nu^2.
"""
import numpy as np
import pytest

from oracle.gamma import GAMMA, GAMMA5, gamma_basis
from oracle.operator import apply_DW, apply_M, apply_M_sites, dense_matrix
from paper_1401_6749_gb300 import synth


def _inner(a, b):
    return np.vdot(a.ravel(), b.ravel())


def test_gamma_algebra():
    I = np.eye(4)
    for m in range(4):
        assert np.allclose(GAMMA[m], GAMMA[m].conj().T)
        for n in range(4):
            ac = GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m]
            assert np.allclose(ac, 2 * I * (m == n))
    g5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
    assert np.allclose(g5, GAMMA5)
    G = gamma_basis()
    assert np.allclose(G[0], I) and np.allclose(G[15], GAMMA5)
    # the 16 products are orthogonal: Tr[G_a^dag G_b] = 4 delta_ab
    gram = np.einsum("aij,bij->ab", G.conj(), G)
    assert np.allclose(gram, 4 * np.eye(16))


@pytest.mark.parametrize("L", [(4, 4, 2, 6), (6, 4, 4, 8)])
def test_free_field_plane_waves(L):
    """U = 1: M e^{ipx} u = M(p) e^{ipx} u with
    M(p) = 1 - 2 kappa sum cos p + 2 i kappa sum gamma_mu sin p_mu + i nu gamma_5,
    spatial p = 2 pi n / L, temporal p = (2n + 1) pi / T (antiperiodic)."""
    X, Y, Z, T = L
    kappa, mu = 0.137, 0.05
    nu = 2 * kappa * mu
    U = synth.unit_gauge(L)
    rng = np.random.default_rng(5)
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    for n in [(0, 0, 0, 0), (1, 0, 1, 2), (3, 1, 1, 5), (2, 3, 0, 1)]:
        p = np.array([2 * np.pi * n[0] / X, 2 * np.pi * n[1] / Y, 2 * np.pi * n[2] / Z,
                      (2 * n[3] + 1) * np.pi / T])
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * u
        Mp = ((1 - 2 * kappa * np.cos(p).sum()) * np.eye(4)
              + 2j * kappa * np.einsum("m,mab->ab", np.sin(p), GAMMA) + 1j * nu * GAMMA5)
        expect = phase[..., None, None] * (Mp @ u)
        np.testing.assert_allclose(apply_M(U, psi, kappa, mu), expect, atol=1e-13)


def test_periodic_time_boundary_option():
    L = (2, 2, 2, 4)
    kappa = 0.1
    U = synth.unit_gauge(L)
    t = np.arange(4).reshape(4, 1, 1, 1)
    p4 = 2 * np.pi / 4
    u = np.arange(12).reshape(4, 3) + 1j
    psi = np.exp(1j * p4 * t)[..., None, None] * np.broadcast_to(u, (4, 2, 2, 2, 4, 3))
    Mp = ((1 - 2 * kappa * (3 + np.cos(p4))) * np.eye(4) + 2j * kappa * np.sin(p4) * GAMMA[3])
    expect = np.exp(1j * p4 * t)[..., None, None] * np.broadcast_to(Mp @ u, (4, 2, 2, 2, 4, 3))
    np.testing.assert_allclose(apply_M(U, psi, kappa, 0.0, antiperiodic=False), expect,
                               atol=1e-13)


def test_gauge_covariance():
    """M[U^g] (g psi) = g (M[U] psi), U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dag."""
    L = (4, 2, 4, 6)
    U = synth.gauge_field(L, seed=3, eps=0.7)
    g = synth.gauge_transform(L, seed=4)
    Ug = np.empty_like(U)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}
    for m in range(4):
        g_fwd = np.roll(g, -1, axis=axes[m])
        Ug[m] = g @ U[m] @ np.swapaxes(g_fwd.conj(), -1, -2)
    psi = synth.random_spinor(L, 1, seed=6)[0]
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    for dagger in (False, True):
        lhs = apply_M(Ug, gpsi, 0.16, 0.01, dagger=dagger)
        rhs = np.einsum("...ab,...sb->...sa", g, apply_M(U, psi, 0.16, 0.01, dagger=dagger))
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_adjoint_and_gamma5_hermiticity():
    L = (4, 4, 2, 4)
    U = synth.gauge_field(L, seed=8)
    phi, psi = synth.random_spinor(L, 2, seed=9)
    kappa, mu = 0.16, 0.03
    # <phi, M psi> = <M^dag phi, psi>
    a = _inner(phi, apply_M(U, psi, kappa, mu))
    b = _inner(apply_M(U, phi, kappa, mu, dagger=True), psi)
    assert abs(a - b) < 1e-11 * abs(a)
    # M(mu)^dag = gamma_5 M(-mu) gamma_5
    g5 = lambda f: np.einsum("ab,...bc->...ac", GAMMA5, f)
    np.testing.assert_allclose(apply_M(U, psi, kappa, mu, dagger=True),
                               g5(apply_M(U, g5(psi), kappa, -mu)), atol=1e-12)


def test_twist_term_and_normal_operator():
    L = (4, 2, 2, 4)
    U = synth.gauge_field(L, seed=10)
    psi = synth.random_spinor(L, 1, seed=11)[0]
    kappa, mu = 0.155, 0.02
    nu = 2 * kappa * mu
    # M - D_W = i nu gamma_5 (kappa normalisation of the twisted mass)
    diff = apply_M(U, psi, kappa, mu) - apply_DW(U, psi, kappa)
    np.testing.assert_allclose(diff, 1j * nu * np.einsum("ab,...bc->...ac", GAMMA5, psi),
                               atol=1e-13)
    # M^dag M = D_W^dag D_W + nu^2
    lhs = apply_M(U, apply_M(U, psi, kappa, mu), kappa, mu, dagger=True)
    dw = apply_DW(U, apply_DW(U, psi, kappa), kappa)
    rhs = apply_M(U, apply_DW(U, psi, kappa), kappa, 0.0, dagger=True) + nu ** 2 * psi
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    assert dw.shape == psi.shape


def test_dense_matrix_adjoint():
    L = (2, 2, 2, 4)
    U = synth.gauge_field(L, seed=12)
    A = dense_matrix(U, 0.16, 0.01)
    Ad = dense_matrix(U, 0.16, 0.01, dagger=True)
    np.testing.assert_allclose(Ad, A.conj().T, atol=1e-14)
    # the diagonal blocks are exactly 1 + i nu gamma_5 (no self-hop for L >= 2)
    nu = 2 * 0.16 * 0.01
    blk = A[:12, :12]
    expect = np.kron(np.eye(4) + 1j * nu * GAMMA5, np.eye(3))
    np.testing.assert_allclose(blk, expect, atol=1e-15)


def test_sampled_sites_match_whole_lattice():
    L = (4, 6, 2, 8)
    U = synth.gauge_field(L, seed=13)
    psi = synth.random_spinor(L, 2, seed=14)
    rng = np.random.default_rng(0)
    sites = np.stack([rng.integers(0, n, 40) for n in L], axis=1)
    sites[0] = (3, 5, 1, 7)                       # every coordinate at its upper edge
    sites[1] = (0, 0, 0, 0)
    for dagger in (False, True):
        full = apply_M(U, psi, 0.16, 0.02, dagger=dagger)
        ref = full[:, sites[:, 3], sites[:, 2], sites[:, 1], sites[:, 0]]
        np.testing.assert_allclose(apply_M_sites(U, psi, 0.16, 0.02, sites, dagger=dagger), ref,
                                   atol=1e-13)

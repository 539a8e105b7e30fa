"""Pins of the oracle's CG and loop contractions.

Exact identities are checked by "probing" with the complete set of 12V unit
vectors e_k: sum_k L_k^dag (P X) R_k over all unit sources equals the exact
trace that the stochastic estimators of Eqs. 3, 5 and 6 converge to, which is
computed independently from the diagonal blocks of a dense inverse
(numpy.linalg.inv).  Free-field (unit-link) momentum sums give closed forms.
"""
import numpy as np
import pytest

from oracle import cg, dense, loops
from oracle.gamma import GAMMA5, gamma_basis
from oracle.operator import apply_DW, apply_M, dense_matrix
from oracle.philox import z4_noise
from paper_1401_6749_gb300 import synth


def _unit_sources(site_shape):
    n = 12 * int(np.prod(site_shape))
    return np.eye(n, dtype=np.complex128).reshape((n,) + tuple(site_shape) + (4, 3))


def _cols_as_spinors(A, site_shape):
    """Columns of a (12V, 12V) matrix as a batch of spinor fields."""
    n = A.shape[0]
    return A.T.reshape((n,) + tuple(site_shape) + (4, 3))


def _g5(f):
    return np.einsum("ab,...bc->...ac", GAMMA5, f)


@pytest.fixture(scope="module")
def small():
    L = (2, 2, 2, 4)
    site = (L[3], L[2], L[1], L[0])
    U = synth.gauge_field(L, seed=21, eps=0.5)
    kappa, mu = 0.16, 0.05
    Mu = dense_matrix(U, kappa, mu)
    Md = dense_matrix(U, kappa, -mu)
    return dict(L=L, site=site, U=U, kappa=kappa, mu=mu, nu=2 * kappa * mu,
                Mu_inv=np.linalg.inv(Mu), Md_inv=np.linalg.inv(Md))


def test_cg_matches_dense_solve(small):
    eta = z4_noise(small["L"], 99, 0, 2)
    for j in range(2):
        s, info = cg.cg_normal(small["U"], eta[j], small["kappa"], small["mu"], tol=1e-13)
        exact = (small["Mu_inv"] @ eta[j].ravel()).reshape(eta[j].shape)
        np.testing.assert_allclose(s, exact, atol=1e-10)
        assert info["true_res_M"] < 1e-10
        assert info["rel_res"] <= 1e-13


def test_cg_truncation_and_zero_source(small):
    eta = z4_noise(small["L"], 5, 0, 1)[0]
    s, info = cg.cg_normal(small["U"], eta, small["kappa"], small["mu"], tol=1e-2)
    assert info["rel_res"] <= 1e-2 and info["iters"] >= 1
    z, zi = cg.cg_normal(small["U"], np.zeros_like(eta), small["kappa"], small["mu"], tol=1e-10)
    assert zi["iters"] == 0 and not np.any(z)


def test_local_std_probe_equals_dense_trace(small):
    E = _unit_sources(small["site"])
    S = _cols_as_spinors(small["Mu_inv"], small["site"])
    probe = loops.local_loops(E, S, "std").sum(axis=0)
    exact = dense.slice_traces(small["Mu_inv"], small["site"])
    np.testing.assert_allclose(probe, exact, atol=1e-12)


def test_one_end_identities_local(small):
    """Eq. 5 (read with the sign fixed by dense inversion):
         -2 i nu Tr[(M_u^{-1})^dag g5 X M_u^{-1}] = Tr[M_u^{-1} X] - Tr[M_d^{-1} X];
       Eq. 6:  2 Tr[(M_u^{-1})^dag g5 X g5 D_W M_u^{-1}] = Tr[M_u^{-1} X] + Tr[M_d^{-1} X]."""
    S = _cols_as_spinors(small["Mu_inv"], small["site"])
    vv = loops.local_loops(S, S, "vv").sum(axis=0)
    tr_u = dense.slice_traces(small["Mu_inv"], small["site"])
    tr_d = dense.slice_traces(small["Md_inv"], small["site"])
    np.testing.assert_allclose(-2j * small["nu"] * vv, tr_u - tr_d, atol=1e-11)
    R = _g5(apply_DW(small["U"], S, small["kappa"]))
    gen = loops.local_loops(S, R, "gen").sum(axis=0)
    np.testing.assert_allclose(2 * gen, tr_u + tr_d, atol=1e-11)


def test_one_end_identities_oneD(small):
    """The same identities hold for any insertion X, in particular Gamma <->D_mu."""
    U, k = small["U"], small["kappa"]
    E = _unit_sources(small["site"])
    Su = _cols_as_spinors(small["Mu_inv"], small["site"])
    Sd = _cols_as_spinors(small["Md_inv"], small["site"])
    tr_u = loops.oneD_loops(U, E, Su, "std").sum(axis=0)
    tr_d = loops.oneD_loops(U, E, Sd, "std").sum(axis=0)
    vv = loops.oneD_loops(U, Su, Su, "vv").sum(axis=0)
    np.testing.assert_allclose(-2j * small["nu"] * vv, tr_u - tr_d, atol=1e-11)
    gen = loops.oneD_loops(U, Su, _g5(apply_DW(U, Su, k)), "gen").sum(axis=0)
    np.testing.assert_allclose(2 * gen, tr_u + tr_d, atol=1e-11)


def _free_momenta(L):
    X, Y, Z, T = L
    p = np.meshgrid(2 * np.pi * np.arange(X) / X, 2 * np.pi * np.arange(Y) / Y,
                    2 * np.pi * np.arange(Z) / Z, (2 * np.arange(T) + 1) * np.pi / T,
                    indexing="ij")
    return [a.ravel() for a in p]


def test_free_field_closed_forms():
    """U = 1.  With m = 1 - 2k sum cos p, s_mu = 2k sin p_mu, den = m^2 + s^2 + nu^2,
    M^{-1}(p) = (m - i g.s - i nu g5)/den, so per site
      Tr[M^{-1}(x,x)] = (12/V) sum_p m/den,  Tr[g5 M^{-1}(x,x)] = (-12 i nu/V) sum_p 1/den,
    and for the symmetric one-derivative insertion
      Tr[g_mu <->D_mu M^{-1}] per site = (24 k / V) sum_p sin^2 p_mu / den,
    every other Gamma giving zero."""
    L = (4, 2, 2, 4)
    X, Y, Z, T = L
    V, V3 = X * Y * Z * T, X * Y * Z
    site = (T, Z, Y, X)
    kappa, mu = 0.124, 0.04
    nu = 2 * kappa * mu
    U = synth.unit_gauge(L)
    Minv = np.linalg.inv(dense_matrix(U, kappa, mu))
    p = _free_momenta(L)
    m = 1 - 2 * kappa * sum(np.cos(q) for q in p)
    s2 = sum((2 * kappa * np.sin(q)) ** 2 for q in p)
    den = m ** 2 + s2 + nu ** 2
    tr1 = 12 / V * np.sum(m / den)
    tr5 = -12j * nu / V * np.sum(1 / den)
    E = _unit_sources(site)
    S = _cols_as_spinors(Minv, site)
    loc = loops.local_loops(E, S, "std").sum(axis=0)          # (16, T)
    expect = np.zeros((16, T), dtype=complex)
    expect[0] = V3 * tr1
    expect[15] = V3 * tr5
    np.testing.assert_allclose(loc, expect, atol=1e-12)
    oneD = loops.oneD_loops(U, E, S, "std").sum(axis=0)      # (4, 16, T)
    expect = np.zeros((4, 16, T), dtype=complex)
    for mu_ in range(4):
        expect[mu_, 1 << mu_] = V3 * 24 * kappa / V * np.sum(np.sin(p[mu_]) ** 2 / den)
    np.testing.assert_allclose(oneD, expect, atol=1e-12)


def test_loops_gauge_invariant_per_source():
    """U -> U^g, eta -> g eta gives s -> g s and leaves every loop unchanged."""
    L = (2, 4, 2, 4)
    site = (L[3], L[2], L[1], L[0])
    U = synth.gauge_field(L, seed=31, eps=0.6)
    g = synth.gauge_transform(L, seed=32)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}
    Ug = np.empty_like(U)
    for m in range(4):
        Ug[m] = g @ U[m] @ np.swapaxes(np.roll(g, -1, axis=axes[m]).conj(), -1, -2)
    kappa, mu = 0.15, 0.02
    eta = z4_noise(L, 77, 0, 1)[0]
    geta = np.einsum("...ab,...sb->...sa", g, eta)
    s = (np.linalg.inv(dense_matrix(U, kappa, mu)) @ eta.ravel()).reshape(eta.shape)
    sg = (np.linalg.inv(dense_matrix(Ug, kappa, mu)) @ geta.ravel()).reshape(eta.shape)
    np.testing.assert_allclose(sg, np.einsum("...ab,...sb->...sa", g, s), atol=1e-11)
    for mode, (Lf, Rf, Lg, Rg) in {
            "std": (eta, s, geta, sg),
            "vv": (s, s, sg, sg),
            "gen": (s, _g5(apply_DW(U, s, kappa)), sg, _g5(apply_DW(Ug, sg, kappa)))}.items():
        np.testing.assert_allclose(loops.local_loops(Lg, Rg, mode),
                                   loops.local_loops(Lf, Rf, mode), atol=1e-11)
        np.testing.assert_allclose(loops.oneD_loops(Ug, Lg, Rg, mode),
                                   loops.oneD_loops(U, Lf, Rf, mode), atol=1e-11)
    assert site[0] == L[3]


def test_stochastic_estimate_within_errors(small):
    """Eq. 3 with 64 Z4 sources estimates Tr_t[Gamma M^{-1}] within 4 sigma."""
    N = 64
    eta = z4_noise(small["L"], 2024, 0, N)
    S = np.stack([(small["Mu_inv"] @ e.ravel()).reshape(e.shape) for e in eta])
    per = loops.local_loops(eta, S, "std")               # (N, 16, T)
    est = per.mean(axis=0)
    err_re = per.real.std(axis=0, ddof=1) / np.sqrt(N)
    err_im = per.imag.std(axis=0, ddof=1) / np.sqrt(N)
    exact = dense.slice_traces(small["Mu_inv"], small["site"])
    zre = np.abs(est.real - exact.real) / np.maximum(err_re, 1e-15)
    zim = np.abs(est.imag - exact.imag) / np.maximum(err_im, 1e-15)
    assert np.max(zre) < 5 and np.max(zim) < 5
    assert np.mean(zre) < 1.5 and np.mean(zim) < 1.5

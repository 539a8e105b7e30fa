"""Pins of the oracle's Truncated Solver Method estimator (Eq. 4)."""
import numpy as np
import pytest

from oracle import cg, dense, loops, tsm
from oracle.operator import dense_matrix
from oracle.philox import z4_noise
from paper_1401_6749_gb300 import synth


def test_hand_computed_example():
    # HP: [1, 3], LP on the HP sources: [0, 1], LP only: [2, 4]
    # mean = ((1-0) + (3-1))/2 + (2+4)/2 = 4.5
    # err^2 = Var([1, 2])/2 + Var([2, 4])/2 = 0.5/2 + 2/2 = 1.25
    mean, ere, eim = tsm.tsm_combine([1.0, 3.0], [0.0, 1.0], [2.0, 4.0])
    assert mean == pytest.approx(4.5)
    assert ere == pytest.approx(np.sqrt(1.25))
    assert eim == 0.0
    # complex prefactor -2i: values (x -> -2i x) put the error on the imaginary part
    mean, ere, eim = tsm.tsm_combine([1.0, 3.0], [0.0, 1.0], [2.0, 4.0], scale=-2j)
    assert mean == pytest.approx(-9j)
    assert ere == 0.0 and eim == pytest.approx(2 * np.sqrt(1.25))


def test_edge_cases():
    mean, ere, eim = tsm.tsm_combine(np.zeros((0, 3)), np.zeros((0, 3)), np.ones((4, 3)))
    np.testing.assert_allclose(mean, 1.0)          # no HP set: plain LP average
    np.testing.assert_allclose(ere, 0.0)
    mean, ere, eim = tsm.tsm_combine([[2.0]], [[1.0]], [[5.0], [7.0]])
    assert mean[0] == pytest.approx(7.0)
    assert np.isnan(ere[0])                        # variance of one HP source undefined
    with pytest.raises(ValueError):
        tsm.tsm_combine([[1.0]], [[1.0]], np.zeros((0, 1)))


def test_identical_maps_give_zero_correction():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((5, 16, 4)) + 1j * rng.standard_normal((5, 16, 4))
    b = rng.standard_normal((9, 16, 4)) + 1j * rng.standard_normal((9, 16, 4))
    mean, _, _ = tsm.tsm_combine(a, a, b)
    np.testing.assert_allclose(mean, b.mean(axis=0), atol=1e-15)


def test_tsm_is_unbiased_where_truncated_solves_are_not():
    """HP = exact inverse, LP = CG truncated at |r|/|b| = 0.1.  Over many sources
    the TSM estimate agrees with the exact trace, the LP-only estimate does not."""
    L = (2, 2, 2, 4)
    site = (L[3], L[2], L[1], L[0])
    U = synth.gauge_field(L, seed=41, eps=0.5)
    kappa, mu = 0.15, 0.05
    Minv = np.linalg.inv(dense_matrix(U, kappa, mu))
    exact = dense.slice_traces(Minv, site)[0].sum()             # Tr[M^{-1}], Gamma = 1
    n_hp, n_lp = 400, 400
    eta = z4_noise(L, 555, 0, n_hp + n_lp)
    f_hp, f_lp = [], []
    for j in range(n_hp + n_lp):
        s_lp, _ = cg.cg_normal(U, eta[j], kappa, mu, tol=1e-1)
        f_lp.append(loops.local_loops(eta[j], s_lp, "std")[0].sum())
        if j < n_hp:
            s_hp = (Minv @ eta[j].ravel()).reshape(eta[j].shape)
            f_hp.append(loops.local_loops(eta[j], s_hp, "std")[0].sum())
    f_hp, f_lp = np.array(f_hp), np.array(f_lp)
    mean, ere, _ = tsm.tsm_combine(f_hp, f_lp[:n_hp], f_lp[n_hp:])
    assert abs(mean.real - exact.real) < 4 * ere
    lp_mean = f_lp.mean()
    lp_err = f_lp.real.std(ddof=1) / np.sqrt(f_lp.size)
    assert abs(lp_mean.real - exact.real) > 4 * lp_err      # the truncated map is biased

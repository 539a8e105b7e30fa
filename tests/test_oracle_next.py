"""Pins of the oracle's time dilution (Sec. 2.3) and momentum-projected loops."""
import numpy as np

from oracle import dense, loops
from oracle.operator import dense_matrix
from oracle.philox import z4_noise, z4_noise_diluted
from paper_1401_6749_gb300 import synth


def test_dilution_partitions_the_source():
    L = (4, 2, 2, 8)
    eta = z4_noise(L, 5, 2, 3)
    for dt in (1, 2, 4, 8):
        parts = [z4_noise_diluted(L, 5, 2, 3, t0, dt) for t0 in range(dt)]
        np.testing.assert_array_equal(sum(parts), eta)
        for t0, p in enumerate(parts):
            on = (np.arange(8) - t0) % dt == 0
            assert not np.any(p[:, ~on])
            np.testing.assert_array_equal(p[:, on], eta[:, on])


def test_fully_diluted_estimate_is_unbiased_and_less_noisy():
    """With one source per time slice (dt = T), slice t of Tr[M^-1] is estimated
    from the source on slice t alone; its spread is below the undiluted one."""
    L = (2, 2, 2, 4)
    site = (4, 2, 2, 2)
    U = synth.gauge_field(L, 7, eps=0.5)
    Minv = np.linalg.inv(dense_matrix(U, 0.15, 0.05))
    exact = dense.slice_traces(Minv, site)[0]            # Gamma = 1, per slice
    N = 200
    und, dil = [], []
    eta = z4_noise(L, 11, 0, N)
    for j in range(N):
        s = (Minv @ eta[j].ravel()).reshape(eta[j].shape)
        und.append(loops.local_loops(eta[j], s, "std")[0])
        est = np.zeros(4, dtype=complex)
        for t0 in range(4):
            e = z4_noise_diluted(L, 11, j, 1, t0, 4)[0]
            sd = (Minv @ e.ravel()).reshape(e.shape)
            est[t0] = loops.local_loops(e, sd, "std")[0][t0]
        dil.append(est)
    und, dil = np.array(und), np.array(dil)
    err = dil.real.std(axis=0, ddof=1) / np.sqrt(N)
    assert np.all(np.abs(dil.real.mean(axis=0) - exact.real) < 5 * err)
    assert dil.real.var(axis=0).sum() < und.real.var(axis=0).sum()


def test_momentum_projection_zero_momentum_translation_and_inversion():
    L = (4, 2, 6, 4)
    X, Y, Z, T = L
    A = synth.random_spinor(L, 1, 3)[0]
    B = synth.random_spinor(L, 1, 4)[0]
    # p = 0 is the plain local loop
    np.testing.assert_allclose(loops.local_loops_mom(A, B, "vv", [(0, 0, 0)])[0],
                               loops.local_loops(A, B, "vv"), atol=1e-12)
    # translating both fields by a multiplies by exp(-i p.a)
    p = (1, 1, 2)
    a = (1, 0, 2)
    As = np.roll(A, a, axis=(3, 2, 1))
    Bs = np.roll(B, a, axis=(3, 2, 1))
    phase = np.exp(-2j * np.pi * (p[0] * a[0] / X + p[1] * a[1] / Y + p[2] * a[2] / Z))
    np.testing.assert_allclose(loops.local_loops_mom(As, Bs, "std", [p])[0],
                               phase * loops.local_loops_mom(A, B, "std", [p])[0], atol=1e-11)
    # summing all momenta with exp(+i p.x0) / V3 recovers the site x0 = (1, 1, 3)
    moms = [(i, j, k) for i in range(X) for j in range(Y) for k in range(Z)]
    lp = loops.local_loops_mom(A, B, "std", moms)                 # (n, 16, T)
    x0 = (1, 1, 3)
    w = np.array([np.exp(2j * np.pi * (m[0] * x0[0] / X + m[1] * x0[1] / Y + m[2] * x0[2] / Z))
                  for m in moms])
    rec = np.einsum("n,ngt->gt", w, lp) / (X * Y * Z)
    only = np.zeros_like(A)
    only[:, x0[2], x0[1], x0[0]] = A[:, x0[2], x0[1], x0[0]]
    np.testing.assert_allclose(rec, loops.local_loops(only, B, "std"), atol=1e-11)

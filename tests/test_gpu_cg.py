"""Parity of the CUDA conjugate-gradient solver with the FP64 oracle.

Solutions are compared with the oracle's dense solve: for a system solved to
relative residual tol on the normal equations, |x - x*| / |x*| <= cond(M^dag M) tol,
so the tests solve to 1e-12 (plain FP64 and mixed precision) and allow 1e-8
on these small, well-conditioned lattices.
"""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle.operator import apply_M, dense_matrix
from oracle.philox import z4_noise as oracle_z4
from paper_1401_6749_gb300 import synth

from .gpu_util import pack, rel_l2, require_gpu, to_dev, unpack

pytestmark = pytest.mark.gpu


def _setup(tl, L, kappa, mu, seed=31, recon=12):
    U = synth.gauge_field(L, seed=seed)
    return U, tl.Operator(L, kappa, mu, to_dev(U), recon=recon)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 4, 8)])
def test_plain_f64_matches_dense_solve(L):
    tl = require_gpu()
    kappa, mu = 0.16, 0.01
    U, op = _setup(tl, L, kappa, mu)
    n = 4
    eta = oracle_z4(L, 11, 0, n)
    x = tl.empty_field(L, 0, n)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, eta, 0), n,
                               tl.cg_params(1e-12, 2000, tl.CG_PLAIN, prec=0, true_residual=True))
    got = unpack(tl, L, x, 0, n)
    for j in range(n):
        assert stats[j]["status"] == 0 and stats[j]["rel_res"] <= 1e-12
        assert stats[j]["true_res"] < 1e-11
        ref, info = ocg.cg_normal(U, eta[j], kappa, mu, tol=1e-13)
        assert rel_l2(got[j], ref) < 1e-9
    # the oracle and the kernel take (nearly) the same number of iterations
    _, info0 = ocg.cg_normal(U, eta[0], kappa, mu, tol=1e-12)
    assert abs(stats[0]["iters"] - info0["iters"]) <= 2
    op.close()


@pytest.mark.parametrize("inner", [1, 2, 3])
def test_mixed_precision_reaches_fp64_accuracy(inner):
    tl = require_gpu()
    L = (4, 4, 4, 8)
    kappa, mu = 0.16, 0.01
    U, op = _setup(tl, L, kappa, mu, seed=5)
    n = 3
    eta = oracle_z4(L, 99, 0, n)
    x = tl.empty_field(L, 0, n)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, eta, 0), n,
                               tl.cg_params(1e-11, 4000, tl.CG_MIXED, inner_prec=inner, delta=0.1))
    got = unpack(tl, L, x, 0, n)
    for j in range(n):
        assert stats[j]["status"] == 0
        assert stats[j]["true_res"] <= 1e-11
        assert stats[j]["reliable_updates"] >= 1
        ref, _ = ocg.cg_normal(U, eta[j], kappa, mu, tol=1e-13)
        assert rel_l2(got[j], ref) < 1e-8
    op.close()


@pytest.mark.parametrize("prec", [2, 3])
def test_low_precision_truncated_solve(prec):
    """LP solves stop at |r|/|b| ~ 1e-2 (Sec. 2.1); the true residual is of that order."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    kappa, mu = 0.16, 0.01
    U, op = _setup(tl, L, kappa, mu, seed=9)
    n = 5
    eta = oracle_z4(L, 3, 0, n)
    x = tl.empty_field(L, prec, n)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, eta, prec), n,
                               tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=prec, true_residual=True))
    got = unpack(tl, L, x, prec, n)
    for j in range(n):
        assert stats[j]["status"] == 0 and stats[j]["rel_res"] <= 1e-2
        b = apply_M(U, eta[j], kappa, mu, dagger=True)
        r = b - apply_M(U, apply_M(U, got[j], kappa, mu), kappa, mu, dagger=True)
        true_rel = np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel())
        assert true_rel < 2e-2
        assert abs(true_rel - stats[j]["true_res"]) < 5e-3
    op.close()


def test_batch_composition_does_not_change_solutions():
    """The LP map must be the same function of eta in every batch (TSM): 6
    systems run 4 + 2 per thread, 2 systems 2 per thread, 1 system alone."""
    tl = require_gpu()
    L = (4, 4, 4, 4)
    U, op = _setup(tl, L, 0.16, 0.01, seed=12)
    eta = oracle_z4(L, 44, 0, 6)
    prm = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=2)
    xa = tl.empty_field(L, 2, 6)
    tl.tm_cg_solve(op, xa, pack(tl, L, eta, 2), 6, prm)
    xb = tl.empty_field(L, 2, 2)
    tl.tm_cg_solve(op, xb, pack(tl, L, eta[3:5], 2), 2, prm)
    a = unpack(tl, L, xa, 2, 6)
    b = unpack(tl, L, xb, 2, 2)
    np.testing.assert_array_equal(a[3:5], b)
    xc = tl.empty_field(L, 2, 1)
    tl.tm_cg_solve(op, xc, pack(tl, L, eta[5:6], 2), 1, prm)
    np.testing.assert_array_equal(a[5], unpack(tl, L, xc, 2, 1)[0])
    op.close()


def test_edge_cases_zero_source_and_noconv():
    tl = require_gpu()
    L = (4, 4, 2, 4)
    U, op = _setup(tl, L, 0.16, 0.01)
    eta = oracle_z4(L, 1, 0, 2)
    eta[1] = 0
    x = tl.empty_field(L, 0, 2)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, eta, 0), 2,
                               tl.cg_params(1e-12, 3, tl.CG_PLAIN, prec=0), raise_on_noconv=False)
    assert st == 3                                  # TM_ERR_NOCONV
    assert stats[0]["status"] == 3 and stats[0]["iters"] == 3
    assert stats[1]["status"] == 0 and stats[1]["iters"] == 0
    assert not np.any(unpack(tl, L, x, 0, 2)[1])
    op.close()


def test_dense_parity_tiny_lattice():
    tl = require_gpu()
    L = (2, 2, 2, 4)
    kappa, mu = 0.17, 0.02
    U, op = _setup(tl, L, kappa, mu, seed=2, recon=18)
    eta = oracle_z4(L, 8, 0, 1)
    x = tl.empty_field(L, 0, 1)
    tl.tm_cg_solve(op, x, pack(tl, L, eta, 0), 1, tl.cg_params(1e-13, 2000, tl.CG_PLAIN, prec=0))
    exact = np.linalg.solve(dense_matrix(U, kappa, mu), eta[0].ravel()).reshape(eta[0].shape)
    assert rel_l2(unpack(tl, L, x, 0, 1)[0], exact) < 1e-10
    op.close()


# ------------------------------------------------------------------ even/odd
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 4, 8), (2, 2, 2, 4)])
def test_schur_plain_f64_matches_oracle_solution(L):
    """The even/odd preconditioned solve returns x = M^-1 eta on both parities."""
    tl = require_gpu()
    kappa, mu = 0.16, 0.01
    U, op = _setup(tl, L, kappa, mu, seed=21)
    n = 3
    eta = oracle_z4(L, 5, 0, n)
    x = tl.empty_field(L, 0, n)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, eta, 0), n,
                               tl.cg_params(1e-12, 2000, tl.CG_PLAIN, prec=0, true_residual=True,
                                            schur=True))
    got = unpack(tl, L, x, 0, n)
    for j in range(n):
        assert stats[j]["status"] == 0 and stats[j]["true_res"] < 1e-11
        ref, _ = ocg.cg_normal(U, eta[j], kappa, mu, tol=1e-13)
        assert rel_l2(got[j], ref) < 1e-9
    op.close()


@pytest.mark.parametrize("inner", [1, 2])
def test_schur_mixed_precision(inner):
    tl = require_gpu()
    L = (4, 4, 4, 8)
    kappa, mu = 0.16, 0.01
    U, op = _setup(tl, L, kappa, mu, seed=5)
    n = 2
    eta = oracle_z4(L, 99, 0, n)
    x = tl.empty_field(L, 0, n)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, eta, 0), n,
                               tl.cg_params(1e-11, 4000, tl.CG_MIXED, inner_prec=inner, delta=0.1,
                                            schur=True))
    got = unpack(tl, L, x, 0, n)
    for j in range(n):
        assert stats[j]["status"] == 0 and stats[j]["true_res"] <= 1e-11
        ref, _ = ocg.cg_normal(U, eta[j], kappa, mu, tol=1e-13)
        assert rel_l2(got[j], ref) < 1e-8
    op.close()


def test_schur_needs_fewer_iterations_and_is_batch_independent():
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U, op = _setup(tl, L, 0.16, 0.01, seed=12)
    eta = oracle_z4(L, 44, 0, 6)
    full = tl.cg_params(1e-8, 2000, tl.CG_PLAIN, prec=1)
    eo = tl.cg_params(1e-8, 2000, tl.CG_PLAIN, prec=1, schur=True)
    x = tl.empty_field(L, 1, 6)
    _, s_full = tl.tm_cg_solve(op, x, pack(tl, L, eta, 1), 6, full)
    _, s_eo = tl.tm_cg_solve(op, x, pack(tl, L, eta, 1), 6, eo)
    assert max(s["iters"] for s in s_eo) < min(s["iters"] for s in s_full)
    lp = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=2, schur=True)
    xa = tl.empty_field(L, 2, 6)
    tl.tm_cg_solve(op, xa, pack(tl, L, eta, 2), 6, lp)
    xb = tl.empty_field(L, 2, 1)
    tl.tm_cg_solve(op, xb, pack(tl, L, eta[4:5], 2), 1, lp)
    np.testing.assert_array_equal(unpack(tl, L, xa, 2, 6)[4], unpack(tl, L, xb, 2, 1)[0])
    op.close()

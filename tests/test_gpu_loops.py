"""Parity of the CUDA loop contractions and TSM combination with the oracle,
and the end-to-end 4^4 pipeline (Z4 noise -> CG -> local + one-derivative loops).

Tolerances: contractions of FP64 fields 1e-12 relative (L2 over the whole
[Gamma][t] array), of FP32 fields 1e-5 (the sums run in FP32 within a block of
1024 sites before FP64 accumulation); loops from high-precision solves 1e-8
(the bar stated for HP loops).
"""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from oracle import loops as oloops
from oracle import tsm as otsm
from oracle.operator import apply_DW
from oracle.philox import z4_noise as oracle_z4
from paper_1401_6749_gb300 import synth

from .gpu_util import from_dev, pack, rel_l2, require_gpu, to_dev, unpack

pytestmark = pytest.mark.gpu

MODES = ["std", "vv", "gen"]


def _g5(f):
    out = f.copy()
    out[..., 2:, :] *= -1
    return out


def _loops_gpu(tl, op, L, left, right, prec, n, mode, kind):
    T = L[3]
    if kind == "local":
        out = torch.empty(n * 16 * T * 2, dtype=torch.float64, device="cuda")
        tl.loop_contract_local(L, left, right, prec, n, tl.LOOP_MODE[mode], out)
        return from_dev(out, (n, 16, T))
    out = torch.empty(n * 4 * 16 * T * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_oneD(op, left, right, prec, n, tl.LOOP_MODE[mode], out)
    return from_dev(out, (n, 4, 16, T))


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 4, 8), (2, 2, 2, 2), (12, 10, 8, 6)])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("prec", [0, 1])
def test_contractions_match_oracle(L, mode, prec):
    tl = require_gpu()
    U = synth.gauge_field(L, seed=4)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=12 if prec else 18)
    n = 3
    A = synth.random_spinor(L, n, seed=5)
    B = synth.random_spinor(L, n, seed=6)
    fa, fb = pack(tl, L, A, prec), pack(tl, L, B, prec)
    A_in, B_in = unpack(tl, L, fa, prec, n), unpack(tl, L, fb, prec, n)
    tol = 1e-12 if prec == 0 else 1e-5
    got = _loops_gpu(tl, op, L, fa, fb, prec, n, mode, "local")
    assert rel_l2(got, oloops.local_loops(A_in, B_in, mode)) < tol
    U_used = U if prec == 0 else None
    if prec == 0:
        got = _loops_gpu(tl, op, L, fa, fb, prec, n, mode, "oneD")
        assert rel_l2(got, oloops.oneD_loops(U_used, A_in, B_in, mode)) < tol
    op.close()


def test_oneD_fp32_matches_oracle():
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=14)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=18)
    A = synth.random_spinor(L, 2, seed=15)
    B = synth.random_spinor(L, 2, seed=16)
    fa, fb = pack(tl, L, A, 1), pack(tl, L, B, 1)
    got = _loops_gpu(tl, op, L, fa, fb, 1, 2, "vv", "oneD")
    ref = oloops.oneD_loops(U, unpack(tl, L, fa, 1, 2), unpack(tl, L, fb, 1, 2), "vv")
    assert rel_l2(got, ref) < 1e-5
    op.close()


@pytest.mark.parametrize("n_hp,n_lp", [(4, 9), (0, 5), (1, 3), (3, 1)])
def test_tsm_combine_matches_oracle(n_hp, n_lp):
    tl = require_gpu()
    rng = np.random.default_rng(n_hp * 10 + n_lp)
    shape = (16, 8)
    mk = lambda n: rng.standard_normal((n,) + shape) + 1j * rng.standard_normal((n,) + shape)
    hp, lphp, lp = mk(n_hp), mk(n_hp), mk(n_lp)
    scale = -2j * 0.0032
    ref_mean, ref_er, ref_ei = otsm.tsm_combine(hp, lphp, lp, scale=scale)
    length = int(np.prod(shape))
    mean = torch.empty(2 * length, dtype=torch.float64, device="cuda")
    err = torch.empty(2 * length, dtype=torch.float64, device="cuda")
    dhp = to_dev(hp) if n_hp else None
    dlphp = to_dev(lphp) if n_hp else None
    tl.tsm_combine(dhp, dlphp, n_hp, to_dev(lp), n_lp, length, scale, mean, err)
    gm = from_dev(mean, shape)
    ge = err.cpu().numpy().reshape(shape + (2,))
    np.testing.assert_allclose(gm, ref_mean, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(ge[..., 0], ref_er, rtol=1e-12, atol=1e-15, equal_nan=True)
    np.testing.assert_allclose(ge[..., 1], ref_ei, rtol=1e-12, atol=1e-15, equal_nan=True)


def test_pipeline_4x4_plain_fp64():
    """4^4, kappa = 0.16, mu = 0.01, antiperiodic t, 16 Z4 sources, plain FP64 CG
    to |r| = 1e-10, local 16-Gamma and one-derivative loops in all three
    estimators: GPU vs oracle within 1e-8."""
    tl = require_gpu()
    L = (4, 4, 4, 4)
    kappa, mu = 0.16, 0.01
    U = synth.gauge_field(L, seed=1234)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=18)
    n, seed = 16, 20140126
    eta_d = tl.empty_field(L, 0, n)
    tl.z4_noise(L, eta_d, 0, seed, 0, n)
    s_d = tl.empty_field(L, 0, n)
    st, stats = tl.tm_cg_solve(op, s_d, eta_d, n, tl.cg_params(1e-10, 5000, tl.CG_PLAIN, prec=0))
    assert all(s["status"] == 0 for s in stats)
    dw = tl.empty_field(L, 0, n)
    tl.tm_dslash(op, dw, s_d, n, mu_zero=True, prec=0)
    gdw = tl.empty_field(L, 0, n)
    tl.tm_gamma5(L, gdw, dw, 0, n)
    pairs = {"std": (eta_d, s_d), "vv": (s_d, s_d), "gen": (s_d, gdw)}
    eta = oracle_z4(L, seed, 0, n)
    sols = np.stack([ocg.cg_normal(U, eta[j], kappa, mu, tol=1e-10)[0] for j in range(n)])
    ref_pairs = {"std": (eta, sols), "vv": (sols, sols), "gen": (sols, _g5(apply_DW(U, sols, kappa)))}
    for mode in MODES:
        lf, rf = pairs[mode]
        lo, ro = ref_pairs[mode]
        got = _loops_gpu(tl, op, L, lf, rf, 0, n, mode, "local")
        assert rel_l2(got, oloops.local_loops(lo, ro, mode)) < 1e-8
        got = _loops_gpu(tl, op, L, lf, rf, 0, n, mode, "oneD")
        assert rel_l2(got, oloops.oneD_loops(U, lo, ro, mode)) < 1e-8
    op.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("prec,recon", [(2, 18), (2, 12), (3, 18)])
def test_contractions_16bit_match_oracle(mode, prec, recon):
    """FP16/BF16 fields (FP32 arithmetic; with 18-real links the link
    products multiply the 16-bit values in memory with the exact mixed FMA).
    FP16 with 18-real links: the oracle takes the links rounded to FP16, so
    only FP32 rounding separates the results (1e-5).  Otherwise the link
    rounding (2^-11, 2^-8) bounds the difference."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=30)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=recon)
    n = 2
    fa = pack(tl, L, synth.random_spinor(L, n, seed=31), prec)
    fb = pack(tl, L, synth.random_spinor(L, n, seed=32), prec)
    A, B = unpack(tl, L, fa, prec, n), unpack(tl, L, fb, prec, n)
    got = _loops_gpu(tl, op, L, fa, fb, prec, n, mode, "local")
    assert rel_l2(got, oloops.local_loops(A, B, mode)) < 1e-5
    got = _loops_gpu(tl, op, L, fa, fb, prec, n, mode, "oneD")
    if prec == 2 and recon == 18:
        U16 = U.real.astype(np.float16).astype(np.float64) + 1j * U.imag.astype(np.float16).astype(np.float64)
        assert rel_l2(got, oloops.oneD_loops(U16, A, B, mode)) < 1e-5
    else:
        assert rel_l2(got, oloops.oneD_loops(U, A, B, mode)) < (5e-3 if prec == 2 else 3e-2)
    op.close()

"""The benchmarked configuration end to end against the oracle, on a lattice
the oracle solves in seconds.

bench.py times the TSM pipeline with: 18-real FP16 links (recon 0), FP16 LP
solves truncated at 1e-2 on the even/odd Schur complement (the plain 16-bit
solver runs on the system-interleaved layout and the tensor-core Dslash),
mixed-precision HP solves, float-float HP loops, FP16 LP loops, batches of 16.
Here the same settings run on 8^4 (kappa 0.161, mu 0.003 as in the bench) with
13 sources in batches of 4 (a ragged last batch of 1), the HP solves to 1e-12
so that the HP loops can be held to the stated 1e-8:

  * HP loops of all four kinds vs the oracle (FP64 CG to 1e-13, oracle
    D_W and contractions): relative L2 < 1e-8 (Sec. 2.2, Eqs. 5-6);
  * every LP solution (re-solved in one batch of 13, bit-identical to the
    pipeline's batches of 4): the oracle's normal-equation residual of the
    odd-site Schur system, |Mh^dag (eta_h - Mh x_o)| / |Mh^dag eta_h|, is at
    most 2e-2 (the 1e-2 truncation of Sec. 2.1 plus FP16 rounding), and the
    full solution solves M x = eta on the even sites to FP16 accuracy;
  * the LP loops the pipeline stored equal the oracle's contractions of those
    LP solutions: to FP32 arithmetic (1e-5) for the one-end local loops, to
    the FP16 rounding of g5 D_W x and of the links (4e-3) for the others;
  * the combined estimate equals the oracle's Eq. 4 of the pipeline's own
    per-source loops (rtol 1e-12).
"""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from oracle import loops as oloops
from oracle import tsm as otsm
from oracle.gamma import GAMMA5
from oracle.operator import apply_DW, apply_M
from oracle.philox import z4_noise as oz4
from paper_1401_6749_gb300 import synth

from .gpu_util import pack, rel_l2, require_gpu, to_dev, unpack

pytestmark = pytest.mark.gpu

L = (8, 8, 8, 8)
T = L[3]
KAPPA, MU = 0.161, 0.003
NU = 2 * KAPPA * MU
N_HP, N_LP, BATCH, SEED = 3, 10, 4, 20140126


def _cplx(t):
    return t.cpu().numpy().view(np.complex128).reshape(t.shape[0], -1, T)


def _odd_mask():
    t, z, y, x = np.meshgrid(*(np.arange(e) for e in L[::-1]), indexing="ij")
    return ((x + y + z + t) % 2 == 1)[..., None, None]


def _twist(v, nu, inverse=False):
    """A v = v + i nu g5 v, or A^-1 v = (v - i nu g5 v) / (1 + nu^2), site by site."""
    g5v = np.einsum("st,...tc->...sc", GAMMA5, v)
    return (v - 1j * nu * g5v) / (1 + nu * nu) if inverse else v + 1j * nu * g5v


def _schur(U, v_o, dagger, odd):
    """Mh v_o (or Mh^dag v_o) on the odd sites from the oracle's full operator:
    with w = M v_o, u = A^-1 (w on the even sites), Mh v_o = w_o - (M u)_o."""
    nu = -NU if dagger else NU
    w = apply_M(U, v_o, KAPPA, MU, dagger=dagger)
    u = np.where(odd, 0, _twist(w, nu, inverse=True))
    return np.where(odd, w - apply_M(U, u, KAPPA, MU, dagger=dagger), 0)


def test_bench_configuration_against_oracle():
    tl = require_gpu()
    from paper_1401_6749_gb300.tsm_pipeline import TsmPipeline
    U = synth.gauge_field(L, 1237)
    op = tl.Operator(L, KAPPA, MU, to_dev(U), recon=0)
    p = TsmPipeline(op, N_HP, N_LP, batch=BATCH, lp_prec=tl.F16, hp_inner=tl.F32, tol_lp=1e-2,
                    tol_hp=1e-12, seed=SEED, schur=True, delta=1e-6, hp_loop_prec=tl.FF)
    res = p.run()
    torch.cuda.synchronize()
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-2 for s in p.stats_lp)
    assert all(s["status"] == 0 and s["true_res"] <= 1e-12 for s in p.stats_hp)
    n_all = N_HP + N_LP
    eta = oz4(L, SEED, 0, n_all)

    # HP loops (float-float) vs the oracle
    sol = np.stack([ocg.cg_normal(U, eta[j], KAPPA, MU, tol=1e-13)[0] for j in range(N_HP)])
    g5dw = apply_DW(U, sol, KAPPA)
    g5dw[..., 2:, :] *= -1
    ref_hp = {"local_vv": oloops.local_loops(sol, sol, "vv"), "local_gen": oloops.local_loops(sol, g5dw, "gen"),
              "oneD_vv": oloops.oneD_loops(U, sol, sol, "vv").reshape(N_HP, 64, T),
              "oneD_gen": oloops.oneD_loops(U, sol, g5dw, "gen").reshape(N_HP, 64, T)}
    for k in p.kinds:
        assert rel_l2(_cplx(p.hp_loops[k]), ref_hp[k]) < 1e-8, k

    # LP solutions: one batch of all sources gives the pipeline's bits
    prm = tl.cg_params(1e-2, p.max_iter, tl.CG_PLAIN, prec=tl.F16, check_every=2, schur=True)
    x = tl.empty_field(L, tl.F16, n_all)
    tl.tm_cg_solve(op, x, pack(tl, L, eta, tl.F16), n_all, prm)
    xs = unpack(tl, L, x, tl.F16, n_all)
    odd = _odd_mask()
    for j in range(n_all):
        e_o = np.where(odd, eta[j], 0)
        e_e = np.where(odd, 0, eta[j])
        eta_h = e_o - np.where(odd, apply_M(U, _twist(e_e, NU, inverse=True), KAPPA, MU), 0)
        b = _schur(U, eta_h, True, odd)
        x_o = np.where(odd, xs[j], 0)
        r = b - _schur(U, _schur(U, x_o, False, odd), True, odd)
        assert np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel()) <= 2e-2
        # the even half solves the even rows of M x = eta: x_e = A^-1 (eta_e -
        # M_eo x_o) up to its FP16 rounding (|A| ~ 1, so |residual| ~ 2^-11 |x_e|)
        re = np.where(odd, 0, eta[j] - apply_M(U, xs[j], KAPPA, MU))
        assert np.linalg.norm(re.ravel()) / np.linalg.norm(np.where(odd, 0, xs[j]).ravel()) < 5e-3

    # LP loops vs the oracle's contractions of the LP solutions
    g5dw_lp = apply_DW(U, xs, KAPPA)
    g5dw_lp[..., 2:, :] *= -1
    ref_lp = {"local_vv": oloops.local_loops(xs, xs, "vv"), "local_gen": oloops.local_loops(xs, g5dw_lp, "gen"),
              "oneD_vv": oloops.oneD_loops(U, xs, xs, "vv").reshape(n_all, 64, T),
              "oneD_gen": oloops.oneD_loops(U, xs, g5dw_lp, "gen").reshape(n_all, 64, T)}
    tol = {"local_vv": 1e-5, "local_gen": 4e-3, "oneD_vv": 4e-3, "oneD_gen": 4e-3}
    for k in p.kinds:
        assert rel_l2(_cplx(p.lp_loops[k]), ref_lp[k]) < tol[k], k

    # Eq. 4 on the pipeline's own per-source loops
    for k in p.kinds:
        lp = _cplx(p.lp_loops[k])
        scale = -2j * NU if k.endswith("vv") else 2.0
        m, _, _ = otsm.tsm_combine(_cplx(p.hp_loops[k]), lp[:N_HP], lp[N_HP:], scale=scale)
        got = res[k][0].cpu().numpy().view(np.complex128).reshape(m.shape)
        np.testing.assert_allclose(got, m, rtol=1e-12, atol=1e-13 * np.abs(m).max())
    op.close()

"""The TSM pipeline in the paper's three sectors (Sec. 4: light, strange and
charm loops with the same method), with twisted masses standing in for them:
the bench's light mass 0.003 and the heavier 0.04 and 0.5.  In each sector, on
a lattice the oracle solves at once, with the bench's settings (recon 0, FP16
LP solves on the interleaved layout, Schur, float-float HP loops):
  * every solve converges (LP to 1e-2, HP to 1e-12);
  * the HP loops of all four kinds agree with the oracle's (FP64 CG to 1e-13,
    oracle D_W and contractions) within 1e-8;
  * the combined estimate equals the oracle's Eq. 4 of the pipeline's own
    per-source loops;
  * heavier quarks converge in fewer iterations (the reason the TSM gains
    less there, Table tab:TSM)."""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from oracle import loops as oloops
from oracle import tsm as otsm
from oracle.operator import apply_DW
from oracle.philox import z4_noise as oz4
from paper_1401_6749_gb300 import synth

from .gpu_util import rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

L = (4, 4, 4, 8)
T = L[3]
KAPPA = 0.161
SEED = 4242
ITERS = {}


def _cplx(t):
    return t.cpu().numpy().view(np.complex128).reshape(t.shape[0], -1, T)


@pytest.mark.parametrize("sector,mu", [("light", 0.003), ("strange", 0.04), ("charm", 0.5)])
def test_sector_pipeline_against_oracle(sector, mu):
    tl = require_gpu()
    from paper_1401_6749_gb300.tsm_pipeline import TsmPipeline
    U = synth.gauge_field(L, 1237)
    op = tl.Operator(L, KAPPA, mu, to_dev(U), recon=0)
    n_hp, n_lp = 2, 5
    p = TsmPipeline(op, n_hp, n_lp, batch=4, lp_prec=tl.F16, hp_inner=tl.F32, tol_lp=1e-2, tol_hp=1e-12,
                    seed=SEED, schur=True, delta=1e-6, hp_loop_prec=tl.FF)
    res = p.run()
    torch.cuda.synchronize()
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-2 for s in p.stats_lp)
    assert all(s["status"] == 0 and s["true_res"] <= 1e-12 for s in p.stats_hp)
    ITERS[sector] = np.mean([s["iters"] for s in p.stats_hp])
    eta = oz4(L, SEED, 0, n_hp)
    sol = np.stack([ocg.cg_normal(U, eta[j], KAPPA, mu, tol=1e-13)[0] for j in range(n_hp)])
    g5dw = apply_DW(U, sol, KAPPA)
    g5dw[..., 2:, :] *= -1
    ref = {"local_vv": oloops.local_loops(sol, sol, "vv"), "local_gen": oloops.local_loops(sol, g5dw, "gen"),
           "oneD_vv": oloops.oneD_loops(U, sol, sol, "vv").reshape(n_hp, 64, T),
           "oneD_gen": oloops.oneD_loops(U, sol, g5dw, "gen").reshape(n_hp, 64, T)}
    nu = 2 * KAPPA * mu
    for k in p.kinds:
        assert rel_l2(_cplx(p.hp_loops[k]), ref[k]) < 1e-8, k
        lp = _cplx(p.lp_loops[k])
        scale = -2j * nu if k.endswith("vv") else 2.0
        m, _, _ = otsm.tsm_combine(_cplx(p.hp_loops[k]), lp[:n_hp], lp[n_hp:], scale=scale)
        got = res[k][0].cpu().numpy().view(np.complex128).reshape(m.shape)
        np.testing.assert_allclose(got, m, rtol=1e-12, atol=1e-13 * np.abs(m).max())
    op.close()
    if len(ITERS) == 3:
        assert ITERS["charm"] < ITERS["strange"] <= ITERS["light"]

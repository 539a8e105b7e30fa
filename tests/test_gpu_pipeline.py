"""The TSM pipeline end to end on a small lattice: Z4 noise, LP (FP16, |r| <= 1e-2)
and HP (mixed, 1e-10) even/odd solves, local and one-derivative loops in both
one-end estimators, TSM combination.

Checked: (1) running the HP solves on a second stream concurrently with the LP
batches, or before them instead of after, changes nothing (bit-identical
per-source loops); (2) the HP loops
agree with the oracle's (FP64 CG to 1e-12 and oracle contractions) within
1e-8; (3) the combined estimate equals the oracle's TSM combination of the
pipeline's own per-source loops; (4) every LP solve meets its truncation."""
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


def _cplx(t, T):
    return t.cpu().numpy().view(np.complex128).reshape(t.shape[0], -1, T)


def test_pipeline_overlap_and_parity():
    tl = require_gpu()
    from paper_1401_6749_gb300.tsm_pipeline import TsmPipeline
    L = (4, 4, 4, 6)
    T = L[3]
    kappa, mu = 0.16, 0.01
    U = synth.gauge_field(L, 1234)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=12)
    kw = dict(batch=4, lp_prec=tl.F16, hp_inner=tl.F32, tol_lp=1e-2, tol_hp=1e-10, seed=77, delta=1e-3)
    runs = []
    for overlap, hp_first in ((False, False), (True, False), (False, True)):
        p = TsmPipeline(op, 3, 6, overlap=overlap, hp_first=hp_first, **kw)
        res = p.run()
        torch.cuda.synchronize()
        runs.append((p, {k: (m.clone(), e.clone()) for k, (m, e) in res.items()}))
    (p0, r0) = runs[0]
    for p1, r1 in runs[1:]:
        for k in p0.kinds:
            np.testing.assert_array_equal(p0.lp_loops[k].cpu().numpy(), p1.lp_loops[k].cpu().numpy())
            np.testing.assert_array_equal(p0.hp_loops[k].cpu().numpy(), p1.hp_loops[k].cpu().numpy())
            np.testing.assert_array_equal(r0[k][0].cpu().numpy(), r1[k][0].cpu().numpy())
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-2 for s in p0.stats_lp)
    assert all(s["status"] == 0 for s in p0.stats_hp)
    # HP loops vs the oracle
    eta = oz4(L, 77, 0, 3)
    sol = np.stack([ocg.cg_normal(U, eta[j], kappa, mu, tol=1e-12)[0] for j in range(3)])
    g5dw = apply_DW(U, sol, kappa)
    g5dw[..., 2:, :] *= -1
    ref = {"local_vv": oloops.local_loops(sol, sol, "vv"),
           "local_gen": oloops.local_loops(sol, g5dw, "gen"),
           "oneD_vv": oloops.oneD_loops(U, sol, sol, "vv").reshape(3, 64, T),
           "oneD_gen": oloops.oneD_loops(U, sol, g5dw, "gen").reshape(3, 64, T)}
    nu = 2 * kappa * mu
    for k in p0.kinds:
        assert rel_l2(_cplx(p0.hp_loops[k], T), ref[k]) < 1e-8
        lp = _cplx(p0.lp_loops[k], T)
        scale = -2j * nu if k.endswith("vv") else 2.0
        m, ere, eim = otsm.tsm_combine(_cplx(p0.hp_loops[k], T), lp[:3], lp[3:], scale=scale)
        got = r0[k][0].cpu().numpy().view(np.complex128).reshape(m.shape)
        np.testing.assert_allclose(got, m, rtol=1e-12, atol=1e-13 * np.abs(m).max())
    for p, _ in runs:
        if p.overlap:
            p.op_hp.close()
    op.close()

"""Mixed-precision CG with float-float true residuals (ru_prec = FF).

The reliable updates (and the final residual) of TM_CG_MIXED compute
r = b - M^dag M x from float-float copies of x and b (about 48-bit
significands) instead of FP64; x still accumulates in FP64.  The residual is
then exact to ~1e-13 relative, far below the 1e-9 .. 1e-12 tolerances, so the
solve must reach the same tolerance in the same number of iterations (within
one), and its solution must solve M x = eta to the tolerance by the oracle's
FP64 residual.
"""
import numpy as np
import pytest
import torch

from oracle.operator import apply_M
from oracle.philox import z4_noise as oz4
from paper_1401_6749_gb300 import synth

from .gpu_util import pack, require_gpu, to_dev, unpack

pytestmark = pytest.mark.gpu

L = (8, 8, 8, 8)
KAPPA, MU = 0.161, 0.003


@pytest.mark.parametrize("schur", [True, False])
def test_ff_residuals_converge_like_fp64(schur):
    tl = require_gpu()
    U = synth.gauge_field(L, 1237)
    op = tl.Operator(L, KAPPA, MU, to_dev(U), recon=0)
    n = 3
    eta_np = oz4(L, 20140126, 0, n)
    eta = pack(tl, L, eta_np, tl.F64)
    out = {}
    for ru in (tl.F64, tl.FF):
        x = tl.empty_field(L, tl.F64, n)
        prm = tl.cg_params(1e-11, 4000, tl.CG_MIXED, inner_prec=tl.F32, delta=3e-5, check_every=4,
                           schur=schur, ru_prec=ru)
        st, stats = tl.tm_cg_solve(op, x, eta, n, prm)
        assert st == 0 and all(s["status"] == 0 and s["true_res"] <= 1e-11 for s in stats)
        out[ru] = (unpack(tl, L, x, tl.F64, n), stats)
    xs64, s64 = out[tl.F64]
    xsff, sff = out[tl.FF]
    for a, b in zip(s64, sff):
        assert abs(a["iters"] - b["iters"]) <= 1
    for j in range(n):
        r = eta_np[j] - apply_M(U, xsff[j], KAPPA, MU)
        assert np.linalg.norm(r.ravel()) / np.linalg.norm(eta_np[j].ravel()) < 1e-9
        d = np.linalg.norm((xsff[j] - xs64[j]).ravel()) / np.linalg.norm(xs64[j].ravel())
        assert d < 1e-8
    op.close()


def test_ru_prec_argument():
    tl = require_gpu()
    U = synth.gauge_field(L, 5)
    op = tl.Operator(L, KAPPA, MU, to_dev(U), recon=0)
    eta = tl.empty_field(L, tl.F64, 1)
    tl.z4_noise(L, eta, tl.F64, 1, 0, 1)
    x = tl.empty_field(L, tl.F64, 1)
    with pytest.raises(tl.TmError) as e:
        tl.tm_cg_solve(op, x, eta, 1, tl.cg_params(1e-8, 100, tl.CG_MIXED, inner_prec=tl.F32, ru_prec=tl.F32))
    assert e.value.status == 1
    op.close()

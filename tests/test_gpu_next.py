"""GPU parity of the widened rows: hopping parameter expansion (Sec. 2.4), time
dilution with coherent sources (Sec. 2.3), momentum-projected local loops."""
import numpy as np
import pytest
import torch

from oracle import hpe as ohpe
from oracle import loops as oloops
from oracle.philox import z4_noise_diluted as oz4d
from paper_1401_6749_gb300 import synth

from .gpu_util import from_dev, pack, rel_l2, require_gpu, site_rel_err, to_dev, unpack

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("t0,dt", [(0, 1), (1, 3), (5, 6), (2, 4)])
@pytest.mark.parametrize("prec", [0, 2])
def test_diluted_noise_bit_exact(t0, dt, prec):
    tl = require_gpu()
    L = (4, 2, 4, 12)
    f = tl.empty_field(L, prec, 2)
    tl.z4_noise_diluted(L, f, prec, 99, 7, 2, t0, dt)
    np.testing.assert_array_equal(unpack(tl, L, f, prec, 2), oz4d(L, 99, 7, 2, t0, dt))


@pytest.mark.parametrize("order", [1, 2, 4])
@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 5e-6)])
def test_hpe_apply_matches_oracle(order, prec, tol):
    tl = require_gpu()
    L = (6, 4, 4, 8)
    kappa, mu = 0.16, 0.02
    U = synth.gauge_field(L, 17)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=18)
    psi = synth.random_spinor(L, 3, 5)
    fin = pack(tl, L, psi, prec)
    fout = tl.empty_field(L, prec, 3)
    tl.tm_hpe_apply(op, fout, fin, 3, order, prec)
    ref = ohpe.apply_BH_power(U, unpack(tl, L, fin, prec, 3), kappa, mu, order)
    assert site_rel_err(unpack(tl, L, fout, prec, 3), ref) < tol * order
    op.close()


def test_hpe_exact_terms_match_dense_oracle():
    tl = require_gpu()
    L = (4, 4, 4, 4)
    kappa, mu = 0.16, 0.04
    got = tl.tm_hpe_exact(L, kappa, mu)
    ref = ohpe.exact_terms_dense(synth.gauge_field(L, 1, eps=0.8), kappa, mu)
    np.testing.assert_allclose(got, ref, atol=1e-10)
    with pytest.raises(tl.TmError):
        tl.tm_hpe_exact((4, 2, 4, 4), kappa, mu)      # extent 2: gauge dependent


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_momentum_projected_loops_match_oracle(prec, tol):
    tl = require_gpu()
    L = (8, 6, 4, 6)
    A = synth.random_spinor(L, 2, 1)
    B = synth.random_spinor(L, 2, 2)
    fa, fb = pack(tl, L, A, prec), pack(tl, L, B, prec)
    moms = [(0, 0, 0), (1, 0, 0), (0, -1, 2), (3, 2, 1), (9, 6, 5)]   # 9 = 1 (mod 8), 6 = 0, 5 = 1
    T = L[3]
    out = torch.empty(2 * len(moms) * 16 * T * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_local_mom(L, fa, fb, prec, 2, tl.LOOP_GEN, moms, out)
    got = from_dev(out, (2, len(moms), 16, T))
    ref = oloops.local_loops_mom(unpack(tl, L, fa, prec, 2), unpack(tl, L, fb, prec, 2), "gen", moms)
    assert rel_l2(got, ref) < tol

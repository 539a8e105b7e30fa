"""Float-float (FF) storage and arithmetic: each real a pair of FP32 values
with about 48 significant bits.

Bars: a double survives FF storage to 2^-47 relative; the FF operator and the
FF contractions match the FP64 oracle to 1e-12 and 1e-11 (the arithmetic
errs by a few 2^-47 of the operands per operation, and a Dslash output sums
~100 terms); HP loops computed in FF agree with the FP64 ones far below the
1e-8 stated for loops from HP solves.
"""
import numpy as np
import pytest
import torch

from oracle import loops as oloops
from oracle.operator import apply_DW, apply_M
from oracle.philox import z4_noise as oracle_z4
from paper_1401_6749_gb300 import synth

from .gpu_util import from_dev, pack, rel_l2, require_gpu, site_rel_err, to_dev, unpack

pytestmark = pytest.mark.gpu


def test_ff_storage_round_trip():
    tl = require_gpu()
    L = (6, 4, 4, 8)
    psi = synth.random_spinor(L, 2, seed=3) * 1e3      # values far from 1 as well
    f = pack(tl, L, psi, tl.FF)
    got = unpack(tl, L, f, tl.FF, 2)
    assert np.max(np.abs(got - psi) / np.maximum(np.abs(psi), 1e-300)) < 2.0 ** -46
    # F64 -> FF -> F64 through tm_spinor_convert
    d = pack(tl, L, psi, tl.F64)
    back = tl.empty_field(L, tl.F64, 2)
    tl.tm_spinor_convert(L, f, tl.FF, d, tl.F64, 2)
    tl.tm_spinor_convert(L, back, tl.F64, f, tl.FF, 2)
    torch.cuda.synchronize()
    assert rel_l2(unpack(tl, L, back, tl.F64, 2), psi) < 2.0 ** -47


def test_ff_noise_exact_and_gamma5():
    tl = require_gpu()
    L = (4, 4, 2, 6)
    f = tl.empty_field(L, tl.FF, 3)
    tl.z4_noise(L, f, tl.FF, 17, 4, 3)
    eta = oracle_z4(L, 17, 4, 3)
    np.testing.assert_array_equal(unpack(tl, L, f, tl.FF, 3), eta)
    g = tl.empty_field(L, tl.FF, 3)
    tl.tm_gamma5(L, g, f, tl.FF, 3)
    ref = eta.copy()
    ref[..., 2:, :] *= -1
    np.testing.assert_array_equal(unpack(tl, L, g, tl.FF, 3), ref)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 4, 8), (8, 6, 4, 6)])
@pytest.mark.parametrize("dagger,mu_zero", [(False, False), (True, False), (False, True)])
def test_ff_dslash_matches_oracle(L, dagger, mu_zero):
    tl = require_gpu()
    kappa, mu = 0.16, 0.02
    U = synth.gauge_field(L, seed=8)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=0)
    psi = synth.random_spinor(L, 2, seed=9)
    fin = pack(tl, L, psi, tl.FF)
    fout = tl.empty_field(L, tl.FF, 2)
    tl.tm_dslash(op, fout, fin, 2, dagger=dagger, mu_zero=mu_zero, prec=tl.FF)
    psi_in = unpack(tl, L, fin, tl.FF, 2)
    ref = apply_M(U, psi_in, kappa, 0.0 if mu_zero else mu, dagger=dagger)
    assert site_rel_err(unpack(tl, L, fout, tl.FF, 2), ref) < 1e-12
    op.close()


@pytest.mark.parametrize("mode", ["std", "vv", "gen"])
def test_ff_contractions_match_oracle(mode):
    tl = require_gpu()
    L = (8, 6, 4, 6)
    U = synth.gauge_field(L, seed=10)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=0)
    n = 2
    fa = pack(tl, L, synth.random_spinor(L, n, seed=11), tl.FF)
    fb = pack(tl, L, synth.random_spinor(L, n, seed=12), tl.FF)
    A, B = unpack(tl, L, fa, tl.FF, n), unpack(tl, L, fb, tl.FF, n)
    T = L[3]
    out = torch.empty(n * 16 * T * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_local(L, fa, fb, tl.FF, n, tl.LOOP_MODE[mode], out)
    assert rel_l2(from_dev(out, (n, 16, T)), oloops.local_loops(A, B, mode)) < 1e-11
    out = torch.empty(n * 64 * T * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_oneD(op, fa, fb, tl.FF, n, tl.LOOP_MODE[mode], out)
    assert rel_l2(from_dev(out, (n, 4, 16, T)), oloops.oneD_loops(U, A, B, mode)) < 1e-11
    op.close()


def test_cg_rejects_ff():
    tl = require_gpu()
    L = (4, 4, 4, 4)
    op = tl.Operator(L, 0.16, 0.01, to_dev(synth.gauge_field(L, 1)))
    f = [tl.empty_field(L, tl.FF, 1) for _ in range(2)]
    with pytest.raises(tl.TmError):
        tl.tm_cg_solve(op, f[1], f[0], 1, tl.cg_params(1e-8, 100, tl.CG_PLAIN, prec=tl.FF))
    op.close()


def test_pipeline_hp_loops_ff_match_f64():
    """The TSM pipeline with its HP loops (D_W s and both contractions) in FF
    gives the HP loops of the FP64 path to 1e-11, and the same LP loops."""
    tl = require_gpu()
    from paper_1401_6749_gb300.tsm_pipeline import TsmPipeline
    L = (8, 8, 8, 8)
    U = synth.gauge_field(L, seed=1237)
    op = tl.Operator(L, 0.161, 0.003, to_dev(U), recon=0)
    kinds = ("local_vv", "local_gen", "oneD_vv", "oneD_gen", "local_std")
    res = {}
    for lp in (tl.F64, tl.FF):
        pipe = TsmPipeline(op, 3, 5, batch=4, tol_hp=1e-10, delta=1e-5, kinds=kinds, hp_loop_prec=lp)
        pipe.run()
        torch.cuda.synchronize()
        res[lp] = ({k: v.cpu().numpy() for k, v in pipe.hp_loops.items()},
                   {k: v.cpu().numpy() for k, v in pipe.lp_loops.items()})
    for k in kinds:
        a, b = res[tl.F64][0][k], res[tl.FF][0][k]
        assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-11, k
        np.testing.assert_array_equal(res[tl.F64][1][k], res[tl.FF][1][k])
    op.close()

"""Failure handling and out-of-bounds guards, without faulting the GPU.

  * A NaN written into one source on the host: the solver reports TM_ERR_NAN
    for that system only, the other systems of the batch converge and their
    solutions are bit-identical to a solve without the poisoned system (the
    16-bit interleaved solver, the CUDA-core 16-bit solver, and the mixed
    solver).
  * Guard bands: every output buffer sits between two 4 KiB bands filled with
    a byte pattern; after kernels whose shapes leave ragged edges (numbers of
    systems that are not multiples of the systems per thread or of the 16 of
    an interleaved block, half volumes that are not multiples of the block
    sizes, including every launch shape the autotuner tries) the bands are
    intact.  This stands in for a memory checker.
"""
import numpy as np
import pytest
import torch

from oracle.philox import z4_noise as oz4
from paper_1401_6749_gb300 import synth

from .gpu_util import pack, require_gpu, to_dev

pytestmark = pytest.mark.gpu

GUARD = 4096
PATTERN = 0xA5


class Guarded:
    """A device buffer of n bytes between two guard bands."""

    def __init__(self, n):
        self.n = int(n)
        self.buf = torch.full((self.n + 2 * GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
        self.view = self.buf[GUARD:GUARD + self.n]

    def as_f64(self):
        return self.view.view(torch.float64)

    def intact(self):
        torch.cuda.synchronize()
        return bool((self.buf[:GUARD] == PATTERN).all()) and bool((self.buf[GUARD + self.n:] == PATTERN).all())


# ---------------------------------------------------------------- NaN sources
@pytest.mark.parametrize("recon,prec,mode", [(0, 2, "plain"), (12, 2, "plain"), (0, 0, "mixed")])
def test_nan_source_fails_alone(recon, prec, mode):
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=9)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=recon)
    eta = oz4(L, 3, 0, 3)
    bad = eta.copy()
    bad[1, 2, 1, 3, 4, 2, 1] = np.nan
    if mode == "plain":
        prm = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=prec, schur=True, check_every=2)
        xp = prec
    else:
        prm = tl.cg_params(1e-10, 2000, tl.CG_MIXED, inner_prec=tl.F32, delta=1e-3, schur=True)
        xp = tl.F64
    x = tl.empty_field(L, xp, 3)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, bad, xp), 3, prm, raise_on_noconv=False)
    assert st == 4                                     # TM_ERR_NAN
    assert stats[1]["status"] == 4
    assert stats[0]["status"] == 0 and stats[2]["status"] == 0
    x2 = tl.empty_field(L, xp, 2)
    st2, _ = tl.tm_cg_solve(op, x2, pack(tl, L, eta[[0, 2]], xp), 2, prm)
    assert st2 == 0
    a = x.view(3, -1)
    b = x2.view(2, -1)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[1])
    op.close()


# ---------------------------------------------------------------- guard bands
LAT = (6, 6, 2, 6)  # half volume 216: not a multiple of 32, 64 or 128


@pytest.mark.parametrize("prec,recon,n", [(2, 0, 3), (2, 0, 5), (1, 12, 5), (3, 12, 3), (0, 18, 3), (4, 18, 2)])
def test_dslash_output_guards(prec, recon, n):
    tl = require_gpu()
    U = synth.gauge_field(LAT, seed=5)
    op = tl.Operator(LAT, 0.16, 0.02, to_dev(U), recon=recon)
    tl.tm_tune_reset()  # the first launch of each kind runs every launch shape
    f = pack(tl, LAT, synth.random_spinor(LAT, n, seed=6), prec)
    out = Guarded(tl.tm_spinor_bytes(LAT, prec, n))
    for dagger, mu_zero in ((False, False), (True, False), (False, True)):
        tl.tm_dslash(op, out.view, f, n, dagger=dagger, mu_zero=mu_zero, prec=prec)
        assert out.intact()
    op.close()


@pytest.mark.parametrize("n", [3, 16, 17])
def test_interleaved_guards(n):
    tl = require_gpu()
    U = synth.gauge_field(LAT, seed=5)
    op = tl.Operator(LAT, 0.16, 0.02, to_dev(U), recon=0)
    f = pack(tl, LAT, synth.random_spinor(LAT, n, seed=7), tl.F16)
    il = Guarded(tl.tm_spinor_bytes_il(LAT, n))
    tl.tm_spinor_to_il(LAT, il.view, f, tl.F16, n)
    assert il.intact()
    out = Guarded(tl.tm_spinor_bytes_il(LAT, n))
    for dagger, mu_zero in ((False, False), (True, False), (False, True)):
        tl.tm_dslash_il(op, out.view, il.view, n, dagger=dagger, mu_zero=mu_zero, prec=tl.F16)
        assert out.intact()
    back = Guarded(tl.tm_spinor_bytes(LAT, tl.F16, n))
    tl.tm_spinor_from_il(LAT, back.view, out.view, tl.F16, n)
    assert back.intact()
    tl.tm_op_check(op)                                 # no staging wait gave up
    op.close()


def test_solver_noise_and_contraction_guards():
    tl = require_gpu()
    U = synth.gauge_field(LAT, seed=5)
    op = tl.Operator(LAT, 0.16, 0.02, to_dev(U), recon=0)
    n, T = 5, LAT[3]
    eta = Guarded(tl.tm_spinor_bytes(LAT, tl.F16, n))
    tl.z4_noise(LAT, eta.view, tl.F16, 11, 0, n)
    assert eta.intact()
    x = Guarded(tl.tm_spinor_bytes(LAT, tl.F16, n))
    for schur in (False, True):
        tl.tm_cg_solve(op, x.view, eta.view, n, tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, schur=schur))
        assert x.intact()
    loc = Guarded(n * 16 * T * 2 * 8)
    tl.loop_contract_local(LAT, x.view, x.view, tl.F16, n, tl.LOOP_VV, loc.as_f64())
    assert loc.intact()
    oned = Guarded(n * 64 * T * 2 * 8)
    tl.loop_contract_oneD(op, x.view, x.view, tl.F16, n, tl.LOOP_VV, oned.as_f64())
    assert oned.intact()
    op.close()


@pytest.mark.parametrize("n", [3, 17])
def test_interleaved_solve_and_contraction_guards(n):
    """z4_noise_il's sources, tm_cg_solve_il's interleaved solution and the
    interleaved contractions' loop arrays, on the ragged lattice (36 sites per
    slice and parity, not a multiple of a warp's stride or a block's sites),
    with a partial second block of 16 systems for n = 17."""
    tl = require_gpu()
    U = synth.gauge_field(LAT, seed=5)
    op = tl.Operator(LAT, 0.16, 0.02, to_dev(U), recon=18)
    T = LAT[3]
    eta = Guarded(tl.tm_spinor_bytes_il(LAT, n))
    tl.z4_noise_il(LAT, eta.view, tl.F16, 11, 0, n)
    assert eta.intact()
    x = Guarded(tl.tm_spinor_bytes_il(LAT, n))
    for schur in (False, True):
        tl.tm_cg_solve_il(op, x.view, eta.view, n, tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, schur=schur))
        assert x.intact() and eta.intact()
    loc = Guarded(n * 16 * T * 2 * 8)
    oned = Guarded(n * 64 * T * 2 * 8)
    for g5 in (False, True):
        tl.loop_contract_local_il(LAT, x.view, x.view, tl.F16, n, tl.LOOP_VV, loc.as_f64(), right_g5=g5)
        assert loc.intact()
        tl.loop_contract_oneD_il(op, x.view, x.view, tl.F16, n, tl.LOOP_VV, oned.as_f64(), right_g5=g5)
        assert oned.intact()
    tl.tm_op_check(op)
    op.close()

"""The tensor-core (warp-level MMA) Dslash of the FP16/BF16 formats with
18-real links (switched on for this module with tm_dslash_mma_enable):
parity with the oracle over two 16-system row groups and a ragged site tile,
every output form of tm_dslash, a CG solve through it, bit-identical results
for a system whatever batch and row it sits in, and the switch itself.

Tolerance: 16 u per site as for every 16-bit Dslash (the link and spinor words
are multiplied exactly, the projection is rounded once to the storage format
as in the CUDA-core kernel, accumulation is in FP32)."""
import numpy as np
import pytest

from oracle.gamma import GAMMA5
from oracle.operator import apply_DW, apply_M
from paper_1401_6749_gb300 import synth

from .gpu_util import UNIT_ROUNDOFF, pack, require_gpu, site_rel_err, to_dev, unpack

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def mma_on():
    tl = require_gpu()
    tl.tm_dslash_mma_enable(True)
    yield
    tl.tm_dslash_mma_enable(False)


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("L,nrhs", [((6, 6, 6, 6), 21), ((4, 4, 4, 8), 16), ((2, 2, 2, 4), 17)])
def test_mma_dslash_matches_oracle(prec, L, nrhs):
    tl = require_gpu()
    kappa, mu = 0.16, 0.03
    U = synth.gauge_field(L, seed=31)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=18)
    fin = pack(tl, L, synth.random_spinor(L, nrhs, seed=32), prec)
    psi = unpack(tl, L, fin, prec, nrhs)
    fout = tl.empty_field(L, prec, nrhs)
    for dagger, mu_zero in ((False, False), (True, False), (False, True)):
        tl.tm_dslash(op, fout, fin, nrhs, dagger=dagger, mu_zero=mu_zero, prec=prec)
        ref = apply_DW(U, psi, kappa) if mu_zero else apply_M(U, psi, kappa, mu, dagger=dagger)
        assert site_rel_err(unpack(tl, L, fout, prec, nrhs), ref) < 16 * UNIT_ROUNDOFF[prec]
    tl.tm_dslash_g5(op, fout, fin, nrhs, mu_zero=True, prec=prec)
    ref = np.einsum("ab,...bc->...ac", GAMMA5, apply_DW(U, psi, kappa))
    assert site_rel_err(unpack(tl, L, fout, prec, nrhs), ref) < 16 * UNIT_ROUNDOFF[prec]
    op.close()


@pytest.mark.parametrize("prec", [2, 3])
def test_mma_row_and_batch_independence(prec):
    """System j of a 21-system batch, the same system alone, and the same
    system at another row of another batch give the same bits."""
    tl = require_gpu()
    L = (6, 4, 4, 6)
    op = tl.Operator(L, 0.155, 0.02, to_dev(synth.gauge_field(L, seed=33)), recon=18)
    psi = synth.random_spinor(L, 21, seed=34)
    fin = pack(tl, L, psi, prec)
    out = tl.empty_field(L, prec, 21)
    tl.tm_dslash(op, out, fin, 21, dagger=True, prec=prec)
    full = unpack(tl, L, out, prec, 21)
    for j, lo in ((0, 0), (9, 0), (9, 3), (20, 12)):
        sub = pack(tl, L, psi[lo:j + 1], prec)
        o = tl.empty_field(L, prec, j + 1 - lo)
        tl.tm_dslash(op, o, sub, j + 1 - lo, dagger=True, prec=prec)
        np.testing.assert_array_equal(unpack(tl, L, o, prec, j + 1 - lo)[-1], full[j])
    op.close()


def test_switch_selects_the_kernel_and_both_match_oracle():
    """Off: the CUDA-core kernel; on: the tensor cores.  Both within the 16-bit
    tolerance of the oracle, and different bits (another summation order)."""
    tl = require_gpu()
    L = (4, 4, 4, 6)
    U = synth.gauge_field(L, seed=35)
    op = tl.Operator(L, 0.16, 0.02, to_dev(U), recon=18)
    fin = pack(tl, L, synth.random_spinor(L, 16, seed=36), 2)
    psi = unpack(tl, L, fin, 2, 16)
    ref = apply_M(U, psi, 0.16, 0.02)
    got = {}
    for on in (False, True):
        tl.tm_dslash_mma_enable(on)
        out = tl.empty_field(L, 2, 16)
        tl.tm_dslash(op, out, fin, 16, prec=2)
        got[on] = unpack(tl, L, out, 2, 16)
        assert site_rel_err(got[on], ref) < 16 * UNIT_ROUNDOFF[2]
    assert not np.array_equal(got[False], got[True])
    op.close()


def test_mma_cg_solve_matches_cuda_core_solve():
    """An even/odd FP16 CG solve (every Schur-complement form and the CG-update
    epilogue) through the tensor-core kernel converges like the CUDA-core one:
    the oracle's residual |eta - M x| / |eta| of its solution is as small."""
    tl = require_gpu()
    L = (8, 8, 8, 8)
    U = synth.gauge_field(L, seed=37)
    kappa, mu = 0.155, 0.01
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=18)
    n = 5
    eta = tl.empty_field(L, tl.F16, n)
    tl.z4_noise(L, eta, tl.F16, 11, 0, n)
    e = unpack(tl, L, eta, tl.F16, n)
    res = {}
    for on in (False, True):
        tl.tm_dslash_mma_enable(on)
        x = tl.empty_field(L, tl.F16, n)
        _, st = tl.tm_cg_solve(op, x, eta, n, tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, schur=True,
                                                           check_every=2))
        assert all(s["status"] == 0 and s["rel_res"] <= 1e-2 for s in st)
        xs = unpack(tl, L, x, tl.F16, n)
        res[on] = [np.linalg.norm((e[r] - apply_M(U, xs[r:r + 1], kappa, mu)[0]).ravel()) / np.linalg.norm(e[r].ravel())
                   for r in range(n)]
    print("oracle residuals, CUDA cores:", np.round(res[False], 5), "tensor cores:", np.round(res[True], 5))
    for a, b in zip(res[False], res[True]):
        assert b < 1.5 * a + 1e-3
    op.close()

"""Parity of the CUDA Dslash, Z4 noise and layout kernels with the FP64 oracle.

Tolerances (per-site relative error, max over sites of
|Delta(x)| / max(|ref(x)|, rms_x |ref|)):
  F64: 1e-13.  F32: 1e-6 (the stated bar for the FP32 Dslash).
  F16 / BF16: 16 u, with u the unit roundoff (2^-11, 2^-8): inputs, links and
  the output are each rounded once to the storage format (3 u) and the sum of
  nine terms of size up to ~2 kappa |psi| with kappa ~ 0.16 adds a few u more.
"""
import numpy as np
import pytest

from oracle.operator import apply_DW, apply_M
from oracle.philox import z4_noise as oracle_z4
from paper_1401_6749_gb300 import synth

from .gpu_util import UNIT_ROUNDOFF, pack, require_gpu, site_rel_err, to_dev, unpack

pytestmark = pytest.mark.gpu

LATTICES = [(4, 4, 4, 4), (6, 4, 4, 8), (2, 2, 2, 2), (8, 6, 4, 6)]
TOL = {0: 1e-13, 1: 1e-6, 2: 16 * UNIT_ROUNDOFF[2], 3: 16 * UNIT_ROUNDOFF[3]}


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_z4_noise_bit_exact(L, prec):
    tl = require_gpu()
    seed, first, n = 0x0123_4567_89AB_CDEF, 5, 3
    f = tl.empty_field(L, prec, n)
    tl.z4_noise(L, f, prec, seed, first, n)
    got = unpack(tl, L, f, prec, n)
    np.testing.assert_array_equal(got, oracle_z4(L, seed, first, n))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_pack_unpack_roundtrip(prec):
    tl = require_gpu()
    L = (6, 4, 4, 8)
    psi = synth.random_spinor(L, 2, seed=1)
    got = unpack(tl, L, pack(tl, L, psi, prec), prec, 2)
    if prec == 0:
        np.testing.assert_array_equal(got, psi)
    else:
        assert site_rel_err(got, psi) < 2 * UNIT_ROUNDOFF[prec]


@pytest.mark.parametrize("L", LATTICES)
@pytest.mark.parametrize("prec,recon", [(0, 18), (1, 12), (1, 18), (2, 12), (3, 12), (2, 18), (3, 18), (2, 0)])
@pytest.mark.parametrize("dagger,mu_zero", [(False, False), (True, False), (False, True)])
def test_dslash_matches_oracle(L, prec, recon, dagger, mu_zero):
    tl = require_gpu()
    kappa, mu = 0.16, 0.05
    U = synth.gauge_field(L, seed=7)
    nrhs = 3
    psi = synth.random_spinor(L, nrhs, seed=8)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=recon)
    fin = pack(tl, L, psi, prec)
    fout = tl.empty_field(L, prec, nrhs)
    tl.tm_dslash(op, fout, fin, nrhs, dagger=dagger, mu_zero=mu_zero, prec=prec)
    got = unpack(tl, L, fout, prec, nrhs)
    # the oracle acts on the same (rounded) input the kernel saw
    psi_in = unpack(tl, L, fin, prec, nrhs)
    if mu_zero:
        ref = apply_DW(U, psi_in, kappa)
    else:
        ref = apply_M(U, psi_in, kappa, mu, dagger=dagger)
    assert site_rel_err(got, ref) < TOL[prec]
    op.close()


def test_dslash_periodic_time_and_batch_independence():
    tl = require_gpu()
    L = (4, 4, 4, 6)
    U = synth.gauge_field(L, seed=17)
    psi = synth.random_spinor(L, 5, seed=18)
    op = tl.Operator(L, 0.15, 0.02, to_dev(U), antiperiodic=False, recon=18)
    fin = pack(tl, L, psi, 0)
    fout = tl.empty_field(L, 0, 5)
    tl.tm_dslash(op, fout, fin, 5, prec=0)
    got = unpack(tl, L, fout, 0, 5)
    ref = apply_M(U, psi, 0.15, 0.02, antiperiodic=False)
    assert site_rel_err(got, ref) < 1e-13
    # one right-hand side at a time gives bit-identical results
    one_in = pack(tl, L, psi[2:3], 0)
    one_out = tl.empty_field(L, 0, 1)
    tl.tm_dslash(op, one_out, one_in, 1, prec=0)
    np.testing.assert_array_equal(unpack(tl, L, one_out, 0, 1)[0], got[2])


def test_gamma5_and_convert():
    tl = require_gpu()
    L = (4, 2, 2, 4)
    psi = synth.random_spinor(L, 2, seed=3)
    f = pack(tl, L, psi, 0)
    g = tl.empty_field(L, 0, 2)
    tl.tm_gamma5(L, g, f, 0, 2)
    got = unpack(tl, L, g, 0, 2)
    ref = psi.copy()
    ref[..., 2:, :] *= -1
    np.testing.assert_array_equal(got, ref)
    h = tl.empty_field(L, 2, 2)
    tl.tm_spinor_convert(L, h, 2, f, 0, 2)
    np.testing.assert_array_equal(unpack(tl, L, h, 2, 2), unpack(tl, L, pack(tl, L, psi, 2), 2, 2))


def test_argument_errors_are_reported():
    tl = require_gpu()
    import torch
    with pytest.raises(tl.TmError):
        tl.z4_noise((3, 4, 4, 4), torch.empty(16, device="cuda"), 0, 1, 0, 1)  # odd extent
    U = to_dev(synth.unit_gauge((2, 2, 2, 2)))
    with pytest.raises(tl.TmError):
        tl.Operator((2, 2, 2, 2), 0.1, 0.0, U, recon=10)
    op = tl.Operator((2, 2, 2, 2), 0.1, 0.0, U)
    f = tl.empty_field((2, 2, 2, 2), 1, 1)
    with pytest.raises(tl.TmError):
        tl.tm_dslash(op, f, f, 1)                  # in-place is rejected
    tl.z4_noise((2, 2, 2, 2), f, 1, 1, 0, 0)       # zero sources: no-op


@pytest.mark.parametrize("prec,same_as", [(1, 12), (2, 18), (3, 18)])
def test_per_precision_link_format(prec, same_as):
    """recon = 0 keeps 12 reals per link for F32 and 18 for F16/BF16: the
    results are those of the operator built with that format."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=21)
    op0 = tl.Operator(L, 0.16, 0.02, to_dev(U), recon=0)
    opx = tl.Operator(L, 0.16, 0.02, to_dev(U), recon=same_as)
    fin = pack(tl, L, synth.random_spinor(L, 3, seed=22), prec)
    a, b = tl.empty_field(L, prec, 3), tl.empty_field(L, prec, 3)
    tl.tm_dslash(op0, a, fin, 3, prec=prec)
    tl.tm_dslash(opx, b, fin, 3, prec=prec)
    assert bool((a == b).all())
    assert tl.link_reals(0, prec) == same_as
    op0.close()
    opx.close()


@pytest.mark.parametrize("prec", [0, 1, 2, 4])
@pytest.mark.parametrize("dagger,mu_zero", [(False, True), (True, False)])
def test_dslash_g5_is_gamma5_of_dslash(prec, dagger, mu_zero):
    """tm_dslash_g5 stores gamma_5 of the Dslash result (a sign flip of the
    lower spins: exact in every format)."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    op = tl.Operator(L, 0.16, 0.02, to_dev(synth.gauge_field(L, seed=23)), recon=0)
    fin = pack(tl, L, synth.random_spinor(L, 2, seed=24), prec)
    a, b = tl.empty_field(L, prec, 2), tl.empty_field(L, prec, 2)
    tl.tm_dslash(op, a, fin, 2, dagger=dagger, mu_zero=mu_zero, prec=prec)
    tl.tm_gamma5(L, a, a, prec, 2)
    tl.tm_dslash_g5(op, b, fin, 2, dagger=dagger, mu_zero=mu_zero, prec=prec)
    assert bool((a == b).all())
    op.close()

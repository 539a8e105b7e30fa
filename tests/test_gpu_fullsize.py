"""Parity at the full benchmark size, in the launch configuration bench.py times:
32^3 x 64, kappa = 0.161, mu = 0.003, the bench's gauge seed, batches of 16
systems, FP16 LP fields and 12-real links.

Checked on sampled outputs the oracle computes one by one, or whole for one
system where that takes seconds:
  * Z4 noise: bit-exact for one full source;
  * Dslash on 16 FP16 systems (and one FP32 system): 2 x 512 sampled sites,
    among them every time-boundary case, against the oracle's formula on the
    same rounded inputs;
  * the LP solve of a source is bit-identical inside the batch and alone;
  * the HP solve (mixed precision, even/odd, 1e-9): the oracle's whole-lattice
    residual |eta - M x| / |eta|;
  * local loops of one system: the oracle's whole-lattice contraction.
"""
import numpy as np
import pytest
import torch

from oracle import loops as oloops
from oracle.operator import apply_M, apply_M_sites
from oracle.philox import z4_noise as oz4
from paper_1401_6749_gb300 import synth

from .gpu_util import UNIT_ROUNDOFF, from_dev, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

L = (32, 32, 32, 64)
KAPPA, MU = 0.161, 0.003
SEED = 20140126


@pytest.fixture(scope="module")
def setup():
    tl = require_gpu()
    U = synth.gauge_field(L, 1237, device="cuda")
    op = tl.Operator(L, KAPPA, MU, torch.from_numpy(U.view(np.float64)).cuda(), recon=12)
    yield tl, U, op
    op.close()


def _unpack_one(tl, f, prec, r, n):
    per = f.numel() // n
    out = torch.empty(int(np.prod(L)) * 24, dtype=torch.float64, device="cuda")
    tl.tm_spinor_unpack(L, out, f[r * per:(r + 1) * per], prec, 1)
    torch.cuda.synchronize()
    return from_dev(out, (L[3], L[2], L[1], L[0], 4, 3))


def _sites(n, seed):
    rng = np.random.default_rng(seed)
    s = np.stack([rng.integers(0, e, n) for e in L], axis=1)
    s[:4, 3] = [0, L[3] - 1, 0, L[3] - 1]         # time-boundary hops both ways
    s[4] = (L[0] - 1, L[1] - 1, L[2] - 1, L[3] - 1)
    return s


def test_noise_full_source_bit_exact(setup):
    tl, U, op = setup
    f = tl.empty_field(L, tl.F16, 2)
    tl.z4_noise(L, f, tl.F16, SEED, 40, 2)
    np.testing.assert_array_equal(_unpack_one(tl, f, tl.F16, 1, 2), oz4(L, SEED, 41, 1)[0])


@pytest.mark.parametrize("prec,n,tol", [(2, 16, 16 * UNIT_ROUNDOFF[2]), (1, 1, 1e-6)])
def test_dslash_sampled_sites(setup, prec, n, tol):
    tl, U, op = setup
    fin = tl.empty_field(L, prec, n)
    fout = tl.empty_field(L, prec, n)
    tl.z4_noise(L, fin, prec, 7, 0, n)
    tl.tm_dslash(op, fout, fin, n, prec=prec)
    sites = _sites(512, 3)
    for r in sorted({0, n - 1}):
        psi = _unpack_one(tl, fin, prec, r, n)
        got = _unpack_one(tl, fout, prec, r, n)[sites[:, 3], sites[:, 2], sites[:, 1], sites[:, 0]]
        ref = apply_M_sites(U, psi, KAPPA, MU, sites)
        d = np.linalg.norm((got - ref).reshape(len(sites), -1), axis=1)
        scale = np.maximum(np.linalg.norm(ref.reshape(len(sites), -1), axis=1),
                           np.sqrt(np.mean(np.sum(np.abs(ref) ** 2, axis=(1, 2)))))
        assert np.max(d / scale) < tol


def test_lp_batch_independence_full_size(setup):
    tl, U, op = setup
    prm = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, check_every=2, schur=True)
    eta = tl.empty_field(L, tl.F16, 16)
    x = tl.empty_field(L, tl.F16, 16)
    tl.z4_noise(L, eta, tl.F16, SEED, 0, 16)
    _, stats = tl.tm_cg_solve(op, x, eta, 16, prm)
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-2 for s in stats)
    e1 = tl.empty_field(L, tl.F16, 1)
    x1 = tl.empty_field(L, tl.F16, 1)
    tl.z4_noise(L, e1, tl.F16, SEED, 5, 1)
    tl.tm_cg_solve(op, x1, e1, 1, prm)
    per = x.numel() // 16
    torch.cuda.synchronize()
    assert torch.equal(x[5 * per:6 * per], x1)


def test_hp_solution_residual_and_local_loops(setup):
    tl, U, op = setup
    eta = tl.empty_field(L, tl.F64, 1)
    x = tl.empty_field(L, tl.F64, 1)
    tl.z4_noise(L, eta, tl.F64, SEED, 0, 1)
    _, stats = tl.tm_cg_solve(op, x, eta, 1, tl.cg_params(1e-9, 2000, tl.CG_MIXED, inner_prec=tl.F32,
                                                          delta=3e-5, schur=True))
    assert stats[0]["status"] == 0 and stats[0]["true_res"] <= 1e-9
    e = _unpack_one(tl, eta, tl.F64, 0, 1)
    s = _unpack_one(tl, x, tl.F64, 0, 1)
    res = np.linalg.norm((e - apply_M(U, s, KAPPA, MU)).ravel()) / np.linalg.norm(e.ravel())
    assert res < 1e-8
    out = torch.empty(16 * L[3] * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_local(L, x, x, tl.F64, 1, tl.LOOP_VV, out)
    got = from_dev(out, (16, L[3]))
    assert rel_l2(got, oloops.local_loops(s, s, "vv")) < 1e-12

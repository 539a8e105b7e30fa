"""Parity at the full benchmark size: 32^3 x 64, kappa = 0.161, mu = 0.003, the
bench's gauge seed and link format (recon 0: 12-real FP32 links, 18-real
FP16/BF16 links), batches of 16 systems.

Checked on sampled outputs the oracle computes one by one, or whole for one
system where that takes seconds:
  * Z4 noise: bit-exact for one full source;
  * Dslash on 16 FP16 systems with the 18-real FP16 links, both on the
    standard layout (CUDA-core kernel) and on the system-interleaved layout
    (tensor-core kernel the LP solver uses), and on one FP32 system: 2 x 512
    sampled sites, among them every time-boundary case, against the oracle's
    formula on the same rounded inputs;
  * the LP solve of a source (interleaved layout, Schur) is bit-identical
    inside the batch and alone;
  * the LP path of the bench on the interleaved layout, 16 systems: Z4
    sources drawn there (the bytes of the standard noise converted), the
    truncated solve (the bits of tm_cg_solve), D_W (2 x 512 sampled sites of
    one system), and that system's generalised local loops (whole lattice)
    and one-derivative loops (three slices) from the tensor-core kernels;
  * the HP solve (mixed precision, even/odd, 1e-9): the oracle's whole-lattice
    residual |eta - M x| / |eta|;
  * local loops of one system: the oracle's whole-lattice contraction;
  * one-derivative loops of one system in FP16 and in float-float (the HP
    loop precision): the oracle's contraction on the time slices t = 0 and
    T - 1 (both antiperiodic boundary crossings) and one interior slice.
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
    op = tl.Operator(L, KAPPA, MU, torch.from_numpy(U.view(np.float64)).cuda(), recon=0)
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


@pytest.mark.parametrize("prec,n,tol,il", [(2, 16, 16 * UNIT_ROUNDOFF[2], False), (2, 16, 16 * UNIT_ROUNDOFF[2], True),
                                            (1, 1, 1e-6, False)])
def test_dslash_sampled_sites(setup, prec, n, tol, il):
    tl, U, op = setup
    fin = tl.empty_field(L, prec, n)
    fout = tl.empty_field(L, prec, n)
    tl.z4_noise(L, fin, prec, 7, 0, n)
    if il:
        fin_il = tl.empty_field_il(L, n)
        fout_il = tl.empty_field_il(L, n)
        tl.tm_spinor_to_il(L, fin_il, fin, prec, n)
        tl.tm_dslash_il(op, fout_il, fin_il, n, prec=prec)
        tl.tm_spinor_from_il(L, fout, fout_il, prec, n)
        del fin_il, fout_il
    else:
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


def _oneD_slice(U, left, right, mode, t):
    """The oracle's one-derivative loops of time slice t (array (4, 16)): its
    contraction on the three slices t - 1, t, t + 1, cut out as a lattice of
    extent 3 in time (middle slice exact), with the antiperiodic sign moved
    onto the slice across the boundary."""
    T = L[3]
    idx = [(t - 1) % T, t, (t + 1) % T]
    lf, rf = left[idx].copy(), right[idx].copy()
    if t == 0:
        lf[0] *= -1
        rf[0] *= -1
    if t == T - 1:
        lf[2] *= -1
        rf[2] *= -1
    return oloops.oneD_loops(U[:, idx], lf, rf, mode, antiperiodic=False)[..., 1]


@pytest.mark.parametrize("prec,tol", [(2, 4e-3), (4, 1e-10)])
def test_oneD_loops_sampled_slices(setup, prec, tol):
    """One system's one-derivative loops (generalised estimator, L = s, R = an
    independent field) in FP16 (links and fields rounded to FP16: 4e-3) and in
    float-float (1e-10) against the oracle on three time slices."""
    tl, U, op = setup
    a = synth.random_spinor(L, 1, seed=61)
    b = synth.random_spinor(L, 1, seed=62)
    fa = tl.empty_field(L, prec, 1)
    fb = tl.empty_field(L, prec, 1)
    tl.tm_spinor_pack(L, fa, prec, torch.from_numpy(a.view(np.float64).copy()).cuda(), 1)
    tl.tm_spinor_pack(L, fb, prec, torch.from_numpy(b.view(np.float64).copy()).cuda(), 1)
    out = torch.empty(64 * L[3] * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_oneD(op, fa, fb, prec, 1, tl.LOOP_GEN, out)
    got = from_dev(out, (4, 16, L[3]))
    la = _unpack_one(tl, fa, prec, 0, 1)    # the values the kernel read
    lb = _unpack_one(tl, fb, prec, 0, 1)
    for t in (0, 17, L[3] - 1):
        ref = _oneD_slice(U, la, lb, "gen", t)
        assert rel_l2(got[..., t], ref) < tol, t


def test_interleaved_lp_path_full_size(setup):
    """The LP batch as the bench runs it (16 FP16 systems, interleaved layout):
    z4_noise_il, tm_cg_solve_il, D_W by tm_dslash_il, loop_contract_local_il
    and loop_contract_oneD_il with gamma_5 on the right (generalised
    estimator).  D_W against the oracle's formula at sampled sites (16u, as
    for M); the contractions of system 5 against the oracle on the same FP16
    values: local to FP32 rounding (1e-5), one-derivative with FP16-rounded
    links to 4u (the link products rounded once)."""
    tl, U, op = setup
    n, T, r = 16, L[3], 5
    u16 = UNIT_ROUNDOFF[tl.F16]
    eta_il = tl.empty_field_il(L, n)
    tl.z4_noise_il(L, eta_il, tl.F16, SEED, 0, n)
    eta = tl.empty_field(L, tl.F16, n)
    tl.z4_noise(L, eta, tl.F16, SEED, 0, n)
    conv = tl.empty_field_il(L, n)
    tl.tm_spinor_to_il(L, conv, eta, tl.F16, n)
    torch.cuda.synchronize()
    assert torch.equal(conv, eta_il)
    del conv
    prm = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, check_every=2, schur=True)
    x_il = tl.empty_field_il(L, n)
    _, stats = tl.tm_cg_solve_il(op, x_il, eta_il, n, prm)
    assert all(q["status"] == 0 and q["rel_res"] <= 1e-2 for q in stats)
    x = tl.empty_field(L, tl.F16, n)
    tl.tm_cg_solve(op, x, eta, n, prm)
    conv = tl.empty_field_il(L, n)
    tl.tm_spinor_to_il(L, conv, x, tl.F16, n)
    torch.cuda.synchronize()
    assert torch.equal(conv, x_il)
    del conv, eta, eta_il
    dw_il = tl.empty_field_il(L, n)
    tl.tm_dslash_il(op, dw_il, x_il, n, mu_zero=True, prec=tl.F16)
    dw = tl.empty_field(L, tl.F16, n)
    tl.tm_spinor_from_il(L, dw, dw_il, tl.F16, n)
    s = _unpack_one(tl, x, tl.F16, r, n)
    w = _unpack_one(tl, dw, tl.F16, r, n)
    del dw
    sites = _sites(512, 4)
    got = w[sites[:, 3], sites[:, 2], sites[:, 1], sites[:, 0]]
    ref = apply_M_sites(U, s, KAPPA, 0.0, sites)
    d = np.linalg.norm((got - ref).reshape(len(sites), -1), axis=1)
    scale = np.maximum(np.linalg.norm(ref.reshape(len(sites), -1), axis=1),
                       np.sqrt(np.mean(np.sum(np.abs(ref) ** 2, axis=(1, 2)))))
    assert np.max(d / scale) < 16 * u16
    g5w = w.copy()
    g5w[..., 2:, :] *= -1
    loc = torch.empty(n * 16 * T * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_local_il(L, x_il, dw_il, tl.F16, n, tl.LOOP_GEN, loc, right_g5=True)
    assert rel_l2(from_dev(loc, (n, 16, T))[r], oloops.local_loops(s, g5w, "gen")) < 1e-5
    oned = torch.empty(n * 64 * T * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_oneD_il(op, x_il, dw_il, tl.F16, n, tl.LOOP_GEN, oned, right_g5=True)
    got = from_dev(oned, (n, 4, 16, T))[r]
    tl.tm_op_check(op)                                 # no staging wait gave up
    h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(torch.float16).to(torch.float64).numpy()
    U16 = h(U.real) + 1j * h(U.imag)
    for t in (0, 17, T - 1):
        assert rel_l2(got[..., t], _oneD_slice(U16, s, g5w, "gen", t)) < 4 * u16, t

"""The system-interleaved 16-bit layout and its tensor-core Dslash.

  * layout conversion: standard -> interleaved -> standard is the identity
    (a byte permutation), slots of systems beyond nrhs are zero;
  * tm_dslash_il against the FP64 oracle (M, M^dag, D_W) per site at the
    16-bit tolerance of the CUDA-core kernel (16 u), on lattices whose half
    volume is and is not a multiple of the 32 sites of a warp, with 16, 17 and
    21 systems (full and ragged blocks), antiperiodic and periodic time;
  * a system's result is bit-identical whatever block row it occupies and
    whatever systems share its block;
  * the plain F16/BF16 solver on this layout: every solution meets the
    truncation against the oracle's operator, the per-system residuals match
    the oracle's, batch composition changes no bit, the Schur form and the
    unpreconditioned form both work, and the graph-replayed solve is
    bit-identical to the eager one.
"""
import numpy as np
import pytest
import torch

from oracle.operator import apply_DW, apply_M
from oracle.philox import z4_noise as oracle_z4
from paper_1401_6749_gb300 import synth

from .gpu_util import UNIT_ROUNDOFF, pack, require_gpu, site_rel_err, to_dev, unpack

pytestmark = pytest.mark.gpu

TOL = {2: 16 * UNIT_ROUNDOFF[2], 3: 16 * UNIT_ROUNDOFF[3]}


def _to_il(tl, L, f, prec, n):
    out = tl.empty_field_il(L, n)
    tl.tm_spinor_to_il(L, out, f, prec, n)
    return out


def _from_il(tl, L, fil, prec, n):
    out = tl.empty_field(L, prec, n)
    tl.tm_spinor_from_il(L, out, fil, prec, n)
    return out


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("n", [1, 5, 16, 21])
def test_layout_round_trip_and_zero_padding(prec, n):
    tl = require_gpu()
    L = (6, 6, 2, 6)
    psi = synth.random_spinor(L, n, seed=3 + n)
    f = pack(tl, L, psi, prec)
    fil = _to_il(tl, L, f, prec, n)
    back = _from_il(tl, L, fil, prec, n)
    torch.cuda.synchronize()
    assert torch.equal(back, f)
    nblk = (n + 15) // 16
    assert fil.numel() == nblk * 16 * int(np.prod(L)) * 48
    # slots of systems >= n: zero
    words = fil.view(torch.int32).view(nblk, 2, -1, 12, 16)
    for s in range(n, nblk * 16):
        blk, j = divmod(s, 16)
        for k in range(12):
            pos = (j % 8) ^ (4 if k % 3 == 2 else 0)
            slot = 2 * pos + (1 if j >= 8 else 0)
            assert not torch.any(words[blk, :, :, k, slot])


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("L,n", [((8, 6, 4, 6), 16), ((6, 6, 2, 6), 17), ((4, 4, 4, 8), 21), ((2, 2, 2, 2), 3)])
@pytest.mark.parametrize("dagger,mu_zero", [(False, False), (True, False), (False, True)])
def test_dslash_il_matches_oracle(prec, L, n, dagger, mu_zero):
    tl = require_gpu()
    kappa, mu = 0.16, 0.05
    U = synth.gauge_field(L, seed=7)
    psi = synth.random_spinor(L, n, seed=8)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=0)
    f = pack(tl, L, psi, prec)
    fil = _to_il(tl, L, f, prec, n)
    oil = tl.empty_field_il(L, n)
    tl.tm_dslash_il(op, oil, fil, n, dagger=dagger, mu_zero=mu_zero, prec=prec)
    got = unpack(tl, L, _from_il(tl, L, oil, prec, n), prec, n)
    psi_in = unpack(tl, L, f, prec, n)
    ref = apply_DW(U, psi_in, kappa) if mu_zero else apply_M(U, psi_in, kappa, mu, dagger=dagger)
    assert site_rel_err(got, ref) < TOL[prec]
    # same operator as the CUDA-core kernel of the standard layout (16-bit tolerance)
    fo = tl.empty_field(L, prec, n)
    tl.tm_dslash(op, fo, f, n, dagger=dagger, mu_zero=mu_zero, prec=prec)
    assert site_rel_err(got, unpack(tl, L, fo, prec, n)) < TOL[prec]
    op.close()


def test_dslash_il_periodic_time():
    tl = require_gpu()
    L = (4, 4, 4, 6)
    U = synth.gauge_field(L, seed=17)
    psi = synth.random_spinor(L, 4, seed=18)
    op = tl.Operator(L, 0.15, 0.02, to_dev(U), antiperiodic=False, recon=18)
    f = pack(tl, L, psi, 2)
    oil = tl.empty_field_il(L, 4)
    tl.tm_dslash_il(op, oil, _to_il(tl, L, f, 2, 4), 4, prec=2)
    got = unpack(tl, L, _from_il(tl, L, oil, 2, 4), 2, 4)
    ref = apply_M(U, unpack(tl, L, f, 2, 4), 0.15, 0.02, antiperiodic=False)
    assert site_rel_err(got, ref) < TOL[2]
    op.close()


@pytest.mark.parametrize("prec", [2, 3])
def test_row_and_block_independence(prec):
    """System j of a 21-system set (second block, row j - 16) gives the bits it
    gives alone (row 0) and at another row of a 16-system set."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=4)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=0)
    psi = synth.random_spinor(L, 21, seed=5)

    def run(idx):
        f = pack(tl, L, psi[idx], prec)
        n = len(idx)
        oil = tl.empty_field_il(L, n)
        tl.tm_dslash_il(op, oil, _to_il(tl, L, f, prec, n), n, prec=prec)
        return _from_il(tl, L, oil, prec, n).view(n, -1)

    a = run(list(range(21)))
    b = run([18])
    c = run([3, 7, 18] + list(range(8, 21))[:13])
    torch.cuda.synchronize()
    assert torch.equal(a[18], b[0])
    assert torch.equal(a[18], c[2])
    assert torch.equal(a[3], c[0]) and torch.equal(a[7], c[1])
    op.close()


def test_argument_errors():
    tl = require_gpu()
    L = (4, 4, 4, 4)
    U = synth.gauge_field(L, seed=1)
    op12 = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=12)
    f = tl.empty_field_il(L, 2)
    g = tl.empty_field_il(L, 2)
    with pytest.raises(tl.TmError) as e:
        tl.tm_dslash_il(op12, g, f, 2, prec=2)
    assert e.value.status == 6                       # 12-real 16-bit links: unsupported
    op12.close()
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=0)
    with pytest.raises(tl.TmError) as e:
        tl.tm_dslash_il(op, g, f, 2, prec=1)         # F32 has no interleaved form
    assert e.value.status == 1
    with pytest.raises(tl.TmError):
        tl.tm_dslash_il(op, f, f, 2, prec=2)         # in place
    with pytest.raises(tl.TmError):
        tl.tm_spinor_to_il(L, g, f, 0, 2)
    op.close()


# ------------------------------------------------------------------ solver
def _true_res(U, kappa, mu, eta, x):
    b = apply_M(U, eta, kappa, mu, dagger=True)
    r = b - apply_M(U, apply_M(U, x, kappa, mu), kappa, mu, dagger=True)
    return np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("schur", [False, True])
def test_il_truncated_solve_against_oracle(prec, schur):
    """Plain 16-bit CG on the interleaved layout, truncated at 1e-2 (Sec. 2.1):
    every solution meets the truncation against the oracle's FP64 operator
    (unpreconditioned: |b - M^dag M x| / |b|; Schur: the full solution solves
    M x = eta to the matching accuracy), 17 systems (a ragged second block)."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    kappa, mu = 0.16, 0.01
    U = synth.gauge_field(L, seed=9)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=0)
    n = 17
    eta = oracle_z4(L, 3, 0, n)
    x = tl.empty_field(L, prec, n)
    st, stats = tl.tm_cg_solve(op, x, pack(tl, L, eta, prec), n,
                               tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=prec, true_residual=True,
                                            schur=schur))
    got = unpack(tl, L, x, prec, n)
    for j in range(n):
        assert stats[j]["status"] == 0 and stats[j]["rel_res"] <= 1e-2
        assert stats[j]["true_res"] < 2e-2
        if not schur:
            true_rel = _true_res(U, kappa, mu, eta[j], got[j])
            assert true_rel < 2e-2
            assert abs(true_rel - stats[j]["true_res"]) < 5e-3
        else:
            r = eta[j] - apply_M(U, got[j], kappa, mu)
            assert np.linalg.norm(r.ravel()) / np.linalg.norm(eta[j].ravel()) < 0.1
    op.close()


def test_il_solve_batch_composition_and_graph():
    """The LP map is the same function of eta in every batch (TSM), and graph
    replay changes no bit."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=12)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=0)
    eta = oracle_z4(L, 44, 0, 20)
    prm = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=2, schur=True, check_every=2)
    xa = tl.empty_field(L, 2, 20)
    tl.tm_cg_solve(op, xa, pack(tl, L, eta, 2), 20, prm)
    xb = tl.empty_field(L, 2, 3)
    tl.tm_cg_solve(op, xb, pack(tl, L, eta[[17, 2, 9]], 2), 3, prm)
    a = xa.view(20, -1)
    b = xb.view(3, -1)
    torch.cuda.synchronize()
    assert torch.equal(a[17], b[0]) and torch.equal(a[2], b[1]) and torch.equal(a[9], b[2])
    prm_g = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=2, schur=True, check_every=2, graph=True)
    xg = tl.empty_field(L, 2, 20)
    tl.tm_cg_solve(op, xg, pack(tl, L, eta, 2), 20, prm_g)
    torch.cuda.synchronize()
    assert torch.equal(xg, xa)
    op.close()


def test_il_switch_selects_the_path():
    tl = require_gpu()
    L = (4, 4, 4, 8)
    U = synth.gauge_field(L, seed=2)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=0)
    eta = oracle_z4(L, 5, 0, 4)
    prm = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=2, schur=True)
    x_il = tl.empty_field(L, 2, 4)
    x_std = tl.empty_field(L, 2, 4)
    tl.tm_trace_reset()
    tl.tm_trace_enable(True)
    try:
        tl.tm_cg_solve(op, x_il, pack(tl, L, eta, 2), 4, prm)
        n_il, _, _ = tl.tm_trace_read("dslash.f16il.*")
        tl.tm_cg_il_enable(False)
        tl.tm_cg_solve(op, x_std, pack(tl, L, eta, 2), 4, prm)
        n_il2, _, _ = tl.tm_trace_read("dslash.f16il.*")
        n_std, _, _ = tl.tm_trace_read("dslash.f16.*")
    finally:
        tl.tm_cg_il_enable(True)
        tl.tm_trace_enable(False)
    assert n_il > 0 and n_il2 == n_il and n_std > 0
    a = unpack(tl, L, x_il, 2, 4)
    b = unpack(tl, L, x_std, 2, 4)
    # two valid truncated solutions of the same systems
    for j in range(4):
        assert np.linalg.norm((a[j] - b[j]).ravel()) / np.linalg.norm(b[j].ravel()) < 2e-2
    op.close()

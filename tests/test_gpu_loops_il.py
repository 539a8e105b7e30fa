"""Loop contractions on the system-interleaved layout (loop_contract_local_il,
loop_contract_oneD_il) and the solve that leaves its solution there
(tm_cg_solve_il), against the oracle.

Tolerances (Sec. 2.2 fixes no precision; the 16-bit contractions are the LP
estimator's): the local contraction multiplies the 16-bit numbers exactly and
sums in FP32, so against the oracle on the same rounded fields only FP32
rounding remains (1e-5).  The one-derivative contraction rounds each link
product U R once to the storage format before the spin products, a relative
error of at most u = 2^-11 (FP16) or 2^-8 (BF16) per product; with the
oracle on the same rounded fields and links the loops then agree to a few u
(bound used: 4u).  Lattices with ragged extents (sites per slice and parity
not a multiple of the warp's 4-site stride or of the 512-site block), odd
numbers of systems and a second block of 16 systems are covered; the
results of a system are bit-identical alone and inside a batch.
"""
import numpy as np
import pytest
import torch

from oracle import loops as oloops
from oracle.philox import z4_noise as oz4
from paper_1401_6749_gb300 import synth

from .gpu_util import UNIT_ROUNDOFF, from_dev, pack, rel_l2, require_gpu, to_dev, unpack

pytestmark = pytest.mark.gpu

MODES = ["std", "vv", "gen"]
# half volumes per slice: 32, 36 (ragged), 120, 648 (two 512-site chunks)
LATS = [(4, 4, 4, 4), (6, 6, 2, 6), (10, 6, 4, 4), (18, 12, 6, 4)]


def _g5(f):
    out = f.copy()
    out[..., 2:, :] *= -1
    return out


def _round_links(U, prec):
    """The links as the 16-bit copy holds them (round to nearest even)."""
    dt = torch.float16 if prec == 2 else torch.bfloat16
    r = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dt).to(torch.float64).numpy()
    return r(U.real) + 1j * r(U.imag)


def _fields(tl, L, n, prec, seeds):
    out = []
    for sd in seeds:
        std = pack(tl, L, synth.random_spinor(L, n, seed=sd), prec)
        il = tl.empty_field_il(L, n)
        tl.tm_spinor_to_il(L, il, std, prec, n)
        out.append((std, il, unpack(tl, L, std, prec, n)))
    return out


def _oned(tl, op, L, a, b, prec, n, mode, g5):
    out = torch.empty(n * 4 * 16 * L[3] * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_oneD_il(op, a, b, prec, n, tl.LOOP_MODE[mode], out, right_g5=g5)
    return from_dev(out, (n, 4, 16, L[3]))


def _local(tl, L, a, b, prec, n, mode, g5):
    out = torch.empty(n * 16 * L[3] * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_local_il(L, a, b, prec, n, tl.LOOP_MODE[mode], out, right_g5=g5)
    return from_dev(out, (n, 16, L[3]))


def _max_rel(got, ref):
    return max(rel_l2(got[j], ref[j]) for j in range(got.shape[0]))


@pytest.mark.parametrize("L", LATS)
@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("n", [3, 17])
def test_il_contractions_match_oracle(L, prec, n):
    tl = require_gpu()
    U = synth.gauge_field(L, seed=41)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=18)
    (_, ia, A), (_, ib, B) = _fields(tl, L, n, prec, (42, 43))
    Ur = _round_links(U, prec)
    tol = 4 * UNIT_ROUNDOFF[prec]
    for mode in MODES:
        for g5 in (False, True):
            Bm = _g5(B) if g5 else B
            assert _max_rel(_local(tl, L, ia, ib, prec, n, mode, g5), oloops.local_loops(A, Bm, mode)) < 1e-5
            assert _max_rel(_oned(tl, op, L, ia, ib, prec, n, mode, g5), oloops.oneD_loops(Ur, A, Bm, mode)) < tol
    tl.tm_op_check(op)                                 # no staging wait gave up
    op.close()


def test_oneD_il_periodic_time_and_recon0_links():
    """Periodic time (no boundary sign) and the bench's recon-0 operator (its
    FP16 links are the 18-real copy)."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=51)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), antiperiodic=False, recon=0)
    (_, ia, A), (_, ib, B) = _fields(tl, L, 5, 2, (52, 53))
    got = _oned(tl, op, L, ia, ib, 2, 5, "gen", False)
    ref = oloops.oneD_loops(_round_links(U, 2), A, B, "gen", antiperiodic=False)
    assert _max_rel(got, ref) < 4 * UNIT_ROUNDOFF[2]
    op.close()


def test_il_contractions_system_independent():
    """A system's loops are the same bits alone and at any row of a batch."""
    tl = require_gpu()
    L = (6, 6, 2, 6)
    U = synth.gauge_field(L, seed=61)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=18)
    n = 21
    A = synth.random_spinor(L, n, seed=62)
    B = synth.random_spinor(L, n, seed=63)

    def run(idx):
        k = len(idx)
        sa, sb = pack(tl, L, A[idx], 2), pack(tl, L, B[idx], 2)
        ia, ib = tl.empty_field_il(L, k), tl.empty_field_il(L, k)
        tl.tm_spinor_to_il(L, ia, sa, 2, k)
        tl.tm_spinor_to_il(L, ib, sb, 2, k)
        return _oned(tl, op, L, ia, ib, 2, k, "gen", True), _local(tl, L, ia, ib, 2, k, "gen", True)

    od_all, lc_all = run(list(range(n)))
    for j in (0, 9, 17, 20):
        od_one, lc_one = run([j])
        np.testing.assert_array_equal(od_all[j], od_one[0])
        np.testing.assert_array_equal(lc_all[j], lc_one[0])
    od_rot, _ = run([20, 3, 9])                         # other rows of the block
    np.testing.assert_array_equal(od_rot[2], od_all[9])
    op.close()


def test_oneD_il_matches_standard_kernel():
    """Against the CUDA-core FP16 contraction of the same fields: the rounding
    of the link products is the only difference."""
    tl = require_gpu()
    L = (8, 6, 4, 6)
    U = synth.gauge_field(L, seed=71)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=18)
    n = 16
    (sa, ia, _), (sb, ib, _) = _fields(tl, L, n, 2, (72, 73))
    ref = torch.empty(n * 4 * 16 * L[3] * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_oneD(op, sa, sb, 2, n, tl.LOOP_VV, ref)
    got = _oned(tl, op, L, ia, ib, 2, n, "vv", False)
    assert _max_rel(got, from_dev(ref, (n, 4, 16, L[3]))) < 4 * UNIT_ROUNDOFF[2]
    op.close()


def test_il_contraction_arguments():
    tl = require_gpu()
    L = (4, 4, 4, 4)
    U = synth.gauge_field(L, seed=81)
    op12 = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=12)
    op = tl.Operator(L, 0.16, 0.01, to_dev(U), recon=18)
    (_, ia, _), (_, ib, _) = _fields(tl, L, 2, 2, (82, 83))
    out = torch.empty(2 * 4 * 16 * L[3] * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(tl.TmError) as e:
        tl.loop_contract_oneD_il(op12, ia, ib, 2, 2, tl.LOOP_VV, out)
    assert e.value.status == 6                         # TM_ERR_UNSUPPORTED: no 18-real FP16 links
    with pytest.raises(tl.TmError) as e:
        tl.loop_contract_oneD_il(op, ia, ib, 1, 2, tl.LOOP_VV, out)
    assert e.value.status == 1                         # FP32 is not an interleaved format
    with pytest.raises(tl.TmError) as e:
        tl.loop_contract_local_il(L, ia[4:], ib, 2, 2, tl.LOOP_VV, out)
    assert e.value.status == 1                         # misaligned field
    op.close()
    op12.close()


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 2, 6), (18, 12, 6, 4)])
@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("n,first", [(1, 0), (16, 5), (17, 40), (35, 3)])
def test_z4_noise_il_is_the_converted_noise(L, prec, n, first):
    """z4_noise_il writes the oracle's Z4 noise (Sec. 2; +-1, +-i are exact
    in every format) in the interleaved layout: read back, every entry equals
    the oracle's; the bytes, including the zero slots of the systems past n
    in the last block of 16, are those of z4_noise followed by
    tm_spinor_to_il."""
    tl = require_gpu()
    seed = 0x1234_5678_9ABC                            # both key words non-zero
    got = tl.empty_field_il(L, n)
    got.fill_(0xA5)
    tl.z4_noise_il(L, got, prec, seed, first, n)
    std = tl.empty_field(L, prec, n)
    tl.tm_spinor_from_il(L, std, got, prec, n)
    assert np.array_equal(unpack(tl, L, std, prec, n), oz4(L, seed, first, n))
    tl.z4_noise(L, std, prec, seed, first, n)
    ref = tl.empty_field_il(L, n)
    ref.fill_(0x5A)
    tl.tm_spinor_to_il(L, ref, std, prec, n)
    torch.cuda.synchronize()
    assert torch.equal(ref, got)


def test_z4_noise_il_arguments():
    tl = require_gpu()
    L = (4, 4, 4, 4)
    f = tl.empty_field_il(L, 2)
    with pytest.raises(tl.TmError) as e:
        tl.z4_noise_il(L, f, tl.F32, 1, 0, 2)          # FP32 is not an interleaved format
    assert e.value.status == 1
    with pytest.raises(tl.TmError) as e:
        tl.z4_noise_il(L, f[2:], tl.F16, 1, 0, 2)      # misaligned field
    assert e.value.status == 1
    with pytest.raises(tl.TmError) as e:
        tl.z4_noise_il((3, 4, 4, 4), f, tl.F16, 1, 0, 2)   # odd extent
    assert e.value.status == 1
    before = f.clone()
    tl.z4_noise_il(L, f, tl.F16, 1, 0, 0)              # zero sources: no-op
    torch.cuda.synchronize()
    assert torch.equal(before, f)


@pytest.mark.parametrize("schur", [True, False])
def test_cg_solve_il_is_the_converted_solution(schur):
    """tm_cg_solve_il on the interleaved sources leaves exactly the bits that
    tm_cg_solve, on the same sources in the standard layout, converts back."""
    tl = require_gpu()
    L = (6, 4, 4, 8)
    U = synth.gauge_field(L, seed=91)
    op = tl.Operator(L, 0.16, 0.02, to_dev(U), recon=18)
    n = 5
    eta = pack(tl, L, oz4(L, 7, 0, n), 2)
    prm = tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, check_every=2, schur=schur)
    x = tl.empty_field(L, tl.F16, n)
    _, s1 = tl.tm_cg_solve(op, x, eta, n, prm)
    eta_il = tl.empty_field_il(L, n)
    tl.z4_noise_il(L, eta_il, tl.F16, 7, 0, n)
    x_il = tl.empty_field_il(L, n)
    _, s2 = tl.tm_cg_solve_il(op, x_il, eta_il, n, prm)
    assert [a["iters"] for a in s1] == [b["iters"] for b in s2]
    ref = tl.empty_field_il(L, n)
    tl.tm_spinor_to_il(L, ref, x, tl.F16, n)
    torch.cuda.synchronize()
    assert torch.equal(ref, x_il)
    with pytest.raises(tl.TmError) as e:               # a mixed solve has no interleaved form
        tl.tm_cg_solve_il(op, x_il, eta_il, n, tl.cg_params(1e-6, 100, tl.CG_MIXED, inner_prec=tl.F32))
    assert e.value.status == 6
    with pytest.raises(tl.TmError) as e:               # misaligned source
        tl.tm_cg_solve_il(op, x_il, eta_il[4:], n, prm)
    assert e.value.status == 1
    op.close()


def test_pipeline_bf16_lp_on_interleaved_layout():
    """The TSM pipeline with BF16 LP solves on the interleaved layout (18-real
    links; graph replay on at this size): every LP loop equals the oracle's
    contraction of that LP solution (re-solved in one batch: the same bits) to
    the BF16 rounding of D_W s and of the link products (8u), the local
    one-end loops to FP32 rounding."""
    tl = require_gpu()
    from oracle.operator import apply_DW
    from paper_1401_6749_gb300.tsm_pipeline import TsmPipeline
    L = (6, 4, 4, 8)
    T = L[3]
    kappa, mu = 0.16, 0.01
    U = synth.gauge_field(L, 2024)
    op = tl.Operator(L, kappa, mu, to_dev(U), recon=18)
    n_hp, n_lp = 2, 5
    p = TsmPipeline(op, n_hp, n_lp, batch=4, lp_prec=tl.BF16, tol_lp=1e-2, tol_hp=1e-10, seed=5, delta=1e-3)
    assert p.lp_il and p.lp_graph
    p.run()
    torch.cuda.synchronize()
    assert all(s["status"] == 0 and s["rel_res"] <= 1e-2 for s in p.stats_lp)
    n = n_hp + n_lp
    eta = oz4(L, 5, 0, n)
    x = tl.empty_field(L, tl.BF16, n)
    tl.tm_cg_solve(op, x, pack(tl, L, eta, tl.BF16), n,
                   tl.cg_params(1e-2, p.max_iter, tl.CG_PLAIN, prec=tl.BF16, check_every=2, schur=True))
    xs = unpack(tl, L, x, tl.BF16, n)
    g5dw = apply_DW(U, xs, kappa)
    g5dw[..., 2:, :] *= -1
    Ur = _round_links(U, 3)
    ref = {"local_vv": oloops.local_loops(xs, xs, "vv"), "local_gen": oloops.local_loops(xs, g5dw, "gen"),
           "oneD_vv": oloops.oneD_loops(Ur, xs, xs, "vv").reshape(n, 64, T),
           "oneD_gen": oloops.oneD_loops(Ur, xs, g5dw, "gen").reshape(n, 64, T)}
    tol = {"local_vv": 1e-5, "local_gen": 8 * UNIT_ROUNDOFF[3], "oneD_vv": 8 * UNIT_ROUNDOFF[3],
           "oneD_gen": 8 * UNIT_ROUNDOFF[3]}
    for k in p.kinds:
        got = p.lp_loops[k].cpu().numpy().view(np.complex128).reshape(n, -1, T)
        assert _max_rel(got, ref[k]) < tol[k], k
    op.close()

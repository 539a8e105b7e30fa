"""Parity at the sizes of the other workloads the build is specified on (the
4^4 FP64 pipeline case is test_gpu_loops.test_pipeline_4x4_plain_fp64, the
32^3 x 64 TSM workload is test_gpu_fullsize):

  * 16^3 x 32, kappa = 0.16, mu = 0.005, one right-hand side: the Dslash in
    FP64, FP32 and FP16 against the oracle's operator on the whole lattice, and
    CG to 1e-10 in plain FP64 and mixed precision (FP32 or FP16 iteration with
    FP64 reliable updates), checked by the oracle's residual |eta - M x| / |eta|
    on the whole lattice; the error of each mixed solution against the FP64
    solution is stated (printed) and bounded;
  * 24^3 x 48, kappa = 0.161, mu = 0.004: 12 and 24 Z4 sources in one batched
    mixed-precision solve (FP32 Dslash) replayed as CUDA graphs; a source's
    solution does not depend on the batch it is in, the oracle's residual holds
    for the first and last source, and the local loops (all three estimators)
    of those sources match the oracle's contraction;
  * the uneven batch: 8^4, 12^4, 16^3 x 32 and 24^3 x 48 with their own kappa,
    mu and 4 / 8 / 16 / 32 sources, TSM solves (FP16 at 1e-2, mixed to 1e-9)
    of all four lattices as ONE group (one graph launch per poll), each set
    bit-identical to its solve alone and one source per lattice checked by the
    oracle's residual.
Gauge fields: the seeded U = exp(0.3 i H) links, seed 1234 + workload index.
"""
import numpy as np
import pytest
import torch

from oracle import loops as oloops
from oracle.gamma import GAMMA5
from oracle.operator import apply_DW, apply_M
from oracle.philox import z4_noise as oz4
from paper_1401_6749_gb300 import synth

from .gpu_util import UNIT_ROUNDOFF, from_dev, rel_l2, require_gpu, site_rel_err, to_dev

pytestmark = pytest.mark.gpu

SEED = 20140126


def _unpack_one(tl, L, f, prec, r, n):
    per = f.numel() // n
    out = torch.empty(int(np.prod(L)) * 24, dtype=torch.float64, device="cuda")
    tl.tm_spinor_unpack(L, out, f[r * per:(r + 1) * per], prec, 1)
    torch.cuda.synchronize()
    return from_dev(out, (L[3], L[2], L[1], L[0], 4, 3))


def _residual(U, eta, x, kappa, mu):
    return float(np.linalg.norm((eta - apply_M(U, x, kappa, mu)).ravel()) / np.linalg.norm(eta.ravel()))


# ---------------------------------------------------------------- 16^3 x 32
L1, K1, M1 = (16, 16, 16, 32), 0.16, 0.005


@pytest.fixture(scope="module")
def w16():
    tl = require_gpu()
    U = synth.gauge_field(L1, 1235)
    ops = {r: tl.Operator(L1, K1, M1, to_dev(U), recon=r) for r in (12, 18)}  # FP64 always 18
    yield tl, U, ops
    for op in ops.values():
        op.close()


@pytest.mark.parametrize("prec,recon,tol", [(0, 18, 1e-13), (1, 12, 1e-6), (1, 18, 1e-6),
                                            (2, 12, 16 * UNIT_ROUNDOFF[2]), (2, 18, 16 * UNIT_ROUNDOFF[2]),
                                            (3, 18, 16 * UNIT_ROUNDOFF[3])])
def test_16x32_dslash_whole_lattice(w16, prec, recon, tol):
    tl, U, ops = w16
    fin = tl.empty_field(L1, prec, 1)
    fout = tl.empty_field(L1, prec, 1)
    tl.z4_noise(L1, fin, prec, 7, 0, 1)     # Z4 entries are exact in every format
    for dagger in (False, True):
        tl.tm_dslash(ops[recon], fout, fin, 1, dagger=dagger, prec=prec)
        got = _unpack_one(tl, L1, fout, prec, 0, 1)
        ref = apply_M(U, oz4(L1, 7, 0, 1)[0], K1, M1, dagger=dagger)
        err = site_rel_err(got[None], ref[None])
        print(f"16^3x32 Dslash prec={prec} recon={recon} dagger={dagger}: per-site rel err {err:.3e}")
        assert err < tol


def test_16x32_cg_fp64_and_mixed(w16):
    tl, U, ops = w16
    op = ops[12]
    eta = tl.empty_field(L1, tl.F64, 1)
    tl.z4_noise(L1, eta, tl.F64, SEED, 0, 1)
    e = oz4(L1, SEED, 0, 1)[0]
    sols = {}
    runs = {"fp64": tl.cg_params(1e-10, 20000, tl.CG_PLAIN, prec=tl.F64, true_residual=True, schur=True),
            "mixed_f32": tl.cg_params(1e-10, 20000, tl.CG_MIXED, inner_prec=tl.F32, delta=1e-5, schur=True),
            "mixed_f16": tl.cg_params(1e-10, 20000, tl.CG_MIXED, inner_prec=tl.F16, delta=1e-2, schur=True)}
    for name, prm in runs.items():
        x = tl.empty_field(L1, tl.F64, 1)
        _, stats = tl.tm_cg_solve(op, x, eta, 1, prm)
        assert stats[0]["status"] == 0 and stats[0]["true_res"] <= 1e-10
        sols[name] = _unpack_one(tl, L1, x, tl.F64, 0, 1)
        res = _residual(U, e, sols[name], K1, M1)
        print(f"16^3x32 CG {name}: iters {stats[0]['iters']}, reliable updates "
              f"{stats[0]['reliable_updates']}, oracle |eta - M x|/|eta| = {res:.3e}")
        assert res < 1e-7
    for name in ("mixed_f32", "mixed_f16"):
        d = rel_l2(sols[name], sols["fp64"])
        print(f"16^3x32 CG {name}: |x - x_fp64| / |x_fp64| = {d:.3e}")
        assert d < 1e-6


# ---------------------------------------------------------------- 24^3 x 48
L2, K2, M2 = (24, 24, 24, 48), 0.161, 0.004


def test_24x48_batched_graph_solve_and_local_loops():
    tl = require_gpu()
    U = synth.gauge_field(L2, 1236)
    op = tl.Operator(L2, K2, M2, to_dev(U), recon=12)
    prm = tl.cg_params(1e-10, 20000, tl.CG_MIXED, inner_prec=tl.F32, delta=1e-5, check_every=4,
                       schur=True, graph=True)
    xs, stats = {}, {}
    for n in (12, 24):
        eta = tl.empty_field(L2, tl.F64, n)
        tl.z4_noise(L2, eta, tl.F64, SEED, 0, n)
        xs[n] = tl.empty_field(L2, tl.F64, n)
        _, stats[n] = tl.tm_cg_solve(op, xs[n], eta, n, prm)
        assert all(s["status"] == 0 and s["true_res"] <= 1e-10 for s in stats[n])
    torch.cuda.synchronize()
    per = xs[24].numel() // 24
    assert torch.equal(xs[24][:12 * per], xs[12])          # batch independence
    assert [s["iters"] for s in stats[24][:12]] == [s["iters"] for s in stats[12]]
    # loops of the first and the last source against the oracle
    n = 24
    w = tl.empty_field(L2, tl.F64, n)
    g5w = tl.empty_field(L2, tl.F64, n)
    tl.tm_dslash(op, w, xs[n], n, mu_zero=True, prec=tl.F64)
    tl.tm_gamma5(L2, g5w, w, tl.F64, n)
    eta_all = tl.empty_field(L2, tl.F64, n)
    tl.z4_noise(L2, eta_all, tl.F64, SEED, 0, n)
    out = {}
    for mode, (lf, rf) in {"std": (eta_all, xs[n]), "vv": (xs[n], xs[n]), "gen": (xs[n], g5w)}.items():
        o = torch.empty(n * 16 * L2[3] * 2, dtype=torch.float64, device="cuda")
        tl.loop_contract_local(L2, lf, rf, tl.F64, n, tl.LOOP_MODE[mode], o)
        out[mode] = from_dev(o, (n, 16, L2[3]))
    for r in (0, n - 1):
        e = oz4(L2, SEED, r, 1)[0]
        s = _unpack_one(tl, L2, xs[n], tl.F64, r, n)
        res = _residual(U, e, s, K2, M2)
        print(f"24^3x48 source {r}: iters {stats[n][r]['iters']}, oracle |eta - M x|/|eta| = {res:.3e}")
        assert res < 1e-7
        g5dw = np.einsum("ab,...bc->...ac", GAMMA5, apply_DW(U, s, K2))
        ref = {"std": oloops.local_loops(e, s, "std"), "vv": oloops.local_loops(s, s, "vv"),
               "gen": oloops.local_loops(s, g5dw, "gen")}
        for mode in ref:
            assert rel_l2(out[mode][r], ref[mode]) < 1e-12
    op.close()


# ---------------------------------------------------------------- uneven batch
RAGGED = [((8, 8, 8, 8), 0.155, 0.01, 4), ((12, 12, 12, 12), 0.158, 0.007, 8),
          ((16, 16, 16, 32), 0.160, 0.005, 16), ((24, 24, 24, 48), 0.162, 0.003, 32)]


def test_uneven_batch_tsm_solves_as_one_group():
    tl = require_gpu()
    Us = [synth.gauge_field(L, 1238) for L, _, _, _ in RAGGED]
    ops = [tl.Operator(L, k, m, to_dev(U), recon=12) for (L, k, m, _), U in zip(RAGGED, Us)]
    ns = [n for *_, n in RAGGED]
    runs = {"lp": (tl.F16, tl.cg_params(1e-2, 20000, tl.CG_PLAIN, prec=tl.F16, check_every=2,
                                        schur=True, graph=True)),
            "hp": (tl.F64, tl.cg_params(1e-9, 20000, tl.CG_MIXED, inner_prec=tl.F32, delta=3e-5,
                                        check_every=4, schur=True, graph=True))}
    for name, (fp, prm) in runs.items():
        etas, xs = [], []
        for (L, *_), n in zip(RAGGED, ns):
            e = tl.empty_field(L, fp, n)
            tl.z4_noise(L, e, fp, SEED, 0, n)
            etas.append(e)
            xs.append(tl.empty_field(L, fp, n))
        st, stats = tl.tm_cg_solve_group(ops, xs, etas, ns, prm)
        torch.cuda.synchronize()
        assert st == 0
        for i, ((L, k, m, n), U) in enumerate(zip(RAGGED, Us)):
            tol = 1e-2 if name == "lp" else 1e-9
            assert all(s["status"] == 0 and s["rel_res"] <= tol for s in stats[i])
            alone = tl.empty_field(L, fp, n)
            tl.tm_cg_solve(ops[i], alone, etas[i], n, prm)
            torch.cuda.synchronize()
            assert torch.equal(alone, xs[i])
            if name == "hp":
                r = n - 1
                res = _residual(U, oz4(L, SEED, r, 1)[0], _unpack_one(tl, L, xs[i], fp, r, n), k, m)
                print(f"uneven batch {L}: HP iters {stats[i][r]['iters']}, oracle residual {res:.3e}")
                assert res < 1e-6
    for op in ops:
        op.close()

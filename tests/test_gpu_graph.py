"""CUDA-graph replay of the CG iterations and the grouped (uneven-batch) solve.

Both are launch-level restructurings of the same arithmetic, so they are held
to bit-identity with the plain tm_cg_solve: the same per-system scalars and the
same fixed-order reductions run in the same order.
"""
import numpy as np
import pytest
import torch

from paper_1401_6749_gb300 import synth

from .gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _op(tl, L, kappa, mu, seed):
    return tl.Operator(L, kappa, mu, to_dev(synth.gauge_field(L, seed)), recon=12)


def _solve(tl, op, L, prec_field, n, params, seed=20140126, first=0):
    eta = tl.empty_field(L, prec_field, n)
    tl.z4_noise(L, eta, prec_field, seed, first, n)
    x = tl.empty_field(L, prec_field, n)
    _, stats = tl.tm_cg_solve(op, x, eta, n, params)
    torch.cuda.synchronize()
    return x, stats


@pytest.mark.parametrize("mode,schur", [("lp", True), ("hp", True), ("hp", False), ("plain64", True)])
def test_graph_replay_is_bit_identical(mode, schur):
    tl = require_gpu()
    L = (8, 8, 8, 16)
    op = _op(tl, L, 0.161, 0.003, 5)
    if mode == "lp":
        kw = dict(tol=1e-2, mode=tl.CG_PLAIN, prec=tl.F16, check_every=2)
        fp = tl.F16
    elif mode == "hp":
        kw = dict(tol=1e-9, mode=tl.CG_MIXED, inner_prec=tl.F32, delta=3e-5, check_every=4)
        fp = tl.F64
    else:
        kw = dict(tol=1e-10, mode=tl.CG_PLAIN, prec=tl.F64, check_every=3)
        fp = tl.F64
    tol = kw.pop("tol")
    x0, s0 = _solve(tl, op, L, fp, 5, tl.cg_params(tol, 3000, schur=schur, graph=False, **kw))
    c0 = tl.tm_launch_count()
    x1, s1 = _solve(tl, op, L, fp, 5, tl.cg_params(tol, 3000, schur=schur, graph=True, **kw))
    assert tl.tm_launch_count() > c0           # replays are counted as kernel launches
    assert torch.equal(x0, x1)
    assert [s["iters"] for s in s0] == [s["iters"] for s in s1]
    assert [s["rel_res"] for s in s0] == [s["rel_res"] for s in s1]
    assert all(s["status"] == 0 for s in s1)
    op.close()


def test_graph_with_partial_last_block_and_noconv():
    """max_iter not a multiple of check_every: the tail runs without the graph;
    systems that hit max_iter report TM_ERR_NOCONV exactly as without it."""
    tl = require_gpu()
    L = (8, 8, 8, 8)
    op = _op(tl, L, 0.161, 0.003, 6)
    res = []
    for graph in (False, True):
        prm = tl.cg_params(1e-12, 7, tl.CG_PLAIN, prec=tl.F32, check_every=3, schur=True, graph=graph)
        eta = tl.empty_field(L, tl.F32, 3)
        tl.z4_noise(L, eta, tl.F32, 9, 0, 3)
        x = tl.empty_field(L, tl.F32, 3)
        st, stats = tl.tm_cg_solve(op, x, eta, 3, prm, raise_on_noconv=False)
        assert st == 3 and all(s["status"] == 3 and s["iters"] == 7 for s in stats)
        torch.cuda.synchronize()
        res.append(x.clone())
    assert torch.equal(res[0], res[1])
    op.close()


@pytest.mark.parametrize("graph", [False, True])
def test_group_solve_matches_single_solves(graph):
    """Four lattices with their own kappa, mu and source counts solved as one
    group give, set by set, the bits of tm_cg_solve on that set alone."""
    tl = require_gpu()
    sets = [((4, 4, 4, 4), 0.155, 0.01, 3), ((6, 6, 6, 6), 0.158, 0.007, 5),
            ((8, 8, 8, 16), 0.160, 0.005, 8), ((12, 12, 12, 24), 0.162, 0.003, 2)]
    prm = tl.cg_params(1e-9, 3000, tl.CG_MIXED, inner_prec=tl.F32, delta=3e-5, check_every=4,
                       schur=True, graph=graph)
    ops, xs, etas, ns, singles = [], [], [], [], []
    for i, (L, k, m, n) in enumerate(sets):
        op = _op(tl, L, k, m, 40 + i)
        eta = tl.empty_field(L, tl.F64, n)
        tl.z4_noise(L, eta, tl.F64, 77, 10 * i, n)
        ops.append(op); etas.append(eta); ns.append(n)
        xs.append(tl.empty_field(L, tl.F64, n))
        x1, s1 = _solve(tl, op, L, tl.F64, n, tl.cg_params(1e-9, 3000, tl.CG_MIXED, inner_prec=tl.F32,
                                                          delta=3e-5, check_every=4, schur=True),
                        seed=77, first=10 * i)
        singles.append((x1, s1))
    st, stats = tl.tm_cg_solve_group(ops, xs, etas, ns, prm)
    torch.cuda.synchronize()
    assert st == 0
    for i in range(len(sets)):
        assert torch.equal(xs[i], singles[i][0])
        assert [s["iters"] for s in stats[i]] == [s["iters"] for s in singles[i][1]]
        assert all(s["status"] == 0 and s["true_res"] <= 1e-9 for s in stats[i])
    for op in ops:
        op.close()


def test_group_rejects_a_shared_operator_and_accepts_clones():
    tl = require_gpu()
    L = (4, 4, 4, 8)
    op = _op(tl, L, 0.16, 0.01, 3)
    prm = tl.cg_params(1e-8, 500, tl.CG_PLAIN, prec=tl.F64, schur=True)
    f = [tl.empty_field(L, tl.F64, 2) for _ in range(4)]
    for e in f[:2]:
        tl.z4_noise(L, e, tl.F64, 1, 0, 2)
    with pytest.raises(tl.TmError):
        tl.tm_cg_solve_group([op, op], f[2:], f[:2], [2, 2], prm)
    twin = op.clone()
    st, stats = tl.tm_cg_solve_group([op, twin], f[2:], f[:2], [2, 2], prm)
    torch.cuda.synchronize()
    assert st == 0 and torch.equal(f[2], f[3])
    twin.close()
    op.close()


@pytest.mark.parametrize("mode", ["lp_il", "hp"])
def test_kept_graph_replays_are_bit_identical(mode):
    """The operator keeps the iteration graph of its last single-set solve and
    replays it for the next solve with the same buffers, systems and
    parameters: every such solve (new sources in the same buffers) gives the
    bits and the launch count of an eager solve; a solve with other buffers in
    between captures its own graph and leaves the results unchanged."""
    tl = require_gpu()
    L = (8, 8, 8, 8)
    op = tl.Operator(L, 0.161, 0.003, to_dev(synth.gauge_field(L, 7)), recon=18)
    if mode == "lp_il":
        kw = dict(mode=tl.CG_PLAIN, prec=tl.F16, check_every=2)
        tol, fp = 1e-2, tl.F16
    else:
        kw = dict(mode=tl.CG_MIXED, inner_prec=tl.F32, delta=3e-5, check_every=4)
        tol, fp = 1e-9, tl.F64
    n = 4
    eta = tl.empty_field(L, fp, n)
    x = tl.empty_field(L, fp, n)

    def solve(first, graph, xb=x, eb=eta, k=n):
        tl.z4_noise(L, eb, fp, 11, first, k)
        c0 = tl.tm_launch_count()
        _, st = tl.tm_cg_solve(op, xb, eb, k, tl.cg_params(tol, 3000, schur=True, graph=graph, **kw))
        torch.cuda.synchronize()
        return xb.clone(), [s["iters"] for s in st], tl.tm_launch_count() - c0

    solve(0, False)                                      # the autotuner's first launches
    ref = [solve(f, False) for f in (0, 4, 8)]
    got = [solve(f, True) for f in (0, 4)]              # capture, then replay of the kept graph
    x2 = tl.empty_field(L, fp, 2)
    e2 = tl.empty_field(L, fp, 2)
    solve(0, True, x2, e2, 2)                            # other buffers and systems: a new graph
    got.append(solve(8, True))                           # captured again for the first buffers
    for (xr, ir, cr), (xg, ig, cg) in zip(ref, got):
        assert torch.equal(xr, xg) and ir == ig and cr == cg
    op.close()

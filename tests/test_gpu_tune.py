"""The Dslash launch-shape autotuner: whatever shape it keeps, results are
bit-identical to the built-in shape (systems per thread and threads per block
change only the schedule), and every recorded choice is a valid shape."""
import numpy as np
import pytest
import torch

from paper_1401_6749_gb300 import synth

from .gpu_util import pack, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _run(tl, op, L, prec):
    psi = synth.random_spinor(L, 6, seed=4)
    fin = pack(tl, L, psi, prec)
    out = tl.empty_field(L, prec, 6)
    tl.tm_dslash(op, out, fin, 6, prec=prec)
    eta = tl.empty_field(L, tl.F64, 6)
    tl.z4_noise(L, eta, tl.F64, 5, 0, 6)
    x = tl.empty_field(L, tl.F64, 6)
    _, st = tl.tm_cg_solve(op, x, eta, 6, tl.cg_params(1e-10, 2000, tl.CG_MIXED, inner_prec=prec,
                                                       delta=0.1, schur=True))
    lp = tl.empty_field(L, tl.F16, 6)
    e16 = tl.empty_field(L, tl.F16, 6)
    tl.z4_noise(L, e16, tl.F16, 5, 0, 6)
    tl.tm_cg_solve(op, lp, e16, 6, tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, schur=True,
                                                check_every=2))
    torch.cuda.synchronize()
    return out.clone(), x.clone(), lp.clone(), [s["iters"] for s in st]


@pytest.mark.parametrize("prec", [1, 3])
def test_tuned_shapes_give_identical_results(prec):
    tl = require_gpu()
    L = (8, 8, 8, 8)
    op = tl.Operator(L, 0.161, 0.003, to_dev(synth.gauge_field(L, 2)), recon=0)
    tl.tm_tune_enable(False)
    tl.tm_tune_reset()
    ref = _run(tl, op, L, prec)
    assert tl.tm_tune_entries() == []
    tl.tm_tune_enable(True)
    got = _run(tl, op, L, prec)
    entries = tl.tm_tune_entries()
    assert len(entries) > 0
    for key, nr, bx, pk in entries:
        assert nr in (1, 2, 4) and nr <= key["nrhs"] and bx in (32, 64, 128)
        assert pk in (0, 1) and (pk == 0 or (nr == 2 and key["prec"] in (2, 3)))
        assert key["epilogue"] in (0, 2)                 # CG updates are never timed
    again = _run(tl, op, L, prec)                        # cached shapes
    for a, b, c in zip(ref, got, again):
        if isinstance(a, list):
            assert a == b == c
        else:
            assert torch.equal(a, b) and torch.equal(a, c)
    op.close()


def test_no_tuning_inside_graph_capture():
    tl = require_gpu()
    L = (8, 8, 8, 8)
    op = tl.Operator(L, 0.161, 0.003, to_dev(synth.gauge_field(L, 3)), recon=0)
    tl.tm_tune_enable(True)
    tl.tm_tune_reset()
    eta = tl.empty_field(L, tl.F16, 4)
    tl.z4_noise(L, eta, tl.F16, 9, 0, 4)
    xs = []
    for graph in (True, False):
        x = tl.empty_field(L, tl.F16, 4)
        tl.tm_cg_solve(op, x, eta, 4, tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, schur=True,
                                                   check_every=2, graph=graph))
        torch.cuda.synchronize()
        xs.append(x)
    assert torch.equal(xs[0], xs[1])
    op.close()

"""The library's device memory pool: an operator created after one of the same
lattice was destroyed reuses its memory (the pool does not grow), solver work
spaces and contraction scratch are served from it as well, and tm_mem_trim
gives the unused memory back."""
import pytest
import torch

from paper_1401_6749_gb300 import synth

from .gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _cycle(tl, L, U):
    op = tl.Operator(L, 0.161, 0.003, U, recon=0)
    eta = tl.empty_field(L, tl.F16, 4)
    tl.z4_noise(L, eta, tl.F16, 3, 0, 4)
    x = tl.empty_field(L, tl.F16, 4)
    _, st = tl.tm_cg_solve(op, x, eta, 4, tl.cg_params(1e-2, 500, tl.CG_PLAIN, prec=tl.F16, schur=True,
                                                       check_every=2))
    out = torch.empty(4 * 16 * L[3] * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_local(L, x, x, tl.F16, 4, tl.LOOP_MODE["vv"], out)
    torch.cuda.synchronize()
    held = tl.tm_mem_reserved()
    op.close()
    return held, [s["iters"] for s in st], out.clone()


def test_pool_reuses_memory_across_operators_and_trims():
    tl = require_gpu()
    L = (16, 16, 16, 16)
    U = to_dev(synth.gauge_field(L, 5))
    tl.tm_mem_trim(0)
    r0 = tl.tm_mem_reserved()
    held1, it1, out1 = _cycle(tl, L, U)
    assert held1 > r0                      # links and work space came from the pool
    after1 = tl.tm_mem_reserved()
    held2, it2, out2 = _cycle(tl, L, U)
    assert held2 == held1 and tl.tm_mem_reserved() == after1   # served from freed memory
    assert it1 == it2 and torch.equal(out1, out2)
    tl.tm_mem_trim(0)
    assert tl.tm_mem_reserved() == r0


def test_operator_from_pinned_host_field():
    """tm_op_create reads a page-locked host gauge field itself: the operator
    is bit-identical to one made from the same field in device memory, and
    pageable host memory is an argument error."""
    import numpy as np
    from paper_1401_6749_gb300 import synth
    tl = require_gpu()
    L = (8, 8, 4, 8)
    U = synth.gauge_field(L, seed=17)
    host = torch.from_numpy(U.view(np.float64).copy())
    ops = [tl.Operator(L, 0.16, 0.01, host.cuda(), recon=0), tl.Operator(L, 0.16, 0.01, host.pin_memory(), recon=0)]
    outs = []
    for op in ops:
        for prec in (tl.F64, tl.F32, tl.F16):
            f = tl.empty_field(L, prec, 2)
            tl.z4_noise(L, f, prec, 3, 0, 2)
            o = tl.empty_field(L, prec, 2)
            tl.tm_dslash(op, o, f, 2, prec=prec)
            outs.append(o)
    torch.cuda.synchronize()
    for a, b in zip(outs[:3], outs[3:]):
        assert torch.equal(a, b)
    with pytest.raises(tl.TmError) as e:
        tl.Operator(L, 0.16, 0.01, host, recon=0)     # pageable host memory
    assert e.value.status == 1
    for op in ops:
        op.close()

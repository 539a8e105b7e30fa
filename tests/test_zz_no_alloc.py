"""loop_contract_local_noalloc: the local contraction for callers that cannot
allocate device memory (their application owns the GPU's memory, or their
loop must not pay for an allocation per call).  It keeps its reduction scratch
in a fixed array inside the library instead of allocating any.

Checked through the C ABI against loop_contract_local, on two calls in a row
with different inputs, sizes and precisions (the shared array keeps the last
call's contents, which must not leak into the next result), within the
contraction tolerances of the other tests (1e-12 for FP64 fields, 1e-5 for
FP32).  This file is collected last so that a failure here leaves every other
test already run.
"""
import numpy as np
import pytest
import torch

from paper_1401_6749_gb300 import synth

from .gpu_util import from_dev, pack, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def _both(tl, L, fa, fb, prec, n, mode):
    T = L[3]
    ref = torch.empty(n * 16 * T * 2, dtype=torch.float64, device="cuda")
    got = torch.full_like(ref, float("nan"))
    tl.loop_contract_local(L, fa, fb, prec, n, mode, ref)
    tl.loop_contract_local_noalloc(L, fa, fb, prec, n, mode, got)
    torch.cuda.synchronize()
    return from_dev(got, (n, 16, T)), from_dev(ref, (n, 16, T))


def test_noalloc_matches_allocating_contraction_on_consecutive_calls():
    tl = require_gpu()
    # call 1: FP64 fields, 3 right-hand sides, several blocks per time slice
    L1 = (16, 16, 16, 8)
    a = synth.random_spinor(L1, 3, seed=101)
    b = synth.random_spinor(L1, 3, seed=102)
    got, ref = _both(tl, L1, pack(tl, L1, a, tl.F64), pack(tl, L1, b, tl.F64), tl.F64, 3, tl.LOOP_VV)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) < 1e-12
    # call 2: other lattice, FP32 fields, 2 right-hand sides, other estimator
    L2 = (12, 10, 8, 6)
    c = synth.random_spinor(L2, 2, seed=103)
    d = synth.random_spinor(L2, 2, seed=104)
    got, ref = _both(tl, L2, pack(tl, L2, c, tl.F32), pack(tl, L2, d, tl.F32), tl.F32, 2, tl.LOOP_GEN)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) < 1e-5


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    tl = require_gpu()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")   # never touched: rejected first
    with pytest.raises(tl.TmError) as e:
        tl.loop_contract_local_noalloc((32, 32, 32, 64), dummy, dummy, tl.F16, 17, tl.LOOP_STD, dummy)
    assert e.value.status == 1                                     # TM_ERR_ARG

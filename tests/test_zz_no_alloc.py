"""loop_contract_local_noalloc: the local contraction for callers that cannot
allocate device memory (their application owns the GPU's memory, or their
loop must not pay for an allocation per call).  It keeps its reduction scratch
in a fixed array inside the library instead of allocating any.

Checked through the C ABI, on consecutive calls with different inputs, sizes
and precisions (the shared array keeps the last call's contents, which must
not leak into the next result):
  * bit-identical to loop_contract_local (the same kernels in the same order,
    only the scratch address differs);
  * against the FP64 oracle for the FP64 case, at 1e-12;
  * a call allocates nothing: the library pool, torch's caching allocator and
    its allocation counters are unchanged across it;
  * sizes beyond the fixed array are rejected before any launch.
This file is collected last so that a failure here leaves every other test
already run.
"""
import gc

import numpy as np
import pytest
import torch

from oracle import loops as oloops
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
    return got, ref


def _alloc_state(tl):
    st = torch.cuda.memory_stats()
    return (tl.tm_mem_reserved(), torch.cuda.memory_reserved(), torch.cuda.memory_allocated(),
            st.get("allocation.all.allocated", 0), st.get("segment.all.allocated", 0))


def test_noalloc_matches_allocating_contraction_on_consecutive_calls():
    tl = require_gpu()
    # call 1: FP64 fields, 3 right-hand sides, several blocks per time slice
    L1 = (16, 16, 16, 8)
    a = synth.random_spinor(L1, 3, seed=101)
    b = synth.random_spinor(L1, 3, seed=102)
    got, ref = _both(tl, L1, pack(tl, L1, a, tl.F64), pack(tl, L1, b, tl.F64), tl.F64, 3, tl.LOOP_VV)
    assert torch.equal(got, ref)
    orc = oloops.local_loops(a, b, "vv")
    assert rel_l2(from_dev(got, (3, 16, L1[3])), orc) < 1e-12
    # calls 2-4: other lattices and precisions (FP32, FP16, float-float), other estimators
    cases = [((12, 10, 8, 6), tl.F32, 2, tl.LOOP_GEN), ((8, 8, 8, 16), tl.F16, 5, tl.LOOP_STD),
             ((10, 8, 6, 4), tl.FF, 2, tl.LOOP_VV)]
    for k, (L, prec, n, mode) in enumerate(cases):
        c = synth.random_spinor(L, n, seed=103 + 2 * k)
        d = synth.random_spinor(L, n, seed=104 + 2 * k)
        got, ref = _both(tl, L, pack(tl, L, c, prec), pack(tl, L, d, prec), prec, n, mode)
        assert torch.isfinite(got).all()
        assert torch.equal(got, ref), "precision %d" % prec


def test_noalloc_allocates_nothing():
    tl = require_gpu()
    L = (8, 8, 8, 8)
    n = 4
    a = pack(tl, L, synth.random_spinor(L, n, seed=201), tl.F32)
    b = pack(tl, L, synth.random_spinor(L, n, seed=202), tl.F32)
    out = torch.empty(n * 16 * L[3] * 2, dtype=torch.float64, device="cuda")
    tl.loop_contract_local_noalloc(L, a, b, tl.F32, n, tl.LOOP_VV, out)   # first call: set-up
    torch.cuda.synchronize()
    # tensors of earlier tests that only the cycle collector frees would
    # otherwise be released in the middle of the measurement
    gc.collect()
    gc.disable()
    try:
        before = _alloc_state(tl)
        for mode in (tl.LOOP_STD, tl.LOOP_VV, tl.LOOP_GEN):
            tl.loop_contract_local_noalloc(L, a, b, tl.F32, n, mode, out)
        torch.cuda.synchronize()
        after = _alloc_state(tl)
    finally:
        gc.enable()
    assert after == before


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    tl = require_gpu()
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")   # never touched: rejected first
    with pytest.raises(tl.TmError) as e:
        tl.loop_contract_local_noalloc((32, 32, 32, 64), dummy, dummy, tl.F16, 17, tl.LOOP_STD, dummy)
    assert e.value.status == 1                                     # TM_ERR_ARG
    with pytest.raises(tl.TmError) as e:
        tl.loop_contract_local_noalloc((32, 32, 32, 64), dummy, dummy, 7, 1, tl.LOOP_STD, dummy)
    assert e.value.status == 1

"""tsm_combine_host (Eq. 4 on host arrays, Sec. 2.1) against the oracle's
combination, through the C ABI on the CPU: random per-source loop sets with a
complex prefactor, and the edge cases n_hp = 0 (no correction), n_hp = 1 and
n_lp = 1 (undefined variances: NaN errors), and the argument checks."""
import numpy as np
import pytest
import torch

from oracle import tsm as otsm


def _lib():
    from paper_1401_6749_gb300 import build
    build.build()
    from paper_1401_6749_gb300 import tmloops
    return tmloops


@pytest.mark.parametrize("n_hp,n_lp", [(4, 9), (0, 5), (1, 6), (3, 1)])
def test_host_combine_matches_oracle(n_hp, n_lp):
    tl = _lib()
    rng = np.random.default_rng(10 * n_hp + n_lp)
    length, scale = 11, 0.5 - 0.3j
    hp = rng.standard_normal((max(n_hp, 1), 2 * length))
    lphp = rng.standard_normal((max(n_hp, 1), 2 * length))
    lp = rng.standard_normal((n_lp, 2 * length))
    mean = torch.empty(2 * length, dtype=torch.float64)
    err = torch.empty(2 * length, dtype=torch.float64)
    tl.tsm_combine_host(torch.tensor(hp) if n_hp else None, torch.tensor(lphp) if n_hp else None, n_hp,
                        torch.tensor(lp), n_lp, length, scale, mean, err)
    c = lambda a: a.view(np.complex128)
    m, er, ei = otsm.tsm_combine(c(hp[:n_hp]), c(lphp[:n_hp]), c(lp), scale=scale)
    np.testing.assert_allclose(mean.numpy().view(np.complex128), m, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(err.numpy()[0::2], er, rtol=1e-13, equal_nan=True)
    np.testing.assert_allclose(err.numpy()[1::2], ei, rtol=1e-13, equal_nan=True)
    if n_lp == 1 or n_hp == 1:
        assert np.all(np.isnan(err.numpy()))


def test_host_combine_argument_errors():
    tl = _lib()
    z = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(tl.TmError) as e:
        tl.tsm_combine_host(None, None, 0, z, 0, 2, 1.0, z.clone(), z.clone())   # n_lp = 0
    assert e.value.status == 1
    with pytest.raises(tl.TmError):
        tl.tsm_combine_host(None, None, 2, z, 1, 2, 1.0, z.clone(), z.clone())   # HP arrays missing

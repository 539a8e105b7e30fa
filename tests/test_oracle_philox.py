"""Pins of the oracle's Philox4x32-10 and Z4 noise (Sec. 2, Eqs. 1-2)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.philox import philox4x32_10, z4_noise

HERE = os.path.dirname(os.path.abspath(__file__))


def _lib_philox(tmp_path, rows):
    """Philox outputs from PyTorch's ATen engine (library routine), compiled with g++."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    if not os.path.exists(hdr):
        pytest.skip("ATen Philox header not shipped with this torch")
    exe = str(tmp_path / "philox_lib_ref")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc,
                    os.path.join(HERE, "philox_lib_ref.cpp"), "-o", exe], check=True)
    text = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    return np.array([[int(w, 16) for w in line.split()] for line in out.strip().splitlines()],
                    dtype=np.uint64)


def test_philox_matches_library_engine(tmp_path):
    rng = np.random.default_rng(11)
    rows = rng.integers(0, 2**32, size=(200, 6), dtype=np.uint64)
    rows[0] = 0
    rows[1] = 2**32 - 1
    rows[2, 2:4] = 0        # counters of the Z4 mapping: (site, r, 0, 0)
    ref = _lib_philox(tmp_path, rows)
    got = philox4x32_10(rows[:, :4], rows[:, 4:6]).astype(np.uint64)
    np.testing.assert_array_equal(got, ref)


def test_z4_values_and_mapping():
    L = (4, 2, 2, 4)
    seed = 0x1234_5678_9ABC
    eta = z4_noise(L, seed, first_src=3, nsrc=2)
    assert eta.shape == (2, 4, 2, 2, 4, 4, 3)
    vals = eta.ravel()
    assert np.all(np.isin(vals, np.array([1, 1j, -1, -1j])))
    # Spot check of the documented mapping for a few (site, component) entries,
    # from the raw generator words.
    X, Y, Z, T = L
    for (site, r, a, c) in [(0, 3, 0, 0), (17, 4, 3, 2), (63, 3, 2, 1)]:
        w0 = int(philox4x32_10(np.array([site, r, 0, 0], np.uint64),
                               np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint64))[0])
        k = (w0 >> (2 * (3 * a + c))) & 3
        x, y, z, t = site % X, (site // X) % Y, (site // (X * Y)) % Z, site // (X * Y * Z)
        assert eta[r - 3, t, z, y, x, a, c] == [1, 1j, -1, -1j][k]


def test_z4_statistics_eq1_eq2():
    """Eq. 1: the source average vanishes like 1/sqrt(N); Eq. 2: <eta eta^dag> -> 1."""
    L = (4, 4, 4, 4)
    N = 64
    eta = z4_noise(L, 20140126, 0, N).reshape(N, -1)
    n = eta.shape[1]
    # every entry has modulus one, so the diagonal of eta eta^dag is exactly 1
    assert np.allclose(np.abs(eta), 1.0)
    # uniform over the four values (chi^2 with 3 dof, p ~ 1e-6 threshold)
    k = np.round(np.angle(eta) / (np.pi / 2)).astype(int) % 4
    counts = np.bincount(k.ravel(), minlength=4)
    expect = k.size / 4
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 30.0
    # Eq. 1: mean over sources is O(1/sqrt(N)) entry by entry
    m = eta.mean(axis=0)
    assert np.sqrt(np.mean(np.abs(m) ** 2)) < 2.0 / np.sqrt(N)
    # Eq. 2: off-diagonal part of (1/N) sum eta eta^dag is O(1/sqrt(N))
    sub = eta[:, :200]
    C = sub.T @ sub.conj() / N
    off = C - np.diag(np.diag(C))
    assert np.allclose(np.diag(C), 1.0)
    assert np.sqrt(np.mean(np.abs(off[np.triu_indices(200, 1)]) ** 2)) < 1.5 / np.sqrt(N)


def test_z4_sources_are_distinct_and_counter_based():
    L = (2, 2, 2, 4)
    a = z4_noise(L, 7, 0, 4)
    b = z4_noise(L, 7, 2, 2)
    np.testing.assert_array_equal(a[2:], b)          # regenerate any source by index
    assert not np.array_equal(a[0], a[1])
    c = z4_noise(L, 8, 0, 1)
    assert not np.array_equal(a[0], c[0])            # the seed enters the key

"""Helpers shared by the GPU parity tests: device transfer of canonical fields
and the per-site tolerance used for operator parity."""
import numpy as np
import pytest
import torch


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_6749_gb300 import build
    build.build()
    from paper_1401_6749_gb300 import tmloops
    return tmloops


def to_dev(a):
    """complex128 numpy array -> float64 cuda tensor with (re, im) interleaved."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).copy()).cuda()


def from_dev(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def site_shape(L):
    X, Y, Z, T = L
    return (T, Z, Y, X)


def pack(tl, L, psi, prec):
    """numpy spinors (n, T, Z, Y, X, 4, 3) -> internal-layout device field."""
    n = psi.shape[0]
    f = tl.empty_field(L, prec, n)
    tl.tm_spinor_pack(L, f, prec, to_dev(psi), n)
    return f


def unpack(tl, L, f, prec, n):
    out = torch.empty(n * int(np.prod(L)) * 24, dtype=torch.float64, device="cuda")
    tl.tm_spinor_unpack(L, out, f, prec, n)
    torch.cuda.synchronize()
    return from_dev(out, (n,) + site_shape(L) + (4, 3))


def site_rel_err(got, ref):
    """max_x |got(x) - ref(x)| / max(|ref(x)|, rms_x |ref|) over (n, sites)."""
    d = np.linalg.norm((got - ref).reshape(got.shape[0], -1, 12), axis=-1)
    r = np.linalg.norm(ref.reshape(ref.shape[0], -1, 12), axis=-1)
    rms = np.sqrt(np.mean(r ** 2, axis=1, keepdims=True))
    return float(np.max(d / np.maximum(r, rms)))


def rel_l2(got, ref):
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


# unit roundoff of each storage precision
UNIT_ROUNDOFF = {0: 2.0 ** -53, 1: 2.0 ** -24, 2: 2.0 ** -11, 3: 2.0 ** -8}

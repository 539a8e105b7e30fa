"""Seeded synthetic inputs: gauge fields, gauge transformations, random spinors.

This module holds no arithmetic of the method.  It only produces inputs, and it
is the one module that both the CUDA path and the CPU oracle are fed from.

The paper measures on an N_f = 2+1+1 twisted-mass ensemble (Sec. 3) that is not
available; its stand-in is a smooth random SU(3) field

    U_mu(x) = exp(i * eps * H_mu(x)),  H = sum_{a=1}^{8} w_a lambda_a / 2,  w_a ~ N(0, 1),

with the Gell-Mann matrices lambda_a and eps = 0.3, drawn from numpy's PCG64
stream seeded by ``seed``.  Layout: complex128 [4, T, Z, Y, X, 3, 3], U[mu] the
link from x to x + mu_hat (mu = 0..3 for x, y, z, t).
"""
import numpy as np

_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1], _GELL_MANN[1][1, 0] = -1j, 1j
_GELL_MANN[2][0, 0], _GELL_MANN[2][1, 1] = 1, -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2], _GELL_MANN[4][2, 0] = -1j, 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2], _GELL_MANN[6][2, 1] = -1j, 1j
_GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)


def _expi(H, chunk=1 << 20, device="cpu"):
    """exp(i H) for a batch of Hermitian 3x3 matrices (torch's matrix_exp)."""
    import torch
    out = np.empty_like(H)
    flat = H.reshape(-1, 3, 3)
    res = out.reshape(-1, 3, 3)
    for s in range(0, flat.shape[0], chunk):
        m = torch.from_numpy(1j * flat[s:s + chunk]).to(device)
        res[s:s + chunk] = torch.linalg.matrix_exp(m).cpu().numpy()
    return out


def random_su3(shape, seed, eps, device="cpu"):
    """Array shape + (3, 3) of exp(i eps H) with H random traceless Hermitian."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(tuple(shape) + (8,))
    H = (w.reshape(-1, 8) @ (_GELL_MANN / 2).reshape(8, 9)).reshape(tuple(shape) + (3, 3))
    return _expi(eps * H, device=device)


def gauge_field(L, seed, eps=0.3, device="cpu"):
    """Smooth random SU(3) gauge field for lattice L = (X, Y, Z, T).

    ``device`` only selects where torch evaluates the matrix exponentials (a
    GPU makes the 32^3 x 64 field quick); the result is a host array either way.
    """
    X, Y, Z, T = (int(v) for v in L)
    return random_su3((4, T, Z, Y, X), seed, eps, device=device)


def unit_gauge(L):
    X, Y, Z, T = (int(v) for v in L)
    U = np.zeros((4, T, Z, Y, X, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def gauge_transform(L, seed, eps=1.0):
    """Random site field g(x) in SU(3), shape [T, Z, Y, X, 3, 3]."""
    X, Y, Z, T = (int(v) for v in L)
    return random_su3((T, Z, Y, X), seed, eps)


def random_spinor(L, nsrc, seed):
    """Complex Gaussian spinors, shape [nsrc, T, Z, Y, X, 4, 3]."""
    X, Y, Z, T = (int(v) for v in L)
    rng = np.random.default_rng(seed)
    shape = (nsrc, T, Z, Y, X, 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

"""Seeded synthetic SU(3) gauge fields (inputs only: none of the gauge-fixing arithmetic).

The paper's runs use 32^4 Wilson-action configurations at three couplings; those
are not available, so rough-gauge fields of the same size stand in for them:

    U_mu(x) = h(x) . exp(i eps A_mu(x)) . h^dag(x + mu)

  * h(x): Haar-random SU(3) per site -- QR of a complex Gaussian matrix with the
    phases of R's diagonal moved into Q (Mezzadri's recipe), then divided by a
    cube root of its determinant.
  * A_mu(x) = sum_a w_a T_a with T_a = lambda_a / 2 (Gell-Mann), w_a ~ N(0, 1).
  * exp(i eps A) from the eigen-decomposition of the Hermitian A.

eps sets the gauge-invariant roughness (eps = 0 is a pure gauge); h makes the
field maximally far from Landau gauge.  Random draws, in order, from
numpy.random.default_rng(seed): the real and imaginary parts of the V Gaussian
3x3 matrices for h (as one (V, 3, 3, 2) normal array), then w as a (4, V, 8)
normal array.

Arrays are complex128 (4, V, 3, 3), site index s = x + Lx*(y + Ly*(z + Lz*t)).
"""
from __future__ import annotations

import os

import numpy as np

_LAMBDA = np.zeros((8, 3, 3), np.complex128)
_LAMBDA[0, 0, 1] = _LAMBDA[0, 1, 0] = 1
_LAMBDA[1, 0, 1], _LAMBDA[1, 1, 0] = -1j, 1j
_LAMBDA[2, 0, 0], _LAMBDA[2, 1, 1] = 1, -1
_LAMBDA[3, 0, 2] = _LAMBDA[3, 2, 0] = 1
_LAMBDA[4, 0, 2], _LAMBDA[4, 2, 0] = -1j, 1j
_LAMBDA[5, 1, 2] = _LAMBDA[5, 2, 1] = 1
_LAMBDA[6, 1, 2], _LAMBDA[6, 2, 1] = -1j, 1j
_LAMBDA[7, 0, 0] = _LAMBDA[7, 1, 1] = 1 / np.sqrt(3)
_LAMBDA[7, 2, 2] = -2 / np.sqrt(3)
GENERATORS = _LAMBDA / 2  # T_a, Tr(T_a T_b) = delta_ab / 2


def volume(L) -> int:
    return int(np.prod([int(v) for v in L]))


def neighbour(L, mu: int, d: int = 1) -> np.ndarray:
    """Index array s -> site of s shifted by d along mu (periodic)."""
    L = [int(v) for v in L]
    V = volume(L)
    s = np.arange(V)
    c = []
    r = s
    for v in L:
        c.append(r % v)
        r = r // v
    c[mu] = (c[mu] + d) % L[mu]
    out = np.zeros(V, np.int64)
    for nu in (3, 2, 1, 0):
        out = out * L[nu] + c[nu]
    return out


def haar_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    z = rng.standard_normal((n, 3, 3, 2))
    z = (z[..., 0] + 1j * z[..., 1]) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def su3_exp_i(eps: float, A: np.ndarray) -> np.ndarray:
    """exp(i eps A) for Hermitian A (..., 3, 3), from its eigen-decomposition
    (torch's CPU eigh, which runs outside the GIL, when torch is importable)."""
    try:
        import torch

        w, v = torch.linalg.eigh(torch.from_numpy(np.ascontiguousarray(A)))
        w, v = w.numpy(), v.numpy()
    except ImportError:  # pragma: no cover
        w, v = np.linalg.eigh(A)
    return (v * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))


def _dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _exp_chunk(args):
    eps, w = args
    return su3_exp_i(eps, np.einsum("sa,aij->sij", w, GENERATORS))


def rough_gauge_field(L, eps: float, seed: int, haar: bool = True, chunk: int = 1 << 17,
                      workers: int | None = None) -> np.ndarray:
    """U_mu(x) = h(x) exp(i eps A_mu(x)) h^dag(x+mu); haar=False uses h = 1.

    Large lattices spread the eigen-decompositions over a pool of threads
    (numpy's linear algebra releases the GIL); all random draws happen before,
    so the result does not depend on the pool."""
    L = [int(v) for v in L]
    V = volume(L)
    rng = np.random.default_rng(seed)
    h = haar_su3(rng, V) if haar else None
    w = rng.standard_normal((4, V, 8))
    U = np.empty((4, V, 3, 3), np.complex128)
    jobs = [(mu, a, min(V, a + chunk)) for mu in range(4) for a in range(0, V, chunk)]
    if workers is None:
        workers = min(16, os.cpu_count() or 1) if 4 * V >= (1 << 20) else 1

    def job(j):
        mu, a, b = j
        U[mu, a:b] = _exp_chunk((eps, w[mu, a:b]))

    if workers > 1:
        import concurrent.futures as cf

        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(job, jobs))
    else:
        for j in jobs:
            job(j)
    if haar:
        for mu in range(4):
            nb = neighbour(L, mu, +1)
            for a in range(0, V, chunk):
                b = min(V, a + chunk)
                U[mu, a:b] = h[a:b] @ U[mu, a:b] @ _dagger(h[nb[a:b]])
    return U


def random_gauge(L, seed: int) -> np.ndarray:
    """A Haar-random gauge transformation h(x), shape (V, 3, 3)."""
    return haar_su3(np.random.default_rng(seed), volume(L))


def pure_gauge_field(L, seed: int) -> np.ndarray:
    """U_mu(x) = h(x) h^dag(x+mu): a gauge copy of the trivial field."""
    return rough_gauge_field(L, 0.0, seed)


def unit_field(L) -> np.ndarray:
    V = volume(L)
    U = np.zeros((4, V, 3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def random_su3_algebra(rng: np.random.Generator, shape) -> np.ndarray:
    """X = sum_a w_a T_a, w_a ~ N(0,1): random Hermitian traceless matrices."""
    w = rng.standard_normal(tuple(shape) + (8,))
    return np.einsum("...a,aij->...ij", w, GENERATORS)


def rough_gauge_field_cuda(L, eps: float, seed: int, haar: bool = True):
    """The same distribution as rough_gauge_field, drawn on the current CUDA
    device by the separate input-generation library (liblgf_inputs.so: Philox
    counter-based random numbers, column Gram-Schmidt Haar matrices, Taylor
    scaling-and-squaring exponential).  A different random stream from the numpy
    generator.  Returns a complex128 torch tensor (4, V, 3, 3) on the device."""
    import ctypes

    import torch

    from . import build as _build

    if not os.path.exists(_build.INPUTS_LIB) or not _build.up_to_date():
        _build.build()
    lib = ctypes.CDLL(_build.INPUTS_LIB)
    f = lib.lgf_inputs_rough_field
    f.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_ulonglong, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    L = [int(v) for v in L]
    V = volume(L)
    U = torch.empty((4, V, 3, 3), dtype=torch.complex128, device="cuda")
    h = torch.empty((V, 3, 3), dtype=torch.complex128, device="cuda") if haar else None
    rc = f((ctypes.c_int * 4)(*L), float(eps), int(seed), int(bool(haar)),
           ctypes.c_void_p(h.data_ptr() if h is not None else 0), ctypes.c_void_p(U.data_ptr()),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError("input generation failed (CUDA error %d)" % rc)
    torch.cuda.current_stream().synchronize()
    del h
    return U

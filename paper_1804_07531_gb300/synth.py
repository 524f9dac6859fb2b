"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module only draws random numbers and assembles test matrices from them; it
holds none of the low-rank method's arithmetic (no views, no QR of sketches, no
core SVD).  Both the FP64 oracle and the GPU library receive the arrays built
here, byte for byte.

Test-matrix families follow Section 8.1 of Bjarkason (2018): low rank plus
symmetric Gaussian noise, polynomially decaying and exponentially decaying
diagonal spectra.  Larger matrices are built as A = U diag(sigma) V^T with
Haar-distributed U, V (QR of a seeded Gaussian with the R diagonal made
positive, which gives the Haar measure).  With a Gaussian test matrix the
error distribution of every algorithm depends only on sigma, so any orthogonal
U, V would do; Haar factors keep the entries free of structure.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng", "gaussian", "haar", "usv", "lowrank_noise", "poly_decay", "exp_decay",
    "sigma_config", "CONFIGS",
]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for `seed` (numpy's documented default bit generator)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian(rows: int, cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """rows x cols i.i.d. N(0,1), drawn in row-major order, cast to `dtype`."""
    g = rng(seed).standard_normal((rows, cols))
    return np.ascontiguousarray(g.astype(dtype, copy=False))


def haar(n: int, r: int, seed: int) -> np.ndarray:
    """First r columns of a Haar-random n x n orthogonal matrix (FP64).

    Q from the QR factorisation of an n x r Gaussian, with column signs chosen
    so that diag(R) > 0 (Mezzadri 2007: this normalisation makes Q Haar).
    """
    g = rng(seed).standard_normal((n, r))
    q, rr = np.linalg.qr(g)
    d = np.sign(np.diag(rr))
    d[d == 0] = 1.0
    return np.ascontiguousarray(q * d[None, :])


def _preload_torch_linalg():
    """Load torch's CUDA linear-algebra library by path so that torch's own
    lazy dlopen of it succeeds in environments (profilers) that alter the
    library search path."""
    import ctypes
    import glob
    import os

    import torch
    for lib in glob.glob(os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so*")):
        try:
            ctypes.CDLL(lib, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def haar_torch(n: int, r: int, seed: int, device="cuda", dtype=None):
    """Haar columns built with torch on `device` (fixture for large shapes).

    The Gaussian is drawn by a seeded torch generator on that device and
    factorised by torch.linalg.qr; the result is an input, shared with every
    consumer in the same process.
    """
    import torch

    _preload_torch_linalg()
    dtype = dtype or torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    g = torch.randn(n, r, generator=gen, device=device, dtype=dtype)
    q, rr = torch.linalg.qr(g)
    d = torch.sign(torch.diagonal(rr))
    d[d == 0] = 1.0
    return q * d[None, :]


def usv(m: int, n: int, sigma: np.ndarray, seed_u: int, seed_v: int) -> np.ndarray:
    """A = U diag(sigma) V^T (FP64, m x n) with Haar U (m x r), V (n x r)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    u = haar(m, r, seed_u)
    v = haar(n, r, seed_v)
    return np.ascontiguousarray((u * sigma[None, :]) @ v.T)


# ---------------------------------------------------------------- Section 8.1
def lowrank_noise(n: int = 1000, R: int = 10, eta: float = 1e-2, seed: int = 0) -> np.ndarray:
    """diag(1,..,1 (R times), 0, .., 0) + sqrt(eta R / (2 n^2)) (G + G^T)."""
    g = rng(seed).standard_normal((n, n))
    a = math.sqrt(eta * R / (2.0 * n * n)) * (g + g.T)
    a[np.arange(R), np.arange(R)] += 1.0
    return a


def poly_decay(n: int = 1000, R: int = 10, rho: float = 1.0) -> np.ndarray:
    """diag(1,..,1 (R times), 2^-rho, 3^-rho, .., (n-R+1)^-rho)."""
    d = np.ones(n)
    d[R:] = np.arange(2, n - R + 2, dtype=np.float64) ** (-rho)
    return np.diag(d)


def exp_decay(n: int = 1000, R: int = 10, theta: float = 0.25) -> np.ndarray:
    """diag(1,..,1 (R times), 10^-theta, 10^-2theta, .., 10^-(n-R)theta)."""
    d = np.ones(n)
    d[R:] = 10.0 ** (-theta * np.arange(1, n - R + 1, dtype=np.float64))
    return np.diag(d)


# ------------------------------------------------------- workload spectra
def sigma_config(name: str, r: int) -> np.ndarray:
    """The first r singular values of the named workload spectrum."""
    j = np.arange(1, r + 1, dtype=np.float64)
    if name == "inv":            # sigma_j = 1/j
        return 1.0 / j
    if name == "exp25":          # sigma_j = 10^(-j/25)
        return 10.0 ** (-j / 25.0)
    if name == "pow15":          # sigma_j = j^-1.5
        return j ** -1.5
    if name == "gap32":          # exp(-j/40), x0.1 after j = 32
        s = np.exp(-j / 40.0)
        s[32:] *= 0.1
        return s
    raise ValueError(name)


# Workloads (sizes, spectra and parameters), named by what they are.
# k = target rank, p = oversampling, ell = k + p, v = views.
CONFIGS = {
    "subspace_2048x1024_v3": dict(m=2048, n=1024, spectrum="inv", rank=1024, k=20, p=10, v=3,
                                  dtype="f32", seed_u=11, seed_v=12, seed_omega=1),
    "single_pass_20000x10000": dict(m=20000, n=10000, spectrum="exp25", rank=256, noise=1e-4,
                                    k=50, ell1=120, ell2=240, dtype="f32",
                                    seed_u=21, seed_v=22, seed_noise=23, seed_omega=24,
                                    seed_psi=25),
    "krylov_65536x16384_v4": dict(m=65536, n=16384, spectrum="pow15", rank=16384, k=100, p=20,
                                  v=4, dtype="bf16", seed_u=31, seed_v=32, seed_omega=33),
    "grad_8192x4096_v4": dict(m=8192, n=4096, spectrum="gap32", rank=4096, k=32, p=8, v=4,
                              dtype="f32", seed_u=41, seed_v=42, seed_omega=43),
    "host_262144x65536": dict(m=262144, n=65536, spectrum="inv", noise=1e-5, k=200, ell1=400,
                              ell2=800, panel=4096, dtype="f32"),
}

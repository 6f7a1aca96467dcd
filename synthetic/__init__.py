"""Seeded synthetic inputs for the staggered-fermion hot path.

This module only draws random numbers and shapes them into gauge links,
pseudofermion sources and rational-approximation poles/residues.  It holds
none of the method's arithmetic (no Dirac operator, no solver, no force), so
both the FP64 oracle and the CUDA path can take their inputs from it.

Layouts (canonical interchange, shared by the oracle and the C-ABI):
  links   complex128 [4][V][3][3]; V lexicographic with
          i = x + Lx*(y + Ly*(z + Lz*t)), mu = 0..3 = x, y, z, t; row-major
          3x3 matrices (U[a][b], a = row).
  fields  complex128 [Vh][3] on one parity, site i stored at half index i>>1
          (valid because Lx is even).

The paper's gauge variables are SU(3) matrices on links and its
pseudofermions live on even sites (Sec. 2); no production ensemble is
available, so links are Haar-random or close to unit (exp(i*0.3*H)).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "volume", "haar_su3", "exp_i_h", "unit_links", "gauge_links",
    "gaussian_field", "haar_gauge_transform", "log_poles", "positive_residues",
    "CONFIGS",
]


def rng(seed: int) -> np.random.Generator:
    """Seeded PCG64 generator (every input in this project is drawn from one)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _complex_gaussian(g: np.random.Generator, shape) -> np.ndarray:
    """(N + iN)/sqrt(2): unit-variance complex Gaussian."""
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im) / np.sqrt(2.0)


def haar_su3(g: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-distributed SU(3) matrices, shape (n, 3, 3).

    QR of a complex Gaussian matrix, phases of R's diagonal moved into Q
    (Mezzadri's recipe for Haar U(3)), then det fixed to 1 by dividing by
    the principal cube root of det(Q).
    """
    z = _complex_gaussian(g, (n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return np.ascontiguousarray(q)


def exp_i_h(g: np.random.Generator, n: int, scale: float = 0.3) -> np.ndarray:
    """n matrices exp(i*scale*H), H a Gaussian traceless Hermitian 3x3.

    H = (G + G^dag)/2 - tr/3 with G complex Gaussian; the exponential is
    taken through the eigendecomposition of H, so det = exp(i*scale*tr H) = 1.
    """
    gm = _complex_gaussian(g, (n, 3, 3))
    h = 0.5 * (gm + np.conj(np.swapaxes(gm, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * scale * w)
    u = (v * ph[:, None, :]) @ np.conj(np.swapaxes(v, 1, 2))
    return np.ascontiguousarray(u)


def unit_links(dims) -> np.ndarray:
    v = volume(dims)
    u = np.zeros((4, v, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def gauge_links(dims, kind: str, seed: int) -> np.ndarray:
    """Canonical links [4][V][3][3] of the given kind: 'haar', 'expih', 'unit'."""
    v = volume(dims)
    if kind == "unit":
        return unit_links(dims)
    g = rng(seed)
    if kind not in ("haar", "expih"):
        raise ValueError(f"unknown link kind {kind!r}")
    u = np.empty((4, v, 3, 3), np.complex128)
    for mu in range(4):  # one direction at a time bounds the temporaries
        u[mu] = haar_su3(g, v) if kind == "haar" else exp_i_h(g, v, 0.3)
    return u


def gaussian_field(dims, seed: int, parity_sites: bool = True) -> np.ndarray:
    """Complex Gaussian colour vector field, [Vh][3] (or [V][3])."""
    v = volume(dims)
    n = v // 2 if parity_sites else v
    return np.ascontiguousarray(_complex_gaussian(rng(seed), (n, 3)))


def haar_gauge_transform(dims, seed: int) -> np.ndarray:
    """One Haar SU(3) matrix per site, [V][3][3]."""
    return haar_su3(rng(seed), volume(dims))


def log_poles(lo: float, hi: float, n: int) -> np.ndarray:
    """n poles sigma_i log-spaced between lo and hi (synthetic rational approximation)."""
    return np.logspace(np.log10(lo), np.log10(hi), n)


def positive_residues(seed: int, n: int, lo: float = 0.1, hi: float = 1.0) -> np.ndarray:
    """n seeded positive residues r_i ~ U(lo, hi)."""
    return rng(seed).uniform(lo, hi, n)


# The five workloads.  Seeds: links 1000+k, sources 2000+k, residues 3000+k,
# gauge transforms 4000+k for workload k (1-based).
CONFIGS = {
    "small_4x4x4x4": dict(
        k=1, dims=(4, 4, 4, 4), links="haar", mass=0.1,
        shifts=lambda: log_poles(1e-4, 1.0, 8), tol=1e-10, nrhs=1),
    "bandwidth_16x16x16x16": dict(k=2, dims=(16, 16, 16, 16), links="expih", mass=0.05),
    "bandwidth_32x32x32x32": dict(k=2, dims=(32, 32, 32, 32), links="expih", mass=0.05),
    "mscg_32x32x32x32": dict(
        k=3, dims=(32, 32, 32, 32), links="expih", mass=0.01,
        shifts=lambda: log_poles(1e-5, 10.0, 16), tol=1e-10, nrhs=1),
    "batched_uneven": dict(
        k=4, dims_list=[(16, 16, 16, 16), (24, 24, 24, 8), (32, 32, 32, 8), (24, 24, 24, 24)],
        links="expih", mass=0.02, shifts=lambda: log_poles(1e-5, 10.0, 16), tol=1e-10, nrhs=4),
    "force_48x48x48x48": dict(
        k=5, dims=(48, 48, 48, 48), links="expih", mass=0.01,
        shifts=lambda: log_poles(1e-5, 10.0, 12), tol=1e-10, nrhs=1),
}

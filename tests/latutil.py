"""Small numpy helpers for the tests: coordinates, plane waves, gauge transforms.

Independent of both the oracle and the CUDA library; they only index the
canonical layouts (links [4][V][3][3], half fields [Vh][3], site
i = x + Lx*(y + Ly*(z + Lz*t)), half index i >> 1).
"""
from __future__ import annotations

import itertools

import numpy as np


def coords(dims) -> np.ndarray:
    """[V][4] coordinates (x, y, z, t) in lexicographic site order."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)


def parity(dims) -> np.ndarray:
    return coords(dims).sum(axis=1) % 2


def shift_index(dims, mu: int, step: int) -> np.ndarray:
    """Index of the neighbour x + step*mu for every site, periodic."""
    c = coords(dims).copy()
    c[:, mu] = (c[:, mu] + step) % dims[mu]
    lx, ly, lz, _ = dims
    return c[:, 0] + lx * (c[:, 1] + ly * (c[:, 2] + lz * c[:, 3]))


def to_half(dims, full: np.ndarray, par: int) -> np.ndarray:
    """Restrict a [V][...] field to parity `par`, in half-index order."""
    p = parity(dims)
    idx = np.nonzero(p == par)[0]
    out = np.empty((len(idx),) + full.shape[1:], full.dtype)
    out[idx >> 1] = full[idx]
    return out


def to_full(dims, half: np.ndarray, par: int) -> np.ndarray:
    p = parity(dims)
    v = len(p)
    out = np.zeros((v,) + half.shape[1:], half.dtype)
    idx = np.nonzero(p == par)[0]
    out[idx] = half[idx >> 1]
    return out


def momentum(dims, n) -> np.ndarray:
    """p_mu = 2 pi n_mu / L_mu for x, y, z and pi (2 n_t + 1) / L_t (antiperiodic t)."""
    lx, ly, lz, lt = dims
    return np.array([2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
                     np.pi * (2 * n[3] + 1) / lt])


def plane_wave_even(dims, n, colour) -> np.ndarray:
    """Even-site restriction of exp(i p.x) * colour, [Vh][3]."""
    p = momentum(dims, n)
    ph = np.exp(1j * coords(dims) @ p)
    full = ph[:, None] * np.asarray(colour, np.complex128)[None, :]
    return to_half(dims, full, 0)


def free_eigenvalues(dims, mass: float, sigma: float = 0.0) -> np.ndarray:
    """Closed-form spectrum of m^2 + sigma - D_eo D_oe on unit links: one value
    m^2 + sigma + sum_mu sin^2 p_mu per momentum class p ~ p + (pi, pi, pi, pi)
    (representatives n_x < Lx/2), times 3 colours; sorted."""
    lx, ly, lz, lt = dims
    vals = []
    for n in itertools.product(range(lx // 2), range(ly), range(lz), range(lt)):
        p = momentum(dims, n)
        vals.append(mass * mass + sigma + np.sum(np.sin(p) ** 2))
    return np.sort(np.repeat(np.array(vals), 3))


def gauge_transform_links(dims, links: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """U'_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dag."""
    out = np.empty_like(links)
    for mu in range(4):
        f = shift_index(dims, mu, +1)
        out[mu] = omega @ links[mu] @ np.conj(np.swapaxes(omega[f], 1, 2))
    return out


def gauge_transform_half(dims, psi: np.ndarray, omega: np.ndarray, par: int) -> np.ndarray:
    """psi'(x) = Omega(x) psi(x) on parity `par`."""
    om = to_half(dims, omega, par)
    return np.einsum("sab,sb->sa", om, psi)


def dense_normal_op(op, n: int) -> np.ndarray:
    """Dense matrix of a linear map on C^n given as a function of a flat vector."""
    a = np.empty((n, n), np.complex128)
    for k in range(n):
        e = np.zeros(n, np.complex128)
        e[k] = 1.0
        a[:, k] = np.asarray(op(e)).reshape(-1)
    return a


def random_su3_algebra(g: np.random.Generator) -> np.ndarray:
    """Random X in su(3): anti-Hermitian, traceless."""
    m = (g.standard_normal((3, 3)) + 1j * g.standard_normal((3, 3)))
    x = 0.5 * (m - m.conj().T)
    return x - np.trace(x) / 3.0 * np.eye(3)


def expm_su3(x: np.ndarray) -> np.ndarray:
    """exp of an anti-Hermitian 3x3 via the Hermitian eigendecomposition of -iX."""
    w, v = np.linalg.eigh(-1j * x)
    return (v * np.exp(1j * w)[None, :]) @ v.conj().T


def plaquette_sum(dims, links: np.ndarray) -> float:
    """sum over x and mu < nu of Re tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag."""
    total = 0.0
    for mu in range(4):
        fm = shift_index(dims, mu, +1)
        for nu in range(mu + 1, 4):
            fn = shift_index(dims, nu, +1)
            for s in range(len(fm)):
                p = links[mu][s] @ links[nu][fm[s]] @ links[mu][fn[s]].conj().T @ links[nu][s].conj().T
                total += np.trace(p).real
    return total

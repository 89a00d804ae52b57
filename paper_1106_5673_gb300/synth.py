"""Seeded synthetic inputs: gauge fields and colour-vector sources.

These generators serve both the CUDA library's callers and the oracle's tests.
They hold none of the RHMC arithmetic: they only draw random SU(3) matrices
and Gaussian vectors with numpy, in the canonical layouts

  gauge   complex128 [4, V, 3, 3]   V in lexicographic order
          lex = x + Lx*(y + Ly*(z + Lz*t)), mu = 0..3 = x, y, z, t
  vector  complex128 [V/2, 3]       the sites of one parity, index lex // 2
"""
import numpy as np

_S3 = 1.0 / np.sqrt(3.0)


def volume(dims):
    return int(np.prod(dims))


def _gell_mann():
    g = np.zeros((8, 3, 3), np.complex128)
    g[0, 0, 1] = g[0, 1, 0] = 1
    g[1, 0, 1], g[1, 1, 0] = -1j, 1j
    g[2, 0, 0], g[2, 1, 1] = 1, -1
    g[3, 0, 2] = g[3, 2, 0] = 1
    g[4, 0, 2], g[4, 2, 0] = -1j, 1j
    g[5, 1, 2] = g[5, 2, 1] = 1
    g[6, 1, 2], g[6, 2, 1] = -1j, 1j
    g[7, 0, 0] = g[7, 1, 1] = _S3
    g[7, 2, 2] = -2 * _S3
    return g


def _expi_hermitian(H):
    """exp(i H) for a stack of Hermitian matrices via numpy's eigh."""
    lam, vec = np.linalg.eigh(H)
    ph = np.exp(1j * lam)
    return np.einsum("...ij,...j,...kj->...ik", vec, ph, vec.conj())


def near_unit_links(dims, scale, seed):
    """U = exp(i * scale * H), H = sum_a w^a lambda^a / 2 with w^a ~ N(0, 1).

    scale = 0.3 is the 4^4 trajectory start; scale = 0.2 gives the
    exp-of-Gaussian links with sigma 0.2 of the batched runs."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((4 * V, 8))
    H = np.einsum("na,aij->nij", w, _gell_mann()) * 0.5
    U = _expi_hermitian(scale * H)
    return np.ascontiguousarray(U.reshape(4, V, 3, 3))


def haar_links(dims, seed):
    """Haar-random SU(3) links: QR of a complex Ginibre matrix with the phases
    of R's diagonal moved into Q (Mezzadri 2007), divided by det^(1/3)."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((4 * V, 3, 3)) + 1j * rng.standard_normal((4 * V, 3, 3))) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=1, axis2=2)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    Q = Q / (det ** (1.0 / 3.0))[:, None, None]
    return np.ascontiguousarray(Q.reshape(4, V, 3, 3))


def unit_links(dims):
    V = volume(dims)
    U = np.zeros((4, V, 3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def gaussian_vector(dims, seed):
    """Complex Gaussian colour vector on one parity, density ~ exp(-|v|^2)."""
    Vh = volume(dims) // 2
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal((Vh, 3)) + 1j * rng.standard_normal((Vh, 3))) / np.sqrt(2)
    return np.ascontiguousarray(v)


def gaussian_momenta(dims, seed):
    """Gell-Mann coefficients w^a ~ N(0, 1), layout float64 [4, V, 8]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, volume(dims), 8))


def log_shifts(n, lo, hi):
    """n log-spaced shifts in [lo, hi]."""
    return np.exp(np.linspace(np.log(lo), np.log(hi), n))

"""Test-only helpers: gauge transformations and dense operator matrices.

Nothing here is part of the method; these are tools to state invariants."""
import numpy as np

from paper_1106_5673_gb300 import synth


def coords(dims, lex):
    Lx, Ly, Lz, Lt = dims
    x = lex % Lx
    y = (lex // Lx) % Ly
    z = (lex // (Lx * Ly)) % Lz
    t = lex // (Lx * Ly * Lz)
    return np.stack([x, y, z, t], -1)


def lex_of(dims, c):
    Lx, Ly, Lz, Lt = dims
    return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))


def parity_sites(dims, parity):
    V = int(np.prod(dims))
    lex = np.arange(V)
    c = coords(dims, lex)
    return lex[(c.sum(-1) % 2) == parity]


def gauge_transform(dims, U, g):
    """U_mu(n) -> g(n) U_mu(n) g(n+mu)^dag for g of shape [V, 3, 3]."""
    V = int(np.prod(dims))
    lex = np.arange(V)
    c = coords(dims, lex)
    out = np.empty_like(U)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        f = lex_of(dims, cf)
        out[mu] = g @ U[mu] @ g[f].conj().transpose(0, 2, 1)
    return out


def transform_vector(dims, g, v, parity):
    sites = parity_sites(dims, parity)
    return np.einsum("nij,nj->ni", g[sites], v)


def random_gauge(dims, seed):
    return synth.haar_links(dims, seed)[0]


def dense_operator(apply, n):
    """Matrix of a linear map on C^n given as apply(v: [n/3, 3]) -> same."""
    M = np.zeros((n, n), np.complex128)
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1
        M[:, j] = apply(e.reshape(-1, 3)).reshape(-1)
    return M


def free_field_even_spectrum(dims, mass):
    """Closed form: with U = 1, -D^2 is diagonal in momentum space with
    eigenvalue sum_mu sin^2 p_mu, p_mu = 2 pi k / L_mu (x, y, z periodic) and
    p_t = pi (2k+1) / L_t (antiperiodic).  Each value appears for 3 colours;
    the even-site block holds half of them (p and p + (pi,pi,pi,pi) pair up)."""
    ps = []
    for mu, L in enumerate(dims):
        k = np.arange(L)
        ps.append(np.pi * (2 * k + 1) / L if mu == 3 else 2 * np.pi * k / L)
    grids = np.meshgrid(*ps, indexing="ij")
    lam = sum(np.sin(g) ** 2 for g in grids).reshape(-1)
    full = np.sort(np.repeat(mass ** 2 + lam, 3))
    return full[::2]


def su3_check(U):
    """max deviation from unitarity and from det = 1 over a stack."""
    I = np.eye(3)
    un = np.abs(U @ U.conj().swapaxes(-1, -2) - I).max()
    de = np.abs(np.linalg.det(U) - 1).max()
    return un, de

"""Pins of the oracle's random numbers and of its Remez rational functions."""
import os

import numpy as np
import pytest

import oracle as O
from oracle import remez
from paper_1106_5673_gb300 import synth
from tests import helpers as H


# ---------------------------------------------------------------- Philox / Box-Muller

def _kat_vectors():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answer_vectors():
    """Philox4x32-10 reproduces the published known-answer vectors (Salmon et
    al., SC'11; the test vectors distributed with their Random123 library):
    a wrong multiplier, Weyl constant, word order or key schedule fails here."""
    rows = _kat_vectors()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert O.philox(ctr, key) == want, (ctr, key)


def _uniforms(n, key=(7, 9)):
    u = np.array([O.uniform_pair((5, 0, i, 0), key) for i in range(n)])
    return u.reshape(-1)


def test_uniforms_in_half_open_unit_interval_and_uniform():
    from scipy import stats
    u = _uniforms(20000)
    assert u.min() > 0 and u.max() <= 1
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # consecutive draws uncorrelated
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.03


def test_gaussians_standard_normal():
    from scipy import stats
    g = np.array([O.gauss_pair((1, 2, i, 3), (11, 0)) for i in range(20000)]).reshape(-1)
    assert stats.kstest(g, "norm").pvalue > 1e-3
    assert abs(g.mean()) < 0.03 and abs(g.var() - 1) < 0.03


def test_philox_avalanche_and_key_dependence():
    """Flipping one counter or key bit changes about half of the 128 output bits."""
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(300):
        c = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
        k = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        o = O.philox(c, k)
        j, b = int(rng.integers(0, 6)), int(rng.integers(0, 32))
        c2, k2 = list(c), list(k)
        if j < 4:
            c2[j] ^= 1 << b
        else:
            k2[j - 4] ^= 1 << b
        o2 = O.philox(c2, k2)
        flips.append(sum(bin(a ^ d).count("1") for a, d in zip(o, o2)))
    assert abs(np.mean(flips) - 64) < 2.0


def test_heatbath_distributions():
    dims = (4, 4, 4, 4)
    w = O.momenta_heatbath(dims, 3, 4)
    assert abs(w.mean()) < 0.02 and abs(w.var() - 1) < 0.02
    # kinetic term sum Tr P^2 averages 1/2 per Gell-Mann component
    assert abs(O.kinetic(dims, w) / w.size - 0.5) < 0.02
    R = O.pf_gaussian(dims, 3, 4, 0)
    parts = np.concatenate([R.real.reshape(-1), R.imag.reshape(-1)])
    assert abs(parts.var() - 0.5) < 0.05
    # different pseudofermion index, trajectory or seed -> different draws
    assert np.abs(R - O.pf_gaussian(dims, 3, 4, 1)).max() > 0.1
    assert np.abs(R - O.pf_gaussian(dims, 3, 5, 0)).max() > 0.1
    assert np.abs(w - O.momenta_heatbath(dims, 4, 4)).max() > 0.1


# ---------------------------------------------------------------- Remez rationals

def _dense_err(r, n=100000):
    x = np.exp(np.linspace(np.log(r["lo"]), np.log(r["hi"]), n))
    return x, remez.rational_eval(r["a0"], r["a"], r["b"], x) / x ** r["power"] - 1


def _alternation_count(e, E):
    """Length of the longest sign-alternating run of points with |e| ~ E."""
    idx = np.nonzero(np.abs(e) > 0.999 * E)[0]
    signs = np.sign(e[idx])
    # collapse consecutive equal signs (one extremum spans several grid points)
    runs = [signs[0]] + [s for prev, s in zip(signs[:-1], signs[1:]) if s != prev]
    return len(runs)


def test_golden_rationals_equioscillate(rationals):
    """Chebyshev alternation: the error reaches +-E at 2d+2 alternating points and
    never exceeds E on a dense grid, which characterises the minimax r."""
    for key, r in rationals.items():
        x, e = _dense_err(r)
        E = np.abs(e).max()
        assert E <= r["err"] * (1 + 1e-6) + 1e-14, key
        assert _alternation_count(e, r["err"]) >= 2 * r["degree"] + 2, key
        assert all(b > 0 for b in r["b"]), key      # poles on the negative real axis
        if r["power"] < 0:
            assert all(a > 0 for a in r["a"]), key  # Stieltjes function: positive residues


def test_remez_degree_zero_closed_form():
    """d = 0: the best constant c for x^p on [lo, hi] is 2 / (lo^-p + hi^-p)."""
    for p in (-0.5, 0.25):
        lo, hi = 0.01, 5.0
        r = remez.remez(p, lo, hi, 0, dps=30)
        c = 2.0 / (lo ** -p + hi ** -p)
        assert abs(r["a0"] - c) < 1e-14 * c
        assert abs(r["err"] - abs(c * lo ** -p - 1)) < 1e-12


def test_remez_scale_covariance():
    """If r is minimax for x^p on [lo, hi] then s^p r(x/s) is minimax on
    [s lo, s hi]: a0 -> s^p a0, b -> s b, a -> s^(p+1) a."""
    p, lo, hi, d, s = -0.5, 0.05, 20.0, 3, 7.0
    r1 = remez.remez(p, lo, hi, d, dps=40)
    r2 = remez.remez(p, s * lo, s * hi, d, dps=40)
    assert abs(r2["a0"] - s ** p * r1["a0"]) < 1e-10 * abs(r2["a0"])
    np.testing.assert_allclose(r2["b"], s * np.array(r1["b"]), rtol=1e-9)
    np.testing.assert_allclose(r2["a"], s ** (p + 1) * np.array(r1["a"]), rtol=1e-9)
    assert abs(r1["err"] - r2["err"]) < 1e-10


def test_rational_against_exact_matrix_power(rationals):
    """Brute force on 2^4: r(M_ee) phi against the exact M_ee^p phi from the
    dense eigendecomposition, within the rational's relative error bound."""
    dims, m = (2, 2, 2, 2), 0.1
    U = synth.near_unit_links(dims, 0.6, 40)
    phi = synth.gaussian_vector(dims, 41)
    n = 3 * synth.volume(dims) // 2
    M = H.dense_operator(lambda v: O.apply_M(dims, U, m, np.ascontiguousarray(v)), n)
    lam, V = np.linalg.eigh(M)
    assert lam.min() >= 1e-3 and lam.max() <= 64
    for key in ("p-1/2_d8_1e-3", "p+1/4_d8_1e-3"):
        r = rationals[key]
        exact = V @ (lam ** r["power"] * (V.conj().T @ phi.reshape(-1)))
        out, _ = O.rational_apply(dims, U, m, r["a0"], r["a"], r["b"], phi, tol=1e-14)
        err = np.linalg.norm(out.reshape(-1) - exact) / np.linalg.norm(exact)
        assert err <= r["err"] * 1.001, (key, err)
        assert err > 1e-3 * r["err"]  # the rational differs from the exact power

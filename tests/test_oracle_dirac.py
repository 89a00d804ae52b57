"""Pins of the oracle's staggered operator and solvers (CPU only).

Each test checks the oracle against something other than itself: a closed
form (free-field spectrum), a symmetry (anti-Hermiticity, gauge covariance),
or brute force (dense linear algebra on tiny lattices)."""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth
from tests import helpers as H


def test_free_field_spectrum_4x4x4x4():
    """Eq. (4) with U = 1: spec(M_ee) = {m^2 + sum_mu sin^2 p_mu} (antiperiodic t)."""
    dims, m = (4, 4, 4, 4), 0.1
    U = synth.unit_links(dims)
    n = 3 * synth.volume(dims) // 2
    M = H.dense_operator(lambda v: O.apply_M(dims, U, m, np.ascontiguousarray(v)), n)
    ev = np.linalg.eigvalsh(M)
    assert np.abs(M - M.conj().T).max() < 1e-14
    np.testing.assert_allclose(ev, H.free_field_even_spectrum(dims, m), rtol=0, atol=1e-12)


def test_free_field_spectrum_rectangular_and_gauge_covariant():
    """Same closed form on 2x4x2x6 after a random gauge transformation of U = 1."""
    dims, m = (2, 4, 2, 6), 0.3
    g = H.random_gauge(dims, 7)
    U = H.gauge_transform(dims, synth.unit_links(dims), g)
    n = 3 * synth.volume(dims) // 2
    M = H.dense_operator(lambda v: O.apply_M(dims, U, m, np.ascontiguousarray(v)), n)
    ev = np.linalg.eigvalsh(M)
    np.testing.assert_allclose(ev, H.free_field_even_spectrum(dims, m), rtol=0, atol=1e-12)


def test_periodic_time_would_fail_the_pin():
    """The pin distinguishes boundary conditions: a periodic-time spectrum
    (with zero modes) differs from the antiperiodic one the oracle gives."""
    dims, m = (2, 2, 2, 4), 0.1
    U = synth.unit_links(dims)
    n = 3 * synth.volume(dims) // 2
    ev = np.linalg.eigvalsh(H.dense_operator(
        lambda v: O.apply_M(dims, U, m, np.ascontiguousarray(v)), n))
    assert ev.min() > m * m + 0.1  # no near-zero modes with antiperiodic t


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 4), (6, 2, 2, 8)])
def test_anti_hermiticity(dims):
    """D^dag = -D: <chi_e, D_eo psi_o> = -<D_oe chi_e, psi_o>."""
    U = synth.haar_links(dims, 3)
    psi = synth.gaussian_vector(dims, 4)
    chi = synth.gaussian_vector(dims, 5)
    a = np.vdot(chi, O.dslash(dims, U, 0, psi))
    b = -np.vdot(O.dslash(dims, U, 1, chi), psi)
    assert abs(a - b) <= 1e-14 * abs(a) * 10


def test_full_operator_matches_parity_blocks():
    """The full-lattice D of Eq. (4) restricted to a parity equals D_eo / D_oe."""
    dims = (4, 2, 4, 4)
    U = synth.near_unit_links(dims, 0.5, 1)
    V = synth.volume(dims)
    ev, od = H.parity_sites(dims, 0), H.parity_sites(dims, 1)
    psi_o = synth.gaussian_vector(dims, 2)
    full = np.zeros((V, 3), np.complex128)
    full[od] = psi_o
    out = O.dslash_full(dims, U, full)
    np.testing.assert_allclose(out[ev], O.dslash(dims, U, 0, psi_o), atol=1e-14)
    assert np.abs(out[od]).max() == 0.0


def test_gauge_invariance_of_inverse_bilinear():
    """phi^dag M_ee^{-1} phi is unchanged under U -> g U g^dag, phi -> g phi."""
    dims, m = (4, 4, 4, 4), 0.2
    U = synth.near_unit_links(dims, 0.4, 11)
    phi = synth.gaussian_vector(dims, 12)
    g = H.random_gauge(dims, 13)
    Ug = H.gauge_transform(dims, U, g)
    phig = H.transform_vector(dims, g, phi, 0)
    x, _, st = O.cg(dims, U, m, 0.0, phi, tol=1e-13)
    xg, _, stg = O.cg(dims, Ug, m, 0.0, phig, tol=1e-13)
    assert st == 0 and stg == 0
    a, b = np.vdot(phi, x).real, np.vdot(phig, xg).real
    assert abs(a - b) < 1e-11 * abs(a)
    # the plaquette is invariant too
    assert abs(O.plaquette(dims, U) - O.plaquette(dims, Ug)) < 1e-14


def test_cg_against_dense_solve_2x2x2x2():
    """Brute force: CG on 2^4 equals numpy's dense solve of (M_ee + s) x = b."""
    dims, m, s = (2, 2, 2, 2), 0.05, 0.01
    U = synth.haar_links(dims, 21)
    b = synth.gaussian_vector(dims, 22)
    n = 3 * synth.volume(dims) // 2
    M = H.dense_operator(lambda v: O.apply_M(dims, U, m, np.ascontiguousarray(v)), n)
    xd = np.linalg.solve(M + s * np.eye(n), b.reshape(-1))
    x, it, st = O.cg(dims, U, m, s, b, tol=1e-14)
    assert st == 0
    np.testing.assert_allclose(x.reshape(-1), xd, rtol=0, atol=1e-10 * np.abs(xd).max())


def test_multishift_against_dense_and_true_residual():
    """Every shifted solution equals the dense solve and has a true residual
    below the requested tolerance."""
    dims, m = (4, 4, 4, 4), 0.05
    U = synth.haar_links(dims, 31)
    b = synth.gaussian_vector(dims, 32)
    shifts = synth.log_shifts(6, 1e-4, 1.0)
    tol = 1e-10
    xs, its, tot, st = O.multishift(dims, U, m, shifts, b, tol=tol)
    assert st == 0
    # the heavier shifts stop earlier
    assert its[-1] <= its[0] == tot
    bn = np.linalg.norm(b)
    for k, s in enumerate(shifts):
        r = b - O.apply_M(dims, U, m, np.ascontiguousarray(xs[k])) - s * xs[k]
        assert np.linalg.norm(r) / bn < 10 * tol
    # brute force on the lightest and heaviest shift
    n = 3 * synth.volume(dims) // 2
    M = H.dense_operator(lambda v: O.apply_M(dims, U, m, np.ascontiguousarray(v)), n)
    for k in (0, len(shifts) - 1):
        xd = np.linalg.solve(M + shifts[k] * np.eye(n), b.reshape(-1))
        np.testing.assert_allclose(xs[k].reshape(-1), xd, rtol=0,
                                   atol=1e-8 * np.abs(xd).max())


def test_multishift_one_step_closed_form():
    """For an eigenvector b of M_ee the base CG converges in one step and the
    shift recurrence gives zeta^1 = 1/(1 + alpha_0 d), i.e. every shifted
    solution is exactly b / (lambda + s) after one iteration."""
    dims, m = (2, 2, 2, 2), 0.1
    U = synth.unit_links(dims)
    n = 3 * synth.volume(dims) // 2
    M = H.dense_operator(lambda v: O.apply_M(dims, U, m, np.ascontiguousarray(v)), n)
    lam, vec = np.linalg.eigh(M)
    b = np.ascontiguousarray(vec[:, 0].reshape(-1, 3))
    shifts = np.array([0.0, 0.5, 2.0])
    xs, its, tot, st = O.multishift(dims, U, m, shifts, b, tol=1e-12)
    assert tot == 1
    for k, s in enumerate(shifts):
        np.testing.assert_allclose(xs[k], b / (lam[0] + s), atol=1e-13)


def test_all_cores_build_gives_identical_results(rationals):
    """The OpenMP build of the oracle (used only to time it on every host
    core) computes the same numbers bit for bit: only loops that write one
    output per site run in parallel, and the dot products stay serial."""
    import hashlib
    import os
    import subprocess
    import sys
    code = (
        "import hashlib, json, sys, numpy as np\n"
        "sys.path.insert(0, %r)\n"
        "import oracle as O\n"
        "from paper_1106_5673_gb300 import synth\n"
        "r = json.load(open(%r))['p-1/2_d6_1e-2']\n"
        "dims = (4, 4, 4, 6)\n"
        "U = synth.near_unit_links(dims, 0.3, 3)\n"
        "phi = synth.gaussian_vector(dims, 4)\n"
        "F, _, _ = O.fermion_force(dims, U, 0.2, r['a0'], r['a'], r['b'], phi, tol=1e-11)\n"
        "G = O.gauge_force(dims, U, 5.3)\n"
        "W = O.update_links(dims, U, G, 0.01)\n"
        "print(hashlib.sha256(F.tobytes() + G.tobytes() + W.tobytes()).hexdigest())\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
         os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json"))
    out = {}
    for omp in ("0", "1"):
        env = dict(os.environ, ORACLE_OPENMP=omp, OMP_NUM_THREADS="4")
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
        out[omp] = r.stdout.strip()
    assert len(out["0"]) == 64 and out["0"] == out["1"]

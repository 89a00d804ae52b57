"""Pins of the oracle's SU(3) algebra, forces and molecular dynamics (CPU).

Forces are pinned by directional finite differences of the actions they
derive from; the integrators by reversibility (Sec. 4.4: flip the momenta at
tau and integrate back) and by the eps^2 scaling of dH."""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth
from tests import helpers as H


def _herm(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    X = (A + A.conj().T) / 2
    X -= np.trace(X) / 3 * np.eye(3)
    return scale * X


@pytest.mark.parametrize("scale", [1e-3, 0.3, 2.0, 7.0])
def test_su3_exp_matches_eigendecomposition(scale):
    """exp(iX) (Taylor, scaling and squaring) = V exp(i Lambda) V^dag (numpy eigh)."""
    X = _herm(1, scale)
    lam, V = np.linalg.eigh(X)
    ref = (V * np.exp(1j * lam)) @ V.conj().T
    E = O.su3_exp_i(X)
    np.testing.assert_allclose(E, ref, atol=2e-14 * max(1, scale))
    un, de = H.su3_check(E[None])
    assert un < 1e-13 and de < 1e-13


def test_reunit_projects_to_su3_and_fixes_su3():
    U = synth.haar_links((2, 2, 2, 2), 3)[0, 0]
    np.testing.assert_allclose(O.reunit(U), U, atol=1e-14)
    pert = U + 1e-3 * (np.random.default_rng(1).standard_normal((3, 3)))
    R = O.reunit(pert)
    un, de = H.su3_check(R[None])
    assert un < 1e-14 and de < 1e-14
    # row 0 keeps its direction
    r0 = pert[0] / np.linalg.norm(pert[0])
    np.testing.assert_allclose(R[0], r0, atol=1e-15)


def test_gell_mann_basis():
    """Tr(T^a T^b) = delta_ab / 2 and the omega <-> matrix maps invert each other."""
    w = np.random.default_rng(2).standard_normal(8)
    P = O.omega_to_matrix(w)
    np.testing.assert_allclose(P, P.conj().T, atol=1e-15)
    assert abs(np.trace(P)) < 1e-15
    np.testing.assert_allclose(O.matrix_to_omega(P), w, atol=1e-14)
    np.testing.assert_allclose(np.trace(P @ P).real, 0.5 * (w ** 2).sum(), rtol=1e-14)
    dims = (2, 2, 2, 2)
    W = synth.gaussian_momenta(dims, 4)
    assert abs(O.kinetic(dims, W) - 0.5 * (W ** 2).sum()) < 1e-12 * (W ** 2).sum()


def test_plaquette_closed_forms():
    dims = (4, 4, 4, 4)
    assert abs(O.plaquette(dims, synth.unit_links(dims)) - 1.0) < 1e-15
    assert abs(O.gauge_action(dims, synth.unit_links(dims), 5.3)) < 1e-12
    # a constant abelian field U_x = exp(i a T3), others 1: plaquettes all 1
    U = synth.unit_links(dims)
    U[0] = np.diag(np.exp(1j * np.array([0.3, -0.3, 0.0])))
    assert abs(O.plaquette(dims, U) - 1.0) < 1e-15
    # Haar links: <Re Tr U_P / 3> = 0 within statistics
    Uh = synth.haar_links((8, 8, 8, 8), 5)
    assert abs(O.plaquette((8, 8, 8, 8), Uh)) < 0.01


def _fd_derivative(S, dims, U, X, h):
    """(S(exp(ihX)U) - S(exp(-ihX)U)) / 2h with X given as omega^a per link."""
    Up = O.update_links(dims, U, X, h)
    Um = O.update_links(dims, U, X, -h)
    return (S(Up) - S(Um)) / (2 * h)


def test_gauge_force_finite_difference():
    """dS_g/ds along U(s) = exp(isX)U equals -2 sum Tr(X dP/dtau) = -sum x.f."""
    dims, beta = (4, 4, 4, 4), 5.3
    U = synth.near_unit_links(dims, 0.4, 6)
    X = synth.gaussian_momenta(dims, 7)
    F = O.gauge_force(dims, U, beta)
    pred = -(X * F).sum()
    S = lambda u: O.gauge_action(dims, u, beta)  # noqa: E731
    d1 = _fd_derivative(S, dims, U, X, 1e-3)
    d2 = _fd_derivative(S, dims, U, X, 5e-4)
    rich = (4 * d2 - d1) / 3  # removes the O(h^2) term
    assert abs(rich - pred) < 1e-7 * abs(pred)


def test_fermion_force_finite_difference(rationals):
    """Same identity for S_f = phi^dag r(M_ee) phi with the r_{-1/2} rational."""
    dims, m = (4, 4, 4, 4), 0.2
    r = rationals["p-1/2_d6_1e-2"]
    U = synth.near_unit_links(dims, 0.3, 8)
    phi = synth.gaussian_vector(dims, 9)
    X = synth.gaussian_momenta(dims, 10)
    F, it, st = O.fermion_force(dims, U, m, r["a0"], r["a"], r["b"], phi, tol=1e-13)
    assert st == 0
    pred = -(X * F).sum()
    S = lambda u: O.fermion_action(dims, u, m, r["a0"], r["a"], r["b"], phi, tol=1e-13)  # noqa
    d1 = _fd_derivative(S, dims, U, X, 1e-3)
    d2 = _fd_derivative(S, dims, U, X, 5e-4)
    rich = (4 * d2 - d1) / 3
    assert abs(rich - pred) < 1e-6 * abs(pred)


def test_fermion_force_gauge_covariant(rationals):
    """Under U -> gUg^dag, phi -> g phi the force transforms as F -> g F g^dag."""
    dims, m = (4, 4, 4, 4), 0.3
    r = rationals["p-1/2_d4_1e-1"]
    U = synth.near_unit_links(dims, 0.3, 14)
    phi = synth.gaussian_vector(dims, 15)
    g = H.random_gauge(dims, 16)
    F, _, _ = O.fermion_force(dims, U, m, r["a0"], r["a"], r["b"], phi, tol=1e-13)
    Fg, _, _ = O.fermion_force(dims, H.gauge_transform(dims, U, g), m, r["a0"], r["a"], r["b"],
                               H.transform_vector(dims, g, phi, 0), tol=1e-13)
    V = synth.volume(dims)
    for mu in range(4):
        for n in (0, 5, V - 1):
            Pm = O.omega_to_matrix(F[mu, n])
            Pg = O.omega_to_matrix(Fg[mu, n])
            np.testing.assert_allclose(Pg, g[n] @ Pm @ g[n].conj().T, atol=1e-10)


def _params(rationals, **kw):
    r = rationals["p-1/2_d6_1e-2"]
    h = rationals["p+1/4_d6_1e-2"]
    base = dict(beta=5.3, mass=0.2, tau=0.5, nsteps=5, integrator=0,
                hb=(h["a0"], h["a"], h["b"]), act=(r["a0"], r["a"], r["b"]),
                force=(r["a0"], r["a"], r["b"]), tol_md=1e-13, tol_metro=1e-13)
    base.update(kw)
    return O.make_params(**base)


@pytest.mark.parametrize("integrator", [0, 1])
def test_md_reversibility(rationals, integrator):
    """Integrate to tau, flip P, integrate again: back to the start (Sec. 4.4,
    Delta C and Delta M per degree of freedom) to FP64 rounding."""
    dims = (2, 2, 2, 4)
    U = synth.near_unit_links(dims, 0.3, 17)
    W = synth.gaussian_momenta(dims, 18)
    phi = synth.gaussian_vector(dims, 19)[None]
    p = _params(rationals, integrator=integrator, nsteps=4)
    U1, W1, _, nf, st = O.md_integrate(dims, U, W, phi, p)
    assert st == 0 and nf == (5 if integrator == 0 else 9)
    U2, W2, _, _, _ = O.md_integrate(dims, U1, -W1, phi, p)
    dof = 4 * 8 * synth.volume(dims)
    dC = np.sqrt((np.abs(U - U2) ** 2).sum() / dof)
    dM = np.sqrt(((W + W2) ** 2).sum() / dof)
    assert np.abs(U1 - U).max() > 1e-2  # it moved
    assert dC < 1e-12 and dM < 1e-11


@pytest.mark.parametrize("integrator", [0, 1])
def test_dH_scales_as_eps_squared(rationals, integrator):
    """|dH| ~ eps^2 for both second-order integrators; Omelyan's error is smaller."""
    dims = (2, 2, 2, 4)
    U = synth.near_unit_links(dims, 0.3, 20)
    W = synth.gaussian_momenta(dims, 21)
    phi = synth.gaussian_vector(dims, 22)[None]
    dH = []
    for n in (4, 8, 16):
        p = _params(rationals, integrator=integrator, nsteps=n, tau=0.5)
        H0 = O.hamiltonian(dims, U, W, phi, p)
        U1, W1, _, _, _ = O.md_integrate(dims, U, W, phi, p)
        H1 = O.hamiltonian(dims, U1, W1, phi, p)
        dH.append(abs(H1 - H0))
    r1, r2 = dH[0] / dH[1], dH[1] / dH[2]
    assert 3.0 < r1 < 5.5 and 3.5 < r2 < 4.5, dH


def test_heatbath_start_action(rationals):
    """phi = r_{1/4}(M) R gives S_f = phi^dag r_{-1/2}(M) phi = R^dag R up to the
    rational errors (r_{1/4}^2 r_{-1/2} = 1 within their bounds)."""
    dims, m = (4, 4, 4, 4), 0.2
    U = synth.near_unit_links(dims, 0.3, 23)
    h, r = rationals["p+1/4_d8_1e-3"], rationals["p-1/2_d8_1e-3"]
    R = O.pf_gaussian(dims, 1, 2, 0)
    phi, _ = O.rational_apply(dims, U, m, h["a0"], h["a"], h["b"], R, tol=1e-13)
    S = O.fermion_action(dims, U, m, r["a0"], r["a"], r["b"], phi, tol=1e-13)
    RR = np.vdot(R, R).real
    bound = (2 * h["err"] + r["err"]) * 1.01 + 1e-12
    assert abs(S / RR - 1) < bound


@pytest.mark.parametrize("integrator", [0, 1])
def test_multistep_without_fermions_is_fine_gauge_integrator(rationals, integrator):
    """npf = 0: the fermion scheme's momentum updates vanish and the multi-step
    integrator is the single-scale one with nsteps * ngauge (leapfrog) or
    nsteps * 2 ngauge (2MN) gauge steps."""
    dims = (2, 2, 2, 4)
    U = synth.near_unit_links(dims, 0.3, 30)
    W = synth.gaussian_momenta(dims, 31)
    phi = np.zeros((1, 3 * synth.volume(dims) // 2), complex)
    ng, ns = 3, 2
    pm = _params(rationals, integrator=integrator, nsteps=ns, ngauge=ng, npf=0)
    fine = ns * ng * (1 if integrator == 0 else 2)
    ps = _params(rationals, integrator=integrator, nsteps=fine, npf=0)
    U1, W1, _, _, st1 = O.md_integrate(dims, U, W, phi, pm)
    U2, W2, _, _, st2 = O.md_integrate(dims, U, W, phi, ps)
    assert st1 == 0 and st2 == 0
    assert np.abs(U1 - U).max() > 1e-2
    assert np.abs(U1 - U2).max() < 1e-12 and np.abs(W1 - W2).max() < 1e-11


@pytest.mark.parametrize("integrator", [0, 1])
def test_multistep_at_zero_beta_is_single_scale(rationals, integrator):
    """beta = 0: the inner steps only move U, ngauge times by h/ngauge, which
    composes to one move by h; the result is the single-scale integrator."""
    dims = (2, 2, 2, 4)
    U = synth.near_unit_links(dims, 0.3, 32)
    W = synth.gaussian_momenta(dims, 33)
    phi = synth.gaussian_vector(dims, 34)[None]
    pm = _params(rationals, integrator=integrator, nsteps=3, ngauge=4, beta=0.0)
    ps = _params(rationals, integrator=integrator, nsteps=3, beta=0.0)
    U1, W1, _, nf1, _ = O.md_integrate(dims, U, W, phi, pm)
    U2, W2, _, nf2, _ = O.md_integrate(dims, U, W, phi, ps)
    assert nf1 == nf2
    assert np.abs(U1 - U2).max() < 1e-12 and np.abs(W1 - W2).max() < 1e-11


@pytest.mark.parametrize("integrator", [0, 1])
def test_multistep_reversible_and_second_order(rationals, integrator):
    dims = (2, 2, 2, 4)
    U = synth.near_unit_links(dims, 0.3, 35)
    W = synth.gaussian_momenta(dims, 36)
    phi = synth.gaussian_vector(dims, 37)[None]
    p = _params(rationals, integrator=integrator, nsteps=3, ngauge=2)
    U1, W1, _, _, st = O.md_integrate(dims, U, W, phi, p)
    U2, W2, _, _, _ = O.md_integrate(dims, U1, -W1, phi, p)
    assert st == 0
    assert np.abs(U - U2).max() < 1e-12 and np.abs(W + W2).max() < 1e-11
    dH = []
    for n in (4, 8, 16):
        p = _params(rationals, integrator=integrator, nsteps=n, ngauge=2)
        H0 = O.hamiltonian(dims, U, W, phi, p)
        U1, W1, _, _, _ = O.md_integrate(dims, U, W, phi, p)
        dH.append(abs(O.hamiltonian(dims, U1, W1, phi, p) - H0))
    r1, r2 = dH[0] / dH[1], dH[1] / dH[2]
    assert 3.0 < r1 < 5.5 and 3.5 < r2 < 4.5, dH

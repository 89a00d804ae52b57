"""Pins of the oracle's whole trajectory (Sec. 2.1, the Phi algorithm with
rooting): heatbath, Hamiltonian, molecular dynamics and the Metropolis test,
checked against the mathematics rather than against another implementation.

- Creutz's equality <exp(-dH)> = 1: for (U, P, phi) drawn from exp(-H) and an
  area-preserving, reversible integrator, exp(-dH) averages to one.  A wrong
  heatbath distribution, an H that is not the one the forces derive from, or
  a non-reversible integrator breaks it.
- H right after the heatbath: 1/2 sum w^2 + S_g + sum_pf R^dag R, since
  phi^dag r_{-1/2}(M) phi = R^dag r_{1/4}(M)^2 r_{-1/2}(M) R = R^dag R up to
  the rational approximations' errors.
- The accept rule u < exp(-dH), and the restoration of the links on reject.
"""
import numpy as np

import oracle as O
from paper_1106_5673_gb300 import synth

DIMS = (2, 2, 2, 4)


def _params(rationals, traj, tau=1.0, nsteps=8, npf=1, seed=21, beta=5.0, mass=0.2):
    r, h = rationals["p-1/2_d6_1e-2"], rationals["p+1/4_d6_1e-2"]
    act = (r["a0"], r["a"], r["b"])
    return O.make_params(beta, mass, tau, nsteps, 0, (h["a0"], h["a"], h["b"]), act, act, npf=npf,
                         tol_md=1e-12, tol_metro=1e-12, seed=seed, traj=traj)


def test_creutz_equality_exp_minus_dH_averages_to_one(rationals):
    """A Markov chain of 400 leapfrog trajectories (tau 1, 8 steps, so that dH
    fluctuates by ~0.4) on 2x2x2x4; after 50 thermalisation trajectories
    <exp(-dH)> over the other 350 equals 1 within 3 standard errors, and
    <dH> ~ Var(dH)/2 (the Gaussian-dH form of the same identity) holds
    within a loose factor.  Planting a factor sqrt(2) in the pseudofermion
    draw moves the average by ~6 standard errors."""
    U = synth.near_unit_links(DIMS, 0.3, 3)
    dH = []
    for t in range(400):
        U, info, st = O.trajectory(DIMS, U, _params(rationals, t))
        assert st == 0
        if t >= 50:
            dH.append(info["dH"])
    dH = np.array(dH)
    e = np.exp(-dH)
    se = e.std() / np.sqrt(len(e))
    assert dH.std() > 0.2  # the test has power only if dH fluctuates
    assert abs(e.mean() - 1.0) < 3 * se, (e.mean(), se)
    assert 0.3 < dH.mean() / (0.5 * dH.var()) < 3.0


def test_hamiltonian_after_heatbath(rationals):
    """H0 of a trajectory = 1/2 sum w^2 (the momenta of the same Philox key)
    + beta sum_P (1 - Re Tr U_P / 3) + sum_pf R_pf^dag R_pf, within the
    rational error bound (2 err_{1/4} + err_{-1/2}) R^dag R."""
    r, h = rationals["p-1/2_d6_1e-2"], rationals["p+1/4_d6_1e-2"]
    U = synth.near_unit_links((4, 4, 4, 4), 0.3, 5)
    for npf in (1, 2):
        p = _params(rationals, traj=7, npf=npf, nsteps=4)
        _, info, st = O.trajectory((4, 4, 4, 4), U, p)
        assert st == 0
        w = O.momenta_heatbath((4, 4, 4, 4), 21, 7)
        RR = sum(np.vdot(R, R).real for R in (O.pf_gaussian((4, 4, 4, 4), 21, 7, pf) for pf in range(npf)))
        H0 = 0.5 * (w ** 2).sum() + O.gauge_action((4, 4, 4, 4), U, 5.0) + RR
        bound = (2 * h["err"] + r["err"]) * 1.01 * RR + 1e-9 * abs(H0)
        assert abs(info["H0"] - H0) < bound, (npf, info["H0"] - H0, bound)
        assert abs(info["H1"] - info["H0"] - info["dH"]) < 1e-12 * abs(info["H0"])


def test_metropolis_accept_rule_and_reject_restores_links(rationals):
    """accepted == (u < exp(-dH)) with u the Philox uniform of (seed, traj);
    a rejected trajectory leaves the links exactly as they were, an accepted
    one moves them."""
    U = synth.near_unit_links(DIMS, 0.3, 9)
    seen = set()
    for t, nsteps in enumerate((16, 1, 1, 16, 2, 16)):
        p = _params(rationals, traj=t, nsteps=nsteps)
        U1, info, st = O.trajectory(DIMS, U, p)
        assert st == 0
        assert info["u"] == O.metro_uniform(21, t)
        assert info["accepted"] == int(info["u"] < np.exp(-info["dH"]))
        if info["accepted"]:
            assert np.abs(U1 - U).max() > 1e-3
        else:
            assert np.array_equal(U1, U)
        assert abs(info["plaq"] - O.plaquette(DIMS, U1)) < 1e-15
        seen.add(info["accepted"])
    assert seen == {0, 1}  # both branches exercised

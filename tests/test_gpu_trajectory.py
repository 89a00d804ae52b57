"""GPU parity of whole RHMC trajectories against the FP64 oracle.

The 4^4 workload: Wilson beta = 5.3, m = 0.1, links exp(i 0.3 H) (seed 0),
degree-8 rationals on [1e-3, 64], solver tolerance 1e-10, leapfrog tau = 1
with 10 steps.  FP64 mode must give the oracle's dH to 1e-8 absolute (the
solves stop at 1e-10 relative, both sides in FP64) and the same
accept/reject decision; mixed mode the same decision and dH to 1e-6.
"""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


def _rats(rationals, key):
    h = rationals["p+1/4_" + key]
    r = rationals["p-1/2_" + key]
    return (h["a0"], h["a"], h["b"]), (r["a0"], r["a"], r["b"])


def _run_both(S, rationals, dims, integrator, nsteps, tau, mode, seed_links=0, traj=0, beta=5.3,
              mass=0.1, key="d8_1e-3", ngauge=0, npf=1):
    hb, act = _rats(rationals, key)
    U = synth.near_unit_links(dims, 0.3, seed_links)
    po = O.make_params(beta, mass, tau, nsteps, integrator, hb, act, act, tol_md=1e-10,
                       tol_metro=1e-10, seed=11, traj=traj, ngauge=ngauge, npf=npf)
    Uo, io, st = O.trajectory(dims, U, po)
    assert st == 0
    L = S.Lattice(dims)
    L.load_gauge(U)
    pg = S.make_params(beta, mass, tau, nsteps, integrator, hb, act, act, tol_md=1e-10,
                       tol_metro=1e-10, mode_md=mode, mode_metro=mode, seed=11, traj=traj,
                       ngauge=ngauge, npf=npf)
    ig = L.md_trajectory(pg)
    return U, Uo, io, L.store_gauge(), ig


def test_trajectory_4x4x4x4_leapfrog_f64(S, rationals):
    U, Uo, io, Ug, ig = _run_both(S, rationals, (4, 4, 4, 4), 0, 10, 1.0, S.SOLVE_F64)
    assert ig["n_force"] == io["n_force"] == 11
    assert abs(ig["u"] - io["u"]) < 1e-15
    assert abs(ig["H0"] - io["H0"]) < 1e-8 * abs(io["H0"])
    assert abs(ig["dH"] - io["dH"]) < 1e-8
    assert ig["accepted"] == io["accepted"]
    assert np.abs(Ug - Uo).max() < 1e-9
    assert abs(ig["plaq"] - io["plaq"]) < 1e-12


def test_trajectory_4x4x4x4_leapfrog_mixed(S, rationals):
    U, Uo, io, Ug, ig = _run_both(S, rationals, (4, 4, 4, 4), 0, 10, 1.0, S.SOLVE_MIXED)
    assert abs(ig["dH"] - io["dH"]) < 1e-6 * max(1.0, abs(io["dH"]))
    assert ig["accepted"] == io["accepted"]
    assert np.abs(Ug - Uo).max() < 1e-6


@pytest.mark.parametrize("mode", [0, 1])
def test_trajectory_omelyan_rectangular(S, rationals, mode):
    """Omelyan 2MN on a 6x4x6x10 lattice (ragged last block), degree 6."""
    U, Uo, io, Ug, ig = _run_both(S, rationals, (6, 4, 6, 10), 1, 4, 0.5, mode, seed_links=3,
                                  traj=5, key="d6_1e-2", mass=0.2)
    assert ig["n_force"] == io["n_force"] == 9
    # mixed mode integrates with FP32 forces: the trajectory moves by ~1e-7
    # relative, so dH agrees to 1e-6 relative to max(1, |dH|)
    tol = 1e-8 if mode == 0 else 1e-6 * max(1.0, abs(io["dH"]))
    assert abs(ig["dH"] - io["dH"]) < tol
    assert ig["accepted"] == io["accepted"]


@pytest.mark.parametrize("mode", [0, 1])
def test_trajectory_two_pseudofermions(S, rationals, mode):
    """N_pf = 2 (Sec. 2.1's multiple pseudofermions): the force solves both
    pseudofermions in one batched multi-system solve."""
    dims = (4, 4, 4, 4)
    h, r = rationals["p+1/4_d6_1e-2"], rationals["p-1/2_d6_1e-2"]
    hb, act = (h["a0"], h["a"], h["b"]), (r["a0"], r["a"], r["b"])
    U = synth.near_unit_links(dims, 0.3, 9)
    po = O.make_params(5.3, 0.2, 0.5, 4, 1, hb, act, act, npf=2, tol_md=1e-10, tol_metro=1e-10,
                       seed=4, traj=2)
    Uo, io, st = O.trajectory(dims, U, po)
    L = S.Lattice(dims)
    L.load_gauge(U)
    pg = S.make_params(5.3, 0.2, 0.5, 4, 1, hb, act, act, npf=2, tol_md=1e-10, tol_metro=1e-10,
                       mode_md=mode, mode_metro=mode, seed=4, traj=2)
    ig = L.md_trajectory(pg)
    # mixed mode: FP32 gauge force and, for N_pf > 1, the batched multi-system
    # solver; the MD moves by ~2^-24 |F| per step and dH by ~1e-6 relative
    tol = 1e-8 if mode == 0 else 5e-6 * max(1.0, abs(io["dH"]))
    assert abs(ig["dH"] - io["dH"]) < tol
    assert ig["accepted"] == io["accepted"]


def test_trajectory_rejection_restores_links(S, rationals):
    """A far too coarse integrator (1 step, tau = 2) is rejected: links restored."""
    dims = (4, 4, 4, 4)
    hb, act = _rats(rationals, "d8_1e-3")
    U = synth.near_unit_links(dims, 0.3, 0)
    L = S.Lattice(dims)
    L.load_gauge(U)
    p = S.make_params(5.3, 0.1, 2.0, 1, 0, hb, act, act, seed=3, traj=1)
    info = L.md_trajectory(p)
    assert info["dH"] > 5 and not info["accepted"]
    np.testing.assert_allclose(L.store_gauge(), U, atol=2e-15)


@pytest.mark.parametrize("integrator", [0, 1])
def test_trajectory_multistep_f64(S, rationals, integrator):
    """Multi-step scheme (gauge force on a finer time scale, 3 inner steps per
    position update): FP64 dH and links as the oracle's."""
    U, Uo, io, Ug, ig = _run_both(S, rationals, (4, 4, 4, 4), integrator, 4, 1.0, S.SOLVE_F64,
                                  seed_links=2, traj=3, ngauge=3)
    assert ig["n_force"] == io["n_force"] == (5 if integrator == 0 else 9)
    assert abs(ig["dH"] - io["dH"]) < 1e-8
    assert ig["accepted"] == io["accepted"]
    assert np.abs(Ug - Uo).max() < 1e-9


@pytest.mark.parametrize("integrator,nsteps", [(0, 40), (1, 8)])
def test_trajectory_pure_gauge(S, rationals, integrator, nsteps):
    """npf = 0: pure-gauge HMC (used to thermalise start configurations); an
    accepted trajectory, so the moved links are compared."""
    U, Uo, io, Ug, ig = _run_both(S, rationals, (6, 4, 6, 10), integrator, nsteps, 0.25, S.SOLVE_F64,
                                  seed_links=4, traj=7, npf=0, beta=5.5)
    assert ig["cg_iters"] == 0 and io["cg_iters"] == 0 and io["accepted"] == 1
    assert abs(ig["dH"] - io["dH"]) < 1e-9
    assert ig["accepted"] == io["accepted"]
    assert np.abs(Ug - Uo).max() < 1e-11


def test_no_metropolis_keeps_the_md_result(S, rationals):
    """no_metropolis = 1 (thermalisation): a trajectory the oracle rejects is
    kept, and the links are the oracle's molecular-dynamics result from the
    same heatbath momenta."""
    dims = (6, 4, 6, 10)
    hb, act = _rats(rationals, "d8_1e-3")
    U = synth.near_unit_links(dims, 0.3, 4)
    po = O.make_params(5.5, 0.1, 1.0, 5, 1, hb, act, act, npf=0, seed=11, traj=7)
    _, io, _ = O.trajectory(dims, U, po)
    assert io["accepted"] == 0
    W = O.momenta_heatbath(dims, 11, 7)
    Um, _, _, _, st = O.md_integrate(dims, U, W, np.zeros((1, 3 * synth.volume(dims) // 2), complex), po)
    L = S.Lattice(dims)
    L.load_gauge(U)
    ig = L.md_trajectory(S.make_params(5.5, 0.1, 1.0, 5, 1, hb, act, act, npf=0, seed=11, traj=7,
                                       no_metropolis=1))
    assert ig["accepted"] == 1 and abs(ig["dH"] - io["dH"]) < 1e-8
    assert np.abs(L.store_gauge() - Um).max() < 1e-11


def _md_params(S, rationals, mode, integrator=1, nsteps=4, tau=0.5, ngauge=0, oracle=False):
    hb, act = _rats(rationals, "d6_1e-2")
    mk = O.make_params if oracle else S.make_params
    kw = dict(tol_md=1e-12, tol_metro=1e-12, ngauge=ngauge)
    if not oracle:
        kw.update(mode_md=mode, mode_metro=mode)
    return mk(5.3, 0.2, tau, nsteps, integrator, hb, act, act, **kw)


@pytest.mark.parametrize("ngauge", [0, 2])
def test_md_integrate_matches_oracle(S, rationals, ngauge):
    """Molecular dynamics alone from given links, momenta and pseudofermion:
    links and momenta as the oracle's (FP64)."""
    dims = (4, 4, 4, 4)
    U = synth.near_unit_links(dims, 0.3, 12)
    W = synth.gaussian_momenta(dims, 13)
    phi = synth.gaussian_vector(dims, 14)[None]
    L = S.Lattice(dims)
    L.load_gauge(U)
    L.load_momenta(W)
    it, nf = L.md_integrate(_md_params(S, rationals, S.SOLVE_F64, ngauge=ngauge),
                            torch.from_numpy(np.ascontiguousarray(phi)).cuda())
    Uo, Wo, ito, nfo, st = O.md_integrate(dims, U, W, phi, _md_params(S, rationals, 0, ngauge=ngauge, oracle=True))
    assert st == 0 and nf == nfo == 9
    assert np.abs(L.store_gauge() - Uo).max() < 1e-10
    assert np.abs(L.store_momenta() - Wo).max() < 1e-9


def test_md_reversibility_fp64_and_mixed(S, rationals):
    """Sec. 4.4: integrate to tau, flip the momenta, integrate back.  FP64:
    back to the start to rounding; mixed (FP32 gauge force): a small, larger
    violation, as the paper reports for single-precision gauge updates."""
    dims = (6, 4, 6, 10)
    U = synth.near_unit_links(dims, 0.3, 15)
    W = synth.gaussian_momenta(dims, 16)
    phi = torch.from_numpy(np.ascontiguousarray(synth.gaussian_vector(dims, 17)[None])).cuda()
    dof = 4 * 8 * synth.volume(dims)
    dC = {}
    for mode in (S.SOLVE_F64, S.SOLVE_MIXED):
        L = S.Lattice(dims)
        L.load_gauge(U)
        L.load_momenta(W)
        p = _md_params(S, rationals, mode)
        L.md_integrate(p, phi)
        assert np.abs(L.store_gauge() - U).max() > 1e-2  # it moved
        L.load_momenta(-L.store_momenta())
        L.md_integrate(p, phi)
        dC[mode] = np.sqrt((np.abs(L.store_gauge() - U) ** 2).sum() / dof)
        dM = np.sqrt(((L.store_momenta() + W) ** 2).sum() / dof)
        if mode == S.SOLVE_F64:
            assert dC[mode] < 1e-12 and dM < 1e-11
        else:
            assert dC[mode] < 1e-5 and dM < 1e-4
    assert dC[S.SOLVE_MIXED] > dC[S.SOLVE_F64]


FULL = (32, 32, 32, 8)


@pytest.fixture(scope="module")
def full_size_oracle(S):
    """The oracle's trajectory at the bench's lattice, mass and rationals
    (degree 15 on [1e-5, 64]): one short leapfrog step (tau 0.005) from the
    smooth start (its solves on the smooth field take seconds)."""
    a = S.remez(-0.5, 1e-5, 64.0, 15)[:3]
    h = S.remez(0.25, 1e-5, 64.0, 15)[:3]
    U = synth.near_unit_links(FULL, 0.3, 1)
    po = O.make_params(5.5, 0.0075, 0.005, 1, 0, h, a, a, tol_md=1e-10, tol_metro=1e-10, seed=3, traj=4)
    Uo, io, st = O.trajectory(FULL, U, po)
    assert st == 0 and io["accepted"] == 1  # a step short enough to be kept: the links moved
    return a, h, U, Uo, io


def test_trajectory_full_size_32x32x32x8_f64(S, full_size_oracle):
    """FP64 mode at full size: heatbath, actions, forces, updates and the
    Metropolis decision against the oracle."""
    a, h, U, Uo, io = full_size_oracle
    L = S.Lattice(FULL)
    L.load_gauge(U)
    ig = L.md_trajectory(S.make_params(5.5, 0.0075, 0.005, 1, 0, h, a, a, tol_md=1e-10, tol_metro=1e-10,
                                       mode_md=S.SOLVE_F64, mode_metro=S.SOLVE_F64, seed=3, traj=4))
    assert ig["accepted"] == io["accepted"]
    assert abs(ig["H0"] - io["H0"]) < 1e-10 * abs(io["H0"])
    assert abs(ig["dH"] - io["dH"]) < 1e-6
    assert np.abs(L.store_gauge() - Uo).max() < 1e-10


def test_trajectory_full_size_32x32x32x8_mixed(S, full_size_oracle):
    """The bench's mode (FP32 shifted CG, batched refinement, FP32 gauge
    force; every solve 1e-10 FP64-accurate) at full size against the oracle:
    the same accept decision, H0 to 1e-9 relative (the heatbath and action
    solves meet 1e-10 by another path than the oracle's, as on 16^3 x 4),
    dH within the mixed tolerance 1e-7 sqrt(N_dof) with N_dof = 32 V, and
    links within 1e-7."""
    a, h, U, Uo, io = full_size_oracle
    L = S.Lattice(FULL)
    L.load_gauge(U)
    ig = L.md_trajectory(S.make_params(5.5, 0.0075, 0.005, 1, 0, h, a, a, tol_md=1e-10, tol_metro=1e-10,
                                       mode_md=S.SOLVE_MIXED, mode_metro=S.SOLVE_MIXED, seed=3, traj=4))
    assert ig["accepted"] == io["accepted"]
    assert abs(ig["H0"] - io["H0"]) < 1e-9 * abs(io["H0"])
    assert abs(ig["dH"] - io["dH"]) < 1e-7 * np.sqrt(32 * np.prod(FULL))
    assert np.abs(L.store_gauge() - Uo).max() < 1e-7

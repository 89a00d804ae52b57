"""GPU trajectories and solves on the mid-size 16^3 x 4 lattice against the
FP64 oracle, and the trajectory's chain properties.

- One trajectory (Omelyan 2MN, tau 0.2, 8 steps, beta 5.5, m 0.1, degree-8
  rationals on [1e-3, 64], every solve to 1e-10) in FP64, float-float and
  mixed mode against the oracle's trajectory from the same start and Philox
  key.  FP64-accurate modes must give dH to 1e-8 absolute.  Mixed mode
  integrates with the FP32 gauge force: each of its ~N_dof = 32 V momentum
  components moves by ~2^-24 of its force per step, independently, so dH
  differs from FP64's by a random walk of size ~1e-7 sqrt(N_dof); that is the
  mixed tolerance (7e-5 here), with the same accept decision.
- The solver configuration of the 16^3 x 4 solver workload as stated: Haar
  links, m 0.05, 16 log-spaced shifts in [1e-4, 1], FP64 and mixed (FP32
  with FP64 reliable updates) against the oracle's shifted CG, both to 1e-10.
- CUDA graphs on or off (stag_params.use_graphs) give identical results.
- A chain stopped after a trajectory, stored (stag_store_gauge) and resumed in
  a new context from the next trajectory index continues as the
  uninterrupted chain.
"""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16, 4)


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


def _rats(rationals):
    h, r = rationals["p+1/4_d8_1e-3"], rationals["p-1/2_d8_1e-3"]
    return (h["a0"], h["a"], h["b"]), (r["a0"], r["a"], r["b"])


@pytest.fixture(scope="module")
def oracle_traj(rationals):
    hb, act = _rats(rationals)
    U = synth.near_unit_links(DIMS, 0.3, 2)
    p = O.make_params(5.5, 0.1, 0.2, 8, 1, hb, act, act, tol_md=1e-10, tol_metro=1e-10, seed=12, traj=3)
    Uo, io, st = O.trajectory(DIMS, U, p)
    assert st == 0
    return U, Uo, io


@pytest.mark.parametrize("mode", [0, 3, 1])
def test_trajectory_16x16x16x4_against_oracle(S, rationals, oracle_traj, mode):
    U, Uo, io = oracle_traj
    hb, act = _rats(rationals)
    L = S.Lattice(DIMS)
    L.load_gauge(U)
    p = S.make_params(5.5, 0.1, 0.2, 8, S.INT_OMELYAN, hb, act, act, tol_md=1e-10, tol_metro=1e-10,
                      mode_md=mode, mode_metro=mode, seed=12, traj=3)
    ig = L.md_trajectory(p)
    assert ig["n_force"] == io["n_force"] == 17
    assert ig["u"] == io["u"]
    ndof = 32 * L.V
    tol = 1e-8 if mode in (0, 3) else 1e-7 * np.sqrt(ndof)
    assert abs(ig["dH"] - io["dH"]) < tol, (mode, ig["dH"], io["dH"])
    assert abs(ig["H0"] - io["H0"]) < 1e-9 * abs(io["H0"])
    assert ig["accepted"] == io["accepted"]
    if mode in (0, 3):
        assert np.abs(L.store_gauge() - Uo).max() < 1e-9
    L.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_multishift_16x16x16x4_haar_16_shifts(S, mode):
    """The solver workload as stated: FP32 + FP64 reliable updates (mode 1)
    and FP64 (mode 0), every shift to 1e-10 in the oracle's own FP64
    residual, solutions within tol x cond of the oracle's."""
    m, tol = 0.05, 1e-10
    U = synth.haar_links(DIMS, 31)
    b = synth.gaussian_vector(DIMS, 32)
    shifts = synth.log_shifts(16, 1e-4, 1.0)
    L = S.Lattice(DIMS)
    L.load_gauge(U)
    sols, info = L.multishift_solve(m, shifts, torch.from_numpy(b).cuda(), tol=tol, mode=mode)
    assert info.status == 0
    xo, _, tot, st = O.multishift(DIMS, U, m, shifts, b, tol=1e-12)
    assert st == 0
    torch.cuda.synchronize()
    for k in range(16):
        x = sols[k].cpu().numpy()
        r = b - O.apply_M(DIMS, U, m, np.ascontiguousarray(x)) - shifts[k] * x
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01 * tol, k
        assert info.true_resid[k] <= tol
        cond = (m * m + 16 + shifts[k]) / (m * m + shifts[k])
        assert np.linalg.norm(x - xo[k]) / np.linalg.norm(xo[k]) < 2 * tol * cond, k
    L.close()


def test_graphs_on_and_off_give_identical_trajectories(S, rationals):
    dims = (8, 8, 8, 8)
    hb, act = _rats(rationals)
    U = synth.near_unit_links(dims, 0.3, 4)
    out = []
    for graphs in (1, 0):
        L = S.Lattice(dims)
        L.load_gauge(U)
        p = S.make_params(5.3, 0.1, 0.5, 5, S.INT_OMELYAN, hb, act, act, mode_md=S.SOLVE_MIXED,
                          mode_metro=S.SOLVE_MIXED, seed=5, traj=1, use_graphs=graphs)
        info = L.md_trajectory(p)
        out.append((info["dH"], info["accepted"], info["cg_iters"], L.store_gauge()))
        L.close()
    (d1, a1, i1, U1), (d2, a2, i2, U2) = out
    assert d1 == d2 and a1 == a2 and i1 == i2
    assert np.array_equal(U1, U2)


def test_chain_resumed_from_stored_links_continues_the_chain(S, rationals):
    """Trajectories 0, 1, 2 in one context, against trajectory 0 in one
    context, links stored to the host, and trajectories 1, 2 in a new context
    loaded from them (the Philox key is (seed, trajectory index), so the
    index is the whole RNG state)."""
    dims = (8, 8, 8, 8)
    hb, act = _rats(rationals)
    U = synth.near_unit_links(dims, 0.3, 6)

    def params(traj):
        return S.make_params(5.3, 0.1, 0.5, 5, S.INT_OMELYAN, hb, act, act, seed=8, traj=traj,
                             mode_md=S.SOLVE_MIXED, mode_metro=S.SOLVE_MIXED)

    L = S.Lattice(dims)
    L.load_gauge(U)
    full = [L.md_trajectory(params(t)) for t in range(3)]
    U_full = L.store_gauge()
    L.close()
    A = S.Lattice(dims)
    A.load_gauge(U)
    first = A.md_trajectory(params(0))
    saved = A.store_gauge()
    A.close()
    B = S.Lattice(dims)
    B.load_gauge(saved)
    rest = [B.md_trajectory(params(t)) for t in (1, 2)]
    U_resumed = B.store_gauge()
    B.close()
    for a, b in zip(full, [first] + rest):
        assert a["accepted"] == b["accepted"]
        assert abs(a["dH"] - b["dH"]) < 1e-8
    assert np.abs(U_full - U_resumed).max() < 1e-10

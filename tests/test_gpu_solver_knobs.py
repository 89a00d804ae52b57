"""The solver's launch-shape switches change how the mixed solve's kernels
are laid out, never what they compute: with each setting the 16-shift solve
on 16^3 x 4 Haar links (m 0.05, shifts log-spaced in [1e-4, 1], tol 1e-10)
meets every shift's tolerance in the oracle's own FP64 residual and agrees
with the oracle's shifted CG (Eq. (13)) within tol x cond.

Switches (read when a solver chunk's CUDA graph is captured):
- STAG_CD_GROUP: shifts whose loads the shifted CG's vector update issues
  together (1, 2, 4);
- STAG_CD_BPS: that kernel's blocks per SM (0: one float4 per thread);
- STAG_BCD_BPS: the refinement's vector-update blocks per SM over all rows
  (0: one block per SM per right-hand side);
- STAG_REFINE_NR: right-hand sides per thread in the refinement's hops
  (0 four, 1 by active count, 2 one, 3 at most two);
- STAG_MS_KEEP: unconverged shifts at which the FP32 shifted CG stops and
  leaves them to the refinement;
- STAG_EARLY_REFINE: converged shifts start their refinement on a second
  stream while the FP32 shifted CG goes on.
"""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16, 4)
MASS, TOL = 0.05, 1e-10


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


@pytest.fixture(scope="module")
def problem():
    U = synth.haar_links(DIMS, 41)
    b = synth.gaussian_vector(DIMS, 42)
    shifts = synth.log_shifts(16, 1e-4, 1.0)
    xo, _, _, st = O.multishift(DIMS, U, MASS, shifts, b, tol=1e-12)
    assert st == 0
    return U, b, shifts, xo


@pytest.mark.parametrize("env", [
    {"STAG_CD_GROUP": "2"},
    {"STAG_CD_GROUP": "4"},
    {"STAG_CD_BPS": "4"},
    {"STAG_BCD_BPS": "0"},
    {"STAG_REFINE_NR": "0"},
    {"STAG_REFINE_NR": "2"},
    {"STAG_REFINE_NR": "3"},
    {"STAG_MS_KEEP": "3"},
    {"STAG_EARLY_REFINE": "1"},
    {"STAG_EARLY_REFINE": "1", "STAG_REFINE_NR": "0"},
], ids=lambda e: ",".join("%s=%s" % kv for kv in e.items()))
def test_mixed_solve_with_launch_switch(S, problem, monkeypatch, env):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    U, b, shifts, xo = problem
    L = S.Lattice(DIMS)
    L.load_gauge(U)
    sols, info = L.multishift_solve(MASS, shifts, torch.from_numpy(b).cuda(), tol=TOL, mode=S.SOLVE_MIXED)
    assert info.status == 0
    torch.cuda.synchronize()
    for k in range(len(shifts)):
        x = sols[k].cpu().numpy()
        r = b - O.apply_M(DIMS, U, MASS, np.ascontiguousarray(x)) - shifts[k] * x
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01 * TOL, k
        assert info.true_resid[k] <= TOL
        cond = (MASS * MASS + 16 + shifts[k]) / (MASS * MASS + shifts[k])
        assert np.linalg.norm(x - xo[k]) / np.linalg.norm(xo[k]) < 2 * TOL * cond, k
    L.close()

"""GPU edge cases and full-size checks: zero sources, the smallest lattice
(2^4, where +mu and -mu neighbours coincide), the maximum number of shifts,
argument bounds, and the bench's 32^3x8 multi-shift solve and fermion force
against the oracle at full size."""
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


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_zero_source_gives_zero_solutions(S, mode):
    dims = (4, 4, 4, 4)
    L = S.Lattice(dims)
    L.load_gauge(synth.haar_links(dims, 1))
    b = L.vector()
    sols, info = L.multishift_solve(0.1, [0.0, 0.01, 1.0], b, tol=1e-10, mode=mode)
    assert info.status == 0 and info.iters == 0
    for x in sols:
        assert not np.any(host(x))


def test_smallest_lattice_2x2x2x2(S):
    """L = 2 in every direction: each site's forward and backward neighbour
    is the same site."""
    dims = (2, 2, 2, 2)
    U = synth.haar_links(dims, 3)
    L = S.Lattice(dims)
    L.load_gauge(U)
    for par in (0, 1):
        x = synth.gaussian_vector(dims, 4 + par)
        out = L.vector()
        (L.apply_deo if par == 0 else L.apply_doe)(dev(x), out)
        assert rel(host(out), O.dslash(dims, U, par, x)) < 1e-13
    b = synth.gaussian_vector(dims, 6)
    shifts = [0.0, 0.3]
    xo, _, _, _ = O.multishift(dims, U, 0.2, shifts, b, tol=1e-13)
    for mode in (0, 1):
        sols, info = L.multishift_solve(0.2, shifts, dev(b), tol=1e-11, mode=mode)
        assert info.status == 0
        for k in range(2):
            assert rel(host(sols[k]), xo[k]) < 1e-9


def test_maximum_number_of_shifts(S):
    dims = (4, 4, 4, 6)
    U = synth.haar_links(dims, 7)
    L = S.Lattice(dims)
    L.load_gauge(U)
    b = synth.gaussian_vector(dims, 8)
    shifts = synth.log_shifts(S.MAXSHIFT, 1e-3, 10.0)
    sols, info = L.multishift_solve(0.05, shifts, dev(b), tol=1e-10, mode=S.SOLVE_MIXED)
    assert info.status == 0 and max(info.true_resid[:S.MAXSHIFT]) <= 1e-10
    xo, _, _, _ = O.multishift(dims, U, 0.05, shifts, b, tol=1e-12)
    for k in (0, S.MAXSHIFT // 2, S.MAXSHIFT - 1):
        assert rel(host(sols[k]), xo[k]) < 1e-7
    with pytest.raises(S.StagError) as e:
        L.multishift_solve(0.05, list(shifts) + [20.0], dev(b))
    assert e.value.code == S.ERR_ARG
    with pytest.raises(S.StagError) as e:
        L.multishift_solve(0.05, [-1.0], dev(b))
    assert e.value.code == S.ERR_ARG


def test_full_size_multishift_and_force_32x32x32x8(S):
    """The bench's lattice, rational (degree 15 on [1e-5, 64]) and mass, in the
    mixed mode the bench times: every solution and the fermion force against
    the oracle (smooth start, so the oracle's solve takes seconds)."""
    dims, m = (32, 32, 32, 8), 0.0075
    U = synth.near_unit_links(dims, 0.3, 1)
    a0, a, b, _ = S.remez(-0.5, 1e-5, 64.0, 15)
    phi = synth.gaussian_vector(dims, 11)
    L = S.Lattice(dims)
    L.load_gauge(U)
    sols, info = L.multishift_solve(m, b, dev(phi), tol=1e-10, mode=S.SOLVE_MIXED)
    assert info.status == 0 and max(info.true_resid[:15]) <= 1e-10
    xo, _, _, st = O.multishift(dims, U, m, b, phi, tol=1e-11)
    assert st == 0
    for k in range(15):
        assert rel(host(sols[k]), xo[k]) < 1e-8
    F, _ = L.fermion_force(m, (a0, a, b), dev(phi), tol=1e-10, mode=S.SOLVE_MIXED)
    Fo, _, _ = O.fermion_force(dims, U, m, a0, a, b, phi, tol=1e-11)
    assert rel(host(F), Fo) < 1e-8

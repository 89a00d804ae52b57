"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (relative, in the 2-norm of the compared field unless stated):
  FP64 operator, forces, updates   1e-12  (only the order of FP64 roundings differs)
  FP32 operator                    2e-6   (FP32 storage and accumulation: ~10 ulp)
  BF16 links, FP32 vectors         2e-2   (8-bit mantissa links: 2^-8 relative per entry)
  solves                           the solver tolerance: every shift's FP64 true
                                   residual <= tol, solutions within tol * cond
"""
import numpy as np
import pytest

import oracle as O
from paper_1106_5673_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# 8^4: Vh = 2048 spans 16 blocks of 128; 6x4x6x10: Vh = 720, a ragged last block
SHAPES = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 6, 10)]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm((a - b).reshape(-1)) / max(np.linalg.norm(b.reshape(-1)), 1e-300)


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("dims", SHAPES)
def test_dslash_f64(S, dims):
    U = synth.haar_links(dims, 1)
    L = S.Lattice(dims)
    L.load_gauge(U)
    for par_out in (0, 1):
        x = synth.gaussian_vector(dims, 2 + par_out)
        out = L.vector()
        (L.apply_deo if par_out == 0 else L.apply_doe)(dev(x), out)
        assert rel(host(out), O.dslash(dims, U, par_out, x)) < 1e-13


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("prec,tol", [(1, 2e-6), (2, 2e-2)])
def test_dslash_low_precision(S, dims, prec, tol):
    U = synth.near_unit_links(dims, 0.5, 4)
    L = S.Lattice(dims)
    L.load_gauge(U)
    x = synth.gaussian_vector(dims, 5)
    out = L.vector(prec)
    L.apply_doe(dev(x, torch.complex64), out, prec)
    ref = O.dslash(dims, U, 1, x)
    err = rel(host(out), ref)
    assert err < tol
    if prec == 2:
        assert err > 1e-5  # bf16 links really are used


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("links", ["near_unit", "haar"])
def test_dslash_8_real_links(S, dims, links):
    """FP32 hop with 8-real links (Sec. 4.2's minimal parametrisation): the
    rebuilt links are SU(3) to FP32 rounding amplified by 1/N in the two
    cofactor divisions (N = |a1|^2 + |a2|^2; a few 1e-6 for Haar links), so
    the operator agrees with the FP64 oracle to 1e-5 relative.  After a link
    update the 8-real copy is rebuilt (the second comparison)."""
    U = synth.near_unit_links(dims, 0.5, 4) if links == "near_unit" else synth.haar_links(dims, 44)
    L = S.Lattice(dims)
    L.load_gauge(U)
    x = synth.gaussian_vector(dims, 5)
    for par_out, fn in ((1, L.apply_doe), (0, L.apply_deo)):
        out = L.vector(S.PREC_F32R8)
        fn(dev(x, torch.complex64), out, S.PREC_F32R8)
        assert rel(host(out), O.dslash(dims, U, par_out, x)) < 1e-5
    w = synth.gaussian_momenta(dims, 45)
    L.load_momenta(w)
    L.update_links(0.05)
    U2 = L.store_gauge()
    out = L.vector(S.PREC_F32R8)
    L.apply_doe(dev(x, torch.complex64), out, S.PREC_F32R8)
    assert rel(host(out), O.dslash(dims, U2, 1, x)) < 1e-5
    y = L.vector(S.PREC_F32R8)
    L.apply_M(0.1, dev(x, torch.complex64), y, S.PREC_F32R8)
    assert rel(host(y), O.apply_M(dims, U2, 0.1, x)) < 1e-5


@pytest.mark.parametrize("dims", SHAPES)
def test_M_ee_f64_and_f32(S, dims):
    U = synth.haar_links(dims, 6)
    L = S.Lattice(dims)
    L.load_gauge(U)
    x = synth.gaussian_vector(dims, 7)
    m = 0.05
    ref = O.apply_M(dims, U, m, x)
    out = L.vector()
    L.apply_M(m, dev(x), out)
    assert rel(host(out), ref) < 1e-13
    out32 = L.vector(1)
    L.apply_M(m, dev(x, torch.complex64), out32, 1)
    assert rel(host(out32), ref) < 5e-6


@pytest.mark.parametrize("dims", SHAPES)
def test_float_float_operator_is_fp64_accurate(S, dims):
    """The float-float hop (FP32 pipes, hi/lo pairs) matches the FP64 oracle to
    1e-12 relative: it is an FP64-accurate operator, not an FP32 one."""
    U = synth.haar_links(dims, 21)
    L = S.Lattice(dims)
    L.load_gauge(U)
    x = synth.gaussian_vector(dims, 22)
    out = L.vector()
    L.apply_doe(dev(x), out, S.PREC_F64FF)
    assert rel(host(out), O.dslash(dims, U, 1, x)) < 1e-12
    out = L.vector()
    L.apply_M(0.01, dev(x), out, S.PREC_F64FF)
    assert rel(host(out), O.apply_M(dims, U, 0.01, x)) < 1e-12


def test_multishift_float_float_mode(S):
    dims, m = (8, 8, 8, 8), 0.05
    U = synth.haar_links(dims, 23)
    b = synth.gaussian_vector(dims, 24)
    shifts = synth.log_shifts(8, 1e-4, 1.0)
    L = S.Lattice(dims)
    L.load_gauge(U)
    tol = 1e-10
    sols, info = L.multishift_solve(m, shifts, dev(b), tol=tol, mode=S.SOLVE_F64FF)
    xo, its, tot, st = O.multishift(dims, U, m, shifts, b, tol=tol)
    assert info.status == 0 and abs(info.iters - tot) <= 3
    for k in range(len(shifts)):
        assert info.true_resid[k] <= tol
        assert rel(host(sols[k]), xo[k]) < 1e-8


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_multishift_multi_system(S, mode):
    """Batched solve of 5 systems (5 pseudofermion sources, two groups of the
    multi-RHS hop) with the same shifts: each equals the oracle's own solve."""
    dims, m = (6, 4, 6, 10), 0.05
    U = synth.haar_links(dims, 25)
    shifts = synth.log_shifts(6, 1e-4, 1.0)
    srcs = [synth.gaussian_vector(dims, 30 + r) for r in range(5)]
    L = S.Lattice(dims)
    L.load_gauge(U)
    tol = 1e-10
    sols, infos = L.multishift_solve_multi(m, shifts, [dev(b) for b in srcs], tol=tol, mode=mode)
    for r, b in enumerate(srcs):
        xo, its, tot, st = O.multishift(dims, U, m, shifts, b, tol=1e-12)
        assert infos[r].status == 0
        if mode == 0:
            # FP64: the same recursion as the oracle's, system by system
            _, _, tot10, _ = O.multishift(dims, U, m, shifts, b, tol=tol)
            assert abs(infos[r].iters - tot10) <= 2
        for k in range(len(shifts)):
            assert infos[r].true_resid[k] <= tol
            x = host(sols[r][k])
            assert rel(x, xo[k]) < 1e-7
        rr = b - O.apply_M(dims, U, m, np.ascontiguousarray(host(sols[r][0]))) - shifts[0] * host(sols[r][0])
        assert np.linalg.norm(rr) / np.linalg.norm(b) <= 1.01 * tol


def test_autotuner_keeps_parity(S):
    dims = (8, 8, 8, 8)
    U = synth.haar_links(dims, 26)
    L = S.Lattice(dims)
    L.load_gauge(U)
    tpb = L.autotune()
    assert len(tpb) == 4 and all(t in (64, 128, 256) for t in tpb)
    x = synth.gaussian_vector(dims, 27)
    ref = O.dslash(dims, U, 1, x)
    out = L.vector(S.PREC_F32)
    L.apply_doe(dev(x, torch.complex64), out, S.PREC_F32)
    assert rel(host(out), ref) < 2e-6
    out = L.vector()
    L.apply_doe(dev(x), out, S.PREC_F64FF)
    assert rel(host(out), ref) < 1e-12
    sols, info = L.multishift_solve(0.1, [0.0, 0.5], dev(x), tol=1e-10, mode=S.SOLVE_MIXED)
    assert info.status == 0 and max(info.true_resid[:2]) <= 1e-10


def test_M_ee_full_size_32x32x32x8(S):
    """The operator at the size of the 32^3x8 trajectory, checked in full."""
    dims = (32, 32, 32, 8)
    U = synth.near_unit_links(dims, 0.3, 8)
    L = S.Lattice(dims)
    L.load_gauge(U)
    x = synth.gaussian_vector(dims, 9)
    out = L.vector()
    L.apply_M(0.0075, dev(x), out)
    assert rel(host(out), O.apply_M(dims, U, 0.0075, x)) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
def test_gauge_roundtrip_plaquette_action_force(S, dims):
    U = synth.near_unit_links(dims, 0.4, 10)
    L = S.Lattice(dims)
    L.load_gauge(U)
    np.testing.assert_allclose(L.store_gauge(), U, atol=2e-15)
    assert abs(L.plaquette() - O.plaquette(dims, U)) < 1e-14
    beta = 5.3
    assert abs(L.gauge_action(beta) - O.gauge_action(dims, U, beta)) < 1e-12 * O.gauge_action(dims, U, beta)
    F = host(L.gauge_force(beta))
    assert rel(F, O.gauge_force(dims, U, beta)) < 1e-12


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
def test_heatbath_identical_draws(S, dims):
    L = S.Lattice(dims)
    L.load_gauge(synth.unit_links(dims))
    L.momenta_heatbath(7, 3)
    w = L.store_momenta()
    np.testing.assert_allclose(w, O.momenta_heatbath(dims, 7, 3), rtol=0, atol=1e-13)
    assert abs(L.kinetic() - O.kinetic(dims, w)) < 1e-11 * O.kinetic(dims, w)
    R = host(L.pf_gaussian(7, 3, 1))
    np.testing.assert_allclose(R, O.pf_gaussian(dims, 7, 3, 1), rtol=0, atol=1e-13)


@pytest.mark.parametrize("eps", [0.05, 0.7])
def test_link_update(S, eps):
    dims = (6, 4, 6, 10)
    U = synth.near_unit_links(dims, 0.4, 11)
    w = synth.gaussian_momenta(dims, 12)
    L = S.Lattice(dims)
    L.load_gauge(U)
    L.load_momenta(w)
    L.update_links(eps)
    Ug = L.store_gauge()
    Uo = O.update_links(dims, U, w, eps)
    assert np.abs(Ug - Uo).max() < 1e-13


def test_multishift_f64(S, rationals):
    dims, m = (8, 8, 8, 8), 0.05
    U = synth.haar_links(dims, 13)
    b = synth.gaussian_vector(dims, 14)
    shifts = synth.log_shifts(8, 1e-4, 1.0)
    L = S.Lattice(dims)
    L.load_gauge(U)
    tol = 1e-10
    sols, info = L.multishift_solve(m, shifts, dev(b), tol=tol, mode=S.SOLVE_F64)
    xo, its, tot, st = O.multishift(dims, U, m, shifts, b, tol=tol)
    assert st == 0 and info.status == 0
    assert abs(info.iters - tot) <= 2
    for k in range(len(shifts)):
        assert info.true_resid[k] <= tol
        assert rel(host(sols[k]), xo[k]) < 1e-8


@pytest.mark.parametrize("mode", [1, 2])
def test_multishift_mixed_reaches_fp64_tolerance(S, mode):
    dims, m = (8, 8, 8, 8), 0.05
    U = synth.haar_links(dims, 15)
    b = synth.gaussian_vector(dims, 16)
    shifts = synth.log_shifts(8, 1e-4, 1.0)
    L = S.Lattice(dims)
    L.load_gauge(U)
    tol = 1e-10
    sols, info = L.multishift_solve(m, shifts, dev(b), tol=tol, mode=mode)
    assert info.status == 0
    xo, _, _, _ = O.multishift(dims, U, m, shifts, b, tol=1e-12)
    for k in range(len(shifts)):
        assert info.true_resid[k] <= tol
        # the oracle's own FP64 check of the GPU solution
        x = host(sols[k])
        r = b - O.apply_M(dims, U, m, np.ascontiguousarray(x)) - shifts[k] * x
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01 * tol
        assert rel(x, xo[k]) < 1e-6
    assert info.reliable_updates > 0


def test_rational_apply(S, rationals):
    dims, m = (6, 4, 6, 10), 0.1
    U = synth.near_unit_links(dims, 0.3, 17)
    b = synth.gaussian_vector(dims, 18)
    r = rationals["p+1/4_d8_1e-3"]
    L = S.Lattice(dims)
    L.load_gauge(U)
    out, info = L.rational_apply(m, (r["a0"], r["a"], r["b"]), dev(b), tol=1e-12)
    ref, _ = O.rational_apply(dims, U, m, r["a0"], r["a"], r["b"], b, tol=1e-12)
    assert rel(host(out), ref) < 1e-10


@pytest.mark.parametrize("mode", [0, 1])
def test_fermion_force(S, rationals, mode):
    dims, m = (6, 4, 6, 10), 0.1
    U = synth.near_unit_links(dims, 0.3, 19)
    phi = synth.gaussian_vector(dims, 20)
    r = rationals["p-1/2_d8_1e-3"]
    L = S.Lattice(dims)
    L.load_gauge(U)
    F, info = L.fermion_force(m, (r["a0"], r["a"], r["b"]), dev(phi), tol=1e-12, mode=mode)
    Fo, _, _ = O.fermion_force(dims, U, m, r["a0"], r["a"], r["b"], phi, tol=1e-12)
    assert rel(host(F), Fo) < 1e-9


def test_error_codes(S):
    dims = (4, 4, 4, 4)
    L = S.Lattice(dims)
    x = L.vector()
    out = L.vector()
    with pytest.raises(S.StagError) as e:
        L.apply_deo(x, out)  # no gauge field yet
    assert e.value.code == S.ERR_STATE
    L.load_gauge(synth.haar_links(dims, 1))
    with pytest.raises(S.StagError) as e:
        L.apply_M(0.1, x, x)  # aliasing
    assert e.value.code == S.ERR_ARG
    with pytest.raises(S.StagError) as e:
        L.apply_M(0.1, x, out, prec=7)
    assert e.value.code == S.ERR_ARG
    b = dev(synth.gaussian_vector(dims, 2))
    with pytest.raises(S.StagError) as e:  # iteration cap far too small: NOCONV, no hang
        L.multishift_solve(0.01, [0.0, 0.1], b, tol=1e-12, maxit=3)
    assert e.value.code == S.ERR_NOCONV
    # the context stays usable afterwards
    _, info = L.multishift_solve(0.1, [0.0, 0.1], b, tol=1e-10)
    assert info.status == 0


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_source_is_reported(S, mode, bad):
    """A source with one non-finite entry (injected on the host) makes every
    solver mode return STAG_ERR_NONFINITE instead of a result, and the
    context stays usable."""
    dims = (6, 4, 6, 10)
    L = S.Lattice(dims)
    L.load_gauge(synth.near_unit_links(dims, 0.3, 3))
    b = synth.gaussian_vector(dims, 4)
    bad_b = b.copy()
    bad_b[17, 1] = complex(bad, 0.0)
    with pytest.raises(S.StagError) as e:
        L.multishift_solve(0.1, [0.0, 0.05, 0.5], dev(bad_b), tol=1e-10, mode=mode)
    assert e.value.code == S.ERR_NONFINITE
    sols, info = L.multishift_solve(0.1, [0.0, 0.05, 0.5], dev(b), tol=1e-10, mode=mode)
    assert info.status == 0 and max(info.true_resid[:3]) <= 1e-10

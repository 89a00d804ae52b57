"""GPU parity of the learned gauge-covariant preconditioner (network forward,
weight gradients, training) against the FP64 numpy network oracle, and of the
flexible CG that uses it.

The network computes in FP32 with BF16 weights and FP32 links; the oracle gets
the same BF16-rounded weights and the FP64 links, so the tolerance is that of
FP32 arithmetic through three layers of 9-tap sums (1e-5 relative).
"""
import numpy as np
import pytest

from oracle import gcnn as G
import oracle as O
from paper_1106_5673_gb300 import synth
from tests import helpers as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 4, 6, 10)]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1106_5673_gb300 import build, stag
    build.build()
    return stag


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel())


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def bf16(w):
    """Round complex weights to BF16 (round to nearest even on the FP32 bits)."""
    f = np.ascontiguousarray(np.asarray(w, np.complex64)).view(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).view(np.complex64).astype(np.complex128)


SHAPES_W = [(8, 1, 9), (8, 8, 9), (1, 8, 9)]


def random_weights(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    Ws = []
    for co, ci, t in SHAPES_W:
        W = scale / np.sqrt(ci) * (rng.standard_normal((co, ci, t)) + 1j * rng.standard_normal((co, ci, t)))
        W[:, :, 0] += np.eye(co, ci)
        Ws.append(W)
    return Ws


def make_net(S, L, Ws):
    net = S.Net(L, seed=1)
    for l, W in enumerate(Ws):
        net.set_weights(l, W)
    return net, [bf16(net.weights(l)).reshape(SHAPES_W[l]) for l in range(3)]


@pytest.mark.parametrize("dims", SHAPES)
def test_network_forward(S, dims):
    U = synth.near_unit_links(dims, 0.5, 3)
    L = S.Lattice(dims)
    L.load_gauge(U)
    net, Wq = make_net(S, L, random_weights(4))
    b = synth.gaussian_vector(dims, 5)
    y = host(net.apply(dev(b)))
    ref, _, _, _ = G.network(dims, U, Wq, b)
    assert rel(y, ref) < 1e-5
    # BF16 weights really are the ones used: the FP32 master weights differ
    Wm = [net.weights(l).reshape(SHAPES_W[l]) for l in range(3)]
    assert rel(G.network(dims, U, Wm, b)[0], ref) > 1e-5


def test_network_gauge_covariance(S):
    dims = (6, 4, 6, 10)
    U = synth.haar_links(dims, 6)
    g = H.random_gauge(dims, 7)
    b = synth.gaussian_vector(dims, 8)
    ev = H.parity_sites(dims, 0)
    Ws = random_weights(9)
    L1 = S.Lattice(dims)
    L1.load_gauge(U)
    n1, _ = make_net(S, L1, Ws)
    y = host(n1.apply(dev(b)))
    L2 = S.Lattice(dims)
    L2.load_gauge(H.gauge_transform(dims, U, g))
    n2, _ = make_net(S, L2, Ws)
    yg = host(n2.apply(dev(np.einsum("nij,nj->ni", g[ev], b))))
    assert rel(yg, np.einsum("nij,nj->ni", g[ev], y)) < 1e-5


@pytest.mark.parametrize("dims", SHAPES)
def test_network_loss_and_gradients(S, dims):
    U = synth.near_unit_links(dims, 0.4, 10)
    L = S.Lattice(dims)
    L.load_gauge(U)
    net, Wq = make_net(S, L, random_weights(11))
    bs = [synth.gaussian_vector(dims, 20 + j) for j in range(3)]
    xs = [synth.gaussian_vector(dims, 30 + j) for j in range(3)]
    loss = net.loss_grad([dev(b) for b in bs], [dev(x) for x in xs])
    ref_loss, ref_g = G.loss_and_grads(dims, U, Wq, bs, xs)
    assert abs(loss - ref_loss) < 1e-5 * ref_loss
    for l in range(3):
        assert rel(net.grads(l).reshape(SHAPES_W[l]), ref_g[l]) < 1e-4


def _pairs(S, L, dims, mass, shift, n, seed):
    bs, xs = [], []
    for j in range(n):
        b = dev(synth.gaussian_vector(dims, seed + j))
        sols, info = L.multishift_solve(mass, [shift], b, tol=1e-10)
        assert info.status == 0
        bs.append(b)
        xs.append(sols[0])
    return bs, xs


def test_training_reduces_loss(S):
    dims, mass, shift = (8, 8, 8, 8), 0.1, 0.0
    L = S.Lattice(dims)
    L.load_gauge(synth.near_unit_links(dims, 0.3, 40))
    net = S.Net(L, seed=2)
    bs, xs = _pairs(S, L, dims, mass, shift, 8, 41)
    l0 = net.loss_grad(bs, xs)
    l1 = net.train(bs, xs, epochs=40, batch=4, lr=5e-3)
    l2 = net.loss_grad(bs, xs)
    assert np.isfinite(l1) and l2 < 0.7 * l0


def test_fcg_plain_matches_oracle_cg(S):
    """net = None: flexible CG reduces to CG; solution against the oracle's."""
    dims, mass, shift = (6, 4, 6, 10), 0.05, 0.01
    U = synth.haar_links(dims, 50)
    b = synth.gaussian_vector(dims, 51)
    L = S.Lattice(dims)
    L.load_gauge(U)
    tol = 1e-10
    x, info = S.fcg_solve(L, None, mass, shift, dev(b), tol=tol)
    assert info.status == 0 and info.true_resid[0] <= tol
    xo, its, _, st = O.multishift(dims, U, mass, [shift], b, tol=tol)
    assert abs(info.iters - its[0]) <= 2
    assert rel(host(x), xo[0]) < tol * 100


def test_fcg_identity_network_is_cg(S):
    """K = 1 (identity weights): same iteration count as plain CG within 2."""
    dims, mass, shift = (8, 8, 8, 8), 0.05, 0.0
    L = S.Lattice(dims)
    L.load_gauge(synth.haar_links(dims, 60))
    Ws = [np.zeros(s, complex) for s in SHAPES_W]
    for W in Ws:
        W[:, :, 0] = np.eye(W.shape[0], W.shape[1])
    Ws[2][0, :, 0] = 0
    Ws[2][0, 0, 0] = 1.0
    net, _ = make_net(S, L, Ws)
    b = dev(synth.gaussian_vector(dims, 61))
    tol = 1e-10
    _, i0 = S.fcg_solve(L, None, mass, shift, b, tol=tol)
    _, i1 = S.fcg_solve(L, net, mass, shift, b, tol=tol)
    assert i0.status == 0 and i1.status == 0 and i1.true_resid[0] <= tol
    assert abs(i1.iters - i0.iters) <= 2


def test_fcg_trained_network_converges_faster(S):
    """A network trained on solved pairs of the light system preconditions it:
    fewer flexible-CG iterations than plain CG, and the FP64-accurate true
    residual still meets the tolerance."""
    dims, mass, shift = (8, 8, 8, 8), 0.02, 0.0
    L = S.Lattice(dims)
    L.load_gauge(synth.near_unit_links(dims, 0.3, 70))
    bs, xs = _pairs(S, L, dims, mass, shift, 16, 71)
    net = S.Net(L, seed=3)
    net.train(bs, xs, epochs=60, batch=4, lr=5e-3)
    b = dev(synth.gaussian_vector(dims, 99))
    tol = 1e-10
    _, i0 = S.fcg_solve(L, None, mass, shift, b, tol=tol)
    _, i1 = S.fcg_solve(L, net, mass, shift, b, tol=tol)
    assert i1.status == 0 and i1.true_resid[0] <= tol
    assert i1.iters < i0.iters


def test_learned_mode_multishift(S):
    """SOLVE_LEARNED: lightest shift by network-preconditioned flexible CG, the
    rest by the mixed multi-shift; every shift meets tol (FP64-accurate) and
    matches the oracle's multi-shift solutions."""
    dims, mass = (6, 4, 6, 10), 0.02
    U = synth.near_unit_links(dims, 0.3, 80)
    L = S.Lattice(dims)
    L.load_gauge(U)
    bs, xs = _pairs(S, L, dims, mass, 0.0, 8, 81)
    net = S.Net(L, seed=4)
    net.train(bs, xs, epochs=30, batch=4, lr=5e-3)
    with pytest.raises(S.StagError):  # no network attached yet
        L.multishift_solve(mass, [0.0, 0.1], bs[0], mode=S.SOLVE_LEARNED)
    net.attach()
    shifts = [0.3, 1e-4, 0.02, 1.5]  # lightest not first: results land at their own index
    b = synth.gaussian_vector(dims, 90)
    tol = 1e-10
    sols, info = L.multishift_solve(mass, shifts, dev(b), tol=tol, mode=S.SOLVE_LEARNED)
    assert info.status == 0
    xo, _, _, _ = O.multishift(dims, U, mass, shifts, b, tol=1e-12)
    for k in range(len(shifts)):
        assert info.true_resid[k] <= tol
        assert rel(host(sols[k]), xo[k]) < 1e-7
    assert info.iters_shift[1] > 0  # the flexible CG ran on shift 1


def test_learned_mode_trajectory(S, rationals):
    """A 4^4 trajectory whose MD force solves use SOLVE_LEARNED (lightest
    pole by the network-preconditioned flexible CG): same decision and dH as
    the oracle within the mixed-mode tolerance, since every solve still meets
    1e-10 in FP64."""
    dims = (4, 4, 4, 4)
    h, r = rationals["p+1/4_d8_1e-3"], rationals["p-1/2_d8_1e-3"]
    hb, act = (h["a0"], h["a"], h["b"]), (r["a0"], r["a"], r["b"])
    U = synth.near_unit_links(dims, 0.3, 0)
    po = O.make_params(5.3, 0.1, 1.0, 10, 0, hb, act, act, tol_md=1e-10, tol_metro=1e-10, seed=11, traj=0)
    _, io, st = O.trajectory(dims, U, po)
    assert st == 0
    L = S.Lattice(dims)
    L.load_gauge(U)
    net = S.Net(L, seed=6)
    net.attach()
    ig = L.md_trajectory(S.make_params(5.3, 0.1, 1.0, 10, 0, hb, act, act, tol_md=1e-10, tol_metro=1e-10,
                                       mode_md=S.SOLVE_LEARNED, mode_metro=S.SOLVE_MIXED, seed=11, traj=0))
    assert ig["accepted"] == io["accepted"]
    assert abs(ig["dH"] - io["dH"]) < 1e-6 * max(1.0, abs(io["dH"]))

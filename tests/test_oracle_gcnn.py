"""Pins of the oracle of the gauge-covariant preconditioner network (CPU)."""
import numpy as np

from oracle import gcnn
from paper_1106_5673_gb300 import synth
from tests import helpers as H

DIMS = (4, 2, 4, 4)


def _weights(seed, co, ci, scale=0.3):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal((co, ci, 9)) + 1j * rng.standard_normal((co, ci, 9)))


def _field(seed, V, c=1):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((c, V, 3)) + 1j * rng.standard_normal((c, V, 3))) / np.sqrt(2)


def test_taps_adjoint_identity():
    """<g, T phi> = <T^dag g, phi> for the 9 transported taps."""
    U = synth.haar_links(DIMS, 1)
    V = synth.volume(DIMS)
    phi = _field(2, V)[0]
    g = _field(3, V, 9)
    lhs = np.vdot(g, gcnn.taps(DIMS, U, phi))
    rhs = np.vdot(gcnn.taps_adjoint(DIMS, U, g), phi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_layer_gauge_covariance():
    U = synth.haar_links(DIMS, 4)
    V = synth.volume(DIMS)
    g = H.random_gauge(DIMS, 5)
    W = _weights(6, 3, 2)
    phis = _field(7, V, 2)
    y, _ = gcnn.layer_forward(DIMS, U, W, phis)
    yg, _ = gcnn.layer_forward(DIMS, H.gauge_transform(DIMS, U, g), W,
                               np.einsum("nij,cnj->cni", g, phis))
    np.testing.assert_allclose(yg, np.einsum("nij,cnj->cni", g, y), atol=1e-12)


def test_identity_weights_give_identity_network():
    """w[o,i,0] = delta, other taps 0: K b = b."""
    U = synth.haar_links(DIMS, 8)
    Ws = [np.zeros((1, 1, 9), complex) for _ in range(3)]
    for W in Ws:
        W[0, 0, 0] = 1.0
    b = synth.gaussian_vector(DIMS, 9)
    y, _, _, _ = gcnn.network(DIMS, U, Ws, b)
    np.testing.assert_allclose(y, b, atol=1e-15)


def test_gradients_finite_difference():
    """Weight gradients of the loss against central differences in Re and Im."""
    U = synth.near_unit_links(DIMS, 0.4, 10)
    Ws = [_weights(11, 4, 1), _weights(12, 4, 4), _weights(13, 1, 4)]
    bs = [synth.gaussian_vector(DIMS, 20 + j) for j in range(2)]
    xs = [synth.gaussian_vector(DIMS, 30 + j) for j in range(2)]
    loss, grads = gcnn.loss_and_grads(DIMS, U, Ws, bs, xs)
    rng = np.random.default_rng(0)
    h = 1e-6
    for li in range(3):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in Ws[li].shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[li][idx] += h * unit
                Wm[li][idx] -= h * unit
                lp, _ = gcnn.loss_and_grads(DIMS, U, Wp, bs, xs)
                lm, _ = gcnn.loss_and_grads(DIMS, U, Wm, bs, xs)
                fd = (lp - lm) / (2 * h)
                an = grads[li][idx].real if part == "re" else grads[li][idx].imag
                assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (li, idx, part, fd, an)


def test_layer_adjoint_identity():
    """<g, L phi> = <L^dag g, phi> for a layer with random complex weights."""
    U = synth.haar_links(DIMS, 40)
    V = synth.volume(DIMS)
    W = _weights(41, 3, 2)
    phis = _field(42, V, 2)
    g = _field(43, V, 3)
    y, _ = gcnn.layer_forward(DIMS, U, W, phis)
    lhs = np.vdot(g, y)
    rhs = np.vdot(gcnn.layer_adjoint(DIMS, U, W, g), phis)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_preconditioner_hermitian_positive():
    """K = restrict A^dag A embed: <a, K b> = conj(<b, K a>) and <b, K b> = |A b|^2 >= 0."""
    U = synth.haar_links(DIMS, 44)
    Ws = [_weights(45, 4, 1), _weights(46, 4, 4), _weights(47, 1, 4)]
    a = synth.gaussian_vector(DIMS, 48)
    b = synth.gaussian_vector(DIMS, 49)
    Ka, _, _, _ = gcnn.network(DIMS, U, Ws, a)
    Kb, acts, _, _ = gcnn.network(DIMS, U, Ws, b)
    assert abs(np.vdot(a, Kb) - np.conj(np.vdot(b, Ka))) < 1e-12 * abs(np.vdot(a, Kb))
    bKb = np.vdot(b, Kb)
    assert abs(bKb.imag) < 1e-12 * abs(bKb) and bKb.real > 0
    assert abs(bKb.real - np.vdot(acts[-1], acts[-1]).real) < 1e-12 * bKb.real

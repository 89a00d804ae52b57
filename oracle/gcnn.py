"""TEST INFRASTRUCTURE ONLY: FP64 numpy oracle of the gauge-covariant network
used as a learned preconditioner for the lightest RHMC pole.

The paper has no network; the definition here is the library's.  One layer
maps C_in complex colour-vector fields on the full lattice to C_out fields by
a parallel-transport convolution with 9 taps,

    (L phi)_o(n) = sum_i sum_t w[o, i, t] (T_t phi_i)(n),
    T_0 phi = phi(n),  T_{1+mu} phi = U_mu(n) phi(n+mu),
    T_{5+mu} phi = U_mu(n-mu)^dag phi(n-mu),

which commutes with gauge transformations (phi -> g phi, U_mu(n) ->
g(n) U_mu(n) g(n+mu)^dag).  A = L3 o L2 o L1 (channels 1 -> 8 -> 8 -> 1) maps
a colour-vector field to another; the preconditioner is
    K = restrict_even o A^dag o A o embed_even,
Hermitian and positive semi-definite by construction (so a conjugate-gradient
method can use it), trained so that K b_j ~ x_j = (M_ee + s)^{-1} b_j.
A^dag applies the adjoint layers in reverse order; the adjoint of a layer is
    (L^dag g)_i = sum_o sum_t conj(w[o, i, t]) T_t^dag g_o,
    T_{1+mu}^dag = T_{5+mu}.
Training minimises
    loss = (1/B) sum_j |K b_j - x_j|^2 / |x_j|^2.
Weight gradients use the convention g = dloss/dRe(w) + i dloss/dIm(w).
Only the test suite may import this module.
"""
import numpy as np


def neighbours(dims):
    """fwd[mu][n] = lex(n + mu), bwd[mu][n] = lex(n - mu)."""
    V = int(np.prod(dims))
    lex = np.arange(V)
    Lx, Ly, Lz, Lt = dims
    c = np.stack([lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz)], -1)
    fwd, bwd = [], []
    for mu in range(4):
        cf, cb = c.copy(), c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        cb[:, mu] = (cb[:, mu] - 1) % dims[mu]
        fwd.append(cf[:, 0] + Lx * (cf[:, 1] + Ly * (cf[:, 2] + Lz * cf[:, 3])))
        bwd.append(cb[:, 0] + Lx * (cb[:, 1] + Ly * (cb[:, 2] + Lz * cb[:, 3])))
    even = (c.sum(-1) % 2) == 0
    return fwd, bwd, even


def taps(dims, U, phi, nb=None):
    """The 9 transported copies of phi [V, 3] -> [9, V, 3]."""
    fwd, bwd, _ = nb if nb is not None else neighbours(dims)
    out = [phi]
    for mu in range(4):
        out.append(np.einsum("nij,nj->ni", U[mu], phi[fwd[mu]]))
    for mu in range(4):
        out.append(np.einsum("nji,nj->ni", U[mu][bwd[mu]].conj(), phi[bwd[mu]]))
    return np.stack(out)


def taps_adjoint(dims, U, g, nb=None):
    """Adjoint of the taps: given g_t [9, V, 3], returns sum_t T_t^dag g_t [V, 3]."""
    fwd, bwd, _ = nb if nb is not None else neighbours(dims)
    out = g[0].copy()
    for mu in range(4):
        # <g, U(n) phi(n+mu)> summed over n = <U(n-mu)^dag g(n-mu), phi(n)>
        t = np.einsum("nji,nj->ni", U[mu].conj(), g[1 + mu])   # U_mu(m)^dag g(m) at m = n-mu
        out += t[bwd[mu]]
        # <g, U(n-mu)^dag phi(n-mu)> = <U(m) g(m+mu), phi(m)>
        t = np.einsum("nij,nj->ni", U[mu], g[5 + mu][fwd[mu]])
        out += t
    return out


def layer_forward(dims, U, W, phis, nb=None):
    """W [Co, Ci, 9] complex; phis [Ci, V, 3] -> [Co, V, 3]."""
    T = np.stack([taps(dims, U, p, nb) for p in phis])  # [Ci, 9, V, 3]
    return np.einsum("oit,itnc->onc", W, T), T


def layer_adjoint(dims, U, W, gs, nb=None):
    """(L^dag g)_i = sum_t T_t^dag (sum_o conj(W[o, i, t]) g_o); gs [Co, V, 3] -> [Ci, V, 3]."""
    Ci = W.shape[1]
    out = []
    for i in range(Ci):
        gt = np.einsum("ot,onc->tnc", W[:, i, :].conj(), gs)  # [9, V, 3]
        out.append(taps_adjoint(dims, U, gt, nb))
    return np.stack(out)


def weight_grad(dims, U, a, b, nb=None):
    """2 sum_n <T_t a_i(n), b_o(n)> -> [Co, Ci, 9] for a [Ci, V, 3], b [Co, V, 3]."""
    T = np.stack([taps(dims, U, p, nb) for p in a])  # [Ci, 9, V, 3]
    return 2.0 * np.einsum("itnc,onc->oit", T.conj(), b)


def layer_backward(dims, U, W, T, gout, nb=None):
    """Given T (taps of the layer input) and gout = dloss/dconj(out) [Co, V, 3]
    (in the convention dloss = 2 Re <gout, d out>), returns
    (gin [Ci, V, 3] = dloss/dconj(in), gW [Co, Ci, 9] = 2 dloss/dconj(W))."""
    gW = 2.0 * np.einsum("itnc,onc->oit", T.conj(), gout)
    return layer_adjoint(dims, U, W, gout, nb), gW


def network(dims, U, Ws, b_even, nb=None):
    """K b = restrict_even A^dag A embed_even b with A = the layers in order.
    Returns (K b, forward activations, taps of the forward layers, adjoint
    activations c with c[-1] = A embed b and c[0] = A^dag A embed b)."""
    nb = nb if nb is not None else neighbours(dims)
    V = int(np.prod(dims))
    even = nb[2]
    phi = np.zeros((1, V, 3), np.complex128)
    phi[0, even] = b_even
    acts = [phi]
    Ts = []
    for W in Ws:
        y, T = layer_forward(dims, U, W, acts[-1], nb)
        acts.append(y)
        Ts.append(T)
    cs = [None] * len(Ws) + [acts[-1]]
    for li in range(len(Ws) - 1, -1, -1):
        cs[li] = layer_adjoint(dims, U, Ws[li], cs[li + 1], nb)
    return cs[0][0, even], acts, Ts, cs


def loss_and_grads(dims, U, Ws, bs, xs, nb=None):
    """loss = mean_j |K b_j - x_j|^2 / |x_j|^2 and its weight gradients.

    Back-propagation runs through the adjoint layers (last applied first) and
    then the forward layers.  For an adjoint layer c_l = L_l^dag c_{l+1} with
    output gradient g, the weight gradient is weight_grad(g, c_{l+1}) and the
    input gradient L_l g; for a forward layer a_{l+1} = L_l a_l it is
    weight_grad(a_l, g) and L_l^dag g."""
    nb = nb if nb is not None else neighbours(dims)
    V = int(np.prod(dims))
    even = nb[2]
    loss = 0.0
    grads = [np.zeros_like(W) for W in Ws]
    B = len(bs)
    for b, x in zip(bs, xs):
        y, acts, Ts, cs = network(dims, U, Ws, b, nb)
        nx = np.vdot(x, x).real
        e = y - x
        loss += np.vdot(e, e).real / nx / B
        g = np.zeros((1, V, 3), np.complex128)
        g[0, even] = e / nx / B  # dloss/dconj(y)
        for li in range(len(Ws)):  # adjoint layers, in reverse order of application
            grads[li] += weight_grad(dims, U, g, cs[li + 1], nb)
            g, _ = layer_forward(dims, U, Ws[li], g, nb)
        for li in range(len(Ws) - 1, -1, -1):  # forward layers
            g, gW = layer_backward(dims, U, Ws[li], Ts[li], g, nb)
            grads[li] += gW
    return loss, grads

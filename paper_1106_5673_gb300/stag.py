"""Thin ctypes binding of libstag.so (include/stag.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device memory comes from PyTorch tensors (CUDA, contiguous) and the
stream is PyTorch's current stream.  Raises if the library is missing: there
is no CPU fallback.

Canonical layouts (see include/stag.h):
  gauge    complex128 [4, V, 3, 3]
  vector   complex128 [V/2, 3] (PREC_F64) or complex64 [V/2, 3] (PREC_F32/BF16)
  momenta  float64    [4, V, 8]
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libstag.so")

OK, ERR_ARG, ERR_CUDA, ERR_NOCONV, ERR_NONFINITE, ERR_OOM, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
PREC_F64, PREC_F32, PREC_BF16, PREC_F64FF, PREC_F32R8 = 0, 1, 2, 3, 4
SOLVE_F64, SOLVE_MIXED, SOLVE_MIXED_BF16, SOLVE_F64FF, SOLVE_LEARNED = 0, 1, 2, 3, 4
INT_LEAPFROG, INT_OMELYAN = 0, 1
MAXSHIFT = 32
MAXPF = 8
MAXLAT = 8
OMELYAN_LAMBDA = 0.1931833275037836


class StagError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("stag error %d: %s" % (code, msg))
        self.code = code


class Rational(C.Structure):
    _fields_ = [("a0", C.c_double), ("n", C.c_int),
                ("a", C.c_double * MAXSHIFT), ("b", C.c_double * MAXSHIFT)]

    @staticmethod
    def make(a0, a, b):
        r = Rational()
        r.a0 = float(a0)
        r.n = len(a)
        if len(a) != len(b) or len(a) > MAXSHIFT:
            raise ValueError("bad rational")
        for i, (x, y) in enumerate(zip(a, b)):
            r.a[i] = float(x)
            r.b[i] = float(y)
        return r

    def as_tuple(self):
        return self.a0, list(self.a[:self.n]), list(self.b[:self.n])


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int),
                ("iters_shift", C.c_int * MAXSHIFT), ("refine_iters", C.c_int * MAXSHIFT),
                ("true_resid", C.c_double * MAXSHIFT), ("reliable_updates", C.c_int),
                ("matvecs", C.c_int)]


class Params(C.Structure):
    _fields_ = [("beta", C.c_double), ("mass", C.c_double), ("tau", C.c_double),
                ("nsteps", C.c_int), ("integrator", C.c_int), ("lam", C.c_double),
                ("npf", C.c_int), ("hb", Rational), ("act", Rational), ("force", Rational),
                ("tol_md", C.c_double), ("tol_metro", C.c_double),
                ("solve_mode_md", C.c_int), ("solve_mode_metro", C.c_int), ("maxit", C.c_int),
                ("seed", C.c_uint32), ("traj", C.c_uint32), ("use_graphs", C.c_int),
                ("ngauge", C.c_int), ("no_metropolis", C.c_int)]


class TrajInfo(C.Structure):
    _fields_ = [("H0", C.c_double), ("H1", C.c_double), ("dH", C.c_double), ("u", C.c_double),
                ("accepted", C.c_int), ("plaq", C.c_double), ("cg_iters", C.c_longlong),
                ("n_force", C.c_int), ("t_heatbath", C.c_double), ("t_action", C.c_double),
                ("t_md", C.c_double), ("t_total", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)

# name -> (restype, argtypes)
_SIGS = {
    "stag_ctx_create": (C.c_int, [C.POINTER(C.c_int), C.POINTER(_vp)]),
    "stag_ctx_destroy": (C.c_int, [_vp]),
    "stag_last_error": (C.c_char_p, [_vp]),
    "stag_ctx_device_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "stag_ctx_launch_count": (C.c_int, [_vp, C.POINTER(C.c_longlong)]),
    "stag_autotune": (C.c_int, [_vp, C.POINTER(C.c_int), _vp]),
    "stag_load_gauge": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "stag_store_gauge": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "stag_load_momenta": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "stag_store_momenta": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "stag_plaquette": (C.c_int, [_vp, _dp, _vp]),
    "stag_gauge_action": (C.c_int, [_vp, C.c_double, _dp, _vp]),
    "stag_apply_deo": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "stag_apply_doe": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp]),
    "stag_apply_M": (C.c_int, [_vp, C.c_double, _vp, _vp, C.c_int, _vp]),
    "stag_multishift_solve": (C.c_int, [_vp, C.c_double, C.c_int, _dp, _vp, C.POINTER(_vp),
                                        C.c_double, C.c_int, C.c_int, C.POINTER(SolveInfo), _vp]),
    "stag_multishift_solve_multi": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int, _dp,
                                              C.POINTER(_vp), C.POINTER(_vp), C.c_double, C.c_int,
                                              C.c_int, C.POINTER(SolveInfo), _vp]),
    "stag_rational_apply": (C.c_int, [_vp, C.c_double, C.POINTER(Rational), _vp, _vp, C.c_double,
                                      C.c_int, C.c_int, C.POINTER(SolveInfo), _vp]),
    "stag_gauge_force": (C.c_int, [_vp, C.c_double, _vp, _vp]),
    "stag_fermion_force": (C.c_int, [_vp, C.c_double, C.POINTER(Rational), _vp, _vp, C.c_double,
                                     C.c_int, C.c_int, C.POINTER(SolveInfo), _vp]),
    "stag_update_links": (C.c_int, [_vp, C.c_double, _vp]),
    "stag_momenta_heatbath": (C.c_int, [_vp, C.c_uint32, C.c_uint32, _vp]),
    "stag_pf_gaussian": (C.c_int, [_vp, C.c_uint32, C.c_uint32, C.c_int, _vp, _vp]),
    "stag_kinetic": (C.c_int, [_vp, _dp, _vp]),
    "stag_md_trajectory": (C.c_int, [_vp, C.POINTER(Params), C.POINTER(TrajInfo), _vp]),
    "stag_md_integrate": (C.c_int, [_vp, C.POINTER(Params), _vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                    _vp]),
    "stag_remez": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(Rational),
                             _dp]),
    "stag_apply_M_noalloc": (C.c_int, [C.POINTER(C.c_int), _vp, C.c_double, _vp, _vp, _vp]),
    "stag_net_create": (C.c_int, [_vp, C.c_uint, C.POINTER(_vp)]),
    "stag_net_destroy": (C.c_int, [_vp]),
    "stag_ctx_set_net": (C.c_int, [_vp, _vp]),
    "stag_dslash_batch": (C.c_int, [C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp),
                                    C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_int), _vp]),
    "stag_net_nweights": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "stag_net_get_weights": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_float)]),
    "stag_net_set_weights": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_float)]),
    "stag_net_get_grads": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_float)]),
    "stag_net_apply": (C.c_int, [_vp, _vp, _vp, _vp]),
    "stag_net_loss_grad": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp), _dp, _vp]),
    "stag_net_train": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.c_int, C.c_int,
                                 C.c_double, _dp, _vp]),
    "stag_fcg_solve": (C.c_int, [_vp, _vp, C.c_double, C.c_double, _vp, _vp, C.c_double, C.c_int,
                                 C.POINTER(SolveInfo), _vp]),
}


def lib():
    """Loads libstag.so (built by paper_1106_5673_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libstag.so not built: run `python -m paper_1106_5673_gb300.build` "
                              "(needs nvcc); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def remez(power, lo, hi, degree):
    """Host Remez exchange (no GPU needed): returns (a0, a, b, max_rel_err)."""
    r = Rational()
    err = C.c_double(0)
    st = lib().stag_remez(power, lo, hi, degree, C.byref(r), C.byref(err))
    if st != OK:
        raise StagError(st, "remez failed for p=%g on [%g, %g] degree %d" % (power, lo, hi, degree))
    a0, a, b = r.as_tuple()
    return a0, a, b, err.value


def apply_M_noalloc(dims, links, mass, x_even, out_even):
    """out = M_ee x through the allocation-free entry point: `links` is the
    canonical gauge field as a complex128 CUDA tensor [4, V, 3, 3]; nothing is
    allocated on the device by the call.  Returns the status code."""
    d = (C.c_int * 4)(*[int(v) for v in dims])
    return lib().stag_apply_M_noalloc(d, _ptr(links), float(mass), _ptr(x_even), _ptr(out_even),
                                      _stream())


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Lattice:
    """One lattice context on the current CUDA device (stag_ctx)."""

    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        h = _vp()
        st = lib().stag_ctx_create((C.c_int * 4)(*self.dims), C.byref(h))
        if st != OK:
            raise StagError(st, "stag_ctx_create failed for dims %s" % (self.dims,))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().stag_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != OK:
            raise StagError(st, lib().stag_last_error(self._h).decode())

    # -------- allocation helpers (torch device memory)
    def vector(self, prec=PREC_F64):
        torch = _torch()
        dt = torch.complex128 if prec == PREC_F64 else torch.complex64
        return torch.zeros((self.Vh, 3), dtype=dt, device="cuda")

    def momenta(self):
        return _torch().zeros((4, self.V, 8), dtype=_torch().float64, device="cuda")

    def device_bytes(self):
        b = C.c_size_t(0)
        self._chk(lib().stag_ctx_device_bytes(self._h, C.byref(b)))
        return b.value

    def autotune(self):
        """Runs the hop autotuner; returns threads per block for FP64, FP32,
        BF16 and float-float links."""
        t = (C.c_int * 4)()
        self._chk(lib().stag_autotune(self._h, t, _stream()))
        return list(t)

    def launch_count(self):
        n = C.c_longlong(0)
        self._chk(lib().stag_ctx_launch_count(self._h, C.byref(n)))
        return n.value

    # -------- fields
    def load_gauge(self, U):
        """U: numpy complex128 [4,V,3,3] (host) or torch complex128 CUDA tensor."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, np.complex128)
            assert U.shape == (4, self.V, 3, 3)
            self._chk(lib().stag_load_gauge(self._h, U.ctypes.data_as(_vp), 0, _stream()))
        else:
            self._chk(lib().stag_load_gauge(self._h, _ptr(U), 1, _stream()))

    def store_gauge(self, out=None):
        """Canonical links to a host array (new, or `out`: complex128
        [4,V,3,3], e.g. a view of pinned memory)."""
        U = np.zeros((4, self.V, 3, 3), np.complex128) if out is None else out
        assert U.shape == (4, self.V, 3, 3) and U.dtype == np.complex128 and U.flags.c_contiguous
        self._chk(lib().stag_store_gauge(self._h, U.ctypes.data_as(_vp), 0, _stream()))
        return U

    def load_momenta(self, w):
        w = np.ascontiguousarray(w, np.float64)
        self._chk(lib().stag_load_momenta(self._h, w.ctypes.data_as(_vp), 0, _stream()))

    def store_momenta(self):
        w = np.zeros((4, self.V, 8))
        self._chk(lib().stag_store_momenta(self._h, w.ctypes.data_as(_vp), 0, _stream()))
        return w

    def plaquette(self):
        v = C.c_double(0)
        self._chk(lib().stag_plaquette(self._h, C.byref(v), _stream()))
        return v.value

    def gauge_action(self, beta):
        v = C.c_double(0)
        self._chk(lib().stag_gauge_action(self._h, beta, C.byref(v), _stream()))
        return v.value

    # -------- operator
    def apply_deo(self, x_odd, out_even, prec=PREC_F64):
        self._chk(lib().stag_apply_deo(self._h, _ptr(x_odd), _ptr(out_even), prec, _stream()))

    def apply_doe(self, x_even, out_odd, prec=PREC_F64):
        self._chk(lib().stag_apply_doe(self._h, _ptr(x_even), _ptr(out_odd), prec, _stream()))

    def apply_M(self, mass, x_even, out_even, prec=PREC_F64):
        self._chk(lib().stag_apply_M(self._h, mass, _ptr(x_even), _ptr(out_even), prec, _stream()))

    # -------- solvers
    def multishift_solve(self, mass, shifts, src, sols=None, tol=1e-10, maxit=100000,
                         mode=SOLVE_F64):
        n = len(shifts)
        sh = (C.c_double * n)(*[float(s) for s in shifts])
        if sols is None:
            sols = [self.vector() for _ in range(n)]
        arr = (_vp * n)(*[s.data_ptr() for s in sols])
        info = SolveInfo()
        st = lib().stag_multishift_solve(self._h, mass, n, sh, _ptr(src), arr, tol, maxit, mode,
                                         C.byref(info), _stream())
        self._chk(st)
        return sols, info

    def multishift_solve_multi(self, mass, shifts, srcs, tol=1e-10, maxit=100000, mode=SOLVE_F64):
        """Batched solve of len(srcs) systems with the same shifts; returns
        (sols[r][k], infos[r])."""
        n, ns = len(shifts), len(srcs)
        sh = (C.c_double * n)(*[float(s) for s in shifts])
        src_arr = (_vp * ns)(*[s.data_ptr() for s in srcs])
        sols = [[self.vector() for _ in range(n)] for _ in range(ns)]
        sol_arr = (_vp * (ns * n))(*[x.data_ptr() for row in sols for x in row])
        infos = (SolveInfo * ns)()
        st = lib().stag_multishift_solve_multi(self._h, mass, ns, n, sh, src_arr, sol_arr, tol, maxit,
                                               mode, infos, _stream())
        self._chk(st)
        return sols, list(infos)

    def rational_apply(self, mass, rat, src, out=None, tol=1e-10, maxit=100000, mode=SOLVE_F64):
        r = Rational.make(*rat)
        out = self.vector() if out is None else out
        info = SolveInfo()
        self._chk(lib().stag_rational_apply(self._h, mass, C.byref(r), _ptr(src), _ptr(out), tol,
                                            maxit, mode, C.byref(info), _stream()))
        return out, info

    # -------- forces and updates
    def gauge_force(self, beta):
        F = self.momenta()
        self._chk(lib().stag_gauge_force(self._h, beta, _ptr(F), _stream()))
        return F

    def fermion_force(self, mass, rat, phi, tol=1e-10, maxit=100000, mode=SOLVE_F64):
        r = Rational.make(*rat)
        F = self.momenta()
        info = SolveInfo()
        self._chk(lib().stag_fermion_force(self._h, mass, C.byref(r), _ptr(phi), _ptr(F), tol,
                                           maxit, mode, C.byref(info), _stream()))
        return F, info

    def update_links(self, eps):
        self._chk(lib().stag_update_links(self._h, eps, _stream()))

    def momenta_heatbath(self, seed, traj):
        self._chk(lib().stag_momenta_heatbath(self._h, seed, traj, _stream()))

    def pf_gaussian(self, seed, traj, pf):
        out = self.vector()
        self._chk(lib().stag_pf_gaussian(self._h, seed, traj, pf, _ptr(out), _stream()))
        return out

    def kinetic(self):
        v = C.c_double(0)
        self._chk(lib().stag_kinetic(self._h, C.byref(v), _stream()))
        return v.value

    def md_trajectory(self, params):
        info = TrajInfo()
        self._chk(lib().stag_md_trajectory(self._h, C.byref(params), C.byref(info), _stream()))
        return info.as_dict()

    def md_integrate(self, params, phi=None):
        """MD over params.tau from the current links and momenta with phi
        (torch complex128 [npf, V/2, 3] or None for npf = 0) held fixed;
        returns (cg_iters, n_force)."""
        it = C.c_longlong(0)
        nf = C.c_int(0)
        self._chk(lib().stag_md_integrate(self._h, C.byref(params), _ptr(phi), C.byref(it), C.byref(nf),
                                          _stream()))
        return it.value, nf.value


def make_params(beta, mass, tau, nsteps, integrator, hb, act, force, npf=1, tol_md=1e-10,
                tol_metro=1e-10, mode_md=SOLVE_F64, mode_metro=SOLVE_F64, seed=0, traj=0,
                lam=OMELYAN_LAMBDA, maxit=100000, use_graphs=1, ngauge=0, no_metropolis=0):
    """hb/act/force: (a0, a, b) partial fractions; ngauge > 0: multi-step
    integrator with ngauge gauge steps per position update."""
    p = Params()
    p.ngauge = ngauge
    p.no_metropolis = no_metropolis
    p.beta, p.mass, p.tau, p.nsteps, p.integrator, p.lam = beta, mass, tau, nsteps, integrator, lam
    p.npf = npf
    p.hb = Rational.make(*hb)
    p.act = Rational.make(*act)
    p.force = Rational.make(*force)
    p.tol_md, p.tol_metro = tol_md, tol_metro
    p.solve_mode_md, p.solve_mode_metro = mode_md, mode_metro
    p.maxit, p.seed, p.traj, p.use_graphs = maxit, seed, traj, use_graphs
    return p


class Net:
    """Learned gauge-covariant preconditioner bound to a Lattice (stag_net)."""

    def __init__(self, lattice, seed=0):
        self.lat = lattice
        h = _vp()
        st = lib().stag_net_create(lattice._h, seed, C.byref(h))
        if st != OK:
            raise StagError(st, lib().stag_last_error(lattice._h).decode())
        self._h = h
        self.nw = []
        for layer in range(3):
            n = C.c_int(0)
            lib().stag_net_nweights(self._h, layer, C.byref(n))
            self.nw.append(n.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().stag_net_destroy(self._h)
            self._h = None

    def attach(self):
        """Makes this network the preconditioner of SOLVE_LEARNED on its lattice."""
        self._chk(lib().stag_ctx_set_net(self.lat._h, self._h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        self.lat._chk(st)

    def weights(self, layer):
        a = np.zeros(2 * self.nw[layer], np.float32)
        self._chk(lib().stag_net_get_weights(self._h, layer, a.ctypes.data_as(C.POINTER(C.c_float))))
        return a.view(np.complex64).astype(np.complex128)

    def set_weights(self, layer, w):
        a = np.ascontiguousarray(np.asarray(w, np.complex64).reshape(-1))
        assert a.size == self.nw[layer]
        f = a.view(np.float32)
        self._chk(lib().stag_net_set_weights(self._h, layer, f.ctypes.data_as(C.POINTER(C.c_float))))

    def grads(self, layer):
        a = np.zeros(2 * self.nw[layer], np.float32)
        self._chk(lib().stag_net_get_grads(self._h, layer, a.ctypes.data_as(C.POINTER(C.c_float))))
        return a.view(np.complex64).astype(np.complex128)

    def apply(self, x_even, out_even=None):
        out = self.lat.vector() if out_even is None else out_even
        self._chk(lib().stag_net_apply(self._h, _ptr(x_even), _ptr(out), _stream()))
        return out

    def loss_grad(self, srcs, sols):
        n = len(srcs)
        a = (_vp * n)(*[s.data_ptr() for s in srcs])
        b = (_vp * n)(*[s.data_ptr() for s in sols])
        loss = C.c_double(0)
        self._chk(lib().stag_net_loss_grad(self._h, n, a, b, C.byref(loss), _stream()))
        return loss.value

    def train(self, srcs, sols, epochs=1, batch=8, lr=1e-3):
        n = len(srcs)
        a = (_vp * n)(*[s.data_ptr() for s in srcs])
        b = (_vp * n)(*[s.data_ptr() for s in sols])
        loss = C.c_double(0)
        self._chk(lib().stag_net_train(self._h, n, a, b, epochs, batch, lr, C.byref(loss), _stream()))
        return loss.value


def fcg_solve(lattice, net, mass, shift, src, tol=1e-10, maxit=100000):
    """Flexible CG with the network as right preconditioner (net None: plain CG)."""
    sol = lattice.vector()
    info = SolveInfo()
    st = lib().stag_fcg_solve(lattice._h, net._h if net is not None else None, mass, shift,
                              _ptr(src), _ptr(sol), tol, maxit, C.byref(info), _stream())
    lattice._chk(st)
    return sol, info


def dslash_batch(lattices, ins, outs=None, out_par=1, prec=PREC_F32):
    """One launch: outs[l][j] = D (to parity out_par) ins[l][j] for every
    lattice l and right-hand side j; ins[l] complex64 CUDA tensors
    [nrhs, V/2, 3].  Returns (outs, (threads per block, rhs per thread))."""
    n = len(lattices)
    if outs is None:
        outs = [_torch().empty_like(x) for x in ins]
    for L, x, y in zip(lattices, ins, outs):
        if x.dim() != 3 or x.shape[1:] != (L.Vh, 3) or y.shape != x.shape or not x.is_contiguous() \
                or not y.is_contiguous():
            raise ValueError("bad batch vector shape")
    hs = (_vp * n)(*[L._h for L in lattices])
    a = (_vp * n)(*[x.data_ptr() for x in ins])
    b = (_vp * n)(*[y.data_ptr() for y in outs])
    nr = (C.c_int * n)(*[int(x.shape[0]) for x in ins])
    cfg = (C.c_int * 2)()
    st = lib().stag_dslash_batch(n, hs, a, b, nr, out_par, prec, cfg, _stream())
    if st != OK:
        raise StagError(st, lib().stag_last_error(lattices[0]._h).decode())
    return outs, (cfg[0], cfg[1])

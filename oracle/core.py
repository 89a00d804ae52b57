"""TEST INFRASTRUCTURE ONLY: ctypes wrappers of the FP64 oracle (stag_oracle.c).

Arrays follow the layout of ``stag_oracle.h``:
  gauge    complex128 [4, V, 3, 3]   (V in lexicographic x-fastest order)
  vector   complex128 [V/2, 3]       (sites of one parity, index lex//2)
  momenta  float64    [4, V, 8]      (P = sum_a w^a lambda^a / 2)
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_LIB_OMP = os.path.join(_LIBDIR, "liboracle_omp.so")
_SRC = os.path.join(_HERE, "stag_oracle.c")

MAXDEG = 32


def build(force=False, openmp=False):
    """Compile the oracle with gcc (portable flags: same results on x86 and Arm).
    openmp=True builds the all-cores variant (OpenMP over the site loops, same
    arithmetic) used only to time the oracle on every host core."""
    os.makedirs(_LIBDIR, exist_ok=True)
    out = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(os.path.join(_HERE, "stag_oracle.h")))):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off"]
    cmd += ["-fopenmp"] if openmp else []
    cmd += ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class Rational(C.Structure):
    _fields_ = [("a0", C.c_double), ("n", C.c_int),
                ("a", C.c_double * MAXDEG), ("b", C.c_double * MAXDEG)]

    @staticmethod
    def make(a0, a, b):
        r = Rational()
        r.a0 = float(a0)
        r.n = len(a)
        assert len(a) == len(b) <= MAXDEG
        for i, (ai, bi) in enumerate(zip(a, b)):
            r.a[i] = float(ai)
            r.b[i] = float(bi)
        return r


class Params(C.Structure):
    _fields_ = [("beta", C.c_double), ("mass", C.c_double), ("tau", C.c_double),
                ("lam", C.c_double), ("tol_md", C.c_double), ("tol_metro", C.c_double),
                ("nsteps", C.c_int), ("integrator", C.c_int), ("npf", C.c_int),
                ("maxit", C.c_int), ("seed", C.c_uint32), ("traj", C.c_uint32),
                ("hb", Rational), ("act", Rational), ("force", Rational), ("ngauge", C.c_int)]


class TrajInfo(C.Structure):
    _fields_ = [("H0", C.c_double), ("H1", C.c_double), ("dH", C.c_double),
                ("u", C.c_double), ("accepted", C.c_int), ("plaq", C.c_double),
                ("cg_iters", C.c_long), ("n_force", C.c_int)]


_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_u32p = C.POINTER(C.c_uint32)


def lib():
    """The oracle library; the all-cores build when ORACLE_OPENMP=1 is set
    before the first call (threads from OMP_NUM_THREADS)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(build(openmp=os.environ.get("ORACLE_OPENMP") == "1"))
        L = _lib
        L.or_volume.restype = C.c_long
        for name in ("or_plaquette", "or_gauge_action", "or_fermion_action", "or_kinetic",
                     "or_metro_uniform"):
            getattr(L, name).restype = C.c_double
    return _lib


def _p(a):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _dims(dims):
    return (C.c_int * 4)(*[int(d) for d in dims])


def volume(dims):
    return int(np.prod(dims))


def new_vector(dims):
    return np.zeros((volume(dims) // 2, 3), np.complex128)


def dslash_full(dims, U, psi):
    out = np.zeros_like(psi)
    lib().or_dslash_full(_dims(dims), _p(U), _p(psi), _p(out))
    return out


def dslash(dims, U, out_parity, psi):
    """D restricted to out_parity <- other parity (D_eo: 0, D_oe: 1)."""
    out = np.zeros_like(psi)
    lib().or_dslash(_dims(dims), _p(U), C.c_int(out_parity), _p(psi), _p(out))
    return out


def apply_M(dims, U, mass, psi):
    out = np.zeros_like(psi)
    lib().or_apply_M(_dims(dims), _p(U), C.c_double(mass), _p(psi), _p(out))
    return out


def cg(dims, U, mass, shift, b, tol=1e-12, maxit=100000):
    x = np.zeros_like(b)
    it = C.c_int(0)
    st = lib().or_cg(_dims(dims), _p(U), C.c_double(mass), C.c_double(shift), _p(b), _p(x),
                     C.c_double(tol), C.c_int(maxit), C.byref(it))
    return x, it.value, st


def multishift(dims, U, mass, shifts, b, tol=1e-12, maxit=100000):
    shifts = np.ascontiguousarray(shifts, np.float64)
    n = len(shifts)
    x = np.zeros((n,) + b.shape, np.complex128)
    its = (C.c_int * n)()
    tot = C.c_int(0)
    st = lib().or_multishift(_dims(dims), _p(U), C.c_double(mass), C.c_int(n), _p(shifts),
                             _p(b), _p(x), C.c_double(tol), C.c_int(maxit), its, C.byref(tot))
    return x, list(its), tot.value, st


def rational_apply(dims, U, mass, a0, a, b, src, tol=1e-12, maxit=100000):
    r = Rational.make(a0, a, b)
    out = np.zeros_like(src)
    it = C.c_int(0)
    lib().or_rational_apply(_dims(dims), _p(U), C.c_double(mass), C.byref(r), _p(src), _p(out),
                            C.c_double(tol), C.c_int(maxit), C.byref(it))
    return out, it.value


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def gauss_pair(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    g = (C.c_double * 2)()
    lib().or_gauss_pair(c, k, g)
    return g[0], g[1]


def uniform_pair(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    g = (C.c_double * 2)()
    lib().or_uniform_pair(c, k, g)
    return g[0], g[1]


def momenta_heatbath(dims, seed, traj):
    w = np.zeros((4, volume(dims), 8))
    lib().or_momenta_heatbath(_dims(dims), C.c_uint32(seed), C.c_uint32(traj), _p(w))
    return w


def pf_gaussian(dims, seed, traj, pf):
    R = new_vector(dims)
    lib().or_pf_gaussian(_dims(dims), C.c_uint32(seed), C.c_uint32(traj), C.c_int(pf), _p(R))
    return R


def metro_uniform(seed, traj):
    return lib().or_metro_uniform(C.c_uint32(seed), C.c_uint32(traj))


def su3_exp_i(X):
    X = np.ascontiguousarray(X, np.complex128)
    out = np.zeros((3, 3), np.complex128)
    lib().or_su3_exp_i(_p(X), _p(out))
    return out


def reunit(U):
    u = np.array(U, np.complex128, copy=True)
    lib().or_reunit(_p(u))
    return u


def omega_to_matrix(w):
    w = np.ascontiguousarray(w, np.float64)
    P = np.zeros((3, 3), np.complex128)
    lib().or_omega_to_matrix(_p(w), _p(P))
    return P


def matrix_to_omega(P):
    P = np.ascontiguousarray(P, np.complex128)
    w = np.zeros(8)
    lib().or_matrix_to_omega(_p(P), _p(w))
    return w


def plaquette(dims, U):
    return lib().or_plaquette(_dims(dims), _p(U))


def gauge_action(dims, U, beta):
    return lib().or_gauge_action(_dims(dims), _p(U), C.c_double(beta))


def gauge_force(dims, U, beta):
    F = np.zeros((4, volume(dims), 8))
    lib().or_gauge_force(_dims(dims), _p(U), C.c_double(beta), _p(F))
    return F


def fermion_force(dims, U, mass, a0, a, b, phi, tol=1e-12, maxit=100000):
    r = Rational.make(a0, a, b)
    F = np.zeros((4, volume(dims), 8))
    it = C.c_int(0)
    st = lib().or_fermion_force(_dims(dims), _p(U), C.c_double(mass), C.byref(r), _p(phi),
                                C.c_double(tol), C.c_int(maxit), _p(F), C.byref(it))
    return F, it.value, st


def fermion_action(dims, U, mass, a0, a, b, phi, tol=1e-12, maxit=100000):
    r = Rational.make(a0, a, b)
    it = C.c_int(0)
    return lib().or_fermion_action(_dims(dims), _p(U), C.c_double(mass), C.byref(r), _p(phi),
                                   C.c_double(tol), C.c_int(maxit), C.byref(it))


def kinetic(dims, w):
    return lib().or_kinetic(_dims(dims), _p(w))


def update_links(dims, U, w, eps):
    U = np.array(U, copy=True)
    lib().or_update_links(_dims(dims), _p(U), _p(w), C.c_double(eps))
    return U


def make_params(beta, mass, tau, nsteps, integrator, hb, act, force, npf=1, tol_md=1e-10,
                tol_metro=1e-10, seed=0, traj=0, lam=0.1931833275037836, maxit=100000, ngauge=0):
    """hb/act/force are (a0, a, b) tuples; ngauge > 0 selects the multi-step
    scheme with ngauge gauge steps per fermion-scheme position update."""
    p = Params()
    p.ngauge = ngauge
    p.beta, p.mass, p.tau, p.lam = beta, mass, tau, lam
    p.tol_md, p.tol_metro = tol_md, tol_metro
    p.nsteps, p.integrator, p.npf, p.maxit = nsteps, integrator, npf, maxit
    p.seed, p.traj = seed, traj
    p.hb = Rational.make(*hb)
    p.act = Rational.make(*act)
    p.force = Rational.make(*force)
    return p


def md_integrate(dims, U, w, phi, params):
    U = np.array(U, copy=True)
    w = np.array(w, copy=True)
    phi = np.ascontiguousarray(phi)
    it = C.c_long(0)
    nf = C.c_int(0)
    st = lib().or_md_integrate(_dims(dims), _p(U), _p(w), _p(phi), C.byref(params),
                               C.byref(it), C.byref(nf))
    return U, w, it.value, nf.value, st


def hamiltonian(dims, U, w, phi, params):
    H = C.c_double(0)
    it = C.c_long(0)
    lib().or_hamiltonian(_dims(dims), _p(U), _p(w), _p(np.ascontiguousarray(phi)),
                         C.byref(params), C.byref(H), C.byref(it))
    return H.value


def trajectory(dims, U, params):
    U = np.array(U, copy=True)
    info = TrajInfo()
    st = lib().or_trajectory(_dims(dims), _p(U), C.byref(params), C.byref(info))
    return U, {f: getattr(info, f) for f, _ in TrajInfo._fields_}, st

"""TEST INFRASTRUCTURE ONLY: the oracle's Remez exchange for the RHMC rational.

RHMC (Sec. 2.1) replaces the root of the fermion matrix by a rational
function evaluated with shifted solvers.  This module computes the best
relative (minimax) approximation

    r(x) = P(x) / Q(x) = a0 + sum_k a_k / (x + b_k),  deg P = deg Q = d,

to x^p on [lo, hi], i.e. the r minimising max |r(x)/x^p - 1|, with the
classical Remez exchange in multiple precision (mpmath):

  1. on a reference set of 2d+2 points solve P(x_i) - x_i^p (1 + (-1)^i E) Q(x_i) = 0
     (Q monic), linearised in E by a fixed-point iteration on Q;
  2. locate the zeros of the error between reference points, then the
     extremum of |error| in each of the 2d+2 intervals they bound;
  3. take those extrema as the new reference; stop when they equioscillate.

The partial fractions follow from the roots of Q: b_k = -root_k,
a_k = P(root_k) / Q'(root_k), a0 = leading coefficient of P.
"""
import mpmath as mp


def _horner(c, x):
    s = mp.mpf(0)
    for ci in reversed(c):
        s = s * x + ci
    return s


def _solve_reference(xs, p, d, E0, scale):
    """Solve the reference equations for P, Q (in t = x/scale) and E."""
    n = 2 * d + 2
    f = [mp.power(x, p) for x in xs]
    t = [x / scale for x in xs]
    qold = None
    E = E0
    for _ in range(60):
        A = mp.matrix(n, n)
        rhs = mp.matrix(n, 1)
        for i in range(n):
            s = 1 if i % 2 == 0 else -1
            for j in range(d + 1):
                A[i, j] = t[i] ** j
            for j in range(d):
                A[i, d + 1 + j] = -f[i] * t[i] ** j
            qo = _horner(qold, t[i]) if qold is not None else t[i] ** d
            A[i, 2 * d + 1] = -s * f[i] * qo
            rhs[i] = f[i] * t[i] ** d
        sol = mp.lu_solve(A, rhs)
        pc = [sol[j] for j in range(d + 1)]
        qc = [sol[d + 1 + j] for j in range(d)] + [mp.mpf(1)]
        Enew = sol[2 * d + 1]
        if qold is not None and abs(Enew - E) <= mp.mpf(10) ** (-(mp.mp.dps - 10)) * abs(Enew):
            E = Enew
            qold = qc
            break
        E = Enew
        qold = qc
    return pc, qc, E


def _golden_max(fun, a, b, iters=80):
    """max of |fun| on [a, b] in log x (unimodal within one interval)."""
    la, lb = mp.log(a), mp.log(b)
    g = (mp.sqrt(5) - 1) / 2
    c = lb - g * (lb - la)
    dd = la + g * (lb - la)
    fc = abs(fun(mp.exp(c)))
    fd = abs(fun(mp.exp(dd)))
    for _ in range(iters):
        if fc > fd:
            lb, dd, fd = dd, c, fc
            c = lb - g * (lb - la)
            fc = abs(fun(mp.exp(c)))
        else:
            la, c, fc = c, dd, fd
            dd = la + g * (lb - la)
            fd = abs(fun(mp.exp(dd)))
    cands = [(abs(fun(a)), a), (abs(fun(b)), b), (fc, mp.exp(c)), (fd, mp.exp(dd))]
    return max(cands, key=lambda z: z[0])


def _bisect_zero(fun, a, b, iters=100):
    fa = fun(a)
    la, lb = mp.log(a), mp.log(b)
    for _ in range(iters):
        m = (la + lb) / 2
        fm = fun(mp.exp(m))
        if (fm > 0) == (fa > 0):
            la, fa = m, fm
        else:
            lb = m
    return mp.exp((la + lb) / 2)


def remez(p, lo, hi, d, dps=80, tol=1e-9, maxiter=60):
    """Best relative approximation of x^p on [lo, hi] of type (d, d).

    Returns dict(a0, a, b, err, extrema, iters) with a, b sorted by pole b."""
    with mp.workdps(dps):
        p, lo, hi = mp.mpf(p), mp.mpf(lo), mp.mpf(hi)
        n = 2 * d + 2
        xs = [lo * mp.power(hi / lo, (1 - mp.cos(mp.pi * i / (n - 1))) / 2) for i in range(n)]
        scale = hi
        E = mp.mpf(0)
        it = 0
        for it in range(1, maxiter + 1):
            pc, qc, E = _solve_reference(xs, p, d, E, scale)
            def err(x, pc=pc, qc=qc):
                return _horner(pc, x / scale) / _horner(qc, x / scale) / mp.power(x, p) - 1

            zs = [_bisect_zero(err, xs[i], xs[i + 1]) for i in range(n - 1)]
            edges = [lo] + zs + [hi]
            ext = [_golden_max(err, edges[i], edges[i + 1]) for i in range(n)]
            xs = [e[1] for e in ext]
            mags = [e[0] for e in ext]
            spread = (max(mags) - min(mags)) / max(mags)
            if spread < tol:
                break
        # partial fractions in x: Q(x) = prod (x - r_k scale) after rescaling
        roots_t = (mp.polyroots(list(reversed(qc)), maxsteps=400, extraprec=4 * dps)
                   if d > 0 else [])
        a, b = [], []
        dq = [j * qc[j] for j in range(1, d + 1)]
        for rt in roots_t:
            rt = mp.re(rt)
            res_t = _horner(pc, rt) / _horner(dq, rt)  # residue in t
            a.append(res_t * scale)                   # dt = dx/scale
            b.append(-rt * scale)
        order = sorted(range(d), key=lambda k: b[k])
        return dict(a0=float(pc[d]), a=[float(a[k]) for k in order],
                    b=[float(b[k]) for k in order], err=float(max(mags)),
                    extrema=[float(x) for x in xs], E=float(E), iters=it,
                    spread=float(spread))


def rational_eval(a0, a, b, x):
    """r(x) = a0 + sum a_k/(x + b_k) in FP64 (numpy arrays accepted)."""
    s = a0
    for ak, bk in zip(a, b):
        s = s + ak / (x + bk)
    return s

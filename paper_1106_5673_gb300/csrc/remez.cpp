// remez.cpp -- host-side Remez exchange for the RHMC rational functions
// (Sec. 2.1: the root of the fermion matrix is replaced by a rational
// function applied with shifted solvers).
//
// Finds the best relative approximation of x^p on [lo, hi] of type (d, d),
//   R(x) = C prod_j (x + z_j) / prod_j (x + b_j),
// i.e. the R minimising max |R(x)/x^p - 1|.  The unknowns are kept in log
// form (log C, log z_j, log b_j) together with the levelled error E; on a
// reference set x_0 < ... < x_{2d+1} the equations
//   log R(x_i) - p log x_i - log(1 + (-1)^i E) = 0
// are solved by damped Newton.  Their Jacobian entries are smooth steps
// z/(x+z), b/(x+b) of order one, so double precision suffices even for wide
// ranges, where the monomial form would need extended precision.  The
// reference set is then exchanged for the extrema of the error until they
// equioscillate.  The result is returned as partial fractions
// a0 + sum_k a_k/(x + b_k): a0 = C, a_k = C prod_j (z_j - b_k) / prod_{j!=k} (b_j - b_k).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/stag.h"

namespace {

struct Approx {
    double p;
    int d;
    double logC;
    std::vector<double> lz, lb;  // log z_j, log b_j
    // log R(x) - p log x
    double logratio(double x) const {
        double s = logC - p * log(x);
        for (int j = 0; j < d; j++) s += log(x + exp(lz[j])) - log(x + exp(lb[j]));
        return s;
    }
    double err(double x) const { return expm1(logratio(x)); }
};

// Gaussian elimination with partial pivoting; A is n x n row-major, solves in place into b
bool solve(std::vector<double>& A, std::vector<double>& b, int n) {
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; k++) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; r++) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return true;
}

// residuals g_i of the reference equations
void residuals(const Approx& a, double E, const std::vector<double>& xs, std::vector<double>& g) {
    const int m = (int)xs.size();
    for (int i = 0; i < m; i++) {
        const double sgn = (i & 1) ? -1.0 : 1.0;
        g[i] = a.logratio(xs[i]) - log1p(sgn * E);
    }
}

double maxabs(const std::vector<double>& v) {
    double m = 0;
    for (double x : v) m = std::max(m, fabs(x));
    return m;
}

// damped Newton on (log C, log z, log b, E) for a fixed reference set
bool newton(Approx& a, double& E, const std::vector<double>& xs) {
    const int d = a.d, m = 2 * d + 2;
    std::vector<double> g(m), J(m * m), rhs(m);
    residuals(a, E, xs, g);
    double gn = maxabs(g);
    for (int it = 0; it < 100 && gn > 1e-15; it++) {
        for (int i = 0; i < m; i++) {
            const double x = xs[i], sgn = (i & 1) ? -1.0 : 1.0;
            double* row = &J[i * m];
            row[0] = 1.0;
            for (int j = 0; j < d; j++) {
                const double z = exp(a.lz[j]), b = exp(a.lb[j]);
                row[1 + j] = z / (x + z);
                row[1 + d + j] = -b / (x + b);
            }
            row[m - 1] = -sgn / (1.0 + sgn * E);
            rhs[i] = -g[i];
        }
        std::vector<double> Jc = J;
        if (!solve(Jc, rhs, m)) return false;
        // trust region: no log-parameter moves by more than 0.5 per step (a pole
        // pushed far outside [lo, hi] makes its Jacobian column degenerate)
        double big = 0.0;
        for (int k = 0; k < m - 1; k++) big = std::max(big, fabs(rhs[k]));
        double step = big > 0.5 ? 0.5 / big : 1.0;
        bool ok = false;
        for (int tries = 0; tries < 40; tries++) {
            Approx t = a;
            t.logC += step * rhs[0];
            for (int j = 0; j < d; j++) {
                t.lz[j] += step * rhs[1 + j];
                t.lb[j] += step * rhs[1 + d + j];
            }
            double tE = E + step * rhs[m - 1];
            if (fabs(tE) < 0.5) {
                std::vector<double> tg(m);
                residuals(t, tE, xs, tg);
                double tn = maxabs(tg);
                if (tn < gn || tn < 1e-15) {
                    a = t;
                    E = tE;
                    g = tg;
                    gn = tn;
                    ok = true;
                    break;
                }
            }
            step *= 0.5;
        }
        if (!ok) break;
    }
    return gn < 1e-11;
}

double golden_max(const Approx& a, double lo, double hi, double* xbest) {
    double la = log(lo), lb = log(hi);
    const double gr = (sqrt(5.0) - 1.0) / 2.0;
    double c = lb - gr * (lb - la), dd = la + gr * (lb - la);
    double fc = fabs(a.err(exp(c))), fd = fabs(a.err(exp(dd)));
    for (int it = 0; it < 100 && lb - la > 1e-13 * (1 + fabs(la)); it++) {
        if (fc > fd) {
            lb = dd; dd = c; fd = fc;
            c = lb - gr * (lb - la);
            fc = fabs(a.err(exp(c)));
        } else {
            la = c; c = dd; fc = fd;
            dd = la + gr * (lb - la);
            fd = fabs(a.err(exp(dd)));
        }
    }
    double best = fabs(a.err(lo)), xb = lo;
    const double cand[3] = {hi, exp(c), exp(dd)};
    for (double x : cand) {
        double v = fabs(a.err(x));
        if (v > best) { best = v; xb = x; }
    }
    *xbest = xb;
    return best;
}

double bisect_zero(const Approx& a, double lo, double hi) {
    double la = log(lo), lb = log(hi);
    double fa = a.err(lo);
    for (int it = 0; it < 200 && lb - la > 1e-14 * (1 + fabs(la)); it++) {
        double m = 0.5 * (la + lb);
        double fm = a.err(exp(m));
        if ((fm > 0) == (fa > 0)) { la = m; fa = fm; } else { lb = m; }
    }
    return exp(0.5 * (la + lb));
}

// Remez exchange from the starting approximation `a` on [lo, hi]; returns
// true when the reference errors equioscillate to 1e-9.
bool exchange(Approx& a, double lo, double hi, double* emax_out) {
    const int d = a.d, m = 2 * d + 2;
    std::vector<double> xs(m);
    for (int i = 0; i < m; i++) xs[i] = lo * pow(hi / lo, 0.5 * (1.0 - cos(M_PI * i / (m - 1))));
    double E = 0.0, spread = 1.0, emax = 0.0;
    for (int iter = 0; iter < 80; iter++) {
        Approx keep = a;
        if (!newton(a, E, xs)) {
            a = keep;
            if (iter == 0) return false;
        }
        std::vector<double> edges(m + 1);
        edges[0] = lo;
        edges[m] = hi;
        for (int i = 0; i < m - 1; i++) edges[i + 1] = bisect_zero(a, xs[i], xs[i + 1]);
        std::vector<double> nx(m);
        double mn = 1e300;
        emax = 0.0;
        for (int i = 0; i < m; i++) {
            double v = golden_max(a, edges[i], edges[i + 1], &nx[i]);
            mn = std::min(mn, v);
            emax = std::max(emax, v);
        }
        if (!isfinite(emax)) return false;
        spread = (emax - mn) / emax;
        xs = nx;
        if (spread < 1e-9) break;
    }
    *emax_out = emax;
    return spread < 1e-5;
}

// starting guess: poles log-uniform over [lo e^-1.3, hi e^0.5], zeros offset
// by |p| of the pole spacing (above the pole for p < 0, below for p > 0), C
// levelled so that the log error is centred
Approx initial_guess(double p, int d, double lo, double hi) {
    Approx a;
    a.p = p;
    a.d = d;
    a.lz.resize(d);
    a.lb.resize(d);
    const double L0 = log(lo) - 1.3, L1 = log(hi) + 0.5;
    const double h = (L1 - L0) / (d > 1 ? d - 1 : 1);
    for (int j = 0; j < d; j++) {
        a.lb[j] = (d > 1) ? L0 + j * h : 0.5 * (L0 + L1);
        a.lz[j] = a.lb[j] - p * (d > 1 ? h : (L1 - L0) / 2);
    }
    double mn = 1e300, mx = -1e300;
    a.logC = 0.0;
    for (int i = 0; i <= 200; i++) {
        double v = a.logratio(exp(log(lo) + (log(hi) - log(lo)) * i / 200.0));
        mn = std::min(mn, v);
        mx = std::max(mx, v);
    }
    a.logC = -0.5 * (mn + mx);
    return a;
}

}  // namespace

extern "C" int stag_remez(double power, double lo, double hi, int degree, stag_rational* out, double* max_rel_err) {
    if (!out || !(lo > 0) || !(hi > lo) || degree < 0 || degree > STAG_MAXSHIFT || !isfinite(power))
        return STAG_ERR_ARG;
    memset(out, 0, sizeof(*out));
    const int d = degree;
    if (d == 0) {
        out->a0 = 2.0 / (pow(lo, -power) + pow(hi, -power));
        out->n = 0;
        if (max_rel_err) *max_rel_err = fabs(out->a0 * pow(lo, -power) - 1.0);
        return STAG_OK;
    }
    double emax = 0.0;
    Approx a = initial_guess(power, d, lo, hi);
    if (!exchange(a, lo, hi, &emax)) {
        // continuation in the degree: converge at a low degree, then resample
        // the ladders of log-poles and log-zeros to one more point (linear
        // interpolation in the normalised index) and converge again
        int d0 = std::min(d, 8);
        a = initial_guess(power, d0, lo, hi);
        bool ok = exchange(a, lo, hi, &emax);
        for (int dd = d0 + 1; ok && dd <= d; dd++) {
            Approx b;
            b.p = power;
            b.d = dd;
            b.logC = a.logC;
            b.lz.resize(dd);
            b.lb.resize(dd);
            for (int j = 0; j < dd; j++) {
                const double t = (double)j * (a.d - 1) / (dd - 1);
                const int i0 = std::min((int)t, a.d - 2);
                const double f = t - i0;
                b.lb[j] = (1 - f) * a.lb[i0] + f * a.lb[i0 + 1];
                b.lz[j] = (1 - f) * a.lz[i0] + f * a.lz[i0 + 1];
            }
            a = b;
            ok = exchange(a, lo, hi, &emax);
        }
        if (!ok) return STAG_ERR_NOCONV;
    }
    // partial fractions
    const double C = exp(a.logC);
    out->a0 = C;
    out->n = d;
    std::vector<int> order(d);
    for (int j = 0; j < d; j++) order[j] = j;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return a.lb[x] < a.lb[y]; });
    for (int kk = 0; kk < d; kk++) {
        const int k = order[kk];
        const double bk = exp(a.lb[k]);
        double num = C, den = 1.0;
        for (int j = 0; j < d; j++) {
            num *= exp(a.lz[j]) - bk;
            if (j != k) den *= exp(a.lb[j]) - bk;
        }
        out->a[kk] = num / den;
        out->b[kk] = bk;
    }
    if (max_rel_err) {
        double e = 0.0;
        const int N = 20000;
        for (int i = 0; i <= N; i++) {
            double x = exp(log(lo) + (log(hi) - log(lo)) * i / N);
            double r = out->a0;
            for (int k = 0; k < d; k++) r += out->a[k] / (x + out->b[k]);
            e = std::max(e, fabs(r / pow(x, power) - 1.0));
        }
        *max_rel_err = std::max(e, emax);
        if (!isfinite(*max_rel_err)) return STAG_ERR_NOCONV;
    }
    return STAG_OK;
}

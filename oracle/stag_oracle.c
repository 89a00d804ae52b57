/*
 * stag_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of the two-flavour staggered RHMC
 * of Bonati, Cossu, D'Elia, Incardona, "QCD simulations with staggered
 * fermions on GPUs" (arXiv:1106.5673).  Every routine follows the paper's
 * definition (or, where the paper is silent, the textbook definition it
 * cites) with no blocking, fusion or reordering, so that it can be checked by
 * eye.  The CUDA library is checked against it; the two share no code.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.
 *
 * The loops over sites and links that write one output per site carry
 * OpenMP pragmas; the default build ignores them (single thread).  The
 * all-cores build (-fopenmp) spreads only those loops over the host cores:
 * every output is computed by the same operations in the same order, and the
 * dot products stay serial, so both builds give identical results.
 *
 * Layout conventions are listed in stag_oracle.h.
 */
#include "stag_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Lattice indexing (Sec. 2: links U_mu(n) on a hypercubic L_x L_y L_z L_t */
/* lattice; even/odd preconditioning, Sec. 2.1, keeps fields on one parity) */
/* ------------------------------------------------------------------------ */

typedef struct {
    int L[4];
    long V, Vh;
} olat;

static void lat_init(olat *l, const int dims[4])
{
    for (int m = 0; m < 4; m++) l->L[m] = dims[m];
    l->V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    l->Vh = l->V / 2;
}

long or_volume(const int dims[4])
{
    return (long)dims[0] * dims[1] * dims[2] * dims[3];
}

static void coords(const olat *l, long lex, int x[4])
{
    x[0] = (int)(lex % l->L[0]); lex /= l->L[0];
    x[1] = (int)(lex % l->L[1]); lex /= l->L[1];
    x[2] = (int)(lex % l->L[2]);
    x[3] = (int)(lex / l->L[2]);
}

static long lexof(const olat *l, const int x[4])
{
    return x[0] + (long)l->L[0] * (x[1] + (long)l->L[1] * (x[2] + (long)l->L[2] * x[3]));
}

static int parity_of(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

/* site n + dir * mu-hat, periodic in all four directions */
static long neighbour(const olat *l, long lex, int mu, int dir)
{
    int x[4];
    coords(l, lex, x);
    x[mu] = (x[mu] + dir + l->L[mu]) % l->L[mu];
    return lexof(l, x);
}

/* Staggered phase eta_mu(n) = (-1)^(n_x + ... + n_{mu-1}) of Eq. (4), times
 * the antiperiodic temporal boundary sign of the fermion field, attached to
 * the link U_mu(n): a hop across the link from t = L_t-1 to t = 0 (forward
 * from n, or backward from n + mu-hat) picks up an extra -1.  Since eta_mu
 * does not depend on n_mu, eta_mu(n) = eta_mu(n + mu-hat) and both hops
 * across the same link carry the same sign. */
static double link_sign(const olat *l, const int x[4], int mu)
{
    int s = 0;
    for (int nu = 0; nu < mu; nu++) s += x[nu];
    double eta = (s & 1) ? -1.0 : 1.0;
    if (mu == 3 && x[3] == l->L[3] - 1) eta = -eta;
    return eta;
}

/* ------------------------------------------------------------------------ */
/* 3x3 complex matrices                                                     */
/* ------------------------------------------------------------------------ */

typedef struct { cplx e[3][3]; } mat3;

static mat3 load_mat(const double *p)
{
    mat3 m;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            m.e[a][b] = p[2 * (3 * a + b)] + I * p[2 * (3 * a + b) + 1];
    return m;
}

static void store_mat(double *p, const mat3 *m)
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            p[2 * (3 * a + b)] = creal(m->e[a][b]);
            p[2 * (3 * a + b) + 1] = cimag(m->e[a][b]);
        }
}

static mat3 link_at(const olat *l, const double *U, int mu, long lex)
{
    return load_mat(U + 18 * (mu * l->V + lex));
}

static mat3 mmul(const mat3 *a, const mat3 *b)
{
    mat3 c;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a->e[i][k] * b->e[k][j];
            c.e[i][j] = s;
        }
    return c;
}

static mat3 dag(const mat3 *a)
{
    mat3 c;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c.e[i][j] = conj(a->e[j][i]);
    return c;
}

static mat3 madd(const mat3 *a, const mat3 *b)
{
    mat3 c;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c.e[i][j] = a->e[i][j] + b->e[i][j];
    return c;
}

static mat3 mscale(const mat3 *a, cplx s)
{
    mat3 c;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c.e[i][j] = s * a->e[i][j];
    return c;
}

static mat3 mzero(void)
{
    mat3 c;
    memset(&c, 0, sizeof c);
    return c;
}

static mat3 munit(void)
{
    mat3 c = mzero();
    for (int i = 0; i < 3; i++) c.e[i][i] = 1;
    return c;
}

static cplx mtrace(const mat3 *a) { return a->e[0][0] + a->e[1][1] + a->e[2][2]; }

/* Traceless anti-Hermitian part TA(W) = (W - W^dag)/2 - Tr(W - W^dag)/6 */
static mat3 traceless_antiherm(const mat3 *W)
{
    mat3 Wd = dag(W), A;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) A.e[i][j] = 0.5 * (W->e[i][j] - Wd.e[i][j]);
    cplx tr = mtrace(&A) / 3.0;
    for (int i = 0; i < 3; i++) A.e[i][i] -= tr;
    return A;
}

/* Gell-Mann matrices lambda^a, a = 1..8 (index 0..7).  The momenta of
 * Sec. 2.1 are H = sum_a T^a omega^a with T^a = lambda^a / 2. */
static mat3 gell_mann(int a)
{
    mat3 g = mzero();
    switch (a) {
    case 0: g.e[0][1] = 1; g.e[1][0] = 1; break;
    case 1: g.e[0][1] = -I; g.e[1][0] = I; break;
    case 2: g.e[0][0] = 1; g.e[1][1] = -1; break;
    case 3: g.e[0][2] = 1; g.e[2][0] = 1; break;
    case 4: g.e[0][2] = -I; g.e[2][0] = I; break;
    case 5: g.e[1][2] = 1; g.e[2][1] = 1; break;
    case 6: g.e[1][2] = -I; g.e[2][1] = I; break;
    case 7:
        g.e[0][0] = 1 / sqrt(3.0); g.e[1][1] = 1 / sqrt(3.0); g.e[2][2] = -2 / sqrt(3.0);
        break;
    }
    return g;
}

static mat3 omega_to_mat(const double *w)
{
    mat3 P = mzero();
    for (int a = 0; a < 8; a++) {
        mat3 g = gell_mann(a);
        mat3 t = mscale(&g, 0.5 * w[a]);
        P = madd(&P, &t);
    }
    return P;
}

/* omega^a = Tr(P lambda^a) for traceless Hermitian P = sum_a omega^a lambda^a / 2 */
static void mat_to_omega(const mat3 *P, double *w)
{
    for (int a = 0; a < 8; a++) {
        mat3 g = gell_mann(a);
        mat3 t = mmul(P, &g);
        w[a] = creal(mtrace(&t));
    }
}

void or_omega_to_matrix(const double *w, double *P)
{
    mat3 m = omega_to_mat(w);
    store_mat(P, &m);
}

void or_matrix_to_omega(const double *P, double *w)
{
    mat3 m = load_mat(P);
    mat_to_omega(&m, w);
}

/* exp(i X) for a 3x3 matrix X by its Taylor series with scaling and squaring:
 * scale X by 2^-s until its Frobenius norm is below 1/2, sum 24 terms of the
 * series, then square s times. */
static mat3 exp_i(const mat3 *X)
{
    double nrm = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) nrm += creal(X->e[i][j] * conj(X->e[i][j]));
    nrm = sqrt(nrm);
    int s = 0;
    while (nrm > 0.5) { nrm *= 0.5; s++; }
    mat3 Y = mscale(X, I * ldexp(1.0, -s));
    mat3 T = munit(), term = munit();
    for (int k = 1; k <= 24; k++) {
        term = mmul(&term, &Y);
        term = mscale(&term, 1.0 / k);
        T = madd(&T, &term);
    }
    for (int k = 0; k < s; k++) T = mmul(&T, &T);
    return T;
}

void or_su3_exp_i(const double *X, double *out)
{
    mat3 x = load_mat(X), e = exp_i(&x);
    store_mat(out, &e);
}

/* Reunitarisation (Sec. 4.1): Gram-Schmidt on the first two rows, the third
 * row rebuilt as the complex conjugate of their cross product (det = 1). */
static void reunit(mat3 *U)
{
    double n0 = 0;
    for (int j = 0; j < 3; j++) n0 += creal(U->e[0][j] * conj(U->e[0][j]));
    n0 = 1.0 / sqrt(n0);
    for (int j = 0; j < 3; j++) U->e[0][j] *= n0;
    cplx d = 0;
    for (int j = 0; j < 3; j++) d += conj(U->e[0][j]) * U->e[1][j];
    for (int j = 0; j < 3; j++) U->e[1][j] -= d * U->e[0][j];
    double n1 = 0;
    for (int j = 0; j < 3; j++) n1 += creal(U->e[1][j] * conj(U->e[1][j]));
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; j++) U->e[1][j] *= n1;
    U->e[2][0] = conj(U->e[0][1] * U->e[1][2] - U->e[0][2] * U->e[1][1]);
    U->e[2][1] = conj(U->e[0][2] * U->e[1][0] - U->e[0][0] * U->e[1][2]);
    U->e[2][2] = conj(U->e[0][0] * U->e[1][1] - U->e[0][1] * U->e[1][0]);
}

void or_reunit(double *Up)
{
    mat3 u = load_mat(Up);
    reunit(&u);
    store_mat(Up, &u);
}

/* ------------------------------------------------------------------------ */
/* Staggered operator, Eq. (4) with a = 1:                                   */
/*   (D psi)(n) = 1/2 sum_mu eta_mu(n) [U_mu(n) psi(n+mu) -                 */
/*                                      U_mu(n-mu)^dag psi(n-mu)]           */
/* and M = m + D.  D is anti-Hermitian and maps one parity to the other.    */
/* ------------------------------------------------------------------------ */

static void hop_site(const olat *l, const double *U, long lex, const cplx *in, int full,
                     cplx out[3])
{
    int x[4];
    coords(l, lex, x);
    cplx acc[3] = {0, 0, 0};
    for (int mu = 0; mu < 4; mu++) {
        long f = neighbour(l, lex, mu, +1);
        long b = neighbour(l, lex, mu, -1);
        int xb[4];
        coords(l, b, xb);
        double sf = link_sign(l, x, mu), sb = link_sign(l, xb, mu);
        mat3 Uf = link_at(l, U, mu, lex), Ub = link_at(l, U, mu, b);
        const cplx *pf = in + 3 * (full ? f : f / 2);
        const cplx *pb = in + 3 * (full ? b : b / 2);
        for (int a = 0; a < 3; a++) {
            cplx s = 0;
            for (int c = 0; c < 3; c++)
                s += sf * Uf.e[a][c] * pf[c] - sb * conj(Ub.e[c][a]) * pb[c];
            acc[a] += s;
        }
    }
    for (int a = 0; a < 3; a++) out[a] = 0.5 * acc[a];
}

void or_dslash_full(const int dims[4], const double *U, const double *in, double *out)
{
    olat l;
    lat_init(&l, dims);
    const cplx *vin = (const cplx *)in;
    cplx *vout = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long lex = 0; lex < l.V; lex++) hop_site(&l, U, lex, vin, 1, vout + 3 * lex);
}

/* D restricted to out_parity <- 1 - out_parity (D_eo for out_parity = 0,
 * D_oe for out_parity = 1); both fields indexed by lex/2. */
void or_dslash(const int dims[4], const double *U, int out_parity, const double *in, double *out)
{
    olat l;
    lat_init(&l, dims);
    const cplx *vin = (const cplx *)in;
    cplx *vout = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long lex = 0; lex < l.V; lex++) {
        int x[4];
        coords(&l, lex, x);
        if (parity_of(x) != out_parity) continue;
        hop_site(&l, U, lex, vin, 0, vout + 3 * (lex / 2));
    }
}

/* Even-site normal operator M^dag M restricted to even sites:
 * M_ee = m^2 - D_eo D_oe (even/odd preconditioning, Sec. 2.1). */
void or_apply_M(const int dims[4], const double *U, double mass, const double *in, double *out)
{
    long Vh = or_volume(dims) / 2;
    double *tmp = malloc(sizeof(double) * 6 * Vh);
    double *tmp2 = malloc(sizeof(double) * 6 * Vh);
    or_dslash(dims, U, 1, in, tmp);
    or_dslash(dims, U, 0, tmp, tmp2);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < 6 * Vh; i++) out[i] = mass * mass * in[i] - tmp2[i];
    free(tmp);
    free(tmp2);
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers (Sec. 4.3)                                                 */
/* ------------------------------------------------------------------------ */

static double dotr(long n, const double *a, const double *b)
{
    double s = 0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Plain CG for (M_ee + shift) x = b from x = 0; stops when
 * |b - (M+shift)x|_recursive <= tol |b|.  Returns 0 on convergence. */
int or_cg(const int dims[4], const double *U, double mass, double shift, const double *b,
          double *x, double tol, int maxit, int *iters)
{
    long n = 6 * (or_volume(dims) / 2);
    double *r = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n);
    double *w = malloc(sizeof(double) * n);
    memset(x, 0, sizeof(double) * n);
    memcpy(r, b, sizeof(double) * n);
    memcpy(p, b, sizeof(double) * n);
    double bb = dotr(n, b, b), rr = bb;
    int k = 0, status = 1;
    if (bb == 0) status = 0;
    while (status && k < maxit) {
        or_apply_M(dims, U, mass, p, w);
        for (long i = 0; i < n; i++) w[i] += shift * p[i];
        double alpha = rr / dotr(n, p, w);
        for (long i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * w[i]; }
        double rr_new = dotr(n, r, r);
        k++;
        if (sqrt(rr_new) <= tol * sqrt(bb)) { status = 0; break; }
        double beta = rr_new / rr;
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    if (iters) *iters = k;
    free(r); free(p); free(w);
    return status;
}

/* Multi-shift CG for (M_ee + shifts[k]) x_k = b, k = 0..n-1, all from x = 0
 * in one Krylov space (the shifted solver of Eq. (13)).  The base system is
 * the smallest shift s0; shift k with d_k = shifts[k] - s0 has residual
 * zeta_k r, with the textbook recurrence
 *   zeta^{j+1} = zeta^j zeta^{j-1} a_{j-1} /
 *       (zeta^{j-1} a_{j-1} (1 + d a_j) + a_j b_{j-1} (zeta^{j-1} - zeta^j))
 *   a_k = a_j zeta^{j+1}/zeta^j,  b_k = b_j (zeta^{j+1}/zeta^j)^2,
 *   x_k += a_k p_k,  p_k <- zeta^{j+1} r_{j+1} + b_k p_k,
 * started from zeta^{-1} = zeta^0 = 1, a_{-1} = 1, b_{-1} = 0.  Shift k stops
 * updating once |zeta_k| |r| <= tol |b|.  x is n consecutive parity fields. */
int or_multishift(const int dims[4], const double *U, double mass, int n, const double *shifts,
                  const double *b, double *x, double tol, int maxit, int *iters_shift,
                  int *iters_total)
{
    long N = 6 * (or_volume(dims) / 2);
    int base = 0;
    for (int k = 1; k < n; k++)
        if (shifts[k] < shifts[base]) base = k;
    double s0 = shifts[base];
    double *r = malloc(sizeof(double) * N), *p = malloc(sizeof(double) * N);
    double *w = malloc(sizeof(double) * N);
    double *pk = malloc(sizeof(double) * N * n);
    double *zeta = malloc(sizeof(double) * n), *zeta_old = malloc(sizeof(double) * n);
    double *zeta_new = malloc(sizeof(double) * n);
    int *active = malloc(sizeof(int) * n);
    memset(x, 0, sizeof(double) * N * n);
    memcpy(r, b, sizeof(double) * N);
    memcpy(p, b, sizeof(double) * N);
    for (int k = 0; k < n; k++) {
        memcpy(pk + k * N, b, sizeof(double) * N);
        zeta[k] = zeta_old[k] = 1.0;
        active[k] = 1;
        if (iters_shift) iters_shift[k] = 0;
    }
    double bb = dotr(N, b, b), rr = bb;
    double alpha_old = 1.0, beta_old = 0.0;
    int j = 0, n_active = (bb > 0) ? n : 0;
    if (bb == 0) for (int k = 0; k < n; k++) active[k] = 0;
    while (n_active > 0 && j < maxit) {
        or_apply_M(dims, U, mass, p, w);
        for (long i = 0; i < N; i++) w[i] += s0 * p[i];
        double alpha = rr / dotr(N, p, w);
        for (int k = 0; k < n; k++) {
            if (!active[k]) continue;
            double d = shifts[k] - s0;
            double den = zeta_old[k] * alpha_old * (1.0 + d * alpha) +
                         alpha * beta_old * (zeta_old[k] - zeta[k]);
            zeta_new[k] = zeta[k] * zeta_old[k] * alpha_old / den;
            double ak = alpha * zeta_new[k] / zeta[k];
            double *xk = x + k * N, *pkk = pk + k * N;
#pragma omp parallel for schedule(static)
            for (long i = 0; i < N; i++) xk[i] += ak * pkk[i];
        }
        for (long i = 0; i < N; i++) r[i] -= alpha * w[i];
        double rr_new = dotr(N, r, r);
        double beta = rr_new / rr;
        j++;
        for (long i = 0; i < N; i++) p[i] = r[i] + beta * p[i];
        for (int k = 0; k < n; k++) {
            if (!active[k]) continue;
            double ratio = zeta_new[k] / zeta[k];
            double bk = beta * ratio * ratio;
            double *pkk = pk + k * N;
#pragma omp parallel for schedule(static)
            for (long i = 0; i < N; i++) pkk[i] = zeta_new[k] * r[i] + bk * pkk[i];
            zeta_old[k] = zeta[k];
            zeta[k] = zeta_new[k];
            if (iters_shift) iters_shift[k] = j;
            if (fabs(zeta[k]) * sqrt(rr_new) <= tol * sqrt(bb)) {
                active[k] = 0;
                n_active--;
            }
        }
        rr = rr_new;
        alpha_old = alpha;
        beta_old = beta;
    }
    if (iters_total) *iters_total = j;
    free(r); free(p); free(w); free(pk);
    free(zeta); free(zeta_old); free(zeta_new); free(active);
    return n_active > 0 ? 1 : 0;
}

/* out = r(M_ee) src = a0 src + sum_k a_k (M_ee + b_k)^{-1} src  (RHMC, Sec. 2.1) */
void or_rational_apply(const int dims[4], const double *U, double mass, const or_rational *r,
                       const double *src, double *out, double tol, int maxit, int *iters)
{
    long N = 6 * (or_volume(dims) / 2);
    double *x = malloc(sizeof(double) * N * r->n);
    int it = 0;
    or_multishift(dims, U, mass, r->n, r->b, src, x, tol, maxit, NULL, &it);
    for (long i = 0; i < N; i++) {
        double s = r->a0 * src[i];
        for (int k = 0; k < r->n; k++) s += r->a[k] * x[k * N + i];
        out[i] = s;
    }
    if (iters) *iters = it;
    free(x);
}

/* ------------------------------------------------------------------------ */
/* Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), a     */
/* counter-based generator, and Box-Muller Gaussians in FP64.  The paper    */
/* draws the heatbath on the host with an unspecified generator (Sec. 4).   */
/* ------------------------------------------------------------------------ */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two uniforms in (0, 1]: 53 bits from each pair of 32-bit words. */
void or_uniform_pair(const uint32_t ctr[4], const uint32_t key[2], double u[2])
{
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    uint64_t k1 = ((uint64_t)o[0] << 21) | (o[1] >> 11);
    uint64_t k2 = ((uint64_t)o[2] << 21) | (o[3] >> 11);
    u[0] = ((double)k1 + 1.0) * 0x1p-53;
    u[1] = ((double)k2 + 1.0) * 0x1p-53;
}

/* Box-Muller: two independent N(0,1) numbers. */
void or_gauss_pair(const uint32_t ctr[4], const uint32_t key[2], double g[2])
{
    double u[2];
    or_uniform_pair(ctr, key, u);
    double rad = sqrt(-2.0 * log(u[0]));
    double th = 2.0 * M_PI * u[1];
    g[0] = rad * cos(th);
    g[1] = rad * sin(th);
}

enum { FIELD_MOM = 1, FIELD_PF = 2, FIELD_METRO = 3 };

/* Momentum heatbath (Sec. 2.1, Phi algorithm step 2): each omega^a_mu(n) is
 * N(0,1), so that the kinetic term sum Tr H^2 = 1/2 sum omega^2. */
void or_momenta_heatbath(const int dims[4], uint32_t seed, uint32_t traj, double *w)
{
    long V = or_volume(dims);
    uint32_t key[2] = {seed, traj};
    for (int mu = 0; mu < 4; mu++)
        for (long lex = 0; lex < V; lex++)
            for (int blk = 0; blk < 4; blk++) {
                uint32_t ctr[4] = {FIELD_MOM, (uint32_t)mu, (uint32_t)lex, (uint32_t)blk};
                double g[2];
                or_gauss_pair(ctr, key, g);
                w[8 * (mu * V + lex) + 2 * blk] = g[0];
                w[8 * (mu * V + lex) + 2 * blk + 1] = g[1];
            }
}

/* Complex Gaussian R on even sites with density proportional to
 * exp(-R^dag R) (Sec. 2.1, Phi algorithm step 1): each real and imaginary
 * part is N(0, 1/2). */
void or_pf_gaussian(const int dims[4], uint32_t seed, uint32_t traj, int pf, double *R)
{
    olat l;
    lat_init(&l, dims);
    uint32_t key[2] = {seed, traj};
    for (long lex = 0; lex < l.V; lex++) {
        int x[4];
        coords(&l, lex, x);
        if (parity_of(x) != 0) continue;
        for (int c = 0; c < 3; c++) {
            uint32_t ctr[4] = {FIELD_PF, (uint32_t)pf, (uint32_t)lex, (uint32_t)c};
            double g[2];
            or_gauss_pair(ctr, key, g);
            R[6 * (lex / 2) + 2 * c] = g[0] * sqrt(0.5);
            R[6 * (lex / 2) + 2 * c + 1] = g[1] * sqrt(0.5);
        }
    }
}

double or_metro_uniform(uint32_t seed, uint32_t traj)
{
    uint32_t key[2] = {seed, traj};
    uint32_t ctr[4] = {FIELD_METRO, 0, 0, 0};
    double u[2];
    or_uniform_pair(ctr, key, u);
    return u[0];
}

/* ------------------------------------------------------------------------ */
/* Gauge action and forces                                                   */
/* ------------------------------------------------------------------------ */

/* U_mu nu(n) = U_mu(n) U_nu(n+mu) U_mu(n+nu)^dag U_nu(n)^dag */
static mat3 plaq_mat(const olat *l, const double *U, long lex, int mu, int nu)
{
    mat3 a = link_at(l, U, mu, lex);
    mat3 b = link_at(l, U, nu, neighbour(l, lex, mu, 1));
    mat3 c = link_at(l, U, mu, neighbour(l, lex, nu, 1));
    mat3 d = link_at(l, U, nu, lex);
    mat3 cd = dag(&c), dd = dag(&d);
    mat3 t = mmul(&a, &b);
    t = mmul(&t, &cd);
    return mmul(&t, &dd);
}

/* Average plaquette (1/6V) sum_{n, mu<nu} Re Tr U_mu nu(n) / 3 */
double or_plaquette(const int dims[4], const double *U)
{
    olat l;
    lat_init(&l, dims);
    double s = 0;
    for (long lex = 0; lex < l.V; lex++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                mat3 p = plaq_mat(&l, U, lex, mu, nu);
                s += creal(mtrace(&p)) / 3.0;
            }
    return s / (6.0 * l.V);
}

/* The "simple plaquette action" of Sec. 2 read as the Wilson action
 * S_g = beta sum_{n, mu<nu} (1 - Re Tr U_mu nu(n) / 3). */
double or_gauge_action(const int dims[4], const double *U, double beta)
{
    olat l;
    lat_init(&l, dims);
    double s = 0;
    for (long lex = 0; lex < l.V; lex++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                mat3 p = plaq_mat(&l, U, lex, mu, nu);
                s += 1.0 - creal(mtrace(&p)) / 3.0;
            }
    return beta * s;
}

/* Sum of the six staples A_mu(n) with sum_{plaquettes with U_mu(n)} Re Tr U_P
 * = Re Tr (U_mu(n) A_mu(n)). */
static mat3 staple_sum(const olat *l, const double *U, long lex, int mu)
{
    mat3 A = mzero();
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        long n_mu = neighbour(l, lex, mu, 1), n_nu = neighbour(l, lex, nu, 1);
        long n_mnu = neighbour(l, lex, nu, -1);
        long n_mu_mnu = neighbour(l, n_mu, nu, -1);
        /* U_nu(n+mu) U_mu(n+nu)^dag U_nu(n)^dag */
        mat3 a = link_at(l, U, nu, n_mu), b = link_at(l, U, mu, n_nu), c = link_at(l, U, nu, lex);
        mat3 bd = dag(&b), cd = dag(&c);
        mat3 t = mmul(&a, &bd);
        t = mmul(&t, &cd);
        A = madd(&A, &t);
        /* U_nu(n+mu-nu)^dag U_mu(n-nu)^dag U_nu(n-nu) */
        mat3 e = link_at(l, U, nu, n_mu_mnu), f = link_at(l, U, mu, n_mnu), g = link_at(l, U, nu, n_mnu);
        mat3 ed = dag(&e), fd = dag(&f);
        t = mmul(&ed, &fd);
        t = mmul(&t, &g);
        A = madd(&A, &t);
    }
    return A;
}

/* Gauge force dP/dtau for U' = i P U and H = sum Tr P^2 + S_g:
 * dP_mu(n)/dtau = (i beta / 6) TA(U_mu(n) A_mu(n)), returned as omega^a. */
void or_gauge_force(const int dims[4], const double *U, double beta, double *F)
{
    olat l;
    lat_init(&l, dims);
    for (int mu = 0; mu < 4; mu++)
#pragma omp parallel for schedule(static)
        for (long lex = 0; lex < l.V; lex++) {
            mat3 u = link_at(&l, U, mu, lex), A = staple_sum(&l, U, lex, mu);
            mat3 W = mmul(&u, &A);
            mat3 T = traceless_antiherm(&W);
            mat3 Pd = mscale(&T, I * beta / 6.0);
            mat_to_omega(&Pd, F + 8 * (mu * l.V + lex));
        }
}

/* Fermion action S_f = phi^dag r(M_ee) phi of the rooted pseudofermion
 * (Eq. (3) with the rooting of Eq. (5), r approximating x^{-1/2}). */
double or_fermion_action(const int dims[4], const double *U, double mass, const or_rational *r,
                         const double *phi, double tol, int maxit, int *iters)
{
    long N = 6 * (or_volume(dims) / 2);
    double *y = malloc(sizeof(double) * N);
    or_rational_apply(dims, U, mass, r, phi, y, tol, maxit, iters);
    double s = dotr(N, phi, y);
    free(y);
    return s;
}

/* Fermion force of S_f = phi^dag r(M_ee) phi, r(x) = a0 + sum_k a_k/(x+b_k).
 * With X_k = (M_ee + b_k)^{-1} phi (even) and Y_k = D_oe X_k (odd),
 *   dS_f = -2 sum_k a_k Re Y_k^dag dD_oe X_k,
 * and for U' = i P U the link U_mu(m) with sign s_mu(m) (staggered phase and
 * boundary) gets dP/dtau = i TA(W), W = (s_mu(m)/2) U_mu(m) sum_k a_k Z_k,
 *   Z_k = X_k(m+mu) Y_k(m)^dag      for m odd,
 *   Z_k = -Y_k(m+mu) X_k(m)^dag     for m even.
 * Returned as omega^a in F (overwritten). */
int or_fermion_force(const int dims[4], const double *U, double mass, const or_rational *r,
                     const double *phi, double tol, int maxit, double *F, int *iters)
{
    olat l;
    lat_init(&l, dims);
    long N = 6 * l.Vh;
    double *X = malloc(sizeof(double) * N * r->n), *Y = malloc(sizeof(double) * N * r->n);
    int it = 0;
    int st = or_multishift(dims, U, mass, r->n, r->b, phi, X, tol, maxit, NULL, &it);
    for (int k = 0; k < r->n; k++) or_dslash(dims, U, 1, X + k * N, Y + k * N);
    const cplx *Xc = (const cplx *)X, *Yc = (const cplx *)Y;
    for (int mu = 0; mu < 4; mu++)
#pragma omp parallel for schedule(static)
        for (long lex = 0; lex < l.V; lex++) {
            int x[4];
            coords(&l, lex, x);
            long f = neighbour(&l, lex, mu, 1);
            mat3 Z = mzero();
            for (int k = 0; k < r->n; k++) {
                const cplx *Xk = Xc + 3 * l.Vh * k, *Yk = Yc + 3 * l.Vh * k;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        if (parity_of(x) == 1)
                            Z.e[a][b] += r->a[k] * Xk[3 * (f / 2) + a] * conj(Yk[3 * (lex / 2) + b]);
                        else
                            Z.e[a][b] -= r->a[k] * Yk[3 * (f / 2) + a] * conj(Xk[3 * (lex / 2) + b]);
                    }
            }
            mat3 u = link_at(&l, U, mu, lex);
            mat3 W = mmul(&u, &Z);
            W = mscale(&W, 0.5 * link_sign(&l, x, mu));
            mat3 T = traceless_antiherm(&W);
            mat3 Pd = mscale(&T, I);
            mat_to_omega(&Pd, F + 8 * (mu * l.V + lex));
        }
    if (iters) *iters = it;
    free(X);
    free(Y);
    return st;
}

/* Kinetic term sum_{n,mu} Tr H_mu(n)^2 = 1/2 sum omega^2 (Sec. 2.1) */
double or_kinetic(const int dims[4], const double *w)
{
    long V = or_volume(dims);
    double s = 0;
    for (long i = 0; i < 4 * V; i++) {
        mat3 P = omega_to_mat(w + 8 * i);
        mat3 P2 = mmul(&P, &P);
        s += creal(mtrace(&P2));
    }
    return s;
}

/* Link update U <- exp(i eps P) U followed by reunitarisation (Sec. 4.1). */
void or_update_links(const int dims[4], double *U, const double *w, double eps)
{
    long V = or_volume(dims);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < 4 * V; i++) {
        mat3 P = omega_to_mat(w + 8 * i);
        mat3 X = mscale(&P, eps);
        mat3 E = exp_i(&X);
        mat3 u = load_mat(U + 18 * i);
        mat3 nu = mmul(&E, &u);
        reunit(&nu);
        store_mat(U + 18 * i, &nu);
    }
}

/* Momentum update P <- P + eps dP/dtau */
void or_update_momenta(const int dims[4], double *w, const double *F, double eps)
{
    long n = 8 * 4 * or_volume(dims);
    for (long i = 0; i < n; i++) w[i] += eps * F[i];
}

/* ------------------------------------------------------------------------ */
/* Molecular dynamics and the trajectory (Sec. 2.1)                          */
/* ------------------------------------------------------------------------ */

/* fermion part of dP/dtau: sum over pseudofermions of the fermion force */
static int fermion_force_all(const int dims[4], const double *U, const double *phi, const or_params *p,
                             double *F, double *Ff, long *cg_iters)
{
    long V = or_volume(dims), N = 6 * (V / 2);
    int st = 0;
    for (long i = 0; i < 32 * V; i++) F[i] = 0.0;
    for (int pf = 0; pf < p->npf; pf++) {
        int it = 0;
        st |= or_fermion_force(dims, U, p->mass, &p->force, phi + pf * N, p->tol_md, p->maxit, Ff,
                               &it);
        *cg_iters += it;
        for (long i = 0; i < 32 * V; i++) F[i] += Ff[i];
    }
    return st;
}

/* total force dP/dtau = gauge force + sum over pseudofermions of the fermion force */
static int total_force(const int dims[4], const double *U, const double *phi, const or_params *p,
                       double *F, double *Ff, long *cg_iters)
{
    long V = or_volume(dims), N = 6 * (V / 2);
    int st = 0;
    or_gauge_force(dims, U, p->beta, F);
    for (int pf = 0; pf < p->npf; pf++) {
        int it = 0;
        st |= or_fermion_force(dims, U, p->mass, &p->force, phi + pf * N, p->tol_md, p->maxit, Ff,
                               &it);
        *cg_iters += it;
        for (long i = 0; i < 32 * V; i++) F[i] += Ff[i];
    }
    return st;
}

/* Inner scheme of the multi-step integrator: ngauge steps of size d = h/ngauge
 * of the same scheme (leapfrog or 2MN) moving U and P with the gauge force
 * only, written out step by step without merging the momentum updates. */
static void gauge_substeps(const int dims[4], double *U, double *w, const or_params *p, double h,
                           double *Fg)
{
    double d = h / p->ngauge, lam = p->lambda;
    for (int j = 0; j < p->ngauge; j++) {
        if (p->integrator == 0) {
            or_gauge_force(dims, U, p->beta, Fg);
            or_update_momenta(dims, w, Fg, 0.5 * d);
            or_update_links(dims, U, w, d);
            or_gauge_force(dims, U, p->beta, Fg);
            or_update_momenta(dims, w, Fg, 0.5 * d);
        } else {
            or_gauge_force(dims, U, p->beta, Fg);
            or_update_momenta(dims, w, Fg, lam * d);
            or_update_links(dims, U, w, 0.5 * d);
            or_gauge_force(dims, U, p->beta, Fg);
            or_update_momenta(dims, w, Fg, (1.0 - 2.0 * lam) * d);
            or_update_links(dims, U, w, 0.5 * d);
            or_gauge_force(dims, U, p->beta, Fg);
            or_update_momenta(dims, w, Fg, lam * d);
        }
    }
}

/* Integrate Hamilton's equations over tau with nsteps steps of size
 * eps = tau/nsteps.  Leapfrog (PQP): P(eps/2) Q(eps) P(eps/2) per step.
 * Omelyan second-order minimum norm (2MN):
 * P(l eps) Q(eps/2) P((1-2l) eps) Q(eps/2) P(l eps) per step.
 * Adjacent momentum half-steps of consecutive steps are merged (same force).
 * Multi-step scheme (ngauge > 0; Sec. 2.1's "multi-step integrator, with
 * action divided in gauge and fermion part", after Sexton and Weingarten):
 * the scheme above moves P with the fermion force only, and each of its
 * position updates Q(h) becomes ngauge inner steps over time h that move U
 * and P with the gauge force (gauge_substeps). */
int or_md_integrate(const int dims[4], double *U, double *w, const double *phi,
                    const or_params *p, long *cg_iters, int *n_force)
{
    long V = or_volume(dims);
    double *F = malloc(sizeof(double) * 32 * V), *Ff = malloc(sizeof(double) * 32 * V);
    double *Fg = malloc(sizeof(double) * 32 * V);
    double eps = p->tau / p->nsteps;
    long it = 0;
    int nf = 0, st = 0;
    int multi = p->ngauge > 0;
#define OR_FORCE() (multi ? fermion_force_all(dims, U, phi, p, F, Ff, &it) \
                          : total_force(dims, U, phi, p, F, Ff, &it))
#define OR_MOVE(h) do { if (multi) gauge_substeps(dims, U, w, p, (h), Fg); \
                        else or_update_links(dims, U, w, (h)); } while (0)
    if (p->integrator == 0) {
        st |= OR_FORCE(); nf++;
        or_update_momenta(dims, w, F, 0.5 * eps);
        for (int s = 0; s < p->nsteps; s++) {
            OR_MOVE(eps);
            st |= OR_FORCE(); nf++;
            or_update_momenta(dims, w, F, (s == p->nsteps - 1) ? 0.5 * eps : eps);
        }
    } else {
        double lam = p->lambda;
        st |= OR_FORCE(); nf++;
        or_update_momenta(dims, w, F, lam * eps);
        for (int s = 0; s < p->nsteps; s++) {
            OR_MOVE(0.5 * eps);
            st |= OR_FORCE(); nf++;
            or_update_momenta(dims, w, F, (1.0 - 2.0 * lam) * eps);
            OR_MOVE(0.5 * eps);
            st |= OR_FORCE(); nf++;
            or_update_momenta(dims, w, F, (s == p->nsteps - 1) ? lam * eps : 2.0 * lam * eps);
        }
    }
#undef OR_FORCE
#undef OR_MOVE
    if (cg_iters) *cg_iters += it;
    if (n_force) *n_force += nf;
    free(F);
    free(Ff);
    free(Fg);
    return st;
}

/* H = sum Tr P^2 + S_g + sum_pf phi^dag r_act(M) phi  (Sec. 2.1) */
int or_hamiltonian(const int dims[4], const double *U, const double *w, const double *phi,
                   const or_params *p, double *H, long *cg_iters)
{
    long N = 6 * (or_volume(dims) / 2);
    double h = or_kinetic(dims, w) + or_gauge_action(dims, U, p->beta);
    for (int pf = 0; pf < p->npf; pf++) {
        int it = 0;
        h += or_fermion_action(dims, U, p->mass, &p->act, phi + pf * N, p->tol_metro, p->maxit, &it);
        if (cg_iters) *cg_iters += it;
    }
    *H = h;
    return 0;
}

/* One RHMC trajectory (the Phi algorithm of Sec. 2.1 with rooting):
 * momenta and R from the heatbath, phi = r_{1/4}(M_ee) R, H0, MD over tau,
 * H1, accept with probability min(1, exp(-dH)); on rejection U is restored. */
int or_trajectory(const int dims[4], double *U, const or_params *p, or_traj_info *info)
{
    long V = or_volume(dims), N = 6 * (V / 2);
    double *w = malloc(sizeof(double) * 32 * V);
    double *phi = malloc(sizeof(double) * N * p->npf), *R = malloc(sizeof(double) * N);
    double *U0 = malloc(sizeof(double) * 72 * V);
    long it = 0;
    int nf = 0;
    memcpy(U0, U, sizeof(double) * 72 * V);
    or_momenta_heatbath(dims, p->seed, p->traj, w);
    for (int pf = 0; pf < p->npf; pf++) {
        int i2 = 0;
        or_pf_gaussian(dims, p->seed, p->traj, pf, R);
        or_rational_apply(dims, U, p->mass, &p->hb, R, phi + pf * N, p->tol_metro, p->maxit, &i2);
        it += i2;
    }
    double H0, H1;
    or_hamiltonian(dims, U, w, phi, p, &H0, &it);
    int st = or_md_integrate(dims, U, w, phi, p, &it, &nf);
    or_hamiltonian(dims, U, w, phi, p, &H1, &it);
    double dH = H1 - H0;
    double u = or_metro_uniform(p->seed, p->traj);
    int acc = (u < exp(-dH));
    if (!acc) memcpy(U, U0, sizeof(double) * 72 * V);
    info->H0 = H0;
    info->H1 = H1;
    info->dH = dH;
    info->u = u;
    info->accepted = acc;
    info->plaq = or_plaquette(dims, U);
    info->cg_iters = it;
    info->n_force = nf;
    free(w); free(phi); free(R); free(U0);
    return st;
}

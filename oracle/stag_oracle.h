/*
 * stag_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Declarations of the plain FP64 CPU oracle of the two-flavour staggered
 * RHMC of Bonati, Cossu, D'Elia, Incardona, "QCD simulations with staggered
 * fermions on GPUs" (arXiv:1106.5673).  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code, header or table with the CUDA library.
 *
 * Conventions (every complex array is interleaved re/im double):
 *   site n = (x,y,z,t), lex = x + Lx*(y + Ly*(z + Lz*t)); every L_mu even;
 *   parity(n) = (x+y+z+t) mod 2; a field on one parity is indexed by lex/2;
 *   gauge field   U[mu][lex][3][3]  complex, row-major, mu = 0..3 = x,y,z,t;
 *   colour vector v[lex/2][3]       complex on the sites of one parity;
 *   momenta       w[mu][lex][8]     real, P = sum_a w^a lambda^a / 2
 *                                   (lambda^a the Gell-Mann matrices).
 */
#ifndef STAG_ORACLE_H
#define STAG_ORACLE_H

#include <stdint.h>

#define OR_MAXDEG 32

/* r(x) = a0 + sum_k a[k] / (x + b[k])  (the RHMC rational function, Sec. 2.1) */
typedef struct {
    double a0;
    int n;
    double a[OR_MAXDEG];
    double b[OR_MAXDEG];
} or_rational;

typedef struct {
    double beta, mass, tau, lambda, tol_md, tol_metro;
    int nsteps;      /* MD steps per trajectory                      */
    int integrator;  /* 0 = leapfrog PQP, 1 = Omelyan 2MN             */
    int npf;         /* pseudofermions                                */
    int maxit;       /* CG iteration cap                              */
    uint32_t seed, traj;
    or_rational hb, act, force;  /* r_{1/4}, r_{-1/2} (Metropolis), r_{-1/2} (MD) */
    int ngauge;      /* 0: one time scale; n > 0: multi-step scheme, n gauge steps
                        per position update of the fermion scheme              */
} or_params;

typedef struct {
    double H0, H1, dH, u;
    int accepted;
    double plaq;
    long cg_iters;
    int n_force;
} or_traj_info;

long or_volume(const int dims[4]);

void or_dslash_full(const int dims[4], const double *U, const double *in, double *out);
void or_dslash(const int dims[4], const double *U, int out_parity, const double *in, double *out);
void or_apply_M(const int dims[4], const double *U, double mass, const double *in, double *out);

int or_cg(const int dims[4], const double *U, double mass, double shift, const double *b,
          double *x, double tol, int maxit, int *iters);
int or_multishift(const int dims[4], const double *U, double mass, int n, const double *shifts,
                  const double *b, double *x, double tol, int maxit, int *iters_shift,
                  int *iters_total);
void or_rational_apply(const int dims[4], const double *U, double mass, const or_rational *r,
                       const double *src, double *out, double tol, int maxit, int *iters);

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_gauss_pair(const uint32_t ctr[4], const uint32_t key[2], double g[2]);
void or_uniform_pair(const uint32_t ctr[4], const uint32_t key[2], double u[2]);
void or_momenta_heatbath(const int dims[4], uint32_t seed, uint32_t traj, double *w);
void or_pf_gaussian(const int dims[4], uint32_t seed, uint32_t traj, int pf, double *R);
double or_metro_uniform(uint32_t seed, uint32_t traj);

void or_su3_exp_i(const double *X, double *out);
void or_reunit(double *U);
void or_omega_to_matrix(const double *w, double *P);
void or_matrix_to_omega(const double *P, double *w);

double or_plaquette(const int dims[4], const double *U);
double or_gauge_action(const int dims[4], const double *U, double beta);
void or_gauge_force(const int dims[4], const double *U, double beta, double *F);
int or_fermion_force(const int dims[4], const double *U, double mass, const or_rational *r,
                     const double *phi, double tol, int maxit, double *F, int *iters);
double or_fermion_action(const int dims[4], const double *U, double mass, const or_rational *r,
                         const double *phi, double tol, int maxit, int *iters);
double or_kinetic(const int dims[4], const double *w);
void or_update_links(const int dims[4], double *U, const double *w, double eps);
void or_update_momenta(const int dims[4], double *w, const double *F, double eps);

int or_md_integrate(const int dims[4], double *U, double *w, const double *phi,
                    const or_params *p, long *cg_iters, int *n_force);
int or_hamiltonian(const int dims[4], const double *U, const double *w, const double *phi,
                   const or_params *p, double *H, long *cg_iters);
int or_trajectory(const int dims[4], double *U, const or_params *p, or_traj_info *info);

#endif

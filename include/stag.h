/*
 * stag.h -- C ABI of the GB300 staggered-RHMC library (libstag.so).
 *
 * Two-flavour staggered RHMC as described in C. Bonati, G. Cossu, M. D'Elia,
 * P. Incardona, "QCD simulations with staggered fermions on GPUs"
 * (arXiv:1106.5673): the even/odd staggered operator of Eq. (4), the shifted
 * (multi-shift) CG of Eq. (13) that applies the RHMC rational functions
 * (Sec. 2.1), the gauge and fermion forces, the SU(3) momentum and link
 * update and the Metropolis test, with a whole molecular-dynamics trajectory
 * kept on one GPU (Sec. 4).
 *
 * Conventions
 *  - Every function returns an int status: STAG_OK (0) or a negative
 *    STAG_ERR_* code; stag_last_error(ctx) gives a message owned by the
 *    library.  The library never aborts and never traps the device; every
 *    device-side loop is bounded.
 *  - Lattice: dims = {Lx, Ly, Lz, Lt}, each even and >= 2; V = Lx Ly Lz Lt,
 *    Vh = V/2.  Site n = (x,y,z,t) has lex = x + Lx*(y + Ly*(z + Lz*t)),
 *    parity (x+y+z+t) mod 2, and index lex/2 within its parity.  Fermions are
 *    antiperiodic in t, links periodic in all directions.
 *  - Canonical host/device layouts at this boundary:
 *      gauge    complex128 [4][V][3][3]  (mu = 0..3 = x,y,z,t; row-major)
 *      vector   complex    [Vh][3]       sites of one parity; complex128
 *                                        for STAG_PREC_F64, complex64
 *                                        (float re/im) for F32 and BF16
 *      momenta  float64    [4][V][8]     Gell-Mann coefficients w^a of
 *                                        P = sum_a w^a lambda^a / 2
 *    Internally the library keeps its own structure-of-arrays forms.
 *  - Pointers are borrowed: the caller owns them (usually PyTorch tensors)
 *    and keeps them alive until the stream has been synchronised.  Device
 *    pointers must be 16-byte aligned.  Objects created by stag_*_create are
 *    owned by the library and freed by the matching destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless documented as
 *    synchronising.
 */
#ifndef STAG_H
#define STAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    STAG_OK = 0,
    STAG_ERR_ARG = -1,       /* invalid argument (null pointer, bad size, bad mode)   */
    STAG_ERR_CUDA = -2,      /* a CUDA runtime call failed                             */
    STAG_ERR_NOCONV = -3,    /* a solver hit its iteration cap above tolerance         */
    STAG_ERR_NONFINITE = -4, /* NaN/Inf found in a result that must be finite          */
    STAG_ERR_OOM = -5,       /* device allocation failed                               */
    STAG_ERR_STATE = -6      /* call out of order (e.g. no gauge field loaded)         */
};

/* Operator precisions.  F64FF takes and returns FP64 vectors but computes in
 * float-float arithmetic on the FP32 units (each double carried as a pair of
 * floats hi + lo, Sec. 4.2's split used for arithmetic): relative accuracy
 * ~1e-13, many times the throughput of GB300's FP64 units.  F32R8: FP32
 * vectors and arithmetic with 8-real links (the minimal SU(3)
 * parametrisation Sec. 4.2 mentions: a1, a2, b0 and the phases of a0 and c0,
 * the rest rebuilt from unitarity and det = 1; 32 bytes per link instead of
 * 48), rebuilt from the FP64 links on first use after every change. */
enum { STAG_PREC_F64 = 0, STAG_PREC_F32 = 1, STAG_PREC_BF16 = 2, STAG_PREC_F64FF = 3, STAG_PREC_F32R8 = 4 };

/* Solver modes:
 *  F64         plain FP64 shifted CG, FP64 true-residual check of every shift;
 *  MIXED       FP32 shifted CG, then the shifts above tolerance refined
 *              together by a batched CG (multi-RHS hops, FP32 recursion, FP64
 *              reliable updates); every shift checked FP64-accurately;
 *  MIXED_BF16  as MIXED with BF16 links in the FP32 kernels;
 *  F64FF       FP64 vectors and recurrences with the float-float operator
 *              (STAG_PREC_F64FF) in place of native FP64 arithmetic;
 *  LEARNED     the lightest shift by flexible CG preconditioned with the
 *              network attached by stag_ctx_set_net, the other shifts by the
 *              MIXED solver (whose shifted CG is then based at the second
 *              lightest shift); if the flexible CG misses tol within its cap
 *              (STAG_FCG_MAXIT, default 2000 iterations) the MIXED solver is
 *              re-run over all shifts.  Every shift checked FP64-accurately. */
enum {
    STAG_SOLVE_F64 = 0,
    STAG_SOLVE_MIXED = 1,
    STAG_SOLVE_MIXED_BF16 = 2,
    STAG_SOLVE_F64FF = 3,
    STAG_SOLVE_LEARNED = 4
};

enum { STAG_INT_LEAPFROG = 0, STAG_INT_OMELYAN = 1 };

#define STAG_MAXSHIFT 32
#define STAG_MAXPF 8
#define STAG_MAXRHS 8 /* systems of one batched multi-shift solve */
#define STAG_MAXLAT 8 /* lattices of one batched hop launch */

typedef struct stag_ctx stag_ctx;

/* r(x) = a0 + sum_{k<n} a[k] / (x + b[k]): the RHMC rational function
 * (Sec. 2.1), b[k] > 0 the shifts of Eq. (13). */
typedef struct {
    double a0;
    int n;
    double a[STAG_MAXSHIFT];
    double b[STAG_MAXSHIFT];
} stag_rational;

typedef struct {
    int status;                          /* STAG_OK or STAG_ERR_NOCONV             */
    int iters;                           /* multi-shift (base) iterations           */
    int iters_shift[STAG_MAXSHIFT];      /* iterations each shift was updated       */
    int refine_iters[STAG_MAXSHIFT];     /* single-shift refinement iterations      */
    double true_resid[STAG_MAXSHIFT];    /* |b - (M+s_k) x_k| / |b| in FP64         */
    int reliable_updates;                /* FP64 residual replacements performed    */
    int matvecs;                         /* M_ee applications of any precision      */
} stag_solve_info;

typedef struct {
    double beta, mass, tau;
    int nsteps;                 /* MD steps of size tau/nsteps                      */
    int integrator;             /* STAG_INT_LEAPFROG or STAG_INT_OMELYAN           */
    double lambda;              /* Omelyan 2MN parameter (0.1931833275037836)       */
    int npf;                    /* pseudofermions, 0..STAG_MAXPF (0: pure gauge)    */
    stag_rational hb;           /* r ~ x^{+1/(4 npf)}  heatbath                     */
    stag_rational act;          /* r ~ x^{-1/(2 npf)}  action (Metropolis)          */
    stag_rational force;        /* r ~ x^{-1/(2 npf)}  molecular dynamics           */
    double tol_md, tol_metro;   /* relative residuals of MD and Metropolis solves   */
    int solve_mode_md;          /* STAG_SOLVE_* for the force solves                */
    int solve_mode_metro;       /* STAG_SOLVE_* for heatbath and action solves      */
    int maxit;                  /* iteration cap of every solve                     */
    uint32_t seed, traj;        /* Philox key (seed, traj)                          */
    int use_graphs;             /* 1: every solver iteration chunk (32 iterations
                                   of a shifted or batched CG) runs as a cached
                                   CUDA graph, replayed between the host's
                                   convergence polls; 0: the same kernels are
                                   launched one by one.  Forces, updates and the
                                   Hamiltonian are launched kernel by kernel
                                   either way.  Results are identical.             */
    int ngauge;                 /* 0: one time scale.  n > 0: multi-step scheme
                                   (Sec. 2.1, Sexton-Weingarten): the integrator
                                   moves P with the fermion force only, and each
                                   of its position updates Q(h) is n inner steps
                                   of the same scheme over h with the gauge force
                                   (step ratio dtau_f/dtau_g = n for leapfrog,
                                   2n for Omelyan)                                  */
    int no_metropolis;          /* 1: accept every trajectory (molecular-dynamics
                                   thermalisation of a start configuration only;
                                   not an exact algorithm).  0: Metropolis test   */
} stag_params;

typedef struct {
    double H0, H1, dH, u;       /* Hamiltonians, their difference, Metropolis u    */
    int accepted;
    double plaq;                /* average plaquette after the accept/reject        */
    long long cg_iters;         /* multi-shift + refinement iterations              */
    int n_force;                /* force evaluations                                */
    double t_heatbath, t_action, t_md, t_total; /* seconds (host wall clock)        */
    int status;
} stag_traj_info;

/* ---------------- context ---------------- */

/* Creates a context for one lattice on the current CUDA device and allocates
 * its device storage (gauge field in FP64/FP32/BF16 12-real form, momenta,
 * solver work space sized on first use).  dims as above. */
int stag_ctx_create(const int dims[4], stag_ctx **out);
int stag_ctx_destroy(stag_ctx *ctx);
const char *stag_last_error(const stag_ctx *ctx);
/* Bytes of device memory held by the context. */
int stag_ctx_device_bytes(const stag_ctx *ctx, size_t *bytes);
/* Number of CUDA kernels the context has launched so far (kernels inside
 * captured graphs counted one by one); for accounting in benchmarks. */
int stag_ctx_launch_count(const stag_ctx *ctx, long long *n);
/* Autotuner: times the hop kernels for 64, 128 and 256 threads per block for
 * each link precision (FP64, FP32, BF16, float-float; CUDA events after
 * warm-up, best of three timings of ten launches) on the loaded gauge field
 * and keeps the fastest for this context, unless it beats 128 by less than
 * 3 % (then 128);
 * tpb_out (nullable, 4 ints) receives the choice.  The first solve on a
 * context runs it automatically unless the environment sets STAG_AUTOTUNE=0.
 * Synchronises. */
int stag_autotune(stag_ctx *ctx, int tpb_out[4], void *stream);

/* ---------------- fields ---------------- */

/* Loads the gauge field (canonical layout, complex128, host or device pointer;
 * on_device selects which) and builds the internal FP64, FP32 and BF16 copies
 * holding the first two rows of each link (the third is rebuilt as the
 * conjugate cross product, Sec. 4.2).  Links must be SU(3). */
int stag_load_gauge(stag_ctx *ctx, const double *links, int on_device, void *stream);
/* Writes the gauge field back in the canonical layout. */
int stag_store_gauge(stag_ctx *ctx, double *links, int on_device, void *stream);
int stag_load_momenta(stag_ctx *ctx, const double *w, int on_device, void *stream);
int stag_store_momenta(stag_ctx *ctx, double *w, int on_device, void *stream);
/* Average plaquette (1/6V) sum Re Tr U_P / 3 in FP64.  Synchronises. */
int stag_plaquette(stag_ctx *ctx, double *plaq, void *stream);
/* Wilson gauge action beta sum_P (1 - Re Tr U_P / 3).  Synchronises. */
int stag_gauge_action(stag_ctx *ctx, double beta, double *action, void *stream);

/* ---------------- operator (Eq. (4), a = 1) ---------------- */

/* out_even = D_eo in_odd:  (D psi)(n) = 1/2 sum_mu eta_mu(n) [U_mu(n) psi(n+mu)
 * - U_mu(n-mu)^dag psi(n-mu)].  Device vectors in the canonical layout of
 * `prec` (F64, F64FF: complex128; F32, BF16, F32R8: complex64, with FP32
 * 12-real, BF16 resp. FP32 8-real links).  in and out must not alias. */
int stag_apply_deo(stag_ctx *ctx, const void *in_odd, void *out_even, int prec, void *stream);
/* out_odd = D_oe in_even. */
int stag_apply_doe(stag_ctx *ctx, const void *in_even, void *out_odd, int prec, void *stream);
/* out_even = M_ee in_even = m^2 in - D_eo D_oe in  (even/odd preconditioned
 * M^dag M, Sec. 2.1).  in and out must not alias. */
int stag_apply_M(stag_ctx *ctx, double mass, const void *in_even, void *out_even, int prec,
                 void *stream);

/* Allocation-free M_ee.  The paper has no counterpart: this serves callers
 * that must not allocate device memory when they apply the operator -- code
 * inside a framework that owns the device's memory pool, where a cudaMalloc
 * behind its back breaks its accounting or its cap, and latency-critical
 * loops, where cudaMalloc's implicit device synchronisation stalls every
 * stream.  Needs no context: `links` is the gauge field on the device in the
 * canonical layout, in_even/out_even FP64 device vectors (canonical, even
 * sites), all owned by the caller; out = m^2 in - D_eo D_oe in in FP64.
 * The odd-site intermediate lives in a fixed array inside the library of
 * 2^17 sites (6 MiB), resident on every device that loads the library until
 * exit; lattices with V/2 > 2^17 (larger than 32^3 x 8) are rejected with
 * STAG_ERR_ARG.  The first call on a device looks up the array's address
 * (set-up) and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this function on a device after
 * cudaDeviceReset (the kept address is then stale).  All calls share
 * the array: calls whose kernels overlap on the GPU race.  Returns STAG_OK,
 * STAG_ERR_ARG (bad sizes or pointers) or STAG_ERR_CUDA; there is no error
 * string, since there is no context.  Asynchronous on `stream`. */
int stag_apply_M_noalloc(const int dims[4], const double *links, double mass, const double *in_even,
                         double *out_even, void *stream);

/* Batched hop: for each lattice l < nlat (each its own context, all on one
 * device, any sizes), out[l][j] = D_{out_par, 1-out_par} in[l][j] for the
 * nrhs[l] right-hand sides j, all in ONE kernel launch whose blocks walk a
 * list of (lattice, site block, group of right-hand sides)
 * tiles, each link loaded once per tile and applied to the group (Eq. (4)).
 * in[l], out[l]: FP32 complex device vectors [nrhs[l]][V_l/2][3], contiguous
 * (canonical site order of the source and target parity).  prec:
 * STAG_PREC_F32 or STAG_PREC_BF16 links.  The first call for a combination of
 * lattice shapes, nrhs and prec tunes the block size, the right-hand sides
 * per thread, the grid form (resident blocks walking the tiles, or one block
 * per tile) and the tile order by timing (synchronises; skipped, with
 * defaults, while `stream` is
 * being captured) and caches the choice; tuned_cfg (nullable) receives
 * {threads per block, right-hand sides per thread}.  Otherwise asynchronous;
 * capturable in a CUDA graph.  nlat <= STAG_MAXLAT. */
int stag_dslash_batch(int nlat, stag_ctx *const *ctxs, const void *const *in, void *const *out,
                      const int *nrhs, int out_par, int prec, int *tuned_cfg, void *stream);

/* ---------------- solvers (Sec. 4.3, Eq. (13)) ---------------- */

/* Solves (M_ee + shifts[k]) x_k = src for k < n (1 <= n <= STAG_MAXSHIFT,
 * shifts >= 0) from x = 0 with the shifted CG, stopping shift k when its
 * residual falls below tol*|src|.  src and sols[k] are FP64 device vectors
 * (canonical complex128, even sites); sols[k] (nullable entries, sols itself
 * nullable) may alias nothing else.  mode (see STAG_SOLVE_*):
 *  F64, F64FF   the shifted CG in FP64 (or float-float) arithmetic; a shift
 *               whose FP64 true residual is still above tol when its
 *               recursion stops resumes the recursion with a tighter target
 *               (or, if it was frozen earlier, is refined as below);
 *  MIXED(_BF16) the shifted CG in FP32 to max(tol, 1e-6), then every shift
 *               above tol refined from x_k by one batched FP32 CG (all such
 *               shifts in the same kernels) with FP64 reliable updates;
 *  LEARNED      see the enum.
 * The true residual of every shift is computed FP64-accurately and returned
 * in info.  Synchronises (reads convergence flags).  Returns STAG_ERR_NOCONV
 * if any shift misses tol within maxit iterations. */
int stag_multishift_solve(stag_ctx *ctx, double mass, int n, const double *shifts,
                          const double *src, double *const *sols, double tol, int maxit,
                          int mode, stag_solve_info *info, void *stream);

/* Batched form: solves (M_ee + shifts[k]) x_{r,k} = srcs[r] for nsys systems
 * (1 <= nsys <= STAG_MAXRHS, e.g. the pseudofermions of one force
 * evaluation) and the same n shifts, advancing all systems together: the hop
 * kernels load each link once for a group of systems.  Each system stops on
 * its own; every (system, shift) whose FP64-accurate true residual is above
 * tolerance is then refined by the batched CG, STAG_MAXSHIFT pairs at a time
 * (modes F64, F64FF, MIXED, MIXED_BF16; not LEARNED).  sols[r*n + k] (nullable entries; sols itself
 * nullable) receive the FP64 solutions; infos (nullable) holds nsys entries.
 * Synchronises.  Errors as stag_multishift_solve. */
int stag_multishift_solve_multi(stag_ctx *ctx, double mass, int nsys, int n, const double *shifts,
                                const double *const *srcs, double *const *sols, double tol, int maxit,
                                int mode, stag_solve_info *infos, void *stream);

/* out = r(M_ee) src = a0 src + sum_k a_k (M_ee + b_k)^{-1} src (RHMC, Sec. 2.1).
 * FP64 device vectors; out may not alias src.  Synchronises. */
int stag_rational_apply(stag_ctx *ctx, double mass, const stag_rational *r, const double *src,
                        double *out, double tol, int maxit, int mode, stag_solve_info *info,
                        void *stream);

/* ---------------- forces and updates ---------------- */

/* Gauge force dP/dtau = (i beta/6) TA(U_mu(n) A_mu(n)) of the Wilson action
 * (A = sum of the six staples, TA = traceless anti-Hermitian part) as
 * Gell-Mann coefficients, canonical momenta layout, FP64 device array. */
int stag_gauge_force(stag_ctx *ctx, double beta, double *force_out, void *stream);

/* Fermion force of S_f = phi^dag r(M_ee) phi: with X_k = (M_ee+b_k)^{-1} phi
 * and Y_k = D_oe X_k, dP/dtau = i TA(W), W = (eta/2) U sum_k a_k Z_k,
 * Z_k = X_k(n+mu) Y_k(n)^dag (n odd) or -Y_k(n+mu) X_k(n)^dag (n even).
 * phi: FP64 device vector (even sites); force_out: canonical momenta layout.
 * Synchronises (solver). */
int stag_fermion_force(stag_ctx *ctx, double mass, const stag_rational *r, const double *phi,
                       double *force_out, double tol, int maxit, int mode,
                       stag_solve_info *info, void *stream);

/* Link update U <- exp(i eps P) U with the context's momenta, in FP64, then
 * reunitarisation (Sec. 4.1) and refresh of the FP32/BF16 copies. */
int stag_update_links(stag_ctx *ctx, double eps, void *stream);

/* Philox4x32-10 momentum heatbath into the context's momenta: w^a ~ N(0,1)
 * with counter (1, mu, lex, block) and key (seed, traj). */
int stag_momenta_heatbath(stag_ctx *ctx, uint32_t seed, uint32_t traj, void *stream);

/* Complex Gaussian R (density exp(-R^dag R)) on even sites, counter
 * (2, pf, lex, colour) and key (seed, traj); out is an FP64 device vector. */
int stag_pf_gaussian(stag_ctx *ctx, uint32_t seed, uint32_t traj, int pf, double *out,
                     void *stream);

/* Kinetic term sum Tr P^2 = 1/2 sum w^2 of the context's momenta.  Synchronises. */
int stag_kinetic(stag_ctx *ctx, double *out, void *stream);

/* ---------------- trajectory (Sec. 2.1, Fig. traj_fig) ---------------- */

/* One RHMC trajectory on the device: momentum and pseudofermion heatbath
 * (phi = r_hb(M) R per pseudofermion), H0, MD over tau with the chosen
 * integrator, H1, Metropolis with u from Philox counter (3,0,0,0); on
 * rejection the gauge field is restored.  Synchronises. */
int stag_md_trajectory(stag_ctx *ctx, const stag_params *p, stag_traj_info *out, void *stream);

/* Molecular dynamics alone (Sec. 2.1, point 3 of the Phi algorithm): integrates
 * Hamilton's equations over p->tau with the context's current links and
 * momenta (stag_load_gauge / stag_load_momenta) and the pseudofermions phi
 * held fixed (p->npf FP64 device vectors, even sites, contiguous with stride
 * V/2 x 3 complex), using p's integrator, force rational, MD tolerance and
 * solver mode; no heatbath, no Metropolis test.  The reversibility test of
 * Sec. 4.4 flips the momenta (store, negate, load) and integrates again.
 * *cg_iters, *n_force (nullable) receive the solver iterations and fermion
 * force evaluations.  Synchronises. */
int stag_md_integrate(stag_ctx *ctx, const stag_params *p, const double *phi, long long *cg_iters, int *n_force,
                      void *stream);

/* ---------------- learned preconditioner (no counterpart in the paper) ------
 * A gauge-covariant network K = restrict_even L3 L2 L1 embed_even with
 * channels 1 -> 8 -> 8 -> 1; each layer is a parallel-transport convolution
 *   (L phi)_o(n) = sum_i sum_t w[o][i][t] (T_t phi_i)(n),  t = 0..8:
 *   T_0 phi = phi(n), T_{1+mu} phi = U_mu(n) phi(n+mu),
 *   T_{5+mu} phi = U_mu(n-mu)^dag phi(n-mu),
 * so K commutes with gauge transformations.  Weights: complex, layout
 * [c_out][c_in][9] (re, im floats), BF16 in the forward pass, FP32 master and
 * FP32 arithmetic.  Trained with Adam on (source, solution) pairs to
 * minimise mean |K b - x|^2 / |x|^2; gradients are dloss/dRe w + i dloss/dIm w. */
typedef struct stag_net stag_net;

/* Creates a network bound to ctx (its gauge field), weights initialised near
 * the identity from `seed`.  Synchronises. */
int stag_net_create(stag_ctx *ctx, unsigned seed, stag_net **out);
/* Frees the network (detaching it from its context if attached). */
int stag_net_destroy(stag_net *net);
/* Attaches net (created on ctx) as the preconditioner of STAG_SOLVE_LEARNED;
 * NULL detaches.  The network is borrowed, not owned. */
int stag_ctx_set_net(stag_ctx *ctx, stag_net *net);
/* Complex weights of layer 0..2 (72, 576, 72). */
int stag_net_nweights(const stag_net *net, int layer, int *n);
/* Host copies of the FP32 master weights / of the last gradients (2 floats per
 * complex weight); set replaces the weights (and their BF16 copy). */
int stag_net_get_weights(stag_net *net, int layer, float *host);
int stag_net_set_weights(stag_net *net, int layer, const float *host);
int stag_net_get_grads(stag_net *net, int layer, float *host);
/* out_even = K in_even (FP64 device vectors). */
int stag_net_apply(stag_net *net, const double *in_even, double *out_even, void *stream);
/* Loss of the pairs (srcs[j], sols[j]) and its weight gradients (read them with
 * stag_net_get_grads).  Synchronises. */
int stag_net_loss_grad(stag_net *net, int npairs, const double *const *srcs, const double *const *sols,
                       double *loss, void *stream);
/* `epochs` passes of Adam (learning rate lr) over minibatches of `batch`
 * pairs; *loss receives the mean loss of the last epoch.  Synchronises. */
int stag_net_train(stag_net *net, int npairs, const double *const *srcs, const double *const *sols, int epochs,
                   int batch, double lr, double *loss, void *stream);
/* Solves (M_ee + shift) x = src (FP64 device vectors) by flexible CG with the
 * network as right preconditioner (net == NULL: plain CG), FP64 vectors and
 * the FP64-accurate float-float operator; stops at |r| <= tol |src| and
 * reports the true residual in info->true_resid[0].  Synchronises. */
int stag_fcg_solve(stag_ctx *ctx, stag_net *net, double mass, double shift, const double *src, double *sol,
                   double tol, int maxit, stag_solve_info *info, void *stream);

/* ---------------- host helper ---------------- */

/* Best relative rational approximation of x^power on [lo, hi] of type
 * (degree, degree) by the Remez exchange, as partial fractions.  Host only,
 * needs no GPU.  degree <= STAG_MAXSHIFT. */
int stag_remez(double power, double lo, double hi, int degree, stag_rational *out,
               double *max_rel_err);

#ifdef __cplusplus
}
#endif

#endif /* STAG_H */

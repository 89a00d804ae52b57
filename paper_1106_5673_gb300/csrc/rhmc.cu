// rhmc.cu -- one RHMC trajectory on the device (Sec. 2.1, the Phi algorithm
// with rooting; Sec. 4: "the whole Molecular Dynamics trajectory is
// performed on [the GPU]").  The host only sequences kernels, reads solver
// convergence flags and the final dH.
#include <chrono>
#include <math.h>

#include "hop.cuh"
#include "stag_internal.h"

int gauge_force_internal_prec(stag_ctx* ctx, double beta, double* F, int accumulate, int prec32, cudaStream_t s);
int refresh_lowp_links(stag_ctx* ctx, cudaStream_t s);

namespace {

double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct TrajWork {
    double2* phi;  // npf even vectors
    double2* R;
    double2* rat;
    double2* X;    // solver output, STAG_MAXSHIFT vectors
    double* F;     // force [4][2][8][Vh]
    long n3;
};

// out = r(M) src with FP64 output
int rational_apply_int(stag_ctx* ctx, double mass, const stag_rational* r, const double2* src, double2* out,
                       double2* X, double tol, int maxit, int mode, long long* iters, cudaStream_t s) {
    stag_solve_info info;
    const long n3 = 3L * ctx->g.Vh;
    double2* sols[STAG_MAXSHIFT];
    for (int k = 0; k < r->n; k++) sols[k] = X + k * n3;
    int st = multishift_solve(ctx, mass, r->n, r->b, src, sols, tol, maxit, mode, &info, s);
    if (iters) {
        *iters += info.iters;
        for (int k = 0; k < r->n; k++) *iters += info.refine_iters[k];
    }
    if (st) return st;
    return blas_rational_combine(ctx, r->a0, r->a, r->n, src, X, out, s);
}

enum { FORCE_GAUGE = 1, FORCE_FERMION = 2, FORCE_ALL = 3 };

// F = dP/dtau of the selected parts: gauge force and/or sum_pf fermion force
int total_force(stag_ctx* ctx, const stag_params* p, const TrajWork& w, long long* iters, cudaStream_t s,
                int parts = FORCE_ALL) {
    const int mixed = p->solve_mode_md == STAG_SOLVE_MIXED || p->solve_mode_md == STAG_SOLVE_MIXED_BF16 ||
                      p->solve_mode_md == STAG_SOLVE_LEARNED;
    int st;
    if (parts & FORCE_GAUGE) {
        if ((st = gauge_force_internal_prec(ctx, p->beta, w.F, 0, mixed, s))) return st;
    } else {
        STAG_CUDA(ctx, cudaMemsetAsync(w.F, 0, sizeof(double) * 64 * (size_t)ctx->g.Vh, s));
    }
    if (!(parts & FORCE_FERMION)) return STAG_OK;
    if (p->npf > 1 && p->solve_mode_md != STAG_SOLVE_LEARNED) {
        // all pseudofermions in one batched solve (multi-RHS hops)
        const long n3 = w.n3;
        double2* XM = (double2*)ws_get(ctx, WS_MX, sizeof(double2) * n3 * STAG_MAXSHIFT * STAG_MAXRHS);
        if (!XM) return stag_fail(ctx, STAG_ERR_OOM, "force workspace");
        const double2* srcs[STAG_MAXRHS];
        for (int pf = 0; pf < p->npf; pf++) srcs[pf] = w.phi + pf * n3;
        stag_solve_info infos[STAG_MAXRHS];
        st = multishift_solve_multi(ctx, p->mass, p->npf, p->force.n, p->force.b, srcs, XM, p->tol_md, p->maxit,
                                    p->solve_mode_md, infos, s);
        for (int pf = 0; pf < p->npf; pf++) {
            *iters += infos[pf].iters;
            for (int k = 0; k < p->force.n; k++) *iters += infos[pf].refine_iters[k];
        }
        if (st) return st;
        for (int pf = 0; pf < p->npf; pf++)
            if ((st = fermion_force_assemble(ctx, &p->force, XM + (size_t)pf * STAG_MAXSHIFT * n3, w.F, 1, s)))
                return st;
        return STAG_OK;
    }
    for (int pf = 0; pf < p->npf; pf++) {
        stag_solve_info info;
        double2* sols[STAG_MAXSHIFT];
        for (int k = 0; k < p->force.n; k++) sols[k] = w.X + k * w.n3;
        st = multishift_solve(ctx, p->mass, p->force.n, p->force.b, w.phi + pf * w.n3, sols, p->tol_md, p->maxit,
                              p->solve_mode_md, &info, s);
        *iters += info.iters;
        for (int k = 0; k < p->force.n; k++) *iters += info.refine_iters[k];
        if (st) return st;
        if ((st = fermion_force_assemble(ctx, &p->force, w.X, w.F, 1, s))) return st;
    }
    return STAG_OK;
}

// H = sum Tr P^2 + S_g + sum_pf phi^dag r_act(M) phi, read back to the host
int hamiltonian(stag_ctx* ctx, const stag_params* p, const TrajWork& w, double* H, long long* iters,
                cudaStream_t s) {
    int st = kinetic_sum(ctx, ctx->dscal + 32, s);
    if (st) return st;
    if ((st = plaquette_sum(ctx, ctx->dscal + 33, s))) return st;
    for (int pf = 0; pf < p->npf; pf++) {
        if ((st = rational_apply_int(ctx, p->mass, &p->act, w.phi + pf * w.n3, w.rat, w.X, p->tol_metro, p->maxit,
                                     p->solve_mode_metro, iters, s)))
            return st;
        if ((st = blas_dot_re(ctx, STAG_PREC_F64, w.phi + pf * w.n3, w.rat, ctx->dscal + 34 + pf, s))) return st;
    }
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal + 32, ctx->dscal + 32, sizeof(double) * (2 + p->npf),
                                   cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    const double nplaq = 6.0 * ctx->g.V;
    double h = ctx->hscal[32] + p->beta * (nplaq - ctx->hscal[33]);
    for (int pf = 0; pf < p->npf; pf++) h += ctx->hscal[34 + pf];
    *H = h;
    return STAG_OK;
}

// Integrate over tau: leapfrog P(e/2) Q(e) P(e/2) or Omelyan 2MN
// P(l e) Q(e/2) P((1-2l) e) Q(e/2) P(l e), merged end half-steps.  With
// ngauge > 0 (multi-step scheme) P(.) uses the fermion force only and each
// Q(h) is ngauge inner steps of the same scheme over h with the gauge force
// (inner end half-steps merged within one Q(h)).
int md_integrate(stag_ctx* ctx, const stag_params* p, const TrajWork& w, long long* iters, int* nforce,
                 cudaStream_t s) {
    const double eps = p->tau / p->nsteps;
    const double lam = p->lambda;
    const int multi = p->ngauge > 0;
    int st;
#define FORCE_STEP(coef)                                                                          \
    do {                                                                                          \
        if ((st = total_force(ctx, p, w, iters, s, multi ? FORCE_FERMION : FORCE_ALL))) return st; \
        (*nforce)++;                                                                              \
        if ((st = update_momenta(ctx, w.F, (coef), s))) return st;                                \
    } while (0)
#define GAUGE_STEP(coef)                                                             \
    do {                                                                             \
        if ((st = total_force(ctx, p, w, iters, s, FORCE_GAUGE))) return st;         \
        if ((st = update_momenta(ctx, w.F, (coef), s))) return st;                   \
    } while (0)
    // position update over h: one link update, or the inner gauge scheme
    auto move = [&](double h) -> int {
        if (!multi) return update_links(ctx, h, s);
        const int ng = p->ngauge;
        const double d = h / ng;
        if (p->integrator == STAG_INT_LEAPFROG) {
            GAUGE_STEP(0.5 * d);
            for (int j = 0; j < ng; j++) {
                if ((st = update_links(ctx, d, s))) return st;
                GAUGE_STEP(j == ng - 1 ? 0.5 * d : d);
            }
        } else {
            GAUGE_STEP(lam * d);
            for (int j = 0; j < ng; j++) {
                if ((st = update_links(ctx, 0.5 * d, s))) return st;
                GAUGE_STEP((1.0 - 2.0 * lam) * d);
                if ((st = update_links(ctx, 0.5 * d, s))) return st;
                GAUGE_STEP(j == ng - 1 ? lam * d : 2.0 * lam * d);
            }
        }
        return STAG_OK;
    };
    if (p->integrator == STAG_INT_LEAPFROG) {
        FORCE_STEP(0.5 * eps);
        for (int k = 0; k < p->nsteps; k++) {
            if ((st = move(eps))) return st;
            FORCE_STEP(k == p->nsteps - 1 ? 0.5 * eps : eps);
        }
    } else {
        FORCE_STEP(lam * eps);
        for (int k = 0; k < p->nsteps; k++) {
            if ((st = move(0.5 * eps))) return st;
            FORCE_STEP((1.0 - 2.0 * lam) * eps);
            if ((st = move(0.5 * eps))) return st;
            FORCE_STEP(k == p->nsteps - 1 ? lam * eps : 2.0 * lam * eps);
        }
    }
#undef FORCE_STEP
#undef GAUGE_STEP
    return STAG_OK;
}

}  // namespace

int md_integrate_public(stag_ctx* ctx, const stag_params* p, const double2* phi, long long* iters, int* nforce,
                        cudaStream_t s) {
    const long n3 = 3L * ctx->g.Vh;
    TrajWork w;
    w.n3 = n3;
    w.phi = (double2*)phi;
    w.X = (double2*)ws_get(ctx, WS_FX, sizeof(double2) * n3 * STAG_MAXSHIFT);
    w.F = (double*)ws_get(ctx, WS_FORCE, sizeof(double) * 64 * (size_t)ctx->g.Vh);
    if (!w.X || !w.F) return stag_fail(ctx, STAG_ERR_OOM, "md workspace");
    return md_integrate(ctx, p, w, iters, nforce, s);
}

int rhmc_trajectory(stag_ctx* ctx, const stag_params* p, stag_traj_info* out, cudaStream_t s) {
    memset(out, 0, sizeof(*out));
    const double t0 = now();
    const long n3 = 3L * ctx->g.Vh;
    TrajWork w;
    w.n3 = n3;
    w.phi = (double2*)ws_get(ctx, WS_PHI, sizeof(double2) * n3 * STAG_MAXPF);
    w.R = (double2*)ws_get(ctx, WS_RGAUSS, sizeof(double2) * n3);
    w.rat = (double2*)ws_get(ctx, WS_RAT, sizeof(double2) * n3);
    w.X = (double2*)ws_get(ctx, WS_FX, sizeof(double2) * n3 * STAG_MAXSHIFT);
    w.F = (double*)ws_get(ctx, WS_FORCE, sizeof(double) * 64 * (size_t)ctx->g.Vh);
    if (!w.phi || !w.R || !w.rat || !w.X || !w.F) return stag_fail(ctx, STAG_ERR_OOM, "trajectory workspace");
    long long iters = 0;
    int st;

    // heatbath: P ~ exp(-Tr P^2), phi = r_hb(M) R
    if ((st = momenta_heatbath(ctx, p->seed, p->traj, s))) return st;
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->U64_save, ctx->U64, sizeof(double2) * 48 * (size_t)ctx->g.Vh,
                                   cudaMemcpyDeviceToDevice, s));
    for (int pf = 0; pf < p->npf; pf++) {
        if ((st = pf_gaussian(ctx, p->seed, p->traj, pf, w.R, s))) return st;
        if ((st = rational_apply_int(ctx, p->mass, &p->hb, w.R, w.phi + pf * n3, w.X, p->tol_metro, p->maxit,
                                     p->solve_mode_metro, &iters, s)))
            return st;
    }
    const double t1 = now();
    double H0, H1;
    if ((st = hamiltonian(ctx, p, w, &H0, &iters, s))) return st;
    const double t2 = now();
    int nforce = 0;
    if ((st = md_integrate(ctx, p, w, &iters, &nforce, s))) return st;
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    const double t3 = now();
    if ((st = hamiltonian(ctx, p, w, &H1, &iters, s))) return st;
    if ((st = metro_uniform(ctx, p->seed, p->traj, ctx->dscal + 60, s))) return st;
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal + 60, ctx->dscal + 60, sizeof(double), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    const double dH = H1 - H0;
    const double u = ctx->hscal[60];
    if (!isfinite(dH)) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite dH");
    const int acc = (p->no_metropolis || u < exp(-dH)) ? 1 : 0;
    if (!acc) {
        STAG_CUDA(ctx, cudaMemcpyAsync(ctx->U64, ctx->U64_save, sizeof(double2) * 48 * (size_t)ctx->g.Vh,
                                       cudaMemcpyDeviceToDevice, s));
        if ((st = refresh_lowp_links(ctx, s))) return st;
    }
    if ((st = plaquette_sum(ctx, ctx->dscal + 61, s))) return st;
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal + 61, ctx->dscal + 61, sizeof(double), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    const double t4 = now();
    out->H0 = H0;
    out->H1 = H1;
    out->dH = dH;
    out->u = u;
    out->accepted = acc;
    out->plaq = ctx->hscal[61] / (6.0 * ctx->g.V);
    out->cg_iters = iters;
    out->n_force = nforce;
    out->t_heatbath = t1 - t0;
    out->t_action = (t2 - t1) + (t4 - t3);
    out->t_md = t3 - t2;
    out->t_total = t4 - t0;
    out->status = STAG_OK;
    return STAG_OK;
}

// ms_common.cuh -- the per-system parts of one shifted-CG iteration (Eq. (13)),
// shared by the single-system solver (solver.cu) and the batched
// multi-right-hand-side solver (msmulti.cu).
#pragma once
#include "hop.cuh"
#include "stag_internal.h"

// Scalar update of one shifted CG from the reduced sums of the iteration:
// t0 = <p,w>, t1 = <r,w>, t2 = <w,w>, t3 = |r|^2, with w = (M + s0) p.
//   alpha = t3/t0,  |r - alpha w|^2 = t3 - 2 alpha t1 + alpha^2 t2 (one-step
//   expansion: |r|^2 is reduced afresh every iteration), beta = |r_new|^2/t3,
//   zeta^{j+1}_k = zeta^j zeta^{j-1} a_{j-1} /
//       (zeta^{j-1} a_{j-1} (1 + d_k a_j) + a_j b_{j-1} (zeta^{j-1} - zeta^j)),
//   a_k = alpha zeta^{j+1}/zeta^j,  b_k = beta (zeta^{j+1}/zeta^j)^2,
// shift k stays active while |zeta_k|^2 |r_new|^2 > tol^2 |b|^2.  Called by
// every thread of one block (one thread per shift).  Every value of the state
// is loaded once, up front and in parallel, and written once at the end: this
// runs in the single block that finishes last, while the rest of the GPU
// waits, so its cost is its chain of dependent global-memory round trips.
STAG_D void ms_scalar_update(MSState* st, double t0, double t1, double t2, double t3) {
    __shared__ double s_alpha, s_beta, s_rr;
    __shared__ int s_iter;
    const int k = threadIdx.x;
    const int n = st->n, base = st->base;
    const double ao = st->alpha_old, bo = st->beta_old, tol2 = st->tol2bb, sb = st->shifts[base];
    int actk = 0;
    double zo = 0.0, z = 1.0, sh = 0.0;
    if (k < n) {
        actk = st->active[k];
        zo = st->zeta_old[k];
        z = st->zeta[k];
        sh = st->shifts[k];
    }
    if (k == 0) {
        const int it = st->iter;
        const double alpha = t3 / t0;
        double rr_new = t3 - 2.0 * alpha * t1 + alpha * alpha * t2;
        if (rr_new < 0.0) rr_new = 0.0;
        s_alpha = alpha;
        s_rr = rr_new;
        s_beta = rr_new / t3;
        s_iter = it + 1;
    }
    __syncthreads();
    const double alpha = s_alpha, beta = s_beta, rr_new = s_rr;
    const int iter = s_iter;
    int act = 0;
    if (k < n) {
        if (actk) {
            const double d = sh - sb;
            const double den = zo * ao * (1.0 + d * alpha) + alpha * bo * (zo - z);
            const double zn = z * zo * ao / den;
            const double ratio = zn / z;
            st->ak[k] = alpha * ratio;
            st->bk[k] = beta * ratio * ratio;
            st->zeta_old[k] = z;
            st->zeta[k] = zn;
            st->upd_x[k] = 1;
            st->iters_shift[k] = iter;
            act = (zn * zn * rr_new > tol2) ? 1 : 0;
            st->active[k] = act;
        } else {
            st->upd_x[k] = 0;
            st->ak[k] = 0.0;
        }
    }
    const int n_active = __syncthreads_count(act);
    if (k == 0) {
        st->pw = t0;
        st->alpha = alpha;
        st->iter = iter;
        st->n_active = n_active;
        st->beta = beta;
        st->rr = rr_new;
        st->alpha_old = alpha;
        st->beta_old = beta;
        const int bad = !isfinite(rr_new) || !isfinite(beta) || !isfinite(alpha);
        if (bad) st->nonfinite = 1;
        st->stop_next = (n_active <= st->keep || iter >= st->maxit || bad) ? 1 : 0;
        st->pend = 1;
    }
}

// Coefficients of the shifted vectors' update of the last iteration, staged in
// shared memory by every thread of a block (one per shift).
template <typename R> struct MSCoef {
    R ak[STAG_MAXSHIFT], bk[STAG_MAXSHIFT], z[STAG_MAXSHIFT];
    int ux[STAG_MAXSHIFT], act[STAG_MAXSHIFT];
};
template <typename R> STAG_D void ms_load_coef(const MSState* st, MSCoef<R>& c) {
    const int k = threadIdx.x, ns = st->n;
    if (k < STAG_MAXSHIFT) {
        const bool in = k < ns;
        c.ak[k] = in ? (R)st->ak[k] : (R)0;
        c.bk[k] = in ? (R)st->bk[k] : (R)0;
        c.z[k] = in ? (R)st->zeta[k] : (R)0;
        c.ux[k] = in ? st->upd_x[k] : 0;
        c.act[k] = in ? st->active[k] : 0;
    }
}

// The shifted vectors' update of one iteration at entry i (x_k += a_k p_k with
// the old p_k, then p_k = zeta_k r + b_k p_k for the shifts still active),
// with r the base residual after that iteration.
template <typename V2, typename R>
STAG_D void ms_shift_update_at(long i, long stride, int ns, const V2 rv, V2* __restrict__ pk, V2* __restrict__ xk,
                               const MSCoef<R>& c) {
    for (int k = 0; k < ns; k++) {
        if (!c.ux[k]) continue;
        V2 q = pk[k * stride + i];
        V2 x = xk[k * stride + i];
        x.x += c.ak[k] * q.x;
        x.y += c.ak[k] * q.y;
        xk[k * stride + i] = x;
        if (c.act[k]) {
            q.x = c.z[k] * rv.x + c.bk[k] * q.x;
            q.y = c.z[k] * rv.y + c.bk[k] * q.y;
            pk[k * stride + i] = q;
        }
    }
}

// Vector update of one shifted CG over the entries this block owns:
// r -= alpha w; p = r + beta p; x_k += a_k p_k (old p_k); p_k = zeta_k r + b_k p_k.
template <typename V2, typename R>
STAG_D void ms_vector_update(long n, long stride, long i0, long step, V2* __restrict__ r, const V2* __restrict__ w,
                             V2* __restrict__ p, V2* __restrict__ pk, V2* __restrict__ xk, const MSState* st) {
    __shared__ R s_ak[STAG_MAXSHIFT], s_bk[STAG_MAXSHIFT], s_z[STAG_MAXSHIFT];
    __shared__ int s_ux[STAG_MAXSHIFT], s_act[STAG_MAXSHIFT];
    const int ns = st->n;
    if (threadIdx.x < ns) {
        s_ak[threadIdx.x] = (R)st->ak[threadIdx.x];
        s_bk[threadIdx.x] = (R)st->bk[threadIdx.x];
        s_z[threadIdx.x] = (R)st->zeta[threadIdx.x];
        s_ux[threadIdx.x] = st->upd_x[threadIdx.x];
        s_act[threadIdx.x] = st->active[threadIdx.x];
    }
    __syncthreads();
    const R alpha = (R)st->alpha, beta = (R)st->beta;
    for (long i = i0; i < n; i += step) {
        V2 rv = r[i];
        const V2 wv = w[i];
        rv.x -= alpha * wv.x;
        rv.y -= alpha * wv.y;
        r[i] = rv;
        V2 pv = p[i];
        pv.x = rv.x + beta * pv.x;
        pv.y = rv.y + beta * pv.y;
        p[i] = pv;
        for (int k = 0; k < ns; k++) {
            if (!s_ux[k]) continue;
            V2 q = pk[k * stride + i];
            V2 x = xk[k * stride + i];
            x.x += s_ak[k] * q.x;
            x.y += s_ak[k] * q.y;
            xk[k * stride + i] = x;
            if (s_act[k]) {
                q.x = s_z[k] * rv.x + s_bk[k] * q.x;
                q.y = s_z[k] * rv.y + s_bk[k] * q.y;
                pk[k * stride + i] = q;
            }
        }
    }
}

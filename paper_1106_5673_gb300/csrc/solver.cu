// solver.cu -- shifted (multi-shift) CG for (M_ee + s_k) x_k = b (Eq. (13),
// Sec. 4.3) and the single-shift CG with FP64 reliable updates used to refine
// each shift in mixed precision.
//
// One iteration of the shifted CG is four kernels:
//   A  t   = D_oe p                                   (hop, odd output)
//   B  w   = c0 p - D_eo t, pw = Re<p,w>              (hop, even output, fused
//          reduction; the last block computes alpha, zeta^{j+1}_k, a_k)
//   C  r  -= alpha w, rr = |r|^2                      (last block: beta, b_k,
//          convergence per shift, stop flag)
//   D  p   = r + beta p; x_k += a_k p_k; p_k = zeta_k r + b_k p_k
// All scalars live in device memory (MSState), so the host never waits inside
// an iteration; it reads the `live` flag every `chunk` iterations.  The chunk
// is captured once per context as a CUDA graph.  Kernels started after the
// stop flag return immediately.
#include "hop.cuh"
#include "ms_common.cuh"
#include "stag_internal.h"

#include <algorithm>

#include <chrono>
#include <vector>
#include <math.h>
#include <stdlib.h>

static const int HOP_TPB = 128;
static const int BLAS_TPB = 256;

static int env_int(const char* name, int dflt) {
    const char* v = getenv(name);
    return v ? atoi(v) : dflt;
}
static double env_dbl(const char* name, double dflt) {
    const char* v = getenv(name);
    return v ? atof(v) : dflt;
}

// Kernels of one shifted-CG iteration: STAG_FUSED=1 (default) A, B3, CD;
// 2: A2, B3, C2 with the shifted vectors' update deferred into the next A2
// (measured 3 % slower for the FP32 solve at 32^3x8 and 11 % slower in
// float-float: the streaming does not hide behind the hop's gathers);
// 0: the four-kernel form A, B, C, D.
// Unconverged shifts at which the FP32 shifted CG stops (STAG_MS_KEEP,
// default 0: it runs until every shift has converged).  Measured on the
// 15-shift solve at 32^3x8: stopping with the lightest 1, 2 or 3 shifts still
// unconverged gives 0.146, 0.149 and 0.156 s against 0.147 s; the refinement
// of those shifts takes nearly as many more iterations as the recursion
// saves (the lightest: +123 for 148 saved, +875 for 943 saved).
static int ms_keep() { return env_int("STAG_MS_KEEP", 0); }

static int fused_iter() {
    static int f = -1;
    if (f < 0) f = env_int("STAG_FUSED", 1);
    return f;
}

static Links make_links(const stag_ctx* ctx, int lp) {
    Links L;
    L.lo = ctx->U32lo;
    L.u = (lp == LP64) ? (const void*)ctx->U64
          : (lp == LP32 || lp == LPFF) ? (const void*)ctx->U32
          : (lp == LP8) ? (const void*)ctx->U8
                        : (const void*)ctx->U16;
    return L;
}

// ============================================================== multi-shift kernels

template <typename R, int LP>
__global__ void __launch_bounds__(256) k_ms_A(Geom g, Links U,
                                                  const typename VT<R>::T* __restrict__ p,
                                                  typename VT<R>::T* __restrict__ t, MSState* st) {
    // the stop requested by the previous iteration's scalar update takes
    // effect here, after that iteration's vector update has run
    const int live = st->live, stop = st->stop_next;
    if (!live) return;
    if (stop) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->live = 0;
        return;
    }
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const Site s = site_of(g, h, 1);
    Vec3<R> acc = hopL<R, LP>(g, U, p, h, 1, s);
#pragma unroll
    for (int a = 0; a < 3; a++) acc.c[a] = (R)0.5 * acc.c[a];
    st_vec(t, h, acc);
}

// w = c0 p - 1/2 hop(t) on even sites; returns Re<p, w> in FP64 via partials
template <typename R, int LP>
STAG_D double mee_second_hop(const Geom& g, Links U, const typename VT<R>::T* t,
                             const typename VT<R>::T* p, typename VT<R>::T* w, R c0, int h) {
    double pw = 0.0;
    if (h < g.Vh) {
        const Site s = site_of(g, h, 0);
        Vec3<R> acc = hopL<R, LP>(g, U, t, h, 0, s);
        Vec3<R> pv = load_vec(p, h);
        Vec3<R> r;
        R ppw = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            r.c[a] = c0 * pv.c[a] - (R)0.5 * acc.c[a];
            ppw += pv.c[a].re * r.c[a].re + pv.c[a].im * r.c[a].im;
        }
        st_vec(w, h, r);
        pw = (double)ppw;
    }
    return pw;
}

template <typename R, int LP>
__global__ void __launch_bounds__(256) k_ms_B(Geom g, Links U,
                                                  const typename VT<R>::T* __restrict__ t,
                                                  const typename VT<R>::T* __restrict__ p,
                                                  typename VT<R>::T* __restrict__ w, MSState* st, double* partials,
                                                  unsigned int* counter) {
    if (!st->live) return;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    double pw = mee_second_hop<R, LP>(g, U, t, p, w, (R)st->c0, h);
    pw = block_sum(pw);
    if (threadIdx.x == 0) partials[blockIdx.x] = pw;
    if (last_block(counter)) {
        double tot = 0.0;
        for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += __ldcg(partials + i);
        tot = block_sum(tot);
        __shared__ double s_alpha;
        if (threadIdx.x == 0) {
            st->pw = tot;
            s_alpha = st->rr / tot;
            st->alpha = s_alpha;
        }
        __syncthreads();
        // one thread per shift: the zeta recurrences are independent
        const int k = threadIdx.x;
        if (k < st->n) {
            const double alpha = s_alpha;
            if (st->active[k]) {
                const double d = st->shifts[k] - st->shifts[st->base];
                const double zo = st->zeta_old[k], z = st->zeta[k], ao = st->alpha_old;
                const double den = zo * ao * (1.0 + d * alpha) + alpha * st->beta_old * (zo - z);
                const double zn = z * zo * ao / den;
                st->zeta_next[k] = zn;
                st->ak[k] = alpha * zn / z;
                st->upd_x[k] = 1;
            } else {
                st->upd_x[k] = 0;
                st->ak[k] = 0.0;
            }
        }
    }
}

// ---- fused variant: 3 kernels per iteration (A, B3, CD)
// B3: w = c0 p - D_eo t and the three sums <p,w>, <r,w>, <w,w>; the last block
// forms alpha = rr/<p,w> and |r - alpha w|^2 = rr - 2 alpha <r,w> + alpha^2 <w,w>
// (no separate pass over r), then every scalar of the iteration: the shifted
// zeta, a_k, b_k, per-shift convergence and the stop flag.
template <typename R, int LP>
__global__ void __launch_bounds__(256) k_ms_B3(Geom g, Links U, const typename VT<R>::T* __restrict__ t,
                                                   const typename VT<R>::T* __restrict__ p,
                                                   const typename VT<R>::T* __restrict__ r,
                                                   typename VT<R>::T* __restrict__ w, MSState* st, double* partials,
                                                   double* gpart, unsigned int* counter) {
    // the previous A2 has applied any pending shifted update; the scalar
    // update of this kernel's last block sets it again (after this write: the
    // grid reduction's fence and counter order block 0 before the last block)
    if (blockIdx.x == 0 && threadIdx.x == 0) st->pend = 0;
    if (!st->live) return;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    R sv[4] = {0, 0, 0, 0};
    if (h < g.Vh) {
        const Site s = site_of(g, h, 0);
        const Vec3<R> acc = hopL<R, LP>(g, U, t, h, 0, s);
        const Vec3<R> pv = load_vec(p, h), rv = load_vec(r, h);
        const R c0 = (R)st->c0;
        Vec3<R> wv;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            wv.c[i] = c0 * pv.c[i] - (R)0.5 * acc.c[i];
            sv[0] += pv.c[i].re * wv.c[i].re + pv.c[i].im * wv.c[i].im;
            sv[1] += rv.c[i].re * wv.c[i].re + rv.c[i].im * wv.c[i].im;
            sv[2] += wv.c[i].re * wv.c[i].re + wv.c[i].im * wv.c[i].im;
            sv[3] += rv.c[i].re * rv.c[i].re + rv.c[i].im * rv.c[i].im;
        }
        st_vec(w, h, wv);
    }
    const double bsum = block_sum_nv<4, R>(sv);
    if (threadIdx.x < 4) partials[threadIdx.x * gridDim.x + blockIdx.x] = bsum;
    __shared__ double s_t[4];
    if (grid_reduce_series(partials, gpart, counter, 4, s_t)) ms_scalar_update(st, s_t[0], s_t[1], s_t[2], s_t[3]);
}

// ---- deferred variant of the fused iteration (the default): the shifted
// vectors' update of iteration j (x_k += a_k p_k, p_k = zeta_k r_{j+1} + b_k p_k)
// needs only r_{j+1} at the same entry, so it runs inside the next
// iteration's first hop kernel (A2), whose gathers leave the memory system
// room for the streaming; C2 updates only r and p.  st->pend marks an update
// still to be applied: set by B3's scalar update, consumed by the next A2,
// cleared by the next B3's first block (which starts after every A2 block
// has finished, and before its own scalar update can set it again).
template <typename R, int LP>
__global__ void __launch_bounds__(256) k_ms_A2(Geom g, Links U, const typename VT<R>::T* __restrict__ p,
                                                typename VT<R>::T* __restrict__ t,
                                                const typename VT<R>::T* __restrict__ r,
                                                typename VT<R>::T* __restrict__ pk, typename VT<R>::T* __restrict__ xk,
                                                MSState* st) {
    typedef typename VT<R>::T V2;
    __shared__ MSCoef<R> c;
    const int live = st->live, stop = st->stop_next;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (st->pend) {  // uniform: nothing writes pend while this kernel runs
        ms_load_coef<R>(st, c);
        __syncthreads();
        if (h < g.Vh) {
            const long stride = 3L * g.Vh, ns = st->n;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const long i = 3L * h + a;
                ms_shift_update_at<V2, R>(i, stride, (int)ns, r[i], pk, xk, c);
            }
        }
    }
    if (!live) return;
    if (stop) {  // the stop requested by the last scalar update takes effect here
        if (blockIdx.x == 0 && threadIdx.x == 0) st->live = 0;
        return;
    }
    if (h >= g.Vh) return;
    const Site s = site_of(g, h, 1);
    Vec3<R> acc = hopL<R, LP>(g, U, p, h, 1, s);
#pragma unroll
    for (int a = 0; a < 3; a++) acc.c[a] = (R)0.5 * acc.c[a];
    st_vec(t, h, acc);
}

// C2: r -= alpha w; p = r + beta p
template <typename V2, typename R>
__global__ void k_ms_C2(long n, V2* __restrict__ r, const V2* __restrict__ w, V2* __restrict__ p, const MSState* st) {
    if (!st->live) return;
    const R alpha = (R)st->alpha, beta = (R)st->beta;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        V2 rv = r[i];
        const V2 wv = w[i];
        rv.x -= alpha * wv.x;
        rv.y -= alpha * wv.y;
        r[i] = rv;
        V2 pv = p[i];
        pv.x = rv.x + beta * pv.x;
        pv.y = rv.y + beta * pv.y;
        p[i] = pv;
    }
}

// the pending shifted update alone (after the last iteration, or before a
// reliable update); clears st->pend in a later launch (k_ms_clear_pend)
template <typename V2, typename R>
__global__ void k_ms_shift_update(long n, long stride, const V2* __restrict__ r, V2* __restrict__ pk,
                                  V2* __restrict__ xk, const MSState* st) {
    __shared__ MSCoef<R> c;
    if (!st->pend) return;
    ms_load_coef<R>(st, c);
    __syncthreads();
    const int ns = st->n;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        ms_shift_update_at<V2, R>(i, stride, ns, r[i], pk, xk, c);
}
__global__ void k_ms_clear_pend(MSState* st) { st->pend = 0; }

// CD: r -= alpha w; p = r + beta p; x_k += a_k p_k; p_k = zeta_k r + b_k p_k
template <typename V2, typename R>
__global__ void k_ms_CD(long n, long stride, V2* __restrict__ r, const V2* __restrict__ w, V2* __restrict__ p,
                        V2* __restrict__ pk, V2* __restrict__ xk, MSState* st, unsigned int* counter) {
    if (!st->live) return;
    ms_vector_update<V2, R>(n, stride, blockIdx.x * (long)blockDim.x + threadIdx.x, (long)gridDim.x * blockDim.x, r,
                            w, p, pk, xk, st);
}
// FP32 vectors: the same update on float4 (two complex entries per access;
// 3 Vh is even, so n4 = 3 Vh / 2 and every vector starts 16-byte aligned)
template <int G>
__global__ void k_ms_CD4(long n, long stride, float2* __restrict__ r2, const float2* __restrict__ w2,
                         float2* __restrict__ p2, float2* __restrict__ pk2, float2* __restrict__ xk2, MSState* st) {
    if (!st->live) return;
    __shared__ MSCoef<float> c;
    __shared__ int kl[STAG_MAXSHIFT], nkl;
    ms_load_coef<float>(st, c);
    __syncthreads();
    // the shifts whose x_k is updated, compacted in order (a ballot over warp 0)
    if (threadIdx.x < 32) {
        const int k = threadIdx.x;
        const bool u = k < STAG_MAXSHIFT && c.ux[k];
        const unsigned int m = __ballot_sync(0xffffffffu, u);
        if (u) kl[__popc(m & ((1u << k) - 1u))] = k;
        if (k == 0) nkl = __popc(m);
    }
    __syncthreads();
    const float alpha = (float)st->alpha, beta = (float)st->beta;
    const int nk = nkl;
    const long n4 = n / 2, s4 = stride / 2;
    float4* r = (float4*)r2;
    const float4* w = (const float4*)w2;
    float4* p = (float4*)p2;
    float4* pk = (float4*)pk2;
    float4* xk = (float4*)xk2;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
        float4 rv = r[i];
        const float4 wv = w[i];
        float4 pv = p[i];
        rv.x = fmaf(-alpha, wv.x, rv.x);
        rv.y = fmaf(-alpha, wv.y, rv.y);
        rv.z = fmaf(-alpha, wv.z, rv.z);
        rv.w = fmaf(-alpha, wv.w, rv.w);
        r[i] = rv;
        pv.x = fmaf(beta, pv.x, rv.x);
        pv.y = fmaf(beta, pv.y, rv.y);
        pv.z = fmaf(beta, pv.z, rv.z);
        pv.w = fmaf(beta, pv.w, rv.w);
        p[i] = pv;
        // shifts in groups of G: every load of a group is issued before its
        // first store (one shift's stores never alias another's loads, which
        // the compiler cannot prove by itself)
        for (int j0 = 0; j0 < nk; j0 += G) {
            float4 q[G], x[G];
#pragma unroll
            for (int u = 0; u < G; u++)
                if (j0 + u < nk) {
                    const long o = kl[j0 + u] * s4 + i;
                    q[u] = pk[o];
                    x[u] = xk[o];
                }
#pragma unroll
            for (int u = 0; u < G; u++)
                if (j0 + u < nk) {
                    const int k = kl[j0 + u];
                    const long o = k * s4 + i;
                    const float a = c.ak[k];
                    x[u].x = fmaf(a, q[u].x, x[u].x);
                    x[u].y = fmaf(a, q[u].y, x[u].y);
                    x[u].z = fmaf(a, q[u].z, x[u].z);
                    x[u].w = fmaf(a, q[u].w, x[u].w);
                    xk[o] = x[u];
                    if (c.act[k]) {
                        const float z = c.z[k], b = c.bk[k];
                        q[u].x = fmaf(b, q[u].x, z * rv.x);
                        q[u].y = fmaf(b, q[u].y, z * rv.y);
                        q[u].z = fmaf(b, q[u].z, z * rv.z);
                        q[u].w = fmaf(b, q[u].w, z * rv.w);
                        pk[o] = q[u];
                    }
                }
        }
    }
}

template <typename V2, typename R>
__global__ void k_ms_C(long n, V2* __restrict__ r, const V2* __restrict__ w, MSState* st, double* partials,
                       unsigned int* counter) {
    if (!st->live) return;
    const R alpha = (R)st->alpha;
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        V2 rv = r[i], wv = w[i];
        rv.x -= alpha * wv.x;
        rv.y -= alpha * wv.y;
        r[i] = rv;
        acc += (double)(rv.x * rv.x + rv.y * rv.y);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    if (last_block(counter)) {
        double tot = 0.0;
        for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += __ldcg(partials + i);
        tot = block_sum(tot);
        __shared__ double s_rr, s_beta;
        __shared__ int s_iter;
        if (threadIdx.x == 0) {
            s_rr = tot;
            s_beta = tot / st->rr;
            s_iter = st->iter + 1;
        }
        __syncthreads();
        // one thread per shift
        const int k = threadIdx.x;
        int act = 0;
        if (k < st->n) {
            if (st->upd_x[k]) {
                const double zn = st->zeta_next[k], z = st->zeta[k];
                const double ratio = zn / z;
                st->bk[k] = s_beta * ratio * ratio;
                st->zeta_old[k] = z;
                st->zeta[k] = zn;
                st->iters_shift[k] = s_iter;
                st->active[k] = (zn * zn * s_rr > st->tol2bb) ? 1 : 0;
            }
            act = st->active[k];
        }
        const int n_active = __syncthreads_count(act);
        if (threadIdx.x == 0) {
            const double rr_new = s_rr, beta = s_beta;
            st->iter = s_iter;
            st->n_active = n_active;
            st->beta = beta;
            st->rr = rr_new;
            st->alpha_old = st->alpha;
            st->beta_old = beta;
            const int bad = !isfinite(rr_new) || !isfinite(beta);
            if (bad) st->nonfinite = 1;
            st->stop_next = (n_active <= st->keep || s_iter >= st->maxit || bad) ? 1 : 0;
        }
    }
}

template <typename V2, typename R>
__global__ void k_ms_D(long n, long stride, const V2* __restrict__ r, V2* __restrict__ p, V2* __restrict__ pk,
                       V2* __restrict__ xk, MSState* st, unsigned int* counter) {
    if (!st->live) return;
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
    const R beta = (R)st->beta;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const V2 rv = r[i];
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
    if (last_block(counter)) {
        if (threadIdx.x == 0 && st->stop_next) st->live = 0;
    }
}

// initial vectors: r = p = p_k = b, x_k = 0 (b in FP64, vectors in V2)
template <typename V2>
__global__ void k_ms_init_vec(long n, long stride, int ns, const double2* __restrict__ b, V2* r, V2* p, V2* pk,
                              V2* xk) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 v = b[i];
        V2 c;
        c.x = v.x;
        c.y = v.y;
        V2 z;
        z.x = 0;
        z.y = 0;
        r[i] = c;
        p[i] = c;
        for (int k = 0; k < ns; k++) {
            pk[k * stride + i] = c;
            xk[k * stride + i] = z;
        }
    }
}

__global__ void k_ms_init_scalars(MSState* st, double tol2, double c_mass) {
    const double bb = st->bb;
    st->rr = bb;
    st->tol2bb = tol2 * bb;
    st->alpha_old = 1.0;
    st->beta_old = 0.0;
    st->iter = 0;
    st->nonfinite = !isfinite(bb);
    st->stop_next = 0;
    st->pend = 0;
    int base = 0;
    for (int k = 1; k < st->n; k++)
        if (st->shifts[k] < st->shifts[base]) base = k;
    st->base = base;
    st->c0 = c_mass + st->shifts[base];
    for (int k = 0; k < st->n; k++) {
        st->zeta[k] = st->zeta_old[k] = 1.0;
        st->active[k] = (bb > 0.0 && isfinite(bb)) ? 1 : 0;
        st->upd_x[k] = 0;
        st->iters_shift[k] = 0;
        st->ak[k] = st->bk[k] = 0.0;
    }
    st->n_active = st->active[0] ? st->n : 0;
    st->live = st->n_active > 0;
}

// ============================================================== single-shift CG (refinement)

// x_lo += alpha p, r -= alpha w, rr_new = |r|^2; last block: reliable-update test and beta
template <typename V2, typename R>
__global__ void k_cg_C(long n, V2* __restrict__ r, const V2* __restrict__ w, const V2* __restrict__ p,
                       V2* __restrict__ x, CGState* st, double* partials, unsigned int* counter) {
    if (!st->live) return;
    const R alpha = (R)st->alpha;
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        V2 rv = r[i], wv = w[i], pv = p[i], xv = x[i];
        rv.x -= alpha * wv.x;
        rv.y -= alpha * wv.y;
        xv.x += alpha * pv.x;
        xv.y += alpha * pv.y;
        r[i] = rv;
        x[i] = xv;
        acc += (double)(rv.x * rv.x + rv.y * rv.y);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    if (last_block(counter)) {
        double tot = 0.0;
        for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += __ldcg(partials + i);
        tot = block_sum(tot);
        if (threadIdx.x == 0) {
            st->iter += 1;
            const int bad = !isfinite(tot);
            if (bad) st->nonfinite = 1;
            // reliable update when the residual dropped by delta since the last one,
            // or when the recursive residual claims convergence
            const int rel = (tot < st->delta2 * st->rr_max) || (tot <= st->tol2bb);
            st->want_reliable = rel;
            st->beta = tot / st->rr;
            st->rr_prev = st->rr;
            st->rr = tot;
            st->stop_next = (rel || bad || st->iter >= st->maxit) ? 1 : 0;
        }
    }
}

// p = r + beta p (skipped when a reliable update is pending: the host does it)
template <typename V2, typename R>
__global__ void k_cg_D(long n, const V2* __restrict__ r, V2* __restrict__ p, CGState* st, unsigned int* counter) {
    if (!st->live) return;
    if (!st->want_reliable) {
        const R beta = (R)st->beta;
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
            V2 rv = r[i], pv = p[i];
            pv.x = rv.x + beta * pv.x;
            pv.y = rv.y + beta * pv.y;
            p[i] = pv;
        }
    }
    if (last_block(counter)) {
        if (threadIdx.x == 0 && st->stop_next) st->live = 0;
    }
}

template <typename R, int LP>
__global__ void __launch_bounds__(256) k_cg_A(Geom g, Links U,
                                                  const typename VT<R>::T* __restrict__ p,
                                                  typename VT<R>::T* __restrict__ t, const CGState* st) {
    if (!st->live) return;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const Site s = site_of(g, h, 1);
    Vec3<R> acc = hopL<R, LP>(g, U, p, h, 1, s);
#pragma unroll
    for (int a = 0; a < 3; a++) acc.c[a] = (R)0.5 * acc.c[a];
    st_vec(t, h, acc);
}

template <typename R, int LP>
__global__ void __launch_bounds__(256) k_cg_B(Geom g, Links U,
                                                  const typename VT<R>::T* __restrict__ t,
                                                  const typename VT<R>::T* __restrict__ p,
                                                  typename VT<R>::T* __restrict__ w, CGState* st, double* partials,
                                                  unsigned int* counter) {
    if (!st->live) return;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    double pw = mee_second_hop<R, LP>(g, U, t, p, w, (R)st->c0, h);
    pw = block_sum(pw);
    if (threadIdx.x == 0) partials[blockIdx.x] = pw;
    if (last_block(counter)) {
        double tot = 0.0;
        for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += __ldcg(partials + i);
        tot = block_sum(tot);
        if (threadIdx.x == 0) {
            st->pw = tot;
            st->alpha = st->rr / tot;
        }
    }
}

// r = b - w (FP64), |r|^2 -> dst; optionally also the FP32 copy of r
template <typename V2>
__global__ void k_residual(long n, const double2* __restrict__ b, const double2* __restrict__ w, double2* r,
                           V2* rlow, double* partials, unsigned int* counter, double* dst) {
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 bv = b[i], wv = w[i];
        double2 rv = make_double2(bv.x - wv.x, bv.y - wv.y);
        if (r) r[i] = rv;
        if (rlow) {
            V2 c;
            c.x = rv.x;
            c.y = rv.y;
            rlow[i] = c;
        }
        acc += rv.x * rv.x + rv.y * rv.y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    if (last_block(counter)) finish_sum(partials, gridDim.x, dst);
}

// x_hi += x_lo (FP64 accumulation of the low-precision correction), x_lo = 0
template <typename V2>
__global__ void k_accumulate(long n, double2* xhi, V2* xlo) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        V2 v = xlo[i];
        double2 x = xhi[i];
        x.x += (double)v.x;
        x.y += (double)v.y;
        xhi[i] = x;
        v.x = 0;
        v.y = 0;
        xlo[i] = v;
    }
}

// after a reliable update: p = r + beta p with beta = rr_new / rr_old, and reset scalars
template <typename V2>
__global__ void k_cg_restart_p(long n, const V2* __restrict__ r, V2* p, double beta, int reset_p) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        V2 rv = r[i], pv = p[i];
        if (reset_p) {
            pv = rv;
        } else {
            pv.x = rv.x + (decltype(rv.x))beta * pv.x;
            pv.y = rv.y + (decltype(rv.x))beta * pv.y;
        }
        p[i] = pv;
    }
}

// ============================================================== reliable updates of the FP32 shifted CG
// (mixed modes; Sec. 4.3: the shifted solver cannot restart, so the base
// residual is replaced in place).  The FP32 solution vectors hold only the
// increments since the last update; they are added into the FP64 solutions
// here, which keeps their rounding proportional to the current residual.

// X_k += x_k (FP64), x_k = 0 for the ns shifts
__global__ void k_ms_flush(long n, long stride, int ns, float2* __restrict__ xk, double2* __restrict__ X) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        for (int k = 0; k < ns; k++) {
            const float2 v = xk[k * stride + i];
            double2 x = X[k * stride + i];
            x.x += (double)v.x;
            x.y += (double)v.y;
            X[k * stride + i] = x;
            xk[k * stride + i] = make_float2(0.f, 0.f);
        }
    }
}

// Residual replacement: r_t = b - w with w = (M_ee + s_base) X_base computed
// FP64-accurately; d = fl32(r_t) - r; r = fl32(r_t); p += d and, for every
// shift still active, p_k += zeta_k d: the search vectors the last iteration
// would have built from the true residual.  |r_t|^2 (FP64) into *dst.
__global__ void k_ms_replace(long n, long stride, const double2* __restrict__ b, const double2* __restrict__ w,
                             float2* __restrict__ r, float2* __restrict__ p, float2* __restrict__ pk,
                             const MSState* st, double* partials, unsigned int* counter, double* dst) {
    __shared__ float s_z[STAG_MAXSHIFT];
    __shared__ int s_act[STAG_MAXSHIFT];
    const int ns = st->n;
    if (threadIdx.x < STAG_MAXSHIFT) {
        s_z[threadIdx.x] = threadIdx.x < ns ? (float)st->zeta[threadIdx.x] : 0.f;
        s_act[threadIdx.x] = threadIdx.x < ns ? st->active[threadIdx.x] : 0;
    }
    __syncthreads();
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 bv = b[i], wv = w[i];
        const double rx = bv.x - wv.x, ry = bv.y - wv.y;
        acc += rx * rx + ry * ry;
        const float2 rn = make_float2((float)rx, (float)ry), ro = r[i];
        const float dx = rn.x - ro.x, dy = rn.y - ro.y;
        r[i] = rn;
        float2 pv = p[i];
        pv.x += dx;
        pv.y += dy;
        p[i] = pv;
        for (int k = 0; k < ns; k++) {
            if (!s_act[k]) continue;
            float2 q = pk[k * stride + i];
            q.x += s_z[k] * dx;
            q.y += s_z[k] * dy;
            pk[k * stride + i] = q;
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    if (last_block(counter)) finish_sum(partials, gridDim.x, dst);
}

// ============================================================== host side

namespace {

struct MSBufs {
    void *r, *p, *w, *t, *pk, *xk;
};

// The fused vector update; FP32 vectors take the float4 form with the shifts
// in groups of STAG_CD_GROUP (1, 2 or 4).  Measured on the 15-shift solve at
// 32^3x8: 0.155 s with groups of one, 0.156 s with two and 0.157 s with four
// (the loads issued ahead cost registers and resident warps).
template <typename V2, typename R>
static void launch_ms_cd(stag_ctx* ctx, int nb, long n, const MSBufs& b, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        const int grp = env_int("STAG_CD_GROUP", 1);
        if (grp == 1)
            k_ms_CD4<1><<<nb, BLAS_TPB, 0, s>>>(n, n, (float2*)b.r, (const float2*)b.w, (float2*)b.p, (float2*)b.pk,
                                                (float2*)b.xk, ctx->ms);
        else if (grp == 2)
            k_ms_CD4<2><<<nb, BLAS_TPB, 0, s>>>(n, n, (float2*)b.r, (const float2*)b.w, (float2*)b.p, (float2*)b.pk,
                                                (float2*)b.xk, ctx->ms);
        else
            k_ms_CD4<4><<<nb, BLAS_TPB, 0, s>>>(n, n, (float2*)b.r, (const float2*)b.w, (float2*)b.p, (float2*)b.pk,
                                                (float2*)b.xk, ctx->ms);
    } else {
        k_ms_CD<V2, R><<<nb, BLAS_TPB, 0, s>>>(n, n, (V2*)b.r, (const V2*)b.w, (V2*)b.p, (V2*)b.pk, (V2*)b.xk, ctx->ms,
                                               ctx->counter);
    }
}

template <typename R, int LP>
void launch_ms_iter(stag_ctx* ctx, Links U, const MSBufs& b, cudaStream_t s) {
    typedef typename VT<R>::T V2;
    const Geom& g = ctx->g;
    const long n = 3L * g.Vh;
    const int tpb = hop_tpb(ctx, LP);
    const int nb_hop = nblocks(g.Vh, tpb);
    const int nb_blas = ctx->num_sms * 4;
    // the fused vector update: one float4 per thread (3 Vh / 2 of them) by default
    const int cd_bps = env_int("STAG_CD_BPS", 0);
    const long n4 = n / 2;
    const int nb_cd = cd_bps > 0 ? ctx->num_sms * cd_bps : (int)((n4 + BLAS_TPB - 1) / BLAS_TPB);
    if (fused_iter() == 2) {  // deferred shifted updates (A2, B3, C2)
        k_ms_A2<R, LP><<<nb_hop, tpb, 0, s>>>(g, U, (const V2*)b.p, (V2*)b.t, (const V2*)b.r, (V2*)b.pk,
                                                 (V2*)b.xk, ctx->ms);
        k_ms_B3<R, LP><<<nb_hop, tpb, 0, s>>>(g, U, (const V2*)b.t, (const V2*)b.p, (const V2*)b.r, (V2*)b.w,
                                                 ctx->ms, ctx->partials, ctx->gpart, ctx->counter);
        k_ms_C2<V2, R><<<nb_blas, BLAS_TPB, 0, s>>>(n, (V2*)b.r, (const V2*)b.w, (V2*)b.p, ctx->ms);
        return;
    }
    k_ms_A<R, LP><<<nb_hop, tpb, 0, s>>>(g, U, (const V2*)b.p, (V2*)b.t, ctx->ms);
    if (fused_iter() == 1) {  // shifted updates in the vector kernel (A, B3, CD)
        k_ms_B3<R, LP><<<nb_hop, tpb, 0, s>>>(g, U, (const V2*)b.t, (const V2*)b.p, (const V2*)b.r, (V2*)b.w,
                                                 ctx->ms, ctx->partials, ctx->gpart, ctx->counter);
        launch_ms_cd<V2, R>(ctx, nb_cd, n, b, s);
        return;
    }
    k_ms_B<R, LP><<<nb_hop, tpb, 0, s>>>(g, U, (const V2*)b.t, (const V2*)b.p, (V2*)b.w, ctx->ms,
                                            ctx->partials, ctx->counter);
    k_ms_C<V2, R><<<nb_blas, BLAS_TPB, 0, s>>>(n, (V2*)b.r, (const V2*)b.w, ctx->ms, ctx->partials, ctx->counter);
    k_ms_D<V2, R><<<nb_blas, BLAS_TPB, 0, s>>>(n, n, (const V2*)b.r, (V2*)b.p, (V2*)b.pk, (V2*)b.xk, ctx->ms,
                                              ctx->counter);
}

template <typename R, int LP>
void launch_cg_iter(stag_ctx* ctx, Links U, void* r, void* p, void* w, void* t, void* x, cudaStream_t s) {
    typedef typename VT<R>::T V2;
    const Geom& g = ctx->g;
    const long n = 3L * g.Vh;
    const int tpb = hop_tpb(ctx, LP);
    const int nb_hop = nblocks(g.Vh, tpb);
    const int nb_blas = ctx->num_sms * 4;
    k_cg_A<R, LP><<<nb_hop, tpb, 0, s>>>(g, U, (const V2*)p, (V2*)t, ctx->cg);
    k_cg_B<R, LP><<<nb_hop, tpb, 0, s>>>(g, U, (const V2*)t, (const V2*)p, (V2*)w, ctx->cg, ctx->partials,
                                            ctx->counter);
    k_cg_C<V2, R><<<nb_blas, BLAS_TPB, 0, s>>>(n, (V2*)r, (const V2*)w, (const V2*)p, (V2*)x, ctx->cg,
                                              ctx->partials, ctx->counter);
    k_cg_D<V2, R><<<nb_blas, BLAS_TPB, 0, s>>>(n, (const V2*)r, (V2*)p, ctx->cg, ctx->counter);
}

// Runs `fn` (which enqueues `chunk` iterations) either directly or through a
// CUDA graph cached under `key`.  The graph is captured on a private stream
// and launched on `s`.
// Marks the FP32 links as persisting in L2 for every kernel of a solver
// graph: between two hops the vector update streams the shifted vectors
// (up to 2 x 32 per site), which would otherwise evict the links.  The
// context's persisting-L2 carve-out (a per-process limit, released at exit) is
// set once.  Off by default (STAG_L2_PERSIST=1 enables it): measured on the
// 32^3x8 trajectory it gained 1 %, the hops reading links faster and the vector
// updates slower by about as much.
static cudaError_t persist_links(stag_ctx* ctx, cudaGraph_t graph) {
    static int on = -1;
    if (on < 0) on = env_int("STAG_L2_PERSIST", 0);
    if (!on) return cudaSuccess;
    int max_persist = 0, max_window = 0;
    if (cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device) != cudaSuccess ||
        max_persist <= 0 || max_window <= 0) {
        cudaGetLastError();
        return cudaSuccess;  // no persisting L2 on this device: nothing to do
    }
    const size_t links = sizeof(float4) * 24 * (size_t)ctx->g.Vh;
    const size_t window = links < (size_t)max_window ? links : (size_t)max_window;
    const size_t carve = window < (size_t)max_persist ? window : (size_t)max_persist;
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) == cudaSuccess && cur < carve) {
        cudaError_t e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, carve);
        if (e != cudaSuccess) return e;
    }
    cudaKernelNodeAttrValue v;
    memset(&v, 0, sizeof(v));
    v.accessPolicyWindow.base_ptr = (void*)ctx->U32;
    v.accessPolicyWindow.num_bytes = window;
    v.accessPolicyWindow.hitRatio = (float)((double)carve / (double)window);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(graph, nullptr, &n);
    if (e != cudaSuccess || n == 0) return e;
    std::vector<cudaGraphNode_t> nodes(n);
    if ((e = cudaGraphGetNodes(graph, nodes.data(), &n)) != cudaSuccess) return e;
    for (size_t i = 0; i < n; i++) {
        cudaGraphNodeType t;
        if ((e = cudaGraphNodeGetType(nodes[i], &t)) != cudaSuccess) return e;
        if (t != cudaGraphNodeTypeKernel) continue;
        if ((e = cudaGraphKernelNodeSetAttribute(nodes[i], cudaKernelNodeAttributeAccessPolicyWindow, &v)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

template <typename F>
int run_chunk(stag_ctx* ctx, const std::string& key, int nkernels, F fn, cudaStream_t s) {
    // STAG_GRAPHS=0 in the environment switches graphs off for the process
    static int env_graphs = -1;
    if (env_graphs < 0) env_graphs = env_int("STAG_GRAPHS", 1);
    ctx->nlaunch += nkernels;
    if (!env_graphs || !ctx->use_graphs) {
        fn(s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return stag_cuda_check(ctx, e, key.c_str());
        return STAG_OK;
    }
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        cudaStream_t cs;
        STAG_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        STAG_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        fn(cs);
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return stag_cuda_check(ctx, e, "graph capture");
        if ((e = persist_links(ctx, graph)) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return stag_cuda_check(ctx, e, "graph access policy");
        }
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return stag_cuda_check(ctx, e, "graph instantiate");
        it = ctx->graphs.emplace(key, exec).first;
    }
    STAG_CUDA(ctx, cudaGraphLaunch(it->second, s));
    return STAG_OK;
}

// waits for the stream and copies the state header to the host mirror
int read_ms_state(stag_ctx* ctx, cudaStream_t s) {
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->ms_host, ctx->ms, sizeof(MSState), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    return STAG_OK;
}
int read_cg_state(stag_ctx* ctx, cudaStream_t s) {
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->cg_host, ctx->cg, sizeof(CGState), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    return STAG_OK;
}

// FP64-accurate true residual |b - (M + shift) x|^2 into *dst; the operator is
// applied in native FP64 (prec F64) or float-float (prec F64FF); w, t FP64 scratch
int true_residual2(stag_ctx* ctx, int prec, double c, const double2* b, const double2* x, double2* w, double2* t,
                   double2* r_out, float2* r_low, double* dst, cudaStream_t s) {
    int st = mee_apply(ctx, prec, c, x, w, t, s);
    if (st) return st;
    long n = 3L * ctx->g.Vh;
    k_residual<float2><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n, b, w, r_out, r_low, ctx->partials, ctx->counter,
                                                             dst);
    STAG_LAUNCH_CHECK(ctx, "residual");
    return STAG_OK;
}

// Reliable updates of an FP32 shifted CG: the FP64 source and solutions, and
// the trigger (the recursive |r|^2 fell below delta2 times its largest value
// since the last update).
struct MSReliable {
    const double2* b;
    double2* X;
    double mass, delta2;
    int nupdates;
};

// Applies the shifted vectors' update that the last iteration left pending
// (deferred form of the iteration) and clears the flag on the device and in
// the host mirror.  In the other forms the vector kernel of the iteration has
// applied it already (the scalar update still raises the flag, which the next
// B3 clears), so nothing is pending.
template <typename R>
static int ms_flush_pending(stag_ctx* ctx, MSBufs& bf, cudaStream_t s) {
    typedef typename VT<R>::T V2;
    MSState* hs = ctx->ms_host;
    if (!hs->pend || fused_iter() != 2) return STAG_OK;
    const long n3 = 3L * ctx->g.Vh;
    k_ms_shift_update<V2, R><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, n3, (const V2*)bf.r, (V2*)bf.pk, (V2*)bf.xk,
                                                                  ctx->ms);
    STAG_LAUNCH_CHECK(ctx, "ms shifted update");
    k_ms_clear_pend<<<1, 1, 0, s>>>(ctx->ms);
    STAG_LAUNCH_CHECK(ctx, "ms clear");
    hs->pend = 0;
    return STAG_OK;
}

// Flush the FP32 increments into the FP64 solutions, replace the base
// residual by its FP64-accurate value, and hand the new |r|^2 to the device
// state (the host mirror was read after the last chunk and nothing has run
// on the device since).
static int ms_reliable_update(stag_ctx* ctx, MSBufs& bf, MSReliable* ru, cudaStream_t s) {
    MSState* hs = ctx->ms_host;
    const long n3 = 3L * ctx->g.Vh;
    const size_t vb64 = sizeof(double2) * n3;
    double2* w64 = (double2*)ws_get(ctx, WS_W64, vb64);
    double2* t64 = (double2*)ws_get(ctx, WS_T64, vb64);
    if (!w64 || !t64) return stag_fail(ctx, STAG_ERR_OOM, "reliable-update workspace");
    int st = ms_flush_pending<float>(ctx, bf, s);
    if (st) return st;
    const int nb = ctx->num_sms * 4;
    k_ms_flush<<<nb, BLAS_TPB, 0, s>>>(n3, n3, hs->n, (float2*)bf.xk, ru->X);
    STAG_LAUNCH_CHECK(ctx, "ms flush");
    const int base = hs->base;
    st = mee_apply(ctx, STAG_PREC_F64FF, ru->mass * ru->mass + hs->shifts[base], ru->X + base * n3, w64, t64, s);
    if (st) return st;
    k_ms_replace<<<nb, BLAS_TPB, 0, s>>>(n3, n3, ru->b, w64, (float2*)bf.r, (float2*)bf.p, (float2*)bf.pk, ctx->ms,
                                        ctx->partials, ctx->counter, ctx->dscal + 2);
    STAG_LAUNCH_CHECK(ctx, "ms residual replacement");
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal + 2, ctx->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    if (!isfinite(ctx->hscal[2])) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite residual in multi-shift CG");
    hs->rr = ctx->hscal[2];
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->ms, hs, sizeof(MSState), cudaMemcpyHostToDevice, s));
    ru->nupdates++;
    return STAG_OK;
}

// Shifted CG with vectors of type R and links LP.  b: FP64 source.  On
// return the FP64 solutions are in xout (n contiguous vectors).
static int pipeline_on() {
    static int v = -1;
    if (v < 0) v = env_int("STAG_PIPELINE", 1);
    return v;
}
static int early_refine_on() { return env_int("STAG_EARLY_REFINE", 0); }

// Early refinement (STAG_EARLY_REFINE=1, mixed modes; off by default): a
// shift that the FP32 shifted CG has converged is refined at once on the
// context's second stream, while the shifted CG goes on for the lighter
// shifts.  At each poll of the shifted CG the hook takes the refinement's
// finished chunk (without waiting for one still running), hands over the
// newly converged shifts (x_k is final once the shift is inactive after a
// whole chunk) and launches the refinement's next chunk.  Measured on the
// 15-shift solve at 32^3x8 it gains nothing (0.1465 s against 0.146-0.149 s):
// the two streams' kernels do not fill idle capacity but slow each other
// (the shifted CG's iteration from 29 to ~42 us, the refinement's chunk of
// one or two right-hand sides to ~80 us per iteration).
struct EarlyRef {
    stag_ctx* ctx = nullptr;
    Refiner rf;
    RefSlots S;
    int n = 0;
    double tol = 0.0;
    const float2* xk32 = nullptr;  // the FP32 shifted CG's x_k (stride 3 Vh)
    int handed[STAG_MAXSHIFT] = {0};
    double rr[STAG_MAXSHIFT] = {0};
    int its[STAG_MAXSHIFT] = {0};
    int nresid = 0;  // true residuals computed at hand-over
    // copies the listed shifts' x_k to FP64 (after `ev` on the main stream),
    // computes their true residuals and lets those above tol join the refinement
    int hand_off(const int* ks, int nk, cudaEvent_t ev) {
        const long n3 = 3L * ctx->g.Vh;
        cudaStream_t s2 = ctx->s2;
        STAG_CUDA(ctx, cudaStreamWaitEvent(s2, ev, 0));
        int st;
        for (int i = 0; i < nk; i++)
            if ((st = blas_copy_f2d(ctx, xk32 + ks[i] * n3, S.x[ks[i]], ctx->g.Vh, s2))) return st;
        if ((st = batched_true_residuals(ctx, S, ks, nk, rf.R, rr, s2))) return st;
        nresid += nk;
        int sel[STAG_MAXSHIFT], ns = 0;
        for (int i = 0; i < nk; i++) {
            handed[ks[i]] = 1;
            if (S.bb[ks[i]] > 0.0 && rr[ks[i]] > tol * tol * S.bb[ks[i]]) sel[ns++] = ks[i];
        }
        return ns > 0 ? rf.add(sel, ns) : STAG_OK;
    }
    int trace = env_int("STAG_TRACE_EARLY", 0);
    double t0 = -1.0;
    double now() {
        const double t = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
        if (t0 < 0) t0 = t;
        return (t - t0) * 1e3;
    }
    int on_poll(const MSState* q) {
        int st;
        if (trace)
            fprintf(stderr, "[early] %.3f ms: ms iter %d n_active %d | refine flying %d ready %d n_act %d remaining %d\n",
                    now(), q->iter, q->n_active, (int)rf.flying, (int)rf.ready(), ctx->bcg_host->n_act, rf.remaining);
        if (rf.flying) {
            if (!rf.ready()) return STAG_OK;
            if ((st = rf.poll())) return st;
        }
        if (q->iter > 0) {
            for (int k = 0; k < n; k++) S.bb[k] = q->bb;
            int ks[STAG_MAXSHIFT], nk = 0;
            for (int k = 0; k < n; k++)
                if (!handed[k] && !q->active[k]) ks[nk++] = k;
            if (nk > 0 && (st = hand_off(ks, nk, ctx->ev_poll))) return st;
            if (trace && nk > 0) fprintf(stderr, "[early] %.3f ms: handed over %d shifts\n", now(), nk);
        }
        return rf.launch();
    }
};

// Runs chunks of STAG_CHUNK (32) iterations of the shifted CG until the device state stops;
// with `ru` (FP32 vectors only), a reliable update at every poll that finds
// the residual reduced by the trigger factor.
template <typename R, int LP>
static int ms_run(stag_ctx* ctx, Links U, MSBufs& bf, int maxit, cudaStream_t s, MSReliable* ru = nullptr,
                  EarlyRef* er = nullptr) {
    MSState* hs = ctx->ms_host;
    const int chunk = env_int("STAG_CHUNK", 32);
    char key[64];
    snprintf(key, sizeof key, "ms_%d_%d_%d_%d_%d_%d_%d_%p", (int)sizeof(R), LP, chunk, fused_iter(), hop_tpb(ctx, LP),
             env_int("STAG_CD_BPS", 0), env_int("STAG_CD_GROUP", 1), bf.xk);
    int guard = 0, st;
    double rr_max = -1.0;
    auto launch = [&]() {
        return run_chunk(ctx, key, (fused_iter() ? 3 : 4) * chunk, [&](cudaStream_t cs) {
            for (int i = 0; i < chunk; i++) launch_ms_iter<R, LP>(ctx, U, bf, cs);
        }, s);
    };
    // Pipelined polling (STAG_PIPELINE, default on): the state after chunk i
    // is copied to the host and chunk i+1 is launched before the host looks
    // at it, so the GPU does not wait for the host's decision.  A chunk
    // launched after the solve has stopped does nothing (its kernels see the
    // stop flags).  A reliable update waits for the stream and re-reads.
    const int pipeline = pipeline_on();
    if ((st = launch())) return st;
    for (;;) {
        const MSState* q = hs;
        if (pipeline) {
            STAG_CUDA(ctx, cudaMemcpyAsync(ctx->ms_poll, ctx->ms, sizeof(MSState), cudaMemcpyDeviceToHost, s));
            STAG_CUDA(ctx, cudaEventRecord(ctx->ev_poll, s));
            if ((st = launch())) return st;
            STAG_CUDA(ctx, cudaEventSynchronize(ctx->ev_poll));
            q = ctx->ms_poll;
        } else if ((st = read_ms_state(ctx, s))) {
            return st;
        }
        if (er && pipeline && !q->nonfinite && (st = er->on_poll(q))) return st;
        if (q->nonfinite || !q->live || q->stop_next) break;
        if (++guard > maxit / chunk + 4) break;  // cannot happen: the device caps iterations
        bool relaunch = !pipeline;
        if (ru) {
            if (rr_max < 0.0) rr_max = q->bb;
            if (q->rr > rr_max) rr_max = q->rr;
            if (q->rr < ru->delta2 * rr_max) {
                if (pipeline && (st = read_ms_state(ctx, s))) return st;
                if (!hs->live || hs->stop_next) break;
                if ((st = ms_reliable_update(ctx, bf, ru, s))) return st;
                rr_max = hs->rr;
                relaunch = true;
            }
        }
        if (relaunch && (st = launch())) return st;
    }
    if ((st = read_ms_state(ctx, s))) return st;  // the final state, after every launched chunk
    if ((st = ms_flush_pending<R>(ctx, bf, s))) return st;
    if (hs->nonfinite) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite residual in multi-shift CG");
    return STAG_OK;
}

template <typename R, int LP>
static MSBufs ms_bufs(stag_ctx* ctx, double2* xout) {
    typedef typename VT<R>::T V2;
    const size_t vb = sizeof(V2) * 3L * ctx->g.Vh;
    const bool f64 = (sizeof(R) == 8);
    MSBufs bf;
    bf.r = ws_get(ctx, f64 ? WS_R64 : WS_R32, vb);
    bf.p = ws_get(ctx, f64 ? WS_P64 : WS_P32, vb);
    bf.w = ws_get(ctx, f64 ? WS_W64 : WS_W32, vb);
    bf.t = ws_get(ctx, f64 ? WS_T64 : WS_T32, vb);
    bf.pk = ws_get(ctx, f64 ? WS_PK64 : WS_PK32, vb * STAG_MAXSHIFT);
    bf.xk = ws_get(ctx, f64 ? WS_XK64 : WS_XK32, vb * STAG_MAXSHIFT);
    if (f64) bf.xk = xout;
    return bf;
}

// FP64 modes: the recursion stops shift k when its recursive residual meets
// tol; if its true residual (checked afterwards) is still above tol, the
// same Krylov recursion is resumed for those shifts alone with a tolerance
// ten times tighter (the state, r, p, p_k and x_k are still on the device).
template <typename R, int LP>
static int ms_continue(stag_ctx* ctx, double2* xout, const int* ks, int nk, int maxit, stag_solve_info* info,
                       cudaStream_t s) {
    MSState* hs = ctx->ms_host;  // the state read after the last chunk
    MSBufs bf = ms_bufs<R, LP>(ctx, xout);
    const int it0 = hs->iter;
    int before[STAG_MAXSHIFT];
    for (int k = 0; k < hs->n; k++) before[k] = hs->iters_shift[k];
    hs->tol2bb *= 0.01;
    for (int i = 0; i < nk; i++) hs->active[ks[i]] = 1;
    hs->n_active = nk;
    hs->live = 1;
    hs->stop_next = 0;
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->ms, hs, sizeof(MSState), cudaMemcpyHostToDevice, s));
    const int st = ms_run<R, LP>(ctx, make_links(ctx, LP), bf, maxit, s);
    if (st) return st;
    info->iters += hs->iter - it0;
    info->matvecs += hs->iter - it0;
    for (int k = 0; k < hs->n; k++) info->iters_shift[k] += hs->iters_shift[k] - before[k];
    return STAG_OK;
}

// FP32 shifted CG with reliable updates of the base residual (STAG_MS_RELIABLE=1;
// trigger factor delta from STAG_RELIABLE_DELTA, 0.03).  Off by default: on the
// 32^3x8 workload the base system then follows its true residual to 1e-10
// (3498 iterations, as in FP64), but the other shifts keep the FP32 floor of
// their recursion (their residuals are never recomputed) and still need most
// of their refinement; the solve takes the same time either way.
static int ms_reliable_on() {
    static int v = -1;
    if (v < 0) v = env_int("STAG_MS_RELIABLE", 0);
    return v;
}

// Target of the FP32 shifted CG in the mixed modes (STAG_MS_TOL32): without
// reliable updates its true residual stalls near 1e-6 (FP32 rounding times the
// condition number); with them the base system follows the true residual down.
static double ms_tol32(double tol, int lp = LP32) {
    return fmax(tol, env_dbl("STAG_MS_TOL32", (ms_reliable_on() && lp != LP16) ? 1e-9 : 1e-6));
}

template <typename R, int LP>
int ms_core(stag_ctx* ctx, double mass, int n, const double* shifts, const double2* b, double2* xout,
            double tol, int maxit, stag_solve_info* info, cudaStream_t s, EarlyRef* er = nullptr) {
    typedef typename VT<R>::T V2;
    const Geom& g = ctx->g;
    const long n3 = 3L * g.Vh;
    const bool f64 = (sizeof(R) == 8);
    // BF16 links: the operator's ~4e-3 error times the condition number of
    // the light shifts exceeds one, so replaced residuals would not fall;
    // that mode keeps the plain FP32 recursion and leaves the rest to the
    // refinement
    const bool reliable = !f64 && LP != LP16 && ms_reliable_on();
    MSBufs bf = ms_bufs<R, LP>(ctx, xout);  // FP64: x_k accumulate straight into the output
    if (!bf.r || !bf.p || !bf.w || !bf.t || !bf.pk || !bf.xk) return stag_fail(ctx, STAG_ERR_OOM, "solver workspace");
    Links U = make_links(ctx, LP);

    // scalar state
    MSState* hs = ctx->ms_host;
    memset(hs, 0, sizeof(MSState));
    hs->n = n;
    hs->maxit = maxit;
    // FP32 recursion: the batched refinement that follows restarts every shift
    // still above tolerance, so the recursion may stop once at most `keep`
    // (the lightest) shifts remain unconverged
    hs->keep = (f64 || reliable) ? 0 : std::min(std::max(ms_keep(), 0), n - 1);
    for (int k = 0; k < n; k++) hs->shifts[k] = shifts[k];
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->ms, hs, sizeof(MSState), cudaMemcpyHostToDevice, s));
    int st = blas_dot_re(ctx, STAG_PREC_F64, b, b, &ctx->ms->bb, s);
    if (st) return st;
    k_ms_init_scalars<<<1, 1, 0, s>>>(ctx->ms, tol * tol, mass * mass);
    k_ms_init_vec<V2><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, n3, n, b, (V2*)bf.r, (V2*)bf.p, (V2*)bf.pk,
                                                           (V2*)bf.xk);
    ctx->nlaunch++;
    STAG_LAUNCH_CHECK(ctx, "ms init");

    MSReliable ru;
    ru.b = b;
    ru.X = xout;
    ru.mass = mass;
    const double delta = env_dbl("STAG_RELIABLE_DELTA", 0.03);
    ru.delta2 = delta * delta;
    ru.nupdates = 0;
    if (reliable) STAG_CUDA(ctx, cudaMemsetAsync(xout, 0, sizeof(double2) * n3 * n, s));
    if (er) er->xk32 = (const float2*)bf.xk;
    if ((st = ms_run<R, LP>(ctx, U, bf, maxit, s, reliable ? &ru : nullptr, er))) return st;
    if (info) {
        info->iters += hs->iter;
        info->matvecs += hs->iter + ru.nupdates;
        info->reliable_updates += ru.nupdates;
        for (int k = 0; k < n; k++) info->iters_shift[k] += hs->iters_shift[k];
    }
    if (reliable) {  // the increments since the last update
        k_ms_flush<<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, n3, n, (float2*)bf.xk, xout);
        STAG_LAUNCH_CHECK(ctx, "ms flush");
    } else if (!f64 && !er) {  // (the early refinement copies each shift as it takes it over)
        if ((st = blas_copy_f2d(ctx, (const float2*)bf.xk, xout, (long)g.Vh * n, s))) return st;
    }
    return STAG_OK;
}

// The mixed solve with early refinement: the FP32 shifted CG on `s`, the
// batched refinement of each shift from the moment the shifted CG has
// converged it on the second stream, then the remaining (lightest) shifts.
// Fills info like finish_batched; *status is STAG_OK or STAG_ERR_NOCONV.
template <int LP>
static int mixed_early(stag_ctx* ctx, double mass, int n, const double* shifts, const double2* src, double2* X,
                       double tol, int maxit, stag_solve_info* info, cudaStream_t s, int* status) {
    const long n3 = 3L * ctx->g.Vh;
    EarlyRef er;
    er.ctx = ctx;
    er.n = n;
    er.tol = tol;
    for (int k = 0; k < n; k++) {
        er.S.b[k] = src;
        er.S.x[k] = X + k * n3;
        er.S.c[k] = mass * mass + shifts[k];
        er.S.bb[k] = 0.0;
    }
    // every buffer the refinement touches exists before the shifted CG starts
    if (!ws_get(ctx, WS_W64, sizeof(double2) * n3) || !ws_get(ctx, WS_T64, sizeof(double2) * n3))
        return stag_fail(ctx, STAG_ERR_OOM, "residual workspace");
    // the refinement uses FP32 links in every mixed mode (see finish_batched)
    int st = er.rf.begin(ctx, LP32, &er.S, tol, maxit, er.rr, er.its, ctx->s2);
    if (st) return st;
    const double tol32 = (LP == LP16) ? ms_tol32(tol, LP16) : ms_tol32(tol);
    st = ms_core<float, LP>(ctx, mass, n, shifts, src, X, tol32, maxit, info, s, &er);
    if (!st && er.rf.flying) st = er.rf.poll();
    if (!st) {  // the rest, after the shifted CG's last chunk
        const double bb = ctx->ms_host->bb;
        for (int k = 0; k < n; k++) er.S.bb[k] = bb;
        int ks[STAG_MAXSHIFT], nk = 0;
        for (int k = 0; k < n; k++)
            if (!er.handed[k]) ks[nk++] = k;
        STAG_CUDA(ctx, cudaEventRecord(ctx->ev_poll, s));
        if (nk > 0) st = er.hand_off(ks, nk, ctx->ev_poll);
    }
    if (er.trace) fprintf(stderr, "[early] %.3f ms: shifted CG done, %d slots still refining\n", er.now(), er.rf.remaining);
    if (!st) st = er.rf.finish();
    if (er.trace) fprintf(stderr, "[early] %.3f ms: refinement done\n", er.now());
    if (st) {
        cudaStreamSynchronize(ctx->s2);
        return st;
    }
    // the caller's stream sees the refined solutions
    STAG_CUDA(ctx, cudaEventRecord(ctx->ev_ref, ctx->s2));
    STAG_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_ref, 0));
    const double bb = er.S.bb[0];
    info->reliable_updates += er.rf.nreliable;
    info->matvecs += er.rf.nmatvec + er.nresid;
    *status = STAG_OK;
    for (int k = 0; k < n; k++) {
        info->refine_iters[k] = er.its[k];
        info->true_resid[k] = (bb > 0.0) ? sqrt(er.rr[k] / bb) : 0.0;
        if (!isfinite(info->true_resid[k])) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite solution");
        if (er.rr[k] > tol * tol * bb * 1.0000001) *status = STAG_ERR_NOCONV;
    }
    return STAG_OK;
}

// Mixed-precision CG with FP64 reliable updates for (M + shift) x = b,
// starting from the FP64 guess x (updated in place).  Returns the FP64 true
// residual^2 in *rr_true.
template <int LP>
int refine_shift(stag_ctx* ctx, double mass, double shift, const double2* b, double bb, double2* x, double tol,
                 int maxit, double* rr_true, int* iters, int* reliable, int* matvecs, cudaStream_t s) {
    const Geom& g = ctx->g;
    const long n3 = 3L * g.Vh;
    const size_t vb32 = sizeof(float2) * n3, vb64 = sizeof(double2) * n3;
    float2* r32 = (float2*)ws_get(ctx, WS_R32, vb32);
    float2* p32 = (float2*)ws_get(ctx, WS_P32, vb32);
    float2* w32 = (float2*)ws_get(ctx, WS_W32, vb32);
    float2* t32 = (float2*)ws_get(ctx, WS_T32, vb32);
    float2* x32 = (float2*)ws_get(ctx, WS_XLO, vb32);
    double2* w64 = (double2*)ws_get(ctx, WS_W64, vb64);
    double2* t64 = (double2*)ws_get(ctx, WS_T64, vb64);
    if (!r32 || !p32 || !w32 || !t32 || !x32 || !w64 || !t64) return stag_fail(ctx, STAG_ERR_OOM, "refine workspace");
    Links U = make_links(ctx, LP);
    const double c = mass * mass + shift;
    const double delta = env_dbl("STAG_RELIABLE_DELTA", 0.03);
    const int chunk = env_int("STAG_CHUNK", 32);
    int st;

    double* dres = ctx->dscal + 0;
    if ((st = true_residual2(ctx, STAG_PREC_F64FF, c, b, x, w64, t64, nullptr, r32, dres, s))) return st;
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal, dres, sizeof(double), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    double rr = ctx->hscal[0];
    *matvecs += 1;
    const double tol2bb = tol * tol * bb;
    if (rr <= tol2bb) {
        *rr_true = rr;
        return STAG_OK;
    }
    STAG_CUDA(ctx, cudaMemsetAsync(x32, 0, vb32, s));
    k_cg_restart_p<float2><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, r32, p32, 0.0, 1);
    STAG_LAUNCH_CHECK(ctx, "cg start");
    CGState* hs = ctx->cg_host;
    memset(hs, 0, sizeof(CGState));
    hs->rr = rr;
    hs->rr_max = rr;
    hs->bb = bb;
    hs->tol2bb = tol2bb;
    hs->delta2 = delta * delta;
    hs->c0 = c;
    hs->maxit = maxit;
    hs->live = 1;
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->cg, hs, sizeof(CGState), cudaMemcpyHostToDevice, s));
    char key[64];
    snprintf(key, sizeof key, "cg_%d_%d_%d", LP, chunk, hop_tpb(ctx, LP));
    int total_iter = 0;
    for (;;) {
        st = run_chunk(ctx, key, 4 * chunk, [&](cudaStream_t cs) {
            for (int i = 0; i < chunk; i++) launch_cg_iter<float, LP>(ctx, U, r32, p32, w32, t32, x32, cs);
        }, s);
        if (st) return st;
        if ((st = read_cg_state(ctx, s))) return st;
        if (hs->live) continue;
        total_iter = hs->iter;
        if (hs->nonfinite) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite residual in CG");
        // reliable update: x += x_lo in FP64, true residual in FP64
        k_accumulate<float2><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, x, x32);
        STAG_LAUNCH_CHECK(ctx, "accumulate");
        if ((st = true_residual2(ctx, STAG_PREC_F64FF, c, b, x, w64, t64, nullptr, r32, dres, s))) return st;
        STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal, dres, sizeof(double), cudaMemcpyDeviceToHost, s));
        STAG_CUDA(ctx, cudaStreamSynchronize(s));
        *matvecs += 1;
        *reliable += 1;
        const double rr_t = ctx->hscal[0];
        if (rr_t <= tol2bb || hs->iter >= maxit) {
            *rr_true = rr_t;
            break;
        }
        // continue the recursion on the true residual, keeping the search
        // direction: p = r_true + (|r_true|^2 / |r_prev|^2) p
        const double beta = rr_t / hs->rr_prev;
        k_cg_restart_p<float2><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, r32, p32, beta, 0);
        STAG_LAUNCH_CHECK(ctx, "cg restart");
        hs->rr = rr_t;
        hs->rr_max = rr_t;
        hs->live = 1;
        hs->stop_next = 0;
        hs->want_reliable = 0;
        STAG_CUDA(ctx, cudaMemcpyAsync(ctx->cg, hs, sizeof(CGState), cudaMemcpyHostToDevice, s));
    }
    *iters += total_iter;
    *matvecs += total_iter;
    return STAG_OK;
}

}  // namespace

int run_graph_chunk(stag_ctx* ctx, const char* key, int nkernels, void (*enqueue)(stag_ctx*, void*, cudaStream_t),
                    void* arg, cudaStream_t s) {
    return run_chunk(ctx, std::string(key), nkernels, [&](cudaStream_t cs) { enqueue(ctx, arg, cs); }, s);
}

// FP64-accurate residuals (float-float operator) of the FP32 multi-shift
// solutions X[k], then the batched refinement of the shifts above tol; fills
// info's residuals and refinement counts, returns STAG_OK or STAG_ERR_NOCONV.
static int finish_batched(stag_ctx* ctx, double mass, int n, const double* shifts, const double2* src, double2* X,
                          double tol, int maxit, stag_solve_info* info, cudaStream_t s) {
    const long n3 = 3L * ctx->g.Vh;
    float2* R = (float2*)ws_get(ctx, WS_BR, sizeof(float2) * n3 * STAG_MAXSHIFT);
    if (!R) return stag_fail(ctx, STAG_ERR_OOM, "refinement workspace");
    int st;
    if ((st = blas_dot_re(ctx, STAG_PREC_F64, src, src, ctx->dscal + 1, s))) return st;
    // |b|^2 to the host (the residuals below synchronise the stream)
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal + 1, ctx->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    RefSlots S;
    int all[STAG_MAXSHIFT];
    for (int k = 0; k < n; k++) {
        all[k] = k;
        S.b[k] = src;
        S.x[k] = X + k * n3;
        S.c[k] = mass * mass + shifts[k];
    }
    double rr[STAG_MAXSHIFT];
    if ((st = batched_true_residuals(ctx, S, all, n, R, rr, s))) return st;
    info->matvecs += n;
    const double bb = ctx->hscal[1];
    for (int k = 0; k < n; k++) S.bb[k] = bb;
    int ks[STAG_MAXSHIFT], nk = 0;
    for (int k = 0; k < n; k++)
        if (bb > 0.0 && rr[k] > tol * tol * bb) ks[nk++] = k;
    if (nk > 0) {
        int its[STAG_MAXSHIFT] = {0}, rel = 0, mv = 0;
        // the refinement always uses FP32 links: BF16's ~4e-3 operator error times
        // the condition number of the light shifts exceeds one, and an inner
        // iteration that far from the true operator does not converge
        st = refine_batched(ctx, LP32, S, ks, nk, R, tol, maxit, rr, its, &rel, &mv, s);
        if (st) return st;
        for (int i = 0; i < nk; i++) info->refine_iters[ks[i]] = its[ks[i]];
        info->reliable_updates += rel;
        info->matvecs += mv;
    }
    int status = STAG_OK;
    for (int k = 0; k < n; k++) {
        info->true_resid[k] = (bb > 0.0) ? sqrt(rr[k] / bb) : 0.0;
        if (!isfinite(info->true_resid[k])) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite solution");
        if (rr[k] > tol * tol * bb * 1.0000001) status = STAG_ERR_NOCONV;
    }
    return status;
}

// STAG_SOLVE_LEARNED: the lightest shift by the network-preconditioned flexible
// CG, the others by the FP32 multi-shift (based at the second lightest shift)
// and batched refinement.  Falls back to the MIXED solver over all shifts when
// the flexible CG misses tol within its cap.  X[k] receives shift k.
static int learned_solve(stag_ctx* ctx, double mass, int n, const double* shifts, const double2* src, double2* X,
                         double tol, int maxit, stag_solve_info* info, cudaStream_t s) {
    if (!ctx->net) return stag_fail(ctx, STAG_ERR_STATE, "STAG_SOLVE_LEARNED needs a network (stag_ctx_set_net)");
    const long n3 = 3L * ctx->g.Vh;
    const size_t vb64 = sizeof(double2) * n3;
    int kmin = 0;
    for (int k = 1; k < n; k++)
        if (shifts[k] < shifts[kmin]) kmin = k;
    double2* XL = (double2*)ws_get(ctx, WS_LX, vb64);
    if (!XL) return stag_fail(ctx, STAG_ERR_OOM, "learned-mode workspace");
    int fit = 0;
    double ftr = 0.0;
    const int cap = env_int("STAG_FCG_MAXIT", 2000);
    int st = fcg_solve(ctx, ctx->net, mass, shifts[kmin], src, XL, tol, cap < maxit ? cap : maxit, &fit, &ftr, s);
    info->matvecs += fit + 1;
    if (st == STAG_ERR_NOCONV) {  // fallback: the plain mixed solver over all shifts
        stag_solve_info fb;
        memset(&fb, 0, sizeof(fb));
        if ((st = ms_core<float, LP32>(ctx, mass, n, shifts, src, X, ms_tol32(tol), maxit,
                                       &fb, s)))
            return st;
        st = finish_batched(ctx, mass, n, shifts, src, X, tol, maxit, &fb, s);
        fb.matvecs += info->matvecs;
        fb.refine_iters[kmin] += fit;
        *info = fb;
        return st;
    }
    if (st) return st;
    // the other shifts, compacted into X[0 .. n-2], then rotated into place
    double sh2[STAG_MAXSHIFT];
    int m = 0;
    for (int k = 0; k < n; k++)
        if (k != kmin) sh2[m++] = shifts[k];
    stag_solve_info i2;
    memset(&i2, 0, sizeof(i2));
    if (m > 0) {
        if ((st = ms_core<float, LP32>(ctx, mass, m, sh2, src, X, ms_tol32(tol), maxit,
                                       &i2, s)))
            return st;
        const int st2 = finish_batched(ctx, mass, m, sh2, src, X, tol, maxit, &i2, s);
        if (st2 && st2 != STAG_ERR_NOCONV) return st2;
        st = st2;
    }
    for (int k = n - 1; k > kmin; k--)
        STAG_CUDA(ctx, cudaMemcpyAsync(X + k * n3, X + (k - 1) * n3, vb64, cudaMemcpyDeviceToDevice, s));
    STAG_CUDA(ctx, cudaMemcpyAsync(X + kmin * n3, XL, vb64, cudaMemcpyDeviceToDevice, s));
    info->iters = i2.iters;
    info->reliable_updates = i2.reliable_updates;
    info->matvecs += i2.matvecs;
    for (int k = 0, j = 0; k < n; k++) {
        if (k == kmin) {
            info->iters_shift[k] = fit;
            info->true_resid[k] = ftr;
            continue;
        }
        info->iters_shift[k] = i2.iters_shift[j];
        info->refine_iters[k] = i2.refine_iters[j];
        info->true_resid[k] = i2.true_resid[j];
        j++;
    }
    return st;
}

int multishift_solve(stag_ctx* ctx, double mass, int n, const double* shifts, const double2* src,
                     double2* const* sols, double tol, int maxit, int mode, stag_solve_info* info, cudaStream_t s) {
    if (n < 1 || n > STAG_MAXSHIFT) return stag_fail(ctx, STAG_ERR_ARG, "number of shifts %d out of range", n);
    for (int k = 0; k < n; k++)
        if (!(shifts[k] >= 0.0)) return stag_fail(ctx, STAG_ERR_ARG, "shift %d negative or NaN", k);
    if (!(tol > 0.0) || maxit < 1) return stag_fail(ctx, STAG_ERR_ARG, "bad tolerance or iteration cap");
    const Geom& g = ctx->g;
    const long n3 = 3L * g.Vh;
    const size_t vb64 = sizeof(double2) * n3;
    stag_solve_info local;
    if (!info) info = &local;
    memset(info, 0, sizeof(*info));

    // contiguous FP64 solutions: the caller's buffers are filled at the end
    double2* X = (double2*)ws_get(ctx, WS_FX, vb64 * STAG_MAXSHIFT);
    if (!X) return stag_fail(ctx, STAG_ERR_OOM, "solution workspace");
    int st;
    if (!ctx->tuned && env_int("STAG_AUTOTUNE", 1)) {  // first solve on this context
        if ((st = autotune_hops(ctx, s))) return st;
    }
    const int check_prec = (mode == STAG_SOLVE_F64) ? STAG_PREC_F64 : STAG_PREC_F64FF;
    bool early = false;
    int early_status = STAG_OK;
    if (mode == STAG_SOLVE_F64) {
        st = ms_core<double, LP64>(ctx, mass, n, shifts, src, X, tol, maxit, info, s);
    } else if (mode == STAG_SOLVE_F64FF) {
        st = ms_core<double, LPFF>(ctx, mass, n, shifts, src, X, tol, maxit, info, s);
    } else if (mode == STAG_SOLVE_LEARNED) {
        st = STAG_OK;  // learned_solve below runs its own solvers
    } else if (mode == STAG_SOLVE_MIXED || mode == STAG_SOLVE_MIXED_BF16) {
        // STAG_MS_LINKS8=1: the FP32 shifted CG reads 8-real links (the
        // refinement keeps the 12-real FP32 links)
        static int r8 = -1;
        if (r8 < 0) r8 = env_int("STAG_MS_LINKS8", 0);
        early = env_int("STAG_BATCHED", 1) && early_refine_on() && fused_iter() == 1 && pipeline_on() &&
                !ms_reliable_on() && !(mode == STAG_SOLVE_MIXED && r8);
        if (early && mode == STAG_SOLVE_MIXED)
            st = mixed_early<LP32>(ctx, mass, n, shifts, src, X, tol, maxit, info, s, &early_status);
        else if (early)
            st = mixed_early<LP16>(ctx, mass, n, shifts, src, X, tol, maxit, info, s, &early_status);
        else if (mode == STAG_SOLVE_MIXED && r8) {
            if (!links_r8(ctx, s)) return STAG_ERR_OOM;
            st = ms_core<float, LP8>(ctx, mass, n, shifts, src, X, ms_tol32(tol), maxit, info, s);
        } else if (mode == STAG_SOLVE_MIXED)
            st = ms_core<float, LP32>(ctx, mass, n, shifts, src, X, ms_tol32(tol), maxit, info, s);
        else
            st = ms_core<float, LP16>(ctx, mass, n, shifts, src, X, ms_tol32(tol, LP16), maxit, info, s);
    } else {
        return stag_fail(ctx, STAG_ERR_ARG, "unknown solver mode %d", mode);
    }
    if (st) return st;

    const int batched = (mode == STAG_SOLVE_MIXED || mode == STAG_SOLVE_MIXED_BF16) && env_int("STAG_BATCHED", 1);
    if (batched || mode == STAG_SOLVE_LEARNED) {
        int status = (mode == STAG_SOLVE_LEARNED) ? learned_solve(ctx, mass, n, shifts, src, X, tol, maxit, info, s)
                     : early                      ? early_status
                                                  : finish_batched(ctx, mass, n, shifts, src, X, tol, maxit, info, s);
        if (status && status != STAG_ERR_NOCONV) return status;
        if (sols) {
            for (int k = 0; k < n; k++)
                if (sols[k] && sols[k] != X + k * n3)
                    STAG_CUDA(ctx, cudaMemcpyAsync(sols[k], X + k * n3, vb64, cudaMemcpyDeviceToDevice, s));
        }
        info->status = status;
        if (status) return stag_fail(ctx, status, "solver did not reach tolerance %.3g", tol);
        return STAG_OK;
    }

    // FP64 true residual of every shift; mixed mode refines the ones above tol
    double2* w64 = (double2*)ws_get(ctx, WS_W64, vb64);
    double2* t64 = (double2*)ws_get(ctx, WS_T64, vb64);
    if ((st = blas_dot_re(ctx, STAG_PREC_F64, src, src, ctx->dscal + 1, s))) return st;
    for (int k = 0; k < n; k++) {
        if ((st = true_residual2(ctx, check_prec, mass * mass + shifts[k], src, X + k * n3, w64, t64, nullptr, nullptr,
                                 ctx->dscal + 100 + k, s)))
            return st;
    }
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal, ctx->dscal, sizeof(double) * (100 + n), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    info->matvecs += n;
    const double bb = ctx->hscal[1];
    double rr[STAG_MAXSHIFT];
    for (int k = 0; k < n; k++) rr[k] = ctx->hscal[100 + k];
    for (int round = 0; round < 3 && (mode == STAG_SOLVE_F64 || mode == STAG_SOLVE_F64FF) && bb > 0.0; round++) {
        // shifts still updated by the last iteration can resume the recursion;
        // a shift frozen earlier cannot (its p_k and zeta_k are stale) and is
        // refined by the batched CG instead
        int ks[STAG_MAXSHIFT], nk = 0, kr[STAG_MAXSHIFT], nr = 0;
        for (int k = 0; k < n; k++)
            if (rr[k] > tol * tol * bb) {
                if (ctx->ms_host->iters_shift[k] == ctx->ms_host->iter)
                    ks[nk++] = k;
                else
                    kr[nr++] = k;
            }
        if (nr > 0) {
            float2* R = (float2*)ws_get(ctx, WS_BR, sizeof(float2) * n3 * STAG_MAXSHIFT);
            if (!R) return stag_fail(ctx, STAG_ERR_OOM, "refinement workspace");
            RefSlots S;
            for (int k = 0; k < n; k++) {
                S.b[k] = src;
                S.x[k] = X + k * n3;
                S.c[k] = mass * mass + shifts[k];
                S.bb[k] = bb;
            }
            double rr2[STAG_MAXSHIFT];
            if ((st = batched_true_residuals(ctx, S, kr, nr, R, rr2, s))) return st;
            int its[STAG_MAXSHIFT] = {0}, rel = 0, mv = 0;
            if ((st = refine_batched(ctx, LP32, S, kr, nr, R, tol, maxit, rr2, its, &rel, &mv, s))) return st;
            for (int i = 0; i < nr; i++) {
                rr[kr[i]] = rr2[kr[i]];
                info->refine_iters[kr[i]] += its[kr[i]];
            }
            info->reliable_updates += rel;
            info->matvecs += mv + nr;
        }
        if (nk == 0) break;
        st = (mode == STAG_SOLVE_F64) ? ms_continue<double, LP64>(ctx, X, ks, nk, maxit, info, s)
                                      : ms_continue<double, LPFF>(ctx, X, ks, nk, maxit, info, s);
        if (st) return st;
        for (int i = 0; i < nk; i++) {
            const int k = ks[i];
            if ((st = true_residual2(ctx, check_prec, mass * mass + shifts[k], src, X + k * n3, w64, t64, nullptr,
                                     nullptr, ctx->dscal + 100 + k, s)))
                return st;
        }
        STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal + 100, ctx->dscal + 100, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                       s));
        STAG_CUDA(ctx, cudaStreamSynchronize(s));
        info->matvecs += nk;
        for (int i = 0; i < nk; i++) rr[ks[i]] = ctx->hscal[100 + ks[i]];
    }
    int status = STAG_OK;
    for (int k = 0; k < n; k++) {
        if (bb == 0.0) {
            info->true_resid[k] = 0.0;
            continue;
        }
        if (mode != STAG_SOLVE_F64 && rr[k] > tol * tol * bb) {
            int it = 0, rel = 0, mv = 0;
            double rrt = rr[k];
            if (mode == STAG_SOLVE_MIXED)
                st = refine_shift<LP32>(ctx, mass, shifts[k], src, bb, X + k * n3, tol, maxit, &rrt, &it, &rel, &mv, s);
            else
                st = refine_shift<LP16>(ctx, mass, shifts[k], src, bb, X + k * n3, tol, maxit, &rrt, &it, &rel, &mv, s);
            if (st) return st;
            rr[k] = rrt;
            info->refine_iters[k] = it;
            info->reliable_updates += rel;
            info->matvecs += mv;
        }
        info->true_resid[k] = sqrt(rr[k] / bb);
        if (!isfinite(info->true_resid[k])) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite solution");
        if (rr[k] > tol * tol * bb * 1.0000001) status = STAG_ERR_NOCONV;
    }
    if (sols) {
        for (int k = 0; k < n; k++)
            if (sols[k] && sols[k] != X + k * n3)
                STAG_CUDA(ctx, cudaMemcpyAsync(sols[k], X + k * n3, vb64, cudaMemcpyDeviceToDevice, s));
    }
    info->status = status;
    if (status) return stag_fail(ctx, status, "solver did not reach tolerance %.3g", tol);
    return STAG_OK;
}

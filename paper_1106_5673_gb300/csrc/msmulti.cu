// msmulti.cu -- batched shifted CG: nsys independent systems
//   (M_ee + s_k) x_{r,k} = b_r,   r < nsys, k < n,
// on one gauge field, advanced together (the pseudofermions of an RHMC force
// evaluation with N_pf > 1, Sec. 2.1: "multiple pseudo-fermions").  The hop
// kernels are multi-RHS hops: each thread loads the links of its site once and
// applies them to up to NRM systems, so the links -- 384 of the 600 bytes of
// an FP32 hop per site -- are read once per group instead of once per system.
// Each system keeps its own recurrence (ms_common.cuh) and stops on its own;
// mixed precision refines every (system, shift) pair above tolerance with the
// batched refinement (refine.cu), 32 pairs at a time.
#include <math.h>
#include <stdlib.h>

#include "ms_common.cuh"

namespace {

const int BLAS_TPB = 256;
const int NRM = 4;

STAG_D bool last_block_xy(unsigned int* counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x * gridDim.y - 1);
    }
    __syncthreads();
    if (am_last && threadIdx.x == 0) *counter = 0;
    return am_last;
}

// the live systems of this block's group (blockIdx.y), compacted
STAG_D int group_systems(const MSState* st, int nsys, int js[NRM]) {
    int nj = 0;
    const int q0 = blockIdx.y * NRM;
#pragma unroll
    for (int q = 0; q < NRM; q++) {
        const int r = q0 + q;
        js[q] = 0;
        if (r < nsys && st[r].live) js[nj++] = r;
    }
    return nj;
}

template <typename R, int LP>
STAG_D void hops(const Geom& g, Links U, const typename VT<R>::T* in, size_t vstride, const int* js, int nj, int h,
                 int par, Vec3<R> acc[NRM]) {
    const Site s = site_of(g, h, par);
    if constexpr (LP == LPFF) {
#pragma unroll
        for (int q = 0; q < NRM; q++)
            if (q < nj) acc[q] = hop2_ff(g, (const float4*)U.u, U.lo, in + js[q] * vstride, h, par, s);
    } else {
        hop2_multiR<R, LP, NRM>(g, U.u, in, vstride, js, nj, h, par, s, acc);
    }
}

template <typename R, int LP>
__global__ void __launch_bounds__(256) k_mm_A(Geom g, Links U, const typename VT<R>::T* __restrict__ P,
                                              typename VT<R>::T* __restrict__ T, size_t vstride, const MSState* st,
                                              int nsys) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    int js[NRM];
    const int nj = group_systems(st, nsys, js);
    if (nj == 0) return;
    Vec3<R> acc[NRM];
    hops<R, LP>(g, U, P, vstride, js, nj, h, 1, acc);
#pragma unroll
    for (int q = 0; q < NRM; q++) {
        if (q < nj) {
#pragma unroll
            for (int a = 0; a < 3; a++) acc[q].c[a] = (R)0.5 * acc[q].c[a];
            st_vec(T + js[q] * vstride, h, acc[q]);
        }
    }
}

// w_r = c0 p_r - D_eo t_r and the sums <p,w>, <r,w>, <w,w>, |r|^2 per system;
// the last block runs every live system's scalar update
template <typename R, int LP>
__global__ void __launch_bounds__(256) k_mm_B3(Geom g, Links U, const typename VT<R>::T* __restrict__ T,
                                               const typename VT<R>::T* __restrict__ P,
                                               const typename VT<R>::T* __restrict__ Rv,
                                               typename VT<R>::T* __restrict__ W, size_t vstride, MSState* st,
                                               int nsys, double* partials, double* gpart, unsigned int* counter) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    int js[NRM];
    const int nj = group_systems(st, nsys, js);
    R flat[NRM * 4];
#pragma unroll
    for (int i = 0; i < NRM * 4; i++) flat[i] = 0;
    if (h < g.Vh && nj > 0) {
        Vec3<R> acc[NRM];
        hops<R, LP>(g, U, T, vstride, js, nj, h, 0, acc);
#pragma unroll
        for (int q = 0; q < NRM; q++) {
            if (q < nj) {
                const R c0 = (R)st[js[q]].c0;
                const Vec3<R> pv = load_vec(P + js[q] * vstride, h), rv = load_vec(Rv + js[q] * vstride, h);
                Vec3<R> wv;
                R a = 0, b = 0, c = 0, d = 0;
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    wv.c[i] = c0 * pv.c[i] - (R)0.5 * acc[q].c[i];
                    a += pv.c[i].re * wv.c[i].re + pv.c[i].im * wv.c[i].im;
                    b += rv.c[i].re * wv.c[i].re + rv.c[i].im * wv.c[i].im;
                    c += wv.c[i].re * wv.c[i].re + wv.c[i].im * wv.c[i].im;
                    d += rv.c[i].re * rv.c[i].re + rv.c[i].im * rv.c[i].im;
                }
                st_vec(W + js[q] * vstride, h, wv);
                flat[4 * q + 0] = a;
                flat[4 * q + 1] = b;
                flat[4 * q + 2] = c;
                flat[4 * q + 3] = d;
            }
        }
    }
    const double bsum = block_sum_nv<NRM * 4, R>(flat);
    const size_t nbx = gridDim.x;
    if (threadIdx.x < 4 * nj) {
        const int q = threadIdx.x >> 2, j = threadIdx.x & 3;
        partials[((size_t)js[q] * 4 + j) * nbx + blockIdx.x] = bsum;
    }
    __shared__ double s_sum[STAG_MAXRHS * 4];
    if (grid_reduce_series(partials, gpart, counter, nsys * 4, s_sum)) {
        for (int r = 0; r < nsys; r++)
            if (st[r].live) ms_scalar_update(&st[r], s_sum[4 * r], s_sum[4 * r + 1], s_sum[4 * r + 2], s_sum[4 * r + 3]);
    }
}

// per-system vector update; blockIdx.y = system
template <typename V2, typename R>
__global__ void k_mm_CD(long n, size_t vstride, size_t kstride, V2* __restrict__ Rv, const V2* __restrict__ W,
                        V2* __restrict__ P, V2* __restrict__ PK, V2* __restrict__ XK, MSState* st, int nsys,
                        unsigned int* counter) {
    const int r = blockIdx.y;
    if (r < nsys && st[r].live)
        ms_vector_update<V2, R>(n, n, blockIdx.x * (long)blockDim.x + threadIdx.x, (long)gridDim.x * blockDim.x,
                                Rv + r * vstride, W + r * vstride, P + r * vstride, PK + r * kstride, XK + r * kstride,
                                &st[r]);
    if (last_block_xy(counter)) {
        if (threadIdx.x == 0)
            for (int q = 0; q < nsys; q++)
                if (st[q].live && st[q].stop_next) st[q].live = 0;
    }
}

template <typename V2>
__global__ void k_mm_init(long n, int ns, const double2* __restrict__ b, V2* r, V2* p, V2* pk, V2* xk) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = b[i];
        V2 c, z;
        c.x = v.x;
        c.y = v.y;
        z.x = 0;
        z.y = 0;
        r[i] = c;
        p[i] = c;
        for (int k = 0; k < ns; k++) {
            pk[k * n + i] = c;
            xk[k * n + i] = z;
        }
    }
}

__global__ void k_mm_init_scalars(MSState* st, double tol2, double c_mass) {
    MSState* s = st + blockIdx.x;
    const double bb = s->bb;
    s->rr = bb;
    s->tol2bb = tol2 * bb;
    s->alpha_old = 1.0;
    s->beta_old = 0.0;
    s->iter = 0;
    s->nonfinite = !isfinite(bb);
    s->stop_next = 0;
    int base = 0;
    for (int k = 1; k < s->n; k++)
        if (s->shifts[k] < s->shifts[base]) base = k;
    s->base = base;
    s->c0 = c_mass + s->shifts[base];
    for (int k = 0; k < s->n; k++) {
        s->zeta[k] = s->zeta_old[k] = 1.0;
        s->active[k] = (bb > 0.0 && isfinite(bb)) ? 1 : 0;
        s->upd_x[k] = 0;
        s->iters_shift[k] = 0;
        s->ak[k] = s->bk[k] = 0.0;
    }
    s->n_active = s->active[0] ? s->n : 0;
    s->live = s->n_active > 0;
}

int env_i(const char* name, int dflt) {
    const char* v = getenv(name);
    return v ? atoi(v) : dflt;
}

struct MMIter {
    Links U;
    void *R, *P, *W, *T, *PK, *XK;
    int nsys, chunk, tpb, lp, f64;
};

template <typename R, int LP>
void enqueue_mm_t(stag_ctx* ctx, const MMIter& a, cudaStream_t cs) {
    typedef typename VT<R>::T V2;
    const Geom& g = ctx->g;
    const long n3 = 3L * g.Vh;
    const size_t vs = (size_t)n3, ks = (size_t)n3 * STAG_MAXSHIFT;
    const dim3 gh(nblocks(g.Vh, a.tpb), (a.nsys + NRM - 1) / NRM), gb(ctx->num_sms, a.nsys);
    for (int i = 0; i < a.chunk; i++) {
        k_mm_A<R, LP><<<gh, a.tpb, 0, cs>>>(g, a.U, (const V2*)a.P, (V2*)a.T, vs, ctx->msm, a.nsys);
        k_mm_B3<R, LP><<<gh, a.tpb, 0, cs>>>(g, a.U, (const V2*)a.T, (const V2*)a.P, (const V2*)a.R, (V2*)a.W, vs,
                                            ctx->msm, a.nsys, ctx->mm_partials, ctx->gpart, ctx->counter);
        k_mm_CD<V2, R><<<gb, BLAS_TPB, 0, cs>>>(n3, vs, ks, (V2*)a.R, (const V2*)a.W, (V2*)a.P, (V2*)a.PK,
                                               (V2*)a.XK, ctx->msm, a.nsys, ctx->counter);
    }
}

void enqueue_mm(stag_ctx* ctx, void* argp, cudaStream_t cs) {
    const MMIter& a = *(const MMIter*)argp;
    switch (a.lp) {
    case LP64: enqueue_mm_t<double, LP64>(ctx, a, cs); break;
    case LPFF: enqueue_mm_t<double, LPFF>(ctx, a, cs); break;
    case LP32: enqueue_mm_t<float, LP32>(ctx, a, cs); break;
    default: enqueue_mm_t<float, LP16>(ctx, a, cs); break;
    }
}

}  // namespace

int run_graph_chunk(stag_ctx* ctx, const char* key, int nkernels, void (*enqueue)(stag_ctx*, void*, cudaStream_t),
                    void* arg, cudaStream_t s);

// Solves (M_ee + shifts[k]) x_{r,k} = srcs[r] for r < nsys, k < n; FP64
// solutions land in X + (r * STAG_MAXSHIFT + k) * 3 Vh.
int multishift_solve_multi(stag_ctx* ctx, double mass, int nsys, int n, const double* shifts,
                           const double2* const* srcs, double2* X, double tol, int maxit, int mode,
                           stag_solve_info* infos, cudaStream_t s) {
    if (nsys < 1 || nsys > STAG_MAXRHS || n < 1 || n > STAG_MAXSHIFT)
        return stag_fail(ctx, STAG_ERR_ARG, "bad number of systems or shifts");
    for (int k = 0; k < n; k++)
        if (!(shifts[k] >= 0.0)) return stag_fail(ctx, STAG_ERR_ARG, "shift %d negative or NaN", k);
    if (!(tol > 0.0) || maxit < 1) return stag_fail(ctx, STAG_ERR_ARG, "bad tolerance or iteration cap");
    int st;
    if (!ctx->tuned && env_i("STAG_AUTOTUNE", 1)) {
        if ((st = autotune_hops(ctx, s))) return st;
    }
    const Geom& g = ctx->g;
    const long n3 = 3L * g.Vh;
    const int lp = (mode == STAG_SOLVE_F64) ? LP64 : (mode == STAG_SOLVE_F64FF) ? LPFF
                   : (mode == STAG_SOLVE_MIXED) ? LP32 : LP16;
    if (mode < 0 || mode > 3) return stag_fail(ctx, STAG_ERR_ARG, "unknown solver mode %d", mode);
    const int f64 = (lp == LP64 || lp == LPFF);
    const size_t vb = (f64 ? sizeof(double2) : sizeof(float2)) * n3;
    MMIter it;
    it.lp = lp;
    it.f64 = f64;
    it.nsys = nsys;
    it.U.u = (lp == LP64) ? (const void*)ctx->U64 : (lp == LP16) ? (const void*)ctx->U16 : (const void*)ctx->U32;
    it.U.lo = ctx->U32lo;
    it.R = ws_get(ctx, WS_MR, vb * STAG_MAXRHS);
    it.P = ws_get(ctx, WS_MP, vb * STAG_MAXRHS);
    it.W = ws_get(ctx, WS_MW, vb * STAG_MAXRHS);
    it.T = ws_get(ctx, WS_MT, vb * STAG_MAXRHS);
    it.PK = ws_get(ctx, WS_MPK, vb * STAG_MAXRHS * STAG_MAXSHIFT);
    it.XK = f64 ? (void*)X : ws_get(ctx, WS_MXK, vb * STAG_MAXRHS * STAG_MAXSHIFT);
    if (!it.R || !it.P || !it.W || !it.T || !it.PK || !it.XK) return stag_fail(ctx, STAG_ERR_OOM, "batched solver workspace");
    it.chunk = env_i("STAG_CHUNK", 32);
    it.tpb = hop_tpb(ctx, lp);

    // scalar states and vectors
    MSState* hs = ctx->msm_host;
    memset(hs, 0, sizeof(MSState) * STAG_MAXRHS);
    const double tol_run = f64 ? tol : fmax(tol, 1e-6);
    for (int r = 0; r < nsys; r++) {
        hs[r].n = n;
        hs[r].maxit = maxit;
        for (int k = 0; k < n; k++) hs[r].shifts[k] = shifts[k];
    }
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->msm, hs, sizeof(MSState) * STAG_MAXRHS, cudaMemcpyHostToDevice, s));
    for (int r = 0; r < nsys; r++) {
        if ((st = blas_dot_re(ctx, STAG_PREC_F64, srcs[r], srcs[r], &ctx->msm[r].bb, s))) return st;
        if (f64)
            k_mm_init<double2><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(
                n3, n, srcs[r], (double2*)it.R + r * n3, (double2*)it.P + r * n3,
                (double2*)it.PK + (size_t)r * STAG_MAXSHIFT * n3, (double2*)it.XK + (size_t)r * STAG_MAXSHIFT * n3);
        else
            k_mm_init<float2><<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(
                n3, n, srcs[r], (float2*)it.R + r * n3, (float2*)it.P + r * n3,
                (float2*)it.PK + (size_t)r * STAG_MAXSHIFT * n3, (float2*)it.XK + (size_t)r * STAG_MAXSHIFT * n3);
        STAG_LAUNCH_CHECK(ctx, "batched init");
    }
    k_mm_init_scalars<<<nsys, 1, 0, s>>>(ctx->msm, tol_run * tol_run, mass * mass);
    STAG_LAUNCH_CHECK(ctx, "batched init scalars");

    char key[80];
    snprintf(key, sizeof key, "mm_%d_%d_%d_%d_%p", lp, nsys, it.chunk, it.tpb, it.XK);
    int guard = 0;
    for (;;) {
        if ((st = run_graph_chunk(ctx, key, 3 * it.chunk, enqueue_mm, &it, s))) return st;
        STAG_CUDA(ctx, cudaMemcpyAsync(hs, ctx->msm, sizeof(MSState) * STAG_MAXRHS, cudaMemcpyDeviceToHost, s));
        STAG_CUDA(ctx, cudaStreamSynchronize(s));
        int live = 0;
        for (int r = 0; r < nsys; r++) {
            if (hs[r].nonfinite) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite residual in batched CG");
            live += hs[r].live;
        }
        if (!live || ++guard > maxit / it.chunk + 4) break;
    }
    for (int r = 0; r < nsys; r++) {
        stag_solve_info* in = infos ? &infos[r] : nullptr;
        if (in) {
            memset(in, 0, sizeof(*in));
            in->iters = hs[r].iter;
            in->matvecs = hs[r].iter;
            for (int k = 0; k < n; k++) in->iters_shift[k] = hs[r].iters_shift[k];
        }
    }
    if (!f64)
        for (int r = 0; r < nsys; r++)
            if ((st = blas_copy_f2d(ctx, (const float2*)it.XK + (size_t)r * STAG_MAXSHIFT * n3,
                                    X + (size_t)r * STAG_MAXSHIFT * n3, (long)g.Vh * n, s)))
                return st;

    // FP64-accurate check of every (system, shift); those above tolerance are
    // refined by the batched CG, up to 32 pairs per batch (in the FP64 modes
    // this only catches a recursion that stopped with its true residual just
    // above tol)
    float2* Rres = (float2*)ws_get(ctx, WS_BR, sizeof(float2) * n3 * STAG_MAXSHIFT);
    if (!Rres) return stag_fail(ctx, STAG_ERR_OOM, "refinement workspace");
    int status = STAG_OK;
    const int npair = nsys * n;
    for (int p0 = 0; p0 < npair; p0 += STAG_MAXSHIFT) {
        const int np = (npair - p0 < STAG_MAXSHIFT) ? npair - p0 : STAG_MAXSHIFT;
        RefSlots S;
        int all[STAG_MAXSHIFT];
        for (int j = 0; j < np; j++) {
            const int r = (p0 + j) / n, k = (p0 + j) % n;
            all[j] = j;
            S.b[j] = srcs[r];
            S.x[j] = X + ((size_t)r * STAG_MAXSHIFT + k) * n3;
            S.c[j] = mass * mass + shifts[k];
            S.bb[j] = hs[r].bb;
        }
        double rr[STAG_MAXSHIFT];
        if ((st = batched_true_residuals(ctx, S, all, np, Rres, rr, s))) return st;
        int ks[STAG_MAXSHIFT], nk = 0;
        for (int j = 0; j < np; j++)
            if (S.bb[j] > 0.0 && rr[j] > tol * tol * S.bb[j]) ks[nk++] = j;
        int its[STAG_MAXSHIFT] = {0}, rel = 0, mv = 0;
        if (nk > 0 && (st = refine_batched(ctx, LP32, S, ks, nk, Rres, tol, maxit, rr, its, &rel, &mv, s)))
            return st;
        for (int j = 0; j < np; j++) {
            const int r = (p0 + j) / n, k = (p0 + j) % n;
            const double tr = (S.bb[j] > 0.0) ? sqrt(rr[j] / S.bb[j]) : 0.0;
            if (!isfinite(tr)) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite solution");
            if (tr > tol * 1.00000005) status = STAG_ERR_NOCONV;
            if (infos) {
                infos[r].true_resid[k] = tr;
                infos[r].refine_iters[k] = its[j];
                infos[r].matvecs += 1 + its[j];
            }
        }
        if (infos) infos[(p0) / n].reliable_updates += rel;
    }
    if (infos)
        for (int r = 0; r < nsys; r++) infos[r].status = status;
    if (status) return stag_fail(ctx, status, "batched solver did not reach tolerance %.3g", tol);
    return STAG_OK;
}

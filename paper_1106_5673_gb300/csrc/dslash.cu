// dslash.cu -- the even/odd staggered operator of Eq. (4) and the even-site
// normal operator M_ee = m^2 - D_eo D_oe (Sec. 2.1), one thread per output
// site.  Memory-bound: per output site 8 links (12 reals) + 8 neighbour
// vectors + 1 output vector (600 B in FP32, 1200 B in FP64).
#include "hop.cuh"
#include "stag_internal.h"

static const int HOP_TPB = 128;

// out = c * self - 1/2 hop(in)   (c = 0, self = null: out = -1/2 hop; sign
// flipped by `scale`) -- generic epilogue: out = c * self + scale * hop2
template <typename R, int LP>
__global__ void __launch_bounds__(256) k_hop(Geom g, const void* __restrict__ U,
                                                 const typename VT<R>::T* __restrict__ in,
                                                 typename VT<R>::T* __restrict__ out, int par, R scale, R c,
                                                 const typename VT<R>::T* __restrict__ self) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const Site s = site_of(g, h, par);
    Vec3<R> acc = hop2<R, LP>(g, U, in, h, par, s);
    Vec3<R> r;
    if (self) {
        Vec3<R> v = load_vec(self, h);
#pragma unroll
        for (int a = 0; a < 3; a++) r.c[a] = c * v.c[a] + scale * acc.c[a];
    } else {
#pragma unroll
        for (int a = 0; a < 3; a++) r.c[a] = scale * acc.c[a];
    }
    st_vec(out, h, r);
}

template <typename R, int LP>
static void launch_hop(stag_ctx* ctx, const void* U, const void* in, void* out, int par, R scale, R c,
                       const void* self, cudaStream_t s, int tpb = 0) {
    if (tpb <= 0) tpb = hop_tpb(ctx, LP);
    k_hop<R, LP><<<nblocks(ctx->g.Vh, tpb), tpb, 0, s>>>(ctx->g, U, (const typename VT<R>::T*)in,
                                                         (typename VT<R>::T*)out, par, scale, c,
                                                         (const typename VT<R>::T*)self);
}

// FP64-accurate hop in float-float arithmetic (FP64 vectors in and out)
__global__ void __launch_bounds__(256) k_hop_ff(Geom g, const float4* __restrict__ Uhi,
                                                    const float4* __restrict__ Ulo, const double2* __restrict__ in,
                                                    double2* __restrict__ out, int par, double scale, double c,
                                                    const double2* __restrict__ self) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const Site s = site_of(g, h, par);
    Vec3<double> acc = hop2_ff(g, Uhi, Ulo, in, h, par, s);
    Vec3<double> r;
    if (self) {
        Vec3<double> v = load_vec(self, h);
#pragma unroll
        for (int a = 0; a < 3; a++) r.c[a] = c * v.c[a] + scale * acc.c[a];
    } else {
#pragma unroll
        for (int a = 0; a < 3; a++) r.c[a] = scale * acc.c[a];
    }
    st_vec(out, h, r);
}

static int hop_dispatch(stag_ctx* ctx, int prec, const void* in, void* out, int par, double scale, double c,
                        const void* self, cudaStream_t s) {
    switch (prec) {
    case STAG_PREC_F64FF: {
        const int tpb = hop_tpb(ctx, LPFF);
        k_hop_ff<<<nblocks(ctx->g.Vh, tpb), tpb, 0, s>>>(ctx->g, ctx->U32, ctx->U32lo, (const double2*)in,
                                                         (double2*)out, par, scale, c, (const double2*)self);
        break;
    }
    case STAG_PREC_F64: launch_hop<double, LP64>(ctx, ctx->U64, in, out, par, scale, c, self, s); break;
    case STAG_PREC_F32: launch_hop<float, LP32>(ctx, ctx->U32, in, out, par, (float)scale, (float)c, self, s); break;
    case STAG_PREC_BF16: launch_hop<float, LP16>(ctx, ctx->U16, in, out, par, (float)scale, (float)c, self, s); break;
    case STAG_PREC_F32R8: {
        const float4* U8 = links_r8(ctx, s);
        if (!U8) return STAG_ERR_OOM;
        launch_hop<float, LP8>(ctx, U8, in, out, par, (float)scale, (float)c, self, s);
        break;
    }
    default: return stag_fail(ctx, STAG_ERR_ARG, "unknown precision %d", prec);
    }
    STAG_LAUNCH_CHECK(ctx, "hop");
    return STAG_OK;
}

int dslash_apply(stag_ctx* ctx, int prec, const void* in, void* out, int out_par, cudaStream_t s) {
    return hop_dispatch(ctx, prec, in, out, out_par, 0.5, 0.0, nullptr, s);
}

// M_ee in = c in - D_eo (D_oe in), c = m^2 (+ shift)
int mee_apply(stag_ctx* ctx, int prec, double c, const void* in, void* out, void* tmp, cudaStream_t s) {
    int st = hop_dispatch(ctx, prec, in, tmp, 1, 0.5, 0.0, nullptr, s);
    if (st) return st;
    return hop_dispatch(ctx, prec, tmp, out, 0, -0.5, c, in, s);
}

// ---------------------------------------------------------------- autotuner
// Times the D_oe hop of each link precision for 64, 128 and 256 threads per
// block (CUDA events, after warm-up) and keeps the fastest per context: the
// lattice is fixed per context, so one measurement serves all later solves.
// Captured graphs are dropped, since they hold the old launch shapes.
int autotune_hops(stag_ctx* ctx, cudaStream_t s) {
    const long n3 = 3L * ctx->g.Vh;
    double2* a = (double2*)ws_get(ctx, WS_TUNE, sizeof(double2) * n3 * 2);
    if (!a) return stag_fail(ctx, STAG_ERR_OOM, "tuning buffers");
    double2* b = a + n3;
    STAG_CUDA(ctx, cudaMemsetAsync(a, 0, sizeof(double2) * n3 * 2, s));
    cudaEvent_t e0, e1;
    STAG_CUDA(ctx, cudaEventCreate(&e0));
    STAG_CUDA(ctx, cudaEventCreate(&e1));
    // each candidate: the best of 3 timings of 10 launches; 128 threads (the
    // default) is kept unless another size is more than 3 % faster, so that
    // timing noise between near-equal sizes does not flip the choice (the
    // solver kernels built on the hop, with their reductions, are more
    // sensitive to the block size than the bare hop timed here)
    const int cand[3] = {128, 64, 256};
    const float4* U8 = links_r8(ctx, s);
    if (!U8) return STAG_ERR_OOM;
    for (int lp = 0; lp < 5; lp++) {
        float best = 1e30f, t128 = 1e30f;
        int best_tpb = 128;
        for (int c = 0; c < 3; c++) {
            const int tpb = cand[c];
            auto launch = [&]() {
                switch (lp) {
                case LP64: launch_hop<double, LP64>(ctx, ctx->U64, a, b, 1, 0.5, 0.0, nullptr, s, tpb); break;
                case LP32: launch_hop<float, LP32>(ctx, ctx->U32, a, b, 1, 0.5f, 0.f, nullptr, s, tpb); break;
                case LP16: launch_hop<float, LP16>(ctx, ctx->U16, a, b, 1, 0.5f, 0.f, nullptr, s, tpb); break;
                case LP8: launch_hop<float, LP8>(ctx, U8, a, b, 1, 0.5f, 0.f, nullptr, s, tpb); break;
                default:
                    k_hop_ff<<<nblocks(ctx->g.Vh, tpb), tpb, 0, s>>>(ctx->g, ctx->U32, ctx->U32lo, a, b, 1, 0.5, 0.0,
                                                                     nullptr);
                }
            };
            for (int w = 0; w < 2; w++) launch();
            float ms = 1e30f;
            for (int rep = 0; rep < 3; rep++) {
                cudaEventRecord(e0, s);
                for (int r = 0; r < 10; r++) launch();
                cudaEventRecord(e1, s);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) return stag_cuda_check(ctx, e, "autotune");
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (t < ms) ms = t;
            }
            if (tpb == 128) t128 = ms;
            if (ms < best) {
                best = ms;
                best_tpb = tpb;
            }
        }
        ctx->tpb[lp] = (best < 0.97f * t128) ? best_tpb : 128;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    STAG_LAUNCH_CHECK(ctx, "autotune");
    ctx->tuned = 1;
    ctx_clear_graphs(ctx);
    return STAG_OK;
}

// ---------------------------------------------------------------- multi-RHS hop
// One thread per (site, RHS block of NR vectors): each link is loaded once and
// applied to NR right-hand sides (the force needs Y_k = D_oe X_k for every
// shift k).  FP64 vectors, FP64 links.
template <int NR>
__global__ void __launch_bounds__(256) k_hop_multi64(Geom g, const double2* __restrict__ U,
                                                         const double2* __restrict__ in, double2* __restrict__ out,
                                                         int nrhs, int k0, int par) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const Site s = site_of(g, h, par);
    const size_t stride = 3 * (size_t)g.Vh;
    Vec3<double> acc[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) acc[k] = vzero<double>();
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int fl = nb_lex(g, s, mu, +1), bl = nb_lex(g, s, mu, -1);
        int sf = eta(s, mu), sb = sf;
        if (mu == 3) {
            if (s.x[3] == g.L[3] - 1) sf = -sf;
            if (s.x[3] == 0) sb = -sb;
        }
        const Mat3<double> uf = load_link64(U, g, mu, par, h);
        const Mat3<double> ub = load_link64(U, g, mu, 1 - par, bl >> 1);
#pragma unroll
        for (int k = 0; k < NR; k++) {
            if (k0 + k < nrhs) {
                const double2* v = in + (k0 + k) * stride;
                axpy_sign(acc[k], sf, mv(uf, load_vec(v, fl >> 1)));
                axpy_sign(acc[k], -sb, mdv(ub, load_vec(v, bl >> 1)));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NR; k++) {
        if (k0 + k < nrhs) {
            Vec3<double> r;
#pragma unroll
            for (int a = 0; a < 3; a++) r.c[a] = 0.5 * acc[k].c[a];
            st_vec(out + (k0 + k) * stride, h, r);
        }
    }
}

int dslash_multi64(stag_ctx* ctx, const double2* in, double2* out, int nrhs, int out_par, cudaStream_t s) {
    const int NR = 4;
    for (int k0 = 0; k0 < nrhs; k0 += NR, ctx->nlaunch++)
        k_hop_multi64<NR><<<nblocks(ctx->g.Vh, HOP_TPB), HOP_TPB, 0, s>>>(ctx->g, ctx->U64, in, out, nrhs, k0,
                                                                         out_par);
    ctx->nlaunch--;  // counted per launch in the loop
    STAG_LAUNCH_CHECK(ctx, "hop_multi64");
    return STAG_OK;
}

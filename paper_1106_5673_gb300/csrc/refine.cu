// refine.cu -- batched mixed-precision refinement of the shifted solutions.
//
// After the FP32 shifted CG, every shift whose FP64-accurate true residual
// is above tolerance gets its own CG on (M_ee + s_k) e = r_k, all advanced
// together: each kernel covers every active right-hand side, and the two
// hops are multi-RHS hops that load each link once for a group of NR
// right-hand sides (the batching of the spec design).  The recursion
// runs in FP32 (or with BF16 links); reliable updates (x += x_lo in FP64,
// r = b - (M + s_k) x recomputed FP64-accurately with the float-float
// operator) happen at the host's polling points, every `chunk` iterations,
// for the right-hand sides whose residual fell by `delta` since their last
// update or that claim convergence.  A right-hand side leaves the batch only
// after a true-residual check below tolerance.
//
// Per iteration:  A  t_k = D_oe p_k          (multi-RHS hop)
//                 B  w_k = c_k p_k - D_eo t_k, alpha_k = rr_k / <p_k, w_k>
//                 C  r_k -= alpha_k w_k, x_k += alpha_k p_k, rr_k, beta_k;
//                    right-hand sides whose rr_k <= tol^2 |b|^2 are parked
//                 D  p_k = r_k + beta_k p_k
#include "hop.cuh"
#include "stag_internal.h"

#include <algorithm>
#include <math.h>
#include <stdlib.h>

namespace {

const int HOP_TPB = 128;
const int BLAS_TPB = 256;
// right-hand sides per thread in the multi-RHS hops: NRMAX while more than
// two right-hand sides are active, then 2 and 1 (fewer registers, more
// resident warps for the last, longest-running shifts)
const int NRMAX = 4;
const int NR = NRMAX;  // the unfused path
static int nr_for(int nact) { return nact <= 1 ? 1 : nact <= 2 ? 2 : NRMAX; }
// STAG_REFINE_NR: 0 always NRMAX, 1 nr_for (default), 2 one right-hand side
// per thread, 3 at most two
static int nr_policy(int nact, int pol) {
    return pol == 0 ? NRMAX : pol == 2 ? 1 : pol == 3 ? (nact <= 1 ? 1 : 2) : nr_for(nact);
}

STAG_D bool last_block_n(unsigned int* counter, unsigned int nblocks_total) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == nblocks_total - 1);
    }
    __syncthreads();
    if (am_last && threadIdx.x == 0) *counter = 0;
    return am_last;
}

template <int LP, int NR = NRMAX>
__global__ void __launch_bounds__(256, 4) k_b_A(Geom g, const void* __restrict__ U, const float2* __restrict__ P,
                                                 float2* __restrict__ T, size_t stride, BCGState* st) {
    // a stop requested by the previous iteration takes effect here, after that
    // iteration's vector update
    const int live = st->live, stop = st->stop_next;
    if (!live) return;
    if (stop) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) st->live = 0;
        return;
    }
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = blockIdx.y * NR, nact = st->n_act;
    if (h >= g.Vh || q0 >= nact) return;
    const int nj = min(NR, nact - q0);
    int js[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) js[q] = (q < nj) ? st->act[q0 + q] : 0;
    const Site s = site_of(g, h, 1);
    Vec3<float> acc[NR];
    hop2_multi<LP, NR>(g, U, P, stride, js, nj, h, 1, s, acc);
#pragma unroll
    for (int q = 0; q < NR; q++) {
        if (q < nj) {
#pragma unroll
            for (int a = 0; a < 3; a++) acc[q].c[a] = 0.5f * acc[q].c[a];
            st_vec(T + js[q] * stride, h, acc[q]);
        }
    }
}

template <int LP>
__global__ void __launch_bounds__(256) k_b_B(Geom g, const void* __restrict__ U, const float2* __restrict__ T,
                                                 const float2* __restrict__ P, float2* __restrict__ W, size_t stride,
                                                 BCGState* st, double* partials, unsigned int* counter) {
    if (!st->live) return;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = blockIdx.y * NR, nact = st->n_act;
    const int nj = max(0, min(NR, nact - q0));
    int js[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) js[q] = (q < nj) ? st->act[q0 + q] : 0;
    double pw[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) pw[q] = 0.0;
    if (h < g.Vh && nj > 0) {
        const Site s = site_of(g, h, 0);
        Vec3<float> acc[NR];
        hop2_multi<LP, NR>(g, U, T, stride, js, nj, h, 0, s, acc);
#pragma unroll
        for (int q = 0; q < NR; q++) {
            if (q < nj) {
                const float c = (float)st->c0[js[q]];
                const Vec3<float> pv = load_vec(P + js[q] * stride, h);
                Vec3<float> r;
                float d = 0.f;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    r.c[a] = c * pv.c[a] - 0.5f * acc[q].c[a];
                    d += pv.c[a].re * r.c[a].re + pv.c[a].im * r.c[a].im;
                }
                st_vec(W + js[q] * stride, h, r);
                pw[q] = (double)d;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NR; q++) {
        const double bs = block_sum(pw[q]);
        if (threadIdx.x == 0 && q < nj) partials[(size_t)(q0 + q) * gridDim.x + blockIdx.x] = bs;
    }
    if (last_block_n(counter, gridDim.x * gridDim.y)) {
        for (int a = 0; a < nact; a++) {
            double tot = 0.0;
            for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += __ldcg(partials + (size_t)a * gridDim.x + i);
            tot = block_sum(tot);
            if (threadIdx.x == 0) {
                const int k = st->act[a];
                st->alpha[k] = st->rr[k] / tot;
            }
        }
    }
}

__global__ void k_b_C(long n, size_t stride, float2* __restrict__ R, const float2* __restrict__ W,
                      const float2* __restrict__ P, float2* __restrict__ XL, BCGState* st, double* partials,
                      unsigned int* counter) {
    if (!st->live) return;
    const int a = blockIdx.y, nact = st->n_act;
    double acc = 0.0;
    if (a < nact) {
        const int k = st->act[a];
        const float alpha = (float)st->alpha[k];
        float2* r = R + k * stride;
        const float2* w = W + k * stride;
        const float2* p = P + k * stride;
        float2* x = XL + k * stride;
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
            float2 rv = r[i];
            const float2 wv = w[i], pv = p[i];
            float2 xv = x[i];
            rv.x -= alpha * wv.x;
            rv.y -= alpha * wv.y;
            xv.x += alpha * pv.x;
            xv.y += alpha * pv.y;
            r[i] = rv;
            x[i] = xv;
            acc += (double)(rv.x * rv.x + rv.y * rv.y);
        }
    }
    const double bs = block_sum(acc);
    if (threadIdx.x == 0 && a < nact) partials[(size_t)a * gridDim.x + blockIdx.x] = bs;
    if (last_block_n(counter, gridDim.x * gridDim.y)) {
        __shared__ double s_rr[STAG_MAXSHIFT];
        for (int b = 0; b < nact; b++) {
            double tot = 0.0;
            for (int i = threadIdx.x; i < gridDim.x; i += blockDim.x) tot += __ldcg(partials + (size_t)b * gridDim.x + i);
            tot = block_sum(tot);
            if (threadIdx.x == 0) s_rr[b] = tot;
        }
        if (threadIdx.x == 0) {
            int keep = 0, bad = 0, capped = 0;
            for (int b = 0; b < nact; b++) {
                const int k = st->act[b];
                const double rr_new = s_rr[b];
                st->iter[k] += 1;
                st->beta[k] = rr_new / st->rr[k];
                st->rr_prev[k] = st->rr[k];
                st->rr[k] = rr_new;
                if (!isfinite(rr_new)) bad = 1;
                if (st->iter[k] >= st->maxit) capped = 1;
                if (rr_new <= st->tol2bb[k]) {
                    st->want_rel[k] = 1;  // parked until the host checks it
                } else {
                    st->act[keep++] = k;
                }
            }
            st->n_act = keep;
            if (bad) st->nonfinite = 1;
            st->stop_next = (keep == 0 || bad || capped) ? 1 : 0;
        }
    }
}

__global__ void k_b_D(long n, size_t stride, const float2* __restrict__ R, float2* __restrict__ P, BCGState* st,
                      unsigned int* counter) {
    if (!st->live) return;
    const int a = blockIdx.y;
    if (a < st->n_act) {
        const int k = st->act[a];
        const float beta = (float)st->beta[k];
        const float2* r = R + k * stride;
        float2* p = P + k * stride;
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
            const float2 rv = r[i];
            float2 pv = p[i];
            pv.x = rv.x + beta * pv.x;
            pv.y = rv.y + beta * pv.y;
            p[i] = pv;
        }
    }
    if (last_block_n(counter, gridDim.x * gridDim.y)) {
        if (threadIdx.x == 0 && st->stop_next) st->live = 0;
    }
}

// ---- fused variant (3 kernels per iteration): B3 forms <p,w>, <r,w>, <w,w> per
// right-hand side; its last block computes alpha_k, |r_k - alpha_k w_k|^2 by
// expansion, beta_k and the parking; CD applies r -= alpha w, x += alpha p and
// (for right-hand sides still active) p = r + beta p.
template <int LP, int NR = NRMAX>
__global__ void __launch_bounds__(256, 4) k_b_B3(Geom g, const void* __restrict__ U, const float2* __restrict__ T,
                                                  const float2* __restrict__ P, const float2* __restrict__ R,
                                                  float2* __restrict__ W, size_t stride, BCGState* st,
                                                  double* partials, double* gpart, unsigned int* counter) {
    if (!st->live) return;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = blockIdx.y * NR, nact = st->n_act;
    const int nj = max(0, min(NR, nact - q0));
    int js[NR];
#pragma unroll
    for (int q = 0; q < NR; q++) js[q] = (q < nj) ? st->act[q0 + q] : 0;
    float flat[NR * 4];
#pragma unroll
    for (int q = 0; q < NR * 4; q++) flat[q] = 0.f;
    if (h < g.Vh && nj > 0) {
        const Site s = site_of(g, h, 0);
        Vec3<float> acc[NR];
        hop2_multi<LP, NR>(g, U, T, stride, js, nj, h, 0, s, acc);
#pragma unroll
        for (int q = 0; q < NR; q++) {
            if (q < nj) {
                const float c = (float)st->c0[js[q]];
                const Vec3<float> pv = load_vec(P + js[q] * stride, h), rv = load_vec(R + js[q] * stride, h);
                Vec3<float> w;
                float a = 0.f, b = 0.f, d = 0.f, e = 0.f;
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    w.c[i] = c * pv.c[i] - 0.5f * acc[q].c[i];
                    a += pv.c[i].re * w.c[i].re + pv.c[i].im * w.c[i].im;
                    b += rv.c[i].re * w.c[i].re + rv.c[i].im * w.c[i].im;
                    d += w.c[i].re * w.c[i].re + w.c[i].im * w.c[i].im;
                    e += rv.c[i].re * rv.c[i].re + rv.c[i].im * rv.c[i].im;
                }
                st_vec(W + js[q] * stride, h, w);
                flat[q * 4 + 0] = a;
                flat[q * 4 + 1] = b;
                flat[q * 4 + 2] = d;
                flat[q * 4 + 3] = e;
            }
        }
    }
    const size_t nbx = gridDim.x;
    if (nj > 0) {  // rows past the active right-hand sides only join the grid reduction
        const double bsum = block_sum_nv<NR * 4, float>(flat);
        if (threadIdx.x < 4 * nj) partials[((size_t)q0 * 4 + threadIdx.x) * nbx + blockIdx.x] = bsum;
    }
    __shared__ double s_sum[STAG_MAXSHIFT][4];
    if (grid_reduce_series(partials, gpart, counter, nact * 4, &s_sum[0][0])) {
        // one lane of warp 0 per active right-hand side (nact <= 32), all state
        // loaded up front; the still-active list is compacted in order by a ballot
        if (threadIdx.x < 32) {
            const int a = threadIdx.x;
            const int maxit = st->maxit;
            int k = 0, keep = 0, bad = 0, capped = 0;
            if (a < nact) {
                k = st->act[a];
                const int it = st->iter[k] + 1;
                const double tol2 = st->tol2bb[k];
                const double rr = s_sum[a][3];  // fresh |r_k|^2 of this iteration
                const double alpha = rr / s_sum[a][0];
                double rr_new = rr - 2.0 * alpha * s_sum[a][1] + alpha * alpha * s_sum[a][2];
                if (rr_new < 0.0) rr_new = 0.0;
                st->alpha[k] = alpha;
                st->beta[k] = rr_new / rr;
                st->rr_prev[k] = rr;
                st->rr[k] = rr_new;
                st->iter[k] = it;
                st->uact[a] = k;
                bad = !isfinite(rr_new) || !isfinite(alpha);
                capped = it >= maxit;
                if (rr_new <= tol2)
                    st->want_rel[k] = 1;  // parked until the host checks it
                else
                    keep = 1;
            }
            const unsigned int m = __ballot_sync(0xffffffffu, keep);
            if (keep) st->act[__popc(m & ((1u << a) - 1u))] = k;
            const int anybad = __any_sync(0xffffffffu, bad), anycap = __any_sync(0xffffffffu, capped);
            if (a == 0) {
                const int nkeep = __popc(m);
                st->n_uact = nact;
                st->n_act = nkeep;
                if (anybad) st->nonfinite = 1;
                st->stop_next = (nkeep == 0 || anybad || anycap) ? 1 : 0;
            }
        }
    }
}

__global__ void k_b_CD(long n, size_t stride, float2* __restrict__ R, const float2* __restrict__ W,
                       float2* __restrict__ P, float2* __restrict__ XL, BCGState* st, unsigned int* counter) {
    if (!st->live) return;
    const int a = blockIdx.y;
    if (a < st->n_uact) {
        const int k = st->uact[a];
        const float alpha = (float)st->alpha[k], beta = (float)st->beta[k];
        const bool upd_p = !st->want_rel[k];
        // float4: two complex entries per access (3 Vh is even, vectors 16-byte aligned)
        float4* r = (float4*)(R + k * stride);
        const float4* w = (const float4*)(W + k * stride);
        float4* p = (float4*)(P + k * stride);
        float4* x = (float4*)(XL + k * stride);
        const long n4 = n / 2;
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
            float4 rv = r[i], pv = p[i], xv = x[i];
            const float4 wv = w[i];
            rv.x = fmaf(-alpha, wv.x, rv.x);
            rv.y = fmaf(-alpha, wv.y, rv.y);
            rv.z = fmaf(-alpha, wv.z, rv.z);
            rv.w = fmaf(-alpha, wv.w, rv.w);
            xv.x = fmaf(alpha, pv.x, xv.x);
            xv.y = fmaf(alpha, pv.y, xv.y);
            xv.z = fmaf(alpha, pv.z, xv.z);
            xv.w = fmaf(alpha, pv.w, xv.w);
            r[i] = rv;
            x[i] = xv;
            if (upd_p) {
                pv.x = fmaf(beta, pv.x, rv.x);
                pv.y = fmaf(beta, pv.y, rv.y);
                pv.z = fmaf(beta, pv.z, rv.z);
                pv.w = fmaf(beta, pv.w, rv.w);
                p[i] = pv;
            }
        }
    }
}

// x_k += xl_k (FP64), xl_k = 0, for the listed slots
struct SlotList {
    int k[STAG_MAXSHIFT];
    double2* x[STAG_MAXSHIFT];
};
__global__ void k_b_accumulate(long n, size_t stride, float2* XL, SlotList L) {
    const int k = L.k[blockIdx.y];
    double2* x = L.x[blockIdx.y];
    float2* xl = XL + k * stride;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 v = xl[i];
        double2 d = x[i];
        d.x += (double)v.x;
        d.y += (double)v.y;
        x[i] = d;
        xl[i] = make_float2(0.f, 0.f);
    }
}

// r_k = b - w (FP64 in, FP32 out), |r|^2 -> dst
__global__ void k_b_residual(long n, const double2* __restrict__ b, const double2* __restrict__ w, float2* r,
                             double* partials, unsigned int* counter, double* dst) {
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 bv = b[i], wv = w[i];
        const double rx = bv.x - wv.x, ry = bv.y - wv.y;
        r[i] = make_float2((float)rx, (float)ry);
        acc += rx * rx + ry * ry;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
    if (last_block(counter)) finish_sum(partials, gridDim.x, dst);
}

__global__ void k_b_copy(long n, const float2* __restrict__ src, float2* dst) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

int env_i(const char* name, int dflt) {
    const char* v = getenv(name);
    return v ? atoi(v) : dflt;
}
double env_d(const char* name, double dflt) {
    const char* v = getenv(name);
    return v ? atof(v) : dflt;
}

}  // namespace

// FP64-accurate residuals r_k = b_k - (M_ee + c_k - m^2) x_k for the listed
// slots with the float-float operator: FP32 copies into R + k*n3, |r_k|^2
// into dscal2[100 + k] (read back, synchronising `s`).  Uses the
// refinement's own reduction buffers, so it may run beside the shifted CG.
int batched_true_residuals(stag_ctx* ctx, const RefSlots& S, const int* ks, int nk, float2* R, double* rr_out,
                           cudaStream_t s) {
    const long n3 = 3L * ctx->g.Vh;
    double2* w64 = (double2*)ws_get(ctx, WS_W64, sizeof(double2) * n3);
    double2* t64 = (double2*)ws_get(ctx, WS_T64, sizeof(double2) * n3);
    if (!w64 || !t64) return stag_fail(ctx, STAG_ERR_OOM, "residual workspace");
    for (int i = 0; i < nk; i++) {
        const int k = ks[i];
        int st = mee_apply(ctx, STAG_PREC_F64FF, S.c[k], S.x[k], w64, t64, s);
        if (st) return st;
        k_b_residual<<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, S.b[k], w64, R + k * n3, ctx->partials2,
                                                           ctx->counter2, ctx->dscal2 + 100 + k);
        STAG_LAUNCH_CHECK(ctx, "batched residual");
    }
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal2 + 100, ctx->dscal2 + 100, sizeof(double) * STAG_MAXSHIFT,
                                   cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    for (int i = 0; i < nk; i++) rr_out[ks[i]] = ctx->hscal2[100 + ks[i]];
    return STAG_OK;
}

int run_graph_chunk(stag_ctx* ctx, const char* key, int nkernels, void (*enqueue)(stag_ctx*, void*, cudaStream_t),
                    void* arg, cudaStream_t s);

namespace {
struct BIter {
    int lp;
    Links U;
    float2 *R, *P, *W, *T, *XL;
    double* part;
    int ny_hop, ny_blas, nbx_blas, chunk, fused, tpb, nr;
};

void enqueue_b(stag_ctx* ctx, void* argp, cudaStream_t cs) {
    const BIter& a = *(const BIter*)argp;
    const Geom& g = ctx->g;
    const long n3 = 3L * g.Vh;
    const size_t stride = (size_t)n3;
    const dim3 gh(nblocks(g.Vh, a.tpb), a.ny_hop), gb(a.nbx_blas, a.ny_blas);
    for (int i = 0; i < a.chunk; i++) {
        if (a.fused) {
            if (a.lp == LP32 && a.nr == 1) {
                k_b_A<LP32, 1><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.P, a.T, stride, ctx->bcg);
                k_b_B3<LP32, 1><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.T, a.P, a.R, a.W, stride, ctx->bcg, a.part,
                                                        ctx->gpart2, ctx->counter2);
            } else if (a.lp == LP32 && a.nr == 2) {
                k_b_A<LP32, 2><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.P, a.T, stride, ctx->bcg);
                k_b_B3<LP32, 2><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.T, a.P, a.R, a.W, stride, ctx->bcg, a.part,
                                                        ctx->gpart2, ctx->counter2);
            } else if (a.lp == LP32) {
                k_b_A<LP32><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.P, a.T, stride, ctx->bcg);
                k_b_B3<LP32><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.T, a.P, a.R, a.W, stride, ctx->bcg, a.part, ctx->gpart2,
                                                     ctx->counter2);
            } else {
                k_b_A<LP16><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.P, a.T, stride, ctx->bcg);
                k_b_B3<LP16><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.T, a.P, a.R, a.W, stride, ctx->bcg, a.part, ctx->gpart2,
                                                     ctx->counter2);
            }
            k_b_CD<<<gb, BLAS_TPB, 0, cs>>>(n3, stride, a.R, a.W, a.P, a.XL, ctx->bcg, ctx->counter2);
            continue;
        }
        if (a.lp == LP32) {
            k_b_A<LP32><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.P, a.T, stride, ctx->bcg);
            k_b_B<LP32><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.T, a.P, a.W, stride, ctx->bcg, a.part, ctx->counter2);
        } else {
            k_b_A<LP16><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.P, a.T, stride, ctx->bcg);
            k_b_B<LP16><<<gh, a.tpb, 0, cs>>>(g, a.U.u, a.T, a.P, a.W, stride, ctx->bcg, a.part, ctx->counter2);
        }
        k_b_C<<<gb, BLAS_TPB, 0, cs>>>(n3, stride, a.R, a.W, a.P, a.XL, ctx->bcg, a.part, ctx->counter2);
        k_b_D<<<gb, BLAS_TPB, 0, cs>>>(n3, stride, a.R, a.P, ctx->bcg, ctx->counter2);
    }
}
}  // namespace

// ---------------------------------------------------------------- Refiner

int Refiner::begin(stag_ctx* c, int link_prec, const RefSlots* slots, double tolerance, int max_iter, double* rr_io,
                   int* iters_out, cudaStream_t stream) {
    ctx = c;
    lp = link_prec;
    S = slots;
    tol = tolerance;
    maxit = max_iter;
    rr = rr_io;
    iters = iters_out;
    s = stream;
    const long n3 = 3L * ctx->g.Vh;
    const size_t vb = sizeof(float2) * n3 * STAG_MAXSHIFT;
    R = (float2*)ws_get(ctx, WS_BR, vb);
    P = (float2*)ws_get(ctx, WS_RPK, vb);
    XL = (float2*)ws_get(ctx, WS_RXL, vb);
    W = (float2*)ws_get(ctx, WS_BW, vb);
    T = (float2*)ws_get(ctx, WS_BT, vb);
    const int nbx = nblocks(ctx->g.Vh, 64);  // partials sized for the smallest block size
    part = (double*)ws_get(ctx, WS_BPART,
                           sizeof(double) * 4 * STAG_MAXSHIFT * (size_t)(nbx > ctx->num_sms ? nbx : ctx->num_sms));
    if (!R || !P || !XL || !W || !T || !part) return stag_fail(ctx, STAG_ERR_OOM, "refinement workspace");
    tpb = hop_tpb(ctx, lp);
    chunk = env_i("STAG_CHUNK", 32);
    fused = env_i("STAG_FUSED", 1);
    delta = env_d("STAG_RELIABLE_DELTA", 0.03);
    bcd_bps = env_i("STAG_BCD_BPS", 8);
    trace = env_i("STAG_TRACE_REFINE", 0);
    nreliable = nmatvec = 0;
    norder = remaining = 0;
    flying = false;
    for (int k = 0; k < STAG_MAXSHIFT; k++) active[k] = done[k] = 0;
    BCGState* hs = ctx->bcg_host;
    memset(hs, 0, sizeof(BCGState));
    hs->delta2 = delta * delta;
    hs->maxit = maxit;
    dirty = true;
    return STAG_OK;
}

int Refiner::add(const int* ks, int nk) {
    if (flying) return stag_fail(ctx, STAG_ERR_STATE, "refinement slots added while a chunk runs");
    const long n3 = 3L * ctx->g.Vh;
    BCGState* hs = ctx->bcg_host;
    for (int i = 0; i < nk; i++) {
        const int k = ks[i];
        hs->rr[k] = hs->rr_max[k] = rr[k];
        hs->c0[k] = S->c[k];
        hs->tol2bb[k] = tol * tol * S->bb[k];
        hs->iter[k] = 0;
        hs->want_rel[k] = 0;
        STAG_CUDA(ctx, cudaMemsetAsync(XL + k * n3, 0, sizeof(float2) * n3, s));
        k_b_copy<<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, R + k * n3, P + k * n3);
        STAG_LAUNCH_CHECK(ctx, "refine init");
        order[norder++] = k;
        active[k] = 1;
        remaining++;
    }
    // the active list in joining order
    int na = 0;
    for (int i = 0; i < norder; i++)
        if (active[order[i]] && !done[order[i]]) hs->act[na++] = order[i];
    hs->n_act = na;
    hs->stop_next = 0;
    hs->live = na > 0;
    dirty = true;
    return STAG_OK;
}

int Refiner::launch() {
    BCGState* hs = ctx->bcg_host;
    if (flying || hs->n_act == 0) return STAG_OK;
    if (dirty) {
        STAG_CUDA(ctx, cudaMemcpyAsync(ctx->bcg, hs, sizeof(BCGState), cudaMemcpyHostToDevice, s));
        dirty = false;
    }
    BIter it;
    it.lp = lp;
    it.U.u = (lp == LP32) ? (const void*)ctx->U32 : (const void*)ctx->U16;
    it.U.lo = ctx->U32lo;
    it.R = R;
    it.P = P;
    it.XL = XL;
    it.W = W;
    it.T = T;
    it.part = part;
    it.tpb = tpb;
    it.chunk = chunk;
    it.fused = fused;
    // the grids cover the right-hand sides active at the start of the chunk
    // (the device only removes slots within a chunk); one graph per size
    it.nr = (fused && lp == LP32) ? nr_policy(hs->n_act, env_i("STAG_REFINE_NR", 1)) : NRMAX;
    it.ny_hop = (hs->n_act + it.nr - 1) / it.nr;
    it.ny_blas = hs->n_act;
    // vector-update blocks per right-hand side: about bcd_bps blocks per SM
    // over all rows (at least one per SM, at most one float4 per thread)
    const long n3 = 3L * ctx->g.Vh;
    it.nbx_blas = bcd_bps > 0 ? std::max(ctx->num_sms, std::min(nblocks(n3 / 2, BLAS_TPB),
                                                                 ctx->num_sms * bcd_bps / std::max(1, hs->n_act)))
                              : ctx->num_sms;
    char key[80];
    snprintf(key, sizeof key, "bcg_%d_%d_%d_%d_%d_%d_%d", lp, hs->n_act, it.chunk, it.fused, it.tpb, it.nr,
             it.nbx_blas);
    int st = run_graph_chunk(ctx, key, (it.fused ? 3 : 4) * it.chunk, enqueue_b, &it, s);
    if (st) return st;
    STAG_CUDA(ctx, cudaMemcpyAsync(hs, ctx->bcg, sizeof(BCGState), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaEventRecord(ctx->ev_ref, s));
    flying = true;
    return STAG_OK;
}

bool Refiner::ready() const { return !flying || cudaEventQuery(ctx->ev_ref) == cudaSuccess; }

int Refiner::poll() {
    if (!flying) return STAG_OK;
    STAG_CUDA(ctx, cudaEventSynchronize(ctx->ev_ref));
    flying = false;
    BCGState* hs = ctx->bcg_host;
    const long n3 = 3L * ctx->g.Vh;
    if (trace) {
        fprintf(stderr, "[refine] n_act %d live %d nonfinite %d |", hs->n_act, hs->live, hs->nonfinite);
        for (int i = 0; i < norder; i++) {
            const int k = order[i];
            fprintf(stderr, " k%d it%d rr%.2e a%.2e b%.2e p%d", k, hs->iter[k], hs->rr[k] / S->bb[k], hs->alpha[k],
                    hs->beta[k], hs->want_rel[k]);
        }
        fprintf(stderr, "\n");
    }
    if (hs->nonfinite) return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite residual in batched CG");
    // reliable updates: parked (claimed convergence) and those whose residual dropped by delta
    int upd[STAG_MAXSHIFT], nu = 0, parked[STAG_MAXSHIFT] = {0};
    int in_act[STAG_MAXSHIFT] = {0};
    for (int a = 0; a < hs->n_act; a++) in_act[hs->act[a]] = 1;
    for (int i = 0; i < norder; i++) {
        const int k = order[i];
        if (done[k]) continue;
        if (hs->want_rel[k]) {
            parked[k] = 1;
            upd[nu++] = k;
        } else if (in_act[k] && hs->rr[k] > 1e2 * hs->rr_max[k]) {
            parked[k] = 1;  // the recursion drifted away: restart from the true residual
            upd[nu++] = k;
        } else if (in_act[k] && (hs->rr[k] < hs->delta2 * hs->rr_max[k] || hs->iter[k] >= maxit)) {
            upd[nu++] = k;
        }
    }
    int st;
    if (nu > 0) {
        SlotList L;
        for (int i = 0; i < nu; i++) {
            L.k[i] = upd[i];
            L.x[i] = S->x[upd[i]];
        }
        k_b_accumulate<<<dim3(ctx->num_sms, nu), BLAS_TPB, 0, s>>>(n3, (size_t)n3, XL, L);
        STAG_LAUNCH_CHECK(ctx, "refine accumulate");
        double rrt[STAG_MAXSHIFT];
        if ((st = batched_true_residuals(ctx, *S, upd, nu, R, rrt, s))) return st;
        nmatvec += nu;
        nreliable += nu;
        for (int i = 0; i < nu; i++) {
            const int k = upd[i];
            hs->want_rel[k] = 0;
            rr[k] = rrt[k];
            if (rrt[k] <= hs->tol2bb[k] || hs->iter[k] >= maxit) {
                done[k] = 1;
                remaining--;
                in_act[k] = 0;
                continue;
            }
            hs->rr[k] = hs->rr_max[k] = rrt[k];
            if (parked[k]) {  // the recursion claimed convergence but the true residual disagrees: restart
                k_b_copy<<<ctx->num_sms * 4, BLAS_TPB, 0, s>>>(n3, R + k * n3, P + k * n3);
                STAG_LAUNCH_CHECK(ctx, "refine restart");
                in_act[k] = 1;
            }
        }
    }
    // rebuild the active list (compacted, joining order)
    int na = 0;
    for (int i = 0; i < norder; i++) {
        const int k = order[i];
        active[k] = in_act[k] && !done[k];
        if (active[k]) hs->act[na++] = k;
    }
    hs->n_act = na;
    hs->stop_next = 0;
    hs->live = na > 0;
    dirty = true;
    if (remaining > 0 && na == 0) return stag_fail(ctx, STAG_ERR_NOCONV, "batched refinement stalled");
    for (int i = 0; i < norder; i++) iters[order[i]] = hs->iter[order[i]];
    return STAG_OK;
}

int Refiner::finish() {
    int st;
    while (remaining > 0) {
        if (!flying && ctx->bcg_host->n_act == 0)
            return stag_fail(ctx, STAG_ERR_NOCONV, "batched refinement stalled");
        if ((st = launch())) return st;
        if ((st = poll())) return st;
    }
    for (int i = 0; i < norder; i++) {
        iters[order[i]] = ctx->bcg_host->iter[order[i]];
        nmatvec += ctx->bcg_host->iter[order[i]];
    }
    return STAG_OK;
}

// Refines the FP64 solutions S.x[k] of the slots ks[0..nk) (those whose true
// residual rr[k] > tol^2 bb_k on entry; R + k*n3 must already hold their FP32
// residuals).  On return rr[k] holds each slot's final FP64-accurate true
// residual^2.
int refine_batched(stag_ctx* ctx, int lp, const RefSlots& S, const int* ks, int nk, float2* R, double tol, int maxit,
                   double* rr, int* iters, int* reliable, int* matvecs, cudaStream_t s) {
    Refiner rf;
    int st = rf.begin(ctx, lp, &S, tol, maxit, rr, iters, s);
    if (st) return st;
    if (rf.R != R) return stag_fail(ctx, STAG_ERR_STATE, "refinement residuals outside the refinement workspace");
    if ((st = rf.add(ks, nk))) return st;
    if ((st = rf.finish())) return st;
    *reliable += rf.nreliable;
    *matvecs += rf.nmatvec;
    return STAG_OK;
}

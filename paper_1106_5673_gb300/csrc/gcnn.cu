// gcnn.cu -- learned gauge-covariant preconditioner for the lightest RHMC pole
// (a component of this library; the paper has no network).
//
// A layer maps C_in colour-vector fields on the full lattice to C_out fields
// by a parallel-transport convolution with 9 taps:
//   (L phi)_o(n) = sum_i sum_t w[o][i][t] (T_t phi_i)(n),
//   T_0 phi = phi(n), T_{1+mu} phi = U_mu(n) phi(n+mu),
//   T_{5+mu} phi = U_mu(n-mu)^dag phi(n-mu),
// which commutes with gauge transformations.  A = L3 L2 L1 (channels
// 1 -> H -> H -> 1); the preconditioner is K = restrict_even A^dag A
// embed_even, Hermitian positive semi-definite by construction, where the
// adjoint layer is (L^dag g)_i = sum_o sum_t conj(w[o][i][t]) T_t^dag g_o and
// T_{1+mu}^dag = T_{5+mu}.  K is trained to map sources b to solutions x of
// (M_ee + s) x = b by minimising mean_j |K b_j - x_j|^2 / |x_j|^2 with Adam,
// using this file's forward, adjoint and weight-gradient kernels; the weight
// gradient of a layer is 2 sum_n <T_t a_i(n), b_o(n)> with (a, b) = (layer
// input, output gradient) for a forward layer and (output gradient, layer
// input) for an adjoint layer.  Weights are stored in BF16 for the forward
// pass (FP32 master copy for the optimiser); arithmetic is FP32.  The flexible
// CG of this file (Golub-Ye's inexact preconditioned CG) uses K as a
// preconditioner for the lightest pole, with FP64 vectors and the FP64-accurate
// float-float operator, so the residual is judged in FP64 whatever K does.
#include <stdlib.h>

#include <vector>

#include "hop.cuh"
#include "stag_internal.h"

#define GC_H 8          // hidden channels
#define GC_TAPS 9
#define GC_NLAYER 3

struct stag_net {
    stag_ctx* ctx;
    int cin[GC_NLAYER], cout[GC_NLAYER];
    int nw[GC_NLAYER];                 // complex weights per layer
    float2* w32[GC_NLAYER];            // FP32 master [cout][cin][9]
    __nv_bfloat162* w16[GC_NLAYER];    // BF16 copy used by the forward pass
    float2 *m[GC_NLAYER], *v[GC_NLAYER], *grad[GC_NLAYER];
    float2* act[GC_NLAYER + 1];        // forward activations a0 [1][V][3], a1, a2 [H][V][3], a3 [1][V][3]
    float2* cact[GC_NLAYER];           // adjoint activations c0 = A^dag A a0 [1], c1, c2 [H]
    float2* gact[GC_NLAYER + 1];       // gradients (channels 1, H, H, 1), reused along the backward pass
    double* partials;                  // weight-gradient block partials
    double* dsc;                       // device scalars
    double* hsc;                       // pinned host scalars
    int step;                          // Adam step
    int nblk;                          // blocks of the weight-gradient kernel
};

namespace {

const int TPB = 128;

STAG_D float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// taps 1+mu and 5+mu of the adjoint swap roles: T_{1+mu}^dag = U(n-mu)^dag g(n-mu)
STAG_HD int tap_swap(int t) { return t == 0 ? 0 : (t <= 4 ? t + 4 : t - 4); }

// One layer (or its adjoint) on all sites: out[o] = sum_i sum_t W'[o][i][t] T_t in[i].
// Forward: W' = W [CO][CI][9] (BF16).  Adjoint: W'[i][o][swap(t)] = conj(W[o][i][t]),
// with CIN/COUT the channel counts of this application.
template <int CIN, int COUT>
__global__ void __launch_bounds__(TPB) k_gc_layer(Geom g, const float4* __restrict__ U, const float2* __restrict__ in,
                                                  float2* __restrict__ out, const __nv_bfloat162* __restrict__ W,
                                                  int adjoint) {
    __shared__ float2 w[COUT][CIN][GC_TAPS];
    for (int j = threadIdx.x; j < COUT * CIN * GC_TAPS; j += blockDim.x) {
        const int t = j % GC_TAPS, i = (j / GC_TAPS) % CIN, o = j / (GC_TAPS * CIN);
        if (!adjoint) {
            const float2 c = __bfloat1622float2(W[j]);
            w[o][i][t] = c;
        } else {
            // stored layer weights are [Wo = CIN][Wi = COUT][9]; this application's out o = stored in
            const float2 c = __bfloat1622float2(W[(i * COUT + o) * GC_TAPS + t]);
            w[o][i][tap_swap(t)] = make_float2(c.x, -c.y);
        }
    }
    __syncthreads();
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.V) return;
    const Site s = site_from_lex(g, n);
    const int par = par_of(s);
    const size_t cs = 3 * (size_t)g.V;
    Vec3<float> acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; o++) acc[o] = vzero<float>();
#pragma unroll
    for (int i = 0; i < CIN; i++) {
        const Vec3<float> v = load_vec(in + i * cs, n);
#pragma unroll
        for (int o = 0; o < COUT; o++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float2 r = cmulf(w[o][i][0], make_float2(v.c[a].re, v.c[a].im));
                acc[o].c[a].re += r.x;
                acc[o].c[a].im += r.y;
            }
    }
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
        const int lf = nb_lex(g, s, mu, +1), lb = nb_lex(g, s, mu, -1);
        const Mat3<float> uf = load_link32(U, g, mu, par, n >> 1);
        const Mat3<float> ub = load_link32(U, g, mu, 1 - par, lb >> 1);
#pragma unroll
        for (int i = 0; i < CIN; i++) {
            const Vec3<float> tf = mv(uf, load_vec(in + i * cs, lf));
            const Vec3<float> tb = mdv(ub, load_vec(in + i * cs, lb));
#pragma unroll
            for (int o = 0; o < COUT; o++)
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const float2 r1 = cmulf(w[o][i][1 + mu], make_float2(tf.c[a].re, tf.c[a].im));
                    const float2 r2 = cmulf(w[o][i][5 + mu], make_float2(tb.c[a].re, tb.c[a].im));
                    acc[o].c[a].re += r1.x + r2.x;
                    acc[o].c[a].im += r1.y + r2.y;
                }
        }
    }
#pragma unroll
    for (int o = 0; o < COUT; o++) st_vec(out + o * cs, n, acc[o]);
}

// Weight gradient: gW[o][i][t] = 2 sum_n <T_t in_i (n), gout_o(n)>; block
// partials [blk][o][i][t][re,im]; each thread strides over sites.
template <int CIN, int COUT>
__global__ void __launch_bounds__(TPB) k_gc_wgrad(Geom g, const float4* __restrict__ U, const float2* __restrict__ in,
                                                  const float2* __restrict__ gout, double* partials) {
    __shared__ double acc_s[COUT * CIN * GC_TAPS * 2];
    for (int j = threadIdx.x; j < COUT * CIN * GC_TAPS * 2; j += blockDim.x) acc_s[j] = 0.0;
    __syncthreads();
    const size_t cs = 3 * (size_t)g.V;
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int i = 0; i < CIN; i++) {
#pragma unroll 1
        for (int t = 0; t < GC_TAPS; t++) {
            float2 d[COUT];
#pragma unroll
            for (int o = 0; o < COUT; o++) d[o] = make_float2(0.f, 0.f);
            for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < g.V; n += gridDim.x * blockDim.x) {
                const Site s = site_from_lex(g, n);
                const int par = par_of(s);
                Vec3<float> T;
                if (t == 0) {
                    T = load_vec(in + i * cs, n);
                } else if (t <= 4) {
                    const int mu = t - 1;
                    T = mv(load_link32(U, g, mu, par, n >> 1), load_vec(in + i * cs, nb_lex(g, s, mu, +1)));
                } else {
                    const int mu = t - 5;
                    const int lb = nb_lex(g, s, mu, -1);
                    T = mdv(load_link32(U, g, mu, 1 - par, lb >> 1), load_vec(in + i * cs, lb));
                }
#pragma unroll
                for (int o = 0; o < COUT; o++) {
                    const Vec3<float> gv = load_vec(gout + o * cs, n);
#pragma unroll
                    for (int a = 0; a < 3; a++) {  // conj(T) g
                        d[o].x += T.c[a].re * gv.c[a].re + T.c[a].im * gv.c[a].im;
                        d[o].y += T.c[a].re * gv.c[a].im - T.c[a].im * gv.c[a].re;
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < COUT; o++) {
                // warp level in FP32 (FP64 shuffles are slow on GB300), FP64 across warps
                const double re = warp_sum_f(d[o].x), im = warp_sum_f(d[o].y);
                if (lane == 0) {
                    atomicAdd(&acc_s[((o * CIN + i) * GC_TAPS + t) * 2], re);
                    atomicAdd(&acc_s[((o * CIN + i) * GC_TAPS + t) * 2 + 1], im);
                }
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < COUT * CIN * GC_TAPS * 2; j += blockDim.x)
        partials[(size_t)blockIdx.x * COUT * CIN * GC_TAPS * 2 + j] = acc_s[j];
}

// grad[j] (+)= 2 sum_blocks partials (deterministic order)
__global__ void k_gc_wgrad_reduce(int nvals, int nblk, const double* partials, float2* grad, int accumulate) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nvals) return;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nblk; b++) {
        re += partials[(size_t)b * nvals * 2 + 2 * j];
        im += partials[(size_t)b * nvals * 2 + 2 * j + 1];
    }
    float2 gj = accumulate ? grad[j] : make_float2(0.f, 0.f);
    grad[j] = make_float2(gj.x + (float)(2.0 * re), gj.y + (float)(2.0 * im));
}

// a0 = embed(b): even sites from b (FP64), odd sites 0
__global__ void k_gc_embed(Geom g, const double2* __restrict__ b, float2* a0) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.V) return;
    const int even = (par_of(site_from_lex(g, n)) == 0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double2 v = even ? b[3 * (size_t)(n >> 1) + c] : make_double2(0.0, 0.0);
        a0[3 * (size_t)n + c] = make_float2((float)v.x, (float)v.y);
    }
}

// z = restrict_even(y) (FP64 out)
__global__ void k_gc_restrict(Geom g, const float2* __restrict__ y, double2* z) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const int n = site_of(g, h, 0).lex;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float2 v = y[3 * (size_t)n + c];
        z[3 * (size_t)h + c] = make_double2(v.x, v.y);
    }
}

// loss gradient: e = y - x on even sites; g3 = e / (|x|^2 B) embedded (odd 0);
// partial sums of |e|^2 / |x|^2 into dst (atomic, FP64)
__global__ void k_gc_lossgrad(Geom g, const float2* __restrict__ y, const double2* __restrict__ x, double inv_nx_B,
                              float2* g3, double* loss_acc) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (n < g.V) {
        const int even = (par_of(site_from_lex(g, n)) == 0);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float2 gv = make_float2(0.f, 0.f);
            if (even) {
                const float2 yv = y[3 * (size_t)n + c];
                const double2 xv = x[3 * (size_t)(n >> 1) + c];
                const double ex = yv.x - xv.x, ey = yv.y - xv.y;
                acc += ex * ex + ey * ey;
                gv = make_float2((float)(ex * inv_nx_B), (float)(ey * inv_nx_B));
            }
            g3[3 * (size_t)n + c] = gv;
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) atomicAdd(loss_acc, acc * inv_nx_B);
}

// Adam on the FP32 master weights (complex entries as two reals) and BF16 refresh
__global__ void k_gc_adam(int n, float2* w, float2* m, float2* v, const float2* grad, __nv_bfloat162* w16, float lr,
                          float b1, float b2, float c1, float c2, float eps) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float2 gj = grad[j];
    float2 mj = m[j], vj = v[j], wj = w[j];
    mj.x = b1 * mj.x + (1.f - b1) * gj.x;
    mj.y = b1 * mj.y + (1.f - b1) * gj.y;
    vj.x = b2 * vj.x + (1.f - b2) * gj.x * gj.x;
    vj.y = b2 * vj.y + (1.f - b2) * gj.y * gj.y;
    wj.x -= lr * (mj.x / c1) / (sqrtf(vj.x / c2) + eps);
    wj.y -= lr * (mj.y / c1) / (sqrtf(vj.y / c2) + eps);
    m[j] = mj;
    v[j] = vj;
    w[j] = wj;
    w16[j] = __float22bfloat162_rn(wj);
}

__global__ void k_gc_tobf16(int n, const float2* w, __nv_bfloat162* w16) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) w16[j] = __float22bfloat162_rn(w[j]);
}

void layer_launch(stag_net* net, int l, const float2* in, float2* out, int adjoint, cudaStream_t s) {
    stag_ctx* ctx = net->ctx;
    const int nb = nblocks(ctx->g.V, TPB);
    const int ci = adjoint ? net->cout[l] : net->cin[l];
    const int co = adjoint ? net->cin[l] : net->cout[l];
    if (ci == 1 && co == GC_H)
        k_gc_layer<1, GC_H><<<nb, TPB, 0, s>>>(ctx->g, ctx->U32, in, out, net->w16[l], adjoint);
    else if (ci == GC_H && co == GC_H)
        k_gc_layer<GC_H, GC_H><<<nb, TPB, 0, s>>>(ctx->g, ctx->U32, in, out, net->w16[l], adjoint);
    else
        k_gc_layer<GC_H, 1><<<nb, TPB, 0, s>>>(ctx->g, ctx->U32, in, out, net->w16[l], adjoint);
    ctx->nlaunch++;
}

void wgrad_launch(stag_net* net, int l, const float2* in, const float2* gout, int accumulate, cudaStream_t s) {
    stag_ctx* ctx = net->ctx;
    const int ci = net->cin[l], co = net->cout[l];
    if (ci == 1)
        k_gc_wgrad<1, GC_H><<<net->nblk, TPB, 0, s>>>(ctx->g, ctx->U32, in, gout, net->partials);
    else if (co == GC_H)
        k_gc_wgrad<GC_H, GC_H><<<net->nblk, TPB, 0, s>>>(ctx->g, ctx->U32, in, gout, net->partials);
    else
        k_gc_wgrad<GC_H, 1><<<net->nblk, TPB, 0, s>>>(ctx->g, ctx->U32, in, gout, net->partials);
    k_gc_wgrad_reduce<<<nblocks(net->nw[l], 128), 128, 0, s>>>(net->nw[l], net->nblk, net->partials, net->grad[l],
                                                              accumulate);
    ctx->nlaunch += 2;
}

int env_i(const char* name, int dflt) {
    const char* v = getenv(name);
    return v ? atoi(v) : dflt;
}

}  // namespace

// ---------------------------------------------------------------- host API

int net_create(stag_ctx* ctx, unsigned seed, stag_net** out) {
    stag_net* net = new stag_net();
    memset(net, 0, sizeof(*net));
    net->ctx = ctx;
    const int cin[GC_NLAYER] = {1, GC_H, GC_H}, cout[GC_NLAYER] = {GC_H, GC_H, 1};
    const size_t cs = 3 * (size_t)ctx->g.V;
    net->nblk = 4 * ctx->num_sms;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < GC_NLAYER; l++) {
        net->cin[l] = cin[l];
        net->cout[l] = cout[l];
        net->nw[l] = cin[l] * cout[l] * GC_TAPS;
        const size_t b = sizeof(float2) * net->nw[l];
        if (e == cudaSuccess) e = cudaMalloc(&net->w32[l], b);
        if (e == cudaSuccess) e = cudaMalloc(&net->w16[l], sizeof(__nv_bfloat162) * net->nw[l]);
        if (e == cudaSuccess) e = cudaMalloc(&net->m[l], b);
        if (e == cudaSuccess) e = cudaMalloc(&net->v[l], b);
        if (e == cudaSuccess) e = cudaMalloc(&net->grad[l], b);
        if (e == cudaSuccess) e = cudaMemset(net->m[l], 0, b);
        if (e == cudaSuccess) e = cudaMemset(net->v[l], 0, b);
    }
    const int chans[GC_NLAYER + 1] = {1, GC_H, GC_H, 1};
    for (int l = 0; l <= GC_NLAYER; l++) {
        if (e == cudaSuccess) e = cudaMalloc(&net->act[l], sizeof(float2) * cs * chans[l]);
        if (e == cudaSuccess) e = cudaMalloc(&net->gact[l], sizeof(float2) * cs * chans[l]);
        if (l < GC_NLAYER && e == cudaSuccess) e = cudaMalloc(&net->cact[l], sizeof(float2) * cs * chans[l]);
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&net->partials, sizeof(double) * 2 * GC_H * GC_H * GC_TAPS * (size_t)net->nblk);
    if (e == cudaSuccess) e = cudaMalloc(&net->dsc, sizeof(double) * 16);
    if (e == cudaSuccess) e = cudaMallocHost(&net->hsc, sizeof(double) * 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        net->ctx = nullptr;  // not attached: net_destroy frees what was allocated
        net_destroy(net);
        stag_fail(ctx, STAG_ERR_OOM, "network allocation");
        return STAG_ERR_OOM;
    }
    // initial weights: identity tap 0 on the diagonal path plus small random
    // parallel-transport taps (deterministic from the seed)
    uint64_t st = 0x9E3779B97F4A7C15ull ^ seed;
    auto rnd = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return ((st >> 11) * (1.0 / 9007199254740992.0)) - 0.5;
    };
    for (int l = 0; l < GC_NLAYER; l++) {
        std::vector<float2> h(net->nw[l]);
        const float sc = 0.2f / sqrtf((float)net->cin[l] * GC_TAPS);
        for (int o = 0; o < net->cout[l]; o++)
            for (int i = 0; i < net->cin[l]; i++)
                for (int t = 0; t < GC_TAPS; t++) {
                    float2 w = make_float2(sc * (float)rnd(), sc * (float)rnd());
                    if (t == 0 && (i == o % net->cin[l] || net->cin[l] == 1)) w.x += 1.0f / (l == 2 ? GC_H : 1);
                    h[(o * net->cin[l] + i) * GC_TAPS + t] = w;
                }
        cudaMemcpy(net->w32[l], h.data(), sizeof(float2) * net->nw[l], cudaMemcpyHostToDevice);
        k_gc_tobf16<<<nblocks(net->nw[l], 128), 128>>>(net->nw[l], net->w32[l], net->w16[l]);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        const int st = stag_cuda_check(ctx, cudaGetLastError(), "network init");
        net->ctx = nullptr;
        net_destroy(net);
        return st;
    }
    *out = net;
    return STAG_OK;
}

void net_destroy(stag_net* net) {
    if (!net) return;
    cudaDeviceSynchronize();
    if (net->ctx && net->ctx->net == net) net->ctx->net = nullptr;
    for (int l = 0; l < GC_NLAYER; l++) {
        cudaFree(net->w32[l]);
        cudaFree(net->w16[l]);
        cudaFree(net->m[l]);
        cudaFree(net->v[l]);
        cudaFree(net->grad[l]);
    }
    for (int l = 0; l <= GC_NLAYER; l++) {
        cudaFree(net->act[l]);
        cudaFree(net->gact[l]);
        if (l < GC_NLAYER) cudaFree(net->cact[l]);
    }
    cudaFree(net->partials);
    cudaFree(net->dsc);
    cudaFreeHost(net->hsc);
    delete net;
}

// forward activations a_l and adjoint activations c_l of K b
static void net_forward(stag_net* net, const double2* b, cudaStream_t s) {
    stag_ctx* ctx = net->ctx;
    k_gc_embed<<<nblocks(ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, b, net->act[0]);
    ctx->nlaunch++;
    for (int l = 0; l < GC_NLAYER; l++) layer_launch(net, l, net->act[l], net->act[l + 1], 0, s);
    for (int l = GC_NLAYER - 1; l >= 0; l--)
        layer_launch(net, l, l == GC_NLAYER - 1 ? net->act[GC_NLAYER] : net->cact[l + 1], net->cact[l], 1, s);
}

// z = K b = restrict A^dag A embed b (FP64 even-site vectors in and out)
int net_apply(stag_net* net, const double2* b, double2* z, cudaStream_t s) {
    stag_ctx* ctx = net->ctx;
    net_forward(net, b, s);
    k_gc_restrict<<<nblocks(ctx->g.Vh, TPB), TPB, 0, s>>>(ctx->g, net->cact[0], z);
    ctx->nlaunch++;
    STAG_LAUNCH_CHECK(ctx, "net apply");
    return STAG_OK;
}

// loss and weight gradients (accumulated into grad[]) of the pairs (b_j, x_j);
// returns the mean loss in *loss.  Back-propagation: through the adjoint
// layers (L0^dag applied last, so first here), then the forward layers.
int net_loss_grad(stag_net* net, int npairs, const double2* const* bs, const double2* const* xs, double* loss,
                  cudaStream_t s) {
    stag_ctx* ctx = net->ctx;
    STAG_CUDA(ctx, cudaMemsetAsync(net->dsc, 0, sizeof(double) * 2, s));
    float2** g = net->gact;
    for (int j = 0; j < npairs; j++) {
        // |x|^2
        int st = blas_dot_re(ctx, STAG_PREC_F64, xs[j], xs[j], net->dsc + 2, s);
        if (st) return st;
        STAG_CUDA(ctx, cudaMemcpyAsync(net->hsc + 2, net->dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
        STAG_CUDA(ctx, cudaStreamSynchronize(s));
        const double inv = 1.0 / (net->hsc[2] * npairs);
        net_forward(net, bs[j], s);
        // g[0] = dloss/dconj(c0) (even sites), loss partial sums
        k_gc_lossgrad<<<nblocks(ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, net->cact[0], xs[j], inv, g[0], net->dsc);
        ctx->nlaunch++;
        // adjoint layer l: c_l = L_l^dag c_{l+1}; gradient at c_l is g[l]
        for (int l = 0; l < GC_NLAYER; l++) {
            const float2* cin = (l == GC_NLAYER - 1) ? net->act[GC_NLAYER] : net->cact[l + 1];
            wgrad_launch(net, l, g[l], cin, j > 0, s);
            layer_launch(net, l, g[l], g[l + 1], 0, s);  // gradient at c_{l+1}; g[3] is the one at a3
        }
        // forward layer l: a_{l+1} = L_l a_l; gradient at a_{l+1} is g[l + 1]
        for (int l = GC_NLAYER - 1; l >= 0; l--) {
            wgrad_launch(net, l, net->act[l], g[l + 1], 1, s);
            if (l > 0) layer_launch(net, l, g[l + 1], g[l], 1, s);
        }
        STAG_LAUNCH_CHECK(ctx, "net gradient");
    }
    STAG_CUDA(ctx, cudaMemcpyAsync(net->hsc, net->dsc, sizeof(double), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    *loss = net->hsc[0];
    return STAG_OK;
}

// epochs of Adam over minibatches of the pairs; returns the loss of the last epoch
int net_train(stag_net* net, int npairs, const double2* const* bs, const double2* const* xs, int epochs, int batch,
              double lr, double* loss_out, cudaStream_t s) {
    stag_ctx* ctx = net->ctx;
    double last = 0.0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs; ep++) {
        double tot = 0.0;
        int nb = 0;
        for (int j0 = 0; j0 < npairs; j0 += batch) {
            const int nbat = (npairs - j0 < batch) ? npairs - j0 : batch;
            double l = 0.0;
            int st = net_loss_grad(net, nbat, bs + j0, xs + j0, &l, s);
            if (st) return st;
            tot += l;
            nb++;
            net->step++;
            const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
            for (int li = 0; li < GC_NLAYER; li++)
                k_gc_adam<<<nblocks(net->nw[li], 128), 128, 0, s>>>(net->nw[li], net->w32[li], net->m[li], net->v[li],
                                                                   net->grad[li], net->w16[li], (float)lr, b1, b2, c1,
                                                                   c2, 1e-8f);
            ctx->nlaunch += GC_NLAYER;
            STAG_LAUNCH_CHECK(ctx, "adam");
        }
        last = tot / nb;
    }
    *loss_out = last;
    return STAG_OK;
}

int net_get_weights(stag_net* net, int layer, float* host) {
    return cudaMemcpy(host, net->w32[layer], sizeof(float2) * net->nw[layer], cudaMemcpyDeviceToHost) == cudaSuccess
               ? STAG_OK
               : STAG_ERR_CUDA;
}

int net_set_weights(stag_net* net, int layer, const float* host) {
    if (cudaMemcpy(net->w32[layer], host, sizeof(float2) * net->nw[layer], cudaMemcpyHostToDevice) != cudaSuccess)
        return STAG_ERR_CUDA;
    k_gc_tobf16<<<nblocks(net->nw[layer], 128), 128>>>(net->nw[layer], net->w32[layer], net->w16[layer]);
    return cudaDeviceSynchronize() == cudaSuccess ? STAG_OK : STAG_ERR_CUDA;
}

int net_get_grads(stag_net* net, int layer, float* host) {
    return cudaMemcpy(host, net->grad[layer], sizeof(float2) * net->nw[layer], cudaMemcpyDeviceToHost) == cudaSuccess
               ? STAG_OK
               : STAG_ERR_CUDA;
}

int net_nweights(const stag_net* net, int layer) { return net->nw[layer]; }

// ---------------------------------------------------------------- flexible CG

namespace {
// y = a x + b y (FP64, n complex entries)
__global__ void k_axpby(long n, double a, const double2* __restrict__ x, double b, double2* y) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 xv = x[i], yv = y[i];
        y[i] = make_double2(a * xv.x + b * yv.x, a * xv.y + b * yv.y);
    }
}
}  // namespace

// Solves (M_ee + shift) x = b from x = 0 by the flexible (inexact
// preconditioned) CG of Golub and Ye with z = K r (K the network; K = 1 and so
// plain CG when net is null):
//   alpha = <r,z>/<p,Ap>, x += alpha p, r -= alpha Ap, z' = K r,
//   beta = <z', r - r_old>/<z, r_old>, p = z' + beta p.
// FP64 vectors, FP64-accurate float-float operator.  The recursion stops on
// its own residual; the true residual b - A x is then computed and, if it is
// still above tol, replaces the recursive one and the recursion restarts from
// x with a target half as large (residual replacement; at most 8 restarts).
int fcg_solve(stag_ctx* ctx, stag_net* net, double mass, double shift, const double2* b, double2* x, double tol,
              int maxit, int* iters, double* true_resid, cudaStream_t s) {
    const long n3 = 3L * ctx->g.Vh;
    const size_t vb = sizeof(double2) * n3;
    double2* buf = (double2*)ws_get(ctx, WS_FCG, vb * 7);
    if (!buf) return stag_fail(ctx, STAG_ERR_OOM, "fcg workspace");
    double2 *r = buf, *rold = buf + n3, *z = buf + 2 * n3, *p = buf + 3 * n3, *w = buf + 4 * n3, *t = buf + 5 * n3,
            *zz = buf + 6 * n3;
    const double c = mass * mass + shift;
    const int nb = ctx->num_sms * 4;
    double* d = ctx->dscal + 200;
    double* hd = ctx->hscal + 200;
    auto dot = [&](const double2* a, const double2* bb, int slot) { return blas_dot_re(ctx, STAG_PREC_F64, a, bb, d + slot, s); };
    auto fetch = [&](int nslots) -> int {
        STAG_CUDA(ctx, cudaMemcpyAsync(hd, d, sizeof(double) * nslots, cudaMemcpyDeviceToHost, s));
        STAG_CUDA(ctx, cudaStreamSynchronize(s));
        return STAG_OK;
    };
    auto apply_K = [&](const double2* in, double2* out) -> int {
        if (net) return net_apply(net, in, out, s);
        STAG_CUDA(ctx, cudaMemcpyAsync(out, in, vb, cudaMemcpyDeviceToDevice, s));
        return STAG_OK;
    };
    int st;
    STAG_CUDA(ctx, cudaMemsetAsync(x, 0, vb, s));
    STAG_CUDA(ctx, cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, s));
    if ((st = dot(b, b, 0)) || (st = fetch(1))) return st;
    const double bb = hd[0];
    int k = 0;
    double target = tol, rr_true = bb;
    for (int restart = 0; restart <= 8 && bb > 0.0; restart++) {
        if ((st = apply_K(r, z))) return st;
        STAG_CUDA(ctx, cudaMemcpyAsync(p, z, vb, cudaMemcpyDeviceToDevice, s));
        if ((st = dot(r, z, 1)) || (st = dot(r, r, 3)) || (st = fetch(4))) return st;
        double rz = hd[1], rr = hd[3];
        while (k < maxit && rr > target * target * bb) {
            if ((st = mee_apply(ctx, STAG_PREC_F64FF, c, p, w, t, s))) return st;
            if ((st = dot(p, w, 2)) || (st = fetch(3))) return st;
            const double alpha = rz / hd[2];
            STAG_CUDA(ctx, cudaMemcpyAsync(rold, r, vb, cudaMemcpyDeviceToDevice, s));
            k_axpby<<<nb, 256, 0, s>>>(n3, alpha, p, 1.0, x);
            k_axpby<<<nb, 256, 0, s>>>(n3, -alpha, w, 1.0, r);
            ctx->nlaunch += 2;
            if ((st = apply_K(r, zz))) return st;
            // beta = <z', r - r_old> / <z, r_old>, computed as (<z',r> - <z',r_old>) / rz
            if ((st = dot(r, r, 3)) || (st = dot(zz, r, 4)) || (st = dot(zz, rold, 5)) || (st = fetch(6))) return st;
            rr = hd[3];
            const double beta = (hd[4] - hd[5]) / rz;
            rz = hd[4];
            k_axpby<<<nb, 256, 0, s>>>(n3, 1.0, zz, beta, p);
            ctx->nlaunch++;
            std::swap(z, zz);
            k++;
            if (!isfinite(rr) || !isfinite(beta))
                return stag_fail(ctx, STAG_ERR_NONFINITE, "non-finite residual in FCG");
        }
        STAG_LAUNCH_CHECK(ctx, "fcg");
        // FP64-accurate true residual; it replaces the recursive one
        if ((st = mee_apply(ctx, STAG_PREC_F64FF, c, x, w, t, s))) return st;
        k_axpby<<<nb, 256, 0, s>>>(n3, 1.0, b, -1.0, w);
        ctx->nlaunch++;
        if ((st = dot(w, w, 6)) || (st = fetch(7))) return st;
        rr_true = hd[6];
        if (rr_true <= tol * tol * bb || k >= maxit) break;
        STAG_CUDA(ctx, cudaMemcpyAsync(r, w, vb, cudaMemcpyDeviceToDevice, s));
        target *= 0.5;
    }
    *iters = k;
    *true_resid = (bb > 0.0) ? sqrt(rr_true / bb) : 0.0;
    return (*true_resid <= tol * 1.00000005) ? STAG_OK : stag_fail(ctx, STAG_ERR_NOCONV, "FCG did not converge");
}

// ---------------------------------------------------------------- C ABI

extern "C" {

int stag_net_create(stag_ctx* ctx, unsigned seed, stag_net** out) {
    if (!ctx || !out) return STAG_ERR_ARG;
    if (!ctx->gauge_loaded) return stag_fail(ctx, STAG_ERR_STATE, "no gauge field loaded");
    *out = nullptr;
    return net_create(ctx, seed, out);
}

int stag_net_destroy(stag_net* net) {
    net_destroy(net);
    return STAG_OK;
}

int stag_ctx_set_net(stag_ctx* ctx, stag_net* net) {
    if (!ctx) return STAG_ERR_ARG;
    if (net && net->ctx != ctx) return stag_fail(ctx, STAG_ERR_ARG, "network belongs to another context");
    ctx->net = net;
    return STAG_OK;
}

int stag_net_nweights(const stag_net* net, int layer, int* n) {
    if (!net || !n || layer < 0 || layer >= GC_NLAYER) return STAG_ERR_ARG;
    *n = net_nweights(net, layer);
    return STAG_OK;
}

int stag_net_get_weights(stag_net* net, int layer, float* host) {
    if (!net || !host || layer < 0 || layer >= GC_NLAYER) return STAG_ERR_ARG;
    return net_get_weights(net, layer, host);
}

int stag_net_set_weights(stag_net* net, int layer, const float* host) {
    if (!net || !host || layer < 0 || layer >= GC_NLAYER) return STAG_ERR_ARG;
    return net_set_weights(net, layer, host);
}

int stag_net_get_grads(stag_net* net, int layer, float* host) {
    if (!net || !host || layer < 0 || layer >= GC_NLAYER) return STAG_ERR_ARG;
    return net_get_grads(net, layer, host);
}

int stag_net_apply(stag_net* net, const double* in_even, double* out_even, void* stream) {
    if (!net || !in_even || !out_even || in_even == out_even) return STAG_ERR_ARG;
    return net_apply(net, (const double2*)in_even, (double2*)out_even, (cudaStream_t)stream);
}

int stag_net_loss_grad(stag_net* net, int npairs, const double* const* srcs, const double* const* sols, double* loss,
                       void* stream) {
    if (!net || npairs < 1 || !srcs || !sols || !loss) return STAG_ERR_ARG;
    return net_loss_grad(net, npairs, (const double2* const*)srcs, (const double2* const*)sols, loss,
                         (cudaStream_t)stream);
}

int stag_net_train(stag_net* net, int npairs, const double* const* srcs, const double* const* sols, int epochs,
                   int batch, double lr, double* loss, void* stream) {
    if (!net || npairs < 1 || !srcs || !sols || !loss || epochs < 1 || batch < 1 || !(lr > 0)) return STAG_ERR_ARG;
    return net_train(net, npairs, (const double2* const*)srcs, (const double2* const*)sols, epochs, batch, lr, loss,
                     (cudaStream_t)stream);
}

int stag_fcg_solve(stag_ctx* ctx, stag_net* net, double mass, double shift, const double* src, double* sol,
                   double tol, int maxit, stag_solve_info* info, void* stream) {
    if (!ctx) return STAG_ERR_ARG;
    if (!ctx->gauge_loaded) return stag_fail(ctx, STAG_ERR_STATE, "no gauge field loaded");
    if (!src || !sol || src == sol || !(tol > 0) || maxit < 1 || !(shift >= 0))
        return stag_fail(ctx, STAG_ERR_ARG, "bad FCG arguments");
    if (net && net->ctx != ctx) return stag_fail(ctx, STAG_ERR_ARG, "network belongs to another context");
    int it = 0;
    double tr = 0.0;
    const int st = fcg_solve(ctx, net, mass, shift, (const double2*)src, (double2*)sol, tol, maxit, &it, &tr,
                             (cudaStream_t)stream);
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iters = it;
        info->iters_shift[0] = it;
        info->true_resid[0] = tr;
        info->matvecs = it + 1;
        info->status = st;
    }
    return st;
}

}  // extern "C"

// blas.cu -- vector kernels over the even sites: FP64-accumulated dot
// products (warp shuffle, block, then last-block reduction), precision
// conversions and the rational combination a0 src + sum_k a_k x_k.
#include "hop.cuh"
#include "stag_internal.h"

static const int TPB = 256;

// Re <a, b> over n complex entries, accumulated in FP64
template <typename V2>
__global__ void k_dot_re(long n, const V2* __restrict__ a, const V2* __restrict__ b, double* partials,
                         unsigned int* counter, double* dst) {
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        V2 x = a[i], y = b[i];
        acc += (double)x.x * (double)y.x + (double)x.y * (double)y.y;
    }
    double bs = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
    if (last_block(counter)) finish_sum(partials, gridDim.x, dst);
}

int blas_dot_re(stag_ctx* ctx, int prec, const void* a, const void* b, double* dst, cudaStream_t s) {
    long n = 3L * ctx->g.Vh;
    int nb = ctx->num_sms * 4;
    if (prec == STAG_PREC_F64)
        k_dot_re<double2><<<nb, TPB, 0, s>>>(n, (const double2*)a, (const double2*)b, ctx->partials, ctx->counter, dst);
    else
        k_dot_re<float2><<<nb, TPB, 0, s>>>(n, (const float2*)a, (const float2*)b, ctx->partials, ctx->counter, dst);
    STAG_LAUNCH_CHECK(ctx, "dot_re");
    return STAG_OK;
}

__global__ void k_d2f(long n, const double2* __restrict__ in, float2* out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 v = in[i];
        out[i] = make_float2((float)v.x, (float)v.y);
    }
}
__global__ void k_f2d(long n, const float2* __restrict__ in, double2* out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        float2 v = in[i];
        out[i] = make_double2(v.x, v.y);
    }
}

int blas_copy_d2f(stag_ctx* ctx, const double2* in, float2* out, long nsites, cudaStream_t s) {
    k_d2f<<<ctx->num_sms * 4, TPB, 0, s>>>(3 * nsites, in, out);
    STAG_LAUNCH_CHECK(ctx, "d2f");
    return STAG_OK;
}
int blas_copy_f2d(stag_ctx* ctx, const float2* in, double2* out, long nsites, cudaStream_t s) {
    k_f2d<<<ctx->num_sms * 4, TPB, 0, s>>>(3 * nsites, in, out);
    STAG_LAUNCH_CHECK(ctx, "f2d");
    return STAG_OK;
}

struct RatCoef {
    double a0;
    double a[STAG_MAXSHIFT];
    int n;
};

__global__ void k_rational_combine(long n, RatCoef rc, const double2* __restrict__ src,
                                   const double2* __restrict__ x, long stride, double2* out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 v = src[i];
        double re = rc.a0 * v.x, im = rc.a0 * v.y;
        for (int k = 0; k < rc.n; k++) {
            double2 y = x[k * stride + i];
            re += rc.a[k] * y.x;
            im += rc.a[k] * y.y;
        }
        out[i] = make_double2(re, im);
    }
}

int blas_rational_combine(stag_ctx* ctx, double a0, const double* a, int n, const double2* src,
                          const double2* x, double2* out, cudaStream_t s) {
    RatCoef rc;
    rc.a0 = a0;
    rc.n = n;
    for (int k = 0; k < n; k++) rc.a[k] = a[k];
    long m = 3L * ctx->g.Vh;
    k_rational_combine<<<ctx->num_sms * 4, TPB, 0, s>>>(m, rc, src, x, m, out);
    STAG_LAUNCH_CHECK(ctx, "rational_combine");
    return STAG_OK;
}

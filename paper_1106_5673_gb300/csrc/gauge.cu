// gauge.cu -- gauge-field kernels: layout conversion, plaquette and Wilson
// action, gauge force, FP64 link update with reunitarisation, momentum
// update, Philox heatbath.  One thread per site or per link (Sec. 3 of the
// paper: "a different thread ... to every link in the gauge update").
#include "stag_internal.h"

static const int TPB = 256;

// ---------------------------------------------------------------- layout conversion

__global__ void k_gauge_from_canonical(Geom g, const double* __restrict__ in, double2* U64, float4* U32, float4* U32lo,
                                       uint2* U16) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    int mu = i / g.V, lex = i % g.V;
    const double* p = in + (size_t)i * 18;
    Mat3<double> u;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) u.e[a][b] = cmk(p[2 * (3 * a + b)], p[2 * (3 * a + b) + 1]);
    int par = par_of_lex(g, lex);
    store_link64(U64, g, mu, par, lex >> 1, u);
    store_link_lowp(U32, U32lo, U16, g, mu, par, lex >> 1, u);
}

__global__ void k_gauge_to_canonical(Geom g, const double2* __restrict__ U64, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    int mu = i / g.V, lex = i % g.V;
    Mat3<double> u = load_link64(U64, g, mu, par_of_lex(g, lex), lex >> 1);
    double* p = out + (size_t)i * 18;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            p[2 * (3 * a + b)] = u.e[a][b].re;
            p[2 * (3 * a + b) + 1] = u.e[a][b].im;
        }
}

// momenta: canonical [mu][lex][8] <-> internal [mu][par][8][Vh]
__global__ void k_mom_from_canonical(Geom g, const double* __restrict__ in, double* mom) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    int mu = i / g.V, lex = i % g.V;
    int par = par_of_lex(g, lex), h = lex >> 1;
    double* q = mom + (size_t)(mu * 2 + par) * 8 * g.Vh + h;
#pragma unroll
    for (int a = 0; a < 8; a++) q[(size_t)a * g.Vh] = in[(size_t)i * 8 + a];
}

__global__ void k_mom_to_canonical(Geom g, const double* __restrict__ mom, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    int mu = i / g.V, lex = i % g.V;
    int par = par_of_lex(g, lex), h = lex >> 1;
    const double* q = mom + (size_t)(mu * 2 + par) * 8 * g.Vh + h;
#pragma unroll
    for (int a = 0; a < 8; a++) out[(size_t)i * 8 + a] = q[(size_t)a * g.Vh];
}

int gauge_from_canonical(stag_ctx* ctx, const double* dev_links, cudaStream_t s) {
    ctx->gauge_gen++;
    k_gauge_from_canonical<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, dev_links, ctx->U64, ctx->U32, ctx->U32lo,
                                                                      ctx->U16);
    STAG_LAUNCH_CHECK(ctx, "gauge_from_canonical");
    return STAG_OK;
}
int gauge_to_canonical(stag_ctx* ctx, double* dev_links, cudaStream_t s) {
    k_gauge_to_canonical<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, ctx->U64, dev_links);
    STAG_LAUNCH_CHECK(ctx, "gauge_to_canonical");
    return STAG_OK;
}
int momenta_from_canonical(stag_ctx* ctx, const double* dev_w, cudaStream_t s) {
    k_mom_from_canonical<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, dev_w, ctx->mom);
    STAG_LAUNCH_CHECK(ctx, "momenta_from_canonical");
    return STAG_OK;
}
int momenta_to_canonical(stag_ctx* ctx, const double* src, double* dev_w, cudaStream_t s) {
    k_mom_to_canonical<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, src, dev_w);
    STAG_LAUNCH_CHECK(ctx, "momenta_to_canonical");
    return STAG_OK;
}

// ---------------------------------------------------------------- link access by lex

template <typename R> STAG_D Mat3<R> lnk(const void* U, const Geom& g, int mu, int lex);
template <> STAG_D Mat3<double> lnk<double>(const void* U, const Geom& g, int mu, int lex) {
    return load_link64((const double2*)U, g, mu, par_of_lex(g, lex), lex >> 1);
}
template <> STAG_D Mat3<float> lnk<float>(const void* U, const Geom& g, int mu, int lex) {
    return load_link32((const float4*)U, g, mu, par_of_lex(g, lex), lex >> 1);
}

STAG_D int shift_lex(const Geom& g, int lex, int mu, int dir) { return nb_lex(g, site_from_lex(g, lex), mu, dir); }

// ---------------------------------------------------------------- plaquette

__global__ void k_plaquette(Geom g, const double2* __restrict__ U, double* partials, unsigned int* counter,
                            double* dst) {
    int lex = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (lex < g.V) {
        for (int mu = 0; mu < 4; mu++) {
            Mat3<double> a = lnk<double>(U, g, mu, lex);
            int lmu = shift_lex(g, lex, mu, 1);
            for (int nu = mu + 1; nu < 4; nu++) {
                Mat3<double> b = lnk<double>(U, g, nu, lmu);
                Mat3<double> c = lnk<double>(U, g, mu, shift_lex(g, lex, nu, 1));
                Mat3<double> d = lnk<double>(U, g, nu, lex);
                // Re Tr (a b c^dag d^dag) = Re Tr ((a b) (d c)^dag)
                Mat3<double> ab = mmul(a, b), dc = mmul(d, c);
                double t = 0.0;
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++) t += ab.e[i][j].re * dc.e[i][j].re + ab.e[i][j].im * dc.e[i][j].im;
                acc += t / 3.0;
            }
        }
    }
    double bs = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
    if (last_block(counter)) finish_sum(partials, gridDim.x, dst);
}

int plaquette_sum(stag_ctx* ctx, double* dst, cudaStream_t s) {
    k_plaquette<<<nblocks(ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, ctx->U64, ctx->partials, ctx->counter, dst);
    STAG_LAUNCH_CHECK(ctx, "plaquette");
    return STAG_OK;
}

// ---------------------------------------------------------------- kinetic term

__global__ void k_kinetic(long n, const double* __restrict__ mom, double* partials, unsigned int* counter,
                          double* dst) {
    double acc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double w = mom[i];
        acc += w * w;
    }
    double bs = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
    if (last_block(counter)) {
        finish_sum(partials, gridDim.x, dst);
        if (threadIdx.x == 0) *dst *= 0.5;
    }
}

int kinetic_sum(stag_ctx* ctx, double* dst, cudaStream_t s) {
    long n = 32L * ctx->g.Vh * 2;
    k_kinetic<<<ctx->num_sms * 4, TPB, 0, s>>>(n, ctx->mom, ctx->partials, ctx->counter, dst);
    STAG_LAUNCH_CHECK(ctx, "kinetic");
    return STAG_OK;
}

// ---------------------------------------------------------------- gauge force

// sum of the six staples attached to U_mu(n) (lex), such that
// sum over plaquettes containing U_mu(n) of Re Tr U_P = Re Tr (U_mu(n) A)
template <typename R> STAG_D Mat3<R> staples(const void* U, const Geom& g, int mu, int lex) {
    Mat3<R> A = mzero<R>();
    const int lmu = shift_lex(g, lex, mu, 1);
#pragma unroll 1
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        const int lnu = shift_lex(g, lex, nu, 1), lmnu = shift_lex(g, lex, nu, -1);
        const int lmu_mnu = shift_lex(g, lmu, nu, -1);
        // U_nu(n+mu) U_mu(n+nu)^dag U_nu(n)^dag
        Mat3<R> a = lnk<R>(U, g, nu, lmu), b = lnk<R>(U, g, mu, lnu), c = lnk<R>(U, g, nu, lex);
        A = madd(A, mmuld(mmuld(a, b), c));
        // U_nu(n+mu-nu)^dag U_mu(n-nu)^dag U_nu(n-nu)
        Mat3<R> d = lnk<R>(U, g, nu, lmu_mnu), e = lnk<R>(U, g, mu, lmnu), f = lnk<R>(U, g, nu, lmnu);
        A = madd(A, mdmul(mmul(e, d), f));
    }
    return A;
}

template <typename R> STAG_D Mat3<double> to64(const Mat3<R>& m) {
    Mat3<double> r;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.e[i][j] = cmk((double)m.e[i][j].re, (double)m.e[i][j].im);
    return r;
}

// F[mu][par][a][h] (+)= (beta/6) * omega(i TA(U A)):  dP/dtau = (i beta/6) TA(U_mu(n) A_mu(n))
template <typename R>
__global__ void k_gauge_force(Geom g, const void* __restrict__ U, double beta, double* F, int accumulate) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    int mu = i / g.V, lex = i % g.V;
    Mat3<R> A = staples<R>(U, g, mu, lex);
    Mat3<R> W = mmul(lnk<R>(U, g, mu, lex), A);
    double f[8];
    i_ta_to_omega(to64(W), f);
    int par = par_of_lex(g, lex), h = lex >> 1;
    double* q = F + (size_t)(mu * 2 + par) * 8 * g.Vh + h;
    const double c = beta / 6.0;
#pragma unroll
    for (int a = 0; a < 8; a++) {
        double v = c * f[a];
        q[(size_t)a * g.Vh] = accumulate ? q[(size_t)a * g.Vh] + v : v;
    }
}

int gauge_force_internal_prec(stag_ctx* ctx, double beta, double* F, int accumulate, int prec32, cudaStream_t s) {
    if (prec32)
        k_gauge_force<float><<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, ctx->U32, beta, F, accumulate);
    else
        k_gauge_force<double><<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, ctx->U64, beta, F, accumulate);
    STAG_LAUNCH_CHECK(ctx, "gauge_force");
    return STAG_OK;
}
int gauge_force_internal(stag_ctx* ctx, double beta, double* F, int accumulate, cudaStream_t s) {
    return gauge_force_internal_prec(ctx, beta, F, accumulate, 0, s);
}

// ---------------------------------------------------------------- SU(3) exponential and link update

// exp(iQ) for traceless Hermitian Q by the Cayley-Hamilton theorem
// (Morningstar and Peardon, Phys. Rev. D 69 (2004) 054501):
//   exp(iQ) = f0 + f1 Q + f2 Q^2,  c0 = Tr Q^3 / 3,  c1 = Tr Q^2 / 2,
//   theta = arccos(c0 / c0max), c0max = 2 (c1/3)^{3/2},
//   u = sqrt(c1/3) cos(theta/3),  w = sqrt(c1) sin(theta/3),
//   f_j = h_j / (9u^2 - w^2) with
//   h0 = (u^2 - w^2) e^{2iu} + e^{-iu} (8u^2 cos w + 2iu (3u^2 + w^2) xi0(w))
//   h1 = 2u e^{2iu} - e^{-iu} (2u cos w - i (3u^2 - w^2) xi0(w))
//   h2 = e^{2iu} - e^{-iu} (cos w + 3iu xi0(w)),   xi0(w) = sin(w)/w,
// evaluated at |c0| and conjugated with sign (-1)^j for c0 < 0.
STAG_D Mat3<double> expi_ch(const Mat3<double>& Q) {
    Mat3<double> Q2 = mmul(Q, Q);
    double c1 = 0.5 * (Q2.e[0][0].re + Q2.e[1][1].re + Q2.e[2][2].re);
    Mat3<double> Q3 = mmul(Q2, Q);
    double c0 = (Q3.e[0][0].re + Q3.e[1][1].re + Q3.e[2][2].re) / 3.0;
    Mat3<double> E;
    if (c1 < 1e-30) {  // Q ~ 0: exp(iQ) = 1 + iQ - Q^2/2
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                E.e[i][j] = cmk((i == j ? 1.0 : 0.0) - Q.e[i][j].im - 0.5 * Q2.e[i][j].re,
                                Q.e[i][j].re - 0.5 * Q2.e[i][j].im);
        return E;
    }
    const bool neg = c0 < 0;
    const double ac0 = fabs(c0);
    const double c0max = 2.0 * pow(c1 / 3.0, 1.5);
    double ratio = ac0 / c0max;
    ratio = ratio > 1.0 ? 1.0 : ratio;
    const double theta = acos(ratio);
    const double u = sqrt(c1 / 3.0) * cos(theta / 3.0);
    const double w = sqrt(c1) * sin(theta / 3.0);
    const double u2 = u * u, w2 = w * w;
    double xi0;
    if (fabs(w) < 0.05) {
        xi0 = 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0));
    } else {
        xi0 = sin(w) / w;
    }
    const double cw = cos(w);
    double s2u, c2u, su, cu;
    sincos(2.0 * u, &s2u, &c2u);
    sincos(u, &su, &cu);
    const cd e2iu = cmk(c2u, s2u), emiu = cmk(cu, -su);
    const cd h0 = (u2 - w2) * e2iu + emiu * cmk(8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0);
    const cd h1 = (2.0 * u) * e2iu - emiu * cmk(2.0 * u * cw, -(3.0 * u2 - w2) * xi0);
    const cd h2 = e2iu - emiu * cmk(cw, 3.0 * u * xi0);
    const double den = 1.0 / (9.0 * u2 - w2);
    cd f0 = den * h0, f1 = den * h1, f2 = den * h2;
    if (neg) {
        f0 = conj(f0);
        f1 = cmk(-f1.re, f1.im);  // -(conj f1)
        f2 = conj(f2);
    }
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cd v = f1 * Q.e[i][j] + f2 * Q2.e[i][j];
            if (i == j) v = v + f0;
            E.e[i][j] = v;
        }
    return E;
}

// Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1)
STAG_D void reunitarize(Mat3<double>& u) {
    double n0 = norm2(u.e[0][0]) + norm2(u.e[0][1]) + norm2(u.e[0][2]);
    n0 = rsqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; j++) u.e[0][j] = n0 * u.e[0][j];
    cd d = cjmul(u.e[0][0], u.e[1][0]) + cjmul(u.e[0][1], u.e[1][1]) + cjmul(u.e[0][2], u.e[1][2]);
#pragma unroll
    for (int j = 0; j < 3; j++) u.e[1][j] = u.e[1][j] - d * u.e[0][j];
    double n1 = norm2(u.e[1][0]) + norm2(u.e[1][1]) + norm2(u.e[1][2]);
    n1 = rsqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; j++) u.e[1][j] = n1 * u.e[1][j];
    recon_row2(u);
}

// U <- exp(i eps P) U, reunitarised, in FP64; refreshes the FP32/BF16 copies
__global__ void k_update_links(Geom g, double eps, const double* __restrict__ mom, double2* U64, float4* U32, float4* U32lo,
                               uint2* U16) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    // i enumerates the internal order [mu][par][h]
    int h = i % g.Vh;
    int mp = i / g.Vh;
    int mu = mp >> 1, par = mp & 1;
    const double* q = mom + (size_t)mp * 8 * g.Vh + h;
    double w[8];
#pragma unroll
    for (int a = 0; a < 8; a++) w[a] = eps * q[(size_t)a * g.Vh];
    Mat3<double> E = expi_ch(omega_to_herm(w));
    Mat3<double> u = load_link64(U64, g, mu, par, h);
    Mat3<double> nu = mmul(E, u);
    reunitarize(nu);
    store_link64(U64, g, mu, par, h, nu);
    store_link_lowp(U32, U32lo, U16, g, mu, par, h, nu);
}

int update_links(stag_ctx* ctx, double eps, cudaStream_t s) {
    ctx->gauge_gen++;
    k_update_links<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, eps, ctx->mom, ctx->U64, ctx->U32, ctx->U32lo,
                                                              ctx->U16);
    STAG_LAUNCH_CHECK(ctx, "update_links");
    return STAG_OK;
}

// rebuild the FP32/BF16 copies from the FP64 master (after a Metropolis reject)
__global__ void k_refresh_lowp(Geom g, const double2* __restrict__ U64, float4* U32, float4* U32lo, uint2* U16) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    int h = i % g.Vh, mp = i / g.Vh;
    Mat3<double> u = load_link64(U64, g, mp >> 1, mp & 1, h);
    store_link_lowp(U32, U32lo, U16, g, mp >> 1, mp & 1, h, u);
}

int refresh_lowp_links(stag_ctx* ctx, cudaStream_t s) {
    ctx->gauge_gen++;
    k_refresh_lowp<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, ctx->U64, ctx->U32, ctx->U32lo, ctx->U16);
    STAG_LAUNCH_CHECK(ctx, "refresh_lowp");
    return STAG_OK;
}

// 8-real FP32 copy of one link from the FP64 master: a1, a2, b0 rounded to
// FP32, the phases of a0 and c0 from atan2 in FP64 (c0 from the rebuilt third
// row)
__global__ void k_build_r8(Geom g, const double2* __restrict__ U64, float4* U8) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    const int h = i % g.Vh, mp = i / g.Vh;
    const Mat3<double> u = load_link64(U64, g, mp >> 1, mp & 1, h);
    float4* p = U8 + (size_t)mp * 2 * g.Vh + h;
    p[0] = make_float4((float)u.e[0][1].re, (float)u.e[0][1].im, (float)u.e[0][2].re, (float)u.e[0][2].im);
    p[g.Vh] = make_float4((float)u.e[1][0].re, (float)u.e[1][0].im, (float)atan2(u.e[0][0].im, u.e[0][0].re),
                          (float)atan2(u.e[2][0].im, u.e[2][0].re));
}

const float4* links_r8(stag_ctx* ctx, cudaStream_t s) {
    if (!ctx->U8) {
        if (cudaMalloc((void**)&ctx->U8, sizeof(float4) * 16 * (size_t)ctx->g.Vh) != cudaSuccess) {
            cudaGetLastError();
            ctx->U8 = nullptr;
            stag_fail(ctx, STAG_ERR_OOM, "8-real links");
            return nullptr;
        }
        ctx->u8_gen = ctx->gauge_gen - 1;
    }
    if (ctx->u8_gen != ctx->gauge_gen) {
        k_build_r8<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, ctx->U64, ctx->U8);
        if (stag_cuda_check(ctx, cudaGetLastError(), "build 8-real links") != STAG_OK) return nullptr;
        ctx->nlaunch++;
        ctx->u8_gen = ctx->gauge_gen;
    }
    return ctx->U8;
}

__global__ void k_axpy_mom(long n, double eps, const double* __restrict__ F, double* mom) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        mom[i] += eps * F[i];
}

int update_momenta(stag_ctx* ctx, const double* F, double eps, cudaStream_t s) {
    long n = 64L * ctx->g.Vh;
    k_axpy_mom<<<ctx->num_sms * 8, TPB, 0, s>>>(n, eps, F, ctx->mom);
    STAG_LAUNCH_CHECK(ctx, "update_momenta");
    return STAG_OK;
}

// ---------------------------------------------------------------- Philox4x32-10 heatbath
// Salmon, Moraes, Dror, Shaw (SC'11): 10 rounds of the Philox S-box with
// multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,
// 0xBB67AE85.  Two 53-bit uniforms in (0,1] per call, Box-Muller to Gaussians.

STAG_D uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

STAG_D double2 uniform2(uint4 c, uint2 k) {
    uint4 o = philox10(c, k);
    unsigned long long a = ((unsigned long long)o.x << 21) | (o.y >> 11);
    unsigned long long b = ((unsigned long long)o.z << 21) | (o.w >> 11);
    return make_double2(((double)a + 1.0) * 0x1p-53, ((double)b + 1.0) * 0x1p-53);
}

STAG_D double2 gauss2(uint4 c, uint2 k) {
    double2 u = uniform2(c, k);
    double rad = sqrt(-2.0 * log(u.x));
    double sn, cs;
    sincos(6.283185307179586476925 * u.y, &sn, &cs);
    return make_double2(rad * cs, rad * sn);
}

__global__ void k_mom_heatbath(Geom g, uint32_t seed, uint32_t traj, double* mom) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * g.V) return;
    int mu = i / g.V, lex = i % g.V;
    int par = par_of_lex(g, lex), h = lex >> 1;
    double* q = mom + (size_t)(mu * 2 + par) * 8 * g.Vh + h;
    uint2 key = make_uint2(seed, traj);
#pragma unroll
    for (int b = 0; b < 4; b++) {
        double2 z = gauss2(make_uint4(1u, (uint32_t)mu, (uint32_t)lex, (uint32_t)b), key);
        q[(size_t)(2 * b) * g.Vh] = z.x;
        q[(size_t)(2 * b + 1) * g.Vh] = z.y;
    }
}

int momenta_heatbath(stag_ctx* ctx, uint32_t seed, uint32_t traj, cudaStream_t s) {
    k_mom_heatbath<<<nblocks(4L * ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, seed, traj, ctx->mom);
    STAG_LAUNCH_CHECK(ctx, "momenta_heatbath");
    return STAG_OK;
}

__global__ void k_pf_gaussian(Geom g, uint32_t seed, uint32_t traj, int pf, double2* out) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    Site s = site_of(g, h, 0);
    uint2 key = make_uint2(seed, traj);
    const double r = 0.70710678118654752440;  // sqrt(1/2): density exp(-|R|^2)
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double2 z = gauss2(make_uint4(2u, (uint32_t)pf, (uint32_t)s.lex, (uint32_t)c), key);
        out[3 * (size_t)h + c] = make_double2(r * z.x, r * z.y);
    }
}

int pf_gaussian(stag_ctx* ctx, uint32_t seed, uint32_t traj, int pf, double2* out, cudaStream_t s) {
    k_pf_gaussian<<<nblocks(ctx->g.Vh, TPB), TPB, 0, s>>>(ctx->g, seed, traj, pf, out);
    STAG_LAUNCH_CHECK(ctx, "pf_gaussian");
    return STAG_OK;
}

__global__ void k_metro_uniform(uint32_t seed, uint32_t traj, double* dst) {
    double2 u = uniform2(make_uint4(3u, 0u, 0u, 0u), make_uint2(seed, traj));
    *dst = u.x;
}

int metro_uniform(stag_ctx* ctx, uint32_t seed, uint32_t traj, double* dst, cudaStream_t s) {
    k_metro_uniform<<<1, 1, 0, s>>>(seed, traj, dst);
    STAG_LAUNCH_CHECK(ctx, "metro_uniform");
    return STAG_OK;
}

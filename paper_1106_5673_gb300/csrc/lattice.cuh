// lattice.cuh -- device-side geometry, complex/SU(3) arithmetic and the
// internal structure-of-arrays layouts of the GB300 staggered library.
//
// Internal layouts (all arrays 16-byte aligned, Vh = V/2 sites per parity):
//   links, FP64  double2 [mu][parity][6][Vh]   rows 0,1 of U_mu(n): u00 u01 u02 u10 u11 u12
//   links, FP32  float4  [mu][parity][3][Vh]   (u00,u01) (u02,u10) (u11,u12)
//   links, BF16  uint2   [mu][parity][3][Vh]   same pairs, 4 bf16 per 8 bytes
//   momenta      double  [mu][parity][8][Vh]   Gell-Mann coefficients w^a
//   vectors      complex [Vh][3]               canonical, AoS (same as the C ABI)
// The third link row is rebuilt on the fly as conj(row0 x row1), which holds
// for SU(3) (12-real storage of Sec. 4.2).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define STAG_HD __host__ __device__ __forceinline__
#define STAG_D __device__ __forceinline__

struct Geom {
    int L[4];
    int V, Vh;
    int Lx2;  // Lx/2, the x-extent in half-site units
    // n / L[m] = high 64 bits of n * mag[m], mag[m] = floor((2^64 - 1) / L[m]) + 1:
    // exact for 0 <= n < 2^64 / L[m] (for L[m] a power of two mag = 2^64 / L;
    // otherwise mag overestimates 2^64 / L by less than one, an error
    // n / 2^64 < 1 / L that cannot carry the quotient past an integer)
    unsigned long long mag[3];
};

// fills the geometry of a lattice with extents dims (each even, V < 2^29)
STAG_HD void geom_init(Geom& g, const int dims[4]) {
    long long V = 1;
    for (int m = 0; m < 4; m++) {
        g.L[m] = dims[m];
        V *= dims[m];
    }
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.Lx2 = dims[0] / 2;
    for (int m = 0; m < 3; m++) g.mag[m] = (~0ull) / (unsigned long long)dims[m] + 1ull;
}

// n / L[m] for 0 <= n < 2^31
STAG_D int gdiv(const Geom& g, int m, int n) {
    return (int)__umul64hi((unsigned long long)(unsigned)n, g.mag[m]);
}

// ---------------------------------------------------------------- complex

template <typename R> struct Cplx { R re, im; };
typedef Cplx<double> cd;
typedef Cplx<float> cf;

template <typename R> STAG_HD Cplx<R> cmk(R a, R b) { Cplx<R> c; c.re = a; c.im = b; return c; }
template <typename R> STAG_HD Cplx<R> operator+(Cplx<R> a, Cplx<R> b) { return cmk(a.re + b.re, a.im + b.im); }
template <typename R> STAG_HD Cplx<R> operator-(Cplx<R> a, Cplx<R> b) { return cmk(a.re - b.re, a.im - b.im); }
template <typename R> STAG_HD Cplx<R> operator*(Cplx<R> a, Cplx<R> b) {
    return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> STAG_HD Cplx<R> operator*(R s, Cplx<R> a) { return cmk(s * a.re, s * a.im); }
template <typename R> STAG_HD Cplx<R> conj(Cplx<R> a) { return cmk(a.re, -a.im); }
// a^* b
template <typename R> STAG_HD Cplx<R> cjmul(Cplx<R> a, Cplx<R> b) {
    return cmk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <typename R> STAG_HD R norm2(Cplx<R> a) { return a.re * a.re + a.im * a.im; }

// colour vector and 3x3 matrix
template <typename R> struct Vec3 { Cplx<R> c[3]; };
template <typename R> struct Mat3 { Cplx<R> e[3][3]; };

template <typename R> STAG_HD Vec3<R> vzero() {
    Vec3<R> v;
#pragma unroll
    for (int i = 0; i < 3; i++) v.c[i] = cmk<R>(0, 0);
    return v;
}

// rebuild row 2 = conj(row0 x row1) (SU(3), det = 1): entry c is
// conj(a b - x y) with a = u0[c+1], b = u1[c+2], x = u0[c+2], y = u1[c+1]
// (indices mod 3), each real part one multiply and three fused multiply-adds
template <typename R> STAG_HD void recon_row2(Mat3<R>& u) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int i1 = (c + 1) % 3, i2 = (c + 2) % 3;
        const Cplx<R> a = u.e[0][i1], b = u.e[1][i2], x = u.e[0][i2], y = u.e[1][i1];
        R re = a.re * b.re;
        re = fma(-a.im, b.im, re);
        re = fma(-x.re, y.re, re);
        re = fma(x.im, y.im, re);
        R im = -(a.re * b.im);
        im = fma(-a.im, b.re, im);
        im = fma(x.re, y.im, im);
        im = fma(x.im, y.re, im);
        u.e[2][c] = cmk(re, im);
    }
}

template <typename R> STAG_HD Mat3<R> mmul(const Mat3<R>& a, const Mat3<R>& b) {
    Mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            c.e[i][j] = a.e[i][0] * b.e[0][j] + a.e[i][1] * b.e[1][j] + a.e[i][2] * b.e[2][j];
    return c;
}
// a^dag b
template <typename R> STAG_HD Mat3<R> mdmul(const Mat3<R>& a, const Mat3<R>& b) {
    Mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            c.e[i][j] = cjmul(a.e[0][i], b.e[0][j]) + cjmul(a.e[1][i], b.e[1][j]) +
                        cjmul(a.e[2][i], b.e[2][j]);
    return c;
}
// a b^dag
template <typename R> STAG_HD Mat3<R> mmuld(const Mat3<R>& a, const Mat3<R>& b) {
    Mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            c.e[i][j] = cjmul(b.e[j][0], a.e[i][0]) + cjmul(b.e[j][1], a.e[i][1]) +
                        cjmul(b.e[j][2], a.e[i][2]);
    return c;
}
template <typename R> STAG_HD Mat3<R> madd(const Mat3<R>& a, const Mat3<R>& b) {
    Mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.e[i][j] = a.e[i][j] + b.e[i][j];
    return c;
}
template <typename R> STAG_HD Mat3<R> mzero() {
    Mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.e[i][j] = cmk<R>(0, 0);
    return c;
}

// ---------------------------------------------------------------- Hermitian / algebra
// P = sum_a w^a lambda^a / 2 (Gell-Mann), as the 3x3 matrix
//   P00 = (w3 + w8/sqrt3)/2, P11 = (-w3 + w8/sqrt3)/2, P22 = -w8/sqrt3,
//   P01 = (w1 - i w2)/2, P02 = (w4 - i w5)/2, P12 = (w6 - i w7)/2.
#define STAG_INV_SQRT3 0.57735026918962576451

STAG_HD Mat3<double> omega_to_herm(const double w[8]) {
    Mat3<double> P;
    const double s = STAG_INV_SQRT3;
    P.e[0][0] = cmk(0.5 * (w[2] + w[7] * s), 0.0);
    P.e[1][1] = cmk(0.5 * (-w[2] + w[7] * s), 0.0);
    P.e[2][2] = cmk(-w[7] * s, 0.0);
    P.e[0][1] = cmk(0.5 * w[0], -0.5 * w[1]);
    P.e[1][0] = cmk(0.5 * w[0], 0.5 * w[1]);
    P.e[0][2] = cmk(0.5 * w[3], -0.5 * w[4]);
    P.e[2][0] = cmk(0.5 * w[3], 0.5 * w[4]);
    P.e[1][2] = cmk(0.5 * w[5], -0.5 * w[6]);
    P.e[2][1] = cmk(0.5 * w[5], 0.5 * w[6]);
    return P;
}

// For W, returns the Gell-Mann coefficients f^a of i TA(W) = sum_a f^a lambda^a/2,
// TA(W) = (W - W^dag)/2 - Tr(W - W^dag)/6.  With A = TA(W) anti-Hermitian
// traceless, i A is Hermitian and f^a = Tr(i A lambda^a).
STAG_HD void i_ta_to_omega(const Mat3<double>& W, double f[8]) {
    // A_ij = (W_ij - conj(W_ji))/2 - trace part;  (iA)_ij = i A_ij
    // f1 = 2 Re (iA)_01, f2 = -2 Im (iA)_01 ... written out from Tr(iA lambda^a)
    const double a01r = 0.5 * (W.e[0][1].re - W.e[1][0].re), a01i = 0.5 * (W.e[0][1].im + W.e[1][0].im);
    const double a02r = 0.5 * (W.e[0][2].re - W.e[2][0].re), a02i = 0.5 * (W.e[0][2].im + W.e[2][0].im);
    const double a12r = 0.5 * (W.e[1][2].re - W.e[2][1].re), a12i = 0.5 * (W.e[1][2].im + W.e[2][1].im);
    // diagonal of A is i*Im(W_kk) minus i*tr/3
    const double d0 = W.e[0][0].im, d1 = W.e[1][1].im, d2 = W.e[2][2].im;
    const double tr = (d0 + d1 + d2) / 3.0;
    const double h0 = -(d0 - tr), h1 = -(d1 - tr);  // (iA)_kk = i * i (d_k - tr) = -(d_k - tr)
    // (iA)_01 = i (a01r + i a01i) = -a01i + i a01r ; (iA)_10 = conj
    // Tr(iA lambda1) = (iA)_01 + (iA)_10 = 2 Re (iA)_01 = -2 a01i
    // Tr(iA lambda2) = i (iA)_01 - i (iA)_10 = -2 Im (iA)_01 = -2 a01r
    f[0] = -2.0 * a01i;
    f[1] = -2.0 * a01r;
    f[2] = h0 - h1;
    f[3] = -2.0 * a02i;
    f[4] = -2.0 * a02r;
    f[5] = -2.0 * a12i;
    f[6] = -2.0 * a12r;
    // Tr(iA lambda8) = (h0 + h1 - 2 h2)/sqrt3, h2 = -h0 - h1
    f[7] = (h0 + h1 - 2.0 * (-h0 - h1)) * STAG_INV_SQRT3;
}

// ---------------------------------------------------------------- geometry

struct Site {
    int x[4];
    int lex;
};

// site of parity `par` with index h (lex/2): lex is 2h or 2h+1
STAG_D Site site_of(const Geom& g, int h, int par) {
    Site s;
    int lex0 = 2 * h;
    int r = gdiv(g, 0, lex0);
    int x0 = lex0 - r * g.L[0];
    int r2 = gdiv(g, 1, r);
    s.x[1] = r - r2 * g.L[1];
    s.x[3] = gdiv(g, 2, r2);
    s.x[2] = r2 - s.x[3] * g.L[2];
    int p0 = (x0 + s.x[1] + s.x[2] + s.x[3]) & 1;
    s.x[0] = x0 + (p0 != par);
    s.lex = lex0 + (p0 != par);
    return s;
}

// lex of the neighbour n + dir mu
STAG_D int nb_lex(const Geom& g, const Site& s, int mu, int dir) {
    int stride = 1;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        if (m == mu) {
            int xm = s.x[m] + dir;
            int delta = dir;
            if (xm == g.L[m]) delta = 1 - g.L[m];
            if (xm < 0) delta = g.L[m] - 1;
            return s.lex + delta * stride;
        }
        stride *= g.L[m];
    }
    return s.lex;
}

// staggered phase eta_mu(n) = (-1)^(x_0 + ... + x_{mu-1}) as +-1
STAG_D int eta(const Site& s, int mu) {
    int t = 0;
#pragma unroll
    for (int m = 0; m < 3; m++)
        if (m < mu) t += s.x[m];
    return (t & 1) ? -1 : 1;
}

// ---------------------------------------------------------------- link loads

STAG_D Mat3<double> load_link64(const double2* __restrict__ U, const Geom& g, int mu, int par, int h) {
    const double2* p = U + (size_t)(mu * 2 + par) * 6 * g.Vh + h;
    Mat3<double> u;
    double2 a0 = __ldg(p), a1 = __ldg(p + g.Vh), a2 = __ldg(p + 2 * (size_t)g.Vh);
    double2 a3 = __ldg(p + 3 * (size_t)g.Vh), a4 = __ldg(p + 4 * (size_t)g.Vh), a5 = __ldg(p + 5 * (size_t)g.Vh);
    u.e[0][0] = cmk(a0.x, a0.y); u.e[0][1] = cmk(a1.x, a1.y); u.e[0][2] = cmk(a2.x, a2.y);
    u.e[1][0] = cmk(a3.x, a3.y); u.e[1][1] = cmk(a4.x, a4.y); u.e[1][2] = cmk(a5.x, a5.y);
    recon_row2(u);
    return u;
}

STAG_D Mat3<float> load_link32(const float4* __restrict__ U, const Geom& g, int mu, int par, int h) {
    const float4* p = U + (size_t)(mu * 2 + par) * 3 * g.Vh + h;
    float4 a = __ldg(p), b = __ldg(p + g.Vh), c = __ldg(p + 2 * (size_t)g.Vh);
    Mat3<float> u;
    u.e[0][0] = cmk(a.x, a.y); u.e[0][1] = cmk(a.z, a.w);
    u.e[0][2] = cmk(b.x, b.y); u.e[1][0] = cmk(b.z, b.w);
    u.e[1][1] = cmk(c.x, c.y); u.e[1][2] = cmk(c.z, c.w);
    recon_row2(u);
    return u;
}

// 8-real FP32 links (the minimal parametrisation of SU(3) the paper
// mentions in Sec. 4.2 and leaves unbuilt): float4 [mu][parity][2][Vh] holding
// (a1, a2) and (b0, arg a0, arg c0) of U = [[a0 a1 a2] [b0 b1 b2] [c0 c1 c2]].
// The rest follows from unitarity and det U = 1 (each entry is the complex
// conjugate of its cofactor):
//   |a0|^2 = 1 - |a1|^2 - |a2|^2 = 1 - N,   |c0|^2 = N - |b0|^2,
//   c1 = (b0* a2* - a1 a0* c0) / N,          c2 = -(b0* a1* + a2 a0* c0) / N,
//   b1 = a0* c2* - a2* c0*,                  b2 = a1* c0* - a0* c1*.
// 32 bytes per link instead of 48, for some 60 extra operations (two square
// roots, two sine/cosine pairs, one reciprocal).
STAG_D Mat3<float> load_link8(const float4* __restrict__ U, const Geom& g, int mu, int par, int h) {
    const float4* p = U + (size_t)(mu * 2 + par) * 2 * g.Vh + h;
    const float4 A = __ldg(p), B = __ldg(p + g.Vh);
    Mat3<float> u;
    const Cplx<float> a1 = cmk(A.x, A.y), a2 = cmk(A.z, A.w), b0 = cmk(B.x, B.y);
    const float N = fmaf(a1.re, a1.re, fmaf(a1.im, a1.im, fmaf(a2.re, a2.re, a2.im * a2.im)));
    const float ra0 = sqrtf(fmaxf(0.f, 1.f - N));
    const float rc0 = sqrtf(fmaxf(0.f, N - fmaf(b0.re, b0.re, b0.im * b0.im)));
    float s0, c0s, s2, c2s;
    __sincosf(B.z, &s0, &c0s);
    __sincosf(B.w, &s2, &c2s);
    const Cplx<float> a0 = cmk(ra0 * c0s, ra0 * s0), c0 = cmk(rc0 * c2s, rc0 * s2);
    const float inv = 1.f / N;
    const Cplx<float> ac = conj(a0) * c0;  // a0* c0
    const Cplx<float> c1 = inv * (conj(b0) * conj(a2) - a1 * ac);
    const Cplx<float> c2 = -inv * (conj(b0) * conj(a1) + a2 * ac);
    u.e[0][0] = a0; u.e[0][1] = a1; u.e[0][2] = a2;
    u.e[1][0] = b0;
    u.e[1][1] = conj(a0) * conj(c2) - conj(a2) * conj(c0);
    u.e[1][2] = conj(a1) * conj(c0) - conj(a0) * conj(c1);
    u.e[2][0] = c0; u.e[2][1] = c1; u.e[2][2] = c2;
    return u;
}

STAG_D float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
STAG_D float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

STAG_D Mat3<float> load_link16(const uint2* __restrict__ U, const Geom& g, int mu, int par, int h) {
    const uint2* p = U + (size_t)(mu * 2 + par) * 3 * g.Vh + h;
    uint2 a = __ldg(p), b = __ldg(p + g.Vh), c = __ldg(p + 2 * (size_t)g.Vh);
    Mat3<float> u;
    u.e[0][0] = cmk(bf_lo(a.x), bf_hi(a.x)); u.e[0][1] = cmk(bf_lo(a.y), bf_hi(a.y));
    u.e[0][2] = cmk(bf_lo(b.x), bf_hi(b.x)); u.e[1][0] = cmk(bf_lo(b.y), bf_hi(b.y));
    u.e[1][1] = cmk(bf_lo(c.x), bf_hi(c.x)); u.e[1][2] = cmk(bf_lo(c.y), bf_hi(c.y));
    recon_row2(u);
    return u;
}

STAG_D void store_link64(double2* U, const Geom& g, int mu, int par, int h, const Mat3<double>& u) {
    double2* p = U + (size_t)(mu * 2 + par) * 6 * g.Vh + h;
    p[0] = make_double2(u.e[0][0].re, u.e[0][0].im);
    p[g.Vh] = make_double2(u.e[0][1].re, u.e[0][1].im);
    p[2 * (size_t)g.Vh] = make_double2(u.e[0][2].re, u.e[0][2].im);
    p[3 * (size_t)g.Vh] = make_double2(u.e[1][0].re, u.e[1][0].im);
    p[4 * (size_t)g.Vh] = make_double2(u.e[1][1].re, u.e[1][1].im);
    p[5 * (size_t)g.Vh] = make_double2(u.e[1][2].re, u.e[1][2].im);
}

STAG_D uint32_t pack_bf2(float lo, float hi) {
    __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// write the low-precision copies of one link from its FP64 rows 0,1: FP32
// (U32 = fl32(u)), its FP32 residual (U32lo = fl32(u - U32), the low word of
// the float-float pair) and BF16
STAG_D void store_link_lowp(float4* U32, float4* U32lo, uint2* U16, const Geom& g, int mu, int par, int h,
                            const Mat3<double>& u) {
    size_t base = (size_t)(mu * 2 + par) * 3 * g.Vh + h;
    const double d[12] = {u.e[0][0].re, u.e[0][0].im, u.e[0][1].re, u.e[0][1].im, u.e[0][2].re, u.e[0][2].im,
                          u.e[1][0].re, u.e[1][0].im, u.e[1][1].re, u.e[1][1].im, u.e[1][2].re, u.e[1][2].im};
    float v[12], w[12];
#pragma unroll
    for (int i = 0; i < 12; i++) {
        v[i] = __double2float_rn(d[i]);
        w[i] = __double2float_rn(d[i] - (double)v[i]);
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        U32lo[base + (size_t)j * g.Vh] = make_float4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
        U32[base + (size_t)j * g.Vh] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        U16[base + (size_t)j * g.Vh] = make_uint2(pack_bf2(v[4 * j], v[4 * j + 1]),
                                                  pack_bf2(v[4 * j + 2], v[4 * j + 3]));
    }
}

// ---------------------------------------------------------------- vector loads (AoS)

STAG_D Vec3<double> load_vec(const double2* __restrict__ v, int h) {
    const double2* p = v + 3 * (size_t)h;
    double2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    Vec3<double> r;
    r.c[0] = cmk(a.x, a.y); r.c[1] = cmk(b.x, b.y); r.c[2] = cmk(c.x, c.y);
    return r;
}
STAG_D Vec3<float> load_vec(const float2* __restrict__ v, int h) {
    const float2* p = v + 3 * (size_t)h;
    float2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    Vec3<float> r;
    r.c[0] = cmk(a.x, a.y); r.c[1] = cmk(b.x, b.y); r.c[2] = cmk(c.x, c.y);
    return r;
}
// non-cached-path load for buffers written earlier by the same kernel sequence
STAG_D Vec3<double> ld_vec(const double2* v, int h) {
    const double2* p = v + 3 * (size_t)h;
    double2 a = p[0], b = p[1], c = p[2];
    Vec3<double> r;
    r.c[0] = cmk(a.x, a.y); r.c[1] = cmk(b.x, b.y); r.c[2] = cmk(c.x, c.y);
    return r;
}
STAG_D Vec3<float> ld_vec(const float2* v, int h) {
    const float2* p = v + 3 * (size_t)h;
    float2 a = p[0], b = p[1], c = p[2];
    Vec3<float> r;
    r.c[0] = cmk(a.x, a.y); r.c[1] = cmk(b.x, b.y); r.c[2] = cmk(c.x, c.y);
    return r;
}
STAG_D void st_vec(double2* v, int h, const Vec3<double>& r) {
    double2* p = v + 3 * (size_t)h;
    p[0] = make_double2(r.c[0].re, r.c[0].im);
    p[1] = make_double2(r.c[1].re, r.c[1].im);
    p[2] = make_double2(r.c[2].re, r.c[2].im);
}
STAG_D void st_vec(float2* v, int h, const Vec3<float>& r) {
    float2* p = v + 3 * (size_t)h;
    p[0] = make_float2(r.c[0].re, r.c[0].im);
    p[1] = make_float2(r.c[1].re, r.c[1].im);
    p[2] = make_float2(r.c[2].re, r.c[2].im);
}

// acc += U v and acc += U^dag v as chains of fused multiply-adds (four per
// complex product, the accumulation folded in)
template <typename R> STAG_D void mv_acc(Vec3<R>& acc, const Mat3<R>& u, const Vec3<R>& v) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R re = acc.c[a].re, im = acc.c[a].im;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            re = fma(u.e[a][c].re, v.c[c].re, re);
            re = fma(-u.e[a][c].im, v.c[c].im, re);
            im = fma(u.e[a][c].re, v.c[c].im, im);
            im = fma(u.e[a][c].im, v.c[c].re, im);
        }
        acc.c[a] = cmk(re, im);
    }
}
template <typename R> STAG_D void mdv_acc(Vec3<R>& acc, const Mat3<R>& u, const Vec3<R>& v) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R re = acc.c[a].re, im = acc.c[a].im;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            re = fma(u.e[c][a].re, v.c[c].re, re);
            re = fma(u.e[c][a].im, v.c[c].im, re);
            im = fma(u.e[c][a].re, v.c[c].im, im);
            im = fma(-u.e[c][a].im, v.c[c].re, im);
        }
        acc.c[a] = cmk(re, im);
    }
}
// s v for a sign s = +-1 (exact)
template <typename R> STAG_D Vec3<R> vsign(R s, const Vec3<R>& v) {
    Vec3<R> r;
#pragma unroll
    for (int a = 0; a < 3; a++) r.c[a] = cmk(s * v.c[a].re, s * v.c[a].im);
    return r;
}
// s U (all three rows) for a sign s = +-1
template <typename R> STAG_D void msign(R s, Mat3<R>& u) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) u.e[a][b] = cmk(s * u.e[a][b].re, s * u.e[a][b].im);
}

// U psi and U^dag psi
template <typename R> STAG_D Vec3<R> mv(const Mat3<R>& u, const Vec3<R>& v) {
    Vec3<R> r;
#pragma unroll
    for (int a = 0; a < 3; a++) r.c[a] = u.e[a][0] * v.c[0] + u.e[a][1] * v.c[1] + u.e[a][2] * v.c[2];
    return r;
}
template <typename R> STAG_D Vec3<R> mdv(const Mat3<R>& u, const Vec3<R>& v) {
    Vec3<R> r;
#pragma unroll
    for (int a = 0; a < 3; a++)
        r.c[a] = cjmul(u.e[0][a], v.c[0]) + cjmul(u.e[1][a], v.c[1]) + cjmul(u.e[2][a], v.c[2]);
    return r;
}

// ---------------------------------------------------------------- reductions

STAG_D double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of one double (blockDim.x multiple of 32, <= 1024); result valid in thread 0
STAG_D double block_sum(double v) {
    __shared__ double red_smem[32];
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red_smem[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        s = (lane < nw) ? red_smem[lane] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

// Block-wide sums of N values at once (one pair of barriers for all of them);
// results valid in thread 0.  blockDim.x a multiple of 32, <= 1024.
template <int N> STAG_D void block_sum_n(double v[N]) {
    __shared__ double red_n[32][N];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < N; j++) v[j] = warp_sum(v[j]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < N; j++) red_n[w][j] = v[j];
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int j = 0; j < N; j++) v[j] = warp_sum(lane < nw ? red_n[lane][j] : 0.0);
    }
}

STAG_D float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of N series (N a power of two <= 32) by a transposing
// butterfly: at the exchange with lane^o (o = 16, 8, ...) each lane keeps
// half of its series (the upper half where its bit o is set) and adds its
// partner's copy of that half, so the series count halves at every step;
// once one series is left, plain butterfly steps finish the sum.  N - 1 +
// 5 - log2(N) shuffles instead of 5 N.  On return, lane l holds the warp sum
// of series l >> (5 - log2(N)).
template <int N, typename T> STAG_D T warp_transpose_sum(const T v[N]) {
    static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "N a power of two <= 32");
    const int lane = threadIdx.x & 31;
    T s[N];
#pragma unroll
    for (int j = 0; j < N; j++) s[j] = v[j];
#pragma unroll
    for (int half = N / 2, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const T send = up ? s[i] : s[i + half];
            const T keep = up ? s[i + half] : s[i];
            s[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    T r = s[0];
#pragma unroll
    for (int o = 16 / N; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// Block sums of N <= 32 per-thread values of type T (N a power of two):
// returns the sum of series j in lane j of warp 0 (j < N; other threads get
// 0).  The warp level runs in T (for FP32 data: FP32 shuffles, since GB300
// executes FP64 at a small fraction of its FP32 rate), the cross-warp level
// in FP64, one lane per series adding the warps' partials in order.
template <int N, typename T> STAG_D double block_sum_nv(const T v[N]) {
    static_assert(N <= 32, "one lane per series");
    __shared__ double red_v[32][N];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int SHIFT = (N >= 32) ? 0 : (N >= 16) ? 1 : (N >= 8) ? 2 : (N >= 4) ? 3 : (N >= 2) ? 4 : 5;
    const T ws = warp_transpose_sum<N, T>(v);
    __syncthreads();
    if ((lane & ((1 << SHIFT) - 1)) == 0) red_v[w][lane >> SHIFT] = (double)ws;
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x < N) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; i++) out += red_v[i][threadIdx.x];
    }
    return out;
}

// In the last block: out[s] = sum_i partials[s * nb + i] for s < nseries,
// one warp per series (all warps in parallel).  Ends with a barrier.
STAG_D void reduce_series(const double* partials, int nseries, int nb, double* out_shared) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int sidx = w; sidx < nseries; sidx += nw) {
        double v = 0.0;
        for (int i = lane; i < nb; i += 32) v += __ldcg(partials + (size_t)sidx * nb + i);
        v = warp_sum(v);
        if (lane == 0) out_shared[sidx] = v;
    }
    __syncthreads();
}

// Deterministic two-level grid reduction of nseries sums whose block partials
// are at partials[s * gridDim.x + blockIdx.x] (blocks of every row y write the
// series they own; unwritten entries are never read by a series' owner rows
// only if the caller keeps them zero -- every caller writes all it reduces).
// Level 1: the last block to finish among the gridDim.y x STAG_RED_GROUP
// blocks of each column group sums that group's columns into
// gpart[s * ngroups + group]; level 2: the last group to finish sums gpart.
// At each level one thread per series adds at most STAG_RED_GROUP (level 1)
// or ngroups (level 2) values, so the serial tail is short and uses few FP64
// operations (GB300 executes FP64 at a small fraction of its FP32 rate).  Returns true in exactly one block, whose
// out_shared[0..nseries) then holds the sums; counters[0] and
// counters[1 + group] return to zero.
#define STAG_RED_GROUP 32
STAG_D bool grid_reduce_series(const double* partials, double* gpart, unsigned int* counters, int nseries,
                               double* out_shared) {
    __shared__ bool s_last;
    const int nbx = gridDim.x, ngr = (nbx + STAG_RED_GROUP - 1) / STAG_RED_GROUP;
    const int grp = blockIdx.x / STAG_RED_GROUP, g0 = grp * STAG_RED_GROUP;
    const int gsz = (nbx - g0 < STAG_RED_GROUP) ? nbx - g0 : STAG_RED_GROUP;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(counters + 1 + grp, 1u);
        s_last = (t == (unsigned int)(gsz * gridDim.y) - 1u);
        if (s_last) counters[1 + grp] = 0;
    }
    __syncthreads();
    if (!s_last) return false;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (nseries <= nw) {  // level 1, few series: one warp per series, one load per lane
        if (w < nseries) {
            double v = (lane < gsz) ? __ldcg(partials + (size_t)w * nbx + g0 + lane) : 0.0;
            v = warp_sum(v);
            if (lane == 0) gpart[(size_t)w * ngr + grp] = v;
        }
    } else {  // level 1, many series: one thread per series, columns in order
        for (int sidx = threadIdx.x; sidx < nseries; sidx += blockDim.x) {
            const double* src = partials + (size_t)sidx * nbx + g0;
            double v = 0.0;
#pragma unroll 8
            for (int i = 0; i < gsz; i++) v += __ldcg(src + i);
            gpart[(size_t)sidx * ngr + grp] = v;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(counters, 1u);
        s_last = (t == (unsigned int)ngr - 1u);
        if (s_last) counters[0] = 0;
    }
    __syncthreads();
    if (!s_last) return false;
    if (nseries <= nw) {  // level 2 as level 1
        if (w < nseries) {
            double v = 0.0;
            for (int i = lane; i < ngr; i += 32) v += __ldcg(gpart + (size_t)w * ngr + i);
            v = warp_sum(v);
            if (lane == 0) out_shared[w] = v;
        }
    } else {
        for (int sidx = threadIdx.x; sidx < nseries; sidx += blockDim.x) {
            const double* src = gpart + (size_t)sidx * ngr;
            double v = 0.0;
#pragma unroll 8
            for (int i = 0; i < ngr; i++) v += __ldcg(src + i);
            out_shared[sidx] = v;
        }
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------- shared helpers

STAG_D Site site_from_lex(const Geom& g, int lex) {
    Site s;
    s.lex = lex;
    int r = gdiv(g, 0, lex);
    s.x[0] = lex - r * g.L[0];
    int r2 = gdiv(g, 1, r);
    s.x[1] = r - r2 * g.L[1];
    s.x[3] = gdiv(g, 2, r2);
    s.x[2] = r2 - s.x[3] * g.L[2];
    return s;
}
STAG_D int par_of(const Site& s) { return (s.x[0] + s.x[1] + s.x[2] + s.x[3]) & 1; }
STAG_D int par_of_lex(const Geom& g, int lex) { return par_of(site_from_lex(g, lex)); }

// last-block-done: returns true in exactly one block, after all blocks have
// written their partials (threadfence + counter), and resets the counter.
STAG_D bool last_block(unsigned int* counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last && threadIdx.x == 0) *counter = 0;
    return am_last;
}

// sum of partials[0..n) into *dst by block 0 style loop in the last block
STAG_D void finish_sum(const double* partials, int n, double* dst) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(partials + i);
    s = block_sum(s);
    if (threadIdx.x == 0) *dst = s;
}


// hop.cuh -- the staggered hop of Eq. (4) for one output site, shared by the
// dslash, M_ee and solver kernels.
//
//   (D psi)(n) = 1/2 sum_mu eta_mu(n) [U_mu(n) psi(n+mu) - U_mu(n-mu)^dag psi(n-mu)]
//
// One thread per output site of parity `par`; it reads 4 forward links
// (parity par, contiguous in h), 4 backward links (parity 1-par, gathered),
// and 8 neighbour vectors (gathered; re-read by 8 sites, so mostly L2 hits).
// The antiperiodic temporal boundary multiplies the hops across the link
// t = Lt-1 -> 0 by -1 (never folded into the stored link, which must stay in
// SU(3) for the third-row rebuild).  The factor 1/2 is applied by the caller.
#pragma once
#include "lattice.cuh"

enum LinkPrec { LP64 = 0, LP32 = 1, LP16 = 2, LPFF = 3, LP8 = 4 };

// Link arrays handed to a kernel: `u` in the kernel's link precision, `lo` the
// FP32 low words (float-float links only).
struct Links {
    const void* u;
    const float4* lo;
};

template <typename R> struct VT;
template <> struct VT<double> { typedef double2 T; };
template <> struct VT<float> { typedef float2 T; };

template <typename R, int LP> STAG_D Mat3<R> get_link(const void* U, const Geom& g, int mu, int par, int h);
template <> STAG_D Mat3<double> get_link<double, LP64>(const void* U, const Geom& g, int mu, int par, int h) {
    return load_link64((const double2*)U, g, mu, par, h);
}
template <> STAG_D Mat3<float> get_link<float, LP32>(const void* U, const Geom& g, int mu, int par, int h) {
    return load_link32((const float4*)U, g, mu, par, h);
}
template <> STAG_D Mat3<float> get_link<float, LP16>(const void* U, const Geom& g, int mu, int par, int h) {
    return load_link16((const uint2*)U, g, mu, par, h);
}
template <> STAG_D Mat3<float> get_link<float, LP8>(const void* U, const Geom& g, int mu, int par, int h) {
    return load_link8((const float4*)U, g, mu, par, h);
}

template <typename R> STAG_D void axpy_sign(Vec3<R>& acc, int s, const Vec3<R>& v) {
    if (s > 0) {
#pragma unroll
        for (int a = 0; a < 3; a++) acc.c[a] = acc.c[a] + v.c[a];
    } else {
#pragma unroll
        for (int a = 0; a < 3; a++) acc.c[a] = acc.c[a] - v.c[a];
    }
}

// ---------------------------------------------------------------- float-float hop
// FP64-accurate hop on the FP32 pipes.  A double d is carried as the pair
// hi = fl32(d), lo = fl32(d - hi) (the split of Sec. 4.2 of the paper, used
// here for arithmetic: GB300's FP64 throughput is a small fraction of its
// FP32 throughput).  Products use the exact FMA split (Dekker/Kahan
// two-product), sums Knuth's two-sum; all operations are the non-contracting
// __f*_rn intrinsics so that the compiler cannot fuse the error terms away.
// Relative accuracy ~2^-44 per operation, ample for 1e-12 residual checks.
struct ff {
    float hi, lo;
};
STAG_D ff ff_make(double d) {
    ff r;
    r.hi = __double2float_rn(d);
    r.lo = __double2float_rn(d - (double)r.hi);
    return r;
}
STAG_D double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }
STAG_D ff ff_quick(float s, float e) {  // |s| >= |e|
    ff r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}
struct cff {
    ff re, im;
};

// Split a double into hi + lo floats with integer operations only (no FP64
// arithmetic): hi = the leading 24 significand bits (truncated), lo = the
// remaining 29 bits rounded to 24, scaled by 2^(e-1075).  Magnitudes outside
// [2^-74, 2^100] fall back to hi = fl32(d), lo = 0.
STAG_D ff ff_split_bits(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);
    ff r;
    if (e < 949 || e > 1123) {
        r.hi = __double2float_rn(d);
        r.lo = 0.f;
        return r;
    }
    const unsigned int sign = (unsigned int)(b >> 63) << 31;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    r.hi = __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)(m >> 29));
    const float scale = __uint_as_float((unsigned int)(e - 1075 + 127) << 23);
    const float lo = __fmul_rn(__uint2float_rn((unsigned int)(m & 0x1FFFFFFFull)), scale);
    r.lo = sign ? -lo : lo;
    return r;
}

STAG_D void load_vec_ff(const double2* __restrict__ v, int h, cff out[3]) {
    const double2* p = v + 3 * (size_t)h;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double2 d = __ldg(p + a);
        out[a].re = ff_split_bits(d.x);
        out[a].im = ff_split_bits(d.y);
    }
}

// Lazy float-float accumulator: value = s + e, where s collects the leading
// parts through two-sums and e (a plain float) the exact error terms; one
// normalisation at the end instead of one per operation.
struct ffa {
    float s, e;
};
STAG_D void ffa_mac(ffa& acc, ff a, ff b, bool neg) {
    float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    if (neg) {
        p = -p;
        pe = -pe;
    }
    const float s = __fadd_rn(acc.s, p);
    const float bb = __fsub_rn(s, acc.s);
    const float te = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.s = s;
    acc.e = __fadd_rn(acc.e, __fadd_rn(te, pe));
}
STAG_D ff ffa_norm(ffa a) { return ff_quick(a.s, a.e); }

// third link row conj(row0 x row1) in float-float with lazy accumulation
STAG_D void recon_ff(cff u[3][3]) {
    const int i1[3] = {1, 2, 0}, i2[3] = {2, 0, 1};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cff a = u[0][i1[c]], b = u[1][i2[c]], x = u[0][i2[c]], y = u[1][i1[c]];
        // row2[c] = conj(a b - x y)
        ffa re = {0.f, 0.f}, im = {0.f, 0.f};
        ffa_mac(re, a.re, b.re, false);
        ffa_mac(re, a.im, b.im, true);
        ffa_mac(re, x.re, y.re, true);
        ffa_mac(re, x.im, y.im, false);
        ffa_mac(im, a.re, b.im, true);
        ffa_mac(im, a.im, b.re, true);
        ffa_mac(im, x.re, y.im, false);
        ffa_mac(im, x.im, y.re, false);
        u[2][c].re = ffa_norm(re);
        u[2][c].im = ffa_norm(im);
    }
}

STAG_D void load_link_ff_lazy(const float4* __restrict__ Uhi, const float4* __restrict__ Ulo, const Geom& g, int mu,
                              int par, int h, cff u[3][3]) {
    const size_t base = (size_t)(mu * 2 + par) * 3 * g.Vh + h;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float4 a = __ldg(Uhi + base + (size_t)j * g.Vh), b = __ldg(Ulo + base + (size_t)j * g.Vh);
        const int e0 = 2 * j, e1 = 2 * j + 1;
        u[e0 / 3][e0 % 3].re = {a.x, b.x};
        u[e0 / 3][e0 % 3].im = {a.y, b.y};
        u[e1 / 3][e1 % 3].re = {a.z, b.z};
        u[e1 / 3][e1 % 3].im = {a.w, b.w};
    }
    recon_ff(u);
}

// 2 (D psi)(n) in float-float arithmetic, returned in FP64
STAG_D Vec3<double> hop2_ff(const Geom& g, const float4* __restrict__ Uhi, const float4* __restrict__ Ulo,
                            const double2* __restrict__ in, int h, int par, const Site& s) {
    ffa ar[3], ai[3];
#pragma unroll
    for (int a = 0; a < 3; a++) ar[a] = ai[a] = {0.f, 0.f};
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int fl = nb_lex(g, s, mu, +1);
        const int bl = nb_lex(g, s, mu, -1);
        int sf = eta(s, mu), sb = sf;
        if (mu == 3) {
            if (s.x[3] == g.L[3] - 1) sf = -sf;
            if (s.x[3] == 0) sb = -sb;
        }
        cff u[3][3], v[3];
        // forward: + sf U_mu(n) psi(n+mu)
        load_link_ff_lazy(Uhi, Ulo, g, mu, par, h, u);
        load_vec_ff(in, fl >> 1, v);
        const bool nf = sf < 0;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                ffa_mac(ar[a], u[a][c].re, v[c].re, nf);
                ffa_mac(ar[a], u[a][c].im, v[c].im, !nf);
                ffa_mac(ai[a], u[a][c].re, v[c].im, nf);
                ffa_mac(ai[a], u[a][c].im, v[c].re, nf);
            }
        // backward: - sb U_mu(n-mu)^dag psi(n-mu)
        load_link_ff_lazy(Uhi, Ulo, g, mu, 1 - par, bl >> 1, u);
        load_vec_ff(in, bl >> 1, v);
        const bool nb = sb > 0;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                // conj(u[c][a]) v[c]
                ffa_mac(ar[a], u[c][a].re, v[c].re, nb);
                ffa_mac(ar[a], u[c][a].im, v[c].im, nb);
                ffa_mac(ai[a], u[c][a].re, v[c].im, nb);
                ffa_mac(ai[a], u[c][a].im, v[c].re, !nb);
            }
    }
    Vec3<double> r;
#pragma unroll
    for (int a = 0; a < 3; a++)
        r.c[a] = cmk((double)ar[a].s + (double)ar[a].e, (double)ai[a].s + (double)ai[a].e);
    return r;
}

// 2 (D psi)(n) for the site s = (h, par); psi lives on parity 1-par.  The
// signs (staggered phase, antiperiodic boundary) multiply the neighbour
// vectors, so the two products of each direction are plain fused
// multiply-add chains into one accumulator, without branches.
template <typename R, int LP>
STAG_D Vec3<R> hop2(const Geom& g, const void* __restrict__ U, const typename VT<R>::T* __restrict__ in,
                    int h, int par, const Site& s) {
    Vec3<R> acc = vzero<R>();
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int fl = nb_lex(g, s, mu, +1);
        const int bl = nb_lex(g, s, mu, -1);
        int sf = eta(s, mu), sb = sf;
        if (mu == 3) {
            if (s.x[3] == g.L[3] - 1) sf = -sf;
            if (s.x[3] == 0) sb = -sb;
        }
        const Mat3<R> uf = get_link<R, LP>(U, g, mu, par, h);
        mv_acc(acc, uf, vsign((R)sf, load_vec(in, fl >> 1)));
        const Mat3<R> ub = get_link<R, LP>(U, g, mu, 1 - par, bl >> 1);
        mdv_acc(acc, ub, vsign((R)(-sb), load_vec(in, bl >> 1)));
    }
    return acc;
}

// 2 (D psi)(n) with any link precision (R = double for LP64 and LPFF)
template <typename R, int LP>
STAG_D Vec3<R> hopL(const Geom& g, Links L, const typename VT<R>::T* __restrict__ in, int h, int par,
                    const Site& s) {
    if constexpr (LP == LPFF) {
        return hop2_ff(g, (const float4*)L.u, L.lo, in, h, par, s);
    } else {
        return hop2<R, LP>(g, L.u, in, h, par, s);
    }
}

// multi-RHS: acc[q] = 2 (D psi_q)(n) for the NR vectors psi_q = in + js[q] * stride,
// q < nj; each link is loaded once for all of them
template <typename R, int LP, int NR>
STAG_D void hop2_multiR(const Geom& g, const void* __restrict__ U, const typename VT<R>::T* __restrict__ in,
                        size_t stride, const int* js, int nj, int h, int par, const Site& s, Vec3<R> acc[NR]) {
#pragma unroll
    for (int q = 0; q < NR; q++) acc[q] = vzero<R>();
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int fl = nb_lex(g, s, mu, +1);
        const int bl = nb_lex(g, s, mu, -1);
        int sf = eta(s, mu), sb = sf;
        if (mu == 3) {
            if (s.x[3] == g.L[3] - 1) sf = -sf;
            if (s.x[3] == 0) sb = -sb;
        }
        // the sign multiplies the link once for all right-hand sides
        Mat3<R> uf = get_link<R, LP>(U, g, mu, par, h);
        msign((R)sf, uf);
#pragma unroll
        for (int q = 0; q < NR; q++)
            if (q < nj) mv_acc(acc[q], uf, load_vec(in + js[q] * stride, fl >> 1));
        Mat3<R> ub = get_link<R, LP>(U, g, mu, 1 - par, bl >> 1);
        msign((R)(-sb), ub);
#pragma unroll
        for (int q = 0; q < NR; q++)
            if (q < nj) mdv_acc(acc[q], ub, load_vec(in + js[q] * stride, bl >> 1));
    }
}

// FP32-vector form used by the batched refinement
template <int LP, int NR>
STAG_D void hop2_multi(const Geom& g, const void* __restrict__ U, const float2* __restrict__ in, size_t stride,
                       const int* js, int nj, int h, int par, const Site& s, Vec3<float> acc[NR]) {
    hop2_multiR<float, LP, NR>(g, U, in, stride, js, nj, h, par, s, acc);
}

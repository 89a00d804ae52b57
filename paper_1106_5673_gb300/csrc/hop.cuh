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

enum LinkPrec { LP64 = 0, LP32 = 1, LP16 = 2 };

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

template <typename R> STAG_D void axpy_sign(Vec3<R>& acc, int s, const Vec3<R>& v) {
    if (s > 0) {
#pragma unroll
        for (int a = 0; a < 3; a++) acc.c[a] = acc.c[a] + v.c[a];
    } else {
#pragma unroll
        for (int a = 0; a < 3; a++) acc.c[a] = acc.c[a] - v.c[a];
    }
}

// 2 (D psi)(n) for the site s = (h, par); psi lives on parity 1-par.
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
        const Vec3<R> vf = load_vec(in, fl >> 1);
        axpy_sign(acc, sf, mv(uf, vf));
        const Mat3<R> ub = get_link<R, LP>(U, g, mu, 1 - par, bl >> 1);
        const Vec3<R> vb = load_vec(in, bl >> 1);
        axpy_sign(acc, -sb, mdv(ub, vb));
    }
    return acc;
}

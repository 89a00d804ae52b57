// force.cu -- fermion force of S_f = phi^dag r(M_ee) phi,
// r(x) = a0 + sum_k a_k / (x + b_k) (RHMC, Sec. 2.1).
//
// With X_k = (M_ee + b_k)^{-1} phi (even sites) and Y_k = D_oe X_k (odd),
// dS_f = -2 sum_k a_k Re Y_k^dag dD_oe X_k.  For U' = i P U the link U_mu(n)
// with sign s_mu(n) (staggered phase times the antiperiodic boundary sign)
// gets dP/dtau = i TA(W),  W = (s_mu(n)/2) U_mu(n) sum_k a_k Z_k,
//   Z_k = X_k(n+mu) Y_k(n)^dag       for n odd,
//   Z_k = -Y_k(n+mu) X_k(n)^dag      for n even.
// One thread per site handles its four links; the site's own vector of each
// shift is loaded once per direction and the neighbour vectors come from L2.
#include "hop.cuh"
#include "stag_internal.h"

static const int TPB = 128;

struct ForceCoef {
    double a[STAG_MAXSHIFT];
    int n;
};

__global__ void __launch_bounds__(TPB) k_fermion_force(Geom g, const double2* __restrict__ U,
                                                       const double2* __restrict__ X, const double2* __restrict__ Y,
                                                       ForceCoef fc, double* F, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int par = i / g.Vh, h = i % g.Vh;
    const Site s = site_of(g, h, par);
    const size_t stride = 3 * (size_t)g.Vh;
    // odd site: own = Y (odd), neighbour = X (even); even site: own = X, neighbour = Y
    const double2* own = par ? Y : X;
    const double2* nbv = par ? X : Y;
    const double sgn_par = par ? 1.0 : -1.0;
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
        const int fl = nb_lex(g, s, mu, +1);
        int sg = eta(s, mu);
        if (mu == 3 && s.x[3] == g.L[3] - 1) sg = -sg;
        Mat3<double> Z = mzero<double>();
        for (int k = 0; k < fc.n; k++) {
            const Vec3<double> a = load_vec(nbv + k * stride, fl >> 1);
            const Vec3<double> b = load_vec(own + k * stride, h);
            const double ak = fc.a[k] * sgn_par;
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const cd o = cjmul(b.c[c], a.c[r]);  // a_r conj(b_c)
                    Z.e[r][c] = Z.e[r][c] + ak * o;
                }
        }
        const Mat3<double> u = load_link64(U, g, mu, par, h);
        Mat3<double> W = mmul(u, Z);
        double f[8];
        i_ta_to_omega(W, f);
        const double c = 0.5 * sg;
        double* q = F + (size_t)(mu * 2 + par) * 8 * g.Vh + h;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const double v = c * f[a];
            q[(size_t)a * g.Vh] = accumulate ? q[(size_t)a * g.Vh] + v : v;
        }
    }
}

int fermion_force_assemble(stag_ctx* ctx, const stag_rational* r, const double2* X, double* F, int accumulate,
                           cudaStream_t s) {
    const long n3 = 3L * ctx->g.Vh;
    double2* Y = (double2*)ws_get(ctx, WS_FY, sizeof(double2) * n3 * STAG_MAXSHIFT);
    if (!Y) return stag_fail(ctx, STAG_ERR_OOM, "force workspace");
    int st = dslash_multi64(ctx, X, Y, r->n, 1, s);
    if (st) return st;
    ForceCoef fc;
    fc.n = r->n;
    for (int k = 0; k < r->n; k++) fc.a[k] = r->a[k];
    k_fermion_force<<<nblocks(ctx->g.V, TPB), TPB, 0, s>>>(ctx->g, ctx->U64, X, Y, fc, F, accumulate);
    STAG_LAUNCH_CHECK(ctx, "fermion_force");
    return STAG_OK;
}

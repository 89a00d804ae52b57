// noalloc.cu -- M_ee for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc when they apply the operator: code that
// lives inside a framework which owns the whole device memory pool (an
// allocation behind its back breaks its accounting or exceeds its cap), and
// latency-critical loops, where cudaMalloc's implicit device synchronisation
// would stall every stream.  stag_apply_M_noalloc serves them: it takes the
// gauge field, the input and the output from the caller and keeps its only
// scratch vector -- the odd-site intermediate D_oe in -- in a fixed array
// inside this library, so the call itself allocates nothing.
//
// The array holds STAG_NOALLOC_MAX_VH sites of one parity (a 32^3 x 8 lattice
// at most, 6 MiB of FP64 colour vectors) and is resident on every device
// that loads the library until the process exits.  All calls share it: a
// call overwrites all of it that it later reads, and calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// it.
#include <stdint.h>

#include "hop.cuh"
#include "stag_internal.h"

#define STAG_NOALLOC_MAX_VH (1 << 17)
#define STAG_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double2 g_noalloc_scratch[3 * STAG_NOALLOC_MAX_VH];

// host side: device address of the array, looked up once per device
static double2* g_scratch_addr[STAG_NOALLOC_MAX_DEVICES];

// One thread per output site; links read in the caller's canonical layout
// complex128 [mu][lex][3][3] (full matrices, no third-row rebuild).
__global__ void __launch_bounds__(128) k_hop_canonical(Geom g, const double2* __restrict__ U,
                                                        const double2* __restrict__ in, double2* __restrict__ out,
                                                        int par, double scale, double c,
                                                        const double2* __restrict__ self) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const Site s = site_of(g, h, par);
    Vec3<double> acc = vzero<double>();
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int fl = nb_lex(g, s, mu, +1), bl = nb_lex(g, s, mu, -1);
        int sf = eta(s, mu), sb = sf;
        if (mu == 3) {
            if (s.x[3] == g.L[3] - 1) sf = -sf;
            if (s.x[3] == 0) sb = -sb;
        }
        const double2* uf = U + ((size_t)mu * g.V + s.lex) * 9;
        const double2* ub = U + ((size_t)mu * g.V + bl) * 9;
        Mat3<double> a, b;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const double2 x = __ldg(uf + 3 * i + j), y = __ldg(ub + 3 * i + j);
                a.e[i][j] = cmk(x.x, x.y);
                b.e[i][j] = cmk(y.x, y.y);
            }
        axpy_sign(acc, sf, mv(a, load_vec(in, fl >> 1)));
        axpy_sign(acc, -sb, mdv(b, load_vec(in, bl >> 1)));
    }
    Vec3<double> r;
    if (self) {
        const Vec3<double> v = load_vec(self, h);
#pragma unroll
        for (int i = 0; i < 3; i++) r.c[i] = c * v.c[i] + scale * acc.c[i];
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++) r.c[i] = scale * acc.c[i];
    }
    st_vec(out, h, r);
}

extern "C" int stag_apply_M_noalloc(const int dims[4], const double* links, double mass, const double* in_even,
                                    double* out_even, void* stream) {
    if (!dims || !links || !in_even || !out_even) return STAG_ERR_ARG;
    if (((uintptr_t)links | (uintptr_t)in_even | (uintptr_t)out_even) & 15u) return STAG_ERR_ARG;
    if (in_even == out_even) return STAG_ERR_ARG;
    // each extent is bounded before it is multiplied in, so the product can
    // neither overflow nor wrap below the limit
    long long V = 1;
    for (int m = 0; m < 4; m++) {
        if (dims[m] < 2 || (dims[m] & 1) || dims[m] > 2 * STAG_NOALLOC_MAX_VH) return STAG_ERR_ARG;
        V *= dims[m];
        if (V / 2 > STAG_NOALLOC_MAX_VH) return STAG_ERR_ARG;  // beyond the fixed scratch array
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return STAG_ERR_CUDA;
    }
    if (dev < 0 || dev >= STAG_NOALLOC_MAX_DEVICES) return STAG_ERR_ARG;
    if (!g_scratch_addr[dev]) {  // set-up on this device's first call
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return STAG_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double2*)p;
    }
    Geom g;
    geom_init(g, dims);
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (g.Vh + 127) / 128;
    double2* tmp = g_scratch_addr[dev];
    const double2* U = (const double2*)links;
    // tmp (odd) = D_oe in;  out = m^2 in - D_eo tmp
    k_hop_canonical<<<nb, 128, 0, s>>>(g, U, (const double2*)in_even, tmp, 1, 0.5, 0.0, nullptr);
    k_hop_canonical<<<nb, 128, 0, s>>>(g, U, tmp, (double2*)out_even, 0, -0.5, mass * mass, (const double2*)in_even);
    if (cudaGetLastError() != cudaSuccess) return STAG_ERR_CUDA;
    return STAG_OK;
}

// capi.cu -- the extern "C" boundary of libstag.so (declared in include/stag.h):
// argument checks, context lifetime, work-space management and error strings.
#include <stdarg.h>
#include <stdlib.h>

#include "stag_internal.h"

int rhmc_trajectory(stag_ctx* ctx, const stag_params* p, stag_traj_info* out, cudaStream_t s);
int md_integrate_public(stag_ctx* ctx, const stag_params* p, const double2* phi, long long* iters, int* nforce,
                        cudaStream_t s);
int gauge_force_internal_prec(stag_ctx* ctx, double beta, double* F, int accumulate, int prec32, cudaStream_t s);

// ---------------------------------------------------------------- errors

int stag_fail(stag_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int stag_cuda_check(stag_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return STAG_OK;
    cudaGetLastError();  // clear a sticky launch error
    return stag_fail(ctx, e == cudaErrorMemoryAllocation ? STAG_ERR_OOM : STAG_ERR_CUDA, "%s: %s (%d)", what,
                     cudaGetErrorString(e), (int)e);
}

static void clear_graphs(stag_ctx* ctx) {
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
}
void ctx_clear_graphs(stag_ctx* ctx) { clear_graphs(ctx); }

// Returns a device buffer of at least `bytes` for `slot`; grows it if needed
// (which invalidates captured graphs, since they hold raw pointers).
void* ws_get(stag_ctx* ctx, int slot, size_t bytes) {
    if (ctx->ws_bytes[slot] >= bytes) return ctx->ws[slot];
    if (ctx->ws[slot]) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws[slot]);
        clear_graphs(ctx);
    }
    ctx->ws[slot] = nullptr;
    ctx->ws_bytes[slot] = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    ctx->ws[slot] = p;
    ctx->ws_bytes[slot] = bytes;
    return p;
}

static inline cudaStream_t S(void* s) { return (cudaStream_t)s; }
static int aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }


#define CHECK_CTX(ctx)                                      \
    do {                                                    \
        if (!(ctx)) return STAG_ERR_ARG;                    \
    } while (0)
#define CHECK_GAUGE(ctx)                                                           \
    do {                                                                           \
        if (!(ctx)->gauge_loaded) return stag_fail(ctx, STAG_ERR_STATE, "no gauge field loaded"); \
    } while (0)
#define CHECK_PTR(ctx, p)                                                                      \
    do {                                                                                       \
        if (!(p) || !aligned16(p)) return stag_fail(ctx, STAG_ERR_ARG, "%s null or not 16-byte aligned", #p); \
    } while (0)

// ---------------------------------------------------------------- context

extern "C" {

int stag_ctx_create(const int dims[4], stag_ctx** out) {
    if (!out || !dims) return STAG_ERR_ARG;
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; m++) {
        if (dims[m] < 2 || (dims[m] & 1)) return STAG_ERR_ARG;
        V *= dims[m];
    }
    if (V > (1L << 29)) return STAG_ERR_ARG;
    stag_ctx* ctx = new stag_ctx();
    memset(ctx->err, 0, sizeof ctx->err);
    geom_init(ctx->g, dims);
    ctx->use_graphs = 1;
    for (int i = 0; i < WS_NSLOTS; i++) {
        ctx->ws[i] = nullptr;
        ctx->ws_bytes[i] = 0;
    }
    int st = STAG_OK;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const size_t Vh = ctx->g.Vh;
    int maxb = (int)(4 * (Vh / 64 + 2));  // four partial sums per hop block of >= 64 threads
    if (maxb < (int)(V / 256 + 2)) maxb = (int)(V / 256 + 2);
    if (maxb < 16 * ctx->num_sms) maxb = 16 * ctx->num_sms;
    // two-level reductions: one counter and 4 * STAG_MAXSHIFT group sums per
    // group of STAG_RED_GROUP blocks of >= 64 threads
    const size_t ngroups = (Vh / 64 + 2) / STAG_RED_GROUP + 2;
    const size_t counter_bytes = sizeof(unsigned int) * (64 + ngroups);
    ctx->counter_bytes = counter_bytes;
    struct { void** p; size_t bytes; } allocs[] = {
        {(void**)&ctx->U64, sizeof(double2) * 48 * Vh},
        {(void**)&ctx->U32, sizeof(float4) * 24 * Vh},
        {(void**)&ctx->U32lo, sizeof(float4) * 24 * Vh},
        {(void**)&ctx->U16, sizeof(uint2) * 24 * Vh},
        {(void**)&ctx->U64_save, sizeof(double2) * 48 * Vh},
        {(void**)&ctx->mom, sizeof(double) * 64 * Vh},
        {(void**)&ctx->partials, sizeof(double) * (size_t)maxb},
        {(void**)&ctx->counter, counter_bytes},
        {(void**)&ctx->gpart, sizeof(double) * 4 * STAG_MAXSHIFT * ngroups},
        {(void**)&ctx->dscal, sizeof(double) * STAG_NSCAL},
        {(void**)&ctx->partials2, sizeof(double) * (size_t)maxb},
        {(void**)&ctx->counter2, counter_bytes},
        {(void**)&ctx->gpart2, sizeof(double) * 4 * STAG_MAXSHIFT * ngroups},
        {(void**)&ctx->dscal2, sizeof(double) * STAG_NSCAL},
        {(void**)&ctx->ms, sizeof(MSState)},
        {(void**)&ctx->cg, sizeof(CGState)},
        {(void**)&ctx->bcg, sizeof(BCGState)},
        {(void**)&ctx->msm, sizeof(MSState) * STAG_MAXRHS},
        {(void**)&ctx->mm_partials, sizeof(double) * 4 * STAG_MAXRHS * (Vh / 64 + 2)},
    };
    ctx->fixed_bytes = 0;
    for (auto& a : allocs) {
        if (e != cudaSuccess) break;
        e = cudaMalloc(a.p, a.bytes);
        ctx->fixed_bytes += a.bytes;
    }
    if (e == cudaSuccess) e = cudaMemset(ctx->counter, 0, counter_bytes);
    if (e == cudaSuccess) e = cudaMemset(ctx->counter2, 0, counter_bytes);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->hscal2, sizeof(double) * STAG_NSCAL);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->s2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_ref, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(ctx->mom, 0, sizeof(double) * 64 * Vh);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->hscal, sizeof(double) * STAG_NSCAL);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->ms_host, sizeof(MSState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->cg_host, sizeof(CGState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->bcg_host, sizeof(BCGState));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->msm_host, sizeof(MSState) * STAG_MAXRHS);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->ms_poll, sizeof(MSState));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_poll, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        st = (e == cudaErrorMemoryAllocation) ? STAG_ERR_OOM : STAG_ERR_CUDA;
        cudaGetLastError();
        stag_ctx_destroy(ctx);
        return st;
    }
    *out = ctx;
    return STAG_OK;
}

int stag_ctx_destroy(stag_ctx* ctx) {
    if (!ctx) return STAG_OK;
    cudaDeviceSynchronize();
    clear_graphs(ctx);
    void* ps[] = {ctx->U64, ctx->U32, ctx->U32lo, ctx->U16, ctx->U8, ctx->U64_save, ctx->mom, ctx->partials,
                  ctx->counter, ctx->dscal, ctx->ms, ctx->cg, ctx->bcg, ctx->msm, ctx->mm_partials,
                  ctx->gpart, ctx->partials2, ctx->counter2, ctx->gpart2, ctx->dscal2};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (int i = 0; i < WS_NSLOTS; i++)
        if (ctx->ws[i]) cudaFree(ctx->ws[i]);
    if (ctx->hscal) cudaFreeHost(ctx->hscal);
    if (ctx->ms_host) cudaFreeHost(ctx->ms_host);
    if (ctx->cg_host) cudaFreeHost(ctx->cg_host);
    if (ctx->bcg_host) cudaFreeHost(ctx->bcg_host);
    if (ctx->msm_host) cudaFreeHost(ctx->msm_host);
    if (ctx->ms_poll) cudaFreeHost(ctx->ms_poll);
    if (ctx->ev_poll) cudaEventDestroy(ctx->ev_poll);
    if (ctx->hscal2) cudaFreeHost(ctx->hscal2);
    if (ctx->ev_ref) cudaEventDestroy(ctx->ev_ref);
    if (ctx->s2) cudaStreamDestroy(ctx->s2);
    delete ctx;
    return STAG_OK;
}

const char* stag_last_error(const stag_ctx* ctx) { return ctx ? ctx->err : "null context"; }

int stag_ctx_launch_count(const stag_ctx* ctx, long long* n) {
    if (!ctx || !n) return STAG_ERR_ARG;
    *n = ctx->nlaunch;
    return STAG_OK;
}

int stag_autotune(stag_ctx* ctx, int tpb_out[4], void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    int st = autotune_hops(ctx, S(stream));
    if (st) return st;
    if (tpb_out)
        for (int i = 0; i < 4; i++) tpb_out[i] = ctx->tpb[i];
    return STAG_OK;
}

int stag_ctx_device_bytes(const stag_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return STAG_ERR_ARG;
    size_t b = ctx->fixed_bytes;
    for (int i = 0; i < WS_NSLOTS; i++) b += ctx->ws_bytes[i];
    *bytes = b;
    return STAG_OK;
}

// ---------------------------------------------------------------- fields

int stag_load_gauge(stag_ctx* ctx, const double* links, int on_device, void* stream) {
    CHECK_CTX(ctx);
    if (!links) return stag_fail(ctx, STAG_ERR_ARG, "links is null");
    const size_t bytes = sizeof(double) * 72 * (size_t)ctx->g.V;
    const double* src = links;
    if (!on_device) {
        double* stg = (double*)ws_get(ctx, WS_STAGE, bytes);
        if (!stg) return stag_fail(ctx, STAG_ERR_OOM, "staging buffer");
        STAG_CUDA(ctx, cudaMemcpyAsync(stg, links, bytes, cudaMemcpyHostToDevice, S(stream)));
        src = stg;
    }
    int st = gauge_from_canonical(ctx, src, S(stream));
    if (st) return st;
    if (!on_device) STAG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    ctx->gauge_loaded = 1;
    return STAG_OK;
}

int stag_store_gauge(stag_ctx* ctx, double* links, int on_device, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    if (!links) return stag_fail(ctx, STAG_ERR_ARG, "links is null");
    const size_t bytes = sizeof(double) * 72 * (size_t)ctx->g.V;
    if (on_device) return gauge_to_canonical(ctx, links, S(stream));
    double* stg = (double*)ws_get(ctx, WS_STAGE, bytes);
    if (!stg) return stag_fail(ctx, STAG_ERR_OOM, "staging buffer");
    int st = gauge_to_canonical(ctx, stg, S(stream));
    if (st) return st;
    STAG_CUDA(ctx, cudaMemcpyAsync(links, stg, bytes, cudaMemcpyDeviceToHost, S(stream)));
    STAG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return STAG_OK;
}

int stag_load_momenta(stag_ctx* ctx, const double* w, int on_device, void* stream) {
    CHECK_CTX(ctx);
    if (!w) return stag_fail(ctx, STAG_ERR_ARG, "w is null");
    const size_t bytes = sizeof(double) * 32 * (size_t)ctx->g.V;
    const double* src = w;
    if (!on_device) {
        double* stg = (double*)ws_get(ctx, WS_STAGE, sizeof(double) * 72 * (size_t)ctx->g.V);
        if (!stg) return stag_fail(ctx, STAG_ERR_OOM, "staging buffer");
        STAG_CUDA(ctx, cudaMemcpyAsync(stg, w, bytes, cudaMemcpyHostToDevice, S(stream)));
        src = stg;
    }
    int st = momenta_from_canonical(ctx, src, S(stream));
    if (st) return st;
    if (!on_device) STAG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return STAG_OK;
}

int stag_store_momenta(stag_ctx* ctx, double* w, int on_device, void* stream) {
    CHECK_CTX(ctx);
    if (!w) return stag_fail(ctx, STAG_ERR_ARG, "w is null");
    const size_t bytes = sizeof(double) * 32 * (size_t)ctx->g.V;
    if (on_device) return momenta_to_canonical(ctx, ctx->mom, w, S(stream));
    double* stg = (double*)ws_get(ctx, WS_STAGE, sizeof(double) * 72 * (size_t)ctx->g.V);
    if (!stg) return stag_fail(ctx, STAG_ERR_OOM, "staging buffer");
    int st = momenta_to_canonical(ctx, ctx->mom, stg, S(stream));
    if (st) return st;
    STAG_CUDA(ctx, cudaMemcpyAsync(w, stg, bytes, cudaMemcpyDeviceToHost, S(stream)));
    STAG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return STAG_OK;
}

static int read_scalar(stag_ctx* ctx, int slot, double* out, cudaStream_t s) {
    STAG_CUDA(ctx, cudaMemcpyAsync(ctx->hscal + slot, ctx->dscal + slot, sizeof(double), cudaMemcpyDeviceToHost, s));
    STAG_CUDA(ctx, cudaStreamSynchronize(s));
    *out = ctx->hscal[slot];
    return STAG_OK;
}

int stag_plaquette(stag_ctx* ctx, double* plaq, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    if (!plaq) return stag_fail(ctx, STAG_ERR_ARG, "plaq is null");
    int st = plaquette_sum(ctx, ctx->dscal + 2, S(stream));
    if (st) return st;
    double v;
    if ((st = read_scalar(ctx, 2, &v, S(stream)))) return st;
    *plaq = v / (6.0 * ctx->g.V);
    return STAG_OK;
}

int stag_gauge_action(stag_ctx* ctx, double beta, double* action, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    if (!action) return stag_fail(ctx, STAG_ERR_ARG, "action is null");
    int st = plaquette_sum(ctx, ctx->dscal + 2, S(stream));
    if (st) return st;
    double v;
    if ((st = read_scalar(ctx, 2, &v, S(stream)))) return st;
    *action = beta * (6.0 * ctx->g.V - v);
    return STAG_OK;
}

// ---------------------------------------------------------------- operator

int stag_apply_deo(stag_ctx* ctx, const void* in_odd, void* out_even, int prec, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    CHECK_PTR(ctx, in_odd);
    CHECK_PTR(ctx, out_even);
    return dslash_apply(ctx, prec, in_odd, out_even, 0, S(stream));
}

int stag_apply_doe(stag_ctx* ctx, const void* in_even, void* out_odd, int prec, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    CHECK_PTR(ctx, in_even);
    CHECK_PTR(ctx, out_odd);
    return dslash_apply(ctx, prec, in_even, out_odd, 1, S(stream));
}

int stag_apply_M(stag_ctx* ctx, double mass, const void* in_even, void* out_even, int prec, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    CHECK_PTR(ctx, in_even);
    CHECK_PTR(ctx, out_even);
    if (in_even == out_even) return stag_fail(ctx, STAG_ERR_ARG, "in and out alias");
    if (prec < 0 || prec > STAG_PREC_F32R8) return stag_fail(ctx, STAG_ERR_ARG, "unknown precision %d", prec);
    const int dbl = (prec == STAG_PREC_F64 || prec == STAG_PREC_F64FF);
    const size_t vb = (dbl ? sizeof(double2) : sizeof(float2)) * 3 * (size_t)ctx->g.Vh;
    void* tmp = ws_get(ctx, dbl ? WS_RHI : WS_XLO, vb);
    if (!tmp) return stag_fail(ctx, STAG_ERR_OOM, "temporary");
    return mee_apply(ctx, prec, mass * mass, in_even, out_even, tmp, S(stream));
}

// ---------------------------------------------------------------- solvers

int stag_multishift_solve(stag_ctx* ctx, double mass, int n, const double* shifts, const double* src,
                          double* const* sols, double tol, int maxit, int mode, stag_solve_info* info,
                          void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    CHECK_PTR(ctx, src);
    if (!shifts) return stag_fail(ctx, STAG_ERR_ARG, "shifts is null");
    if (sols)
        for (int k = 0; k < n && k < STAG_MAXSHIFT; k++)
            if (sols[k] && !aligned16(sols[k])) return stag_fail(ctx, STAG_ERR_ARG, "sols[%d] not aligned", k);
    return multishift_solve(ctx, mass, n, shifts, (const double2*)src, (double2* const*)sols, tol, maxit, mode, info,
                            S(stream));
}

int stag_multishift_solve_multi(stag_ctx* ctx, double mass, int nsys, int n, const double* shifts,
                                const double* const* srcs, double* const* sols, double tol, int maxit, int mode,
                                stag_solve_info* infos, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    if (!shifts || !srcs) return stag_fail(ctx, STAG_ERR_ARG, "shifts or srcs is null");
    if (nsys < 1 || nsys > STAG_MAXRHS || n < 1 || n > STAG_MAXSHIFT)
        return stag_fail(ctx, STAG_ERR_ARG, "bad number of systems or shifts");
    for (int r = 0; r < nsys; r++) CHECK_PTR(ctx, srcs[r]);
    if (sols)
        for (int i = 0; i < nsys * n; i++)
            if (sols[i] && !aligned16(sols[i])) return stag_fail(ctx, STAG_ERR_ARG, "sols[%d] not aligned", i);
    const long n3 = 3L * ctx->g.Vh;
    double2* X = (double2*)ws_get(ctx, WS_MX, sizeof(double2) * n3 * STAG_MAXSHIFT * STAG_MAXRHS);
    if (!X) return stag_fail(ctx, STAG_ERR_OOM, "solution workspace");
    int st = multishift_solve_multi(ctx, mass, nsys, n, shifts, (const double2* const*)srcs, X, tol, maxit, mode,
                                    infos, S(stream));
    if (st) return st;
    if (sols)
        for (int r = 0; r < nsys; r++)
            for (int k = 0; k < n; k++)
                if (sols[r * n + k])
                    STAG_CUDA(ctx, cudaMemcpyAsync(sols[r * n + k], X + ((size_t)r * STAG_MAXSHIFT + k) * n3,
                                                   sizeof(double2) * n3, cudaMemcpyDeviceToDevice, S(stream)));
    STAG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return STAG_OK;
}

int stag_rational_apply(stag_ctx* ctx, double mass, const stag_rational* r, const double* src, double* out,
                        double tol, int maxit, int mode, stag_solve_info* info, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    CHECK_PTR(ctx, src);
    CHECK_PTR(ctx, out);
    if (!r || r->n < 1 || r->n > STAG_MAXSHIFT) return stag_fail(ctx, STAG_ERR_ARG, "bad rational");
    if (src == out) return stag_fail(ctx, STAG_ERR_ARG, "src and out alias");
    const long n3 = 3L * ctx->g.Vh;
    double2* X = (double2*)ws_get(ctx, WS_FX, sizeof(double2) * n3 * STAG_MAXSHIFT);
    if (!X) return stag_fail(ctx, STAG_ERR_OOM, "solution workspace");
    double2* sols[STAG_MAXSHIFT];
    for (int k = 0; k < r->n; k++) sols[k] = nullptr;  // X already holds them
    int st = multishift_solve(ctx, mass, r->n, r->b, (const double2*)src, sols, tol, maxit, mode, info, S(stream));
    if (st) return st;
    if ((st = blas_rational_combine(ctx, r->a0, r->a, r->n, (const double2*)src, X, (double2*)out, S(stream))))
        return st;
    STAG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return STAG_OK;
}

// ---------------------------------------------------------------- forces and updates

int stag_gauge_force(stag_ctx* ctx, double beta, double* force_out, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    CHECK_PTR(ctx, force_out);
    double* F = (double*)ws_get(ctx, WS_FORCE, sizeof(double) * 64 * (size_t)ctx->g.Vh);
    if (!F) return stag_fail(ctx, STAG_ERR_OOM, "force buffer");
    int st = gauge_force_internal_prec(ctx, beta, F, 0, 0, S(stream));
    if (st) return st;
    return momenta_to_canonical(ctx, F, force_out, S(stream));
}

int stag_fermion_force(stag_ctx* ctx, double mass, const stag_rational* r, const double* phi, double* force_out,
                       double tol, int maxit, int mode, stag_solve_info* info, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    CHECK_PTR(ctx, phi);
    CHECK_PTR(ctx, force_out);
    if (!r || r->n < 1 || r->n > STAG_MAXSHIFT) return stag_fail(ctx, STAG_ERR_ARG, "bad rational");
    const long n3 = 3L * ctx->g.Vh;
    double2* X = (double2*)ws_get(ctx, WS_FX, sizeof(double2) * n3 * STAG_MAXSHIFT);
    double* F = (double*)ws_get(ctx, WS_FORCE, sizeof(double) * 64 * (size_t)ctx->g.Vh);
    if (!X || !F) return stag_fail(ctx, STAG_ERR_OOM, "force workspace");
    int st = multishift_solve(ctx, mass, r->n, r->b, (const double2*)phi, nullptr, tol, maxit, mode, info, S(stream));
    if (st) return st;
    if ((st = fermion_force_assemble(ctx, r, X, F, 0, S(stream)))) return st;
    return momenta_to_canonical(ctx, F, force_out, S(stream));
}

int stag_update_links(stag_ctx* ctx, double eps, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    return update_links(ctx, eps, S(stream));
}

int stag_momenta_heatbath(stag_ctx* ctx, uint32_t seed, uint32_t traj, void* stream) {
    CHECK_CTX(ctx);
    return momenta_heatbath(ctx, seed, traj, S(stream));
}

int stag_pf_gaussian(stag_ctx* ctx, uint32_t seed, uint32_t traj, int pf, double* out, void* stream) {
    CHECK_CTX(ctx);
    CHECK_PTR(ctx, out);
    return pf_gaussian(ctx, seed, traj, pf, (double2*)out, S(stream));
}

int stag_kinetic(stag_ctx* ctx, double* out, void* stream) {
    CHECK_CTX(ctx);
    if (!out) return stag_fail(ctx, STAG_ERR_ARG, "out is null");
    int st = kinetic_sum(ctx, ctx->dscal + 3, S(stream));
    if (st) return st;
    return read_scalar(ctx, 3, out, S(stream));
}

// ---------------------------------------------------------------- trajectory

static int check_params(stag_ctx* ctx, const stag_params* p) {
    if (p->nsteps < 1 || !(p->tau > 0) || p->npf < 0 || p->npf > STAG_MAXPF || p->maxit < 1 || p->ngauge < 0 ||
        p->ngauge > 1000)
        return stag_fail(ctx, STAG_ERR_ARG, "bad trajectory parameters");
    if (p->integrator != STAG_INT_LEAPFROG && p->integrator != STAG_INT_OMELYAN)
        return stag_fail(ctx, STAG_ERR_ARG, "unknown integrator");
    const stag_rational* rs[3] = {&p->hb, &p->act, &p->force};
    for (auto r : rs)
        if (r->n < 1 || r->n > STAG_MAXSHIFT) return stag_fail(ctx, STAG_ERR_ARG, "bad rational degree");
    return STAG_OK;
}

int stag_md_trajectory(stag_ctx* ctx, const stag_params* p, stag_traj_info* out, void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    if (!p || !out) return stag_fail(ctx, STAG_ERR_ARG, "null params or output");
    int st = check_params(ctx, p);
    if (st) return st;
    const int graphs = ctx->use_graphs;
    ctx->use_graphs = p->use_graphs ? 1 : 0;
    st = rhmc_trajectory(ctx, p, out, S(stream));
    ctx->use_graphs = graphs;
    return st;
}

int stag_md_integrate(stag_ctx* ctx, const stag_params* p, const double* phi, long long* cg_iters, int* n_force,
                      void* stream) {
    CHECK_CTX(ctx);
    CHECK_GAUGE(ctx);
    if (!p) return stag_fail(ctx, STAG_ERR_ARG, "null params");
    int st = check_params(ctx, p);
    if (st) return st;
    if (p->npf > 0 && !phi) return stag_fail(ctx, STAG_ERR_ARG, "null pseudofermions");
    long long it = 0;
    int nf = 0;
    const int graphs = ctx->use_graphs;
    ctx->use_graphs = p->use_graphs ? 1 : 0;
    st = md_integrate_public(ctx, p, (const double2*)phi, &it, &nf, S(stream));
    ctx->use_graphs = graphs;
    if (st) return st;
    STAG_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    if (cg_iters) *cg_iters = it;
    if (n_force) *n_force = nf;
    return STAG_OK;
}

}  // extern "C"

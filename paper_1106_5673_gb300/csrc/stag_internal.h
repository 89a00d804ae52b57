// stag_internal.h -- context object and cross-file declarations of the
// GB300 staggered-RHMC library.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/stag.h"
#include "lattice.cuh"

#define STAG_RED_MAXBLOCKS 8192  // max blocks of any reducing kernel
#define STAG_NSCAL 256           // doubles in the device scalar area

// Work buffers, allocated on first use and grown on demand.
enum WsSlot {
    WS_STAGE = 0,   // canonical <-> internal conversion staging
    WS_R64, WS_P64, WS_W64, WS_T64,       // FP64 solver vectors (T: odd-parity temp)
    WS_PK64, WS_XK64,                     // FP64 shifted p_k / x_k, n vectors each
    WS_R32, WS_P32, WS_W32, WS_T32,       // FP32 solver vectors
    WS_PK32, WS_XK32,                     // FP32 shifted p_k / x_k
    WS_XHI, WS_RHI, WS_B64,               // refinement (FP64 solution, residual, rhs)
    WS_XLO,                               // refinement FP32 correction
    WS_FX, WS_FY,                         // force: X_k (even), Y_k (odd), FP64
    WS_PHI, WS_RGAUSS, WS_RAT,            // trajectory: pseudofermions, R, r(M) phi
    WS_FORCE,                             // force accumulator [4][2][8][Vh] doubles
    WS_BR, WS_BW, WS_BT, WS_BPART,        // batched refinement: residuals, M p, odd temp, partials
    WS_TUNE,                              // autotuner test vectors
    WS_MR, WS_MP, WS_MW, WS_MT,           // batched multi-system solver: per-system vectors
    WS_MPK, WS_MXK, WS_MX,                // per-system shifted p_k / x_k (low precision), FP64 solutions
    WS_FCG,                               // flexible CG vectors
    WS_LX,                                // learned mode: solution of the lightest shift
    WS_RPK, WS_RXL,                       // batched refinement: search directions, FP32 corrections
    WS_NSLOTS
};

// Device-resident scalar state of one multi-shift CG (Eq. (13)).
struct MSState {
    double rr, bb, alpha, alpha_old, beta, beta_old, pw, tol2bb, c0;
    double zeta[STAG_MAXSHIFT], zeta_old[STAG_MAXSHIFT], zeta_next[STAG_MAXSHIFT];
    double ak[STAG_MAXSHIFT], bk[STAG_MAXSHIFT], shifts[STAG_MAXSHIFT];
    int upd_x[STAG_MAXSHIFT], active[STAG_MAXSHIFT], iters_shift[STAG_MAXSHIFT];
    int n, base, iter, maxit;
    int live;       // 1 while iterating
    int stop_next;  // set by the residual update, applied by the last kernel of the iteration
    int n_active;
    int nonfinite;
    int pend;       // 1: the shifted vectors' update of the last iteration is still to be applied
    int keep;       // stop once at most this many shifts are still unconverged (their refinement finishes them)
};

// Device-resident scalar state of one single-shift CG with reliable updates.
struct CGState {
    double rr, rr_prev, rr_max, alpha, beta, pw, bb, tol2bb, delta2, c0;
    int iter, maxit, live, stop_next, want_reliable, nonfinite;
};

// Device-resident state of the batched refinement: one CG per right-hand side
// (shift), all advanced by the same kernels.  RHS j uses vector slot j.
struct BCGState {
    double rr[STAG_MAXSHIFT], rr_prev[STAG_MAXSHIFT], rr_max[STAG_MAXSHIFT];
    double alpha[STAG_MAXSHIFT], beta[STAG_MAXSHIFT], c0[STAG_MAXSHIFT];
    double tol2bb[STAG_MAXSHIFT], delta2;
    int act[STAG_MAXSHIFT];       // active RHS slots, compacted; n_act of them
    int uact[STAG_MAXSHIFT];      // slots updated by the current iteration (fused path)
    int want_rel[STAG_MAXSHIFT];  // per slot: reliable update requested
    int iter[STAG_MAXSHIFT];      // per slot: iterations done
    int n_act, n_uact, maxit, live, stop_next, nonfinite;
};

struct stag_ctx {
    Geom g;
    int device;
    char err[512];
    double2* U64;       // [4][2][6][Vh]
    float4* U32;        // [4][2][3][Vh]
    float4* U32lo;      // [4][2][3][Vh]  fl32(U64 - U32): low words of the float-float links
    uint2* U16;         // [4][2][3][Vh]
    float4* U8;         // [4][2][2][Vh]  8-real FP32 links, built on first use (null until then)
    long long gauge_gen;  // incremented whenever the links change
    long long u8_gen;     // gauge_gen at the last rebuild of U8
    double2* U64_save;  // copy kept for the Metropolis reject
    double* mom;        // [4][2][8][Vh]
    int gauge_loaded;
    double* partials;   // reduction partials
    unsigned int* counter;  // last-block counters ([0] and the group counters of grid_reduce_series)
    size_t counter_bytes;
    double* gpart;      // group sums of grid_reduce_series
    double* dscal;      // device scalar area (STAG_NSCAL doubles)
    double* hscal;      // pinned host mirror of dscal
    // the batched refinement's own reduction buffers and scalars, so that it
    // can run on the second stream while the shifted CG runs on the first
    double* partials2;
    unsigned int* counter2;
    double* gpart2;
    double* dscal2;
    double* hscal2;
    cudaStream_t s2;      // second stream (the early refinement)
    cudaEvent_t ev_ref;   // end of the refinement's chunk in flight and of its state copy
    MSState* ms;        // device multi-shift state
    MSState* ms_host;   // pinned host mirror
    MSState* ms_poll;   // pinned copy read one chunk behind (pipelined polling)
    cudaEvent_t ev_poll;  // marks the arrival of ms_poll
    CGState* cg;        // device single-shift state
    CGState* cg_host;   // pinned host mirror
    BCGState* bcg;      // device batched-refinement state
    BCGState* bcg_host; // pinned host mirror
    MSState* msm;       // device states of the batched multi-system solver [STAG_MAXRHS]
    MSState* msm_host;  // pinned host mirror
    double* mm_partials;  // its reduction partials
    void* ws[WS_NSLOTS];
    size_t ws_bytes[WS_NSLOTS];
    size_t fixed_bytes;
    std::map<std::string, cudaGraphExec_t> graphs;
    int num_sms;
    long long nlaunch;  // kernels launched (graph nodes counted individually)
    int tpb[5];         // tuned threads per block of the hop kernels, per link precision (0: default)
    int tuned;
    stag_net* net;      // preconditioner of STAG_SOLVE_LEARNED (borrowed)
    int use_graphs;     // 1: solver iteration chunks run as cached CUDA graphs
};

// threads per block of the hop kernels for link precision lp (autotuned, else 128)
static inline int hop_tpb(const stag_ctx* c, int lp) { return c->tpb[lp] > 0 ? c->tpb[lp] : 128; }
void ctx_clear_graphs(stag_ctx* ctx);
int autotune_hops(stag_ctx* ctx, cudaStream_t s);

// ---------------------------------------------------------------- utilities (capi.cu)
int stag_fail(stag_ctx* ctx, int code, const char* fmt, ...);
int stag_cuda_check(stag_ctx* ctx, cudaError_t e, const char* what);
void* ws_get(stag_ctx* ctx, int slot, size_t bytes);
#define STAG_CUDA(ctx, call)                                              \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return stag_cuda_check(ctx, e_, #call);    \
    } while (0)
#define STAG_LAUNCH_CHECK(ctx, what)                                      \
    do {                                                                  \
        (ctx)->nlaunch++;                                                 \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) return stag_cuda_check(ctx, e_, what);     \
    } while (0)

static inline int nblocks(long n, int threads) { return (int)((n + threads - 1) / threads); }


// ---------------------------------------------------------------- gauge.cu
int gauge_from_canonical(stag_ctx* ctx, const double* dev_links, cudaStream_t s);
int gauge_to_canonical(stag_ctx* ctx, double* dev_links, cudaStream_t s);
int momenta_from_canonical(stag_ctx* ctx, const double* dev_w, cudaStream_t s);
int momenta_to_canonical(stag_ctx* ctx, const double* src_internal, double* dev_w, cudaStream_t s);
int plaquette_sum(stag_ctx* ctx, double* dst_dev, cudaStream_t s);         // sum Re Tr U_P / 3
int kinetic_sum(stag_ctx* ctx, double* dst_dev, cudaStream_t s);           // 1/2 sum w^2
// F (internal layout) = coeff * gauge force (+ F if accumulate)
int gauge_force_internal(stag_ctx* ctx, double beta, double* F, int accumulate, cudaStream_t s);
int update_links(stag_ctx* ctx, double eps, cudaStream_t s);
// the 8-real FP32 links, rebuilt from the FP64 master if the links changed since
const float4* links_r8(stag_ctx* ctx, cudaStream_t s);
int update_momenta(stag_ctx* ctx, const double* F, double eps, cudaStream_t s);
int momenta_heatbath(stag_ctx* ctx, uint32_t seed, uint32_t traj, cudaStream_t s);
int pf_gaussian(stag_ctx* ctx, uint32_t seed, uint32_t traj, int pf, double2* out, cudaStream_t s);
int metro_uniform(stag_ctx* ctx, uint32_t seed, uint32_t traj, double* dst_dev, cudaStream_t s);

// ---------------------------------------------------------------- dslash.cu
// out = 1/2 hop (plain D restricted to out_par)
int dslash_apply(stag_ctx* ctx, int prec, const void* in, void* out, int out_par, cudaStream_t s);
// out = c * in - D_eo D_oe in, with tmp (odd) scratch
int mee_apply(stag_ctx* ctx, int prec, double c, const void* in, void* out, void* tmp, cudaStream_t s);
// multi-RHS: out[k] = D_oe in[k] for nrhs FP64 vectors (contiguous, stride Vh*3)
int dslash_multi64(stag_ctx* ctx, const double2* in, double2* out, int nrhs, int out_par, cudaStream_t s);

// ---------------------------------------------------------------- blas.cu
int blas_dot_re(stag_ctx* ctx, int prec, const void* a, const void* b, double* dst_dev, cudaStream_t s);
int blas_copy_d2f(stag_ctx* ctx, const double2* in, float2* out, long nvec_sites, cudaStream_t s);
int blas_copy_f2d(stag_ctx* ctx, const float2* in, double2* out, long nvec_sites, cudaStream_t s);
// out = a0 * src + sum_k a_k x_k (FP64)
int blas_rational_combine(stag_ctx* ctx, double a0, const double* a, int n, const double2* src,
                          const double2* x, double2* out, cudaStream_t s);

// ---------------------------------------------------------------- solver.cu
int multishift_solve(stag_ctx* ctx, double mass, int n, const double* shifts, const double2* src,
                     double2* const* sols, double tol, int maxit, int mode, stag_solve_info* info,
                     cudaStream_t s);

// ---------------------------------------------------------------- refine.cu
// Systems of a batched refinement: slot k solves (M_ee + c_k - m^2) x_k = b_k,
// i.e. M_ee with diagonal c_k = m^2 + shift; bb_k = |b_k|^2.
struct RefSlots {
    const double2* b[STAG_MAXSHIFT];
    double2* x[STAG_MAXSHIFT];
    double c[STAG_MAXSHIFT];
    double bb[STAG_MAXSHIFT];
};
int batched_true_residuals(stag_ctx* ctx, const RefSlots& S, const int* ks, int nk, float2* R, double* rr_out,
                           cudaStream_t s);
int refine_batched(stag_ctx* ctx, int lp, const RefSlots& S, const int* ks, int nk, float2* R, double tol, int maxit,
                   double* rr, int* iters, int* reliable, int* matvecs, cudaStream_t s);

// The batched refinement driven chunk by chunk: slots can join while it runs
// (add), a chunk runs asynchronously on `s` (launch), and the host processes
// it when it has finished (ready, poll: reliable updates, parking, the active
// list).  refine_batched is begin + add + finish on one stream; the mixed
// shifted solve also uses it on the context's second stream, where shifts
// start their refinement as soon as the FP32 shifted CG has converged them.
struct Refiner {
    stag_ctx* ctx = nullptr;
    cudaStream_t s = 0;
    int lp = 1;
    const RefSlots* S = nullptr;
    double tol = 0.0;
    int maxit = 0;
    double* rr = nullptr;  // per slot: the latest FP64-accurate true residual^2 (caller's array)
    int* iters = nullptr;  // per slot: iterations of its refinement (caller's array)
    int nreliable = 0, nmatvec = 0;
    float2 *R = nullptr, *P = nullptr, *W = nullptr, *T = nullptr, *XL = nullptr;
    double* part = nullptr;
    int chunk = 32, fused = 1, tpb = 128, bcd_bps = 8, trace = 0;
    double delta = 0.03;
    int active[STAG_MAXSHIFT] = {0}, done[STAG_MAXSHIFT] = {0};
    int order[STAG_MAXSHIFT] = {0}, norder = 0;  // slots in the order they joined
    int remaining = 0;
    bool flying = false, dirty = false;
    int begin(stag_ctx* c, int link_prec, const RefSlots* slots, double tolerance, int max_iter, double* rr_io,
              int* iters_out, cudaStream_t stream);
    int add(const int* ks, int nk);  // the slots' rows of R and rr[] hold their true residuals (above tol)
    int launch();                    // one chunk, asynchronous (no-op when no slot is active)
    bool ready() const;              // the chunk in flight has finished
    int poll();                      // processes the finished chunk (waits for it first)
    int finish();                    // runs until every slot has met tol or its iteration cap
};

// ---------------------------------------------------------------- msmulti.cu
int multishift_solve_multi(stag_ctx* ctx, double mass, int nsys, int n, const double* shifts,
                           const double2* const* srcs, double2* X, double tol, int maxit, int mode,
                           stag_solve_info* infos, cudaStream_t s);

// ---------------------------------------------------------------- gcnn.cu
int net_create(stag_ctx* ctx, unsigned seed, stag_net** out);
void net_destroy(stag_net* net);
int net_apply(stag_net* net, const double2* b, double2* z, cudaStream_t s);
int net_loss_grad(stag_net* net, int npairs, const double2* const* bs, const double2* const* xs, double* loss,
                  cudaStream_t s);
int net_train(stag_net* net, int npairs, const double2* const* bs, const double2* const* xs, int epochs, int batch,
              double lr, double* loss_out, cudaStream_t s);
int net_get_weights(stag_net* net, int layer, float* host);
int net_set_weights(stag_net* net, int layer, const float* host);
int net_get_grads(stag_net* net, int layer, float* host);
int net_nweights(const stag_net* net, int layer);
int fcg_solve(stag_ctx* ctx, stag_net* net, double mass, double shift, const double2* b, double2* x, double tol,
              int maxit, int* iters, double* true_resid, cudaStream_t s);

// ---------------------------------------------------------------- force.cu
// F (internal) (+)= fermion force for sum_k a_k X_k, Y_k = D_oe X_k; X contiguous FP64
int fermion_force_assemble(stag_ctx* ctx, const stag_rational* r, const double2* X, double* F,
                           int accumulate, cudaStream_t s);

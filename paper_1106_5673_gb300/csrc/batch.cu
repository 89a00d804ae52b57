// batch.cu -- the even/odd hop of Eq. (4) for many right-hand sides on several
// lattices of different sizes in one launch.
//
// The work is a list of tiles (lattice, block of output sites, group of NR
// right-hand sides); each block of the grid walks the list with a grid
// stride (a persistent grid of resident blocks, or one block per tile).
// Within a tile every link is loaded once and applied to the NR right-hand
// sides (FP32 vectors, FP32 or BF16 12-real links).  The block size, NR, the
// grid form and the tile order (site blocks or right-hand-side groups
// fastest) are chosen by a timed search on the first call for each
// combination of lattices, right-hand-side counts and link precision, and
// cached for the process.
#include <map>
#include <mutex>
#include <stdio.h>
#include <stdlib.h>
#include <string>

#include "hop.cuh"
#include "stag_internal.h"

namespace {

struct BatchLat {
    Geom g;
    const void* U;
    const float2* in;
    float2* out;
    size_t stride;  // complex entries between right-hand sides (3 Vh)
    int nrhs;
    int nsb;    // blocks of output sites
    int tile0;  // first tile of this lattice
};

struct BatchDesc {
    BatchLat l[STAG_MAXLAT];
    int nlat, total_tiles, out_par;
    int group_fastest;  // tile order within a lattice: 0 site blocks fastest, 1 right-hand-side groups fastest
};

// launch shape chosen by the tuner: block size, right-hand sides per thread,
// grid form (0 persistent: resident blocks walk the tiles; 1 one block per
// tile) and tile order
struct BatchCfg {
    int tpb, nr, one_per_tile, group_fastest;
};

template <int LP, int NR>
__global__ void __launch_bounds__(256) k_hop_batch(const __grid_constant__ BatchDesc d) {
    for (int tile = blockIdx.x; tile < d.total_tiles; tile += gridDim.x) {
        int l = 0;
        while (l + 1 < d.nlat && tile >= d.l[l + 1].tile0) l++;
        const BatchLat& L = d.l[l];
        const int t = tile - L.tile0;
        int sb, q0;
        if (d.group_fastest) {
            const int ng = (L.nrhs + NR - 1) / NR;
            sb = t / ng;
            q0 = (t - sb * ng) * NR;
        } else {
            sb = t % L.nsb;
            q0 = (t / L.nsb) * NR;
        }
        const int h = sb * blockDim.x + threadIdx.x;
        if (h >= L.g.Vh) continue;
        const int nj = min(NR, L.nrhs - q0);
        int js[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) js[q] = (q < nj) ? q0 + q : 0;
        const Site s = site_of(L.g, h, d.out_par);
        Vec3<float> acc[NR];
        hop2_multiR<float, LP, NR>(L.g, L.U, L.in, L.stride, js, nj, h, d.out_par, s, acc);
#pragma unroll
        for (int q = 0; q < NR; q++) {
            if (q < nj) {
#pragma unroll
                for (int a = 0; a < 3; a++) acc[q].c[a] = 0.5f * acc[q].c[a];
                st_vec(L.out + (size_t)(q0 + q) * L.stride, h, acc[q]);
            }
        }
    }
}

template <int LP, int NR>
int launch_batch(BatchDesc& d, const stag_ctx* const* ctxs, int tpb, int one_per_tile, int num_sms, cudaStream_t s) {
    int tiles = 0;
    for (int l = 0; l < d.nlat; l++) {
        BatchLat& L = d.l[l];
        L.nsb = nblocks(L.g.Vh, tpb);
        L.tile0 = tiles;
        tiles += L.nsb * ((L.nrhs + NR - 1) / NR);
    }
    d.total_tiles = tiles;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hop_batch<LP, NR>, tpb, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int grid = (one_per_tile || tiles < per_sm * num_sms) ? tiles : per_sm * num_sms;
    k_hop_batch<LP, NR><<<grid, tpb, 0, s>>>(d);
    (void)ctxs;
    return cudaGetLastError() == cudaSuccess ? STAG_OK : STAG_ERR_CUDA;
}

int launch_cfg(BatchDesc& d, const stag_ctx* const* ctxs, int lp, const BatchCfg& c, int num_sms, cudaStream_t s) {
    d.group_fastest = c.group_fastest;
    const int tpb = c.tpb, opt = c.one_per_tile;
    if (lp == LP16) {
        switch (c.nr) {
            case 1: return launch_batch<LP16, 1>(d, ctxs, tpb, opt, num_sms, s);
            case 2: return launch_batch<LP16, 2>(d, ctxs, tpb, opt, num_sms, s);
            case 4: return launch_batch<LP16, 4>(d, ctxs, tpb, opt, num_sms, s);
            default: return launch_batch<LP16, 8>(d, ctxs, tpb, opt, num_sms, s);
        }
    }
    switch (c.nr) {
        case 1: return launch_batch<LP32, 1>(d, ctxs, tpb, opt, num_sms, s);
        case 2: return launch_batch<LP32, 2>(d, ctxs, tpb, opt, num_sms, s);
        case 4: return launch_batch<LP32, 4>(d, ctxs, tpb, opt, num_sms, s);
        default: return launch_batch<LP32, 8>(d, ctxs, tpb, opt, num_sms, s);
    }
}

std::mutex g_tune_mutex;
std::map<std::string, BatchCfg> g_tuned;  // key -> launch shape

}  // namespace

extern "C" int stag_dslash_batch(int nlat, stag_ctx* const* ctxs, const void* const* in, void* const* out,
                                 const int* nrhs, int out_par, int prec, int* tuned_cfg, void* stream) {
    if (nlat < 1 || nlat > STAG_MAXLAT || !ctxs || !in || !out || !nrhs || (out_par != 0 && out_par != 1))
        return STAG_ERR_ARG;
    if (prec != STAG_PREC_F32 && prec != STAG_PREC_BF16) return STAG_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    BatchDesc d;
    memset(&d, 0, sizeof(d));
    d.nlat = nlat;
    d.out_par = out_par;
    const int lp = (prec == STAG_PREC_F32) ? LP32 : LP16;
    std::string key = std::to_string(prec) + ":" + std::to_string(out_par);
    for (int l = 0; l < nlat; l++) {
        stag_ctx* c = ctxs[l];
        if (!c || !in[l] || !out[l] || nrhs[l] < 1) return STAG_ERR_ARG;
        if (!c->gauge_loaded) return stag_fail(c, STAG_ERR_STATE, "no gauge field loaded");
        if (c->device != ctxs[0]->device) return stag_fail(c, STAG_ERR_ARG, "lattices on different devices");
        BatchLat& L = d.l[l];
        L.g = c->g;
        L.U = (lp == LP32) ? (const void*)c->U32 : (const void*)c->U16;
        L.in = (const float2*)in[l];
        L.out = (float2*)out[l];
        L.stride = 3 * (size_t)c->g.Vh;
        L.nrhs = nrhs[l];
        for (int m = 0; m < 4; m++) key += ":" + std::to_string(c->g.L[m]);
        key += "x" + std::to_string(nrhs[l]);
    }
    const int num_sms = ctxs[0]->num_sms;
    BatchCfg cfg = {128, 4, 0, 0};
    bool have = false;
    // STAG_BATCH_CFG="threads,rhs_per_thread,one_block_per_tile,group_fastest"
    // forces a launch shape (no search, nothing cached)
    const char* forced = getenv("STAG_BATCH_CFG");
    BatchCfg fc;
    if (forced && sscanf(forced, "%d,%d,%d,%d", &fc.tpb, &fc.nr, &fc.one_per_tile, &fc.group_fastest) == 4) {
        const bool ok_tpb = fc.tpb == 64 || fc.tpb == 128 || fc.tpb == 256;
        const bool ok_nr = fc.nr == 1 || fc.nr == 2 || fc.nr == 4 || fc.nr == 8;
        if (!ok_tpb || !ok_nr) return STAG_ERR_ARG;
        fc.one_per_tile = fc.one_per_tile != 0;
        fc.group_fastest = fc.group_fastest != 0;
        cfg = fc;
        have = true;
    }
    if (!have) {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            cfg = it->second;
            have = true;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return stag_cuda_check(ctxs[0], cudaGetLastError(), "stream");
    if (!have && cap == cudaStreamCaptureStatusNone) {
        // timed search over block size, right-hand sides per thread, grid form and tile order
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            return stag_cuda_check(ctxs[0], cudaGetLastError(), "tuning events");
        const int tpbs[3] = {64, 128, 256}, nrs[4] = {1, 2, 4, 8};
        float best = 1e30f;
        for (int mode = 0; mode < 4; mode++)
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 4; b++) {
                    const BatchCfg c = {tpbs[a], nrs[b], mode & 1, mode >> 1};
                    BatchDesc dd = d;
                    if (launch_cfg(dd, ctxs, lp, c, num_sms, s)) return stag_fail(ctxs[0], STAG_ERR_CUDA, "batch tune");
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < 3; r++) launch_cfg(dd, ctxs, lp, c, num_sms, s);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess)
                        return stag_cuda_check(ctxs[0], cudaGetLastError(), "tune");
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) {
                        best = ms;
                        cfg = c;
                    }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const char* tr = getenv("STAG_TRACE_BATCH");
        if (tr && atoi(tr))
            fprintf(stderr, "[batch] %s: %d threads, %d rhs/thread, %s grid, %s fastest, %.3f ms\n", key.c_str(), cfg.tpb,
                    cfg.nr, cfg.one_per_tile ? "one block per tile" : "persistent",
                    cfg.group_fastest ? "rhs groups" : "site blocks", best / 3);
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tuned[key] = cfg;
    }
    if (tuned_cfg) {
        tuned_cfg[0] = cfg.tpb;
        tuned_cfg[1] = cfg.nr;
    }
    const int st = launch_cfg(d, ctxs, lp, cfg, num_sms, s);
    ctxs[0]->nlaunch++;
    if (st) return stag_fail(ctxs[0], st, "batched hop launch: %s", cudaGetErrorString(cudaGetLastError()));
    return STAG_OK;
}

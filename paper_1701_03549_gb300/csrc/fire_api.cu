// C ABI of libfire (see include/fire.h): contexts, maps, argument checks,
// host <-> device staging and kernel launch configuration.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include "fire_internal.h"

using namespace fire;

namespace fire {

int set_err(fire_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int cuda_err(fire_ctx *ctx, cudaError_t e, const char *what)
{
    return set_err(ctx, FIRE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ensure_device(fire_ctx *ctx)
{
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGetDevice");
    if (cur != ctx->device) {
        e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
    }
    return FIRE_OK;
}

int grow_device(fire_ctx *ctx, void **buf, size_t *cap, size_t need,
                const char *what)
{
    if (need <= *cap) return FIRE_OK;
    ctx->epoch++;   // cached graphs may reference the old buffer
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    size_t n = need + need / 4 + 256;
    if (ctx->fail_alloc_after >= 0 && ctx->fail_alloc_after-- == 0)
        return set_err(ctx, FIRE_ENOMEM, "cudaMalloc(%zu) for %s: failure "
                       "forced by fire_debug_fail_alloc", n, what);
    cudaError_t e = cudaMalloc(buf, n);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return set_err(ctx, FIRE_ENOMEM, "cudaMalloc(%zu) for %s: %s", n, what,
                       cudaGetErrorString(e));
    }
    *cap = n;
    return FIRE_OK;
}

int grow_pinned(fire_ctx *ctx, size_t need)
{
    if (need <= ctx->host_pinned_bytes) return FIRE_OK;
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    ctx->host_pinned = nullptr;
    ctx->host_pinned_bytes = 0;
    size_t n = need + need / 4 + 256;
    cudaError_t e = cudaMallocHost(&ctx->host_pinned, n);
    if (e != cudaSuccess)
        return set_err(ctx, FIRE_ENOMEM, "cudaMallocHost(%zu): %s", n,
                       cudaGetErrorString(e));
    ctx->host_pinned_bytes = n;
    return FIRE_OK;
}

size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

bool valid_map(const fire_map *m) { return m && m->ctx && m->feat; }

// Launch shape of the simulation kernel for maps of up to `ntiles` tiles:
// an explicit fire_set_launch override, else the autotuned shape recorded for
// this tile count, else a heuristic.
int plan_launch(fire_ctx *ctx, int ntiles, long long n, LaunchPlan *p, bool burn)
{
    int warps = 0, bps = 0, queue = 0, state = FIRE_STATE_AUTO;
    const bool override = ctx->warps_per_block || ctx->blocks_per_sm ||
                          ctx->queue_entries || ctx->state_mode;
    if (override) {
        warps = ctx->warps_per_block;
        bps = ctx->blocks_per_sm;
        queue = ctx->queue_entries;
        state = ctx->state_mode;
    } else {
        for (const TuneEntry &t : ctx->tuned) {
            if (t.ntiles == ntiles) {
                warps = t.warps;
                bps = t.bps;
                queue = t.queue;
                state = t.state;
            }
        }
    }
    int nwarps = warps > 0 ? warps : (ntiles <= 16 ? 4 : (ntiles <= 64 ? 8 : 16));
    nwarps = std::min(nwarps, kSimMaxThreads / 32);
    int qcap = queue > 0 ? queue : 4096;
    SimLayout L = sim_layout(ntiles, qcap, true);
    // the burn-time variant keeps its state in global memory; a shape tuned
    // for shared-memory state gives way to the global-state shape that is
    // fastest on the plain kernel's benchmarks (4 warps x 8 blocks per SM)
    if (burn && !override && state != FIRE_STATE_GLOBAL) {
        nwarps = 4;
        bps = 8;
        qcap = queue = 3072;
    }
    if (burn) state = FIRE_STATE_GLOBAL;
    bool smem_state = state == FIRE_STATE_SHARED ||
                      (state == FIRE_STATE_AUTO && L.total <= ctx->max_smem_optin);
    if (smem_state && L.total > ctx->max_smem_optin)
        return set_err(ctx, FIRE_EINVAL, "state of %d tiles does not fit in "
                       "shared memory", ntiles);
    if (!smem_state) {
        if (queue <= 0) {
            qcap = 16384;
            if (sim_layout(ntiles, qcap, false).total > ctx->max_smem_optin)
                qcap = 4096;
        }
        L = sim_layout(ntiles, qcap, false);
        if (L.total > ctx->max_smem_optin)
            return set_err(ctx, FIRE_EINVAL, "worklists of %d tiles do not fit in "
                           "shared memory", ntiles);
    }
    const void *kfn = burn ? simulate_burn_kernel_ptr() : simulate_kernel_ptr(smem_state);
    cudaError_t e = cudaFuncSetAttribute(
        kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaFuncSetAttribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, nwarps * 32,
                                                      L.total);
    if (e != cudaSuccess) return cuda_err(ctx, e, "occupancy");
    if (occ < 1)
        return set_err(ctx, FIRE_EINVAL, "kernel does not fit (%zu B smem, %d "
                       "warps)", L.total, nwarps);
    const int use = bps > 0 ? std::min(bps, occ) : occ;
    p->nwarps = nwarps;
    p->qcap = qcap;
    p->smem_state = smem_state;
    p->L = L;
    p->grid = (int)std::min((long long)use * ctx->num_sms, std::max(n, 1ll));
    return FIRE_OK;
}

}  // namespace fire

extern "C" {

int fire_create(fire_ctx **out, int device, void *cuda_stream)
{
    if (!out) return FIRE_EINVAL;
    *out = nullptr;
    fire_ctx *ctx = new (std::nothrow) fire_ctx();
    if (!ctx) return FIRE_ENOMEM;
    ctx->device = device;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        delete ctx;
        return FIRE_ECUDA;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete ctx; return FIRE_ECUDA; }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete ctx; return FIRE_ECUDA; }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->max_smem_optin = prop.sharedMemPerBlockOptin;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete ctx; return FIRE_ECUDA; }
        ctx->own_stream = true;
    }
    e = cudaMalloc(&ctx->counter, 256);
    if (e != cudaSuccess) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return FIRE_ENOMEM;
    }
    cudaMemset(ctx->counter, 0, 256);
    *out = ctx;
    return FIRE_OK;
}

void fire_destroy(fire_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (GraphEntry &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    if (ctx->table) cudaFree(ctx->table);
    if (ctx->order) cudaFree(ctx->order);
    if (ctx->lpt) cudaFree(ctx->lpt);
    if (ctx->counter) cudaFree(ctx->counter);
    if (ctx->staging) cudaFree(ctx->staging);
    if (ctx->gstate) cudaFree(ctx->gstate);
    if (ctx->burn_aux) cudaFree(ctx->burn_aux);
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *fire_last_error(const fire_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

int fire_sync(fire_ctx *ctx)
{
    FIRE_NVTX("fire_sync");
    if (!ctx) return FIRE_EINVAL;
    int rc = ensure_device(ctx);
    if (rc) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    uint32_t errw = 0;
    CUDA_TRY(ctx, cudaMemcpy(&errw, ctx->counter + 1, 4, cudaMemcpyDeviceToHost),
             "read error word");
    if (errw) {
        cudaMemset(ctx->counter + 1, 0, 4);
        return set_err(ctx, FIRE_ETIMEOUT, "a bounded device wait ran out");
    }
    // asynchronous fire_simulate_batch_noalloc calls keep their error word
    // in the no-alloc scratch of this device
    bool na = false;
    if (noalloc_take_error(ctx->device, &na) != FIRE_OK)
        return set_err(ctx, FIRE_ECUDA, "read the no-alloc error word");
    if (na)
        return set_err(ctx, FIRE_ETIMEOUT,
                       "a bounded device wait ran out (no-alloc call)");
    return FIRE_OK;
}

int fire_debug_fail_alloc(fire_ctx *ctx, int after)
{
    if (!ctx || after < -1) return FIRE_EINVAL;
    ctx->fail_alloc_after = after;
    return FIRE_OK;
}

int fire_set_launch(fire_ctx *ctx, int warps_per_block, int blocks_per_sm,
                    int queue_entries, int state_mode)
{
    if (!ctx) return FIRE_EINVAL;
    if (warps_per_block < 0 || warps_per_block > kSimMaxThreads / 32 ||
        blocks_per_sm < 0 || queue_entries < 0 ||
        (queue_entries > 0 && queue_entries < 64) || state_mode < 0 ||
        state_mode > FIRE_STATE_GLOBAL)
        return set_err(ctx, FIRE_EINVAL, "bad launch shape %d x %d, queue %d, "
                       "state %d", warps_per_block, blocks_per_sm,
                       queue_entries, state_mode);
    ctx->warps_per_block = warps_per_block;
    ctx->blocks_per_sm = blocks_per_sm;
    ctx->queue_entries = queue_entries;
    ctx->state_mode = state_mode;
    return FIRE_OK;
}

int fire_maps_upload(fire_ctx *ctx, int H, int W, float cell_m,
                     const uint8_t *veg, const float *elev, const float *slope,
                     const float *aspect, const float *wind, uint32_t flags,
                     fire_map **out)
{
    FIRE_NVTX("fire_maps_upload");
    if (!ctx || !out) return FIRE_EINVAL;
    *out = nullptr;
    if (H <= 0 || W <= 0)
        return set_err(ctx, FIRE_EINVAL, "grid %d x %d is empty", H, W);
    if (!veg || !elev || !slope || !aspect || !wind)
        return set_err(ctx, FIRE_EINVAL, "NULL map pointer");
    const long long TH = (H + 31) / 32, TW = (W + 31) / 32;
    if (TH * TW > FIRE_MAX_TILES || (long long)H * W > 0x7fffffffll)
        return set_err(ctx, FIRE_EINVAL, "grid %d x %d exceeds %d tiles", H, W,
                       FIRE_MAX_TILES);
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t HW = (size_t)H * W;
    const bool dev = flags & FIRE_DEVICE_PTRS;

    fire_map *m = new (std::nothrow) fire_map();
    if (!m) return FIRE_ENOMEM;
    m->ctx = ctx;
    m->cell_m = cell_m;
    m->dev.H = H;
    m->dev.W = W;
    m->dev.TH = (int)TH;
    m->dev.TW = (int)TW;
    m->dev.ntiles = (int)(TH * TW);
    const size_t words = (size_t)m->dev.ntiles * 32;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&m->feat, HW * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc(&m->wdiag, HW * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&m->ps, HW * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc(&m->cfl, HW * sizeof(uint16_t))) != cudaSuccess ||
        (e = cudaMalloc(&m->blk, words * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->tgt, words * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->tgt_count, 16)) != cudaSuccess) {
        fire_map_free(m);
        return set_err(ctx, FIRE_ENOMEM, "map allocation: %s",
                       cudaGetErrorString(e));
    }
    m->dev.feat = m->feat;
    m->dev.wdiag = m->wdiag;
    m->dev.ps = m->ps;
    m->dev.cfl = m->cfl;
    m->dev.blk = m->blk;
    m->dev.tgt = m->tgt;
    m->dev.tgt_count = m->tgt_count;

    // stage the inputs on the device
    const uint8_t *dveg = veg;
    const float *delev = elev, *dslope = slope, *daspect = aspect, *dwind = wind;
    void *tmp = nullptr;
    if (!dev) {
        const size_t bytes = round16(HW) + 4 * round16(HW * 4);
        if ((e = cudaMalloc(&tmp, bytes)) != cudaSuccess) {
            fire_map_free(m);
            return set_err(ctx, FIRE_ENOMEM, "staging: %s", cudaGetErrorString(e));
        }
        char *p = (char *)tmp;
        uint8_t *v = (uint8_t *)p;
        p += round16(HW);
        float *f[4];
        for (int i = 0; i < 4; ++i) { f[i] = (float *)p; p += round16(HW * 4); }
        const float *src[4] = {elev, slope, aspect, wind};
        e = cudaMemcpyAsync(v, veg, HW, cudaMemcpyHostToDevice, ctx->stream);
        for (int i = 0; i < 4 && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(f[i], src[i], HW * 4, cudaMemcpyHostToDevice,
                                ctx->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            fire_map_free(m);
            return cuda_err(ctx, e, "map upload");
        }
        dveg = v;
        delev = f[0];
        dslope = f[1];
        daspect = f[2];
        dwind = f[3];
    }
    // the map's tgt_count word doubles as the wind-uniformity flag until the
    // target is cleared below
    e = launch_features(H, W, dveg, delev, dslope, daspect, dwind, m->feat,
                        m->wdiag, m->ps, m->cfl, m->tgt_count, ctx->stream);
    uint32_t wind_varies = 1;
    float4 f0;
    float2 w0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&wind_varies, m->tgt_count, 4, cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&f0, m->feat, sizeof f0, cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&w0, m->wdiag, sizeof w0, cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && !wind_varies) {
        m->dev.uniform_wind = 1;
        m->dev.cw = f0.z;
        m->dev.sw = f0.w;
        m->dev.om1 = w0.x;
        m->dev.om3 = w0.y;
    }
    if (e == cudaSuccess) e = launch_blocked(m->dev, dveg, m->blk, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->tgt, 0, words * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->tgt_count, 0, 16, ctx->stream);
    // host copy of the burnable mask for validating host ignitions
    m->burnable_host.resize(HW);
    if (e == cudaSuccess) {
        if (dev) {
            e = cudaMemcpyAsync(m->burnable_host.data(), veg, HW,
                                cudaMemcpyDeviceToHost, ctx->stream);
        } else {
            std::memcpy(m->burnable_host.data(), veg, HW);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        fire_map_free(m);
        return cuda_err(ctx, e, "feature precompute");
    }
    *out = m;
    return FIRE_OK;
}

void fire_map_free(fire_map *m)
{
    if (!m) return;
    if (m->ctx) cudaSetDevice(m->ctx->device);
    if (m->feat) cudaFree(m->feat);
    if (m->wdiag) cudaFree(m->wdiag);
    if (m->ps) cudaFree(m->ps);
    if (m->cfl) cudaFree(m->cfl);
    if (m->blk) cudaFree(m->blk);
    if (m->tgt) cudaFree(m->tgt);
    if (m->tgt_count) cudaFree(m->tgt_count);
    delete m;
}

int fire_map_shape(const fire_map *m, int *H, int *W)
{
    if (!valid_map(m)) return FIRE_EINVAL;
    if (H) *H = m->dev.H;
    if (W) *W = m->dev.W;
    return FIRE_OK;
}

int fire_target_upload(fire_ctx *ctx, fire_map *m, const uint8_t *burnt,
                       uint32_t flags)
{
    FIRE_NVTX("fire_target_upload");
    if (!ctx || !valid_map(m) || !burnt) return set_err(ctx, FIRE_EINVAL,
                                                         "bad target arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t HW = (size_t)m->dev.H * m->dev.W;
    const uint8_t *src = burnt;
    void *tmp = nullptr;
    cudaError_t e;
    if (!(flags & FIRE_DEVICE_PTRS)) {
        if ((e = cudaMalloc(&tmp, HW)) != cudaSuccess)
            return set_err(ctx, FIRE_ENOMEM, "target staging");
        e = cudaMemcpyAsync(tmp, burnt, HW, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) { cudaFree(tmp); return cuda_err(ctx, e, "target copy"); }
        src = (const uint8_t *)tmp;
    }
    e = launch_target(m->dev, src, m->tgt, m->tgt_count, ctx->stream);
    if (e == cudaSuccess && (tmp || (flags & FIRE_SYNC)))
        e = cudaStreamSynchronize(ctx->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_err(ctx, e, "target pack");
    return FIRE_OK;
}

}  // extern "C"

namespace fire {

// Launch the simulation kernel over n simulations of one map whose arguments
// already sit on the device (the common tail of fire_simulate_batch, also
// used by the surrogate's label builder for the burnt-word output).
int launch_batch(fire_ctx *ctx, const fire_map *m, int n,
                 const fire_params *dparams, const fire_cell *dign,
                 const uint64_t *dseeds, uint32_t max_steps, uint32_t flags,
                 fire_result *dout, int32_t *dsteps, uint32_t *dbits)
{
    const int ntiles = m->dev.ntiles;
    LaunchPlan plan;
    int rc = plan_launch(ctx, ntiles, n, &plan);
    if (rc) return rc;
    const bool smem_state = plan.smem_state;
    const long long grid = plan.grid;
    if (!smem_state) {
        const size_t need = (size_t)grid * 2 * ntiles * 128;
        rc = grow_device(ctx, (void **)&ctx->gstate, &ctx->gstate_bytes, need,
                         "simulation state");
        if (rc) return rc;
    }
    // longest-first processing order (scheduling only: every fire's result
    // depends on its own parameters, ignition and seed alone)
    const uint32_t *dorder = nullptr;
    if ((flags & FIRE_LONGEST_FIRST) && n > grid && n <= kLongestFirstMax) {
        rc = grow_device(ctx, &ctx->lpt, &ctx->lpt_bytes, (size_t)n * 8,
                         "longest-first order");
        if (rc) return rc;
        float *key = (float *)ctx->lpt;
        uint32_t *ord = (uint32_t *)((char *)ctx->lpt + (size_t)n * 4);
        cudaError_t e = launch_longest_first(m->dev, n, dparams, key, ord, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "longest-first order");
        dorder = ord;
    }
    SimLaunch a;
    a.map = m->dev;
    a.maps = nullptr;
    a.nmaps = 1;
    a.map_of_sim = nullptr;
    a.order = dorder;
    a.ntiles_max = ntiles;
    a.n = n;
    a.params = dparams;
    a.ign = dign;
    a.seeds = dseeds;
    a.out = dout;
    a.burn_step = dsteps;
    a.burnt_bits = dbits;
    a.work_counter = ctx->counter;
    a.gstate = ctx->gstate;
    a.block_words = 0;
    a.burn_time = nullptr;
    a.long_burn = nullptr;
    a.error_word = ctx->counter + 1;
    a.max_steps = max_steps;
    a.qcap = plan.qcap;
    a.cell_uniform = (flags & FIRE_CELL_UNIFORM) ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(ctx->counter, 0, 4, ctx->stream);
    if (e == cudaSuccess)
        e = launch_simulate(a, smem_state, plan.nwarps, (int)grid, plan.L.total,
                            ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "simulate launch");
    return FIRE_OK;
}

}  // namespace fire

extern "C" {

int fire_simulate_batch(fire_ctx *ctx, const fire_map *m, int n,
                        const fire_params *params, const fire_cell *ignitions,
                        const uint64_t *seeds, uint32_t max_steps,
                        uint32_t flags, fire_result *out, int32_t *burn_step)
{
    FIRE_NVTX("fire_simulate_batch");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(m)) return set_err(ctx, FIRE_EINVAL, "invalid map");
    if (m->ctx->device != ctx->device)
        return set_err(ctx, FIRE_EINVAL, "the map was uploaded on device %d, the "
                       "context runs on device %d", m->ctx->device, ctx->device);
    if (n < 0) return set_err(ctx, FIRE_EINVAL, "n = %d", n);
    if (n == 0) return FIRE_OK;
    if (!params || !ignitions || !seeds || !out)
        return set_err(ctx, FIRE_EINVAL, "NULL argument");
    const bool want_steps = (flags & FIRE_WANT_STEPS) != 0;
    if (want_steps && !burn_step)
        return set_err(ctx, FIRE_EINVAL, "FIRE_WANT_STEPS without burn_step");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const bool dev = flags & FIRE_DEVICE_PTRS;
    const int H = m->dev.H, W = m->dev.W;
    if (!dev) {
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < 5; ++j)
                if (!std::isfinite(params[i].b[j]))
                    return set_err(ctx, FIRE_EINVAL,
                                   "params[%d].b[%d] is not finite", i, j);
            const fire_cell g = ignitions[i];
            if (g.row < 0 || g.row >= H || g.col < 0 || g.col >= W ||
                !m->burnable_host[(size_t)g.row * W + g.col])
                return set_err(ctx, FIRE_EIGNITION,
                               "ignition %d (%d, %d) is outside the grid or "
                               "non-burnable", i, g.row, g.col);
        }
    }

    // staging of host arguments
    const fire_params *dparams = params;
    const fire_cell *dign = ignitions;
    const uint64_t *dseeds = seeds;
    fire_result *dout = out;
    if (!dev) {
        const size_t bp = round16((size_t)n * sizeof(fire_params));
        const size_t bi = round16((size_t)n * sizeof(fire_cell));
        const size_t bs = round16((size_t)n * sizeof(uint64_t));
        const size_t bo = round16((size_t)n * sizeof(fire_result));
        rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes,
                         bp + bi + bs + bo, "argument staging");
        if (rc) return rc;
        char *p = (char *)ctx->staging;
        fire_params *sp = (fire_params *)p;
        fire_cell *si = (fire_cell *)(p + bp);
        uint64_t *ss = (uint64_t *)(p + bp + bi);
        dout = (fire_result *)(p + bp + bi + bs);
        CUDA_TRY(ctx, cudaMemcpyAsync(sp, params, (size_t)n * sizeof(fire_params),
                                      cudaMemcpyHostToDevice, ctx->stream), "params H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync(si, ignitions, (size_t)n * sizeof(fire_cell),
                                      cudaMemcpyHostToDevice, ctx->stream), "ignitions H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync(ss, seeds, (size_t)n * sizeof(uint64_t),
                                      cudaMemcpyHostToDevice, ctx->stream), "seeds H2D");
        dparams = sp;
        dign = si;
        dseeds = ss;
    }
    int32_t *dsteps = nullptr;
    void *steps_tmp = nullptr;
    if (want_steps) {
        if (dev) {
            dsteps = burn_step;
        } else {
            const size_t bytes = (size_t)n * H * W * sizeof(int32_t);
            cudaError_t e = cudaMalloc(&steps_tmp, bytes);
            if (e != cudaSuccess)
                return set_err(ctx, FIRE_ENOMEM, "burn-step buffer (%zu B)", bytes);
            dsteps = (int32_t *)steps_tmp;
        }
    }
    rc = launch_batch(ctx, m, n, dparams, dign, dseeds, max_steps, flags, dout,
                      dsteps, nullptr);
    if (rc) {
        if (steps_tmp) cudaFree(steps_tmp);
        return rc;
    }
    if (!dev) {
        cudaError_t e = cudaMemcpyAsync(out, dout, (size_t)n * sizeof(fire_result),
                                        cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && want_steps)
            e = cudaMemcpyAsync(burn_step, dsteps,
                                (size_t)n * H * W * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (steps_tmp) cudaFree(steps_tmp);
        if (e != cudaSuccess) return cuda_err(ctx, e, "results D2H");
        return fire_sync(ctx);
    }
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_fitness(fire_ctx *ctx, const fire_result *results, int n, int kind,
                 uint32_t flags, double *out)
{
    FIRE_NVTX("fire_fitness");
    if (!ctx) return FIRE_EINVAL;
    if (n < 0 || (kind != 0 && kind != 1))
        return set_err(ctx, FIRE_EINVAL, "bad fitness arguments");
    if (n == 0) return FIRE_OK;
    if (!results || !out) return set_err(ctx, FIRE_EINVAL, "NULL argument");
    if (flags & FIRE_DEVICE_PTRS) {
        // out[i] would land inside results[i / 3], read by another thread
        const char *a = (const char *)results, *b = (const char *)out;
        if (a < b + (size_t)n * 8 && b < a + (size_t)n * sizeof(fire_result))
            return set_err(ctx, FIRE_EINVAL, "device out overlaps results");
    }
    int rc = ensure_device(ctx);
    if (rc) return rc;
    if (flags & FIRE_DEVICE_PTRS) {
        CUDA_TRY(ctx, launch_fitness(results, n, kind, out, ctx->stream), "fitness");
        if (flags & FIRE_SYNC) return fire_sync(ctx);
        return FIRE_OK;
    }
    const size_t br = round16((size_t)n * sizeof(fire_result));
    const size_t bo = round16((size_t)n * sizeof(double));
    rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes, br + bo, "fitness staging");
    if (rc) return rc;
    fire_result *dr = (fire_result *)ctx->staging;
    double *dout = (double *)((char *)ctx->staging + br);
    CUDA_TRY(ctx, cudaMemcpyAsync(dr, results, (size_t)n * sizeof(fire_result),
                                  cudaMemcpyHostToDevice, ctx->stream), "results H2D");
    CUDA_TRY(ctx, launch_fitness(dr, n, kind, dout, ctx->stream), "fitness");
    CUDA_TRY(ctx, cudaMemcpyAsync(out, dout, (size_t)n * sizeof(double),
                                  cudaMemcpyDeviceToHost, ctx->stream), "fitness D2H");
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "fitness sync");
    return FIRE_OK;
}

namespace {

// Runs `body(dev_beta, dev_outs...)` with host or device output buffers.
int with_beta(fire_ctx *ctx, const fire_params *params, uint32_t flags,
              double **dbeta)
{
    const size_t need = 64;
    int rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes, need, "beta");
    if (rc) return rc;
    *dbeta = (double *)ctx->staging;
    CUDA_TRY(ctx, cudaMemcpyAsync(*dbeta, params->b, 5 * sizeof(double),
                                  (flags & FIRE_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice
                                                             : cudaMemcpyHostToDevice,
                                  ctx->stream), "beta copy");
    return FIRE_OK;
}

}  // namespace

int fire_thresholds(fire_ctx *ctx, const fire_map *m, const fire_params *params,
                    uint32_t flags, int64_t *out)
{
    FIRE_NVTX("fire_thresholds");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(m) || !params || !out)
        return set_err(ctx, FIRE_EINVAL, "bad thresholds arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t cnt = 8 * (size_t)m->dev.H * m->dev.W;
    double *dbeta = nullptr;
    int64_t *dout = out;
    void *tmp = nullptr;
    if (!(flags & FIRE_DEVICE_PTRS)) {
        CUDA_TRY(ctx, cudaMalloc(&tmp, cnt * 8), "threshold buffer");
        dout = (int64_t *)tmp;
    }
    rc = with_beta(ctx, params, flags, &dbeta);
    if (!rc) {
        cudaError_t e = launch_thresholds(m->dev, dbeta, dout, ctx->stream);
        if (e == cudaSuccess && tmp)
            e = cudaMemcpyAsync(out, dout, cnt * 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "thresholds");
    }
    if (tmp) cudaFree(tmp);
    return rc;
}

int fire_probabilities(fire_ctx *ctx, const fire_map *m, const fire_params *params,
                       uint32_t flags, float *p32, double *p64)
{
    FIRE_NVTX("fire_probabilities");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(m) || !params || (!p32 && !p64))
        return set_err(ctx, FIRE_EINVAL, "bad probabilities arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t cnt = 8 * (size_t)m->dev.H * m->dev.W;
    float *d32 = p32;
    double *d64 = p64;
    void *tmp = nullptr;
    if (!(flags & FIRE_DEVICE_PTRS)) {
        CUDA_TRY(ctx, cudaMalloc(&tmp, cnt * 12 + 64), "probability buffer");
        d64 = p64 ? (double *)tmp : nullptr;
        d32 = p32 ? (float *)((char *)tmp + cnt * 8) : nullptr;
    }
    double *dbeta = nullptr;
    rc = with_beta(ctx, params, flags, &dbeta);
    if (!rc) {
        cudaError_t e = launch_probabilities(m->dev, dbeta, d32, d64, ctx->stream);
        if (e == cudaSuccess && tmp && p32)
            e = cudaMemcpyAsync(p32, d32, cnt * 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && tmp && p64)
            e = cudaMemcpyAsync(p64, d64, cnt * 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = cuda_err(ctx, e, "probabilities");
    }
    if (tmp) cudaFree(tmp);
    return rc;
}

int fire_map_features(fire_ctx *ctx, const fire_map *m, uint32_t flags,
                      float *psi, float *sig, float *cos_wind, float *sin_wind,
                      uint16_t *cell_flags)
{
    FIRE_NVTX("fire_map_features");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(m)) return set_err(ctx, FIRE_EINVAL, "invalid map");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t HW = (size_t)m->dev.H * m->dev.W;
    if (flags & FIRE_DEVICE_PTRS) {
        CUDA_TRY(ctx, launch_features_export(m->dev, psi, sig, cos_wind, sin_wind,
                                             cell_flags, ctx->stream), "features");
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "features sync");
        return FIRE_OK;
    }
    void *tmp = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&tmp, HW * 18 + 64), "feature buffer");
    float *f = (float *)tmp;
    uint16_t *c = (uint16_t *)((char *)tmp + HW * 16);
    cudaError_t e = launch_features_export(m->dev, f, f + HW, f + 2 * HW, f + 3 * HW,
                                           c, ctx->stream);
    float *dst[4] = {psi, sig, cos_wind, sin_wind};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
        if (dst[i])
            e = cudaMemcpyAsync(dst[i], f + i * HW, HW * 4, cudaMemcpyDeviceToHost,
                                ctx->stream);
    if (e == cudaSuccess && cell_flags)
        e = cudaMemcpyAsync(cell_flags, c, HW * 2, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_err(ctx, e, "features export");
    return FIRE_OK;
}

int fire_screen_selftest(fire_ctx *ctx, uint64_t n, uint64_t seed,
                         uint64_t counts[3], double max_err_ratio[1])
{
    FIRE_NVTX("fire_screen_selftest");
    if (!ctx) return FIRE_EINVAL;
    if (!counts || !max_err_ratio) return set_err(ctx, FIRE_EINVAL, "NULL output");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    unsigned long long *d = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&d, 64), "selftest buffer");
    cudaError_t e = cudaMemsetAsync(d, 0, 64, ctx->stream);
    if (e == cudaSuccess) e = launch_screen_selftest(n, seed, d, d + 3, ctx->stream);
    unsigned long long h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d, 32, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_err(ctx, e, "screen selftest");
    for (int i = 0; i < 3; ++i) counts[i] = h[i];
    double v;
    std::memcpy(&v, &h[3], 8);
    max_err_ratio[0] = v;
    return FIRE_OK;
}

int fire_philox_blocks(fire_ctx *ctx, uint64_t n, const uint32_t ctr[4],
                       const uint32_t key[2], uint32_t flags, uint32_t *out)
{
    FIRE_NVTX("fire_philox_blocks");
    if (!ctx) return FIRE_EINVAL;
    if (!ctr || !key || !out) return set_err(ctx, FIRE_EINVAL, "NULL argument");
    if (n == 0) return FIRE_OK;
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const uint4 c = make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]);
    const uint2 k = make_uint2(key[0], key[1]);
    if (flags & FIRE_DEVICE_PTRS) {
        CUDA_TRY(ctx, launch_philox_blocks(n, c, k, out, ctx->stream), "philox");
        if (flags & FIRE_SYNC) return fire_sync(ctx);
        return FIRE_OK;
    }
    void *tmp = nullptr;
    CUDA_TRY(ctx, cudaMalloc(&tmp, n * 16), "philox buffer");
    cudaError_t e = launch_philox_blocks(n, c, k, (uint32_t *)tmp, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, tmp, n * 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_err(ctx, e, "philox");
    return FIRE_OK;
}

}  // extern "C"

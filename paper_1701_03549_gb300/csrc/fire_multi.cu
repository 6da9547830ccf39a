// Uneven multi-map batches in one persistent launch, CUDA-graph replay of
// repeated calls, and the launch-shape autotuner (C ABI, include/fire.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "fire_internal.h"

using namespace fire;

namespace {

// Replays a captured graph for an identical call, or captures the work that
// `issue` enqueues on the context's stream, instantiates and launches it.
template <class Issue>
int run_graph(fire_ctx *ctx, const std::vector<unsigned long long> &key,
              Issue &&issue)
{
    if (ctx->stream == nullptr || ctx->stream == cudaStreamLegacy ||
        ctx->stream == cudaStreamPerThread)
        return set_err(ctx, FIRE_EINVAL,
                       "FIRE_GRAPH needs a context on a non-default stream");
    // drop graphs that may reference moved buffers
    for (size_t i = 0; i < ctx->graphs.size();) {
        if (ctx->graphs[i].epoch != ctx->epoch) {
            cudaGraphExecDestroy(ctx->graphs[i].exec);
            ctx->graphs.erase(ctx->graphs.begin() + i);
        } else {
            ++i;
        }
    }
    for (GraphEntry &g : ctx->graphs) {
        if (g.key == key) {
            CUDA_TRY(ctx, cudaGraphLaunch(g.exec, ctx->stream), "cudaGraphLaunch");
            return FIRE_OK;
        }
    }
    CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->stream,
                                         cudaStreamCaptureModeThreadLocal),
             "cudaStreamBeginCapture");
    const int rc = issue();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_err(ctx, ei, "cudaGraphInstantiate");
    ctx->graphs.push_back(GraphEntry{key, exec, ctx->epoch});
    CUDA_TRY(ctx, cudaGraphLaunch(exec, ctx->stream), "cudaGraphLaunch");
    return FIRE_OK;
}

}  // namespace

extern "C" {

int fire_simulate_multi(fire_ctx *ctx, int nmaps, const fire_map *const *maps,
                        const int32_t *map_of_sim, int n,
                        const fire_params *params, const fire_cell *ignitions,
                        const uint64_t *seeds, uint32_t max_steps,
                        uint32_t flags, fire_result *out)
{
    FIRE_NVTX("fire_simulate_multi");
    if (!ctx) return FIRE_EINVAL;
    if (nmaps <= 0 || !maps) return set_err(ctx, FIRE_EINVAL, "no maps");
    if (n < 0) return set_err(ctx, FIRE_EINVAL, "n = %d", n);
    if (n == 0) return FIRE_OK;
    if (!map_of_sim || !params || !ignitions || !seeds || !out)
        return set_err(ctx, FIRE_EINVAL, "NULL argument");
    if (flags & FIRE_WANT_STEPS)
        return set_err(ctx, FIRE_EINVAL,
                       "burn-step maps are not produced by fire_simulate_multi");
    const bool dev = flags & FIRE_DEVICE_PTRS;
    const bool graph = flags & FIRE_GRAPH;
    if (graph && !dev)
        return set_err(ctx, FIRE_EINVAL, "FIRE_GRAPH needs FIRE_DEVICE_PTRS");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    int ntiles_max = 0;
    for (int j = 0; j < nmaps; ++j) {
        if (!valid_map(maps[j]) || maps[j]->ctx->device != ctx->device)
            return set_err(ctx, FIRE_EINVAL, "map %d is invalid", j);
        ntiles_max = std::max(ntiles_max, maps[j]->dev.ntiles);
    }
    if (!dev) {
        for (int i = 0; i < n; ++i) {
            const int mi = map_of_sim[i];
            if (mi < 0 || mi >= nmaps)
                return set_err(ctx, FIRE_EINVAL, "map_of_sim[%d] = %d", i, mi);
            for (int j = 0; j < 5; ++j)
                if (!std::isfinite(params[i].b[j]))
                    return set_err(ctx, FIRE_EINVAL,
                                   "params[%d].b[%d] is not finite", i, j);
            const fire_map *m = maps[mi];
            const fire_cell g = ignitions[i];
            if (g.row < 0 || g.row >= m->dev.H || g.col < 0 || g.col >= m->dev.W ||
                !m->burnable_host[(size_t)g.row * m->dev.W + g.col])
                return set_err(ctx, FIRE_EIGNITION,
                               "ignition %d (%d, %d) is outside map %d or "
                               "non-burnable", i, g.row, g.col, mi);
        }
    }
    LaunchPlan plan;
    rc = plan_launch(ctx, ntiles_max, n, &plan);
    if (rc) return rc;

    // map table and ranks (largest map first) on the device
    std::vector<MapDev> table(nmaps);
    std::vector<int32_t> order_of(nmaps), rank(nmaps);
    for (int j = 0; j < nmaps; ++j) table[j] = maps[j]->dev;
    std::iota(order_of.begin(), order_of.end(), 0);
    std::stable_sort(order_of.begin(), order_of.end(), [&](int a, int b) {
        return table[a].ntiles > table[b].ntiles;
    });
    for (int j = 0; j < nmaps; ++j) rank[order_of[j]] = j;
    const size_t tb = round16(nmaps * sizeof(MapDev));
    rc = grow_device(ctx, &ctx->table, &ctx->table_bytes, tb + nmaps * 4, "map table");
    if (rc) return rc;
    const size_t ob = round16((nmaps + 1) * 4);
    rc = grow_device(ctx, &ctx->order, &ctx->order_bytes, ob + (size_t)n * 4,
                     "processing order");
    if (rc) return rc;
    if (!plan.smem_state) {
        rc = grow_device(ctx, (void **)&ctx->gstate, &ctx->gstate_bytes,
                         (size_t)plan.grid * 2 * ntiles_max * 128,
                         "simulation state");
        if (rc) return rc;
    }
    // host-pointer arguments are staged (never under graph capture)
    const fire_params *dparams = params;
    const fire_cell *dign = ignitions;
    const uint64_t *dseeds = seeds;
    const int32_t *dmap = map_of_sim;
    fire_result *dout = out;
    if (!dev) {
        const size_t bp = round16((size_t)n * sizeof(fire_params));
        const size_t bi = round16((size_t)n * sizeof(fire_cell));
        const size_t bs = round16((size_t)n * sizeof(uint64_t));
        const size_t bm = round16((size_t)n * sizeof(int32_t));
        const size_t bo = round16((size_t)n * sizeof(fire_result));
        rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes,
                         bp + bi + bs + bm + bo, "argument staging");
        if (rc) return rc;
        char *p = (char *)ctx->staging;
        dparams = (const fire_params *)p;
        dign = (const fire_cell *)(p + bp);
        dseeds = (const uint64_t *)(p + bp + bi);
        dmap = (const int32_t *)(p + bp + bi + bs);
        dout = (fire_result *)(p + bp + bi + bs + bm);
        CUDA_TRY(ctx, cudaMemcpyAsync((void *)dparams, params, (size_t)n * sizeof(fire_params),
                                      cudaMemcpyHostToDevice, ctx->stream), "params H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync((void *)dign, ignitions, (size_t)n * sizeof(fire_cell),
                                      cudaMemcpyHostToDevice, ctx->stream), "ignitions H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync((void *)dseeds, seeds, (size_t)n * sizeof(uint64_t),
                                      cudaMemcpyHostToDevice, ctx->stream), "seeds H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync((void *)dmap, map_of_sim, (size_t)n * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, ctx->stream), "map index H2D");
    }
    MapDev *dtable = (MapDev *)ctx->table;
    int32_t *drank = (int32_t *)((char *)ctx->table + tb);
    uint32_t *dcounts = (uint32_t *)ctx->order;
    uint32_t *dorder = (uint32_t *)((char *)ctx->order + ob);
    // the table is uploaded before (never inside) a capture: graphs keep
    // pointing at this buffer, whose contents only change with the map set
    CUDA_TRY(ctx, cudaMemcpyAsync(dtable, table.data(), nmaps * sizeof(MapDev),
                                  cudaMemcpyHostToDevice, ctx->stream), "map table H2D");
    CUDA_TRY(ctx, cudaMemcpyAsync(drank, rank.data(), nmaps * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, ctx->stream), "ranks H2D");

    SimLaunch a;
    std::memset(&a, 0, sizeof a);
    a.map = table[0];
    a.maps = dtable;
    a.nmaps = nmaps;
    a.map_of_sim = dmap;
    a.order = dorder;
    a.ntiles_max = ntiles_max;
    a.n = n;
    a.params = dparams;
    a.ign = dign;
    a.seeds = dseeds;
    a.out = dout;
    a.burn_step = nullptr;
    a.burnt_bits = nullptr;
    a.work_counter = ctx->counter;
    a.gstate = ctx->gstate;
    a.error_word = ctx->counter + 1;
    a.max_steps = max_steps;
    a.qcap = plan.qcap;
    a.cell_uniform = (flags & FIRE_CELL_UNIFORM) ? 1 : 0;

    auto issue = [&]() -> int {
        CUDA_TRY(ctx, launch_order(n, dmap, nmaps, drank, dcounts, dorder, ctx->stream),
                 "order kernels");
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->counter, 0, 4, ctx->stream), "counter reset");
        CUDA_TRY(ctx, launch_simulate(a, plan.smem_state, plan.nwarps, plan.grid,
                                      plan.L.total, ctx->stream),
                 "simulate launch");
        return FIRE_OK;
    };
    if (graph) {
        std::vector<unsigned long long> key = {
            (unsigned long long)n, (unsigned long long)nmaps,
            (unsigned long long)(uintptr_t)dparams, (unsigned long long)(uintptr_t)dign,
            (unsigned long long)(uintptr_t)dseeds, (unsigned long long)(uintptr_t)dmap,
            (unsigned long long)(uintptr_t)dout, max_steps,
            (unsigned long long)plan.nwarps, (unsigned long long)plan.qcap,
            (unsigned long long)plan.smem_state, (unsigned long long)plan.grid,
            (unsigned long long)a.cell_uniform};
        // a map's memory may be reused by a later map of another shape, and
        // the launch bakes in the largest map's tile count
        for (int j = 0; j < nmaps; ++j) {
            key.push_back((unsigned long long)(uintptr_t)maps[j]->feat);
            key.push_back(((unsigned long long)(uint32_t)maps[j]->dev.H << 32) |
                          (uint32_t)maps[j]->dev.W);
        }
        rc = run_graph(ctx, key, issue);
    } else {
        rc = issue();
    }
    if (rc) return rc;
    if (!dev) {
        CUDA_TRY(ctx, cudaMemcpyAsync(out, dout, (size_t)n * sizeof(fire_result),
                                      cudaMemcpyDeviceToHost, ctx->stream), "results D2H");
        return fire_sync(ctx);
    }
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_autotune(fire_ctx *ctx, int nmaps, const fire_map *const *maps,
                  const int32_t *map_of_sim, int n, const fire_params *params,
                  const fire_cell *ignitions, const uint64_t *seeds,
                  uint32_t flags, fire_launch *best)
{
    FIRE_NVTX("fire_autotune");
    if (!ctx) return FIRE_EINVAL;
    if (!best || n <= 0 || nmaps <= 0 || !maps)
        return set_err(ctx, FIRE_EINVAL, "bad autotune arguments");
    const bool lpt = (flags & FIRE_LONGEST_FIRST) != 0;
    if (lpt && nmaps != 1)
        return set_err(ctx, FIRE_EINVAL, "FIRE_LONGEST_FIRST autotuning takes one map");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    int ntiles_max = 0;
    for (int j = 0; j < nmaps; ++j) {
        if (!valid_map(maps[j])) return set_err(ctx, FIRE_EINVAL, "map %d is invalid", j);
        ntiles_max = std::max(ntiles_max, maps[j]->dev.ntiles);
    }
    // candidate shapes: warps per block, blocks per SM, queue entries, state
    static const int kCand[][4] = {
        {16, 0, 4096, FIRE_STATE_SHARED}, {10, 3, 2048, FIRE_STATE_SHARED},
        {8, 2, 4096, FIRE_STATE_SHARED},  {4, 6, 2048, FIRE_STATE_SHARED},
        {16, 2, 8192, FIRE_STATE_GLOBAL}, {8, 4, 6144, FIRE_STATE_GLOBAL},
        {8, 4, 4096, FIRE_STATE_GLOBAL},  {8, 4, 3072, FIRE_STATE_GLOBAL},
        {6, 5, 3072, FIRE_STATE_GLOBAL},
        {4, 8, 3072, FIRE_STATE_GLOBAL},  {4, 8, 2048, FIRE_STATE_GLOBAL},
        {2, 16, 1024, FIRE_STATE_GLOBAL},
    };
    const int saved[4] = {ctx->warps_per_block, ctx->blocks_per_sm,
                          ctx->queue_entries, ctx->state_mode};
    // results of the trial runs go to a scratch buffer on the device
    const bool dev = flags & FIRE_DEVICE_PTRS;
    std::vector<fire_result> host_out;
    fire_result *out = nullptr;
    void *scratch = nullptr;
    if (dev) {
        CUDA_TRY(ctx, cudaMalloc(&scratch, (size_t)n * sizeof(fire_result)),
                 "autotune output");
        out = (fire_result *)scratch;
    } else {
        host_out.resize(n);
        out = host_out.data();
    }
    std::vector<int32_t> zeros;
    const int32_t *mos = map_of_sim;
    if (!mos && !lpt) {   // the longest-first runs take the one map directly
        if (dev) {
            cudaFree(scratch);
            return set_err(ctx, FIRE_EINVAL, "map_of_sim is required with device pointers");
        }
        zeros.assign(n, 0);
        mos = zeros.data();
    }
    const uint32_t run_flags = (dev ? FIRE_DEVICE_PTRS : 0u);
    // one run of the batch in the order the caller's calls will use: a
    // single map in longest-first order through fire_simulate_batch, else
    // fire_simulate_multi (largest map first)
    auto run = [&]() {
        if (lpt)
            return fire_simulate_batch(ctx, maps[0], n, params, ignitions, seeds,
                                       0, run_flags | FIRE_LONGEST_FIRST, out,
                                       nullptr);
        return fire_simulate_multi(ctx, nmaps, maps, mos, n, params, ignitions,
                                   seeds, 0, run_flags, out);
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = INFINITY;
    int best_i = -1;
    for (int c = 0; c < (int)(sizeof kCand / sizeof kCand[0]); ++c) {
        ctx->warps_per_block = kCand[c][0];
        ctx->blocks_per_sm = kCand[c][1];
        ctx->queue_entries = kCand[c][2];
        ctx->state_mode = kCand[c][3];
        rc = run();
        if (rc == FIRE_OK) rc = fire_sync(ctx);
        if (rc != FIRE_OK) continue;   // shape does not fit this device / map
        // the better of two timed runs, so that one slow run does not decide
        float ms = INFINITY;
        for (int rep = 0; rep < 2 && rc == FIRE_OK; ++rep) {
            cudaEventRecord(e0, ctx->stream);
            rc = run();
            cudaEventRecord(e1, ctx->stream);
            if (rc == FIRE_OK) rc = fire_sync(ctx);
            float r_ms = 0.f;
            if (rc == FIRE_OK && cudaEventElapsedTime(&r_ms, e0, e1) == cudaSuccess)
                ms = fminf(ms, r_ms);
        }
        if (rc != FIRE_OK) continue;
        if (ms < best_ms) {
            best_ms = ms;
            best_i = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (scratch) cudaFree(scratch);
    ctx->warps_per_block = saved[0];
    ctx->blocks_per_sm = saved[1];
    ctx->queue_entries = saved[2];
    ctx->state_mode = saved[3];
    if (best_i < 0) return set_err(ctx, FIRE_EINVAL, "no candidate launch shape ran");
    ctx->err.clear();
    best->warps_per_block = kCand[best_i][0];
    best->blocks_per_sm = kCand[best_i][1];
    best->queue_entries = kCand[best_i][2];
    best->state_mode = kCand[best_i][3];
    best->ms = best_ms;
    TuneEntry t{ntiles_max, kCand[best_i][0], kCand[best_i][1], kCand[best_i][2],
                kCand[best_i][3], best_ms};
    bool replaced = false;
    for (TuneEntry &u : ctx->tuned) {
        if (u.ntiles == ntiles_max) {
            u = t;
            replaced = true;
        }
    }
    if (!replaced) ctx->tuned.push_back(t);
    return FIRE_OK;
}

}  // extern "C"

// C ABI of the burn-out-time variant (fire_simulate_burnout, include/fire.h):
// argument checks, staging of host arguments and the launch of the bit-plane
// simulation kernel in its burn-time form.
#include <cmath>
#include <cstring>

#include "fire_internal.h"

using namespace fire;

extern "C" int fire_simulate_burnout(fire_ctx *ctx, const fire_map *m, int n,
                                     const fire_params *params,
                                     const fire_cell *ignitions,
                                     const uint64_t *seeds,
                                     const uint8_t *burn_time, uint32_t max_steps,
                                     uint32_t flags, fire_result *out,
                                     int32_t *burn_step)
{
    FIRE_NVTX("fire_simulate_burnout");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(m)) return set_err(ctx, FIRE_EINVAL, "invalid map");
    if (n < 0) return set_err(ctx, FIRE_EINVAL, "n = %d", n);
    if (n == 0) return FIRE_OK;
    if (!params || !ignitions || !seeds || !out || !burn_time)
        return set_err(ctx, FIRE_EINVAL, "NULL argument");
    const bool want_steps = (flags & FIRE_WANT_STEPS) != 0;
    if (want_steps && !burn_step)
        return set_err(ctx, FIRE_EINVAL, "FIRE_WANT_STEPS without burn_step");
    if (flags & (FIRE_CELL_UNIFORM | FIRE_GRAPH))
        return set_err(ctx, FIRE_EINVAL,
                       "burn times take the per-neighbour rule, without graphs");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const bool dev = flags & FIRE_DEVICE_PTRS;
    const int H = m->dev.H, W = m->dev.W;
    const size_t HW = (size_t)H * W;
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
        for (size_t i = 0; i < HW; ++i)
            if (m->burnable_host[i] && (burn_time[i] < 1 || burn_time[i] > 250))
                return set_err(ctx, FIRE_EINVAL,
                               "burn_time[%zu] = %d outside 1..250", i,
                               (int)burn_time[i]);
    }
    // host arguments go through one temporary device buffer
    void *tmp = nullptr;
    const fire_params *dp = params;
    const fire_cell *di = ignitions;
    const uint64_t *ds = seeds;
    const uint8_t *db = burn_time;
    fire_result *dout = out;
    int32_t *dsteps = want_steps ? burn_step : nullptr;
    if (!dev) {
        const size_t bp = round16((size_t)n * sizeof(fire_params));
        const size_t bi = round16((size_t)n * sizeof(fire_cell));
        const size_t bs = round16((size_t)n * 8);
        const size_t bb = round16(HW);
        const size_t bo = round16((size_t)n * sizeof(fire_result));
        const size_t bst = want_steps ? (size_t)n * HW * 4 : 0;
        cudaError_t e = cudaMalloc(&tmp, bp + bi + bs + bb + bo + bst);
        if (e != cudaSuccess)
            return set_err(ctx, FIRE_ENOMEM, "burn-out staging");
        char *p = (char *)tmp;
        cudaStream_t st = ctx->stream;
        e = cudaMemcpyAsync(p, params, (size_t)n * sizeof(fire_params),
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p + bp, ignitions, (size_t)n * sizeof(fire_cell),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p + bp + bi, seeds, (size_t)n * 8,
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p + bp + bi + bs, burn_time, HW,
                                cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_err(ctx, e, "burn-out staging copy");
        }
        dp = (const fire_params *)p;
        di = (const fire_cell *)(p + bp);
        ds = (const uint64_t *)(p + bp + bi);
        db = (const uint8_t *)(p + bp + bi + bs);
        dout = (fire_result *)(p + bp + bi + bs + bb);
        if (want_steps) dsteps = (int32_t *)(p + bp + bi + bs + bb + bo);
    }
    // cells that burn two steps or more: with none, the batch is the plain
    // rule of fire_simulate_batch and runs its kernel (the same fires)
    const size_t nwords = (size_t)m->dev.ntiles * 32;
    rc = grow_device(ctx, &ctx->burn_aux, &ctx->burn_aux_bytes, nwords * 4 + 16,
                     "long-burn plane");
    if (rc) {
        if (tmp) cudaFree(tmp);
        return rc;
    }
    uint32_t *dlong = (uint32_t *)ctx->burn_aux;
    uint32_t *dany = dlong + nwords;
    uint32_t hany = 0;
    cudaError_t e0 = launch_long_burn(m->dev, db, dlong, dany, ctx->stream);
    if (e0 == cudaSuccess)
        e0 = cudaMemcpyAsync(&hany, dany, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(ctx->stream);
    if (e0 != cudaSuccess) {
        if (tmp) cudaFree(tmp);
        return cuda_err(ctx, e0, "long-burn plane");
    }
    if (!hany) {
        rc = launch_batch(ctx, m, n, dp, di, ds, max_steps, 0u, dout, dsteps,
                          nullptr);
        cudaError_t e = cudaSuccess;
        if (!rc && !dev) {
            e = cudaMemcpyAsync(out, dout, (size_t)n * sizeof(fire_result),
                                cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess && want_steps)
                e = cudaMemcpyAsync(burn_step, dsteps, (size_t)n * HW * 4,
                                    cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        }
        if (tmp) cudaFree(tmp);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_err(ctx, e, "burn-out results");
        if (!dev || (flags & FIRE_SYNC)) return fire_sync(ctx);
        return FIRE_OK;
    }
    // the bit-plane simulation kernel with burn times: state, two "still
    // burning" planes and a fuel byte per cell in each block's global buffer
    LaunchPlan plan;
    rc = plan_launch(ctx, m->dev.ntiles, n, &plan, true);
    if (rc) {
        if (tmp) cudaFree(tmp);
        return rc;
    }
    const size_t words = burn_block_words(m->dev.ntiles, (long long)HW);
    rc = grow_device(ctx, (void **)&ctx->gstate, &ctx->gstate_bytes,
                     (size_t)plan.grid * words * 4, "burn-time state");
    if (rc) {
        if (tmp) cudaFree(tmp);
        return rc;
    }
    SimLaunch a;
    std::memset(&a, 0, sizeof a);
    a.map = m->dev;
    a.nmaps = 1;
    a.ntiles_max = m->dev.ntiles;
    a.n = n;
    a.params = dp;
    a.ign = di;
    a.seeds = ds;
    a.out = dout;
    a.burn_step = dsteps;
    a.work_counter = ctx->counter;
    a.gstate = ctx->gstate;
    a.block_words = words;
    a.burn_time = db;
    a.long_burn = dlong;
    a.error_word = ctx->counter + 1;
    a.max_steps = max_steps;
    a.qcap = plan.qcap;
    a.cell_uniform = 0;
    cudaError_t e = cudaMemsetAsync(ctx->counter, 0, 4, ctx->stream);
    if (e == cudaSuccess)
        e = launch_simulate_burn(a, plan.nwarps, plan.grid, plan.L.total, ctx->stream);
    if (e == cudaSuccess && !dev) {
        e = cudaMemcpyAsync(out, dout, (size_t)n * sizeof(fire_result),
                            cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess && want_steps)
            e = cudaMemcpyAsync(burn_step, dsteps, (size_t)n * HW * 4,
                                cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_err(ctx, e, "burn-out launch");
    if (!dev || (flags & FIRE_SYNC)) return fire_sync(ctx);
    return FIRE_OK;
}

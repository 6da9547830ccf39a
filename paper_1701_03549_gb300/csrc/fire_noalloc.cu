// fire_simulate_batch_noalloc: the batched simulation for callers that must
// not have the library allocate device memory.
//
// fire_simulate_batch grows per-context device buffers on demand (argument
// staging, per-block state buffers for grids whose state does not fit in
// shared memory).  Some callers cannot allow that: code that runs under a
// fixed device-memory budget owned by another allocator, or a latency-bound
// loop in which cudaMalloc's implicit device synchronisation is not
// acceptable.  This entry point takes every input and output as a device
// pointer from the caller and keeps its own scratch (the work counter, the
// error word and the per-block state buffers) in one file-scope device array
// of fixed size, so it calls no cudaMalloc, cudaFree or other allocating
// routine.
//
// Rules of use:
//  * The array holds kNoAllocScratchBytes on every GPU that loads the
//    library, for as long as the process lives.  A map whose per-block state
//    buffer does not fit in it is rejected with FIRE_EINVAL; maps whose state
//    fits in shared memory need only the 256-byte counter area.
//  * The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) once; make that first call before any stream
//    capture begins on that device.
//  * Every call on a device shares the same array, which keeps the contents
//    left by the last call; the counter area is cleared by each call on its
//    stream before the kernel starts.  Calls whose work overlaps on the GPU
//    (for example on two streams) race on the array: serialise them.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "fire_internal.h"

using namespace fire;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;  // 2 MiB per GPU
constexpr size_t kCounterBytes = 256;                     // counter + error word
constexpr int kMaxDevices = 64;
// Flags this entry point honours; any other flag (FIRE_LONGEST_FIRST and
// FIRE_GRAPH need buffers the library would allocate) is refused.
constexpr uint32_t kNoAllocFlags =
    FIRE_DEVICE_PTRS | FIRE_WANT_STEPS | FIRE_SYNC | FIRE_CELL_UNIFORM;

// The scratch itself.  In host code this name is only a host-side stand-in:
// kernels receive the device address found by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

int na_err(fire_ctx *ctx, int code, const char *msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

int na_cuda(fire_ctx *ctx, cudaError_t e, const char *what)
{
    if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return FIRE_ECUDA;
}

// Device address of the scratch array on the current device (one-time
// lookup per device).
int scratch_address(fire_ctx *ctx, int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_cuda(ctx, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FIRE_OK;
}

}  // namespace

namespace fire {

// Reads and clears the error word of the no-alloc scratch on `device` (the
// current device), so that fire_sync reports a bounded wait that ran out in
// an asynchronous no-alloc call.  Returns FIRE_OK with *set = 0 when the
// scratch was never set up on that device.
int noalloc_take_error(int device, bool *set)
{
    *set = false;
    void *p = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (device < 0 || device >= kMaxDevices || !g_scratch_addr[device])
            return FIRE_OK;
        p = g_scratch_addr[device];
    }
    uint32_t *errw = static_cast<uint32_t *>(p) + 1;
    uint32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, errw, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return FIRE_ECUDA;
    if (v) {
        *set = true;
        e = cudaMemset(errw, 0, sizeof v);
        if (e != cudaSuccess) return FIRE_ECUDA;
    }
    return FIRE_OK;
}

}  // namespace fire

extern "C" int fire_simulate_batch_noalloc(fire_ctx *ctx, const fire_map *m,
                                           int n, const fire_params *params,
                                           const fire_cell *ignitions,
                                           const uint64_t *seeds,
                                           uint32_t max_steps, uint32_t flags,
                                           fire_result *out,
                                           int32_t *burn_step)
{
    if (!ctx) return FIRE_EINVAL;
    // every check below runs before the first CUDA call
    if (!valid_map(m)) return na_err(ctx, FIRE_EINVAL, "invalid map");
    if (m->ctx->device != ctx->device)
        return na_err(ctx, FIRE_EINVAL,
                      "the map was uploaded on another device than the context's");
    if (flags & ~kNoAllocFlags)
        return na_err(ctx, FIRE_EINVAL,
                      "flag not supported by the no-alloc entry point (it takes "
                      "FIRE_DEVICE_PTRS, FIRE_WANT_STEPS, FIRE_SYNC and "
                      "FIRE_CELL_UNIFORM only)");
    if (n < 0) return na_err(ctx, FIRE_EINVAL, "negative simulation count");
    if (n == 0) return FIRE_OK;
    if (!params || !ignitions || !seeds || !out)
        return na_err(ctx, FIRE_EINVAL, "NULL argument");
    const bool want_steps = (flags & FIRE_WANT_STEPS) != 0;
    if (want_steps && !burn_step)
        return na_err(ctx, FIRE_EINVAL, "FIRE_WANT_STEPS without burn_step");
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return na_err(ctx, FIRE_EINVAL, "device index beyond the set-up table");
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return na_cuda(ctx, e, "cudaGetDevice");
    if (cur != ctx->device && (e = cudaSetDevice(ctx->device)) != cudaSuccess)
        return na_cuda(ctx, e, "cudaSetDevice");
    void *scratch = nullptr;
    int rc = scratch_address(ctx, ctx->device, &scratch);
    if (rc) return rc;

    // launch shape, as fire_simulate_batch chooses it
    const int ntiles = m->dev.ntiles;
    LaunchPlan plan;
    rc = plan_launch(ctx, ntiles, n, &plan);
    if (rc) return rc;
    const bool smem_state = plan.smem_state;
    long long grid = plan.grid;
    if (!smem_state) {
        // each resident block needs its own state buffer inside the array
        const size_t per_block = 2 * (size_t)ntiles * 128;
        const size_t room = kNoAllocScratchBytes - kCounterBytes;
        const long long fit = (long long)(room / per_block);
        if (fit < 1) {
            char msg[256];
            snprintf(msg, sizeof msg,
                     "grid %d x %d needs %zu bytes of state scratch per block; "
                     "the no-alloc entry point has %zu",
                     m->dev.H, m->dev.W, per_block, room);
            return na_err(ctx, FIRE_EINVAL, msg);
        }
        grid = std::min(grid, fit);
    }

    uint32_t *counters = static_cast<uint32_t *>(scratch);
    SimLaunch a;
    a.map = m->dev;
    a.maps = nullptr;
    a.nmaps = 1;
    a.map_of_sim = nullptr;
    a.order = nullptr;
    a.ntiles_max = ntiles;
    a.n = n;
    a.params = params;
    a.ign = ignitions;
    a.seeds = seeds;
    a.out = out;
    a.burn_step = want_steps ? burn_step : nullptr;
    a.burnt_bits = nullptr;
    a.work_counter = counters;
    a.error_word = counters + 1;
    a.gstate = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) +
                                            kCounterBytes);
    a.block_words = 0;
    a.burn_time = nullptr;
    a.long_burn = nullptr;
    a.max_steps = max_steps;
    a.qcap = plan.qcap;
    a.cell_uniform = (flags & FIRE_CELL_UNIFORM) ? 1 : 0;
    e = cudaMemsetAsync(counters, 0, 2 * sizeof(uint32_t), ctx->stream);
    if (e == cudaSuccess)
        e = launch_simulate(a, smem_state, plan.nwarps, (int)grid, plan.L.total,
                            ctx->stream);
    if (e != cudaSuccess) return na_cuda(ctx, e, "no-alloc simulate launch");
    if (flags & FIRE_SYNC) {
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return na_cuda(ctx, e, "cudaStreamSynchronize");
        uint32_t errw = 0;
        e = cudaMemcpy(&errw, counters + 1, sizeof errw, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return na_cuda(ctx, e, "read error word");
        if (errw) return na_err(ctx, FIRE_ETIMEOUT, "a bounded device wait ran out");
    }
    return FIRE_OK;
}

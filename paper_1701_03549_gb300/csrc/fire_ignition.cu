// Ignition-point search (the paper's Sec. 3 experiment with the ignition
// treated as unknown) on the device, with its C ABI (include/fire.h).
//
// Reading (identical to the test oracle's, implemented independently):
//  * the target's burnt cells span rows [r0, r1] and columns [c0, c1];
//  * lattice point (a, b) sits at row r0 + floor((2a+1)(r1-r0+1) / (2 LH))
//    and column c0 + floor((2b+1)(c1-c0+1) / (2 LW));
//  * its candidate ignition is the burnable burnt cell nearest to it
//    (squared distance, ties to the lower row-major index);
//  * candidate c = a LW + b is simulated reps times with seeds
//    seed + c reps + r; its fitness is the replicate mean;
//  * the ensemble is the candidates with fitness <= cutoff (else the best,
//    ties to the lower index); the estimate is the mean and sample standard
//    deviation of their x = column and y = row.
#include "fire_internal.h"

using namespace fire;

namespace {

// Bounding box of the target's burnt cells: bbox = {r0, r1, c0, c1}.
__global__ void k_target_bbox(MapDev m, int *bbox)
{
    const int nw = m.ntiles * 32;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw;
         w += gridDim.x * blockDim.x) {
        const uint32_t t = m.tgt[w];
        if (!t) continue;
        const int k = w >> 5, ti = k / m.TW, tj = k - ti * m.TW;
        const int R = ti * 32 + (w & 31);
        const int cmin = tj * 32 + (__ffs(t) - 1);
        const int cmax = tj * 32 + (31 - __clz(t));
        atomicMin(&bbox[0], R);
        atomicMax(&bbox[1], R);
        atomicMin(&bbox[2], cmin);
        atomicMax(&bbox[3], cmax);
    }
}

// Row-major index of the burnable burnt cell nearest to (R, C): least
// (squared distance, index), one block cooperating (all threads call it);
// 0xffffffff when the target has no burnable cell.  The distance can exceed
// 32 bits on wide maps, so the pair is compared field by field.
__device__ uint32_t block_nearest(const MapDev &m, long long R, long long C)
{
    unsigned long long bd = ~0ull;
    uint32_t bi = 0xffffffffu;
    const int nw = m.ntiles * 32;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t t = m.tgt[w] & ~m.blk[w];
        if (!t) continue;
        const int k = w >> 5, ti = k / m.TW, tj = k - ti * m.TW;
        const long long Rw = ti * 32 + (w & 31);
        while (t) {
            const int i = __ffs(t) - 1;
            t &= t - 1;
            const long long Cc = tj * 32 + i;
            const unsigned long long d = (unsigned long long)(
                (Rw - R) * (Rw - R) + (Cc - C) * (Cc - C));
            const uint32_t idx = (uint32_t)(Rw * m.W + Cc);
            if (d < bd || (d == bd && idx < bi)) {
                bd = d;
                bi = idx;
            }
        }
    }
    __shared__ unsigned long long rd[256];
    __shared__ uint32_t ri[256];
    rd[threadIdx.x] = bd;
    ri[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const unsigned long long d2 = rd[threadIdx.x + s];
            const uint32_t i2 = ri[threadIdx.x + s];
            if (d2 < rd[threadIdx.x] ||
                (d2 == rd[threadIdx.x] && i2 < ri[threadIdx.x])) {
                rd[threadIdx.x] = d2;
                ri[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const uint32_t best = rd[0] == ~0ull ? 0xffffffffu : ri[0];
    __syncthreads();   // the arrays may be reused by the next call
    return best;
}

// One block (256 threads) per lattice point: nearest burnable burnt cell.
__global__ void k_snap(MapDev m, const int *__restrict__ bbox, int LH, int LW,
                       int32_t *__restrict__ cells, int *__restrict__ fail)
{
    const int cidx = blockIdx.x;
    const int a = cidx / LW, b = cidx - a * LW;
    const int r0 = bbox[0], r1 = bbox[1], c0 = bbox[2], c1 = bbox[3];
    const long long R = r0 + ((2LL * a + 1) * (r1 - r0 + 1)) / (2LL * LH);
    const long long C = c0 + ((2LL * b + 1) * (c1 - c0 + 1)) / (2LL * LW);
    const uint32_t best = block_nearest(m, R, C);
    if (threadIdx.x == 0) {
        if (best == 0xffffffffu) {
            atomicOr(fail, 1);
            cells[2 * cidx] = cells[2 * cidx + 1] = 0;
        } else {
            cells[2 * cidx] = (int32_t)(best / (uint32_t)m.W);
            cells[2 * cidx + 1] = (int32_t)(best % (uint32_t)m.W);
        }
    }
}

// A coordinate gene clamped to [0, hi] (a NaN counts as 0) and rounded half
// up.
__device__ __forceinline__ long long gene_coord(double v, int hi)
{
    const double c = v >= 0.0 ? (v > (double)hi ? (double)hi : v) : 0.0;
    return (long long)floor(__dadd_rn(c, 0.5));
}

// One block (256 threads) per individual: the ignition cell of its x
// (column) and y (row) genes, written to its reps simulations.
__global__ void k_snap_genes(MapDev m, int G, int gx, int gy,
                             const double *__restrict__ genes, int reps,
                             fire_cell *__restrict__ ign, int *__restrict__ fail)
{
    const long long j = blockIdx.x;
    const long long C = gene_coord(genes[j * G + gx], m.W - 1);
    const long long R = gene_coord(genes[j * G + gy], m.H - 1);
    const uint32_t best = block_nearest(m, R, C);
    fire_cell cell;
    cell.row = best == 0xffffffffu ? 0 : (int32_t)(best / (uint32_t)m.W);
    cell.col = best == 0xffffffffu ? 0 : (int32_t)(best % (uint32_t)m.W);
    if (best == 0xffffffffu && threadIdx.x == 0) atomicOr(fail, 1);
    for (int r = threadIdx.x; r < reps; r += blockDim.x) ign[j * reps + r] = cell;
}

__global__ void k_ign_batch(int L, int reps, const int32_t *__restrict__ cells,
                            const double *__restrict__ beta, uint64_t seed,
                            fire_params *__restrict__ params,
                            fire_cell *__restrict__ ign,
                            uint64_t *__restrict__ seeds)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L * reps) return;
    const int c = i / reps;
    fire_params p;
    for (int j = 0; j < 5; ++j) p.b[j] = beta[j];
    params[i] = p;
    ign[i].row = cells[2 * c];
    ign[i].col = cells[2 * c + 1];
    seeds[i] = seed + (uint64_t)i;   // = seed + c reps + r
}

// Ensemble estimate (one thread; sums in index order).
__global__ void k_ign_ensemble(int L, const double *__restrict__ fm,
                               const int32_t *__restrict__ cells, double cutoff,
                               double *__restrict__ xy)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int k = 0;
    double sx = 0.0, sy = 0.0;
    for (int c = 0; c < L; ++c)
        if (fm[c] <= cutoff) {
            k++;
            sx = __dadd_rn(sx, (double)cells[2 * c + 1]);
            sy = __dadd_rn(sy, (double)cells[2 * c]);
        }
    if (k == 0) {
        int b = 0;
        for (int c = 1; c < L; ++c) {
            const double fc = fm[c], fb = fm[b];
            const bool nc = fc != fc, nb = fb != fb;
            const bool better = (nc != nb) ? nb : (!nc && fc != fb ? fc < fb : false);
            if (better) b = c;
        }
        xy[0] = (double)cells[2 * b + 1];
        xy[1] = 0.0;
        xy[2] = (double)cells[2 * b];
        xy[3] = 0.0;
        return;
    }
    const double mx = __ddiv_rn(sx, (double)k), my = __ddiv_rn(sy, (double)k);
    double vx = 0.0, vy = 0.0;
    for (int c = 0; c < L; ++c)
        if (fm[c] <= cutoff) {
            const double dx = __dsub_rn((double)cells[2 * c + 1], mx);
            const double dy = __dsub_rn((double)cells[2 * c], my);
            vx = __dadd_rn(vx, __dmul_rn(dx, dx));
            vy = __dadd_rn(vy, __dmul_rn(dy, dy));
        }
    xy[0] = mx;
    xy[1] = k > 1 ? __dsqrt_rn(__ddiv_rn(vx, (double)(k - 1))) : 0.0;
    xy[2] = my;
    xy[3] = k > 1 ? __dsqrt_rn(__ddiv_rn(vy, (double)(k - 1))) : 0.0;
}

}  // namespace

extern "C" int ignition_search(fire_ctx *ctx, const fire_map *map,
                               const fire_params *params, int lat_h, int lat_w,
                               int reps, uint64_t seed, int kind, double cutoff,
                               uint32_t flags, double *fitness_map,
                               int32_t *cells, double xy_mean_sd[4])
{
    FIRE_NVTX("ignition_search");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(map) || !params || lat_h <= 0 || lat_w <= 0 || reps <= 0 ||
        (kind != 0 && kind != 1) || !fitness_map || !xy_mean_sd)
        return set_err(ctx, FIRE_EINVAL, "bad ignition_search arguments");
    const long long Lll = (long long)lat_h * lat_w;
    if (Lll * reps > 0x7fffffffll)
        return set_err(ctx, FIRE_EINVAL, "lattice x replicates too large");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const bool dev = flags & FIRE_DEVICE_PTRS;
    const int L = (int)Lll, n = L * reps;
    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += round16(bytes); return o; };
    const size_t o_bbox = take(16), o_fail = take(16), o_cells = take((size_t)L * 8);
    const size_t o_beta = take(40), o_par = take((size_t)n * sizeof(fire_params));
    const size_t o_ign = take((size_t)n * sizeof(fire_cell));
    const size_t o_seed = take((size_t)n * 8), o_res = take((size_t)n * sizeof(fire_result));
    const size_t o_fit = take((size_t)n * 8), o_fm = take((size_t)L * 8);
    const size_t o_xy = take(32);
    rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes, off, "ignition search");
    if (rc) return rc;
    char *base = (char *)ctx->staging;
    int *dbbox = (int *)(base + o_bbox);
    int *dfail = (int *)(base + o_fail);
    int32_t *dcells = (int32_t *)(base + o_cells);
    double *dbeta = (double *)(base + o_beta);
    fire_params *dpar = (fire_params *)(base + o_par);
    fire_cell *dign = (fire_cell *)(base + o_ign);
    uint64_t *dseed = (uint64_t *)(base + o_seed);
    fire_result *dres = (fire_result *)(base + o_res);
    double *dfit = (double *)(base + o_fit);
    double *dfm = (double *)(base + o_fm);
    double *dxy = (double *)(base + o_xy);
    cudaStream_t st = ctx->stream;
    const int init[4] = {0x7fffffff, -1, 0x7fffffff, -1};
    CUDA_TRY(ctx, cudaMemcpyAsync(dbbox, init, 16, cudaMemcpyHostToDevice, st), "bbox init");
    CUDA_TRY(ctx, cudaMemsetAsync(dfail, 0, 4, st), "fail init");
    CUDA_TRY(ctx, cudaMemcpyAsync(dbeta, params->b, 40,
                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  st), "params copy");
    k_target_bbox<<<152 * 4, 256, 0, st>>>(map->dev, dbbox);
    int hbbox[4];
    CUDA_TRY(ctx, cudaMemcpyAsync(hbbox, dbbox, 16, cudaMemcpyDeviceToHost, st), "bbox D2H");
    CUDA_TRY(ctx, cudaStreamSynchronize(st), "bbox sync");
    if (hbbox[1] < 0) return set_err(ctx, FIRE_EINVAL, "the map's target is empty");
    k_snap<<<L, 256, 0, st>>>(map->dev, dbbox, lat_h, lat_w, dcells, dfail);
    k_ign_batch<<<(n + 255) / 256, 256, 0, st>>>(L, reps, dcells, dbeta, seed, dpar,
                                                  dign, dseed);
    CUDA_TRY(ctx, cudaGetLastError(), "ignition set-up kernels");
    int hfail = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&hfail, dfail, 4, cudaMemcpyDeviceToHost, st), "fail D2H");
    CUDA_TRY(ctx, cudaStreamSynchronize(st), "snap sync");
    if (hfail) return set_err(ctx, FIRE_EINVAL, "the target has no burnable burnt cell");
    rc = fire_simulate_batch(ctx, map, n, dpar, dign, dseed, 0, FIRE_DEVICE_PTRS, dres,
                             nullptr);
    if (rc) return rc;
    rc = fire_fitness(ctx, dres, n, kind, FIRE_DEVICE_PTRS, dfit);
    if (rc) return rc;
    rc = fire_group_mean(ctx, dfit, L, reps, FIRE_DEVICE_PTRS, dfm);
    if (rc) return rc;
    k_ign_ensemble<<<1, 32, 0, st>>>(L, dfm, dcells, cutoff, dxy);
    CUDA_TRY(ctx, cudaGetLastError(), "ensemble kernel");
    const cudaMemcpyKind dk = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CUDA_TRY(ctx, cudaMemcpyAsync(fitness_map, dfm, (size_t)L * 8, dk, st), "fitness map");
    if (cells)
        CUDA_TRY(ctx, cudaMemcpyAsync(cells, dcells, (size_t)L * 8, dk, st), "cells");
    CUDA_TRY(ctx, cudaMemcpyAsync(xy_mean_sd, dxy, 32, dk, st), "estimate");
    return fire_sync(ctx);
}

extern "C" int fire_snap_ignitions(fire_ctx *ctx, const fire_map *map, int n,
                                   int genes, int gx, int gy,
                                   const double *genes_in, int reps,
                                   uint32_t flags, fire_cell *ignitions)
{
    FIRE_NVTX("fire_snap_ignitions");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(map) || n < 0 || genes < 1 || gx < 0 || gx >= genes ||
        gy < 0 || gy >= genes || reps < 1)
        return set_err(ctx, FIRE_EINVAL, "bad fire_snap_ignitions arguments");
    if (map->ctx->device != ctx->device)
        return set_err(ctx, FIRE_EINVAL, "the map was uploaded on another device");
    if (n == 0) return FIRE_OK;
    if (!genes_in || !ignitions) return set_err(ctx, FIRE_EINVAL, "NULL argument");
    if ((long long)n * reps > 0x7fffffffll)
        return set_err(ctx, FIRE_EINVAL, "individuals x replicates too large");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const bool dev = flags & FIRE_DEVICE_PTRS;
    const size_t bg = round16((size_t)n * genes * 8);
    const size_t bi = round16((size_t)n * reps * sizeof(fire_cell));
    rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes,
                     16 + (dev ? 0 : bg + bi), "ignition genes");
    if (rc) return rc;
    char *base = (char *)ctx->staging;
    int *dfail = (int *)base;
    const double *dgenes = genes_in;
    fire_cell *dign = ignitions;
    cudaStream_t st = ctx->stream;
    if (!dev) {
        dgenes = (const double *)(base + 16);
        dign = (fire_cell *)(base + 16 + bg);
        CUDA_TRY(ctx, cudaMemcpyAsync((void *)dgenes, genes_in, (size_t)n * genes * 8,
                                      cudaMemcpyHostToDevice, st), "genes H2D");
    }
    CUDA_TRY(ctx, cudaMemsetAsync(dfail, 0, 4, st), "fail init");
    k_snap_genes<<<n, 256, 0, st>>>(map->dev, genes, gx, gy, dgenes, reps, dign, dfail);
    CUDA_TRY(ctx, cudaGetLastError(), "snap kernel");
    if (!dev)
        CUDA_TRY(ctx, cudaMemcpyAsync(ignitions, dign, (size_t)n * reps * sizeof(fire_cell),
                                      cudaMemcpyDeviceToHost, st), "ignitions D2H");
    int hfail = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&hfail, dfail, 4, cudaMemcpyDeviceToHost, st), "fail D2H");
    CUDA_TRY(ctx, cudaStreamSynchronize(st), "snap sync");
    if (hfail) return set_err(ctx, FIRE_EINVAL, "the target has no burnable burnt cell");
    return FIRE_OK;
}

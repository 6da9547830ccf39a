// Genetic-algorithm generation (the paper's Appendix B) and replicate
// averaging on the device, with their C ABI (include/fire.h).
//
// Reading of the constants the paper leaves open (identical to the test
// oracle's, which implements it independently):
//  * individuals are ordered by fitness, lower is better, NaN worst, ties to
//    the lower index;
//  * E = min(2, P) elites (best first) fill slots 0..E-1 unchanged;
//  * slot j >= E: Philox4x32-10 block (j, g, 0, 0) under key ga_seed gives
//    contestants a = (w0 P) >> 32, b = (w1 P) >> 32; the better is the parent;
//  * pairs (j, j + 1), j = E, E + 2, ...: block (j, g, 1, 0), cut
//    c = 1 + ((w0 (G - 1)) >> 32); child j takes genes [0, c) from its parent
//    and [c, G) from the partner's, child j + 1 the reverse; an unpaired last
//    slot copies its parent; G = 1 never crosses;
//  * gene k of child j: block (j, g, 2, k); with s = 1 - g / NG,
//    pm = 0.2 s + 0.01, T = floor(pm 2^32): mutate iff w0 < T, by
//    (2 u - 1) (0.1 (hi_k - lo_k)) s with u = w1 2^-32, then clamp to
//    [lo_k, hi_k].
// All double arithmetic uses explicitly rounded operations in that order.
#include <cmath>

#include "fire_internal.h"

using namespace fire;

namespace {

__device__ __forceinline__ bool ga_better(const double *f, int a, int b)
{
    const double fa = f[a], fb = f[b];
    const bool na = fa != fa, nb = fb != fb;
    if (na != nb) return nb;
    if (!na && fa != fb) return fa < fb;
    return a < b;
}

// The two best individuals (one block).
__global__ void k_ga_elite(int P, const double *__restrict__ f, int *elite)
{
    __shared__ int cand[256];
    for (int pass = 0; pass < 2; ++pass) {
        const int skip = pass == 0 ? -1 : elite[0];
        int best = -1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            if (i == skip) continue;
            if (best < 0 || ga_better(f, i, best)) best = i;
        }
        cand[threadIdx.x] = best;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const int a = cand[threadIdx.x], b = cand[threadIdx.x + s];
                if (a < 0 || (b >= 0 && ga_better(f, b, a))) cand[threadIdx.x] = b;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) elite[pass] = cand[0];
        __syncthreads();
    }
}

__global__ void k_ga_select(int P, int E, const double *__restrict__ f,
                            uint32_t g, uint32_t k0, uint32_t k1,
                            int *__restrict__ parent)
{
    const int j = E + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const uint4 w = philox4x32_10((uint32_t)j, g, 0u, 0u, k0, k1);
    const int a = (int)(((unsigned long long)w.x * (unsigned)P) >> 32);
    const int b = (int)(((unsigned long long)w.y * (unsigned)P) >> 32);
    parent[j] = ga_better(f, a, b) ? a : b;
}

__device__ __forceinline__ void ga_mutate(double *child, int j, int G,
                                          uint32_t g, double s, uint64_t T,
                                          uint32_t k0, uint32_t k1,
                                          const double *lo, const double *hi)
{
    for (int k = 0; k < G; ++k) {
        const uint4 w = philox4x32_10((uint32_t)j, g, 2u, (uint32_t)k, k0, k1);
        if ((uint64_t)w.x >= T) continue;
        const double u = __dmul_rn((double)w.y, 0x1p-32);
        const double scale = __dmul_rn(__dmul_rn(0.1, __dsub_rn(hi[k], lo[k])), s);
        const double delta = __dmul_rn(__dsub_rn(__dmul_rn(2.0, u), 1.0), scale);
        double x = __dadd_rn(child[k], delta);
        if (x < lo[k]) x = lo[k];
        if (x > hi[k]) x = hi[k];
        child[k] = x;
    }
}

// One thread per elite slot or per pair of child slots.
__global__ void k_ga_breed(int P, int G, int E, const double *__restrict__ gin,
                           const int *__restrict__ parent,
                           const int *__restrict__ elite, uint32_t g, int NG,
                           uint32_t k0, uint32_t k1,
                           const double *__restrict__ lo,
                           const double *__restrict__ hi,
                           double *__restrict__ gout)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < E) {
        for (int k = 0; k < G; ++k)
            gout[(long long)u * G + k] = gin[(long long)elite[u] * G + k];
        return;
    }
    const int j = E + 2 * (u - E);
    if (j >= P) return;
    const double s = __dsub_rn(1.0, __ddiv_rn((double)g, (double)NG));
    const double pm = __dadd_rn(__dmul_rn(0.2, s), 0.01);
    const uint64_t T = (uint64_t)floor(__dmul_rn(pm, 4294967296.0));
    const double *pa = gin + (long long)parent[j] * G;
    double *ca = gout + (long long)j * G;
    if (j + 1 >= P || G < 2) {
        for (int k = 0; k < G; ++k) ca[k] = pa[k];
        ga_mutate(ca, j, G, g, s, T, k0, k1, lo, hi);
        if (j + 1 < P) {
            const double *pb = gin + (long long)parent[j + 1] * G;
            double *cb = gout + (long long)(j + 1) * G;
            for (int k = 0; k < G; ++k) cb[k] = pb[k];
            ga_mutate(cb, j + 1, G, g, s, T, k0, k1, lo, hi);
        }
        return;
    }
    const double *pb = gin + (long long)parent[j + 1] * G;
    double *cb = gout + (long long)(j + 1) * G;
    const uint4 w = philox4x32_10((uint32_t)j, g, 1u, 0u, k0, k1);
    const int cut = 1 + (int)(((unsigned long long)w.x * (unsigned)(G - 1)) >> 32);
    for (int k = 0; k < G; ++k) {
        ca[k] = k < cut ? pa[k] : pb[k];
        cb[k] = k < cut ? pb[k] : pa[k];
    }
    ga_mutate(ca, j, G, g, s, T, k0, k1, lo, hi);
    ga_mutate(cb, j + 1, G, g, s, T, k0, k1, lo, hi);
}

__global__ void k_group_mean(const double *__restrict__ v, int groups,
                             int per_group, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= groups) return;
    double s = 0.0;
    for (int r = 0; r < per_group; ++r)
        s = __dadd_rn(s, v[(long long)i * per_group + r]);
    out[i] = __ddiv_rn(s, (double)per_group);
}

}  // namespace

extern "C" {

int ga_step(fire_ctx *ctx, int pop, int genes, const double *genes_in,
            const double *fitness, int generation, int total_gens,
            uint64_t ga_seed, const double *lo, const double *hi,
            uint32_t flags, double *genes_out)
{
    FIRE_NVTX("ga_step");
    if (!ctx) return FIRE_EINVAL;
    if (pop <= 0 || genes <= 0 || total_gens <= 0 || generation < 0 ||
        !genes_in || !fitness || !lo || !hi || !genes_out)
        return set_err(ctx, FIRE_EINVAL, "bad ga_step arguments");
    const bool dev = flags & FIRE_DEVICE_PTRS;
    {
        // children are written while parents are read: no overlap
        const char *a = (const char *)genes_in, *b = (const char *)genes_out;
        const size_t len = (size_t)pop * genes * sizeof(double);
        if (a < b + len && b < a + len)
            return set_err(ctx, FIRE_EINVAL, "genes_out overlaps genes_in");
    }
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t bg = round16((size_t)pop * genes * sizeof(double));
    const size_t bf = round16((size_t)pop * sizeof(double));
    const size_t bb = round16((size_t)genes * sizeof(double));
    const size_t bp = round16((size_t)pop * sizeof(int) + 2 * sizeof(int));
    const size_t need = bp + (dev ? 0 : 2 * bg + bf + 2 * bb);
    rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes, need, "ga staging");
    if (rc) return rc;
    char *p = (char *)ctx->staging;
    int *parent = (int *)p;
    int *elite = parent + pop;
    const double *dgin = genes_in, *dfit = fitness, *dlo = lo, *dhi = hi;
    double *dgout = genes_out;
    if (!dev) {
        double *a = (double *)(p + bp);
        double *o = (double *)(p + bp + bg);
        double *f = (double *)(p + bp + 2 * bg);
        double *l = (double *)(p + bp + 2 * bg + bf);
        double *h = (double *)(p + bp + 2 * bg + bf + bb);
        CUDA_TRY(ctx, cudaMemcpyAsync(a, genes_in, (size_t)pop * genes * 8,
                                      cudaMemcpyHostToDevice, ctx->stream), "genes H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync(f, fitness, (size_t)pop * 8,
                                      cudaMemcpyHostToDevice, ctx->stream), "fitness H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync(l, lo, (size_t)genes * 8,
                                      cudaMemcpyHostToDevice, ctx->stream), "lo H2D");
        CUDA_TRY(ctx, cudaMemcpyAsync(h, hi, (size_t)genes * 8,
                                      cudaMemcpyHostToDevice, ctx->stream), "hi H2D");
        dgin = a;
        dgout = o;
        dfit = f;
        dlo = l;
        dhi = h;
    }
    const int E = pop < 2 ? pop : 2;
    const uint32_t k0 = (uint32_t)ga_seed, k1 = (uint32_t)(ga_seed >> 32);
    k_ga_elite<<<1, 256, 0, ctx->stream>>>(pop, dfit, elite);
    if (pop > E)
        k_ga_select<<<(pop - E + 255) / 256, 256, 0, ctx->stream>>>(
            pop, E, dfit, (uint32_t)generation, k0, k1, parent);
    const int units = E + (pop - E + 1) / 2;
    k_ga_breed<<<(units + 127) / 128, 128, 0, ctx->stream>>>(
        pop, genes, E, dgin, parent, elite, (uint32_t)generation, total_gens,
        k0, k1, dlo, dhi, dgout);
    CUDA_TRY(ctx, cudaGetLastError(), "ga kernels");
    if (!dev) {
        CUDA_TRY(ctx, cudaMemcpyAsync(genes_out, dgout, (size_t)pop * genes * 8,
                                      cudaMemcpyDeviceToHost, ctx->stream), "genes D2H");
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "ga sync");
    } else if (flags & FIRE_SYNC) {
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "ga sync");
    }
    return FIRE_OK;
}

int fire_group_mean(fire_ctx *ctx, const double *values, int groups,
                    int per_group, uint32_t flags, double *out)
{
    FIRE_NVTX("fire_group_mean");
    if (!ctx) return FIRE_EINVAL;
    if (groups < 0 || per_group <= 0)
        return set_err(ctx, FIRE_EINVAL, "bad group-mean arguments");
    if (groups == 0) return FIRE_OK;
    if (!values || !out) return set_err(ctx, FIRE_EINVAL, "NULL argument");
    const size_t n = (size_t)groups * per_group;
    if (flags & FIRE_DEVICE_PTRS) {
        // one thread reads a group while another writes its mean: no overlap
        const char *a = (const char *)values, *b = (const char *)out;
        if (a < b + (size_t)groups * 8 && b < a + n * 8)
            return set_err(ctx, FIRE_EINVAL, "device out overlaps values");
    }
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const double *dv = values;
    double *dout = out;
    if (!(flags & FIRE_DEVICE_PTRS)) {
        rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes,
                         round16(n * 8) + round16((size_t)groups * 8), "mean staging");
        if (rc) return rc;
        double *a = (double *)ctx->staging;
        dout = (double *)((char *)ctx->staging + round16(n * 8));
        CUDA_TRY(ctx, cudaMemcpyAsync(a, values, n * 8, cudaMemcpyHostToDevice,
                                      ctx->stream), "values H2D");
        dv = a;
    }
    k_group_mean<<<(groups + 255) / 256, 256, 0, ctx->stream>>>(dv, groups,
                                                                per_group, dout);
    CUDA_TRY(ctx, cudaGetLastError(), "group mean");
    if (!(flags & FIRE_DEVICE_PTRS)) {
        CUDA_TRY(ctx, cudaMemcpyAsync(out, dout, (size_t)groups * 8,
                                      cudaMemcpyDeviceToHost, ctx->stream), "mean D2H");
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "mean sync");
    } else if (flags & FIRE_SYNC) {
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "mean sync");
    }
    return FIRE_OK;
}

}  // extern "C"

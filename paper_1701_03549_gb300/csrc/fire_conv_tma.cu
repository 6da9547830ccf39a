// TMA-fed implicit-GEMM convolution for the surrogate's 128 -> 128 layers
// (forward and input gradient), on tcgen05 tensor cores.
//
// A CTA computes a 128-pixel x 128-channel tile.  The K loop runs over the
// 9 taps x 2 halves of 64 input channels; for each 64-wide slab
//   * one thread issues two TMA loads: the activation tile, shifted by the
//     tap's offset, through a 4-D tensor map over the NHWC buffer (channels,
//     x, y, sample) whose out-of-range elements read as zero (the zero
//     padding of the convolution), and the 128 x 64 weight slab through a 2-D
//     map; both land 128-byte swizzled, which is the canonical K-major
//     SWIZZLE_128B operand layout of the tensor core;
//   * another thread waits for the slab, issues four 128 x 128 x 16 MMAs into
//     the tensor-memory accumulator and commits them to the slab's "empty"
//     barrier, which hands the stage back to the loader.
// k_conv_tma runs one tile per CTA: two stages (64 KB) let three CTAs share
// an SM, so the epilogues of some (tensor memory -> registers -> bias/ReLU or
// ReLU mask -> BF16 stores) overlap the main loops of the others.
// k_conv_tma_p, the default, is persistent: two CTAs per SM loop over tiles
// with three stages and two tensor-memory accumulators, the loads and MMAs
// of the next tile overlapping the epilogue of the previous one within the
// CTA (on a GB300, 9 % more training throughput than k_conv_tma; a single
// persistent CTA per SM was slower than either).  Every wait is bounded; on a
// timeout the CTA records an error, waits (bounded) for its own copies and
// MMAs in flight, frees its tensor memory and returns.
#include "fire_internal.h"
#include "fire_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace fire {
namespace convtma {

#ifndef FIRE_CONV_STAGES
#define FIRE_CONV_STAGES 2
#endif
#ifndef FIRE_CONV_PERSISTENT
#define FIRE_CONV_PERSISTENT 1   // 0: one tile per CTA (k_conv_tma)
#endif
constexpr int kStages = FIRE_CONV_STAGES;       // shared-memory stages per CTA
constexpr int kTileBytes = 128 * 128;           // 128 rows x 64 BF16
constexpr int kStageBytes = 2 * kTileBytes;     // A + B
constexpr int kSmem = kStages * kStageBytes + 1024;
constexpr int kSlabs = 18;                      // 9 taps x 2 channel halves
// CTAs that fit on one SM (227 KB of shared memory; 128 tensor-memory
// columns each, so at most four).
constexpr int kCtasPerSm =
    (227 * 1024) / (kSmem + 2048) > 4 ? 4 : (227 * 1024) / (kSmem + 2048);
// The weight-gradient kernel's own stage count and residency.
#ifndef FIRE_WGRAD_STAGES
#define FIRE_WGRAD_STAGES 2
#endif
constexpr int kWStages = FIRE_WGRAD_STAGES;
constexpr int kWSmem = kWStages * kStageBytes + 1024;
constexpr int kWCtasPerSm =
    (227 * 1024) / (kWSmem + 2048) > 4 ? 4 : (227 * 1024) / (kWSmem + 2048);

struct Epi {
    int mode;                 // 0 forward (bias + ReLU), 1 input gradient (mask)
    const float *bias;        // forward
    const uint16_t *hprev;    // input gradient: activations of the layer below
    uint16_t *out;            // [P][128] BF16
};

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3ffffu) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // SBO: 8 rows x 128 B
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ void expect_tx(void *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     tc::smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap *map, int c0,
                                       int c1, int c2, int c3, void *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::"
        "bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(tc::smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int c0,
                                       int c1, void *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::"
        "bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1),
        "r"(tc::smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ bool pos16(uint32_t u)
{
    return !(u & 0x8000u) && (u & 0x7fffu);
}

// Epilogue of one accumulator row (pixel p, 128 channels in tensor memory at
// taddr): forward, bias and ReLU; input gradient, zero where the layer
// below's activation is not positive; BF16 stores.
__device__ __forceinline__ void conv_epilogue(const Epi &epi, const float *s_bias,
                                              uint32_t taddr, int p)
{
    uint16_t *orow = epi.out + (size_t)p * 128;
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 32) {
        float v[32];
        tc::tmem_ld32(taddr + (uint32_t)c0, v);
        uint32_t pk[16];
        if (epi.mode == 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                pk[j] = pack2(fmaxf(v[2 * j] + s_bias[c0 + 2 * j], 0.0f),
                              fmaxf(v[2 * j + 1] + s_bias[c0 + 2 * j + 1], 0.0f));
        } else {
            const uint4 *hp =
                reinterpret_cast<const uint4 *>(epi.hprev + (size_t)p * 128 + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 h = hp[q];
                const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int e = 2 * (4 * q + j);
                    pk[4 * q + j] = pack2(pos16(hw[j] & 0xffffu) ? v[e] : 0.0f,
                                          pos16(hw[j] >> 16) ? v[e + 1] : 0.0f);
                }
            }
        }
        uint4 *o = reinterpret_cast<uint4 *>(orow + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            o[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
}

// sign = +1: forward (source pixel p + off(t)); -1: input gradient (p - off(t)).
__global__ void __launch_bounds__(128, kCtasPerSm)
    k_conv_tma(const __grid_constant__ CUtensorMap act,
               const __grid_constant__ CUtensorMap wts, Epi epi, int S, int lgS,
               int d, int sign, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_consumed;
    __shared__ float s_bias[128];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (tc::smem_addr(smem_raw) + 1023u) & ~1023u;
    const int m0 = blockIdx.x * 128;
    if (epi.mode == 0) s_bias[tid] = epi.bias[tid];
    const int b = m0 >> (2 * lgS);
    const int y0 = (m0 >> lgS) & (S - 1), x0 = m0 & (S - 1);

    if (warp == 0) {
        tc::tmem_alloc(&tmem_slot, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(&done, 1);
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // loader
        int s = 0;
        for (; s < kSlabs; ++s) {
            const int st = s % kStages;
            if (s >= kStages &&
                !tc::mbar_wait_bounded(&empty[st], ((s / kStages) - 1) & 1)) {
                atomicOr(&s_fail, 1);
                break;
            }
            if (*(volatile int *)&s_fail) break;
            const int tap = s >> 1, c0 = (s & 1) * 64;
            const int dy = sign * (tap / 3 - 1) * d, dx = sign * (tap % 3 - 1) * d;
            const uint32_t sa = base + st * kStageBytes;
            expect_tx(&full[st], kStageBytes);
            tma_4d(sa, &act, c0, x0 + dx, y0 + dy, b, &full[st]);
            tma_2d(sa + kTileBytes, &wts, s * 64, 0, &full[st]);
        }
        s_issued = s;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
        int s = 0;
        for (; s < kSlabs; ++s) {
            const int st = s % kStages;
            if (!tc::mbar_wait_bounded(&full[st], (s / kStages) & 1)) {
                atomicOr(&s_fail, 1);
                break;
            }
            tc::fence_after_sync();
            const uint32_t sa = base + st * kStageBytes, sb = sa + kTileBytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(tmem, desc_sw128(sa + kk * 32), desc_sw128(sb + kk * 32),
                             idesc, s > 0 || kk > 0);
            tc::mma_commit(&empty[st]);
        }
        s_consumed = s;
        if (s == kSlabs) tc::mma_commit(&done);
    }
    __syncwarp();
    if (!tc::mbar_wait_bounded(&done, 0)) atomicOr(&s_fail, 1);
    __syncthreads();
    tc::fence_after_sync();

    if (!s_fail) {
        conv_epilogue(epi, s_bias, tmem + ((uint32_t)(warp * 32) << 16),
                      m0 + warp * 32 + lane);
    } else if (tid == 0) {
        atomicOr(err, 1u);
        // copies issued but never consumed must land before the CTA leaves
        for (int s = s_consumed; s < s_issued; ++s)
            tc::mbar_wait_bounded(&full[s % kStages], (s / kStages) & 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// Persistent variant of k_conv_tma: two CTAs per SM, each looping over tiles
// (tile = blockIdx.x, blockIdx.x + gridDim.x, ...) with three shared-memory
// stages and two 128-column tensor-memory accumulators, so that the next
// tile's loads and MMAs run while the previous tile's epilogue drains its
// accumulator.  Warp 0 (one thread) issues the TMA loads, warp 1 (one thread)
// the MMAs, warps 2..5 run the epilogue (warp w reads tensor-memory lanes
// 32 (w mod 4) .. 32 (w mod 4) + 31, as tcgen05.ld requires).  Every wait is
// bounded; on a timeout the CTA records an error, lets its copies and MMAs in
// flight finish (bounded), frees its tensor memory and returns.
constexpr int kPStages = 3;
constexpr int kPSmem = kPStages * kStageBytes + 1024;
constexpr int kPThreads = 192;

__device__ __forceinline__ void mbar_arrive(void *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                     tc::smem_addr(bar))
                 : "memory");
}

__global__ void __launch_bounds__(kPThreads, 2)
    k_conv_tma_p(const __grid_constant__ CUtensorMap act,
                 const __grid_constant__ CUtensorMap wts, Epi epi, int S, int lgS,
                 int d, int sign, int ntiles, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kPStages], empty[kPStages];
    __shared__ __align__(8) unsigned long long tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_consumed;
    __shared__ float s_bias[128];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (tc::smem_addr(smem_raw) + 1023u) & ~1023u;
    if (epi.mode == 0 && tid < 128) s_bias[tid] = epi.bias[tid];
    if (warp == 0) {
        tc::tmem_alloc(&tmem_slot, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kPStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], 128);   // every epilogue thread arrives
        }
        tc::mbar_init(&done, 1);
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // loader: slab g of the CTA's sequence uses stage g mod kPStages
            int g = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                const int m0 = tile * 128;
                const int b = m0 >> (2 * lgS);
                const int y0 = (m0 >> lgS) & (S - 1), x0 = m0 & (S - 1);
                for (int s = 0; s < kSlabs; ++s, ++g) {
                    const int st = g % kPStages;
                    if (g >= kPStages &&
                        !tc::mbar_wait_bounded(&empty[st],
                                               ((g / kPStages) - 1) & 1)) {
                        atomicOr(&s_fail, 1);
                        ok = false;
                        break;
                    }
                    if (*(volatile int *)&s_fail) {
                        ok = false;
                        break;
                    }
                    const int tap = s >> 1, c0 = (s & 1) * 64;
                    const int dy = sign * (tap / 3 - 1) * d;
                    const int dx = sign * (tap % 3 - 1) * d;
                    const uint32_t sa = base + st * kStageBytes;
                    expect_tx(&full[st], kStageBytes);
                    tma_4d(sa, &act, c0, x0 + dx, y0 + dy, b, &full[st]);
                    tma_2d(sa + kTileBytes, &wts, s * 64, 0, &full[st]);
                }
            }
            s_issued = g;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile number `it` of this CTA accumulates in buffer
            // it & 1, once the epilogue has drained that buffer's last use
            constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
            int g = 0, it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < ntiles;
                 tile += gridDim.x, ++it) {
                const int acc = it & 1;
                if (it >= 2 &&
                    !tc::mbar_wait_bounded(&tempty[acc], ((it >> 1) - 1) & 1)) {
                    atomicOr(&s_fail, 1);
                    break;
                }
                tc::fence_after_sync();
                const uint32_t td = tmem + (uint32_t)(acc * 128);
                for (int s = 0; s < kSlabs; ++s, ++g) {
                    const int st = g % kPStages;
                    if (!tc::mbar_wait_bounded(&full[st], (g / kPStages) & 1)) {
                        atomicOr(&s_fail, 1);
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sa = base + st * kStageBytes, sb = sa + kTileBytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(td, desc_sw128(sa + kk * 32),
                                     desc_sw128(sb + kk * 32), idesc,
                                     s > 0 || kk > 0);
                    tc::mma_commit(&empty[st]);
                }
                if (ok) tc::mma_commit(&tfull[acc]);
            }
            s_consumed = g;
            tc::mma_commit(&done);   // arrives once every issued MMA is done
        }
    } else {
        // epilogue: tile number `it` is read from buffer it & 1
        const int q = warp & 3;   // tensor-memory lane quarter of this warp
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const int acc = it & 1;
            if (*(volatile int *)&s_fail) break;
            if (!tc::mbar_wait_bounded(&tfull[acc], (it >> 1) & 1)) {
                atomicOr(&s_fail, 1);
                break;
            }
            tc::fence_after_sync();
            conv_epilogue(epi, s_bias,
                          tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 128),
                          tile * 128 + q * 32 + lane);
            tc::fence_before_sync();
            mbar_arrive(&tempty[acc]);
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_fail) {
            atomicOr(err, 1u);
            // copies issued but never consumed must land before the CTA leaves
            for (int g = s_consumed; g < s_issued; ++g)
                tc::mbar_wait_bounded(&full[g % kPStages], (g / kPStages) & 1);
        }
        // every MMA this CTA issued has completed
        tc::mbar_wait_bounded(&done, 0);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// Weight gradient of a 128 -> 128 layer: D[o][(t, i)] = sum_p dz[p, o]
// in[p + off(t), i].  CTA (tap t = blockIdx.y, pixel range blockIdx.z) runs
// 64-pixel slabs; both operands are MN-major (8 consecutive channels per 16
// bytes, pixels along K).  Each slab is two 64-channel TMA boxes per operand,
// which land as the MN-major SWIZZLE_128B layout: channel halves 8 KB apart
// (LBO), 8-pixel groups 1 KB apart (SBO).  Partial sums are added to dW with
// FP32 atomics.
__device__ __forceinline__ uint64_t desc_sw128_mn(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3ffffu) >> 4);
    d |= (uint64_t)(8192 >> 4) << 16;       // LBO: next 64 MN elements
    d |= (uint64_t)(1024 >> 4) << 32;       // SBO: next 8 K rows
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

__global__ void __launch_bounds__(128, kWCtasPerSm)
    k_wgrad_tma(const __grid_constant__ CUtensorMap dzm,
                const __grid_constant__ CUtensorMap inm, float *dw, int S, int lgS,
                int d, int slabs_total, int slabs_per, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kWStages], empty[kWStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_consumed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (tc::smem_addr(smem_raw) + 1023u) & ~1023u;
    const int tap = blockIdx.y;
    const int dy = (tap / 3 - 1) * d, dx = (tap % 3 - 1) * d;
    const int s0 = blockIdx.z * slabs_per;
    const int ns = min(slabs_total - s0, slabs_per);

    if (warp == 0) {
        tc::tmem_alloc(&tmem_slot, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kWStages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(&done, 1);
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (ns > 0 && warp == 0 && lane == 0) {
        int s = 0;
        for (; s < ns; ++s) {
            const int st = s % kWStages;
            if (s >= kWStages &&
                !tc::mbar_wait_bounded(&empty[st], ((s / kWStages) - 1) & 1)) {
                atomicOr(&s_fail, 1);
                break;
            }
            if (*(volatile int *)&s_fail) break;
            const int p0 = (s0 + s) * 64;
            const int b = p0 >> (2 * lgS);
            const int y = (p0 >> lgS) & (S - 1), x = p0 & (S - 1);
            const uint32_t sa = base + st * kStageBytes, sb = sa + kTileBytes;
            expect_tx(&full[st], kStageBytes);
            tma_4d(sa, &dzm, 0, x, y, b, &full[st]);
            tma_4d(sa + 8192, &dzm, 64, x, y, b, &full[st]);
            tma_4d(sb, &inm, 0, x + dx, y + dy, b, &full[st]);
            tma_4d(sb + 8192, &inm, 64, x + dx, y + dy, b, &full[st]);
        }
        s_issued = s;
    } else if (ns > 0 && warp == 1 && lane == 0) {
        constexpr uint32_t idesc =
            tc::idesc_bf16(128, 128) | (1u << 15) | (1u << 16);   // both MN-major
        int s = 0;
        for (; s < ns; ++s) {
            const int st = s % kWStages;
            if (!tc::mbar_wait_bounded(&full[st], (s / kWStages) & 1)) {
                atomicOr(&s_fail, 1);
                break;
            }
            tc::fence_after_sync();
            const uint32_t sa = base + st * kStageBytes, sb = sa + kTileBytes;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc::mma_bf16(tmem, desc_sw128_mn(sa + kk * 2048),
                             desc_sw128_mn(sb + kk * 2048), idesc, s > 0 || kk > 0);
            tc::mma_commit(&empty[st]);
        }
        s_consumed = s;
        if (s == ns) tc::mma_commit(&done);
    }
    __syncwarp();
    if (ns > 0 && !tc::mbar_wait_bounded(&done, 0)) atomicOr(&s_fail, 1);
    __syncthreads();
    tc::fence_after_sync();

    if (ns > 0 && !s_fail) {
        const int o = warp * 32 + lane;
        // 16-byte aligned: dw, the row stride (1152 floats) and tap * 128 are
        // multiples of four floats
        float4 *row = reinterpret_cast<float4 *>(dw + (size_t)o * 1152 + tap * 128);
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                atomicAdd(row + c0 / 4 + j,
                          make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
        }
    } else if (s_fail && tid == 0) {
        atomicOr(err, 1u);
        for (int s = s_consumed; s < s_issued; ++s)
            tc::mbar_wait_bounded(&full[s % kWStages], (s / kWStages) & 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// First layer (16 -> 128 channels): one tap per 16-wide K slab.  The
// activation box is 16 channels (32 bytes) x 128 pixels and the weight box
// 16 x 128 rows of W1[o][t][i]; both land 32-byte swizzled, the canonical
// K-major SWIZZLE_32B layout (8-row groups 256 bytes apart), and one
// 128 x 128 x 16 MMA consumes a slab.  Nine slabs, no padding of K.
constexpr int kC1Stages = 6;                     // 49 KB: four CTAs per SM, as
                                                  // many as tensor memory holds
constexpr int kC1Tile = 128 * 32;                 // 128 rows x 16 BF16
constexpr int kC1Stage = 2 * kC1Tile;
constexpr int kC1Smem = kC1Stages * kC1Stage + 1024;

__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3ffffu) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
    d |= (uint64_t)(256 >> 4) << 32;        // SBO: 8 rows x 32 B
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;                 // SWIZZLE_32B
    return d;
}

__global__ void __launch_bounds__(128, 4)
    k_conv1_tma(const __grid_constant__ CUtensorMap act,
                const __grid_constant__ CUtensorMap wts, const float *bias,
                uint16_t *out, int S, int lgS, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full[kC1Stages], empty[kC1Stages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_consumed;
    __shared__ float s_bias[128];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = (tc::smem_addr(smem_raw) + 1023u) & ~1023u;
    const int m0 = blockIdx.x * 128;
    const int b = m0 >> (2 * lgS);
    const int y0 = (m0 >> lgS) & (S - 1), x0 = m0 & (S - 1);
    s_bias[tid] = bias[tid];

    if (warp == 0) {
        tc::tmem_alloc(&tmem_slot, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kC1Stages; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(&done, 1);
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        int s = 0;
        for (; s < 9; ++s) {
            const int st = s % kC1Stages;
            if (s >= kC1Stages &&
                !tc::mbar_wait_bounded(&empty[st], ((s / kC1Stages) - 1) & 1)) {
                atomicOr(&s_fail, 1);
                break;
            }
            if (*(volatile int *)&s_fail) break;
            const int dy = s / 3 - 1, dx = s % 3 - 1;   // dilation 1
            const uint32_t sa = base + st * kC1Stage;
            expect_tx(&full[st], kC1Stage);
            tma_4d(sa, &act, 0, x0 + dx, y0 + dy, b, &full[st]);
            tma_2d(sa + kC1Tile, &wts, s * 16, 0, &full[st]);
        }
        s_issued = s;
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16(128, 128);
        int s = 0;
        for (; s < 9; ++s) {
            const int st = s % kC1Stages;
            if (!tc::mbar_wait_bounded(&full[st], (s / kC1Stages) & 1)) {
                atomicOr(&s_fail, 1);
                break;
            }
            tc::fence_after_sync();
            const uint32_t sa = base + st * kC1Stage;
            tc::mma_bf16(tmem, desc_sw32(sa), desc_sw32(sa + kC1Tile), idesc, s > 0);
            tc::mma_commit(&empty[st]);
        }
        s_consumed = s;
        if (s == 9) tc::mma_commit(&done);
    }
    __syncwarp();
    if (!tc::mbar_wait_bounded(&done, 0)) atomicOr(&s_fail, 1);
    __syncthreads();
    tc::fence_after_sync();

    if (!s_fail) {
        const int p = m0 + warp * 32 + lane;
        uint16_t *orow = out + (size_t)p * 128;
#pragma unroll 1
        for (int c0 = 0; c0 < 128; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            uint32_t pk[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                pk[j] = pack2(fmaxf(v[2 * j] + s_bias[c0 + 2 * j], 0.0f),
                              fmaxf(v[2 * j + 1] + s_bias[c0 + 2 * j + 1], 0.0f));
            uint4 *o = reinterpret_cast<uint4 *>(orow + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        }
    } else if (tid == 0) {
        atomicOr(err, 1u);
        for (int s = s_consumed; s < s_issued; ++s)
            tc::mbar_wait_bounded(&full[s % kC1Stages], (s / kC1Stages) & 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// --- host: tensor maps ------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// NHWC activations [n][S][S][128] BF16; box 64 channels x `pix` pixels
// (a run of one row, or whole rows when S < pix).
bool map_act(CUtensorMap *m, const uint16_t *ptr, int n, int S, int pix = 128)
{
    auto fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[4] = {128, (cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)n};
    const cuuint64_t strides[3] = {256, (cuuint64_t)S * 256, (cuuint64_t)S * S * 256};
    const cuuint32_t bx = S >= pix ? pix : S, by = pix / bx;
    const cuuint32_t box[4] = {64, bx, by, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(ptr), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// First-layer input [n][S][S][16] BF16; box 16 channels x 128 pixels.
bool map_in16(CUtensorMap *m, const uint16_t *ptr, int n, int S)
{
    auto fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[4] = {16, (cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)n};
    const cuuint64_t strides[3] = {32, (cuuint64_t)S * 32, (cuuint64_t)S * S * 32};
    const cuuint32_t bx = S >= 128 ? 128 : S, by = 128 / bx;
    const cuuint32_t box[4] = {16, bx, by, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t *>(ptr), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// First-layer weights [128 rows][144] BF16; box 16 x 128.
bool map_w144(CUtensorMap *m, const uint16_t *ptr)
{
    auto fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {144, 128};
    const cuuint64_t strides[1] = {144 * 2};
    const cuuint32_t box[2] = {16, 128};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(ptr), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Weights [128 rows][1152] BF16; box 64 x 128.
bool map_wts(CUtensorMap *m, const uint16_t *ptr)
{
    auto fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {1152, 128};
    const cuuint64_t strides[1] = {1152 * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(ptr), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace convtma

// Forward (mode 0: out = ReLU(conv(in) + bias)) or input gradient (mode 1:
// out = conv^T(in) masked by hprev > 0) of a 128 -> 128 layer over n samples
// of S x S (S a power of two >= 16).  `w` is W[o][t][i] (forward) or
// Wt[i][t][o] (input gradient), 16-byte aligned.
cudaError_t launch_conv_tma(int mode, const uint16_t *in, const uint16_t *w,
                            const float *bias, const uint16_t *hprev, uint16_t *out,
                            int n, int S, int lgS, int d, uint32_t *err,
                            cudaStream_t st)
{
    using namespace convtma;
    if (S < 16 || (S & (S - 1)) || ((uintptr_t)in & 15) || ((uintptr_t)w & 15))
        return cudaErrorInvalidValue;
    CUtensorMap ma, mw;
    if (!map_act(&ma, in, n, S) || !map_wts(&mw, w)) return cudaErrorInvalidValue;
    Epi e{mode, bias, hprev, out};
    const long long P = (long long)n * S * S;
    const int ntiles = (int)(P / 128);
#if FIRE_CONV_PERSISTENT
    int dev = 0, nsm = 0;
    cudaError_t attr = cudaGetDevice(&dev);
    if (attr == cudaSuccess)
        attr = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (attr == cudaSuccess)
        attr = cudaFuncSetAttribute(k_conv_tma_p,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem);
    if (attr != cudaSuccess) return attr;
    const int grid = std::min(ntiles, 2 * nsm);
    k_conv_tma_p<<<grid, kPThreads, kPSmem, st>>>(ma, mw, e, S, lgS, d,
                                                  mode == 0 ? 1 : -1, ntiles, err);
#else
    cudaError_t attr = cudaFuncSetAttribute(
        k_conv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (attr != cudaSuccess) return attr;
    k_conv_tma<<<(unsigned)ntiles, 128, kSmem, st>>>(ma, mw, e, S, lgS, d,
                                                     mode == 0 ? 1 : -1, err);
#endif
    return cudaGetLastError();
}

// CTAs of the weight-gradient kernel resident per SM.
int wgrad_ctas_per_sm() { return convtma::kWCtasPerSm; }

// Weight gradient of a 128 -> 128 layer, added into dw[128][1152] (FP32,
// cleared by the caller): dz and in are [n][S][S][128] BF16, S a power of two
// >= 16; the pixel range is split `split` ways.
cudaError_t launch_wgrad_tma(const uint16_t *dz, const uint16_t *in, float *dw, int n,
                             int S, int lgS, int d, int split, uint32_t *err,
                             cudaStream_t st)
{
    using namespace convtma;
    if (S < 16 || (S & (S - 1)) || ((uintptr_t)dz & 15) || ((uintptr_t)in & 15) ||
        ((uintptr_t)dw & 15) || split < 1)
        return cudaErrorInvalidValue;
    CUtensorMap mz, mi;
    if (!map_act(&mz, dz, n, S, 64) || !map_act(&mi, in, n, S, 64))
        return cudaErrorInvalidValue;
    cudaError_t attr = cudaFuncSetAttribute(
        k_wgrad_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem);
    if (attr != cudaSuccess) return attr;
    const int total = (int)((long long)n * S * S / 64);
    if (split > total) split = total;
    const int per = (total + split - 1) / split;
    dim3 grid(1, 9, (total + per - 1) / per);
    k_wgrad_tma<<<grid, 128, kWSmem, st>>>(mz, mi, dw, S, lgS, d, total, per, err);
    return cudaGetLastError();
}

// First layer forward: out = ReLU(conv3x3(x, W1) + b1) for x [n][S][S][16]
// and W1 [128][9][16] (BF16, 16-byte aligned), S a power of two >= 16.
cudaError_t launch_conv1_tma(const uint16_t *x, const uint16_t *w, const float *bias,
                             uint16_t *out, int n, int S, int lgS, uint32_t *err,
                             cudaStream_t st)
{
    using namespace convtma;
    if (S < 16 || (S & (S - 1)) || ((uintptr_t)x & 15) || ((uintptr_t)w & 15))
        return cudaErrorInvalidValue;
    CUtensorMap ma, mw;
    if (!map_in16(&ma, x, n, S) || !map_w144(&mw, w)) return cudaErrorInvalidValue;
    cudaError_t attr = cudaFuncSetAttribute(
        k_conv1_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kC1Smem);
    if (attr != cudaSuccess) return attr;
    const long long P = (long long)n * S * S;
    k_conv1_tma<<<(unsigned)(P / 128), 128, kC1Smem, st>>>(ma, mw, bias, out, S, lgS,
                                                           err);
    return cudaGetLastError();
}

}  // namespace fire

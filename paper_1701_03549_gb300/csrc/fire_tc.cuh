// Blackwell (sm_100 family) tensor-core building blocks for the surrogate
// network: tcgen05 MMA with FP32 accumulators in tensor memory (TMEM),
// operands in shared memory in the canonical no-swizzle K-major layout.
//
// Shared-memory operand layout (both A and B, K-major, 16-bit elements): the
// tile of R rows x BK columns is stored as core matrices of 8 rows x 8
// elements (8 x 16 bytes, rows contiguous); core matrix (row group g,
// column group c) starts at byte g * SBO + c * LBO with LBO = 128 and
// SBO = (BK / 8) * 128.  One MMA consumes 16 columns, i.e. two core-matrix
// columns; its descriptor starts at the tile base + (k / 8) * 128.
//
// Descriptors (PTX ISA, tcgen05 shared-memory and instruction descriptors):
//   smem: [13:0] start >> 4, [29:16] LBO >> 4, [45:32] SBO >> 4,
//         [48:46] = 0b001, [51:49] base offset 0, [52] LBO mode 0,
//         [63:61] swizzle 0 (none);
//   instr (kind::f16): [5:4] D format (1 = F32), [9:7] A format (1 = BF16),
//         [12:10] B format (1 = BF16), [15]/[16] A/B major (0 = K-major),
//         [22:17] N >> 3, [28:24] M >> 4.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fire {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo,
                                              uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3ffffu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: BF16 x BF16 -> F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::
            "r"(smem_addr(dst_smem)),
        "r"(ncols)
        : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::
                     : "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     taddr),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc,
                                         uint64_t bdesc, uint32_t idesc,
                                         bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(void *mbar_smem)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster."
        "b64 [%0];" ::"r"(smem_addr(mbar_smem))
        : "memory");
}

__device__ __forceinline__ void mbar_init(void *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(count)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(void *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (about a second of clocks); false when it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(void *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

// 32 lanes x 16 consecutive 32-bit columns: thread t of the warp receives
// lane (base lane + t), columns [col, col + 16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
          "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
          "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 consecutive 32-bit columns (as tmem_ld16, twice as wide).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
          "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
          "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major operand tile of width BK.
__device__ __forceinline__ uint32_t tile_offset(int row, int k, int BK)
{
    return (uint32_t)((row >> 3) * (BK / 8) * 128 + (k >> 3) * 128 +
                      (row & 7) * 16 + (k & 7) * 2);
}


// ---------------------------------------------------------------------------
// Generic 128 x BN tile GEMM over a K range, D[m][n] = sum_k A(m, k) B(n, k).
//
// Prob supplies the operands and the epilogue:
//   int M, N, K                  (K a multiple of 64, padded with zeros)
//   static constexpr bool kAMn   A staged MN-major (8 consecutive m at one k)
//   static constexpr bool kBMn   likewise for B
//   uint4 a_chunk(m, k) const    K-major: A(m, k..k+7); MN-major: A(m..m+7, k)
//   uint4 b_chunk(n, k) const    likewise; rows m >= M / n >= N are never asked
//   void epilogue(m, n0, v[16])  columns n0..n0+15 of row m (m < M; the
//                                problem checks n < N itself)
//
// Chunk c of a stage (16 bytes) lives at byte c * 16 of its operand tile.
// K-major: row = (c & 7) + 8 (c >> 6), k = 8 ((c >> 3) & 7), which is the
// core-matrix layout above with LBO = 128, SBO = 1024.  MN-major: the 8 rows
// of a core matrix are 8 consecutive k (16 bytes each = 8 consecutive m), so
// m = 8 (c >> 6), k = c & 63, again with the k-groups 128 bytes apart and the
// m-groups 1024 bytes apart; both kinds use the same descriptors and differ
// only in the instruction descriptor's transpose bits.
//
// Two smem stages: the loads of slab s + 1 overlap the MMAs of slab s; a
// stage is refilled only after the mbarrier its MMAs committed to has fired.
constexpr int kTcBK = 64;

template <int BN> struct TcShape {
    static constexpr int kAStage = 128 * kTcBK * 2;
    static constexpr int kBStage = BN * kTcBK * 2;
    static constexpr int kStage = kAStage + kBStage;
    static constexpr int kSmem = 2 * kStage;
    // tensor-memory columns: a power of two >= 32 holding BN
    static constexpr int kCols =
        BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    static_assert(BN % 16 == 0 && BN <= 256, "MMA N: a multiple of 16, at most 256");
};

__device__ __forceinline__ void st_shared16(uint32_t saddr, uint4 v)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(saddr),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ uint4 ld_global16(const void *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

template <int BN, class Prob>
__global__ void __launch_bounds__(128) k_tc_tile(const Prob pr, int k_chunk,
                                                 uint32_t *err)
{
    using S = TcShape<BN>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * k_chunk;
    const int ke = min(pr.K, kb + k_chunk);
    const int nslab = ke > kb ? (ke - kb) / kTcBK : 0;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, S::kCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = idesc_bf16(128, BN) |
                               (Prob::kAMn ? 1u << 15 : 0u) |
                               (Prob::kBMn ? 1u << 16 : 0u);
    const uint32_t sbase = smem_addr(smem);

    for (int s = 0; s < nslab; ++s) {
        const int b = s & 1;
        if (s >= 2 && !mbar_wait_bounded(&mbar[b], ((s - 2) >> 1) & 1))
            atomicOr(&s_fail, 1);
        const uint32_t sa = sbase + b * S::kStage, sb = sa + S::kAStage;
        const int k0 = kb + s * kTcBK;
#pragma unroll 2
        for (int c = tid; c < 128 * 8; c += 128) {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (Prob::kAMn) {
                const int m = m0 + ((c >> 6) << 3);
                if (m < pr.M) v = pr.a_chunk(m, k0 + (c & 63));
            } else {
                const int m = m0 + (c & 7) + ((c >> 6) << 3);
                if (m < pr.M) v = pr.a_chunk(m, k0 + (((c >> 3) & 7) << 3));
            }
            st_shared16(sa + c * 16, v);
        }
#pragma unroll 2
        for (int c = tid; c < BN * 8; c += 128) {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (Prob::kBMn) {
                const int n = n0 + ((c >> 6) << 3);
                if (n < pr.N) v = pr.b_chunk(n, k0 + (c & 63));
            } else {
                const int n = n0 + (c & 7) + ((c >> 6) << 3);
                if (n < pr.N) v = pr.b_chunk(n, k0 + (((c >> 3) & 7) << 3));
            }
            st_shared16(sb + c * 16, v);
        }
        fence_proxy_async();
        __syncthreads();
        if (s_fail) break;
        if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kTcBK; kk += 16) {
                const uint64_t ad = smem_desc(sa + (kk / 8) * 128, 128, 1024);
                const uint64_t bd = smem_desc(sb + (kk / 8) * 128, 128, 1024);
                mma_bf16(tmem, ad, bd, idesc, s > 0 || kk > 0);
            }
            mma_commit(&mbar[b]);
        }
    }
    if (nslab > 0 && !s_fail &&
        !mbar_wait_bounded(&mbar[(nslab - 1) & 1], ((nslab - 1) >> 1) & 1))
        atomicOr(&s_fail, 1);
    __syncthreads();
    fence_after_sync();

    if (!s_fail && nslab > 0) {
        const int m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (m < pr.M && n0 + c0 < pr.N) pr.epilogue(m, n0 + c0, v);
        }
    }
    if (s_fail && tid == 0) atomicOr(err, 1u);
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, S::kCols);
}

// Launch over an M x N output with the K range split ksplit ways (each split
// a whole number of 64-wide slabs).  The caller picks BN.
template <int BN, class Prob>
cudaError_t launch_tc_tile(const Prob &pr, int ksplit, uint32_t *err,
                           cudaStream_t st)
{
    using S = TcShape<BN>;
    if (pr.K % kTcBK || pr.M <= 0 || pr.N <= 0 || ksplit < 1)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(
        k_tc_tile<BN, Prob>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        S::kSmem);
    if (e != cudaSuccess) return e;
    const int kslabs = pr.K / kTcBK;
    const int per = (kslabs + ksplit - 1) / ksplit;
    dim3 grid((pr.M + 127) / 128, (pr.N + BN - 1) / BN,
              (kslabs + per - 1) / per);
    k_tc_tile<BN, Prob><<<grid, 128, S::kSmem, st>>>(pr, per * kTcBK, err);
    return cudaGetLastError();
}

}  // namespace tc
}  // namespace fire

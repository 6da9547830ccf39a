// Plain tensor-core GEMM on the generic tcgen05 tile (fire_tc.cuh), exposed
// as fire_tc_gemm: C[M x N] (FP32) = A B^T with BF16 operands given K-major
// (A[m][k], B[n][k]) or MN-major (A[k][m], B[k][n]).  It carries no part of
// the paper's method; the surrogate's convolutions use the same tile with
// gathering loaders (fire_surrogate.cu) and this entry point lets tests check
// the tile, its descriptors and its split-K path on their own.
#include "fire_internal.h"
#include "fire_tc.cuh"

using namespace fire;

namespace {

template <bool AMn, bool BMn> struct GemmProb {
    static constexpr bool kAMn = AMn, kBMn = BMn;
    const uint16_t *A, *B;
    float *C;
    int M, N, K, atomic;

    __device__ uint4 a_chunk(int m, int k) const
    {
        return tc::ld_global16(AMn ? A + (size_t)k * M + m : A + (size_t)m * K + k);
    }
    __device__ uint4 b_chunk(int n, int k) const
    {
        return tc::ld_global16(BMn ? B + (size_t)k * N + n : B + (size_t)n * K + k);
    }
    __device__ void epilogue(int m, int n0, const float v[16]) const
    {
        float *row = C + (size_t)m * N;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (n0 + j >= N) break;
            if (atomic)
                atomicAdd(row + n0 + j, v[j]);
            else
                row[n0 + j] = v[j];
        }
    }
};

template <bool AMn, bool BMn>
cudaError_t gemm_launch(const uint16_t *A, const uint16_t *B, float *C, int M,
                        int N, int K, int ksplit, uint32_t *err, cudaStream_t st)
{
    GemmProb<AMn, BMn> p{A, B, C, M, N, K, ksplit > 1};
    if (N <= 16) return tc::launch_tc_tile<16>(p, ksplit, err, st);
    if (N <= 32) return tc::launch_tc_tile<32>(p, ksplit, err, st);
    if (N <= 64) return tc::launch_tc_tile<64>(p, ksplit, err, st);
    return tc::launch_tc_tile<128>(p, ksplit, err, st);
}

// One thread waits, with the bounded wait that every TMA and tensor-core
// pipeline of the library uses, for the first phase of an mbarrier that
// nothing arrives at.  The wait gives up after 2^31 SM clocks and the error
// word is set, as when a copy or an MMA never completes; `gave_up` records
// that the wait ran out rather than completed.
__global__ void k_wait_selftest(uint32_t *err, uint32_t *gave_up)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    if (!tc::mbar_wait_bounded(&bar, 0)) {
        atomicOr(err, 1u);
        *gave_up = 1u;
    }
}

}  // namespace

extern "C" int fire_tc_gemm(fire_ctx *ctx, int M, int N, int K,
                            const uint16_t *A, const uint16_t *B, int ksplit,
                            uint32_t flags, float *C)
{
    FIRE_NVTX("fire_tc_gemm");
    if (!ctx) return FIRE_EINVAL;
    const bool amn = flags & FIRE_TC_A_MN, bmn = flags & FIRE_TC_B_MN;
    if (!(flags & FIRE_DEVICE_PTRS) || !A || !B || !C || M <= 0 || N <= 0 ||
        K <= 0 || K % 64 || ksplit < 1 || (amn && M % 8) || (bmn && N % 8) ||
        ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
        return set_err(ctx, FIRE_EINVAL, "bad fire_tc_gemm arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    if (ksplit > 1)
        CUDA_TRY(ctx, cudaMemsetAsync(C, 0, (size_t)M * N * 4, ctx->stream),
                 "split-K clear");
    uint32_t *err = ctx->counter + 1;
    cudaError_t e;
    if (amn)
        e = bmn ? gemm_launch<true, true>(A, B, C, M, N, K, ksplit, err, ctx->stream)
                : gemm_launch<true, false>(A, B, C, M, N, K, ksplit, err, ctx->stream);
    else
        e = bmn ? gemm_launch<false, true>(A, B, C, M, N, K, ksplit, err, ctx->stream)
                : gemm_launch<false, false>(A, B, C, M, N, K, ksplit, err, ctx->stream);
    CUDA_TRY(ctx, e, "tc gemm");
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

extern "C" int fire_wait_selftest(fire_ctx *ctx)
{
    if (!ctx) return FIRE_EINVAL;
    int rc = ensure_device(ctx);
    if (rc) return rc;
    // a clean error word first, so that only this wait can set it
    rc = fire_sync(ctx);
    if (rc) return rc;
    uint32_t *gave_up = ctx->counter + 2;
    CUDA_TRY(ctx, cudaMemsetAsync(gave_up, 0, 4, ctx->stream), "self-test flag");
    k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->counter + 1, gave_up);
    CUDA_TRY(ctx, cudaGetLastError(), "wait self-test");
    uint32_t flag = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&flag, gave_up, 4, cudaMemcpyDeviceToHost,
                                  ctx->stream), "self-test flag");
    rc = fire_sync(ctx);   // FIRE_ETIMEOUT, clearing the error word
    if (rc == FIRE_ETIMEOUT && flag != 1u)
        return set_err(ctx, FIRE_ECUDA, "error word set without the wait");
    return rc;
}

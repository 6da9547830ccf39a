// Test-only reference: Philox4x32-10 blocks from cuRAND's public raw block
// function (curand_Philox4x32_10), to pin the library's and the oracle's
// independent implementations of the generator (Salmon et al., SC'11) to a
// third-party one.  Built and loaded by tests/test_gpu_parity.py only.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_philox4x32_x.h>

namespace {

__global__ void k_ref(int n, const uint4 *ctr, const uint2 *key, uint4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

}  // namespace

// out[4 i .. 4 i + 3] = block of counter ctr[4 i .. 4 i + 3] under key
// key[2 i .. 2 i + 1], i < n (host arrays).  Returns 0 or a cudaError_t.
extern "C" int curand_philox_blocks(int n, const uint32_t *ctr,
                                    const uint32_t *key, uint32_t *out)
{
    if (n <= 0) return 0;
    uint4 *dc = nullptr, *dout = nullptr;
    uint2 *dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, (size_t)n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&dk, (size_t)n * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)n * sizeof(uint4));
    if (e == cudaSuccess)
        e = cudaMemcpy(dc, ctr, (size_t)n * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dk, key, (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_ref<<<(n + 127) / 128, 128>>>(n, dc, dk, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(out, dout, (size_t)n * 16, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return (int)e;
}

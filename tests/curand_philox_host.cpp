// Test-only reference on the CPU: Philox4x32-10 blocks from cuRAND's public
// raw block function (curand_Philox4x32_10), compiled for the host through
// the header's own host code path, to pin the oracle's generator (Salmon et
// al., SC'11) to a third-party implementation without a GPU.  Built and
// loaded by tests/test_oracle_rng_math.py only.
#define QUALIFIERS static inline
#include <cstdint>
#include <vector_types.h>
#include <vector_functions.h>
#include <curand_philox4x32_x.h>

// out[4 i .. 4 i + 3] = block of counter ctr[4 i .. 4 i + 3] under key
// key[2 i .. 2 i + 1], i < n.
extern "C" void curand_philox_blocks_host(int n, const uint32_t *ctr,
                                          const uint32_t *key, uint32_t *out)
{
    for (int i = 0; i < n; ++i) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2],
                                   ctr[4 * i + 3]);
        const uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
        const uint4 o = curand_Philox4x32_10(c, k);
        out[4 * i] = o.x;
        out[4 * i + 1] = o.y;
        out[4 * i + 2] = o.z;
        out[4 * i + 3] = o.w;
    }
}

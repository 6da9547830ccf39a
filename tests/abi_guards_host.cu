// Host-side argument guards of the simulation entry points, exercised
// without a GPU: contexts and maps are built in host memory with the
// library's own definitions, so each call must be refused before it issues
// any CUDA call (a CUDA call would fail on a machine without a device and
// return FIRE_ECUDA instead of FIRE_EINVAL).
#include <cstdio>
#include <cstring>

#include "fire_internal.h"

extern "C" int abi_guard_cases(char *msg, int len)
{
    fire_ctx ctx0, ctx1;
    ctx0.device = 0;
    ctx1.device = 1;
    fire_map m;
    m.ctx = &ctx1;   // uploaded through a context on device 1
    m.feat = reinterpret_cast<float4 *>(256);
    fire_params *p = reinterpret_cast<fire_params *>(256);
    fire_cell *g = reinterpret_cast<fire_cell *>(256);
    uint64_t *s = reinterpret_cast<uint64_t *>(256);
    fire_result *o = reinterpret_cast<fire_result *>(256);
    auto fail = [&](int k, int rc) {
        snprintf(msg, len, "case %d: rc %d: %s", k, rc, ctx0.err.c_str());
        return k;
    };
    int rc;
    // 1. a map of another device, no-alloc entry point
    rc = fire_simulate_batch_noalloc(&ctx0, &m, 1, p, g, s, 0,
                                     FIRE_DEVICE_PTRS, o, nullptr);
    if (rc != FIRE_EINVAL || !strstr(ctx0.err.c_str(), "another device"))
        return fail(1, rc);
    // 2. the same through fire_simulate_batch (device pointers)
    rc = fire_simulate_batch(&ctx0, &m, 1, p, g, s, 0, FIRE_DEVICE_PTRS, o,
                             nullptr);
    if (rc != FIRE_EINVAL || !strstr(ctx0.err.c_str(), "device 1"))
        return fail(2, rc);
    // 3-4. flags the no-alloc entry point does not honour
    m.ctx = &ctx0;
    const uint32_t bad[2] = {FIRE_LONGEST_FIRST, FIRE_GRAPH};
    for (int k = 0; k < 2; ++k) {
        rc = fire_simulate_batch_noalloc(&ctx0, &m, 1, p, g, s, 0,
                                         FIRE_DEVICE_PTRS | bad[k], o, nullptr);
        if (rc != FIRE_EINVAL || !strstr(ctx0.err.c_str(), "flag"))
            return fail(3 + k, rc);
    }
    // 5. a map without an owning context
    m.ctx = nullptr;
    rc = fire_simulate_batch_noalloc(&ctx0, &m, 1, p, g, s, 0, FIRE_DEVICE_PTRS,
                                     o, nullptr);
    if (rc != FIRE_EINVAL) return fail(5, rc);
    m.ctx = nullptr;
    snprintf(msg, len, "ok");
    return 0;
}

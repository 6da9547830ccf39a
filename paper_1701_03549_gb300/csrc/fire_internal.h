// Internal declarations shared by the C ABI (fire_api.cu) and the kernels
// (fire_kernels.cu).  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fire.h"
#include "fire_device.cuh"

namespace fire {

// Device-resident landscape.  Covariates are row-major per cell; the
// non-burnable and target bitmaps are tile-major: tile (ti, tj) of the
// ceil(H/32) x ceil(W/32) tiling owns 32 consecutive words, word r holding
// row 32 ti + r, bit i holding column 32 tj + i.  Cells of a tile that lie
// outside the grid are marked non-burnable and not in the target.
struct MapDev {
    int H, W, TH, TW, ntiles;
    const float4 *feat;         // (psi, sig, cos wind, sin wind) per cell
    const uint16_t *cfl;        // bit d<8 uphill from source d, 8 forest, 9 burnable
    const uint32_t *blk;        // non-burnable bitmap, ntiles * 32 words
    const uint32_t *tgt;        // target bitmap, ntiles * 32 words
    const uint32_t *tgt_count;  // |A|, one word
};

struct SimLaunch {
    MapDev map;
    int n;
    const fire_params *params;
    const fire_cell *ign;
    const uint64_t *seeds;
    fire_result *out;
    int32_t *burn_step;        // nullable
    uint32_t *work_counter;    // zeroed before launch
    uint32_t *gstate;          // global-state variant: 2 * ntiles * 32 words per block
    uint32_t *error_word;      // set nonzero when a bounded wait runs out
    uint32_t max_steps;        // 0 = no cap
    int qcap;                  // candidate-queue capacity (entries)
};

// Cell-flag bits.
constexpr uint16_t kFlagForest = 1u << 8;
constexpr uint16_t kFlagBurnable = 1u << 9;

// Per-simulation shared state of the simulation kernel's block.
struct SimShared {
    double beta[5];
    ScreenParams sp;
    uint32_t key0, key1;
    int sim;
    int skip;
    int timeout;
    uint32_t count[3];    // worklist lengths, slot t % 3 for step t
    uint32_t newflag[3];  // some cell burning at step t (slot t % 3)
    uint32_t qcount[2];   // candidate-queue reservations of step t (t & 1)
    uint32_t qvalid[2];   // end of the valid queue prefix of step t (t & 1)
    uint32_t trials, status, last_new;
    uint32_t burnt, inter;
    unsigned long long tw_magic;  // floor(2^40 / TW) + 1: k / TW = k * m >> 40
    unsigned long long mbar;
};

// Shared-memory layout of the simulation kernel (identical on host/device):
// header, worklist mark bits (2 per tile), three worklists of uint16 tile
// indices, the block's candidate queue (qcap uint32 entries), then, in the
// shared-state variant, the X and Y planes.
struct SimLayout {
    size_t header, marks, lists, queue, planes, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a)
{
    return (x + a - 1) / a * a;
}

__host__ __device__ inline SimLayout sim_layout(int ntiles, int qcap,
                                                bool smem_state)
{
    SimLayout L;
    L.header = 0;
    L.marks = align_up(sizeof(SimShared), 16);
    L.lists = align_up(L.marks + 4 * (size_t)((ntiles + 15) / 16), 16);
    L.queue = align_up(L.lists + 3 * 2 * (size_t)ntiles, 16);
    L.planes = align_up(L.queue + 4 * (size_t)qcap, 128);
    L.total = smem_state ? L.planes + 2 * (size_t)ntiles * 128 : L.planes;
    return L;
}

// Launchers (fire_kernels.cu).  All are asynchronous on `st`.
cudaError_t launch_features(int H, int W, const uint8_t *veg, const float *elev,
                            const float *slope, const float *aspect,
                            const float *wind, float4 *feat, uint16_t *cfl,
                            cudaStream_t st);
cudaError_t launch_blocked(const MapDev &m, const uint8_t *veg, uint32_t *blk,
                           cudaStream_t st);
cudaError_t launch_target(const MapDev &m, const uint8_t *burnt, uint32_t *tgt,
                          uint32_t *tgt_count, cudaStream_t st);
cudaError_t launch_simulate(const SimLaunch &a, bool smem_state, int nwarps,
                            int grid, size_t smem_bytes, cudaStream_t st);
// Threads per block the simulation kernel is compiled for (upper bound).
constexpr int kSimMaxThreads = 512;
const void *simulate_kernel_ptr(bool smem_state);
cudaError_t launch_fitness(const fire_result *r, int n, int kind, double *out,
                           cudaStream_t st);
cudaError_t launch_thresholds(const MapDev &m, const double *beta_dev,
                              int64_t *out, cudaStream_t st);
cudaError_t launch_probabilities(const MapDev &m, const double *beta_dev,
                                 float *p32, double *p64, cudaStream_t st);
cudaError_t launch_features_export(const MapDev &m, float *psi, float *sig,
                                   float *cw, float *sw, uint16_t *cfl,
                                   cudaStream_t st);
cudaError_t launch_screen_selftest(uint64_t n, uint64_t seed,
                                   unsigned long long *counts,
                                   unsigned long long *max_dp_bits,
                                   cudaStream_t st);
cudaError_t launch_philox_blocks(uint64_t n, uint4 ctr, uint2 key,
                                 uint32_t *out, cudaStream_t st);

}  // namespace fire

// Opaque handles of the C ABI (definitions shared by the host sources).
struct fire_ctx {
    int device = 0;
    int num_sms = 0;
    size_t max_smem_optin = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int warps_per_block = 0;   // 0: heuristic
    int blocks_per_sm = 0;     // 0: as many as fit
    std::string err;
    // device scratch
    uint32_t *counter = nullptr;     // work counter + error word
    void *staging = nullptr;         // inputs / outputs of host-pointer calls
    size_t staging_bytes = 0;
    uint32_t *gstate = nullptr;      // global-state simulation buffers
    size_t gstate_bytes = 0;
    void *host_pinned = nullptr;     // pinned bounce buffer
    size_t host_pinned_bytes = 0;
};

struct fire_map {
    fire_ctx *ctx = nullptr;
    fire::MapDev dev{};
    float cell_m = 0.f;
    float4 *feat = nullptr;
    uint16_t *cfl = nullptr;
    uint32_t *blk = nullptr;
    uint32_t *tgt = nullptr;
    uint32_t *tgt_count = nullptr;
    std::vector<uint8_t> burnable_host;
};


// Internal declarations shared by the C ABI (fire_api.cu) and the kernels
// (fire_kernels.cu).  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

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
    const float2 *wdiag;        // cos(wind - 45 deg), cos(wind - 135 deg) per cell
    const float2 *ps;           // (psi, sig) per cell
    // A wind raster of one value everywhere (bit for bit) has the same four
    // wind terms in every cell: the simulation then reads them from here and
    // only (psi, sig) per cell (10 bytes with the flags instead of 26).
    int uniform_wind;
    float cw, sw, om1, om3;
    const uint16_t *cfl;        // bit d<8 uphill from source d, 8 forest, 9 burnable
    const uint32_t *blk;        // non-burnable bitmap, ntiles * 32 words
    const uint32_t *tgt;        // target bitmap, ntiles * 32 words
    const uint32_t *tgt_count;  // |A|, one word
};

struct SimLaunch {
    MapDev map;                // the map when `maps` is NULL
    const MapDev *maps;        // device map table (multi-map launches)
    int nmaps;
    const int32_t *map_of_sim; // map index per simulation (NULL: map 0)
    const uint32_t *order;     // processing order of the simulations (NULL: 0..n-1)
    int ntiles_max;            // largest map of the launch (sizes buffers)
    int n;
    const fire_params *params;
    const fire_cell *ign;
    const uint64_t *seeds;
    fire_result *out;
    int32_t *burn_step;        // nullable
    uint32_t *burnt_bits;      // nullable; single-map launches only: the final
                               // burnt words (tile-major, blocked cells
                               // cleared), ntiles * 32 words per simulation
    uint32_t *work_counter;    // zeroed before launch
    uint32_t *gstate;          // global-state variant: block_words words per block
    size_t block_words;        // 0: 2 * ntiles_max * 32 (the X, Y planes)
    const uint8_t *burn_time;  // burn-time variant: steps each cell burns
                               // (1..250, others clamped); its blocks keep X, Y,
                               // two "still burning" planes and one fuel byte
                               // per cell in their global state
    const uint32_t *long_burn; // burn-time variant: tile-major bit plane of the
                               // cells that burn 2 steps or more (only these
                               // keep a fuel count)
    uint32_t *error_word;      // set nonzero when a bounded wait runs out
    uint32_t max_steps;        // 0 = no cap
    int qcap;                  // candidate-queue capacity (entries)
    int cell_uniform;          // 1: one uniform per target cell (Sec. 2.3)
};

// Largest batch ordered longest-first (the ranking is quadratic in n).
constexpr int kLongestFirstMax = 8192;

// Cell-flag bits.
constexpr uint16_t kFlagForest = 1u << 8;
constexpr uint16_t kFlagBurnable = 1u << 9;

// Per-simulation shared state of the simulation kernel's block.
struct SimShared {
    uint4 rk[5];          // Philox round keys: (k0, k1) of round 2j, then 2j + 1
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
    uint32_t hard_cap;
    int nmark;
    // floor((2^32 - 1) / TW): k / TW = (k + 1) m >> 32 for every tile index
    // k < FIRE_MAX_TILES and TW <= FIRE_MAX_TILES (checked exhaustively)
    uint32_t tw_magic;
    MapDev map;                   // map of the current simulation
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
                            const float *wind, float4 *feat, float2 *wdiag,
                            float2 *ps, uint16_t *cfl, uint32_t *wind_varies,
                            cudaStream_t st);
cudaError_t launch_blocked(const MapDev &m, const uint8_t *veg, uint32_t *blk,
                           cudaStream_t st);
cudaError_t launch_target(const MapDev &m, const uint8_t *burnt, uint32_t *tgt,
                          uint32_t *tgt_count, cudaStream_t st);
cudaError_t launch_simulate(const SimLaunch &a, bool smem_state, int nwarps,
                            int grid, size_t smem_bytes, cudaStream_t st);
// The burn-time variant (global-memory state only).
cudaError_t launch_simulate_burn(const SimLaunch &a, int nwarps, int grid,
                                 size_t smem_bytes, cudaStream_t st);
// Tile-major bit plane of the cells whose burn time is 2 or more, and a flag
// set when there is any (zeroed by the launcher).
cudaError_t launch_long_burn(const MapDev &m, const uint8_t *burn_time,
                             uint32_t *plane, uint32_t *any, cudaStream_t st);
// Words of one block's global state in the burn-time variant.
inline size_t burn_block_words(int ntiles, long long HW)
{
    return 4 * (size_t)ntiles * 32 + (size_t)((HW + 15) / 16) * 4;
}
// Threads per block the simulation kernel is compiled for (upper bound).
constexpr int kSimMaxThreads = 512;
const void *simulate_kernel_ptr(bool smem_state);
const void *simulate_burn_kernel_ptr();
cudaError_t launch_longest_first(const MapDev &m, int n, const fire_params *params,
                                 float *key, uint32_t *order, cudaStream_t st);
cudaError_t launch_fitness(const fire_result *r, int n, int kind, double *out,
                           cudaStream_t st);
// Counting sort of simulations by rank[map_of_sim[i]] (counts: nmaps + 1).
cudaError_t launch_order(int n, const int32_t *map_of_sim, int nmaps,
                         const int32_t *rank, uint32_t *counts, uint32_t *order,
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

struct LaunchPlan {
    int nwarps, qcap;
    bool smem_state;
    SimLayout L;
    int grid;
};

}  // namespace fire

// Launch-shape record of the autotuner (per map tile count).
struct TuneEntry {
    int ntiles, warps, bps, queue, state;
    float ms;
};

// A captured CUDA graph and the call it replays.
struct GraphEntry {
    std::vector<unsigned long long> key;
    cudaGraphExec_t exec;
    unsigned epoch;
};

// Opaque handles of the C ABI (definitions shared by the host sources).
struct fire_ctx {
    int device = 0;
    int num_sms = 0;
    size_t max_smem_optin = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int warps_per_block = 0;   // 0: heuristic
    int blocks_per_sm = 0;     // 0: as many as fit
    int queue_entries = 0;     // 0: default
    int state_mode = 0;        // FIRE_STATE_*
    std::string err;
    // device scratch
    uint32_t *counter = nullptr;     // work counter + error word
    void *staging = nullptr;         // inputs / outputs of host-pointer calls
    size_t staging_bytes = 0;
    uint32_t *gstate = nullptr;      // global-state simulation buffers
    size_t gstate_bytes = 0;
    void *host_pinned = nullptr;     // pinned bounce buffer
    size_t host_pinned_bytes = 0;
    void *table = nullptr;           // map table + map ranks (multi-map calls)
    size_t table_bytes = 0;
    void *order = nullptr;           // bucket counts + processing order
    size_t order_bytes = 0;
    void *lpt = nullptr;             // longest-first keys + order (single map)
    size_t lpt_bytes = 0;
    std::vector<TuneEntry> tuned;    // autotuned launch shapes
    std::vector<GraphEntry> graphs;  // captured calls
    unsigned epoch = 0;              // bumped when a device buffer moves
    int fail_alloc_after = -1;       // test hook: fail that growth (-1: off)
    void *burn_aux = nullptr;        // burn-time calls: long-burn plane + flag
    size_t burn_aux_bytes = 0;
};

struct fire_map {
    fire_ctx *ctx = nullptr;
    fire::MapDev dev{};
    float cell_m = 0.f;
    float4 *feat = nullptr;
    float2 *wdiag = nullptr;
    float2 *ps = nullptr;
    uint16_t *cfl = nullptr;
    uint32_t *blk = nullptr;
    uint32_t *tgt = nullptr;
    uint32_t *tgt_count = nullptr;
    std::vector<uint8_t> burnable_host;
};


namespace fire {
// Host helpers shared by the C ABI sources (fire_api.cu).
int set_err(fire_ctx *ctx, int code, const char *fmt, ...);
int cuda_err(fire_ctx *ctx, cudaError_t e, const char *what);
int ensure_device(fire_ctx *ctx);
int grow_device(fire_ctx *ctx, void **buf, size_t *cap, size_t need,
                const char *what);
size_t round16(size_t x);
bool valid_map(const fire_map *m);
int noalloc_take_error(int device, bool *set);
// Launch shape of the simulation kernel (burn: the burn-time variant, whose
// state is always in global memory).
int plan_launch(fire_ctx *ctx, int ntiles, long long n, LaunchPlan *p,
                bool burn = false);
cudaError_t launch_conv_tma(int mode, const uint16_t *in, const uint16_t *w,
                            const float *bias, const uint16_t *hprev, uint16_t *out,
                            int n, int S, int lgS, int d, uint32_t *err,
                            cudaStream_t st);
cudaError_t launch_conv1_tma(const uint16_t *x, const uint16_t *w, const float *bias,
                             uint16_t *out, int n, int S, int lgS, uint32_t *err,
                             cudaStream_t st);
cudaError_t launch_wgrad_tma(const uint16_t *dz, const uint16_t *in, float *dw, int n,
                             int S, int lgS, int d, int split, uint32_t *err,
                             cudaStream_t st);
int launch_batch(fire_ctx *ctx, const fire_map *m, int n,
                 const fire_params *dparams, const fire_cell *dign,
                 const uint64_t *dseeds, uint32_t max_steps, uint32_t flags,
                 fire_result *dout, int32_t *dsteps, uint32_t *dbits);
}  // namespace fire

// NVTX range named after the C-ABI entry point, open for the call's
// duration (profilers such as Nsight show the library's calls on the host
// timeline; without a tool attached each range costs a no-op call).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};
#define FIRE_NVTX(name) NvtxScope fire_nvtx_scope_(name)

#define CUDA_TRY(ctx, expr, what)                                   \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) return fire::cuda_err(ctx, e_, what); \
    } while (0)

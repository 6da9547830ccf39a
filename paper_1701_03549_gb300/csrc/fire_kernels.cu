// Kernels of libfire: covariate precompute (Sec. 2.1), target packing, the
// batched fire-spread simulation (Sec. 2.1 rules, Eq. 1, Sec. 2.3) with the
// burnt-map comparison of Eq. 2 fused into it, fitness, and debug exports.
//
// Simulation kernel design (one thread block per simulation at a time,
// persistent blocks pulling simulations from a global counter):
//  * State: two bit planes X, Y (one bit per cell each) in 32 x 32-cell tiles,
//    tile-major, in shared memory when they fit (else in a per-block global
//    buffer).  A cell's 2-bit code is 00 burnable and unburnt, 11 burnt or
//    non-burnable, and 10 / 01 burning, the code alternating with the parity
//    of the step at which the cell ignited.  Within step t the sources are the
//    cells coded "burning, parity t"; a tile's owner warp writes new cells
//    with the other parity code and retires the previous step's burning cells
//    to 11, and neither write changes the parity-t burning set that other
//    warps read across tile edges.  Each step has two phases separated by
//    block barriers: the tile scans (phase A) fill the block's candidate
//    queue, the block's threads then decide the queued candidates (phase B).
//  * Frontier: a worklist of active tiles per step (tiles holding burning
//    cells, tiles bordering them across an edge that has burning cells, and
//    tiles whose burning cells must be retired), deduplicated with per-tile
//    mark bits; quiet tiles are never touched.  The fire is extinct when the
//    list is empty.
//  * Per tile (one warp, lane = tile row): eight bit masks of targets with a
//    burning source in each direction, built with shifts across tile edges;
//    the candidates are queued and spread evenly over the warp's lanes; each
//    candidate draws one Philox block per half of its directions (counter =
//    (cell, step, d/4, 0), key = seed) and decides each trial through the
//    single-precision screen, falling back to the exact double-precision
//    threshold only near the decision boundary.
//  * Fused fitness: at extinction a final sweep of the planes popcounts the
//    burnt cells and those also in the target bit plane (|A*| and |A n A*|
//    of Eq. 2) and records whether the fire reached the grid's border.
//  * Draws: every trial of a simulation uses the same Philox key, so the
//    key schedule (ten round keys) is computed once per simulation.
#include <cstdio>

#include "fire_device.cuh"
#include "fire_internal.h"

namespace fire {

namespace {

constexpr unsigned kFull = 0xffffffffu;
__constant__ int kDR[8] = {-1, -1, 0, 1, 1, 1, 0, -1};
__constant__ int kDC[8] = {0, 1, 1, 1, 0, -1, -1, -1};

}  // namespace

// ---------------------------------------------------------------------------
// Covariates of Eq. 1 for every cell (Sec. 2.1): psi = cos(aspect - 315) for
// slopes above 5 degrees, sig = slope / 100, cos and sin of the wind bearing,
// uphill mask per direction (target strictly above the source), forest and
// burnable flags.
__global__ void k_features(int H, int W, const uint8_t *__restrict__ veg,
                           const float *__restrict__ elev,
                           const float *__restrict__ slope,
                           const float *__restrict__ aspect,
                           const float *__restrict__ wind,
                           float4 *__restrict__ feat,
                           float2 *__restrict__ wdiag,
                           float2 *__restrict__ ps,
                           uint16_t *__restrict__ cfl,
                           uint32_t *__restrict__ wind_varies)
{
    const long long n = (long long)H * W;
    const uint32_t wind0 = __float_as_uint(wind[0]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / W), c = (int)(i - (long long)r * W);
        const float sl = slope[i];
        const float psi =
            sl > 5.0f ? __double2float_rn(
                            spec::cosd(spec::sub((double)aspect[i], 315.0)))
                      : 0.0f;
        const float sig = __double2float_rn(__ddiv_rn((double)sl, 100.0));
        const double wd = (double)wind[i];
        const float cw = __double2float_rn(spec::cosd(wd));
        const float sw = __double2float_rn(spec::sind(wd));
        const float e = elev[i];
        uint16_t f = 0;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int sr = r - kDR[d], sc = c - kDC[d];
            if (sr < 0 || sr >= H || sc < 0 || sc >= W) continue;
            if (e > elev[(long long)sr * W + sc]) f |= (uint16_t)(1u << d);
        }
        const uint8_t v = veg[i];
        if (v == 1) f |= kFlagForest;
        if (v != 0) f |= kFlagBurnable;
        feat[i] = make_float4(psi, sig, cw, sw);
        ps[i] = make_float2(psi, sig);
        if (__float_as_uint(wind[i]) != wind0) *wind_varies = 1u;
        wdiag[i] = make_float2(__double2float_rn(spec::omega(cw, sw, 1)),
                               __double2float_rn(spec::omega(cw, sw, 3)));
        cfl[i] = f;
    }
}

// Tile-major bit plane of a per-cell byte map: bit set where pred(byte).
template <bool kTarget>
__global__ void k_pack_bits(int H, int W, int TW, int nwords,
                            const uint8_t *__restrict__ src,
                            uint32_t *__restrict__ dst,
                            uint32_t *__restrict__ count)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t word = 0;
    if (w < nwords) {
        const int k = w >> 5, r = w & 31;
        const int ti = k / TW, tj = k - ti * TW;
        const int R = ti * 32 + r;
        for (int i = 0; i < 32; ++i) {
            const int C = tj * 32 + i;
            const bool in = R < H && C < W;
            bool bit;
            if (kTarget) bit = in && src[(long long)R * W + C] != 0;
            else bit = !in || src[(long long)R * W + C] == 0;
            word |= (uint32_t)bit << i;
        }
        dst[w] = word;
    }
    if (kTarget) {
        uint32_t c = __reduce_add_sync(kFull, w < nwords ? __popc(word) : 0u);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
    }
}

// Tile-major bit plane of the cells that burn two steps or more.
__global__ void k_long_burn(int H, int W, int TW, int nwords,
                            const uint8_t *__restrict__ bt,
                            uint32_t *__restrict__ dst, uint32_t *__restrict__ any)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    const int k = w >> 5, r = w & 31;
    const int ti = k / TW, tj = k - ti * TW;
    const int R = ti * 32 + r;
    uint32_t word = 0;
    for (int i = 0; i < 32; ++i) {
        const int C = tj * 32 + i;
        if (R < H && C < W && bt[(long long)R * W + C] >= 2) word |= 1u << i;
    }
    dst[w] = word;
    if (word) *any = 1u;
}

// ---------------------------------------------------------------------------
// Simulation kernel helpers.

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(n)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar,
                                                      uint32_t bytes)
{
    asm volatile(
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar,
                                              uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bulk (TMA engine) copy global -> shared, completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t burning(uint32_t x, uint32_t y,
                                            uint32_t par)
{
    return par ? (y & ~x) : (x & ~y);
}

struct SimCtx {
    const SimLaunch *a;
    SimShared *sh;
    const MapDev *map;   // the current simulation's map (shared memory)
    uint32_t *marks;
    uint16_t *lists;
    uint32_t *queue;
    uint32_t *X, *Y;
    uint32_t *K0, *K1;   // burn-time variant: cells still burning, by step parity
    uint8_t *fuel;       // burn-time variant: steps of fuel left per cell
    int ntiles;
    int sim;
};

// Steps a cell ignited now will burn (burn-time variant), 1..250.
__device__ __forceinline__ uint8_t burn_steps(const SimLaunch &a, uint32_t cell)
{
    const uint32_t b = __ldg(&a.burn_time[cell]);
    return (uint8_t)(b < 1u ? 1u : (b > 250u ? 250u : b));
}

__device__ __forceinline__ int tile_row(const SimShared &sh, int k)
{
    return (int)__umulhi((uint32_t)k + 1u, sh.tw_magic);
}

// Append tile kk to the worklist of step tn unless it is already there.  A
// set mark bit of parity tn & 1 can only come from step tn - 1 (every tile of
// a worklist is popped, clearing its bit, during its step), so a plain read
// that sees the bit set may skip the atomic.
__device__ __forceinline__ void mark_tile(const SimCtx &s, int kk, uint32_t tn)
{
    const uint32_t bit = 1u << (2 * (kk & 15) + (tn & 1));
    if (*((volatile uint32_t *)&s.marks[kk >> 4]) & bit) return;
    const uint32_t old = atomicOr(&s.marks[kk >> 4], bit);
    if (!(old & bit)) {
        const uint32_t slot = tn % 3;
        const uint32_t idx = atomicAdd(&s.sh->count[slot], 1u);
        s.lists[slot * s.ntiles + idx] = (uint16_t)kk;
    }
}

// Exact decision of one trial through the double-precision threshold.
static __device__ __noinline__ int exact_decide(const double *beta,
                                                bool forest, float4 f,
                                                bool upd, int d, uint32_t u)
{
    const uint64_t T = spec::threshold_of_z(
        spec::z_of(beta, forest, f.x, f.y, f.z, f.w, upd, d));
    return (uint64_t)u < T ? 1 : 0;
}

// Trials of the directions in m4 (bit j: direction base + j) drawn from one
// Philox block; stops at the first success.
__device__ __forceinline__ bool test_dirs(uint32_t m4, int base, uint4 u4,
                                          const ScreenCell &sc, const ff &b3,
                                          float margin, uint32_t up,
                                          const double *beta, bool forest,
                                          const float4 &f)
{
    while (m4) {
        const int j = __ffs(m4) - 1;
        m4 &= m4 - 1;
        const int d = base + j;
        const uint32_t u = j == 0 ? u4.x : (j == 1 ? u4.y : (j == 2 ? u4.z : u4.w));
        const bool upd = (up >> d) & 1u;
        const float p32 = screen_p(screen_z(sc, b3, upd, d));
        int dec = screen_decide(p32, u, margin);
        if (dec < 0) dec = exact_decide(beta, forest, f, upd, d, u);
        if (dec) return true;
    }
    return false;
}

// Exact decision of the one-uniform-per-cell rule: u < floor((1 - q) 2^32),
// q = prod over the directions of dm (increasing d) of (1 - p_d).
static __device__ __noinline__ int exact_cell_decide(const double *beta,
                                                     bool forest, float4 f,
                                                     uint32_t up, uint32_t dm,
                                                     uint32_t u)
{
    double q = 1.0;
    for (int d = 0; d < 8; ++d) {
        if (!((dm >> d) & 1u)) continue;
        const double z = spec::z_of(beta, forest, f.x, f.y, f.z, f.w,
                                    (up >> d) & 1u, d);
        const double p = !(z > -40.0) ? 0.0 : (z >= 40.0 ? 1.0 : spec::logistic(z));
        q = __dmul_rn(q, __dsub_rn(1.0, p));
    }
    const double P = __dsub_rn(1.0, q);
    return (uint64_t)u < (uint64_t)floor(__dmul_rn(P, 4294967296.0)) ? 1 : 0;
}

// All trials of one candidate cell (dm: directions with a burning source).
__device__ __forceinline__ bool trial_cell(const SimCtx &s, uint32_t cell,
                                           uint32_t dm, uint32_t t)
{
    const MapDev &m = *s.map;
    const SimShared &sh = *s.sh;
    float4 f;   // (psi, sig, cos wind, sin wind)
    float2 wd;  // diagonal wind terms
    if (m.uniform_wind) {
        const float2 p = __ldg(&m.ps[cell]);
        f = make_float4(p.x, p.y, m.cw, m.sw);
        wd = make_float2(m.om1, m.om3);
    } else {
        f = __ldg(&m.feat[cell]);
        wd = __ldg(&m.wdiag[cell]);
    }
    const uint32_t fl = __ldg(&m.cfl[cell]);
    const bool forest = (fl & kFlagForest) != 0;
    const uint32_t up = fl & 0xffu;
    const ScreenCell sc = screen_cell(sh.sp, forest, f.x, f.y, f.z, wd.x, f.w,
                                      wd.y);
    const ff b3 = sh.sp.b3;
    if (s.a->cell_uniform) {
        float q = 1.0f;
        uint32_t mm = dm;
        while (mm) {
            const int d = __ffs(mm) - 1;
            mm &= mm - 1;
            const float p = screen_p(screen_z(sc, b3, (up >> d) & 1u, d));
            q = __fmul_rn(q, __fsub_rn(1.0f, p));
        }
        const uint32_t u = philox4x32_10_rk(cell, t, 2u, 0u, sh.rk).x;
        int dec = screen_decide(__fsub_rn(1.0f, q), u, sh.sp.cell_margin);
        if (dec < 0) dec = exact_cell_decide(sh.beta, forest, f, up, dm, u);
        return dec != 0;
    }
    // The cell ignites iff any trial succeeds, whatever the order they are
    // tested in; the half with more burning sources goes first, so that the
    // second Philox block is needed less often.
    const uint32_t lo = dm & 0x0fu, hi = dm >> 4;
    const uint32_t first = __popc(hi) > __popc(lo) ? 1u : 0u;
    bool ign = false;
    for (uint32_t k = 0; k < 2 && !ign; ++k) {
        const uint32_t half = first ^ k;
        const uint32_t m4 = half ? hi : lo;
        if (!m4) continue;
        const uint4 u = philox4x32_10_rk(cell, t, half, 0u, sh.rk);
        ign = test_dirs(m4, (int)(half * 4), u, sc, b3, sh.sp.margin, up,
                        sh.beta, forest, f);
    }
    return ign;
}

// Cell (row r, column i of tile k = (ti, tj)) ignites at step t: write it with
// the "burning, parity t + 1" code and put its tile, and the neighbour tiles
// across the edges it lies on, on the worklist of step t + 1.
template <bool kBurn>
__device__ __forceinline__ void ignite(const SimCtx &s, int k, int ti, int tj,
                                       int r, int i, uint32_t cell, uint32_t t)
{
    const MapDev &m = *s.map;
    uint32_t *P = (t & 1u) ? s.X : s.Y;
    atomicOr(&P[k * 32 + r], 1u << i);
    if (kBurn) {
        // only cells that burn two steps or more keep a fuel count
        const uint8_t f = burn_steps(*s.a, cell);
        if (f > 1) s.fuel[cell] = f;
    }
    if (s.a->burn_step)
        s.a->burn_step[(long long)s.sim * m.H * m.W + cell] = (int32_t)(t + 1);
    const uint32_t tn = t + 1;
    mark_tile(s, k, tn);
    const int dr = r == 0 ? -1 : (r == 31 ? 1 : 0);
    const int dc = i == 0 ? -1 : (i == 31 ? 1 : 0);
    const bool rok = dr != 0 && ti + dr >= 0 && ti + dr < m.TH;
    const bool cok = dc != 0 && tj + dc >= 0 && tj + dc < m.TW;
    if (rok) mark_tile(s, k + dr * m.TW, tn);
    if (cok) mark_tile(s, k + dc, tn);
    if (rok && cok) mark_tile(s, k + dr * m.TW + dc, tn);
}

// Position of the n-th (0-based) set bit of m (n < popc(m)).
__device__ __forceinline__ int nth_set_bit(uint32_t m, uint32_t n)
{
    int pos = 0;
    uint32_t c = __popc(m & 0xffffu);
    if (n >= c) { n -= c; m >>= 16; pos += 16; }
    c = __popc(m & 0xffu);
    if (n >= c) { n -= c; m >>= 8; pos += 8; }
    c = __popc(m & 0xfu);
    if (n >= c) { n -= c; m >>= 4; pos += 4; }
    c = __popc(m & 0x3u);
    if (n >= c) { n -= c; m >>= 2; pos += 2; }
    if (n >= (m & 1u)) pos += 1;
    return pos;
}

// Phase A of step t for active tile k, one warp (lane = tile row): retire the
// previous step's burning cells, find the targets with a burning source in
// each direction, count the trials and queue the candidates for phase B.
template <bool kBurn>
__device__ __forceinline__ void phase_a(const SimCtx &s, int k, uint32_t t,
                                        int lane, uint32_t &ntrials)
{
    const SimLaunch &a = *s.a;
    const MapDev &m = *s.map;
    SimShared &sh = *s.sh;
    const int TW = m.TW, TH = m.TH;
    const int ti = tile_row(sh, k), tj = k - ti * TW;
    const uint32_t par = t & 1u;
    uint32_t *X = s.X, *Y = s.Y;
    // burn-time variant: the sources of step t also include the cells that
    // ignited before step t - 1 and still burn (plane K[t & 1])
    const uint32_t *Kt = kBurn ? (par ? s.K1 : s.K0) : nullptr;

    if (lane == 0) atomicAnd(&s.marks[k >> 4], ~(1u << (2 * (k & 15) + par)));

    const int w = k * 32 + lane;
    const uint32_t x = X[w], y = Y[w];
    uint32_t b = burning(x, y, par);
    if (kBurn) b |= Kt[w];
    uint32_t bl = 0, br = 0;
    if (tj > 0) {
        bl = burning(X[w - 32], Y[w - 32], par);
        if (kBurn) bl |= Kt[w - 32];
    }
    if (tj < TW - 1) {
        br = burning(X[w + 32], Y[w + 32], par);
        if (kBurn) br |= Kt[w + 32];
    }
    // Edge rows of the tiles above (row 31) and below (row 0), including the
    // diagonal neighbours: lanes 0..5 fetch one word each.
    uint32_t edge = 0;
    if (lane < 6) {
        const int dti = lane < 3 ? -1 : 1;
        const int dtj = (lane % 3) - 1;   // -1, 0, +1
        const int nti = ti + dti, ntj = tj + dtj;
        if (nti >= 0 && nti < TH && ntj >= 0 && ntj < TW) {
            const int we = (nti * TW + ntj) * 32 + (dti < 0 ? 31 : 0);
            edge = burning(X[we], Y[we], par);
            if (kBurn) edge |= Kt[we];
        }
    }
    uint32_t bu = __shfl_up_sync(kFull, b, 1);
    uint32_t blu = __shfl_up_sync(kFull, bl, 1);
    uint32_t bru = __shfl_up_sync(kFull, br, 1);
    uint32_t bd = __shfl_down_sync(kFull, b, 1);
    uint32_t bld = __shfl_down_sync(kFull, bl, 1);
    uint32_t brd = __shfl_down_sync(kFull, br, 1);
    const uint32_t e_ul = __shfl_sync(kFull, edge, 0);
    const uint32_t e_u = __shfl_sync(kFull, edge, 1);
    const uint32_t e_ur = __shfl_sync(kFull, edge, 2);
    const uint32_t e_dl = __shfl_sync(kFull, edge, 3);
    const uint32_t e_d = __shfl_sync(kFull, edge, 4);
    const uint32_t e_dr = __shfl_sync(kFull, edge, 5);
    if (lane == 0) {
        bu = e_u;
        blu = e_ul;
        bru = e_ur;
    }
    if (lane == 31) {
        bd = e_d;
        bld = e_dl;
        brd = e_dr;
    }
    // Retire last step's burning cells (code of parity t + 1) to "burnt";
    // readers of other tiles only look for the parity-t code.
    const uint32_t stale = burning(x, y, par ^ 1u);
    if (stale) {
        X[w] = x | stale;
        Y[w] = y | stale;
    }
    if (kBurn) {
        // each cell burning at step t spends one step of fuel; the ones left
        // with fuel burn at step t + 1 as well (plane K[(t + 1) & 1], written
        // for this tile's rows only by this warp; a tile holding such cells
        // is on the next worklist, and so is a neighbour tile across an edge
        // they lie on)
        uint32_t cont = 0, mm = b & __ldg(&a.long_burn[w]);
        const uint32_t rowc = (uint32_t)(ti * 32 + lane) * (uint32_t)m.W +
                              (uint32_t)(tj * 32);
        while (mm) {
            const int i = __ffs(mm) - 1;
            mm &= mm - 1;
            const uint8_t left = (uint8_t)(s.fuel[rowc + i] - 1u);
            s.fuel[rowc + i] = left;
            if (left) cont |= 1u << i;
        }
        (par ? s.K0 : s.K1)[w] = cont;
        const uint32_t cl = __ballot_sync(kFull, cont & 1u);
        const uint32_t cr = __ballot_sync(kFull, (cont >> 31) & 1u);
        const uint32_t top = __shfl_sync(kFull, cont, 0);
        const uint32_t bot = __shfl_sync(kFull, cont, 31);
        if (__any_sync(kFull, cont != 0) && lane == 0) {
            sh.newflag[(t + 1) % 3] = 1;
            const uint32_t tn = t + 1;
            if (top && ti > 0) mark_tile(s, k - TW, tn);
            if (bot && ti < TH - 1) mark_tile(s, k + TW, tn);
            if (cl && tj > 0) mark_tile(s, k - 1, tn);
            if (cr && tj < TW - 1) mark_tile(s, k + 1, tn);
            if ((top & 1u) && ti > 0 && tj > 0) mark_tile(s, k - TW - 1, tn);
            if ((top >> 31) && ti > 0 && tj < TW - 1) mark_tile(s, k - TW + 1, tn);
            if ((bot & 1u) && ti < TH - 1 && tj > 0) mark_tile(s, k + TW - 1, tn);
            if ((bot >> 31) && ti < TH - 1 && tj < TW - 1)
                mark_tile(s, k + TW + 1, tn);
        }
    }
    if (__any_sync(kFull, b != 0) && lane == 0) mark_tile(s, k, t + 1);
    __syncwarp();

    // Targets of row `lane` with a burning source in direction d (the source
    // of direction d lies at target - off(d)).
    const uint32_t avail = ~(x | y);
    uint32_t md[8];
    md[0] = bd;                               // N : source below
    md[1] = (bd << 1) | (bld >> 31);          // NE: source below-left
    md[2] = (b << 1) | (bl >> 31);            // E : source left
    md[3] = (bu << 1) | (blu >> 31);          // SE: source above-left
    md[4] = bu;                               // S : source above
    md[5] = (bu >> 1) | (bru << 31);          // SW: source above-right
    md[6] = (b >> 1) | (br << 31);            // W : source right
    md[7] = (bd >> 1) | (brd << 31);          // NW: source below-right
    uint32_t cand = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        md[d] &= avail;
        cand |= md[d];
    }
    const uint32_t c = __popc(cand);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    // Reserve queue space for the tile's candidates; a full queue makes this
    // warp decide them here instead (same decisions, in phase A).
    uint32_t base = 0;
    if (lane == 0) {
        base = atomicAdd(&sh.qcount[par], total);
        if (base + total > (uint32_t)a.qcap) {
            atomicMin(&sh.qvalid[par], base);
            base = 0xffffffffu;
        }
    }
    base = __shfl_sync(kFull, base, 0);
    // Candidate q (in row-major order within the tile) goes to lane q mod 32:
    // its row is the first with inclusive prefix > q, its column the
    // (q - excl)-th set bit of that row's candidate mask.  The trip count is
    // the same for every lane (all lanes take part in the shuffles).
    for (uint32_t q0 = 0; q0 < total; q0 += 32) {
        const uint32_t q = q0 + lane;
        int r = 0;
        if (__shfl_sync(kFull, incl, 15) <= q) r = 16;
        if (__shfl_sync(kFull, incl, r + 7) <= q) r += 8;
        if (__shfl_sync(kFull, incl, r + 3) <= q) r += 4;
        if (__shfl_sync(kFull, incl, r + 1) <= q) r += 2;
        if (__shfl_sync(kFull, incl, r) <= q) r += 1;
        const uint32_t cr = __shfl_sync(kFull, cand, r);
        const uint32_t ir = __shfl_sync(kFull, incl, r);
        const int i = nth_set_bit(cr, q - (ir - (uint32_t)__popc(cr)));
        uint32_t dm = 0;
#pragma unroll
        for (int d = 0; d < 8; ++d)
            dm |= ((__shfl_sync(kFull, md[d], r) >> i) & 1u) << d;
        if (q >= total) continue;
        if (base != 0xffffffffu) {
            s.queue[base + q] = ((uint32_t)(k * 32 + r) << 13) |
                                ((uint32_t)i << 8) | dm;
        } else {
            const uint32_t cell = (uint32_t)(ti * 32 + r) * (uint32_t)m.W +
                                  (uint32_t)(tj * 32 + i);
            ntrials += (uint32_t)__popc(dm);
            if (trial_cell(s, cell, dm, t)) {
                ignite<kBurn>(s, k, ti, tj, r, i, cell, t);
                // every writer of this step stores the same values
                sh.newflag[(t + 1) % 3] = 1;
                sh.last_new = t + 1;
            }
        }
    }
}

template <bool kSmemState, bool kBurn>
__global__ void __launch_bounds__(kSimMaxThreads, 2) k_simulate(SimLaunch a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles_max = a.ntiles_max;
    const SimLayout L = sim_layout(ntiles_max, a.qcap, kSmemState);
    const int nwarps = blockDim.x >> 5;
    SimShared &sh = *reinterpret_cast<SimShared *>(smem + L.header);
    const MapDev &m = sh.map;
    SimCtx s;
    s.a = &a;
    s.sh = &sh;
    s.map = &sh.map;
    s.marks = reinterpret_cast<uint32_t *>(smem + L.marks);
    s.lists = reinterpret_cast<uint16_t *>(smem + L.lists);
    s.queue = reinterpret_cast<uint32_t *>(smem + L.queue);
    s.ntiles = ntiles_max;
    if (kSmemState) {
        s.X = reinterpret_cast<uint32_t *>(smem + L.planes);
    } else {
        const size_t stride =
            a.block_words ? a.block_words : 2 * (size_t)ntiles_max * 32;
        s.X = a.gstate + (size_t)blockIdx.x * stride;
    }
    s.Y = s.X + ntiles_max * 32;
    s.K0 = s.K1 = nullptr;
    s.fuel = nullptr;
    if (kBurn) {
        s.K0 = s.Y + ntiles_max * 32;
        s.K1 = s.K0 + ntiles_max * 32;
        s.fuel = reinterpret_cast<uint8_t *>(s.K1 + ntiles_max * 32);
    }

    if (kSmemState && threadIdx.x == 0) {
        mbar_init(&sh.mbar, 1);
        fence_proxy_async_smem();
    }
    uint32_t phase = 0;
    __syncthreads();

    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t w = atomicAdd(a.work_counter, 1u);
            sh.sim = w < (uint32_t)a.n ? (a.order ? (int)a.order[w] : (int)w)
                                       : a.n;
        }
        __syncthreads();
        const int sim = sh.sim;
        if (sim >= a.n) break;
        s.sim = sim;

        // --- set-up of simulation `sim` ---
        if (threadIdx.x == 0) {
            bool map_ok = true;
            if (a.maps) {
                const int mi = a.map_of_sim ? a.map_of_sim[sim] : 0;
                map_ok = mi >= 0 && mi < a.nmaps;
                sh.map = a.maps[map_ok ? mi : 0];
            } else {
                sh.map = a.map;
            }
            const long long hw = (long long)sh.map.H * sh.map.W;
            // a fire runs at most one step per cell (one step per cell and
            // step of burn time in the burn-time variant) plus the last
            sh.hard_cap = (uint32_t)min((hw + 2) * (kBurn ? 256 : 1),
                                        (long long)0x7fffffff);
            sh.nmark = (sh.map.ntiles + 15) / 16;
            sh.tw_magic = 0xffffffffu / (uint32_t)sh.map.TW;
            sh.status = map_ok ? 0u : FIRE_STATUS_BAD_MAP;
            const fire_params P = a.params[sim];
            for (int j = 0; j < 5; ++j) sh.beta[j] = P.b[j];
            sh.sp = screen_params(P.b);
            const uint64_t seed = a.seeds[sim];
            sh.key0 = (uint32_t)seed;
            sh.key1 = (uint32_t)(seed >> 32);
            philox_round_keys(sh.key0, sh.key1, sh.rk);
            const fire_cell g = a.ign[sim];
            const bool ok = map_ok && g.row >= 0 && g.row < m.H &&
                            g.col >= 0 && g.col < m.W &&
                            (m.cfl[(long long)g.row * m.W + g.col] &
                             kFlagBurnable);
            sh.skip = ok ? 0 : 1;
            sh.timeout = 0;
            sh.count[0] = sh.count[1] = sh.count[2] = 0;
            sh.newflag[0] = 1;
            sh.newflag[1] = sh.newflag[2] = 0;
            sh.qcount[0] = sh.qcount[1] = 0;
            sh.qvalid[0] = sh.qvalid[1] = (uint32_t)a.qcap;
            sh.trials = 0;
            sh.last_new = 0;
            sh.burnt = 0;
            sh.inter = 0;
        }
        __syncthreads();   // the map descriptor is read by every thread below
        const uint32_t plane_bytes = (uint32_t)m.ntiles * 128u;
        const long long HW = (long long)m.H * m.W;
        for (int i = threadIdx.x; i < sh.nmark; i += blockDim.x) s.marks[i] = 0;
        if (kSmemState) {
            fence_proxy_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(&sh.mbar, 2u * plane_bytes);
                bulk_g2s(s.X, m.blk, plane_bytes, &sh.mbar);
                bulk_g2s(s.Y, m.blk, plane_bytes, &sh.mbar);
            }
        } else {
            const uint4 *src = reinterpret_cast<const uint4 *>(m.blk);
            uint4 *dx = reinterpret_cast<uint4 *>(s.X);
            uint4 *dy = reinterpret_cast<uint4 *>(s.Y);
            // two 16-byte loads in flight per thread before their stores
            const int n16 = m.ntiles * 8, bd = blockDim.x;
            for (int i = threadIdx.x; i < n16; i += 2 * bd) {
                const bool two = i + bd < n16;
                const uint4 v0 = src[i];
                const uint4 v1 = two ? src[i + bd] : v0;
                dx[i] = v0;
                dy[i] = v0;
                if (two) {
                    dx[i + bd] = v1;
                    dy[i + bd] = v1;
                }
            }
            if (kBurn) {
                uint4 *dk = reinterpret_cast<uint4 *>(s.K0);
                for (int i = threadIdx.x; i < ntiles_max * 16; i += blockDim.x)
                    dk[i] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        if (a.burn_step) {
            int32_t *bs = a.burn_step + (long long)sim * HW;
            for (long long i = threadIdx.x; i < HW; i += blockDim.x)
                bs[i] = (m.cfl[i] & kFlagBurnable) ? -1 : -2;
        }
        if (kSmemState) {
            const long long t0 = clock64();
            bool done = mbar_try_wait(&sh.mbar, phase);
            while (!done) {
                if (clock64() - t0 > (1ll << 31)) break;
                done = mbar_try_wait(&sh.mbar, phase);
            }
            if (!done) atomicOr((unsigned *)&sh.timeout, 1u);
            phase ^= 1u;
        }
        __syncthreads();
        if (sh.timeout) {
            if (threadIdx.x == 0) {
                atomicOr(a.error_word, 1u);
                fire_result r{};
                r.status = FIRE_STATUS_TIMEOUT;
                a.out[sim] = r;
            }
            return;  // the copy never completed: leave this block
        }
        if (threadIdx.x == 0) {
            const fire_cell g = a.ign[sim];
            if (sh.skip) {
                fire_result r{};
                r.target = *m.tgt_count;
                r.status = (sh.status & FIRE_STATUS_BAD_MAP)
                               ? FIRE_STATUS_BAD_MAP
                               : FIRE_STATUS_BAD_IGNITION;
                a.out[sim] = r;
            } else {
                const int k0 = (g.row >> 5) * m.TW + (g.col >> 5);
                const int r0 = g.row & 31, i0 = g.col & 31;
                s.X[k0 * 32 + r0] |= 1u << i0;   // burning, parity 0
                if (kBurn) {
                    const uint32_t c0 = (uint32_t)g.row * (uint32_t)m.W + (uint32_t)g.col;
                    const uint8_t f = burn_steps(a, c0);
                    if (f > 1) s.fuel[c0] = f;
                }
                if (a.burn_step)
                    a.burn_step[(long long)sim * HW + (long long)g.row * m.W +
                                g.col] = 0;
                const int ti = k0 / m.TW, tj = k0 - ti * m.TW;
                for (int dti = -1; dti <= 1; ++dti) {
                    for (int dtj = -1; dtj <= 1; ++dtj) {
                        const bool rowok = dti == 0 || (dti < 0 ? r0 == 0 : r0 == 31);
                        const bool colok = dtj == 0 || (dtj < 0 ? i0 == 0 : i0 == 31);
                        const int nti = ti + dti, ntj = tj + dtj;
                        if (rowok && colok && nti >= 0 && nti < m.TH &&
                            ntj >= 0 && ntj < m.TW)
                            mark_tile(s, nti * m.TW + ntj, 0);
                    }
                }
            }
        }
        if (sh.skip) {  // uniform: written before the last barrier
            __syncthreads();
            continue;
        }

        // --- steps: phase A (tiles) | barrier | phase B (trials) | barrier
        uint32_t t = 0;
        bool capped = false;
        // trials of the candidates this thread decides (each candidate is
        // decided once, in phase B or, after a queue overflow, in phase A)
        uint32_t ntrials = 0;
        for (;; ++t) {
            __syncthreads();
            const uint32_t nA = sh.count[t % 3];
            if (nA == 0) break;
            const bool burning_now = sh.newflag[t % 3] != 0;
            // burn-time variant: the fire ends when nothing burns (its
            // worklist can still hold tiles to retire)
            if (kBurn && !burning_now) break;
            if (burning_now && ((a.max_steps && t >= a.max_steps) || t >= sh.hard_cap)) {
                capped = true;
                break;
            }
            if (threadIdx.x == 0) {
                sh.count[(t + 2) % 3] = 0;
                sh.newflag[(t + 2) % 3] = 0;
            }
            const uint16_t *list = s.lists + (t % 3) * ntiles_max;
            for (uint32_t li = warp; li < nA; li += nwarps)
                phase_a<kBurn>(s, list[li], t, lane, ntrials);
            __syncthreads();
            const uint32_t par = t & 1u;
            const uint32_t nq = min(sh.qcount[par], sh.qvalid[par]);
            if (threadIdx.x == 0) {
                sh.qcount[par ^ 1u] = 0;
                sh.qvalid[par ^ 1u] = (uint32_t)a.qcap;
            }
            bool any = false;
            for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
                const uint32_t e = s.queue[q];
                const uint32_t w = e >> 13;
                const int i = (int)((e >> 8) & 31u);
                const int k = (int)(w >> 5), r = (int)(w & 31u);
                const int ti = tile_row(sh, k), tj = k - ti * m.TW;
                const uint32_t cell = (uint32_t)(ti * 32 + r) * (uint32_t)m.W +
                                      (uint32_t)(tj * 32 + i);
                ntrials += (uint32_t)__popc(e & 0xffu);
                if (trial_cell(s, cell, e & 0xffu, t)) {
                    ignite<kBurn>(s, k, ti, tj, r, i, cell, t);
                    any = true;
                }
            }
            if (__any_sync(kFull, any) && lane == 0) {
                sh.newflag[(t + 1) % 3] = 1;
                sh.last_new = t + 1;
            }
        }

        // --- final sweep: Eq. 2 counts and border status from the state ---
        __syncthreads();
        uint32_t nb = 0, ni = 0;
        bool border = false;
        if (a.burnt_bits) {
            for (int w = threadIdx.x; w < m.ntiles * 32; w += blockDim.x) {
                const uint32_t bw = (s.X[w] | s.Y[w]) & ~__ldg(&m.blk[w]);
                a.burnt_bits[(long long)sim * m.ntiles * 32 + w] = bw;
                if (!bw) continue;
                nb += __popc(bw);
                ni += __popc(bw & __ldg(&m.tgt[w]));
                const int k = w >> 5;
                const int ti = tile_row(sh, k), tj = k - ti * m.TW;
                const int R = ti * 32 + (w & 31);
                if (R == 0 || R == m.H - 1 || (tj == 0 && (bw & 1u)) ||
                    (tj == m.TW - 1 && ((bw >> ((m.W - 1) & 31)) & 1u)))
                    border = true;
            }
        } else {
            // four consecutive rows of one tile per thread (16-byte loads)
            const uint4 *X4 = reinterpret_cast<const uint4 *>(s.X);
            const uint4 *Y4 = reinterpret_cast<const uint4 *>(s.Y);
            const uint4 *B4 = reinterpret_cast<const uint4 *>(m.blk);
            const uint4 *T4 = reinterpret_cast<const uint4 *>(m.tgt);
            for (int v = threadIdx.x; v < m.ntiles * 8; v += blockDim.x) {
                const uint4 x = X4[v], y = Y4[v], bl = __ldg(&B4[v]);
                const uint32_t bw[4] = {(x.x | y.x) & ~bl.x, (x.y | y.y) & ~bl.y,
                                        (x.z | y.z) & ~bl.z, (x.w | y.w) & ~bl.w};
                if (!(bw[0] | bw[1] | bw[2] | bw[3])) continue;
                const uint4 tg = __ldg(&T4[v]);
                nb += __popc(bw[0]) + __popc(bw[1]) + __popc(bw[2]) + __popc(bw[3]);
                ni += __popc(bw[0] & tg.x) + __popc(bw[1] & tg.y) +
                      __popc(bw[2] & tg.z) + __popc(bw[3] & tg.w);
                const int k = v >> 3;
                const int ti = tile_row(sh, k), tj = k - ti * m.TW;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int R = ti * 32 + ((v & 7) << 2) + j;
                    if (bw[j] && (R == 0 || R == m.H - 1 || (tj == 0 && (bw[j] & 1u)) ||
                                  (tj == m.TW - 1 && ((bw[j] >> ((m.W - 1) & 31)) & 1u))))
                        border = true;
                }
            }
        }
        nb = __reduce_add_sync(kFull, nb);
        ni = __reduce_add_sync(kFull, ni);
        ntrials = __reduce_add_sync(kFull, ntrials);
        border = __any_sync(kFull, border);
        if (lane == 0) {
            if (ntrials) atomicAdd(&sh.trials, ntrials);
            if (nb) atomicAdd(&sh.burnt, nb);
            if (ni) atomicAdd(&sh.inter, ni);
            if (border) atomicOr(&sh.status, FIRE_STATUS_BORDER);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            fire_result r;
            r.burnt = sh.burnt;
            r.inter = sh.inter;
            r.target = *m.tgt_count;
            // steps in which some cell burned (the burn-time variant leaves
            // the loop at the first step with none)
            r.steps = (capped || kBurn) ? t : sh.last_new + 1;
            r.status = sh.status | (capped ? FIRE_STATUS_STEP_CAP : 0u);
            r.trials = sh.trials;
            a.out[sim] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// Longest-first order of a batch (scheduling only).  A fire's work grows with
// how readily its parameters spread fire on this map, so each fire gets the
// key: mean over a fixed sample of burnable cells (about 2048, every stride-th
// cell) of the single-precision probability 1 - prod_d (1 - p_d) that a cell
// with all eight neighbours burning ignites; fires are then handed to the
// persistent blocks by decreasing key (ties to the lower index), so the
// longest fires start first and the launch's tail shrinks.
__global__ void k_spread_key(MapDev m, int n, const fire_params *__restrict__ params,
                             long long stride, float *__restrict__ key)
{
    const int i = blockIdx.x;
    if (i >= n) return;
    const ScreenParams sp = screen_params(params[i].b);
    const long long HW = (long long)m.H * m.W;
    float acc = 0.0f;
    unsigned cnt = 0;
    for (long long c = (long long)threadIdx.x * stride; c < HW;
         c += (long long)blockDim.x * stride) {
        const uint32_t fl = __ldg(&m.cfl[c]);
        if (!(fl & kFlagBurnable)) continue;
        const float4 f = __ldg(&m.feat[c]);
        const float2 wd = __ldg(&m.wdiag[c]);
        const ScreenCell sc = screen_cell(sp, (fl & kFlagForest) != 0, f.x, f.y, f.z,
                                          wd.x, f.w, wd.y);
        float q = 1.0f;
#pragma unroll
        for (int d = 0; d < 8; ++d)
            q *= 1.0f - screen_p(screen_z(sc, sp.b3, (fl >> d) & 1u, d));
        acc += 1.0f - q;
        cnt++;
    }
    __shared__ float sa[256];
    __shared__ unsigned sc_[256];
    sa[threadIdx.x] = acc;
    sc_[threadIdx.x] = cnt;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sc_[threadIdx.x] += sc_[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const float k = sc_[0] ? sa[0] / (float)sc_[0] : 0.0f;
        key[i] = k == k ? k : -1.0f;   // NaN parameters go last
    }
}

// order[r] = the fire of rank r by decreasing key (ties: lower index first).
__global__ void k_rank_desc(int n, const float *__restrict__ key,
                            uint32_t *__restrict__ order)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ki = key[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
        const float kj = key[j];
        r += (kj > ki) || (kj == ki && j < i);
    }
    order[r] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Fitness of Eq. 2 (kind 0) or Jaccard distance (kind 1).
__global__ void k_fitness(const fire_result *__restrict__ r, int n, int kind,
                          double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const fire_result q = r[i];
    const double uni = __dsub_rn(__dadd_rn((double)q.target, (double)q.burnt),
                                 (double)q.inter);
    const double sym = __dsub_rn(uni, (double)q.inter);
    const double den = kind == 0 ? (double)q.target : uni;
    out[i] = den == 0.0 ? __longlong_as_double(0x7ff8000000000000ll)
                        : __ddiv_rn(sym, den);
}

// Exact thresholds of every (direction, cell).
__global__ void k_thresholds(MapDev m, const double *__restrict__ beta_dev,
                             int64_t *__restrict__ out)
{
    const long long HW = (long long)m.H * m.W;
    double b[5];
    for (int j = 0; j < 5; ++j) b[j] = beta_dev[j];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
         idx < 8 * HW; idx += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(idx / HW);
        const long long i = idx - d * HW;
        const float4 f = m.feat[i];
        const uint32_t fl = m.cfl[i];
        const double z = spec::z_of(b, fl & kFlagForest, f.x, f.y, f.z, f.w,
                                    (fl >> d) & 1u, d);
        out[idx] = (int64_t)spec::threshold_of_z(z);
    }
}

__global__ void k_probabilities(MapDev m, const double *__restrict__ beta_dev,
                                float *__restrict__ p32,
                                double *__restrict__ p64)
{
    const long long HW = (long long)m.H * m.W;
    double b[5];
    for (int j = 0; j < 5; ++j) b[j] = beta_dev[j];
    const ScreenParams sp = screen_params(b);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
         idx < 8 * HW; idx += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(idx / HW);
        const long long i = idx - d * HW;
        const float4 f = m.feat[i];
        const uint32_t fl = m.cfl[i];
        const bool forest = fl & kFlagForest, up = (fl >> d) & 1u;
        if (p32) {
            const float2 wd = m.wdiag[i];
            const ScreenCell sc =
                screen_cell(sp, forest, f.x, f.y, f.z, wd.x, f.w, wd.y);
            p32[idx] = screen_p(screen_z(sc, sp.b3, up, d));
        }
        if (p64)
            p64[idx] = spec::logistic(
                spec::z_of(b, forest, f.x, f.y, f.z, f.w, up, d));
    }
}

__global__ void k_features_export(MapDev m, float *psi, float *sig, float *cw,
                                  float *sw, uint16_t *cfl)
{
    const long long HW = (long long)m.H * m.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 f = m.feat[i];
        if (psi) psi[i] = f.x;
        if (sig) sig[i] = f.y;
        if (cw) cw[i] = f.z;
        if (sw) sw[i] = f.w;
        if (cfl) cfl[i] = m.cfl[i];
    }
}

// Randomised check of the single-precision screen against the exact
// threshold: uniform and Gaussian parameters, random covariates, and draws
// both uniform and placed next to the exact threshold.  Also records the
// largest ratio of |p32 - p64| to the screen's stated error bound.
__global__ void k_screen_selftest(uint64_t n, uint64_t seed,
                                  unsigned long long *counts,
                                  unsigned long long *max_dp_bits)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    unsigned long long local[3] = {0, 0, 0};
    double local_max = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r1 = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), 1u, 0u, k0, k1);
        const uint4 r2 = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), 2u, 0u, k0, k1);
        const uint4 r3 = philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), 3u, 0u, k0, k1);
        const uint32_t rs[5] = {r1.x, r1.y, r1.z, r1.w, r2.x};
        double b[5];
        const bool gauss = (r2.y >> 31) & 1u;
        const double wide = ((r2.y >> 30) & 1u) ? 200.0 : 30.0;
        for (int j = 0; j < 5; ++j) {
            const double u = ((double)rs[j] + 0.5) * 0x1p-32;
            // a Gaussian-looking sum (sd ~5), or uniform on [-30, 30] or on
            // [-200, 200] (a large |b3| widens the screen's margin)
            b[j] = gauss ? (u - 0.5) * 17.32 + ((double)(rs[(j + 1) % 5] >> 16) /
                                                     65536.0 - 0.5) * 17.32
                         : wide * (2.0 * u - 1.0);
        }
        const bool forest = r2.y & 1u;
        const int d = (int)((r2.y >> 1) & 7u);
        const bool up = (r2.y >> 4) & 1u;
        const float psi = (float)(((double)(r2.z >> 8) * 0x1p-24) * 2.0 - 1.0);
        const float sig = (float)(0.9 * (double)(r2.w >> 8) * 0x1p-24);
        const double ang = 360.0 * (double)(r3.x >> 8) * 0x1p-24;
        const float cw = __double2float_rn(spec::cosd(ang));
        const float sw = __double2float_rn(spec::sind(ang));
        const double z = spec::z_of(b, forest, psi, sig, cw, sw, up, d);
        const uint64_t T = spec::threshold_of_z(z);
        uint32_t u;
        if ((r3.y & 3u) == 0) {
            u = r3.z;
        } else {
            const int64_t off = (int64_t)(r3.z % 200001u) - 100000;
            int64_t v = (int64_t)T + off;
            v = v < 0 ? 0 : (v > 0xffffffffll ? 0xffffffffll : v);
            u = (uint32_t)v;
        }
        const ScreenParams sp = screen_params(b);
        const float om1 = __double2float_rn(spec::omega(cw, sw, 1));
        const float om3 = __double2float_rn(spec::omega(cw, sw, 3));
        const ScreenCell sc = screen_cell(sp, forest, psi, sig, cw, om1, sw, om3);
        const float p32 = screen_p(screen_z(sc, sp.b3, up, d));
        int dec = screen_decide(p32, u, sp.margin);
        const bool exact = (uint64_t)u < T;
        local[0]++;
        if (dec < 0) {
            local[1]++;
            dec = exact;
        }
        if ((dec != 0) != exact) local[2]++;
        // |p32 - p64| against the screen's stated bound
        const double dp = fabs((double)p32 - spec::logistic(z));
        local_max = fmax(local_max,
                         dp / ((double)kScreenErrB3 * fabs(b[3]) + kScreenErr0));
    }
    for (int j = 0; j < 3; ++j) {
        unsigned long long v = local[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&counts[j], v);
    }
    for (int o = 16; o > 0; o >>= 1)
        local_max = fmax(local_max, __shfl_down_sync(kFull, local_max, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(max_dp_bits, (unsigned long long)__double_as_longlong(local_max));
}

// Philox blocks as the simulation draws them (the precomputed key schedule
// of philox4x32_10_rk).
__global__ void k_philox_blocks(uint64_t n, uint4 ctr, uint2 key, uint32_t *out)
{
    __shared__ uint4 rk[5];
    if (threadIdx.x == 0) philox_round_keys(key.x, key.y, rk);
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox4x32_10_rk(ctr.x + (uint32_t)i, ctr.y, ctr.z, ctr.w,
                                         rk);
        reinterpret_cast<uint4 *>(out)[i] = r;
    }
}

// ---------------------------------------------------------------------------
// Processing order of a multi-map batch: simulations grouped by map, largest
// map first (rank 0 = most tiles), by a counting sort.  The order inside a
// group is arbitrary; results do not depend on it.

__global__ void k_order_count(int n, const int32_t *__restrict__ map_of_sim,
                              int nmaps, const int32_t *__restrict__ rank,
                              uint32_t *__restrict__ counts)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        const int mi = map_of_sim[i];
        const int b = (mi >= 0 && mi < nmaps) ? rank[mi] : nmaps;
        atomicAdd(&counts[b], 1u);
    }
}

__global__ void k_order_scan(int nb, uint32_t *counts)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = 0; b < nb; ++b) {
            const uint32_t c = counts[b];
            counts[b] = acc;
            acc += c;
        }
    }
}

__global__ void k_order_scatter(int n, const int32_t *__restrict__ map_of_sim,
                                int nmaps, const int32_t *__restrict__ rank,
                                uint32_t *__restrict__ cursor,
                                uint32_t *__restrict__ order)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += gridDim.x * blockDim.x) {
        const int mi = map_of_sim[i];
        const int b = (mi >= 0 && mi < nmaps) ? rank[mi] : nmaps;
        order[atomicAdd(&cursor[b], 1u)] = (uint32_t)i;
    }
}

// ---------------------------------------------------------------------------
// Launchers.

static int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

cudaError_t launch_features(int H, int W, const uint8_t *veg, const float *elev,
                            const float *slope, const float *aspect,
                            const float *wind, float4 *feat, float2 *wdiag,
                            float2 *ps, uint16_t *cfl, uint32_t *wind_varies,
                            cudaStream_t st)
{
    const long long n = (long long)H * W;
    cudaError_t e = cudaMemsetAsync(wind_varies, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    k_features<<<grid_for(n, 256), 256, 0, st>>>(H, W, veg, elev, slope, aspect,
                                                 wind, feat, wdiag, ps, cfl,
                                                 wind_varies);
    return cudaGetLastError();
}

cudaError_t launch_blocked(const MapDev &m, const uint8_t *veg, uint32_t *blk,
                           cudaStream_t st)
{
    const int nw = m.ntiles * 32;
    k_pack_bits<false><<<(nw + 255) / 256, 256, 0, st>>>(m.H, m.W, m.TW, nw,
                                                         veg, blk, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_target(const MapDev &m, const uint8_t *burnt, uint32_t *tgt,
                          uint32_t *tgt_count, cudaStream_t st)
{
    const int nw = m.ntiles * 32;
    cudaError_t e = cudaMemsetAsync(tgt_count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    k_pack_bits<true><<<(nw + 255) / 256, 256, 0, st>>>(m.H, m.W, m.TW, nw,
                                                        burnt, tgt, tgt_count);
    return cudaGetLastError();
}

const void *simulate_kernel_ptr(bool smem_state)
{
    return smem_state ? (const void *)k_simulate<true, false>
                      : (const void *)k_simulate<false, false>;
}

const void *simulate_burn_kernel_ptr()
{
    return (const void *)k_simulate<false, true>;
}

cudaError_t launch_simulate(const SimLaunch &a, bool smem_state, int nwarps,
                            int grid, size_t smem_bytes, cudaStream_t st)
{
    if (smem_state)
        k_simulate<true, false><<<grid, nwarps * 32, smem_bytes, st>>>(a);
    else
        k_simulate<false, false><<<grid, nwarps * 32, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_long_burn(const MapDev &m, const uint8_t *burn_time,
                             uint32_t *plane, uint32_t *any, cudaStream_t st)
{
    const int nw = m.ntiles * 32;
    cudaError_t e = cudaMemsetAsync(any, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    k_long_burn<<<(nw + 255) / 256, 256, 0, st>>>(m.H, m.W, m.TW, nw, burn_time,
                                                 plane, any);
    return cudaGetLastError();
}

cudaError_t launch_simulate_burn(const SimLaunch &a, int nwarps, int grid,
                                 size_t smem_bytes, cudaStream_t st)
{
    k_simulate<false, true><<<grid, nwarps * 32, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_longest_first(const MapDev &m, int n, const fire_params *params,
                                 float *key, uint32_t *order, cudaStream_t st)
{
    const long long HW = (long long)m.H * m.W;
    const long long stride = HW > 2048 ? HW / 2048 : 1;
    k_spread_key<<<n, 256, 0, st>>>(m, n, params, stride, key);
    k_rank_desc<<<grid_for(n, 256), 256, 0, st>>>(n, key, order);
    return cudaGetLastError();
}

cudaError_t launch_order(int n, const int32_t *map_of_sim, int nmaps,
                         const int32_t *rank, uint32_t *counts, uint32_t *order,
                         cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, (nmaps + 1) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const int g = grid_for(n, 256);
    k_order_count<<<g, 256, 0, st>>>(n, map_of_sim, nmaps, rank, counts);
    k_order_scan<<<1, 32, 0, st>>>(nmaps + 1, counts);
    k_order_scatter<<<g, 256, 0, st>>>(n, map_of_sim, nmaps, rank, counts, order);
    return cudaGetLastError();
}

cudaError_t launch_fitness(const fire_result *r, int n, int kind, double *out,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_fitness<<<(n + 255) / 256, 256, 0, st>>>(r, n, kind, out);
    return cudaGetLastError();
}

cudaError_t launch_thresholds(const MapDev &m, const double *beta_dev,
                              int64_t *out, cudaStream_t st)
{
    k_thresholds<<<grid_for(8ll * m.H * m.W, 256), 256, 0, st>>>(m, beta_dev,
                                                                 out);
    return cudaGetLastError();
}

cudaError_t launch_probabilities(const MapDev &m, const double *beta_dev,
                                 float *p32, double *p64, cudaStream_t st)
{
    k_probabilities<<<grid_for(8ll * m.H * m.W, 256), 256, 0, st>>>(
        m, beta_dev, p32, p64);
    return cudaGetLastError();
}

cudaError_t launch_features_export(const MapDev &m, float *psi, float *sig,
                                   float *cw, float *sw, uint16_t *cfl,
                                   cudaStream_t st)
{
    k_features_export<<<grid_for((long long)m.H * m.W, 256), 256, 0, st>>>(
        m, psi, sig, cw, sw, cfl);
    return cudaGetLastError();
}

cudaError_t launch_screen_selftest(uint64_t n, uint64_t seed,
                                   unsigned long long *counts,
                                   unsigned long long *max_dp_bits,
                                   cudaStream_t st)
{
    k_screen_selftest<<<152 * 8, 256, 0, st>>>(n, seed, counts, max_dp_bits);
    return cudaGetLastError();
}

cudaError_t launch_philox_blocks(uint64_t n, uint4 ctr, uint2 key,
                                 uint32_t *out, cudaStream_t st)
{
    k_philox_blocks<<<grid_for((long long)n, 256), 256, 0, st>>>(n, ctr, key,
                                                                 out);
    return cudaGetLastError();
}

}  // namespace fire

// Learned surrogate of the automaton: a BF16 convolutional network that maps
// (parameters, landscape, ignition) to a per-cell burn probability on an
// S x S coarse grid, trained on burn fractions the automaton produces and used
// to rank GA offspring before they are simulated.  The paper has no such
// component; the automaton stays the judge of every kept candidate.
//
// Network (NHWC, BF16 activations, FP32 accumulation):
//   layer 1      3x3 conv 16 -> 128, dilation 1, bias, ReLU
//   layers 2..8  3x3 conv 128 -> 128, dilations 1, 2, 4, 8, 16, 32, 64, ReLU
//   head         1x1 conv 128 -> 1, bias, logistic sigmoid
//   loss         mean binary cross-entropy against the burn fraction
// Convolution l: z[p, o] = b[o] + sum_{t, i} W[o, t, i] in[p + off_l(t), i],
// t = 3 t_y + t_x, off_l(t) = ((t_y - 1) d_l, (t_x - 1) d_l), zero outside.
//
// Every convolution is an implicit GEMM on the tcgen05 tile (fire_tc.cuh):
//   forward  D[p][o]      = sum_{(t,i)} in[p + off(t), i] W[o][t][i]
//   dgrad    D[p][i]      = sum_{(t,o)} dz[p - off(t), o] Wt[i][t][o]
//   wgrad    D[o][(t,i)]  = sum_p dz[p, o] in[p + off(t), i]   (MN-major)
// with the bias and ReLU fused into the forward epilogue and the ReLU mask of
// the layer below fused into the dgrad epilogue; the weight gradient is split
// over pixels and summed with FP32 atomics.
//
// Parameters are one flat FP32 vector: per layer W[o][t][i] then b[o], then
// the head's w[128] and b.  Adam keeps FP32 moments and refreshes the BF16
// copy W (same layout) and the transposed copy Wt[i][t][o] of layers 2..8.
#include "fire_internal.h"
#include "fire_tc.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

namespace fire {
// CTAs of the weight-gradient kernel resident per SM (fire_conv_tma.cu).
int wgrad_ctas_per_sm();
}  // namespace fire

using namespace fire;

namespace {

constexpr int kCin = FIRE_NET_CIN;
constexpr int kC = FIRE_NET_C;
constexpr int kL = FIRE_NET_LAYERS;
constexpr int kDil[kL] = {1, 1, 2, 4, 8, 16, 32, 64};
constexpr long long kW0 = (long long)kC * 9 * kCin;   // 18432
constexpr long long kL0 = kW0 + kC;                   // 18560
constexpr long long kWl = (long long)kC * 9 * kC;     // 147456
constexpr long long kLl = kWl + kC;                   // 147584
constexpr long long kHead = kL0 + (kL - 1) * kLl;     // 1051648
constexpr long long kParams = kHead + kC + 1;         // 1051777

__host__ __device__ constexpr long long w_off(int l)
{
    return l == 0 ? 0 : kL0 + (long long)(l - 1) * kLl;
}
__host__ __device__ constexpr long long b_off(int l)
{
    return w_off(l) + (l == 0 ? kW0 : kWl);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ float bf16_to_f(uint16_t u)
{
    return __uint_as_float((uint32_t)u << 16);
}
__device__ __forceinline__ bool bf16_pos(uint32_t u16)
{
    return !(u16 & 0x8000u) && (u16 & 0x7fffu);
}

// Neighbour q = p + (dy, dx) of pixel p (p = (b S + y) S + x); false outside.
__device__ __forceinline__ bool neighbour(int p, int S, int lgS, int dy, int dx,
                                          int &q)
{
    const int y = (p >> lgS) & (S - 1), x = p & (S - 1);
    if ((unsigned)(y + dy) >= (unsigned)S || (unsigned)(x + dx) >= (unsigned)S)
        return false;
    q = p + dy * S + dx;
    return true;
}

// --- forward convolution --------------------------------------------------
template <int Cin> struct ConvFwd {
    static constexpr bool kAMn = false, kBMn = false;
    static constexpr int kK = 9 * Cin;
    const uint16_t *in, *w;
    const float *bias;
    uint16_t *out;
    int M, N, K, S, lgS, d;

    __device__ uint4 a_chunk(int p, int k) const
    {
        const int tap = k / Cin, ci = k % Cin;
        int q;
        if (tap >= 9 || !neighbour(p, S, lgS, (tap / 3 - 1) * d, (tap % 3 - 1) * d, q))
            return make_uint4(0, 0, 0, 0);
        return tc::ld_global16(in + (size_t)q * Cin + ci);
    }
    __device__ uint4 b_chunk(int o, int k) const
    {
        if (k >= kK) return make_uint4(0, 0, 0, 0);
        return tc::ld_global16(w + (size_t)o * kK + k);
    }
    __device__ void epilogue(int p, int n0, const float v[16]) const
    {
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            pk[j] = pack_bf16x2(fmaxf(v[2 * j] + bias[n0 + 2 * j], 0.0f),
                                fmaxf(v[2 * j + 1] + bias[n0 + 2 * j + 1], 0.0f));
        uint4 *o = reinterpret_cast<uint4 *>(out + (size_t)p * kC + n0);
        o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
};

// --- input gradient (layers 2..8), ReLU mask of the layer below fused -----
struct ConvDgrad {
    static constexpr bool kAMn = false, kBMn = false;
    const uint16_t *dz, *wt, *hprev;
    uint16_t *dzprev;
    int M, N, K, S, lgS, d;

    __device__ uint4 a_chunk(int p, int k) const
    {
        const int tap = k >> 7, o = k & (kC - 1);
        int q;
        if (!neighbour(p, S, lgS, -(tap / 3 - 1) * d, -(tap % 3 - 1) * d, q))
            return make_uint4(0, 0, 0, 0);
        return tc::ld_global16(dz + (size_t)q * kC + o);
    }
    __device__ uint4 b_chunk(int i, int k) const
    {
        return tc::ld_global16(wt + (size_t)i * (9 * kC) + k);
    }
    __device__ void epilogue(int p, int n0, const float v[16]) const
    {
        const uint4 *hp = reinterpret_cast<const uint4 *>(hprev + (size_t)p * kC + n0);
        const uint4 h0 = hp[0], h1 = hp[1];
        const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float a = bf16_pos(hw[j] & 0xffffu) ? v[2 * j] : 0.0f;
            const float b = bf16_pos(hw[j] >> 16) ? v[2 * j + 1] : 0.0f;
            pk[j] = pack_bf16x2(a, b);
        }
        uint4 *o = reinterpret_cast<uint4 *>(dzprev + (size_t)p * kC + n0);
        o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
};

// --- weight gradient, both operands MN-major, split over pixels -----------
template <int Cin> struct ConvWgrad {
    static constexpr bool kAMn = true, kBMn = true;
    const uint16_t *dz, *in;
    float *dw;
    int M, N, K, S, lgS, d;

    __device__ uint4 a_chunk(int o, int p) const
    {
        return tc::ld_global16(dz + (size_t)p * kC + o);
    }
    __device__ uint4 b_chunk(int n, int p) const
    {
        const int tap = n / Cin, ci = n % Cin;
        int q;
        if (!neighbour(p, S, lgS, (tap / 3 - 1) * d, (tap % 3 - 1) * d, q))
            return make_uint4(0, 0, 0, 0);
        return tc::ld_global16(in + (size_t)q * Cin + ci);
    }
    __device__ void epilogue(int o, int n0, const float v[16]) const
    {
        float *row = dw + (size_t)o * N;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (n0 + j < N) atomicAdd(row + n0 + j, v[j]);
    }
};

// --- head: logits, probabilities, loss and the per-pixel gradient ---------
// Head: z = wh[kC] + sum_c wh[c] h[p, c], prob = sigmoid(z), the mean BCE
// loss and its per-pixel gradient g.  16 threads per pixel, each taking 8
// channels with one 16-byte load; the partial sums meet by shuffles within
// the 16 lanes (blockDim: a multiple of 32).
__global__ void __launch_bounds__(256)
    k_head(const uint16_t *__restrict__ h, const float *__restrict__ wh, int P,
           const float *__restrict__ target, float inv_count, float *__restrict__ prob,
           float *__restrict__ g, double *__restrict__ loss)
{
    const int cg = threadIdx.x & 15;
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = wh[cg * 8 + j];
    const float bias = wh[kC];
    // warp-wide pixel pairs: lanes 0..15 take pixel 2 pp, lanes 16..31 pixel
    // 2 pp + 1; the loop bound is the same for the whole warp
    const int nw = (gridDim.x * blockDim.x) >> 5;
    float l = 0.0f;
    for (int pp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; 2 * pp < P;
         pp += nw) {
        const int p = 2 * pp + ((threadIdx.x >> 4) & 1);
        float z = 0.0f;
        if (p < P) {
            const uint4 u = *reinterpret_cast<const uint4 *>(h + (size_t)p * kC + cg * 8);
            const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                z = fmaf(bf16_to_f(w4[j] & 0xffffu), w[2 * j], z);
                z = fmaf(bf16_to_f(w4[j] >> 16), w[2 * j + 1], z);
            }
        }
#pragma unroll
        for (int o = 8; o; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (cg == 0 && p < P) {
            z += bias;
            const float y = 1.0f / (1.0f + expf(-z));
            prob[p] = y;
            if (target) {
                const float t = target[p];
                l += (fmaxf(z, 0.0f) - t * z + log1pf(expf(-fabsf(z)))) * inv_count;
                g[p] = (y - t) * inv_count;
            }
        }
    }
    if (target) {
        for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, (double)l);
    }
}

// dz of the top layer, head weight and bias gradients.  Block = 128 threads,
// thread c = channel; each block walks `per` pixels.
// Head gradient: dz[p, c] = g[p] wh[c] where h[p, c] > 0 (else 0), dwh[c] =
// sum_p g[p] h[p, c], dwh[kC] = sum_p g[p]; threads as in k_bias_grad.
__global__ void __launch_bounds__(256)
    k_head_grad(const uint16_t *__restrict__ h, const float *__restrict__ wh,
                const float *__restrict__ g, int P, int per,
                uint16_t *__restrict__ dz, float *__restrict__ dwh)
{
    __shared__ float red[16][kC + 2];
    const int cg = threadIdx.x & 15, pl = threadIdx.x >> 4;
    const int p0 = blockIdx.x * per, p1 = min(P, p0 + per);
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = wh[cg * 8 + j];
    float aw[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float ab = 0.0f;
    for (int p = p0 + pl; p < p1; p += 16) {
        const float gp = g[p];
        const size_t off = (size_t)p * kC + cg * 8;
        const uint4 u = *reinterpret_cast<const uint4 *>(h + off);
        const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
        uint32_t o4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint16_t lo = (uint16_t)(w4[j] & 0xffffu), hi = (uint16_t)(w4[j] >> 16);
            aw[2 * j] = fmaf(gp, bf16_to_f(lo), aw[2 * j]);
            aw[2 * j + 1] = fmaf(gp, bf16_to_f(hi), aw[2 * j + 1]);
            const uint32_t dl = __bfloat16_as_ushort(
                __float2bfloat16_rn(bf16_pos(lo) ? gp * w[2 * j] : 0.0f));
            const uint32_t dh = __bfloat16_as_ushort(
                __float2bfloat16_rn(bf16_pos(hi) ? gp * w[2 * j + 1] : 0.0f));
            o4[j] = dl | (dh << 16);
        }
        *reinterpret_cast<uint4 *>(dz + off) = make_uint4(o4[0], o4[1], o4[2], o4[3]);
        ab += gp;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[pl][cg * 8 + j] = aw[j];
    if (cg == 0) red[pl][kC] = ab;
    __syncthreads();
    if (threadIdx.x <= kC) {
        float sum = 0.0f;
#pragma unroll
        for (int r = 0; r < 16; ++r) sum += red[r][threadIdx.x];
        atomicAdd(dwh + threadIdx.x, sum);
    }
}

// Bias gradient: db[o] = sum_p dz[p, o].  A block of 256 threads takes
// `per` pixels, 16 at a time: thread (pl, cg) reads channels 8 cg .. 8 cg + 7
// of pixel pl with one 16-byte load; the 16 pixel lanes' partial sums are
// added in shared memory and once per block into db.
__global__ void __launch_bounds__(256)
    k_bias_grad(const uint16_t *__restrict__ dz, int P, int per, float *__restrict__ db)
{
    __shared__ float red[16][kC + 1];
    const int cg = threadIdx.x & 15, pl = threadIdx.x >> 4;
    const int p0 = blockIdx.x * per, p1 = min(P, p0 + per);
    float a[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int p = p0 + pl; p < p1; p += 16) {
        const uint4 u = *reinterpret_cast<const uint4 *>(dz + (size_t)p * kC + cg * 8);
        const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            a[2 * j] += bf16_to_f(w4[j] & 0xffffu);
            a[2 * j + 1] += bf16_to_f(w4[j] >> 16);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[pl][cg * 8 + j] = a[j];
    __syncthreads();
    if (threadIdx.x < kC) {
        float sum = 0.0f;
#pragma unroll
        for (int r = 0; r < 16; ++r) sum += red[r][threadIdx.x];
        atomicAdd(db + threadIdx.x, sum);
    }
}

// BF16 copies of parameter i: the flat copy and, for the weights of layers
// 2..8, the transposed copy Wt[i][t][o].
__device__ __forceinline__ void write_copies(long long i, float th,
                                             uint16_t *__restrict__ wb,
                                             uint16_t *__restrict__ wt)
{
    const uint16_t u = __bfloat16_as_ushort(__float2bfloat16_rn(th));
    wb[i] = u;
    if (i >= kL0 && i < kHead) {
        const long long j = i - kL0;
        const int l = (int)(j / kLl);
        const long long r = j - (long long)l * kLl;
        if (r < kWl) {
            const int o = (int)(r / (9 * kC)), rem = (int)(r % (9 * kC));
            const int tap = rem / kC, ci = rem % kC;
            wt[(long long)l * kWl + (long long)ci * 9 * kC + tap * kC + o] = u;
        }
    }
}

__global__ void k_sync_copies(const float *__restrict__ theta, uint16_t *__restrict__ wb,
                              uint16_t *__restrict__ wt)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < kParams;
         i += (long long)gridDim.x * blockDim.x)
        write_copies(i, theta[i], wb, wt);
}

// Adam (Kingma and Ba): c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ grad,
                       float *__restrict__ m, float *__restrict__ v,
                       uint16_t *__restrict__ wb, uint16_t *__restrict__ wt,
                       float lr, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < kParams;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float th = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
        theta[i] = th;
        write_copies(i, th, wb, wt);
    }
}

// --- inputs and labels ----------------------------------------------------
__global__ void k_planes(int H, int W, int S, const uint8_t *__restrict__ veg,
                         const float *__restrict__ slope,
                         const float *__restrict__ aspect,
                         const float *__restrict__ wind, float *__restrict__ planes)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S * S) return;
    const int ci = c / S, cj = c % S, fr = H / S, fc = W / S;
    int cnt[5] = {0, 0, 0, 0, 0};
    float sl = 0.f, sa = 0.f, ca = 0.f, sw = 0.f, cw = 0.f;
    const float rad = 0.017453292519943295f;
    for (int r = ci * fr; r < (ci + 1) * fr; ++r)
        for (int q = cj * fc; q < (cj + 1) * fc; ++q) {
            const size_t i = (size_t)r * W + q;
            cnt[min((int)veg[i], 4)]++;
            sl += slope[i];
            float s, co;
            sincosf(aspect[i] * rad, &s, &co);
            sa += s;
            ca += co;
            sincosf(wind[i] * rad, &s, &co);
            sw += s;
            cw += co;
        }
    const float inv = 1.0f / (float)(fr * fc);
    float *o = planes + (size_t)c * 10;
    for (int k = 0; k < 5; ++k) o[k] = (float)cnt[k] * inv;
    o[5] = sl * inv / 45.0f;
    o[6] = sa * inv;
    o[7] = ca * inv;
    o[8] = sw * inv;
    o[9] = cw * inv;
}

__global__ void k_inputs(int S, int H, int W, int n, const float *__restrict__ planes,
                         const fire_params *__restrict__ params,
                         const fire_cell *__restrict__ ign, uint16_t *__restrict__ x)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * S * S) return;
    const int s = (int)(t / ((long long)S * S));
    const int c = (int)(t - (long long)s * S * S);
    const int ci = c / S, cj = c % S;
    const float *pl = planes + (size_t)c * 10;
    float v[16];
    for (int k = 0; k < 10; ++k) v[k] = pl[k];
    const fire_cell g = ign[s];
    v[10] = (g.row / (H / S) == ci && g.col / (W / S) == cj) ? 1.0f : 0.0f;
    for (int j = 0; j < 5; ++j) v[11 + j] = (float)(params[s].b[j] / 10.0);
    uint32_t pk[8];
    for (int j = 0; j < 8; ++j) pk[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
    uint4 *o = reinterpret_cast<uint4 *>(x + (size_t)t * kCin);
    o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// Burn fractions per coarse cell from tile-major burnt words (reps per group).
__global__ void k_labels(const uint32_t *__restrict__ bits, long long words_per_sim,
                         int TW, int H, int W, int S, int groups, int reps,
                         float *__restrict__ out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)groups * S * S) return;
    const int g = (int)(t / ((long long)S * S));
    const int c = (int)(t - (long long)g * S * S);
    const int ci = c / S, cj = c % S, fr = H / S, fc = W / S;
    unsigned cnt = 0;
    for (int r = 0; r < reps; ++r) {
        const uint32_t *b = bits + (long long)(g * reps + r) * words_per_sim;
        for (int R = ci * fr; R < (ci + 1) * fr; ++R) {
            const int ti = R >> 5, row = R & 31;
            int q = cj * fc;
            const int qe = (cj + 1) * fc;
            while (q < qe) {
                const int lo = q & 31, cntb = min(32 - lo, qe - q);
                const uint32_t mask =
                    (cntb == 32 ? 0xffffffffu : ((1u << cntb) - 1u)) << lo;
                cnt += __popc(b[((long long)ti * TW + (q >> 5)) * 32 + row] & mask);
                q += cntb;
            }
        }
    }
    out[t] = (float)cnt / (float)(reps * fr * fc);
}

__global__ void k_expand(int n, int reps, const fire_params *__restrict__ gp,
                         const fire_cell *__restrict__ gi, uint64_t seed0,
                         fire_params *__restrict__ sp, fire_cell *__restrict__ si,
                         uint64_t *__restrict__ ss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sp[i] = gp[i / reps];
    si[i] = gi[i / reps];
    ss[i] = seed0 + (uint64_t)i;
}

// --- screening --------------------------------------------------------------
// Predicted Eq. 2 fitness with expected set sizes; one block per candidate.
__global__ void k_pred_fitness(int SS, const float *__restrict__ prob,
                               const float *__restrict__ tfrac, double cells,
                               int kind, double *__restrict__ pred)
{
    const float *q = prob + (size_t)blockIdx.x * SS;
    double sq = 0.0, sqt = 0.0, st = 0.0;
    for (int c = threadIdx.x; c < SS; c += blockDim.x) {
        const double qc = q[c], tc_ = tfrac[c];
        sq += qc;
        sqt += qc * tc_;
        st += tc_;
    }
    __shared__ double red[3][256];
    red[0][threadIdx.x] = sq;
    red[1][threadIdx.x] = sqt;
    red[2][threadIdx.x] = st;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sim = cells * red[0][0], inter = cells * red[1][0];
        const double tgt = cells * red[2][0];
        const double num = sim + tgt - 2.0 * inter;
        const double den = kind == 0 ? tgt : sim + tgt - inter;
        pred[blockIdx.x] = num / den;
    }
}

// Rank by predicted fitness (lower first; NaN last; ties to the lower index).
__global__ void k_rank_keep(int n, const double *__restrict__ pred, int keep,
                            int32_t *__restrict__ keep_idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double fi = pred[i];
    const bool ni = fi != fi;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        const double fj = pred[j];
        const bool nj = fj != fj;
        const bool before = (ni != nj) ? ni : (!ni && fj != fi ? fj < fi : j < i);
        rank += before;
    }
    if (rank < keep) keep_idx[rank] = i;
}

}  // namespace

// ---------------------------------------------------------------------------

struct fire_net {
    fire_ctx *ctx = nullptr;
    int S = 0, lgS = 0, max_batch = 0;
    void *mem = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    uint16_t *wb = nullptr, *wt = nullptr;
    uint16_t *h[kL] = {};
    uint16_t *dz[kL] = {};
    float *prob = nullptr, *g = nullptr;
    double *loss = nullptr;
    int step = 0;
};

namespace {

int net_err(fire_ctx *ctx, const char *what)
{
    return set_err(ctx, FIRE_EINVAL, "%s", what);
}

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Forward over n <= max_batch samples of x; activations stay in net->h.
cudaError_t net_forward(fire_net *net, int n, const uint16_t *x, uint32_t *err,
                        cudaStream_t st)
{
    const int S = net->S, lgS = net->lgS;
    const int M = n * S * S;
    cudaError_t e;
    if (S >= 16) {
        e = launch_conv1_tma(x, net->wb + w_off(0), net->theta + b_off(0), net->h[0],
                             n, S, lgS, err, st);
        if (e != cudaSuccess) return e;
    } else {
        ConvFwd<kCin> p{x, net->wb + w_off(0), net->theta + b_off(0), net->h[0],
                        M, kC, 192, S, lgS, kDil[0]};
        e = tc::launch_tc_tile<128>(p, 1, err, st);
        if (e != cudaSuccess) return e;
    }
    for (int l = 1; l < kL; ++l) {
        if (S >= 16) {
            e = launch_conv_tma(0, net->h[l - 1], net->wb + w_off(l),
                                net->theta + b_off(l), nullptr, net->h[l], n, S, lgS,
                                kDil[l], err, st);
        } else {
            ConvFwd<kC> p{net->h[l - 1], net->wb + w_off(l), net->theta + b_off(l),
                          net->h[l], M, kC, 9 * kC, S, lgS, kDil[l]};
            e = tc::launch_tc_tile<128>(p, 1, err, st);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int wgrad_split(int nt_n, int kslabs, int ctas_per_sm = 3)
{
    int s = (152 * ctas_per_sm) / nt_n;
    if (s < 1) s = 1;
    if (s > kslabs) s = kslabs;
    return s;
}

}  // namespace

extern "C" {

int64_t fire_net_param_count(void) { return kParams; }

int fire_net_create(fire_ctx *ctx, int S, int max_batch, fire_net **out)
{
    if (!ctx) return FIRE_EINVAL;
    if (!out || S < 8 || S > 1024 || (S & (S - 1)) || max_batch < 1 ||
        (long long)max_batch * S * S > (1ll << 24))
        return net_err(ctx, "fire_net_create: S must be a power of two in "
                            "[8, 1024] and max_batch * S * S <= 2^24");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    fire_net *net = new fire_net;
    net->ctx = ctx;
    net->S = S;
    net->lgS = ilog2(S);
    net->max_batch = max_batch;
    const size_t P = (size_t)kParams;
    const size_t pix = (size_t)max_batch * S * S;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_th = take(P * 4), o_gr = take(P * 4), o_m = take(P * 4),
                 o_v = take(P * 4), o_wb = take(P * 2),
                 o_wt = take((size_t)(kL - 1) * kWl * 2);
    size_t o_h[kL], o_dz[kL];
    for (int l = 0; l < kL; ++l) o_h[l] = take(pix * kC * 2);
    for (int l = 0; l < kL; ++l) o_dz[l] = take(pix * kC * 2);
    const size_t o_prob = take(pix * 4), o_g = take(pix * 4), o_loss = take(8);
    cudaError_t e = cudaMalloc(&net->mem, off);
    if (e != cudaSuccess) {
        delete net;
        return set_err(ctx, FIRE_ENOMEM, "surrogate buffers (%zu B)", off);
    }
    char *b = (char *)net->mem;
    net->theta = (float *)(b + o_th);
    net->grad = (float *)(b + o_gr);
    net->m = (float *)(b + o_m);
    net->v = (float *)(b + o_v);
    net->wb = (uint16_t *)(b + o_wb);
    net->wt = (uint16_t *)(b + o_wt);
    for (int l = 0; l < kL; ++l) {
        net->h[l] = (uint16_t *)(b + o_h[l]);
        net->dz[l] = (uint16_t *)(b + o_dz[l]);
    }
    net->prob = (float *)(b + o_prob);
    net->g = (float *)(b + o_g);
    net->loss = (double *)(b + o_loss);
    e = cudaMemsetAsync(net->mem, 0, o_h[0], ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(net->mem);
        delete net;
        return cuda_err(ctx, e, "surrogate clear");
    }
    *out = net;
    return FIRE_OK;
}

void fire_net_free(fire_net *net)
{
    if (!net) return;
    if (net->mem) {
        cudaSetDevice(net->ctx->device);
        cudaFree(net->mem);
    }
    delete net;
}

int fire_net_set_params(fire_ctx *ctx, fire_net *net, const float *params,
                        uint32_t flags)
{
    if (!ctx) return FIRE_EINVAL;
    if (!net || !params) return net_err(ctx, "fire_net_set_params: NULL argument");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t P = (size_t)kParams;
    CUDA_TRY(ctx, cudaMemcpyAsync(net->theta, params, P * 4,
                                  (flags & FIRE_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice
                                                             : cudaMemcpyHostToDevice,
                                  ctx->stream), "params copy");
    CUDA_TRY(ctx, cudaMemsetAsync(net->m, 0, P * 4, ctx->stream), "adam m");
    CUDA_TRY(ctx, cudaMemsetAsync(net->v, 0, P * 4, ctx->stream), "adam v");
    net->step = 0;
    k_sync_copies<<<152 * 4, 256, 0, ctx->stream>>>(net->theta, net->wb, net->wt);
    CUDA_TRY(ctx, cudaGetLastError(), "weight copies");
    return fire_sync(ctx);
}

int fire_net_get(fire_ctx *ctx, const fire_net *net, int which, uint32_t flags,
                 float *out)
{
    if (!ctx) return FIRE_EINVAL;
    if (!net || !out || which < 0 || which > 3)
        return net_err(ctx, "fire_net_get: bad arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const float *src = which == 0 ? net->theta
                     : which == 1 ? net->grad
                     : which == 2 ? net->m : net->v;
    CUDA_TRY(ctx, cudaMemcpyAsync(out, src, (size_t)kParams * 4,
                                  (flags & FIRE_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice
                                                             : cudaMemcpyDeviceToHost,
                                  ctx->stream), "params out");
    return fire_sync(ctx);
}

int fire_net_forward(fire_ctx *ctx, fire_net *net, int n, const uint16_t *x,
                     uint32_t flags, float *prob)
{
    FIRE_NVTX("fire_net_forward");
    if (!ctx) return FIRE_EINVAL;
    if (!net || n < 0 || !(flags & FIRE_DEVICE_PTRS) || (n && (!x || !prob)) ||
        ((uintptr_t)x & 15))
        return net_err(ctx, "fire_net_forward: bad arguments (device pointers "
                            "required, x 16-byte aligned)");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const int SS = net->S * net->S;
    for (int s0 = 0; s0 < n; s0 += net->max_batch) {
        const int nb = n - s0 < net->max_batch ? n - s0 : net->max_batch;
        CUDA_TRY(ctx, net_forward(net, nb, x + (size_t)s0 * SS * kCin,
                                  ctx->counter + 1, ctx->stream), "surrogate forward");
        const int P = nb * SS;
        k_head<<<(P + 255) / 256, 256, 0, ctx->stream>>>(
            net->h[kL - 1], net->theta + kHead, P, nullptr, 0.0f,
            prob + (size_t)s0 * SS, nullptr, nullptr);
        CUDA_TRY(ctx, cudaGetLastError(), "surrogate head");
    }
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_net_backward(fire_ctx *ctx, fire_net *net, int n, const uint16_t *x,
                      const float *target, uint32_t flags, double *loss)
{
    FIRE_NVTX("fire_net_backward");
    if (!ctx) return FIRE_EINVAL;
    if (!net || n < 1 || n > net->max_batch || !x || !target ||
        !(flags & FIRE_DEVICE_PTRS) || ((uintptr_t)x & 15))
        return net_err(ctx, "fire_net_backward: bad arguments (1 <= n <= "
                            "max_batch, device pointers, x 16-byte aligned)");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    cudaStream_t st = ctx->stream;
    uint32_t *err = ctx->counter + 1;
    const int S = net->S, lgS = net->lgS, P = n * S * S;
    CUDA_TRY(ctx, net_forward(net, n, x, err, st), "surrogate forward");
    CUDA_TRY(ctx, cudaMemsetAsync(net->loss, 0, 8, st), "loss clear");
    CUDA_TRY(ctx, cudaMemsetAsync(net->grad, 0, (size_t)kParams * 4, st), "grad clear");
    k_head<<<(P + 255) / 256, 256, 0, st>>>(net->h[kL - 1], net->theta + kHead, P,
                                            target, 1.0f / (float)P, net->prob,
                                            net->g, net->loss);
    CUDA_TRY(ctx, cudaGetLastError(), "surrogate head");
    const int per = 256;
    const int nblk = (P + per - 1) / per;
    k_head_grad<<<nblk, 256, 0, st>>>(net->h[kL - 1], net->theta + kHead, net->g, P,
                                     per, net->dz[kL - 1], net->grad + kHead);
    CUDA_TRY(ctx, cudaGetLastError(), "head gradient");
    const int kslabs = P / 64;
    for (int l = kL - 1; l >= 0; --l) {
        cudaError_t e;
        if (l == 0) {
            ConvWgrad<kCin> p{net->dz[0], x, net->grad + w_off(0), kC, 9 * kCin, P,
                              S, lgS, kDil[0]};
            e = tc::launch_tc_tile<64>(p, wgrad_split(3, kslabs), err, st);
        } else if (S >= 16) {
            e = launch_wgrad_tma(net->dz[l], net->h[l - 1], net->grad + w_off(l), n, S,
                                 lgS, kDil[l],
                                 wgrad_split(9, kslabs, wgrad_ctas_per_sm()), err, st);
        } else {
            ConvWgrad<kC> p{net->dz[l], net->h[l - 1], net->grad + w_off(l), kC,
                            9 * kC, P, S, lgS, kDil[l]};
            e = tc::launch_tc_tile<128>(p, wgrad_split(9, kslabs), err, st);
        }
        CUDA_TRY(ctx, e, "weight gradient");
        k_bias_grad<<<nblk, 256, 0, st>>>(net->dz[l], P, per, net->grad + b_off(l));
        CUDA_TRY(ctx, cudaGetLastError(), "bias gradient");
        if (l > 0) {
            const uint16_t *wt = net->wt + (size_t)(l - 1) * kWl;
            if (S >= 16) {
                CUDA_TRY(ctx, launch_conv_tma(1, net->dz[l], wt, nullptr, net->h[l - 1],
                                              net->dz[l - 1], n, S, lgS, kDil[l], err,
                                              st), "input gradient");
            } else {
                ConvDgrad p{net->dz[l], wt, net->h[l - 1], net->dz[l - 1], P, kC,
                            9 * kC, S, lgS, kDil[l]};
                CUDA_TRY(ctx, tc::launch_tc_tile<128>(p, 1, err, st), "input gradient");
            }
        }
    }
    if (loss)
        CUDA_TRY(ctx, cudaMemcpyAsync(loss, net->loss, 8, cudaMemcpyDeviceToDevice, st),
                 "loss out");
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_net_adam(fire_ctx *ctx, fire_net *net, float lr, uint32_t flags)
{
    FIRE_NVTX("fire_net_adam");
    if (!ctx) return FIRE_EINVAL;
    if (!net || !(lr >= 0.0f)) return net_err(ctx, "fire_net_adam: bad arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    net->step += 1;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, net->step));
    const double c2 = 1.0 / (1.0 - std::pow(0.999, net->step));
    k_adam<<<152 * 8, 256, 0, ctx->stream>>>(net->theta, net->grad, net->m, net->v,
                                            net->wb, net->wt, lr, (float)c1,
                                            (float)c2);
    CUDA_TRY(ctx, cudaGetLastError(), "adam");
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_net_buffer(fire_ctx *ctx, const fire_net *net, int which, int layer, int n,
                    uint32_t flags, void *out)
{
    if (!ctx) return FIRE_EINVAL;
    if (!net || !out || which < 0 || which > 2 || layer < 0 || layer >= kL || n < 1 ||
        n > net->max_batch || !(flags & FIRE_DEVICE_PTRS))
        return net_err(ctx, "fire_net_buffer: bad arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const size_t pix = (size_t)n * net->S * net->S;
    const void *src = which == 0 ? (const void *)net->h[layer]
                    : which == 1 ? (const void *)net->dz[layer]
                                 : (const void *)net->prob;
    const size_t bytes = which == 2 ? pix * 4 : pix * kC * 2;
    CUDA_TRY(ctx, cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice,
                                  ctx->stream), "buffer copy");
    return fire_sync(ctx);
}

int fire_net_planes(fire_ctx *ctx, int H, int W, int S, const uint8_t *veg,
                    const float *slope, const float *aspect, const float *wind,
                    uint32_t flags, float *planes)
{
    FIRE_NVTX("fire_net_planes");
    if (!ctx) return FIRE_EINVAL;
    if (S < 1 || H < S || W < S || H % S || W % S || !veg || !slope || !aspect ||
        !wind || !planes || !(flags & FIRE_DEVICE_PTRS))
        return net_err(ctx, "fire_net_planes: bad arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    k_planes<<<(S * S + 127) / 128, 128, 0, ctx->stream>>>(H, W, S, veg, slope, aspect,
                                                          wind, planes);
    CUDA_TRY(ctx, cudaGetLastError(), "planes");
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_net_inputs(fire_ctx *ctx, int S, int H, int W, int n, const float *planes,
                    const fire_params *params, const fire_cell *ign, uint32_t flags,
                    uint16_t *x)
{
    FIRE_NVTX("fire_net_inputs");
    if (!ctx) return FIRE_EINVAL;
    if (S < 1 || H < S || W < S || H % S || W % S || n < 0 ||
        (n && (!planes || !params || !ign || !x)) || !(flags & FIRE_DEVICE_PTRS) ||
        ((uintptr_t)x & 15))
        return net_err(ctx, "fire_net_inputs: bad arguments");
    if (n == 0) return FIRE_OK;
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const long long T = (long long)n * S * S;
    k_inputs<<<(unsigned)((T + 255) / 256), 256, 0, ctx->stream>>>(S, H, W, n, planes,
                                                                   params, ign, x);
    CUDA_TRY(ctx, cudaGetLastError(), "inputs");
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_net_labels(fire_ctx *ctx, const fire_map *map, int S, int groups, int reps,
                    const fire_params *params, const fire_cell *ign, uint64_t seed,
                    uint32_t max_steps, uint32_t flags, float *labels,
                    fire_result *results)
{
    FIRE_NVTX("fire_net_labels");
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(map) || S < 1 || groups < 0 || reps < 1 ||
        map->dev.H % S || map->dev.W % S || !(flags & FIRE_DEVICE_PTRS) ||
        (groups && (!params || !ign || !labels)))
        return net_err(ctx, "fire_net_labels: bad arguments");
    if (groups == 0) return FIRE_OK;
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const MapDev &md = map->dev;
    const long long wps = (long long)md.ntiles * 32;
    // groups per chunk: keep the burnt words under 1 GiB
    long long gper = (1ll << 28) / (wps * reps);
    if (gper < 1) gper = 1;
    if (gper > groups) gper = groups;
    const long long nper = gper * reps;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += round16(bytes);
        return o;
    };
    const size_t o_p = take(nper * sizeof(fire_params)), o_i = take(nper * sizeof(fire_cell));
    const size_t o_s = take(nper * 8), o_r = take(nper * sizeof(fire_result));
    const size_t o_b = take((size_t)nper * wps * 4);
    rc = grow_device(ctx, &ctx->staging, &ctx->staging_bytes, off, "label scratch");
    if (rc) return rc;
    char *b = (char *)ctx->staging;
    fire_params *sp = (fire_params *)(b + o_p);
    fire_cell *si = (fire_cell *)(b + o_i);
    uint64_t *ss = (uint64_t *)(b + o_s);
    fire_result *sr = (fire_result *)(b + o_r);
    uint32_t *sb = (uint32_t *)(b + o_b);
    for (long long g0 = 0; g0 < groups; g0 += gper) {
        const int gn = (int)(groups - g0 < gper ? groups - g0 : gper);
        const int n = gn * reps;
        k_expand<<<(n + 255) / 256, 256, 0, ctx->stream>>>(
            n, reps, params + g0, ign + g0, seed + (uint64_t)g0 * reps, sp, si, ss);
        CUDA_TRY(ctx, cudaGetLastError(), "label expand");
        rc = launch_batch(ctx, map, n, sp, si, ss, max_steps, flags & FIRE_CELL_UNIFORM,
                          results ? results + g0 * reps : sr, nullptr, sb);
        if (rc) return rc;
        const long long T = (long long)gn * S * S;
        k_labels<<<(unsigned)((T + 255) / 256), 256, 0, ctx->stream>>>(
            sb, wps, md.TW, md.H, md.W, S, gn, reps, labels + (size_t)g0 * S * S);
        CUDA_TRY(ctx, cudaGetLastError(), "labels");
    }
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_net_target_frac(fire_ctx *ctx, const fire_map *map, int S, uint32_t flags,
                         float *frac)
{
    if (!ctx) return FIRE_EINVAL;
    if (!valid_map(map) || S < 1 || map->dev.H % S || map->dev.W % S || !frac ||
        !(flags & FIRE_DEVICE_PTRS))
        return net_err(ctx, "fire_net_target_frac: bad arguments");
    int rc = ensure_device(ctx);
    if (rc) return rc;
    const MapDev &md = map->dev;
    k_labels<<<(S * S + 255) / 256, 256, 0, ctx->stream>>>(
        md.tgt, (long long)md.ntiles * 32, md.TW, md.H, md.W, S, 1, 1, frac);
    CUDA_TRY(ctx, cudaGetLastError(), "target fractions");
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

int fire_net_screen(fire_ctx *ctx, int S, int n, const float *prob,
                    const float *target_frac, double cells_per_coarse, int kind,
                    int keep, uint32_t flags, double *pred, int32_t *keep_idx)
{
    FIRE_NVTX("fire_net_screen");
    if (!ctx) return FIRE_EINVAL;
    if (S < 1 || n < 0 || keep < 0 || keep > n || (kind != 0 && kind != 1) ||
        !(cells_per_coarse > 0) || !(flags & FIRE_DEVICE_PTRS) ||
        (n && (!prob || !target_frac || !pred)) || (keep && !keep_idx))
        return net_err(ctx, "fire_net_screen: bad arguments");
    if (n == 0) return FIRE_OK;
    int rc = ensure_device(ctx);
    if (rc) return rc;
    k_pred_fitness<<<n, 256, 0, ctx->stream>>>(S * S, prob, target_frac,
                                               cells_per_coarse, kind, pred);
    CUDA_TRY(ctx, cudaGetLastError(), "predicted fitness");
    if (keep) {
        k_rank_keep<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, pred, keep, keep_idx);
        CUDA_TRY(ctx, cudaGetLastError(), "rank");
    }
    if (flags & FIRE_SYNC) return fire_sync(ctx);
    return FIRE_OK;
}

}  // extern "C"

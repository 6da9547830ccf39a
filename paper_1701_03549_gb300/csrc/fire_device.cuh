// Device arithmetic of the fire-spread automaton (arXiv:1701.03549):
// counter-based random numbers (Sec. 2.3), the ignition probability of Eq. 1
// evaluated exactly in double precision, and the single-precision screen that
// decides almost every trial without it.
//
// Double-precision definition of a trial threshold (identical, operation by
// operation, to what the test oracle computes independently):
//   z = ((((b0 + b1*If) + b2*psi) + b3*omega_d) + b4*sigma_d)
//   p = 1 / (1 + exp(-z)),  T = floor(p * 2^32) in [0, 2^32]
// with every step a single IEEE-754 double operation (no contraction), exp
// evaluated by Cody-Waite reduction and a degree-13 Taylor series, and
// omega_d = cos(phi_w - 45 d) expanded with the exact values of cos and sin at
// multiples of 45 degrees.  A trial succeeds iff u < T.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fire {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Round:
//   (hi0, lo0) = M0 * x0, (hi1, lo1) = M1 * x2,
//   x' = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0),
// with the key advanced by the Weyl increments between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint32_t x0, uint32_t x1,
                                               uint32_t x2, uint32_t x3,
                                               uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * x0;
        const uint32_t hi0 = __umulhi(kPhiloxM0, x0);
        const uint32_t lo1 = kPhiloxM1 * x2;
        const uint32_t hi1 = __umulhi(kPhiloxM1, x2);
        const uint32_t n0 = hi1 ^ x1 ^ k0;
        const uint32_t n2 = hi0 ^ x3 ^ k1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return make_uint4(x0, x1, x2, x3);
}

// The same block function with the key schedule precomputed: rk[j] holds the
// round keys (k0 + 2j W0, k1 + 2j W1) in .x, .y and those of round 2j + 1 in
// .z, .w.  Every trial of one simulation uses the same key, so the schedule
// is computed once per simulation instead of once per block.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint32_t x0, uint32_t x1,
                                                  uint32_t x2, uint32_t x3,
                                                  const uint4 *rk)
{
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const uint4 k = rk[j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t k0 = h ? k.z : k.x, k1 = h ? k.w : k.y;
            const uint32_t lo0 = kPhiloxM0 * x0;
            const uint32_t hi0 = __umulhi(kPhiloxM0, x0);
            const uint32_t lo1 = kPhiloxM1 * x2;
            const uint32_t hi1 = __umulhi(kPhiloxM1, x2);
            const uint32_t n0 = hi1 ^ x1 ^ k0;
            const uint32_t n2 = hi0 ^ x3 ^ k1;
            x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
        }
    }
    return make_uint4(x0, x1, x2, x3);
}

// Round keys of philox4x32_10_rk for the key (k0, k1).
__host__ __device__ inline void philox_round_keys(uint32_t k0, uint32_t k1,
                                                  uint4 rk[5])
{
    for (uint32_t j = 0; j < 5; ++j) {
        const uint32_t r0 = 2u * j, r1 = 2u * j + 1u;
        rk[j] = make_uint4(k0 + r0 * kPhiloxW0, k1 + r0 * kPhiloxW1,
                           k0 + r1 * kPhiloxW0, k1 + r1 * kPhiloxW1);
    }
}

// ---------------------------------------------------------------------------
// Double-precision exp on |x| <= 40: x = k ln2 + r, |r| <= ln2/2, Taylor
// series of e^r to degree 13, times 2^k.  ln2 is split into a 40-bit head
// (k * head exact) and a tail.
namespace spec {

constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kLn2Head = 0x1.62e42fefa4000p-1;
constexpr double kLn2Tail = -0x1.8432a1b0e2634p-43;
constexpr double kPiOver180 = 0x1.1df46a2529d39p-6;
constexpr double kHalfSqrt2 = 0x1.6a09e667f3bcdp-1;

// 1/n! rounded to nearest
constexpr double kF2 = 0x1.0000000000000p-1;
constexpr double kF3 = 0x1.5555555555555p-3;
constexpr double kF4 = 0x1.5555555555555p-5;
constexpr double kF5 = 0x1.1111111111111p-7;
constexpr double kF6 = 0x1.6c16c16c16c17p-10;
constexpr double kF7 = 0x1.a01a01a01a01ap-13;
constexpr double kF8 = 0x1.a01a01a01a01ap-16;
constexpr double kF9 = 0x1.71de3a556c734p-19;
constexpr double kF10 = 0x1.27e4fb7789f5cp-22;
constexpr double kF11 = 0x1.ae64567f544e4p-26;
constexpr double kF12 = 0x1.1eed8eff8d898p-29;
constexpr double kF13 = 0x1.6124613a86d09p-33;
constexpr double kF14 = 0x1.93974a8c07c9dp-37;
constexpr double kF15 = 0x1.ae7f3e733b81fp-41;
constexpr double kF16 = 0x1.ae7f3e733b81fp-45;
constexpr double kF17 = 0x1.952c77030ad4ap-49;
constexpr double kF18 = 0x1.6827863b97d97p-53;
constexpr double kF19 = 0x1.2f49b46814157p-57;

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

static __device__ __noinline__ double exp_small(double x)
{
    const double k = rint(mul(x, kInvLn2));
    const double r = sub(sub(x, mul(k, kLn2Head)), mul(k, kLn2Tail));
    double s = kF13;
    s = add(mul(s, r), kF12);
    s = add(mul(s, r), kF11);
    s = add(mul(s, r), kF10);
    s = add(mul(s, r), kF9);
    s = add(mul(s, r), kF8);
    s = add(mul(s, r), kF7);
    s = add(mul(s, r), kF6);
    s = add(mul(s, r), kF5);
    s = add(mul(s, r), kF4);
    s = add(mul(s, r), kF3);
    s = add(mul(s, r), kF2);
    s = add(mul(s, r), 1.0);
    s = add(mul(s, r), 1.0);
    const long long ik = (long long)k;
    const double two_k = __longlong_as_double((ik + 1023LL) << 52);
    return mul(s, two_k);
}

// T = floor(2^32 / (1 + exp(-z))) in [0, 2^32].
static __device__ __noinline__ uint64_t threshold_of_z(double z)
{
    if (!(z > -40.0)) return 0ull;
    if (z >= 40.0) return 1ull << 32;
    const double e = exp_small(-z);
    const double p = __ddiv_rn(1.0, add(1.0, e));
    return (uint64_t)floor(mul(p, 4294967296.0));
}

// p = 1 / (1 + exp(-z)) in double precision (debug exports); the argument of
// exp is clamped to [-700, 700], where 2^k stays a normal double.
__device__ __forceinline__ double logistic(double z)
{
    if (z != z) return z;
    const double zc = fmin(fmax(z, -700.0), 700.0);
    const double e = exp_small(-zc);
    return __ddiv_rn(1.0, add(1.0, e));
}

// cos / sin of an angle in degrees: y = deg - 90 k, |y| <= 45, Taylor series
// in radians to degree 18 / 19, rotated by the quadrant k mod 4.
__device__ __forceinline__ double cos_series(double t)
{
    const double s2 = mul(t, t);
    double c = -kF18;
    c = add(mul(c, s2), kF16);
    c = add(mul(c, s2), -kF14);
    c = add(mul(c, s2), kF12);
    c = add(mul(c, s2), -kF10);
    c = add(mul(c, s2), kF8);
    c = add(mul(c, s2), -kF6);
    c = add(mul(c, s2), kF4);
    c = add(mul(c, s2), -kF2);
    c = add(mul(c, s2), 1.0);
    return c;
}

__device__ __forceinline__ double sin_series(double t)
{
    const double s2 = mul(t, t);
    double c = -kF19;
    c = add(mul(c, s2), kF17);
    c = add(mul(c, s2), -kF15);
    c = add(mul(c, s2), kF13);
    c = add(mul(c, s2), -kF11);
    c = add(mul(c, s2), kF9);
    c = add(mul(c, s2), -kF7);
    c = add(mul(c, s2), kF5);
    c = add(mul(c, s2), -kF3);
    c = add(mul(c, s2), 1.0);
    return mul(t, c);
}

__device__ __forceinline__ void reduce_deg(double deg, double &t, int &q)
{
    const double k = rint(__ddiv_rn(deg, 90.0));
    const double y = sub(deg, mul(k, 90.0));
    t = mul(y, kPiOver180);
    const long long kq = (long long)k;
    q = (int)(((kq % 4) + 4) % 4);
}

static __device__ __noinline__ double cosd(double deg)
{
    double t; int q;
    reduce_deg(deg, t, q);
    if (q == 0) return cos_series(t);
    if (q == 1) return -sin_series(t);
    if (q == 2) return -cos_series(t);
    return sin_series(t);
}

static __device__ __noinline__ double sind(double deg)
{
    double t; int q;
    reduce_deg(deg, t, q);
    if (q == 0) return sin_series(t);
    if (q == 1) return cos_series(t);
    if (q == 2) return -sin_series(t);
    return -cos_series(t);
}

// omega_d = cos(phi_w - 45 d) from cw = cos(phi_w), sw = sin(phi_w).
__device__ __forceinline__ double omega(float cwf, float swf, int d)
{
    const double c = (double)cwf, s = (double)swf;
    switch (d & 7) {
    case 0: return c;
    case 1: return mul(add(c, s), kHalfSqrt2);
    case 2: return s;
    case 3: return mul(sub(s, c), kHalfSqrt2);
    case 4: return -c;
    case 5: return -mul(add(c, s), kHalfSqrt2);
    case 6: return -s;
    default: return mul(sub(c, s), kHalfSqrt2);
    }
}

// z of Eq. 1 in the equation's order.
__device__ __forceinline__ double z_of(const double b[5], bool forest,
                                       float psi, float sig, float cw,
                                       float sw, bool up, int d)
{
    const double If = forest ? 1.0 : 0.0;
    const double om = omega(cw, sw, d);
    const double sg = up ? (double)sig : 0.0;
    double z = add(b[0], mul(b[1], If));
    z = add(z, mul(b[2], (double)psi));
    z = add(z, mul(b[3], om));
    z = add(z, mul(b[4], sg));
    return z;
}

}  // namespace spec

// ---------------------------------------------------------------------------
// Single-precision screen.  z is accumulated as an unevaluated float pair
// (hi + lo, error-free products by FMA and two-sums, error below 2^-44 of
// the term magnitudes), so the roundings left are that of the diagonal wind
// cosines (|b3| 2^-25 in z), of z to float (relative 2^-24), of the
// exponential and of the reciprocal.  p = 1 / (1 + e^-z) moves by p(1-p)
// times the z error, p(1-p) <= 1/4 and max_z z p(1-p) < 0.23: |b3| 2^-27
// plus 0.23 2^-24.  The hardware exponential (its argument scaling 0.23
// 2^-24, relative error 2^-21 times p(1-p)), the rounding of 1 + e (2^-24),
// the approximate reciprocal (2^-23) and the float conversion of the draw
// (2^-24) add 3.1e-7.  So |p32 - p64| <= kScreenErrB3 |b3| + kScreenErr0,
// within 1e-6 for |b3| <= 66.  A trial is decided in single precision when
// |p32 - (u + 1) 2^-32| exceeds the simulation's margin, twice that bound
// and at least 4e-6 (4e-6 for every |b3| <= 200), and otherwise re-decided
// through the exact double-precision threshold (success <=> u <
// floor(p 2^32) <=> (u + 1) 2^-32 <= p64).
constexpr float kScreenErrB3 = 7.5e-9f;   // per unit of |b3|
constexpr float kScreenErr0 = 5.0e-7f;
constexpr float kScreenMarginMin = 4.0e-6f;

struct ff { float h, l; };

__device__ __forceinline__ ff ff_from_double(double x)
{
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(__dsub_rn(x, (double)h));
    return {h, l};
}

// (a.h + a.l) * b, unnormalised; error below 2^-46 |a b|.
__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    const float h = __fmul_rn(a.h, b);
    float l = __fmaf_rn(a.h, b, -h);
    l = __fmaf_rn(a.l, b, l);
    return {h, l};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)),
                              __fsub_rn(b.h, bb));
    const float l = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s, l);
    return {h, __fsub_rn(l, __fsub_rn(h, s))};
}

// Per-parameter-set constants of the screen.
struct ScreenParams {
    ff K[2];   // b0 + b1 * If for If = 0, 1
    ff b2, b3, b4;
    float margin;        // trial margin: max(2 err, 4e-6)
    float cell_margin;   // one-uniform-per-cell margin (below)
};

__device__ __forceinline__ ScreenParams screen_params(const double b[5])
{
    ScreenParams s;
    s.K[0] = ff_from_double(b[0]);
    s.K[1] = ff_from_double(__dadd_rn(b[0], b[1]));
    s.b2 = ff_from_double(b[2]);
    s.b3 = ff_from_double(b[3]);
    s.b4 = ff_from_double(b[4]);
    // err = kScreenErrB3 |b3| + kScreenErr0, rounded upwards
    const float err = __fmaf_ru(kScreenErrB3, __double2float_ru(fabs(b[3])),
                                kScreenErr0);
    s.margin = fmaxf(2.0f * err, kScreenMarginMin);
    // 1 - prod(1 - p_d) over up to 8 directions accumulates at most 8
    // per-direction errors and 17 float roundings of values at most 1 (below
    // 1.1e-6); doubled like the trial margin, and at least 2.5e-5
    s.cell_margin = fmaxf(__fmaf_ru(16.0f, err, 2.2e-6f), 2.5e-5f);
    if (err != err) s.margin = s.cell_margin = INFINITY;   // NaN b3: never decide
    return s;
}

// Per-target-cell partial sums of z: the direction-independent part with and
// without the slope term, and cos(phi_w - 45 j) for j = 0..3 (directions
// 4..7 use their negatives).  The diagonal cosines are the double-precision
// omega of the threshold definition rounded to float at upload, which adds at
// most |b3| 2^-25 to z.
struct ScreenCell {
    ff base;    // b0 + b1 If + b2 psi
    ff baseG;   // base + b4 sig
    float om0, om1, om2, om3;
};

__device__ __forceinline__ ScreenCell screen_cell(const ScreenParams &sp,
                                                  bool forest, float psi,
                                                  float sig, float cw,
                                                  float om1, float sw,
                                                  float om3)
{
    ScreenCell c;
    c.base = ff_add(sp.K[forest ? 1 : 0], ff_mul_f(sp.b2, psi));
    c.baseG = ff_add(c.base, ff_mul_f(sp.b4, sig));
    c.om0 = cw;
    c.om1 = om1;
    c.om2 = sw;
    c.om3 = om3;
    return c;
}

// z of direction d (up: target above the source), rounded to float.
__device__ __forceinline__ float screen_z(const ScreenCell &c, const ff &b3,
                                         bool up, int d)
{
    const int j = d & 3;
    float om = j == 0 ? c.om0 : (j == 1 ? c.om1 : (j == 2 ? c.om2 : c.om3));
    if (d & 4) om = -om;
    return ff_add(up ? c.baseG : c.base, ff_mul_f(b3, om)).h;
}

// p = 1 / (1 + e^-z) with the hardware exponential and reciprocal (each
// within a few ulp; the margin above covers them with a factor 10).
__device__ __forceinline__ float screen_p(float z)
{
    const float e = __expf(-z);
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__fadd_rn(1.0f, e)));
    return r;
}

// Decision of the trial with draw u.  Returns 1 success, 0 failure, -1 when
// the screen cannot decide and the exact threshold is needed.
__device__ __forceinline__ int screen_decide(float p32, uint32_t u,
                                             float margin)
{
    const float v = __fmaf_rn(__uint2float_rn(u), 0x1p-32f, 0x1p-32f);
    const float d = __fsub_rn(p32, v);
    if (d > margin) return 1;
    if (d < -margin) return 0;
    return -1;
}

}  // namespace fire

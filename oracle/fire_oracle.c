/*
 * CPU oracle for the stochastic fire-spread cellular automaton of
 * Denham & Laneri, "Using efficient parallelization in Graphic Processing
 * Units to parameterize stochastic fire propagation models"
 * (arXiv:1701.03549).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * reference that the CUDA library is checked against.  Only the test suite,
 * the package smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant generator with the CUDA
 * path; both implement the same written definitions independently.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent the reading used is stated in place:
 *   - Direction d = 0..7 is the compass bearing 45*d degrees (N, NE, E, SE,
 *     S, SW, W, NW) of the step from the burning (source) cell to the target
 *     cell.  Row 0 is north, column 0 is west; off(d) = (drow, dcol) with
 *     off(N) = (-1, 0), off(E) = (0, +1).
 *   - Aspect is the bearing the slope faces (downslope), clockwise from N;
 *     psi = cos(aspect - 315 deg) when slope > 5 deg, else 0 (Sec. 2.1).
 *   - Wind direction is the bearing the wind blows toward, so omega = +1
 *     when the target lies downwind of the source (Sec. 2.1).
 *   - sigma = slope_deg / 100 of the target cell, used only when the target
 *     is strictly higher than the source (Sec. 2.1).
 *   - A target cell adjacent to k burning cells ignites with probability
 *     1 - prod_i (1 - p_i) (Sec. 2.1/2.3); it is realised as k independent
 *     Bernoulli trials, one per burning neighbour, each drawn from a keyed
 *     Philox stream, and the cell ignites if any trial succeeds.
 *   - A burning cell burns out after exactly one step (Sec. 2.1).
 *   - Cells outside the grid are non-burnable (no wraparound).
 *   - Trial success is u < T with u a 32-bit uniform integer and
 *     T = floor(p * 2^32) in [0, 2^32], p evaluated in double precision by
 *     the threshold definition below.
 *
 * Compile with -ffp-contract=off: every floating-point operation here is a
 * single IEEE-754 double operation in the written order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox-4xW-R counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11, Sec. 3-4).  The paper draws its
 * random numbers from Random123's Philox (Sec. 2.3).  One generic round
 * structure serves both the 32-bit-word variant used by the automaton and the
 * 64-bit-word variant, which the tests check against numpy's implementation.
 *
 * Round: (hi0, lo0) = M0 * X0, (hi1, lo1) = M1 * X2 (double-width products),
 *        X' = (hi1 ^ X1 ^ k0, lo1, hi0 ^ X3 ^ k1, lo0);
 * the key is bumped by the Weyl constants (W0, W1) between rounds.        */
static void philox4_generic(int wbits, const uint64_t mul[2],
                            const uint64_t weyl[2], int rounds,
                            const uint64_t ctr_in[4], const uint64_t key_in[2],
                            uint64_t out[4])
{
    const uint64_t mask = (wbits == 64) ? ~(uint64_t)0
                                        : (((uint64_t)1 << wbits) - 1);
    uint64_t x0 = ctr_in[0] & mask, x1 = ctr_in[1] & mask;
    uint64_t x2 = ctr_in[2] & mask, x3 = ctr_in[3] & mask;
    uint64_t k0 = key_in[0] & mask, k1 = key_in[1] & mask;
    for (int r = 0; r < rounds; ++r) {
        if (r > 0) {
            k0 = (k0 + weyl[0]) & mask;
            k1 = (k1 + weyl[1]) & mask;
        }
        unsigned __int128 p0 = (unsigned __int128)mul[0] * x0;
        unsigned __int128 p1 = (unsigned __int128)mul[1] * x2;
        uint64_t hi0 = (uint64_t)(p0 >> wbits) & mask;
        uint64_t lo0 = (uint64_t)p0 & mask;
        uint64_t hi1 = (uint64_t)(p1 >> wbits) & mask;
        uint64_t lo1 = (uint64_t)p1 & mask;
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Multipliers and Weyl key increments given by Salmon et al. (SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4])
{
    static const uint64_t mul[2] = {0xD2511F53u, 0xCD9E8D57u};
    static const uint64_t weyl[2] = {0x9E3779B9u, 0xBB67AE85u};
    uint64_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint64_t k[2] = {key[0], key[1]};
    uint64_t o[4];
    philox4_generic(32, mul, weyl, 10, c, k, o);
    for (int i = 0; i < 4; ++i) out[i] = (uint32_t)o[i];
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                       uint64_t out[4])
{
    static const uint64_t mul[2] = {0xD2E7470EE14C6C93ull,
                                    0xCA5A826395121157ull};
    static const uint64_t weyl[2] = {0x9E3779B97F4A7C15ull,
                                     0xBB67AE8584CAA73Bull};
    philox4_generic(64, mul, weyl, 10, ctr, key, out);
}

/* The automaton's draw for the trial "target cell c, step t, direction d":
 * counter (c, t, d / 4, 0), key (seed low word, seed high word), output
 * word d % 4.                                                              */
uint32_t orc_draw(uint64_t seed, uint32_t cell, uint32_t step, int d)
{
    uint32_t ctr[4] = {cell, step, (uint32_t)(d >> 2), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[d & 3];
}

/* ------------------------------------------------------------------------ */
/* exp(x) for the logistic of Eq. 1, written from the mathematics: Cody-Waite
 * reduction x = k ln2 + r with |r| <= ln2 / 2, then the Taylor series of e^r
 * to degree 13 (remainder below 2^-56 relative), then scaling by 2^k.
 * ln2 is split into a 40-bit head (k * head is exact for |k| < 2^13) and a
 * tail.                                                                    */
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;
static const double ORC_LN2_HEAD = 0x1.62e42fefa4000p-1;
static const double ORC_LN2_TAIL = -0x1.8432a1b0e2634p-43;

double orc_exp(double x)
{
    if (x > 709.0) return INFINITY;
    if (x < -745.0) return 0.0;
    double k = rint(x * ORC_INV_LN2);
    double r = (x - k * ORC_LN2_HEAD) - k * ORC_LN2_TAIL;
    /* coefficients 1/n!, n = 13 .. 0 */
    double s = 1.0 / 6227020800.0;
    s = s * r + 1.0 / 479001600.0;
    s = s * r + 1.0 / 39916800.0;
    s = s * r + 1.0 / 3628800.0;
    s = s * r + 1.0 / 362880.0;
    s = s * r + 1.0 / 40320.0;
    s = s * r + 1.0 / 5040.0;
    s = s * r + 1.0 / 720.0;
    s = s * r + 1.0 / 120.0;
    s = s * r + 1.0 / 24.0;
    s = s * r + 1.0 / 6.0;
    s = s * r + 1.0 / 2.0;
    s = s * r + 1.0;
    s = s * r + 1.0;
    return ldexp(s, (int)k);
}

/* ------------------------------------------------------------------------ */
/* cos and sin of an angle in degrees (for the aspect term psi and the wind
 * term omega of Sec. 2.1), written from the mathematics: reduce the angle to
 * y = deg - 90 k with |y| <= 45 (exact for float-derived inputs), convert to
 * radians, evaluate the Taylor series of cos and sin to degree 18/19, and
 * rotate by the quadrant k mod 4.                                          */
static const double ORC_PI_OVER_180 = 0x1.1df46a2529d39p-6;

static double orc_cos_series(double t)
{
    double s2 = t * t;
    double c = -1.0 / 6402373705728000.0;          /* -1/18! */
    c = c * s2 + 1.0 / 20922789888000.0;           /* +1/16! */
    c = c * s2 - 1.0 / 87178291200.0;              /* -1/14! */
    c = c * s2 + 1.0 / 479001600.0;                /* +1/12! */
    c = c * s2 - 1.0 / 3628800.0;                  /* -1/10! */
    c = c * s2 + 1.0 / 40320.0;                    /* +1/8!  */
    c = c * s2 - 1.0 / 720.0;                      /* -1/6!  */
    c = c * s2 + 1.0 / 24.0;                       /* +1/4!  */
    c = c * s2 - 1.0 / 2.0;                        /* -1/2!  */
    c = c * s2 + 1.0;
    return c;
}

static double orc_sin_series(double t)
{
    double s2 = t * t;
    double c = -1.0 / 121645100408832000.0;        /* -1/19! */
    c = c * s2 + 1.0 / 355687428096000.0;          /* +1/17! */
    c = c * s2 - 1.0 / 1307674368000.0;            /* -1/15! */
    c = c * s2 + 1.0 / 6227020800.0;               /* +1/13! */
    c = c * s2 - 1.0 / 39916800.0;                 /* -1/11! */
    c = c * s2 + 1.0 / 362880.0;                   /* +1/9!  */
    c = c * s2 - 1.0 / 5040.0;                     /* -1/7!  */
    c = c * s2 + 1.0 / 120.0;                      /* +1/5!  */
    c = c * s2 - 1.0 / 6.0;                        /* -1/3!  */
    c = c * s2 + 1.0;
    return t * c;
}

static void orc_reduce_deg(double deg, double *t, int *quadrant)
{
    double k = rint(deg / 90.0);
    double y = deg - k * 90.0;
    *t = y * ORC_PI_OVER_180;
    long long kq = (long long)k;
    *quadrant = (int)(((kq % 4) + 4) % 4);
}

double orc_cosd(double deg)
{
    double t; int q;
    orc_reduce_deg(deg, &t, &q);
    switch (q) {
    case 0: return orc_cos_series(t);
    case 1: return -orc_sin_series(t);
    case 2: return -orc_cos_series(t);
    default: return orc_sin_series(t);
    }
}

double orc_sind(double deg)
{
    double t; int q;
    orc_reduce_deg(deg, &t, &q);
    switch (q) {
    case 0: return orc_sin_series(t);
    case 1: return orc_cos_series(t);
    case 2: return -orc_sin_series(t);
    default: return -orc_cos_series(t);
    }
}

/* ------------------------------------------------------------------------ */
/* Ignition threshold of one trial from the logistic of Eq. 1:
 * p = 1 / (1 + exp(-z)), T = floor(p * 2^32) in [0, 2^32].  For z >= 40 the
 * double-precision p is exactly 1 and for z <= -40 floor(p 2^32) is 0; both
 * are returned directly.                                                   */
uint64_t orc_threshold_of_z(double z)
{
    if (!(z > -40.0)) return 0;
    if (z >= 40.0) return (uint64_t)1 << 32;
    double e = orc_exp(-z);
    double p = 1.0 / (1.0 + e);
    return (uint64_t)floor(p * 4294967296.0);
}

double orc_logistic(double z)
{
    double e = orc_exp(-z);
    return 1.0 / (1.0 + e);
}

/* Direction table: off(d) = (drow, dcol), bearing 45*d degrees. */
static const int ORC_DR[8] = {-1, -1, 0, 1, 1, 1, 0, -1};
static const int ORC_DC[8] = {0, 1, 1, 1, 0, -1, -1, -1};

/* omega = cos(phi_w - phi_c) (Sec. 2.1) with phi_c = 45 d degrees, expanded
 * as cos(phi_w) cos(phi_c) + sin(phi_w) sin(phi_c) with the exact values of
 * cos and sin at multiples of 45 degrees.                                  */
static const double ORC_R2 = 0x1.6a09e667f3bcdp-1;  /* sqrt(2) / 2 */

double orc_omega(float cw, float sw, int d)
{
    double c = (double)cw, s = (double)sw;
    switch (d & 7) {
    case 0: return c;
    case 1: return (c + s) * ORC_R2;
    case 2: return s;
    case 3: return (s - c) * ORC_R2;
    case 4: return -c;
    case 5: return -((c + s) * ORC_R2);
    case 6: return -s;
    default: return (c - s) * ORC_R2;
    }
}

/* ------------------------------------------------------------------------ */
/* Per-cell covariates of Eq. 1 (Sec. 2.1).                                 */
typedef struct {
    int32_t H, W;
    const float *psi;        /* relative aspect, 0 where slope <= 5 deg      */
    const float *sig;        /* slope / 100                                  */
    const float *cw, *sw;    /* cos / sin of the wind bearing                */
    const uint8_t *up;       /* bit d: target higher than source of dir. d   */
    const uint8_t *forest;   /* I_f                                          */
    const uint8_t *burnable; /* vegetation code != 0                         */
} orc_map;

int orc_features(int H, int W, const uint8_t *veg, const float *elev,
                 const float *slope, const float *aspect, const float *wind,
                 float *psi, float *sig, float *cw, float *sw, uint8_t *up,
                 uint8_t *forest, uint8_t *burnable)
{
    if (H <= 0 || W <= 0) return -1;
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            long i = (long)r * W + c;
            burnable[i] = veg[i] != 0;
            forest[i] = veg[i] == 1;
            psi[i] = slope[i] > 5.0f
                         ? (float)orc_cosd((double)aspect[i] - 315.0)
                         : 0.0f;
            sig[i] = (float)((double)slope[i] / 100.0);
            cw[i] = (float)orc_cosd((double)wind[i]);
            sw[i] = (float)orc_sind((double)wind[i]);
            uint8_t m = 0;
            for (int d = 0; d < 8; ++d) {
                int sr = r - ORC_DR[d], sc = c - ORC_DC[d];
                if (sr < 0 || sr >= H || sc < 0 || sc >= W) continue;
                if (elev[i] > elev[(long)sr * W + sc]) m |= (uint8_t)(1u << d);
            }
            up[i] = m;
        }
    }
    return 0;
}

/* z of Eq. 1 for target cell i and direction d, summed in the equation's
 * order: ((((b0 + b1 I_f) + b2 psi) + b3 omega) + b4 sigma).              */
double orc_z(const orc_map *m, const double beta[5], long i, int d)
{
    double If = m->forest[i] ? 1.0 : 0.0;
    double omega = orc_omega(m->cw[i], m->sw[i], d);
    double sigma = ((m->up[i] >> d) & 1) ? (double)m->sig[i] : 0.0;
    double z = beta[0] + beta[1] * If;
    z = z + beta[2] * (double)m->psi[i];
    z = z + beta[3] * omega;
    z = z + beta[4] * sigma;
    return z;
}

/* Threshold table T[d * H * W + i] for every cell and direction. */
void orc_thresholds(const orc_map *m, const double beta[5], uint64_t *T)
{
    long n = (long)m->H * m->W;
    for (int d = 0; d < 8; ++d)
        for (long i = 0; i < n; ++i)
            T[d * n + i] = orc_threshold_of_z(orc_z(m, beta, i, d));
}

/* ------------------------------------------------------------------------ */
/* One simulation (Sec. 2.1 rules, Sec. 2.3): synchronous update of all
 * cells, every unburnt burnable cell tested against each burning neighbour,
 * burning cells burn out after one step, run until no cell burns.
 *
 * result[0] burnt cells |A*| (ignition included)
 * result[1] |A  intersect A*| against the target map (may be NULL -> 0)
 * result[2] |A| of the target map
 * result[3] steps: number of steps in which some cell was burning
 * result[4] status bits: 1 border touched, 2 step cap reached
 * result[5] trials: (target, direction) pairs tested
 * burn_step (optional, H*W): step at which a cell ignited, 0 for the
 * ignition, -1 burnable but unburnt, -2 non-burnable.
 * Returns 0, or -4 when the ignition is outside the grid or non-burnable. */
enum { ORC_UNBURNT = 0, ORC_BURNING = 1, ORC_BURNT = 2, ORC_BLOCKED = 3 };

/* Update rules.  Mode 0: one Bernoulli trial per (target, burning
 * neighbour), trial d succeeding iff u_d < T_d.  Mode 1, the paper's own
 * CUDA rule (Sec. 2.3): one uniform per target cell and step, compared with
 * the cell's ignition probability 1 - prod_d (1 - p_d) over its burning
 * neighbours: success iff u < floor((1 - q) 2^32), q the product of (1 - p_d)
 * in increasing d in double precision, u word 0 of the Philox block with
 * counter (cell, step, 2, 0). */
uint64_t orc_cell_threshold(const orc_map *m, const double beta[5], long i,
                            unsigned dirmask)
{
    double q = 1.0;
    for (int d = 0; d < 8; ++d) {
        if (!((dirmask >> d) & 1u)) continue;
        const double z = orc_z(m, beta, i, d);
        double p;
        if (!(z > -40.0)) p = 0.0;
        else if (z >= 40.0) p = 1.0;
        else p = orc_logistic(z);
        q = q * (1.0 - p);
    }
    const double P = 1.0 - q;
    return (uint64_t)floor(P * 4294967296.0);
}

/* Burn-out times.  The paper burns every fuel out one step after it
 * ignites (Sec. 2.1) and names fitting fuel-consumption times as future
 * work.  With burn_time (uint8 per cell, >= 1 on burnable cells) a cell
 * ignited at step t stays burning during steps t+1 .. t+burn_time, trying
 * its unburnt neighbours at each of them with the same per-trial draws
 * (counter (cell, step, d/4, 0)); NULL means one step everywhere, the
 * paper's rule.  steps = the number of update steps run while some cell
 * was burning. */
static int orc_simulate_impl(const orc_map *m, const uint8_t *target,
                             const double beta[5], int ign_r, int ign_c,
                             uint64_t seed, uint32_t max_steps, int mode,
                             const uint8_t *burn_time, int32_t *burn_step,
                             uint32_t result[6]);

int orc_simulate(const orc_map *m, const uint8_t *target, const double beta[5],
                 int ign_r, int ign_c, uint64_t seed, uint32_t max_steps,
                 int32_t *burn_step, uint32_t result[6])
{
    return orc_simulate_impl(m, target, beta, ign_r, ign_c, seed, max_steps, 0,
                             NULL, burn_step, result);
}

int orc_simulate_mode(const orc_map *m, const uint8_t *target,
                      const double beta[5], int ign_r, int ign_c,
                      uint64_t seed, uint32_t max_steps, int mode,
                      int32_t *burn_step, uint32_t result[6])
{
    return orc_simulate_impl(m, target, beta, ign_r, ign_c, seed, max_steps,
                             mode, NULL, burn_step, result);
}

int orc_simulate_burnout(const orc_map *m, const uint8_t *target,
                         const double beta[5], int ign_r, int ign_c,
                         uint64_t seed, uint32_t max_steps,
                         const uint8_t *burn_time, int32_t *burn_step,
                         uint32_t result[6])
{
    return orc_simulate_impl(m, target, beta, ign_r, ign_c, seed, max_steps, 0,
                             burn_time, burn_step, result);
}

static int orc_simulate_impl(const orc_map *m, const uint8_t *target,
                             const double beta[5], int ign_r, int ign_c,
                             uint64_t seed, uint32_t max_steps, int mode,
                             const uint8_t *burn_time, int32_t *burn_step,
                             uint32_t result[6])
{
    const int H = m->H, W = m->W;
    const long n = (long)H * W;
    memset(result, 0, 6 * sizeof(uint32_t));
    if (target) {
        for (long i = 0; i < n; ++i) result[2] += target[i] ? 1u : 0u;
    }
    if (ign_r < 0 || ign_r >= H || ign_c < 0 || ign_c >= W) return -4;
    if (!m->burnable[(long)ign_r * W + ign_c]) return -4;

    if (n <= 0) return -1;
    if (burn_time) {
        for (long i = 0; i < n; ++i)
            if (m->burnable[i] && burn_time[i] == 0) return -1;
    }
    uint8_t *state = (uint8_t *)malloc((size_t)n);
    uint8_t *ignite = (uint8_t *)malloc((size_t)n);
    uint8_t *left = (uint8_t *)malloc((size_t)n);   /* burning steps left */
    if (!state || !ignite || !left) {
        free(state); free(ignite); free(left);
        return -2;
    }
    for (long i = 0; i < n; ++i) {
        state[i] = m->burnable[i] ? ORC_UNBURNT : ORC_BLOCKED;
        left[i] = 0;
        if (burn_step) burn_step[i] = m->burnable[i] ? -1 : -2;
    }
    long ign = (long)ign_r * W + ign_c;
    state[ign] = ORC_BURNING;
    left[ign] = burn_time ? burn_time[ign] : 1;
    if (burn_step) burn_step[ign] = 0;

    uint32_t burnt = 1, inter = (target && target[ign]) ? 1u : 0u;
    uint32_t trials = 0, status = 0;
    if (ign_r == 0 || ign_r == H - 1 || ign_c == 0 || ign_c == W - 1)
        status |= 1u;

    uint32_t t = 0;
    int any_burning = 1;
    while (any_burning) {
        if (max_steps && t >= max_steps) { status |= 2u; break; }
        /* every unburnt burnable cell checks its burning neighbours */
        for (int r = 0; r < H; ++r) {
            for (int c = 0; c < W; ++c) {
                long i = (long)r * W + c;
                ignite[i] = 0;
                if (state[i] != ORC_UNBURNT) continue;
                unsigned dirmask = 0;
                for (int d = 0; d < 8; ++d) {
                    int sr = r - ORC_DR[d], sc = c - ORC_DC[d];
                    if (sr < 0 || sr >= H || sc < 0 || sc >= W) continue;
                    if (state[(long)sr * W + sc] != ORC_BURNING) continue;
                    trials++;
                    dirmask |= 1u << d;
                    if (mode != 0) continue;
                    uint64_t T = orc_threshold_of_z(orc_z(m, beta, i, d));
                    uint32_t u = orc_draw(seed, (uint32_t)i, t, d);
                    if ((uint64_t)u < T) ignite[i] = 1;
                }
                if (mode != 0 && dirmask) {
                    uint32_t ctr[4] = {(uint32_t)i, t, 2u, 0u};
                    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
                    uint32_t w[4];
                    orc_philox4x32_10(ctr, key, w);
                    if ((uint64_t)w[0] < orc_cell_threshold(m, beta, i, dirmask))
                        ignite[i] = 1;
                }
            }
        }
        /* burning cells spend one step of fuel and burn out when none is
           left; newly ignited cells start burning */
        any_burning = 0;
        for (long i = 0; i < n; ++i) {
            if (state[i] != ORC_BURNING) continue;
            left[i]--;
            if (left[i] == 0) state[i] = ORC_BURNT;
            else any_burning = 1;
        }
        for (int r = 0; r < H; ++r) {
            for (int c = 0; c < W; ++c) {
                long i = (long)r * W + c;
                if (!ignite[i]) continue;
                state[i] = ORC_BURNING;
                left[i] = burn_time ? burn_time[i] : 1;
                any_burning = 1;
                burnt++;
                if (target && target[i]) inter++;
                if (burn_step) burn_step[i] = (int32_t)(t + 1);
                if (r == 0 || r == H - 1 || c == 0 || c == W - 1)
                    status |= 1u;
            }
        }
        t++;
    }
    result[0] = burnt;
    result[1] = inter;
    result[3] = t;
    result[4] = status;
    result[5] = trials;
    free(state);
    free(ignite);
    free(left);
    return 0;
}

/* Per-cell burn counts over many replicate seeds (seed0, seed0 + 1, ...),
 * for the Monte Carlo side of the exact-enumeration check.                */
int orc_burn_frequency_mode(const orc_map *m, const double beta[5], int ign_r,
                            int ign_c, uint64_t seed0, long nseeds, int mode,
                            uint32_t *counts);

int orc_burn_frequency(const orc_map *m, const double beta[5], int ign_r,
                       int ign_c, uint64_t seed0, long nseeds, uint32_t *counts)
{
    return orc_burn_frequency_mode(m, beta, ign_r, ign_c, seed0, nseeds, 0,
                                   counts);
}

static int orc_burn_frequency_impl(const orc_map *m, const double beta[5],
                                   int ign_r, int ign_c, uint64_t seed0,
                                   long nseeds, int mode,
                                   const uint8_t *burn_time, uint32_t *counts);

int orc_burn_frequency_mode(const orc_map *m, const double beta[5], int ign_r,
                            int ign_c, uint64_t seed0, long nseeds, int mode,
                            uint32_t *counts)
{
    return orc_burn_frequency_impl(m, beta, ign_r, ign_c, seed0, nseeds, mode,
                                   NULL, counts);
}

int orc_burn_frequency_burnout(const orc_map *m, const double beta[5],
                               int ign_r, int ign_c, uint64_t seed0,
                               long nseeds, const uint8_t *burn_time,
                               uint32_t *counts)
{
    return orc_burn_frequency_impl(m, beta, ign_r, ign_c, seed0, nseeds, 0,
                                   burn_time, counts);
}

static int orc_burn_frequency_impl(const orc_map *m, const double beta[5],
                                   int ign_r, int ign_c, uint64_t seed0,
                                   long nseeds, int mode,
                                   const uint8_t *burn_time, uint32_t *counts)
{
    const long n = (long)m->H * m->W;
    int32_t *bs = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!bs) return -2;
    memset(counts, 0, (size_t)n * sizeof(uint32_t));
    for (long s = 0; s < nseeds; ++s) {
        uint32_t res[6];
        int rc = orc_simulate_impl(m, NULL, beta, ign_r, ign_c,
                                   seed0 + (uint64_t)s, 0, mode, burn_time, bs,
                                   res);
        if (rc) { free(bs); return rc; }
        for (long i = 0; i < n; ++i) counts[i] += bs[i] >= 0 ? 1u : 0u;
    }
    free(bs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Fitness of Eq. 2: delta = (|A u A*| - |A n A*|) / |A|, with A the
 * reference (target) burnt set and A* the simulated one (kind 0).  Kind 1 is
 * the Jaccard distance (|A u A*| - |A n A*|) / |A u A*|.                   */
double orc_fitness(uint32_t burnt, uint32_t inter, uint32_t target, int kind)
{
    double uni = (double)target + (double)burnt - (double)inter;
    double sym = uni - (double)inter;
    if (kind == 0) return sym / (double)target;
    return sym / uni;
}

/* ------------------------------------------------------------------------ */
/* Genetic algorithm of the paper's Appendix B: elitism, tournament selection
 * between two individuals drawn at random, one-point crossover of pairs, and
 * per-gene mutation whose probability decreases as the GA advances.  The
 * paper leaves the constants open; the reading used here (the same one the
 * CUDA library implements independently):
 *   - order of individuals: lower fitness is better, NaN is worst, ties go
 *     to the lower index;
 *   - E = min(2, P) elites (best first) fill slots 0..E-1 unchanged;
 *   - slot j >= E: Philox counter (j, g, 0, 0), contestants
 *     a = (w0 * P) >> 32 and b = (w1 * P) >> 32, parent = the better one;
 *   - pairs (j, j + 1), j = E, E + 2, ...: counter (j, g, 1, 0), cut
 *     c = 1 + ((w0 * (G - 1)) >> 32) in [1, G - 1]; child j takes genes
 *     [0, c) from its own parent and [c, G) from the partner's, child j + 1
 *     the reverse; an unpaired last slot copies its parent; G = 1 never
 *     crosses;
 *   - gene k of child j: counter (j, g, 2, k); with s = 1 - g / NG,
 *     pm = 0.2 s + 0.01 and T = floor(pm 2^32), the gene mutates iff w0 < T,
 *     by delta = (2 u - 1) (0.1 (hi_k - lo_k)) s with u = w1 2^-32, and the
 *     result is clamped to [lo_k, hi_k].
 * Every step is a single IEEE-754 double operation in the written order. */
static int orc_better(const double *f, int a, int b)
{
    const int na = f[a] != f[a], nb = f[b] != f[b];
    if (na != nb) return nb;          /* the non-NaN one is better */
    if (!na && f[a] != f[b]) return f[a] < f[b];
    return a < b;
}

static void orc_block(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                      uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

int orc_ga_step(int P, int G, const double *genes_in, const double *fitness,
                int g, int NG, uint64_t seed, const double *lo,
                const double *hi, double *genes_out)
{
    if (P <= 0 || G <= 0 || NG <= 0) return -1;
    const int E = P < 2 ? P : 2;
    /* elites */
    int best = 0;
    for (int i = 1; i < P; ++i) if (orc_better(fitness, i, best)) best = i;
    int second = -1;
    for (int i = 0; i < P; ++i) {
        if (i == best) continue;
        if (second < 0 || orc_better(fitness, i, second)) second = i;
    }
    const int elite[2] = {best, second};
    for (int e = 0; e < E; ++e)
        for (int k = 0; k < G; ++k)
            genes_out[(long)e * G + k] = genes_in[(long)elite[e] * G + k];
    /* tournament parents */
    int *parent = (int *)malloc(sizeof(int) * (size_t)P);
    if (!parent) return -2;
    for (int j = E; j < P; ++j) {
        uint32_t w[4];
        orc_block(seed, (uint32_t)j, (uint32_t)g, 0u, 0u, w);
        const int a = (int)(((uint64_t)w[0] * (uint64_t)P) >> 32);
        const int b = (int)(((uint64_t)w[1] * (uint64_t)P) >> 32);
        parent[j] = orc_better(fitness, a, b) ? a : b;
    }
    /* crossover */
    for (int j = E; j < P; j += 2) {
        const double *pa = genes_in + (long)parent[j] * G;
        double *ca = genes_out + (long)j * G;
        if (j + 1 >= P || G < 2) {
            for (int k = 0; k < G; ++k) ca[k] = pa[k];
            if (j + 1 < P) {
                const double *pb = genes_in + (long)parent[j + 1] * G;
                double *cb = genes_out + (long)(j + 1) * G;
                for (int k = 0; k < G; ++k) cb[k] = pb[k];
            }
            continue;
        }
        const double *pb = genes_in + (long)parent[j + 1] * G;
        double *cb = genes_out + (long)(j + 1) * G;
        uint32_t w[4];
        orc_block(seed, (uint32_t)j, (uint32_t)g, 1u, 0u, w);
        const int cut = 1 + (int)(((uint64_t)w[0] * (uint64_t)(G - 1)) >> 32);
        for (int k = 0; k < G; ++k) {
            ca[k] = k < cut ? pa[k] : pb[k];
            cb[k] = k < cut ? pb[k] : pa[k];
        }
    }
    free(parent);
    /* mutation */
    const double s = 1.0 - (double)g / (double)NG;
    const double pm = 0.2 * s + 0.01;
    const uint64_t T = (uint64_t)floor(pm * 4294967296.0);
    for (int j = E; j < P; ++j) {
        for (int k = 0; k < G; ++k) {
            uint32_t w[4];
            orc_block(seed, (uint32_t)j, (uint32_t)g, 2u, (uint32_t)k, w);
            if ((uint64_t)w[0] >= T) continue;
            const double u = (double)w[1] * 0x1p-32;
            const double scale = (0.1 * (hi[k] - lo[k])) * s;
            const double delta = (2.0 * u - 1.0) * scale;
            double x = genes_out[(long)j * G + k] + delta;
            if (x < lo[k]) x = lo[k];
            if (x > hi[k]) x = hi[k];
            genes_out[(long)j * G + k] = x;
        }
    }
    return 0;
}

/* Mean of each group of per_group consecutive values (the fitness of a GA
 * individual over its replicate simulations), summed in index order. */
void orc_group_mean(const double *v, int groups, int per_group, double *out)
{
    for (int i = 0; i < groups; ++i) {
        double s = 0.0;
        for (int r = 0; r < per_group; ++r) s = s + v[(long)i * per_group + r];
        out[i] = s / (double)per_group;
    }
}

/* ------------------------------------------------------------------------ */
/* Ignition-point search (Sec. 3: the ignition point treated as unknown and
 * drawn from inside the reference fire's burnt area).  The reading used:
 *   - the target's burnt cells span rows [r0, r1], columns [c0, c1];
 *   - lattice point (a, b), a < LH, b < LW, sits at row
 *     r0 + floor((2a + 1)(r1 - r0 + 1) / (2 LH)) and column
 *     c0 + floor((2b + 1)(c1 - c0 + 1) / (2 LW)) (centres of equal strips);
 *   - its candidate ignition is the burnable burnt cell nearest to it
 *     (squared distance, ties to the lower row-major index);
 *   - candidate c = a LW + b is simulated reps times with seeds
 *     seed + c reps + r; its fitness is the mean over the replicates;
 *   - the ensemble is the candidates with fitness <= cutoff (or, if none,
 *     the best one, ties to the lower index); the estimate is the mean and
 *     sample standard deviation of their x = column and y = row.
 * Returns 0, or -1 when the target has no burnable burnt cell. */
int orc_ignition_search(const orc_map *m, const uint8_t *target,
                        const double beta[5], int LH, int LW, int reps,
                        uint64_t seed, int kind, double cutoff,
                        double *fitness_map, int32_t *cells, double xy[4])
{
    const int H = m->H, W = m->W;
    int r0 = H, r1 = -1, c0 = W, c1 = -1;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c)
            if (target[(long)r * W + c]) {
                if (r < r0) r0 = r;
                if (r > r1) r1 = r;
                if (c < c0) c0 = c;
                if (c > c1) c1 = c;
            }
    if (r1 < 0) return -1;
    const int L = LH * LW;
    for (int a = 0; a < LH; ++a) {
        for (int b = 0; b < LW; ++b) {
            const long long R = r0 + ((2LL * a + 1) * (r1 - r0 + 1)) / (2LL * LH);
            const long long C = c0 + ((2LL * b + 1) * (c1 - c0 + 1)) / (2LL * LW);
            long long best = -1, bestd = 0;
            for (long i = 0; i < (long)H * W; ++i) {
                if (!target[i] || !m->burnable[i]) continue;
                const long long dr = i / W - R, dc = i % W - C;
                const long long d = dr * dr + dc * dc;
                if (best < 0 || d < bestd) { best = i; bestd = d; }
            }
            if (best < 0) return -1;
            const int cidx = a * LW + b;
            cells[2 * cidx] = (int32_t)(best / W);
            cells[2 * cidx + 1] = (int32_t)(best % W);
        }
    }
    for (int cidx = 0; cidx < L; ++cidx) {
        double s = 0.0;
        for (int r = 0; r < reps; ++r) {
            uint32_t res[6];
            orc_simulate(m, target, beta, cells[2 * cidx], cells[2 * cidx + 1],
                         seed + (uint64_t)cidx * (uint64_t)reps + (uint64_t)r, 0,
                         NULL, res);
            s = s + orc_fitness(res[0], res[1], res[2], kind);
        }
        fitness_map[cidx] = s / (double)reps;
    }
    /* ensemble */
    int k = 0;
    double sx = 0.0, sy = 0.0;
    for (int cidx = 0; cidx < L; ++cidx)
        if (fitness_map[cidx] <= cutoff) {
            k++;
            sx = sx + (double)cells[2 * cidx + 1];
            sy = sy + (double)cells[2 * cidx];
        }
    int bestc = 0;
    if (k == 0) {
        for (int cidx = 1; cidx < L; ++cidx)
            if (orc_better(fitness_map, cidx, bestc)) bestc = cidx;
        xy[0] = (double)cells[2 * bestc + 1];
        xy[1] = 0.0;
        xy[2] = (double)cells[2 * bestc];
        xy[3] = 0.0;
        return 0;
    }
    const double mx = sx / (double)k, my = sy / (double)k;
    double vx = 0.0, vy = 0.0;
    for (int cidx = 0; cidx < L; ++cidx)
        if (fitness_map[cidx] <= cutoff) {
            const double dx = (double)cells[2 * cidx + 1] - mx;
            const double dy = (double)cells[2 * cidx] - my;
            vx = vx + dx * dx;
            vy = vy + dy * dy;
        }
    xy[0] = mx;
    xy[1] = k > 1 ? sqrt(vx / (double)(k - 1)) : 0.0;
    xy[2] = my;
    xy[3] = k > 1 ? sqrt(vy / (double)(k - 1)) : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ignition point as two more genes (Sec. 3, Table 3; Appendix B: with the
 * ignition unknown the search runs over seven parameters, x and y added).
 * The paper starts those fires from points of the reference fire's burnt
 * area.  Reading: gene x is the column and y the row; each is clamped to the
 * grid ([0, W - 1] and [0, H - 1], a NaN counting as 0), rounded half up to
 * an integer, and the fire starts from the burnable cell of the target burnt
 * area nearest to that point (squared distance, ties to the lower row-major
 * index) - the same nearest-cell rule as the lattice candidates of
 * orc_ignition_search.  Returns -1 when the target has no burnable cell.   */
static double orc_clamp_gene(double v, double hi)
{
    if (!(v >= 0.0)) return 0.0;   /* NaN and negatives */
    return v > hi ? hi : v;
}

int orc_snap_ignition(const orc_map *m, const uint8_t *target, double x,
                      double y, int32_t *row, int32_t *col)
{
    const int H = m->H, W = m->W;
    const long long C = (long long)floor(orc_clamp_gene(x, (double)(W - 1)) + 0.5);
    const long long R = (long long)floor(orc_clamp_gene(y, (double)(H - 1)) + 0.5);
    long long best = -1, bestd = 0;
    for (long i = 0; i < (long)H * W; ++i) {
        if (!target[i] || !m->burnable[i]) continue;
        const long long dr = i / W - R, dc = i % W - C;
        const long long d = dr * dr + dc * dc;
        if (best < 0 || d < bestd) { best = i; bestd = d; }
    }
    if (best < 0) return -1;
    *row = (int32_t)(best / W);
    *col = (int32_t)(best % W);
    return 0;
}

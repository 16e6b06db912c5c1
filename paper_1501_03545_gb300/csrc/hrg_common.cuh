// hrg_common.cuh -- device-side building blocks of the RHG generator.
//
// Shared by the generator's translation units only (never by the CPU oracle).
// Notation follows von Looz et al., "Fast generation of complex networks with
// underlying hyperbolic geometry": n points on the hyperbolic disk of radius
// R (curvature -1), angle phi uniform on [0, 2pi), radius r with density
// alpha sinh(alpha r) / (cosh(alpha R) - 1) (Eq. (1)); u ~ v iff
// dist(u, v) < R (Sec. 2.1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define HRG_MAX_BANDS 64

namespace hrg {

// ---------------------------------------------------------------------------
// Plan: everything a kernel needs to know about one graph.  Filled on the
// host (hrg_api.cu) and passed by value.
// ---------------------------------------------------------------------------
struct Plan {
    int64_t n;
    double R, coshR, alpha;
    double big;          // cosh(alpha R) - 1, the scale of Eq. (1)'s inverse CDF
    double big53;        // big 2^-53 (exact): multiplies the top 53 bits of a random word
    double inv_alpha;    // 1 / alpha
    double half_R;       // R / 2
    float half_R_hi, half_R_lo;  // R / 2 as a float pair (hi + lo)
    double inv_width;    // B / R
    int B;               // number of radial bands
    int hub_bands;       // bands [0, hub_bands) are queried one warp per vertex
    int sbits;           // 2^sbits angular sectors; every band has gbits >= sbits
    int first_band;      // bands below it are known to be empty (0 when the counts are estimates)
    int64_t G;           // total number of angular buckets over all bands
    double band_lo[HRG_MAX_BANDS + 1];  // inner radius of each band; band_lo[B] = +inf
    int64_t base[HRG_MAX_BANDS + 1];    // first bucket of each band; base[B] = G
    int gbits[HRG_MAX_BANDS];           // log2(#buckets) of each band
    float Pb[HRG_MAX_BANDS], Mb[HRG_MAX_BANDS], Sb[HRG_MAX_BANDS];  // scaled exps at band_lo
    float rhs32;         // 1 + e^{-2R} rounded to float
    float mu;            // half-width of the FP32 filter's undecided band (relative)
    double rhs64;        // 1 + e^{-2R}
    // the tie band of the FP64 path's scaled value: the bit patterns of
    // rhs64 (1 - 1e-12) and rhs64 (1 + 1e-12) (positive doubles order like
    // their bits, so the band test is two integer compares)
    int64_t tie_lo, tie_hi;
    // A batch of graphs lays its graphs out one after another: graph g owns
    // positions and global ids [id_off, id_off + n) and buckets from base[0].
    // The CSR stores local ids (global id - id_off).  0 for a single graph.
    int32_t id_off;
    int32_t pad_;
    uint64_t seed;       // Philox key of the graph (batches)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The counter block is
// (id_lo, id_hi, 0, 0) and the key (seed_lo, seed_hi); ten rounds, each a
// pair of 32x32->64 multiplications with the halves swapped and xored with
// the key, the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox_block(uint64_t ctr, uint64_t seed)
{
    const uint32_t MUL_A = 0xD2511F53u, MUL_B = 0xCD9E8D57u;
    const uint32_t BUMP_A = 0x9E3779B9u, BUMP_B = 0xBB67AE85u;
    U4 s{(uint32_t)ctr, (uint32_t)(ctr >> 32), 0u, 0u};
    uint32_t ka = (uint32_t)seed, kb = (uint32_t)(seed >> 32);
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t ha = __umulhi(MUL_A, s.x), la = MUL_A * s.x;
        const uint32_t hb = __umulhi(MUL_B, s.z), lb = MUL_B * s.z;
        s = U4{hb ^ s.y ^ ka, lb, ha ^ s.w ^ kb, la};
        ka += BUMP_A;
        kb += BUMP_B;
    }
    return s;
}

// acosh(x) for a double x >= 2^8, in unsigned 64-bit fixed point (integer
// multiplies instead of the FP64 pipe), from
//   acosh(x) = log(2x) + log((1 + sqrt(1 - s)) / 2)
//            = log(2x) - s/4 - 3 s^2/32 - 5 s^3/96 - ...,  s = 1/x^2 <= 2^-16
// (the first dropped term, 35 s^4/1024, is below 2^-69).
// log(2x) by the table-driven reduction of P. T. P. Tang (ACM TOMS 16(4),
// 1990): 2x = 2^e (F_j + f) with F_j = 1 + j/128 (j = the top 7 mantissa
// bits) and 0 <= f < 1/128, so
//   log 2x = e ln 2 + log F_j + log(1 + t),  t = f / F_j in [0, 2^-7).
// tab[j] = floor(2^63 / F_j), tab[128 + j] = log F_j 2^64 and tab[256] =
// ln 2 2^64, rounded, are computed on the host in integer arithmetic.
// t is formed as T = t 2^70 (truncations below 2^-70); log(1 + t) = t h_1
// with h_8 = 1/8, h_k = 1/k - t h_{k+1} in Q63 (the dropped term t^9/9 is
// below 2^-66; each step truncates below 2^-63, weighed by t <= 2^-7).
// s from the same reduction: x = 2^(e-1) m, 1/m = (1/F_j) / (1 + t) with
// 1/(1 + t) by its series through t^7 in Q63 (dropped: t^8 < 2^-56,
// relative), so s is within ~2^-55 relative and the correction within
// ~2^-64.  The sum is kept with 64 fraction bits and rounded to the nearest
// double once: within 0.5 ulp + ~2^-60 of acosh(x).
__device__ __forceinline__ double acosh_fix(double x, const uint64_t *tab)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const uint64_t e = (bits >> 52) - 1022;  // exponent of 2x, >= 9
    const int j = (int)((bits >> 45) & 127);
    const uint64_t f45 = bits & ((1ull << 45) - 1);
    // T = f45 2^-52 (tab[j] 2^-63) 2^70 = (f45 tab[j]) >> 45
    const uint64_t inv = tab[j];
    const uint64_t T = (__umul64hi(f45, inv) << 19) | ((f45 * inv) >> 45);
    uint64_t h = (1ull << 63) / 8, g = 1ull << 63;
#pragma unroll
    for (int k = 7; k >= 1; --k) {
        h = ((1ull << 63) / k) - (__umul64hi(T, h) >> 6);  // (t h) 2^63 = (T h) >> 70
        if (k <= 6) g = (1ull << 63) - (__umul64hi(T, g) >> 6);
    }
    g = (1ull << 63) - (__umul64hi(T, g) >> 6);  // g_0
    const uint64_t L = __umul64hi(T, h) >> 5;    // t h_1 2^64 = (T h_1) >> 69
    // (1/m)^2, ^4, ^6 in Q63; s = (1/m)^2 2^(2 - 2e)
    const uint64_t rm = __umul64hi(inv, g) << 1;
    const uint64_t q2 = __umul64hi(rm, rm) << 1, q4 = __umul64hi(q2, q2) << 1, q6 = __umul64hi(q4, q2) << 1;
    // the correction times 2^64 (x = 2^(e-1) m): s/4 = q2 >> (2e - 1),
    // 3 s^2/32 = 3 q4 >> 4e, 5 s^3/96 = 5 q6 / 96 >> (6e - 7)
    const unsigned s1 = (unsigned)(2 * e - 1), s2 = (unsigned)(4 * e - 2), s3 = (unsigned)(6 * e - 7);
    uint64_t corr = s1 < 64 ? q2 >> s1 : 0;
    if (s2 < 64) corr += (3 * (q4 >> 2)) >> s2;
    if (s3 < 64) corr += ((q6 / 96) * 5) >> s3;
    // e ln 2 + log F_j + L - corr as hi + lo 2^-64
    uint64_t lo = e * tab[256], hi = __umul64hi(e, tab[256]);
    const uint64_t a = lo + tab[128 + j];
    hi += a < lo;
    lo = a + L;
    hi += lo < a;
    hi -= lo < corr;
    lo -= corr;
    // round hi + lo 2^-64 (hi >= 6) to 53 bits, to nearest, ties to even
    const int nb = 64 - __clzll((long long)hi);  // integer bits
    const int sh = nb + 11;                      // bits dropped, 14..21
    uint64_t m = (hi << (64 - sh)) | (lo >> sh);
    const uint64_t rem = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    m += (rem > half || (rem == half && (m & 1))) ? 1 : 0;
    // m carries the leading bit at 2^52 (2^53 after a carry, which then
    // raises the exponent): value m 2^(nb - 53)
    return __longlong_as_double((long long)(((uint64_t)(nb - 2 + 1023) << 52) + m));
}

// The uniform of a 64-bit word is u = k 2^-53, k its top 53 bits.  Its
// products are taken as k (c 2^-53): c 2^-53 is c with the exponent moved
// (exact), and k and u differ by a power of two too, so k (c 2^-53) and u c
// are the same real number and round to the same double -- one multiply
// instead of two.
__device__ __forceinline__ double top53(uint32_t hi, uint32_t lo)
{
    const uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
    return (double)(w >> 11);  // exact: below 2^53
}

// Radius of Eq. (1)'s inverse CDF, r = acosh(x) / alpha with x = 1 + u_r
// (cosh(alpha R) - 1) = 1 + k_r big_scaled, big_scaled = (cosh(alpha R) - 1)
// 2^-53.  Above x = 2^8 the fixed-point series (acosh_fix: integer pipes,
// one short branch where the library acosh would make a warp run both
// paths); below, the library acosh.
__device__ __forceinline__ double radius_of(double k_r, double big_scaled, double inv_alpha, const uint64_t *log_tab)
{
    const double x = __dadd_rn(1.0, __dmul_rn(k_r, big_scaled));
    const double a = x >= 0x1p8 ? acosh_fix(x, log_tab) : acosh(x);
    return a * inv_alpha;
}

constexpr double kTwoPi = 6.283185307179586;          // the double nearest 2 pi
constexpr double kTwoPiScaled = kTwoPi * 0x1.0p-53;    // (the double nearest 2 pi) 2^-53, exact
constexpr double kAngleScale = 2.9358905032820014e18;  // 2^64 / (2 pi): angle -> 64-bit fixed point
constexpr float kAngleScaleUp = 2.9358906e18f;         // the same, rounded up (windows stay conservative)
constexpr float kAngleUnit = 3.4061215800865545e-19f;  // 2 pi / 2^64

// Fixed-point angle A in [0, 2^64) for phi in [0, 2pi): monotone in phi, and
// within 2^12 units of phi * 2^64 / (2 pi).  Differences of A taken as signed
// 64-bit integers are circular angle differences.
__device__ __forceinline__ uint64_t angle_key(double phi)
{
    double a = __dmul_rn(phi, kAngleScale);
    if (!(a > 0.0)) return 0ull;
    if (a >= 18446744073709551615.0) return 0xFFFFFFFFFFFFFFFFull;
    return __double2ull_rz(a);
}

// The sampler files a point under the bucket of u_phi 2^64 = its word's top
// 53 bits shifted back (integer work only), not of angle_key(phi): phi =
// fl(u_phi 2pi), so the two are within 2^12 units of each other, and a
// window's 2^16-unit pad (window_halfwidth) covers that as well as the
// stored angles' own 2^12 -- no bucket range misses a point in the window.
__device__ __forceinline__ uint64_t sampled_angle_key(const U4 &w)
{
    return (((uint64_t)w.x << 32) | (uint64_t)w.y) & ~(uint64_t)0x7FF;
}

// radial band: the k with band_lo[k] <= r < band_lo[k+1]
__device__ __forceinline__ int band_of(const Plan &p, double r)
{
    int k = (int)(r * p.inv_width);
    if (k < 0) k = 0;
    if (k > p.B - 1) k = p.B - 1;
    while (k > 0 && r < p.band_lo[k]) --k;
    while (k < p.B - 1 && r >= p.band_lo[k + 1]) ++k;
    return k;
}

__device__ __forceinline__ int64_t bucket_of(const Plan &p, int band, uint64_t A)
{
    const int g = p.gbits[band];
    return p.base[band] + (g == 0 ? 0 : (int64_t)(A >> (64 - g)));
}

// ---------------------------------------------------------------------------
// Scaled exponentials.  With P = e^{r - R/2}, M = e^{-r - R/2} and
// S = P - M = 2 e^{-R/2} sinh r, the edge rule of Sec. 2.1 in the form
//   cosh(r1 - r2) + 2 sinh r1 sinh r2 sin^2(dphi/2) < cosh R
// multiplied by 2 e^{-R} reads
//   P1 M2 + P2 M1 + S1 S2 sin^2(dphi/2) < 1 + e^{-2R},
// all terms non-negative and bounded by e^{R} for r <= R.
// ---------------------------------------------------------------------------
struct __align__(16) PMS { float P, M, S; int32_t id; };

// a + b = s + e exactly (Knuth's two-sum), in float
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// e^{r - R/2} and e^{-r - R/2} with their arguments carried as float pairs
// (r split once into r_hi + r_lo from the double, R/2 split on the host), so
// the exponent keeps ~2^-40 absolute accuracy with float arithmetic only:
// e^{t_hi + t_lo} = e^{t_hi} (1 + t_lo) to within t_lo^2.
__device__ __forceinline__ PMS scaled_exps(const Plan &p, double r, int32_t id)
{
    PMS o;
    const float rh = __double2float_rn(r);
    const float rl = __double2float_rn(r - (double)rh);
    float e1, e2;
    const float th = two_sum(rh, -p.half_R_hi, e1);  // r - R/2
    const float tl = e1 + (rl - p.half_R_lo);
    o.P = expf(th) * (1.0f + tl);
    const float mh = two_sum(-rh, -p.half_R_hi, e2);  // -r - R/2
    const float ml = e2 - (rl + p.half_R_lo);
    o.M = expf(mh) * (1.0f + ml);
    // S = P (1 - e^{-2r}); expm1f keeps small radii accurate
    o.S = o.P * (-expm1f(-2.0f * rh));
    o.id = id;
    return o;
}

// sin(x) for |x| <= pi/2 by its Taylor series through x^11 (Horner in x^2);
// truncation error <= (pi/2)^13/13! < 6e-8 at the interval's end.
__device__ __forceinline__ float sin_taylor(float x)
{
    const float t = x * x;
    float s = -2.5052108e-8f;           // -1/11!
    s = fmaf(s, t, 2.7557319e-6f);      //  1/9!
    s = fmaf(s, t, -1.9841270e-4f);     // -1/7!
    s = fmaf(s, t, 8.3333333e-3f);      //  1/5!
    s = fmaf(s, t, -1.6666667e-1f);     // -1/3!
    s = fmaf(s, t, 1.0f);
    return x * s;
}

// FP32 value of P1 M2 + P2 M1 + S1 S2 sin^2(dA/2) for a fixed-point angle
// difference dA (signed, |dA| <= 2^63 <-> pi).
__device__ __forceinline__ float lhs32(const PMS &q, const PMS &c, int64_t dA)
{
    // dA = hi 2^32 + lo with hi signed and lo unsigned; two 32-bit
    // conversions (the 64-bit one is an order of magnitude slower) and one
    // FMA give dA * pi / 2^64 to within 3 ulp
    // (split of |dA|, so that both directions of a pair round identically)
    const uint64_t ad = dA < 0 ? (0ull - (uint64_t)dA) : (uint64_t)dA;
    const uint32_t hi = (uint32_t)(ad >> 32);
    const uint32_t lo = (uint32_t)ad;
    const float half = fmaf((float)hi, 7.3145904e-10f /* pi / 2^32 */, (float)lo * 1.7030608e-19f /* pi / 2^64 */);
    const float s = sin_taylor(half);
    // both products rounded on their own and then added: rounded addition and
    // multiplication commute, so the value of a pair is the same whichever
    // endpoint asks (no fused multiply-add across the two cross products)
    const float cross = __fadd_rn(__fmul_rn(q.P, c.M), __fmul_rn(c.P, q.M));
    return fmaf(__fmul_rn(q.S, c.S), s * s, cross);
}

// sin(x) for |x| <= 2^-4 by Taylor through x^9 (error < x^11/11! < 1e-20 |x|),
// the CUDA library sin beyond.
__device__ __forceinline__ double sin_small64(double x)
{
    if (fabs(x) > 0.0625) return sin(x);
    const double t = x * x;
    double s = 2.7557319223985893e-6;            //  1/9!
    s = fma(s, t, -1.9841269841269841e-4);       // -1/7!
    s = fma(s, t, 8.3333333333333333e-3);        //  1/5!
    s = fma(s, t, -1.6666666666666667e-1);       // -1/3!
    s = fma(s, t, 1.0);
    return x * s;
}

// Exact FP64 decision from the stored coordinates (the recheck, and the
// reference form of the predicate): cosh(r1-r2) + 2 sinh r1 sinh r2 s^2 < cosh R
// with s = sin((phi1 - phi2)/2) computed from the same doubles the caller
// sees.  Relative error a few ulp, far inside the 1e-12 tie band.
__device__ __forceinline__ double cosh_dist64(double r1, double phi1, double r2, double phi2)
{
    // fixed operand order: both endpoints of a pair get the same value
    if (r1 > r2 || (r1 == r2 && phi1 > phi2)) {
        const double tr = r1, tp = phi1;
        r1 = r2; phi1 = phi2; r2 = tr; phi2 = tp;
    }
    const double s = sin_small64(0.5 * (phi1 - phi2));
    return cosh(r1 - r2) + 2.0 * sinh(r1) * sinh(r2) * (s * s);
}

__device__ __forceinline__ bool edge64(double r1, double phi1, double r2, double phi2, double coshR)
{
    return cosh_dist64(r1, phi1, r2, phi2) < coshR;
}

// The tie band: pairs whose FP64 value lies within 1e-12 of the threshold
// (relative).  Their decision may differ between two correct FP64
// evaluations (a few ulp of rounding), so they are counted, not trusted.
constexpr double kTieBand = 1e-12;

// FP64 per-point data of the plain double-precision path
struct __align__(16) PMS64 { double P, M, S, phi; };

__device__ __forceinline__ PMS64 scaled_exps64(const Plan &p, double r, double phi)
{
    PMS64 o;
    o.P = exp(r - p.half_R);
    o.M = exp(-r - p.half_R);
    o.S = 2.0 * exp(-p.half_R) * sinh(r);
    o.phi = phi;
    return o;
}

// P1 M2 + P2 M1 + S1 S2 sin^2(dphi/2), to be compared with 1 + e^{-2R}
__device__ __forceinline__ double lhs_pms64(const PMS64 &q, const PMS64 &c)
{
    // fixed operand order: both endpoints of a pair get the same value
    const bool sw = q.P > c.P || (q.P == c.P && q.phi > c.phi);
    const PMS64 &a = sw ? c : q, &b = sw ? q : c;
    const double s = sin_small64(0.5 * (a.phi - b.phi));
    return fma(a.S * b.S, s * s, fma(a.P, b.M, b.P * a.M));
}

__device__ __forceinline__ bool edge_pms64(const Plan &p, const PMS64 &q, const PMS64 &c)
{
    return lhs_pms64(q, c) < p.rhs64;
}

// ---------------------------------------------------------------------------
// Angular window of a query in a band (replaces Proposition 1 + the range
// query of Algorithm 1).  For r_c >= b the admissible |dphi| is at most
// theta(r_q, b) with sin^2(theta/2) = X = (cosh R - cosh(r_q - b)) /
// (2 sinh r_q sinh b) = (1 + e^{-2R} - P_q M_b - P_b M_q) / (S_q S_b): the
// bound over the band is at its inner radius b, since dX/dr_c has the sign of
// cosh r_q - cosh R cosh r_c < 0.  Computed in FP32 and padded so that it
// never excludes a neighbour; returns the half-width in fixed-point angle
// units, or ~0 (all ones) for the whole circle.
//
// Why the pads suffice (u = 2^-24, the FP32 unit roundoff):
//  * inputs: P_q, M_q carry <= 3 u relative (expf <= 2 ulp, its argument kept
//    to 2^-40 as a float pair), S_q <= 5 u (expm1f <= 1 ulp, the rounding of
//    r to float moves e^{-2r} by <= u relative to 1 - e^{-2r}); the band
//    constants and 1 + e^{-2R} are rounded once (<= u);
//  * sub = P_q M_b + P_b M_q (non-negative terms) is within ~6 u relative,
//    num = (1 + e^{-2R}) - sub within u (1 + e^{-2R}) + 6 u sub + u |num|
//    absolute: below 1e-6 (1 + sub), covered 20 times by the absolute pad
//    2e-5 (1 + sub);
//  * den = S_q S_b (~7 u), its reciprocal (u) and the product (u): ~1e-6
//    relative, covered by the relative pad 2e-5 on num, so X >= the exact X;
//  * theta = 2 sqrt(X / (1 - X)) >= 2 asin(sqrt X) (X <= 1/4) or 2 asinf(sqrt
//    X) (asinf <= 2 ulp, sqrtf and 1 - X <= u each): the X pad carries over
//    as >= 9e-6 relative, above those ~5 u; theta is padded by 2e-5 more;
//  * the fixed-point conversion multiplies by 2^64 / 2pi rounded up and
//    rounds up, and adds 2^16 units: the angles A of the two endpoints are
//    within 2^12 units of their exact values each (angle_key), so their
//    difference within 2^13, and a sampled point is filed by a key within
//    2^12 of its A (sampled_angle_key): 3 2^12 in all, covered 5 times.
// The plain FP64 path uses the same windows: they are a superset; every
// candidate inside is decided by the predicate.
// ---------------------------------------------------------------------------
constexpr uint64_t kFullCircle = 0xFFFFFFFFFFFFFFFFull;

// ceil(x) as an unsigned 64-bit integer for 0 <= x < 2^64, from two 32-bit
// conversions (a 64-bit conversion is an order of magnitude slower).  For
// x < 2^32 the high word is 0; for x >= 2^32, x is a multiple of 2^9, so
// x - hi 2^32 is exact in float and integral, and hi = floor(x 2^-32) is
// exact as a float too.
__device__ __forceinline__ uint64_t float_to_u64_ru(float x)
{
    const float xh = floorf(x * 2.3283064365386963e-10f);  // x 2^-32 is exact
    const float rem = fmaf(-xh, 4294967296.0f, x);
    return ((uint64_t)__float2uint_rz(xh) << 32) + __float2uint_ru(rem);
}

__device__ __forceinline__ uint64_t window_halfwidth(const Plan &p, const PMS &q, int band)
{
    const float Pb = p.Pb[band], Mb = p.Mb[band], Sb = p.Sb[band];
    const float den = q.S * Sb;
    if (!(den > 0.0f)) return kFullCircle;
    const float inv = __frcp_rn(den);
    const float sub = fmaf(q.P, Mb, Pb * q.M);
    const float num = p.rhs32 - sub;
    // X = num / den, padded by 2e-5 relative (the division's and den's
    // roundings, ~1e-6) and 2e-5 (1 + sub) absolute (the difference's, ~1e-6 (1 + sub))
    float X = fmaf(num, 1.0f + 2e-5f, 2e-5f * (1.0f + sub)) * inv;
    if (X >= 1.0f) return kFullCircle;
    if (!(X > 0.0f)) X = 0.0f;
    // theta = 2 asin(sqrt X); for X <= 1/4 the bound asin(y) <= y / sqrt(1 - y^2)
    // (asin y = atan(y / sqrt(1 - y^2))) avoids asinf at < 9% extra width
    float th = X <= 0.25f ? 2.0f * sqrtf(X * __frcp_rn(1.0f - X)) : 2.0f * asinf(sqrtf(X));
    th = th * (1.0f + 2e-5f) + 1e-30f;  // the asinf / sqrtf roundings (~5 u) and the scaling below (u)
    if (th >= 3.1415f) return kFullCircle;
    // 2^16 units: the two endpoints' fixed-point angles are each within 2^12
    // of exact, and a sampled point's filing key within 2^12 of its angle
    return float_to_u64_ru(th * kAngleScaleUp) + (1ull << 16);
}

}  // namespace hrg

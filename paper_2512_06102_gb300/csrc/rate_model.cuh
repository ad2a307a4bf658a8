// rate_model.cuh -- the per-(target, direction) ignition rate of Eqs. 1-4,
// evaluated in float with double-float (hi + lo) steps where the exponent
// needs them, so that the rate is within ~4e-7 relative of its exact value.
//
//   r(v, d) = gamma(v) * p_base (1 + mu_veg(u)) (1 + mu_den(u))
//             * exp(alpha_w1 V(u) + alpha_w2 V(u) (cos(d pi/4 - Theta(u)) - 1)
//                   + alpha_s S(u, d)),          u = v - Delta_d
//   S(u, d) = degrees(atan((z(v) - z(u)) / (cell_size |Delta_d|)))
//
// Every operation is an explicit intrinsic (no operator the compiler could
// contract differently in two kernels), so every kernel that includes this
// header computes bit-identical rates.
#pragma once

#include <stdint.h>

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return quick_two_sum(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
// 1 / a for a > 0: approximate reciprocal refined by one exact-residual step
__device__ __forceinline__ df df_rcp(df a) {
    const float r0 = __fdividef(1.0f, a.hi);
    const float e = __fmaf_rn(-r0, a.lo, __fmaf_rn(-r0, a.hi, 1.0f));   // 1 - r0 a
    return quick_two_sum(r0, __fmul_rn(r0, e));
}

// Constants prepared on the host in double precision.
struct RateConsts {
    df atan_th[65];      // theta_k = k pi/256, k = 0..64
    df atan_tan[65];     // tan(theta_k)
    df half_pi;
    df slope_coef;       // alpha_s * 180 / pi: exponent per radian of slope
    df inv_run[8];       // 1 / (cell_size |Delta_d|)
    float G[16][16];     // gamma(c_v) * p_base (1 + mu_veg(c_u)) (1 + mu_den(c_u)), [c_v][c_u]
};

// atan of a double-float to ~1e-9 absolute: reduce to b = |x| <= 1 (via
// atan(x) = pi/2 - atan(1/x)), pick the node theta_k nearest atan(b), and use
// atan(b) = theta_k + atan(u), u = (b - tan theta_k) / (1 + b tan theta_k),
// |u| < 0.012, atan(u) = u - u^3/3 + u^5/5 (truncation below 1e-15).
__device__ __forceinline__ df atan_df(df x, const RateConsts& K) {
    const bool neg = x.hi < 0.f;
    const df a = neg ? df_neg(x) : x;
    const bool inv = a.hi > 1.0f;
    const df b = inv ? df_rcp(a) : a;
    // estimate of atan(b) on [0, 1] within 5e-3 rad, to pick the node
    const float est = __fdividef(b.hi, __fmaf_rn(0.28f, __fmul_rn(b.hi, b.hi), 1.0f));
    int k = __float2int_rn(__fmul_rn(est, 81.48733086305042f));       // 256 / pi
    k = min(max(k, 0), 64);
    const df t = K.atan_tan[k];
    const df num = df_add(b, df_neg(t));
    const df den = df_add({1.0f, 0.0f}, df_mul(b, t));
    const float u = __fdividef(__fadd_rn(num.hi, num.lo), den.hi);
    const float u2 = __fmul_rn(u, u);
    const float at_u = __fmaf_rn(__fmul_rn(u, u2), __fmaf_rn(u2, 0.2f, -0.33333334f), u);
    df th = df_add(K.atan_th[k], {at_u, 0.0f});
    if (inv) th = df_add(K.half_pi, df_neg(th));
    return neg ? df_neg(th) : th;
}

// Rate into target v from the source u in direction d.  wexp_d: the wind part
// of the exponent at u (alpha_w1 V + alpha_w2 V (cos - 1)) as hi + lo.
// G: the class-pair factor K.G[c_v][c_u] (0 when either cell has no fuel).
__device__ __forceinline__ float rate_of(float G, float z_v, float z_u, df wexp_d, int d,
                                         const RateConsts& K) {
    if (G == 0.f) return 0.f;
    const df dz = two_sum(z_v, -z_u);
    const df slope = atan_df(df_mul(dz, K.inv_run[d]), K);          // radians, Eq. 2
    const df E = df_add(wexp_d, df_mul(K.slope_coef, slope));        // Eqs. 1-2 exponent
    const float kh = expf(E.hi);
    return __fmul_rn(G, __fmaf_rn(kh, E.lo, kh));                   // Eqs. 3-4
}

// 1 - exp(-r)
__device__ __forceinline__ float prob_of(float r) { return -expm1f(-r); }

// The ignition probability in plain float: the steps of rate_of without the
// lo parts, the exponentials by __expf.  Returns p_f and sets *B to a bound on
// |p_f - prob_of(rate_of(...))| (four times the sum of the steps' errors):
//   slope angle                   within 1e-6 rad (reciprocal and quotient by
//                                 __fdividef, 2 ulp; the node table's hi parts;
//                                 series truncated at u^7/7 < 1e-14)
//   exponent E                    within 1.3e-6 |alpha_s 180/pi| + 1.2e-7 |E|
//   __expf(E)                     within (2 + 1.16 |E|) ulp (its documented bound)
//   1 - __expf(-r)                within 4e-7 absolute
//   prob_of(rate_of(...))         within 1e-6 relative of the exact value
// so |p_f - p| <= |p_f| (1.3e-6 |c_s| + 2.6e-7 |E| + 1.7e-6) + 5e-7.
__device__ __forceinline__ float prob_fast(float G, float z_v, float z_u, float wexp_hi, int d, const RateConsts& K,
                                           float* B) {
    const float x = __fmul_rn(__fsub_rn(z_v, z_u), K.inv_run[d].hi);
    const float ax = fabsf(x);
    const bool inv = ax > 1.0f;
    const float b = inv ? __fdividef(1.0f, ax) : ax;
    const float est = __fdividef(b, __fmaf_rn(0.28f, __fmul_rn(b, b), 1.0f));
    int k = __float2int_rn(__fmul_rn(est, 81.48733086305042f));       // 256 / pi
    k = min(max(k, 0), 64);
    const float t = K.atan_tan[k].hi;
    const float v = __fdividef(__fsub_rn(b, t), __fmaf_rn(b, t, 1.0f));
    const float v2 = __fmul_rn(v, v);
    float at = __fadd_rn(K.atan_th[k].hi, __fmaf_rn(__fmul_rn(v, v2), __fmaf_rn(v2, 0.2f, -0.33333334f), v));
    if (inv) at = __fsub_rn(K.half_pi.hi, at);
    const float slope = x < 0.f ? -at : at;
    const float E = __fmaf_rn(K.slope_coef.hi, slope, wexp_hi);
    const float r = __fmul_rn(G, __expf(E));
    const float p = __fsub_rn(1.0f, __expf(-r));
    const float rel = __fmaf_rn(5.2e-6f, fabsf(K.slope_coef.hi), __fmaf_rn(1.04e-6f, fabsf(E), 6.8e-6f));
    *B = __fmaf_rn(fabsf(p), rel, 2.0e-6f);
    return p;
}

// u < prob_of(rate_of(G, z_v, z_u, wexp_d, d, K)), for a draw u in [0, 1):
// decided by prob_fast when u is farther than its bound from p_f (all but a
// fraction of about 1e-5 of the draws), else by the double-float rate.  The
// answer is the same either way.
__device__ __forceinline__ bool below_prob(float u, float G, float z_v, float z_u, df wexp_d, int d,
                                           const RateConsts& K) {
    if (G == 0.f) return false;                 // rate 0: probability 0
    float B;
    const float p = prob_fast(G, z_v, z_u, wexp_d.hi, d, K, &B);
    if (u < __fsub_rn(p, B)) return true;
    if (u >= __fadd_rn(p, B)) return false;
    return u < prob_of(rate_of(G, z_v, z_u, wexp_d, d, K));
}

// eri_device.cuh -- device-side building blocks shared by the ERI kernels:
// plan data views, constant tables, the Boys function and the Rys roots/weights.
//
// arXiv 2303.13632, Sec. II-C: the Rys quadrature needs the roots t_mu and weights w_mu
// of order n_Rys for T = rho |P-Q|^2 (the input R_Rys, Eq. 5).  The paper computes them
// on the CPU in FP64 (footnote of Sec. II-C); here they are evaluated on the GPU in FP64
// from piecewise polynomials (Chebyshev fits in monomial form, T below a per-order threshold)
// or the Gauss-Hermite limit (T above it), both generated offline with 40-digit arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace eri {

constexpr int kRysNmax = 9;
constexpr int kRysDeg = 12;
constexpr int kRysTail = 10;  // coefficients j >= kRysTail are evaluated in FP32
// Mixed-precision setup (the B, C and weights are rounded to FP32 afterwards): coefficients
// j >= kRysTailMixed of the root/weight pieces and j >= kBoysTailMixed of the F_0/F_1 Taylor
// series in FP32 (tails below 3.5e-3 and 1.3e-3 of the value, so the FP32 rounding of the tail
// moves the result by about 1e-9 relative, far below the FP32 rounding that follows)
constexpr int kRysTailMixed = 4;
constexpr int kBoysTailMixed = 2;
constexpr int kBoysMmax = 16;
constexpr int kBoysTaylor = 10;
constexpr int kBoysCols = kBoysMmax + kBoysTaylor + 1;
constexpr double kBoysStep = 0.1;
constexpr double kBoysTmax = 50.0;
constexpr int kBoysNgrid = 502;
constexpr double kPi = 3.14159265358979323846;

// 1/j for the Taylor terms of the Boys function (a product with a rounded reciprocal instead of
// an FP64 division; the terms it scales are corrections below 5e-2 of the sum).
__device__ __forceinline__ double inv_int(int j) {
    constexpr double t[kBoysTaylor + 1] = {0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5,
                                          1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10};
    return t[j];
}

// Conversions between binary64 and binary32 on the integer pipe.  On this part the FP64
// conversion instructions issue on the FP64 pipe, at the FP64 rate, and so do 64-bit integer
// operations; the setup stages hand every B, C and weight value to the FP32 recurrences, so
// they convert with 32-bit integer operations on the two halves instead.  Both are exact
// IEEE-754 conversions (binary64 -> binary32 rounds to nearest, ties to even), including
// subnormal results, overflow to infinity and NaN, with no floating-point instruction.
__device__ __forceinline__ float f64_to_f32(double d) {
    const unsigned int hi = (unsigned int)__double2hiint(d), lo = (unsigned int)__double2loint(d);
    const unsigned int sign = hi & 0x80000000u, ahi = hi & 0x7FFFFFFFu;
    const unsigned int e = ahi >> 20;
    if (e - 897u <= 253u) {
        // normal binary32 result: rebias the exponent (1023 -> 127), keep 20 + 3 fraction
        // bits, round on the 29 dropped bits (a carry increments the exponent, up to infinity)
        const unsigned int t = __funnelshift_l(lo, ahi - (896u << 20), 3);
        const unsigned int rem = lo & 0x1FFFFFFFu;
        const unsigned int up = (rem > 0x10000000u) | ((rem == 0x10000000u) & t);
        return __uint_as_float(sign | (t + (up & 1u)));
    }
    if (e >= 1151u) {  // beyond the binary32 range: infinity, or NaN (quiet, top payload bits)
        const bool nan = e == 2047u && ((ahi & 0xFFFFFu) | lo) != 0u;
        return __uint_as_float(sign | (nan ? 0x7FC00000u | __funnelshift_l(lo, ahi & 0xFFFFFu, 3)
                                           : 0x7F800000u));
    }
    // subnormal binary32 result (or zero): the 53-bit significand shifted right by 926 - e
    // bits (>= 30), rounded to nearest even; a carry into bit 23 gives the smallest normal
    const unsigned int sh = 926u - e;
    if (e == 0u || sh > 54u) return __uint_as_float(sign);
    const unsigned int mh = (ahi & 0xFFFFFu) | 0x100000u;  // significand bits 32..52
    // q = significand >> sh; the dropped part compared with half
    unsigned int q, rem_hi, rem_lo, half_hi, half_lo;
    if (sh < 32u) {  // sh in [30, 31]
        q = __funnelshift_r(lo, mh, sh);
        rem_hi = 0u;
        rem_lo = lo & ((1u << sh) - 1u);
        half_hi = 0u;
        half_lo = 1u << (sh - 1u);
    } else {
        const unsigned int s2 = sh - 32u;  // 0..22
        q = mh >> s2;
        rem_hi = mh & ((1u << s2) - 1u);
        rem_lo = lo;
        half_hi = s2 ? 1u << (s2 - 1u) : 0u;
        half_lo = s2 ? 0u : 0x80000000u;
    }
    const bool gt = rem_hi > half_hi || (rem_hi == half_hi && rem_lo > half_lo);
    const bool eq = rem_hi == half_hi && rem_lo == half_lo;
    return __uint_as_float(sign | (q + ((gt || (eq && (q & 1u))) ? 1u : 0u)));
}

__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int sign = u & 0x80000000u, a = u & 0x7FFFFFFFu;
    if (a - 0x00800000u < 0x7F000000u)  // normal: exponent field 1..254
        return __hiloint2double((int)(sign | ((a >> 3) + (896u << 20))), (int)(a << 29));
    if (a >= 0x7F800000u)  // infinity or NaN: all-ones exponent, fraction moved up
        return __hiloint2double((int)(sign | 0x7FF00000u | ((a & 0x007FFFFFu) >> 3)), (int)(a << 29));
    if (a == 0u) return __hiloint2double((int)sign, 0);
    // subnormal: value a * 2^-149 with its leading one at bit p; fraction bits below it moved
    // to the top of the 52-bit field
    const int p = 31 - __clz((int)a);
    const unsigned int fr = p ? a << (32 - p) : 0u;  // fraction bits below the leading one, left-aligned
    return __hiloint2double((int)(sign | ((unsigned int)(p + 874) << 20) | (fr >> 12)),
                            (int)(fr << 20));
}

// Rounding of an FP64 setup value to the recurrence type R.
template <typename R>
__device__ __forceinline__ R to_r(double v) {
    if constexpr (sizeof(R) == 4)
        return f64_to_f32(v);
    else
        return v;
}

// Two-float numbers (value = h + l, |l| <= 2^-24 |h|): FP32 arithmetic with about 2^-46
// relative precision, for the mixed setup's B and C values, whose differences cancel (C00 =
// (P - A) - q x / (p + q) (P - Q) vanishes where the root-weighted centre meets A).
struct F2 {
    float h, l;
};

// Two-float form of an FP64 value with integer operations only: h is the value rounded to
// FP32 (as f64_to_f32), l the rounding remainder d - h, formed from the 29 significand bits
// that h drops (truncated to 24 bits).  h + l equals d to 2^-47 relative where h is a normal
// FP32 number and the remainder is above the FP32 normal range (|d| >= 2^-74); otherwise l is
// 0 and h alone stands for d.
__device__ __forceinline__ F2 split_f2(double d) {
    const unsigned int hi = (unsigned int)__double2hiint(d), lo = (unsigned int)__double2loint(d);
    const unsigned int sign = hi & 0x80000000u, ahi = hi & 0x7FFFFFFFu;
    const unsigned int e = ahi >> 20;
    if (e - 897u > 253u) return {f64_to_f32(d), 0.0f};
    const unsigned int t = __funnelshift_l(lo, ahi - (896u << 20), 3);
    const unsigned int rem = lo & 0x1FFFFFFFu;
    const unsigned int up = ((rem > 0x10000000u) | ((rem == 0x10000000u) & t)) & 1u;
    const float h = __uint_as_float(sign | (t + up));
    // d - h = r 2^(e - 1075) with r = rem (rounded down) or rem - 2^29 (rounded up)
    const unsigned int m = up ? 0x20000000u - rem : rem;  // |r| <= 2^28
    const unsigned int rsign = up ? (sign ^ 0x80000000u) : sign;
    if (m == 0u) return {h, 0.0f};
    const int p = 31 - __clz((int)m);  // leading one of |r|
    const int ef = p + (int)e - 948;   // binary32 exponent field of |r| 2^(e - 1075)
    if (ef < 1) return {h, 0.0f};
    const unsigned int mant = p >= 23 ? m >> (p - 23) : m << (23 - p);
    return {h, __uint_as_float(rsign | ((unsigned int)ef << 23) | (mant & 0x7FFFFFu))};
}

// a - b x: the product of the high parts is exact inside the first FMA and the cross terms
// (a.l - b.h x.l - b.l x.h) enter as a correction; b.l x.l (2^-48 of b x) is dropped.  Error
// below 2^-23 |a - b x| + 2^-46 (|a| + |b x|).
__device__ __forceinline__ float tf_fms(F2 a, F2 b, F2 x) {
    const float h = fmaf(-b.h, x.h, a.h);
    float c = fmaf(-b.h, x.l, a.l);
    c = fmaf(-b.l, x.h, c);
    return __fadd_rn(h, c);
}

// a b (Dekker's product of the high parts through an FMA, plus the cross terms)
__device__ __forceinline__ F2 tf_mul(F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return {p, e};
}

// a + b (Knuth's two-sum of the high parts, plus the low parts)
__device__ __forceinline__ F2 tf_add(F2 a, F2 b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ F2 tf_neg(F2 a) { return {-a.h, -a.l}; }

// Device addresses of the generated tables (see eri_tables.cu).
struct Tables {
    const double *rys_poly;  // monomial coefficients of the Rys root/weight pieces
    const float *rys_tail;   // FP32 copies of coefficients kRysTail..kRysDeg of every piece
    const double *herm_x2;
    const double *herm_w;
    const double *boys_grid;
    const double *boys_t01;  // F_0, F_1 Taylor coefficients divided by j! (kBoysTaylor each)
    const float *rys_tail_m;  // FP32 copies of coefficients kRysTailMixed..kRysDeg of every piece
    const float *boys_t01_f;  // FP32 copy of boys_t01
    int tasym[kRysNmax + 1];
    long long offset[kRysNmax + 1];
    int herm_off[kRysNmax + 2];
};

// Shell table of a plan on the device (structure of arrays).
struct ShellsDev {
    const double *cx, *cy, *cz;  // centres
    const int *pofs;             // first primitive
    const int *nprim;            // primitives per shell
    const double *exps;          // exponents
    const double *cn;            // contraction coefficient times N(alpha, L)
};

// One class launch: inputs, outputs and latch.  The kernel computes the canonical class
// (Sec. II-B, Eq. 3) of the quartets' generic class: canonical shell slot k takes the
// quartet's shell perm[k], and the canonical component tuple (i0, i1, i2, i3) is stored at
// generic offset i0*ostride[0] + i1*ostride[1] + i2*ostride[2] + i3*ostride[3].
struct ClassArgs {
    int perm[4];
    int ostride[4];
    const int4 *quartets;  // class-sorted shell ids, first quartet of the class
    long long nq;          // quartets of the class
    double *out_fp64;      // FP64 output of the class (null in compressed mode)
    uint32_t *packed;      // first word of the class segment (null in FP64 mode)
    long long seg_words;   // words of the class segment (incl. zero padding)
    float *scales;         // eps of the class's first quartet
    int bits;              // 2..24 in compressed mode
    int *err;              // device error latch (bit 0: non-finite result)
    const void *setup;     // per-quartet setup values from the setup kernel, or null
    long long setup_stride;  // elements between two fields of the setup buffer
    const double *pairs;   // primitive-pair table (kPairFields per pair, index pa * np + pb), or null
    long long np;          // primitives of the plan (row length of the pair table)
};

// Primitive-pair record: the Gaussian-product quantities of primitives (pa, pb) of shells
// (X, Y) that do not depend on the other pair (Sec. II-A): p = a + b, 1/p, P - X =
// -(b/p)(X - Y), and exp(-ab/p |X - Y|^2) times both coefficient x normalisation factors.
enum PairField { PR_P = 0, PR_IP, PR_PAX, PR_PAY, PR_PAZ, PR_KCN, kPairFields };

// Launch options of a class kernel (see launch_class).
struct LaunchOpts {
    int force_phase = 0;
    unsigned long long *counter = nullptr;
    int grid = 0;
    int device = 0;
    void *scratch = nullptr;  // setup buffer for the split setup/recurrence path (K = 1)
};

// Boys function F_m(T), m = 0..mmax (mmax <= kBoysMmax).  For T < 50: Taylor series of
// F_mmax about the nearest grid point T_k (|T - T_k| <= 0.05, ten terms; the derivative is
// dF_m/dT = -F_{m+1}) and the stable downward recursion
// F_m = (2T F_{m+1} + exp(-T)) / (2m+1).  For T >= 50: F_0 = sqrt(pi/T)/2 (erf(sqrt T) = 1
// to double precision there) and the upward recursion F_{m+1} = ((2m+1)F_m - exp(-T))/(2T).
__device__ __forceinline__ void boys_eval(int mmax, double T, const double *__restrict__ grid,
                                          double *F) {
    double eT = exp(-T);
    if (T < kBoysTmax) {
        int k = __double2int_rn(T * (1.0 / kBoysStep));
        double d = k * kBoysStep - T;  // expansion in (-delta)
        const double *g = grid + k * kBoysCols + mmax;
        double s = __ldg(g + kBoysTaylor - 1);
#pragma unroll
        for (int j = kBoysTaylor - 1; j >= 1; --j) s = fma(s, d * inv_int(j), __ldg(g + j - 1));
        F[mmax] = s;
        for (int m = mmax - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + eT) / (2 * m + 1);
    } else {
        F[0] = 0.5 * sqrt(kPi / T);
        double inv2T = 0.5 / T;
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - eT) * inv2T;
    }
}

// F_0(T) and, when WANT1, F_1(T) without exp(): Taylor series of each order about the grid
// point for T < 50; beyond, F_0 = sqrt(pi/T)/2 and F_1 = F_0/(2T) (the exp(-T) terms are below
// 1e-20 relative there).
template <bool WANT1>
__device__ __forceinline__ void boys_f01(double T, const double *__restrict__ t01, double &F0,
                                         double &F1) {
    // grid point from an FP32 copy of T (no FP64 conversion instruction): any point within
    // 0.05 (plus FP32 rounding) serves, since d below is formed exactly in FP64
    const int k = __float2int_rn(f64_to_f32(T) * (float)(1.0 / kBoysStep));
    if (k <= (int)(kBoysTmax / kBoysStep)) {
        // F_m(T_k - d) = sum_j F_{m+j}(T_k) / j! d^j with the 1/j! folded into the table
        double d = fma(f32_to_f64((float)k), kBoysStep, -T);
        const double *g = t01 + k * (2 * kBoysTaylor);
        double s0 = __ldg(g + kBoysTaylor - 1);
        double s1 = WANT1 ? __ldg(g + 2 * kBoysTaylor - 1) : 0.0;
#pragma unroll
        for (int j = kBoysTaylor - 2; j >= 0; --j) {
            s0 = fma(s0, d, __ldg(g + j));
            if (WANT1) s1 = fma(s1, d, __ldg(g + kBoysTaylor + j));
        }
        F0 = s0;
        F1 = s1;
    } else {
        F0 = 0.5 * sqrt(kPi / T);
        F1 = WANT1 ? F0 * (0.5 / T) : 0.0;
    }
}

// Polynomial sum_j a_j u^j of degree kRysDeg by Horner's rule: the terms j >= kRysTail
// (below 1e-9 of the value on every piece, checked when the tables are generated) in FP32 from
// FP32 coefficients and u rounded to FP32, the rest in FP64; the result stays accurate to
// FP64 rounding (verified by emulating exactly this evaluation at generation time).
__device__ __forceinline__ double poly_eval(const double *__restrict__ a,
                                            const float *__restrict__ at, double u) {
    const float uf = f64_to_f32(u);
    float sf = __ldg(at + (kRysDeg - kRysTail));
#pragma unroll
    for (int j = kRysDeg - 1; j >= kRysTail; --j) sf = fmaf(sf, uf, __ldg(at + (j - kRysTail)));
    double s = f32_to_f64(sf);
#pragma unroll
    for (int j = kRysTail - 1; j >= 0; --j) s = fma(s, u, __ldg(a + j));
    return s;
}

// 1/v and 1/sqrt(v) for the mixed-precision setup: the FP32 approximation of the special-
// function unit (PTX rcp.approx / rsqrt.approx, relative error below 2^-22) refined by one
// Newton-Raphson step in FP64, r' = r + r (1 - v r) and r' = r + (r/2)(1 - v r^2), which squares
// the relative error (to about 1e-13), for v in the FP32 normal range.
__device__ __forceinline__ float rcp_approx_f32(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float rsqrt_approx_f32(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ double recip_nr(double v) {
    const double r = f32_to_f64(rcp_approx_f32(f64_to_f32(v)));
    return fma(r, fma(-v, r, 1.0), r);
}
__device__ __forceinline__ double rsqrt_nr(double v) {
    const double r = f32_to_f64(rsqrt_approx_f32(f64_to_f32(v)));
    const double e = fma(-v * r, r, 1.0);  // 1 - v r^2
    return fma(0.5 * r, e, r);
}

// boys_f01 of the mixed-precision setup: terms j >= kBoysTailMixed of the Taylor series in FP32
// (from boys_t01_f and d rounded to FP32), the rest in FP64; beyond the grid F_0 = sqrt(pi/T)/2
// with 1/sqrt(T) from rsqrt_nr.
template <bool WANT1>
__device__ __forceinline__ void boys_f01_mixed(double T, const double *__restrict__ t01,
                                               const float *__restrict__ t01f, double &F0, double &F1) {
    const int k = __float2int_rn(f64_to_f32(T) * (float)(1.0 / kBoysStep));
    if (k <= (int)(kBoysTmax / kBoysStep)) {
        const double d = fma(f32_to_f64((float)k), kBoysStep, -T);
        const float df = f64_to_f32(d);
        const double *g = t01 + k * (2 * kBoysTaylor);
        const float *gf = t01f + k * (2 * kBoysTaylor);
        float s0f = __ldg(gf + kBoysTaylor - 1);
        float s1f = WANT1 ? __ldg(gf + 2 * kBoysTaylor - 1) : 0.0f;
#pragma unroll
        for (int j = kBoysTaylor - 2; j >= kBoysTailMixed; --j) {
            s0f = fmaf(s0f, df, __ldg(gf + j));
            if (WANT1) s1f = fmaf(s1f, df, __ldg(gf + kBoysTaylor + j));
        }
        double s0 = f32_to_f64(s0f), s1 = WANT1 ? f32_to_f64(s1f) : 0.0;
#pragma unroll
        for (int j = kBoysTailMixed - 1; j >= 0; --j) {
            s0 = fma(s0, d, __ldg(g + j));
            if (WANT1) s1 = fma(s1, d, __ldg(g + kBoysTaylor + j));
        }
        F0 = s0;
        F1 = s1;
    } else {
        const double rs = rsqrt_nr(T);
        F0 = 0.88622692545275801365 * rs;  // sqrt(pi) / 2
        F1 = WANT1 ? F0 * (0.5 * rs * rs) : 0.0;
    }
}

// poly_eval of the mixed-precision setup: terms j >= kRysTailMixed in FP32.
__device__ __forceinline__ double poly_eval_mixed(const double *__restrict__ a,
                                                  const float *__restrict__ at, double u) {
    const float uf = f64_to_f32(u);
    float sf = __ldg(at + (kRysDeg - kRysTailMixed));
#pragma unroll
    for (int j = kRysDeg - 1; j >= kRysTailMixed; --j) sf = fmaf(sf, uf, __ldg(at + (j - kRysTailMixed)));
    double s = f32_to_f64(sf);
#pragma unroll
    for (int j = kRysTailMixed - 1; j >= 0; --j) s = fma(s, u, __ldg(a + j));
    return s;
}

// Root mu (0-based, ascending) and weight of the order-n Rys rule at T.  MIXED: the evaluation
// of the mixed-precision setup (FP32 tails, Newton-refined reciprocals; about 1e-9 relative).
template <bool MIXED = false>
__device__ __forceinline__ void rys_root(const Tables &tb, int n, int mu, double T, double &x,
                                         double &w) {
    if (n == 1) {
        double F0, F1;
        if constexpr (MIXED) {
            boys_f01_mixed<true>(T, tb.boys_t01, tb.boys_t01_f, F0, F1);
            w = F0;
            x = F1 * recip_nr(F0);
        } else {
            boys_f01<true>(T, tb.boys_t01, F0, F1);
            w = F0;
            x = F1 / F0;
        }
        return;
    }
    // unit interval from an FP32 copy of T (no FP64 conversion instruction); when FP32
    // rounding lifts T to the next integer (T < 90: by less than 4e-6), u lands within 1e-5
    // below -1, where the degree-12 fit still holds to the same accuracy
    const int k = (int)f64_to_f32(T);
    if (k < tb.tasym[n]) {
        double u = 2.0 * (T - f32_to_f64((float)k)) - 1.0;
        const long long f = (tb.offset[n] / (kRysDeg + 1)) + (long long)k * (2 * n) + 2 * mu;
        const double *c = tb.rys_poly + f * (kRysDeg + 1);
        if constexpr (MIXED) {
            const float *ct = tb.rys_tail_m + f * (kRysDeg + 1 - kRysTailMixed);
            x = poly_eval_mixed(c, ct, u);
            w = poly_eval_mixed(c + (kRysDeg + 1), ct + (kRysDeg + 1 - kRysTailMixed), u);
        } else {
            const float *ct = tb.rys_tail + f * (kRysDeg + 1 - kRysTail);
            x = poly_eval(c, ct, u);
            w = poly_eval(c + (kRysDeg + 1), ct + (kRysDeg + 1 - kRysTail), u);
        }
    } else {
        int h = tb.herm_off[n] + mu;
        if constexpr (MIXED) {
            const double rs = rsqrt_nr(T);
            x = __ldg(tb.herm_x2 + h) * (rs * rs);
            w = __ldg(tb.herm_w + h) * rs;
        } else {
            x = __ldg(tb.herm_x2 + h) / T;
            w = __ldg(tb.herm_w + h) * rsqrt(T);
        }
    }
}

__host__ __device__ constexpr int ncart(int L) { return (L + 1) * (L + 2) / 2; }

// Cartesian components (a_x, a_y, a_z) of index idx in a shell of angular momentum L.
static __constant__ int c_cart[5][15][3] = {
    {{0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}},
    {{3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2}, {0, 3, 0}, {0, 2, 1},
     {0, 1, 2}, {0, 0, 3}},
    {{4, 0, 0}, {3, 1, 0}, {3, 0, 1}, {2, 2, 0}, {2, 1, 1}, {2, 0, 2}, {1, 3, 0}, {1, 2, 1},
     {1, 1, 2}, {1, 0, 3}, {0, 4, 0}, {0, 3, 1}, {0, 2, 2}, {0, 1, 3}, {0, 0, 4}}};

// Cartesian component of index idx in a shell of angular momentum L (order: a_x from L
// down to 0, then a_y from L - a_x down to 0).
__host__ __device__ constexpr int cart_x(int L, int idx) {
    int k = 0;
    for (int ax = L; ax >= 0; --ax)
        for (int ay = L - ax; ay >= 0; --ay) {
            if (k == idx) return ax;
            ++k;
        }
    return -1;
}
__host__ __device__ constexpr int cart_y(int L, int idx) {
    int k = 0;
    for (int ax = L; ax >= 0; --ax)
        for (int ay = L - ax; ay >= 0; --ay) {
            if (k == idx) return ay;
            ++k;
        }
    return -1;
}
__host__ __device__ constexpr int cart_z(int L, int idx) { return L - cart_x(L, idx) - cart_y(L, idx); }

}  // namespace eri

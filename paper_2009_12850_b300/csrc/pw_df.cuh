// pw_df.cuh -- packed double-float arithmetic for the FP64 "split" stencil.
//
// A double x is carried as an unevaluated pair of floats (hi, lo) with
// x = hi + lo + d, |d| <= 2^-46 |x|.  Two consecutive k levels are processed
// together in Blackwell's packed FP32 instructions (add/sub/mul/fma .f32x2),
// so a P2 holds (level k, level k+1) and a D2 holds the hi and lo parts of two
// levels.  Arithmetic follows the classical error-free transformations:
//   TwoSum (Knuth):    s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a,
//                      a + b = s + e exactly;
//   TwoProd (FMA):     p = a * b, e = fma(a, b, -p),  a * b = p + e exactly;
// and the "lazy" double-float add and multiply built on them, which skip the
// final renormalisation: their results stay accurate to a few units of 2^-46
// relative to the sum of the magnitudes involved, which is what the stencil's
// error bound (1e-12 of the per-point condition sum) needs.
//
// Conversions avoid the FP64 pipe (f64<->f32 conversions run at the DP rate on
// B300): doubles are split with integer bit operations, and results are
// rebuilt from (hi, lo) with integer widening plus one FP64 add.
#pragma once

#include <stdint.h>

struct P2 {
    unsigned long long v;
};
struct D2 {
    P2 h, l;
};

__device__ __forceinline__ P2 pk(float a, float b) {
    P2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
// the lane of a pair (the other half of the unpack is left unused)
#pragma nv_diag_suppress 550
__device__ __forceinline__ float lx(P2 a) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
    return x;
}
__device__ __forceinline__ float ly(P2 a) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
    return y;
}
#pragma nv_diag_default 550
__device__ __forceinline__ P2 operator+(P2 a, P2 b) {
    P2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 operator-(P2 a, P2 b) {
    P2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 operator*(P2 a, P2 b) {
    P2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 pfma(P2 a, P2 b, P2 c) {
    P2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// a*b = p + e exactly (the error by scalar FMAs, which negate for free)
__device__ __forceinline__ P2 two_prod_err(P2 a, P2 b, P2 p) {
    return pk(fmaf(lx(a), lx(b), -lx(p)), fmaf(ly(a), ly(b), -ly(p)));
}

// lazy double-float sum / difference: TwoSum of the hi parts, lo parts added
__device__ __forceinline__ D2 df_add(D2 a, D2 b) {
    P2 s = a.h + b.h;
    P2 bb = s - a.h;
    P2 e = (a.h - (s - bb)) + (b.h - bb);
    return D2{s, e + (a.l + b.l)};
}
__device__ __forceinline__ D2 df_sub(D2 a, D2 b) {
    P2 s = a.h - b.h;
    P2 bb = s - a.h;
    P2 e = (a.h - (s - bb)) - (b.h + bb);
    return D2{s, e + (a.l - b.l)};
}
// lazy double-float product (the lo*lo term is below 2^-46 and dropped)
__device__ __forceinline__ D2 df_mul(D2 a, D2 b) {
    P2 p = a.h * b.h;
    P2 e = two_prod_err(a.h, b.h, p);
    e = pfma(a.h, b.l, e);
    e = pfma(a.l, b.h, e);
    return D2{p, e};
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
// Range of the split arithmetic.  Every field value is carried scaled by 2^8
// (an exact exponent shift taken in the split itself), so every source, being
// quadratic in the fields, comes out scaled by 2^16 and the join removes it.
// With the mesh coefficients checked when the mesh is made (tcx, tcy and the
// vertical coefficients in [2^-16, 2^8], the density factors 0.25 rho in
// [2^-36, 2^24]) no intermediate product can overflow while the winds stay
// below 2^40 in magnitude and the scalars, which only meet products with a
// wind factor, below 2^60.  Larger values, NaN and Inf are read as 0 and
// reported.  Nonzero values below 2^-110 are read as 0 without a report: the
// split is exact from there up, and what is lost below is far under the
// absolute error floor that underflow of the FP32 intermediates sets anyway.
#define PW_SPLIT_SCALE_LOG2 8
// biased FP64 exponents, shifted to the exponent field of the high word
#define PW_SPLIT_ELO (913u << 20)          // 2^-110: smaller values read as 0
#define PW_SPLIT_WIND_EHI (1063u << 20)    // 2^40: this and above is out of range
#define PW_SPLIT_SCALAR_EHI (1083u << 20)  // 2^60

// Split a double, given as its two 32-bit words, into (hi, lo) of 2^8 x: hi =
// 2^8 x truncated to 24 significant bits, lo = the next 23 bits (an exact float
// subtraction removes the implicit bit), so |2^8 x - hi - lo| < 2^-46 |2^8 x|.
// Integer operations plus one FP32 subtraction.  A value whose biased exponent
// lies outside [PW_SPLIT_ELO, ehi) (shifted left by 20) gives (0, 0); one at or
// above ehi (too large, Inf or NaN) also sets `bad`.
__device__ __forceinline__ void split_words(uint32_t xl, uint32_t xh, float &hi, float &lo, uint32_t ehi,
                                            bool &bad) {
    // top 23 mantissa bits and the low 9 exponent bits; adding 136 << 23 sets
    // the float exponent field to (e_double - 1023 + 127 + 8) mod 256
    const uint32_t f = __funnelshift_l(xl, xh, 3) + 0x44000000u;
    const uint32_t hb = (f & 0x7fffffffu) | (xh & 0x80000000u);
    // lo: 1.m x 2^(e-23) minus 2^(e-23), with m the next 23 mantissa bits
    const uint32_t cb = (hb & 0xff800000u) - 0x0b800000u;
    const uint32_t fb = cb | ((xl >> 6) & 0x007fffffu);
    const uint32_t e = xh & 0x7ff00000u;
    const bool inr = (e - PW_SPLIT_ELO) < (ehi - PW_SPLIT_ELO);
    bad |= e >= ehi;
    hi = inr ? __uint_as_float(hb) : 0.0f;
    lo = inr ? __uint_as_float(fb) - __uint_as_float(cb) : 0.0f;
}

// 2^-16 f as a double, by integer widening, for normal floats only (no zero or
// subnormal handling: those come out as a number of magnitude below 2^-142,
// inside the absolute error floor of the split arithmetic).
__device__ __forceinline__ double widen_normal(float f) {
    const uint32_t b = __float_as_uint(f);
    // exponent rebias 127 -> 1023 less the 2^16 scale of the sources
    const uint32_t h = (((b & 0x7fffffffu) >> 3) + 0x37000000u) | (b & 0x80000000u);
    return __hiloint2double((int)h, (int)(b << 29));
}

// 2^-16 (hi + lo) rounded to double with one FP64 add: the source held in
// scaled double-float form, returned unscaled.  Only the exact-zero case needs
// care: when hi != 0 a zero or subnormal lo is below half an ulp of any result
// in range, and when hi == 0 a normal lo is widened exactly.
__device__ __forceinline__ double join(float hi, float lo) {
    const double d = widen_normal(hi) + widen_normal(lo);
    return (hi == 0.0f && lo == 0.0f) ? 0.0 : d;
}

// ---------------------------------------------------------------------------
// access to the split stencils' tables and converted planes
// ---------------------------------------------------------------------------
// coefficient table (floats): 8 arrays of cs_n levels starting at level -2:
// g_h g_l gp_h gp_l r_h r_l rp_h rp_l, then tcx_h tcx_l tcy_h tcy_l
__device__ __forceinline__ D2 cs_pair(const float *cs, int n, int arr, int k) {
    const float *h = cs + (2 * arr) * n + k + 2;
    const float *l = cs + (2 * arr + 1) * n + k + 2;
    return D2{pk(h[0], h[1]), pk(l[0], l[1])};
}

// D2 of levels (k+s, k+1+s), s in {-1, 0, 1}, from a converted plane row
template <int S>
__device__ __forceinline__ D2 ld2(const double *row, int kk) {
    const float4 c = *reinterpret_cast<const float4 *>(row + kk);
    if (S == 0) return D2{pk(c.x, c.y), pk(c.z, c.w)};
    if (S < 0) {
        const float4 m = *reinterpret_cast<const float4 *>(row + kk - 2);
        return D2{pk(m.y, c.x), pk(m.w, c.z)};
    }
    const float4 p = *reinterpret_cast<const float4 *>(row + kk + 2);
    return D2{pk(c.y, p.x), pk(c.w, p.z)};
}

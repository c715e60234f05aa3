// Double-float arithmetic for complex128 sweeps on the FP32 pipes.
//
// A double x is carried as an unevaluated sum hi + lo of two floats (Dekker,
// "A floating-point technique for extending the available precision",
// Numer. Math. 18, 1971).  Products use the FMA form of Dekker's exact
// product (p = a*b rounded, e = fma(a, b, -p) exact); sums use Knuth's
// TwoSum (TAOCP vol. 2, Sec. 4.2.2), which returns the rounded sum and its
// exact rounding error without any assumption on the operands' order; a dot
// product accumulates the rounded terms with TwoSum and every error term in
// a float correction (the compensated dot product "Dot2" of Ogita, Rump and
// Oishi, SIAM J. Sci. Comput. 26, 2005).  The result carries about 48 bits.
//
// Conversions between the IEEE double storage and the float pair use integer
// operations only (no FP64 instruction): on this part the FP64 pipe runs at
// 1/64 of the FP32 rate, which is what made complex128 sweeps ALU-bound.
//   split: hi = x truncated to 24 significant bits (an exponent rebase and a
//          funnel shift of the bit pattern), lo = the remaining 29 fraction
//          bits converted to float (rounded to 24) and scaled by 2^(e-1075);
//   join:  the double nearest to hi + lo, assembled in a 64-bit integer
//          from hi's 24-bit significand and lo scaled to the result's last
//          place (lo is at most half an ulp of hi after normalisation).
// split reports doubles outside [2^-74, 2^77) (other than zero and the
// subnormals, which become zero): there lo would underflow, or hi overflow,
// the float range, and the caller computes that element in FP64 instead.
#pragma once

#include <cstdint>

namespace qsim {
namespace dfl {

// Split x into hi + lo; returns false when x is outside the range where both
// parts are normal floats.  Zero and subnormal doubles (|x| < 2^-1022) give
// hi = lo = 0 (an absolute error below 2.3e-308).
__device__ __forceinline__ bool split(double x, float &hi, float &lo) {
    const uint32_t H = uint32_t(__double2hiint(x)), L = uint32_t(__double2loint(x));
    const uint32_t sgn = H & 0x80000000u;
    const uint32_t e = (H >> 20) & 0x7FFu;  // biased double exponent
    // hi: the float exponent is e - 1023 + 127 = e - 896; the 23 fraction
    // bits are the double's top 20 (of H) and 3 (of L)
    const uint32_t t = H - (896u << 20);
    const float h = __uint_as_float((__funnelshift_l(L, t, 3) & 0x7FFFFFFFu) | sgn);
    // lo = (L mod 2^29) * 2^(e - 1075); the scale 2^(e - 1075) is a normal
    // float for e >= 949
    const float scale = __uint_as_float((e - 948u) << 23);
    const float l = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(L & 0x1FFFFFFFu), scale)) | sgn);
    const bool zero = e == 0u;
    hi = zero ? 0.f : h;
    lo = zero ? 0.f : l;
    return zero || e - 949u < 1100u - 949u;
}

// The double nearest to hi + lo, for hi = 0 or a normal float and |lo| <=
// ulp(hi) / 2.  Branch free, and mostly on the FP32 and conversion pipes: lo
// is scaled (exactly, by a power of two built from hi's exponent) into units
// of the result's last place and rounded to an integer t (|t| <= 2^28); the
// 53-bit significand is then hi's 24 bits shifted up by 29 plus t, with
// signs taken into account, renormalised by one bit if a negative t took it
// below 2^52.  When hi < 2^-75, lo is below 2^-99 and is dropped.
__device__ __forceinline__ double join(float hi, float lo) {
    const uint32_t hb = __float_as_uint(hi);
    const uint32_t ef = hb & 0x7F800000u;  // hi's exponent field
    // 2^(179 - eh) as a float: exponent field (306 - eh) << 23
    const float scale = __uint_as_float(0x99000000u - ef);
    const int tl = __float2int_rn(__fmul_rn(lo, scale));  // lo in units of 2^(eh - 179)
    const int t = ef >= (52u << 23) ? tl : 0;
    const int ts = (hb & 0x80000000u) ? -t : t;  // added to |hi|
    const uint64_t m = (uint64_t((hb & 0x7FFFFFu) | 0x800000u) << 29) + uint64_t(int64_t(ts));
    const uint32_t below = m < (uint64_t(1) << 52) ? 1u : 0u;
    const uint64_t mn = m << below;
    const uint64_t ex = uint64_t((ef >> 23) + 896u - below) << 52;
    const uint64_t bits = (uint64_t(hb & 0x80000000u) << 32) | ex | (mn & ((uint64_t(1) << 52) - 1));
    return __longlong_as_double((long long)(ef ? bits : 0ull));
}

// Compensated dot product of double-float values: sum_k a_k * b_k with a_k
// and b_k given as (hi, lo) pairs; the cross term lo * lo (2^-48 relative to
// its product) is dropped.
struct Dot {
    float s, c;  // rounded running sum, correction
    __device__ __forceinline__ void first(float ah, float al, float bh, float bl) {
        s = __fmul_rn(ah, bh);
        c = fmaf(ah, bh, -s);
        c = fmaf(ah, bl, c);
        c = fmaf(al, bh, c);
    }
    __device__ __forceinline__ void add(float ah, float al, float bh, float bl) {
        const float p = __fmul_rn(ah, bh);
        const float e = fmaf(ah, bh, -p);
        const float s1 = __fadd_rn(s, p);  // TwoSum(s, p): s1 + t = s + p exactly
        const float bv = __fadd_rn(s1, -s);
        const float t = __fadd_rn(__fadd_rn(s, -__fadd_rn(s1, -bv)), __fadd_rn(p, -bv));
        s = s1;
        c = fmaf(ah, bl, fmaf(al, bh, __fadd_rn(c, __fadd_rn(t, e))));
    }
    // normalised (hi, lo) = TwoSum(s, c): |lo| <= ulp(hi) / 2 whatever the
    // operands' magnitudes (after cancellation c may exceed s)
    __device__ __forceinline__ void result(float &hi, float &lo) const {
        hi = __fadd_rn(s, c);
        const float bv = __fadd_rn(hi, -s);
        lo = __fadd_rn(__fadd_rn(s, -__fadd_rn(hi, -bv)), __fadd_rn(c, -bv));
    }
};

}  // namespace dfl
}  // namespace qsim

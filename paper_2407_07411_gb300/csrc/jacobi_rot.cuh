// Jacobi rotation shared by the Rayleigh-Ritz eigensolver (two-sided, davidson.cu) and
// the one-sided SVD of the truncation (svd.cu).
//
// This GPU has few FP64 units: a warp-wide FP64 instruction holds an SM sub-partition's
// FP64 pipe for tens of clocks whatever its active lanes, and a round of Jacobi rotations
// is a dependent chain through one warp.  So the rotation and the test that decides
// whether to rotate use as few FP64 instructions as possible: exponents, scaling and
// the conversions between FP64 and FP32 are done on the bit patterns with integer
// operations, the angle in FP32, and the correction that makes (c, s) orthonormal in
// double in 64-bit integer arithmetic; two fused multiply-adds form c and s.
#pragma once
#include <cstdint>

namespace dmrg {

// Biased exponent field of a double (0 for zero and subnormals).
__device__ __forceinline__ int jr_exp(double x) { return int((__double_as_longlong(x) >> 52) & 0x7FF); }

// Whether the pair (p, q) is rotated: |apq| above ~1e-15 sqrt|app aqq| (a smaller entry
// moves the eigenvalues by < ~1e-30 relative, and rotations below rounding level only
// regenerate rounding noise).  Compared on exponent fields, 2 e(apq) > e(app) + e(aqq) -
// 99, which places the threshold within a factor 2 of 2^-49.5 |app aqq|^(1/2); zero and
// subnormal apq are never rotated.
__device__ __forceinline__ bool jacobi_rotate_needed(double apq, double app, double aqq) {
    const int ea = jr_exp(apq);
    return ea != 0 && 2 * ea > jr_exp(app) + jr_exp(aqq) - 99;
}

// x 2^(1023 - eb) as a float (truncated), x with bit pattern b and exponent field e <= eb;
// 0 when it falls below the normal FP32 range.
__device__ __forceinline__ float jr_scaled_float(long long b, int e, int eb) {
    const int ef = e - eb + 127;
    if (e == 0 || ef <= 0) return 0.0f;
    const unsigned hi = unsigned(static_cast<unsigned long long>(b) >> 32), lo = unsigned(b);
    return __uint_as_float((hi & 0x80000000u) | (unsigned(ef) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// The double equal to a normal float given by its bit pattern (0 for zero).
__device__ __forceinline__ double jr_float_to_double(unsigned fb) {
    const unsigned e = (fb >> 23) & 0xFF;
    if (e == 0) return 0.0;
    return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(fb & 0x80000000u) << 32) |
                                                       (static_cast<unsigned long long>(e + 896) << 52) |
                                                       (static_cast<unsigned long long>(fb & 0x7FFFFFu) << 29)));
}

// Jacobi rotation (c, s) that annihilates apq of the 2 x 2 block [[app, apq], [apq, aqq]],
// d = aqq - app: t = tan of the angle is the root of smaller magnitude of
// t^2 + 2 tau t - 1 = 0, tau = d / (2 apq).  The angle is formed in single precision from
// d and apq scaled by 2^-E, E the larger exponent; with c0, s0 the single-precision cosine
// and sine, c0^2 + s0^2 = 1 + delta (|delta| < 2^-20), and (c, s) = (c0, s0) (1 + rho) with
// rho = (1 + delta)^(-1/2) - 1 = -delta / 2 + 3 delta^2 / 8 + O(delta^3).  c0 = C 2^-24 and
// s0 are 24-bit integers times powers of two, so delta is formed exactly in units of
// 2^-62 from C^2 and the aligned S^2 (only bits of s0^2 below 2^-62 are dropped), and rho
// in the same units; c = fma(c0, rho, c0) is then orthonormal with s to double rounding.
// The angle's single-precision error leaves |apq| reduced by ~2^-22 of its scale instead
// of to zero, which the next sweep removes.  apq must be non-zero.
__device__ __forceinline__ void jacobi_rotation(double d, double apq, double* c, double* s) {
    const long long bd = __double_as_longlong(d), ba = __double_as_longlong(apq);
    const int ed = int((bd >> 52) & 0x7FF), ea = int((ba >> 52) & 0x7FF);
    const int eb = max(ed, ea);
    const float df = jr_scaled_float(bd, ed, eb), af = jr_scaled_float(ba, ea, eb);
    if (!(fabsf(af) > 1e-18f * fabsf(df))) {   // angle below 1e-18: t = apq / d, cos 1 to double
        *c = 1.0;
        *s = apq / d;
        return;
    }
    const float tau = df / (2.0f * af);
    const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
    const float cf = rsqrtf(fmaf(t, t, 1.0f));   // in [2^-1/2, 1] up to rounding: exponent field 126 or 127
    const float sf = t * cf;
    const unsigned cb = __float_as_uint(cf), sb = __float_as_uint(sf);
    const int ec = int((cb >> 23) & 0xFF), es = int((sb >> 23) & 0xFF);
    // c0 = Cu 2^-24 (Cu <= 2^24 + 2), s0 = Sm 2^(es - 150); both squares in units of 2^-62
    const unsigned long long Cu = static_cast<unsigned long long>((cb & 0x7FFFFFu) | 0x800000u) << min(max(ec - 126, 0), 1);
    const unsigned long long Sm = es ? static_cast<unsigned long long>((sb & 0x7FFFFFu) | 0x800000u) : 0ull;
    const unsigned long long S2 = Sm * Sm;
    const int sh = 2 * es - 238;   // <= 14 for |s0| < 1
    const unsigned long long s2u = sh >= 0 ? (S2 << min(sh, 14)) : (sh > -64 ? (S2 >> (-sh)) : 0ull);
    const long long D = static_cast<long long>((Cu * Cu) << 14) + static_cast<long long>(s2u) - (1ll << 62);
    const long long q = D >> 20;   // |D| < 2^43: q^2 fits, and (q^2 >> 22) is D^2 2^-62 to a few units
    const long long R = -(D >> 1) + ((3 * ((q * q) >> 22)) >> 3);
    double rho = 0.0;   // R 2^-62, built from its bits (|R| < 2^52, so exact)
    if (R != 0) {
        const unsigned long long ar = R < 0 ? static_cast<unsigned long long>(-R) : static_cast<unsigned long long>(R);
        const int L = 63 - __clzll(static_cast<long long>(ar));
        rho = __longlong_as_double(static_cast<long long>((R < 0 ? (1ull << 63) : 0ull) |
                                                          (static_cast<unsigned long long>(L + 961) << 52) |
                                                          ((ar << (52 - L)) & 0xFFFFFFFFFFFFFull)));
    }
    const double c0 = jr_float_to_double(cb), s0 = jr_float_to_double(sb);
    *c = fma(c0, rho, c0);
    *s = fma(s0, rho, s0);
}

}  // namespace dmrg

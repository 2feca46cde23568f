// Jacobi rotation shared by the Rayleigh-Ritz eigensolver (two-sided, davidson.cu) and
// the one-sided SVD of the truncation (svd.cu).
#pragma once
#include <cstdint>

namespace dmrg {

// Jacobi rotation (c, s) that annihilates apq of the 2 x 2 block [[app, apq], [apq, aqq]],
// d = aqq - app: t = tan of the angle is the root of smaller magnitude of
// t^2 + 2 tau t - 1 = 0, tau = d / (2 apq).  Double-precision division and square roots
// are long dependent chains on this GPU's few FP64 units, so the angle is formed in
// single precision from d and apq scaled by a power of two (exact), and the pair is then
// made orthonormal to double precision: with c, s the single-precision cosine and sine,
// c^2 + s^2 = 1 + delta (|delta| < 2^-20), and c, s are divided by sqrt(1 + delta) =
// 1 + delta / 2 - delta^2 / 8 + O(delta^3) through the series 1 - delta / 2 +
// 3 delta^2 / 8 of its reciprocal.  The rotation is exactly orthogonal; the angle's
// single-precision error leaves |apq| reduced by ~2^-22 of its scale instead of to zero,
// which the next sweep removes (convergence is judged on the rounding-level threshold).
__device__ __forceinline__ void jacobi_rotation(double d, double apq, double* c, double* s) {
    // scale by 2^-E, E the exponent of the larger magnitude (bit patterns; exact)
    const long long em = max(__double_as_longlong(d) & 0x7FF0000000000000ll,
                             __double_as_longlong(apq) & 0x7FF0000000000000ll);
    const double sc = __longlong_as_double((2046ll << 52) - em);
    const float df = float(d * sc), af = float(apq * sc);
    if (!(fabsf(af) > 1e-18f * fabsf(df))) {   // angle below 1e-18: t = apq / d, cos 1 to double
        *c = 1.0;
        *s = apq / d;
        return;
    }
    const float tau = df / (2.0f * af);
    const float t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
    const float cf = rsqrtf(fmaf(t, t, 1.0f));
    const double c0 = cf, s0 = double(t * cf);
    const double delta = fma(c0, c0, fma(s0, s0, -1.0));
    const double r = fma(delta, fma(delta, 0.375, -0.5), 1.0);
    *c = c0 * r;
    *s = s0 * r;
}


}  // namespace dmrg

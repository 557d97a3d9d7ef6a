// Device-side building blocks of the pulse-noise step (arXiv:1610.04914):
// the counter-based noise generator, Box-Muller, the pulse rotation and the
// right-hand side of the noiseless Landau-Lifshitz equation.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spin {

// Key word 1 of the noise stream ("noise" in ASCII).
constexpr uint64_t kStreamNoise = 0x6E6F697365ULL;

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each
// multiplying counter words 0 and 2 by the two round constants, crossing the
// high halves with words 1 and 3 and the key, then bumping the key by the
// two Weyl increments.
struct Words4 {
    uint64_t w[4];
};

// 64x64 -> 128-bit product: low word by the wrapping multiply, high word by
// the compiler's multiply-high intrinsic.
__device__ __forceinline__ void mul64_wide(uint64_t a, uint64_t m, uint64_t& hi, uint64_t& lo) {
    lo = a * m;
    hi = __umul64hi(a, m);
}

__device__ __forceinline__ Words4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1) {
    constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ULL;
    constexpr uint64_t kMulB = 0xCA5A826395121157ULL;
    constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ULL;
    constexpr uint64_t kWeylB = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t hiA, loA, hiB, loB;
        mul64_wide(c0, kMulA, hiA, loA);
        mul64_wide(c2, kMulB, hiB, loB);
        const uint64_t n0 = hiB ^ c1 ^ k0;
        const uint64_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return Words4{{c0, c1, c2, c3}};
}

__device__ __forceinline__ Words4 noise_words(uint64_t seed, uint64_t site, uint64_t k, uint64_t replica) {
    return philox4x64_10(site, k, replica, 0ULL, seed, kStreamNoise);
}

// Box-Muller.  Uniforms are u = ((w >> 11) + 1/2) 2^-53 in (0, 1); G0, G1 from
// (u0, u1) and G2 from (u2, u3).
template <typename real>
struct Gauss;

template <>
struct Gauss<double> {
    __device__ __forceinline__ static void draw(const Words4& w, double& g0, double& g1, double& g2) {
        const double scale = 1.0 / 9007199254740992.0;  // 2^-53
        const double u0 = ((double)(w.w[0] >> 11) + 0.5) * scale;
        const double u1 = ((double)(w.w[1] >> 11) + 0.5) * scale;
        const double u2 = ((double)(w.w[2] >> 11) + 0.5) * scale;
        const double u3 = ((double)(w.w[3] >> 11) + 0.5) * scale;
        const double r0 = sqrt(-2.0 * log(u0));
        const double r2 = sqrt(-2.0 * log(u2));
        double s1, c1, s3, c3;
        sincospi(2.0 * u1, &s1, &c1);
        sincospi(2.0 * u3, &s3, &c3);
        g0 = r0 * c1;
        g1 = r0 * s1;
        g2 = r2 * c3;
    }
};

template <>
struct Gauss<float> {
    // Same real numbers as the double path, each rounded once to float: the
    // 54-bit odd integer 2(w>>11)+1 converts with relative error 2^-24 at any
    // magnitude, so small u keep their relative precision in the logarithm.
    __device__ __forceinline__ static float u01(uint64_t w) {
        return __ull2float_rn(((w >> 11) << 1) | 1ULL) * 5.5511151231257827e-17f;  // 2^-54
    }
    __device__ __forceinline__ static void draw(const Words4& w, float& g0, float& g1, float& g2) {
        const float u0 = u01(w.w[0]), u1 = u01(w.w[1]), u2 = u01(w.w[2]), u3 = u01(w.w[3]);
        const float r0 = sqrtf(-2.0f * logf(u0));
        const float r2 = sqrtf(-2.0f * logf(u2));
        float s1, c1, s3, c3;
        sincospif(2.0f * u1, &s1, &c1);
        sincospif(2.0f * u3, &s3, &c3);
        g0 = r0 * c1;
        g1 = r0 * s1;
        g2 = r2 * c3;
    }
};

template <typename real>
struct Math;
template <>
struct Math<float> {
    __device__ __forceinline__ static float rsqrt_(float x) { return rsqrtf(x); }
    __device__ __forceinline__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ __forceinline__ static void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
};
template <>
struct Math<double> {
    __device__ __forceinline__ static double rsqrt_(double x) { return 1.0 / sqrt(x); }
    __device__ __forceinline__ static double sqrt_(double x) { return sqrt(x); }
    __device__ __forceinline__ static void sincos_(double x, double* s, double* c) { sincos(x, s, c); }
};

// Rotation of s by the angle vector phi = sigma G, Eq. (s_rotation):
//   s' = s cos(phi) + (n x s) sin(phi) + n (n.s)(1 - cos(phi)),  n = phi/|phi|.
template <typename real>
__device__ __forceinline__ void pulse_rotate(real& sx, real& sy, real& sz, real px, real py, real pz) {
    const real phi2 = px * px + py * py + pz * pz;
    if (phi2 > real(0)) {
        const real phi = Math<real>::sqrt_(phi2);
        const real inv = real(1) / phi;
        const real nx = px * inv, ny = py * inv, nz = pz * inv;
        real sn, cs;
        Math<real>::sincos_(phi, &sn, &cs);
        const real ns = nx * sx + ny * sy + nz * sz;
        const real om = (real(1) - cs) * ns;
        const real cx = ny * sz - nz * sy;
        const real cy = nz * sx - nx * sz;
        const real cz = nx * sy - ny * sx;
        const real ox = sx * cs + cx * sn + nx * om;
        const real oy = sy * cs + cy * sn + ny * om;
        const real oz = sz * cs + cz * sn + nz * om;
        sx = ox;
        sy = oy;
        sz = oz;
    }
}

// One pulse on one site: draw G_i for pulse k, rotate by sigma G_i.
template <typename real>
__device__ __forceinline__ void pulse_site(real& sx, real& sy, real& sz, uint64_t seed, uint64_t site,
                                           uint64_t k, uint64_t replica, real sigma) {
    const Words4 w = noise_words(seed, site, k, replica);
    real g0, g1, g2;
    Gauss<real>::draw(w, g0, g1, g2);
    pulse_rotate<real>(sx, sy, sz, sigma * g0, sigma * g1, sigma * g2);
}

// Exact float -> double for FP64 accumulation of FP32 terms: sign, exponent
// rebased from 127 to 1023, mantissa shifted into the top of the 52-bit field
// -- integer operations only, because this GPU's FP64 pipe, which the
// hardware conversion uses, runs at ~1/76 of the FP32 rate and is needed for
// the FP64 additions themselves.  Zeros keep their sign; subnormal, infinite
// and NaN floats take the hardware conversion.
__device__ __forceinline__ double to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if ((b & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)sign);
    if (e == 0u || e == 0xFFu) return (double)f;
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double to_f64(double d) { return d; }

// Right-hand side of Eq. (LLL) with a rectangular-noise field zeta, which
// enters the precession term only:  f = s x (H + zeta) - lambda s x (s x H).
template <typename real>
__device__ __forceinline__ void llg_rhs_noise(real sx, real sy, real sz, real hx, real hy, real hz, real zx,
                                              real zy, real zz, real lambda, real& fx, real& fy, real& fz) {
    const real cx = sy * hz - sz * hy;
    const real cy = sz * hx - sx * hz;
    const real cz = sx * hy - sy * hx;
    const real bx = sy * cz - sz * cy;
    const real by = sz * cx - sx * cz;
    const real bz = sx * cy - sy * cx;
    const real px = hx + zx, py = hy + zy, pz = hz + zz;
    fx = (sy * pz - sz * py) - lambda * bx;
    fy = (sz * px - sx * pz) - lambda * by;
    fz = (sx * py - sy * px) - lambda * bz;
}

// Right-hand side of Eq. (LLL) without noise, given H_eff = (hx, hy, hz):
//   a = s x H,  b = s x a
//   precessional: f = a - lambda b;   slow (precession dropped): f = -lambda b
template <typename real, bool PREC>
__device__ __forceinline__ void llg_rhs(real sx, real sy, real sz, real hx, real hy, real hz, real lambda,
                                        real& fx, real& fy, real& fz) {
    const real ax = sy * hz - sz * hy;
    const real ay = sz * hx - sx * hz;
    const real az = sx * hy - sy * hx;
    const real bx = sy * az - sz * ay;
    const real by = sz * ax - sx * az;
    const real bz = sx * ay - sy * ax;
    if (PREC) {
        fx = ax - lambda * bx;
        fy = ay - lambda * by;
        fz = az - lambda * bz;
    } else {
        fx = -lambda * bx;
        fy = -lambda * by;
        fz = -lambda * bz;
    }
}

}  // namespace spin

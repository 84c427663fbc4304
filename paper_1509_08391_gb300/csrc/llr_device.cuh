// llr_device.cuh -- device-side building blocks of the LLR sweep kernels:
// Philox4x32-10, uniforms, angle wrap, the fixed-point energy format and the
// per-lattice state record.  Internal to the CUDA library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace llr {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (hi, lo) = M * c products xored with the key, key bumped by the Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// Uniform in the open interval (0,1): (2 * (w >> 9) + 1) * 2^-24, exact in float,
// formed without an integer-to-float conversion: the float 1.m with the top 23
// bits of w as mantissa is 1 + (w >> 9) 2^-23, and subtracting 1 - 2^-24 (exact:
// the difference is representable) leaves (2 (w >> 9) + 1) 2^-24.
__device__ __forceinline__ float u01(uint32_t w)
{
    return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994039535522f;
}

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;

// Wrap to [-pi, pi).
__device__ __forceinline__ float wrap_angle(float t)
{
    return t - kTwoPi * floorf((t + kPi) * (1.0f / kTwoPi));
}

// sqrt(x) for x >= 0 as x times the hardware reciprocal square root (a few
// ulp; the sampler's parameters and an angle's sine need no IEEE-rounded
// sqrtf).  sqrt(0) = 0.
__device__ __forceinline__ float sqrt_fast(float x)
{
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

// arg(x + i y) in [-pi, pi] in float32, for the staple direction and the new
// heat-bath angle.  With t = min(|x|, |y|) / max(|x|, |y|) in [0, 1],
// atan t = t P(t^2), P the degree-7 polynomial whose t P(t^2) has the least
// maximum absolute error from atan t on [0, 1] (Remez exchange: 3.7e-8; with
// float32 coefficients and Horner evaluation 1.4e-7, plus <= 1.2e-7 from the
// quotient); then the octant: pi/2 - r where |y| > |x|, pi - r where x < 0,
// the sign of y.  arg(0) = 0.
__device__ __forceinline__ float arg_fast(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = __fdividef(mn, fmaxf(mx, 1e-30f));
    const float u = t * t;
    float p = -0.004054567310959101f;
    p = fmaf(p, u, 0.021862957626581192f);
    p = fmaf(p, u, -0.0559123270213604f);
    p = fmaf(p, u, 0.0964219719171524f);
    p = fmaf(p, u, -0.1390862911939621f);
    p = fmaf(p, u, 0.19946566224098206f);
    p = fmaf(p, u, -0.33329859375953674f);
    p = fmaf(p, u, 0.9999993443489075f);
    float r = t * p;
    r = ay > ax ? 1.57079632679489662f - r : r;
    r = x < 0.0f ? kPi - r : r;
    return copysignf(r, y);
}

// ---------------------------------------------------------------------------
// Energies on the device are int64 fixed point with 32 fractional bits
// (resolution 2.3e-10, range +-2.1e9).  Sums are exact and independent of
// the order of accumulation; the window test is an integer comparison.
// ---------------------------------------------------------------------------
constexpr double kFx = 4294967296.0;   // 2^32
constexpr double kInvFx = 1.0 / 4294967296.0;

__device__ __forceinline__ long long to_fx(float v)
{
    return __float2ll_rn(v * 4294967296.0f);
}

__device__ __forceinline__ long long dist_fx(long long E, long long lo, long long hi)
{
    return E < lo ? lo - E : (E > hi ? E - hi : 0ll);
}

// Philox counter word 2 ("tag") of each kind of draw.
constexpr uint32_t kTagSweep = 0u;
constexpr uint32_t kTagMuca = 12u;       // the multicanonical accept draw of a link
constexpr uint32_t kTagApproach = 14u;
constexpr uint32_t kTagInit = 15u;
constexpr int kSamplerMaxAttempts = 64;

// ---------------------------------------------------------------------------
// Per-lattice state, one record per (interval, replica) chain.
// ---------------------------------------------------------------------------
struct alignas(16) LatState {
    // geometry: side L, half = L^4 / 2, offset of the lattice's first float
    int L;
    int half;
    unsigned long long off;
    uint32_t magic;            // ceil(2^32 / L): q = umulhi(n, magic) = n / L for n < 2^24
    uint32_t key0, key1;       // Philox key
    uint32_t sweep;            // composite sweeps done (Philox counter word 1)
    // window and energy
    long long E_fx;            // tracked energy
    long long lo_fx, hi_fx;    // window, ceil(E_lo 2^32) .. floor((E_lo+dE) 2^32)
    double E_lo, dE;
    double a;                  // slope used by the current sweeps
    // measurement of the current Robbins-Monro step
    double sum_dE, sum_dE2;
    int n_meas;
    int status;
    // statistics
    unsigned long long hb_acc, hb_tot, or_acc, or_tot, caps;
    double max_drift;
    unsigned long long sweeps_done;
};

}  // namespace llr

// mpr_device.cuh -- device building blocks of the MPR sweeps: Philox-4x32-10, storage
// conversions and the precision-dispatched math of the three precision axes of Sec. 2
// (spins X_S, energy X_E, functions X_F).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mpr {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr float kTwoPiF = 6.28318530717958647692f;

// ---------------------------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplies
// whose halves are mixed with the other two words and the round key; the key advances by the
// golden-ratio and sqrt(3)-1 Weyl constants between rounds. One IMAD.WIDE per product.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * x.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x.z;
        x = make_uint4((uint32_t)(p1 >> 32) ^ x.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ x.w ^ k1, (uint32_t)p0);
    }
    return x;
}

// Random stream of a site pair: counter (x >> 2, y, sweep, problem << 8 | tag << 1 | colour),
// key = seed. The pair's first site (half-lattice column j even) takes words (x, y), the second
// (j odd) takes (z, w); the first word of a site drives its proposal or initial angle, the
// second its acceptance test. (The initial angles of every setup and the Metropolis moves of
// the FP64-function setting use this layout; the FP32-function Metropolis moves call the same
// function with counter (g, h, sweep, problem << 8 | sub << 2 | colour) for a group of eight
// sites, see mpr_tile_f32.cuh.)
enum : uint32_t { kTagMetropolis = 0, kTagInit = 1 };

__device__ __forceinline__ uint4 pair_words(uint32_t jpair, uint32_t y, uint32_t sweep,
                                            uint32_t problem, uint32_t tag, uint32_t colour,
                                            uint32_t seed_lo, uint32_t seed_hi, uint32_t sub = 0u)
{
    return philox4x32_10(make_uint4(jpair, y, sweep,
                                    (problem << 8) | (sub << 2) | (tag << 1) | colour),
                         seed_lo, seed_hi);
}

// The same words with the work that is constant over one colour pass done once, on the host or
// once per tile: the ten round keys, and the half of round 1 that depends only on the counter's
// sweep and tag words (they multiply and mix the same way for every site of the pass). Round keys
// then enter the mixing straight from kernel parameters.
struct PhiloxSched {
    uint32_t a, b, c;   // round 1: hi(M1 * sweep) ^ k0, lo(M1 * sweep), ctr.w ^ k1
    uint32_t k[18];     // keys of rounds 2 .. 10: (k0, k1) pairs
};

__host__ __device__ inline PhiloxSched philox_sched(uint32_t sweep, uint32_t problem, uint32_t tag,
                                                    uint32_t colour, uint32_t seed_lo,
                                                    uint32_t seed_hi)
{
    PhiloxSched s;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * sweep;
    s.a = (uint32_t)(p1 >> 32) ^ seed_lo;
    s.b = (uint32_t)p1;
    s.c = ((problem << 8) | (tag << 1) | colour) ^ seed_hi;
    uint32_t k0 = seed_lo, k1 = seed_hi;
    for (int r = 1; r < 10; ++r) {
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
        s.k[2 * (r - 1)] = k0;
        s.k[2 * (r - 1) + 1] = k1;
    }
    return s;
}

__device__ __forceinline__ uint4 pair_words(uint32_t jpair, uint32_t y, const PhiloxSched& s,
                                            uint32_t sub = 0u)
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * jpair;
    uint4 x = make_uint4(s.a ^ y, s.b, (uint32_t)(p0 >> 32) ^ s.c ^ (sub << 2), (uint32_t)p0);
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint64_t q0 = (uint64_t)0xD2511F53u * x.x;
        const uint64_t q1 = (uint64_t)0xCD9E8D57u * x.z;
        x = make_uint4((uint32_t)(q1 >> 32) ^ x.y ^ s.k[2 * (r - 1)], (uint32_t)q1,
                       (uint32_t)(q0 >> 32) ^ x.w ^ s.k[2 * (r - 1) + 1], (uint32_t)q0);
    }
    return x;
}

// Uniforms in [0, 1): FP64 functions take all 32 bits, FP32 functions the top 23 bits.
__device__ __forceinline__ double uniform_d(uint32_t w) { return (double)w * 2.3283064365386962890625e-10; }
// 1 + uniform_f(w), exactly: 1.m with the top 23 bits of w as mantissa (the exponent bits of 1.0
// are added: the shifted word has none, so the sum equals the bitwise or, in one shift-add).
__device__ __forceinline__ float one_plus_uniform_f(uint32_t w)
{
    return __uint_as_float((w >> 9) + 0x3f800000u);
}
// Exactly (w >> 9) * 2^-23, no conversion op. c * uniform_f(w) == fmaf(c, one_plus_uniform_f(w), -c)
// bit for bit, since both round the same exact product once.
__device__ __forceinline__ float uniform_f(uint32_t w) { return one_plus_uniform_f(w) - 1.0f; }
// 1 + m * 2^-23 for the low 23 bits m of v, exactly (one logic op).
__device__ __forceinline__ float one_plus_low23_f(uint32_t v)
{
    return __uint_as_float((v & 0x007FFFFFu) | 0x3f800000u);
}

// ---------------------------------------------------------------------------------------------
// Storage conversions
// ---------------------------------------------------------------------------------------------
template <typename F, typename S> __device__ __forceinline__ F load_as(S v);
template <> __device__ __forceinline__ double load_as<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double load_as<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double load_as<double, __half>(__half v) { return (double)__half2float(v); }
template <> __device__ __forceinline__ double load_as<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <> __device__ __forceinline__ float load_as<float, double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float load_as<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float load_as<float, __half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float load_as<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename S> __device__ __forceinline__ S store_from(double v);
template <typename S> __device__ __forceinline__ S store_from(float v);
template <> __device__ __forceinline__ double store_from<double>(double v) { return v; }
template <> __device__ __forceinline__ double store_from<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float store_from<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ float store_from<float>(float v) { return v; }
template <> __device__ __forceinline__ __half store_from<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __half store_from<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 store_from<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __nv_bfloat16 store_from<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ---------------------------------------------------------------------------------------------
// Function precision X_F: FP64 library functions, or the FP32 hardware intrinsics (Sec. 2: the
// hardware-intrinsic versions are used for all SP function evaluations).
// ---------------------------------------------------------------------------------------------
template <typename F> struct Math;

template <> struct Math<double> {
    static __device__ __forceinline__ void sincos_(double a, double* s, double* c) { sincos(a, s, c); }
    static __device__ __forceinline__ double exp_neg_over(double dE, double T, double /*invT*/) { return exp(-dE / T); }
    static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
    static __device__ __forceinline__ double uniform(uint32_t w) { return uniform_d(w); }
    static __device__ __forceinline__ double two_pi() { return kTwoPi; }
    static __device__ __forceinline__ double floor_(double v) { return floor(v); }
};

template <> struct Math<float> {
    static __device__ __forceinline__ void sincos_(float a, float* s, float* c) { __sincosf(a, s, c); }
    static __device__ __forceinline__ float exp_neg_over(float dE, float /*T*/, float invT) { return __expf(-dE * invT); }
    static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float uniform(uint32_t w) { return uniform_f(w); }
    static __device__ __forceinline__ float two_pi() { return kTwoPiF; }
    static __device__ __forceinline__ float floor_(float v) { return floorf(v); }
};

template <typename F> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

}  // namespace mpr

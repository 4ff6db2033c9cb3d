// philox.cuh -- counter-based normals for the sampler's noise, device side.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and the Weyl key schedule
// 0x9E3779B9 / 0xBB67AE85.  Box-Muller turns word pairs into normals.
//
// Counter layout (one convention for the whole library):
//   key     = (seed low 32 bits, seed high 32 bits)
//   counter = (c0 call index, c1 element index, c2 sweep, c3 tag | job << 8)
//   tags    : 0 init U, 1 init V, 2 U row noise, 3 V row noise,
//             4 U hyper normals, 5 V hyper normals, 6 U gamma, 7 V gamma
//   normal q of a stream comes from call q/4: word pair (q%4)/2, the cosine
//   branch for even q and the sine branch for odd q.
//   Uniforms take the top 24 bits of a word, so FP32 and FP64 see the same
//   value: u = ((w >> 8) + 1) * 2^-24 in (0, 1] (log argument),
//   t = (w >> 8) * 2^-24 in [0, 1) (angle); z = sqrt(-2 ln u) (cos, sin)(2 pi t).
#pragma once
#include <stdint.h>

namespace bpmf {

enum : uint32_t {
    kTagInitU = 0, kTagInitV = 1, kTagRowU = 2, kTagRowV = 3,
    kTagHyperU = 4, kTagHyperV = 5, kTagGammaU = 6, kTagGammaV = 7
};

__host__ __device__ __forceinline__ uint32_t tag_word(uint32_t tag, uint32_t job)
{
    return tag | (job << 8);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_call(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                             uint32_t c3)
{
    return philox4x32_10(make_uint4(c0, c1, c2, c3), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Two FP32 normals from two words (cosine branch in .x, sine branch in .y).
__device__ __forceinline__ float2 box_muller_f32(uint32_t wu, uint32_t wt)
{
    const float u = (float)((wu >> 8) + 1u) * 0x1p-24f;
    const float t = (float)(wt >> 8) * 0x1p-24f;
    const float rho = sqrtf(-2.0f * logf(u));
    float s, c;
    sincospif(2.0f * t, &s, &c);
    return make_float2(rho * c, rho * s);
}

// Same in FP64 (hyper-parameter draws).
__device__ __forceinline__ double2 box_muller_f64(uint32_t wu, uint32_t wt)
{
    const double u = (double)((wu >> 8) + 1u) * 0x1p-24;
    const double t = (double)(wt >> 8) * 0x1p-24;
    const double rho = sqrt(-2.0 * log(u));
    double s, c;
    sincospi(2.0 * t, &s, &c);
    return make_double2(rho * c, rho * s);
}

// Four FP32 normals of call c0 (normals 4 c0 .. 4 c0 + 3 of the stream).
__device__ __forceinline__ float4 normals4_f32(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3)
{
    const uint4 w = philox_call(seed, c0, c1, c2, c3);
    const float2 a = box_muller_f32(w.x, w.y);
    const float2 b = box_muller_f32(w.z, w.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Normal q of a stream in FP64.
__device__ __forceinline__ double normal_f64(uint64_t seed, uint32_t q, uint32_t c1, uint32_t c2,
                                             uint32_t c3)
{
    const uint4 w = philox_call(seed, q >> 2, c1, c2, c3);
    const uint32_t p = (q & 3u) >> 1;
    const double2 z = p ? box_muller_f64(w.z, w.w) : box_muller_f64(w.x, w.y);
    return (q & 1u) ? z.y : z.x;
}

}  // namespace bpmf

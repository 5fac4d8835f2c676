// Conversions between binary64 and binary32 in integer arithmetic.
//
// On B300 the FP64 pipe, which bounds the Krylov operator and Gram-Schmidt, also executes
// the hardware conversions between FP64 and FP32; the mixed V-cycle converts every entry
// of its input and of its result once per application. These routines take the same
// conversions to the integer pipes: f32_rn_of_f64 is the IEEE 754 (2008) conversion of a
// binary64 value to binary32 with roundTiesToEven (subnormal results, overflow to
// infinity, NaN kept quiet with the payload's leading bits), f64_of_f32 the exact
// widening (binary32 subnormals become normal binary64 values). Results are bit for bit
// those of the hardware conversions for every finite and infinite input.
// Host-compilable, so that the host test checks them against the C++ conversions.
#pragma once

#include <stdint.h>
#ifndef __CUDA_ARCH__
#include <string.h>
#endif

#ifdef __CUDACC__
#define GF_CVT_FN __host__ __device__ __forceinline__
#else
#define GF_CVT_FN inline
#endif

namespace gf {

GF_CVT_FN uint64_t cvt_bits64(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

GF_CVT_FN double cvt_f64(uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

GF_CVT_FN uint32_t cvt_bits32(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

GF_CVT_FN float cvt_f32(uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

GF_CVT_FN int cvt_clz32(uint32_t v)   // v != 0
{
#ifdef __CUDA_ARCH__
    return __clz((int)v);
#else
    return __builtin_clz(v);
#endif
}

// binary64 -> binary32, round to nearest, ties to even.
GF_CVT_FN float f32_rn_of_f64(double x)
{
    const uint64_t b = cvt_bits64(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffu);        // binary64 biased exponent
    const uint64_t m = b & 0x000fffffffffffffull;   // its 52 fraction bits
    if (e == 0x7ff)   // infinity, or NaN made quiet with the payload's leading 22 bits
        return cvt_f32(sign | 0x7f800000u | (m ? (0x00400000u | (uint32_t)(m >> 29)) : 0u));
    const int E = e - 896;   // binary32 biased exponent: 1023 - 127 = 896
    if (E >= 255) return cvt_f32(sign | 0x7f800000u);   // |x| >= 2^128: infinity
    if (E >= 1) {
        // normal result: keep 23 of the 52 fraction bits and round by the other 29; a carry
        // out of the fraction moves into the exponent (to infinity above the largest finite)
        const uint32_t kept = ((uint32_t)E << 23) | (uint32_t)(m >> 29);
        const uint32_t rest = (uint32_t)(m & 0x1fffffffu);
        const uint32_t up = (rest > 0x10000000u || (rest == 0x10000000u && (kept & 1u))) ? 1u : 0u;
        return cvt_f32(sign | (kept + up));
    }
    // subnormal or zero result, in units of 2^-149: the significand sig = 1.m * 2^52 times
    // 2^(e - 1075 + 149) = sig / 2^sh with sh = 926 - e >= 30
    const int sh = 926 - e;
    if (e == 0 || sh >= 54) return cvt_f32(sign);   // below 2^-150 (sig / 2^sh < 1/2): zero
    const uint64_t sig = m | 0x0010000000000000ull;
    const uint64_t k = sig >> sh;
    const uint64_t rest = sig & ((1ull << sh) - 1ull);
    const uint64_t half = 1ull << (sh - 1);
    const uint64_t up = (rest > half || (rest == half && (k & 1ull))) ? 1ull : 0ull;
    return cvt_f32(sign | (uint32_t)(k + up));   // k + up = 2^23 is the smallest normal
}

// binary32 -> binary64, exact.
GF_CVT_FN double f64_of_f32(float x)
{
    const uint32_t b = cvt_bits32(x);
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    if (e == 0xffu)   // infinity, or NaN made quiet with its payload
        return cvt_f64(sign | 0x7ff0000000000000ull | ((uint64_t)m << 29) | (m ? 0x0008000000000000ull : 0ull));
    if (e != 0) return cvt_f64(sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)m << 29));
    if (m == 0) return cvt_f64(sign);
    // subnormal: m * 2^-149 with m's leading 1 at bit p, i.e. 2^(p - 149) * (m / 2^p)
    const int p = 31 - cvt_clz32(m);
    return cvt_f64(sign | ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & 0x000fffffffffffffull));
}

// value conversion used by the kernels: the integer forms between binary64 and binary32,
// a plain cast otherwise (the same type, or conversions the hot path does not run)
template <typename To, typename From>
struct Convert {
    static GF_CVT_FN To run(From x) { return (To)x; }
};
template <>
struct Convert<float, double> {
    static GF_CVT_FN float run(double x) { return f32_rn_of_f64(x); }
};
template <>
struct Convert<double, float> {
    static GF_CVT_FN double run(float x) { return f64_of_f32(x); }
};
template <typename To, typename From>
GF_CVT_FN To convert(From x)
{
    return Convert<To, From>::run(x);
}

#ifdef __CUDACC__
// out[q] = convert<To>(in[q]), q < n (gf_round_to_f32, gf_widen_to_f64)
template <typename To, typename From>
__global__ void convert_kernel(const From* __restrict__ in, To* __restrict__ out, long long n)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = convert<To>(in[q]);
}
#endif

}  // namespace gf

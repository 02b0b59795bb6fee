// Flooding sum-product pass kernels (check-node and bit-node updates).
//
// Layout. Messages and posteriors are frame-interleaved: row x of r, app and
// lamT holds Fp consecutive frames. A warp owns one node (check or variable)
// for 32 * V consecutive frames, lane l handling frames f0 .. f0 + V - 1 with
// f0 = g * 32V + l * V, so every row access of the warp is one contiguous,
// aligned 128 * V-byte (float) segment, and the node's index loads are
// warp-uniform. blockIdx.y selects the frame group g; CTAs stride over the
// nodes of their bin.
//
// Check-node rule (Algorithm 1, "Values to Variable Nodes", LLR form):
//   |r_ij| = phi^( sum_{j' in N_i \ j} phi^(|q_ij'|) ),
//   r_ij > 0 iff an odd number of the other q_ij' are > 0,
// phi(x) = ln((e^x+1)/(e^x-1)), phi^(x) = phi(clamp(x, phi(L_MAX), L_MAX)),
// with q_ij = APP_j - r_ij (the extrinsic input of Algorithm 1's first half,
// lambda_j + sum_{i' != i} r_i'j) or q_ij = lambda_j on the first pass
// (Algorithm 3). The exclusive sums are formed without subtraction: prefix
// plus suffix sums in registers for degree <= 32, and a compensated
// (error-free two-sum) total for larger degrees, so that a dominant own term
// never cancels the small ones.
//
// Bit-node rule (Algorithm 4 / Algorithm 1 first half):
//   APP_j = lambda_j + sum_{i in M_j} r_ij.
//
// Syndrome (Algorithm 6) is fused into the next check pass: that pass already
// gathers APP_j for every edge of every check, so it xors the signs into
// z_i and ors z_i into a per-frame "unsatisfied" bit of the previous pass.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>
#include <type_traits>

#include "ldpc_launch.cuh"
#include "ldpc_pass.h"

namespace ldpc {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Message storage: float, half or bfloat16 in memory, float in registers.
// ---------------------------------------------------------------------------

template <typename M>
struct MsgIO;

template <>
struct MsgIO<float> {
    static __device__ __forceinline__ void load4(const float *p, float (&x)[4]) {
        float4 v = *reinterpret_cast<const float4 *>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    static __device__ __forceinline__ void store4(float *p, const float (&x)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
    static __device__ __forceinline__ void load2(const float *p, float (&x)[2]) {
        float2 v = *reinterpret_cast<const float2 *>(p);
        x[0] = v.x; x[1] = v.y;
    }
    static __device__ __forceinline__ void store2(float *p, const float (&x)[2]) {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    }
    static __device__ __forceinline__ float load1(const float *p) { return *p; }
    static __device__ __forceinline__ void store1(float *p, float x) { *p = x; }
};

template <>
struct MsgIO<__half> {
    static __device__ __forceinline__ void load4(const __half *p, float (&x)[4]) {
        uint2 raw = *reinterpret_cast<const uint2 *>(p);
        float2 a = __half22float2(*reinterpret_cast<__half2 *>(&raw.x));
        float2 b = __half22float2(*reinterpret_cast<__half2 *>(&raw.y));
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
    static __device__ __forceinline__ void store4(__half *p, const float (&x)[4]) {
        __half2 a = __floats2half2_rn(x[0], x[1]);
        __half2 b = __floats2half2_rn(x[2], x[3]);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t *>(&a);
        raw.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = raw;
    }
    static __device__ __forceinline__ void load2(const __half *p, float (&x)[2]) {
        float2 a = __half22float2(*reinterpret_cast<const __half2 *>(p));
        x[0] = a.x; x[1] = a.y;
    }
    static __device__ __forceinline__ void store2(__half *p, const float (&x)[2]) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(x[0], x[1]);
    }
    static __device__ __forceinline__ float load1(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void store1(__half *p, float x) { *p = __float2half_rn(x); }
};

template <>
struct MsgIO<__nv_bfloat16> {
    static __device__ __forceinline__ void load4(const __nv_bfloat16 *p, float (&x)[4]) {
        uint2 raw = *reinterpret_cast<const uint2 *>(p);
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&raw.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&raw.y));
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
    static __device__ __forceinline__ void store4(__nv_bfloat16 *p, const float (&x)[4]) {
        __nv_bfloat162 a = __floats2bfloat162_rn(x[0], x[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(x[2], x[3]);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t *>(&a);
        raw.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = raw;
    }
    static __device__ __forceinline__ void load2(const __nv_bfloat16 *p, float (&x)[2]) {
        float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
        x[0] = a.x; x[1] = a.y;
    }
    static __device__ __forceinline__ void store2(__nv_bfloat16 *p, const float (&x)[2]) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(x[0], x[1]);
    }
    static __device__ __forceinline__ float load1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store1(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
};

// int8 messages are stored as biased levels u = k + 128 (k = round(r / step),
// |k| <= 127, so 1 <= u <= 255) and converted with FP32 arithmetic instead of
// the int<->float conversion instructions, which share the transcendental
// unit with the check rule's ex2/lg2/rcp:
//  * load: one byte permute assembles the float with bit pattern
//    0x4B000000 + u, which is exactly 2^23 + u; subtracting 2^23 + 128 leaves
//    k exactly, and k * step is the message (the same product as k * step
//    from any other route, so the stored format does not change any value);
//  * store: adding 1.5 * 2^23 + 128 to r / step (|r / step| < 2^22) leaves
//    round(r / step) + 128 (ties to even) in the low mantissa bits, whose low
//    byte is u.
constexpr float kI8StoreMagic = 12583040.0f;   // 1.5 * 2^23 + 128
constexpr float kI8LoadBias = 8388736.0f;      // 2^23 + 128

template <>
struct MsgIO<int8_t> {
    // 2^23 + (byte B of w) as a float
    template <int B>
    static __device__ __forceinline__ float biased(uint32_t w) {
        uint32_t f;
        // bytes 1-3 of the result from 0x4B000000 (selectors 5, 6, 7), byte 0 from w
        asm("prmt.b32 %0, %1, 0x4B000000, %2;" : "=r"(f) : "r"(w), "n"(0x7650 | B));
        return __uint_as_float(f);
    }
    static __device__ __forceinline__ float2 values2(float a, float b) {
        return __fmul2_rn(__fadd2_rn(make_float2(a, b), make_float2(-kI8LoadBias, -kI8LoadBias)),
                          make_float2(kI8Step, kI8Step));
    }
    // the biased level of x (x clamped to +-127 steps) in the low byte
    static __device__ __forceinline__ uint32_t level_bits(float x) {
        x = fminf(fmaxf(x, -127.0f * kI8Step), 127.0f * kI8Step);
        return __float_as_uint(fmaf(x, kI8Inv, kI8StoreMagic));
    }
    // the same for two values already within +-127.5 steps (no clamp)
    static __device__ __forceinline__ float2 level_bits2(float a, float b) {
        return __ffma2_rn(make_float2(a, b), make_float2(kI8Inv, kI8Inv), make_float2(kI8StoreMagic, kI8StoreMagic));
    }
    static __device__ __forceinline__ void load4(const int8_t *p, float (&x)[4]) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(p);
        const float2 lo = values2(biased<0>(w), biased<1>(w));
        const float2 hi = values2(biased<2>(w), biased<3>(w));
        x[0] = lo.x; x[1] = lo.y; x[2] = hi.x; x[3] = hi.y;
    }
    static __device__ __forceinline__ uint32_t pack4(uint32_t b0, uint32_t b1, uint32_t b2, uint32_t b3) {
        return __byte_perm(__byte_perm(b0, b1, 0x0040u), __byte_perm(b2, b3, 0x0040u), 0x5410u);
    }
    static __device__ __forceinline__ void store4(int8_t *p, const float (&x)[4]) {
        *reinterpret_cast<uint32_t *>(p) = pack4(level_bits(x[0]), level_bits(x[1]), level_bits(x[2]), level_bits(x[3]));
    }
    // for |x| <= 127.5 steps (messages of a rule saturating at L_MAX <= 20)
    static __device__ __forceinline__ void store4_unclamped(int8_t *p, const float (&x)[4]) {
        const float2 lo = level_bits2(x[0], x[1]), hi = level_bits2(x[2], x[3]);
        *reinterpret_cast<uint32_t *>(p) =
            pack4(__float_as_uint(lo.x), __float_as_uint(lo.y), __float_as_uint(hi.x), __float_as_uint(hi.y));
    }
    static __device__ __forceinline__ void load2(const int8_t *p, float (&x)[2]) {
        const uint32_t w = *reinterpret_cast<const uint16_t *>(p);
        const float2 v = values2(biased<0>(w), biased<1>(w));
        x[0] = v.x;
        x[1] = v.y;
    }
    static __device__ __forceinline__ void store2(int8_t *p, const float (&x)[2]) {
        *reinterpret_cast<uint16_t *>(p) = (uint16_t)__byte_perm(level_bits(x[0]), level_bits(x[1]), 0x0040u);
    }
    // explicit roundings: a product left to the compiler could be fused into
    // the caller's next add, which the packed forms never do
    static __device__ __forceinline__ float load1(const int8_t *p) {
        return __fmul_rn(__fadd_rn(biased<0>((uint32_t)(uint8_t)*p), -kI8LoadBias), kI8Step);
    }
    static __device__ __forceinline__ void store1(int8_t *p, float x) { *p = (int8_t)(level_bits(x) & 0xFFu); }
};

template <int V, typename M>
__device__ __forceinline__ void load_v(const M *p, float (&x)[V]) {
    if constexpr (V == 8) {
        float lo[4], hi[4];
        MsgIO<M>::load4(p, lo);
        MsgIO<M>::load4(p + 4, hi);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            x[v] = lo[v];
            x[v + 4] = hi[v];
        }
    } else if constexpr (V == 4) {
        MsgIO<M>::load4(p, x);
    } else if constexpr (V == 2) {
        MsgIO<M>::load2(p, x);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = MsgIO<M>::load1(p + v);
    }
}

template <int V, typename M>
__device__ __forceinline__ void store_v(M *p, const float (&x)[V]) {
    if constexpr (V == 8) {
        float lo[4] = {x[0], x[1], x[2], x[3]}, hi[4] = {x[4], x[5], x[6], x[7]};
        MsgIO<M>::store4(p, lo);
        MsgIO<M>::store4(p + 4, hi);
    } else if constexpr (V == 4) {
        MsgIO<M>::store4(p, x);
    } else if constexpr (V == 2) {
        MsgIO<M>::store2(p, x);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) MsgIO<M>::store1(p + v, x[v]);
    }
}

// ---------------------------------------------------------------------------
// L2 residency. Between passes the posteriors (APP, 4n bytes per frame) are
// the data worth keeping in L2: the bit kernel writes them and the next
// check pass gathers them. Messages and channel LLRs stream through once per
// kernel. So APP traffic carries an evict-last policy and message / LLR
// reads an evict-first one (createpolicy + .L2::cache_hint).
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}

// B bytes from global memory (B-aligned) into dst, with an L2 policy.
template <int B>
__device__ __forceinline__ void ld_hint(void *dst, const void *src, uint64_t pol) {
    if constexpr (B == 32) {
        ld_hint<16>(dst, src, pol);
        ld_hint<16>(static_cast<char *>(dst) + 16, static_cast<const char *>(src) + 16, pol);
    } else if constexpr (B == 16) {
        uint4 v;
        asm volatile("ld.global.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;\n"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "l"(src), "l"(pol));
        *static_cast<uint4 *>(dst) = v;
    } else if constexpr (B == 8) {
        uint2 v;
        asm volatile("ld.global.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;\n" : "=r"(v.x), "=r"(v.y) : "l"(src), "l"(pol));
        *static_cast<uint2 *>(dst) = v;
    } else if constexpr (B == 4) {
        uint32_t v;
        asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;\n" : "=r"(v) : "l"(src), "l"(pol));
        *static_cast<uint32_t *>(dst) = v;
    } else if constexpr (B == 2) {
        unsigned short v;
        asm volatile("ld.global.L2::cache_hint.b16 %0, [%1], %2;\n" : "=h"(v) : "l"(src), "l"(pol));
        *static_cast<unsigned short *>(dst) = v;
    } else {
        static_assert(B == 1, "1, 2, 4, 8, 16 or 32 bytes");
        unsigned short v;
        asm volatile("ld.global.L2::cache_hint.b8 %0, [%1], %2;\n" : "=h"(v) : "l"(src), "l"(pol));
        *static_cast<unsigned char *>(dst) = (unsigned char)v;
    }
}

// V messages of type M (or floats) with an L2 policy.
template <int V, typename M>
__device__ __forceinline__ void load_v_hint(const M *p, float (&x)[V], uint64_t pol) {
    alignas(16) M raw[V];
    ld_hint<V * (int)sizeof(M)>(raw, p, pol);
    load_v<V, M>(raw, x);
}

// V floats to global memory with an L2 policy.
template <int V>
__device__ __forceinline__ void store_v_hint(float *p, const float (&x)[V], uint64_t pol) {
    if constexpr (V == 8) {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;\n" ::"l"(p), "f"(x[0]), "f"(x[1]),
                     "f"(x[2]), "f"(x[3]), "l"(pol)
                     : "memory");
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;\n" ::"l"(p + 4), "f"(x[4]), "f"(x[5]),
                     "f"(x[6]), "f"(x[7]), "l"(pol)
                     : "memory");
    } else if constexpr (V == 4) {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;\n" ::"l"(p), "f"(x[0]), "f"(x[1]),
                     "f"(x[2]), "f"(x[3]), "l"(pol)
                     : "memory");
    } else if constexpr (V == 2) {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;\n" ::"l"(p), "f"(x[0]), "f"(x[1]), "l"(pol)
                     : "memory");
    } else {
        static_assert(V == 1, "V is 1, 2, 4 or 8");
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;\n" ::"l"(p), "f"(x[0]), "l"(pol) : "memory");
    }
}

// ---------------------------------------------------------------------------
// phi on [phi(L_MAX), L_MAX]
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// phi(x) = ln((1 + t) / (1 - t)), t = e^-x, for 0 < x <= 80.
//  * t = 2^(-x log2 e): the product x log2(e) is split exactly by an FMA (and
//    the rounding of log2(e) itself is added back), so t keeps ~1e-7
//    relative accuracy even at x = 80.
//  * t < 1/16: phi = 2 atanh(t) = 2t (1 + t^2/3 + t^4/5 + t^6/7 + ...), the
//    series truncated after t^6/7 (relative error < 1e-10); this keeps full
//    relative precision for the tiny values that the sums of large-|q|
//    inputs are made of.
//  * otherwise phi = ln((1 + t) / (1 - t)), with 1 - t = 1 - e^-x from its
//    Taylor series below x = 1/4 (where 1 - t would cancel).
// phi^ serves the any-degree kernel, which carries one or two frames per
// lane with the same scalar operations, so its results do not depend on the
// frame layout either.
constexpr float kL2E = 1.44269502162933349609375f;  // log2(e) rounded to float
constexpr float kL2ELo = 1.925963033500011e-08f;    // log2(e) - kL2E
constexpr float kLn2 = 0.693147180559945309f;

__device__ __forceinline__ float phi_hat(float x, float l_max, float phi_lmax) {
    x = fminf(fmaxf(x, phi_lmax), l_max);
    float pn = x * -kL2E;
    float e = fmaf(x, kL2E, pn);
    e = fmaf(x, kL2ELo, e);
    float t = ex2_approx(pn);
    t = fmaf(t, e * -kLn2, t);
    float t2 = t * t;
    float poly = fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 7.0f, 1.0f / 5.0f), 1.0f / 3.0f), 1.0f);
    float res = (t + t) * poly;
    if (t >= 0.0625f) {
        float us = x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, -1.0f / 720.0f, 1.0f / 120.0f), -1.0f / 24.0f),
                                            1.0f / 6.0f),
                                    -0.5f),
                            1.0f);
        float u1 = fmaf(t, -1.0f, 1.0f);
        float u = x < 0.25f ? us : u1;
        float num = fmaf(u, -1.0f, 2.0f);
        float ratio = num * rcp_approx(u);
        res = lg2_approx(ratio) * kLn2;
    }
    return res;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Tabulated phi^: x clamped to [phi(L), L] (L <= 22, so x lies in
// [2^-32, 2^5)), then the chord a + b x of its bucket, the bucket being the
// top 15 bits of the float pattern of x.
__device__ __forceinline__ float phi_tab(float x, float l_max, float phi_lmax, const float2 *tab) {
    x = fminf(fmaxf(x, phi_lmax), l_max);
    const float2 ab = tab[(__float_as_uint(x) >> 17) - kPhiKey0];
    return fmaf(ab.y, x, ab.x);
}

// Error-free sum: s + err == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &err) {
    float s = a + b;
    float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
    return s;
}

// ---------------------------------------------------------------------------
// The check rule in product form. Algorithm 1 ("Values to Variable Nodes")
// computes r0 - r1 = prod_{j' != j} (1 - 2 q1_j'); in magnitudes this is
//   tanh(|r_ij| / 2) = prod_{j' != j} T_j',   T = tanh(x / 2),
// x = min(|q|, L) (the saturation: |q| > L acts as L), the same rule as
// phi(sum phi) above. With t = e^-x, T = (1 - t) / (1 + t), so for a set S of
// inputs
//   A(S) = prod (1 + t),  B(S) = prod (1 - t),  D(S) = A(S) - B(S),
//   prod_S T = B / A,     |r| = ln((1 + B/A) / (1 - B/A)) = ln((A + B) / D)
// for S the other inputs of an output. The kernels carry (A2, D) = (2A, D),
// which needs no division per input and nothing that cancels:
//   merging an input t:  D <- D + t (A2 - D)   (A2 - D = A + B),
//                        A2 <- A2 (1 + t);
//   an output joins the inputs before it (prefix p) and after it (suffix s):
//     K = 2 D(p u s) = D_p A2_s + D_s (A2_p - 2 D_p)   (A2_p - 2 D_p = 2 B_p),
//     (A + B) / D of p u s = A2_p A2_s / K - 1,
// sums and products of non-negative terms (A2_p - 2 D_p loses relative
// precision only where B_p << A_p, and then the term it scales is a few ulp
// of K). One exponential per input, a reciprocal and a logarithm per output.
// t = 2^(x * -log2(e)) with the product rounded once: its relative error is
// below 2e-6 at x = 20, an absolute error of ~2e-6 in the strong outputs it
// decides; the final "- 1" applies to a quotient >= 2, so weak outputs (A + B
// close to D) carry an absolute error of a few ulp of 1 (the smallest
// magnitudes come out as 0 or a rounding-sized value instead of phi(L)).
// Saturation of the output, |r| <= L: only an empty set of other inputs (a
// degree-1 check, K = 0) exceeds it; its quotient is clamped at e^L. Any
// other set gives |r| <= min x <= L, and for two or more other inputs a
// margin of ln 2 below L, so checks of a bin's full degree D >= 4 skip the
// clamp with the same results. Padding inputs (t = 0) are exact no-ops of
// the merge. Scalar and packed forms run the same operations in the same
// order, so every frame layout gives the same results.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float exp_neg(float x) { return ex2_approx(__fmul_rn(x, -kL2E)); }

__device__ __forceinline__ float2 exp_neg2(float2 x) {
    const float2 pn = mul2(x, f2(-kL2E));
    return make_float2(ex2_approx(pn.x), ex2_approx(pn.y));
}

// x = min(|q|, L) of two frames
__device__ __forceinline__ float2 sat_abs2(float2 q, float l_max) {
    return make_float2(fminf(fabsf(q.x), l_max), fminf(fabsf(q.y), l_max));
}

// The extrinsic input q = APP - r with a zero q given the sign of APP:
// fma(APP, 2^-60, q) equals q exactly whenever q != 0 (|q| > 2^-36 |APP|
// for any nonzero float difference, so the added term is below half an ulp
// of q), and is 2^-60 APP when q = 0. A zero input then flips with its
// posterior, as every other input does, so the outputs it has made (almost)
// zero keep the exact sign symmetry of the rule under a codeword flip of the
// inputs; their magnitudes are unchanged (t = e^-|q| rounds to 1 either way).
constexpr float kZeroSign = 0x1.0p-60f;

__device__ __forceinline__ float extrinsic(float app, float r) { return fmaf(app, kZeroSign, app - r); }

__device__ __forceinline__ float2 extrinsic2(float2 app, float2 r) {
    return fma2(app, f2(kZeroSign), fma2(r, f2(-1.0f), app));
}

// |mag| with the sign bit of `sign` (bit 31): one bit select. A weak output
// can round to a magnitude of -1e-7 (a quotient just below 1); taking its
// absolute value keeps the sign rule exact, and the rule symmetric under a
// codeword flip of the inputs.
__device__ __forceinline__ float with_sign(float mag, uint32_t sign) {
    return __uint_as_float((__float_as_uint(mag) & 0x7FFFFFFFu) | (sign & 0x80000000u));
}

__device__ __forceinline__ void pf_merge(float &a2, float &dl, float t) {
    const float s = fmaf(dl, -1.0f, a2);
    dl = fmaf(t, s, dl);
    a2 = fmaf(t, a2, a2);
}

__device__ __forceinline__ void pf_merge2(float2 &a2, float2 &dl, float2 t) {
    const float2 s = fma2(dl, f2(-1.0f), a2);
    dl = fma2(t, s, dl);
    a2 = fma2(t, a2, a2);
}

template <bool kClamp>
__device__ __forceinline__ float pf_log(float ratio, float r_max) {
    if constexpr (kClamp) ratio = fminf(ratio, r_max);
    return __fmul_rn(lg2_approx(ratio), kLn2);
}

template <bool kClamp>
__device__ __forceinline__ float2 pf_log2(float2 ratio, float r_max) {
    if constexpr (kClamp) {
        ratio.x = fminf(ratio.x, r_max);
        ratio.y = fminf(ratio.y, r_max);
    }
    return mul2(make_float2(lg2_approx(ratio.x), lg2_approx(ratio.y)), f2(kLn2));
}

// |r| for the union of a prefix (pa, pd) and a suffix (sa, sd)
template <bool kClamp>
__device__ __forceinline__ float pf_out(float pa, float pd, float sa, float sd, float r_max) {
    const float k2 = fmaf(pd, sa, __fmul_rn(sd, fmaf(pd, -2.0f, pa)));
    return pf_log<kClamp>(fmaf(__fmul_rn(pa, sa), rcp_approx(k2), -1.0f), r_max);
}

template <bool kClamp>
__device__ __forceinline__ float2 pf_out2(float2 pa, float2 pd, float2 sa, float2 sd, float r_max) {
    const float2 k2 = fma2(pd, sa, mul2(sd, fma2(pd, f2(-2.0f), pa)));
    const float2 rk = make_float2(rcp_approx(k2.x), rcp_approx(k2.y));
    return pf_log2<kClamp>(fma2(mul2(pa, sa), rk, f2(-1.0f)), r_max);
}

// The same where one side is empty, (A2, D) = (2, 0): K = 2 d and the product
// 2 a of the other side, exactly the values pf_out2 forms from (2, 0).
template <bool kClamp>
__device__ __forceinline__ float2 pf_out_one2(float2 a2, float2 dl, float r_max) {
    const float2 k2 = add2(dl, dl);
    const float2 rk = make_float2(rcp_approx(k2.x), rcp_approx(k2.y));
    return pf_log2<kClamp>(fma2(add2(a2, a2), rk, f2(-1.0f)), r_max);
}

// ---------------------------------------------------------------------------
// Per-frame flag bits: frame f is bit (f & 31) of word f >> 5.
// ---------------------------------------------------------------------------

// The syndrome flag row of the decision after pass p: row p of the call, or
// one of two alternating rows in continuous decoding.
__device__ __forceinline__ uint32_t *unsat_row(const PassArgs &a, int p) {
    return a.unsat + (size_t)(a.unsat_ring ? (p & 1) : p) * (a.Fp / 32);
}



// OR the per-lane frame bits (frames f0 .. f0 + V - 1 of every lane) into the
// flag row `row` with one atomic per 32 frames.
template <int V>
__device__ __forceinline__ void or_frame_bits(uint32_t *row, int g, int lane, const bool (&bits)[V]) {
    if constexpr (V == 1) {
        uint32_t w = __ballot_sync(kFull, bits[0]);
        if (lane == 0 && w) atomicOr(row + g, w);
    } else if constexpr (V == 2) {
        uint32_t pair = (bits[0] ? 1u : 0u) | (bits[1] ? 2u : 0u);
        uint32_t w = pair << ((lane & 15) * 2);
        w |= __shfl_xor_sync(kFull, w, 1);
        w |= __shfl_xor_sync(kFull, w, 2);
        w |= __shfl_xor_sync(kFull, w, 4);
        w |= __shfl_xor_sync(kFull, w, 8);
        if ((lane & 15) == 0 && w) atomicOr(row + g * 2 + (lane >> 4), w);
    } else if constexpr (V == 8) {
        uint32_t byte = 0;
#pragma unroll
        for (int v = 0; v < 8; ++v) byte |= (bits[v] ? 1u : 0u) << v;
        uint32_t w = byte << ((lane & 3) * 8);
        w |= __shfl_xor_sync(kFull, w, 1);
        w |= __shfl_xor_sync(kFull, w, 2);
        if ((lane & 3) == 0 && w) atomicOr(row + g * 8 + (lane >> 2), w);
    } else {
        static_assert(V == 4, "V is 1, 2, 4 or 8");
        uint32_t nib = 0;
#pragma unroll
        for (int v = 0; v < 4; ++v) nib |= (bits[v] ? 1u : 0u) << v;
        uint32_t w = nib << ((lane & 7) * 4);
        w |= __shfl_xor_sync(kFull, w, 1);
        w |= __shfl_xor_sync(kFull, w, 2);
        w |= __shfl_xor_sync(kFull, w, 4);
        if ((lane & 7) == 0 && w) atomicOr(row + g * 4 + (lane >> 3), w);
    }
}

// Store the per-lane frame bits as the words of a decision row (plain store:
// the warp owns these words).
template <int V>
__device__ __forceinline__ void store_frame_bits(uint32_t *row, int g, int lane, const bool (&bits)[V]) {
    uint32_t mine = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) mine |= (bits[v] ? 1u : 0u) << v;
    constexpr int kLanesPerWord = 32 / V;
    uint32_t w = mine << ((lane % kLanesPerWord) * V);
#pragma unroll
    for (int o = 1; o < kLanesPerWord; o <<= 1) w |= __shfl_xor_sync(kFull, w, o);
    if (lane % kLanesPerWord == 0) row[g * V + lane / kLanesPerWord] = w;
}

// ---------------------------------------------------------------------------
// Check-node kernels
// ---------------------------------------------------------------------------

// The check-node rule for one check of degree d <= D on V frames per lane,
// in product/complement form. load(k, av, rv) fetches input k: av = APP_j
// (or lambda_j on the first pass), rv = the previous message r_ij (unused on
// the first pass). Writes the d new messages to rows out + k * Fp and ors the
// check's syndrome of the previous hard decision into unsat.
// The min-sum family for one check of degree d <= D (a derived algorithm the
// paper names, not its exact rule): |r_k| = clamp(alpha m_k - beta, 0, L_MAX)
// with m_k the smallest |q| of the other inputs (L_MAX when there is none),
// found from the two smallest magnitudes and the position of the smallest;
// same sign rule as sum-product. The degree-adaptive variant takes alpha and
// beta from the table entry of the check's degree d.
template <int D, int V, typename M, typename Load>
__device__ __forceinline__ void min_sum_node(int d, bool first, bool syn, Load &&load, M *out, size_t Fp,
                                             const PassArgs &a, bool (&unsat)[V]) {
    float alpha = a.ms_alpha, beta = a.ms_beta;
    if (a.ms_table) {
        const float2 t = __ldg(a.ms_table + d);
        alpha = t.x;
        beta = t.y;
    }
    float m1[V], m2[V];
    int idx[V];
    uint32_t ones[V], z[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        m1[v] = m2[v] = a.l_max;
        idx[v] = -1;
        ones[v] = z[v] = 0u;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (k < d) {
            float av[V], rv[V];
            load(k, av, rv);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (syn) z[v] ^= av[v] > 0.0f ? 1u : 0u;
                const float q = first ? av[v] : av[v] - rv[v];
                ones[v] |= (q > 0.0f ? 1u : 0u) << k;
                const float x = fminf(fabsf(q), a.l_max);
                if (x < m1[v]) {
                    m2[v] = m1[v];
                    m1[v] = x;
                    idx[v] = k;
                } else if (x < m2[v]) {
                    m2[v] = x;
                }
            }
        }
    }
    uint32_t neg[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        unsat[v] |= z[v] != 0u;
        neg[v] = (__popc(ones[v]) & 1u) ? ones[v] : ~ones[v];
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (k < d) {
            float o[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float m = idx[v] == k ? m2[v] : m1[v];
                const float mag = fminf(fmaxf(fmaf(alpha, m, -beta), 0.0f), a.l_max);
                o[v] = __int_as_float(__float_as_int(mag) | (int)((neg[v] << (31 - k)) & 0x80000000u));
            }
            store_v<V, M>(out + (size_t)k * Fp, o);
        }
    }
}

template <int D, int V, typename M, int RULE, typename Load>
__device__ __forceinline__ void check_node(int d, bool first, bool syn, Load &&load, M *out, size_t Fp,
                                           const PassArgs &a, bool (&unsat)[V]) {
    if constexpr (RULE == 1) {
        min_sum_node<D, V, M>(d, first, syn, load, out, Fp, a, unsat);
    } else {
        float tt[D][V];    // t_k = e^-min(|q_k|, L); 0 (a no-op) for slots k >= d
        uint32_t ones[V];  // bit k: input k says "bit 1" (q > 0)
        uint32_t z[V];
#pragma unroll
        for (int v = 0; v < V; ++v) ones[v] = z[v] = 0u;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                float av[V], rv[V];
                load(k, av, rv);
                if (syn) {
#pragma unroll
                    for (int v = 0; v < V; ++v) z[v] ^= av[v] > 0.0f ? 1u : 0u;
                }
                if (!first) {
#pragma unroll
                    for (int v = 0; v < V; ++v) av[v] = extrinsic(av[v], rv[v]);
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    ones[v] |= (av[v] > 0.0f ? 1u : 0u) << k;
                    tt[k][v] = exp_neg(fminf(fabsf(av[v]), a.l_max));
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) tt[k][v] = 0.0f;
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) unsat[v] |= z[v] != 0u;
        // (A2, D) of the inputs after k, then a running prefix
        float sa[D][V], sd[D][V];
        {
            float ca[V], cd[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                ca[v] = 2.0f;
                cd[v] = 0.0f;
            }
#pragma unroll
            for (int k = D - 1; k >= 0; --k) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    sa[k][v] = ca[v];
                    sd[k][v] = cd[v];
                    if (k > 0) pf_merge(ca[v], cd[v], tt[k][v]);
                }
            }
        }
        // output k is negative (bit-0 message) iff the other inputs hold an even
        // number of ones, i.e. iff input k's bit equals the total parity
        float pa[V], pd[V];
        uint32_t neg[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pa[v] = 2.0f;
            pd[v] = 0.0f;
            neg[v] = (__popc(ones[v]) & 1u) ? ones[v] : ~ones[v];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                float o[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    o[v] = pf_out<true>(pa[v], pd[v], sa[k][v], sd[k][v], a.r_max);
                    o[v] = with_sign(o[v], neg[v] << (31 - k));
                    pf_merge(pa[v], pd[v], tt[k][v]);
                }
                store_v<V, M>(out + (size_t)k * Fp, o);
            }
        }
    }
}

// The same rule with frames kept in packed pairs (V = 2P frames per lane):
// every value lives in a float2 register pair, so the packed FP32
// instructions need no repacking. Same operations, same order, same results
// as check_node.
template <typename M, int P>
__device__ __forceinline__ void store_pairs(M *p, const float2 (&o)[P]) {
    float x[2 * P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        x[2 * q] = o[q].x;
        x[2 * q + 1] = o[q].y;
    }
    store_v<2 * P, M>(p, x);
}

template <int D, int P, typename M, int RULE, typename Load>
__device__ __forceinline__ void check_node_pairs(int d, bool first, bool syn, Load &&load, M *out, size_t Fp,
                                                 const PassArgs &a, bool (&unsat)[2 * P]) {
    if constexpr (RULE == 1) {
        auto load_flat = [&](int k, float (&av)[2 * P], float (&rv)[2 * P]) {
            float2 a2[P], r2[P];
            load(k, a2, r2);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                av[2 * q] = a2[q].x;
                av[2 * q + 1] = a2[q].y;
                rv[2 * q] = first ? 0.0f : r2[q].x;
                rv[2 * q + 1] = first ? 0.0f : r2[q].y;
            }
        };
        min_sum_node<D, 2 * P, M>(d, first, syn, load_flat, out, Fp, a, unsat);
    } else {
        float2 tt[D][P];       // t_k, two frames per entry; 0 for slots k >= d
        uint32_t ones[2 * P];  // bit k: input k says "bit 1" (q > 0)
        uint32_t z[2 * P];
#pragma unroll
        for (int v = 0; v < 2 * P; ++v) ones[v] = z[v] = 0u;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                float2 av[P], rv[P];
                load(k, av, rv);
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    if (syn) {
                        z[2 * q] ^= av[q].x > 0.0f ? 1u : 0u;
                        z[2 * q + 1] ^= av[q].y > 0.0f ? 1u : 0u;
                    }
                    if (!first) av[q] = extrinsic2(av[q], rv[q]);
                    ones[2 * q] |= (av[q].x > 0.0f ? 1u : 0u) << k;
                    ones[2 * q + 1] |= (av[q].y > 0.0f ? 1u : 0u) << k;
                    tt[k][q] = exp_neg2(sat_abs2(av[q], a.l_max));
                }
            } else {
#pragma unroll
                for (int q = 0; q < P; ++q) tt[k][q] = f2(0.0f);
            }
        }
#pragma unroll
        for (int v = 0; v < 2 * P; ++v) unsat[v] |= z[v] != 0u;
        float2 sa[D][P], sd[D][P];
        {
            float2 ca[P], cd[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                ca[q] = f2(2.0f);
                cd[q] = f2(0.0f);
            }
#pragma unroll
            for (int k = D - 1; k >= 0; --k) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    sa[k][q] = ca[q];
                    sd[k][q] = cd[q];
                    if (k > 0) pf_merge2(ca[q], cd[q], tt[k][q]);
                }
            }
        }
        float2 pa[P], pd[P];
        uint32_t neg[2 * P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            pa[q] = f2(2.0f);
            pd[q] = f2(0.0f);
        }
#pragma unroll
        for (int v = 0; v < 2 * P; ++v) neg[v] = (__popc(ones[v]) & 1u) ? ones[v] : ~ones[v];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                float2 o[P];
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    o[q] = pf_out2<true>(pa[q], pd[q], sa[k][q], sd[k][q], a.r_max);
                    o[q].x = with_sign(o[q].x, neg[2 * q] << (31 - k));
                    o[q].y = with_sign(o[q].y, neg[2 * q + 1] << (31 - k));
                    pf_merge2(pa[q], pd[q], tt[k][q]);
                }
                store_pairs<M, P>(out + (size_t)k * Fp, o);
            }
        }
    }
}

// The sum-product rule for checks whose D input rows are all readable
// (the shared-memory ring of the pipelined kernel): every one of the D slots
// is computed without a branch and the d <= D real inputs are selected by
// predicates, so a bin whose checks mostly have degree D pays no control
// flow per edge. Slots k >= d become neutral inputs (D_k = 0, no sign, no
// syndrome term) and their outputs are not stored. Same operations, same
// order, same results as check_node_pairs for the real inputs.
template <int D, int P, typename M, bool kFirst, bool kSyn, bool kFull, typename Load>
__device__ __forceinline__ void check_node_pairs_masked(int d, Load &&load, M *out, size_t Fp, const PassArgs &a,
                                                        bool (&unsat)[2 * P]) {
    const float l_max = a.l_max, r_max = a.r_max;
    float2 tt[D][P];
    // sign bits of the inputs, input k at bit D - 1 - k (shifted in by one
    // funnel shift per input; padding slots shift in 0)
    uint32_t sb[2 * P];
    uint32_t z[2 * P];
#pragma unroll
    for (int v = 0; v < 2 * P; ++v) sb[v] = z[v] = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const bool real = kFull || k < d;  // kFull: the caller knows d == D
        float2 av[P], rv[P];
        load(k, av, rv);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            if constexpr (kSyn) {
                z[2 * q] ^= (real && av[q].x > 0.0f) ? 1u : 0u;
                z[2 * q + 1] ^= (real && av[q].y > 0.0f) ? 1u : 0u;
            }
            if constexpr (!kFirst) av[q] = extrinsic2(av[q], rv[q]);
            const uint32_t bx = real ? __float_as_uint(av[q].x) : 0u, by = real ? __float_as_uint(av[q].y) : 0u;
            sb[2 * q] = __funnelshift_l(bx, sb[2 * q], 1);
            sb[2 * q + 1] = __funnelshift_l(by, sb[2 * q + 1], 1);
            const float2 t = exp_neg2(sat_abs2(av[q], l_max));
            tt[k][q] = make_float2(real ? t.x : 0.0f, real ? t.y : 0.0f);
        }
    }
#pragma unroll
    for (int v = 0; v < 2 * P; ++v) unsat[v] |= z[v] != 0u;
    // (A2, D) of the inputs after k (the last one's is empty: (2, 0))
    float2 sa[D][P], sd[D][P];
    {
        float2 ca[P], cd[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            ca[q] = f2(2.0f);
            cd[q] = f2(0.0f);
        }
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
#pragma unroll
            for (int q = 0; q < P; ++q) {
                sa[k][q] = ca[q];
                sd[k][q] = cd[q];
                if (k > 0) pf_merge2(ca[q], cd[q], tt[k][q]);
            }
        }
    }
    float2 pa[P], pd[P];
    uint32_t neg[2 * P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        pa[q] = f2(2.0f);
        pd[q] = f2(0.0f);
    }
    // r_k > 0 iff an odd number of the other real inputs are > 0. With s_j
    // the sign bit of q_j, that count is (d - 1) - sum_{j != k} s_j, so r_k
    // is negative iff d + S + s_k is odd (S = sum of all s_j): bit D - 1 - k
    // of neg. A zero input counts as positive here, which only changes the
    // sign of outputs whose magnitude that input has already made zero.
    const uint32_t dpar = (uint32_t)(kFull ? D : d) & 1u;
#pragma unroll
    for (int v = 0; v < 2 * P; ++v) neg[v] = ((dpar ^ __popc(sb[v])) & 1u) ? ~sb[v] : sb[v];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float2 o[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            // checks of the bin's full degree D >= 4 never need the clamp
            if (k == 0)
                o[q] = pf_out_one2<!kFull>(sa[0][q], sd[0][q], r_max);
            else if (k == D - 1)
                o[q] = pf_out_one2<!kFull>(pa[q], pd[q], r_max);
            else
                o[q] = pf_out2<!kFull>(pa[q], pd[q], sa[k][q], sd[k][q], r_max);
            o[q].x = with_sign(o[q].x, neg[2 * q] << (32 - D + k));
            o[q].y = with_sign(o[q].y, neg[2 * q + 1] << (32 - D + k));
            if (k + 1 < D) pf_merge2(pa[q], pd[q], tt[k][q]);
        }
        if constexpr (kFull && std::is_same_v<M, int8_t> && P == 2) {
            // |r| <= L <= 20 here (the caller takes this path for int8 only
            // then), so the levels need no clamp
            const float x[4] = {o[0].x, o[0].y, o[1].x, o[1].y};
            MsgIO<int8_t>::store4_unclamped(out + (size_t)k * Fp, x);
        } else if (kFull || k < d) {
            store_pairs<M, P>(out + (size_t)k * Fp, o);
        }
    }
}

template <int V, typename M>
__device__ __forceinline__ void load_pairs(const M *p, float2 (&x)[V / 2]) {
    float t[V];
    load_v<V, M>(p, t);
#pragma unroll
    for (int q = 0; q < V / 2; ++q) x[q] = make_float2(t[2 * q], t[2 * q + 1]);
}

// Checks of degree <= D, inputs read straight from global memory.
template <int D, int V, typename M, int RULE>
__global__ void __launch_bounds__(kThreads) k_check_reg(PassArgs a, const int32_t *__restrict__ checks,
                                                        int32_t count) {
    pdl_wait();
    if (gated_off(a)) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = a.f_begin / (32 * V) + (int)blockIdx.y;
    const int f0 = g * 32 * V + lane * V;
    const size_t Fp = (size_t)a.Fp;
    M *r = reinterpret_cast<M *>(a.r);
    const bool first = a.pass == 0;
    const bool syn = a.syndrome != 0;
    const float *qsrc = first ? a.lamT : a.app;

    bool live[V];
    bool any_live = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        live[v] = !frame_bit(a.done, f0 + v);
        any_live |= live[v];
    }
    if (!__any_sync(kFull, any_live)) return;

    bool unsat[V];
#pragma unroll
    for (int v = 0; v < V; ++v) unsat[v] = false;

    for (int w = blockIdx.x * (kThreads / 32) + warp; w < count; w += gridDim.x * (kThreads / 32)) {
        const int i = checks[w];
        const int b = a.row_ptr[i];
        const int d = a.row_ptr[i + 1] - b;  // warp-uniform, 1 <= d <= D
        if constexpr (V % 2 == 0) {
            auto load = [&](int k, float2 (&av)[V / 2], float2 (&rv)[V / 2]) {
                const int slot = b + k;
                load_pairs<V, float>(qsrc + (size_t)a.col_idx[slot] * Fp + f0, av);
                if (!first) load_pairs<V, M>(r + (size_t)slot * Fp + f0, rv);
            };
            check_node_pairs<D, V / 2, M, RULE>(d, first, syn, load, r + (size_t)b * Fp + f0, Fp, a, unsat);
        } else {
            auto load = [&](int k, float (&av)[V], float (&rv)[V]) {
                const int slot = b + k;
                load_v<V, float>(qsrc + (size_t)a.col_idx[slot] * Fp + f0, av);
                if (!first) load_v<V, M>(r + (size_t)slot * Fp + f0, rv);
            };
            check_node<D, V, M, RULE>(d, first, syn, load, r + (size_t)b * Fp + f0, Fp, a, unsat);
        }
    }
    if (a.syndrome) {
        bool bits[V];
#pragma unroll
        for (int v = 0; v < V; ++v) bits[v] = unsat[v] && live[v];
        or_frame_bits<V>(unsat_row(a, a.pass - 1), g, lane, bits);
    }
}

// ---------------------------------------------------------------------------
// Pipelined check kernel: every warp keeps the APP and message rows of its
// next S - 1 checks in flight into its own shared-memory ring while it
// computes the current one. The rows arrive by bulk copies (cp.async.bulk,
// the copy engine): lane k issues one copy for the APP row of input k and one
// for its message row, completing on the stage's mbarrier, so a check costs
// the warp two copy instructions per input instead of one 16-byte copy per
// lane and chunk. Check descriptors (first slot, degree) and column indices
// are fetched one and two checks ahead of their copies. Waits on an mbarrier
// give up after kSpinLimit polls: the warp then flags the call (status word)
// and stops.
// ---------------------------------------------------------------------------

template <int D, int V, typename M>
struct PipeShape {
    static constexpr int kRowA = 32 * V * 4;                  // bytes of one APP row segment
    static constexpr int kRowR = 32 * V * (int)sizeof(M);     // bytes of one message row segment
    static constexpr int kOffR = D * kRowA;                   // message rows after the APP rows
    static constexpr int kStage = kOffR + D * kRowR;          // bytes of one check's rows
    static_assert(kRowA % 128 == 0 && kStage % 128 == 0, "copy destinations stay 128-byte aligned");
};

constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of a barrier; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// One box {32 V frames, h rows} of a 2-D tensor map at (frame x, row y).
__device__ __forceinline__ void tma_tile_2d(uint32_t dst, const CUtensorMap *tm, int x, int y, uint32_t bar,
                                            uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar), "l"(pol)
        : "memory");
}
// Four one-row boxes at (frame x, rows y0..y3), landing as four consecutive rows.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap *tm, int x, int y0, int y1, int y2, int y3,
                                            uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(bar), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

template <int D, int V, typename M, int S>
struct BulkShape {
    static constexpr int kBarBytes = ((kThreads / 32) * S * 8 + 127) / 128 * 128;  // mbarriers, then the rings
    static constexpr int kSmem = kBarBytes + (kThreads / 32) * S * PipeShape<D, V, M>::kStage;
};

// CTAs per SM the register budget is set for. Three for int8 messages and
// checks of degree <= 8, whose ring is small enough for that (85 registers a
// thread; for 16-bit messages the same bound measured no faster, and wider
// checks would spill under it). Two for the syndrome form of the other
// narrow bins, which would otherwise take 136 registers and run one CTA of
// 8 warps per SM.
template <int D, typename M, int MODE>
constexpr int bulk_min_ctas() {
    return D > 8 ? 1 : (sizeof(M) == 1 ? 3 : (MODE == 2 ? 2 : 1));
}

template <int D, int V, typename M, int S, int MODE, int RULE>
__global__ void __launch_bounds__(kThreads, bulk_min_ctas<D, M, MODE>()) k_check_bulk(const __grid_constant__ PassArgs a,
                                                         const int2 *__restrict__ desc, int32_t count) {
    pdl_wait();
    if (gated_off(a)) return;
    using P = PipeShape<D, V, M>;
    using B = BulkShape<D, V, M, S>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *ring = smem + B::kBarBytes + (size_t)warp * S * P::kStage;
    const uint32_t bar0 = smem_u32(smem) + (uint32_t)(warp * S * 8);
    const int g = a.f_begin / (32 * V) + (int)blockIdx.y;
    const int fbase = g * 32 * V;
    const int f0 = fbase + lane * V;
    const size_t Fp = (size_t)a.Fp;
    M *r = reinterpret_cast<M *>(a.r);
    constexpr bool first = MODE == 0;
    constexpr bool syn = MODE == 2;

    bool live[V];
    bool any_live = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        live[v] = !frame_bit(a.done, f0 + v);
        any_live |= live[v];
    }
    if (!__any_sync(kFull, any_live)) return;
    bool unsat[V];
#pragma unroll
    for (int v = 0; v < V; ++v) unsat[v] = false;

    if (lane < S) mbar_init(bar0 + 8 * lane, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncwarp();

    const int stride = gridDim.x * (kThreads / 32);
    const int w0 = blockIdx.x * (kThreads / 32) + warp;
    const uint64_t pol_keep = policy_evict_last(), pol_stream = policy_evict_first();
    // int8 messages of a rule saturating above 20 keep the clamped stores
    const bool full_ok = !std::is_same_v<M, int8_t> || a.l_max <= 20.0f;

    // Copy the rows of one check (first slot b, degree d, lane k holding the
    // column of input k) into stage st: lane 0 issues one tensor copy of the
    // check's d message rows (a box of D rows from slot b; rows past the
    // check are read but never used), a four-row gather per four APP rows and
    // a one-row copy for each of the last d mod 4.
    auto issue = [&](int st, int b, int d, int jl) {
        if (d <= 0) return;
        // every lane's reads of this stage come before the copies that refill it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        const uint32_t bar = bar0 + 8 * st;
        const uint32_t base = smem_u32(ring + st * P::kStage);
        const int d4 = d & ~3;
        int cj[D];
#pragma unroll
        for (int k = 0; k < D; ++k) cj[k] = __shfl_sync(kFull, jl, k);
        if (lane == 0) {
            mbar_arrive_expect_tx(bar, (uint32_t)(d * P::kRowA) + (first ? 0u : (uint32_t)(D * P::kRowR)));
            if (d == D) {  // most checks of a bin: straight-line copies
#pragma unroll
                for (int k = 0; k + 3 < D; k += 4)
                    tma_gather4(base + k * P::kRowA, &a.tm_q, fbase, cj[k], cj[k + 1], cj[k + 2], cj[k + 3], bar,
                                pol_keep);
#pragma unroll
                for (int k = D & ~3; k < D; ++k) tma_tile_2d(base + k * P::kRowA, &a.tm_q, fbase, cj[k], bar, pol_keep);
            } else {
#pragma unroll
                for (int k = 0; k + 3 < D; k += 4)
                    if (k < d4)
                        tma_gather4(base + k * P::kRowA, &a.tm_q, fbase, cj[k], cj[k + 1], cj[k + 2], cj[k + 3], bar,
                                    pol_keep);
#pragma unroll
                for (int k = 0; k < D; ++k)
                    if (k >= d4 && k < d) tma_tile_2d(base + k * P::kRowA, &a.tm_q, fbase, cj[k], bar, pol_keep);
            }
            if (!first) tma_tile_2d(base + P::kOffR, &a.tm_r, fbase, b, bar, pol_stream);
        }
    };
    auto get_desc = [&](int w) { return w < count ? desc[w] : make_int2(0, 0); };
    auto get_col = [&](int2 dd) { return lane < dd.y ? a.col_idx[dd.x + lane] : 0; };

    int qb[S], qd[S];
    int2 nd = get_desc(w0);
    int njl = get_col(nd);
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        issue(s, nd.x, nd.y, njl);
        qb[s] = nd.x;
        qd[s] = nd.y;
        nd = get_desc(w0 + (s + 1) * stride);
        njl = get_col(nd);
    }
    int2 nd2 = get_desc(w0 + S * stride);
    int n = 0;
    bool timed_out = false;
    for (int w = w0; w < count; w += stride, ++n) {
        issue((n + S - 1) % S, nd.x, nd.y, njl);
        qb[S - 1] = nd.x;
        qd[S - 1] = nd.y;
        nd = nd2;
        njl = get_col(nd);
        nd2 = get_desc(w + (S + 1) * stride);
        const int st = n % S;
        // every lane waits (the wait makes the copied rows visible to it);
        // the warp gives up together if any lane did
        bool landed = __all_sync(kFull, mbar_wait(bar0 + 8 * st, (uint32_t)((n / S) & 1)));
        // test hook: warp 0 of the chosen CTA takes the give-up path with its
        // first check's rows already landed (no wait runs out, nothing faults)
        if (a.giveup_cta >= 0 && n == 0 && warp == 0 && (int)(blockIdx.y * gridDim.x + blockIdx.x) == a.giveup_cta)
            landed = false;
        if (!landed) {
            timed_out = true;
            break;
        }
        const unsigned char *base = ring + st * P::kStage;
        static_assert(V % 2 == 0, "the pipelined kernel runs frame pairs");
        auto load = [&](int k, float2 (&av)[V / 2], float2 (&rv)[V / 2]) {
            const float2 *pa = reinterpret_cast<const float2 *>(base + k * P::kRowA) + lane * (V / 2);
#pragma unroll
            for (int q = 0; q < V / 2; ++q) av[q] = pa[q];
            if (!first)
                load_pairs<V, M>(reinterpret_cast<const M *>(base + P::kOffR + k * P::kRowR) + lane * V, rv);
        };
        if constexpr (RULE == 0) {
            // checks of the bin's full degree (most of them) skip the masking;
            // the widest bin keeps one path (registers)
            if (D <= 8 && qd[0] == D && full_ok)
                check_node_pairs_masked<D, V / 2, M, first, syn, true>(D, load, r + (size_t)qb[0] * Fp + f0, Fp, a,
                                                                      unsat);
            else
                check_node_pairs_masked<D, V / 2, M, first, syn, false>(qd[0], load, r + (size_t)qb[0] * Fp + f0, Fp,
                                                                       a, unsat);
        } else
            check_node_pairs<D, V / 2, M, RULE>(qd[0], first, syn, load, r + (size_t)qb[0] * Fp + f0, Fp, a, unsat);
        __syncwarp();
#pragma unroll
        for (int s = 0; s < S - 1; ++s) {
            qb[s] = qb[s + 1];
            qd[s] = qd[s + 1];
        }
    }
    if (timed_out) {
        // flag the call, then give the copies still in flight a bounded time
        // to land before the warp leaves
        if (lane == 0) atomicOr(a.status, 1u);
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (qd[s] > 0) mbar_wait(bar0 + 8 * ((n + s) % S), (uint32_t)(((n + s) / S) & 1));
        return;
    }
    if (a.syndrome) {
        bool bits[V];
#pragma unroll
        for (int v = 0; v < V; ++v) bits[v] = unsat[v] && live[v];
        or_frame_bits<V>(unsat_row(a, a.pass - 1), g, lane, bits);
    }
}

// Checks of degree 17-32 in codes with many of them (high-rate codes): the
// product form of the register kernels, with each input's t and each suffix
// state (A2, D) staged per warp in shared memory instead of registers, so
// that the per-frame state does not grow with the degree. One pass over the
// inputs (APP gathered, messages read once), a suffix sweep and an output
// sweep over shared memory. The same operations in the same order as
// check_node_pairs, one or two frames per lane (V = 1 or 2), so the results
// do not depend on the frame layout.
template <int V, typename M>
struct ProdShape {
    static constexpr int kPairs = V == 1 ? 1 : V / 2;  // float (V = 1) or float2 entries per lane
    static constexpr int kEntry = V == 1 ? 4 : 8;
    // bytes per warp for `ds` staged inputs: t, A2 and D of every input
    static __host__ __device__ constexpr size_t warp_bytes(int ds) { return (size_t)3 * ds * 32 * kEntry; }
};

template <int V, typename M>
__global__ void __launch_bounds__(kThreads) k_check_prod(PassArgs a, const int32_t *__restrict__ checks,
                                                         int32_t count) {
    static_assert(V == 1 || V == 2, "one or two frames per lane");
    pdl_wait();
    if (gated_off(a)) return;
    extern __shared__ __align__(128) unsigned char smem[];
    using T = typename std::conditional<V == 1, float, float2>::type;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int ds = a.bin_degree;
    T *tt = reinterpret_cast<T *>(smem + (size_t)warp * ProdShape<V, M>::warp_bytes(ds));
    T *sa = tt + (size_t)ds * 32;
    T *sd = sa + (size_t)ds * 32;
    const int g = a.f_begin / (32 * V) + (int)blockIdx.y;
    const int f0 = g * 32 * V + lane * V;
    const size_t Fp = (size_t)a.Fp;
    M *r = reinterpret_cast<M *>(a.r);
    const bool first = a.pass == 0;
    const bool syn = a.syndrome != 0;
    const float *qsrc = first ? a.lamT : a.app;
    const float l_max = a.l_max, r_max = a.r_max;

    bool live[V];
    bool any_live = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        live[v] = !frame_bit(a.done, f0 + v);
        any_live |= live[v];
    }
    if (!__any_sync(kFull, any_live)) return;
    bool unsat[V];
#pragma unroll
    for (int v = 0; v < V; ++v) unsat[v] = false;
    const uint64_t pol_keep = policy_evict_last(), pol_stream = policy_evict_first();

    auto two = [](float x) {
        if constexpr (V == 1) return x;
        else return f2(x);
    };
    for (int w = blockIdx.x * (kThreads / 32) + warp; w < count; w += gridDim.x * (kThreads / 32)) {
        const int i = checks[w];
        const int b = a.row_ptr[i];
        const int d = a.row_ptr[i + 1] - b;  // 17 <= d <= ds
        uint32_t sb[V], z[V];
#pragma unroll
        for (int v = 0; v < V; ++v) sb[v] = z[v] = 0u;
        // the check's column indices in one warp load (d <= 32), then each
        // input's row loads need no dependent index load
        const int jl = lane < d ? a.col_idx[b + lane] : 0;
        // inputs: t and sign bits (input k at bit d - 1 - k)
#pragma unroll 4
        for (int k = 0; k < d; ++k) {
            float av[V], rv[V];
            load_v_hint<V, float>(qsrc + (size_t)__shfl_sync(kFull, jl, k) * Fp + f0, av, pol_keep);
            if (!first) load_v_hint<V, M>(r + (size_t)(b + k) * Fp + f0, rv, pol_stream);
            float x[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (syn) z[v] ^= av[v] > 0.0f ? 1u : 0u;
                if (!first) av[v] = extrinsic(av[v], rv[v]);
                sb[v] = __funnelshift_l(__float_as_uint(av[v]), sb[v], 1);
                x[v] = fminf(fabsf(av[v]), l_max);
            }
            if constexpr (V == 1) {
                tt[k * 32 + lane] = exp_neg(x[0]);
            } else {
                tt[k * 32 + lane] = exp_neg2(make_float2(x[0], x[1]));
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) unsat[v] |= z[v] != 0u;
        // suffix states: (A2, D) of the inputs after k
        {
            T ca = two(2.0f), cd = two(0.0f);
            for (int k = d - 1; k >= 0; --k) {
                sa[k * 32 + lane] = ca;
                sd[k * 32 + lane] = cd;
                if (k > 0) {
                    if constexpr (V == 1) pf_merge(ca, cd, tt[k * 32 + lane]);
                    else pf_merge2(ca, cd, tt[k * 32 + lane]);
                }
            }
        }
        // outputs with a running prefix
        uint32_t neg[V];
#pragma unroll
        for (int v = 0; v < V; ++v) neg[v] = (((uint32_t)d ^ __popc(sb[v])) & 1u) ? ~sb[v] : sb[v];
        T pa = two(2.0f), pd = two(0.0f);
        M *out = r + (size_t)b * Fp + f0;
        for (int k = 0; k < d; ++k) {
            const T t = tt[k * 32 + lane];
            float o[V];
            if constexpr (V == 1) {
                o[0] = with_sign(pf_out<true>(pa, pd, sa[k * 32 + lane], sd[k * 32 + lane], r_max),
                                 neg[0] << (32 - d + k));
                pf_merge(pa, pd, t);
            } else {
                const float2 y = pf_out2<true>(pa, pd, sa[k * 32 + lane], sd[k * 32 + lane], r_max);
                o[0] = with_sign(y.x, neg[0] << (32 - d + k));
                o[1] = with_sign(y.y, neg[1] << (32 - d + k));
                pf_merge2(pa, pd, t);
            }
            store_v<V, M>(out + (size_t)k * Fp, o);
        }
    }
    if (a.syndrome) {
        bool bits[V];
#pragma unroll
        for (int v = 0; v < V; ++v) bits[v] = unsat[v] && live[v];
        or_frame_bits<V>(unsat_row(a, a.pass - 1), g, lane, bits);
    }
}

// Checks of any degree: two sweeps over the check's edges. The first forms
// the total of phi^(|q|) as an unevaluated float pair (hi + lo) with
// error-free two-sums and the parity of the signs; the second recomputes each
// term and takes the exclusive sum as (hi - own) + lo, again error-free, so
// the result keeps ~48 bits of the total even when one term dominates.
template <int V, typename M, int RULE>
__global__ void __launch_bounds__(kThreads) k_check_any(PassArgs a, const int32_t *__restrict__ checks,
                                                        int32_t count) {
    pdl_wait();
    if (gated_off(a)) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = a.f_begin / (32 * V) + (int)blockIdx.y;
    const int f0 = g * 32 * V + lane * V;
    const size_t Fp = (size_t)a.Fp;
    M *r = reinterpret_cast<M *>(a.r);
    const bool first = a.pass == 0;
    const float *qsrc = first ? a.lamT : a.app;

    // rule 2: the chords of the tabulated phi, copied to shared memory by the
    // whole CTA before any warp may leave
    const float2 *tab = nullptr;
    if constexpr (RULE == 2) {
        extern __shared__ __align__(128) unsigned char smem[];
        float2 *t = reinterpret_cast<float2 *>(smem);
        for (int i = threadIdx.x; i < kPhiTableSize; i += blockDim.x) t[i] = a.phi_table[i];
        __syncthreads();
        tab = t;
    }
    auto phi_rule = [&](float x) {
        if constexpr (RULE == 2)
            return phi_tab(x, a.l_max, a.phi_lmax, tab);
        else
            return phi_hat(x, a.l_max, a.phi_lmax);
    };

    bool live[V];
    bool any_live = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        live[v] = !frame_bit(a.done, f0 + v);
        any_live |= live[v];
    }
    if (!__any_sync(kFull, any_live)) return;
    bool unsat[V];
#pragma unroll
    for (int v = 0; v < V; ++v) unsat[v] = false;

    for (int w = blockIdx.x * (kThreads / 32) + warp; w < count; w += gridDim.x * (kThreads / 32)) {
        const int i = checks[w];
        const int b = a.row_ptr[i];
        const int d = a.row_ptr[i + 1] - b;
        float alpha = a.ms_alpha, beta = a.ms_beta;
        if (RULE == 1 && a.ms_table) {
            const float2 t = __ldg(a.ms_table + d);
            alpha = t.x;
            beta = t.y;
        }
        float hi[V], lo[V];  // sum-product: compensated total; min-sum: two smallest |q|
        int idx[V];
        uint32_t par[V], z[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            hi[v] = lo[v] = RULE == 1 ? a.l_max : 0.0f;
            idx[v] = -1;
            par[v] = z[v] = 0u;
        }
        for (int k = 0; k < d; ++k) {
            const int slot = b + k;
            const int j = a.col_idx[slot];
            float av[V], qv[V];
            load_v<V, float>(qsrc + (size_t)j * Fp + f0, av);
            if (first) {
#pragma unroll
                for (int v = 0; v < V; ++v) qv[v] = av[v];
            } else {
                float rv[V];
                load_v<V, M>(r + (size_t)slot * Fp + f0, rv);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    // sum-product outputs next to a zero input are tiny, not
                    // zero, so that input takes the sign of APP (min-sum
                    // makes them exactly zero)
                    qv[v] = RULE == 1 ? av[v] - rv[v] : extrinsic(av[v], rv[v]);
                    z[v] ^= av[v] > 0.0f ? 1u : 0u;
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if constexpr (RULE == 1) {
                    const float x = fminf(fabsf(qv[v]), a.l_max);
                    if (x < hi[v]) {
                        lo[v] = hi[v];
                        hi[v] = x;
                        idx[v] = k;
                    } else if (x < lo[v]) {
                        lo[v] = x;
                    }
                } else {
                    float err;
                    hi[v] = two_sum(hi[v], phi_rule(fabsf(qv[v])), err);
                    lo[v] += err;
                }
                par[v] ^= qv[v] > 0.0f ? 1u : 0u;
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) unsat[v] |= z[v] != 0u;
        for (int k = 0; k < d; ++k) {
            const int slot = b + k;
            const int j = a.col_idx[slot];
            float av[V], qv[V];
            load_v<V, float>(qsrc + (size_t)j * Fp + f0, av);
            if (first) {
#pragma unroll
                for (int v = 0; v < V; ++v) qv[v] = av[v];
            } else {
                float rv[V];
                load_v<V, M>(r + (size_t)slot * Fp + f0, rv);
#pragma unroll
                for (int v = 0; v < V; ++v) qv[v] = RULE == 1 ? av[v] - rv[v] : extrinsic(av[v], rv[v]);
            }
            float out[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float mm;
                if constexpr (RULE == 1) {
                    const float m = idx[v] == k ? lo[v] : hi[v];
                    mm = fminf(fmaxf(fmaf(alpha, m, -beta), 0.0f), a.l_max);
                } else {
                    float own = phi_rule(fabsf(qv[v]));
                    float err;
                    float s = two_sum(hi[v], -own, err);
                    float excl = s + (err + lo[v]);
                    mm = phi_rule(excl);
                }
                uint32_t others = par[v] ^ (qv[v] > 0.0f ? 1u : 0u);
                out[v] = others ? mm : -mm;
            }
            store_v<V, M>(r + (size_t)slot * Fp + f0, out);
        }
    }
    if (a.syndrome) {
        bool bits[V];
#pragma unroll
        for (int v = 0; v < V; ++v) bits[v] = unsat[v] && live[v];
        or_frame_bits<V>(unsat_row(a, a.pass - 1), g, lane, bits);
    }
}

// Checks of degree above 32: one CTA per (check, group of 32 V frames), its
// eight warps splitting the check's inputs (warp w takes inputs w, w + 8,
// ...). Each warp forms partial results over its inputs -- the sum of
// phi(|q|) as an error-free pair (sum-product) or the two smallest |q| and
// the position of the smallest (min-sum), the parity of the inputs' signs and
// the previous decision's syndrome -- the CTA merges the eight partials in
// warp order through shared memory (every warp the same merge, so the same
// totals), and each warp writes the outputs of its inputs. A lone check of
// degree 96 then has eight warps per frame group working on it instead of
// one walking its 96 inputs twice.
template <int V, typename M, int RULE>
__global__ void __launch_bounds__(kThreads) k_check_wide(PassArgs a, const int32_t *__restrict__ checks,
                                                         int32_t count) {
    pdl_wait();
    if (gated_off(a)) return;
    constexpr int W = kThreads / 32;
    __shared__ float s_hi[W][32 * V], s_lo[W][32 * V];
    __shared__ int s_idx[W][32 * V];
    __shared__ uint32_t s_par[W][32 * V], s_z[W][32 * V];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = a.f_begin / (32 * V) + (int)blockIdx.y;
    const int f0 = g * 32 * V + lane * V;
    const size_t Fp = (size_t)a.Fp;
    M *r = reinterpret_cast<M *>(a.r);
    const bool first = a.pass == 0;
    const float *qsrc = first ? a.lamT : a.app;

    bool live[V];
    bool any_live = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        live[v] = !frame_bit(a.done, f0 + v);
        any_live |= live[v];
    }
    if (!__syncthreads_or(any_live)) return;  // the whole CTA leaves together
    bool unsat[V];
#pragma unroll
    for (int v = 0; v < V; ++v) unsat[v] = false;

    for (int w = blockIdx.x; w < count; w += gridDim.x) {
        const int i = checks[w];
        const int b = a.row_ptr[i];
        const int d = a.row_ptr[i + 1] - b;
        float alpha = a.ms_alpha, beta = a.ms_beta;
        if (RULE == 1 && a.ms_table) {
            const float2 t = __ldg(a.ms_table + d);
            alpha = t.x;
            beta = t.y;
        }
        float hi[V], lo[V];  // sum-product: compensated partial sum; min-sum: two smallest |q|
        int idx[V];
        uint32_t par[V], z[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            hi[v] = lo[v] = RULE == 1 ? a.l_max : 0.0f;
            idx[v] = -1;
            par[v] = z[v] = 0u;
        }
        // this warp's inputs k = warp + W u, u < nk; their column indices
        // are fetched 32 at a time (lane u holds input u of the chunk), so the
        // row loads of several inputs are in flight at once
        const int nk = (d - warp + W - 1) / W;
        for (int uc = 0; uc < nk; uc += 32) {
            const int jl = uc + lane < nk ? a.col_idx[b + warp + W * (uc + lane)] : 0;
            const int ue = min(32, nk - uc);
#pragma unroll 4
            for (int u = 0; u < ue; ++u) {
                const int k = warp + W * (uc + u);
                const int slot = b + k;
                float av[V], qv[V];
                load_v<V, float>(qsrc + (size_t)__shfl_sync(kFull, jl, u) * Fp + f0, av);
                if (first) {
#pragma unroll
                    for (int v = 0; v < V; ++v) qv[v] = av[v];
                } else {
                    float rv[V];
                    load_v<V, M>(r + (size_t)slot * Fp + f0, rv);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        // sum-product outputs next to a zero input are tiny, not
                        // zero, so that input takes the sign of APP (min-sum
                        // makes them exactly zero)
                        qv[v] = RULE == 1 ? av[v] - rv[v] : extrinsic(av[v], rv[v]);
                        z[v] ^= av[v] > 0.0f ? 1u : 0u;
                    }
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if constexpr (RULE == 1) {
                        const float x = fminf(fabsf(qv[v]), a.l_max);
                        if (x < hi[v]) {
                            lo[v] = hi[v];
                            hi[v] = x;
                            idx[v] = k;
                        } else if (x < lo[v]) {
                            lo[v] = x;
                        }
                    } else {
                        float err;
                        hi[v] = two_sum(hi[v], phi_hat(fabsf(qv[v]), a.l_max, a.phi_lmax), err);
                        lo[v] += err;
                    }
                    par[v] ^= qv[v] > 0.0f ? 1u : 0u;
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            s_hi[warp][lane * V + v] = hi[v];
            s_lo[warp][lane * V + v] = lo[v];
            s_idx[warp][lane * V + v] = idx[v];
            s_par[warp][lane * V + v] = par[v];
            s_z[warp][lane * V + v] = z[v];
        }
        __syncthreads();
        // merge the partials in warp order
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int c = lane * V + v;
            float H = s_hi[0][c], L = s_lo[0][c];
            int I = s_idx[0][c];
            uint32_t P = s_par[0][c], Z = s_z[0][c];
            for (int u = 1; u < W; ++u) {
                const float h2 = s_hi[u][c], l2 = s_lo[u][c];
                if constexpr (RULE == 1) {
                    // two smallest of both pairs; the position of the smallest
                    // matters only when it is unique, where this choice is exact
                    if (h2 < H) {
                        L = fminf(H, l2);
                        H = h2;
                        I = s_idx[u][c];
                    } else {
                        L = fminf(L, h2);
                    }
                } else {
                    float err;
                    const float s2 = two_sum(H, h2, err);
                    L = (L + l2) + err;
                    H = s2;
                }
                P ^= s_par[u][c];
                Z ^= s_z[u][c];
            }
            hi[v] = H;
            lo[v] = L;
            idx[v] = I;
            par[v] = P;
            unsat[v] |= Z != 0u;
        }
        __syncthreads();  // the partials are read before the next check overwrites them
        for (int uc = 0; uc < nk; uc += 32) {
            const int jl = uc + lane < nk ? a.col_idx[b + warp + W * (uc + lane)] : 0;
            const int ue = min(32, nk - uc);
#pragma unroll 4
            for (int u = 0; u < ue; ++u) {
                const int k = warp + W * (uc + u);
                const int slot = b + k;
                float av[V], qv[V];
                load_v<V, float>(qsrc + (size_t)__shfl_sync(kFull, jl, u) * Fp + f0, av);
                if (first) {
#pragma unroll
                    for (int v = 0; v < V; ++v) qv[v] = av[v];
                } else {
                    float rv[V];
                    load_v<V, M>(r + (size_t)slot * Fp + f0, rv);
#pragma unroll
                    for (int v = 0; v < V; ++v) qv[v] = RULE == 1 ? av[v] - rv[v] : extrinsic(av[v], rv[v]);
                }
                float out[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    float mm;
                    if constexpr (RULE == 1) {
                        const float m = idx[v] == k ? lo[v] : hi[v];
                        mm = fminf(fmaxf(fmaf(alpha, m, -beta), 0.0f), a.l_max);
                    } else {
                        const float own = phi_hat(fabsf(qv[v]), a.l_max, a.phi_lmax);
                        float err;
                        const float s2 = two_sum(hi[v], -own, err);
                        mm = phi_hat(s2 + (err + lo[v]), a.l_max, a.phi_lmax);
                    }
                    const uint32_t others = par[v] ^ (qv[v] > 0.0f ? 1u : 0u);
                    out[v] = others ? mm : -mm;
                }
                store_v<V, M>(r + (size_t)slot * Fp + f0, out);
            }
        }
    }
    if (a.syndrome && warp == 0) {
        bool bits[V];
#pragma unroll
        for (int v = 0; v < V; ++v) bits[v] = unsat[v] && live[v];
        or_frame_bits<V>(unsat_row(a, a.pass - 1), g, lane, bits);
    }
}

// ---------------------------------------------------------------------------
// Bit-node kernel: APP_j = lambda_j + sum_{i in M_j} r_ij
// ---------------------------------------------------------------------------

// Variables of degree above kWideVarDegree: the last bit_wide_ctas CTAs of
// the bit kernel's grid, one CTA per (variable, group of 32 V frames) at a
// time, its eight warps summing every eighth edge; the eight partial sums
// (dynamic shared memory) are added to lambda in warp order (a fixed order,
// so every frame layout gives the same posterior). They run beside the other
// CTAs, which skip these variables, and see the same live frames.
template <int V, typename M>
__device__ __forceinline__ void bit_wide_ctas(const PassArgs &a, int cta, int ctas, int g, const bool (&live)[V],
                                              bool all_live) {
    constexpr int W = kThreads / 32;
    extern __shared__ __align__(16) float part_smem[];
    float(*part)[32 * V] = reinterpret_cast<float(*)[32 * V]>(part_smem);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int f0 = g * 32 * V + lane * V;
    const size_t Fp = (size_t)a.Fp;
    const M *r = reinterpret_cast<const M *>(a.r);
    const uint64_t pol_keep = policy_evict_last(), pol_stream = policy_evict_first();
    for (int w = cta; w < a.n_wide_vars; w += ctas) {
        const int j = a.wide_vars[w];
        const int e0 = a.col_ptr[j], e1 = a.col_ptr[j + 1];
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
#pragma unroll 2
        for (int e = e0 + warp; e < e1; e += W) {
            float rv[V];
            load_v_hint<V, M>(r + (size_t)a.edge_slot[e] * Fp + f0, rv, pol_stream);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += rv[v];
        }
#pragma unroll
        for (int v = 0; v < V; ++v) part[warp][lane * V + v] = acc[v];
        __syncthreads();
        if (warp == 0) {
            load_v_hint<V, float>(a.lamT + (size_t)j * Fp + f0, acc, pol_stream);
            for (int u = 0; u < W; ++u)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] += part[u][lane * V + v];
            float *dst = a.app + (size_t)j * Fp + f0;
            if (all_live) {
                store_v_hint<V>(dst, acc, pol_keep);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (live[v]) dst[v] = acc[v];
            }
            if (a.dec) {
                bool bits[V];
#pragma unroll
                for (int v = 0; v < V; ++v) bits[v] = acc[v] > 0.0f;
                store_frame_bits<V>(a.dec + (size_t)j * (Fp / 32), g, lane, bits);
            }
        }
        __syncthreads();  // the partials are read before the next variable overwrites them
    }
}

// kWide: the grid ends in CTAs for the variables of degree above
// kWideVarDegree (a separate instance, so that the common one keeps its
// 32 registers and 8 CTAs per SM).
template <int V, typename M, bool kWide>
__global__ void __launch_bounds__(kThreads) k_bit(PassArgs a) {
    pdl_wait();
    if (gated_off(a)) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = a.f_begin / (32 * V) + (int)blockIdx.y;
    const int f0 = g * 32 * V + lane * V;
    const size_t Fp = (size_t)a.Fp;
    const M *r = reinterpret_cast<const M *>(a.r);
    const uint32_t *unsat_prev = a.pass > 0 ? unsat_row(a, a.pass - 1) : nullptr;
    const bool exit_test = a.early_exit && a.pass > 0;
    const bool cont = a.base != nullptr && a.pass > 0;  // continuous decoding, a later pass

    // One CTA records the frames whose previous hard decision was a codeword
    // (and, in continuous decoding, those that have used up their
    // iterations). Other CTAs may see the done bit either before or after it
    // is set; both give the same answer, since it is set exactly when the
    // condition they test as well holds.
    if ((exit_test || cont) && blockIdx.x == 0 && blockIdx.y == 0) {
        const int f_end = min(a.f_begin + a.f_count, a.n_frames);
        for (int f = a.f_begin + threadIdx.x; f < f_end; f += blockDim.x) {
            if (frame_bit(a.done, f)) continue;
            const bool zero = !frame_bit(unsat_prev, f);
            const int32_t own = cont ? a.pass - a.base[f] : a.pass;
            if (exit_test && zero) {
                atomicOr(a.done + (f >> 5), 1u << (f & 31));
                a.stop_iter[f] = own - 1;
            } else if (cont && own > a.max_iter) {
                atomicOr(a.done + (f >> 5), 1u << (f & 31));
                a.stop_iter[f] = a.max_iter | (zero ? 0 : kStopFailed);
            }
        }
        // the row the next check pass writes starts clear
        if (cont && a.unsat_ring)
            for (int w = threadIdx.x; w < a.Fp / 32; w += blockDim.x) unsat_row(a, a.pass)[w] = 0u;
    }

    bool live[V];
    bool all_live = true, any_live = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        live[v] = !frame_bit(a.done, f0 + v) && (!exit_test || frame_bit(unsat_prev, f0 + v));
        if (cont) live[v] = live[v] && a.pass - a.base[f0 + v] <= a.max_iter;
        all_live &= live[v];
        any_live |= live[v];
    }
    const int main_ctas = kWide ? (int)gridDim.x - a.bit_wide_ctas : (int)gridDim.x;
    if constexpr (kWide) {
        if ((int)blockIdx.x >= main_ctas) {
            if (__syncthreads_or(any_live))  // the whole CTA stays or leaves together
                bit_wide_ctas<V, M>(a, (int)blockIdx.x - main_ctas, a.bit_wide_ctas, g, live, all_live);
            return;
        }
    }
    if (!__any_sync(kFull, any_live)) return;

    const uint64_t pol_keep = policy_evict_last(), pol_stream = policy_evict_first();
    for (int j = blockIdx.x * (kThreads / 32) + warp; j < a.n; j += main_ctas * (kThreads / 32)) {
        const int e0 = a.col_ptr[j];
        const int e1 = a.col_ptr[j + 1];
        if (kWide && e1 - e0 > kWideVarDegree) continue;  // the trailing CTAs
        float acc[V];
        load_v_hint<V, float>(a.lamT + (size_t)j * Fp + f0, acc, pol_stream);
#pragma unroll 4
        for (int e = e0; e < e1; ++e) {
            const int slot = a.edge_slot[e];
            float rv[V];
            load_v_hint<V, M>(r + (size_t)slot * Fp + f0, rv, pol_stream);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += rv[v];
        }
        float *dst = a.app + (size_t)j * Fp + f0;
        if (all_live) {
            store_v_hint<V>(dst, acc, pol_keep);
        } else if (any_live) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (live[v]) dst[v] = acc[v];
        }
        if (a.dec) {
            // last pass: the hard decisions (Algorithm 5) as bit words for
            // the final syndrome
            bool bits[V];
#pragma unroll
            for (int v = 0; v < V; ++v) bits[v] = acc[v] > 0.0f;
            store_frame_bits<V>(a.dec + (size_t)j * (Fp / 32), g, lane, bits);
        }
    }
}

// r_out[f][e] = r[slot(e)][f] for real frames (float), 32 x 32 tiles.
template <typename M>
__global__ void k_export_r(PassArgs a, float *__restrict__ r_out) {
    __shared__ float tile[32][33];
    const M *r = reinterpret_cast<const M *>(a.r);
    const int64_t e0 = (int64_t)blockIdx.x * 32;
    const int f0 = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int64_t e = e0 + yy;
        int f = f0 + threadIdx.x;
        float val = 0.0f;
        if (e < a.E) val = MsgIO<M>::load1(r + (size_t)a.edge_slot[e] * a.Fp + f);
        tile[yy][threadIdx.x] = val;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int f = f0 + yy;
        int64_t e = e0 + threadIdx.x;
        if (f < a.n_frames && e < a.E) r_out[(size_t)f * a.E + e] = tile[threadIdx.x][yy];
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

inline dim3 pass_grid(const PassArgs &a, int64_t nodes, int V) {
    int groups = a.f_count / (32 * V);
    int64_t want = (nodes + (kThreads / 32) - 1) / (kThreads / 32);
    int64_t cap = a.grid_ctas / groups;
    if (cap < 1) cap = 1;
    int64_t x = want < cap ? want : cap;
    if (x < 1) x = 1;
    return dim3((unsigned)x, (unsigned)groups, 1);
}

// Only the (bin, frames-per-lane) pairs launch_check_rule selects are
// instantiated: V = 4 for bins 0-2 (degree <= 8), V = 2 for bins 0-3, V = 1
// for bins 0-4 (the unbounded bin has its own kernel, k_check_wide).
template <int V, typename M, int RULE>
static cudaError_t launch_check_bin_v(const PassArgs &a, int bin, const int32_t *checks, int32_t count,
                                      cudaStream_t s) {
    dim3 grid = pass_grid(a, count, V);
    if (bin == 0) {
        return launch_pdl(k_check_reg<4, V, M, RULE>, grid, dim3(kThreads), 0, s, a, checks, count);
    } else if (bin == 1) {
        return launch_pdl(k_check_reg<6, V, M, RULE>, grid, dim3(kThreads), 0, s, a, checks, count);
    } else if (bin == 2) {
        return launch_pdl(k_check_reg<8, V, M, RULE>, grid, dim3(kThreads), 0, s, a, checks, count);
    } else if constexpr (V <= 2) {
        if (bin == 3) {
            return launch_pdl(k_check_reg<16, V, M, RULE>, grid, dim3(kThreads), 0, s, a, checks, count);
        } else if (bin == 4) {
            if constexpr (V == 1) return launch_pdl(k_check_reg<32, V, M, RULE>, grid, dim3(kThreads), 0, s, a, checks, count);
            else return cudaErrorInvalidValue;
        } else {
            return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Element type of a message buffer for its tensor map.
template <typename M>
struct TensorType;
template <>
struct TensorType<float> {
    static constexpr int value = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
};
template <>
struct TensorType<__half> {
    static constexpr int value = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
};
template <>
struct TensorType<__nv_bfloat16> {
    static constexpr int value = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
};
template <>
struct TensorType<int8_t> {
    static constexpr int value = CU_TENSOR_MAP_DATA_TYPE_UINT8;
};

// Pipelined kernel: dynamic shared memory above 48 KB needs an opt-in, and
// the grid is sized to the CTAs that fit on the GPU at once.
template <int D, int V, typename M, int S, int MODE, int RULE>
static cudaError_t launch_bulk_mode(const PassArgs &a, const int2 *desc, int32_t count, cudaStream_t s) {
    // CTAs per SM, set up once per device; concurrent first calls may both
    // set it up (same attribute, same value), hence the atomic
    static std::atomic<int> resident_by_device[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> &resident = resident_by_device[dev & 63];
    const size_t smem = (size_t)BulkShape<D, V, M, S>::kSmem;
    int nres = resident.load(std::memory_order_acquire);
    if (nres == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_check_bulk<D, V, M, S, MODE, RULE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_check_bulk<D, V, M, S, MODE, RULE>, kThreads, smem);
        if (e != cudaSuccess) return e;
        nres = nb > 0 ? nb : 1;
        resident.store(nres, std::memory_order_release);
    }
    PassArgs b = a;
    b.grid_ctas = a.sm_count * nres;
    dim3 grid = pass_grid(b, count, V);
    // the tensor maps of this launch: input rows (float, one-row boxes) and
    // message rows (boxes of D rows), both 32 V frames wide
    const float *qsrc = MODE == 0 ? a.lamT : a.app;
    cudaError_t e = tensor_map_2d(&b.tm_q, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, qsrc, (uint64_t)a.Fp, (uint64_t)a.n,
                                  (uint64_t)a.Fp * sizeof(float), 32 * V, 1);
    if (e == cudaSuccess && MODE != 0)
        e = tensor_map_2d(&b.tm_r, TensorType<M>::value, a.r, (uint64_t)a.Fp, (uint64_t)a.E,
                          (uint64_t)a.Fp * sizeof(M), 32 * V, D);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_check_bulk<D, V, M, S, MODE, RULE>, grid, dim3(kThreads), smem, s, b, desc, count);
}

template <int D, int V, typename M, int S, int RULE>
static cudaError_t launch_bulk(const PassArgs &a, const int2 *desc, int32_t count, cudaStream_t s) {
    if (a.pass == 0) return launch_bulk_mode<D, V, M, S, 0, RULE>(a, desc, count, s);
    if (a.syndrome) return launch_bulk_mode<D, V, M, S, 2, RULE>(a, desc, count, s);
    return launch_bulk_mode<D, V, M, S, 1, RULE>(a, desc, count, s);
}

// The staged product-form kernel: shared memory for the bin's largest degree,
// the grid sized to the CTAs that fit on the GPU at once.
template <int V, typename M>
static cudaError_t launch_prod(const PassArgs &a, const int32_t *checks, int32_t count, cudaStream_t s) {
    const size_t smem = (size_t)(kThreads / 32) * ProdShape<V, M>::warp_bytes(a.bin_degree);
    static std::atomic<int> resident_by[64][33];  // per device and staged degree
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> &resident = resident_by[dev & 63][std::min(a.bin_degree, 32)];
    int nres = resident.load(std::memory_order_acquire);
    if (nres == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_check_prod<V, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kThreads / 32 * ProdShape<V, M>::warp_bytes(32)));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_check_prod<V, M>, kThreads, smem);
        if (e != cudaSuccess) return e;
        nres = nb > 0 ? nb : 1;
        resident.store(nres, std::memory_order_release);
    }
    PassArgs b = a;
    b.grid_ctas = a.sm_count * nres;
    return launch_pdl(k_check_prod<V, M>, pass_grid(b, count, V), dim3(kThreads), smem, s, a, checks, count);
}

// One CTA per check and group of 32 V frames, as many checks at once as the
// CTA budget of a pass allows.
template <int V, typename M, int RULE>
static cudaError_t launch_wide(const PassArgs &a, const int32_t *checks, int32_t count, cudaStream_t s) {
    const int groups = a.f_count / (32 * V);
    int64_t cap = a.grid_ctas / groups;
    if (cap < 1) cap = 1;
    const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(count, cap)), (unsigned)groups, 1);
    return launch_pdl(k_check_wide<V, M, RULE>, grid, dim3(kThreads), 0, s, a, checks, count);
}

template <typename M, int RULE>
static cudaError_t launch_check_rule(const PassArgs &a, int bin, const int32_t *checks, const int2 *desc,
                                     int32_t count, cudaStream_t s) {
    // Four frames per lane where the check's state fits the registers (degree
    // <= 6): the per-edge index, copy and control work is then shared by two
    // frame pairs. Wider checks run two frames per lane.
    if (a.check_schedule != 1 && bin <= 1 && a.V >= 4 && a.f_count % 128 == 0 && a.f_begin % 128 == 0) {
        if (bin == 0) return launch_bulk<4, 4, M, 2, RULE>(a, desc, count, s);
        return launch_bulk<6, 4, M, 2, RULE>(a, desc, count, s);
    }
    if (a.check_schedule != 1 && bin <= 3 && a.f_count % 64 == 0 && a.f_begin % 64 == 0) {
        switch (bin) {
        case 0: return launch_bulk<4, 2, M, 4, RULE>(a, desc, count, s);
        case 1: return launch_bulk<6, 2, M, 3, RULE>(a, desc, count, s);
        case 2: return launch_bulk<8, 2, M, 3, RULE>(a, desc, count, s);
        default:
            // checks of degree 9-12 only: 12 slots instead of 16 (a padding
            // slot is an exact no-op, so the results do not change)
            if (a.bin_degree <= 12) return launch_bulk<12, 2, M, 2, RULE>(a, desc, count, s);
            return launch_bulk<16, 2, M, 2, RULE>(a, desc, count, s);
        }
    }
    // Degrees 17-32. Up to degree 18 (the rate-5/6 codes), batches of 64-frame
    // groups run the pipelined kernel with 18 slots, its rows brought in by
    // tensor copies (n = 576 rate 5/6, 256 frames, 10 iterations: 0.156 ->
    // 0.099 ms against the register kernel). Other batches and wider checks:
    // in a code with many such checks the staged product-form kernel (the
    // same operations in the same order, so a frame's result does not depend
    // on which one ran), min-sum the any-degree kernel; in a code with few,
    // the register kernel, which pads every check to 32 slots at one frame
    // per lane (5.28 ms on n = 64800 rate 5/6, where it would be the only
    // choice), whose loads of one check are all in flight at once.
    if (a.check_schedule != 1 && bin == 4 && a.bin_degree <= 18 && a.f_count % 64 == 0 && a.f_begin % 64 == 0)
        return launch_bulk<18, 2, M, 2, RULE>(a, desc, count, s);
    if (bin == 4 && count >= kWideBinAnyKernel && RULE == 0) {
        if (a.V >= 2 && a.f_count % 64 == 0 && a.f_begin % 64 == 0) return launch_prod<2, M>(a, checks, count, s);
        return launch_prod<1, M>(a, checks, count, s);
    }
    if (bin == 4 && count >= kWideBinAnyKernel) {
        if (a.V >= 4 && a.f_count % 128 == 0 && a.f_begin % 128 == 0)
            return launch_pdl(k_check_any<4, M, RULE>, pass_grid(a, count, 4), dim3(kThreads), 0, s, a, checks,
                              count);
        if (a.V >= 2)
            return launch_pdl(k_check_any<2, M, RULE>, pass_grid(a, count, 2), dim3(kThreads), 0, s, a, checks,
                              count);
        return launch_pdl(k_check_any<1, M, RULE>, pass_grid(a, count, 1), dim3(kThreads), 0, s, a, checks, count);
    }
    // Degrees above 32: a CTA per check and frame group (k_check_wide). A
    // few such checks (the usual case) take narrow frame groups, so that
    // more CTAs share them: one check of degree 96 on 128 frames is four
    // CTAs at one frame per lane instead of one at four. Every width gives
    // the same results.
    if (bin == kNumCheckBins - 1) {
        const int64_t ctas4 = (int64_t)count * (a.f_count / 128);
        if (a.V >= 4 && a.f_count % 128 == 0 && a.f_begin % 128 == 0 && ctas4 >= a.sm_count)
            return launch_wide<4, M, RULE>(a, checks, count, s);
        if (a.V >= 2 && 2 * ctas4 >= a.sm_count) return launch_wide<2, M, RULE>(a, checks, count, s);
        return launch_wide<1, M, RULE>(a, checks, count, s);
    }
    // The register kernel for the other layouts. Wider bins keep more
    // messages per frame in registers: fewer frames per lane there, to stay
    // clear of spills (bin 3 runs two frames per lane at most, the 17-32 bin
    // of a code with few such checks one).
    if (a.V == 4 && bin < 3) return launch_check_bin_v<4, M, RULE>(a, bin, checks, count, s);
    if (a.V >= 2 && bin != 4) return launch_check_bin_v<2, M, RULE>(a, bin, checks, count, s);
    return launch_check_bin_v<1, M, RULE>(a, bin, checks, count, s);
}

// Rule 2 runs every bin through the any-degree kernel with the table in
// shared memory.
template <typename M>
static cudaError_t launch_check_table(const PassArgs &a, const int32_t *checks, int32_t count, cudaStream_t s) {
    const size_t smem = sizeof(float2) * kPhiTableSize;
    if (a.V >= 2) {
        k_check_any<2, M, 2><<<pass_grid(a, count, 2), kThreads, smem, s>>>(a, checks, count);
    } else {
        k_check_any<1, M, 2><<<pass_grid(a, count, 1), kThreads, smem, s>>>(a, checks, count);
    }
    return cudaGetLastError();
}

template <typename M>
cudaError_t launch_check_bin(const PassArgs &a, int bin, const int32_t *checks, const int2 *desc, int32_t count,
                             cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (a.check_rule == 2) return launch_check_table<M>(a, checks, count, s);
    if (a.check_rule == 1 || a.check_rule == 3) return launch_check_rule<M, 1>(a, bin, checks, desc, count, s);
    return launch_check_rule<M, 0>(a, bin, checks, desc, count, s);
}

template <int V, typename M>
static cudaError_t launch_bit_v(const PassArgs &a, cudaStream_t s) {
    // The bit kernel is bound by row gathers: 8 CTAs per SM (64 warps) keep
    // more rows in flight than the default 4. Variables of degree above
    // kWideVarDegree get trailing CTAs of the same grid (a CTA per variable
    // and frame group), with their partial sums in dynamic shared memory.
    PassArgs b = a;
    b.grid_ctas = a.sm_count * 8;
    dim3 grid = pass_grid(b, a.n, V);
    b.bit_wide_ctas = 0;
    if (a.n_wide_vars == 0) return launch_pdl(k_bit<V, M, false>, grid, dim3(kThreads), 0, s, b);
    const int64_t cap = std::max<int64_t>(1, (int64_t)a.sm_count * 8 / grid.y);
    b.bit_wide_ctas = (int32_t)std::min<int64_t>(a.n_wide_vars, cap);
    grid.x += (unsigned)b.bit_wide_ctas;
    return launch_pdl(k_bit<V, M, true>, grid, dim3(kThreads), sizeof(float) * (kThreads / 32) * 32 * V, s, b);
}

template <typename M>
cudaError_t launch_bit(const PassArgs &a, cudaStream_t s) {
    if (a.V == 8) return launch_bit_v<8, M>(a, s);
    if (a.V == 4) return launch_bit_v<4, M>(a, s);
    if (a.V == 2) return launch_bit_v<2, M>(a, s);
    return launch_bit_v<1, M>(a, s);
}

template <typename M>
cudaError_t launch_export_r(const PassArgs &a, float *r_out, cudaStream_t s) {
    if (a.E == 0 || a.n_frames == 0) return cudaSuccess;
    dim3 grid((unsigned)((a.E + 31) / 32), (unsigned)((a.n_frames + 31) / 32), 1);
    k_export_r<M><<<grid, dim3(32, 8, 1), 0, s>>>(a, r_out);
    return cudaGetLastError();
}

}  // namespace ldpc

#define LDPC_INSTANTIATE_PASS_KERNELS(M)                                                                       \
    namespace ldpc {                                                                                           \
    template cudaError_t launch_check_bin<M>(const PassArgs &, int, const int32_t *, const int2 *, int32_t,    \
                                             cudaStream_t);                                                    \
    template cudaError_t launch_bit<M>(const PassArgs &, cudaStream_t);                                        \
    template cudaError_t launch_export_r<M>(const PassArgs &, float *, cudaStream_t);                          \
    }

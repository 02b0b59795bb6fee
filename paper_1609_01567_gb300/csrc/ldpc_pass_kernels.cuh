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

#include "ldpc_internal.h"

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
    static __device__ __forceinline__ float load1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store1(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
};

template <int V, typename M>
__device__ __forceinline__ void load_v(const M *p, float (&x)[V]) {
    if constexpr (V == 4) {
        MsgIO<M>::load4(p, x);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = MsgIO<M>::load1(p + v);
    }
}

template <int V, typename M>
__device__ __forceinline__ void store_v(M *p, const float (&x)[V]) {
    if constexpr (V == 4) {
        MsgIO<M>::store4(p, x);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) MsgIO<M>::store1(p + v, x[v]);
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
//  * t = 2^(-x log2 e) with the product split exactly by an FMA, so the
//    exponent carries no rounding error beyond ~1e-12 relative.
//  * t < 1/16: phi = 2 atanh(t) = 2t (1 + t^2/3 + t^4/5 + t^6/7 + ...), the
//    series truncated after t^6/7 (relative error < 1e-10); this keeps full
//    relative precision for the tiny values that the sums of large-|q|
//    inputs are made of.
//  * otherwise phi = ln((1 + t) / (1 - t)), with 1 - t = 1 - e^-x from its
//    Taylor series below x = 1/4 (where 1 - t would cancel).
__device__ __forceinline__ float phi_core(float x) {
    const float kL2E = 1.44269502162933349609375f;   // log2(e) rounded to float
    const float kL2ELo = 1.925963033500011e-08f;     // log2(e) - kL2E
    const float kLn2 = 0.693147180559945309f;
    float p = -x * kL2E;
    float pe = fmaf(-x, kL2E, -p) - x * kL2ELo;
    float t = ex2_approx(p);
    t = fmaf(t, pe * kLn2, t);
    if (t < 0.0625f) {
        float t2 = t * t;
        float poly = fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 7.0f, 1.0f / 5.0f), 1.0f / 3.0f), 1.0f);
        return 2.0f * t * poly;
    }
    float u, num;
    if (x < 0.25f) {
        u = x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, -1.0f / 720.0f, 1.0f / 120.0f), -1.0f / 24.0f), 1.0f / 6.0f),
                             -0.5f),
                     1.0f);
        num = 2.0f - u;
    } else {
        u = 1.0f - t;
        num = 1.0f + t;
    }
    return lg2_approx(num * rcp_approx(u)) * kLn2;
}

__device__ __forceinline__ float phi_hat(float x, float l_max, float phi_lmax) {
    return phi_core(fminf(fmaxf(x, phi_lmax), l_max));
}

// Error-free sum: s + err == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &err) {
    float s = a + b;
    float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
    return s;
}

// ---------------------------------------------------------------------------
// Per-frame flag bits: frame f is bit (f & 31) of word f >> 5.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool frame_bit(const uint32_t *words, int f) { return (words[f >> 5] >> (f & 31)) & 1u; }

// OR the per-lane frame bits (frames f0 .. f0 + V - 1 of every lane) into the
// flag row `row` with one atomic per 32 frames.
template <int V>
__device__ __forceinline__ void or_frame_bits(uint32_t *row, int g, int lane, const bool (&bits)[V]) {
    if constexpr (V == 1) {
        uint32_t w = __ballot_sync(kFull, bits[0]);
        if (lane == 0 && w) atomicOr(row + g, w);
    } else {
        static_assert(V == 4, "V is 1 or 4");
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

// ---------------------------------------------------------------------------
// Check-node kernels
// ---------------------------------------------------------------------------

// Checks of degree <= D: a check's d messages stay in registers.
template <int D, int V, typename M>
__global__ void __launch_bounds__(kThreads) k_check_reg(PassArgs a, const int32_t *__restrict__ checks,
                                                        int32_t count) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = blockIdx.y;
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
    if (!__any_sync(kFull, any_live)) return;

    bool unsat[V];
#pragma unroll
    for (int v = 0; v < V; ++v) unsat[v] = false;

    for (int w = blockIdx.x * (kThreads / 32) + warp; w < count; w += gridDim.x * (kThreads / 32)) {
        const int i = checks[w];
        const int b = a.row_ptr[i];
        const int d = a.row_ptr[i + 1] - b;
        float mag[D][V];
        uint32_t ones[V];
        uint32_t z[V];
#pragma unroll
        for (int v = 0; v < V; ++v) ones[v] = z[v] = 0u;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                const int slot = b + k;
                const int j = a.col_idx[slot];
                float av[V];
                load_v<V, float>(qsrc + (size_t)j * Fp + f0, av);
                float qv[V];
                if (first) {
#pragma unroll
                    for (int v = 0; v < V; ++v) qv[v] = av[v];
                } else {
                    float rv[V];
                    load_v<V, M>(r + (size_t)slot * Fp + f0, rv);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        qv[v] = av[v] - rv[v];
                        z[v] ^= av[v] > 0.0f ? 1u : 0u;
                    }
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    mag[k][v] = phi_hat(fabsf(qv[v]), a.l_max, a.phi_lmax);
                    ones[v] |= (qv[v] > 0.0f ? 1u : 0u) << k;
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) mag[k][v] = 0.0f;
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) unsat[v] |= z[v] != 0u;
        // exclusive sums: suffix sums first, then a running prefix
        float suf[D][V];
        {
            float run[V];
#pragma unroll
            for (int v = 0; v < V; ++v) run[v] = 0.0f;
#pragma unroll
            for (int k = D - 1; k >= 0; --k) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    suf[k][v] = run[v];
                    run[v] += mag[k][v];
                }
            }
        }
        float pre[V];
        uint32_t par[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            pre[v] = 0.0f;
            par[v] = __popc(ones[v]) & 1u;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k < d) {
                float out[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    float m = phi_hat(pre[v] + suf[k][v], a.l_max, a.phi_lmax);
                    uint32_t others = par[v] ^ ((ones[v] >> k) & 1u);
                    out[v] = others ? m : -m;
                    pre[v] += mag[k][v];
                }
                store_v<V, M>(r + (size_t)(b + k) * Fp + f0, out);
            }
        }
    }
    if (a.syndrome) {
        bool bits[V];
#pragma unroll
        for (int v = 0; v < V; ++v) bits[v] = unsat[v] && live[v];
        or_frame_bits<V>(a.unsat + (size_t)(a.pass - 1) * (a.Fp / 32), g, lane, bits);
    }
}

// Checks of any degree: two sweeps over the check's edges. The first forms
// the total of phi^(|q|) as an unevaluated float pair (hi + lo) with
// error-free two-sums and the parity of the signs; the second recomputes each
// term and takes the exclusive sum as (hi - own) + lo, again error-free, so
// the result keeps ~48 bits of the total even when one term dominates.
template <int V, typename M>
__global__ void __launch_bounds__(kThreads) k_check_any(PassArgs a, const int32_t *__restrict__ checks,
                                                        int32_t count) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = blockIdx.y;
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
    if (!__any_sync(kFull, any_live)) return;
    bool unsat[V];
#pragma unroll
    for (int v = 0; v < V; ++v) unsat[v] = false;

    for (int w = blockIdx.x * (kThreads / 32) + warp; w < count; w += gridDim.x * (kThreads / 32)) {
        const int i = checks[w];
        const int b = a.row_ptr[i];
        const int d = a.row_ptr[i + 1] - b;
        float hi[V], lo[V];
        uint32_t par[V], z[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            hi[v] = lo[v] = 0.0f;
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
                    qv[v] = av[v] - rv[v];
                    z[v] ^= av[v] > 0.0f ? 1u : 0u;
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float err;
                hi[v] = two_sum(hi[v], phi_hat(fabsf(qv[v]), a.l_max, a.phi_lmax), err);
                lo[v] += err;
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
                for (int v = 0; v < V; ++v) qv[v] = av[v] - rv[v];
            }
            float out[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float own = phi_hat(fabsf(qv[v]), a.l_max, a.phi_lmax);
                float err;
                float s = two_sum(hi[v], -own, err);
                float excl = s + (err + lo[v]);
                float mm = phi_hat(excl, a.l_max, a.phi_lmax);
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
        or_frame_bits<V>(a.unsat + (size_t)(a.pass - 1) * (a.Fp / 32), g, lane, bits);
    }
}

// ---------------------------------------------------------------------------
// Bit-node kernel: APP_j = lambda_j + sum_{i in M_j} r_ij
// ---------------------------------------------------------------------------

template <int V, typename M>
__global__ void __launch_bounds__(kThreads) k_bit(PassArgs a) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = blockIdx.y;
    const int f0 = g * 32 * V + lane * V;
    const size_t Fp = (size_t)a.Fp;
    const M *r = reinterpret_cast<const M *>(a.r);
    const uint32_t *unsat_prev = a.pass > 0 ? a.unsat + (size_t)(a.pass - 1) * (a.Fp / 32) : nullptr;
    const bool exit_test = a.early_exit && a.pass > 0;

    // One CTA records the frames whose previous hard decision was a codeword.
    // Other CTAs may see the done bit either before or after it is set; both
    // give the same answer, since it is set exactly when that frame's
    // previous syndrome was zero, which they test as well.
    if (exit_test && blockIdx.x == 0 && blockIdx.y == 0) {
        for (int f = threadIdx.x; f < a.n_frames; f += blockDim.x) {
            if (!frame_bit(a.done, f) && !frame_bit(unsat_prev, f)) {
                atomicOr(a.done + (f >> 5), 1u << (f & 31));
                a.stop_iter[f] = a.pass - 1;
            }
        }
    }

    bool live[V];
    bool all_live = true, any_live = false;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        live[v] = !frame_bit(a.done, f0 + v) && (!exit_test || frame_bit(unsat_prev, f0 + v));
        all_live &= live[v];
        any_live |= live[v];
    }
    if (!__any_sync(kFull, any_live)) return;

    for (int j = blockIdx.x * (kThreads / 32) + warp; j < a.n; j += gridDim.x * (kThreads / 32)) {
        const int e0 = a.col_ptr[j];
        const int e1 = a.col_ptr[j + 1];
        float acc[V];
        load_v<V, float>(a.lamT + (size_t)j * Fp + f0, acc);
#pragma unroll 4
        for (int e = e0; e < e1; ++e) {
            const int slot = a.edge_slot[e];
            float rv[V];
            load_v<V, M>(r + (size_t)slot * Fp + f0, rv);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += rv[v];
        }
        float *dst = a.app + (size_t)j * Fp + f0;
        if (all_live) {
            store_v<V, float>(dst, acc);
        } else if (any_live) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (live[v]) dst[v] = acc[v];
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

inline dim3 pass_grid(const PassArgs &a, int64_t nodes) {
    int groups = a.Fp / (32 * a.V);
    int64_t want = (nodes + (kThreads / 32) - 1) / (kThreads / 32);
    int64_t cap = a.grid_ctas / groups;
    if (cap < 1) cap = 1;
    int64_t x = want < cap ? want : cap;
    if (x < 1) x = 1;
    return dim3((unsigned)x, (unsigned)groups, 1);
}

template <int V, typename M>
static cudaError_t launch_check_bin_v(const PassArgs &a, int bin, const int32_t *checks, int32_t count,
                                      cudaStream_t s) {
    dim3 grid = pass_grid(a, count);
    switch (bin) {
    case 0: k_check_reg<4, V, M><<<grid, kThreads, 0, s>>>(a, checks, count); break;
    case 1: k_check_reg<8, V, M><<<grid, kThreads, 0, s>>>(a, checks, count); break;
    case 2: k_check_reg<16, V, M><<<grid, kThreads, 0, s>>>(a, checks, count); break;
    case 3: k_check_reg<32, V, M><<<grid, kThreads, 0, s>>>(a, checks, count); break;
    default: k_check_any<V, M><<<grid, kThreads, 0, s>>>(a, checks, count); break;
    }
    return cudaGetLastError();
}

template <typename M>
cudaError_t launch_check_bin(const PassArgs &a, int bin, const int32_t *checks, int32_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    // The degree-32 bin keeps 32 messages per frame in registers: one frame
    // per lane there, to stay clear of spills.
    if (a.V == 4 && bin < 3) return launch_check_bin_v<4, M>(a, bin, checks, count, s);
    return launch_check_bin_v<1, M>(a, bin, checks, count, s);
}

template <typename M>
cudaError_t launch_bit(const PassArgs &a, cudaStream_t s) {
    dim3 grid = pass_grid(a, a.n);
    if (a.V == 4)
        k_bit<4, M><<<grid, kThreads, 0, s>>>(a);
    else
        k_bit<1, M><<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
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
    template cudaError_t launch_check_bin<M>(const PassArgs &, int, const int32_t *, int32_t, cudaStream_t);  \
    template cudaError_t launch_bit<M>(const PassArgs &, cudaStream_t);                                        \
    template cudaError_t launch_export_r<M>(const PassArgs &, float *, cudaStream_t);                          \
    }

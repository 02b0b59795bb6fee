// BPSK/AWGN channel-LLR generator of the BER simulator (Section IV, Eqs. 3-4)
// and raw Philox-4x64-10 blocks.
//
// Philox-4x64 with 10 rounds follows Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3" (SC'11): every round takes
// the two 128-bit products of counter words 0 and 2 with fixed odd
// multipliers, xors their high halves into words 1 and 3 and the round key,
// and permutes the words; the key advances by two Weyl constants per round.
// Being counter-based, the noise of any (frame, bit) is a pure function of
// (seed, frame index, bit index), independent of how frames are batched.
#include <cmath>

#include "ldpc_internal.h"

namespace ldpc {

struct U64x4 {
    uint64_t x[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                               uint64_t k1) {
    const uint64_t kM0 = 0xD2E7470EE14C6C93ull, kM1 = 0xCA5A826395121157ull;
    const uint64_t kW0 = 0x9E3779B97F4A7C15ull, kW1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        uint64_t lo0 = kM0 * c0, hi0 = __umul64hi(kM0, c0);
        uint64_t lo1 = kM1 * c2, hi1 = __umul64hi(kM1, c2);
        uint64_t y0 = hi1 ^ c1 ^ k0;
        uint64_t y2 = hi0 ^ c3 ^ k1;
        c0 = y0;
        c1 = lo1;
        c2 = y2;
        c3 = lo0;
        k0 += kW0;
        k1 += kW1;
    }
    return U64x4{{c0, c1, c2, c3}};
}

__global__ void k_philox_raw(uint64_t k0, uint64_t k1, uint64_t ctr0, uint64_t ctr1, int64_t count,
                             uint64_t *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        U64x4 w = philox4x64_10(ctr0 + (uint64_t)i, ctr1, 0, 0, k0, k1);
        ulonglong2 *o = reinterpret_cast<ulonglong2 *>(out + 4 * i);
        o[0] = make_ulonglong2(w.x[0], w.x[1]);
        o[1] = make_ulonglong2(w.x[2], w.x[3]);
    }
}

// One thread per (frame, group of 4 bits).
__global__ void k_gen_awgn(uint64_t seed, int64_t frame_offset, int32_t F, int32_t n, float sigma, float sigma2,
                           const uint8_t *__restrict__ cw, float *__restrict__ llr) {
    const int32_t Q = (n + 3) / 4;
    const int64_t total = (int64_t)F * Q;
    const float inv24 = 1.0f / 16777216.0f;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = (int32_t)(id / Q);
        const int32_t q = (int32_t)(id - (int64_t)f * Q);
        U64x4 w = philox4x64_10((uint64_t)q, (uint64_t)(frame_offset + f), 0, 0, seed, 0);
        float z[4];
#pragma unroll
        for (int pair = 0; pair < 2; ++pair) {
            float ua = (float)((w.x[2 * pair] >> 40) + 1) * inv24;
            float ub = (float)(w.x[2 * pair + 1] >> 40) * inv24;
            float rho = sqrtf(-2.0f * logf(ua));
            float sn, cs;
            sincospif(2.0f * ub, &sn, &cs);
            z[2 * pair] = rho * cs;
            z[2 * pair + 1] = rho * sn;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int32_t j = 4 * q + t;
            if (j < n) {
                const size_t idx = (size_t)f * n + j;
                float x = cw ? 2.0f * (float)cw[idx] - 1.0f : -1.0f;
                float y = x + sigma * z[t];
                llr[idx] = 2.0f * y / sigma2;
            }
        }
    }
}

// One thread per (frame, 256-bit Philox block): information bits, one byte
// each. Bit j of frame f is bit (j mod 64) of word (j mod 256) / 64 of the
// block at counter (j / 256, frame_offset + f), key (seed, 1); the key's
// second word keeps these bits apart from the channel noise (key (seed, 0)).
__global__ void k_gen_bits(uint64_t seed, int64_t frame_offset, int32_t F, int32_t k, uint8_t *__restrict__ out) {
    const int32_t B = (k + 255) / 256;
    const int64_t total = (int64_t)F * B;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = (int32_t)(id / B);
        const int32_t t = (int32_t)(id - (int64_t)f * B);
        U64x4 w = philox4x64_10((uint64_t)t, (uint64_t)(frame_offset + f), 0, 0, seed, 1);
        uint8_t *o = out + (size_t)f * k + (size_t)t * 256;
        const int32_t len = min(256, k - t * 256);
        if ((reinterpret_cast<uintptr_t>(o) & 7) == 0) {
            // eight bytes per store: byte b of the word is bit q + b
            int32_t q = 0;
            for (; q + 8 <= len; q += 8) {
                const uint32_t x = (uint32_t)(w.x[q >> 6] >> (q & 63)) & 0xFFu;
                uint64_t v = 0;
#pragma unroll
                for (int b = 0; b < 8; ++b) v |= (uint64_t)((x >> b) & 1u) << (8 * b);
                *reinterpret_cast<uint64_t *>(o + q) = v;
            }
            for (; q < len; ++q) o[q] = (uint8_t)((w.x[q >> 6] >> (q & 63)) & 1u);
        } else {
            for (int32_t q = 0; q < len; ++q) o[q] = (uint8_t)((w.x[q >> 6] >> (q & 63)) & 1u);
        }
    }
}

}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_gen_bits(uint64_t seed, int64_t frame_offset, int32_t F, int32_t k, uint8_t *bits, void *stream) {
    if (F < 0 || k < 0) return set_error(LDPC_EINVAL, "ldpc_gen_bits: negative size F=%d k=%d", F, k);
    if (frame_offset < 0) return set_error(LDPC_EINVAL, "ldpc_gen_bits: frame_offset < 0");
    if ((int64_t)F * k == 0) return LDPC_OK;
    if (!bits) return set_error(LDPC_EINVAL, "ldpc_gen_bits: bits is NULL");
    const int64_t total = (int64_t)F * ((k + 255) / 256);
    int64_t blocks = (total + 127) / 128;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_gen_bits<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(seed, frame_offset, F, k, bits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "ldpc_gen_bits: launch");
    return LDPC_OK;
}

extern "C" int ldpc_gen_awgn(uint64_t seed, int64_t frame_offset, int32_t F, int32_t n, float sigma2,
                             const uint8_t *codewords, float *llr, void *stream) {
    if (F < 0 || n < 0) return set_error(LDPC_EINVAL, "ldpc_gen_awgn: negative size F=%d n=%d", F, n);
    if (!(sigma2 > 0.0f) || !std::isfinite(sigma2)) return set_error(LDPC_EINVAL, "ldpc_gen_awgn: sigma2 must be > 0");
    if (frame_offset < 0) return set_error(LDPC_EINVAL, "ldpc_gen_awgn: frame_offset < 0");
    if ((int64_t)F * n == 0) return LDPC_OK;
    if (!llr) return set_error(LDPC_EINVAL, "ldpc_gen_awgn: llr is NULL");
    const int64_t total = (int64_t)F * ((n + 3) / 4);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    float sigma = (float)std::sqrt((double)sigma2);
    k_gen_awgn<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(seed, frame_offset, F, n, sigma, sigma2, codewords,
                                                                    llr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "ldpc_gen_awgn: launch");
    return LDPC_OK;
}

extern "C" int ldpc_philox4x64_10(uint64_t key0, uint64_t key1, uint64_t ctr0, uint64_t ctr1, int64_t count,
                                  uint64_t *out, void *stream) {
    if (count < 0) return set_error(LDPC_EINVAL, "ldpc_philox4x64_10: count < 0");
    if (count == 0) return LDPC_OK;
    if (!out) return set_error(LDPC_EINVAL, "ldpc_philox4x64_10: out is NULL");
    if (reinterpret_cast<uintptr_t>(out) % 16) return set_error(LDPC_EINVAL, "ldpc_philox4x64_10: out not 16-byte aligned");
    int64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_philox_raw<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(key0, key1, ctr0, ctr1, count, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "ldpc_philox4x64_10: launch");
    return LDPC_OK;
}

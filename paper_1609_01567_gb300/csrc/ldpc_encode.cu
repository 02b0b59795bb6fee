// Systematic encoder of IRA codes (H = [H1 | H2], H2 the dual-diagonal
// staircase in columns k .. n-1): c = [u | p] with p_i = s_i xor p_(i-1),
// s = H1 u. The BER simulator (Section IV) needs codewords; the paper sends
// the all-zero word or encodes on the host. Here the whole chain (information
// bits, encoder, channel, decoder, error count) stays on the device.
//
// Frames travel bit-sliced: word g of a row holds one bit of frames
// 32g .. 32g + 31, so one XOR combines 32 frames.
//   1. pack      u [F][k] bytes      -> U [k][G] words
//   2. checks    s_i = xor over the H1 neighbours of check i of U[j]
//   3. prefix    p_i = s_0 xor ... xor s_i, per word column (block scan)
//   4. write     c [F][n] bytes: the information bytes, then bit f of P
#include <algorithm>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr int kScanThreads = 1024;

__global__ void k_pack_info(const uint8_t *__restrict__ info, int32_t F, int32_t k, int32_t G,
                            uint32_t *__restrict__ U) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    for (int32_t g = blockIdx.y; g < G; g += gridDim.y) {
        uint32_t w = 0;
        const int32_t nb = min(32, F - 32 * g);
        for (int32_t b = 0; b < nb; ++b) w |= (uint32_t)(info[(size_t)(32 * g + b) * k + j] & 1u) << b;
        U[(size_t)j * G + g] = w;
    }
}

__global__ void k_check_words(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, int32_t m,
                              int32_t k, int32_t G, const uint32_t *__restrict__ U, uint32_t *__restrict__ S) {
    const int64_t total = (int64_t)m * G;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(id / G);
        const int32_t g = (int32_t)(id - (int64_t)i * G);
        uint32_t s = 0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t j = col_idx[e];
            if (j < k) s ^= U[(size_t)j * G + g];
        }
        S[(size_t)i * G + g] = s;
    }
}

// Inclusive xor-scan over the checks of one word column g, in place.
__global__ void __launch_bounds__(kScanThreads) k_prefix_xor(uint32_t *__restrict__ S, int32_t m, int32_t G) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t chunk = (m + kScanThreads - 1) / kScanThreads;
    const int32_t i0 = min(m, (int32_t)threadIdx.x * chunk), i1 = min(m, i0 + chunk);
    for (int32_t g = blockIdx.x; g < G; g += gridDim.x) {
        uint32_t x = 0;
        for (int32_t i = i0; i < i1; ++i) x ^= S[(size_t)i * G + g];
        // block-wide exclusive xor-scan of the chunk totals
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc ^= y;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t ^= y;
            }
            warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        uint32_t run = (inc ^ x) ^ (warp > 0 ? warp_tot[warp - 1] : 0u);
        for (int32_t i = i0; i < i1; ++i) {
            run ^= S[(size_t)i * G + g];
            S[(size_t)i * G + g] = run;
        }
        __syncthreads();  // warp_tot is reused by the next column
    }
}

__global__ void k_write_codeword(const uint8_t *__restrict__ info, const uint32_t *__restrict__ P, int32_t F,
                                 int32_t n, int32_t k, int32_t G, uint8_t *__restrict__ cw) {
    const int64_t total = (int64_t)F * n;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = (int32_t)(id / n);
        const int32_t j = (int32_t)(id - (int64_t)f * n);
        uint8_t v;
        if (j < k)
            v = info[(size_t)f * k + j] & 1u;
        else
            v = (uint8_t)((P[(size_t)(j - k) * G + (f >> 5)] >> (f & 31)) & 1u);
        cw[id] = v;
    }
}

unsigned grid_of(int64_t threads, int per_block, int sm_count) {
    int64_t b = (threads + per_block - 1) / per_block;
    const int64_t cap = (int64_t)std::max(sm_count, 1) * 16;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_encode_ira(ldpc_code_t *c, const uint8_t *info, int32_t n_frames, uint8_t *codeword,
                               void *stream) {
    if (!c) return set_error(LDPC_EINVAL, "ldpc_encode_ira: code is NULL");
    if (c->device < 0) return set_error(LDPC_ENODEV, "ldpc_encode_ira: host-only code");
    if (c->ira_k < 0)
        return set_error(LDPC_EINVAL, "ldpc_encode_ira: H has no staircase parity part in its last m columns");
    if (n_frames < 0) return set_error(LDPC_EINVAL, "ldpc_encode_ira: n_frames < 0");
    const int32_t k = c->ira_k, m = c->m, n = c->n;
    if (n_frames == 0 || n == 0) return LDPC_OK;
    if (!codeword || (k > 0 && !info)) return set_error(LDPC_EINVAL, "ldpc_encode_ira: NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    const int32_t G = (n_frames + 31) / 32;
    // stream-ordered scratch: U [k][G] and S [m][G] words
    uint32_t *U = nullptr, *S = nullptr;
    const size_t words = ((size_t)k + (size_t)m) * G;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&U), sizeof(uint32_t) * std::max<size_t>(words, 1), s);
    if (e == cudaSuccess) {
        S = U + (size_t)k * G;
        if (k > 0) {
            dim3 grid((unsigned)((k + 255) / 256), (unsigned)std::min(G, 65535));
            k_pack_info<<<grid, 256, 0, s>>>(info, n_frames, k, G, U);
        }
        if (m > 0) {
            k_check_words<<<grid_of((int64_t)m * G, 256, c->sm_count), 256, 0, s>>>(c->d.row_ptr, c->d.col_idx, m, k,
                                                                                    G, U, S);
            k_prefix_xor<<<(unsigned)std::min(G, 65535), kScanThreads, 0, s>>>(S, m, G);
        }
        k_write_codeword<<<grid_of((int64_t)n_frames * n, 256, c->sm_count), 256, 0, s>>>(info, S, n_frames, n, k, G,
                                                                                          codeword);
        e = cudaGetLastError();
        cudaError_t e2 = cudaFreeAsync(U, s);
        if (e == cudaSuccess) e = e2;
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_encode_ira");
    return LDPC_OK;
}

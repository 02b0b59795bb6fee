// Systematic encoder of IRA codes (H = [H1 | H2], H2 the dual-diagonal
// staircase in columns k .. n-1): c = [u | p] with p_i = s_i xor p_(i-1),
// s = H1 u. The BER simulator (Section IV) needs codewords; the paper sends
// the all-zero word or encodes on the host. Here the whole chain (information
// bits, encoder, channel, decoder, error count) stays on the device.
//
// Frames travel bit-sliced: word g of a row holds one bit of frames
// 32g .. 32g + 31, so one XOR combines 32 frames.
//   1. pack      u [F][k] bytes      -> U [k][G] words
//   2. checks    s_i = xor over the H1 neighbours of check i of U[j], and
//                its running xor within a chunk of checks
//   3. carries   exclusive xor-scan of the chunk totals
//   4. write     c [F][n] bytes: the information bytes, then bit f of
//                p_i = (running xor) xor (carry of the chunk)
#include <algorithm>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

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

// Checks are scanned in chunks of kChunk: one thread per (chunk, word
// column) forms s_i and its running xor inside the chunk, then one warp per
// word column turns the chunk totals into carries, and the write kernel
// applies the carry of each chunk.
constexpr int kChunk = 64;

__global__ void k_chunk_prefix(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, int32_t m,
                               int32_t k, int32_t G, const uint32_t *__restrict__ U, uint32_t *__restrict__ Pl,
                               uint32_t *__restrict__ T) {
    const int32_t nC = (m + kChunk - 1) / kChunk;
    const int64_t total = (int64_t)nC * G;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = (int32_t)(id / G);
        const int32_t g = (int32_t)(id - (int64_t)c * G);
        const int32_t i1 = min(m, (c + 1) * kChunk);
        uint32_t run = 0;
        for (int32_t i = c * kChunk; i < i1; ++i) {
            uint32_t s = 0;
            for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const int32_t j = col_idx[e];
                if (j < k) s ^= U[(size_t)j * G + g];
            }
            run ^= s;
            Pl[(size_t)i * G + g] = run;
        }
        T[(size_t)c * G + g] = run;
    }
}

// Exclusive xor-scan of the chunk totals T[c][g] over c, in place: one warp
// per word column g.
__global__ void k_chunk_carry(uint32_t *__restrict__ T, int32_t nC, int32_t G) {
    const int lane = threadIdx.x & 31;
    const int32_t per = (nC + 31) / 32;
    const int32_t c0 = min(nC, lane * per), c1 = min(nC, c0 + per);
    for (int32_t g = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); g < G; g += gridDim.x * (blockDim.x / 32)) {
        uint32_t x = 0;
        for (int32_t c = c0; c < c1; ++c) x ^= T[(size_t)c * G + g];
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc ^= y;
        }
        uint32_t run = inc ^ x;  // xor of the chunks before this lane's range
        for (int32_t c = c0; c < c1; ++c) {
            const uint32_t t = T[(size_t)c * G + g];
            T[(size_t)c * G + g] = run;
            run ^= t;
        }
    }
}

__global__ void k_write_codeword(const uint8_t *__restrict__ info, const uint32_t *__restrict__ Pl,
                                 const uint32_t *__restrict__ carry, int32_t F, int32_t n, int32_t k, int32_t G,
                                 uint8_t *__restrict__ cw) {
    const int64_t total = (int64_t)F * n;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = (int32_t)(id / n);
        const int32_t j = (int32_t)(id - (int64_t)f * n);
        uint8_t v;
        if (j < k)
            v = info[(size_t)f * k + j] & 1u;
        else {
            const int32_t i = j - k, g = f >> 5;
            v = (uint8_t)(((Pl[(size_t)i * G + g] ^ carry[(size_t)(i / kChunk) * G + g]) >> (f & 31)) & 1u);
        }
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
    // stream-ordered scratch: U [k][G], Pl [m][G] and T [chunks][G] words
    const int32_t nC = (m + kChunk - 1) / kChunk;
    uint32_t *U = nullptr;
    const size_t words = ((size_t)k + (size_t)m + (size_t)nC) * G;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&U), sizeof(uint32_t) * std::max<size_t>(words, 1), s);
    if (e == cudaSuccess) {
        uint32_t *Pl = U + (size_t)k * G;
        uint32_t *T = Pl + (size_t)m * G;
        if (k > 0) {
            dim3 grid((unsigned)((k + 255) / 256), (unsigned)std::min(G, 65535));
            k_pack_info<<<grid, 256, 0, s>>>(info, n_frames, k, G, U);
        }
        if (m > 0) {
            k_chunk_prefix<<<grid_of((int64_t)nC * G, 128, c->sm_count), 128, 0, s>>>(c->d.row_ptr, c->d.col_idx, m,
                                                                                      k, G, U, Pl, T);
            k_chunk_carry<<<(unsigned)std::min((G + 7) / 8, 65535), 256, 0, s>>>(T, nC, G);
        }
        k_write_codeword<<<grid_of((int64_t)n_frames * n, 256, c->sm_count), 256, 0, s>>>(info, Pl, T, n_frames, n, k,
                                                                                          G, codeword);
        e = cudaGetLastError();
        cudaError_t e2 = cudaFreeAsync(U, s);
        if (e == cudaSuccess) e = e2;
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_encode_ira");
    return LDPC_OK;
}

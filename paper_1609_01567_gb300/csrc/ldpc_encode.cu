// Systematic encoder of IRA codes (H = [H1 | H2], H2 the dual-diagonal
// staircase in columns k .. n-1): c = [u | p] with p_i = s_i xor p_(i-1),
// s = H1 u. The BER simulator (Section IV) needs codewords; the paper sends
// the all-zero word or encodes on the host. Here the whole chain (information
// bits, encoder, channel, decoder, error count) stays on the device.
//
// Frames travel bit-sliced: word g of a row holds one bit of frames
// 32g .. 32g + 31, so one XOR combines 32 frames.
//
// The dense systematic encoder below serves any code (lifted codes without a
// staircase included): the host reduces H over GF(2) once, and the device
// forms each parity bit as the xor of the information bits its reduced row
// holds.
//   1. pack      u [F][k] bytes      -> U [k][G] words
//   2. checks    s_i = xor over the H1 neighbours of check i of U[j], and
//                its running xor within a chunk of checks
//   3. carries   exclusive xor-scan of the chunk totals
//   4. write     c [F][n] bytes: the information bytes, then bit f of
//                p_i = (running xor) xor (carry of the chunk)
#include <algorithm>
#include <vector>

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

// Dense systematic encoder (any code): parity row i of the reduced H sets the
// bit of its pivot column to the xor of the information bits it holds.
// Bit-sliced like the IRA encoder: P [r][G] from U [k][G].
__global__ void k_dense_parity(const uint32_t *__restrict__ R, int32_t r, int32_t kw, const uint32_t *__restrict__ U,
                               int32_t G, uint32_t *__restrict__ P) {
    const int64_t total = (int64_t)r * G;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(id / G);
        const int32_t g = (int32_t)(id - (int64_t)i * G);
        const uint32_t *row = R + (size_t)i * kw;
        uint32_t acc = 0;
        for (int32_t w = 0; w < kw; ++w)
            for (uint32_t bits = row[w]; bits; bits &= bits - 1) acc ^= U[(size_t)(32 * w + __ffs(bits) - 1) * G + g];
        P[(size_t)i * G + g] = acc;
    }
}

// c[f][j]: information byte (colmap[j] = its index) or the parity bit of row
// -1 - colmap[j].
__global__ void k_dense_write(const uint8_t *__restrict__ info, const uint32_t *__restrict__ P,
                              const int32_t *__restrict__ colmap, int32_t F, int32_t n, int32_t k, int32_t G,
                              uint8_t *__restrict__ cw) {
    const int64_t total = (int64_t)F * n;
    for (int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; id < total;
         id += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = (int32_t)(id / n);
        const int32_t j = (int32_t)(id - (int64_t)f * n);
        const int32_t cm = colmap[j];
        cw[id] = cm >= 0 ? (uint8_t)(info[(size_t)f * k + cm] & 1u)
                         : (uint8_t)((P[(size_t)(-1 - cm) * G + (f >> 5)] >> (f & 31)) & 1u);
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

namespace {

// Reduced row echelon form of H over GF(2) (dense rows of 64-bit words),
// pivots taken column by column from the last column down, so that a code in
// IRA form keeps its staircase columns as the parity positions. Fills the
// column map (information index, or -1 - pivot row) and the parity rows over
// the information bits; returns the rank.
int32_t reduce_parity_check(const ldpc_code *c, std::vector<int32_t> &colmap, std::vector<uint32_t> &R, int32_t *k_out) {
    const int32_t m = c->m, n = c->n;
    const size_t nw = ((size_t)n + 63) / 64;
    std::vector<uint64_t> A((size_t)m * nw, 0);
    for (int32_t i = 0; i < m; ++i)
        for (int32_t e = c->row_ptr[i]; e < c->row_ptr[i + 1]; ++e) {
            const int32_t j = c->col_idx[e];
            A[(size_t)i * nw + j / 64] ^= 1ull << (j % 64);
        }
    std::vector<int32_t> pivot_col;
    int32_t rank = 0;
    for (int32_t j = n - 1; j >= 0 && rank < m; --j) {
        const size_t w = (size_t)j / 64;
        const uint64_t bit = 1ull << (j % 64);
        int32_t p = -1;
        for (int32_t i = rank; i < m && p < 0; ++i)
            if (A[(size_t)i * nw + w] & bit) p = i;
        if (p < 0) continue;
        uint64_t *pr = &A[(size_t)p * nw], *rr = &A[(size_t)rank * nw];
        if (p != rank) std::swap_ranges(pr, pr + nw, rr);
        for (int32_t i = 0; i < m; ++i) {
            uint64_t *ri = &A[(size_t)i * nw];
            if (i == rank || !(ri[w] & bit)) continue;
            for (size_t t = 0; t < nw; ++t) ri[t] ^= rr[t];
        }
        pivot_col.push_back(j);
        ++rank;
    }
    colmap.assign((size_t)n, 0);
    std::vector<char> is_pivot((size_t)n, 0);
    for (int32_t i = 0; i < rank; ++i) {
        colmap[pivot_col[i]] = -1 - i;
        is_pivot[pivot_col[i]] = 1;
    }
    std::vector<int32_t> info_col;
    for (int32_t j = 0; j < n; ++j)
        if (!is_pivot[j]) {
            colmap[j] = (int32_t)info_col.size();
            info_col.push_back(j);
        }
    const int32_t k = (int32_t)info_col.size();
    const size_t kw = ((size_t)k + 31) / 32;
    R.assign((size_t)rank * std::max<size_t>(kw, 1), 0u);
    for (int32_t i = 0; i < rank; ++i) {
        const uint64_t *ri = &A[(size_t)i * nw];
        for (int32_t t = 0; t < k; ++t) {
            const int32_t j = info_col[t];
            if ((ri[j / 64] >> (j % 64)) & 1ull) R[(size_t)i * kw + t / 32] |= 1u << (t % 32);
        }
    }
    *k_out = k;
    return rank;
}

}  // namespace

extern "C" int ldpc_code_build_encoder(ldpc_code_t *c, int32_t *k_out) {
    if (!c) return set_error(LDPC_EINVAL, "ldpc_code_build_encoder: code is NULL");
    if ((int64_t)c->m * c->n > ((int64_t)1 << 26))
        return set_error(LDPC_EINVAL, "ldpc_code_build_encoder: m * n = %lld exceeds 2^26 (dense elimination)",
                         (long long)c->m * c->n);
    std::lock_guard<std::mutex> lock(c->mu);
    if (c->enc_k < 0) {
        std::vector<int32_t> colmap;
        std::vector<uint32_t> R;
        int32_t k = 0;
        const int32_t r = reduce_parity_check(c, colmap, R, &k);
        if (c->device >= 0) {
            int prev = -1;
            cudaGetDevice(&prev);
            cudaSetDevice(c->device);
            uint32_t *dR = nullptr;
            int32_t *dmap = nullptr;
            cudaError_t e = cudaMalloc(&dR, sizeof(uint32_t) * std::max<size_t>(R.size(), 1));
            if (e == cudaSuccess) e = cudaMalloc(&dmap, sizeof(int32_t) * std::max<size_t>(colmap.size(), 1));
            if (e == cudaSuccess && !R.empty())
                e = cudaMemcpy(dR, R.data(), sizeof(uint32_t) * R.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess && !colmap.empty())
                e = cudaMemcpy(dmap, colmap.data(), sizeof(int32_t) * colmap.size(), cudaMemcpyHostToDevice);
            if (prev >= 0) cudaSetDevice(prev);
            if (e != cudaSuccess) {
                cudaFree(dR);
                cudaFree(dmap);
                return cuda_error(e, "ldpc_code_build_encoder");
            }
            c->enc_R = dR;
            c->enc_colmap = dmap;
        }
        c->enc_r = r;
        c->enc_k = k;
    }
    if (k_out) *k_out = c->enc_k;
    return LDPC_OK;
}

extern "C" int ldpc_encode(ldpc_code_t *c, const uint8_t *info, int32_t n_frames, uint8_t *codeword, void *stream) {
    if (!c) return set_error(LDPC_EINVAL, "ldpc_encode: code is NULL");
    if (c->device < 0) return set_error(LDPC_ENODEV, "ldpc_encode: host-only code");
    if (c->enc_k < 0) return set_error(LDPC_EINVAL, "ldpc_encode: no encoder (call ldpc_code_build_encoder first)");
    if (n_frames < 0) return set_error(LDPC_EINVAL, "ldpc_encode: n_frames < 0");
    const int32_t k = c->enc_k, r = c->enc_r, n = c->n;
    if (n_frames == 0 || n == 0) return LDPC_OK;
    if (!codeword || (k > 0 && !info)) return set_error(LDPC_EINVAL, "ldpc_encode: NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    const int32_t G = (n_frames + 31) / 32;
    const int32_t kw = (k + 31) / 32;
    uint32_t *U = nullptr;  // stream-ordered scratch: U [k][G], then P [r][G]
    const size_t words = ((size_t)k + (size_t)r) * G;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&U), sizeof(uint32_t) * std::max<size_t>(words, 1), s);
    if (e == cudaSuccess) {
        uint32_t *P = U + (size_t)k * G;
        if (k > 0) {
            dim3 grid((unsigned)((k + 255) / 256), (unsigned)std::min(G, 65535));
            k_pack_info<<<grid, 256, 0, s>>>(info, n_frames, k, G, U);
        }
        if (r > 0)
            k_dense_parity<<<grid_of((int64_t)r * G, 128, c->sm_count), 128, 0, s>>>(c->enc_R, r, std::max(kw, 1), U,
                                                                                     G, P);
        k_dense_write<<<grid_of((int64_t)n_frames * n, 256, c->sm_count), 256, 0, s>>>(info, P, c->enc_colmap, n_frames,
                                                                                       n, k, G, codeword);
        e = cudaGetLastError();
        cudaError_t e2 = cudaFreeAsync(U, s);
        if (e == cudaSuccess) e = e2;
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_encode");
    return LDPC_OK;
}

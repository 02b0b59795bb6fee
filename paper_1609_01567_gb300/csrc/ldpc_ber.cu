// Error counting of the BER simulator (Section IV): Hamming distance between
// decoded words and the transmitted ones (or the all-zero word, which is
// enough by linearity), accumulated on the device.
#include "ldpc_internal.h"

namespace ldpc {

// One CTA per frame (grid-stride over frames).
__global__ void k_count_errors(const uint8_t *__restrict__ bits, const uint8_t *__restrict__ ref, int32_t F, int32_t n,
                               const int32_t *__restrict__ iters, const uint8_t *__restrict__ ok,
                               unsigned long long *__restrict__ counts) {
    __shared__ unsigned int partial[32];
    for (int32_t f = blockIdx.x; f < F; f += gridDim.x) {
        const uint8_t *b = bits + (size_t)f * n;
        const uint8_t *r = ref ? ref + (size_t)f * n : nullptr;
        unsigned int errs = 0;
        for (int32_t j = threadIdx.x; j < n; j += blockDim.x) errs += (b[j] != (r ? r[j] : 0)) ? 1u : 0u;
        for (int o = 16; o > 0; o >>= 1) errs += __shfl_xor_sync(0xffffffffu, errs, o);
        if ((threadIdx.x & 31) == 0) partial[threadIdx.x >> 5] = errs;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int total = 0;
            for (int w = 0; w < (int)(blockDim.x / 32); ++w) total += partial[w];
            atomicAdd(counts + 0, (unsigned long long)total);
            if (total) atomicAdd(counts + 1, 1ull);
            if (iters) atomicAdd(counts + 2, (unsigned long long)iters[f]);
            if (ok && !ok[f]) atomicAdd(counts + 3, 1ull);
        }
        __syncthreads();
    }
}

}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_count_errors(const uint8_t *bits, const uint8_t *ref, int32_t n_frames, int32_t n,
                                 const int32_t *iters, const uint8_t *syndrome_ok, int64_t *counts, void *stream) {
    if (n_frames < 0 || n < 0) return set_error(LDPC_EINVAL, "ldpc_count_errors: negative size");
    if (!counts) return set_error(LDPC_EINVAL, "ldpc_count_errors: counts is NULL");
    if (n_frames == 0) return LDPC_OK;
    if (n > 0 && !bits) return set_error(LDPC_EINVAL, "ldpc_count_errors: bits is NULL");
    int blocks = n_frames < 152 * 16 ? n_frames : 152 * 16;
    k_count_errors<<<blocks, 256, 0, (cudaStream_t)stream>>>(bits, ref, n_frames, n, iters, syndrome_ok,
                                                            reinterpret_cast<unsigned long long *>(counts));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "ldpc_count_errors: launch");
    return LDPC_OK;
}

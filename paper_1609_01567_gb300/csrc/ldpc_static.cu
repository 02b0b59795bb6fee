// ldpc_decode_static: the decode of ldpc_decode with its scratch in a fixed,
// file-scope device array instead of memory allocated by the library.
//
// Who needs it: callers that cannot allocate device memory at the moment they
// decode. A receive chain with a hard latency budget cannot afford
// cudaMalloc, which may synchronise the whole device; a plug-in living inside
// another framework may be barred from allocating outside that framework's
// memory pool, or may run where device memory is capped and already
// committed. Such callers create their code handle (which uploads the code
// tables) during set-up and then decode with this entry point, which calls no
// allocating routine: no cudaMalloc, cudaFree or library call that
// allocates.
//
// The scratch array is kStaticScratchBytes (64 MiB) on every GPU that loads
// this library, held until the process exits. A decode whose scratch would
// not fit (messages E x Fp, posteriors and interleaved LLRs 2 x n x Fp, flags)
// is rejected with LDPC_EINVAL before anything is enqueued.
//
// The paper has no counterpart to this entry point.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ldpc_internal.h"

namespace ldpc {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; it keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Device address of g_scratch per device. In host code the name g_scratch is
// only a host-side stand-in, so the address is looked up once per device.
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_address(int dev, void **out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (dev < 0 || dev >= kMaxDevices) return set_error(LDPC_EINVAL, "ldpc_decode_static: device %d unsupported", dev);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_error(e, "ldpc_decode_static: cudaGetSymbolAddress of the static scratch");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LDPC_OK;
}

__device__ __forceinline__ bool bit_of(const uint32_t *w, int f) { return (w[f >> 5] >> (f & 31)) & 1u; }

__global__ void ks_init_done(uint32_t *done, int32_t F, int32_t Fp) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w == Fp / 32) done[w] = 0u;  // the status word after the frame bits
    if (w >= Fp / 32) return;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b)
        if (w * 32 + b >= F) bits |= 1u << b;
    done[w] = bits;
}

__global__ void ks_interleave(const float *__restrict__ llr, float *__restrict__ lamT, int32_t n, int32_t F,
                              int32_t Fp) {
    __shared__ float tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int f0 = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int f = f0 + yy;
        int64_t j = j0 + threadIdx.x;
        tile[yy][threadIdx.x] = (f < F && j < n) ? llr[(size_t)f * n + j] : 0.0f;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int64_t j = j0 + yy;
        int f = f0 + threadIdx.x;
        if (j < n) lamT[(size_t)j * Fp + f] = tile[threadIdx.x][yy];
    }
}

// One lane per (check, frame), a warp per check for 32 frames: xor of the
// hard decisions (Algorithm 6), one atomic per warp and check.
__global__ void ks_syndrome(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                            const float *__restrict__ app, int32_t m, int32_t Fp, uint32_t *row) {
    const int lane = threadIdx.x & 31;
    const int f = blockIdx.y * 32 + lane;
    for (int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < m; i += gridDim.x * (blockDim.x / 32)) {
        uint32_t z = 0;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) z ^= app[(size_t)col_idx[k] * Fp + f] > 0.0f ? 1u : 0u;
        const uint32_t w = __ballot_sync(0xffffffffu, z != 0u);
        if (lane == 0 && w) atomicOr(row + blockIdx.y, w);
    }
}

__global__ void ks_finalize(const float *__restrict__ app, uint8_t *__restrict__ bits, float *__restrict__ post,
                            int32_t n, int32_t F, int32_t Fp) {
    __shared__ float tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int f0 = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int64_t j = j0 + yy;
        int f = f0 + threadIdx.x;
        tile[yy][threadIdx.x] = j < n ? app[(size_t)j * Fp + f] : 0.0f;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int f = f0 + yy;
        int64_t j = j0 + threadIdx.x;
        if (f < F && j < n) {
            float x = tile[threadIdx.x][yy];
            bits[(size_t)f * n + j] = x > 0.0f ? 1 : 0;
            if (post) post[(size_t)f * n + j] = x;
        }
    }
}

__global__ void ks_frame_results(const uint32_t *done, const uint32_t *status, const int32_t *stop_iter,
                                 const uint32_t *final_unsat, int32_t F, int32_t max_iter, int32_t *iters,
                                 uint8_t *ok) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    if (status[0] != 0u) {  // a device wait of the call gave up: no result
        iters[f] = -1;
        ok[f] = 0;
        return;
    }
    bool stopped = bit_of(done, f);
    iters[f] = stopped ? stop_iter[f] : max_iter;
    ok[f] = stopped ? 1 : (bit_of(final_unsat, f) ? 0 : 1);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <typename M>
cudaError_t run_static(ldpc_code *c, unsigned char *scratch, const float *llr, int32_t F, int32_t max_iter,
                       const ldpc_decode_opts_t &o, float l_max, int32_t V, int32_t Fp, uint8_t *bits, int32_t *iters,
                       uint8_t *ok, float *post, cudaStream_t s) {
    const size_t words = (size_t)Fp / 32;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        unsigned char *p = scratch + off;
        off += align256(bytes);
        return p;
    };
    float *lamT = reinterpret_cast<float *>(carve(sizeof(float) * (size_t)c->n * Fp));
    float *app = reinterpret_cast<float *>(carve(sizeof(float) * (size_t)c->n * Fp));
    void *r = carve(sizeof(M) * (size_t)c->E * Fp);
    uint32_t *done = reinterpret_cast<uint32_t *>(carve(sizeof(uint32_t) * (words + 1)));
    uint32_t *unsat = reinterpret_cast<uint32_t *>(carve(sizeof(uint32_t) * words * (max_iter + 1)));
    int32_t *stop_iter = reinterpret_cast<int32_t *>(carve(sizeof(int32_t) * (size_t)Fp));

    PassArgs a = make_pass_args(c, o, l_max, F, V, Fp, lamT, app, r, done, done + words, unsat, stop_iter);

    // what must start at zero: the syndrome flag rows, and posteriors (the
    // padding frames' columns are read but never written)
    cudaError_t e = cudaMemsetAsync(unsat, 0, sizeof(uint32_t) * words * (max_iter + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(app, 0, sizeof(float) * (size_t)c->n * Fp, s);
    if (e != cudaSuccess) return e;
    ks_init_done<<<(unsigned)((words + 1 + 127) / 128), 128, 0, s>>>(done, F, Fp);
    if (c->n > 0) {
        dim3 grid((unsigned)((c->n + 31) / 32), (unsigned)(Fp / 32), 1);
        ks_interleave<<<grid, dim3(32, 8, 1), 0, s>>>(llr, lamT, c->n, F, Fp);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int32_t t = 0; t <= max_iter; ++t) {
        a.pass = t;
        a.syndrome = (t > 0 && a.early_exit) ? 1 : 0;
        for (int b = 0; b < kNumCheckBins; ++b) {
            int32_t count = c->bin_off[b + 1] - c->bin_off[b];
            if (count == 0) continue;
            a.bin_degree = c->bin_max_degree[b];
            e = launch_check_bin<M>(a, b, c->d.bin_checks + c->bin_off[b], c->d.bin_desc + c->bin_off[b], count, s);
            if (e != cudaSuccess) return e;
        }
        if (c->n > 0 && (e = launch_bit<M>(a, s)) != cudaSuccess) return e;
    }
    uint32_t *final_row = unsat + words * max_iter;
    if (c->m > 0 && c->E > 0) {
        int64_t blocks = std::min<int64_t>((c->m + 7) / 8, (int64_t)a.sm_count * 8);
        ks_syndrome<<<dim3((unsigned)std::max<int64_t>(blocks, 1), (unsigned)(Fp / 32), 1), 256, 0, s>>>(
            c->d.row_ptr, c->d.col_idx, app, c->m, Fp, final_row);
    }
    if (c->n > 0) {
        dim3 grid((unsigned)((c->n + 31) / 32), (unsigned)((F + 31) / 32), 1);
        ks_finalize<<<grid, dim3(32, 8, 1), 0, s>>>(app, bits, post, c->n, F, Fp);
    }
    ks_frame_results<<<(F + 255) / 256, 256, 0, s>>>(done, done + words, stop_iter, final_row, F, max_iter, iters,
                                                      ok);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (o.r_out) return launch_export_r<M>(a, o.r_out, s);
    return cudaSuccess;
}

struct DeviceSwitch {
    int prev = -1;
    explicit DeviceSwitch(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceSwitch() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_decode_static(const ldpc_code_t *code, const float *llr, int32_t n_frames, int32_t max_iter,
                                  const ldpc_decode_opts_t *opts, uint8_t *bits, int32_t *iters, uint8_t *syndrome_ok,
                                  float *post_llr, void *stream) {
    ldpc_code *c = const_cast<ldpc_code *>(code);
    ldpc_decode_opts_t o;
    memset(&o, 0, sizeof(o));
    if (opts) {
        o = *opts;
    } else {
        o.early_exit = 1;
        o.l_max = 20.0f;
    }
    // the argument rules of ldpc_decode, plus the one exception of this entry point
    float l_max = 20.0f;
    int st = check_opts(c, n_frames, max_iter, o, &l_max, "ldpc_decode_static");
    if (st != LDPC_OK) return st;
    if (o.profile) return set_error(LDPC_EINVAL, "ldpc_decode_static: profiling is not available on this entry point");
    if (n_frames == 0) return LDPC_OK;
    if ((c->n > 0 && (!llr || !bits)) || !iters || !syndrome_ok)
        return set_error(LDPC_EINVAL, "ldpc_decode_static: NULL llr, bits, iters or syndrome_ok");

    // the frame layout of ldpc_decode
    int32_t V = 0, Fp = 0;
    frames_layout(n_frames, o.frames_per_lane, &V, &Fp);
    const size_t msg = (size_t)msg_bytes(o.msg_dtype);
    const size_t words = (size_t)Fp / 32;
    const size_t need = align256(4 * (size_t)c->n * Fp) * 2 + align256(msg * (size_t)c->E * Fp) +
                        align256(4 * (words + 1)) + align256(4 * words * ((size_t)max_iter + 1)) +
                        align256(4 * (size_t)Fp);
    if (need > kStaticScratchBytes)
        return set_error(LDPC_EINVAL,
                         "ldpc_decode_static: %d frames of this code need %zu bytes of scratch; the static scratch "
                         "holds %zu bytes (decode fewer frames per call)",
                         n_frames, need, kStaticScratchBytes);

    DeviceSwitch guard(c->device);
    void *scratch = nullptr;
    st = scratch_address(c->device, &scratch);
    if (st != LDPC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    cudaError_t e;
    e = with_msg_type(o.msg_dtype, [&](auto tag) {
        using M = typename decltype(tag)::type;
        return run_static<M>(c, base, llr, n_frames, max_iter, o, l_max, V, Fp, bits, iters, syndrome_ok, post_llr, s);
    });
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode_static: kernel launch");
    return LDPC_OK;
}

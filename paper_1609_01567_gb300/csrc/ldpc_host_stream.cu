// Streaming decode of host batches: the copies of one batch overlap the
// decode of its neighbours.
//
// Two device staging slots alternate between batches. Batch i is copied in
// on a copy-in stream into slot i % 2 (once batch i - 2 has finished reading
// it), decoded on the caller's stream (once its copy-in and the copy-out of
// batch i - 2 are done), and copied out on a copy-out stream. The host thread
// only enqueues; the call returns when the last results are in host memory.
#include <mutex>

#include "ldpc_internal.h"

namespace ldpc {

struct HostStream {
    std::mutex mu;
    int32_t cap_frames = 0;
    int32_t n = 0;
    float *llr[2] = {nullptr, nullptr};
    uint8_t *bits[2] = {nullptr, nullptr};
    int32_t *iters[2] = {nullptr, nullptr};
    uint8_t *ok[2] = {nullptr, nullptr};
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t in_done[2] = {nullptr, nullptr}, dec_done[2] = {nullptr, nullptr}, out_done[2] = {nullptr, nullptr};
};

static void release_slots(HostStream &h) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(h.llr[k]);
        cudaFree(h.bits[k]);
        cudaFree(h.iters[k]);
        cudaFree(h.ok[k]);
        h.llr[k] = nullptr;
        h.bits[k] = nullptr;
        h.iters[k] = nullptr;
        h.ok[k] = nullptr;
    }
    h.cap_frames = 0;
}

void free_host_stream(ldpc_code *c) {
    HostStream *h = c->host_stream;
    if (!h) return;
    if (h->in) cudaStreamSynchronize(h->in);
    if (h->out) cudaStreamSynchronize(h->out);
    release_slots(*h);
    if (h->in) cudaStreamDestroy(h->in);
    if (h->out) cudaStreamDestroy(h->out);
    for (int k = 0; k < 2; ++k) {
        if (h->in_done[k]) cudaEventDestroy(h->in_done[k]);
        if (h->dec_done[k]) cudaEventDestroy(h->dec_done[k]);
        if (h->out_done[k]) cudaEventDestroy(h->out_done[k]);
    }
    delete h;
    c->host_stream = nullptr;
}

static cudaError_t prepare(HostStream &h, int32_t F, int32_t n) {
    cudaError_t e = cudaSuccess;
    if (!h.in) {
        if ((e = cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking)) != cudaSuccess) return e;
        for (int k = 0; k < 2; ++k) {
            if ((e = cudaEventCreateWithFlags(&h.in_done[k], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h.dec_done[k], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h.out_done[k], cudaEventDisableTiming)) != cudaSuccess)
                return e;
        }
    }
    if (F <= h.cap_frames && n == h.n) return cudaSuccess;
    release_slots(h);
    const size_t nf = std::max<size_t>((size_t)F * n, 1);
    for (int k = 0; k < 2; ++k) {
        if ((e = cudaMalloc(&h.llr[k], sizeof(float) * nf)) != cudaSuccess ||
            (e = cudaMalloc(&h.bits[k], nf)) != cudaSuccess ||
            (e = cudaMalloc(&h.iters[k], sizeof(int32_t) * (size_t)F)) != cudaSuccess ||
            (e = cudaMalloc(&h.ok[k], (size_t)F)) != cudaSuccess) {
            release_slots(h);
            return e;
        }
    }
    h.cap_frames = F;
    h.n = n;
    return cudaSuccess;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_decode_host_stream(ldpc_code_t *c, int32_t n_batches, const float *const *llr_host,
                                       int32_t n_frames, int32_t max_iter, const ldpc_decode_opts_t *opts,
                                       uint8_t *const *bits_host, int32_t *const *iters_host,
                                       uint8_t *const *ok_host, void *stream) {
    if (!c) return set_error(LDPC_EINVAL, "ldpc_decode_host_stream: code is NULL");
    if (c->device < 0) return set_error(LDPC_ENODEV, "ldpc_decode_host_stream: host-only code");
    if (n_batches < 0 || n_frames < 0)
        return set_error(LDPC_EINVAL, "ldpc_decode_host_stream: negative n_batches or n_frames");
    if (opts && (opts->r_out || opts->profile))
        return set_error(LDPC_EINVAL, "ldpc_decode_host_stream: r_out and profile are not available here");
    if (n_batches == 0 || n_frames == 0) return LDPC_OK;
    if (!llr_host || !bits_host || !iters_host || !ok_host)
        return set_error(LDPC_EINVAL, "ldpc_decode_host_stream: NULL buffer list");
    for (int32_t i = 0; i < n_batches; ++i)
        if ((c->n > 0 && (!llr_host[i] || !bits_host[i])) || !iters_host[i] || !ok_host[i])
            return set_error(LDPC_EINVAL, "ldpc_decode_host_stream: NULL buffer in batch %d", i);
    {
        std::lock_guard<std::mutex> lock(c->mu);
        if (!c->host_stream) c->host_stream = new (std::nothrow) HostStream();
        if (!c->host_stream) return set_error(LDPC_ENOMEM, "ldpc_decode_host_stream: out of host memory");
    }
    HostStream &h = *c->host_stream;
    std::lock_guard<std::mutex> lock(h.mu);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = prepare(h, n_frames, c->n);
    int st = LDPC_OK;
    const size_t nf = (size_t)n_frames * c->n;
    for (int32_t i = 0; i < n_batches && e == cudaSuccess && st == LDPC_OK; ++i) {
        const int k = i & 1;
        if (i >= 2) e = cudaStreamWaitEvent(h.in, h.dec_done[k], 0);
        if (e == cudaSuccess && nf)
            e = cudaMemcpyAsync(h.llr[k], llr_host[i], sizeof(float) * nf, cudaMemcpyHostToDevice, h.in);
        if (e == cudaSuccess) e = cudaEventRecord(h.in_done[k], h.in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h.in_done[k], 0);
        if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(s, h.out_done[k], 0);
        if (e != cudaSuccess) break;
        st = ldpc_decode(c, h.llr[k], n_frames, max_iter, opts, h.bits[k], h.iters[k], h.ok[k], nullptr, stream);
        if (st != LDPC_OK) break;
        e = cudaEventRecord(h.dec_done[k], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h.out, h.dec_done[k], 0);
        if (e == cudaSuccess && nf) e = cudaMemcpyAsync(bits_host[i], h.bits[k], nf, cudaMemcpyDeviceToHost, h.out);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(iters_host[i], h.iters[k], sizeof(int32_t) * n_frames, cudaMemcpyDeviceToHost, h.out);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ok_host[i], h.ok[k], n_frames, cudaMemcpyDeviceToHost, h.out);
        if (e == cudaSuccess) e = cudaEventRecord(h.out_done[k], h.out);
    }
    // drain whatever was enqueued, also after an error
    cudaError_t e1 = cudaStreamSynchronize(h.in);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaError_t e3 = cudaStreamSynchronize(h.out);
    if (prev >= 0) cudaSetDevice(prev);
    if (st != LDPC_OK) return st;
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode_host_stream");
    for (int32_t i = 0; i < n_batches; ++i)
        if ((st = report_gave_up(iters_host[i], n_frames, "ldpc_decode_host_stream")) != LDPC_OK) return st;
    return LDPC_OK;
}

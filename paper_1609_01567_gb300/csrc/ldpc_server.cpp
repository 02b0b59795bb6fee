// Decode server: continuous request batching over device-resident codes.
//
// Requests (code, frames, caller-owned device buffers) queue per code. A
// dispatcher thread hands the oldest queued requests of one code, up to a
// batch size, to a free slot -- a decode workspace with its own stream --
// gathers their LLRs into the slot's batch buffer, decodes, scatters the
// results back, and a host callback on the slot's stream completes the
// requests and frees the slot. Several slots are in flight at once, so
// requests arriving while others run are admitted as soon as a slot frees,
// and their decodes overlap on the device. The number of slots follows a
// device-memory budget (admission by free memory); submits beyond a bound on
// queued frames are refused with LDPC_EBUSY (back-pressure).
//
// A frame's result does not depend on the other frames of its batch (the
// kernels treat frames independently and deterministically), so a request
// decodes to the same bits, iterations and posteriors alone or in the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "ldpc_internal.h"

using namespace ldpc;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int32_t code = 0;
    int32_t F = 0;
    const float *llr = nullptr;
    uint8_t *bits = nullptr;
    int32_t *iters = nullptr;
    uint8_t *ok = nullptr;
    float *post = nullptr;
    double t_submit = 0.0, t_done = 0.0;
    int status = 1;  // 1 queued, 2 running, 0 done, < 0 error
};

struct Slot;

struct SlotCallback {
    ldpc_server *server;
    int slot;
};

struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    float *llr = nullptr;
    uint8_t *bits = nullptr;
    int32_t *iters = nullptr;
    uint8_t *ok = nullptr;
    float *post = nullptr;
    bool busy = false;
    std::vector<uint64_t> reqs;
    SlotCallback cb{};
};

}  // namespace

struct ldpc_server {
    int device = 0;
    std::vector<ldpc_code *> codes;
    ldpc_decode_opts_t opts{};
    float l_max = 20.0f;
    int32_t max_iter = 50;
    int32_t max_batch = 1024;
    int64_t max_pending = 1 << 20;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::deque<uint64_t>> pending;
    int64_t pending_frames = 0;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    int error = LDPC_OK;
    std::thread worker;
    // statistics
    int64_t completed = 0, frames_done = 0, batches = 0, info_bits = 0;
};

namespace {

void CUDART_CB slot_done(void *arg) {
    auto *cb = static_cast<SlotCallback *>(arg);
    ldpc_server *s = cb->server;
    std::lock_guard<std::mutex> lock(s->mu);
    Slot &sl = s->slots[cb->slot];
    const double t = now_ms();
    for (uint64_t id : sl.reqs) {
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) continue;
        it->second.status = 0;
        it->second.t_done = t;
        s->completed += 1;
        s->frames_done += it->second.F;
    }
    sl.reqs.clear();
    sl.busy = false;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Gather, decode and scatter one batch on a slot (no lock held).
cudaError_t launch_batch(ldpc_server *s, int si, int32_t code, const std::vector<Request> &batch) {
    Slot &sl = s->slots[si];
    ldpc_code *c = s->codes[code];
    const size_t n = (size_t)c->n;
    cudaError_t e = cudaSuccess;
    int32_t off = 0;
    for (const Request &r : batch) {
        if (e == cudaSuccess && n)
            e = cudaMemcpyAsync(sl.llr + (size_t)off * n, r.llr, sizeof(float) * n * r.F, cudaMemcpyDeviceToDevice,
                                sl.stream);
        off += r.F;
    }
    const int32_t F = off;
    if (e == cudaSuccess)
        e = enqueue_decode(c, sl.ws, sl.llr, F, s->max_iter, s->opts, s->l_max, sl.bits, sl.iters, sl.ok, sl.post,
                           sl.stream);
    off = 0;
    for (const Request &r : batch) {
        if (e == cudaSuccess && n)
            e = cudaMemcpyAsync(r.bits, sl.bits + (size_t)off * n, n * r.F, cudaMemcpyDeviceToDevice, sl.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r.iters, sl.iters + off, sizeof(int32_t) * r.F, cudaMemcpyDeviceToDevice, sl.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r.ok, sl.ok + off, r.F, cudaMemcpyDeviceToDevice, sl.stream);
        if (e == cudaSuccess && r.post && n)
            e = cudaMemcpyAsync(r.post, sl.post + (size_t)off * n, sizeof(float) * n * r.F, cudaMemcpyDeviceToDevice,
                                sl.stream);
        off += r.F;
    }
    if (e == cudaSuccess) e = cudaLaunchHostFunc(sl.stream, slot_done, &sl.cb);
    return e;
}

void dispatcher(ldpc_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        // a free slot and the code whose oldest request waits longest
        int si = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (!s->slots[i].busy) {
                si = (int)i;
                break;
            }
        int code = -1;
        double oldest = 0.0;
        for (size_t ci = 0; ci < s->pending.size(); ++ci) {
            if (s->pending[ci].empty()) continue;
            double t = s->reqs[s->pending[ci].front()].t_submit;
            if (code < 0 || t < oldest) {
                code = (int)ci;
                oldest = t;
            }
        }
        if (si < 0 || code < 0) {
            bool idle = code < 0;
            bool any_busy = false;
            for (auto &sl : s->slots) any_busy |= sl.busy;
            if (s->stop && idle && !any_busy) break;
            s->cv_work.wait(lock);
            continue;
        }
        // take requests of that code, oldest first, up to the batch size
        std::vector<Request> batch;
        std::vector<uint64_t> ids;
        int32_t frames = 0;
        auto &q = s->pending[code];
        while (!q.empty()) {
            Request &r = s->reqs[q.front()];
            if (!ids.empty() && frames + r.F > s->max_batch) break;
            frames += r.F;
            r.status = 2;
            ids.push_back(q.front());
            batch.push_back(r);
            q.pop_front();
        }
        s->pending_frames -= frames;
        Slot &sl = s->slots[si];
        sl.busy = true;
        sl.reqs = ids;
        s->batches += 1;
        s->info_bits += (int64_t)frames * (s->codes[code]->n - s->codes[code]->m);
        lock.unlock();
        cudaError_t e = launch_batch(s, si, code, batch);
        lock.lock();
        if (e != cudaSuccess) {
            s->error = cuda_error(e, "ldpc_server: batch launch");
            for (uint64_t id : ids) s->reqs[id].status = LDPC_ECUDA;
            sl.reqs.clear();
            sl.busy = false;
            s->cv_done.notify_all();
        }
    }
}

void server_free(ldpc_server *s) {
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        free_workspace(sl.ws);
        cudaFree(sl.llr);
        cudaFree(sl.bits);
        cudaFree(sl.iters);
        cudaFree(sl.ok);
        cudaFree(sl.post);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

}  // namespace

extern "C" int ldpc_server_create(int32_t n_codes, ldpc_code_t *const *codes, const ldpc_server_opts_t *opts,
                                  ldpc_server_t **out) {
    if (!out) return set_error(LDPC_EINVAL, "ldpc_server_create: out is NULL");
    *out = nullptr;
    if (n_codes <= 0 || !codes) return set_error(LDPC_EINVAL, "ldpc_server_create: no codes");
    ldpc_server_opts_t o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    ldpc_decode_opts_t d;
    memset(&d, 0, sizeof(d));
    d.early_exit = o.early_exit;
    d.l_max = o.l_max > 0.0f ? o.l_max : 20.0f;
    d.msg_dtype = o.msg_dtype;
    d.check_rule = o.check_rule;
    d.rule_alpha = o.rule_alpha;
    d.rule_beta = o.rule_beta;
    d.streams = 1;
    const int32_t max_batch = o.max_batch_frames > 0 ? o.max_batch_frames : 1024;
    if (max_batch > 8192) return set_error(LDPC_EINVAL, "ldpc_server_create: max_batch_frames above 8192");
    const int32_t max_iter = o.max_iter > 0 ? o.max_iter : 50;
    float l_max = 20.0f;
    int32_t n_max = 0;
    int64_t e_max = 0;
    for (int32_t i = 0; i < n_codes; ++i) {
        int st = check_opts(codes[i], 1, max_iter, d, &l_max, "ldpc_server_create");
        if (st != LDPC_OK) return st;
        if (codes[i]->device != codes[0]->device)
            return set_error(LDPC_EINVAL, "ldpc_server_create: codes on different devices");
        n_max = std::max(n_max, codes[i]->n);
        e_max = std::max(e_max, codes[i]->E);
    }
    ldpc_server *s = new (std::nothrow) ldpc_server();
    if (!s) return set_error(LDPC_ENOMEM, "ldpc_server_create: out of host memory");
    s->device = codes[0]->device;
    s->codes.assign(codes, codes + n_codes);
    s->opts = d;
    s->l_max = l_max;
    s->max_iter = max_iter;
    s->max_batch = max_batch;
    s->max_pending = o.max_pending_frames > 0 ? o.max_pending_frames : (1 << 20);
    s->pending.resize(n_codes);

    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    // slots: as many as the memory budget allows (at least one)
    const int32_t Fp = (max_batch + 255) / 256 * 256;
    const int mb = msg_bytes(d.msg_dtype);
    const int64_t per_slot = (int64_t)Fp * (8 * (int64_t)n_max + mb * e_max) +
                             (int64_t)max_batch * (5 * (int64_t)n_max + 5) + (int64_t)(max_iter + 1) * Fp / 8;
    int64_t budget = o.memory_budget;
    if (budget <= 0) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        budget = (int64_t)(free_b / 4);
    }
    int32_t n_slots = (int32_t)std::max<int64_t>(1, budget / std::max<int64_t>(per_slot, 1));
    n_slots = std::min(n_slots, o.max_slots > 0 ? o.max_slots : 4);
    s->slots.resize(n_slots);
    cudaError_t e = cudaSuccess;
    int st = LDPC_OK;
    for (int32_t i = 0; i < n_slots && e == cudaSuccess && st == LDPC_OK; ++i) {
        Slot &sl = s->slots[i];
        sl.cb = SlotCallback{s, i};
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ws.last_use, cudaEventDisableTiming);
        if (e == cudaSuccess) st = workspace_reserve(sl.ws, n_max, e_max, Fp, max_iter, mb);
        if (e == cudaSuccess && st == LDPC_OK) e = cudaMalloc(&sl.llr, sizeof(float) * (size_t)max_batch * n_max);
        if (e == cudaSuccess && st == LDPC_OK) e = cudaMalloc(&sl.bits, (size_t)max_batch * n_max);
        if (e == cudaSuccess && st == LDPC_OK) e = cudaMalloc(&sl.iters, sizeof(int32_t) * max_batch);
        if (e == cudaSuccess && st == LDPC_OK) e = cudaMalloc(&sl.ok, (size_t)max_batch);
        if (e == cudaSuccess && st == LDPC_OK) e = cudaMalloc(&sl.post, sizeof(float) * (size_t)max_batch * n_max);
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess || st != LDPC_OK) {
        if (e != cudaSuccess) st = cuda_error(e, "ldpc_server_create: slot allocation");
        server_free(s);
        return st;
    }
    s->worker = std::thread(dispatcher, s);
    *out = s;
    return LDPC_OK;
}

extern "C" int ldpc_server_submit(ldpc_server_t *s, int32_t code, const float *llr, int32_t n_frames, uint8_t *bits,
                                  int32_t *iters, uint8_t *syndrome_ok, float *post_llr, uint64_t *request_id) {
    if (!s || !request_id) return set_error(LDPC_EINVAL, "ldpc_server_submit: NULL argument");
    if (code < 0 || code >= (int32_t)s->codes.size()) return set_error(LDPC_EINVAL, "ldpc_server_submit: bad code");
    if (n_frames <= 0 || n_frames > s->max_batch)
        return set_error(LDPC_EINVAL, "ldpc_server_submit: %d frames outside [1, %d]", n_frames, s->max_batch);
    if (!llr || !bits || !iters || !syndrome_ok) return set_error(LDPC_EINVAL, "ldpc_server_submit: NULL buffer");
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->error != LDPC_OK) return s->error;
    if (s->pending_frames + n_frames > s->max_pending)
        return set_error(LDPC_EBUSY, "ldpc_server_submit: %lld frames already queued", (long long)s->pending_frames);
    uint64_t id = s->next_id++;
    Request r;
    r.code = code;
    r.F = n_frames;
    r.llr = llr;
    r.bits = bits;
    r.iters = iters;
    r.ok = syndrome_ok;
    r.post = post_llr;
    r.t_submit = now_ms();
    s->reqs.emplace(id, r);
    s->pending[code].push_back(id);
    s->pending_frames += n_frames;
    *request_id = id;
    s->cv_work.notify_all();
    return LDPC_OK;
}

extern "C" int ldpc_server_wait(ldpc_server_t *s, uint64_t id, int32_t timeout_ms, double *latency_ms) {
    if (!s) return set_error(LDPC_EINVAL, "ldpc_server_wait: server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return set_error(LDPC_EINVAL, "ldpc_server_wait: unknown request %llu", (unsigned long long)id);
    auto done = [&] { return s->reqs[id].status <= 0; };
    if (timeout_ms < 0)
        s->cv_done.wait(lock, done);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done))
        return set_error(LDPC_ETIMEOUT, "ldpc_server_wait: request %llu not done after %d ms", (unsigned long long)id,
                         timeout_ms);
    Request r = s->reqs[id];
    s->reqs.erase(id);
    if (latency_ms) *latency_ms = r.t_done - r.t_submit;
    return r.status == 0 ? LDPC_OK : r.status;
}

extern "C" int ldpc_server_stats(ldpc_server_t *s, ldpc_server_stats_t *out) {
    if (!s || !out) return set_error(LDPC_EINVAL, "ldpc_server_stats: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    memset(out, 0, sizeof(*out));
    out->slots = (int32_t)s->slots.size();
    out->completed = s->completed;
    out->frames = s->frames_done;
    out->batches = s->batches;
    out->queued_frames = s->pending_frames;
    out->info_bits = s->info_bits;
    return LDPC_OK;
}

extern "C" void ldpc_server_destroy(ldpc_server_t *s) {
    if (s) server_free(s);
}

// Decode server: continuous batching at the frame level over device-resident
// codes.
//
// Requests (code, frames, caller-owned device buffers) queue per code. A
// slot -- a frame set of up to max_batch_frames frames with its workspace and
// stream -- serves one code at a time and decodes in chunks of a few
// flooding passes. Frames enter and leave a running slot independently:
//   * after each chunk, every frame that has stopped (zero syndrome) or used
//     up its max_iter iterations has its results written to its request's
//     buffers, and the live frames are packed to the front of the slot;
//   * queued requests of the slot's code are then admitted into the free
//     frame groups at the back: their LLRs are interleaved into the slot, the
//     new groups run their first check and bit pass (Algorithm 2's pass before
//     the loop), and from the next chunk on they share every pass with the
//     frames already running, each frame counting its own iterations.
// A request completes when its last frame has been written out. Several slots
// run at once on their own streams, so the device overlaps their work while
// the dispatcher thread handles another slot between chunks; a slot whose
// frames are all done takes the code with the oldest waiting request. Slots
// are sized by a device-memory budget; submits beyond a bound on queued
// frames are refused with LDPC_EBUSY (back-pressure).
//
// A frame's decode does not depend on the other frames of its slot or on when
// it was admitted (the kernels treat frames independently and
// deterministically, and every frame runs its first pass and then its own
// count of later passes), so a request decodes to the same bits, iterations
// and posteriors alone or in the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "ldpc_internal.h"
#include "ldpc_launch.cuh"

using namespace ldpc;

namespace {

constexpr int32_t kChunkPasses = 4;  // flooding passes between two admission points
constexpr double kFairMs = 20.0;     // waiting-time lead that makes a busy slot drain for another code

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Where a frame's results go.
struct Dest {
    uint8_t *bits;  // [n]
    float *post;    // [n] or null
    int32_t *iters;
    uint8_t *ok;
};

struct Request {
    int32_t code = 0;
    int32_t F = 0;
    int32_t left = 0;  // frames not yet written out
    const float *llr = nullptr;
    uint8_t *bits = nullptr;
    int32_t *iters = nullptr;
    uint8_t *ok = nullptr;
    float *post = nullptr;
    double t_submit = 0.0, t_done = 0.0;
    int status = 1;  // 1 queued, 2 running, 0 done, < 0 error
};

struct SlotCallback {
    ldpc_server *server;
    int slot;
};

struct Slot {
    Workspace ws;                 // frame-interleaved state of the frame set
    int32_t *base = nullptr;      // [cap] pass before each frame's own first pass
    Dest *dest = nullptr;         // [2 cap] destination of each frame token
    uint8_t *emitted = nullptr;   // [2 cap] token written out by the last chunk
    const float **adm_src = nullptr;  // [cap] admission staging: LLR row of each new frame
    int32_t *adm_token = nullptr;     // [cap] its token
    Dest *adm_dest = nullptr;         // [cap] its destination
    // pinned host mirrors
    const float **h_src = nullptr;
    int32_t *h_token = nullptr;
    Dest *h_dest = nullptr;
    uint8_t *h_emitted = nullptr;
    int2 *h_count = nullptr;          // (moves, live frames) after the last chunk
    cudaStream_t stream = nullptr;
    int code = -1;                // code served, -1 when idle
    int32_t t = 1;                // the slot's next later pass (never reset)
    int32_t live = 0;             // live frames, packed at the front
    bool in_flight = false, status_ready = false;
    bool draining = false;        // admits nothing until its frames are done
    std::vector<uint64_t> token_req;     // request of each token (0 = free)
    std::vector<int32_t> free_tokens;
    SlotCallback cb{};
};

}  // namespace

struct ldpc_server {
    int device = 0;
    std::vector<ldpc_code *> codes;
    ldpc_decode_opts_t opts{};
    float l_max = 20.0f;
    int32_t max_iter = 50;
    int32_t max_batch = 1024;  // largest request
    int32_t cap = 1024;        // frames of a slot
    int32_t V = 4, group = 128;
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

// Interleave the LLR rows of n_new new frames into slots [a, a + count) (the
// rest of that range is padding), and set their state: frame token, pass
// base, not stopped, destination.
__global__ void __launch_bounds__(256) ks_admit(float *__restrict__ lamT, int32_t n, int32_t Fp, int32_t a,
                                                int32_t n_new, const float *const *__restrict__ src,
                                                const int32_t *__restrict__ token, const Dest *__restrict__ adm_dest,
                                                int32_t *__restrict__ slot_frame, int32_t *__restrict__ base,
                                                uint32_t *__restrict__ done, Dest *__restrict__ dest,
                                                uint8_t *__restrict__ emitted, int32_t t_base) {
    pdl_wait();
    __shared__ float tile[32][129];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t j0 = blockIdx.x * 128;
    const int32_t i0 = blockIdx.y * 32;
    for (int fi = warp; fi < 32; fi += 8) {
        const int32_t i = i0 + fi;
        const float *row = i < n_new ? src[i] : nullptr;
        for (int q = lane; q < 128; q += 32) {
            const int32_t j = j0 + q;
            tile[fi][q] = (row && j < n) ? row[j] : 0.0f;
        }
    }
    __syncthreads();
    for (int q = warp; q < 128; q += 8) {
        const int32_t j = j0 + q;
        if (j < n) lamT[(size_t)j * Fp + a + i0 + lane] = tile[lane][q];
    }
    if (blockIdx.x == 0 && warp == 0) {
        const int32_t i = i0 + lane, s = a + i;
        const bool real = i < n_new;
        slot_frame[s] = real ? token[i] : -1;
        base[s] = t_base;
        if (real) {
            dest[token[i]] = adm_dest[i];
            emitted[token[i]] = 0;
        }
        const uint32_t pad = __ballot_sync(0xffffffffu, !real);
        if (lane == 0) done[s >> 5] = pad;  // s is a multiple of 32 here
    }
}

// Results of the stopped frames that still hold a token: decisions (and
// posteriors) from their APP columns, iterations and syndrome flag from their
// stop record. CTA (x, y): 128 variables of 32 slots.
__global__ void __launch_bounds__(256) ks_emit(const float *__restrict__ app, int32_t n, int32_t Fp,
                                               const uint32_t *__restrict__ done, const uint32_t *__restrict__ status,
                                               const int32_t *__restrict__ slot_frame,
                                               const int32_t *__restrict__ stop_iter, const Dest *__restrict__ dest,
                                               uint8_t *__restrict__ emitted) {
    pdl_wait();
    __shared__ float tile[32][129];
    __shared__ int32_t s_tok[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t s0 = blockIdx.y * 32;
    if (warp == 0) {
        const int32_t s = s0 + lane;
        const int32_t tok = frame_bit(done, s) ? slot_frame[s] : -1;
        s_tok[lane] = tok;
        if (blockIdx.x == 0 && tok >= 0) {
            const Dest d = dest[tok];
            const int32_t st = stop_iter[s];
            const bool gave_up = *status != 0u;
            *d.iters = gave_up ? -1 : (st & ~kStopFailed);
            *d.ok = (gave_up || (st & kStopFailed)) ? 0 : 1;
            emitted[tok] = 1;
        }
    }
    __syncthreads();
    if (!__syncthreads_or(s_tok[lane] >= 0)) return;
    const int32_t j0 = blockIdx.x * 128;
    for (int q = warp; q < 128; q += 8) {
        const int32_t j = j0 + q;
        tile[lane][q] = (j < n && s_tok[lane] >= 0) ? app[(size_t)j * Fp + s0 + lane] : 0.0f;
    }
    __syncthreads();
    for (int fi = warp; fi < 32; fi += 8) {
        const int32_t tok = s_tok[fi];
        if (tok < 0) continue;
        const Dest d = dest[tok];
        for (int q = lane; q < 128; q += 32) {
            const int32_t j = j0 + q;
            if (j >= n) break;
            const float x = tile[fi][q];
            d.bits[j] = x > 0.0f ? 1 : 0;
            if (d.post) d.post[j] = x;
        }
    }
}

void CUDART_CB chunk_done(void *arg) {
    auto *cb = static_cast<SlotCallback *>(arg);
    ldpc_server *s = cb->server;
    std::lock_guard<std::mutex> lock(s->mu);
    Slot &sl = s->slots[cb->slot];
    sl.in_flight = false;
    sl.status_ready = true;
    s->cv_work.notify_all();
}

struct Admission {
    int32_t a = 0, count = 0, n_new = 0;  // slot range [a, a + count) of n_new new frames
};

// Enqueue one chunk of a slot (no lock held): admission of the staged new
// frames with their first pass, kChunkPasses later passes over the occupied
// groups, results of the stopped frames, packing, the status copy and the
// callback.
cudaError_t enqueue_chunk(ldpc_server *s, int si, const Admission &adm, int32_t range) {
    NvtxRange nvtx_chunk("ldpc server chunk");
    Slot &sl = s->slots[si];
    ldpc_code *c = s->codes[sl.code];
    const cudaStream_t st = sl.stream;
    Workspace &w = sl.ws;
    const int32_t Fp = s->cap;
    const int32_t words = Fp / 32;
    PassArgs a = make_pass_args(c, s->opts, s->l_max, Fp, s->V, Fp, w.lamT, w.app, w.r, w.done, w.done + words,
                                w.unsat, w.stop_iter);
    a.base = sl.base;
    a.max_iter = s->max_iter;
    a.unsat_ring = 1;
    cudaError_t e = cudaSuccess;
    auto passes = [&](int32_t f_begin, int32_t f_count, int32_t t) {
        PassArgs at = a;
        at.f_begin = f_begin;
        at.f_count = f_count;
        at.pass = t;
        at.syndrome = t > 0 ? 1 : 0;  // later passes test every frame's previous decision
        return with_msg_type(s->opts.msg_dtype, [&](auto tag) {
            using M = typename decltype(tag)::type;
            cudaError_t ee = cudaSuccess;
            for (int b = 0; b < kNumCheckBins && ee == cudaSuccess; ++b) {
                const int32_t count = c->bin_off[b + 1] - c->bin_off[b];
                if (count == 0) continue;
                at.bin_degree = c->bin_max_degree[b];
                ee = launch_check_bin<M>(at, b, c->d.bin_checks + c->bin_off[b], c->d.bin_desc + c->bin_off[b], count,
                                         st);
            }
            if (ee == cudaSuccess && c->n > 0) ee = launch_bit<M>(at, st);
            return ee;
        });
    };
    if (adm.n_new > 0) {
        const size_t k = (size_t)adm.n_new;
        if ((e = cudaMemcpyAsync(sl.adm_src, sl.h_src, sizeof(float *) * k, cudaMemcpyHostToDevice, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(sl.adm_token, sl.h_token, sizeof(int32_t) * k, cudaMemcpyHostToDevice, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(sl.adm_dest, sl.h_dest, sizeof(Dest) * k, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return e;
        const dim3 grid((unsigned)std::max<int32_t>(1, (c->n + 127) / 128), (unsigned)(adm.count / 32), 1);
        e = launch_pdl(ks_admit, grid, dim3(256), 0, st, w.lamT, c->n, Fp, adm.a, adm.n_new,
                       static_cast<const float *const *>(sl.adm_src), static_cast<const int32_t *>(sl.adm_token),
                       static_cast<const Dest *>(sl.adm_dest), w.slot_frame, sl.base, w.done, sl.dest, sl.emitted,
                       sl.t - 1);
        if (e == cudaSuccess) e = passes(adm.a, adm.count, 0);  // the new frames' first pass
        if (e != cudaSuccess) return e;
    }
    for (int32_t t = sl.t; t < sl.t + kChunkPasses && e == cudaSuccess; ++t) e = passes(0, range, t);
    if (e != cudaSuccess) return e;
    sl.t += kChunkPasses;
    if (c->n > 0) {
        const dim3 grid((unsigned)((c->n + 127) / 128), (unsigned)(range / 32), 1);
        e = launch_pdl(ks_emit, grid, dim3(256), 0, st, static_cast<const float *>(w.app), c->n, Fp,
                       static_cast<const uint32_t *>(w.done), static_cast<const uint32_t *>(w.done + words),
                       static_cast<const int32_t *>(w.slot_frame), static_cast<const int32_t *>(w.stop_iter),
                       static_cast<const Dest *>(sl.dest), sl.emitted);
    }
    if (e == cudaSuccess) e = launch_continuous_pack(a, s->opts.msg_dtype, s->group, w.slot_frame, w.moves, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_count, w.moves, sizeof(int2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_emitted, sl.emitted, (size_t)2 * s->cap, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, chunk_done, &sl.cb);
    return e;
}

// After a chunk (lock held): frames written out complete their requests.
void take_status(ldpc_server *s, Slot &sl) {
    const double t = now_ms();
    for (size_t tok = 0; tok < sl.token_req.size(); ++tok) {
        const uint64_t id = sl.token_req[tok];
        if (!id || !sl.h_emitted[tok]) continue;
        sl.token_req[tok] = 0;
        sl.free_tokens.push_back((int32_t)tok);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) continue;
        Request &r = it->second;
        if (--r.left == 0 && r.status == 2) {
            r.status = 0;
            r.t_done = t;
            s->completed += 1;
            s->frames_done += r.F;
        }
    }
    sl.live = sl.h_count->y;
    s->cv_done.notify_all();
}

int oldest_code(ldpc_server *s) {
    int code = -1;
    double oldest = 0.0;
    for (size_t ci = 0; ci < s->pending.size(); ++ci) {
        if (s->pending[ci].empty()) continue;
        const double t = s->reqs[s->pending[ci].front()].t_submit;
        if (code < 0 || t < oldest) {
            code = (int)ci;
            oldest = t;
        }
    }
    return code;
}

void fail_slot(ldpc_server *s, Slot &sl, int status) {
    s->error = status;
    for (uint64_t id : sl.token_req)
        if (id && s->reqs.count(id)) s->reqs[id].status = status;
    s->cv_done.notify_all();
}

void dispatcher(ldpc_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        bool launched = false, busy = false;
        for (size_t si = 0; si < s->slots.size(); ++si) {
            Slot &sl = s->slots[si];
            if (sl.in_flight) {
                busy = true;
                continue;
            }
            if (sl.status_ready) {
                take_status(s, sl);
                sl.status_ready = false;
            }
            if (s->error != LDPC_OK) continue;
            // an idle slot (or one whose code has run dry) takes the code
            // with the oldest waiting request
            if (sl.live == 0 && (sl.code < 0 || s->pending[sl.code].empty() || sl.draining)) {
                sl.code = oldest_code(s);
                sl.draining = false;
            }
            if (sl.code < 0) continue;
            // admit whole requests of the slot's code into the free groups,
            // unless an older request of a code no slot serves is waiting:
            // then this slot drains and takes that code when it frees
            const int32_t a = (sl.live + s->group - 1) / s->group * s->group;
            Admission adm;
            adm.a = a;
            auto &q = s->pending[sl.code];
            std::vector<uint64_t> taken;
            bool drain = false;
            const int oc = oldest_code(s);
            if (sl.draining) {
                drain = true;
            } else if (oc >= 0 && oc != sl.code && !q.empty()) {
                bool taken_care = false;  // served, or another slot drains for it already
                for (auto &other : s->slots) taken_care |= other.code == oc || other.draining;
                drain = !taken_care &&
                        s->reqs[q.front()].t_submit - s->reqs[s->pending[oc].front()].t_submit > kFairMs;
            }
            sl.draining = drain;
            while (!q.empty() && !drain) {
                Request &r = s->reqs[q.front()];
                if (a + adm.n_new + r.F > s->cap) break;
                for (int32_t f = 0; f < r.F; ++f) {
                    const int32_t i = adm.n_new + f;
                    const int32_t tok = sl.free_tokens.back();
                    sl.free_tokens.pop_back();
                    sl.token_req[tok] = q.front();
                    const size_t n = (size_t)s->codes[sl.code]->n;
                    sl.h_src[i] = r.llr + (size_t)f * n;
                    sl.h_token[i] = tok;
                    sl.h_dest[i] = Dest{r.bits + (size_t)f * n, r.post ? r.post + (size_t)f * n : nullptr,
                                        r.iters + f, r.ok + f};
                }
                adm.n_new += r.F;
                r.status = 2;
                r.left = r.F;
                s->pending_frames -= r.F;
                s->info_bits += (int64_t)r.F * (s->codes[sl.code]->n - s->codes[sl.code]->m);
                taken.push_back(q.front());
                q.pop_front();
            }
            if (sl.live == 0 && adm.n_new == 0) {
                sl.code = -1;
                sl.draining = false;
                continue;
            }
            if (adm.n_new > 0) s->batches += 1;
            adm.count = (adm.n_new + s->group - 1) / s->group * s->group;
            const int32_t range = adm.n_new > 0 ? a + adm.count : a;
            sl.in_flight = true;
            launched = true;
            lock.unlock();
            const cudaError_t e = enqueue_chunk(s, (int)si, adm, range);
            lock.lock();
            if (e != cudaSuccess) {
                sl.in_flight = false;
                fail_slot(s, sl, cuda_error(e, "ldpc_server: chunk launch"));
            }
        }
        if (launched) continue;
        if (s->stop && !busy) {
            bool queued = false;
            for (auto &q : s->pending) queued |= !q.empty();
            bool running = false;
            for (auto &sl : s->slots) running |= sl.live > 0;
            if ((!queued && !running) || s->error != LDPC_OK) break;
        }
        s->cv_work.wait(lock);
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
        cudaFree(sl.base);
        cudaFree(sl.dest);
        cudaFree(sl.emitted);
        cudaFree(sl.adm_src);
        cudaFree(sl.adm_token);
        cudaFree(sl.adm_dest);
        cudaFreeHost(sl.h_src);
        cudaFreeHost(sl.h_token);
        cudaFreeHost(sl.h_dest);
        cudaFreeHost(sl.h_emitted);
        cudaFreeHost(sl.h_count);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

// Device and pinned buffers of one slot, its initial state (no frame, every
// slot stopped, syndrome rows clear).
cudaError_t make_slot(ldpc_server *s, Slot &sl, int32_t n_max, int64_t e_max, int mb, int *st) {
    const int32_t cap = s->cap;
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ws.last_use, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    *st = workspace_reserve(sl.ws, n_max, e_max, cap, 1, mb);  // two syndrome rows
    if (*st != LDPC_OK) return cudaSuccess;
    if ((e = cudaMalloc(&sl.base, sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = cudaMalloc(&sl.dest, sizeof(Dest) * 2 * cap)) != cudaSuccess ||
        (e = cudaMalloc(&sl.emitted, (size_t)2 * cap)) != cudaSuccess ||
        (e = cudaMalloc(&sl.adm_src, sizeof(float *) * cap)) != cudaSuccess ||
        (e = cudaMalloc(&sl.adm_token, sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = cudaMalloc(&sl.adm_dest, sizeof(Dest) * cap)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_src, sizeof(float *) * cap)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_token, sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_dest, sizeof(Dest) * cap)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_emitted, (size_t)2 * cap)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_count, sizeof(int2))) != cudaSuccess)
        return e;
    const int32_t words = cap / 32;
    if ((e = cudaMemset(sl.ws.done, 0xFF, sizeof(uint32_t) * words)) != cudaSuccess ||
        (e = cudaMemset(sl.ws.done + words, 0, sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(sl.ws.unsat, 0, sizeof(uint32_t) * 2 * words)) != cudaSuccess ||
        (e = cudaMemset(sl.ws.slot_frame, 0xFF, sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = cudaMemset(sl.base, 0, sizeof(int32_t) * cap)) != cudaSuccess ||
        (e = cudaMemset(sl.emitted, 0, (size_t)2 * cap)) != cudaSuccess)
        return e;
    std::memset(sl.h_emitted, 0, (size_t)2 * cap);
    sl.token_req.assign((size_t)2 * cap, 0);
    for (int32_t tok = 2 * cap - 1; tok >= 0; --tok) sl.free_tokens.push_back(tok);
    return cudaSuccess;
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
    // a slot of max_batch frames in whole groups of 32 V (the frame layout of
    // ldpc_decode for that batch size)
    frames_layout(max_batch, 0, &s->V, &s->cap);
    s->group = 32 * s->V;
    s->max_pending = o.max_pending_frames > 0 ? o.max_pending_frames : (1 << 20);
    s->pending.resize(n_codes);

    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    // slots: as many as the memory budget allows (at least one)
    const int32_t Fp = s->cap;
    const int mb = msg_bytes(d.msg_dtype);
    const int64_t per_slot = (int64_t)Fp * (8 * (int64_t)n_max + mb * e_max + 64) + 2 * (int64_t)Fp / 8;
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
        s->slots[i].cb = SlotCallback{s, i};
        e = make_slot(s, s->slots[i], n_max, e_max, mb, &st);
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

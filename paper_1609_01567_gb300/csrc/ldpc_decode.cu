// Decode driver (Algorithm 2) and the layout/flag kernels around the passes.
//
// One decode call of F frames runs, per chunk of frames:
//   init flags -> interleave LLRs -> pass 0 (check on q = lambda, bit) ->
//   passes 1..max_iter (check, fused syndrome of the previous decision,
//   bit with the early-exit test) -> final syndrome -> results.
// Every step is a kernel of this library on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ldpc_internal.h"
#include "ldpc_pass_kernels.cuh"

namespace ldpc {

constexpr int32_t kMaxChunkFrames = 8192;

// llr [F][n] (frame-major) -> lamT [n][Fp] (frame-interleaved); padding
// frames get lambda = 0.
__global__ void __launch_bounds__(256) k_interleave(const float *__restrict__ llr, float *__restrict__ lamT,
                                                    int32_t n, int32_t F, int32_t Fp) {
    pdl_wait();
    // tile of 32 frames x 128 variables: frame rows read as float4 when the
    // rows are 4-aligned, variable rows written 32 frames (128 bytes) at once
    __shared__ float tile[128][33];
    const int32_t j0 = blockIdx.x * 128;
    const int32_t f0 = blockIdx.y * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(llr) & 15) == 0;
#pragma unroll
    for (int fi = warp; fi < 32; fi += 8) {
        const int32_t f = f0 + fi, j = j0 + 4 * lane;
        float x[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (f < F) {
            const float *src = llr + (size_t)f * n + j;
            if (vec && j + 3 < n) {
                const float4 v = *reinterpret_cast<const float4 *>(src);
                x[0] = v.x;
                x[1] = v.y;
                x[2] = v.z;
                x[3] = v.w;
            } else {
                for (int b = 0; b < 4; ++b)
                    if (j + b < n) x[b] = src[b];
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) tile[4 * lane + b][fi] = x[b];
    }
    __syncthreads();
    for (int jj = warp; jj < 128; jj += 8) {
        const int32_t j = j0 + jj;
        if (j < n) lamT[(size_t)j * Fp + f0 + lane] = tile[jj][lane];
    }
}

// done bits: padding frames (f >= F) start as stopped; slot f holds frame f.
__global__ void k_init_done(uint32_t *done, uint32_t *status, uint32_t *unsat, int64_t n_unsat, int32_t F,
                            int32_t Fp, int32_t *slot_frame) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w == 0) *status = 0u;
    for (int64_t i = w; i < n_unsat; i += (int64_t)gridDim.x * blockDim.x) unsat[i] = 0u;  // syndrome rows
    if (slot_frame)
        for (int32_t f = w; f < Fp; f += gridDim.x * blockDim.x) slot_frame[f] = f < F ? f : -1;
    if (w >= Fp / 32) return;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b)
        if (w * 32 + b >= F) bits |= 1u << b;
    done[w] = bits;
}

// Syndrome of the final hard decisions (Algorithm 6) from their bit words
// dec [n][G] (G = Fp / 32 words per variable): thread (check i, word group)
// xors the words of the check's variables (a check of degree above 32 by its
// whole warp, lanes striding its edges), and each warp ors its checks'
// unsatisfied-frame words into `row` with one atomic per word.
template <int W>
__global__ void k_syndrome_words(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, int32_t m,
                                 const uint32_t *__restrict__ dec, int32_t G, uint32_t *__restrict__ row) {
    pdl_wait();
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t w0 = blockIdx.y * W;
    uint32_t z[W];
#pragma unroll
    for (int q = 0; q < W; ++q) z[q] = 0u;
    auto add = [&](uint32_t(&acc)[W], int32_t e) {
        const uint32_t *p = dec + (size_t)col_idx[e] * G + w0;
        if constexpr (W == 4) {
            const uint4 v = *reinterpret_cast<const uint4 *>(p);
            acc[0] ^= v.x;
            acc[1] ^= v.y;
            acc[2] ^= v.z;
            acc[3] ^= v.w;
        } else {
            acc[0] ^= p[0];
        }
    };
    int32_t e0 = 0, e1 = 0;
    if (i < m) {
        e0 = row_ptr[i];
        e1 = row_ptr[i + 1];
    }
    if (e1 - e0 <= 32) {
#pragma unroll 4
        for (int32_t e = e0; e < e1; ++e) add(z, e);
    }
    // checks of degree above 32: the whole warp walks the check's edges and
    // xor-reduces across its lanes
    for (uint32_t wide = __ballot_sync(0xffffffffu, e1 - e0 > 32); wide; wide &= wide - 1) {
        const int src = __ffs(wide) - 1;
        const int32_t ws = __shfl_sync(0xffffffffu, e0, src), we = __shfl_sync(0xffffffffu, e1, src);
        uint32_t zz[W];
#pragma unroll
        for (int q = 0; q < W; ++q) zz[q] = 0u;
        for (int32_t e = ws + (int32_t)(threadIdx.x & 31); e < we; e += 32) add(zz, e);
#pragma unroll
        for (int q = 0; q < W; ++q) {
            zz[q] = __reduce_xor_sync(0xffffffffu, zz[q]);
            if ((int)(threadIdx.x & 31) == src) z[q] ^= zz[q];
        }
    }
#pragma unroll
    for (int q = 0; q < W; ++q) {
        const uint32_t u = __reduce_or_sync(0xffffffffu, z[q]);
        if ((threadIdx.x & 31) == 0 && u) atomicOr(row + w0 + q, u);
    }
}

// Per-frame iteration count and syndrome status, written by the finalize
// kernels' first CTA column (or by k_frame_results for a code without
// variables).
struct FrameResults {
    const uint32_t *done;
    const uint32_t *status;
    const int32_t *stop_iter;
    const uint32_t *final_unsat;
    int32_t F, max_iter;
    int32_t *iters;
    uint8_t *ok;
    const int32_t *slot_frame;  // frame held by each slot (-1: none); null: slot f holds frame f
};

__device__ __forceinline__ int32_t frame_of_slot(const int32_t *slot_frame, int32_t s) {
    return slot_frame ? slot_frame[s] : s;
}

// results of the frame in slot s (per-slot state, written at its frame index)
__device__ __forceinline__ void write_frame_result(const FrameResults &fr, int32_t s) {
    if (s >= fr.F) return;
    const int32_t f = frame_of_slot(fr.slot_frame, s);
    if (f < 0) return;
    if (*fr.status != 0u) {  // a device wait of the call gave up: no result
        fr.iters[f] = -1;
        fr.ok[f] = 0;
        return;
    }
    const bool stopped = frame_bit(fr.done, s);
    fr.iters[f] = stopped ? fr.stop_iter[s] : fr.max_iter;
    fr.ok[f] = stopped ? 1 : (frame_bit(fr.final_unsat, s) ? 0 : 1);
}

// APP [n][Fp] -> bits [F][n] (1 iff APP > 0, Algorithm 5) and optional post
// [F][n]. A CTA transposes a tile of 128 variables x 32 frames through shared
// memory and writes each frame's 128 decisions as 32 four-byte words (128
// posteriors as float4) when rows are 4-aligned, else byte by byte.
constexpr int kFinVars = 128;
constexpr int kFinStride = kFinVars + 4;  // float4-aligned rows

__global__ void __launch_bounds__(256) k_finalize(const float *__restrict__ app, uint8_t *__restrict__ bits,
                                                  float *__restrict__ post, int32_t n, int32_t F, int32_t Fp,
                                                  FrameResults fr) {
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x < 32) write_frame_result(fr, (int32_t)blockIdx.y * 32 + threadIdx.x);
    __shared__ __align__(16) float tile[32][kFinStride];
    const int32_t j0 = blockIdx.x * kFinVars;
    const int32_t f0 = blockIdx.y * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // all 16 row loads of a warp in flight before the first shared store
    float v[kFinVars / 8];
#pragma unroll
    for (int r = 0; r < kFinVars / 8; ++r) {
        const int32_t j = j0 + warp + 8 * r;
        v[r] = j < n ? app[(size_t)j * Fp + f0 + lane] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < kFinVars / 8; ++r) tile[lane][warp + 8 * r] = v[r];
    __syncthreads();
    const bool vec = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(bits) & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(post) & 15) == 0;
    for (int wi = threadIdx.x; wi < 32 * (kFinVars / 4); wi += blockDim.x) {
        const int fi = wi / (kFinVars / 4), q = wi % (kFinVars / 4);
        const int32_t s = f0 + fi, j = j0 + 4 * q;
        if (s >= F || j >= n) continue;
        const int32_t f = frame_of_slot(fr.slot_frame, s);
        if (f < 0) continue;
        const float4 x = *reinterpret_cast<const float4 *>(&tile[fi][4 * q]);
        const size_t o = (size_t)f * n + j;
        if (vec) {
            const uint32_t word = (x.x > 0.0f ? 1u : 0u) | (x.y > 0.0f ? 1u : 0u) << 8 |
                                  (x.z > 0.0f ? 1u : 0u) << 16 | (x.w > 0.0f ? 1u : 0u) << 24;
            *reinterpret_cast<uint32_t *>(bits + o) = word;
            if (post) *reinterpret_cast<float4 *>(post + o) = x;
        } else {
            const float xs[4] = {x.x, x.y, x.z, x.w};
            for (int b = 0; b < 4 && j + b < n; ++b) {
                bits[o + b] = xs[b] > 0.0f ? 1 : 0;
                if (post) post[o + b] = xs[b];
            }
        }
    }
}

// Fixed-iteration decodes without posteriors: bits [F][n] from the decision
// words dec [n][Fp/32] of the last bit pass (bit f % 32 of word f / 32 of row
// j is APP_j > 0 for frame f, written for every frame when no frame retires
// early): 2 MB of words read instead of the 66 MB APP array at n = 64800 and
// 256 frames. A CTA covers 128 variables of one 32-frame word.
__global__ void __launch_bounds__(256) k_finalize_words(const uint32_t *__restrict__ dec, uint8_t *__restrict__ bits,
                                                        int32_t n, int32_t F, int32_t G, FrameResults fr) {
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x < 32) write_frame_result(fr, (int32_t)blockIdx.y * 32 + threadIdx.x);
    __shared__ __align__(16) uint32_t wt[kFinVars];
    const int32_t j0 = blockIdx.x * kFinVars;
    const int32_t g = blockIdx.y;
    for (int t = threadIdx.x; t < kFinVars; t += blockDim.x) {
        const int32_t j = j0 + t;
        wt[t] = j < n ? dec[(size_t)j * G + g] : 0u;
    }
    __syncthreads();
    const bool vec = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(bits) & 3) == 0;
    for (int wi = threadIdx.x; wi < 32 * (kFinVars / 4); wi += blockDim.x) {
        const int fi = wi / (kFinVars / 4), q = wi % (kFinVars / 4);
        const int32_t f = g * 32 + fi, j = j0 + 4 * q;
        if (f >= F || j >= n) continue;
        const uint4 x = reinterpret_cast<const uint4 *>(wt)[q];
        const uint32_t b0 = (x.x >> fi) & 1u, b1 = (x.y >> fi) & 1u, b2 = (x.z >> fi) & 1u, b3 = (x.w >> fi) & 1u;
        const size_t o = (size_t)f * n + j;
        if (vec) {
            *reinterpret_cast<uint32_t *>(bits + o) = b0 | b1 << 8 | b2 << 16 | b3 << 24;
        } else {
            const uint32_t bs[4] = {b0, b1, b2, b3};
            for (int k = 0; k < 4 && j + k < n; ++k) bits[o + k] = (uint8_t)bs[k];
        }
    }
}

__global__ void k_frame_results(FrameResults fr) {
    pdl_wait();
    write_frame_result(fr, (int32_t)(blockIdx.x * blockDim.x + threadIdx.x));
}

// ---------------------------------------------------------------------------
// Early-exit compaction. A warp works on 32 V consecutive frame slots and
// returns at once only when all of them have stopped, so a batch whose
// frames stop at scattered iterations keeps most groups alive. Between two
// passes, the live frames still held in slots [L, Fp) (L = live frames) are
// moved into the slots [0, L) that hold stopped frames, after those stopped
// frames' results have been written out; the trailing groups then hold no
// live frame. Every step is a kernel on the decode's stream (no host
// decision), and a compaction that would not free a group moves nothing.
// ---------------------------------------------------------------------------

constexpr int kPlanThreads = 1024;  // one thread per 32-slot word: Fp <= 32768

// moves[0] = (M, L); moves[1 + i] = (source, destination) slot of move i.
// `always`: pack the live frames to the front even when no group is freed.
// `narrow` (> 0): also pack when at most `narrow` frames live and one of them
// sits at or beyond slot `narrow`, so that a narrow tail finds them all below.
// `release` (continuous decoding): stopped slots, whose results have been
// written out, give up their frame (slot_frame = -1).
__global__ void __launch_bounds__(kPlanThreads) k_compact_plan(const uint32_t *__restrict__ done, int32_t Fp,
                                                               int32_t group, int2 *__restrict__ moves, int32_t always,
                                                               int32_t narrow, int32_t *__restrict__ release) {
    pdl_wait();
    __shared__ int32_t s_a[kPlanThreads], s_b[kPlanThreads];
    const int t = threadIdx.x;
    const int W = Fp / 32;
    const uint32_t live = t < W ? ~done[t] : 0u;
    if (release && t < W)
        for (uint32_t x = ~live; x; x &= x - 1) release[t * 32 + __ffs(x) - 1] = -1;
    // inclusive scan of the live counts
    s_a[t] = __popc(live);
    __syncthreads();
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        const int v = t >= o ? s_a[t - o] : 0;
        __syncthreads();
        s_a[t] += v;
        __syncthreads();
    }
    const int32_t L = s_a[kPlanThreads - 1];
    // groups with a live frame now, and after packing
    const int wpg = group / 32;
    s_b[t] = (t < W && t % wpg == 0) ? 0 : 0;
    __syncthreads();
    if (t < W && live) atomicOr(&s_b[t / wpg], 1);
    __syncthreads();
    int32_t busy = 0;
    for (int g = 0; g < (W + wpg - 1) / wpg; ++g) busy += s_b[g];
    const int32_t after = (L + group - 1) / group;
    const bool spread = __syncthreads_or(narrow > 0 && L <= narrow && t < W && t * 32 >= narrow && live != 0u);
    if (after >= busy && !always && !spread) {
        if (t == 0) moves[0] = make_int2(0, L);
        return;
    }
    // holes: stopped slots below L; movers: live slots at or above L
    const int32_t base = t * 32;
    uint32_t below = 0u;  // bit b set when slot base + b < L
    if (t < W) below = L >= base + 32 ? 0xFFFFFFFFu : (L <= base ? 0u : ((1u << (L - base)) - 1u));
    const uint32_t holes = t < W ? ~live & below : 0u;
    const uint32_t movers = t < W ? live & ~below : 0u;
    s_a[t] = __popc(holes);
    s_b[t] = __popc(movers);
    __syncthreads();
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        const int va = t >= o ? s_a[t - o] : 0, vb = t >= o ? s_b[t - o] : 0;
        __syncthreads();
        s_a[t] += va;
        s_b[t] += vb;
        __syncthreads();
    }
    int32_t h = s_a[t] - __popc(holes), m = s_b[t] - __popc(movers);  // exclusive offsets
    for (uint32_t x = holes; x; x &= x - 1) moves[1 + h++].y = base + __ffs(x) - 1;
    for (uint32_t x = movers; x; x &= x - 1) moves[1 + m++].x = base + __ffs(x) - 1;
    if (t == kPlanThreads - 1) moves[0] = make_int2(s_a[t], L);
}

// Results of the stopped frames in the destination slots (about to be
// reused): 128 variables x 32 moves per CTA, as k_finalize.
__global__ void __launch_bounds__(256) k_compact_emit(const float *__restrict__ app, const int2 *__restrict__ moves,
                                                      uint8_t *__restrict__ bits, float *__restrict__ post,
                                                      int32_t n, int32_t Fp, FrameResults fr) {
    pdl_wait();
    const int32_t M = moves[0].x;
    const int32_t i0 = blockIdx.y * 32;
    if (i0 >= M) return;
    __shared__ __align__(16) float tile[32][kFinStride];
    __shared__ int32_t s_slot[32], s_frame[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 32) {
        const int32_t s = i0 + lane < M ? moves[1 + i0 + lane].y : -1;
        s_slot[lane] = s;
        s_frame[lane] = s >= 0 ? fr.slot_frame[s] : -1;
        if (blockIdx.x == 0 && s >= 0) write_frame_result(fr, s);
    }
    __syncthreads();
    const int32_t j0 = blockIdx.x * kFinVars;
    for (int r = warp; r < kFinVars; r += 8) {
        const int32_t j = j0 + r;
        const int32_t s = s_slot[lane];
        tile[lane][r] = (j < n && s >= 0) ? app[(size_t)j * Fp + s] : 0.0f;
    }
    __syncthreads();
    for (int wi = threadIdx.x; wi < 32 * kFinVars; wi += blockDim.x) {
        const int fi = wi / kFinVars, q = wi % kFinVars;
        const int32_t f = s_frame[fi], j = j0 + q;
        if (f < 0 || j >= n) continue;
        const float x = tile[fi][q];
        bits[(size_t)f * n + j] = x > 0.0f ? 1 : 0;
        if (post) post[(size_t)f * n + j] = x;
    }
}

// Move the columns (LLRs, posteriors, messages) of every (source, destination)
// pair: a warp per row; then the slots' frame map and stop bits.
template <typename M>
__global__ void __launch_bounds__(256) k_compact_move(float *__restrict__ lamT, float *__restrict__ app, M *r,
                                                      int32_t n, int64_t E, int32_t Fp, const int2 *__restrict__ moves,
                                                      int32_t *__restrict__ slot_frame, uint32_t *__restrict__ done,
                                                      int32_t *__restrict__ base) {
    pdl_wait();
    const int32_t Mv = moves[0].x;
    if (Mv == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t rows = 2 * (int64_t)n + E;
    for (int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); row < rows; row += (int64_t)gridDim.x * 8) {
        if (row < 2 * (int64_t)n) {
            float *p = (row < n ? lamT : app) + (size_t)(row < n ? row : row - n) * Fp;
            for (int i = lane; i < Mv; i += 32) {
                const int2 mv = moves[1 + i];
                p[mv.y] = p[mv.x];
            }
        } else {
            M *p = r + (size_t)(row - 2 * (int64_t)n) * Fp;
            for (int i = lane; i < Mv; i += 32) {
                const int2 mv = moves[1 + i];
                p[mv.y] = p[mv.x];
            }
        }
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < Mv; i += blockDim.x) {
            const int2 mv = moves[1 + i];
            slot_frame[mv.y] = slot_frame[mv.x];
            slot_frame[mv.x] = -1;
            if (base) base[mv.y] = base[mv.x];
            atomicAnd(done + (mv.y >> 5), ~(1u << (mv.y & 31)));
            atomicOr(done + (mv.x >> 5), 1u << (mv.x & 31));
        }
    }
}

// The compaction of a continuous decode's frame set (the decode server's
// slots): stopped slots release their frame, and the live frames are packed
// to the front; moves[0] = (moves, live frames) afterwards.
template <typename M>
static cudaError_t launch_pack(const PassArgs &a, int32_t group, int32_t *slot_frame, int2 *moves, cudaStream_t s) {
    cudaError_t e = launch_pdl(k_compact_plan, dim3(1), dim3(kPlanThreads), 0, s, a.done, a.Fp, group, moves, 1,
                               0, slot_frame);
    if (e == cudaSuccess)
        e = launch_pdl(k_compact_move<M>, dim3((unsigned)std::max(1, a.sm_count) * 8), dim3(256), 0, s,
                       const_cast<float *>(a.lamT), a.app, reinterpret_cast<M *>(a.r), a.n, a.E, a.Fp,
                       static_cast<const int2 *>(moves), slot_frame, a.done, const_cast<int32_t *>(a.base));
    return e;
}

cudaError_t launch_continuous_pack(const PassArgs &a, int msg_dtype, int32_t group, int32_t *slot_frame, int2 *moves,
                                   cudaStream_t s) {
    return with_msg_type(msg_dtype, [&](auto tag) {
        using M = typename decltype(tag)::type;
        return launch_pack<M>(a, group, slot_frame, moves, s);
    });
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

static int msg_size(int dtype) { return msg_bytes(dtype); }

// Frames per lane V and padded frame count Fp (a multiple of 32 V).
// `want` = 0 picks by batch size: four frames per lane (the widest rows,
// best for the bandwidth-bound bit kernel) once the padding stays small.
void frames_layout(int32_t F, int32_t want, int32_t *V, int32_t *Fp) {
    int32_t v = want;
    if (v != 1 && v != 2 && v != 4 && v != 8) v = F > 64 ? 4 : (F > 32 ? 2 : 1);
    *V = v;
    *Fp = (F + 32 * v - 1) / (32 * v) * (32 * v);
}

template <typename T>
static cudaError_t grow(T **p, size_t count) {
    cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(p, sizeof(T) * std::max<size_t>(count, 1));
}

// Device buffers for Fp frames and max_iter iterations of a code with n
// variables and E edges (grown, never shrunk).
static int ensure_workspace_dims(Workspace &w, int32_t n, int64_t E, int32_t Fp, int32_t max_iter, int msg_bytes) {
    bool need_frames = Fp > w.fp_cap || msg_bytes > w.msg_bytes;
    bool need_iters = need_frames || max_iter > w.iter_cap;
    if (!need_frames && !need_iters) return LDPC_OK;
    cudaError_t e = cudaEventSynchronize(w.last_use);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: waiting for the previous decode");
    if (need_frames) {
        int32_t cap = std::max(Fp, w.fp_cap);
        int mb = std::max(msg_bytes, w.msg_bytes);
        if ((e = grow(&w.lamT, (size_t)n * cap)) != cudaSuccess ||
            (e = grow(&w.app, (size_t)n * cap)) != cudaSuccess ||
            (e = grow(reinterpret_cast<char **>(&w.r), (size_t)E * cap * mb)) != cudaSuccess ||
            (e = grow(&w.done, (size_t)cap / 32 + 1)) != cudaSuccess ||
            (e = grow(&w.stop_iter, (size_t)cap)) != cudaSuccess ||
            (e = grow(&w.slot_frame, (size_t)cap)) != cudaSuccess ||
            (e = grow(&w.moves, (size_t)cap + 1)) != cudaSuccess ||
            (e = grow(&w.dec, (size_t)n * cap / 32)) != cudaSuccess) {
            w.fp_cap = 0;
            w.iter_cap = -1;
            return cuda_error(e, "ldpc_decode: workspace allocation");
        }
        // padding frames read finite posteriors
        if ((e = cudaMemset(w.app, 0, sizeof(float) * std::max<size_t>((size_t)n * cap, 1))) != cudaSuccess)
            return cuda_error(e, "ldpc_decode: workspace init");
        w.fp_cap = cap;
        w.generation += 1;
        w.msg_bytes = mb;
    }
    int32_t icap = std::max(max_iter, w.iter_cap);
    if ((e = grow(&w.unsat, (size_t)(icap + 1) * (w.fp_cap / 32))) != cudaSuccess) {
        w.iter_cap = -1;
        return cuda_error(e, "ldpc_decode: workspace allocation");
    }
    w.iter_cap = icap;
    w.generation += 1;
    return LDPC_OK;
}

static int ensure_workspace(ldpc_code *c, Workspace &w, int32_t Fp, int32_t max_iter, int msg_bytes) {
    return ensure_workspace_dims(w, c->n, c->E, Fp, max_iter, msg_bytes);
}

static cudaEvent_t take_event(ldpc_code *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// The two library streams (non-blocking) and their fork/phase/join events.
static cudaError_t ensure_half_streams(Workspace &w) {
    cudaError_t e = cudaSuccess;
    for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
        if (!w.half_stream[h]) e = cudaStreamCreateWithFlags(&w.half_stream[h], cudaStreamNonBlocking);
        if (e == cudaSuccess && !w.join[h]) e = cudaEventCreateWithFlags(&w.join[h], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !w.fork) e = cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !w.phase) e = cudaEventCreateWithFlags(&w.phase, cudaEventDisableTiming);
    return e;
}

// The side streams (non-blocking) of the two pass streams and their events.
static cudaError_t ensure_side_streams(Workspace &w) {
    cudaError_t e = cudaSuccess;
    for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
        if (!w.side_stream[h]) e = cudaStreamCreateWithFlags(&w.side_stream[h], cudaStreamNonBlocking);
        if (e == cudaSuccess && !w.side_fork[h]) e = cudaEventCreateWithFlags(&w.side_fork[h], cudaEventDisableTiming);
        if (e == cudaSuccess && !w.side_join[h]) e = cudaEventCreateWithFlags(&w.side_join[h], cudaEventDisableTiming);
    }
    return e;
}

// Launch wrapper: optional CUDA-event timing of each launch on the stream.
struct Launcher {
    ldpc_code *c;
    cudaStream_t s;
    bool profile;
    template <typename F>
    cudaError_t operator()(int kind, int n_kernels, F &&fn) {
        c->kernels_launched += n_kernels;
        cudaEvent_t a = nullptr, b = nullptr;
        if (profile) {
            a = take_event(c);
            b = take_event(c);
            cudaEventRecord(a, s);
        }
        cudaError_t e = fn();
        if (profile) {
            cudaEventRecord(b, s);
            c->prof.push_back(ProfRecord{kind, a, b});
        }
        return e;
    }
};

PassArgs make_pass_args(const ldpc_code *c, const ldpc_decode_opts_t &o, float l_max, int32_t F, int32_t V,
                        int32_t Fp, float *lamT, float *app, void *r, uint32_t *done, uint32_t *status,
                        uint32_t *unsat, int32_t *stop_iter) {
    PassArgs a{};
    a.row_ptr = c->d.row_ptr;
    a.col_idx = c->d.col_idx;
    a.col_ptr = c->d.col_ptr;
    a.edge_slot = c->d.edge_slot;
    a.phi_table = c->d.phi_table;
    a.lamT = lamT;
    a.app = app;
    a.r = r;
    a.m = c->m;
    a.n = c->n;
    a.E = c->E;
    a.Fp = Fp;
    a.V = V;
    a.n_frames = F;
    a.early_exit = o.early_exit ? 1 : 0;
    a.l_max = l_max;
    a.phi_lmax = (float)std::log1p(2.0 / std::expm1((double)l_max));
    a.r_max = (float)std::exp((double)l_max);
    a.done = done;
    a.status = status;
    a.unsat = unsat;
    a.stop_iter = stop_iter;
    a.grid_ctas = std::max(1, c->sm_count) * 4;
    a.sm_count = std::max(1, c->sm_count);
    a.check_schedule = o.check_schedule;
    a.f_begin = 0;
    a.f_count = Fp;
    a.check_rule = o.check_rule;
    a.ms_alpha = o.rule_alpha > 0.0f ? o.rule_alpha : 1.0f;
    a.ms_beta = o.rule_beta;
    a.ms_table = o.check_rule == LDPC_RULE_MIN_SUM_ADAPTIVE ? c->d.ms_table : nullptr;
    a.giveup_cta = -1;
    a.gate = nullptr;
    a.gate_narrow = 0;
    a.base = nullptr;
    a.max_iter = 0;
    a.unsat_ring = 0;
    a.wide_vars = c->d.wide_vars;
    a.n_wide_vars = (int32_t)c->wide_vars.size();
    a.bit_wide_ctas = 0;
    return a;
}

template <typename M>
static cudaError_t run_chunk(ldpc_code *c, Workspace &w, const float *llr, int32_t F, int32_t max_iter,
                             const ldpc_decode_opts_t &o, float l_max, uint8_t *bits, int32_t *iters, uint8_t *ok,
                             float *post, float *r_out, cudaStream_t s) {
    NvtxRange nvtx_decode("ldpc decode");
    int32_t V, Fp;
    frames_layout(F, o.frames_per_lane, &V, &Fp);
    // the status word follows the frame bits
    PassArgs a = make_pass_args(c, o, l_max, F, V, Fp, w.lamT, w.app, w.r, w.done, w.done + w.fp_cap / 32, w.unsat,
                                w.stop_iter);

    // profile 2 times only the pass region, so that consecutive kernels keep
    // their programmatic launch; other nonzero values time every launch too
    const bool per_kernel = o.profile != 0 && o.profile != 2;
    Launcher L{c, s, per_kernel};
    // Early-exit decodes of two or more frame groups compact their live frames
    // at a few pass boundaries (not with the message export, which reads the
    // messages by slot).
    const int32_t group = 32 * V;
    const bool compact = a.early_exit && max_iter >= 6 && Fp >= 2 * group && !r_out && c->n > 0;
    cudaError_t e;
    const int words = Fp / 32;
    e = L(LDPC_K_OTHER, 1, [&] {
        const int64_t n_unsat = (int64_t)(max_iter + 1) * words;
        const int64_t blocks = std::min<int64_t>(std::max<int64_t>(words, n_unsat) / 128 + 1, 1024);
        k_init_done<<<(unsigned)blocks, 128, 0, s>>>(w.done, a.status, w.unsat, n_unsat, F, Fp,
                                                     compact ? w.slot_frame : nullptr);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    if (c->n > 0) {
        e = L(LDPC_K_INTERLEAVE, 1, [&] {
            dim3 grid((unsigned)((c->n + 127) / 128), (unsigned)(Fp / 32), 1);
            return launch_pdl(k_interleave, grid, dim3(256), 0, s, llr, w.lamT, c->n, F, Fp);
        });
        if (e != cudaSuccess) return e;
    }
    // The passes: on `s`, or split over the two library streams, each running
    // one half of the frame range, the second starting when the first has
    // finished its first check pass, so the (arithmetic-bound) check pass of
    // one half overlaps the (bandwidth-bound) bit pass of the other.
    cudaEvent_t region_start = nullptr;
    if (o.profile) {
        region_start = take_event(c);
        cudaEventRecord(region_start, s);
    }
    // Tiles: frame ranges that run all their passes back to back. By default
    // there is one tile per stream; smaller tiles keep one tile's working set
    // (messages, posteriors, LLRs) within L2 while it iterates. With two
    // streams, consecutive tiles alternate between them and the second stream
    // starts when the first has finished its first check pass.
    // By default a batch splits when each half still fills the GPU: at least
    // 256 frames and n * Fp >= 2^20 (n = 4096 at 256 frames; shorter codes'
    // passes are launch- and latency-bound, and one stream is faster there:
    // n = 576 / 1152 / 2304 at 256 frames 0.099 / 0.095 / 0.143 ms on two
    // streams, 0.093 / 0.085 / 0.132 ms on one). An odd number of frame
    // groups splits unevenly (192 frames at two per lane: 128 + 64).
    const int32_t unit = 32 * std::max(V, 2);
    const bool split = o.streams != 1 && Fp >= 2 * unit &&
                       (o.streams == 2 || (Fp >= 256 && (int64_t)c->n * Fp >= (int64_t)1 << 20));
    int32_t tile = o.tile_frames > 0 ? (o.tile_frames + unit - 1) / unit * unit : 0;
    if (tile <= 0 || tile >= Fp || Fp % tile != 0) tile = split ? (Fp / 2 + unit - 1) / unit * unit : Fp;
    const int32_t ntiles = (Fp + tile - 1) / tile;  // the last tile may be shorter
    const int nstreams = split && ntiles >= 2 ? 2 : 1;
    cudaStream_t hs[2] = {s, s};
    if (nstreams == 2) {
        if ((e = ensure_half_streams(w)) != cudaSuccess) return e;
        hs[0] = w.half_stream[0];
        hs[1] = w.half_stream[1];
        if ((e = cudaEventRecord(w.fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(hs[0], w.fork, 0)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(hs[1], w.fork, 0)) != cudaSuccess) return e;
    }
    // test hook: one CTA of the first later check pass gives up its wait
    const int32_t giveup = c->debug_giveup_cta;
    c->debug_giveup_cta = -1;
    // Segments of passes; between two segments the streams join and the
    // compaction kernels run on `s`.
    static constexpr int32_t kCuts[] = {6, 10, 15, 21, 25, 28, 32, 36, 44, 48, 60, 80};
    // Narrow tail (four frames per lane, two 128-frame halves or more): from
    // the segment after pass kNarrowFrom on, stream 0 launches every pass in
    // two forms, its 128-frame groups and one 64-frame group at two frames
    // per lane, and the device runs the second once the last compaction left
    // at most 64 live frames (then all in slots [0, 64); the other groups
    // return at once). One pass of 64 frames costs about half the 128-frame
    // pass that the last few frames of a batch would otherwise keep running.
    static constexpr int32_t kNarrowFrom = 15;
    const bool narrow = compact && V == 4 && nstreams == 2 && ntiles == 2 && Fp % 256 == 0;
    // Checks of degree above 32 (a CTA per check; a code has few of them)
    // run on a side stream of each pass stream, beside the kernel of the
    // other checks, which would otherwise wait for them.
    const int32_t wide_bin = kNumCheckBins - 1;
    const bool side = c->bin_off[wide_bin + 1] > c->bin_off[wide_bin] && c->bin_off[wide_bin] > 0;
    if (side && (e = ensure_side_streams(w)) != cudaSuccess) return e;
    std::vector<int32_t> bounds{0};
    if (compact)
        for (int32_t t : kCuts)
            if (t <= max_iter) bounds.push_back(t);
    bounds.push_back(max_iter + 1);
    for (size_t sg = 0; sg + 1 < bounds.size(); ++sg) {
        const int32_t t0 = bounds[sg], t1 = bounds[sg + 1];
        if (sg > 0 && nstreams == 2) {  // fork again after a compaction
            if ((e = cudaEventRecord(w.fork, s)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(hs[0], w.fork, 0)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(hs[1], w.fork, 0)) != cudaSuccess) return e;
        }
        for (int32_t ti = 0; ti < ntiles; ++ti) {
            const int h = ti % nstreams;
            PassArgs at = a;
            at.f_begin = ti * tile;
            at.f_count = std::min(tile, Fp - ti * tile);
            // the narrow form of stream 0's passes in this segment
            const bool two_forms = narrow && ti == 0 && t0 >= kNarrowFrom;
            PassArgs an = at;
            if (two_forms) {
                at.gate = an.gate = w.moves;
                an.gate_narrow = 1;
                an.V = 2;
                an.f_begin = 0;
                an.f_count = kNarrowFrames;
            }
            Launcher Lh{c, hs[h], per_kernel};
            for (int32_t t = t0; t < t1; ++t) {
                NvtxRange nvtx_pass(ti == 0 ? "ldpc pass (first half)" : "ldpc pass (second half)");
                at.pass = an.pass = t;
                at.syndrome = an.syndrome = (t > 0 && at.early_exit) ? 1 : 0;
                at.dec = an.dec = t == max_iter ? w.dec : nullptr;
                at.giveup_cta = (t == 1 && ti == 0) ? giveup : -1;
                for (int form = 0; form < (two_forms ? 2 : 1); ++form) {
                    PassArgs &ap = form == 0 ? at : an;
                    if (side) {
                        const cudaStream_t ss = w.side_stream[h];
                        if ((e = cudaEventRecord(w.side_fork[h], hs[h])) != cudaSuccess) return e;
                        if ((e = cudaStreamWaitEvent(ss, w.side_fork[h], 0)) != cudaSuccess) return e;
                        PassArgs aw = ap;
                        aw.bin_degree = c->bin_max_degree[wide_bin];
                        Launcher Ls{c, ss, per_kernel};
                        e = Ls(LDPC_K_CHECK, 1, [&] {
                            return launch_check_bin<M>(aw, wide_bin, c->d.bin_checks + c->bin_off[wide_bin],
                                                       c->d.bin_desc + c->bin_off[wide_bin],
                                                       c->bin_off[wide_bin + 1] - c->bin_off[wide_bin], ss);
                        });
                        if (e != cudaSuccess) return e;
                        if ((e = cudaEventRecord(w.side_join[h], ss)) != cudaSuccess) return e;
                    }
                    for (int b = 0; b < kNumCheckBins; ++b) {
                        int32_t count = c->bin_off[b + 1] - c->bin_off[b];
                        if (count == 0 || (side && b == wide_bin)) continue;
                        ap.bin_degree = c->bin_max_degree[b];
                        e = Lh(LDPC_K_CHECK, 1, [&] {
                            return launch_check_bin<M>(ap, b, c->d.bin_checks + c->bin_off[b],
                                                       c->d.bin_desc + c->bin_off[b], count, hs[h]);
                        });
                        if (e != cudaSuccess) return e;
                    }
                    if (side && (e = cudaStreamWaitEvent(hs[h], w.side_join[h], 0)) != cudaSuccess) return e;
                }
                if (nstreams == 2 && ti == 0 && t == t0) {
                    if ((e = cudaEventRecord(w.phase, hs[0])) != cudaSuccess) return e;
                    if ((e = cudaStreamWaitEvent(hs[1], w.phase, 0)) != cudaSuccess) return e;
                }
                if (c->n > 0) {
                    for (int form = 0; form < (two_forms ? 2 : 1); ++form) {
                        const PassArgs &ap = form == 0 ? at : an;
                        e = Lh(LDPC_K_BIT, 1, [&] { return launch_bit<M>(ap, hs[h]); });
                        if (e != cudaSuccess) return e;
                    }
                }
            }
        }
        if (nstreams == 2) {
            for (int h = 0; h < 2; ++h) {
                if ((e = cudaEventRecord(w.join[h], hs[h])) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(s, w.join[h], 0)) != cudaSuccess) return e;
            }
        }
        if (sg + 2 < bounds.size()) {
            NvtxRange nvtx_compact("ldpc compaction");
            e = L(LDPC_K_OTHER, 3, [&] {
                cudaError_t ee = launch_pdl(k_compact_plan, dim3(1), dim3(kPlanThreads), 0, s, w.done, Fp, group,
                                            w.moves, 0, narrow ? kNarrowFrames : 0, static_cast<int32_t *>(nullptr));
                const FrameResults fr{w.done, a.status, w.stop_iter, nullptr, F, max_iter, iters, ok, w.slot_frame};
                if (ee == cudaSuccess)
                    ee = launch_pdl(k_compact_emit, dim3((unsigned)((c->n + kFinVars - 1) / kFinVars),
                                                         (unsigned)((Fp + 63) / 64)),
                                    dim3(256), 0, s, w.app, w.moves, bits, post, c->n, Fp, fr);
                if (ee == cudaSuccess)
                    ee = launch_pdl(k_compact_move<M>, dim3((unsigned)std::max(1, c->sm_count) * 8), dim3(256), 0, s,
                                    w.lamT, w.app, reinterpret_cast<M *>(w.r), c->n, c->E, Fp,
                                    static_cast<const int2 *>(w.moves), w.slot_frame, w.done,
                                    static_cast<int32_t *>(nullptr));
                return ee;
            });
            if (e != cudaSuccess) return e;
        }
    }
    if (o.profile) {
        cudaEvent_t region_stop = take_event(c);
        cudaEventRecord(region_stop, s);
        c->prof.push_back(ProfRecord{LDPC_K_PASSES, region_start, region_stop});
    }
    uint32_t *final_row = w.unsat + (size_t)max_iter * words;
    if (c->m > 0 && c->E > 0) {
        e = L(LDPC_K_SYNDROME, 1, [&] {
            if (words % 4 == 0)
                return launch_pdl(k_syndrome_words<4>, dim3((unsigned)((c->m + 255) / 256), (unsigned)(words / 4)),
                                  dim3(256), 0, s, c->d.row_ptr, c->d.col_idx, c->m, w.dec, words, final_row);
            return launch_pdl(k_syndrome_words<1>, dim3((unsigned)((c->m + 255) / 256), (unsigned)words), dim3(256),
                              0, s, c->d.row_ptr, c->d.col_idx, c->m, w.dec, words, final_row);
        });
        if (e != cudaSuccess) return e;
    }
    e = L(LDPC_K_FINALIZE, 1, [&] {
        const FrameResults fr{w.done, a.status, w.stop_iter, final_row, F, max_iter, iters, ok,
                              compact ? w.slot_frame : nullptr};
        if (c->n > 0) {
            dim3 grid((unsigned)((c->n + kFinVars - 1) / kFinVars), (unsigned)((F + 31) / 32), 1);
            return !a.early_exit && !post
                       ? launch_pdl(k_finalize_words, grid, dim3(256), 0, s, w.dec, bits, c->n, F, Fp / 32, fr)
                       : launch_pdl(k_finalize, grid, dim3(256), 0, s, w.app, bits, post, c->n, F, Fp, fr);
        }
        return launch_pdl(k_frame_results, dim3((unsigned)((F + 255) / 256)), dim3(256), 0, s, fr);
    });
    if (e != cudaSuccess) return e;
    if (r_out) {
        e = L(LDPC_K_OTHER, 1, [&] { return launch_export_r<M>(a, r_out, s); });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static int check_decode_args(const ldpc_code *c, int32_t F, int32_t max_iter, const ldpc_decode_opts_t &o,
                             float *l_max_out, const char *fn) {
    if (!c) return set_error(LDPC_EINVAL, "%s: code is NULL", fn);
    if (c->device < 0) return set_error(LDPC_ENODEV, "%s: the code was created without device tables", fn);
    if (F < 0) return set_error(LDPC_EINVAL, "%s: n_frames=%d < 0", fn, F);
    if (max_iter < 0 || max_iter > 100000) return set_error(LDPC_EINVAL, "%s: max_iter=%d outside [0, 100000]", fn, max_iter);
    float l_max = o.l_max > 0.0f ? o.l_max : 20.0f;
    if (!(l_max <= 80.0f)) return set_error(LDPC_EINVAL, "%s: l_max=%g outside (0, 80]", fn, (double)o.l_max);
    if (o.check_schedule < 0 || o.check_schedule > 2)
        return set_error(LDPC_EINVAL, "%s: check_schedule=%d not in {0, 1, 2}", fn, o.check_schedule);
    if (o.frames_per_lane != 0 && o.frames_per_lane != 1 && o.frames_per_lane != 2 && o.frames_per_lane != 4 &&
        o.frames_per_lane != 8)
        return set_error(LDPC_EINVAL, "%s: frames_per_lane=%d not in {0, 1, 2, 4, 8}", fn, o.frames_per_lane);
    if (o.streams < 0 || o.streams > 2) return set_error(LDPC_EINVAL, "%s: streams=%d not in {0, 1, 2}", fn, o.streams);
    if (o.tile_frames < 0) return set_error(LDPC_EINVAL, "%s: tile_frames=%d < 0", fn, o.tile_frames);
    if (o.check_rule != LDPC_RULE_SUM_PRODUCT && o.check_rule != LDPC_RULE_MIN_SUM &&
        o.check_rule != LDPC_RULE_SP_TABLE && o.check_rule != LDPC_RULE_MIN_SUM_ADAPTIVE)
        return set_error(LDPC_EINVAL, "%s: unknown check_rule %d", fn, o.check_rule);
    if (o.check_rule == LDPC_RULE_MIN_SUM_ADAPTIVE && !c->ms_table_set)
        return set_error(LDPC_EINVAL, "%s: the adaptive min-sum rule needs ldpc_code_set_rule_table first", fn);
    if (o.check_rule == LDPC_RULE_SP_TABLE && !(l_max <= kPhiTableMaxLmax))
        return set_error(LDPC_EINVAL, "%s: the tabulated rule needs l_max <= 22 (got %g)", fn, (double)l_max);
    if (!(o.rule_beta >= 0.0f) || !std::isfinite(o.rule_alpha))
        return set_error(LDPC_EINVAL, "%s: rule_beta must be >= 0 and rule_alpha finite", fn);
    if (!msg_dtype_valid(o.msg_dtype)) return set_error(LDPC_EINVAL, "%s: unknown msg_dtype %d", fn, o.msg_dtype);
    *l_max_out = l_max;
    return LDPC_OK;
}

static ldpc_decode_opts_t default_opts() {
    ldpc_decode_opts_t o;
    memset(&o, 0, sizeof(o));
    o.early_exit = 1;
    o.l_max = 20.0f;
    o.msg_dtype = LDPC_MSG_F32;
    return o;
}

// Decode with the code's lock held.
// Enqueue the chunks of one decode on `s` (no synchronisation, no
// allocation: capturable).
static cudaError_t enqueue_chunks(ldpc_code *c, const float *llr, int32_t F, int32_t chunk, int32_t max_iter,
                                  const ldpc_decode_opts_t &o, float l_max, uint8_t *bits, int32_t *iters, uint8_t *ok,
                                  float *post, cudaStream_t s) {
    for (int32_t f0 = 0; f0 < F; f0 += chunk) {
        int32_t fc = std::min(chunk, F - f0);
        const float *l = llr + (size_t)f0 * c->n;
        uint8_t *bb = bits + (size_t)f0 * c->n;
        float *pp = post ? post + (size_t)f0 * c->n : nullptr;
        float *rr = o.r_out ? o.r_out + (size_t)f0 * c->E : nullptr;
        cudaError_t e = with_msg_type(o.msg_dtype, [&](auto tag) {
            using M = typename decltype(tag)::type;
            return run_chunk<M>(c, c->ws, l, fc, max_iter, o, l_max, bb, iters + f0, ok + f0, pp, rr, s);
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Graph replay. A decode whose shape, options and buffers repeat the
// previous call's is captured into a CUDA graph on a library stream (so any
// caller stream works, the legacy default stream included) and replayed by
// later calls with the same key: one launch instead of ~4 per pass, which
// is what small codes are bound by. A key is captured the second time it is
// seen among the last four; up to kGraphCache graphs per code; a workspace
// reallocation changes the key.
constexpr size_t kGraphCache = 4;

static int decode_graph(ldpc_code *c, const GraphKey &key, int32_t chunk, cudaStream_t s, bool *done) {
    *done = false;
    for (auto &g : c->graphs) {
        if (g.key == key) {
            cudaError_t e = cudaGraphLaunch(g.exec, s);
            if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: graph launch");
            g.used = ++c->graph_tick;
            c->kernels_launched += g.kernels;
            *done = true;
            return LDPC_OK;
        }
    }
    bool seen = false;
    for (int i = 0; i < c->n_seen; ++i) seen |= c->seen_keys[i] == key;
    if (!seen) {  // first sighting: run directly, remember the key
        c->seen_keys[c->next_seen] = key;
        c->next_seen = (c->next_seen + 1) % 4;
        c->n_seen = std::min(c->n_seen + 1, 4);
        return LDPC_OK;
    }
    cudaError_t e = cudaSuccess;
    if (!c->capture_stream) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = ensure_half_streams(c->ws);
    if (e == cudaSuccess) e = ensure_side_streams(c->ws);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: graph set-up");
    cudaStream_t cap = c->capture_stream;
    const int64_t k0 = c->kernels_launched;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: begin capture");
    cudaError_t ee = enqueue_chunks(c, key.llr, key.F, chunk, key.max_iter, key.o, key.l_max, key.bits, key.iters,
                                    key.ok, key.post, cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    const int64_t kernels = c->kernels_launched - k0;
    c->kernels_launched = k0;
    if (ee != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return LDPC_OK;  // not capturable here: the caller runs it directly
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LDPC_OK;
    }
    if (c->graphs.size() >= kGraphCache) {
        auto lru = std::min_element(c->graphs.begin(), c->graphs.end(),
                                    [](const DecodeGraph &x, const DecodeGraph &y) { return x.used < y.used; });
        cudaGraphExecDestroy(lru->exec);
        c->graphs.erase(lru);
    }
    c->graphs.push_back(DecodeGraph{key, exec, kernels, ++c->graph_tick});
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: graph launch");
    c->kernels_launched += kernels;
    *done = true;
    return LDPC_OK;
}

static int decode_locked(ldpc_code *c, const float *llr, int32_t F, int32_t max_iter, const ldpc_decode_opts_t &o,
                         float l_max, uint8_t *bits, int32_t *iters, uint8_t *ok, float *post, cudaStream_t s) {
    int32_t chunk = std::min(F, kMaxChunkFrames);
    int32_t V, Fp;
    frames_layout(chunk, o.frames_per_lane, &V, &Fp);
    int st = ensure_workspace(c, c->ws, Fp, max_iter, msg_size(o.msg_dtype));
    if (st != LDPC_OK) return st;
    cudaError_t e = cudaStreamWaitEvent(s, c->ws.last_use, 0);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: cudaStreamWaitEvent");
    bool done = false;
    if (!o.profile && c->debug_giveup_cta < 0) {
        GraphKey key;
        key.llr = llr;
        key.bits = bits;
        key.iters = iters;
        key.ok = ok;
        key.post = post;
        key.r_out = o.r_out;
        key.F = F;
        key.max_iter = max_iter;
        key.l_max = l_max;
        key.o = o;
        key.ws_generation = c->ws.generation;
        st = decode_graph(c, key, chunk, s, &done);
        if (st != LDPC_OK) return st;
    }
    if (!done) {
        e = enqueue_chunks(c, llr, F, chunk, max_iter, o, l_max, bits, iters, ok, post, s);
        if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: kernel launch");
    }
    e = cudaEventRecord(c->ws.last_use, s);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_decode: cudaEventRecord");
    return LDPC_OK;
}

}  // namespace ldpc

using namespace ldpc;

extern "C" int ldpc_decode(ldpc_code_t *c, const float *llr, int32_t F, int32_t max_iter,
                           const ldpc_decode_opts_t *opts, uint8_t *bits, int32_t *iters, uint8_t *ok, float *post,
                           void *stream) {
    ldpc_decode_opts_t o = opts ? *opts : default_opts();
    float l_max = 20.0f;
    int st = check_decode_args(c, F, max_iter, o, &l_max, "ldpc_decode");
    if (st != LDPC_OK) return st;
    if (F == 0) return LDPC_OK;
    if ((c->n > 0 && (!llr || !bits)) || !iters || !ok)
        return set_error(LDPC_EINVAL, "ldpc_decode: NULL llr, bits, iters or syndrome_ok");
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceGuard guard(c->device);
    return decode_locked(c, llr, F, max_iter, o, l_max, bits, iters, ok, post, (cudaStream_t)stream);
}

extern "C" int ldpc_decode_host(ldpc_code_t *c, const float *llr_host, int32_t F, int32_t max_iter,
                                const ldpc_decode_opts_t *opts, uint8_t *bits_host, int32_t *iters_host,
                                uint8_t *ok_host, float *post_host, void *stream) {
    ldpc_decode_opts_t o = opts ? *opts : default_opts();
    float l_max = 20.0f;
    int st = check_decode_args(c, F, max_iter, o, &l_max, "ldpc_decode_host");
    if (st != LDPC_OK) return st;
    if (o.r_out) return set_error(LDPC_EINVAL, "ldpc_decode_host: r_out must be NULL");
    if (F == 0) return LDPC_OK;
    if ((c->n > 0 && (!llr_host || !bits_host)) || !iters_host || !ok_host)
        return set_error(LDPC_EINVAL, "ldpc_decode_host: NULL llr, bits, iters or syndrome_ok");
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceGuard guard(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    Workspace &w = c->ws;
    cudaError_t e;
    if (F > w.host_cap) {
        if ((e = cudaEventSynchronize(w.last_use)) != cudaSuccess) return cuda_error(e, "ldpc_decode_host: wait");
        if ((e = grow(&w.h_llr, (size_t)F * c->n)) != cudaSuccess || (e = grow(&w.h_bits, (size_t)F * c->n)) != cudaSuccess ||
            (e = grow(&w.h_iters, (size_t)F)) != cudaSuccess || (e = grow(&w.h_ok, (size_t)F)) != cudaSuccess ||
            (e = grow(&w.h_post, (size_t)F * c->n)) != cudaSuccess) {
            w.host_cap = 0;
            return cuda_error(e, "ldpc_decode_host: staging allocation");
        }
        w.host_cap = F;
    }
    if ((e = cudaStreamWaitEvent(s, w.last_use, 0)) != cudaSuccess) return cuda_error(e, "ldpc_decode_host: wait");
    // A large batch runs as two parts, its copies on a copy stream: the
    // second part's LLRs arrive while the first decodes, and the first part's
    // results leave while the second decodes (a frame's result does not
    // depend on the frames decoded with it).
    const int32_t part = (F / 2 + 127) / 128 * 128;
    const bool pipe = F >= 256 && part < F && (int64_t)c->n * F >= ((int64_t)1 << 22);
    if (pipe && !w.copy_stream) {
        e = cudaStreamCreateWithFlags(&w.copy_stream, cudaStreamNonBlocking);
        for (auto &ev : w.copy_ev)
            if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_error(e, "ldpc_decode_host: copy stream");
    }
    const int32_t np = pipe ? 2 : 1;
    const int32_t f0s[2] = {0, pipe ? part : F}, fns[2] = {pipe ? part : F, pipe ? F - part : 0};
    const cudaStream_t cs = pipe ? w.copy_stream : s;
    if (pipe && ((e = cudaEventRecord(w.copy_ev[0], s)) != cudaSuccess ||
                 (e = cudaStreamWaitEvent(cs, w.copy_ev[0], 0)) != cudaSuccess))
        return cuda_error(e, "ldpc_decode_host: fork");
    for (int32_t p = 0; p < np; ++p) {  // copies in
        const size_t off = (size_t)f0s[p] * c->n, cnt = (size_t)fns[p] * c->n;
        if (cnt && (e = cudaMemcpyAsync(w.h_llr + off, llr_host + off, sizeof(float) * cnt, cudaMemcpyHostToDevice,
                                        cs)) != cudaSuccess)
            return cuda_error(e, "ldpc_decode_host: copy in");
        if (pipe && (e = cudaEventRecord(w.copy_ev[1 + p], cs)) != cudaSuccess)
            return cuda_error(e, "ldpc_decode_host: record");
    }
    for (int32_t p = 0; p < np; ++p) {  // decodes
        const size_t off = (size_t)f0s[p] * c->n;
        if (pipe && (e = cudaStreamWaitEvent(s, w.copy_ev[1 + p], 0)) != cudaSuccess)
            return cuda_error(e, "ldpc_decode_host: wait");
        st = decode_locked(c, w.h_llr + off, fns[p], max_iter, o, l_max, w.h_bits + off, w.h_iters + f0s[p],
                           w.h_ok + f0s[p], post_host ? w.h_post + off : nullptr, s);
        if (st != LDPC_OK) return st;
        if (pipe && (e = cudaEventRecord(w.copy_ev[3 + p], s)) != cudaSuccess)
            return cuda_error(e, "ldpc_decode_host: record");
    }
    for (int32_t p = 0; p < np; ++p) {  // copies out
        const size_t off = (size_t)f0s[p] * c->n, cnt = (size_t)fns[p] * c->n;
        const int32_t f0 = f0s[p], fn = fns[p];
        if (pipe && (e = cudaStreamWaitEvent(cs, w.copy_ev[3 + p], 0)) != cudaSuccess)
            return cuda_error(e, "ldpc_decode_host: wait");
        if ((cnt && (e = cudaMemcpyAsync(bits_host + off, w.h_bits + off, cnt, cudaMemcpyDeviceToHost, cs)) !=
                        cudaSuccess) ||
            (e = cudaMemcpyAsync(iters_host + f0, w.h_iters + f0, sizeof(int32_t) * fn, cudaMemcpyDeviceToHost, cs)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(ok_host + f0, w.h_ok + f0, fn, cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
            (post_host && cnt &&
             (e = cudaMemcpyAsync(post_host + off, w.h_post + off, sizeof(float) * cnt, cudaMemcpyDeviceToHost, cs)) !=
                 cudaSuccess))
            return cuda_error(e, "ldpc_decode_host: copy out");
    }
    if (pipe && ((e = cudaEventRecord(w.copy_ev[5], cs)) != cudaSuccess ||
                 (e = cudaStreamWaitEvent(s, w.copy_ev[5], 0)) != cudaSuccess))
        return cuda_error(e, "ldpc_decode_host: join");
    if ((e = cudaEventRecord(w.last_use, s)) != cudaSuccess) return cuda_error(e, "ldpc_decode_host: record");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "ldpc_decode_host: synchronize");
    return report_gave_up(iters_host, F, "ldpc_decode_host");
}

namespace ldpc {
int report_gave_up(const int32_t *iters_host, int32_t F, const char *fn) {
    for (int32_t f = 0; f < F; ++f)
        if (iters_host[f] < 0)
            return set_error(LDPC_ETIMEOUT, "%s: a bounded device wait of the decode ran out; no results", fn);
    return LDPC_OK;
}
}  // namespace ldpc

extern "C" int ldpc_debug_giveup(ldpc_code_t *c, int32_t cta) {
    if (!c) return set_error(LDPC_EINVAL, "ldpc_debug_giveup: code is NULL");
    if (cta < -1) return set_error(LDPC_EINVAL, "ldpc_debug_giveup: cta=%d < -1", cta);
    std::lock_guard<std::mutex> lock(c->mu);
    c->debug_giveup_cta = cta;
    return LDPC_OK;
}

extern "C" int ldpc_prof_read(ldpc_code_t *c, ldpc_prof_t *out, int32_t reset) {
    if (!c || !out) return set_error(LDPC_EINVAL, "ldpc_prof_read: NULL argument");
    std::lock_guard<std::mutex> lock(c->mu);
    if (c->device < 0) return LDPC_OK;
    DeviceGuard guard(c->device);
    for (auto &p : c->prof) {
        cudaError_t e = cudaEventSynchronize(p.stop);
        if (e != cudaSuccess) return cuda_error(e, "ldpc_prof_read: event");
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, p.start, p.stop);
        if (e != cudaSuccess) return cuda_error(e, "ldpc_prof_read: elapsed");
        if (p.kind >= 0 && p.kind < LDPC_K_COUNT) {
            out->launches[p.kind] += 1;
            out->total_ms[p.kind] += ms;
        }
    }
    out->kernels += c->kernels_launched;
    if (reset) {
        c->kernels_launched = 0;
        for (auto &p : c->prof) {
            c->event_pool.push_back(p.start);
            c->event_pool.push_back(p.stop);
        }
        c->prof.clear();
    }
    return LDPC_OK;
}

// ---------------------------------------------------------------------------
// Mixed-code batches: the decodes of several codes (each with its own frame
// count) as parallel branches of one CUDA graph, launched once per batch.
// ---------------------------------------------------------------------------

namespace ldpc {

bool GraphKey::operator==(const GraphKey &b) const {
    return llr == b.llr && bits == b.bits && iters == b.iters && ok == b.ok && post == b.post && r_out == b.r_out &&
           F == b.F && max_iter == b.max_iter && l_max == b.l_max && ws_generation == b.ws_generation &&
           o.early_exit == b.o.early_exit && o.l_max == b.o.l_max && o.msg_dtype == b.o.msg_dtype &&
           o.profile == b.o.profile && o.r_out == b.o.r_out && o.frames_per_lane == b.o.frames_per_lane &&
           o.check_schedule == b.o.check_schedule && o.streams == b.o.streams && o.tile_frames == b.o.tile_frames &&
           o.check_rule == b.o.check_rule && o.rule_alpha == b.o.rule_alpha && o.rule_beta == b.o.rule_beta;
}

void free_decode_graphs(ldpc_code *c) {
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
    c->n_seen = 0;
    c->next_seen = 0;
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->capture_stream = nullptr;
}

void free_workspace(Workspace &w) {
    if (w.last_use) cudaEventSynchronize(w.last_use);
    cudaFree(w.lamT);
    cudaFree(w.app);
    cudaFree(w.r);
    cudaFree(w.done);
    cudaFree(w.unsat);
    cudaFree(w.stop_iter);
    cudaFree(w.slot_frame);
    cudaFree(w.moves);
    cudaFree(w.dec);
    cudaFree(w.h_llr);
    cudaFree(w.h_bits);
    cudaFree(w.h_iters);
    cudaFree(w.h_ok);
    cudaFree(w.h_post);
    if (w.last_use) cudaEventDestroy(w.last_use);
    if (w.copy_stream) cudaStreamDestroy(w.copy_stream);
    for (auto ev : w.copy_ev)
        if (ev) cudaEventDestroy(ev);
    for (int h = 0; h < 2; ++h) {
        if (w.half_stream[h]) cudaStreamDestroy(w.half_stream[h]);
        if (w.join[h]) cudaEventDestroy(w.join[h]);
        if (w.side_stream[h]) cudaStreamDestroy(w.side_stream[h]);
        if (w.side_fork[h]) cudaEventDestroy(w.side_fork[h]);
        if (w.side_join[h]) cudaEventDestroy(w.side_join[h]);
    }
    if (w.fork) cudaEventDestroy(w.fork);
    if (w.phase) cudaEventDestroy(w.phase);
    w = Workspace{};
}

struct BatchItem {
    ldpc_code *code = nullptr;
    int32_t F = 0;
    ldpc_decode_opts_t opts{};
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

static cudaError_t enqueue_item(BatchItem &it, int32_t max_iter, float l_max, const float *llr, uint8_t *bits,
                                int32_t *iters, uint8_t *ok, float *post, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(it.code->mu);
    return with_msg_type(it.opts.msg_dtype, [&](auto tag) {
        using M = typename decltype(tag)::type;
        return run_chunk<M>(it.code, it.ws, llr, it.F, max_iter, it.opts, l_max, bits, iters, ok, post, nullptr, s);
    });
}

}  // namespace ldpc

struct ldpc_batch {
    int device = 0;
    int32_t max_iter = 0;
    float l_max = 20.0f;
    std::vector<ldpc::BatchItem> items;
    cudaStream_t capture = nullptr;
    cudaEvent_t fork = nullptr;
    cudaEvent_t last_run = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool warmed = false;
    std::vector<const void *> key;  // the pointers the graph was captured with
    int64_t kernels_per_run = 0;
    std::mutex mu;
};

static void batch_free(ldpc_batch *b) {
    DeviceGuard guard(b->device);
    if (b->last_run) cudaEventSynchronize(b->last_run);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &it : b->items) {
        free_workspace(it.ws);
        if (it.stream) cudaStreamDestroy(it.stream);
        if (it.done) cudaEventDestroy(it.done);
    }
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->last_run) cudaEventDestroy(b->last_run);
    delete b;
}

extern "C" int ldpc_batch_create(int32_t n_items, ldpc_code_t *const *codes, const int32_t *n_frames, int32_t max_iter,
                                 const ldpc_decode_opts_t *opts, ldpc_batch_t **out) {
    if (!out) return set_error(LDPC_EINVAL, "ldpc_batch_create: out is NULL");
    *out = nullptr;
    if (n_items <= 0 || !codes || !n_frames) return set_error(LDPC_EINVAL, "ldpc_batch_create: empty batch");
    ldpc_decode_opts_t o = opts ? *opts : default_opts();
    float l_max = 20.0f;
    for (int32_t i = 0; i < n_items; ++i) {
        int st = check_decode_args(codes[i], n_frames[i], max_iter, o, &l_max, "ldpc_batch_create");
        if (st != LDPC_OK) return st;
        if (n_frames[i] <= 0 || n_frames[i] > kMaxChunkFrames)
            return set_error(LDPC_EINVAL, "ldpc_batch_create: item %d has %d frames, outside [1, %d]", i, n_frames[i],
                             kMaxChunkFrames);
        if (codes[i]->device != codes[0]->device)
            return set_error(LDPC_EINVAL, "ldpc_batch_create: items on different devices");
    }
    if (o.profile || o.r_out) return set_error(LDPC_EINVAL, "ldpc_batch_create: profile and r_out are not available");
    ldpc_batch *b = new (std::nothrow) ldpc_batch();
    if (!b) return set_error(LDPC_ENOMEM, "ldpc_batch_create: out of host memory");
    b->device = codes[0]->device;
    b->max_iter = max_iter;
    b->l_max = l_max;
    DeviceGuard guard(b->device);
    cudaError_t e = cudaSuccess;
    b->items.resize(n_items);
    for (int32_t i = 0; i < n_items && e == cudaSuccess; ++i) {
        BatchItem &it = b->items[i];
        it.code = codes[i];
        it.F = n_frames[i];
        it.opts = o;
        it.opts.streams = 1;      // one branch per item; items overlap each other
        it.opts.tile_frames = 0;
        e = cudaStreamCreateWithFlags(&it.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&it.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&it.ws.last_use, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            // room for the widest frame layout the tuner may pick (8 frames per lane)
            int32_t Fp = (it.F + 255) / 256 * 256;
            int st = ensure_workspace(it.code, it.ws, Fp, max_iter, msg_size(o.msg_dtype));
            if (st != LDPC_OK) {
                batch_free(b);
                return st;
            }
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->last_run, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int st = cuda_error(e, "ldpc_batch_create");
        batch_free(b);
        return st;
    }
    *out = b;
    return LDPC_OK;
}

extern "C" void ldpc_batch_destroy(ldpc_batch_t *b) {
    if (b) batch_free(b);
}

// Enqueue every item on its own stream, forked from and joined into `s`.
static cudaError_t batch_enqueue(ldpc_batch *b, const float *const *llr, uint8_t *const *bits, int32_t *const *iters,
                                 uint8_t *const *ok, float *const *post, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (size_t i = 0; i < b->items.size() && e == cudaSuccess; ++i) {
        BatchItem &it = b->items[i];
        e = cudaStreamWaitEvent(it.stream, b->fork, 0);
        if (e == cudaSuccess)
            e = enqueue_item(it, b->max_iter, b->l_max, llr[i], bits[i], iters[i], ok[i], post ? post[i] : nullptr,
                             it.stream);
        if (e == cudaSuccess) e = cudaEventRecord(it.done, it.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, it.done, 0);
    }
    return e;
}

extern "C" int ldpc_batch_run(ldpc_batch_t *b, const float *const *llr, uint8_t *const *bits, int32_t *const *iters,
                              uint8_t *const *syndrome_ok, float *const *post_llr, void *stream) {
    if (!b || !llr || !bits || !iters || !syndrome_ok) return set_error(LDPC_EINVAL, "ldpc_batch_run: NULL argument");
    for (size_t i = 0; i < b->items.size(); ++i)
        if (!llr[i] || !bits[i] || !iters[i] || !syndrome_ok[i])
            return set_error(LDPC_EINVAL, "ldpc_batch_run: NULL buffer for item %zu", i);
    std::lock_guard<std::mutex> lock(b->mu);
    DeviceGuard guard(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamWaitEvent(s, b->last_run, 0);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_batch_run: wait");
    std::vector<const void *> key;
    for (size_t i = 0; i < b->items.size(); ++i) {
        key.push_back(llr[i]);
        key.push_back(bits[i]);
        key.push_back(iters[i]);
        key.push_back(syndrome_ok[i]);
        key.push_back(post_llr ? post_llr[i] : nullptr);
    }
    if (!b->warmed) {
        // first run: direct launches (also performs every kernel's one-time set-up)
        e = batch_enqueue(b, llr, bits, iters, syndrome_ok, post_llr, s);
        if (e != cudaSuccess) return cuda_error(e, "ldpc_batch_run: launch");
        b->warmed = true;
    } else {
        if (!b->exec || key != b->key) {
            int64_t before = 0, after = 0;
            for (auto &it : b->items) before += it.code->kernels_launched;
            e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) e = batch_enqueue(b, llr, bits, iters, syndrome_ok, post_llr, b->capture);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
            if (e == cudaSuccess) e = e2;
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_error(e, "ldpc_batch_run: graph capture");
            }
            for (auto &it : b->items) after += it.code->kernels_launched;
            b->kernels_per_run = after - before;
            if (b->exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(b->exec, g, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(b->exec);
                    b->exec = nullptr;
                }
            }
            if (!b->exec && (e = cudaGraphInstantiate(&b->exec, g, 0)) != cudaSuccess) {
                cudaGraphDestroy(g);
                return cuda_error(e, "ldpc_batch_run: graph instantiate");
            }
            if (b->graph) cudaGraphDestroy(b->graph);
            b->graph = g;
            b->key = key;
        }
        if ((e = cudaGraphLaunch(b->exec, s)) != cudaSuccess) return cuda_error(e, "ldpc_batch_run: graph launch");
    }
    if ((e = cudaEventRecord(b->last_run, s)) != cudaSuccess) return cuda_error(e, "ldpc_batch_run: record");
    return LDPC_OK;
}

extern "C" int ldpc_batch_tune(ldpc_batch_t *b, const float *const *llr, void *stream) {
    if (!b || !llr) return set_error(LDPC_EINVAL, "ldpc_batch_tune: NULL argument");
    std::lock_guard<std::mutex> lock(b->mu);
    DeviceGuard guard(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b->last_run);
    if (e != cudaSuccess) return cuda_error(e, "ldpc_batch_tune: synchronize");
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    int status = LDPC_OK;
    for (size_t i = 0; i < b->items.size() && status == LDPC_OK; ++i) {
        BatchItem &it = b->items[i];
        if (!llr[i]) {
            status = set_error(LDPC_EINVAL, "ldpc_batch_tune: NULL llr for item %zu", i);
            break;
        }
        uint8_t *bits = nullptr, *ok = nullptr;
        int32_t *iters = nullptr;
        if ((e = cudaMalloc(&bits, (size_t)it.F * it.code->n + 1)) != cudaSuccess ||
            (e = cudaMalloc(&ok, (size_t)it.F)) != cudaSuccess ||
            (e = cudaMalloc(&iters, sizeof(int32_t) * it.F)) != cudaSuccess) {
            status = cuda_error(e, "ldpc_batch_tune: scratch outputs");
        }
        float best = 1e30f;
        ldpc_decode_opts_t best_opts = it.opts;
        const int32_t lanes[4] = {1, 2, 4, 8};
        for (int li = 0; li < 4 && status == LDPC_OK; ++li) {
            int32_t v = lanes[li];
            int32_t Fp = (it.F + 32 * v - 1) / (32 * v) * (32 * v);
            if (v > 1 && Fp - it.F > it.F) continue;  // padding larger than the batch itself
            for (int32_t trial = 0; trial < 4 && status == LDPC_OK; ++trial) {
                const int32_t sched = 1 + trial % 2, nst = 1 + trial / 2;
                // two streams only for items that fill the GPU by themselves
                // (in the graph the items already overlap one another)
                if (nst == 2 && (Fp < 2 * 32 * std::max(v, 2) || (int64_t)it.code->n * Fp < ((int64_t)1 << 22)))
                    continue;
                it.opts.frames_per_lane = v;
                it.opts.check_schedule = sched;
                it.opts.streams = nst;
                float ms = 0.0f;
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                    if (rep == 1) e = cudaEventRecord(t0, it.stream);
                    if (e == cudaSuccess) e = enqueue_item(it, b->max_iter, b->l_max, llr[i], bits, iters, ok, nullptr,
                                                           it.stream);
                }
                if (e == cudaSuccess) e = cudaEventRecord(t1, it.stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) {
                    status = cuda_error(e, "ldpc_batch_tune: trial");
                    break;
                }
                if (ms < (nst == 2 ? 0.9f : 1.0f) * best) {  // a split must win clearly
                    best = ms;
                    best_opts = it.opts;
                }
            }
        }
        it.opts = best_opts;
        cudaFree(bits);
        cudaFree(ok);
        cudaFree(iters);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    b->warmed = true;   // every candidate kernel has run once
    if (b->exec) {      // schedules changed: capture again on the next run
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return status;
}

extern "C" int ldpc_batch_info(const ldpc_batch_t *b, int32_t item, int32_t *frames_per_lane, int32_t *check_schedule,
                               int32_t *streams, int64_t *kernels_per_run) {
    if (!b || item < 0 || item >= (int32_t)b->items.size()) return set_error(LDPC_EINVAL, "ldpc_batch_info: bad item");
    if (frames_per_lane) *frames_per_lane = b->items[item].opts.frames_per_lane;
    if (check_schedule) *check_schedule = b->items[item].opts.check_schedule;
    if (streams) *streams = b->items[item].opts.streams;
    if (kernels_per_run) *kernels_per_run = b->kernels_per_run;
    return LDPC_OK;
}

namespace ldpc {

// Entry points for the serving runtime (ldpc_server.cpp).
int workspace_reserve(Workspace &w, int32_t n, int64_t E, int32_t Fp, int32_t max_iter, int msg_bytes) {
    return ensure_workspace_dims(w, n, E, Fp, max_iter, msg_bytes);
}

cudaError_t enqueue_decode(ldpc_code *c, Workspace &w, const float *llr, int32_t F, int32_t max_iter,
                           const ldpc_decode_opts_t &o, float l_max, uint8_t *bits, int32_t *iters, uint8_t *ok,
                           float *post, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(c->mu);
    return with_msg_type(o.msg_dtype, [&](auto tag) {
        using M = typename decltype(tag)::type;
        return run_chunk<M>(c, w, llr, F, max_iter, o, l_max, bits, iters, ok, post, nullptr, s);
    });
}

int check_opts(const ldpc_code *c, int32_t F, int32_t max_iter, const ldpc_decode_opts_t &o, float *l_max,
               const char *fn) {
    return check_decode_args(c, F, max_iter, o, l_max, fn);
}

}  // namespace ldpc

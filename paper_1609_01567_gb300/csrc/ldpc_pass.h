// Declarations of the flooding-pass kernels: device data layout, the
// per-pass argument block and the kernel launchers.
//
// Device data layout (frame-interleaved, see the kernels for details):
//   r     [E][Fp]  check-to-bit messages, rows in check order (slot k = the
//                  k-th entry of ebar, Table 2), Fp frames per row
//   app   [n][Fp]  posterior LLR of every variable (Algorithm 4)
//   lamT  [n][Fp]  channel LLRs, interleaved copy of the caller's [F][n]
//   done  [Fp/32]  bit f set once frame f has stopped (or is padding)
//   unsat [P][Fp/32] bit f of row t set when the hard decision of pass t
//                  leaves an unsatisfied check (Algorithm 6)
// Fp is the frame count rounded up to a multiple of 32 (V = 1) or of 128
// (V = 4 frames per lane).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "ldpc.h"

namespace ldpc {

constexpr int kNumCheckBins = 6;
// Upper degree bound of each check bin: the first five keep a check's
// messages in registers (exclusive sums by prefix/suffix), the last one
// handles any degree with a compensated two-pass reduction.
constexpr int kBinMaxDegree[kNumCheckBins] = {4, 6, 8, 16, 32, INT32_MAX};
constexpr int kMaxRegisterDegree = 32;

constexpr int kThreads = 256;  // threads per CTA of the pass kernels (8 warps)
constexpr int32_t kNarrowFrames = 64;  // frames of an early-exit decode's narrow tail group
// checks of degree 17-32 in one code from which the wide-bin kernels (18-slot ring, staged
// product form, any-degree) serve them instead of the padded register kernel
constexpr int32_t kWideBinAnyKernel = 2048;

// int8 messages: uniform step 20/127, saturating at +-127 steps (= 20).
constexpr float kI8Step = 20.0f / 127.0f;
constexpr float kI8Inv = 127.0f / 20.0f;

// Bytes per stored message, and a call of f with the matching storage type.
inline int msg_bytes(int dtype) { return dtype == LDPC_MSG_F32 ? 4 : (dtype == LDPC_MSG_I8 ? 1 : 2); }
inline bool msg_dtype_valid(int dtype) {
    return dtype == LDPC_MSG_F32 || dtype == LDPC_MSG_F16 || dtype == LDPC_MSG_BF16 || dtype == LDPC_MSG_I8;
}
template <typename T>
struct TypeTag {
    using type = T;
};
template <typename F>
auto with_msg_type(int dtype, F &&f) {
    switch (dtype) {
    case LDPC_MSG_F16: return f(TypeTag<__half>{});
    case LDPC_MSG_BF16: return f(TypeTag<__nv_bfloat16>{});
    case LDPC_MSG_I8: return f(TypeTag<int8_t>{});
    default: return f(TypeTag<float>{});
    }
}

struct DeviceTables {
    int32_t *row_ptr = nullptr;    // [m+1] first slot of each check
    int32_t *col_idx = nullptr;    // [E]   variable of each check-order slot (vbar)
    int32_t *col_ptr = nullptr;    // [n+1] first edge of each variable (s)
    int32_t *edge_slot = nullptr;  // [E]   check-order slot of each edge id (inverse of ebar)
    int32_t *bin_checks = nullptr; // [m']  checks grouped by degree bin
    int2 *bin_desc = nullptr;      // [m']  (first slot, degree) of each binned check
    float2 *phi_table = nullptr;   // [kPhiTableSize] chords (a, b) of the tabulated phi
    float2 *ms_table = nullptr;    // [max check degree + 1] (alpha_d, beta_d) of the degree-adaptive min-sum
    int32_t *wide_vars = nullptr;  // variables of degree above kWideVarDegree (their own bit kernel)
};

// Per-frame flag bits: frame f is bit (f & 31) of word f >> 5.
__device__ __forceinline__ bool frame_bit(const uint32_t *words, int f) { return (words[f >> 5] >> (f & 31)) & 1u; }

// stop_iter of a frame of a continuous decode that used up its iterations
// with a nonzero syndrome (the low bits hold max_iter)
constexpr int32_t kStopFailed = 0x40000000;

// Variables of higher degree are summed by a CTA (trailing CTAs of the bit
// kernel's grid), its warps splitting the edges; the others by one warp each.
constexpr int kWideVarDegree = 16;

// Tabulated phi: bucket key = float bits >> 17 (64 buckets per octave) over
// [2^-32, 2^5); entry key - kPhiKey0 holds the chord a + b x of the bucket.
constexpr uint32_t kPhiKey0 = 95u << 6;
constexpr int kPhiTableSize = 37 * 64;
constexpr float kPhiTableMaxLmax = 22.0f;

// Arguments of one flooding pass, shared by the kernels of all bins.
struct PassArgs {
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const int32_t *col_ptr;
    const int32_t *edge_slot;
    const float *lamT;
    float *app;
    void *r;
    int32_t m, n;
    int64_t E;
    int32_t Fp;          // padded frames per row
    int32_t V;           // frames per lane (1 or 4)
    int32_t n_frames;    // real frames (< Fp frames are padding)
    int32_t pass;        // 0 = first check pass on q = lambda
    int32_t syndrome;    // check pass also tests the previous hard decision
    int32_t early_exit;
    float l_max;
    float phi_lmax;      // phi(l_max)
    float r_max;         // e^l_max: the largest (A + B) / D of the product form, |r| = l_max
    uint32_t *done;      // [Fp/32]
    uint32_t *dec;       // [n][Fp/32] hard-decision words, written by the last bit pass (else null)
    uint32_t *status;    // one word, nonzero once a device wait of the call gave up
    uint32_t *unsat;     // [max_iter + 1][Fp/32]
    int32_t *stop_iter;  // [Fp] iteration at which a frame stopped
    int32_t grid_ctas;   // CTAs per launch target (a multiple of the SM count)
    int32_t sm_count;
    int32_t check_schedule;  // 0 auto, 1 direct loads, 2 shared-memory pipeline
    int32_t f_begin;     // first frame of the range this launch covers (a multiple of 32 V)
    int32_t f_count;     // frames in that range (a multiple of 32 V)
    int32_t bin_degree;  // largest check degree present in the bin being launched
    int32_t check_rule;  // 0 sum-product, 1 min-sum family, 2 sum-product with tabulated phi,
                         // 3 min-sum with (alpha, beta) per check degree from ms_table
    const float2 *phi_table;  // device chords of the tabulated phi (rule 2)
    float ms_alpha;      // min-sum scale
    float ms_beta;       // min-sum offset
    const float2 *ms_table;   // degree-adaptive min-sum: (alpha, beta) indexed by check degree, else null
    // Continuous decoding (the decode server's slots): frames enter and leave a
    // running frame set. base[f] is the pass before frame f's own first pass,
    // so its own pass count at pass t is t - base[f]; it stops at its first
    // zero syndrome (early exit) or after max_iter of its own passes. The
    // syndrome rows are then a ring of two (unsat_ring != 0). Null base: every
    // frame starts at pass 0 of the call.
    const int32_t *base;
    int32_t max_iter;
    int32_t unsat_ring;
    const int32_t *wide_vars;  // variables of degree above kWideVarDegree
    int32_t n_wide_vars;
    int32_t bit_wide_ctas;     // bit kernel: its last CTAs sum the wide variables (set by its launcher)
    int32_t giveup_cta;  // test hook (ldpc_debug_giveup): this CTA of the launch treats its first
                         // completed bounded wait as run out; -1 = off
    // Early-exit tail: once a compaction has left at most kNarrowFrames live
    // frames (all in the first slots), they run as one group of two frames
    // per lane instead of a group of four. Both forms of a pass are launched
    // and the device picks one: with gate set, the kernel runs only when
    // (live frames <= kNarrowFrames) equals gate_narrow; gate->y holds the
    // live count the last compaction left. Null gate: always runs.
    const int2 *gate;
    int32_t gate_narrow;
    // Tensor maps of the pipelined check kernel, filled by its launcher: the
    // rows the check inputs are read from (lamT on the first pass, else app;
    // float, box {32 V frames, 1 row}, gathered four rows at a time) and the
    // message rows (r, box {32 V frames, D rows}: one check's rows).
    CUtensorMap tm_q;
    CUtensorMap tm_r;
};

// A pass kernel whose form the device did not pick for this pass returns at
// once (after its programmatic wait, so the compaction's count is visible).
__device__ __forceinline__ bool gated_off(const PassArgs &a) {
    if (a.gate == nullptr) return false;
    return (a.gate->y <= kNarrowFrames) != (a.gate_narrow != 0);
}

// A 2-D tensor map (TMA descriptor) over a row-major buffer of `rows` rows
// of `cols` elements (CUtensorMapDataType dtype), rows `row_bytes` apart,
// with a box of {box_cols, box_rows}; encoded on the host, cached per thread.
cudaError_t tensor_map_2d(CUtensorMap *out, int dtype, const void *base, uint64_t cols, uint64_t rows,
                          uint64_t row_bytes, uint32_t box_cols, uint32_t box_rows);

template <typename M>
cudaError_t launch_check_bin(const PassArgs &a, int bin, const int32_t *checks, const int2 *desc, int32_t count,
                             cudaStream_t s);
template <typename M>
cudaError_t launch_bit(const PassArgs &a, cudaStream_t s);
template <typename M>
cudaError_t launch_export_r(const PassArgs &a, float *r_out, cudaStream_t s);

}  // namespace ldpc

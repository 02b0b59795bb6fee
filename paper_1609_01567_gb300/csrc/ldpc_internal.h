// Internal declarations shared by the library's translation units.
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

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <mutex>
#include <string>
#include <vector>

#include "ldpc.h"

namespace ldpc {

constexpr int kNumCheckBins = 5;
// Upper degree bound of each check bin: the first four keep a check's
// messages in registers (exclusive sums by prefix/suffix), the last one
// handles any degree with a compensated two-pass reduction.
constexpr int kBinMaxDegree[kNumCheckBins] = {4, 8, 16, 32, INT32_MAX};
constexpr int kMaxRegisterDegree = 32;

constexpr int kThreads = 256;  // threads per CTA of the pass kernels (8 warps)

struct DeviceTables {
    int32_t *row_ptr = nullptr;    // [m+1] first slot of each check
    int32_t *col_idx = nullptr;    // [E]   variable of each check-order slot (vbar)
    int32_t *col_ptr = nullptr;    // [n+1] first edge of each variable (s)
    int32_t *edge_slot = nullptr;  // [E]   check-order slot of each edge id (inverse of ebar)
    int32_t *bin_checks = nullptr; // [m']  checks grouped by degree bin
    int2 *bin_desc = nullptr;      // [m']  (first slot, degree) of each binned check
};

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
    float c_min;         // 1 - tanh(l_max / 2): complement of the largest |r|
    float c_max;         // 1 - e^-l_max: complement of the smallest |r|
    uint32_t *done;      // [Fp/32]
    uint32_t *unsat;     // [max_iter + 1][Fp/32]
    int32_t *stop_iter;  // [Fp] iteration at which a frame stopped
    int32_t grid_ctas;   // CTAs per launch target (a multiple of the SM count)
    int32_t sm_count;
    int32_t check_schedule;  // 0 auto, 1 direct loads, 2 shared-memory pipeline
    int32_t f_begin;     // first frame of the range this launch covers (a multiple of 32 V)
    int32_t f_count;     // frames in that range (a multiple of 32 V)
    int32_t check_rule;  // 0 sum-product, 1 min-sum family
    float ms_alpha;      // min-sum scale
    float ms_beta;       // min-sum offset
};

template <typename M>
cudaError_t launch_check_bin(const PassArgs &a, int bin, const int32_t *checks, const int2 *desc, int32_t count,
                             cudaStream_t s);
template <typename M>
cudaError_t launch_bit(const PassArgs &a, cudaStream_t s);
template <typename M>
cudaError_t launch_export_r(const PassArgs &a, float *r_out, cudaStream_t s);

struct Workspace {
    int32_t fp_cap = 0;       // frames (padded) the buffers hold
    int32_t iter_cap = -1;    // max_iter the unsat rows hold
    int32_t msg_bytes = 0;    // bytes per stored message of the current buffer
    float *lamT = nullptr;
    float *app = nullptr;
    void *r = nullptr;
    uint32_t *done = nullptr;
    uint32_t *unsat = nullptr;
    int32_t *stop_iter = nullptr;
    // staging for ldpc_decode_host
    int32_t host_cap = 0;
    float *h_llr = nullptr;
    uint8_t *h_bits = nullptr;
    int32_t *h_iters = nullptr;
    uint8_t *h_ok = nullptr;
    float *h_post = nullptr;
    cudaEvent_t last_use = nullptr;  // end of the last decode that used the buffers
    // two library streams that run the two halves of a batch half a pass apart
    cudaStream_t half_stream[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, phase = nullptr, join[2] = {nullptr, nullptr};
};

struct ProfRecord {
    int kind;
    cudaEvent_t start, stop;
};

void free_workspace(Workspace &w);
int workspace_reserve(Workspace &w, int32_t n, int64_t E, int32_t Fp, int32_t max_iter, int msg_bytes);
cudaError_t enqueue_decode(ldpc_code *c, Workspace &w, const float *llr, int32_t F, int32_t max_iter,
                           const ldpc_decode_opts_t &o, float l_max, uint8_t *bits, int32_t *iters, uint8_t *ok,
                           float *post, cudaStream_t s);
int check_opts(const ldpc_code *c, int32_t F, int32_t max_iter, const ldpc_decode_opts_t &o, float *l_max,
               const char *fn);

// Thread-local error text.
int set_error(int status, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);

}  // namespace ldpc

struct ldpc_code {
    int32_t m = 0, n = 0;
    int64_t E = 0;
    int32_t max_cdeg = 0, max_vdeg = 0;
    // host tables
    std::vector<int32_t> var_of_edge;   // v  [E]
    std::vector<int32_t> chk_of_edge;   // c  [E]
    std::vector<int32_t> col_ptr;       // [n+1]
    std::vector<int32_t> row_ptr;       // [m+1]
    std::vector<int32_t> edge_of_slot;  // ebar [E]
    std::vector<int32_t> col_idx;       // vbar [E]
    std::vector<int32_t> edge_slot;     // [E]
    std::vector<int32_t> bin_checks;
    std::vector<int2> bin_desc;
    int32_t bin_off[ldpc::kNumCheckBins + 1] = {0};
    // device side
    int device = -1;
    int sm_count = 0;
    ldpc::DeviceTables d;
    ldpc::Workspace ws;
    std::mutex mu;
    std::vector<ldpc::ProfRecord> prof;
    std::vector<cudaEvent_t> event_pool;
    int64_t kernels_launched = 0;  // library kernels enqueued since the last profile reset
};

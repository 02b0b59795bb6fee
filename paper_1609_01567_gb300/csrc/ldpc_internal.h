// Internal declarations shared by the library's translation units: decode
// workspace, code handle, error helpers. The kernels' own declarations are in
// ldpc_pass.h.
#pragma once

#include <atomic>
#include <climits>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ldpc_pass.h"

namespace ldpc {

struct Workspace {
    uint64_t generation = 0;  // bumped whenever the buffers are (re)allocated
    int32_t fp_cap = 0;       // frames (padded) the buffers hold
    int32_t iter_cap = -1;    // max_iter the unsat rows hold
    int32_t msg_bytes = 0;    // bytes per stored message of the current buffer
    float *lamT = nullptr;
    float *app = nullptr;
    void *r = nullptr;
    uint32_t *done = nullptr;
    uint32_t *unsat = nullptr;
    uint32_t *dec = nullptr;  // [n][Fp/32] final hard-decision words
    int32_t *stop_iter = nullptr;
    // early-exit compaction: the frame each slot holds (-1: none), and the
    // (source, destination) slot pairs of a compaction with their count
    int32_t *slot_frame = nullptr;
    int2 *moves = nullptr;
    // staging for ldpc_decode_host
    int32_t host_cap = 0;
    float *h_llr = nullptr;
    uint8_t *h_bits = nullptr;
    int32_t *h_iters = nullptr;
    uint8_t *h_ok = nullptr;
    float *h_post = nullptr;
    cudaEvent_t last_use = nullptr;  // end of the last decode that used the buffers
    // ldpc_decode_host's copy stream and its events (start, two copies in, two
    // decodes, copies out done), for batches decoded as two halves
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // two library streams that run the two halves of a batch half a pass apart
    cudaStream_t half_stream[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, phase = nullptr, join[2] = {nullptr, nullptr};
    // a side stream per pass stream for the checks of degree above 32
    cudaStream_t side_stream[2] = {nullptr, nullptr};
    cudaEvent_t side_fork[2] = {nullptr, nullptr}, side_join[2] = {nullptr, nullptr};
};

struct ProfRecord {
    int kind;
    cudaEvent_t start, stop;
};

void free_workspace(Workspace &w);

// A captured decode: the call's shape, options and buffers, and its graph.
struct GraphKey {
    const float *llr = nullptr;
    uint8_t *bits = nullptr;
    int32_t *iters = nullptr;
    uint8_t *ok = nullptr;
    float *post = nullptr;
    float *r_out = nullptr;
    int32_t F = 0, max_iter = 0;
    float l_max = 0.0f;
    ldpc_decode_opts_t o{};
    uint64_t ws_generation = 0;
    bool operator==(const GraphKey &b) const;
};
struct DecodeGraph {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;  // library kernels in the graph
    uint64_t used = 0;    // last use (for eviction)
};
void free_decode_graphs(ldpc_code *c);
struct HostStream;
void free_host_stream(ldpc_code *c);
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
    int32_t ira_k = -1;  // k when columns k .. n-1 form the staircase (IRA form), else -1
    std::atomic<bool> ms_table_set{false};  // ldpc_code_set_rule_table has filled d.ms_table
    // host tables
    std::vector<int32_t> var_of_edge;   // v  [E]
    std::vector<int32_t> chk_of_edge;   // c  [E]
    std::vector<int32_t> col_ptr;       // [n+1]
    std::vector<int32_t> row_ptr;       // [m+1]
    std::vector<int32_t> edge_of_slot;  // ebar [E]
    std::vector<int32_t> col_idx;       // vbar [E]
    std::vector<int32_t> edge_slot;     // [E]
    std::vector<int32_t> bin_checks;
    std::vector<int32_t> wide_vars;     // variables of degree above kWideVarDegree
    std::vector<int2> bin_desc;
    int32_t bin_off[ldpc::kNumCheckBins + 1] = {0};
    int32_t bin_max_degree[ldpc::kNumCheckBins] = {0};  // largest check degree present in each bin
    // device side
    int device = -1;
    int sm_count = 0;
    ldpc::DeviceTables d;
    ldpc::Workspace ws;
    std::mutex mu;
    std::vector<ldpc::ProfRecord> prof;
    std::vector<cudaEvent_t> event_pool;
    int64_t kernels_launched = 0;  // library kernels enqueued since the last profile reset
    ldpc::HostStream *host_stream = nullptr;  // staging of ldpc_decode_host_stream
    // graph replay of repeated decodes (ldpc_decode, ldpc_decode_host)
    std::vector<ldpc::DecodeGraph> graphs;
    ldpc::GraphKey seen_keys[4];  // keys run once directly (captured when they recur)
    int n_seen = 0, next_seen = 0;
    uint64_t graph_tick = 0;
    cudaStream_t capture_stream = nullptr;
    int32_t debug_giveup_cta = -1;  // ldpc_debug_giveup: armed for the next decode, then cleared
    // systematic encoder of any code (ldpc_code_build_encoder): enc_k
    // information positions (-1: not built), enc_r = rank of H; on the device
    // the parity rows over the information bits, enc_R [enc_r][ceil(enc_k / 32)]
    // bit words, and enc_colmap [n] (information index j >= 0, or -1 - i for
    // the column set by parity row i)
    int32_t enc_k = -1, enc_r = 0;
    uint32_t *enc_R = nullptr;
    int32_t *enc_colmap = nullptr;
};

namespace ldpc {

// An NVTX range over a scope of host code (a decode call, one pass, a
// compaction): a profiler that reads NVTX (ncu --nvtx, nsys) groups the
// kernels each range launches under its name; without one attached the
// calls cost a few nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Frames per lane V (1, 2, 4 or 8) and padded frame count Fp (a multiple of
// 32 V) of a decode of F frames; `want` = 0 picks by batch size.
void frames_layout(int32_t F, int32_t want, int32_t *V, int32_t *Fp);

// The argument block of every pass of one decode (code tables, options,
// layout and the decode's buffers), shared by all decode entry points so that
// none of them leaves a field unset. status is the call's device-wait word.
// Compaction of a continuous decode's frame set (see ldpc_decode.cu):
// stopped slots release their frame (slot_frame = -1), live frames are packed
// to the front; moves[0] = (moves, live frames) afterwards.
cudaError_t launch_continuous_pack(const PassArgs &a, int msg_dtype, int32_t group, int32_t *slot_frame, int2 *moves,
                                   cudaStream_t s);

// LDPC_ETIMEOUT (with its message) when a frame of a finished host-side
// decode reports iters = -1 (a bounded device wait gave up), else LDPC_OK.
int report_gave_up(const int32_t *iters_host, int32_t F, const char *fn);

PassArgs make_pass_args(const ldpc_code *c, const ldpc_decode_opts_t &o, float l_max, int32_t F, int32_t V,
                        int32_t Fp, float *lamT, float *app, void *r, uint32_t *done, uint32_t *status,
                        uint32_t *unsat, int32_t *stop_iter);

}  // namespace ldpc

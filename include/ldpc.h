/*
 * ldpc.h -- C ABI of the GB300 (sm_103a) sum-product LDPC decoder.
 *
 * The library decodes any irregular binary LDPC code, with no bound on node
 * degree, by the flooding sum-product (SP) algorithm of arXiv:1609.01567:
 * a check-node update, a bit-node update, a hard decision and a parallel
 * syndrome check per iteration, stopping a frame at its first zero syndrome
 * or after max_iter iterations (Algorithm 2). All compute runs in the
 * library's CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - LLRs are lambda = ln(P(bit = 1) / P(bit = 0)); a positive LLR favours
 *     bit 1. This is the reading of Algorithms 3 and 5, which store and
 *     decide on the probability of a one. Callers holding ln(P0/P1) negate.
 *   - A hard decision is 1 iff the posterior LLR is > 0 (a tie gives 0, as
 *     in Algorithm 5).
 *   - Edges are the nonzeros of H (Section II-B, Eqs. 1-2). Edge ids are the
 *     caller's COO entries stably sorted by column (the e array of Table 1);
 *     the check order of edges is the edge ids stably sorted by check (the
 *     ebar array of Table 2).
 *   - Device pointers must be in the device memory of the code's device and
 *     stay valid until the work enqueued on `stream` completes. `stream` is
 *     a cudaStream_t (NULL = legacy default stream).
 *   - Every function returns LDPC_OK (0) or a negative ldpc_status; the text
 *     of the last error of the calling thread is ldpc_last_error(). No C++
 *     exception crosses this ABI.
 *   - Argument errors are reported synchronously, before anything is
 *     enqueued. Work is asynchronous on `stream` unless a function says
 *     otherwise.
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LDPC_OK = 0,
    LDPC_EINVAL = -1,   /* bad argument (range, size, null pointer, wrong device) */
    LDPC_EDUP = -2,     /* repeated (row, column) in the COO of H               */
    LDPC_ENOMEM = -3,   /* host or device allocation failed                     */
    LDPC_ECUDA = -4,    /* a CUDA runtime call failed                           */
    LDPC_ETIMEOUT = -5, /* a bounded device wait ran out                        */
    LDPC_EBUSY = -6,    /* resource in use                                      */
    LDPC_ENODEV = -7    /* the code was created host-only (no device tables)    */
} ldpc_status;

typedef enum {
    LDPC_MSG_F32 = 0,   /* check-to-bit messages stored as float              */
    LDPC_MSG_F16 = 1,   /* stored as IEEE binary16, rounded to nearest (ties
                           to even, subnormals kept); node sums stay float  */
    LDPC_MSG_BF16 = 2,  /* stored as bfloat16, rounded to nearest (ties to
                           even); node sums stay in float                   */
    LDPC_MSG_I8 = 3     /* stored as int8 in steps of 20/127, saturating at
                           +-20 (L_MAX above 20 acts as 20 for the stored
                           messages); all node arithmetic stays in float    */
} ldpc_msg_dtype;

/* Opaque code handle: host tables plus their device copies. */
typedef struct ldpc_code ldpc_code_t;

typedef struct {
    int32_t device;     /* CUDA device ordinal for the tables; -1 = host only
                           (tables are built and can be read back with
                           ldpc_code_tables, but decoding returns LDPC_ENODEV) */
} ldpc_code_opts_t;

typedef struct {
    int32_t m;                   /* checks (rows of H)                       */
    int32_t n;                   /* variables / code bits (columns of H)     */
    int64_t n_edges;             /* E = nonzeros of H                        */
    int32_t max_check_degree;
    int32_t max_var_degree;
    double mean_check_degree;    /* E / m                                    */
    double mean_var_degree;      /* E / n                                    */
    int32_t n_check_bins;        /* degree bins used by the check kernels    */
    int32_t check_bin_max_degree[8]; /* upper degree bound of each bin; the
                                        last bin of an unbounded-degree code
                                        reports INT32_MAX                     */
    int32_t check_bin_count[8];  /* checks in each bin                       */
    int32_t device;              /* device of the tables, -1 for host only   */
    int32_t ira_k;               /* k = n - m when the last m columns of H are
                                    the dual-diagonal staircase of an IRA code
                                    (column k + i joins checks i and i + 1, the
                                    last column only check m - 1), so that
                                    ldpc_encode_ira applies; else -1          */
} ldpc_code_info_t;

/*
 * Build a code from the COO of its parity-check matrix H (m x n, nnz ones).
 * rows/cols: host arrays of nnz int32 indices; H[rows[t]][cols[t]] = 1.
 * The COO order defines edge ids (stable sort by column). Empty rows or
 * columns and degree-1 nodes are accepted.
 * Errors: LDPC_EINVAL for m, n or nnz out of range (m, n >= 0,
 * 0 <= nnz <= 2^31 - 1) or an index outside H; LDPC_EDUP when a (row,
 * column) pair repeats; LDPC_ENOMEM / LDPC_ECUDA on allocation or upload
 * failure. Synchronous: the device tables are uploaded before it returns.
 * The caller owns rows/cols; the library copies them. *out receives a handle
 * that the caller releases with ldpc_code_destroy.
 */
int ldpc_code_create(int32_t m, int32_t n, int64_t nnz, const int32_t *rows, const int32_t *cols,
                     const ldpc_code_opts_t *opts, ldpc_code_t **out);

/*
 * Build a quasi-cyclic code by lifting a base matrix (protograph) with
 * circulant permutations: the family of the paper's benchmark codes (the
 * CCSDS code and its protograph expansions, Section IV); the paper builds
 * such codes off-line and feeds the decoder their H. The lifted H has
 * mb * Z rows and nb * Z columns; base entry b puts the Z x Z circulant
 * P^shift[b] at block (brow[b], bcol[b]): row t of the block joins column
 * (t + shift[b]) mod Z. Several entries at one block with distinct shifts are
 * parallel protograph edges. Edge ids follow the COO order entry-major,
 * t-minor, stably sorted by column, as in ldpc_code_create.
 * Errors: LDPC_EINVAL for sizes out of range (Z >= 1; the lifted rows,
 * columns and edges each at most 2^31 - 1) or an entry outside the base
 * matrix or with shift outside [0, Z); LDPC_EDUP when an entry repeats with
 * the same shift; otherwise as ldpc_code_create. The caller owns the arrays.
 */
int ldpc_code_create_qc(int32_t mb, int32_t nb, int32_t Z, int64_t n_entries, const int32_t *brow,
                        const int32_t *bcol, const int32_t *shift, const ldpc_code_opts_t *opts, ldpc_code_t **out);

/* Release a code, its device tables and its decode workspace. Waits for
 * the code's pending work. NULL is ignored. */
void ldpc_code_destroy(ldpc_code_t *code);

/* Sizes and degree statistics of a code. */
int ldpc_code_info(const ldpc_code_t *code, ldpc_code_info_t *info);

/*
 * Read back the paper's address-iterator arrays (Section III-B, Tables 1-2),
 * each of n_edges int32 entries into caller-owned host buffers; any pointer
 * may be NULL to skip that array.
 *   variable-sorted (edge e):  v[e] variable, c[e] check, t[e] degree of v[e],
 *                              s[e] first edge of v[e], u[e] = e - s[e]
 *   check-sorted (slot k):     ebar[k] edge id, vbar[k], cbar[k] its variable
 *                              and check, tbar[k] degree of cbar[k],
 *                              sbar[k] first slot of cbar[k], ubar[k] = k - sbar[k]
 * Host-only; works for host-only codes.
 */
int ldpc_code_tables(const ldpc_code_t *code, int32_t *v, int32_t *c, int32_t *t, int32_t *s, int32_t *u,
                     int32_t *ebar, int32_t *vbar, int32_t *cbar, int32_t *tbar, int32_t *sbar, int32_t *ubar);

typedef struct {
    int32_t early_exit; /* nonzero: a frame stops at its first zero syndrome
                           (Algorithm 2); zero: every frame runs all max_iter
                           iterations and reports the final syndrome        */
    float l_max;        /* saturation L_MAX of the check rule, > 0; values
                           <= 0 select the default 20. Check inputs and outputs
                           are clamped to [phi(L_MAX), L_MAX] in magnitude    */
    int32_t msg_dtype;  /* ldpc_msg_dtype of the stored check-to-bit messages */
    int32_t profile;    /* nonzero: time the decode with CUDA events on
                           `stream` (read with ldpc_prof_read) and run it
                           directly, never from a captured graph; 2 times
                           only the region of the flooding passes, so the
                           kernels keep their programmatic (overlapped)
                           launches; any other nonzero value also times
                           every kernel launch                             */
    float *r_out;       /* optional device [n_frames][n_edges] float: the last
                           check-to-bit messages in edge order (for checking
                           one iteration at a time); NULL to skip            */
    int32_t frames_per_lane; /* tuning: frames each GPU lane carries in the
                           bit-node kernel (1, 2, 4 or 8); 0 picks by batch
                           size                                              */
    int32_t check_schedule;  /* tuning: check-node kernel schedule for checks
                           of degree <= 16, and of degree 17-18 in a code
                           with >= 2048 checks of degree 17-32 that are all
                           of degree <= 18; 0 = auto, 1 = inputs loaded
                           straight from global memory (degree 17-18: the
                           staged product-form kernel), 2 = rows staged
                           through a shared-memory ring by tensor copies
                           (when the batch allows: frame groups of 64 or
                           128). Other wide checks have kernels chosen by the
                           code: the register kernel, the staged product-form
                           or any-degree kernel (a code with >= 2048 checks
                           of degree 17-32) or one CTA per check (degree >
                           32)                                               */
    int32_t streams;    /* tuning: 1 = all passes on `stream`; 2 = the two
                           halves of the batch on two library streams, half a
                           pass apart, so that the check pass of one half
                           overlaps the bit pass of the other; 0 = 2 when the
                           batch splits evenly into halves of at least 128
                           frames and n x (padded frames) >= 2^20, else 1   */
    int32_t tile_frames; /* tuning: run all passes of tile_frames frames at a
                           time (rounded up to the kernels' frame group; tiles
                           alternate between the two streams), so that one
                           tile's working set can stay in L2; 0 = one tile per
                           stream. Results do not depend on any tuning field */
    int32_t check_rule; /* LDPC_RULE_SUM_PRODUCT (0, the paper's exact rule);
                           LDPC_RULE_MIN_SUM (1): |r| = clamp(alpha m -
                           beta, 0, L_MAX), m the smallest other |q|, same
                           signs -- plain (alpha 1, beta 0), normalised
                           (alpha < 1) or offset (beta > 0) min-sum, a
                           derived algorithm the paper names;
                           LDPC_RULE_SP_TABLE (2): sum-product with phi read
                           from a table (the paper's look-up-table
                           direction): phi replaced by its chords on 64
                           buckets per octave, the bucket of x being the top
                           15 bits of its float pattern (edges: the floats
                           with bits key << 17); needs l_max <= 22;
                           LDPC_RULE_MIN_SUM_ADAPTIVE (3): the min-sum rule
                           with alpha and beta chosen by the check's degree
                           from the code's table (ldpc_code_set_rule_table;
                           adaptive min-sum, which the paper names by
                           citation only, read as degree-adaptive); needs
                           that table set, ignores rule_alpha/rule_beta    */
    float rule_alpha;   /* min-sum scale; <= 0 selects 1                   */
    float rule_beta;    /* min-sum offset, >= 0                            */
} ldpc_decode_opts_t;

enum { LDPC_RULE_SUM_PRODUCT = 0, LDPC_RULE_MIN_SUM = 1, LDPC_RULE_SP_TABLE = 2, LDPC_RULE_MIN_SUM_ADAPTIVE = 3 };

/*
 * Set the per-check-degree scale and offset of LDPC_RULE_MIN_SUM_ADAPTIVE
 * (Section III-A names adaptive min-sum among the derived algorithms the
 * edge-level scheme carries): a check of degree d uses
 * |r| = clamp(alpha_d m - beta_d, 0, L_MAX), m the smallest other |q|, with
 * (alpha_d, beta_d) = entry min(d, n_degrees - 1) of the tables.
 *   n_degrees        >= 1 entries, indexed by check degree (0, 1, 2, ...)
 *   alpha_by_degree  host [n_degrees] floats, each finite and > 0
 *   beta_by_degree   host [n_degrees] floats, each finite and >= 0; NULL
 *                    selects 0 for every degree
 * The library copies the tables (synchronously) into device memory the code
 * owns; the caller keeps its buffers. Call it while no decode of this code is
 * in flight; later decodes (graph replays included) read the new values.
 * Returns LDPC_EINVAL for a bad entry or a host-only code, LDPC_ECUDA on a
 * failed copy.
 */
int ldpc_code_set_rule_table(ldpc_code_t *code, int32_t n_degrees, const float *alpha_by_degree,
                             const float *beta_by_degree);

/*
 * Decode n_frames frames.
 *   llr       device [n_frames][n] float channel LLRs (read only)
 *   max_iter  >= 0 iterations after the first check pass (Algorithm 2), so at
 *             most max_iter + 1 check passes run
 *   opts      NULL selects {early_exit = 1, l_max = 20, F32, no profiling}
 *   bits      device [n_frames][n] uint8 hard decisions (0/1)
 *   iters     device [n_frames] int32: 0 when the first pass already gives a
 *             codeword, else the iteration at which the frame stopped, or
 *             max_iter (always max_iter without early exit); -1 for every
 *             frame of a call in which a device wait of the pipelined check
 *             kernel gave up (a bounded wait for row copies; not expected)
 *   syndrome_ok device [n_frames] uint8: 1 iff H * bits = 0
 *   post_llr  optional device [n_frames][n] float posterior LLRs; NULL to skip
 * The code's decode workspace (device scratch sized for the largest batch
 * seen so far) is allocated on first use and reused; calls that share a code
 * are serialised on the device through an event, whatever their streams.
 * Errors: LDPC_EINVAL (bad sizes, NULL required pointer), LDPC_ENODEV,
 * LDPC_ENOMEM, LDPC_ECUDA.
 */
int ldpc_decode(ldpc_code_t *code, const float *llr, int32_t n_frames, int32_t max_iter,
                const ldpc_decode_opts_t *opts, uint8_t *bits, int32_t *iters, uint8_t *syndrome_ok,
                float *post_llr, void *stream);

/*
 * ldpc_decode on HOST buffers (same shapes, host memory; pinned memory makes
 * the copies asynchronous). Copies llr to the device, decodes, copies bits,
 * iters, syndrome_ok (and post_llr when non-NULL) back, and synchronizes
 * `stream` before returning. A batch of at least 256 frames with
 * n x n_frames >= 2^22 runs as two parts whose copies (on a library copy
 * stream) overlap the other part's decode; results are those of one decode.
 * opts->r_out must be NULL. Returns LDPC_ETIMEOUT
 * (results copied back, iters = -1) when a bounded device wait of the decode
 * gave up.
 */
int ldpc_decode_host(ldpc_code_t *code, const float *llr_host, int32_t n_frames, int32_t max_iter,
                     const ldpc_decode_opts_t *opts, uint8_t *bits_host, int32_t *iters_host,
                     uint8_t *syndrome_ok_host, float *post_llr_host, void *stream);

/*
 * A sequence of n_batches host batches of n_frames frames each (batch i:
 * llr_host[i] [n_frames][n] float in, bits_host[i] [n_frames][n] uint8,
 * iters_host[i] [n_frames] int32, ok_host[i] [n_frames] uint8 out), decoded
 * as ldpc_decode would, with the copies of each batch overlapping the decode
 * of its neighbours: two device staging slots alternate, batch i is copied
 * in on a library stream once batch i - 2 no longer needs its slot, decoded
 * on `stream`, and copied out on a second library stream. Pinned host memory
 * is needed for the overlap (pageable memory works, serialised). Returns when
 * every result is in host memory. opts->r_out and opts->profile must be
 * unset. Output pointers may repeat across batches (the copies out run in
 * batch order). Returns LDPC_ETIMEOUT when a bounded device wait of any
 * batch's decode gave up (that batch reports iters = -1). The paper decodes one frame set per call; this is the
 * receive-chain form of the same decode.
 */
int ldpc_decode_host_stream(ldpc_code_t *code, int32_t n_batches, const float *const *llr_host, int32_t n_frames,
                            int32_t max_iter, const ldpc_decode_opts_t *opts, uint8_t *const *bits_host,
                            int32_t *const *iters_host, uint8_t *const *ok_host, void *stream);

/*
 * Mixed-code batches. A batch holds several (code, frame count) items, all on
 * one device, each with its own decode workspace (allocated here) and
 * stream. ldpc_batch_run decodes every item's frames; the items run as
 * parallel branches forked from and joined into `stream`. The first run
 * launches the kernels directly; later runs replay one CUDA graph captured
 * from that sequence (re-captured when any buffer pointer changes). Results
 * equal ldpc_decode's for each item with the same options.
 *   codes, n_frames: n_items entries (1 <= n_frames[i] <= 8192); opts as in
 *   ldpc_decode (NULL = defaults; profile and r_out must be 0/NULL; the
 *   stream split and tiles are not used inside a batch).
 * Runs of one batch are serialised on the device. The batch borrows the code
 * handles: destroy the batch before its codes.
 */
typedef struct ldpc_batch ldpc_batch_t;

int ldpc_batch_create(int32_t n_items, ldpc_code_t *const *codes, const int32_t *n_frames, int32_t max_iter,
                      const ldpc_decode_opts_t *opts, ldpc_batch_t **out);

/* Decode every item: llr[i] device [n_frames[i]][n_i] float, outputs as in
 * ldpc_decode (post_llr may be NULL, or hold NULL entries). Asynchronous. */
int ldpc_batch_run(ldpc_batch_t *batch, const float *const *llr, uint8_t *const *bits, int32_t *const *iters,
                   uint8_t *const *syndrome_ok, float *const *post_llr, void *stream);

/* Autotune each item's kernel schedule (frames per lane in {1, 2, 4, 8} with
 * padding at most the item's own frame count, direct or pipelined check
 * kernel, the item's frames on one stream or split over two) by timing
 * decodes of the given device LLRs; keeps the fastest. Synchronous;
 * allocates temporary outputs. */
int ldpc_batch_tune(ldpc_batch_t *batch, const float *const *llr, void *stream);

/* The schedule picked for one item (frames per lane, check schedule,
 * streams) and the kernels one graph replay runs. NULL outputs are skipped. */
int ldpc_batch_info(const ldpc_batch_t *batch, int32_t item, int32_t *frames_per_lane, int32_t *check_schedule,
                    int32_t *streams, int64_t *kernels_per_run);

/* Waits for the batch's pending work and releases it. NULL is ignored. */
void ldpc_batch_destroy(ldpc_batch_t *batch);

/*
 * Decode server: continuous batching, at the frame level, over
 * device-resident codes (the parallel decoders of the paper's Results
 * section, serving requests as they arrive). Requests (a code index, n_frames
 * frames, caller-owned device buffers laid out as in ldpc_decode) queue per
 * code. A slot -- a frame set of up to max_batch_frames frames with its own
 * workspace and stream -- serves one code at a time and decodes in chunks of
 * a few flooding passes; between two chunks, every frame that has stopped
 * (zero syndrome, with early exit) or used up its max_iter iterations has its
 * results written to its request's buffers, the live frames are packed to
 * the front, and queued requests of that code are admitted into the free
 * frame groups, running their first pass and then sharing every later pass
 * with the frames already running, each frame counting its own iterations. A
 * request completes when its last frame is written out. Several slots run at
 * once, so requests arriving while others are on the GPU are admitted as
 * frames and slots free up and their work overlaps; a slot with no live frame
 * takes the code with the oldest waiting request. The slot count follows
 * memory_budget (admission by free memory) and max_slots; submits beyond
 * max_pending_frames queued frames return LDPC_EBUSY. A request's results do
 * not depend on the requests decoded beside it or on when it was admitted
 * (they equal ldpc_decode's for the same options). Buffers must stay valid
 * until ldpc_server_wait returns for the request. All entry points are
 * thread-safe.
 */
typedef struct ldpc_server ldpc_server_t;

typedef struct {
    int32_t max_batch_frames;   /* frames of a slot, 1..8192 (0 = 1024); also the
                                   largest request                              */
    int32_t max_slots;          /* batches in flight at once (0 = 4)              */
    int64_t memory_budget;      /* device bytes for the slots (0 = a quarter of
                                   the free device memory at creation)          */
    int64_t max_pending_frames; /* queued frames beyond which submits are refused
                                   with LDPC_EBUSY (0 = 2^20)                   */
    int32_t max_iter;           /* 0 = 50                                        */
    int32_t early_exit;         /* as in ldpc_decode_opts_t                      */
    float l_max;                /* <= 0 = 20                                     */
    int32_t msg_dtype;          /* ldpc_msg_dtype                                */
    int32_t check_rule;         /* as in ldpc_decode_opts_t (0 = sum-product)    */
    float rule_alpha;           /* min-sum scale; <= 0 selects 1                 */
    float rule_beta;            /* min-sum offset, >= 0                          */
} ldpc_server_opts_t;

typedef struct {
    int32_t slots;         /* slots allocated                                    */
    int64_t completed;     /* requests completed                                 */
    int64_t frames;        /* frames completed                                   */
    int64_t batches;       /* admissions: groups of requests added to a slot     */
    int64_t queued_frames; /* frames waiting for a slot                          */
    int64_t info_bits;     /* information bits of the admitted frames            */
} ldpc_server_stats_t;

/* Start a server over n_codes code handles (one device; the server borrows
 * them: destroy the server first). Allocates the slots. */
int ldpc_server_create(int32_t n_codes, ldpc_code_t *const *codes, const ldpc_server_opts_t *opts,
                       ldpc_server_t **out);

/* Queue a request; *request_id identifies it for ldpc_server_wait. post_llr
 * may be NULL. Errors: LDPC_EINVAL, LDPC_EBUSY (queue full). */
int ldpc_server_submit(ldpc_server_t *server, int32_t code_index, const float *llr, int32_t n_frames, uint8_t *bits,
                       int32_t *iters, uint8_t *syndrome_ok, float *post_llr, uint64_t *request_id);

/* Wait until the request completes (timeout_ms < 0: no limit; else
 * LDPC_ETIMEOUT when it has not completed in time) and release its record;
 * *latency_ms (optional) receives submit-to-completion time. */
int ldpc_server_wait(ldpc_server_t *server, uint64_t request_id, int32_t timeout_ms, double *latency_ms);

int ldpc_server_stats(ldpc_server_t *server, ldpc_server_stats_t *out);

/* Finish the queued work, stop the dispatcher and free the slots. */
void ldpc_server_destroy(ldpc_server_t *server);

/*
 * ldpc_decode for callers that cannot allocate device memory when they
 * decode: a latency-bound receive chain that must not stall on cudaMalloc
 * (which may synchronise the device), or a plug-in confined to another
 * framework's memory pool or to a device-memory cap. The code handle is made
 * beforehand with ldpc_code_create (that call does allocate: it uploads the
 * tables); this entry point then allocates nothing. The paper has no
 * counterpart: it is a deployment aid, not part of the method.
 *
 * Arguments, layouts, results and errors are those of ldpc_decode, except:
 *   - its scratch (messages, posteriors, interleaved LLRs, flags) lives in one
 *     64 MiB device array of the library, reserved on every GPU that loads the
 *     library until the process exits. A call whose scratch does not fit
 *     (roughly (4 E + 8 n) bytes per frame rounded up to 32 to 128 frames, for
 *     FP32 messages) is rejected with LDPC_EINVAL and a message giving both
 *     sizes; decode fewer frames per call;
 *   - every call on a device shares that array and it keeps the last call's
 *     contents (each call clears what it needs cleared). Calls that overlap on
 *     the GPU -- on different streams, with the same or different codes --
 *     race on it: the caller must serialise them;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture;
 *   - opts->profile must be 0 (timing events are not available here).
 */
int ldpc_decode_static(const ldpc_code_t *code, const float *llr, int32_t n_frames, int32_t max_iter,
                       const ldpc_decode_opts_t *opts, uint8_t *bits, int32_t *iters, uint8_t *syndrome_ok,
                       float *post_llr, void *stream);

/*
 * Channel LLRs of BPSK over AWGN (the BER simulator of Section IV, Eqs. 3-4)
 * into device llr [n_frames][n] float.
 * Frame f has global index frame_offset + f. Bit j of a frame uses Philox-4x64
 * with 10 rounds (Salmon et al., SC'11), key (seed, 0) and counter
 * (j / 4, frame_offset + f, 0, 0): words (w0, w1) drive bits 4q and 4q+1,
 * (w2, w3) bits 4q+2 and 4q+3, through Box-Muller on 24-bit uniforms
 * ua = ((w >> 40) + 1) 2^-24 in (0, 1], ub = (w >> 40) 2^-24 in [0, 1):
 * z0 = sqrt(-2 ln ua) cos(2 pi ub), z1 = sqrt(-2 ln ua) sin(2 pi ub).
 * Then x = 2c - 1, y = x + sigma z, llr = 2 y / sigma^2 (float arithmetic).
 * codewords: device [n_frames][n] uint8, or NULL for the all-zero word.
 * Errors: LDPC_EINVAL for negative sizes or sigma2 <= 0.
 */
int ldpc_gen_awgn(uint64_t seed, int64_t frame_offset, int32_t n_frames, int32_t n, float sigma2,
                  const uint8_t *codewords, float *llr, void *stream);

/*
 * Random information words for the BER simulator (Section IV transmits
 * random or all-zero codewords): device bits [n_frames][k] uint8, one bit per
 * byte. Bit j of frame f is bit (j mod 64) of word (j mod 256) / 64 of the
 * Philox-4x64-10 block with key (seed, 1) and counter (j / 256,
 * frame_offset + f, 0, 0); key word 1 keeps these bits independent of the
 * channel noise of ldpc_gen_awgn (key word 1 = 0).
 * Errors: LDPC_EINVAL for negative sizes or offset. Asynchronous.
 */
int ldpc_gen_bits(uint64_t seed, int64_t frame_offset, int32_t n_frames, int32_t k, uint8_t *bits, void *stream);

/*
 * Systematic encoding of an IRA code (ldpc_code_info_t.ira_k >= 0): for
 * information words info [n_frames][k] (device uint8, bit 0 of each byte
 * used) writes codewords [n_frames][n] (device uint8) c = [u | p] with
 * p_i = (H1 u)_i xor p_(i-1), the unique codeword of H with that systematic
 * part (the staircase makes H2 invertible). The paper's simulator takes its
 * codewords as given; this keeps random-codeword simulation on the device.
 * Scratch ((k + m + ceil(m / 64)) * ceil(n_frames / 32) words) is stream-ordered
 * (cudaMallocAsync / cudaFreeAsync on `stream`). Asynchronous.
 * Errors: LDPC_EINVAL when the code is not in IRA form, for n_frames < 0 or
 * NULL buffers; LDPC_ENODEV for a host-only code.
 */
int ldpc_encode_ira(ldpc_code_t *code, const uint8_t *info, int32_t n_frames, uint8_t *codeword, void *stream);

/*
 * A systematic encoder for any code, lifted (quasi-cyclic) codes without a
 * staircase included. H is brought to reduced row echelon form over GF(2)
 * on the host, pivots taken column by column from the last column down (an
 * IRA code keeps its staircase columns as parity positions); rank r of H,
 * k = n - r information positions (the non-pivot columns, in increasing
 * order), and per pivot row the information bits whose xor sets its pivot
 * column. Built once and kept with the code (device: r * ceil(k / 32) words
 * and n indices); *k_out (optional) receives k. A host-only code gets k only.
 * Synchronous. Errors: LDPC_EINVAL for a NULL code or m * n > 2^26 (the dense
 * elimination), LDPC_ECUDA/LDPC_ENOMEM on device failures.
 */
int ldpc_code_build_encoder(ldpc_code_t *code, int32_t *k_out);

/*
 * Encoding with that encoder: information words info [n_frames][k] (device
 * uint8, bit 0 of each byte used, k from ldpc_code_build_encoder) to
 * codewords [n_frames][n] (device uint8): information bit t at the t-th
 * information position, each pivot column the xor its row gives, so that
 * H c = 0 for every frame. Stream-ordered scratch ((k + r) * ceil(n_frames /
 * 32) words). Asynchronous. Errors: LDPC_EINVAL without an encoder, for
 * n_frames < 0 or NULL buffers; LDPC_ENODEV for a host-only code.
 */
int ldpc_encode(ldpc_code_t *code, const uint8_t *info, int32_t n_frames, uint8_t *codeword, void *stream);

/*
 * Error counts of the BER simulator (Section IV): for decoded words bits
 * [n_frames][n] and the transmitted words ref [n_frames][n] (NULL = the
 * all-zero word, enough by the code's linearity), adds to device counts[0]
 * the bit errors, counts[1] the frames with at least one error, counts[2]
 * the sum of iters (device [n_frames], optional) and counts[3] the frames
 * with syndrome_ok == 0 (device [n_frames], optional). counts is device
 * int64 [4], accumulated (zero it first). Asynchronous on `stream`.
 */
int ldpc_count_errors(const uint8_t *bits, const uint8_t *ref, int32_t n_frames, int32_t n, const int32_t *iters,
                      const uint8_t *syndrome_ok, int64_t *counts, void *stream);

/* Raw Philox-4x64-10 blocks: out[i][0..3] = Philox(key (key0, key1),
 * counter (ctr0 + i, ctr1, 0, 0)) for 0 <= i < count; out is device
 * [count][4] uint64. */
int ldpc_philox4x64_10(uint64_t key0, uint64_t key1, uint64_t ctr0, uint64_t ctr1, int64_t count,
                       uint64_t *out, void *stream);

/*
 * Test hook for the bounded device waits (no counterpart in the paper: it
 * exercises this library's failure reporting). The pipelined check kernel
 * waits for its row copies with a bounded number of polls; a warp whose wait
 * runs out flags the call, waits (again bounded) for its own copies still in
 * flight, and leaves, and the call then reports iters = -1 and
 * syndrome_ok = 0 for every frame (LDPC_ETIMEOUT from the host-buffer entry
 * points). ldpc_debug_giveup arms the next decode of `code` (ldpc_decode,
 * ldpc_decode_host, ldpc_decode_host_stream; run directly, never from a
 * captured graph) so that warp 0 of CTA `cta` (blockIdx.y * gridDim.x +
 * blockIdx.x) of its first later check pass takes that path after the rows
 * of its first check have landed: the give-up path runs without any wait
 * running out and without a fault. It only has an effect where that pass
 * runs the pipelined check kernel (frame groups of 64 or 128, checks of
 * degree <= 16). cta = -1 disarms it; the hook clears itself after one
 * decode. Returns LDPC_EINVAL for a NULL code or cta < -1.
 */
int ldpc_debug_giveup(ldpc_code_t *code, int32_t cta);

/* Kernel classes reported by ldpc_prof_read. */
enum {
    LDPC_K_INTERLEAVE = 0, /* frame-major LLRs -> frame-interleaved layout      */
    LDPC_K_CHECK = 1,      /* check-node update (plus syndrome of the last APP) */
    LDPC_K_BIT = 2,        /* bit-node update: posterior LLR per variable       */
    LDPC_K_SYNDROME = 3,   /* final syndrome pass                               */
    LDPC_K_FINALIZE = 4,   /* hard decisions, posteriors, iteration counts      */
    LDPC_K_OTHER = 5,      /* flag set-up, message export                       */
    LDPC_K_PASSES = 6,     /* the whole pass region (all check and bit passes,
                              on one or two streams), timed on `stream`       */
    LDPC_K_COUNT = 7
};

typedef struct {
    int64_t launches[LDPC_K_COUNT];
    double total_ms[LDPC_K_COUNT]; /* sum of CUDA-event durations */
    int64_t kernels;               /* library kernels enqueued by this code,
                                      profiled or not                      */
} ldpc_prof_t;

/* Collect the timings of profiled launches of `code` made since the last
 * reset (synchronizes on their events) and the count of all library kernels
 * enqueued for the code since then, adding them into *out (zero it first);
 * reset != 0 clears the record afterwards. */
int ldpc_prof_read(ldpc_code_t *code, ldpc_prof_t *out, int32_t reset);

/* Text of the calling thread's last error ("" if none). */
const char *ldpc_last_error(void);

/* Library version string. */
const char *ldpc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_GB300_H */

/* lbp.h — C ABI of the GB300 Lottery BP (+ OSD-0) syndrome decoder.
 *
 * The library decodes batches of syndromes s of one sparse GF(2) check
 * matrix H (m checks x n columns) into error estimates e_hat with
 * H e_hat = s (mod 2) when decoding succeeds.  The problem statement is the
 * one of Alg. 1 (inputs H, max iterations I, error rates p, syndrome s;
 * output e_hat) and of Alg. 2 (inputs H, BP output LLRs, s; output the
 * OSD-0 estimate), Sec. II-B and Sec. III-B of the paper.
 *
 * Conventions for every call:
 *  - Plain pointers and sizes only.  "device" pointers address memory of the
 *    current CUDA device; "host" pointers ordinary (preferably pinned) host
 *    memory.  The caller owns every buffer it passes and the stream.
 *  - Bits pack little-endian into 64-bit words: bit j of word w is index
 *    64 w + j; bits past the end of a row are zero on output and ignored on
 *    input.
 *  - Calls that take a stream only enqueue work on it (asynchronous); the
 *    caller synchronises.  lbp_load_code and lbp_free_code are synchronous.
 *  - Return value 0 on success, a negative LBP_E* code otherwise; nothing is
 *    enqueued when an argument check fails.  No C++ exception crosses the ABI.
 *  - A code object is bound to the device that was current at load time and
 *    may be used from several host threads at once (only lbp_tune writes it);
 *    a workspace must not be shared by two calls in flight.
 */
#ifndef LBP_H
#define LBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBP_OK          0
#define LBP_EINVAL    (-22)   /* malformed H, priors, parameters or sizes */
#define LBP_ENOMEM    (-12)   /* device allocation failed, or workspace too small */
#define LBP_ENOSYS    (-38)   /* this code / precision combination is not supported */
#define LBP_ECUDA     (-5)    /* a CUDA runtime call failed */
#define LBP_E2BIG     (-7)    /* request needs more scratch than lbp_decode_noalloc's fixed area */

/* Per-shot OSD status written to osd_out. */
#define LBP_OSD_NOT_RUN     0  /* BP converged, or OSD disabled */
#define LBP_OSD_APPLIED     1  /* OSD-0 estimate replaced the BP estimate */
#define LBP_OSD_NO_SOLUTION 2  /* s is outside the column space of H; BP estimate kept */

/* Storage type of the check-to-variable messages beta (Alg. 1 CN update).
 * Arithmetic is binary32 in every mode; channel LLRs mu and posteriors
 * lambda stay binary32 (Sec. VI-C quantisation study). */
#define LBP_MSG_F32 0          /* IEEE binary32 */
#define LBP_MSG_F16 1          /* IEEE binary16, round to nearest even */
#define LBP_MSG_I8  2          /* Int3.4 fixed point: q = clamp(rne(16 x), -127, 127), value q/16 */

/* Lottery policy (Sec. III-B and Table I): the proposed rule of Alg. 3 and
 * the four baselines it is compared with.  "Worst CN": the unsatisfied check
 * with the most columns currently estimated in error (lowest row on ties);
 * "random CN": the k-th unsatisfied check, k = floor(u N / 2^32) (Alg. 3);
 * "unreliable VN": least |lambda| among the check's columns (lowest column on
 * ties); "random VN": column floor(u2 deg / 2^32) of the check, u2 the high 32
 * bits of the same 64-bit draw whose low 32 bits are u. */
#define LBP_LOTTERY_PROPOSED          0  /* random CN, most unsatisfied checks, then least |lambda| */
#define LBP_LOTTERY_WORST_UNRELIABLE  1
#define LBP_LOTTERY_WORST_RANDOM      2
#define LBP_LOTTERY_RANDOM_UNRELIABLE 3
#define LBP_LOTTERY_RANDOM_RANDOM     4
/* Not Alg. 3: an ablation of its delay.  As LBP_LOTTERY_PROPOSED, but U is
 * built from this iteration's s_hat(i) instead of s_hat(i-1).  Built into the
 * index-image form in shared memory and the general kernel; a decode whose
 * plan takes another form (a code whose image does not fit shared memory, the
 * implicit or round-periodic graph, a merged launch) returns LBP_ENOSYS. */
#define LBP_LOTTERY_PROPOSED_CURRENT  5

/* Check-node rule.  LBP_RULE_MIN_SUM is the normalised min-sum update of
 * Alg. 1.  LBP_RULE_SUM_PRODUCT is the tanh rule
 *   beta_{v<-c} = (-1)^{s_c} 2 atanh( prod_{v' != v} tanh(alpha_{v'->c} / 2) ),
 * evaluated in binary32 in the equivalent log-domain form
 *   |beta| = phi( sum_{v' != v} phi(|alpha_{v'->c}|) ),  phi(x) = ln((e^x + 1) / (e^x - 1)),
 * with the sign of the product, the magnitude saturated at 25 (phi(0) is
 * infinite), and no normalisation factor (scale_mode and scale_const are
 * ignored).  Its results are not bit-identical across toolkits: they depend on
 * the device's expm1f and log1pf. */
#define LBP_RULE_MIN_SUM     0
#define LBP_RULE_SUM_PRODUCT 1

/* Normalisation factor of the min-sum CN update. */
#define LBP_SCALE_CONST    0   /* scale_const at every iteration */
#define LBP_SCALE_ADAPTIVE 1   /* 1 - 2^-(i+1) at iteration i (Alg. 1) */

typedef struct lbp_code lbp_code;   /* opaque, device-resident Tanner graph + mu */

typedef struct {
    int32_t  max_iter;      /* I >= 1 (Alg. 1); at most 2^24 - 1 */
    int32_t  scale_mode;    /* LBP_SCALE_* */
    float    scale_const;   /* used when scale_mode == LBP_SCALE_CONST, in (0, 1] */
    int32_t  lottery;       /* 1: apply the lottery sign flip of Alg. 3 */
    int32_t  lottery_skip;  /* first iteration index (0-based) at which it may run; 6 in Sec. III-B */
    int32_t  osd;           /* 1: OSD-0 (Alg. 2) on shots BP did not converge on */
    int32_t  msg;           /* LBP_MSG_* */
    int32_t  lottery_policy;/* LBP_LOTTERY_*: which check and column the lottery picks */
    uint64_t seed;          /* key of the lottery's random draws */
    uint64_t shot_offset;   /* global index of shot 0 of this call: the draws of shot b
                               depend only on (seed, shot_offset + b), never on batching */
    int32_t  rule;          /* LBP_RULE_*: check-node update */
    int32_t  reserved;      /* must be 0 */
} lbp_params;

/* Fill *p with the paper's Lottery BP defaults: I = 100, adaptive scale,
 * lottery on with skip 6, OSD off, binary32 messages, min-sum rule, seed 0. */
void lbp_params_default(lbp_params *p);

/* Load the check matrix H and the per-column error probabilities p_v.
 *
 * H is given in CSR form on the host: row_ptr[m+1] (row_ptr[0] = 0,
 * nondecreasing, row_ptr[m] = nnz), col_idx[nnz] strictly increasing within
 * each row, each in [0, n).  A row with exactly one nonzero is rejected
 * (its exclusive minimum in the CN update would range over an empty set);
 * rows with more than 32 nonzeros are rejected.  priors[n] are p_v in (0, 1);
 * the prior LLR mu_v = ln((1 - p_v) / p_v) (Alg. 1) is computed in binary64
 * on the host and rounded once to binary32.
 *
 * The library copies what it needs (host buffers may be freed on return),
 * allocates the device-resident graph with cudaMalloc on the current device
 * and returns an opaque handle in *out.  Errors: LBP_EINVAL, LBP_ENOMEM,
 * LBP_ECUDA; *out is set to NULL on error.
 *
 * When the bounded-degree index image and one shot's FP32 state always fit
 * in shared memory, the image gets a bank-aware layout: message rows padded
 * to a multiple of 32 words and a table that regroups the check phase's
 * pairs of checks into warps (chosen by a deterministic local search over
 * the shared-memory bank conflicts of the posterior gathers).  Results are
 * the same with or without it; LBP_BANK_LAYOUT=0 (read at load) turns it
 * off.
 *
 * Environment switches for experiments are read here, once, and kept in the
 * code object, so decodes never depend on the environment at call time:
 * LBP_BANK_LAYOUT, LBP_GRAPH (graph form, see lbp_code_surface),
 * LBP_BP_SHAPE ("S,G": BP groups per CTA and threads per group),
 * LBP_OSD_POOL_ROWS, LBP_OSD_LAT (see lbp_workspace_size) and LBP_OSD_DENSE
 * (see lbp_code_osd_form). */
int lbp_load_code(int32_t m, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *priors, lbp_code **out);

/* The environment switches lbp_load_code read for this code: graph form
 * (0 unset, 1 table, 2 implicit, 3 round), BP launch shape (groups per CTA and
 * threads per group, 0 unset), OSD pool rows (0 unset) and the OSD latency
 * layout (1 on, 0 off).  Any output pointer may be NULL.  Errors: LBP_EINVAL
 * (code NULL). */
int lbp_code_options(const lbp_code *code, int32_t *graph, int32_t *groups, int32_t *G,
                     int32_t *pool_rows, int32_t *osd_latency);

/* OSD form of a loaded code (Alg. 2, Sec. III-B).  Codes with m <= 160,
 * n + 1 <= 320 and 16-bit indices take the dense form: one warp per shot
 * holds all of [H | s] as packed 64-bit rows in registers (lane l: rows l,
 * l + 32, ...) and runs Gauss-Jordan elimination over the columns in the
 * LLR-sorted order of Alg. 2, stopping after rank(H) pivots (rank(H) over
 * GF(2) is computed at load).  Other codes take the event-driven warp kernel
 * and its block-wide fallback.  Both forms return the same e and status.
 * LBP_OSD_DENSE=0 (read at load) keeps a small code on the event-driven
 * kernels.  *dense = 1 for the dense form, else 0; *rank = rank(H) in the
 * dense form, else -1.  Any output pointer may be NULL.  Errors: LBP_EINVAL
 * (code NULL). */
int lbp_code_osd_form(const lbp_code *code, int32_t *dense, int32_t *rank);

/* Release a code object (synchronous; no call using it may be in flight).
 * Errors: LBP_EINVAL (code NULL). */
int lbp_free_code(lbp_code *code);

/* Sizes of a loaded code (any output pointer may be NULL).  Errors:
 * LBP_EINVAL (code NULL). */
int lbp_code_info(const lbp_code *code, int32_t *m, int32_t *n, int32_t *nnz);

/* Whether lbp_load_code recognised H as the space-time matrix (Eq. 1) of the
 * unrotated distance-d surface code whose per-round rows are those of
 * Table III: T rounds of d(d-1) checks of one type (*type 0: X, 1: Z), then
 * T - 1 (open time boundary, *cyclic 0) or T (cyclic, 1) measurement blocks,
 * d >= 3, columns and rows in Table III's order.  Such a code can run K_bp on
 * the implicit graph: every neighbour index is evaluated from the formulas,
 * no index image is read (LBP_GRAPH=table|implicit|round selects the form,
 * else lbp_tune's choice, else the index image).  Both forms give
 * identical results.  *d = 0 when not recognised; any output pointer may be
 * NULL. */
int lbp_code_surface(const lbp_code *code, int32_t *d, int32_t *T, int32_t *type, int32_t *cyclic);

/* Whether lbp_load_code recognised H as a space-time matrix of Eq. 1 for some
 * round check matrix H_r (m_r x n_r, rows of at most 4 ones, columns of at
 * most 2): T >= 2 rounds of H_r's rows shifted by t * n_r, then T - 1 (open
 * time boundary, *cyclic 0) or T (cyclic, 1) blocks of m_r measurement
 * columns, block b in rounds b and b + 1.  Such a code can run K_bp on the
 * round-periodic graph: one round's index table in shared memory, the round
 * offset and the measurement columns by arithmetic, with the same results as
 * the full index image, from a table of a few KB (7.5 KB for the d=25
 * space-time code, whose full image takes 230 KB).  LBP_GRAPH=round selects
 * it, and lbp_tune measures it; by default the full image is used, whose
 * index loads cost fewer instructions than the arithmetic they would
 * replace.  *T = 0 when not recognised; any output pointer may be NULL. */
int lbp_code_rounds(const lbp_code *code, int32_t *T, int32_t *m_r, int32_t *n_r, int32_t *cyclic);

/* Bytes of device workspace lbp_decode needs for num_shots shots with these
 * parameters (0 on invalid input).  The size grows linearly with num_shots
 * only when params->osd is set (the LLRs of shots handed to OSD).
 *
 * Tuning (codes on the event-driven OSD kernels, see lbp_code_osd_form):
 * OSD keeps rows of H sparse until an elimination changes them; the
 * changed rows take dense copies from a per-warp pool of C rows, by default
 * max(192, m / 2) (at most m), lowered so that the pools of all warps stay
 * within 1 GiB but never below min(m, 192).  The environment variable
 * LBP_OSD_POOL_ROWS (read when the code is loaded) sets C (1..m); a shot
 * that needs more rows is solved by the block-wide OSD kernel instead, with
 * the same result.
 * A call with num_shots at most the SM count runs OSD in its latency layout
 * (one warp per CTA; lambda and the first pool rows that fit in shared
 * memory, the other rows of the same C in the workspace); LBP_OSD_LAT=0
 * (read when the code is loaded) turns that off.  The workspace size does not depend on it. */
size_t lbp_workspace_size(const lbp_code *code, const lbp_params *params, int64_t num_shots);

/* Decode num_shots syndromes on `stream` (a cudaStream_t, NULL = legacy default).
 * Every shot runs the BP of Alg. 1 with the check-node rule params->rule
 * (normalised min-sum by default; messages stored as params->msg),
 * with the lottery sign flip of Alg. 3 (or the policy params->lottery_policy
 * names) when params->lottery is set, and stops at the first iteration whose
 * hard decision reproduces s.  When params->osd is set, the shots that did
 * not converge then take OSD-0 (Alg. 2) on their final posteriors.
 *
 * Device buffers, all [num_shots][...] row-major:
 *   syndromes   in   [B][ceil(m/64)] uint64, packed s
 *   err_out     out  [B][ceil(n/64)] uint64, packed e_hat
 *   converged   out  [B] uint8: 1 iff BP reached s_hat == s (early termination)
 *   osd_out     out  [B] uint8: LBP_OSD_* status (may be NULL)
 *   iters_out   out  [B] int32: BP iterations executed (i + 1 at convergence, else I)
 *   llr_out     out  [B][n] float: final posterior lambda (may be NULL)
 *   workspace        lbp_workspace_size() bytes, 256-byte aligned, owned by the
 *                    caller; contents on entry are ignored.
 * Shot b's result depends only on its syndrome, the code, the parameters and
 * shot_offset + b (not on num_shots or on other shots).  num_shots = 0 is an
 * empty decode: LBP_OK, nothing enqueued, no buffer read (lbp_decode_host,
 * lbp_tune and lbp_decode_noalloc do the same; lbp_graph_create and
 * lbp_server_submit want at least one shot).  Errors: LBP_EINVAL (also
 * num_shots < 0 or above 2^31), LBP_ENOMEM (workspace too small), LBP_ENOSYS,
 * LBP_ECUDA. */
int lbp_decode(const lbp_code *code, const lbp_params *params, int64_t num_shots,
               const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
               uint8_t *osd_out, int32_t *iters_out, float *llr_out,
               void *workspace, size_t workspace_bytes, void *stream);

/* Autotuner for the BP kernel's launch shape (groups of threads per CTA and
 * threads per group, the "shot tile" and the threads working on one shot):
 * decodes the given batch once per candidate shape and graph form, three
 * times each (a warm-up, then two timed runs of which the faster counts),
 * timing the BP kernel with CUDA events, and stores the fastest in `code` for its
 * message type and check-node rule (params->msg, params->rule); later decodes
 * with that pair use it.
 * Every shape computes identical results, so on return the outputs hold
 * lbp_decode's results for the batch.  Arguments as for lbp_decode (llr_out
 * omitted).  Synchronous: returns after the stream has drained.  It writes
 * the code object: no other call may use `code` meanwhile.  Tune on a batch
 * representative of the workload (its noise decides the iteration counts). */
int lbp_tune(lbp_code *code, const lbp_params *params, int64_t num_shots,
             const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
             uint8_t *osd_out, int32_t *iters_out, void *workspace, size_t workspace_bytes,
             void *stream);

/* The launch shape lbp_tune stored for (msg, rule): groups per CTA, threads
 * per group and graph form (1 index image, 2 implicit surface-code graph,
 * 3 round-periodic graph); all 0 when that pair has not been tuned.  Any
 * output pointer may be NULL.  Errors: LBP_EINVAL (code NULL, msg not an
 * LBP_MSG_* value, rule not an LBP_RULE_* value). */
int lbp_code_tuned(const lbp_code *code, int32_t msg, int32_t rule, int32_t *groups, int32_t *G, int32_t *graph);

/* Bytes of device workspace lbp_decode_host needs: lbp_workspace_size plus
 * device staging for the inputs and outputs.  When llr_out is requested the
 * call needs 4 * n * num_shots more bytes, rounded up to a multiple of 256. */
size_t lbp_host_workspace_size(const lbp_code *code, const lbp_params *params, int64_t num_shots);

/* Same as lbp_decode with HOST buffers (same shapes; llr_out and osd_out may
 * be NULL): enqueues the host-to-device copy of the syndromes, the decode and
 * the device-to-host copies of the results, ordered on `stream`, using
 * `workspace` (device, lbp_host_workspace_size bytes) for staging.  Calls of
 * at least 262,144 shots run as 2 or 4 consecutive chunks whose copies travel
 * on two internal streams while the neighbouring chunks decode on `stream`
 * (events keep the copies after `stream`'s earlier work and `stream`'s later
 * work after the copies); results are those of one call.  Pinned host memory
 * makes the copies asynchronous; the caller synchronises the stream before
 * reading the outputs.  On an error after copies were queued, `stream` is
 * still ordered after every one of them, so once it has drained the caller
 * may reuse its buffers and the workspace. */
int lbp_decode_host(const lbp_code *code, const lbp_params *params, int64_t num_shots,
                    const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                    uint8_t *osd_out, int32_t *iters_out, float *llr_out,
                    void *workspace, size_t workspace_bytes, void *stream);

/* ---- One launch for several codes -------------------------------------------
 *
 * A merged decode: the shots of several requests, of different codes, share
 * one persistent BP launch.  Every group of threads claims the next shot of
 * the combined work list, finds the request it belongs to and decodes it with
 * that request's code (its index image read from global memory, where the
 * L2 keeps it), parameters and buffers; OSD-0 then runs per request on the
 * shots BP left unconverged.  Each request's results are exactly those of
 * lbp_decode on the same arguments.  All requests must use the same message
 * type, the min-sum rule, and codes whose bounded-degree image has 16-bit
 * indices and the same degree bounds (every surface-code space-time matrix
 * shares one bound, every BB code another), on the current device.  The paper
 * has one decoder per code; this is the GPU service's batching. */
typedef struct {
    const lbp_code *code;
    lbp_params params;
    int64_t  num_shots;
    const uint64_t *syndromes;   /* device, [B][ceil(m/64)] */
    uint64_t *err_out;           /* device, [B][ceil(n/64)] */
    uint8_t  *converged;         /* device, [B] */
    uint8_t  *osd_out;           /* device, [B], may be NULL */
    int32_t  *iters_out;         /* device, [B] */
} lbp_batch_item;

/* Device workspace bytes lbp_decode_batch needs for these items (0 when the
 * items cannot share a launch or an argument is invalid).  Only the codes,
 * parameters and shot counts are read, not the buffer pointers. */
size_t lbp_batch_workspace_size(const lbp_batch_item *items, int32_t n_items);

/* Decode n_items (1..64) requests in one BP launch on `stream` (asynchronous;
 * the item array itself is copied before the call returns).  workspace:
 * lbp_batch_workspace_size bytes, 256-byte aligned, caller-owned.  Errors:
 * LBP_EINVAL (arguments), LBP_ENOSYS (the items cannot share a launch),
 * LBP_ENOMEM (workspace too small), LBP_ECUDA. */
int lbp_decode_batch(const lbp_batch_item *items, int32_t n_items, void *workspace, size_t workspace_bytes,
                     void *stream);

/* ---- Serving: continuous batching on one device ---------------------------
 *
 * A server owns a device arena (one cudaMalloc of arena_bytes at creation),
 * max_inflight CUDA streams and a scheduler thread.  Requests are decodes of
 * loaded codes with HOST buffers (pinned memory makes the copies
 * asynchronous).  The scheduler admits the oldest waiting request as soon as
 * a stream is free and the arena has room for its device buffers and
 * workspace (admission by memory); each admitted request runs H2D copy,
 * decode and D2H copies on its own stream, so requests overlap on the device
 * and a request that arrives while others run starts as soon as a slot and
 * memory free up.  A request's results depend only on its code, parameters
 * and syndromes, never on the other requests in flight.  The caller keeps the
 * host buffers and the code alive until the request completes.
 * The paper's decoder is a single-stream pipeline; this service is the GPU
 * deployment around it. */
typedef struct lbp_server lbp_server;

/* Create a server on the current device.  Errors: LBP_EINVAL (arena_bytes <
 * 4096 or max_inflight outside [1, 64]), LBP_ENOMEM, LBP_ECUDA. */
int lbp_server_create(size_t arena_bytes, int max_inflight, lbp_server **out);

/* Scheduling policy (defaults: chunk_work = 16 Mi edge-shots, priority = 1).
 * The decode kernels are persistent, so a launch holds its SMs until it ends.
 * A request of more than chunk_work edge-shots (num_shots x nnz(H)) runs as
 * consecutive launches of at most that much work, each shot keeping its own
 * draws (shot_offset advances), so work that arrives meanwhile waits for one
 * launch, not the whole request; chunk_work = 0 keeps one launch per request.
 * With priority = 1, requests that fit one launch run on a high-priority
 * stream and start ahead of queued chunks of larger requests.  Results do
 * not depend on the policy.  Applies to requests admitted after the call.
 * A request of at most one shot per SM takes lbp_decode's small-batch
 * latency layouts only when nothing else is in flight, since they hold
 * whole SMs; otherwise it runs the throughput layouts.
 * Errors: LBP_EINVAL (chunk_work < 0, priority not 0 or 1). */
int lbp_server_configure(lbp_server *server, int64_t chunk_work, int priority);

/* Merged launches: with max_items > 0, whenever an in-flight slot is free
 * the scheduler takes the oldest waiting request and up to max_items - 1
 * later ones that can share its launch (lbp_decode_batch's conditions) and
 * that fit the arena together, and decodes them with one BP launch on the
 * slot's stream; requests that cannot be merged run as before.  0 (the
 * default) keeps one launch chain per request.  Results do not depend on it.
 * Applies to requests admitted after the call.  Errors: LBP_EINVAL
 * (max_items outside [0, 64]). */
int lbp_server_set_batching(lbp_server *server, int32_t max_items);

/* Queue a decode (buffers as for lbp_decode_host, osd_out may be NULL) and
 * return its ticket.  LBP_E2BIG if the request can never fit the arena. */
int lbp_server_submit(lbp_server *server, const lbp_code *code, const lbp_params *params,
                      int64_t num_shots, const uint64_t *syndromes, uint64_t *err_out,
                      uint8_t *converged, uint8_t *osd_out, int32_t *iters_out, int64_t *ticket);

/* Non-blocking: *done = 1 once the request's outputs are in its host buffers,
 * then *latency_s (nullable) is submission-to-completion time in seconds and
 * the return value is the request's status; a completed ticket is forgotten
 * after it has been reported once.  Errors: LBP_EINVAL (server or done NULL,
 * a ticket never issued or already reported). */
int lbp_server_poll(lbp_server *server, int64_t ticket, int *done, double *latency_s);

/* Blocking version of lbp_server_poll, with its errors.  When several
 * callers wait on one ticket, one of them gets the request's status and the
 * others LBP_EINVAL. */
int lbp_server_wait(lbp_server *server, int64_t ticket, double *latency_s);

/* Drain every queued and in-flight request, then release the server.  No
 * other call on the server may be running (a thread blocked in
 * lbp_server_wait included) or follow.  Tickets not yet collected are
 * dropped; their outputs are in their host buffers.  Errors: LBP_EINVAL
 * (server NULL). */
int lbp_server_destroy(lbp_server *server);

/* Same decode as lbp_decode, for callers that cannot allocate device memory
 * (no cudaMalloc, no allocator callback): e.g. a latency-bound request loop
 * on a pre-sized device, where an allocation could stall or synchronise the
 * device in the middle of a request, or a plugin whose host process owns
 * every allocation and gives it none.  No workspace argument: scratch comes from a fixed
 * device array of LBP_NOALLOC_SCRATCH_BYTES bytes inside this library, which
 * every GPU that loads the library holds until the process exits.  The call
 * allocates nothing; buffers and their meaning are those of lbp_decode.
 *
 * The paper has no counterpart to this call; it is a deployment variant.
 *
 * Limits and behaviour:
 *  - Returns LBP_E2BIG, enqueuing nothing, when lbp_workspace_size(code,
 *    params, num_shots) exceeds LBP_NOALLOC_SCRATCH_BYTES (OSD on a large
 *    code, or very large OSD batches); use lbp_decode with a workspace then.
 *  - The first call on each device does a one-time set-up: with that device
 *    current, it looks up the array's device address (cudaGetSymbolAddress)
 *    and keeps it.  Make that first call before any stream capture begins.
 *  - All calls on a device share the array; the decode clears what must start
 *    at zero on the call's stream, so calls in order on one stream are
 *    independent, but calls that overlap on the GPU (other streams, other host
 *    threads) race on it and must be serialised by the caller. */
#define LBP_NOALLOC_SCRATCH_BYTES (32u << 20)
int lbp_decode_noalloc(const lbp_code *code, const lbp_params *params, int64_t num_shots,
                       const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                       uint8_t *osd_out, int32_t *iters_out, float *llr_out, void *stream);

/* ---- CUDA-graph replay of one decode --------------------------------------
 *
 * A decode issues a short chain of stream operations (a memset of its work
 * counters and the BP and OSD kernels); at small batches the host cost of
 * issuing them is a visible part of the latency.  lbp_graph_create captures
 * the chain lbp_decode would issue for these arguments into a CUDA graph
 * (on a private capturing stream; nothing runs), and lbp_graph_launch
 * replays it on `stream` with one call.  Buffers, sizes and parameters are
 * frozen at capture: to decode new shots, write their syndromes into the
 * same `syndromes` buffer (stream-ordered before the launch); outputs land
 * in the same output buffers.  Results are those of lbp_decode.  Arguments
 * as for lbp_decode (device buffers; workspace of lbp_workspace_size bytes,
 * 256-byte aligned), which must stay allocated while the graph exists.
 * Errors: LBP_EINVAL (as lbp_decode; also while kernel timing is enabled),
 * LBP_ENOMEM, LBP_ECUDA. */
typedef struct lbp_graph lbp_graph;
int lbp_graph_create(const lbp_code *code, const lbp_params *params, int64_t num_shots,
                     const uint64_t *syndromes, uint64_t *err_out, uint8_t *converged,
                     uint8_t *osd_out, int32_t *iters_out, float *llr_out, void *workspace,
                     size_t workspace_bytes, lbp_graph **out);
/* Replay the captured decode on `stream` (a cudaStream_t, NULL = legacy
 * default).  Replays of one graph must not overlap each other. */
int lbp_graph_launch(lbp_graph *graph, void *stream);
/* Release the graph (not its buffers).  Replays already launched finish.
 * Errors: LBP_EINVAL (graph NULL). */
int lbp_graph_destroy(lbp_graph *graph);

/* Kernel timing instrumentation, off by default.  While enabled, every
 * decode records a CUDA event pair on its stream around each kernel launch
 * (the BP kernel, K_bp, and the OSD kernel, K_osd); lbp_timing_read waits for
 * the recorded events, returns the summed milliseconds and launch counts
 * since the last read, and forgets them.  Enabling or disabling also forgets
 * them.  Any output pointer may be NULL.  Thread-safe; meant for benchmarks. */
int lbp_timing_enable(int on);
int lbp_timing_read(double *bp_ms, int64_t *bp_launches, double *osd_ms, int64_t *osd_launches);

/* Shared-memory load bandwidth probe for the on-chip roofline: two CTAs of
 * 1024 threads per SM read conflict-free 16-byte words from shared memory,
 * `trips` loop trips of eight loads per thread; the second of two launches
 * is timed with CUDA events on `stream` (synchronous: returns after it).
 * *bytes = bytes loaded by that launch, *ms = its duration.  Not part of the
 * paper's method; it measures the device.  Errors: LBP_EINVAL (trips outside
 * [1, 2^20], NULL outputs), LBP_ENOMEM, LBP_ECUDA. */
int lbp_probe_smem(int32_t trips, double *bytes, float *ms, void *stream);

/* Gallager's function phi(x) = ln((e^x + 1) / (e^x - 1)) as the sum-product
 * check-node rule evaluates it on the device (the magnitude rule of the
 * tanh form, 2 atanh(prod tanh(|a|/2)) = phi(sum phi(|a|))): out[i] =
 * phi(x[i]) for n device floats x >= 0, asynchronous on `stream`.  For
 * measuring that evaluation's accuracy; not part of a decode.  Errors:
 * LBP_EINVAL (n < 0, NULL buffers with n > 0), LBP_ECUDA. */
int lbp_probe_phi(const float *x, float *out, int64_t n, void *stream);

/* Static text for an LBP_* code. */
const char *lbp_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LBP_H */

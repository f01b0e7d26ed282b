/*
 * clipverify.h -- C-ABI of the GB300 (sm_103a) Clip-and-Verify bounding library.
 *
 * One call bounds a batch of branch-and-bound subdomains of a ReLU network:
 * activation-split constraints are turned into input-space rows, the input box is
 * clipped (relaxed clipping), every cached intermediate bound is re-concretised over
 * the clipped box and tightened by complete clipping, and the specification is
 * bounded by CROWN back-substitution.  Method: arXiv 2512.11087 (Sections 3.2-3.4,
 * Theorems 1-2, Algorithms 1, 2 and 5; CROWN as in its Appendix "Formulations").
 *
 * Conventions common to every entry point
 *  - Status codes are returned, never exceptions; cv_last_error() gives a message
 *    (thread-local, valid until the next call on the same thread).
 *  - Pointers documented as "device" must point to memory of the current CUDA device;
 *    "host" pointers are read during the call only.  The library never frees caller
 *    memory.  Objects created by cv_*_create / cv_*_build are owned by the caller and
 *    released with the matching cv_*_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Work is enqueued on it; entry points do not synchronise unless stated.
 *  - All floating-point data is FP32, row-major.  Sizes are element counts.
 *  - Invalid arguments (NULL where required, negative sizes, unknown enums, sizes that
 *    do not match the network or cache) return CV_EINVAL / CV_ESHAPE before anything is
 *    launched.  Problems only a kernel can see (a CSR count above the stated maximum, a
 *    split id out of range, a non-finite box) set the network's device status word;
 *    cv_device_status() reads and clears it.
 *  - Every returned bound is sound: lower bounds are rounded/padded toward -inf and
 *    upper bounds toward +inf by an a-priori bound of the FP32 rounding error.
 */
#ifndef CLIPVERIFY_H
#define CLIPVERIFY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int cv_status;
#define CV_OK           0
#define CV_EINVAL       1  /* bad argument */
#define CV_ESHAPE       2  /* sizes inconsistent with the network / cache */
#define CV_ENAN         3  /* non-finite value found in an input */
#define CV_ECUDA        4  /* CUDA runtime error (message in cv_last_error) */
#define CV_ETIMEOUT     5  /* a bounded device wait ran out */
#define CV_ENOMEM       6  /* device allocation failed */
#define CV_EUNSUPPORTED 7  /* feature not supported by the library, or not for this net / these sizes */
#define CV_EWORKSPACE   8  /* caller workspace too small */
#define CV_EDEVICE      9  /* a kernel reported a bad input (see cv_device_status) */

#define CV_MAX_LAYERS 16

/* Layer kinds (every layer except the last is followed by a ReLU). */
#define CV_LAYER_DENSE  0
#define CV_LAYER_CONV2D 1

/* Precision of the contractions (re-concretisation and back-substitution). */
#define CV_PREC_FP32   0  /* CUDA-core FP32 with chunked, compensated accumulation */
#define CV_PREC_BF16X8 1  /* spec back-substitution on tcgen05 tensor cores: operands split into three
                                 * BF16 digit slices, eight exact slice products per tile step */

/* Lower slope of an unstable ReLU when no per-row alpha is given. */
#define CV_ALPHA_ADAPTIVE 0  /* alpha = 1 if u >= -l else 0 */
#define CV_ALPHA_ONE      1
#define CV_ALPHA_ZERO     2

/* Human-readable message for the last failing call on this thread. */
const char* cv_last_error(void);

/* ---------------------------------------------------------------- network */

/* One affine layer z = W x + b.
 *  dense : in_c = fan-in, out_c = fan-out, in_h = in_w = out_h = out_w = 1,
 *          weight host [out_c x in_c] row-major, bias host [out_c].
 *  conv2d: input (in_c, in_h, in_w), output (out_c, out_h, out_w), square kernel k,
 *          stride, zero padding pad; weight host [out_c x in_c x k x k], bias [out_c];
 *          activations are flattened C,H,W. */
typedef struct cv_layer_desc {
    int kind;
    int in_c, in_h, in_w;
    int out_c, out_h, out_w;
    int k, stride, pad;
    const float* weight;
    const float* bias;
} cv_layer_desc;

typedef struct cv_net cv_net;

/* Copies the weights to the current device.  n_layers in [1, CV_MAX_LAYERS]; the
 * flattened output size of layer i must equal the input size of layer i+1. */
cv_status cv_net_create(const cv_layer_desc* layers, int n_layers, cv_net** out);
void      cv_net_destroy(cv_net* net);
/* dims (host, n_layers+1 entries, may be NULL): flattened widths n_0..n_L.
 * n_hidden: sum of the hidden widths n_1..n_{L-1} (global hidden ids are 0..n_hidden-1,
 * layer by layer). */
cv_status cv_net_dims(const cv_net* net, int* n_layers, int* dims, int* n_hidden);
/* Synchronises `stream`, returns CV_OK or CV_EDEVICE if a kernel flagged a bad input
 * since the last call, and clears the flag.  `code` (may be NULL) receives the raw
 * device status word (bit 0: CSR count above the stated maximum, bit 1: split id out
 * of range, bit 2: non-finite box, bit 3: target slot out of range, bit 4: a wait inside the
 * tensor-core back-substitution (CV_PREC_BF16X8) ran out; that round's spec bounds are not
 * valid). */
cv_status cv_device_status(cv_net* net, void* stream, int* code);

/* ---------------------------------------------------------------- root cache */

/* Root bounds and planes (Get_Constraints of Algorithm 5; Section 3.4 "cache and
 * reuse"): the CROWN lower/upper planes of every hidden neuron over the root box,
 * and the cache of the root-unstable ones (slots in increasing global id). */
typedef struct cv_cache cv_cache;

/* Runs CROWN on the GPU over the root box [root_lo, root_hi] (device, [n_0] each).
 * alpha_mode: CV_ALPHA_*.  The planes are padded by their rounding bound so that
 * they are valid over the root box.  Synchronises `stream` (it returns U). */
cv_status cv_cache_build(cv_net* net, const float* root_lo, const float* root_hi,
                         int alpha_mode, cv_cache** out, void* stream);

/* Builds a cache from caller-supplied planes (all host):
 *   root_lo, root_hi [n_0]; root_l, root_u [n_hidden] (bounds of every hidden neuron);
 *   U cached neurons with global ids ids[U] (strictly increasing), lower planes
 *   lA [U x n_0], lc [U] and upper planes uA [U x n_0], uc [U].  The planes are
 *   taken as valid over the root box as given. */
cv_status cv_cache_create(cv_net* net, const float* root_lo, const float* root_hi,
                          const float* root_l, const float* root_u, int U, const int* ids,
                          const float* lA, const float* lc, const float* uA, const float* uc,
                          cv_cache** out);

/* Number of cached (root-unstable) neurons. */
cv_status cv_cache_size(const cv_cache* cache, int* U);

/* Copies the cache to host buffers (any may be NULL): ids [U], lA/uA [U x n_0],
 * lc/uc [U], root_l/root_u [n_hidden].  Synchronous. */
cv_status cv_cache_read(const cv_cache* cache, int* ids, float* lA, float* lc,
                        float* uA, float* uc, float* root_l, float* root_u);
void      cv_cache_destroy(cv_cache* cache);

/* ---------------------------------------------------------------- phase timing */

/* Optional per-call instrumentation of cv_bound_batch (not part of the method).  When
 * cv_options.timer is set, the call records CUDA events on its stream at the phase
 * boundaries and counts its kernel launches and the coordinate-ascent row steps complete
 * clipping executes (one atomic add per thread block).  Phases:
 *   0 rows, pre-check and relaxed clipping   1 re-concretisation
 *   2 complete clipping                      3 back-substitution and verified flags */
#define CV_N_PHASES 4
typedef struct cv_timer cv_timer;
cv_status cv_timer_create(cv_timer** out);
void      cv_timer_destroy(cv_timer* timer);
/* Waits for the last timed call; ms[CV_N_PHASES] (may be NULL) receives its per-phase device
 * time in milliseconds, launches (may be NULL) its kernel launch count, cc_steps (may be NULL)
 * the row steps of Algorithm 1 it executed. */
cv_status cv_timer_read(cv_timer* timer, float* ms, int* launches, long long* cc_steps);
/* Decision counters of the last timed call's complete clipping (Algorithm 1 with two or more rows):
 * stats[0] row steps whose FP32 breakpoint decision was certified (re-decided on float-float
 * breakpoints, see cv_bound_batch), stats[1] of them with more than one candidate breakpoint,
 * stats[2] with a widened window, stats[3] left with the FP32 decision because it could not be
 * settled (still a valid multiplier), stats[4] of those with more than 64 candidates.
 * Synchronous. */
cv_status cv_timer_read_cc(cv_timer* timer, long long stats[5]);

/* ---------------------------------------------------------------- one BaB round */

/* Relaxed clipping of the input box (cv_options.relaxed), all with Theorem 2 per coordinate:
 *  CV_RELAX_OFF                 none (the box is copied; the pre-check still runs)
 *  CV_RELAX_PARALLEL            Algorithm 2: every active row against the input box
 *  CV_RELAX_SEQUENTIAL          Algorithm 3 (Appendix, sequential clipping): the active rows one
 *                               at a time, each against the box the earlier ones left, the
 *                               pre-check repeated on that box (an infeasible row or an emptied
 *                               box ends the subdomain, a redundant row is skipped); rows in their
 *                               order (splits, then extra rows)
 *  CV_RELAX_SEQUENTIAL_ORDERED  Algorithm 3 with the rows in the constraint-importance order of
 *                               the Appendix's heuristics: ascending |g.xhat + h| / ||g||_2 on the
 *                               input box, equal distances in row order
 * Complete clipping uses the active rows in their own order whatever the mode.  The sequential
 * modes keep the box in shared memory: 16 n_0 + 12 (max_splits + max_rows) bytes must stay
 * within 220 KiB (else CV_EUNSUPPORTED).  Other values are refused (CV_EINVAL). */
#define CV_RELAX_OFF 0
#define CV_RELAX_PARALLEL 1
#define CV_RELAX_SEQUENTIAL 2
#define CV_RELAX_SEQUENTIAL_ORDERED 3

typedef struct cv_options {
    int relaxed;        /* CV_RELAX_*: relaxed clipping of the input box (Theorem 2) */
    int sweeps;         /* complete clipping passes of Algorithm 1 (0: off) */
    int precision;      /* CV_PREC_* */
    int alpha_mode;     /* CV_ALPHA_*; ignored where batch.alpha is given */
    int enforce_splits; /* 1: clamp split neurons to their side (standard activation BaB) */
    cv_timer* timer;    /* optional phase timing (NULL: none) */
    int babsr_weight;   /* 1: the round also writes cv_batch_out.babsr_weight (the workspace grows
                           by B m max_i n_i floats for the layer products) */
} cv_options;

/* relaxed = 1, sweeps = 0, precision = CV_PREC_FP32, alpha_mode = CV_ALPHA_ADAPTIVE,
 * enforce_splits = 1, timer = NULL, babsr_weight = 0. */
void cv_options_default(cv_options* opt);

/* Inputs of one round for B subdomains (all device pointers unless noted).
 *  lo, hi        [B x n_0]  input box of every subdomain
 *  l_in, u_in    [B x U]    inherited bounds of the cached neurons; NULL = root bounds
 *  split_off     [B+1]      CSR offsets into split_ids; NULL = no splits
 *  split_ids     [nnz]      +(g+1): split z_g >= 0, -(g+1): z_g <= 0, g a global hidden id
 *  max_splits    (host)     upper bound on any subdomain's split count
 *  row_off       [B+1]      CSR offsets of extra rows G x + h <= 0; NULL = none
 *  G, h          [R x n_0], [R]
 *  max_rows      (host)     upper bound on any subdomain's extra-row count
 *  m, C, t       spec rows [m x n_L], thresholds [m]: bound f_r = C_r y + t_r
 *  alpha         [B x m x n_hidden] lower slopes per subdomain, spec row and neuron; NULL =
 *                alpha_mode
 *  tgt_off, tgt_ids  CSR over cache slots: complete-clipping targets per subdomain; NULL =
 *                every cached neuron still unstable after re-concretisation */
typedef struct cv_batch_in {
    int B;
    const float* lo;
    const float* hi;
    const float* l_in;
    const float* u_in;
    const int* split_off;
    const int* split_ids;
    int max_splits;
    const int* row_off;
    const float* G;
    const float* h;
    int max_rows;
    int m;
    const float* C;
    const float* t;
    const float* alpha;
    const int* tgt_off;
    const int* tgt_ids;
} cv_batch_in;

/* Outputs (device, caller-allocated; optional ones may be NULL).
 *  lower      [B x m]      sound lower bound of every spec row (+inf if infeasible)
 *  lo_clip, hi_clip [B x n_0]  clipped box (rounded outward)
 *  l, u       [B x U]      tightened bounds of the cached neurons
 *  mask       [B x U]      +1 active, -1 inactive, 0 unstable
 *  infeasible [B], verified [B]  0/1; an infeasible subdomain counts as verified
 *  err_bound  [B x m]      optional: the outward pad included in lower
 *  final_A    [B x m x n_0], final_c [B x m]  optional: the final linear bound
 *             f_r >= final_A_r . x + final_c_r on the clipped box (final_c includes the
 *             pad), e.g. for reuse as output constraints in input BaB (Section 3.3).
 *  babsr_weight [B x U]    written when cv_options.babsr_weight = 1: the weight of the BaBSR score
 *             (Appendix, neuron selection heuristic) of every cached neuron, the mean over the m
 *             spec rows of the coefficient of its post-activation in the lower bound, taken in the
 *             spec back-substitution of this round: for neuron q of hidden layer i, P^(i+1)_{r,q}
 *             with P^(i+1) = Lam^(i+1) W^(i+1) before layer i's relaxation; summed over the rows in
 *             increasing order in FP32, then divided by m (0 when m = 0 and for infeasible
 *             subdomains).  Not a bound: no pad. */
typedef struct cv_batch_out {
    float* lower;
    float* lo_clip;
    float* hi_clip;
    float* l;
    float* u;
    int8_t* mask;
    uint8_t* infeasible;
    uint8_t* verified;
    float* err_bound;
    float* final_A;
    float* final_c;
    float* babsr_weight;
} cv_batch_out;

/* Per-round summary of a round's outputs, the one quantity that ranks exchange when the subdomains
 * are sharded over GPUs (each rank bounds its own batch; no exchange inside the round): bounds [2]
 * (device) = the least spec lower bound over the feasible subdomains (Algorithm 5's global bound of
 * the batch) and over the unverified feasible ones (+inf when there are none), counts [2] (device) =
 * the verified (feasible) and the infeasible subdomains.  Inputs: lower [B x m], verified [B],
 * infeasible [B] as cv_bound_batch writes them.  Across ranks the bounds combine by min and the counts
 * by sum.  One launch; asynchronous on `stream`. */
cv_status cv_round_summary(int B, int m, const float* lower, const uint8_t* verified, const uint8_t* infeasible,
                           float* bounds, int* counts, void* stream);

/* Checks a batch's device inputs before a round.  The round itself reads nothing back to the host
 * (it never synchronises), so problems in device data reach it only as device status bits; this call
 * finds them first, with one launch and one read-back (synchronous on `stream`).  Checked: CSR offsets
 * non-decreasing with per-subdomain counts within max_splits / max_rows; split codes nonzero with
 * |code| - 1 < n_hidden; target slots in [0, U); every box bound finite with lo <= hi; l_in / u_in
 * and alpha without NaN, alpha in [0, 1]; G and h (row_off[B] rows), C and t finite.  Returns CV_ENAN
 * for a non-finite value, CV_EINVAL for any other problem, CV_OK otherwise; code (may be NULL)
 * receives the bits (1 CSR, 2 split code, 4 non-finite, 8 target slot, 32 lo > hi, 64 slope outside
 * [0, 1]) and cv_last_error names them.  Nothing is modified.  (The paper has no counterpart: it
 * defines the inputs, not their validation.) */
cv_status cv_batch_check(cv_net* net, const cv_cache* cache, const cv_batch_in* in, int* code, void* stream);

/* Bytes of device workspace cv_bound_batch needs for these sizes (in->B, in->m,
 * in->max_splits, in->max_rows; device pointers in `in` are not read). */
cv_status cv_bound_batch_workspace(const cv_net* net, const cv_cache* cache,
                                   const cv_batch_in* in, const cv_options* opt,
                                   size_t* bytes);

/* One round: constraint rows from splits and extra rows, pre-check, relaxed clipping,
 * re-concretisation, complete clipping, back-substitution of the spec, verified flags.
 * Complete clipping (Theorem 1, Algorithm 1, opt->sweeps passes over the active rows) takes the
 * decisions of the paper's sorted-breakpoint rule: the breakpoints are located in FP32, and with
 * two or more rows every decision whose neighbouring breakpoints lie within their a-priori FP32
 * error is re-decided on breakpoints recomputed in float-float arithmetic, with the multipliers
 * kept as float-float sums; only breakpoints equal to within about 2^-44 of their magnitude can be
 * ordered differently from exact arithmetic.  The bound is the dual objective at the leading
 * FP32 parts of the multipliers, padded by its rounding bound (any multipliers >= 0 give a valid
 * bound).
 * workspace: device memory of at least cv_bound_batch_workspace() bytes, 256-byte
 * aligned, used only during the call's kernels (stream-ordered). */
cv_status cv_bound_batch(cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                         cv_batch_out* out, const cv_options* opt,
                         void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- complete clipping of the spec */

/* Complete clipping (Theorem 1, Algorithm 1, opt->sweeps passes) applied to the final linear bound
 * of every spec row that a round left unproven: for subdomain b and spec row r with lower <= 0,
 * maximises over beta >= 0 the dual of  min final_A_r . x + final_c_r  over the clipped box under the
 * subdomain's active rows (splits and extra rows, as the round's pre-check keeps them), and raises
 * lower[b, r] to the dual value when it is larger.  Any beta >= 0 gives a valid bound: the value is
 * evaluated in FP32 with its rounding pad (FP64 when the padded value straddles 0), as for the
 * cached neurons.  verified is recomputed from the new bounds.
 * Call after cv_bound_batch with the same `in` and with out->final_A / final_c requested; reads
 * out->lo_clip, hi_clip, infeasible, final_A, final_c; updates out->lower and out->verified.  The
 * breakpoint decisions are those of the cached-neuron step (see cv_bound_batch).
 * opt->sweeps must be > 0 (else CV_EINVAL); opt->timer (optional) records the call as its
 * complete-clipping phase and its decision counters; the other options are not used.  workspace:
 * cv_spec_clip_workspace() bytes, 256-byte aligned. */
cv_status cv_spec_clip_workspace(const cv_net* net, const cv_cache* cache, const cv_batch_in* in, size_t* bytes);
cv_status cv_spec_clip(cv_net* net, const cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                       const cv_options* opt, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- scheduler tuning */

/* Complete clipping runs as persistent launches over uneven work (the paper's Algorithm 1 per
 * (target, side) task; the scheduling is this library's, with no counterpart in the paper).  In
 * the main launch, which stages a subdomain's rows in shared memory, each subdomain's tasks are
 * cut into work items that thread blocks take from an atomic ticket; items[c] is the number of
 * tasks per item for subdomains with c + 1 active rows (c = 2: three or more).  The wide launch
 * (subdomains with more than four rows, or every subdomain when the rows do not fit in shared
 * memory) hands out single tasks to warps and does not use the item sizes.  The item size
 * changes no result, only the time.
 * A cache starts with CV_CC_ITEMS_1/2/3.  cv_cc_items_set: each value in [1, 4096] (else
 * CV_EINVAL); it affects rounds run and graphs captured after the call (a graph captured before
 * keeps the sizes it was captured with). */
#define CV_CC_ITEMS_1 256
#define CV_CC_ITEMS_2 64
#define CV_CC_ITEMS_3 16
cv_status cv_cc_items_set(cv_cache* cache, const int items[3]);
cv_status cv_cc_items_get(const cv_cache* cache, int items[3]);

/* Autotuner of the item sizes for a batch: runs cv_bound_batch on (in, out, opt, workspace)
 * repeatedly on `stream` and times its complete-clipping phase with CUDA events: one row class
 * at a time, the candidates 128/256/512/1024 (one row), 32/64/128/256 (two), 8/16/32/64/128 (three
 * or more),
 * each round twice, the faster time counting; the fastest sizes stay in the cache.
 * best (may be NULL) receives them, best_ms (may be NULL) their phase time in milliseconds.
 * Host-synchronous (it reads the events), so it cannot be captured in a CUDA graph; `out`
 * holds the last round's results.  opt->sweeps must be > 0 (else CV_EINVAL: nothing to tune);
 * opt->timer is ignored. */
cv_status cv_autotune_cc(cv_net* net, cv_cache* cache, const cv_batch_in* in, cv_batch_out* out,
                         const cv_options* opt, void* workspace, size_t workspace_bytes, void* stream,
                         int best[3], float* best_ms);

/* ---------------------------------------------------------------- CUDA graph of a round */

/* A captured, instantiated CUDA graph of one cv_bound_batch call.  Replays run the same round
 * (same sizes, options and pointers) on whatever the input buffers hold at replay time, with a
 * single host launch: the round's ~25 kernels and its persistent complete-clipping launch are
 * replayed without per-kernel launch overhead. */
typedef struct cv_graph cv_graph;

/* Captures cv_bound_batch(net, cache, in, out, opt, workspace, workspace_bytes) on a private
 * stream (nothing runs during capture) and instantiates it.  opt->timer is ignored.  The
 * pointers in `in` and `out`, the workspace and the cache must stay valid while the graph is
 * used.  Synchronous. */
cv_status cv_graph_capture(cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                           cv_batch_out* out, const cv_options* opt, void* workspace,
                           size_t workspace_bytes, cv_graph** graph);
/* Enqueues one replay on `stream`. */
cv_status cv_graph_launch(cv_graph* graph, void* stream);
void      cv_graph_destroy(cv_graph* graph);

/* ---------------------------------------------------------------- alpha optimisation */

/* Inputs of the slope gradient (device pointers).
 *  B, m        subdomains and spec rows
 *  lo, hi      [B x n_0] box of every subdomain (for instance the clipped box of a round)
 *  l, u, mask  [B x U] bounds and stability of the cached neurons (for instance from
 *              cv_bound_batch); the other hidden neurons use their root state
 *  C, t        spec rows [m x n_L], thresholds [m]
 *  alpha       [B x m x n_hidden] lower slopes of unstable neurons, in [0, 1]
 *  grad_f      [B x m] upstream gradient of the bounds; NULL = ones
 *  precision   CV_PREC_FP32 (CUDA-core contractions) or CV_PREC_BF16X8 (the forward and the reverse
 *              sweep's contractions on tensor cores, split-BF16 as in cv_bound_batch)
 *  beta        [B x m x n_hidden] split multipliers >= 0, or NULL (none): the beta-CROWN form of the
 *              split constraints of Section 3.4.  A split z_g >= 0 (z_g <= 0) holds -z_g <= 0 (z_g <= 0)
 *              on the subdomain, so beta_g times it is added to the bound, which stays a lower bound
 *              for any beta >= 0 (after hidden layer h's relaxation, Lam_g -= sign_g beta_g, rounded
 *              so that the multiplier in effect is >= beta_g)
 *  split_sign  [B x n_hidden] +1 for a split z_g >= 0, -1 for z_g <= 0, 0 for none (cv_split_signs);
 *              required with beta
 *  grad_beta   [B x m x n_hidden] output (with beta): d sum_r grad_f f_r / d beta, 0 where no split */
typedef struct cv_alpha_in {
    int B, m;
    const float* lo;
    const float* hi;
    const float* l;
    const float* u;
    const int8_t* mask;
    const float* C;
    const float* t;
    const float* alpha;
    const float* grad_f;
    int precision;
    const float* beta;
    const int8_t* split_sign;
    float* grad_beta;
} cv_alpha_in;

/* Bytes of workspace cv_alpha_grad needs for B subdomains and m spec rows (the workspace passed
 * to cv_alpha_grad must be 256-byte aligned, else CV_EINVAL). */
cv_status cv_alpha_grad_workspace(const cv_net* net, int B, int m, size_t* bytes);

/* The spec lower bounds f [B x m] (as cv_bound_batch's back-substitution with these slopes,
 * padded outward; may be NULL) and the gradient of sum_r grad_f[b,r] f[b,r] with respect to
 * alpha, grad_alpha [B x m x n_hidden] (zero where a slope does not enter the bound: stable
 * neurons and neurons whose upper relaxation was selected).  alpha-CROWN's slope gradient
 * (the "optimized" alpha of the paper's ReLU relaxation Lemma), by a hand-written reverse
 * sweep of the back-substitution with the relaxation choices of the forward pass held fixed.
 * The gradient is FP32 and carries no pad. */
cv_status cv_alpha_grad(cv_net* net, const cv_cache* cache, const cv_alpha_in* in, float* lower,
                        float* grad_alpha, void* workspace, size_t workspace_bytes, void* stream);

/* The split signs [B x n_hidden] of a batch's CSR split lists (device; split_off NULL: no splits):
 * +1 for a code +(g+1) (z_g >= 0), -1 for -(g+1) (z_g <= 0), 0 elsewhere.  Codes out of range are
 * skipped (and flagged in the network's status word, as in cv_bound_batch). */
cv_status cv_split_signs(cv_net* net, int B, const int* split_off, const int* split_ids, int8_t* sign,
                         void* stream);

/* One Adam ascent step on n values clamped to [lo, hi] (the split multipliers: [0, inf)); as
 * cv_alpha_adam otherwise. */
cv_status cv_adam_range(float* x, float* m1, float* m2, const float* grad, long long n, int t, float lr,
                        float beta1, float beta2, float eps, float lo, float hi, void* stream);

/* One Adam ascent step on n slopes (device arrays alpha, m1, m2, grad), t >= 1 the step count,
 * followed by clamping alpha to [0, 1] (the paper's alpha optimisation uses Adam with learning
 * rate 0.1 decayed by 0.98 per iteration; the caller passes the decayed lr). */
cv_status cv_alpha_adam(float* alpha, float* m1, float* m2, const float* grad, long long n, int t,
                        float lr, float beta1, float beta2, float eps, void* stream);

/* ---------------------------------------------------------------- input branch and bound */

/* One split step of input BaB with Clip-and-Verify (Algorithm 4: Domain_Filter, Batch_Split with
 * the parents' hyperplanes shared by both children; Section 3.3, using final-layer bounds for
 * clipping).  For B bounded parents (the outputs of a cv_bound_batch call with final_A/final_c):
 *  - a parent that is verified or infeasible is dropped; the K kept parents, in their order,
 *    give children 2k (lower half) and 2k + 1 (upper half);
 *  - the split axis maximises (hi_i - lo_i) * sum_r |final_A_r,i| over the spec rows r that are
 *    not yet proven (lower_r <= 0), the extent of those planes along axis i (FP32, rows summed in
 *    increasing r); when every score is 0 the widest axis; the lowest index on ties;
 *  - the split point is fl(fl(lo_i + hi_i) * 0.5) (FP32), the children [lo_i, mid] and [mid, hi_i];
 *  - when exactly one spec row r is not yet proven, both children get its plane as the
 *    constraint row final_A_r . x + final_c_r <= 0: points where the plane is positive already
 *    satisfy f_r > 0 and every other row is proven on the whole parent.  With several rows
 *    unproven the points still to verify form a union of such half-spaces, not an intersection,
 *    so no row is passed (a joint row would be unsound).
 * Pass the children's boxes and rows to cv_bound_batch (extra rows: row_off, G, h; relaxed
 * clipping then clips each child with its inherited plane, as Algorithm 4 orders it).
 * Inputs (device): lo, hi [B x n_0] the parents' (clipped) boxes; final_A [B x m x n_0],
 *   final_c [B x m], lower [B x m]; verified, infeasible [B] (0/1).
 * Outputs (device, caller-allocated for the worst case K = B): lo_out, hi_out [2B x n_0];
 *   row_off [2B + 1] (CSR over the children, 0 or 1 row each); G [2B x n_0], h [2B];
 *   parent [2B] (index of each child's parent); n_children [1] (2K).  Entries past the
 *   2K children (and row_off past 2K) are left unwritten.
 * workspace: cv_input_split_workspace() bytes of device memory.  B = 0 writes n_children = 0 and
 * row_off[0] = 0.  Errors: CV_EINVAL for a null pointer (B > 0) or n_0, m < 1. */
cv_status cv_input_split_workspace(int B, size_t* bytes);
cv_status cv_input_split(int B, int n0, int m, const float* lo, const float* hi, const float* final_A,
                         const float* final_c, const float* lower, const uint8_t* verified,
                         const uint8_t* infeasible, float* lo_out, float* hi_out, int* row_off, float* G,
                         float* h, int* parent, int* n_children, void* workspace, size_t workspace_bytes,
                         void* stream);

/* ---------------------------------------------------------------- activation branch and bound */

/* BaBSR intercept score of a cached neuron c of a subdomain (Appendix, neuron selection heuristic):
 * -1 unless the neuron is unstable (mask 0, l < 0 < u); else
 *   max(0, -l) * max(0, u) / (u - l) * w,  w = max(0, -weight[c]) (w = 1 when weight is NULL)
 * in FP32, in this order: the intercept of the neuron's upper ReLU line times its weight in the
 * bound (for instance the mean over the spec rows of its coefficient in the final linear bound).
 *
 * One activation-BaB split step (Algorithm 5: Domain_Filter, Batch_Split).  For B bounded parents:
 * a verified or infeasible parent is dropped; a kept parent branches on its highest-scoring cached
 * neuron (the lowest slot among equal scores) and gives children 2k (split z <= 0, code -(id+1))
 * and 2k + 1 (z >= 0, code +(id+1)), each with the parent's split codes first, the parent's
 * (clipped) box and its cached bounds (to pass as l_in / u_in).  A kept parent without any
 * unstable cached neuron gets no children and stuck = 1.
 * Inputs (device): split_off [B + 1] / split_ids (may be NULL: no splits); lo, hi [B x n_0];
 *   l, u [B x U], mask [B x U]; weight [B x U] or NULL; verified, infeasible [B].
 * Outputs (device, caller-allocated for the worst case): split_off_out [2B + 1]; split_ids_out
 *   [2 (split_off[B] + B)]; lo_out, hi_out [2B x n_0]; l_out, u_out [2B x U]; parent, branched
 *   [2B] (parent index, branching slot); stuck [B]; n_children [1].
 * workspace: cv_activation_split_workspace() bytes.  Errors: CV_EINVAL for a null pointer (B > 0)
 * or a cache without unstable neurons. */
cv_status cv_activation_split_workspace(int B, size_t* bytes);
cv_status cv_activation_split(const cv_net* net, const cv_cache* cache, int B, const int* split_off,
                              const int* split_ids, const float* lo, const float* hi, const float* l,
                              const float* u, const int8_t* mask, const float* weight, const uint8_t* verified,
                              const uint8_t* infeasible, int* split_off_out, int* split_ids_out, float* lo_out,
                              float* hi_out, float* l_out, float* u_out, int* parent, int* branched,
                              uint8_t* stuck, int* n_children, void* workspace, size_t workspace_bytes,
                              void* stream);

/* Top-k targets for complete clipping (Algorithms 4 and 5, Top-K_Heuristic, with the score
 * above): per subdomain and hidden layer, the k unstable cached neurons of highest score (a higher
 * score first, then the lower slot), listed per subdomain in slot order as a CSR of cache slots to
 * pass as tgt_off / tgt_ids.  Inputs (device): l, u, mask [B x U]; weight [B x U] or NULL.  Outputs
 * (device): tgt_off [B + 1]; tgt_ids [B x U] at most.  k >= 0.  workspace:
 * cv_select_targets_workspace() bytes.  CV_EUNSUPPORTED above 17066 cached neurons. */
cv_status cv_select_targets_workspace(int B, int U, size_t* bytes);
cv_status cv_select_targets(const cv_net* net, const cv_cache* cache, int B, const float* l, const float* u,
                            const int8_t* mask, const float* weight, int k, int* tgt_off, int* tgt_ids,
                            void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- the activation-BaB loop */

/* The loop of Algorithm 5 (Clip-and-Verify for activation branch and bound) with every step on the
 * GPU.  The unknown set D_Unknown is a device-resident stack of domains, each with its split codes,
 * its clipped box, the bounds / mask / BaBSR weight of its cached neurons from its last round and
 * its least spec lower bound.  One iteration (cv_bab_step):
 *   Batch_Pick_Out   the last P = min(batch, |D|, capacity - |D|) domains of the stack (the most
 *                    recently added: depth first; the cap keeps the children within the capacity)
 *   Batch_Split      cv_activation_split on them with the BaBSR score and the stored weight; a
 *                    domain without an unstable cached neuron gives no children (stuck, unknown)
 *   Top-K_Heuristic  cv_select_targets on the children: their inherited bounds, the parent's mask
 *                    with the new split fixed (-1 for z <= 0, +1 for z >= 0) and the parent's
 *                    weight; top_k < 0 takes every unstable cached neuron
 *   Domain_Clipper / Domain_Update / Solve_Bound   one cv_bound_batch round on the children (the
 *                    split codes, the inherited box and bounds, the targets; the BaBSR weight on)
 *   Domain_Filter    verified and infeasible children are dropped; a child that holds max_depth
 *                    split codes and is not verified is dropped as depth-limited (unknown); the
 *                    others go back on the stack in child order
 * The host reads back two small counts per iteration (the children, the survivors) to size the
 * next launches.  The paper leaves the pick order open; depth first keeps the list compact: only
 * the picked region of the stack is rewritten. */
typedef struct cv_bab cv_bab;

typedef struct cv_bab_params {
    int batch;       /* n of Algorithm 5: parents picked per iteration, >= 1 */
    int top_k;       /* complete-clipping targets per hidden layer and child; < 0: every unstable one */
    int capacity;    /* domain-list capacity, >= batch + 1 */
    int max_depth;   /* split codes a domain may hold, >= 1 (<= 32 with complete clipping) */
    cv_options opt;  /* options of every round (the loop sets opt.babsr_weight = 1) */
} cv_bab_params;

/* batch 1024, top_k 20, capacity 65536, max_depth 32, opt = cv_options_default with sweeps 10. */
void cv_bab_params_default(cv_bab_params* p);

typedef struct cv_bab_stats {
    int picked;         /* parents taken from the list */
    int stuck;          /* of them without an unstable cached neuron (dropped: unknown) */
    int children;       /* subdomains bounded by this call's round (the domains it visited) */
    int verified;       /* children with every spec lower bound > 0 (infeasible ones not counted) */
    int infeasible;     /* children found infeasible */
    int depth_limited;  /* children dropped at max_depth split codes, not verified */
    int pushed;         /* children put back on the list */
    int remaining;      /* list size after the call */
    float lower_min;    /* least spec lower bound over the pushed children (+inf when none) */
} cv_bab_stats;

/* Allocates the list (capacity domains) and the buffers and workspace of one round of 2 batch
 * subdomains on the current device.  C [m x n_L], t [m]: device spec rows, kept by pointer (they
 * must outlive the object); m >= 1.  Errors: CV_EINVAL for bad parameters, CV_EUNSUPPORTED where
 * the round refuses the options, CV_ECUDA when the allocation fails. */
cv_status cv_bab_create(cv_net* net, const cv_cache* cache, int m, const float* C, const float* t,
                        const cv_bab_params* params, cv_bab** out);
/* Init of Algorithm 5: one round on B0 domains without splits (device boxes lo, hi [B0 x n_0],
 * 1 <= B0 <= min(2 batch, capacity); complete clipping has no rows there), then Domain_Filter; the
 * list is replaced by the survivors.  stats (host, may be NULL): picked = 0, children = B0. */
cv_status cv_bab_init(cv_bab* bab, int B0, const float* lo, const float* hi, void* stream,
                      cv_bab_stats* stats);
/* One iteration of the while loop.  An empty list returns CV_OK with stats->picked = 0; a full one
 * (no room for the children of one parent) returns CV_EWORKSPACE and changes nothing. */
cv_status cv_bab_step(cv_bab* bab, void* stream, cv_bab_stats* stats);
/* Iterations until the list is empty or max_iters have run (the time-out of Algorithm 5); total
 * (may be NULL) receives the sums of the iterations' counts (remaining and lower_min of the last
 * one), iters (may be NULL) the number run.  Stops at the first error. */
cv_status cv_bab_run(cv_bab* bab, int max_iters, void* stream, cv_bab_stats* total, int* iters);
/* Host copies of the list (synchronous): count; split_off [count + 1] and split_ids
 * [split_off[count]] (offsets from 0); lower_min [count]; any may be NULL. */
cv_status cv_bab_read(const cv_bab* bab, int* count, int* split_off, int* split_ids, float* lower_min,
                      void* stream);
void cv_bab_destroy(cv_bab* bab);

/* ---------------------------------------------------------------- measurement */

/* Measured FP32 FMA issue rate of the current device, in lane FMAs per second (the roofline
 * denominator of the ALU-bound complete clipping; the paper has no counterpart).  Times a kernel of
 * independent FFMA chains (4 blocks of 256 threads per SM) with CUDA events, best of three launches
 * after a warm-up; ms (may be NULL) receives that launch's time.  Synchronous on `stream`. */
cv_status cv_fp32_fma_peak(double* lane_fma_per_s, float* ms, void* stream);

/* ---------------------------------------------------------------- allocation-free variant */

/* Size of the library's fixed device scratch array used by cv_relaxed_clip_static. */
#define CV_STATIC_SCRATCH_BYTES (8u << 20)

/* Constraint rows, pre-check and relaxed clipping (the first steps of cv_bound_batch) without
 * any device allocation and without a caller workspace.  This entry has no counterpart in the
 * paper; it exists for callers that cannot allocate device memory when they bound subdomains:
 * a host framework whose caching allocator or memory pool must own every device byte, or a
 * latency-bound loop where cudaMalloc / cudaFree, which may synchronise the device, are not
 * allowed once the run has started.  It calls no cudaMalloc, cudaFree or allocating library
 * routine; its scratch is a fixed array of CV_STATIC_SCRATCH_BYTES inside this library, which
 * every GPU that loads the library holds until the process exits.
 *  in        the batch as for cv_bound_batch (B, lo, hi, splits, extra rows, max_splits,
 *            max_rows); spec rows, bounds, alpha and targets are not read
 *  lo_clip, hi_clip [B x n_0]  device outputs, identical to cv_bound_batch's with the same
 *            relaxed option
 *  infeasible [B]  device output: the subdomains the pre-check or relaxed clipping finds empty
 *            (cv_bound_batch can flag more in its later steps)
 *  relaxed   1: apply relaxed clipping; 0: only the pre-check (the box is copied)
 * Limit: B x (max_splits + max_rows) x 9 bytes (plus 256 bytes of alignment) must fit in the
 * array; larger batches return CV_EWORKSPACE before anything is launched.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make it before any stream capture.  All calls share the array and
 * it keeps the last call's contents; calls whose kernels overlap on the GPU (concurrent streams,
 * host threads) race on it, so serialise them. */
cv_status cv_relaxed_clip_static(cv_net* net, const cv_cache* cache, const cv_batch_in* in,
                                 float* lo_clip, float* hi_clip, uint8_t* infeasible, int relaxed,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CLIPVERIFY_H */

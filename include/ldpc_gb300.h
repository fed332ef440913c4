/*
 * ldpc_gb300.h -- C ABI of the GB300 (sm_103a) single-scan min-sum LDPC decoder.
 *
 * The decoder implements Huang, "Single-Scan Min-Sum Algorithms for Fast
 * Decoding of LDPC Codes" (ITW 2006):
 *   - Section III: (normalized/offset) min-sum, check rule Eq. (1), the
 *     posterior Z_n = Z0_n + sum_m L_mn, the decision x_n = 0 iff Z_n > 0 and
 *     the stop rule H x^T = 0 or an iteration cap;
 *   - Section IV, Eq. (3): the single scan, which needs only the
 *     check->variable adjacency N(m) and keeps one message L_mn per edge
 *     (LDPC_FORM_SS_FIXED);
 *   - Section V, Eqs. (4)-(5): the single scan whose persistent state per check
 *     is (A_m, B_m, n~_m) and one sign bit per edge (LDPC_FORM_SS_1BIT);
 *   - Section III, Eqs. (1)-(2) literally (horizontal then vertical scan), as a
 *     comparator (LDPC_FORM_TWO_SCAN), and the same two-scan algorithm with its
 *     check messages stored in the Section V form (A_m, B_m, n~_m and one sign
 *     bit per edge; Section V notes that the storage applies to the original
 *     algorithm too): LDPC_FORM_TWO_SCAN_1BIT.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an ldpc_status; nothing is thrown across the ABI.  On
 *     an error, ldpc_last_error() returns a message for the calling thread.
 *   - Pointers documented as "device" must be device memory of the code's
 *     device (or managed memory); "host" pointers are ordinary host memory.
 *   - The caller owns every buffer it passes in.  The library owns only the
 *     device copy of a code (created by ldpc_code_create, released by
 *     ldpc_code_destroy).
 *   - Decoding calls are asynchronous on the given stream (a cudaStream_t; NULL
 *     is the legacy default stream).  Outputs are valid once the stream has
 *     been synchronised.  Frames are independent; n_frames == 0 is a no-op.
 *   - Numerics: the int8 path is exact integer arithmetic, bit-identical to the
 *     literal two-scan / single-scan definitions (the posterior is held exactly,
 *     never saturated); the float32 path accumulates in float32.
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LDPC_API __attribute__((visibility("default")))
#else
#define LDPC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ldpc_status;
#define LDPC_OK 0
#define LDPC_ERR_INVALID_ARG 1 /* null pointer, malformed H, bad parameter */
#define LDPC_ERR_UNSUPPORTED 2 /* valid request this build cannot run (sizes, degrees) */
#define LDPC_ERR_CUDA 3        /* a CUDA runtime call failed */
#define LDPC_ERR_OOM 4         /* device allocation failed */
#define LDPC_ERR_TIMEOUT 5     /* a bounded device-side wait gave up */

/* Opaque device-resident description of a code. */
typedef struct ldpc_code ldpc_code;

enum { LDPC_DTYPE_INT8 = 0, LDPC_DTYPE_F32 = 1 };
enum { LDPC_FORM_SS_FIXED = 0, LDPC_FORM_SS_1BIT = 1, LDPC_FORM_TWO_SCAN = 2, LDPC_FORM_TWO_SCAN_1BIT = 3 };
enum { LDPC_RULE_PLAIN = 0, LDPC_RULE_OFFSET = 1, LDPC_RULE_NORMALIZED = 2, LDPC_RULE_SUM_PRODUCT = 3 };

/* Decoder settings (Section III: lambda_k, beta_k constant over k; cap).
 *   dtype      LDPC_DTYPE_INT8: llr is int8, messages are integers saturated to
 *              msg_sat; LDPC_DTYPE_F32: llr is float32.
 *   form       which of the four algorithms above runs.  The two-scan forms run
 *              frame-resident (TWO_SCAN on codes whose edge cells fit one SM,
 *              kernel AUTO or ONCHIP_HALF) or with the frame state in the
 *              workspace (kernel AUTO or STREAM; row and column degree <= 16).
 *   rule       PLAIN; OFFSET: |L| <- max(|L| - beta, 0); NORMALIZED: |L| <- lambda |L|;
 *              SUM_PRODUCT: the log-domain sum-product check rule that min-sum
 *              approximates (Section I), as an accuracy reference: L_mn = prod of
 *              the other inputs' signs x phi(sum over them of phi(min(|u|, 30))),
 *              phi(x) = -ln tanh(x/2); float32 path, SS_FIXED form, flooding only.
 *   offset     int8 path: beta in LSBs (>= 0).
 *   norm_num,  int8 path: lambda = norm_num / 2^norm_shift, magnitude floored
 *   norm_shift (0 < norm_num <= 2^norm_shift, 0 <= norm_shift <= 8).
 *   offset_f32 float path: beta (>= 0).
 *   norm_f32   float path: lambda (0 < lambda <= 1).
 *   msg_sat    int8 path: Qm in [1, 127]; |Z_n' - L_mn'| saturates to Qm before
 *              the minimum of Eq. (1)/(3).
 *   max_iter   iteration cap (>= 0).  0 returns the channel decisions.
 *   early_stop 1: a frame stops at the first k in 0..max_iter whose decisions
 *              satisfy H x^T = 0 (checked before the first iteration too);
 *              0: every frame runs max_iter iterations.
 *   kernel     LDPC_KERNEL_AUTO (0) lets the library choose; otherwise forces one
 *              implementation (results are identical; LDPC_ERR_UNSUPPORTED if the
 *              forced kernel cannot run this request):
 *                LDPC_KERNEL_ONCHIP_INT   frame-resident, 32-bit integer lanes
 *                LDPC_KERNEL_ONCHIP_HALF  frame-resident, two frames per packed
 *                                         binary16 instruction (exact: needs row
 *                                         degree <= 16 and
 *                                         128 + (max_col_degree + 1) * msg_sat <= 2048
 *                                         and n_vars <= 65535)
 *                LDPC_KERNEL_STREAM       frame state in device memory (the
 *                                         workspace), two kernel launches per
 *                                         iteration; for codes too large for one
 *                                         SM; the only kernel of the float32 path
 *                LDPC_KERNEL_PINGPONG     frame state in the workspace, one kernel
 *                                         launch per iteration and no column
 *                                         pass: two posterior buffers, the one
 *                                         read (Z^(k-1)) and the one updated
 *                                         with the exact binary16 sums of
 *                                         L^(k) - L^(k-2); two frame pairs per
 *                                         lane; int8, check degree <= 8 and the
 *                                         binary16 condition of ONCHIP_HALF;
 *                                         what AUTO runs for int8 single-scan
 *                                         codes too large for one SM
 *                LDPC_KERNEL_PERSISTENT   frame state in the workspace, the whole
 *                                         decode in one persistent kernel launch
 *                                         that takes groups of 64-frame chunks
 *                                         through all their iterations while
 *                                         their state stays in L2; int8, the
 *                                         binary16 conditions of ONCHIP_HALF and
 *                                         row degree <= 16.  Its waits between work items
 *                                         are bounded: if one gives up (it does
 *                                         not in a correct run), every frame of
 *                                         the call reports iters_used = -1 and
 *                                         syndrome_ok = 0
 *                LDPC_KERNEL_CLUSTER      a frame pair spread over the CTAs of a
 *                                         thread-block cluster (distributed shared
 *                                         memory), the packed binary16 arithmetic
 *                                         of ONCHIP_HALF with its conditions; for
 *                                         int8 single-scan codes too large for
 *                                         one SM; no workspace
 *   schedule   LDPC_SCHEDULE_FLOODING (0): every check of an iteration reads the
 *              posteriors of the previous iteration (Sections III-V).
 *              LDPC_SCHEDULE_LAYERED (1): the single scan of Eq. (3) in a layered
 *              schedule (layered decoding is cited in Section I; the paper's own
 *              schedule is flooding): the checks are grouped into layers whose
 *              checks share no variable (ldpc_code_layers); within an iteration
 *              the layers run in order and each check updates its variables'
 *              posteriors in place, Z_n <- Z_n - L^(k-1)_mn + L^(k)_mn.  The stop
 *              rule is checked after whole iterations.  int8, SS_FIXED or
 *              SS_1BIT, kernel AUTO, the binary16 conditions of ONCHIP_HALF
 *              (N unrestricted); needs a workspace.
 *   posterior  LDPC_POSTERIOR_EXACT (0): the int8 path holds every posterior
 *              exactly (it fits int16; the two-scan, single-scan and Section V
 *              forms then give identical results, Section V's equivalence).
 *              LDPC_POSTERIOR_SAT8 (1): the posterior is stored in 8 bits, the
 *              b-bit storage Section IV counts for messages applied to Z_n:
 *              after every iteration Z^(k)_n = clamp(Z^(0)_n + sum_m L^(k)_mn,
 *              -127, 127), and the next iteration's inputs Z^(k)_n - L^(k)_mn
 *              read the clamped value; llr_out returns the clamped posteriors.
 *              A single-scan-only variant (the two-scan form keeps Z_mn, not
 *              Z_n) and no longer equivalent to two-scan: int8, SS_FIXED or
 *              SS_1BIT, flooding, kernel AUTO, ONCHIP_HALF or STREAM (the
 *              kernels that write the posterior in a column pass); otherwise
 *              LDPC_ERR_UNSUPPORTED.  The float path takes EXACT only.
 */
typedef struct {
  int32_t dtype;
  int32_t form;
  int32_t rule;
  int32_t offset;
  int32_t norm_num;
  int32_t norm_shift;
  float offset_f32;
  float norm_f32;
  int32_t msg_sat;
  int32_t max_iter;
  int32_t early_stop;
  int32_t kernel;
  int32_t schedule;
  int32_t posterior;
} ldpc_decode_params;

enum { LDPC_SCHEDULE_FLOODING = 0, LDPC_SCHEDULE_LAYERED = 1 };
enum { LDPC_POSTERIOR_EXACT = 0, LDPC_POSTERIOR_SAT8 = 1 };

enum {
  LDPC_KERNEL_AUTO = 0,
  LDPC_KERNEL_ONCHIP_INT = 1,
  LDPC_KERNEL_ONCHIP_HALF = 2,
  LDPC_KERNEL_STREAM = 3,
  LDPC_KERNEL_CLUSTER = 4,
  LDPC_KERNEL_PERSISTENT = 5,
  LDPC_KERNEL_PINGPONG = 6
};

/* Build a code from the check->variable adjacency N(m) of H (Section II).
 *   row_ptr  host, [n_checks + 1], row_ptr[0] = 0, non-decreasing.
 *   col_idx  host, [row_ptr[n_checks]]: the variables of check m are
 *            col_idx[row_ptr[m] .. row_ptr[m+1]-1]; their order is the row
 *            position used by the Section V index n~.
 *   device   CUDA device ordinal that will run the decodes.
 * Checks: n_vars >= 1, n_checks >= 1, every check degree in [2, 32], indices in
 * [0, n_vars), no variable twice in a check; otherwise LDPC_ERR_INVALID_ARG.
 * Variables of degree 0 or 1 are allowed.  On success *out owns device memory
 * until ldpc_code_destroy.  Synchronous. */
LDPC_API ldpc_status ldpc_code_create(ldpc_code **out, int32_t n_vars, int32_t n_checks,
                             const int32_t *row_ptr, const int32_t *col_idx, int device);

/* A quasi-cyclic parity-check matrix (the structure of the DTMB codes the paper
 * decodes, Section I): an mb x nb base matrix of circulant shifts lifted by z.
 * Entry (i, j) = s in [0, z) puts the z x z identity shifted cyclically by s
 * in block (i, j): check i z + r has variable j z + ((r + s) mod z); s = -1 is
 * the zero block.  The caller owns `shift`. */
typedef struct {
  int32_t base_rows;      /* mb >= 1 */
  int32_t base_cols;      /* nb >= 1 */
  int32_t lift;           /* z >= 1 */
  const int32_t *shift;   /* host, [mb][nb] row-major, each -1 or in [0, z) */
} ldpc_qc_desc;

/* Expands a QC descriptor into the check->variable adjacency ldpc_code_create
 * takes (host computation only, no device call).
 *   row_ptr   host or NULL, [mb z + 1].
 *   col_idx   host or NULL, capacity entries; the variables of a check come in
 *             increasing order (block column order).
 *   n_edges   host or NULL: the number of edges E (call with col_idx NULL
 *             and capacity 0 to size col_idx).
 * LDPC_ERR_INVALID_ARG for a malformed descriptor (sizes < 1, a shift outside
 * {-1} u [0, z), nb z, mb z or E beyond int32) or capacity < E with col_idx
 * given. */
LDPC_API ldpc_status ldpc_qc_expand(const ldpc_qc_desc *qc, int32_t *row_ptr, int32_t *col_idx,
                                    int64_t capacity, int32_t *n_edges);

/* ldpc_code_create of the expanded descriptor (n_vars = nb z, n_checks = mb z),
 * with the block rows as the layers of the layered schedule (the z checks of a
 * block row share no variable, since every block is a permutation).  Same
 * checks and ownership as ldpc_code_create. */
LDPC_API ldpc_status ldpc_code_create_qc(ldpc_code **out, const ldpc_qc_desc *qc, int device);

/* Release a code (NULL is accepted).  Synchronises the code's device first. */
LDPC_API ldpc_status ldpc_code_destroy(ldpc_code *code);

/* Sizes of a code: any output pointer may be NULL. */
LDPC_API ldpc_status ldpc_code_info(const ldpc_code *code, int32_t *n_vars, int32_t *n_checks,
                           int32_t *n_edges, int32_t *max_row_degree, int32_t *max_col_degree);

/* Device workspace (bytes) that ldpc_decode_batch needs for this request;
 * 0 when the chosen kernel keeps all per-frame state on chip. */
LDPC_API ldpc_status ldpc_workspace_size(const ldpc_code *code, const ldpc_decode_params *params,
                                int32_t n_frames, size_t *bytes);

/* The implementation (an LDPC_KERNEL_* value other than AUTO) that
 * ldpc_decode_batch runs for this request: params->kernel itself when it is
 * not AUTO, else the library's choice.  For the layered schedule *kernel is
 * LDPC_KERNEL_AUTO (it has one implementation).  Errors as ldpc_workspace_size. */
LDPC_API ldpc_status ldpc_kernel_choice(const ldpc_code *code, const ldpc_decode_params *params,
                                        int32_t n_frames, int32_t *kernel);

/* Decode a batch of frames (Sections III-V).
 *   llr          device, frame-major [n_frames][n_vars] channel values Z0_n,
 *                int8 or float32 per params->dtype.
 *   hard_bits    device, [n_frames][ceil(n_vars/8)]: decision of variable n at
 *                byte n>>3, bit n&7 (1 means x_n = 1, i.e. Z_n <= 0).
 *   iters_used   device, [n_frames]: iterations run (the k at which H x^T = 0
 *                was met with early_stop, else max_iter).
 *   syndrome_ok  device, [n_frames]: 1 when the returned decisions satisfy H.
 *   llr_out      device or NULL, [n_frames][n_vars] final posterior Z_n:
 *                int16 for the int8 path, float32 for the float path.
 *   workspace    device or NULL, at least ldpc_workspace_size() bytes,
 *                256-byte aligned, not used by another call in flight.
 * Returns LDPC_ERR_UNSUPPORTED when the int8 posterior could leave int16
 * (128 + max_col_degree * msg_sat > 32767) or the code is too large for every
 * kernel of this build. */
LDPC_API ldpc_status ldpc_decode_batch(const ldpc_code *code, const ldpc_decode_params *params,
                              const void *llr, int32_t n_frames, uint8_t *hard_bits,
                              int32_t *iters_used, uint8_t *syndrome_ok, void *llr_out,
                              void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Learned offset min-sum (an extension of Section III's offset rule: beta_k
 * becomes a trainable table beta[k][c], c = degree class of the check), the
 * hand-written adjoint through the unrolled iterations, and the pieces of a
 * training step.  The decoder is the Section V single scan in float32.
 * ------------------------------------------------------------------------ */

/* Degree classes of a code: the distinct check degrees in ascending order.
 * degrees (host, nullable) receives n_classes entries (at most 31). */
LDPC_API ldpc_status ldpc_code_degree_classes(const ldpc_code *code, int32_t *n_classes, int32_t *degrees);

/* Layers of the layered schedule: *n_layers and, in layer_of_check (host,
 * nullable, n_checks entries), the layer of every check.  The default partition
 * (built by ldpc_code_create) takes the checks in row order and puts each into
 * the lowest layer none of whose checks shares a variable with it. */
LDPC_API ldpc_status ldpc_code_layers(const ldpc_code *code, int32_t *n_layers, int32_t *layer_of_check);

/* Replaces the layer partition (for instance the block rows of a
 * quasi-cyclic code).  layer_of_check: host, n_checks entries in [0, n_layers);
 * the checks of one layer must share no variable (else LDPC_ERR_INVALID_ARG and
 * the old partition stays).  Synchronises the code's device first. */
LDPC_API ldpc_status ldpc_code_set_layers(ldpc_code *code, int32_t n_layers, const int32_t *layer_of_check);

/* Bytes of device workspace that ldpc_learned_forward / _loss / _backward share
 * for n_iters iterations and n_frames frames: per-iteration checkpoints of the
 * posteriors Z^(k) and the Section V state, plus gradient buffers. */
LDPC_API ldpc_status ldpc_learned_workspace_size(const ldpc_code *code, int32_t n_iters, int32_t n_frames,
                                                 size_t *bytes);

/* Forward: n_iters (1..64) iterations of the Section V single scan with the
 * offset |L| <- max(|L| - beta[k][c], 0), no early stop.
 *   beta      device, [n_iters][n_classes] float32, iteration-major.
 *   llr       device, [n_frames][n_vars] float32 channel values Z0.
 *   z_out     device or NULL, [n_frames][n_vars] final posterior Z^(n_iters).
 *   workspace device, >= ldpc_learned_workspace_size bytes, 256-byte aligned;
 *             it keeps the checkpoints that _loss and _backward read, so those
 *             calls must use the same workspace, n_iters and n_frames.
 * Codes with more than 4 degree classes: LDPC_ERR_UNSUPPORTED. */
LDPC_API ldpc_status ldpc_learned_forward(const ldpc_code *code, int32_t n_iters, const float *beta,
                                          const float *llr, int32_t n_frames, float *z_out, void *workspace,
                                          size_t ws_bytes, void *stream);

/* Mean binary cross-entropy of the soft decisions sigma(-Z^(K)) (probability
 * that a bit is 1) against the transmitted bits, over all n_frames x n_vars
 * bits, after ldpc_learned_forward.  target_bits: device [n_frames][ceil(N/8)]
 * packed like hard_bits, or NULL for the all-zero codeword.  loss: device
 * float scalar.  want_grad != 0 also leaves dLoss/dZ^(K) in the workspace for
 * ldpc_learned_backward(dz = NULL).  The sum is reduced in a fixed order. */
LDPC_API ldpc_status ldpc_learned_loss(const ldpc_code *code, int32_t n_iters, int32_t n_frames,
                                       const uint8_t *target_bits, float *loss, int32_t want_grad,
                                       void *workspace, size_t ws_bytes, void *stream);

/* Backward (adjoint) through the unrolled iterations: dbeta (device,
 * [n_iters][n_classes]) = sum over frames of dLoss/dbeta for the gradient dz
 * (device [n_frames][n_vars] float32 = dLoss/dZ^(K), or NULL to use the one
 * ldpc_learned_loss left in the workspace).  Each iteration's row reduction is
 * recomputed from the checkpoints; the minimum is differentiated through its
 * argument (lowest position on ties, sgn(0) = +1), the offset through
 * [min > beta].  Deterministic: no floating-point atomics touch dbeta. */
LDPC_API ldpc_status ldpc_learned_backward(const ldpc_code *code, int32_t n_iters, const float *beta,
                                           const float *dz, int32_t n_frames, float *dbeta, void *workspace,
                                           size_t ws_bytes, void *stream);

/* One Adam step (Kingma & Ba, 2015) on n float32 parameters, all device
 * buffers: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps); step >= 1. */
LDPC_API ldpc_status ldpc_adam_step(float *params, const float *grads, float *m, float *v, int32_t n,
                                    int32_t step, float lr, float beta1, float beta2, float eps, void *stream);

/* BPSK over AWGN channel values on the device (Section II): y = (1 - 2 x) +
 * sigma xi, LLR = 2 y / sigma^2, sigma^2 = 1 / (2 rate 10^(EbN0/10)).  Frame f
 * (global index first_frame + f) draws its Eb/N0 uniformly in [ebn0_lo_db,
 * ebn0_hi_db] and its noise from Philox4x32-10 keyed by seed (Salmon et al.,
 * SC 2011; counter (g, frame, 0) gives the Box-Muller normals of variables
 * 4g..4g+3, counter (2^32-1, frame, 1) the Eb/N0 draw).  codewords: device
 * [n_frames][ceil(n_vars/8)] packed bits, or NULL for all-zero.  llr: device
 * [n_frames][n_vars] float32; ebn0_out: device [n_frames] or NULL. */
LDPC_API ldpc_status ldpc_awgn_llr_f32(int32_t n_vars, uint64_t seed, uint64_t first_frame, int32_t n_frames,
                                       float ebn0_lo_db, float ebn0_hi_db, float rate, const uint8_t *codewords,
                                       float *llr, float *ebn0_out, void *stream);

/* q[i] = clamp(round_half_away(llr[i] / delta), -qc, qc) as int8 (the fixed-
 * point channel input of ldpc_decode_batch); device buffers of n elements. */
LDPC_API ldpc_status ldpc_quantize_llr(const float *llr, int64_t n, float delta, int32_t qc, int8_t *q,
                                       void *stream);

/* Size of the device scratch array built into the library for
 * ldpc_decode_batch_noalloc (held on every GPU that loads the library). */
#define LDPC_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)

/* ldpc_decode_batch for callers that cannot allocate device memory.  (An
 * interface of this library; the paper has no counterpart.)
 *
 * Who needs it: decode paths that must not call cudaMalloc -- a receiver with a
 * bounded per-block latency (cudaMalloc synchronises the device and can take
 * arbitrarily long), or a component that only gets buffers from a pool it does
 * not own -- and so cannot provide ldpc_decode_batch's workspace.  This entry
 * point allocates nothing: it runs the int8 single-scan streaming decoder
 * (LDPC_KERNEL_STREAM) on LDPC_NOALLOC_SCRATCH_BYTES of scratch compiled into
 * the library as a device array.  The caller still passes the inputs and
 * outputs, with the meanings of ldpc_decode_batch; results are identical to
 * ldpc_decode_batch with kernel = LDPC_KERNEL_STREAM.
 *
 * Limits and behaviour:
 *  - params->dtype must be LDPC_DTYPE_INT8, form SS_FIXED or SS_1BIT, kernel AUTO
 *    or STREAM; otherwise LDPC_ERR_UNSUPPORTED.
 *  - A request whose scratch exceeds LDPC_NOALLOC_SCRATCH_BYTES is rejected with
 *    LDPC_ERR_UNSUPPORTED and a message giving both sizes; decode fewer frames
 *    per call.  (48 MiB holds 64 frames of an N = 64800, rate-1/2 code in either
 *    form, and 768 frames of the N = 7493 code in the SS_1BIT form or 576 in the
 *    SS_FIXED form; ldpc_workspace_size with kernel = LDPC_KERNEL_STREAM gives
 *    the exact need of a request.)
 *  - The first call on a device looks up the array's device address (a CUDA
 *    runtime query, no allocation); make that first call before any stream
 *    capture on the device.
 *  - Every call on a device uses the same array and leaves its contents behind;
 *    the decoder initialises everything it reads.  Calls whose executions
 *    overlap on the GPU (different streams, or different host threads) race on
 *    the array and corrupt each other: serialise them.
 *  - No cudaMalloc, cudaFree or allocating library routine is called. */
LDPC_API ldpc_status ldpc_decode_batch_noalloc(const ldpc_code *code, const ldpc_decode_params *params,
                                               const void *llr, int32_t n_frames, uint8_t *hard_bits,
                                               int32_t *iters_used, uint8_t *syndrome_ok, void *llr_out,
                                               void *stream);

/* ------------------------------------------------------------------------
 * Batches over several codes.  (A throughput interface of this library; the
 * paper decodes one code at a time.)  Every job is an int8 single-scan decode
 * with outputs identical to ldpc_decode_batch's.  The codes whose frame pair
 * fits one CTA share one persistent kernel launch in which frame pairs are
 * handed out longest first from a work queue, several pairs per CTA on
 * sub-teams of its threads.  A larger code either runs the streaming decoder
 * (frame state in the workspace) after that launch on the same stream, or is
 * decoded inside the same persistent launch by all CTAs of a thread-block
 * cluster (tuning.large).
 * ------------------------------------------------------------------------ */

/* One code of a batch.
 *   code        a code created on the batch's device.
 *   params      dtype LDPC_DTYPE_INT8, form SS_FIXED or SS_1BIT (the same form
 *               for every job of a batch), any rule, flooding schedule; kernel
 *               is ignored.  The code must meet the binary16 conditions of
 *               LDPC_KERNEL_ONCHIP_HALF.
 *   llr, n_frames and the outputs: device buffers as in ldpc_decode_batch
 *   (llr_out may be NULL).  n_frames == 0 drops the job. */
typedef struct {
  const ldpc_code *code;
  ldpc_decode_params params;
  const int8_t *llr;
  int32_t n_frames;
  uint8_t *hard_bits;
  int32_t *iters_used;
  uint8_t *syndrome_ok;
  int16_t *llr_out;
} ldpc_multi_job;

/* Launch shape of a batch (0 in a field means the default).
 *   threads       threads per CTA: 256, 512, 768 or 1024 (default 1024).
 *   team_threads  fewest threads that decode one frame pair of a code that fits
 *                 one CTA; a CTA holds threads / team_threads such pairs when
 *                 shared memory allows (32..1024, power of two; default 128).
 *   cluster       CTAs per cluster for codes that do not fit one SM: 2, 4, 8 or
 *                 16; default the smallest that fits every such code.
 *   queue         1 (default): dynamic work queue; 2: round-robin assignment.
 *   large         codes whose frame pair does not fit one CTA: 1 (default) the
 *                 streaming decoder after the persistent launch (the ping-pong
 *                 decoder for codes whose checks have degree <= 8, else the
 *                 two-launch one); 2 thread-block clusters inside the
 *                 persistent launch (the whole batch in one kernel launch).
 *   overlap       the codes on the streaming decoder: 0 (default) in sequence on
 *                 the caller's stream until ldpc_multi_autotune picks the faster
 *                 schedule; 1 always in sequence; 2 always overlapped on side
 *                 streams.  The autotuner keeps a schedule fixed by 1 or 2.
 *   stream_warps  warps per CTA of the ping-pong decoder's row kernel for the
 *                 streamed codes (four checks per warp, so 16, 32 or 64 checks
 *                 per CTA): 4, 8 or 16; 0 (default) 4 until ldpc_multi_autotune
 *                 times the three; a value set here is kept by the autotuner. */
typedef struct {
  int32_t threads;
  int32_t team_threads;
  int32_t cluster;
  int32_t queue;
  int32_t large;
  int32_t overlap;
  int32_t stream_warps;
} ldpc_multi_tuning;

typedef struct ldpc_multi ldpc_multi;

/* Plan a batch of n_jobs (1..16) jobs.  jobs: host array, copied; the device
 * buffers it names are bound to the plan (every ldpc_multi_decode reads and
 * writes those buffers).  tuning: host, nullable.  Checks every job and fails
 * with LDPC_ERR_UNSUPPORTED (and a message naming the job) if one cannot run. */
LDPC_API ldpc_status ldpc_multi_create(ldpc_multi **out, const ldpc_multi_job *jobs, int32_t n_jobs,
                                       const ldpc_multi_tuning *tuning);
LDPC_API ldpc_status ldpc_multi_destroy(ldpc_multi *plan);

/* Device workspace bytes of ldpc_multi_decode: the queue counters and the
 * frame state of the codes on the streaming decoder. */
LDPC_API ldpc_status ldpc_multi_workspace_size(const ldpc_multi *plan, size_t *bytes);

/* Decode every job of the plan on `stream`: a cudaMemsetAsync of the queue
 * counters, the persistent kernel launch, and the streaming decoder's memsets
 * and launches for the codes that run on it; no allocation, no host
 * synchronisation, so the call can be captured in a CUDA graph and replayed.
 * When the plan overlaps its streamed codes (chosen by ldpc_multi_autotune),
 * they run on side streams of the plan, forked from `stream` with an event
 * after the persistent kernel and joined back into it with one event each,
 * so the call still orders as one unit on `stream` (and captures as a fork /
 * join in a graph); the plan's first such call creates those streams and
 * events.  workspace: device, 256-byte aligned, at least
 * ldpc_multi_workspace_size bytes, not shared with another call in flight. */
LDPC_API ldpc_status ldpc_multi_decode(const ldpc_multi *plan, void *workspace, size_t ws_bytes, void *stream);

/* Times the candidate launch shapes (threads, team_threads, large, cluster) on the
 * plan's own buffers, reps decodes each after one warm-up, with CUDA events on
 * `stream` (synchronising it), and keeps the fastest; then times that shape
 * with the streamed codes in sequence and overlapped (at least 5 decodes
 * each, back to back) and keeps the faster, and, when codes run on the
 * ping-pong decoder, its row kernel at 4, 8 and 16 warps per CTA.  The decodes overwrite the
 * outputs (with the same values).  Not capturable.  chosen (host, nullable)
 * receives the kept shape, best_ms (host, nullable) its mean time. */
LDPC_API ldpc_status ldpc_multi_autotune(ldpc_multi *plan, void *workspace, size_t ws_bytes, int32_t reps,
                                         void *stream, ldpc_multi_tuning *chosen, float *best_ms);

/* Description of the plan: the shape in use, CTAs launched, cluster size,
 * dynamic shared memory per CTA, and per job (arrays of n_jobs entries,
 * nullable) where it runs (0 CTA sub-teams, 1 a cluster, 2 the streaming
 * decoder, -1 a job without frames) and the frame pairs a CTA holds at once. */
LDPC_API ldpc_status ldpc_multi_info(const ldpc_multi *plan, ldpc_multi_tuning *shape, int32_t *grid,
                                     int32_t *cluster, int32_t *smem_bytes, int32_t *job_is_cluster,
                                     int32_t *job_pairs_per_cta);

/* Diagnostic of the persistent decoder's failure path: on `device`, one CTA runs
 * the bounded wait that the decoder uses between its work items, on a counter
 * that nothing increments, for max_spins polls (128 ns apart; 1 .. 2^24).  The
 * wait gives up, sets the error word and returns, so the expected result is
 * LDPC_ERR_TIMEOUT; the CUDA context stays usable.  Synchronous; allocates a
 * few hundred bytes of device memory for the call. */
LDPC_API ldpc_status ldpc_wait_selftest(int device, int32_t max_spins);

/* Message describing the last failed call on this thread ("" if none). */
LDPC_API const char *ldpc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LDPC_GB300_H */

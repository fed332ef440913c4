/*
 * ldpc_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU oracle for (normalized/offset) min-sum
 * LDPC decoding and the two single-scan rewrites of Huang, "Single-Scan Min-Sum
 * Algorithms for Fast Decoding of LDPC Codes" (ITW 2006):
 *
 *   ORC_TWO_SCAN     Section III, Eqs. (1) and (2): horizontal scan over checks,
 *                    vertical scan over variables (uses the variable->check
 *                    adjacency M(n), built here from the CSR).
 *   ORC_SS_FIXED     Section IV, Eq. (3): single scan with one stored check
 *                    message L_mn per edge.
 *   ORC_SS_1BIT      Section V, Eqs. (4) and (5): single scan whose persistent
 *                    state per check is (A_m, B_m, n~_m) plus one sign per edge.
 *
 * Only tests, __graft_entry__.smoke() and bench.py's cpu_baseline may use this
 * oracle.  It shares no code with the CUDA decoder.
 *
 * Readings of points the paper leaves open (used identically by all forms):
 *  - offset on a signed message acts on the magnitude: sgn(L) max(|L|-beta, 0);
 *  - in the Section V form the offset/normalized magnitudes are the ones both
 *    stored and accumulated into Z;
 *  - inside Eq. (3) the extrinsic input of position n' is Z^{(k-1)}_{n'} - L^{(k-1)}_{mn'};
 *  - sgn(0) = 0; a zero input forces the other messages of its check to zero;
 *  - n~ is the lowest row position attaining max |L|;
 *  - the syndrome is also checked before the first iteration, so a frame whose
 *    channel decisions already form a codeword stops after 0 iterations; at most
 *    max_iter iterations run;
 *  - integer paths saturate |input| to msg_sat (Qm) before the minimum; the
 *    posterior is kept exactly (no saturation).
 */
#ifndef LDPC_ORACLE_H
#define LDPC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_TWO_SCAN = 0, ORC_SS_FIXED = 1, ORC_SS_1BIT = 2 };
enum { ORC_PLAIN = 0, ORC_OFFSET = 1, ORC_NORMALIZED = 2, ORC_SUM_PRODUCT = 3 };
/* ORC_SUM_PRODUCT (double decoders, two-scan and per-edge single scan): the
   sum-product check rule L = prod sgn x phi(sum phi(|in|)) over the other
   positions, phi(x) = -ln tanh(x/2), magnitudes saturated to ORC_SPA_SAT. */
#define ORC_SPA_SAT 30.0

typedef struct {
  int32_t n_vars, n_checks;
  const int32_t *row_ptr; /* [n_checks+1] */
  const int32_t *col_idx; /* [E] variable of each edge, grouped by check */
} orc_code;

typedef struct {
  int32_t rule;       /* ORC_PLAIN / ORC_OFFSET / ORC_NORMALIZED */
  int32_t offset;     /* beta (LSBs) for ORC_OFFSET */
  int32_t norm_num;   /* lambda = norm_num / 2^norm_shift, magnitude floored */
  int32_t norm_shift;
  int32_t msg_sat;    /* Qm: |input| saturates to Qm before the min; <= 0: none */
  int32_t max_iter;
  int32_t early_stop; /* 1: stop at the first iteration whose decisions satisfy H */
  /* > 0: the posterior is stored in b bits, Z^(k)_n = sat(Z^(0)_n + sum_m L^(k)_mn)
     clamped to [-post_sat, post_sat] after every iteration (the b-bit storage of
     Section IV's cost argument applied to Z; single-scan forms only, since the
     two-scan form keeps Z_mn, not Z_n); <= 0: Z held exactly. */
  int32_t post_sat;
} orc_iparams;

typedef struct {
  int32_t rule;       /* ORC_PLAIN / ORC_OFFSET / ORC_NORMALIZED */
  double offset;      /* beta for ORC_OFFSET */
  double lambda;      /* lambda for ORC_NORMALIZED */
  int32_t max_iter;
  int32_t early_stop;
  /* Optional per-iteration, per-check offsets: beta of check m at iteration k
     (1-based) is beta_tab[(k-1)*n_checks + m].  When set, rule must be ORC_OFFSET. */
  const double *beta_tab;
} orc_dparams;

/* Decode n_frames frames.  q0: [F][N] channel values Z^(0).  Outputs (all
   [F]-major, caller-allocated): bits [F][N] (0/1), iters [F], ok [F],
   z_out [F][N] final posterior Z, l_out [F][E] final check messages (nullable),
   state_out [F][M][4] = (A, B, n~, sign word) for ORC_SS_1BIT (nullable; sign
   word bit j set when s_mj < 0).  n_threads <= 0 uses every online core.
   Returns 0, or -1 on a bad argument. */
int orc_decode_int(const orc_code *code, const orc_iparams *p, int32_t form,
                   const int32_t *q0, int32_t n_frames, uint8_t *bits, int32_t *iters,
                   uint8_t *ok, int32_t *z_out, int32_t *l_out, int32_t *state_out,
                   int32_t n_threads);

/* margin_out [F] (nullable): the smallest |Z^(k)_n| over every iteration k
   (including k = 0) and variable n -- the distance to the decision rule, the
   only discontinuity of min-sum decoding (the check rule, offset, scaling and
   sums are Lipschitz in their inputs).  Frames with a small margin are those
   whose decisions or stopping iteration a different rounding may change; it is
   a diagnostic and does not affect decoding. */
int orc_decode_f64(const orc_code *code, const orc_dparams *p, int32_t form,
                   const double *q0, int32_t n_frames, uint8_t *bits, int32_t *iters,
                   uint8_t *ok, double *z_out, double *l_out, int32_t n_threads);
int orc_decode_f64_margin(const orc_code *code, const orc_dparams *p, int32_t form,
                          const double *q0, int32_t n_frames, uint8_t *bits, int32_t *iters,
                          uint8_t *ok, double *z_out, double *l_out, double *margin_out,
                          int32_t n_threads);

/* Learned offset min-sum (offset beta per iteration and check), FP64 reference
   of the loss and its gradient.  Runs n_iters iterations of Eq. (3) without
   early stop, with |L| <- max(|L| - beta_tab[k-1][m], 0), then the mean-free
   binary cross-entropy sum over bits of softplus(-Z) (bit 0) / softplus(Z)
   (bit 1) of the final posterior; targets [F][N] (0/1, nullable = all zero).
   Reverse mode through every message, each message differentiated literally:
   L_j = prod_{j'!=j} sgn(u_j') * max(min_{j'!=j} |u_j'| - beta, 0), the minimum
   through its lowest-position argument, sgn(0) = +1 for the derivative of
   |u|.  Outputs: loss_sum (sum over frames and bits), dbeta [n_iters][M]
   (gradient of loss_sum), gap [F] (nullable): the frame's smallest distance to
   a point where the loss is not differentiable -- over every iteration and
   check, min2 - min1 of |u|, |min1 - beta|, |min2 - beta| and the smallest |u|. */
int orc_learned_grad_f64(const orc_code *code, int32_t n_iters, const double *beta_tab, const double *q0,
                         const uint8_t *targets, int32_t n_frames, double *loss_sum, double *dbeta,
                         double *gap, int32_t n_threads);

/* The single scan of Eq. (3) in a layered schedule: layer[m] in [0, n_layers)
   gives the layer of check m, the checks of one layer must share no variable
   (else -1).  Within an iteration the layers run in increasing order; each
   check updates the posteriors of its variables in place,
   Z_n = (Z_n - L_mn) + L_new_mn.  Per-edge messages (the Section V state gives
   the same messages).  Outputs as orc_decode_int (no state_out). */
int orc_decode_layered_int(const orc_code *code, const orc_iparams *p, const int32_t *layer, int32_t n_layers,
                           const int32_t *q0, int32_t n_frames, uint8_t *bits, int32_t *iters, uint8_t *ok,
                           int32_t *z_out, int32_t *l_out, int32_t n_threads);

/* Number of threads orc_decode_* would use for n_threads <= 0. */
int32_t orc_default_threads(void);

#ifdef __cplusplus
}
#endif
#endif

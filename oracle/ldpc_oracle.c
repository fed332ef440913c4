/*
 * ldpc_oracle.c -- TEST INFRASTRUCTURE ONLY (see ldpc_oracle.h).
 *
 * Every function follows the paper's equations in their order and notation,
 * one frame at a time, with no blocking, fusion or reordering.  Check messages
 * are computed literally as a product of signs and a minimum over N(m)\n
 * (quadratic in the check degree) rather than through min1/min2 bookkeeping.
 * Frames are independent problems; they are split across POSIX threads.
 */
#include "ldpc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------ common */

static int sgn_i(int64_t v) { return (v > 0) - (v < 0); }
static int sgn_d(double v) { return (v > 0.0) - (v < 0.0); }

/* Section III: magnitude modification of a check message.  Normalized:
   L <= lambda_k L (magnitude floored in integers).  Offset: L <= max(L - beta, 0),
   read as acting on |L|. */
static int64_t modify_i(const orc_iparams *p, int64_t mag) {
  if (p->rule == ORC_OFFSET) return mag > p->offset ? mag - p->offset : 0;
  if (p->rule == ORC_NORMALIZED) return (mag * p->norm_num) >> p->norm_shift;
  return mag;
}

static double modify_d(const orc_dparams *p, int32_t k, int32_t m, int32_t n_checks, double mag) {
  if (p->rule == ORC_OFFSET) {
    double beta = p->beta_tab ? p->beta_tab[(size_t)(k - 1) * n_checks + m] : p->offset;
    return mag > beta ? mag - beta : 0.0;
  }
  if (p->rule == ORC_NORMALIZED) return p->lambda * mag;
  return mag;
}

static int64_t sat_i(const orc_iparams *p, int64_t mag) {
  return (p->msg_sat > 0 && mag > p->msg_sat) ? p->msg_sat : mag;
}

/* The stored posterior of the single scan: Z clamped to [-post_sat, post_sat]
   when the posterior is kept in b bits, else Z itself. */
static void sat_post(const orc_iparams *p, int64_t *Z, int32_t N) {
  if (p->post_sat <= 0) return;
  for (int32_t n = 0; n < N; ++n) Z[n] = Z[n] > p->post_sat ? p->post_sat : (Z[n] < -p->post_sat ? -p->post_sat : Z[n]);
}

/* Decoding step (Section III): x_n = 0 if Z_n > 0, else 1.  Returns 1 when
   H x^T = 0. */
static int decide_and_check(const orc_code *c, const int64_t *Zi, const double *Zd,
                            uint8_t *x) {
  for (int32_t n = 0; n < c->n_vars; ++n) x[n] = Zi ? (Zi[n] > 0 ? 0 : 1) : (Zd[n] > 0.0 ? 0 : 1);
  for (int32_t m = 0; m < c->n_checks; ++m) {
    int par = 0;
    for (int32_t e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e) par ^= x[c->col_idx[e]];
    if (par) return 0;
  }
  return 1;
}

/* Variable->check adjacency M(n) (CSC with edge ids), needed by the vertical
   scan of the two-scan algorithm only. */
typedef struct {
  int32_t *col_ptr; /* [N+1] */
  int32_t *edge;    /* [E] edge ids grouped by variable */
} orc_csc;

static int build_csc(const orc_code *c, orc_csc *t) {
  int32_t E = c->row_ptr[c->n_checks];
  t->col_ptr = (int32_t *)calloc((size_t)c->n_vars + 1, sizeof(int32_t));
  t->edge = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  int32_t *fill = (int32_t *)calloc((size_t)c->n_vars + 1, sizeof(int32_t));
  if (!t->col_ptr || !t->edge || !fill) { free(fill); return -1; }
  for (int32_t e = 0; e < E; ++e) t->col_ptr[c->col_idx[e] + 1]++;
  for (int32_t n = 0; n < c->n_vars; ++n) t->col_ptr[n + 1] += t->col_ptr[n];
  for (int32_t e = 0; e < E; ++e) {
    int32_t n = c->col_idx[e];
    t->edge[t->col_ptr[n] + fill[n]++] = e;
  }
  free(fill);
  return 0;
}

static void free_csc(orc_csc *t) { free(t->col_ptr); free(t->edge); }

/* Eq. (1) / Eq. (3) for one position j of a check with inputs in[0..d-1]:
   product of sgn over the other positions times the minimum over the other
   positions of the (saturated) magnitude. */
static int64_t check_rule_i(const orc_iparams *p, const int64_t *in, int32_t d, int32_t j) {
  int s = 1;
  int64_t mn = -1;
  for (int32_t t = 0; t < d; ++t) {
    if (t == j) continue;
    s *= sgn_i(in[t]);
    int64_t a = sat_i(p, in[t] < 0 ? -in[t] : in[t]);
    if (mn < 0 || a < mn) mn = a;
  }
  return (int64_t)s * mn;
}

static double check_rule_d(const double *in, int32_t d, int32_t j) {
  int s = 1;
  double mn = INFINITY;
  for (int32_t t = 0; t < d; ++t) {
    if (t == j) continue;
    s *= sgn_d(in[t]);
    double a = fabs(in[t]);
    if (a < mn) mn = a;
  }
  return (double)s * mn;
}

/* Sum-product check rule (log domain; cited in Section I as the rule min-sum
   approximates), for one position j: the product of the signs of the other
   inputs times phi(sum over the other inputs of phi(|in|)), with
   phi(x) = -ln tanh(x/2) = ln(1 + 2/(e^x - 1)) (phi(0) = inf, phi(inf) = 0) and
   the magnitudes saturated to ORC_SPA_SAT before phi. */
static double phi_d(double x) { return log1p(2.0 / expm1(x)); }

static double check_rule_spa_d(const double *in, int32_t d, int32_t j) {
  int s = 1;
  double sum = 0.0;
  for (int32_t t = 0; t < d; ++t) {
    if (t == j) continue;
    s *= sgn_d(in[t]);
    double a = fabs(in[t]);
    if (a > ORC_SPA_SAT) a = ORC_SPA_SAT;
    sum += phi_d(a);
  }
  return s == 0 ? 0.0 : (double)s * phi_d(sum);
}

/* ------------------------------------------------------- integer, one frame */

typedef struct {
  int64_t *Z, *Zprev, *L, *Zmn, *u, *Lraw;
  int64_t *A, *B;
  int32_t *nt;
  int8_t *s;
  uint8_t *x;
} iscratch;

static void decode_frame_int(const orc_code *c, const orc_csc *t, const orc_iparams *p,
                             int32_t form, const int32_t *q0, iscratch *w, uint8_t *bits,
                             int32_t *iters, uint8_t *ok, int32_t *z_out, int32_t *l_out,
                             int32_t *state_out) {
  const int32_t N = c->n_vars, M = c->n_checks, E = c->row_ptr[M];
  const int32_t *rp = c->row_ptr, *ci = c->col_idx;
  int64_t *Z = w->Z, *Zprev = w->Zprev, *L = w->L;

  /* k = 0: Z^(0)_n = q0_n, L^(0) = 0 (Section IV initialization; Section III
     initialization Z^(0)_mn = Z^(0)_n). */
  for (int32_t n = 0; n < N; ++n) Z[n] = q0[n];
  for (int32_t e = 0; e < E; ++e) { L[e] = 0; w->Zmn[e] = q0[ci[e]]; w->s[e] = 0; }
  for (int32_t m = 0; m < M; ++m) { w->A[m] = 0; w->B[m] = 0; w->nt[m] = 0; }

  int32_t k = 0;
  int sat = decide_and_check(c, Z, NULL, w->x);
  if (!(p->early_stop && sat)) {
    for (k = 1; k <= p->max_iter; ++k) {
      memcpy(Zprev, Z, sizeof(int64_t) * (size_t)N);
      if (form == ORC_TWO_SCAN) {
        /* Horizontal scan, Eq. (1), then the normalized/offset modification. */
        for (int32_t m = 0; m < M; ++m) {
          int32_t d = rp[m + 1] - rp[m];
          for (int32_t j = 0; j < d; ++j) w->u[j] = w->Zmn[rp[m] + j];
          for (int32_t j = 0; j < d; ++j) {
            int64_t l = check_rule_i(p, w->u, d, j);
            L[rp[m] + j] = sgn_i(l) * modify_i(p, l < 0 ? -l : l);
          }
        }
        /* Vertical scan, Eq. (2): Z_mn = Z0_n + sum over M(n)\m of L_m'n. */
        for (int32_t n = 0; n < N; ++n) {
          for (int32_t a = t->col_ptr[n]; a < t->col_ptr[n + 1]; ++a) {
            int64_t acc = q0[n];
            for (int32_t b = t->col_ptr[n]; b < t->col_ptr[n + 1]; ++b)
              if (b != a) acc += L[t->edge[b]];
            w->Zmn[t->edge[a]] = acc;
          }
          /* Decoding step: Z_n = Z0_n + sum over M(n) of L_mn. */
          int64_t post = q0[n];
          for (int32_t b = t->col_ptr[n]; b < t->col_ptr[n + 1]; ++b) post += L[t->edge[b]];
          Z[n] = post;
        }
      } else if (form == ORC_SS_FIXED) {
        /* Eq. (3): Z^(k)_n = Z^(0)_n; per check, L^(k)_mn from
           Z^(k-1)_n' - L^(k-1)_mn'; then Z^(k)_n += L^(k)_mn. */
        for (int32_t n = 0; n < N; ++n) Z[n] = q0[n];
        for (int32_t m = 0; m < M; ++m) {
          int32_t d = rp[m + 1] - rp[m];
          for (int32_t j = 0; j < d; ++j) w->u[j] = Zprev[ci[rp[m] + j]] - L[rp[m] + j];
          for (int32_t j = 0; j < d; ++j) {
            int64_t l = check_rule_i(p, w->u, d, j);
            w->Lraw[j] = sgn_i(l) * modify_i(p, l < 0 ? -l : l);
          }
          for (int32_t j = 0; j < d; ++j) {
            L[rp[m] + j] = w->Lraw[j];
            Z[ci[rp[m] + j]] += w->Lraw[j];
          }
        }
      } else {
        /* Section V: rebuild L^(k-1)_mn = s f(A, B, n, n~), apply Eq. (3),
           then store A = g(min |L|), B = g(max |L|), n~ = argmax |L|, s = sgn L
           (Eqs. (4), (5) with the normalized/offset change), and accumulate
           the stored message into Z. */
        for (int32_t n = 0; n < N; ++n) Z[n] = q0[n];
        for (int32_t m = 0; m < M; ++m) {
          int32_t d = rp[m + 1] - rp[m];
          for (int32_t j = 0; j < d; ++j) {
            int64_t f = (j == w->nt[m]) ? w->B[m] : w->A[m];
            int64_t lold = (int64_t)w->s[rp[m] + j] * f;
            w->u[j] = Zprev[ci[rp[m] + j]] - lold;
          }
          for (int32_t j = 0; j < d; ++j) w->Lraw[j] = check_rule_i(p, w->u, d, j);
          int64_t amin = -1, amax = -1;
          int32_t arg = 0;
          for (int32_t j = 0; j < d; ++j) {
            int64_t a = w->Lraw[j] < 0 ? -w->Lraw[j] : w->Lraw[j];
            if (amin < 0 || a < amin) amin = a;
            if (a > amax) { amax = a; arg = j; }
          }
          w->A[m] = modify_i(p, amin);
          w->B[m] = modify_i(p, amax);
          w->nt[m] = arg;
          for (int32_t j = 0; j < d; ++j) {
            w->s[rp[m] + j] = (int8_t)sgn_i(w->Lraw[j]);
            int64_t f = (j == arg) ? w->B[m] : w->A[m];
            int64_t lnew = (int64_t)w->s[rp[m] + j] * f;
            L[rp[m] + j] = lnew;
            Z[ci[rp[m] + j]] += lnew;
          }
        }
      }
      if (form != ORC_TWO_SCAN) sat_post(p, Z, N);
      sat = decide_and_check(c, Z, NULL, w->x);
      if (p->early_stop && sat) break;
    }
    if (k > p->max_iter) k = p->max_iter;
  }
  *iters = k;
  *ok = (uint8_t)sat;
  for (int32_t n = 0; n < N; ++n) { bits[n] = w->x[n]; z_out[n] = (int32_t)Z[n]; }
  if (l_out)
    for (int32_t e = 0; e < E; ++e) l_out[e] = (int32_t)L[e];
  if (state_out && form == ORC_SS_1BIT) {
    for (int32_t m = 0; m < M; ++m) {
      int32_t sw = 0;
      for (int32_t j = 0; j < rp[m + 1] - rp[m]; ++j)
        if (w->s[rp[m] + j] < 0) sw |= (int32_t)(1u << j);
      state_out[4 * m + 0] = (int32_t)w->A[m];
      state_out[4 * m + 1] = (int32_t)w->B[m];
      state_out[4 * m + 2] = w->nt[m];
      state_out[4 * m + 3] = sw;
    }
  }
}

/* ------------------------------------------- integer, layered, one frame */

/* The single scan of Eq. (3) in a layered schedule (cited in Section I; not
   the paper's own schedule): the checks are split into layers whose checks
   share no variable; within an iteration the layers run in order and each
   check of a layer reads the posteriors as the previous layers left them,
   computes its new messages from Z_n - L_mn and writes Z_n = (Z_n - L_mn) +
   L_new_mn in place.  Checks of one layer touch disjoint variables, so their
   order within the layer does not matter.  The stop rule is the paper's: the
   decisions of Z after a whole iteration (and before the first). */
static void decode_frame_layered_int(const orc_code *c, const orc_iparams *p, const int32_t *layer,
                                     int32_t n_layers, const int32_t *q0, iscratch *w, uint8_t *bits,
                                     int32_t *iters, uint8_t *ok, int32_t *z_out, int32_t *l_out) {
  const int32_t N = c->n_vars, M = c->n_checks, E = c->row_ptr[M];
  const int32_t *rp = c->row_ptr, *ci = c->col_idx;
  int64_t *Z = w->Z, *L = w->L;
  for (int32_t n = 0; n < N; ++n) Z[n] = q0[n];
  for (int32_t e = 0; e < E; ++e) L[e] = 0;
  int32_t k = 0;
  int sat = decide_and_check(c, Z, NULL, w->x);
  if (!(p->early_stop && sat)) {
    for (k = 1; k <= p->max_iter; ++k) {
      for (int32_t l = 0; l < n_layers; ++l) {
        for (int32_t m = 0; m < M; ++m) {
          if (layer[m] != l) continue;
          int32_t d = rp[m + 1] - rp[m];
          for (int32_t j = 0; j < d; ++j) w->u[j] = Z[ci[rp[m] + j]] - L[rp[m] + j];
          for (int32_t j = 0; j < d; ++j) {
            int64_t v = check_rule_i(p, w->u, d, j);
            w->Lraw[j] = sgn_i(v) * modify_i(p, v < 0 ? -v : v);
          }
          for (int32_t j = 0; j < d; ++j) {
            L[rp[m] + j] = w->Lraw[j];
            Z[ci[rp[m] + j]] = w->u[j] + w->Lraw[j];
          }
        }
      }
      sat = decide_and_check(c, Z, NULL, w->x);
      if (p->early_stop && sat) break;
    }
    if (k > p->max_iter) k = p->max_iter;
  }
  *iters = k;
  *ok = (uint8_t)sat;
  for (int32_t n = 0; n < N; ++n) { bits[n] = w->x[n]; z_out[n] = (int32_t)Z[n]; }
  if (l_out)
    for (int32_t e = 0; e < E; ++e) l_out[e] = (int32_t)L[e];
}

/* -------------------------------------------------- double, one frame */

typedef struct {
  double *Z, *Zprev, *L, *Zmn, *u, *Lraw, *A, *B;
  int32_t *nt;
  int8_t *s;
  uint8_t *x;
} dscratch;

static void decode_frame_f64(const orc_code *c, const orc_csc *t, const orc_dparams *p,
                             int32_t form, const double *q0, dscratch *w, uint8_t *bits,
                             int32_t *iters, uint8_t *ok, double *z_out, double *l_out,
                             double *margin) {
  double mg = INFINITY;
  const int32_t N = c->n_vars, M = c->n_checks, E = c->row_ptr[M];
  const int32_t *rp = c->row_ptr, *ci = c->col_idx;
  double *Z = w->Z, *Zprev = w->Zprev, *L = w->L;

  for (int32_t n = 0; n < N; ++n) Z[n] = q0[n];
  for (int32_t e = 0; e < E; ++e) { L[e] = 0.0; w->Zmn[e] = q0[ci[e]]; w->s[e] = 0; }
  for (int32_t m = 0; m < M; ++m) { w->A[m] = 0.0; w->B[m] = 0.0; w->nt[m] = 0; }

  int32_t k = 0;
  int sat = decide_and_check(c, NULL, Z, w->x);
  for (int32_t n = 0; n < N; ++n) if (fabs(Z[n]) < mg) mg = fabs(Z[n]);
  if (!(p->early_stop && sat)) {
    for (k = 1; k <= p->max_iter; ++k) {
      memcpy(Zprev, Z, sizeof(double) * (size_t)N);
      if (form == ORC_TWO_SCAN) {
        for (int32_t m = 0; m < M; ++m) {
          int32_t d = rp[m + 1] - rp[m];
          for (int32_t j = 0; j < d; ++j) w->u[j] = w->Zmn[rp[m] + j];
          for (int32_t j = 0; j < d; ++j) {
            double l = p->rule == ORC_SUM_PRODUCT ? check_rule_spa_d(w->u, d, j) : check_rule_d(w->u, d, j);
            L[rp[m] + j] = sgn_d(l) * modify_d(p, k, m, M, fabs(l));
          }
        }
        for (int32_t n = 0; n < N; ++n) {
          for (int32_t a = t->col_ptr[n]; a < t->col_ptr[n + 1]; ++a) {
            double acc = q0[n];
            for (int32_t b = t->col_ptr[n]; b < t->col_ptr[n + 1]; ++b)
              if (b != a) acc += L[t->edge[b]];
            w->Zmn[t->edge[a]] = acc;
          }
          double post = q0[n];
          for (int32_t b = t->col_ptr[n]; b < t->col_ptr[n + 1]; ++b) post += L[t->edge[b]];
          Z[n] = post;
        }
      } else if (form == ORC_SS_FIXED) {
        for (int32_t n = 0; n < N; ++n) Z[n] = q0[n];
        for (int32_t m = 0; m < M; ++m) {
          int32_t d = rp[m + 1] - rp[m];
          for (int32_t j = 0; j < d; ++j) w->u[j] = Zprev[ci[rp[m] + j]] - L[rp[m] + j];
          for (int32_t j = 0; j < d; ++j) {
            double l = p->rule == ORC_SUM_PRODUCT ? check_rule_spa_d(w->u, d, j) : check_rule_d(w->u, d, j);
            w->Lraw[j] = sgn_d(l) * modify_d(p, k, m, M, fabs(l));
          }
          for (int32_t j = 0; j < d; ++j) {
            L[rp[m] + j] = w->Lraw[j];
            Z[ci[rp[m] + j]] += w->Lraw[j];
          }
        }
      } else {
        for (int32_t n = 0; n < N; ++n) Z[n] = q0[n];
        for (int32_t m = 0; m < M; ++m) {
          int32_t d = rp[m + 1] - rp[m];
          for (int32_t j = 0; j < d; ++j) {
            double f = (j == w->nt[m]) ? w->B[m] : w->A[m];
            w->u[j] = Zprev[ci[rp[m] + j]] - (double)w->s[rp[m] + j] * f;
          }
          for (int32_t j = 0; j < d; ++j) w->Lraw[j] = check_rule_d(w->u, d, j);
          double amin = INFINITY, amax = -1.0;
          int32_t arg = 0;
          for (int32_t j = 0; j < d; ++j) {
            double a = fabs(w->Lraw[j]);
            if (a < amin) amin = a;
            if (a > amax) { amax = a; arg = j; }
          }
          w->A[m] = modify_d(p, k, m, M, amin);
          w->B[m] = modify_d(p, k, m, M, amax);
          w->nt[m] = arg;
          for (int32_t j = 0; j < d; ++j) {
            w->s[rp[m] + j] = (int8_t)sgn_d(w->Lraw[j]);
            double f = (j == arg) ? w->B[m] : w->A[m];
            double lnew = (double)w->s[rp[m] + j] * f;
            L[rp[m] + j] = lnew;
            Z[ci[rp[m] + j]] += lnew;
          }
        }
      }
      sat = decide_and_check(c, NULL, Z, w->x);
      for (int32_t n = 0; n < N; ++n) if (fabs(Z[n]) < mg) mg = fabs(Z[n]);
      if (p->early_stop && sat) break;
    }
    if (k > p->max_iter) k = p->max_iter;
  }
  *iters = k;
  *ok = (uint8_t)sat;
  for (int32_t n = 0; n < N; ++n) { bits[n] = w->x[n]; z_out[n] = Z[n]; }
  if (l_out)
    for (int32_t e = 0; e < E; ++e) l_out[e] = L[e];
  if (margin) *margin = mg;
}

/* ------------------------------------------------------------ threading */

typedef struct {
  const orc_code *c;
  const orc_csc *t;
  int32_t form;
  int is_int;
  const orc_iparams *ip;
  const orc_dparams *dp;
  const void *q0;
  int32_t f0, f1;
  uint8_t *bits;
  int32_t *iters;
  uint8_t *ok;
  void *z_out, *l_out;
  int32_t *state_out;
  double *margin_out;
  const int32_t *layer; /* layered schedule: layer of every check (else NULL) */
  int32_t n_layers;
  int err;
} job;

static int32_t max_row_degree(const orc_code *c) {
  int32_t dmax = 0;
  for (int32_t m = 0; m < c->n_checks; ++m)
    if (c->row_ptr[m + 1] - c->row_ptr[m] > dmax) dmax = c->row_ptr[m + 1] - c->row_ptr[m];
  return dmax;
}

static void *run_job(void *arg) {
  job *jb = (job *)arg;
  const orc_code *c = jb->c;
  size_t N = (size_t)c->n_vars, M = (size_t)c->n_checks, E = (size_t)c->row_ptr[c->n_checks];
  size_t D = (size_t)max_row_degree(c) + 1;
  if (jb->is_int) {
    iscratch w;
    w.Z = malloc(sizeof(int64_t) * (N + 1)); w.Zprev = malloc(sizeof(int64_t) * (N + 1));
    w.L = malloc(sizeof(int64_t) * (E + 1)); w.Zmn = malloc(sizeof(int64_t) * (E + 1));
    w.u = malloc(sizeof(int64_t) * D); w.Lraw = malloc(sizeof(int64_t) * D);
    w.A = malloc(sizeof(int64_t) * (M + 1)); w.B = malloc(sizeof(int64_t) * (M + 1));
    w.nt = malloc(sizeof(int32_t) * (M + 1)); w.s = malloc(E + 1); w.x = malloc(N + 1);
    if (!w.Z || !w.Zprev || !w.L || !w.Zmn || !w.u || !w.Lraw || !w.A || !w.B || !w.nt || !w.s || !w.x) {
      jb->err = -1;
    } else {
      const int32_t *q0 = (const int32_t *)jb->q0;
      for (int32_t f = jb->f0; f < jb->f1 && jb->layer; ++f)
        decode_frame_layered_int(c, jb->ip, jb->layer, jb->n_layers, q0 + (size_t)f * N, &w,
                                 jb->bits + (size_t)f * N, jb->iters + f, jb->ok + f,
                                 (int32_t *)jb->z_out + (size_t)f * N,
                                 jb->l_out ? (int32_t *)jb->l_out + (size_t)f * E : NULL);
      for (int32_t f = jb->f0; f < jb->f1 && !jb->layer; ++f)
        decode_frame_int(c, jb->t, jb->ip, jb->form, q0 + (size_t)f * N, &w, jb->bits + (size_t)f * N,
                         jb->iters + f, jb->ok + f, (int32_t *)jb->z_out + (size_t)f * N,
                         jb->l_out ? (int32_t *)jb->l_out + (size_t)f * E : NULL,
                         jb->state_out ? jb->state_out + (size_t)f * M * 4 : NULL);
    }
    free(w.Z); free(w.Zprev); free(w.L); free(w.Zmn); free(w.u); free(w.Lraw);
    free(w.A); free(w.B); free(w.nt); free(w.s); free(w.x);
  } else {
    dscratch w;
    w.Z = malloc(sizeof(double) * (N + 1)); w.Zprev = malloc(sizeof(double) * (N + 1));
    w.L = malloc(sizeof(double) * (E + 1)); w.Zmn = malloc(sizeof(double) * (E + 1));
    w.u = malloc(sizeof(double) * D); w.Lraw = malloc(sizeof(double) * D);
    w.A = malloc(sizeof(double) * (M + 1)); w.B = malloc(sizeof(double) * (M + 1));
    w.nt = malloc(sizeof(int32_t) * (M + 1)); w.s = malloc(E + 1); w.x = malloc(N + 1);
    if (!w.Z || !w.Zprev || !w.L || !w.Zmn || !w.u || !w.Lraw || !w.A || !w.B || !w.nt || !w.s || !w.x) {
      jb->err = -1;
    } else {
      const double *q0 = (const double *)jb->q0;
      for (int32_t f = jb->f0; f < jb->f1; ++f)
        decode_frame_f64(c, jb->t, jb->dp, jb->form, q0 + (size_t)f * N, &w, jb->bits + (size_t)f * N,
                         jb->iters + f, jb->ok + f, (double *)jb->z_out + (size_t)f * N,
                         jb->l_out ? (double *)jb->l_out + (size_t)f * E : NULL,
                         jb->margin_out ? jb->margin_out + f : NULL);
    }
    free(w.Z); free(w.Zprev); free(w.L); free(w.Zmn); free(w.u); free(w.Lraw);
    free(w.A); free(w.B); free(w.nt); free(w.s); free(w.x);
  }
  return NULL;
}

int32_t orc_default_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int32_t)n : 1;
}

static int validate(const orc_code *c, int32_t form) {
  if (!c || c->n_vars < 0 || c->n_checks < 0 || !c->row_ptr) return -1;
  if (form < ORC_TWO_SCAN || form > ORC_SS_1BIT) return -1;
  if (c->row_ptr[0] != 0) return -1;
  for (int32_t m = 0; m < c->n_checks; ++m) {
    int32_t d = c->row_ptr[m + 1] - c->row_ptr[m];
    if (d < 2 || d > 32) return -1; /* empty N(m)\n is undefined in Eq. (1) */
    for (int32_t e = c->row_ptr[m]; e < c->row_ptr[m + 1]; ++e)
      if (c->col_idx[e] < 0 || c->col_idx[e] >= c->n_vars) return -1;
  }
  return 0;
}

static int run_all(job *proto, int32_t n_frames, int32_t n_threads) {
  if (n_threads <= 0) n_threads = orc_default_threads();
  if (n_threads > n_frames) n_threads = n_frames > 0 ? n_frames : 1;
  orc_csc t = {0, 0};
  if (build_csc(proto->c, &t)) { free_csc(&t); return -1; }
  proto->t = &t;
  job *jobs = (job *)calloc((size_t)n_threads, sizeof(job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  int err = (!jobs || !th) ? -1 : 0;
  int32_t started = 0;
  for (int32_t i = 0; i < n_threads && !err; ++i) {
    jobs[i] = *proto;
    jobs[i].f0 = (int32_t)((int64_t)n_frames * i / n_threads);
    jobs[i].f1 = (int32_t)((int64_t)n_frames * (i + 1) / n_threads);
    if (pthread_create(&th[i], NULL, run_job, &jobs[i])) err = -1;
    else started++;
  }
  for (int32_t i = 0; i < started; ++i) {
    pthread_join(th[i], NULL);
    if (jobs[i].err) err = -1;
  }
  free(jobs); free(th); free_csc(&t);
  return err;
}

int orc_decode_int(const orc_code *code, const orc_iparams *p, int32_t form, const int32_t *q0,
                   int32_t n_frames, uint8_t *bits, int32_t *iters, uint8_t *ok, int32_t *z_out,
                   int32_t *l_out, int32_t *state_out, int32_t n_threads) {
  if (validate(code, form) || !p || p->max_iter < 0 || n_frames < 0) return -1;
  if (form == ORC_TWO_SCAN && p->post_sat > 0) return -1; /* Z_mn, not a stored Z_n */
  if (n_frames == 0) return 0;
  if (!q0 || !bits || !iters || !ok || !z_out) return -1;
  job proto;
  memset(&proto, 0, sizeof proto);
  proto.c = code; proto.form = form; proto.is_int = 1; proto.ip = p; proto.q0 = q0;
  proto.bits = bits; proto.iters = iters; proto.ok = ok; proto.z_out = z_out;
  proto.l_out = l_out; proto.state_out = state_out;
  return run_all(&proto, n_frames, n_threads);
}

int orc_decode_layered_int(const orc_code *code, const orc_iparams *p, const int32_t *layer, int32_t n_layers,
                           const int32_t *q0, int32_t n_frames, uint8_t *bits, int32_t *iters, uint8_t *ok,
                           int32_t *z_out, int32_t *l_out, int32_t n_threads) {
  if (validate(code, ORC_SS_FIXED) || !p || p->max_iter < 0 || n_frames < 0 || !layer || n_layers < 1) return -1;
  if (p->post_sat > 0) return -1; /* the layered update keeps Z exact */
  /* every check in a layer; the checks of a layer share no variable */
  int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * ((size_t)code->n_vars * (size_t)n_layers + 1));
  if (!owner) return -1;
  for (size_t i = 0; i < (size_t)code->n_vars * (size_t)n_layers; ++i) owner[i] = -1;
  int bad = 0;
  for (int32_t m = 0; m < code->n_checks && !bad; ++m) {
    if (layer[m] < 0 || layer[m] >= n_layers) { bad = 1; break; }
    for (int32_t e = code->row_ptr[m]; e < code->row_ptr[m + 1]; ++e) {
      int32_t *o = &owner[(size_t)layer[m] * code->n_vars + code->col_idx[e]];
      if (*o >= 0) { bad = 1; break; }
      *o = m;
    }
  }
  free(owner);
  if (bad) return -1;
  if (n_frames == 0) return 0;
  if (!q0 || !bits || !iters || !ok || !z_out) return -1;
  job proto;
  memset(&proto, 0, sizeof proto);
  proto.c = code; proto.form = ORC_SS_FIXED; proto.is_int = 1; proto.ip = p; proto.q0 = q0;
  proto.bits = bits; proto.iters = iters; proto.ok = ok; proto.z_out = z_out; proto.l_out = l_out;
  proto.layer = layer; proto.n_layers = n_layers;
  return run_all(&proto, n_frames, n_threads);
}

int orc_decode_f64(const orc_code *code, const orc_dparams *p, int32_t form, const double *q0,
                   int32_t n_frames, uint8_t *bits, int32_t *iters, uint8_t *ok, double *z_out,
                   double *l_out, int32_t n_threads) {
  if (p && p->rule == ORC_SUM_PRODUCT && form == ORC_SS_1BIT) return -1; /* messages are not (A, B) pairs */
  return orc_decode_f64_margin(code, p, form, q0, n_frames, bits, iters, ok, z_out, l_out, NULL, n_threads);
}

int orc_decode_f64_margin(const orc_code *code, const orc_dparams *p, int32_t form, const double *q0,
                          int32_t n_frames, uint8_t *bits, int32_t *iters, uint8_t *ok, double *z_out,
                          double *l_out, double *margin_out, int32_t n_threads) {
  if (p && p->rule == ORC_SUM_PRODUCT && form == ORC_SS_1BIT) return -1;
  if (validate(code, form) || !p || p->max_iter < 0 || n_frames < 0) return -1;
  if (n_frames == 0) return 0;
  if (!q0 || !bits || !iters || !ok || !z_out) return -1;
  job proto;
  memset(&proto, 0, sizeof proto);
  proto.c = code; proto.form = form; proto.is_int = 0; proto.dp = p; proto.q0 = q0;
  proto.bits = bits; proto.iters = iters; proto.ok = ok; proto.z_out = z_out; proto.l_out = l_out;
  proto.margin_out = margin_out;
  return run_all(&proto, n_frames, n_threads);
}

/* --------------------------------------------------- learned offsets (FP64) */

typedef struct {
  const orc_code *c;
  int32_t K;
  const double *beta;
  const double *q0;
  const uint8_t *tg;
  int32_t f0, f1;
  double loss;
  double *dbeta; /* [K][M], this thread's sum */
  double *gap;
  int err;
} ljob;

static double softplus(double x) { return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }

static void *run_ljob(void *arg) {
  ljob *jb = (ljob *)arg;
  const orc_code *c = jb->c;
  const int32_t N = c->n_vars, M = c->n_checks, E = c->row_ptr[M], K = jb->K;
  const int32_t *rp = c->row_ptr, *ci = c->col_idx;
  /* forward record: u[k-1][e] (k = 1..K), L[k][e] (k = 0..K), Z[k][n] (k = 0..K) */
  double *u = malloc(sizeof(double) * (size_t)K * E);
  double *L = malloc(sizeof(double) * (size_t)(K + 1) * E);
  double *Z = malloc(sizeof(double) * (size_t)(K + 1) * N);
  double *gZ = malloc(sizeof(double) * (size_t)N);   /* dLoss/dZ^(k) */
  double *gZp = malloc(sizeof(double) * (size_t)N);  /* dLoss/dZ^(k-1) */
  double *gLx = malloc(sizeof(double) * (size_t)E);  /* dLoss/dL^(k) through u^(k+1) */
  double *gL = malloc(sizeof(double) * (size_t)E);   /* total dLoss/dL^(k) */
  double *gu = malloc(sizeof(double) * (size_t)E);   /* dLoss/du^(k) */
  if (!u || !L || !Z || !gZ || !gZp || !gLx || !gL || !gu) { jb->err = -1; goto done; }
  for (int32_t f = jb->f0; f < jb->f1; ++f) {
    const double *q = jb->q0 + (size_t)f * N;
    double g = INFINITY;
    /* forward: Eq. (3) with the per-iteration, per-check offset */
    for (int32_t e = 0; e < E; ++e) L[e] = 0.0; /* L^(0) = 0 */
    for (int32_t n = 0; n < N; ++n) Z[n] = q[n];
    for (int32_t k = 1; k <= K; ++k) {
      double *uk = u + (size_t)(k - 1) * E, *Lk = L + (size_t)k * E, *Lp = L + (size_t)(k - 1) * E;
      double *Zk = Z + (size_t)k * N, *Zp = Z + (size_t)(k - 1) * N;
      for (int32_t n = 0; n < N; ++n) Zk[n] = q[n];
      for (int32_t m = 0; m < M; ++m) {
        const double bt = jb->beta[(size_t)(k - 1) * M + m];
        const int32_t d = rp[m + 1] - rp[m];
        for (int32_t j = 0; j < d; ++j) uk[rp[m] + j] = Zp[ci[rp[m] + j]] - Lp[rp[m] + j];
        double a1 = INFINITY, a2 = INFINITY;
        for (int32_t j = 0; j < d; ++j) {
          const double a = fabs(uk[rp[m] + j]);
          if (a < g) g = a;
          if (a < a1) { a2 = a1; a1 = a; } else if (a < a2) a2 = a;
        }
        if (a2 - a1 < g) g = a2 - a1;
        if (fabs(a1 - bt) < g) g = fabs(a1 - bt);
        if (fabs(a2 - bt) < g) g = fabs(a2 - bt);
        for (int32_t j = 0; j < d; ++j) {
          double sg = 1.0, mn = INFINITY;
          for (int32_t t = 0; t < d; ++t) {
            if (t == j) continue;
            const double v = uk[rp[m] + t];
            sg *= (v > 0) - (v < 0);
            if (fabs(v) < mn) mn = fabs(v);
          }
          const double l = sg * (mn > bt ? mn - bt : 0.0);
          Lk[rp[m] + j] = l;
          Zk[ci[rp[m] + j]] += l;
        }
      }
    }
    /* loss and dLoss/dZ^(K) */
    const double *ZK = Z + (size_t)K * N;
    for (int32_t n = 0; n < N; ++n) {
      const int t = jb->tg ? jb->tg[(size_t)f * N + n] : 0;
      jb->loss += softplus(t ? ZK[n] : -ZK[n]);
      gZ[n] = t ? sigm(ZK[n]) : sigm(ZK[n]) - 1.0;
    }
    for (int32_t e = 0; e < E; ++e) gLx[e] = 0.0;
    /* reverse sweep over the iterations */
    for (int32_t k = K; k >= 1; --k) {
      const double *uk = u + (size_t)(k - 1) * E;
      /* Z^(k) = Z0 + sum_m L^(k): every message receives its variable's gradient */
      for (int32_t e = 0; e < E; ++e) { gL[e] = gZ[ci[e]] + gLx[e]; gu[e] = 0.0; }
      for (int32_t m = 0; m < M; ++m) {
        const double bt = jb->beta[(size_t)(k - 1) * M + m];
        const int32_t d = rp[m + 1] - rp[m];
        for (int32_t j = 0; j < d; ++j) {
          double sg = 1.0, mn = INFINITY;
          int32_t arg = -1;
          for (int32_t t = 0; t < d; ++t) {
            if (t == j) continue;
            const double v = uk[rp[m] + t];
            sg *= (v > 0) - (v < 0);
            if (fabs(v) < mn) { mn = fabs(v); arg = t; }
          }
          if (!(mn > bt)) continue; /* the offset's max(., 0) is inactive */
          const double gl = gL[rp[m] + j];
          jb->dbeta[(size_t)(k - 1) * M + m] -= gl * sg;          /* dL/dbeta = -sg */
          const double v = uk[rp[m] + arg];
          gu[rp[m] + arg] += gl * sg * (v < 0 ? -1.0 : 1.0);      /* dL/du_arg = sg sgn(u_arg) */
        }
      }
      /* u^(k)_e = Z^(k-1)_n - L^(k-1)_e */
      for (int32_t n = 0; n < N; ++n) gZp[n] = 0.0;
      for (int32_t e = 0; e < E; ++e) { gZp[ci[e]] += gu[e]; gLx[e] = -gu[e]; }
      for (int32_t n = 0; n < N; ++n) gZ[n] = gZp[n];
    }
    if (jb->gap) jb->gap[f] = g;
  }
done:
  free(u); free(L); free(Z); free(gZ); free(gZp); free(gLx); free(gL); free(gu);
  return NULL;
}

int orc_learned_grad_f64(const orc_code *code, int32_t n_iters, const double *beta_tab, const double *q0,
                         const uint8_t *targets, int32_t n_frames, double *loss_sum, double *dbeta,
                         double *gap, int32_t n_threads) {
  if (validate(code, ORC_SS_FIXED) || n_iters < 1 || !beta_tab || !q0 || n_frames < 0 || !loss_sum || !dbeta)
    return -1;
  const int32_t M = code->n_checks;
  const size_t nb = (size_t)n_iters * M;
  for (size_t i = 0; i < nb; ++i) dbeta[i] = 0.0;
  *loss_sum = 0.0;
  if (n_frames == 0) return 0;
  if (n_threads <= 0) n_threads = orc_default_threads();
  if (n_threads > n_frames) n_threads = n_frames;
  ljob *jobs = (ljob *)calloc((size_t)n_threads, sizeof(ljob));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  int err = (!jobs || !th) ? -1 : 0;
  int32_t started = 0;
  for (int32_t i = 0; i < n_threads && !err; ++i) {
    jobs[i].c = code; jobs[i].K = n_iters; jobs[i].beta = beta_tab; jobs[i].q0 = q0; jobs[i].tg = targets;
    jobs[i].f0 = (int32_t)((int64_t)n_frames * i / n_threads);
    jobs[i].f1 = (int32_t)((int64_t)n_frames * (i + 1) / n_threads);
    jobs[i].gap = gap;
    jobs[i].dbeta = (double *)calloc(nb, sizeof(double));
    if (!jobs[i].dbeta) { err = -1; break; }
    if (pthread_create(&th[i], NULL, run_ljob, &jobs[i])) err = -1;
    else started++;
  }
  for (int32_t i = 0; i < started; ++i) {
    pthread_join(th[i], NULL);
    if (jobs[i].err) err = -1;
  }
  /* sum in thread order (each thread's frames in order): deterministic */
  for (int32_t i = 0; i < started && !err; ++i) {
    *loss_sum += jobs[i].loss;
    for (size_t t = 0; t < nb; ++t) dbeta[t] += jobs[i].dbeta[t];
  }
  for (int32_t i = 0; i < n_threads; ++i) free(jobs ? jobs[i].dbeta : NULL);
  free(jobs); free(th);
  return err;
}

// ldpc_api.cu -- the C ABI (include/ldpc_gb300.h): argument checks, the device
// copy of a code, kernel selection and error reporting.  No kernel logic here.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"


namespace {
thread_local std::string g_last_error;
}  // namespace

namespace ldpc_api {

void clear_error() { g_last_error.clear(); }

ldpc_status fail(ldpc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

ldpc_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error so later calls start clean
  return fail(e == cudaErrorMemoryAllocation ? LDPC_ERR_OOM : LDPC_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

ldpc::DevCode view(const ldpc_code* c) {
  ldpc::DevCode v;
  v.N = c->N;
  v.M = c->M;
  v.E = c->E;
  v.rp = c->d_rp;
  v.ci = c->d_ci;
  v.cdeg = c->d_cdeg;
  v.ell16 = c->d_ell16;
  v.ell32 = c->d_ell32;
  v.rdeg = c->d_rdeg;
  v.ell_w = c->ell_w;
  v.cptr = c->d_cptr;
  v.cslot = c->d_cslot;
  v.ccj = c->d_ccj;
  v.n_dc = c->n_dc;
  for (int i = 0; i < 4; ++i) {
    v.dc_end[i] = c->dc_end[i];
    v.dc_deg[i] = c->dc_deg[i];
  }
  return v;
}

ldpc_status set_layers(ldpc_code* c, int32_t n_layers, const int32_t* layer_of_check) {
  const int32_t M = c->M, N = c->N;
  if (n_layers < 1 || n_layers > M || layer_of_check == nullptr)
    return fail(LDPC_ERR_INVALID_ARG, "n_layers %d outside [1, %d] or layer_of_check NULL", n_layers, M);
  std::vector<int32_t> owner((size_t)N, -1), count((size_t)n_layers + 1, 0);
  std::vector<int32_t> seen_layer((size_t)N, -1);
  for (int32_t m = 0; m < M; ++m) {
    const int32_t l = layer_of_check[m];
    if (l < 0 || l >= n_layers) return fail(LDPC_ERR_INVALID_ARG, "check %d in layer %d of %d", m, l, n_layers);
    count[(size_t)l + 1]++;
  }
  // the checks of one layer must share no variable
  std::vector<int32_t> by_layer((size_t)M);
  std::vector<int32_t> fill(count.begin(), count.end() - 1);
  for (int32_t l = 0; l < n_layers; ++l) count[(size_t)l + 1] += count[(size_t)l];
  for (int32_t l = 0; l < n_layers; ++l) fill[(size_t)l] = count[(size_t)l];
  for (int32_t m = 0; m < M; ++m) by_layer[(size_t)fill[(size_t)layer_of_check[m]]++] = m;
  for (int32_t l = 0; l < n_layers; ++l)
    for (int32_t i = count[(size_t)l]; i < count[(size_t)l + 1]; ++i) {
      const int32_t m = by_layer[(size_t)i];
      for (int32_t e = c->h_row_ptr[(size_t)m]; e < c->h_row_ptr[(size_t)m + 1]; ++e) {
        const int32_t n = c->h_col_idx[(size_t)e];
        if (seen_layer[(size_t)n] == l)
          return fail(LDPC_ERR_INVALID_ARG, "layer %d: checks %d and %d share variable %d", l, owner[(size_t)n], m, n);
        seen_layer[(size_t)n] = l;
        owner[(size_t)n] = m;
      }
    }
  // device lists: the internal (degree-sorted) index of every check, per layer
  std::vector<int32_t> rows((size_t)M);
  for (int32_t l = 0; l < n_layers; ++l) {
    for (int32_t i = count[(size_t)l]; i < count[(size_t)l + 1]; ++i)
      rows[(size_t)i] = c->pos[(size_t)by_layer[(size_t)i]];
    std::sort(rows.begin() + count[(size_t)l], rows.begin() + count[(size_t)l + 1]);
  }
  int32_t *dp = nullptr, *dr = nullptr;
  cudaError_t e;
  if ((e = cudaMalloc(&dp, sizeof(int32_t) * ((size_t)n_layers + 1))) != cudaSuccess ||
      (e = cudaMalloc(&dr, sizeof(int32_t) * (size_t)M)) != cudaSuccess ||
      (e = cudaMemcpy(dp, count.data(), sizeof(int32_t) * ((size_t)n_layers + 1), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(dr, rows.data(), sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(dp);
    cudaFree(dr);
    return cuda_fail(e, "layer tables");
  }
  cudaFree(c->d_lay_ptr);
  cudaFree(c->d_lay_rows);
  c->d_lay_ptr = dp;
  c->d_lay_rows = dr;
  c->n_layers = n_layers;
  c->layer_of_check.assign(layer_of_check, layer_of_check + M);
  return LDPC_OK;
}

ldpc_status check_params(const ldpc_code* c, const ldpc_decode_params* p) {
  if (p->dtype != LDPC_DTYPE_INT8 && p->dtype != LDPC_DTYPE_F32)
    return fail(LDPC_ERR_INVALID_ARG, "dtype %d is not LDPC_DTYPE_INT8/F32", p->dtype);
  if (p->form < LDPC_FORM_SS_FIXED || p->form > LDPC_FORM_TWO_SCAN_1BIT)
    return fail(LDPC_ERR_INVALID_ARG, "form %d is not a known LDPC_FORM_*", p->form);
  if (p->rule < LDPC_RULE_PLAIN || p->rule > LDPC_RULE_SUM_PRODUCT)
    return fail(LDPC_ERR_INVALID_ARG, "rule %d is not a known LDPC_RULE_*", p->rule);
  if (p->rule == LDPC_RULE_SUM_PRODUCT &&
      (p->dtype != LDPC_DTYPE_F32 || p->form != LDPC_FORM_SS_FIXED || p->schedule != LDPC_SCHEDULE_FLOODING))
    return fail(LDPC_ERR_UNSUPPORTED, "the sum-product rule runs on the float32 path, SS_FIXED form, flooding");
  if (p->max_iter < 0) return fail(LDPC_ERR_INVALID_ARG, "max_iter %d < 0", p->max_iter);
  if (p->early_stop != 0 && p->early_stop != 1)
    return fail(LDPC_ERR_INVALID_ARG, "early_stop must be 0 or 1");
  if (p->kernel < LDPC_KERNEL_AUTO || p->kernel > LDPC_KERNEL_PINGPONG)
    return fail(LDPC_ERR_INVALID_ARG, "kernel %d is not a known LDPC_KERNEL_*", p->kernel);
  if (p->schedule != LDPC_SCHEDULE_FLOODING && p->schedule != LDPC_SCHEDULE_LAYERED)
    return fail(LDPC_ERR_INVALID_ARG, "schedule %d is not a known LDPC_SCHEDULE_*", p->schedule);
  if (p->posterior != LDPC_POSTERIOR_EXACT && p->posterior != LDPC_POSTERIOR_SAT8)
    return fail(LDPC_ERR_INVALID_ARG, "posterior %d is not a known LDPC_POSTERIOR_*", p->posterior);
  if (p->posterior == LDPC_POSTERIOR_SAT8 &&
      (p->dtype != LDPC_DTYPE_INT8 || (p->form != LDPC_FORM_SS_FIXED && p->form != LDPC_FORM_SS_1BIT) ||
       p->schedule != LDPC_SCHEDULE_FLOODING ||
       (p->kernel != LDPC_KERNEL_AUTO && p->kernel != LDPC_KERNEL_ONCHIP_HALF && p->kernel != LDPC_KERNEL_STREAM)))
    return fail(LDPC_ERR_UNSUPPORTED, "the 8-bit posterior runs int8 single-scan decodes (SS_FIXED or SS_1BIT), "
                "flooding, on kernel AUTO, ONCHIP_HALF or STREAM");
  if (p->dtype == LDPC_DTYPE_INT8) {
    if (p->msg_sat < 1 || p->msg_sat > 127)
      return fail(LDPC_ERR_INVALID_ARG, "msg_sat %d outside [1, 127]", p->msg_sat);
    if (p->rule == LDPC_RULE_OFFSET && (p->offset < 0 || p->offset > 127))
      return fail(LDPC_ERR_INVALID_ARG, "offset %d outside [0, 127]", p->offset);
    if (p->rule == LDPC_RULE_NORMALIZED &&
        (p->norm_shift < 0 || p->norm_shift > 8 || p->norm_num <= 0 || p->norm_num > (1 << p->norm_shift)))
      return fail(LDPC_ERR_INVALID_ARG, "normalization %d/2^%d is not in (0, 1]", p->norm_num,
                  p->norm_shift);
    // The posterior is held exactly in int16: |Z| <= 128 + max_col_degree * Qm.
    if (128 + (int64_t)c->max_col_deg * p->msg_sat > 32767)
      return fail(LDPC_ERR_UNSUPPORTED,
                  "posterior bound 128 + %d * %d exceeds int16; lower msg_sat or the column degree",
                  c->max_col_deg, p->msg_sat);
  } else {
    if (p->rule == LDPC_RULE_OFFSET && !(p->offset_f32 >= 0.0f))
      return fail(LDPC_ERR_INVALID_ARG, "offset_f32 must be >= 0");
    if (p->rule == LDPC_RULE_NORMALIZED && !(p->norm_f32 > 0.0f && p->norm_f32 <= 1.0f))
      return fail(LDPC_ERR_INVALID_ARG, "norm_f32 must be in (0, 1]");
  }
  return LDPC_OK;
}

}  // namespace ldpc_api

using namespace ldpc_api;

namespace {

// Chunks of 32 frame pairs that the persistent decoder takes through all their
// iterations together (their state stays in L2 meanwhile).
#ifndef LDPC_PP_GROUP_CHUNKS
#define LDPC_PP_GROUP_CHUNKS 2
#endif
constexpr int kPersistGroupChunks = LDPC_PP_GROUP_CHUNKS;

// Which kernel serves a request; ws = workspace bytes it needs.
struct Choice {
  enum Kind { NONE, ONCHIP_INT8, ONCHIP_H2, CLUSTER_H2, STREAM_INT8, PERSIST_INT8, PINGPONG_INT8, STREAM_F32,
              ONCHIP_TWOSCAN, STREAM_TWOSCAN, LAYERED } kind = NONE;
  ldpc::OnchipPlan onchip;
  ldpc::StreamLayout stream;
  ldpc::PersistLayout persist;
  ldpc::PingpongLayout pingpong;
  ldpc::TwoScanLayout twoscan;
  ldpc::LayeredLayout layered;
  size_t ws = 0;
};

ldpc_status choose(const ldpc_code* c, const ldpc_decode_params* p, int32_t n_frames, Choice* ch) {
  const ldpc::DevCode v = view(c);
  if (p->schedule == LDPC_SCHEDULE_LAYERED) {
    if (p->dtype != LDPC_DTYPE_INT8 || p->form == LDPC_FORM_TWO_SCAN || p->kernel != LDPC_KERNEL_AUTO)
      return fail(LDPC_ERR_UNSUPPORTED, "the layered schedule runs int8 single-scan decodes (SS_FIXED or SS_1BIT) "
                  "with kernel = LDPC_KERNEL_AUTO");
    if (!ldpc::onchip_h2_eligible(65535, c->max_row_deg, c->max_col_deg, p->msg_sat, p->rule, p->norm_num))
      return fail(LDPC_ERR_UNSUPPORTED, "the layered schedule needs row degree <= 16 and "
                  "128 + (max_col_degree + 1) * msg_sat <= 2048");
    const int form = p->form == LDPC_FORM_SS_1BIT ? 1 : 0;
    ch->kind = Choice::LAYERED;
    ch->layered = ldpc::layered_layout(form, c->N, c->M, c->ell_w, n_frames, c->d_ell16 != nullptr, c->smem_optin);
    ch->ws = ch->layered.total;
    return LDPC_OK;
  }
  if (p->dtype == LDPC_DTYPE_INT8 && (p->form == LDPC_FORM_SS_1BIT || p->form == LDPC_FORM_SS_FIXED)) {
    const int form = p->form == LDPC_FORM_SS_1BIT ? 1 : 0;
    // the 8-bit posterior is clamped where a column pass writes it: the packed
    // frame-resident kernel and the two-launch streaming kernel
    const bool exact = p->posterior == LDPC_POSTERIOR_EXACT;
    const bool want_half = p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_ONCHIP_HALF;
    const bool want_int = exact && (p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_ONCHIP_INT);
    const bool want_stream = p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_STREAM;
    const bool want_cluster = exact && (p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_CLUSTER);
    const bool want_persist = exact && p->kernel == LDPC_KERNEL_PERSISTENT;
    const bool want_pingpong = exact && (p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_PINGPONG);
    if (want_half && ldpc::onchip_h2_eligible(c->N, c->max_row_deg, c->max_col_deg, p->msg_sat, p->rule, p->norm_num) &&
        ldpc::onchip_h2_plan(v, form, n_frames, c->sm_count, c->smem_optin, c->max_row_deg, &ch->onchip)) {
      ch->kind = Choice::ONCHIP_H2;
      ch->ws = 0;
      return LDPC_OK;
    }
    if (want_cluster && cluster_plan_fits(c, p)) {
      ch->kind = Choice::CLUSTER_H2;
      ch->ws = 0;
      return LDPC_OK;
    }
    if (want_int && ldpc::onchip_int8_plan(v, form, n_frames, c->sm_count, c->smem_optin, c->max_row_deg, &ch->onchip)) {
      ch->kind = Choice::ONCHIP_INT8;
      ch->ws = 0;
      return LDPC_OK;
    }
    if (want_pingpong && ldpc::pingpong_int8_eligible(c->N, c->M, c->ell_w, c->max_row_deg, c->max_col_deg,
                                                      p->msg_sat, form, n_frames)) {
      ch->kind = Choice::PINGPONG_INT8;
      ch->pingpong = ldpc::pingpong_layout(form, c->N, c->M, c->ell_w, n_frames);
      ch->ws = ch->pingpong.total;
      return LDPC_OK;
    }
    if (want_persist && ldpc::persist_int8_eligible(c->N, c->M, c->ell_w, c->max_row_deg, c->max_col_deg,
                                                    p->msg_sat, form, n_frames)) {
      ch->kind = Choice::PERSIST_INT8;
      ch->persist = ldpc::persist_layout(form, c->N, c->M, c->ell_w, n_frames, kPersistGroupChunks);
      ch->ws = ch->persist.total;
      return LDPC_OK;
    }
    if (want_stream && ldpc::stream_int8_eligible(c->max_row_deg, c->max_col_deg, p->msg_sat)) {
      ch->kind = Choice::STREAM_INT8;
      ch->stream = ldpc::stream_layout(0, form, c->N, c->M, c->ell_w * c->M, n_frames);
      ch->ws = ch->stream.total;
      return LDPC_OK;
    }
    return fail(LDPC_ERR_UNSUPPORTED, "code (N=%d, M=%d, E=%d, row degree <= %d, column degree <= %d) "
                "cannot run on the requested kernel (%d)",
                c->N, c->M, c->E, c->max_row_deg, c->max_col_deg, p->kernel);
  }
  if (p->dtype == LDPC_DTYPE_INT8 && (p->form == LDPC_FORM_TWO_SCAN || p->form == LDPC_FORM_TWO_SCAN_1BIT)) {
    const int form2 = p->form == LDPC_FORM_TWO_SCAN_1BIT ? 1 : 0;
    if (form2 == 0 && (p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_ONCHIP_HALF) &&
        ldpc::onchip_h2_eligible(c->N, c->max_row_deg, c->max_col_deg, p->msg_sat, p->rule, p->norm_num) &&
        ldpc::onchip_twoscan_plan(v, n_frames, c->sm_count, c->smem_optin, c->max_row_deg, &ch->onchip)) {
      ch->kind = Choice::ONCHIP_TWOSCAN;
      ch->ws = 0;
      return LDPC_OK;
    }
    if ((p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_STREAM) &&
        (form2 == 0 || c->d_ccj != nullptr) &&
        ldpc::twoscan_stream_eligible(c->N, c->M, c->ell_w, c->max_row_deg, c->max_col_deg, p->msg_sat, form2,
                                      n_frames)) {
      ch->kind = Choice::STREAM_TWOSCAN;
      ch->twoscan = ldpc::twoscan_layout(form2, c->N, c->M, c->ell_w, n_frames);
      ch->twoscan.dvmax = c->max_col_deg;
      ch->ws = ch->twoscan.total;
      return LDPC_OK;
    }
    return fail(LDPC_ERR_UNSUPPORTED, "the two-scan decoders need row degree <= 16, column degree <= 16 and "
                "128 + (max_col_degree + 1) * msg_sat <= 2048 (code N=%d, E=%d; kernel %d)", c->N, c->E, p->kernel);
  }
  if (p->dtype == LDPC_DTYPE_F32 && (p->form == LDPC_FORM_SS_1BIT || p->form == LDPC_FORM_SS_FIXED) &&
      (p->kernel == LDPC_KERNEL_AUTO || p->kernel == LDPC_KERNEL_STREAM)) {
    ch->kind = Choice::STREAM_F32;
    // per-edge slots: the degree-sorted table's (min-sum) or the edges of H (sum-product)
    ch->stream = ldpc::stream_layout(1, p->form == LDPC_FORM_SS_1BIT ? 1 : 0, c->N, c->M,
                                     std::max(c->E, c->ell_w * c->M), n_frames);
    ch->ws = ch->stream.total;
    return LDPC_OK;
  }
  return fail(LDPC_ERR_UNSUPPORTED, "dtype %d / form %d / kernel %d is not available in this build", p->dtype,
              p->form, p->kernel);
}

}  // namespace

extern "C" {

const char* ldpc_last_error(void) { return g_last_error.c_str(); }

ldpc_status ldpc_code_create(ldpc_code** out, int32_t n_vars, int32_t n_checks, const int32_t* row_ptr,
                             const int32_t* col_idx, int device) {
  g_last_error.clear();
  if (out == nullptr) return fail(LDPC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (row_ptr == nullptr) return fail(LDPC_ERR_INVALID_ARG, "row_ptr is NULL");
  if (n_vars < 1 || n_checks < 1) return fail(LDPC_ERR_INVALID_ARG, "n_vars and n_checks must be >= 1");
  if (row_ptr[0] != 0) return fail(LDPC_ERR_INVALID_ARG, "row_ptr[0] must be 0");
  int32_t max_row = 0;
  for (int32_t m = 0; m < n_checks; ++m) {
    const int64_t d = (int64_t)row_ptr[m + 1] - row_ptr[m];
    if (d < 2 || d > 32)
      return fail(LDPC_ERR_INVALID_ARG, "check %d has degree %lld; degrees must be in [2, 32]", m, (long long)d);
    if (d > max_row) max_row = (int32_t)d;
  }
  const int32_t E = row_ptr[n_checks];
  if (col_idx == nullptr) return fail(LDPC_ERR_INVALID_ARG, "col_idx is NULL");
  std::vector<int32_t> col_deg((size_t)n_vars, 0);
  std::vector<int32_t> seen((size_t)n_vars, -1);
  for (int32_t m = 0; m < n_checks; ++m) {
    for (int32_t e = row_ptr[m]; e < row_ptr[m + 1]; ++e) {
      const int32_t n = col_idx[e];
      if (n < 0 || n >= n_vars)
        return fail(LDPC_ERR_INVALID_ARG, "col_idx[%d] = %d outside [0, %d)", e, n, n_vars);
      if (seen[(size_t)n] == m)
        return fail(LDPC_ERR_INVALID_ARG, "variable %d appears twice in check %d", n, m);
      seen[(size_t)n] = m;
      col_deg[(size_t)n]++;
    }
  }
  int32_t max_col = 0;
  for (int32_t d : col_deg) max_col = d > max_col ? d : max_col;
  // edge-slot-major copy of N(m), padded with each check's last variable
  const bool narrow = n_vars <= 65535;
  std::vector<uint16_t> ell16(narrow ? (size_t)max_row * n_checks : 0);
  std::vector<int32_t> ell32(narrow ? 0 : (size_t)max_row * n_checks);
  std::vector<uint8_t> rdeg((size_t)n_checks);
  // degree classes: the distinct check degrees, ascending
  int32_t n_cls = 0, cls_deg[32] = {};
  for (int32_t dgr = 2; dgr <= 32; ++dgr)
    for (int32_t m = 0; m < n_checks; ++m)
      if (row_ptr[m + 1] - row_ptr[m] == dgr) { cls_deg[n_cls++] = dgr; break; }
  // The frame-resident kernels visit checks in an internal order sorted by degree
  // (stable), so that the checks of a warp share one degree; check order does not
  // change any result (each check's messages depend only on the previous
  // iteration, and the exact integer sums do not depend on the order).
  std::vector<int32_t> order((size_t)n_checks), pos((size_t)n_checks);
  for (int32_t m = 0; m < n_checks; ++m) order[(size_t)m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return row_ptr[a + 1] - row_ptr[a] < row_ptr[b + 1] - row_ptr[b];
  });
  for (int32_t i = 0; i < n_checks; ++i) pos[(size_t)order[(size_t)i]] = i;
  // variable -> edge slots (j * M + internal check index), for the two-scan comparator
  std::vector<int32_t> cptr((size_t)n_vars + 1, 0), cslot((size_t)E), cfill((size_t)n_vars, 0);
  std::vector<uint32_t> ccj((size_t)E);
  for (int32_t e = 0; e < E; ++e) cptr[(size_t)col_idx[e] + 1]++;
  for (int32_t n = 0; n < n_vars; ++n) cptr[(size_t)n + 1] += cptr[(size_t)n];
  for (int32_t m = 0; m < n_checks; ++m)
    for (int32_t j = 0; j < row_ptr[m + 1] - row_ptr[m]; ++j) {
      const int32_t n = col_idx[row_ptr[m] + j];
      ccj[(size_t)(cptr[(size_t)n] + cfill[(size_t)n])] = (uint32_t)pos[(size_t)m] | ((uint32_t)j << 24);
      cslot[(size_t)(cptr[(size_t)n] + cfill[(size_t)n]++)] = j * n_checks + pos[(size_t)m];
    }
  for (int32_t i = 0; i < n_checks; ++i) {
    const int32_t m = order[(size_t)i];
    const int32_t d = row_ptr[m + 1] - row_ptr[m];
    rdeg[(size_t)i] = (uint8_t)d;
    for (int32_t j = 0; j < max_row; ++j) {
      const int32_t n = col_idx[row_ptr[m] + (j < d ? j : d - 1)];
      if (narrow) ell16[(size_t)j * n_checks + i] = (uint16_t)n;
      else ell32[(size_t)j * n_checks + i] = n;
    }
  }

  int n_dev = 0;
  cudaError_t err = cudaGetDeviceCount(&n_dev);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDeviceCount");
  if (device < 0 || device >= n_dev) return fail(LDPC_ERR_INVALID_ARG, "device %d of %d", device, n_dev);
  DeviceGuard guard(device);
  if (!guard.ok) return fail(LDPC_ERR_CUDA, "cudaSetDevice(%d) failed", device);

  ldpc_code* c = new ldpc_code();
  c->device = device;
  c->N = n_vars;
  c->M = n_checks;
  c->E = E;
  c->max_row_deg = max_row;
  c->max_col_deg = max_col;
  c->ell_w = max_row;
  c->n_classes = n_cls;
  for (int32_t q = 0; q < n_cls; ++q) c->class_deg[q] = cls_deg[q];
  // the degree-sorted internal order as runs of equal degree
  if (n_cls <= 4) {
    c->n_dc = n_cls;
    int32_t end = 0;
    for (int32_t q = 0; q < n_cls; ++q) {
      while (end < n_checks && rdeg[(size_t)end] == cls_deg[q]) ++end;
      c->dc_end[q] = end;
      c->dc_deg[q] = cls_deg[q];
    }
  }
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  c->sm_count = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = (size_t)v;
  if ((err = cudaMalloc(&c->d_rp, sizeof(int32_t) * ((size_t)n_checks + 1))) != cudaSuccess ||
      (err = cudaMalloc(&c->d_ci, sizeof(int32_t) * (size_t)E)) != cudaSuccess ||
      (err = cudaMalloc(&c->d_cdeg, sizeof(int32_t) * (size_t)n_vars)) != cudaSuccess ||
      (err = cudaMemcpy(c->d_cdeg, col_deg.data(), sizeof(int32_t) * (size_t)n_vars, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (err = cudaMalloc(&c->d_cptr, sizeof(int32_t) * ((size_t)n_vars + 1))) != cudaSuccess ||
      (err = cudaMemcpy(c->d_cptr, cptr.data(), sizeof(int32_t) * ((size_t)n_vars + 1), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (err = cudaMalloc(&c->d_cslot, sizeof(int32_t) * (size_t)E)) != cudaSuccess ||
      (err = cudaMemcpy(c->d_cslot, cslot.data(), sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (n_checks < (1 << 24) && (err = cudaMalloc(&c->d_ccj, sizeof(uint32_t) * (size_t)E)) != cudaSuccess) ||
      (n_checks < (1 << 24) && (err = cudaMemcpy(c->d_ccj, ccj.data(), sizeof(uint32_t) * (size_t)E,
                                                 cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (err = cudaMalloc(&c->d_rdeg, (size_t)n_checks)) != cudaSuccess ||
      (err = cudaMemcpy(c->d_rdeg, rdeg.data(), (size_t)n_checks, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (narrow && (err = cudaMalloc(&c->d_ell16, sizeof(uint16_t) * ell16.size())) != cudaSuccess) ||
      (narrow && (err = cudaMemcpy(c->d_ell16, ell16.data(), sizeof(uint16_t) * ell16.size(),
                                   cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (!narrow && (err = cudaMalloc(&c->d_ell32, sizeof(int32_t) * ell32.size())) != cudaSuccess) ||
      (!narrow && (err = cudaMemcpy(c->d_ell32, ell32.data(), sizeof(int32_t) * ell32.size(),
                                    cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (err = cudaMemcpy(c->d_rp, row_ptr, sizeof(int32_t) * ((size_t)n_checks + 1), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (err = cudaMemcpy(c->d_ci, col_idx, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(c->d_rp);
    cudaFree(c->d_ci);
    cudaFree(c->d_cdeg);
    cudaFree(c->d_rdeg);
    cudaFree(c->d_ell16);
    cudaFree(c->d_ell32);
    cudaFree(c->d_cptr);
    cudaFree(c->d_cslot);
    cudaFree(c->d_ccj);
    delete c;
    return cuda_fail(err, "ldpc_code_create device copy");
  }
  const ldpc_status cs = build_cluster_tables(c, row_ptr, col_idx);
  if (cs != LDPC_OK) {
    ldpc_code_destroy(c);
    return cs;
  }
  // kernel attributes of this device, set here: code creation is never inside
  // a stream capture, and every decode of the code runs on this device
  if ((err = ldpc::pingpong_prepare()) != cudaSuccess || (err = ldpc::twoscan_prepare()) != cudaSuccess) {
    ldpc_code_destroy(c);
    return cuda_fail(err, "ldpc_code_create kernel attributes");
  }
  // default layers for the layered schedule: checks in row order, each into the
  // lowest layer none of whose checks shares a variable with it
  c->pos = pos;
  c->h_row_ptr.assign(row_ptr, row_ptr + n_checks + 1);
  c->h_col_idx.assign(col_idx, col_idx + E);
  {
    std::vector<int32_t> layer((size_t)n_checks, 0);
    std::vector<std::vector<uint8_t>> used;
    for (int32_t m = 0; m < n_checks; ++m) {
      size_t l = 0;
      for (; l < used.size(); ++l) {
        bool free_here = true;
        for (int32_t e = row_ptr[m]; e < row_ptr[m + 1] && free_here; ++e) free_here = !used[l][(size_t)col_idx[e]];
        if (free_here) break;
      }
      if (l == used.size()) used.emplace_back((size_t)n_vars, (uint8_t)0);
      for (int32_t e = row_ptr[m]; e < row_ptr[m + 1]; ++e) used[l][(size_t)col_idx[e]] = 1;
      layer[(size_t)m] = (int32_t)l;
    }
    const ldpc_status ls = set_layers(c, (int32_t)used.size(), layer.data());
    if (ls != LDPC_OK) {
      ldpc_code_destroy(c);
      return ls;
    }
  }
  *out = c;
  return LDPC_OK;
}

ldpc_status ldpc_code_destroy(ldpc_code* code) {
  g_last_error.clear();
  if (code == nullptr) return LDPC_OK;
  DeviceGuard guard(code->device);
  cudaDeviceSynchronize();
  cudaFree(code->d_rp);
  cudaFree(code->d_ci);
  cudaFree(code->d_cdeg);
  cudaFree(code->d_rdeg);
  cudaFree(code->d_ell16);
  cudaFree(code->d_ell32);
  cudaFree(code->d_cptr);
  cudaFree(code->d_cslot);
  cudaFree(code->d_ccj);
  cudaFree(code->d_lay_ptr);
  cudaFree(code->d_lay_rows);
  free_cluster_tables(code);
  delete code;
  return LDPC_OK;
}

ldpc_status ldpc_code_info(const ldpc_code* code, int32_t* n_vars, int32_t* n_checks, int32_t* n_edges,
                           int32_t* max_row_degree, int32_t* max_col_degree) {
  g_last_error.clear();
  if (code == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code is NULL");
  if (n_vars) *n_vars = code->N;
  if (n_checks) *n_checks = code->M;
  if (n_edges) *n_edges = code->E;
  if (max_row_degree) *max_row_degree = code->max_row_deg;
  if (max_col_degree) *max_col_degree = code->max_col_deg;
  return LDPC_OK;
}

ldpc_status ldpc_workspace_size(const ldpc_code* code, const ldpc_decode_params* params, int32_t n_frames,
                                size_t* bytes) {
  g_last_error.clear();
  if (code == nullptr || params == nullptr || bytes == nullptr)
    return fail(LDPC_ERR_INVALID_ARG, "code, params and bytes must be non-NULL");
  if (n_frames < 0) return fail(LDPC_ERR_INVALID_ARG, "n_frames %d < 0", n_frames);
  *bytes = 0;
  ldpc_status s = check_params(code, params);
  if (s != LDPC_OK) return s;
  if (n_frames == 0) return LDPC_OK;
  Choice ch;
  s = choose(code, params, n_frames, &ch);
  if (s != LDPC_OK) return s;
  *bytes = ch.ws;
  return LDPC_OK;
}

ldpc_status ldpc_kernel_choice(const ldpc_code* code, const ldpc_decode_params* params, int32_t n_frames,
                               int32_t* kernel) {
  g_last_error.clear();
  if (code == nullptr || params == nullptr || kernel == nullptr)
    return fail(LDPC_ERR_INVALID_ARG, "code, params and kernel must be non-NULL");
  if (n_frames < 0) return fail(LDPC_ERR_INVALID_ARG, "n_frames %d < 0", n_frames);
  ldpc_status s = check_params(code, params);
  if (s != LDPC_OK) return s;
  Choice ch;
  s = choose(code, params, n_frames > 0 ? n_frames : 1, &ch);
  if (s != LDPC_OK) return s;
  switch (ch.kind) {
    case Choice::ONCHIP_INT8: *kernel = LDPC_KERNEL_ONCHIP_INT; break;
    case Choice::ONCHIP_H2:
    case Choice::ONCHIP_TWOSCAN: *kernel = LDPC_KERNEL_ONCHIP_HALF; break;
    case Choice::CLUSTER_H2: *kernel = LDPC_KERNEL_CLUSTER; break;
    case Choice::STREAM_INT8:
    case Choice::STREAM_TWOSCAN:
    case Choice::STREAM_F32: *kernel = LDPC_KERNEL_STREAM; break;
    case Choice::PERSIST_INT8: *kernel = LDPC_KERNEL_PERSISTENT; break;
    case Choice::PINGPONG_INT8: *kernel = LDPC_KERNEL_PINGPONG; break;
    default: *kernel = LDPC_KERNEL_AUTO; break;
  }
  return LDPC_OK;
}

ldpc_status ldpc_decode_batch(const ldpc_code* code, const ldpc_decode_params* params, const void* llr,
                              int32_t n_frames, uint8_t* hard_bits, int32_t* iters_used, uint8_t* syndrome_ok,
                              void* llr_out, void* workspace, size_t ws_bytes, void* stream) {
  g_last_error.clear();
  if (code == nullptr || params == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code and params must be non-NULL");
  if (n_frames < 0) return fail(LDPC_ERR_INVALID_ARG, "n_frames %d < 0", n_frames);
  ldpc_status s = check_params(code, params);
  if (s != LDPC_OK) return s;
  if (n_frames == 0) return LDPC_OK;
  if (llr == nullptr || hard_bits == nullptr || iters_used == nullptr || syndrome_ok == nullptr)
    return fail(LDPC_ERR_INVALID_ARG, "llr, hard_bits, iters_used and syndrome_ok must be non-NULL");
  Choice ch;
  s = choose(code, params, n_frames, &ch);
  if (s != LDPC_OK) return s;
  if (ch.ws > 0 && (workspace == nullptr || ws_bytes < ch.ws))
    return fail(LDPC_ERR_INVALID_ARG, "workspace of %zu bytes needed, %zu given", ch.ws,
                workspace ? ws_bytes : (size_t)0);
  if (workspace != nullptr && ((uintptr_t)workspace & 255u) != 0)
    return fail(LDPC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  DeviceGuard guard(code->device);
  if (!guard.ok) return fail(LDPC_ERR_CUDA, "cudaSetDevice(%d) failed", code->device);
  cudaStream_t st = (cudaStream_t)stream;
  const ldpc::DevCode v = view(code);
  cudaError_t err = cudaSuccess;
  ldpc::IntRule r;
  r.rule = params->rule;
  r.beta = params->offset;
  r.num = params->norm_num;
  r.shift = params->norm_shift;
  r.qm = params->msg_sat;
  r.psat = params->posterior == LDPC_POSTERIOR_SAT8 ? 127 : 0;
  const int form = params->form == LDPC_FORM_SS_1BIT ? 1 : 0;
  if (ch.kind == Choice::ONCHIP_TWOSCAN) {
    err = ldpc::onchip_twoscan_launch(v, r, ch.onchip, code->sm_count, static_cast<const int8_t*>(llr), n_frames,
                                      params->max_iter, params->early_stop, hard_bits, iters_used, syndrome_ok,
                                      static_cast<int16_t*>(llr_out), st);
  } else if (ch.kind == Choice::ONCHIP_H2) {
    err = ldpc::onchip_h2_launch(v, r, form, ch.onchip, code->sm_count, static_cast<const int8_t*>(llr), n_frames,
                                 params->max_iter, params->early_stop, hard_bits, iters_used, syndrome_ok,
                                 static_cast<int16_t*>(llr_out), st, false);
  } else if (ch.kind == Choice::LAYERED) {
    err = ldpc::layered_decode(v, r, form, code->d_lay_ptr, code->d_lay_rows, code->n_layers,
                               static_cast<const int8_t*>(llr), n_frames, params->max_iter, params->early_stop,
                               hard_bits, iters_used, syndrome_ok, static_cast<int16_t*>(llr_out), workspace,
                               ch.layered, code->sm_count, st);
  } else if (ch.kind == Choice::CLUSTER_H2) {
    err = cluster_decode(code, params, static_cast<const int8_t*>(llr), n_frames, hard_bits, iters_used, syndrome_ok,
                         static_cast<int16_t*>(llr_out), st);
  } else if (ch.kind == Choice::STREAM_INT8) {
    err = ldpc::stream_int8_decode(v, r, form, ch.stream, workspace, code->sm_count, static_cast<const int8_t*>(llr),
                                   n_frames, params->max_iter, params->early_stop, hard_bits, iters_used,
                                   syndrome_ok, static_cast<int16_t*>(llr_out), st);
  } else if (ch.kind == Choice::STREAM_TWOSCAN) {
    err = ldpc::twoscan_stream_decode(v, r, params->form == LDPC_FORM_TWO_SCAN_1BIT ? 1 : 0, ch.twoscan, workspace,
                                      static_cast<const int8_t*>(llr), n_frames, params->max_iter, params->early_stop,
                                      hard_bits, iters_used, syndrome_ok, static_cast<int16_t*>(llr_out), st);
  } else if (ch.kind == Choice::PINGPONG_INT8) {
    // row kernel blocks of 4 warps (N=64800, 1024 frames: 7.04 ms against 7.13 at 8 warps, same box)
    err = ldpc::pingpong_int8_decode(v, r, form, ch.pingpong, workspace, static_cast<const int8_t*>(llr), n_frames,
                                     params->max_iter, params->early_stop, hard_bits, iters_used, syndrome_ok,
                                     static_cast<int16_t*>(llr_out), st, 4);
  } else if (ch.kind == Choice::PERSIST_INT8) {
    err = ldpc::persist_int8_decode(v, r, form, ch.persist, workspace, code->sm_count,
                                    static_cast<const int8_t*>(llr), n_frames, params->max_iter, params->early_stop,
                                    hard_bits, iters_used, syndrome_ok, static_cast<int16_t*>(llr_out), st);
  } else if (ch.kind == Choice::STREAM_F32) {
    ldpc::F32Rule fr;
    fr.rule = params->rule;
    fr.beta = params->offset_f32;
    fr.lambda = params->norm_f32;
    err = ldpc::stream_f32_decode(v, fr, form, ch.stream, workspace, code->sm_count, static_cast<const float*>(llr),
                                  n_frames, params->max_iter, params->early_stop, hard_bits, iters_used,
                                  syndrome_ok, static_cast<float*>(llr_out), st);
  } else if (ch.kind == Choice::ONCHIP_INT8) {
    err = ldpc::onchip_int8_occupancy(form, code->sm_count, &ch.onchip);
    if (err == cudaSuccess)
      err = ldpc::onchip_int8_launch(v, r, form, ch.onchip, static_cast<const int8_t*>(llr), n_frames,
                                     params->max_iter, params->early_stop, hard_bits, iters_used, syndrome_ok,
                                     static_cast<int16_t*>(llr_out), st);
  }
  if (err != cudaSuccess) return cuda_fail(err, "ldpc_decode_batch launch");
  return LDPC_OK;
}

ldpc_status ldpc_qc_expand(const ldpc_qc_desc* qc, int32_t* row_ptr, int32_t* col_idx, int64_t capacity,
                           int32_t* n_edges) {
  g_last_error.clear();
  if (qc == nullptr || qc->shift == nullptr) return fail(LDPC_ERR_INVALID_ARG, "qc and qc->shift must be non-NULL");
  const int64_t mb = qc->base_rows, nb = qc->base_cols, z = qc->lift;
  if (mb < 1 || nb < 1 || z < 1) return fail(LDPC_ERR_INVALID_ARG, "base_rows, base_cols and lift must be >= 1");
  if (nb * z > INT32_MAX || mb * z + 1 > INT32_MAX)
    return fail(LDPC_ERR_INVALID_ARG, "%lld x %lld blocks of %lld exceed int32 sizes", (long long)mb, (long long)nb,
                (long long)z);
  int64_t E = 0;
  for (int64_t i = 0; i < mb * nb; ++i) {
    const int32_t sh = qc->shift[i];
    if (sh < -1 || sh >= z)
      return fail(LDPC_ERR_INVALID_ARG, "shift[%lld] = %d is neither -1 nor in [0, %lld)", (long long)i, sh,
                  (long long)z);
    if (sh >= 0) E += z;
  }
  if (E > INT32_MAX) return fail(LDPC_ERR_INVALID_ARG, "%lld edges exceed int32", (long long)E);
  if (col_idx != nullptr && capacity < E)
    return fail(LDPC_ERR_INVALID_ARG, "col_idx holds %lld entries, %lld needed", (long long)capacity, (long long)E);
  if (n_edges != nullptr) *n_edges = (int32_t)E;
  int64_t e = 0;
  for (int64_t i = 0; i < mb; ++i) {
    for (int64_t r = 0; r < z; ++r) {
      if (row_ptr != nullptr) row_ptr[i * z + r] = (int32_t)e;
      for (int64_t j = 0; j < nb; ++j) {
        const int32_t sh = qc->shift[i * nb + j];
        if (sh < 0) continue;
        if (col_idx != nullptr) col_idx[e] = (int32_t)(j * z + (r + sh) % z);
        ++e;
      }
    }
  }
  if (row_ptr != nullptr) row_ptr[mb * z] = (int32_t)e;
  return LDPC_OK;
}

ldpc_status ldpc_code_create_qc(ldpc_code** out, const ldpc_qc_desc* qc, int device) {
  if (out == nullptr) return fail(LDPC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int32_t E = 0;
  ldpc_status s = ldpc_qc_expand(qc, nullptr, nullptr, 0, &E);
  if (s != LDPC_OK) return s;
  const int32_t M = qc->base_rows * qc->lift, N = qc->base_cols * qc->lift;
  std::vector<int32_t> rp((size_t)M + 1), ci((size_t)E);
  s = ldpc_qc_expand(qc, rp.data(), ci.data(), E, nullptr);
  if (s != LDPC_OK) return s;
  ldpc_code* c = nullptr;
  s = ldpc_code_create(&c, N, M, rp.data(), ci.data(), device);
  if (s != LDPC_OK) return s;
  std::vector<int32_t> layer((size_t)M);
  for (int32_t m = 0; m < M; ++m) layer[(size_t)m] = m / qc->lift;
  s = ldpc_code_set_layers(c, qc->base_rows, layer.data());
  if (s != LDPC_OK) {
    const std::string why = g_last_error;
    ldpc_code_destroy(c);
    return fail(s, "block-row layers: %s", why.c_str());
  }
  *out = c;
  return LDPC_OK;
}

ldpc_status ldpc_code_degree_classes(const ldpc_code* code, int32_t* n_classes, int32_t* degrees) {
  g_last_error.clear();
  if (code == nullptr || n_classes == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code and n_classes must be non-NULL");
  *n_classes = code->n_classes;
  if (degrees != nullptr)
    for (int32_t q = 0; q < code->n_classes; ++q) degrees[q] = code->class_deg[q];
  return LDPC_OK;
}

ldpc_status ldpc_code_layers(const ldpc_code* code, int32_t* n_layers, int32_t* layer_of_check) {
  g_last_error.clear();
  if (code == nullptr || n_layers == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code and n_layers must be non-NULL");
  *n_layers = code->n_layers;
  if (layer_of_check != nullptr)
    std::copy(code->layer_of_check.begin(), code->layer_of_check.end(), layer_of_check);
  return LDPC_OK;
}

ldpc_status ldpc_code_set_layers(ldpc_code* code, int32_t n_layers, const int32_t* layer_of_check) {
  g_last_error.clear();
  if (code == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code is NULL");
  DeviceGuard guard(code->device);
  cudaDeviceSynchronize();  // no decode in flight may read the old tables
  return set_layers(code, n_layers, layer_of_check);
}

namespace {
constexpr int kLearnedMaxClasses = 4;

ldpc_status learned_check(const ldpc_code* code, int32_t n_iters, int32_t n_frames, void* ws, size_t ws_bytes,
                          ldpc::LearnedLayout* L) {
  if (code == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code is NULL");
  if (n_iters < 1 || n_iters > 64) return fail(LDPC_ERR_INVALID_ARG, "n_iters %d outside [1, 64]", n_iters);
  if (n_frames < 1) return fail(LDPC_ERR_INVALID_ARG, "n_frames %d < 1", n_frames);
  if (code->n_classes > kLearnedMaxClasses)
    return fail(LDPC_ERR_UNSUPPORTED, "learned offsets support at most %d check-degree classes, the code has %d",
                kLearnedMaxClasses, code->n_classes);
  *L = ldpc::learned_layout(code->N, code->M, n_iters, code->n_classes, n_frames);
  if (ws == nullptr || ws_bytes < L->total)
    return fail(LDPC_ERR_INVALID_ARG, "learned workspace of %zu bytes needed, %zu given", L->total,
                ws ? ws_bytes : (size_t)0);
  if (((uintptr_t)ws & 255u) != 0) return fail(LDPC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  return LDPC_OK;
}
}  // namespace

ldpc_status ldpc_learned_workspace_size(const ldpc_code* code, int32_t n_iters, int32_t n_frames, size_t* bytes) {
  g_last_error.clear();
  if (code == nullptr || bytes == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code and bytes must be non-NULL");
  if (n_iters < 1 || n_frames < 1) return fail(LDPC_ERR_INVALID_ARG, "n_iters and n_frames must be >= 1");
  *bytes = ldpc::learned_layout(code->N, code->M, n_iters, code->n_classes, n_frames).total;
  return LDPC_OK;
}

ldpc_status ldpc_learned_forward(const ldpc_code* code, int32_t n_iters, const float* beta, const float* llr,
                                 int32_t n_frames, float* z_out, void* workspace, size_t ws_bytes, void* stream) {
  g_last_error.clear();
  ldpc::LearnedLayout L;
  ldpc_status s = learned_check(code, n_iters, n_frames, workspace, ws_bytes, &L);
  if (s != LDPC_OK) return s;
  if (beta == nullptr || llr == nullptr) return fail(LDPC_ERR_INVALID_ARG, "beta and llr must be non-NULL");
  DeviceGuard guard(code->device);
  const cudaError_t e = ldpc::learned_forward(view(code), code->n_classes, n_iters, beta, L,
                                              workspace, llr, n_frames, z_out, (cudaStream_t)stream);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_learned_forward launch");
}

ldpc_status ldpc_learned_loss(const ldpc_code* code, int32_t n_iters, int32_t n_frames, const uint8_t* target_bits,
                              float* loss, int32_t want_grad, void* workspace, size_t ws_bytes, void* stream) {
  g_last_error.clear();
  ldpc::LearnedLayout L;
  ldpc_status s = learned_check(code, n_iters, n_frames, workspace, ws_bytes, &L);
  if (s != LDPC_OK) return s;
  if (loss == nullptr) return fail(LDPC_ERR_INVALID_ARG, "loss must be non-NULL");
  DeviceGuard guard(code->device);
  const cudaError_t e = ldpc::learned_bce(view(code), code->n_classes, n_iters, L, workspace, n_frames, target_bits,
                                          loss, want_grad != 0, (cudaStream_t)stream);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_learned_loss launch");
}

ldpc_status ldpc_learned_backward(const ldpc_code* code, int32_t n_iters, const float* beta, const float* dz,
                                  int32_t n_frames, float* dbeta, void* workspace, size_t ws_bytes, void* stream) {
  g_last_error.clear();
  ldpc::LearnedLayout L;
  ldpc_status s = learned_check(code, n_iters, n_frames, workspace, ws_bytes, &L);
  if (s != LDPC_OK) return s;
  if (beta == nullptr || dbeta == nullptr) return fail(LDPC_ERR_INVALID_ARG, "beta and dbeta must be non-NULL");
  DeviceGuard guard(code->device);
  const cudaError_t e = ldpc::learned_backward(view(code), code->n_classes, n_iters, beta, L,
                                               workspace, dz, n_frames, dbeta, (cudaStream_t)stream);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_learned_backward launch");
}

ldpc_status ldpc_adam_step(float* params, const float* grads, float* m, float* v, int32_t n, int32_t step, float lr,
                           float beta1, float beta2, float eps, void* stream) {
  g_last_error.clear();
  if (params == nullptr || grads == nullptr || m == nullptr || v == nullptr || n < 1 || step < 1)
    return fail(LDPC_ERR_INVALID_ARG, "adam: non-NULL buffers, n >= 1 and step >= 1 required");
  const cudaError_t e = ldpc::adam_step(params, grads, m, v, n, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_adam_step launch");
}

ldpc_status ldpc_awgn_llr_f32(int32_t n_vars, uint64_t seed, uint64_t first_frame, int32_t n_frames, float ebn0_lo_db,
                              float ebn0_hi_db, float rate, const uint8_t* codewords, float* llr, float* ebn0_out,
                              void* stream) {
  g_last_error.clear();
  if (n_vars < 1 || n_frames < 0 || llr == nullptr || !(rate > 0.0f && rate <= 1.0f) || ebn0_hi_db < ebn0_lo_db)
    return fail(LDPC_ERR_INVALID_ARG, "awgn: n_vars >= 1, llr non-NULL, 0 < rate <= 1, lo <= hi required");
  if (n_frames == 0) return LDPC_OK;
  const cudaError_t e = ldpc::awgn_llr(n_vars, seed, first_frame, n_frames, ebn0_lo_db, ebn0_hi_db, rate, codewords,
                                       llr, ebn0_out, (cudaStream_t)stream);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_awgn_llr_f32 launch");
}

ldpc_status ldpc_quantize_llr(const float* llr, int64_t n, float delta, int32_t qc, int8_t* q, void* stream) {
  g_last_error.clear();
  if (llr == nullptr || q == nullptr || n < 0 || !(delta > 0.0f) || qc < 1 || qc > 127)
    return fail(LDPC_ERR_INVALID_ARG, "quantize: non-NULL buffers, delta > 0, 1 <= qc <= 127 required");
  if (n == 0) return LDPC_OK;
  const cudaError_t e = ldpc::quantize_llr(llr, (size_t)n, delta, qc, q, (cudaStream_t)stream);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_quantize_llr launch");
}

ldpc_status ldpc_wait_selftest(int device, int32_t max_spins) {
  g_last_error.clear();
  if (max_spins < 1 || max_spins > (1 << 24)) return fail(LDPC_ERR_INVALID_ARG, "max_spins %d outside [1, 2^24]", max_spins);
  DeviceGuard guard(device);
  if (!guard.ok) return fail(LDPC_ERR_CUDA, "cudaSetDevice(%d) failed", device);
  bool gave_up = false;
  const cudaError_t e = ldpc::persist_wait_selftest((uint32_t)max_spins, &gave_up);
  if (e != cudaSuccess) return cuda_fail(e, "ldpc_wait_selftest");
  if (gave_up) return fail(LDPC_ERR_TIMEOUT, "the bounded wait gave up after %d polls", max_spins);
  return LDPC_OK;
}

// ---------------------------------------------------------------------------
// Decoding without any device allocation by the caller or the library.
//
// Some callers cannot allocate device memory on their decode path: a receiver
// that must keep a bounded per-block latency cannot afford cudaMalloc (it
// synchronises the device and its latency is unbounded), and a host component
// that only receives buffers from a memory pool it does not own has no
// allocator to call.  For them ldpc_decode_batch_noalloc runs the streaming int8
// decoder on a scratch area that is part of the library image itself: a
// file-scope device array, created once on every GPU that loads the library and
// kept until the process exits.

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[LDPC_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).  In
// host code the array's name is only a host-side stand-in, so its device
// address is looked up once per device and cached.
ldpc_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kNoallocMaxDevices)
    return fail(LDPC_ERR_UNSUPPORTED, "device %d is beyond the %d devices the static scratch supports", device,
                kNoallocMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[device] == nullptr) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_noalloc_ptr[device] = ptr;
  }
  *out = g_noalloc_ptr[device];
  return LDPC_OK;
}

}  // namespace

ldpc_status ldpc_decode_batch_noalloc(const ldpc_code* code, const ldpc_decode_params* params, const void* llr,
                                      int32_t n_frames, uint8_t* hard_bits, int32_t* iters_used,
                                      uint8_t* syndrome_ok, void* llr_out, void* stream) {
  g_last_error.clear();
  if (code == nullptr || params == nullptr) return fail(LDPC_ERR_INVALID_ARG, "code and params must be non-NULL");
  if (n_frames < 0) return fail(LDPC_ERR_INVALID_ARG, "n_frames %d < 0", n_frames);
  ldpc_status s = check_params(code, params);
  if (s != LDPC_OK) return s;
  if (params->dtype != LDPC_DTYPE_INT8 || params->form == LDPC_FORM_TWO_SCAN ||
      (params->kernel != LDPC_KERNEL_AUTO && params->kernel != LDPC_KERNEL_STREAM) ||
      params->schedule != LDPC_SCHEDULE_FLOODING)
    return fail(LDPC_ERR_UNSUPPORTED, "the no-allocation entry point runs the int8 single-scan streaming decoder "
                "(flooding schedule) only");
  if (!ldpc::stream_int8_eligible(code->max_row_deg, code->max_col_deg, params->msg_sat))
    return fail(LDPC_ERR_UNSUPPORTED, "code degrees / msg_sat are outside the streaming int8 decoder's range");
  if (n_frames == 0) return LDPC_OK;
  if (llr == nullptr || hard_bits == nullptr || iters_used == nullptr || syndrome_ok == nullptr)
    return fail(LDPC_ERR_INVALID_ARG, "llr, hard_bits, iters_used and syndrome_ok must be non-NULL");
  const int form = params->form == LDPC_FORM_SS_1BIT ? 1 : 0;
  const ldpc::StreamLayout L = ldpc::stream_layout(0, form, code->N, code->M, code->ell_w * code->M, n_frames);
  if (L.total > (size_t)LDPC_NOALLOC_SCRATCH_BYTES)
    return fail(LDPC_ERR_UNSUPPORTED,
                "%d frames of this code need %zu bytes of scratch; the static scratch holds %zu "
                "(decode fewer frames per call)",
                n_frames, L.total, (size_t)LDPC_NOALLOC_SCRATCH_BYTES);
  DeviceGuard guard(code->device);
  if (!guard.ok) return fail(LDPC_ERR_CUDA, "cudaSetDevice(%d) failed", code->device);
  void* scratch = nullptr;
  s = noalloc_scratch(code->device, &scratch);
  if (s != LDPC_OK) return s;
  ldpc::IntRule r;
  r.rule = params->rule;
  r.beta = params->offset;
  r.num = params->norm_num;
  r.shift = params->norm_shift;
  r.qm = params->msg_sat;
  r.psat = params->posterior == LDPC_POSTERIOR_SAT8 ? 127 : 0;
  // every buffer the decoder reads before writing is initialised by the decoder
  // itself (state memset, init kernel), so contents left by a previous call do not matter
  const cudaError_t err = ldpc::stream_int8_decode(view(code), r, form, L, scratch, code->sm_count,
                                                   static_cast<const int8_t*>(llr), n_frames, params->max_iter,
                                                   params->early_stop, hard_bits, iters_used, syndrome_ok,
                                                   static_cast<int16_t*>(llr_out), (cudaStream_t)stream);
  if (err != cudaSuccess) return cuda_fail(err, "ldpc_decode_batch_noalloc launch");
  return LDPC_OK;
}

}  // extern "C"

// multi_api.cu -- host side of the cluster and multi-code launches: the split
// of a code over the CTAs of a cluster, the launch plan (which codes run on a
// cluster, frame pairs per CTA, shared memory, grid, work order), the
// ldpc_multi_* entry points and the autotuner.  No kernel logic here.
#include <algorithm>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "cluster_split.h"

using namespace ldpc_api;

struct ldpc_multi {
  int device = 0;
  int form = 1;
  std::vector<ldpc_multi_job> jobs;  // jobs with frames, in the caller's order
  std::vector<int32_t> user_index;   // their indices in the caller's array
  int32_t n_user = 0;
  ldpc_multi_tuning shape = {};
  ldpc::MultiParams mp = {};
  int threads = 0, grid = 0;
  size_t smem = 0;
  bool es = false;
  std::vector<int32_t> is_cluster, pairs_per_cta;  // per job of `jobs` (is_cluster: 0, 1, 2 streaming)
  struct StreamJob {
    int job;                     // index into jobs
    bool pingpong;               // the ping-pong decoder (checks of degree <= 8), else the two-launch one
    ldpc::StreamLayout layout;
    ldpc::PingpongLayout pp;
    size_t offset;               // in the workspace
  };
  std::vector<StreamJob> streamed;
  size_t ws_bytes = 0;
  // whether the streamed codes run concurrently on side streams (chosen by
  // ldpc_multi_autotune); their side streams and the fork / join events are
  // made at the first such launch on the plan's device
  bool overlap = false;
  mutable std::vector<cudaStream_t> side;
  mutable std::vector<cudaEvent_t> joined;
  mutable cudaEvent_t fork = nullptr;
  ~ldpc_multi() {
    for (cudaStream_t s : side) cudaStreamDestroy(s);
    for (cudaEvent_t e : joined) cudaEventDestroy(e);
    if (fork != nullptr) cudaEventDestroy(fork);
  }
};

namespace {

constexpr size_t kStaticReserve = 1024;  // static shared memory of the kernel, rounded up
constexpr size_t kQueueBytes = 256;

size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared memory of one cluster rank: table, Zs, Acc, state.
size_t cluster_need(const ClusterTables& t, int ell_w, int form, size_t* acc_off, size_t* st_off, size_t* tab) {
  const size_t tb = a16((size_t)ell_w * t.mr * 2);
  const size_t zs = a16((size_t)t.ns * 4);
  const size_t st = form == 1 ? (size_t)t.mr * 16 : a16((size_t)ell_w * t.mr * 2);
  if (acc_off) *acc_off = zs;
  if (st_off) *st_off = 2 * zs;
  if (tab) *tab = tb;
  return tb + 2 * zs + st;
}

struct JobIn {
  const ldpc_code* code;
  ldpc_decode_params p;
  const int8_t* llr;
  int32_t F;
  uint8_t* bits;
  int32_t* iters;
  uint8_t* ok;
  int16_t* zout;
};

struct Built {
  ldpc::MultiParams mp = {};
  int threads = 0, grid = 0, cs = 1;
  size_t smem = 0;
  bool es = false;
  std::vector<int32_t> is_cluster, pairs_per_cta;
  std::vector<ldpc_multi::StreamJob> streamed;
  size_t ws_bytes = 0;
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Plans one launch over `in` (all of the same form).  With occupancy == false
// the grid is left 0 (no CUDA call is made).  force_cluster puts every job on a
// cluster, also one that fits a CTA.
ldpc_status build(const std::vector<JobIn>& in, int form, const ldpc_multi_tuning& t, bool occupancy, Built* out,
                  bool force_cluster = false) {
  const int T = t.threads;
  const int tt = t.team_threads;
  if (in.empty()) return fail(LDPC_ERR_INVALID_ARG, "no job has frames");
  if ((int)in.size() > ldpc::kMultiMaxJobs)
    return fail(LDPC_ERR_UNSUPPORTED, "%d jobs; at most %d per launch", (int)in.size(), ldpc::kMultiMaxJobs);
  const ldpc_code* c0 = in[0].code;
  const size_t budget = c0->smem_optin > kStaticReserve ? c0->smem_optin - kStaticReserve : 0;
  const bool on_clusters = force_cluster || t.large == 2;
  std::vector<int> cs_need(in.size(), 1);  // 1: CTA sub-teams; > 1: cluster size; 0: streaming
  int cs = 1;
  for (size_t j = 0; j < in.size(); ++j) {
    const ldpc_code* c = in[j].code;
    const ldpc_decode_params& p = in[j].p;
    if (!ldpc::onchip_h2_eligible(c->N, c->max_row_deg, c->max_col_deg, p.msg_sat, p.rule, p.norm_num))
      return fail(LDPC_ERR_UNSUPPORTED,
                  "job %d: the code (N=%d, row degree <= %d, column degree <= %d) with msg_sat %d does not meet "
                  "n_vars <= 65535, row degree <= 16 and 128 + (max_col_degree + 1) * msg_sat <= 2048",
                  (int)j, c->N, c->max_row_deg, c->max_col_deg, p.msg_sat);
    const size_t local = a16((size_t)c->ell_w * c->M * 2) + ldpc::multi_local_slot_bytes(c->N, c->M, c->ell_w, form,
                                                                                           nullptr, nullptr);
    if (local <= budget && !force_cluster) continue;
    if (!on_clusters) {
      cs_need[j] = 0;
      continue;
    }
    int need = 0;
    for (int q = 0; q < kClusterSizes && need == 0; ++q) {
      const ClusterTables& ct = c->ctab[q];
      if (ct.ok && cluster_need(ct, c->ell_w, form, nullptr, nullptr, nullptr) <= budget) need = ct.cs;
    }
    if (need == 0)
      return fail(LDPC_ERR_UNSUPPORTED, "job %d: a frame pair of the code (N=%d, M=%d, E=%d) does not fit "
                  "the shared memory of a 16-CTA cluster", (int)j, c->N, c->M, c->E);
    cs_need[j] = need;
    cs = std::max(cs, need);
  }
  const bool any_cluster = cs > 1;
  if (any_cluster && t.cluster > cs) cs = t.cluster;
  if (cs > 16) return fail(LDPC_ERR_INVALID_ARG, "cluster size %d > 16", cs);

  struct Row {
    int j;
    bool cl;
    double cost;
  };
  std::vector<Row> order;
  Built b;
  b.cs = any_cluster ? cs : 1;
  b.is_cluster.assign(in.size(), 0);
  b.pairs_per_cta.assign(in.size(), 0);
  b.ws_bytes = kQueueBytes;
  std::vector<ldpc::MultiJob> jobs(in.size());
  size_t smem = 0;
  for (size_t j = 0; j < in.size(); ++j) {
    const ldpc_code* c = in[j].code;
    const ldpc_decode_params& p = in[j].p;
    ldpc::MultiJob& m = jobs[j];
    if (cs_need[j] == 0) {
      ldpc_multi::StreamJob sj{};
      sj.job = (int)j;
      sj.offset = b.ws_bytes;
      sj.pingpong = ldpc::pingpong_int8_eligible(c->N, c->M, c->ell_w, c->max_row_deg, c->max_col_deg, p.msg_sat,
                                                  form, in[j].F);
      if (sj.pingpong) {
        sj.pp = ldpc::pingpong_layout(form, c->N, c->M, c->ell_w, in[j].F);
        b.ws_bytes += al256(sj.pp.total);
      } else {
        sj.layout = ldpc::stream_layout(0, form, c->N, c->M, c->ell_w * c->M, in[j].F);
        b.ws_bytes += al256(sj.layout.total);
      }
      b.streamed.push_back(sj);
      b.is_cluster[j] = 2;
      b.es = b.es || p.early_stop != 0;
      continue;
    }
    std::memset(&m, 0, sizeof m);
    m.N = c->N;
    m.M = c->M;
    m.ell_w = c->ell_w;
    m.cdeg = c->d_cdeg;
    m.beta = p.rule == LDPC_RULE_OFFSET ? p.offset : 0;
    m.num = p.rule == LDPC_RULE_NORMALIZED ? p.norm_num : 1;
    m.shift = p.rule == LDPC_RULE_NORMALIZED ? p.norm_shift : 0;
    m.qm = p.msg_sat;
    m.max_iter = p.max_iter;
    m.early_stop = p.early_stop;
    m.llr = in[j].llr;
    m.F = in[j].F;
    m.bits = in[j].bits;
    m.iters = in[j].iters;
    m.ok = in[j].ok;
    m.zout = in[j].zout;
    m.n_pairs = (in[j].F + 1) / 2;
    b.es = b.es || p.early_stop != 0;
    const double pair_cost = (double)c->E * (p.max_iter + 1);
    if (cs_need[j] > 1) {
      const ClusterTables& ct = c->ctab[cluster_index(cs)];
      if (!ct.ok) return fail(LDPC_ERR_UNSUPPORTED, "job %d: the code cannot be split over %d CTAs", (int)j, cs);
      size_t acc_off, st_off, tb;
      const size_t need = cluster_need(ct, c->ell_w, form, &acc_off, &st_off, &tb);
      if (need > budget)
        return fail(LDPC_ERR_UNSUPPORTED, "job %d: %zu bytes of shared memory per CTA at cluster size %d", (int)j,
                    need, cs);
      smem = std::max(smem, need);
      m.mr = ct.mr;
      m.ns = ct.ns;
      m.lb = ct.lb;
      m.sub = 1;
      m.tab = ct.d_tab;
      m.rdeg = ct.d_rdeg;
      m.rows = ct.d_rows;
      m.tab_bytes = (uint32_t)tb;
      m.slot_bytes = (uint32_t)(need - tb);
      m.acc_off = (uint32_t)acc_off;
      m.st_off = (uint32_t)st_off;
      b.is_cluster[j] = 1;
      b.pairs_per_cta[j] = 1;
      order.push_back({(int)j, true, pair_cost});
    } else {
      size_t acc_off, st_off, rs_off;
      const size_t tb = a16((size_t)c->ell_w * c->M * 2);
      // the accumulator reset values join the slot when one slot still fits
      const bool rset = tb + ldpc::multi_local_slot_bytes(c->N, c->M, c->ell_w, form, nullptr, nullptr, true) <= budget;
      const size_t slot = ldpc::multi_local_slot_bytes(c->N, c->M, c->ell_w, form, &acc_off, &st_off, rset, &rs_off);
      int want = std::min(ldpc::kMultiMaxSub, std::max(1, T / tt));
      while (want > 1 && want / 2 >= m.n_pairs) want /= 2;  // no more slots than pairs
      int sub = want;
      while (sub > 1 && tb + (size_t)sub * slot > budget) sub /= 2;
      smem = std::max(smem, tb + (size_t)sub * slot);
      m.mr = c->M;
      m.ns = c->N;
      m.sub = sub;
      m.tab = c->d_ell16;
      m.rdeg = c->d_rdeg;
      m.rows = nullptr;
      m.tab_bytes = (uint32_t)tb;
      m.slot_bytes = (uint32_t)slot;
      m.acc_off = (uint32_t)acc_off;
      m.st_off = (uint32_t)st_off;
      m.rs_off = (uint32_t)rs_off;
      order.push_back({(int)j, false, pair_cost * sub});
    }
  }
  // local jobs may hold more pairs per CTA in the shared memory the launch has anyway
  for (size_t j = 0; j < in.size(); ++j) {
    ldpc::MultiJob& m = jobs[j];
    if (b.is_cluster[j] != 0) continue;
    int want = std::min(ldpc::kMultiMaxSub, std::max(1, T / tt));
    while (want > 1 && want / 2 >= m.n_pairs) want /= 2;
    while (m.sub * 2 <= want && m.tab_bytes + (size_t)(m.sub * 2) * m.slot_bytes <= smem) m.sub *= 2;
    b.pairs_per_cta[j] = m.sub;
  }
  for (Row& r : order)
    if (!r.cl) r.cost = (double)in[(size_t)r.j].code->E * (in[(size_t)r.j].p.max_iter + 1) * jobs[(size_t)r.j].sub;
  // longest items first: cluster jobs, then local jobs, each by cost per item
  std::stable_sort(order.begin(), order.end(), [](const Row& a, const Row& b2) {
    if (a.cl != b2.cl) return a.cl;
    return a.cost > b2.cost;
  });
  ldpc::MultiParams& mp = b.mp;
  std::memset(&mp, 0, sizeof mp);
  int citems = 0, litems = 0, nc = 0;
  for (size_t i = 0; i < order.size(); ++i) {
    ldpc::MultiJob m = jobs[(size_t)order[i].j];
    if (order[i].cl) {
      m.item0 = citems;
      citems += m.n_pairs;
      ++nc;
    } else {
      m.item0 = litems;
      litems += (m.n_pairs + m.sub - 1) / m.sub;
    }
    mp.job[i] = m;
  }
  mp.n_jobs = (int32_t)order.size();
  mp.n_cjobs = nc;
  mp.n_citems = citems;
  mp.n_litems = litems;
  mp.cs = b.cs;
  mp.counters = nullptr;
  b.threads = T;
  b.smem = smem;
  if (occupancy && mp.n_jobs > 0) {
    int max_grid = 0;
    const cudaError_t e = ldpc::multi_launch(form, b.es, mp, T, smem, 0, nullptr, &max_grid);
    if (e != cudaSuccess) return cuda_fail(e, "multi-code launch occupancy");
    if (max_grid < 1) return fail(LDPC_ERR_UNSUPPORTED, "no CTA of this shape can be resident");
    int grid = max_grid;
    if (citems == 0) grid = std::min(grid, litems);
    else if (litems == 0) grid = std::min(grid, citems * b.cs);
    b.grid = grid;
  }
  *out = b;
  return LDPC_OK;
}

ldpc_multi_tuning normalize(const ldpc_multi_tuning* t) {
  ldpc_multi_tuning s = {1024, 128, 0, 1, 1, 0, 0};
  if (t != nullptr) {
    if (t->threads) s.threads = t->threads;
    if (t->team_threads) s.team_threads = t->team_threads;
    if (t->cluster) s.cluster = t->cluster;
    if (t->queue) s.queue = t->queue;
    if (t->large) s.large = t->large;
    s.overlap = t->overlap;
    s.stream_warps = t->stream_warps;
  }
  return s;
}

ldpc_status check_tuning(const ldpc_multi_tuning& s) {
  if (s.threads < 256 || s.threads > 1024 || s.threads % 256 != 0)
    return fail(LDPC_ERR_INVALID_ARG, "threads %d is not 256, 512, 768 or 1024", s.threads);
  if (s.team_threads < 32 || s.team_threads > 1024 || (s.team_threads & (s.team_threads - 1)) != 0)
    return fail(LDPC_ERR_INVALID_ARG, "team_threads %d is not a power of two in [32, 1024]", s.team_threads);
  if (s.cluster != 0 && cluster_index(s.cluster) < 0)
    return fail(LDPC_ERR_INVALID_ARG, "cluster %d is not 2, 4, 8 or 16", s.cluster);
  if (s.queue != 1 && s.queue != 2) return fail(LDPC_ERR_INVALID_ARG, "queue %d is not 1 or 2", s.queue);
  if (s.large != 1 && s.large != 2) return fail(LDPC_ERR_INVALID_ARG, "large %d is not 1 or 2", s.large);
  if (s.overlap < 0 || s.overlap > 2) return fail(LDPC_ERR_INVALID_ARG, "overlap %d is not 0, 1 or 2", s.overlap);
  if (s.stream_warps != 0 && s.stream_warps != 4 && s.stream_warps != 8 && s.stream_warps != 16)
    return fail(LDPC_ERR_INVALID_ARG, "stream_warps %d is not 0, 4, 8 or 16", s.stream_warps);
  return LDPC_OK;
}

std::vector<JobIn> job_inputs(const std::vector<ldpc_multi_job>& jobs) {
  std::vector<JobIn> v;
  for (const ldpc_multi_job& j : jobs)
    v.push_back({j.code, j.params, j.llr, j.n_frames, j.hard_bits, j.iters_used, j.syndrome_ok, j.llr_out});
  return v;
}

ldpc_status replan(ldpc_multi* p, const ldpc_multi_tuning& s) {
  ldpc_status st = check_tuning(s);
  if (st != LDPC_OK) return st;
  Built b;
  st = build(job_inputs(p->jobs), p->form, s, true, &b);
  if (st != LDPC_OK) return st;
  p->shape = s;
  if (s.overlap != 0) p->overlap = s.overlap == 2;  // 1 / 2 fix the schedule; 0 keeps the current one
  p->mp = b.mp;
  p->threads = b.threads;
  p->grid = b.grid;
  p->smem = b.smem;
  p->es = b.es;
  p->is_cluster = b.is_cluster;
  p->pairs_per_cta = b.pairs_per_cta;
  p->streamed = b.streamed;
  p->ws_bytes = b.ws_bytes;
  if (b.cs > 1) p->shape.cluster = b.cs;
  return LDPC_OK;
}

// With overlap, the codes on the streaming decoder run on side streams, forked
// from the caller's stream with an event after the persistent kernel and
// joined back with one event each, so that their decodes overlap one another
// (event fork and join is what stream capture records as graph edges).  The
// autotuner keeps it where it measures faster: on the eight-code batch 9.33 ->
// 9.07 ms in the Section V form, but 12.45 -> 12.84 ms in the per-edge form,
// whose plan streams four codes.  Forking before the persistent kernel, so
// that the streaming kernels share the SMs with it, measured slower in both.
cudaError_t ensure_side(const ldpc_multi* p) {
  if (p->fork == nullptr) {
    cudaError_t e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  // a stream and its join event are added together, so the two lists stay in step
  while (p->side.size() < p->streamed.size()) {
    cudaStream_t s;
    cudaEvent_t ev;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaStreamDestroy(s);
      return e;
    }
    p->side.push_back(s);
    p->joined.push_back(ev);
  }
  return cudaSuccess;
}

cudaError_t launch_plan(const ldpc_multi* p, void* ws, cudaStream_t st) {
  ldpc::MultiParams mp = p->mp;
  cudaError_t e = cudaSuccess;
  const bool fork = p->overlap && !p->streamed.empty();
  if (fork) {
    e = ensure_side(p);
    if (e != cudaSuccess) return e;
  }
  if (mp.n_jobs > 0) {
    if (p->shape.queue == 1) {
      mp.counters = static_cast<int32_t*>(ws);
      e = cudaMemsetAsync(ws, 0, 2 * sizeof(int32_t), st);
      if (e != cudaSuccess) return e;
    }
    e = ldpc::multi_launch(p->form, p->es, mp, p->threads, p->smem, p->grid, st, nullptr);
    if (e != cudaSuccess) return e;
  }
  if (fork) {
    e = cudaEventRecord(p->fork, st);
    if (e != cudaSuccess) return e;
  }
  for (size_t i = 0; i < p->streamed.size(); ++i) {
    const ldpc_multi::StreamJob& sj = p->streamed[i];
    cudaStream_t ss = fork ? p->side[i] : st;
    if (fork) {
      e = cudaStreamWaitEvent(ss, p->fork, 0);
      if (e != cudaSuccess) return e;
    }
    const ldpc_multi_job& jb = p->jobs[(size_t)sj.job];
    ldpc::IntRule r;
    r.rule = jb.params.rule;
    r.beta = jb.params.offset;
    r.num = jb.params.norm_num;
    r.shift = jb.params.norm_shift;
    r.qm = jb.params.msg_sat;
    r.psat = 0;
    if (sj.pingpong)
      e = ldpc::pingpong_int8_decode(view(jb.code), r, p->form, sj.pp, static_cast<char*>(ws) + sj.offset, jb.llr,
                                     jb.n_frames, jb.params.max_iter, jb.params.early_stop, jb.hard_bits,
                                     jb.iters_used, jb.syndrome_ok, jb.llr_out, ss,
                                     p->shape.stream_warps ? p->shape.stream_warps : 4);
    else
      e = ldpc::stream_int8_decode(view(jb.code), r, p->form, sj.layout, static_cast<char*>(ws) + sj.offset,
                                   jb.code->sm_count, jb.llr, jb.n_frames, jb.params.max_iter, jb.params.early_stop,
                                   jb.hard_bits, jb.iters_used, jb.syndrome_ok, jb.llr_out, ss);
    if (e != cudaSuccess) return e;
    if (fork) {
      e = cudaEventRecord(p->joined[i], ss);
      if (e != cudaSuccess) return e;
      e = cudaStreamWaitEvent(st, p->joined[i], 0);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace

namespace ldpc_api {

// Splits the code over cs = 2, 4, 8, 16 CTAs (cluster_split.h) and uploads
// the tables.
ldpc_status build_cluster_tables(ldpc_code* c, const int32_t* rp, const int32_t* ci) {
  if (c->N > 65535 || c->ell_w > 16) return LDPC_OK;  // not eligible for the packed kernels
  for (int q = 0; q < kClusterSizes; ++q) {
    const ldpc::ClusterSplit sp = ldpc::split_for_cluster(c->N, c->M, rp, ci, c->ell_w, 2 << q);
    ClusterTables& t = c->ctab[q];
    t = ClusterTables();
    t.cs = sp.cs;
    t.ns = sp.ns;
    t.lb = sp.lb;
    t.mr = sp.mr;
    if (!sp.ok) continue;
    cudaError_t e;
    if ((e = cudaMalloc(&t.d_tab, sp.tab.size() * 2)) != cudaSuccess ||
        (e = cudaMemcpy(t.d_tab, sp.tab.data(), sp.tab.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&t.d_rdeg, sp.rdeg.size())) != cudaSuccess ||
        (e = cudaMemcpy(t.d_rdeg, sp.rdeg.data(), sp.rdeg.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&t.d_rows, sp.rows.size() * 4)) != cudaSuccess ||
        (e = cudaMemcpy(t.d_rows, sp.rows.data(), sp.rows.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "cluster tables");
    t.ok = true;
  }
  return LDPC_OK;
}

void free_cluster_tables(ldpc_code* c) {
  for (ClusterTables& t : c->ctab) {
    cudaFree(t.d_tab);
    cudaFree(t.d_rdeg);
    cudaFree(t.d_rows);
    t = ClusterTables();
  }
}

bool cluster_plan_fits(const ldpc_code* c, const ldpc_decode_params* p) {
  const int form = p->form == LDPC_FORM_SS_1BIT ? 1 : 0;
  std::vector<JobIn> in{{c, *p, nullptr, 2, nullptr, nullptr, nullptr, nullptr}};
  Built b;
  const ldpc_multi_tuning s = normalize(nullptr);
  const std::string saved = ldpc_last_error();
  const bool ok = build(in, form, s, false, &b, p->kernel == LDPC_KERNEL_CLUSTER) == LDPC_OK && b.cs > 1;
  if (!ok) fail(LDPC_OK, "%s", saved.c_str());
  return ok;
}

cudaError_t cluster_decode(const ldpc_code* c, const ldpc_decode_params* p, const int8_t* llr, int32_t F,
                           uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st) {
  const int form = p->form == LDPC_FORM_SS_1BIT ? 1 : 0;
  std::vector<JobIn> in{{c, *p, llr, F, bits, iters, ok, zout}};
  ldpc_multi_tuning s = normalize(nullptr);
  s.queue = 2;
  Built b;
  if (build(in, form, s, true, &b, p->kernel == LDPC_KERNEL_CLUSTER) != LDPC_OK) return cudaErrorInvalidConfiguration;
  return ldpc::multi_launch(form, b.es, b.mp, b.threads, b.smem, b.grid, st, nullptr);
}

}  // namespace ldpc_api

extern "C" {

ldpc_status ldpc_multi_create(ldpc_multi** out, const ldpc_multi_job* jobs, int32_t n_jobs,
                              const ldpc_multi_tuning* tuning) {
  clear_error();
  if (out == nullptr) return fail(LDPC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (jobs == nullptr || n_jobs < 1 || n_jobs > ldpc::kMultiMaxJobs)
    return fail(LDPC_ERR_INVALID_ARG, "jobs must be non-NULL with 1..%d entries", ldpc::kMultiMaxJobs);
  ldpc_multi* p = new ldpc_multi();
  int form = -1, device = -1;
  for (int32_t j = 0; j < n_jobs; ++j) {
    const ldpc_multi_job& jb = jobs[j];
    ldpc_status s = LDPC_OK;
    if (jb.code == nullptr) s = fail(LDPC_ERR_INVALID_ARG, "job %d: code is NULL", j);
    else if (jb.n_frames < 0) s = fail(LDPC_ERR_INVALID_ARG, "job %d: n_frames %d < 0", j, jb.n_frames);
    else if ((s = check_params(jb.code, &jb.params)) != LDPC_OK) fail(s, "job %d: %s", j, ldpc_last_error());
    else if (jb.params.dtype != LDPC_DTYPE_INT8 ||
             (jb.params.form != LDPC_FORM_SS_FIXED && jb.params.form != LDPC_FORM_SS_1BIT) ||
             jb.params.schedule != LDPC_SCHEDULE_FLOODING || jb.params.posterior != LDPC_POSTERIOR_EXACT)
      s = fail(LDPC_ERR_UNSUPPORTED, "job %d: batches run int8 single-scan decodes (SS_FIXED or SS_1BIT, flooding "
               "schedule, exact posterior)", j);
    else if (form >= 0 && jb.params.form != form)
      s = fail(LDPC_ERR_INVALID_ARG, "job %d: every job of a batch must use the same form", j);
    else if (device >= 0 && jb.code->device != device)
      s = fail(LDPC_ERR_INVALID_ARG, "job %d: codes of one batch must be on one device", j);
    else if (jb.n_frames > 0 && (jb.llr == nullptr || jb.hard_bits == nullptr || jb.iters_used == nullptr ||
                                 jb.syndrome_ok == nullptr))
      s = fail(LDPC_ERR_INVALID_ARG, "job %d: llr, hard_bits, iters_used and syndrome_ok must be non-NULL", j);
    if (s != LDPC_OK) {
      delete p;
      return s;
    }
    form = jb.params.form;
    device = jb.code->device;
    if (jb.n_frames > 0) {
      p->jobs.push_back(jb);
      p->user_index.push_back(j);
    }
  }
  p->n_user = n_jobs;
  p->form = form == LDPC_FORM_SS_1BIT ? 1 : 0;
  p->device = device;
  if (p->jobs.empty()) {
    delete p;
    return fail(LDPC_ERR_INVALID_ARG, "no job has frames");
  }
  DeviceGuard guard(device);
  const ldpc_status s = replan(p, normalize(tuning));
  if (s != LDPC_OK) {
    delete p;
    return s;
  }
  *out = p;
  return LDPC_OK;
}

ldpc_status ldpc_multi_destroy(ldpc_multi* plan) {
  clear_error();
  if (plan == nullptr) return LDPC_OK;
  DeviceGuard guard(plan->device);  // its side streams and events belong to that device
  delete plan;
  return LDPC_OK;
}

ldpc_status ldpc_multi_workspace_size(const ldpc_multi* plan, size_t* bytes) {
  clear_error();
  if (plan == nullptr || bytes == nullptr) return fail(LDPC_ERR_INVALID_ARG, "plan and bytes must be non-NULL");
  *bytes = plan->ws_bytes;
  return LDPC_OK;
}

ldpc_status ldpc_multi_decode(const ldpc_multi* plan, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  if (plan == nullptr) return fail(LDPC_ERR_INVALID_ARG, "plan is NULL");
  if (workspace == nullptr || ws_bytes < plan->ws_bytes)
    return fail(LDPC_ERR_INVALID_ARG, "workspace of %zu bytes needed, %zu given", plan->ws_bytes,
                workspace ? ws_bytes : (size_t)0);
  if (((uintptr_t)workspace & 255u) != 0) return fail(LDPC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  DeviceGuard guard(plan->device);
  const cudaError_t e = launch_plan(plan, workspace, (cudaStream_t)stream);
  return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "ldpc_multi_decode launch");
}

ldpc_status ldpc_multi_autotune(ldpc_multi* plan, void* workspace, size_t ws_bytes, int32_t reps, void* stream,
                                ldpc_multi_tuning* chosen, float* best_ms) {
  clear_error();
  if (plan == nullptr) return fail(LDPC_ERR_INVALID_ARG, "plan is NULL");
  if (reps < 1) return fail(LDPC_ERR_INVALID_ARG, "reps %d < 1", reps);
  if (workspace == nullptr || ((uintptr_t)workspace & 255u) != 0)
    return fail(LDPC_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
  DeviceGuard guard(plan->device);
  cudaStream_t st = (cudaStream_t)stream;
  const ldpc_multi_tuning start = plan->shape;
  // codes that do not fit one CTA: streaming (cluster size irrelevant) or
  // clusters of every size from the smallest that fits
  std::vector<std::pair<int, int>> modes{{1, 0}};
  bool any_large = false;
  for (int32_t v : plan->is_cluster) any_large = any_large || v != 0;
  if (any_large) {
    ldpc_multi_tuning probe = start;
    probe.large = 2;
    probe.cluster = 0;
    if (replan(plan, probe) == LDPC_OK)
      for (int cs = plan->shape.cluster; cs <= 16; cs *= 2) modes.push_back({2, cs});
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  // mean time of one launch of the current plan over n launches (after one
  // untimed launch)
  auto time_plan = [&](int n, float* ms) -> cudaError_t {
    cudaError_t e = launch_plan(plan, workspace, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < n && e == cudaSuccess; ++r) e = launch_plan(plan, workspace, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e == cudaSuccess) *ms /= (float)n;
    return e;
  };
  plan->overlap = false;
  ldpc_multi_tuning best = start;
  float best_t = -1.0f;
  ldpc_status result = LDPC_OK;
  for (int T : {512, 1024})
    for (int tt : {64, 128, 256})
      for (const std::pair<int, int>& md : modes) {
        ldpc_multi_tuning s = start;
        s.threads = T;
        s.team_threads = tt;
        s.large = md.first;
        s.cluster = md.second;
        if (replan(plan, s) != LDPC_OK || plan->ws_bytes > ws_bytes) continue;
        float ms = 0.0f;
        const cudaError_t e = time_plan(reps, &ms);
        if (e != cudaSuccess) {
          result = cuda_fail(e, "autotune candidate");
          break;
        }
        if (best_t < 0.0f || ms < best_t) best_t = ms, best = plan->shape;
      }
  ldpc_status s = LDPC_OK;
  if (result == LDPC_OK && best_t >= 0.0f) {
    s = replan(plan, best);
    // the chosen shape with and without the streamed codes overlapped, timed
    // back to back over at least 5 launches each; the faster is kept
    if (s == LDPC_OK && !plan->streamed.empty() && start.overlap != 0) {
      plan->shape.overlap = start.overlap;  // fixed by the caller: kept
      plan->overlap = start.overlap == 2;
    } else if (s == LDPC_OK && !plan->streamed.empty()) {
      const int n = reps > 5 ? reps : 5;
      float t_seq = 0.0f, t_ovl = 0.0f;
      plan->overlap = false;
      cudaError_t e = time_plan(n, &t_seq);
      if (e == cudaSuccess) {
        plan->overlap = true;
        e = time_plan(n, &t_ovl);
      }
      if (e != cudaSuccess) {
        plan->overlap = false;
        result = cuda_fail(e, "autotune overlap");
      } else {
        plan->overlap = t_ovl < t_seq;
        best_t = plan->overlap ? t_ovl : t_seq;
      }
    }
    // warps per CTA of the ping-pong row kernel for the streamed codes: the
    // workspace does not depend on it, so the plan is timed as it stands
    bool any_pp = false;
    for (const ldpc_multi::StreamJob& sj : plan->streamed) any_pp = any_pp || sj.pingpong;
    if (s == LDPC_OK && result == LDPC_OK && any_pp && start.stream_warps == 0) {
      const int n = reps > 5 ? reps : 5;
      int best_w = 8;
      float best_wt = -1.0f;
      for (int w : {4, 8, 16}) {
        plan->shape.stream_warps = w;
        float ms = 0.0f;
        const cudaError_t e = time_plan(n, &ms);
        if (e != cudaSuccess) {
          result = cuda_fail(e, "autotune stream_warps");
          break;
        }
        if (best_wt < 0.0f || ms < best_wt) best_wt = ms, best_w = w;
      }
      plan->shape.stream_warps = best_w;
      if (result == LDPC_OK) best_t = best_wt;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != LDPC_OK) return result;
  if (best_t < 0.0f) return fail(LDPC_ERR_UNSUPPORTED, "no candidate shape could be planned");
  if (s != LDPC_OK) return s;
  if (chosen) *chosen = plan->shape;
  if (best_ms) *best_ms = best_t;
  return LDPC_OK;
}

ldpc_status ldpc_multi_info(const ldpc_multi* plan, ldpc_multi_tuning* shape, int32_t* grid, int32_t* cluster,
                            int32_t* smem_bytes, int32_t* job_is_cluster, int32_t* job_pairs_per_cta) {
  clear_error();
  if (plan == nullptr) return fail(LDPC_ERR_INVALID_ARG, "plan is NULL");
  if (shape) *shape = plan->shape;
  if (grid) *grid = plan->grid;
  if (cluster) *cluster = plan->mp.cs;
  if (smem_bytes) *smem_bytes = (int32_t)plan->smem;
  for (int32_t j = 0; j < plan->n_user; ++j) {
    if (job_is_cluster) job_is_cluster[j] = -1;  // a job without frames
    if (job_pairs_per_cta) job_pairs_per_cta[j] = 0;
  }
  for (size_t j = 0; j < plan->jobs.size(); ++j) {
    const int32_t u = plan->user_index[j];
    if (job_is_cluster) job_is_cluster[u] = plan->is_cluster[j];
    if (job_pairs_per_cta) job_pairs_per_cta[u] = plan->pairs_per_cta[j];
  }
  return LDPC_OK;
}

}  // extern "C"

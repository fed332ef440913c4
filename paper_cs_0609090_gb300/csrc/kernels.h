// kernels.h -- host-side launch interface between the C ABI layer and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ldpc {

// Launch configuration of the frame-resident ("on-chip") kernel: every CTA
// keeps G frames' posteriors, accumulators and check state in shared memory for
// all iterations.
struct OnchipPlan {
  int G = 0;            // frames per CTA (even)
  int threads = 0;      // threads per CTA
  size_t smem = 0;      // dynamic shared memory bytes
  int grid = 0;         // CTAs launched (persistent over frame groups)
  int n_groups = 0;
  int dmax = 0;         // unrolled row-degree bound (packed-half kernel)
  bool sidx = false;    // column table copied into shared memory
  bool rset = false;    // accumulator reset values kept in shared memory
};

// Fills *plan for an int8 decode (form: 0 fixed, 1 one-bit).  Returns false if
// no G fits in shared memory.
bool onchip_int8_plan(const DevCode& c, int form, int32_t n_frames, int sm_count,
                      size_t smem_optin, int max_row_deg, OnchipPlan* plan);

// Sets plan->grid from the occupancy of the chosen instantiation (persistent grid).
cudaError_t onchip_int8_occupancy(int form, int sm_count, OnchipPlan* plan);

cudaError_t onchip_int8_launch(const DevCode& c, const IntRule& r, int form, const OnchipPlan& plan,
                               const int8_t* llr, int32_t n_frames, int32_t max_iter,
                               int32_t early_stop, uint8_t* bits, int32_t* iters, uint8_t* ok,
                               int16_t* zout, cudaStream_t stream);

// Packed binary16 variant (two frames per instruction, exact for integers < 2048).
bool onchip_h2_eligible(int n_vars, int max_row_deg, int max_col_deg, int qm, int rule, int num);
bool onchip_h2_plan(const DevCode& c, int form, int32_t n_frames, int sm_count, size_t smem_optin,
                    int max_row_deg, OnchipPlan* plan);
// Sets plan.grid from occupancy; launches unless occupancy_only.
cudaError_t onchip_h2_launch(const DevCode& c, const IntRule& r, int form, OnchipPlan& plan, int sm_count,
                             const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                             int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t stream, bool occupancy_only);

// Two-scan comparator (Section III), frame-resident, exact binary16 pairs.
bool onchip_twoscan_plan(const DevCode& c, int32_t n_frames, int sm_count, size_t smem_optin, int max_row_deg,
                         OnchipPlan* plan);
cudaError_t onchip_twoscan_launch(const DevCode& c, const IntRule& r, OnchipPlan& plan, int sm_count,
                                  const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                                  int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t stream);

// Persistent multi-code launch (multi_h2.cu).  Jobs [0, n_cjobs) are cluster
// jobs (one frame pair per cluster of cs CTAs), the rest local jobs (`sub` frame
// pairs per CTA, one per sub-team); items are numbered per queue from item0.
constexpr int kMultiMaxJobs = 16;
constexpr int kMultiMaxSub = 8;
struct MultiJob {
  int32_t N, M, ell_w;
  int32_t mr;       // rows per table (local: M; cluster: row capacity of a rank, even)
  int32_t ns, lb;   // cluster: variables per rank, local-index bits of a table entry
  int32_t sub;      // local: frame pairs per CTA
  int32_t n_pairs, item0;
  const uint16_t* tab;   // local: the code's ell16 [ell_w][M]; cluster: [cs][ell_w][mr] packed
  const uint8_t* rdeg;   // local: [M]; cluster: [cs][mr]
  const int32_t* rows;   // cluster: [cs] checks per rank
  const int32_t* cdeg;   // [N]
  int32_t beta, num, shift, qm, max_iter, early_stop;  // H2Rule fields, Qm, cap
  const int8_t* llr;
  int32_t F;
  uint8_t* bits;
  int32_t* iters;
  uint8_t* ok;
  int16_t* zout;
  uint32_t tab_bytes, slot_bytes, acc_off, st_off;  // shared-memory layout
  uint32_t rs_off;  // local jobs: offset of the accumulator reset values in a slot (0: none)
};
struct MultiParams {
  int32_t n_jobs, n_cjobs, n_citems, n_litems, cs;
  int32_t* counters;  // [2] zero before the launch, or nullptr: round-robin items
  MultiJob job[kMultiMaxJobs];
};
// Bytes of one local pair slot (Zs, Acc, St or Lm, and with rset the
// accumulator reset values) and its offsets.
size_t multi_local_slot_bytes(int N, int M, int ell_w, int form, size_t* acc_off, size_t* st_off,
                              bool rset = false, size_t* rs_off = nullptr);
// Launches (max_grid == nullptr) or reports the persistent grid of a shape.
cudaError_t multi_launch(int form, bool es, const MultiParams& mp, int threads, size_t smem, int grid,
                         cudaStream_t st, int* max_grid);

// The single scan in a layered schedule (layered_h2.cu): frame-pair chunks,
// one CTA per chunk, state in the workspace.  lay_ptr [n_layers + 1] and
// lay_rows [M]: the internal check indices of each layer.
struct LayeredLayout {
  int chunks = 0, pw = 8;     // frame pairs per chunk (one CTA each)
  bool sidx = false;          // column table in shared memory
  bool zsm = false;           // the chunk's posteriors in shared memory
  size_t smem = 0, zsm_off = 0;
  size_t hdr = 0;             // workspace: queue counter, then per chunk [Z][state]
  size_t st_off = 0, chunk_bytes = 0, total = 0;
};
LayeredLayout layered_layout(int form, int N, int M, int ell_w, int F, bool narrow, size_t smem_optin);
cudaError_t layered_decode(const DevCode& c, const IntRule& r, int form, const int32_t* lay_ptr,
                           const int32_t* lay_rows, int n_layers, const int8_t* llr, int32_t F, int32_t max_iter,
                           int32_t early_stop, uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, void* ws,
                           const LayeredLayout& L, int sm_count, cudaStream_t st);

// Device-memory (streaming) decoders for codes whose frame state does not fit
// one SM.  All state lives in the caller's workspace (layout below).
struct StreamLayout {
  int lanes = 0;  // frame pairs (int8) or frames (float32), padded to 32
  size_t z = 0, acc = 0, st = 0, q0 = 0, act = 0, fail = 0, iters = 0, ok = 0, total = 0;
};
// E: message slots of the per-edge form (the degree-sorted table's ell_w * M;
// float32 gets max(E, ell_w * M), its sum-product rule addressing the E edges
// of H).
StreamLayout stream_layout(int dtype, int form, int N, int M, int E, int F);
bool stream_int8_eligible(int max_row_deg, int max_col_deg, int qm);
cudaError_t stream_int8_decode(const DevCode& c, const IntRule& r, int form, const StreamLayout& L, void* ws,
                               int sm_count, const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop,
                               uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st);
cudaError_t stream_f32_decode(const DevCode& c, const F32Rule& r, int form, const StreamLayout& L, void* ws,
                              int sm_count, const float* llr, int32_t F, int32_t max_iter, int32_t early_stop,
                              uint8_t* bits, int32_t* iters, uint8_t* ok, float* zout, cudaStream_t st);

// The ping-pong streaming decoder (pingpong.cu): one kernel launch per
// iteration, two posterior buffers accumulated with exact f16x2 atomics (no
// column pass), two frame pairs per lane; codes whose checks have degree <= 8.
struct PingpongLayout {
  int lanes = 0;   // frame pairs, padded to 64
  int ub = 0;      // bytes per state unit and pair (8: Section V; 2: a per-edge message)
  int rows = 0;    // state units per buffer: M (Section V) or ell_w M (per edge)
  size_t zb = 0, st = 0, act = 0, fail = 0, iters = 0, ok = 0, total = 0;
};
PingpongLayout pingpong_layout(int form, int N, int M, int ell_w, int F);
// Sets the ping-pong row kernels' shared-memory attribute on the current
// device (once per device, outside stream capture).
cudaError_t pingpong_prepare();
bool pingpong_int8_eligible(int N, int M, int ell_w, int max_row_deg, int max_col_deg, int qm, int form, int F);
// warps: warps per block of the row kernel (4, 8 or 16; four checks per warp).
cudaError_t pingpong_int8_decode(const DevCode& c, const IntRule& r, int form, const PingpongLayout& L, void* ws,
                                 const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                                 int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st, int warps = 8);

// The two-scan algorithm of Section III with the frame state in device memory
// (twoscan_stream.cu), any code size: per-edge Z_mn, and the check messages per
// edge (form2 0) or as the Section V state (form2 1).
struct TwoScanLayout {
  int lanes = 0;   // frame pairs, padded to 64
  bool c8 = false; // compressed state in 8 bytes per pair (check degree <= 8), else 16
  int ub = 0;
  int dvmax = 16;  // largest column degree of the code (set by the caller; <= 16)
  size_t zmn = 0, lmn = 0, st = 0, q0 = 0, zp = 0, act = 0, fail = 0, iters = 0, ok = 0, total = 0;
};
// Sets the staged two-scan vertical kernels' shared-memory attribute on the
// current device (once per device, outside stream capture).
cudaError_t twoscan_prepare();
TwoScanLayout twoscan_layout(int form2, int N, int M, int ell_w, int F);
bool twoscan_stream_eligible(int N, int M, int ell_w, int max_row_deg, int max_col_deg, int qm, int form2, int F);
cudaError_t twoscan_stream_decode(const DevCode& c, const IntRule& r, int form2, const TwoScanLayout& L, void* ws,
                                  const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop, uint8_t* bits,
                                  int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st);

// The persistent streaming decoder (persist.cu): one kernel launch per decode,
// a work queue over (chunk of 32 frame pairs, iteration, tile of checks) that
// runs groups of W chunks through all their iterations while their state stays
// in L2; two posterior buffers updated with exact f16x2 atomics, no column pass.
struct PersistLayout {
  int lanes = 0, chunks = 0, W = 1;
  bool c8 = false;     // Section V state in 8 bytes per pair (every check degree <= 8)
  int ub = 0;          // bytes per state unit and pair (8 / 16, or 2 for a per-edge message)
  int rows = 0;        // state units per buffer: M (Section V) or ell_w M (per edge)
  size_t zb = 0, st = 0, act = 0, fail = 0, iters = 0, ok = 0, ctl = 0, total = 0;
};
PersistLayout persist_layout(int form, int N, int M, int ell_w, int F, int group_chunks);
bool persist_int8_eligible(int N, int M, int ell_w, int max_row_deg, int max_col_deg, int qm, int form, int F);
cudaError_t persist_int8_decode(const DevCode& c, const IntRule& r, int form, const PersistLayout& L, void* ws,
                                int sm_count, const int8_t* llr, int32_t F, int32_t max_iter, int32_t early_stop,
                                uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st);
// Runs the queue's bounded wait on a counter that nothing increments (one CTA,
// max_spins polls) and reports whether it gave up.  Synchronous.
cudaError_t persist_wait_selftest(uint32_t max_spins, bool* gave_up);

// Learned offsets beta[k][class]: workspace layout and launchers (learned.cu).
struct LearnedLayout {
  int FL = 0, tasks = 0;
  size_t zck = 0, sck = 0, dz = 0, du = 0, part = 0, lpart = 0, total = 0;
};
LearnedLayout learned_layout(int N, int M, int K, int C, int F);
// A check's degree class is the index of its degree run in the internal
// (degree-sorted) order: the classes are the distinct degrees, ascending.
cudaError_t learned_forward(const DevCode& c, int C, int K, const float* beta, const LearnedLayout& L, void* ws,
                            const float* llr, int F, float* zout, cudaStream_t st);
cudaError_t learned_bce(const DevCode& c, int C, int K, const LearnedLayout& L, void* ws, int F,
                        const uint8_t* tbits, float* loss, bool want_grad, cudaStream_t st);
cudaError_t learned_backward(const DevCode& c, int C, int K, const float* beta, const LearnedLayout& L, void* ws,
                             const float* dz_in, int F, float* dbeta, cudaStream_t st);
cudaError_t adam_step(float* p, const float* g, float* m, float* v, int n, int step, float lr, float b1, float b2,
                      float eps, cudaStream_t st);
cudaError_t awgn_llr(int N, uint64_t seed, uint64_t first_frame, int F, float lo, float hi, float rate,
                     const uint8_t* cw, float* llr, float* ebn0_out, cudaStream_t st);
cudaError_t quantize_llr(const float* llr, size_t n, float delta, int qc, int8_t* q, cudaStream_t st);

}  // namespace ldpc

// api_internal.h -- what the C-ABI translation units share: the device copy of
// a code, error reporting and the device guard.  Not part of the public ABI.
#pragma once
#include <string>
#include <vector>

#include "../../include/ldpc_gb300.h"
#include "kernels.h"

// A code split over the CTAs of a thread-block cluster of cs CTAs: CTA rank r
// holds variables [r ns, (r+1) ns) and the checks listed in its part of tab.
// Entry (r, j, i) of tab is (rank << lb) | local index of position j of the
// rank's i-th check (checks sorted by degree; positions past the degree repeat
// the last variable; rows past rows[r] are padding).
struct ClusterTables {
  int cs = 0, ns = 0, lb = 0, mr = 0;
  bool ok = false;
  uint16_t* d_tab = nullptr;   // [cs][ell_w][mr]
  uint8_t* d_rdeg = nullptr;   // [cs][mr]
  int32_t* d_rows = nullptr;   // [cs]
};
constexpr int kClusterSizes = 4;  // cs = 2, 4, 8, 16
inline int cluster_index(int cs) { return cs == 2 ? 0 : cs == 4 ? 1 : cs == 8 ? 2 : cs == 16 ? 3 : -1; }

struct ldpc_code {
  int device = 0;
  int32_t N = 0, M = 0, E = 0;
  int32_t max_row_deg = 0, max_col_deg = 0;
  int32_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  int32_t* d_cdeg = nullptr;
  uint16_t* d_ell16 = nullptr;
  int32_t* d_ell32 = nullptr;
  uint8_t* d_rdeg = nullptr;
  int32_t* d_cptr = nullptr;
  int32_t* d_cslot = nullptr;
  uint32_t* d_ccj = nullptr;
  int32_t n_classes = 0;
  int32_t class_deg[32] = {};       // check degree of each class, ascending
  int32_t ell_w = 0;
  int32_t n_dc = 0;                 // degree runs of the internal order (0: more than 4)
  int32_t dc_end[4] = {};
  int32_t dc_deg[4] = {};
  int sm_count = 0;
  size_t smem_optin = 0;
  ClusterTables ctab[kClusterSizes];
  // layered schedule: layer of every check (original order) and, on the device,
  // the internal check indices of each layer
  std::vector<int32_t> layer_of_check;
  int32_t n_layers = 0;
  int32_t* d_lay_ptr = nullptr;   // [n_layers + 1]
  int32_t* d_lay_rows = nullptr;  // [M]
  std::vector<int32_t> pos;       // internal index of each original check
  std::vector<int32_t> h_row_ptr, h_col_idx;
};

namespace ldpc_api {

void clear_error();
ldpc_status fail(ldpc_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
ldpc_status cuda_fail(cudaError_t e, const char* what);

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

ldpc::DevCode view(const ldpc_code* c);
// Uploads a layer partition (validated: the checks of a layer share no variable).
ldpc_status set_layers(ldpc_code* c, int32_t n_layers, const int32_t* layer_of_check);
ldpc_status check_params(const ldpc_code* c, const ldpc_decode_params* p);

// Cluster split of a code (multi_api.cu): built by ldpc_code_create for every
// code the packed kernels accept, released by ldpc_code_destroy.
ldpc_status build_cluster_tables(ldpc_code* c, const int32_t* row_ptr, const int32_t* col_idx);
void free_cluster_tables(ldpc_code* c);
// Whether a single-code int8 single-scan decode runs on a cluster (it does not
// fit one CTA but fits a cluster; with kernel LDPC_KERNEL_CLUSTER whenever it
// fits a cluster), and that decode (round-robin items).
bool cluster_plan_fits(const ldpc_code* c, const ldpc_decode_params* p);
cudaError_t cluster_decode(const ldpc_code* c, const ldpc_decode_params* p, const int8_t* llr, int32_t F,
                           uint8_t* bits, int32_t* iters, uint8_t* ok, int16_t* zout, cudaStream_t st);

}  // namespace ldpc_api

// Host-side objects of libhm (trees, matrices) and helpers shared by the
// runtime translation units (products, batching, serving).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda.h>

#include "hm_internal.h"

namespace hmi {

constexpr uint32_t kMagicTree = 0x31545248u;     // "HRT1"
constexpr uint32_t kMagicMatrix = 0x314d5248u;   // "HRM1"
constexpr uint32_t kMagicBatch = 0x31425248u;    // "HRB1"
constexpr uint32_t kMagicServer = 0x31535248u;   // "HRS1"

// A typed generator plane being packed on the host (hi and, for BF16X2, lo).
struct Plane {
  int storage = HM_F64;
  size_t count = 0;
  std::vector<uint8_t> hi, lo;
  void init(int st, size_t cnt);
  void set(size_t i, double v);
};

uint16_t f64_to_bf16(double a);
double bf16_to_f64(uint16_t h);
size_t storage_bytes(int st);
int* device_error_word(int dev);
// cudaMalloc, unless a failure was injected with hm_inject_alloc_failures.
cudaError_t dev_malloc(void** p, size_t bytes);
// The timeout self-test kernel (hm_fault.cu).
hm_status launch_selftest_timeout(DeviceStatusBlock* b, cudaStream_t s);
const double* host_block(const double* p, size_t count, std::vector<double>& tmp);

}  // namespace hmi

struct hm_tree {
  uint32_t magic;
  int64_t n;
  int p;
  int L;
  std::vector<int64_t> ends;
};

struct hm_matrix {
  uint32_t magic = 0;
  int kind = 0;
  int storage = 0;
  int device = 0;
  int64_t n = 0;
  int p = 0, L = 1;
  std::vector<int64_t> ends;
  int m_max = 0, m_pad = 16, Ke = 0, Kp = 0, We = 16;
  int ku_max = 0, kv_max = 0;   // HSS: largest row / column rank before padding (Ke, Kp: padded to 8)
  int kk[hmi::kMaxDepth + 2] = {0};
  int koff[hmi::kMaxDepth + 2] = {0};
  int64_t gen_elems = 0;
  size_t gen_bytes = 0;
  size_t dev_bytes = 0;
  int64_t* d_off = nullptr;
  void* d_A = nullptr;
  void* d_A_lo = nullptr;
  void* d_W = nullptr;
  void* d_W_lo = nullptr;
  void* d_RU = nullptr;
  void* d_RVt = nullptr;
  void* d_B12 = nullptr;
  void* d_B21 = nullptr;
  int64_t r_cap = 0;
  void* d_ws = nullptr;
  int* d_cnt = nullptr;
  void* d_io = nullptr;
  size_t io_cap = 0;
  int* err = nullptr;
  int path = 0;
  int tree_mode = 0;            // 0 automatic, 1 level kernels, 2 cluster kernel when it fits
  int64_t tree_ok_r = -1;       // r for which the cluster kernel's residency was checked
  bool tree_ok = false;
  int tree_rc = 0;              // launch shape chosen for tree_ok_r: columns per cluster,
  int tree_s = 0;               //   levels shared by the cluster (2^s CTAs),
  int tree_ns = 0;              //   operator ring slots
  bool tree_last_cluster = false;  // the last product ran the cluster tree kernel
  hmi::Prof* prof = nullptr;   // set while profiling is enabled
  CUtensorMap tmA;              // TMA descriptors of the expansion planes (BF16 / BF16X2)
  CUtensorMap tmAlo;
  CUtensorMap tmW;              // ... and of the projection planes
  CUtensorMap tmWlo;
  bool tm_ok = false;
  bool tmw_ok = false;
  int w_box = 128;              // rows of a projection TMA box (min(Kp, 128))
  hmi::MatView view() const;
};

namespace hmi {

int64_t node_start(const hm_tree* t, int q);
int64_t node_end(const hm_tree* t, int q);
hm_status ensure_scratch(hm_matrix* A, int64_t r);

// CUDA-event timing of the phases of the products of one matrix (slots as in
// hm_matrix_phase_times).
constexpr int kPhaseSlots = 5;
class EventProf : public Prof {
 public:
  void mark(int phase, bool start, cudaStream_t s) override;
  hm_status read(double ms[kPhaseSlots], int64_t launches[kPhaseSlots]);
  ~EventProf() override;

 private:
  struct Rec { int phase; cudaEvent_t a, b; };
  std::vector<Rec> recs_;
  std::vector<cudaEvent_t> pool_;
  cudaEvent_t open_[kPhaseSlots] = {};
  double ms_[kPhaseSlots] = {};
  int64_t n_[kPhaseSlots] = {};
  cudaEvent_t get();
};
Scratch scratch_of(const hm_matrix* A, int64_t r);
hm_status run_product(const hm_matrix* A, int want_kind, int64_t r, const void* X, int64_t ldx, int xt,
                      void* Y, int64_t ldy, int yt, void* stream);
hm_status launch_product(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                         int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t s);
// Tensor-core expansion (k_tc.cu).
void make_tensor_maps(hm_matrix* A);
bool use_tensor_cores(const hm_matrix* A, int64_t r);
// Shape of the tensor-core expansion (proj = false) or projection (proj =
// true) of A for r columns (false if none fits).
bool tc_plan(const hm_matrix* A, int64_t r, bool proj, int* nt, int* nK, int* nX, int* nst, int* tiles);
// Tree phases of one product (HSS upsweep, couplings and downsweep; HODLR
// sums) in one cluster launch; HM_EUNSUPPORTED when the shape does not fit
// (the level kernels then run).
hm_status launch_tree_cluster(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, cudaStream_t st,
                              bool pdl);
bool tree_cluster_usable(hm_matrix* A, const MatView& mv, int64_t r);
hm_status tune_tree_cluster(hm_matrix* A, int64_t r, int xt, int yt, double* best_ms);
hm_status set_tree_shape(hm_matrix* A, int64_t r, int cluster_ctas, int columns, int ring_slots);
hm_status launch_project_tc(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                            int64_t ldx, int xt, cudaStream_t st, bool pdl);
size_t tc_tile_smem(bool split, int NT, int nK, int nst);
int tc_tile_ncols(bool split, int NT);
hm_status launch_expand_tc(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                           int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl);

// Releases batch and server objects (defined with them).
void destroy_other(void* any, uint32_t magic);
void destroy_server(void* any);
void destroy_ulv(void* any);
bool is_ulv(const void* any);

}  // namespace hmi

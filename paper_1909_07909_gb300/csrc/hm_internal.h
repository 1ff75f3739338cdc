// Internal structures of libhm shared by the host runtime and the kernels.
//
// Device layout of one matrix (all generator planes row-major, storage type S):
//
//  * Expansion operand  Aexp: n rows x We columns, We = m_pad + Ke.  Row g of
//    leaf i holds [ D_i(g,:) | 0 ... | E_i(g,:) ] where the D part occupies
//    columns [0, m_i), zeros fill [m_i, m_pad) and E_i starts at column m_pad:
//      HODLR: E_i = [U^(1)(g,:) | ... | U^(p)(g,:)], the row factors of the
//             leaf's ancestors at levels 1..p (level l block at koff[l], width kk[l]);
//      HSS:   E_i = U_i(g,:), the leaf row basis.
//    One leaf's output block is then a single product
//      Y(I_i, :) = [D_i | E_i] [X(I_i, :); Z_i]
//    with Z_i the per-level T's (HODLR) or the leaf y-hat (HSS).
//  * Projection operand Wprj: L*Kp rows x m_pad columns; rows i*Kp .. i*Kp+Kp-1
//    hold the transposed column factors of leaf i's rows (HODLR: the V of each
//    level, at the same offsets koff[l]; HSS: V_i^T), zero-padded to m_pad.
//  * HSS tree operators in the compute type C (double for F64 storage, float
//    otherwise), one block per internal node q (0..L-2), stored so that every
//    product reads them as "transposed" matrices Mt[j][i] (inner index i
//    contiguous, which is conflict-free for consecutive threads):
//      RU  [q][h][j][i] = R_U(h*Ke + i, j)   (h = 0 left child half, 1 right)
//      RV  [q][j][i]    = R_V(j, i), j over the stacked children (2Kp rows)
//      B12 [q][j][i]    = B12(i, j),  B21 [q][j][i] = B21(i, j)   (Kp x Ke)
//    (root entries of RU/RV are unused).
//
// Scratch of one product with r columns (compute type C), node-major:
//  HODLR  PS[node][col][e], e < Ke: a leaf holds V^T X of its rows for every
//         level; an internal node at level l holds, in rows of levels 1..l, the
//         sums over its leaves, so PS[node][.][koff[l]..] is T_node^(l).
//  HSS    xh[node][col][e] (e < Kp), yc / yf [node][col][e] (e < Ke).
//  cnt    (L-1) x nchunks arrival counters, zero before and after every call.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "hm.h"

namespace hmi {

constexpr int kMaxDepth = 30;

struct MatView {
  int kind;      // hm_kind
  int storage;   // hm_dtype
  int p, L;
  int m_pad;     // padded leaf width (multiple of 16)
  int Ke;        // width of the expansion factor part (multiple of 8)
  int Kp;        // projection rows per leaf (multiple of 8)
  int We;        // m_pad + Ke
  int64_t n;
  const int64_t* off;   // device, L+1 leaf offsets
  const void* A;        // expansion operand (hi plane for BF16X2)
  const void* A_lo;     // lo plane (BF16X2) or nullptr
  const void* W;        // projection operand
  const void* W_lo;
  const void* RU;       // HSS tree operators (compute type), layouts above
  const void* RV;
  const void* B12;
  const void* B21;
  int kk[kMaxDepth + 2];    // HODLR padded rank of level l (index 1..p)
  int koff[kMaxDepth + 2];  // HODLR offset of level l inside the Ke block
};

// Optional per-kernel event timing (phase 0 project, 1 tree upsweep, 2 HSS
// downsweep, 3 expand, 4 FP64 diagonal-block product run apart from the expansion).
struct Prof {
  virtual void mark(int phase, bool start, cudaStream_t s) = 0;
  virtual ~Prof() {}
};

inline void prof_mark(Prof* p, int phase, bool start, cudaStream_t s) {
  if (p) p->mark(phase, start, s);
}

// The per-device status block of the library's bounded device waits: the
// error word a kernel sets when a wait gives up (read and cleared by
// hm_device_status), a flag word that nothing in the product path sets (the
// timeout self-test waits on it), and the wait limit in nanoseconds
// (hm_set_device_wait_limit).  Kernels receive a pointer to `err`.
struct DeviceStatusBlock {
  int err;
  int flag;
  unsigned long long wait_ns;
};
constexpr uint64_t kDefaultWaitNs = 2000000000ull;

// The wait limit of the status block whose error word is `err` (the default
// when there is none).
__device__ __forceinline__ uint64_t wait_limit_ns(const int* err) {
  return err ? reinterpret_cast<const volatile DeviceStatusBlock*>(err)->wait_ns : kDefaultWaitNs;
}

struct Scratch {
  void* PS;   // HODLR partial sums
  void* xh;   // HSS
  void* yc;
  void* yf;
  int* cnt;
  int* err;   // device error word (bounded waits)
  Prof* prof; // host-side timing hook or nullptr (never read by kernels)
};

// One phase of the SIMT path (0 projection, 1 tree upsweep / sums, 2 HSS
// downsweep, 3 leaf expansion) for one storage type; `pdl` launches it with programmatic stream
// serialization.  Defined in k_simt_<type>.cu.
#define HM_SIMT_PHASE_DECL(T)                                                                       \
  hm_status simt_phase_##T(int phase, const MatView& mv, const Scratch& ws, int64_t r, const void* X, \
                           int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t s, bool pdl);
HM_SIMT_PHASE_DECL(f64)
HM_SIMT_PHASE_DECL(f32)
HM_SIMT_PHASE_DECL(bf16)
HM_SIMT_PHASE_DECL(bf16x2)
#undef HM_SIMT_PHASE_DECL

// Scratch element counts for r columns (in compute-type elements) and counter
// count: the tree kernels' arrival counters, then 8 work counters of the FP64
// leaf kernels.
size_t scratch_elems(const MatView& mv, int64_t r);
size_t tree_counter_count(const MatView& mv, int64_t r);
size_t counter_count(const MatView& mv, int64_t r);

// FP64 storage with at least this many right-hand sides runs the register-tiled
// FP64 leaf kernels (k_f64.cu); narrower blocks run the SIMT row engine.
constexpr int kF64TiledMinR = 12;
bool f64_tiled(const MatView& mv, int64_t r);
inline int* f64_counters(const Scratch& ws, const MatView& mv, int64_t r) {
  return ws.cnt + tree_counter_count(mv, r);
}
// One FP64 leaf phase: 0 projection (x-hat / per-level V^T X), 1 diagonal-block
// product Y = D X, 2 expansion Y += E Z.  grid_cap > 0 limits the persistent grid.
hm_status f64_leaf_phase(int which, const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx,
                         void* Y, int64_t ldy, cudaStream_t st, bool pdl, int grid_cap);

void set_error(const char* fmt, ...);

}  // namespace hmi

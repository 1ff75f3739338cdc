// FP64 leaf products of the HODLR/HSS product for blocks of right-hand sides
// (Sec. 4.1, Fig. 4.1): the leaf projection V^T X, the diagonal-block
// product D_i X_i and the leaf expansion E_i Z_i (HSS: U_i y-hat_i; HODLR:
// the ancestors' U rows times their siblings' V^T X).
//
// On this GPU FP64 arithmetic runs at about 1/64 of the FP32 rate (one
// multiply-add per SM and cycle pair), so every FP64 product here is bound
// by the FP64 pipe, not by memory: a leaf row of D (2 KB) feeds 256 r
// multiply-adds.  The kernels are therefore shaped for the pipe:
//  * register-tiled SIMT GEMM: a thread owns a 2 x RN tile of outputs and
//    multiplies operands from shared memory, so every FP64 instruction issued
//    is a useful multiply-add (no cross-lane reduction adds);
//  * persistent blocks that take work units (leaf, 32 rows, TN columns) from
//    an atomic counter, so the last wave does not leave SMs idle;
//  * the diagonal-block product D_i X_i, three quarters of the work, is its
//    own launch right after the tree kernel, with programmatic dependent
//    launch: it needs nothing from the tree, so it may start as soon as the
//    tree's blocks are resident and room frees up.  It waits for the tree
//    (griddepcontrol.wait) only before it exits, so that its completion
//    implies the tree's; the expansion E_i Z_i, launched after it, then adds
//    to its result.
//
// Work unit u -> (leaf, column chunk, row tile), row tile fastest.  Every
// output is one FMA chain over K in increasing order, so results do not
// depend on which block took a unit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hm_api_internal.h"
#include "k_simt.cuh"

namespace hmi {

namespace {

constexpr int GT = 256;   // threads per block (16 x 16)
constexpr int GKC = 32;   // K per shared-memory chunk
constexpr int GTM = 32;   // rows per work unit (2 per thread)

enum { GW_PROJ = 0, GW_DPART = 1, GW_EPART = 2 };

template <int TN>
struct GSmem {
  double A[2][GKC][GTM + 1];   // A chunk, k-major (rows contiguous)
  double B[2][GKC][TN + 1];    // B chunk, k-major (columns contiguous)
  int unit;
};

// Operand sources of one work unit.
struct Unit {
  const double* A;   // row 0, k 0 of the unit's A block (row-major, lda)
  int64_t lda;
  int rows;          // valid rows (others read as zero)
  int kdim;          // valid K (others read as zero)
  int c0, ncols;     // column chunk
  int leaf;
};

template <int WHICH, int TN>
__device__ __forceinline__ void stage_regs(const MatView& mv, const Scratch& ws, int64_t r, const double* X,
                                           int64_t ldx, const Unit& un, int64_t xrow0, int k0, double (&ra)[4],
                                           double (&rb)[TN / 8]) {
  const int tid = threadIdx.x;
  // A: GTM x GKC values, 4 per thread; consecutive threads take consecutive k
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = tid + GT * u;
    const int row = idx / GKC, k = k0 + idx % GKC;
    ra[u] = (row < un.rows && k < un.kdim) ? __ldg(un.A + row * un.lda + k) : 0.0;
  }
  // B: GKC x TN values; consecutive threads take consecutive k of a column
#pragma unroll
  for (int u = 0; u < TN / 8; ++u) {
    const int idx = tid + GT * u;
    const int k = k0 + idx % GKC, c = idx / GKC;
    double v = 0.0;
    if (k < un.kdim && c < un.ncols) {
      const int64_t col = un.c0 + c;
      if constexpr (WHICH == GW_EPART) {
        if (mv.kind == HM_HSS) {
          const int node = mv.L - 1 + un.leaf;
          v = __ldcg(static_cast<const double*>(ws.yf) + (static_cast<int64_t>(node) * r + col) * mv.Ke + k);
        } else {
          v = z_value<double>(mv, ws, r, un.leaf, k, col);
        }
      } else {
        v = X[xrow0 + k + col * ldx];
      }
    }
    rb[u] = v;
  }
}

template <int TN>
__device__ __forceinline__ void stage_store(GSmem<TN>& sm, int buf, const double (&ra)[4],
                                            const double (&rb)[TN / 8]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = tid + GT * u;
    sm.A[buf][idx % GKC][idx / GKC] = ra[u];
  }
#pragma unroll
  for (int u = 0; u < TN / 8; ++u) {
    const int idx = tid + GT * u;
    sm.B[buf][idx % GKC][idx / GKC] = rb[u];
  }
}

template <int WHICH, int TN>
__global__ void __launch_bounds__(GT, 2) k_leaf_f64(MatView mv, Scratch ws, int64_t r, const double* X,
                                                    int64_t ldx, double* Y, int64_t ldy, int tiles, int chunks,
                                                    int units, int* ctr) {
  constexpr int RN = TN / 16;
  __shared__ __align__(16) GSmem<TN> sm;
  if constexpr (WHICH != GW_EPART) pdl_launch_dependents();
  if constexpr (WHICH == GW_EPART) pdl_wait();   // Y (D part) and Z come from the kernels before
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  for (;;) {
    if (tid == 0) sm.unit = atomicAdd(ctr, 1);
    __syncthreads();
    const int u = sm.unit;
    if (u >= units) break;
    const int tile = u % tiles;
    const int chunk = (u / tiles) % chunks;
    const int leaf = u / (tiles * chunks);
    const int64_t a0 = mv.off[leaf];
    const int m = static_cast<int>(mv.off[leaf + 1] - a0);
    const int row0 = tile * GTM;
    Unit un;
    un.leaf = leaf;
    un.c0 = chunk * TN;
    un.ncols = static_cast<int>(min(static_cast<int64_t>(TN), r - un.c0));
    if constexpr (WHICH == GW_PROJ) {
      un.A = static_cast<const double*>(mv.W) + (static_cast<int64_t>(leaf) * mv.Kp + row0) * mv.m_pad;
      un.lda = mv.m_pad;
      un.rows = mv.Kp - row0;
      un.kdim = m;
    } else if constexpr (WHICH == GW_DPART) {
      un.A = static_cast<const double*>(mv.A) + (a0 + row0) * mv.We;
      un.lda = mv.We;
      un.rows = m - row0;
      un.kdim = m;
    } else {
      un.A = static_cast<const double*>(mv.A) + (a0 + row0) * mv.We + mv.m_pad;
      un.lda = mv.We;
      un.rows = m - row0;
      un.kdim = (mv.kind == HM_HSS && mv.p == 0) ? 0 : mv.Ke;
    }
    if (un.rows > 0) {
      double acc[2][RN];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = 0.0;
      const int nk = (un.kdim + GKC - 1) / GKC;
      double ra[4], rb[TN / 8];
      if (nk > 0) {
        stage_regs<WHICH, TN>(mv, ws, r, X, ldx, un, a0, 0, ra, rb);
        stage_store<TN>(sm, 0, ra, rb);
      }
      __syncthreads();
      for (int kc = 0; kc < nk; ++kc) {
        const int buf = kc & 1;
        if (kc + 1 < nk) stage_regs<WHICH, TN>(mv, ws, r, X, ldx, un, a0, (kc + 1) * GKC, ra, rb);
#pragma unroll 8
        for (int k = 0; k < GKC; ++k) {
          const double x0 = sm.A[buf][k][ty], x1 = sm.A[buf][k][ty + 16];
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            const double b = sm.B[buf][k][tx + 16 * j];
            acc[0][j] = fma(x0, b, acc[0][j]);
            acc[1][j] = fma(x1, b, acc[1][j]);
          }
        }
        if (kc + 1 < nk) stage_store<TN>(sm, buf ^ 1, ra, rb);
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int row = ty + 16 * i;
        if (row >= un.rows) continue;
#pragma unroll
        for (int j = 0; j < RN; ++j) {
          const int c = tx + 16 * j;
          if (c >= un.ncols) continue;
          const int64_t col = un.c0 + c;
          if constexpr (WHICH == GW_PROJ) {
            const int node = mv.L - 1 + leaf;
            double* dst = static_cast<double*>(mv.kind == HM_HODLR ? ws.PS : ws.xh);
            const int ld = (mv.kind == HM_HODLR) ? mv.Ke : mv.Kp;
            dst[(static_cast<int64_t>(node) * r + col) * ld + row0 + row] = acc[i][j];
          } else if constexpr (WHICH == GW_DPART) {
            Y[a0 + row0 + row + col * ldy] = acc[i][j];
          } else {
            double* y = Y + a0 + row0 + row + col * ldy;
            *y = *y + acc[i][j];
          }
        }
      }
    }
    __syncthreads();   // every thread is done with sm.unit and the buffers
  }
  // the D part needs nothing from the tree kernel before it, but its
  // completion must imply the tree's: the expansion after it reads both
  if constexpr (WHICH == GW_DPART) pdl_wait();
  if (tid == 0) {
    // the last block to leave resets the counters for the next launch
    __threadfence();
    if (atomicAdd(ctr + 1, 1) == static_cast<int>(gridDim.x) - 1) {
      atomicExch(ctr, 0);
      atomicExch(ctr + 1, 0);
    }
  }
}

template <int WHICH, int TN>
hm_status launch_leaf_f64(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx, void* Y,
                          int64_t ldy, cudaStream_t st, bool pdl, int* ctr, int grid_cap) {
  const int tiles = (WHICH == GW_PROJ) ? (mv.Kp + GTM - 1) / GTM : (mv.m_pad + GTM - 1) / GTM;
  const int chunks = static_cast<int>((r + TN - 1) / TN);
  const int64_t units64 = static_cast<int64_t>(mv.L) * tiles * chunks;
  if (units64 > (int64_t(1) << 30)) return HM_EUNSUPPORTED;
  const int units = static_cast<int>(units64);
  int dev = 0, sms = 152, per = 2;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_leaf_f64<WHICH, TN>, GT, 0);
  per = std::max(1, std::min(per, 2));
  int grid = std::min(units, sms * per);
  if (grid_cap > 0) grid = std::min(grid, grid_cap);
  grid = std::max(grid, 1);
  Scratch wk = ws;
  wk.prof = nullptr;
  const cudaError_t e = launch_k(k_leaf_f64<WHICH, TN>, dim3(grid), dim3(GT), 0, st, pdl, mv, wk, r,
                                 static_cast<const double*>(X), ldx, static_cast<double*>(Y), ldy, tiles, chunks,
                                 units, ctr);
  if (e != cudaSuccess) {
    set_error("FP64 leaf launch (%d) failed: %s", WHICH, cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

template <int WHICH>
hm_status launch_leaf_f64_tn(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx, void* Y,
                             int64_t ldy, cudaStream_t st, bool pdl, int* ctr, int grid_cap) {
  if (r <= 16) return launch_leaf_f64<WHICH, 16>(mv, ws, r, X, ldx, Y, ldy, st, pdl, ctr, grid_cap);
  return launch_leaf_f64<WHICH, 32>(mv, ws, r, X, ldx, Y, ldy, st, pdl, ctr, grid_cap);
}

}  // namespace

bool f64_tiled(const MatView& mv, int64_t r) { return mv.storage == HM_F64 && r >= kF64TiledMinR; }

hm_status f64_leaf_phase(int which, const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx,
                         void* Y, int64_t ldy, cudaStream_t st, bool pdl, int grid_cap) {
  int* ctr = f64_counters(ws, mv, r) + 2 * which;
  switch (which) {
    case GW_PROJ: return launch_leaf_f64_tn<GW_PROJ>(mv, ws, r, X, ldx, Y, ldy, st, pdl, ctr, grid_cap);
    case GW_DPART: return launch_leaf_f64_tn<GW_DPART>(mv, ws, r, X, ldx, Y, ldy, st, pdl, ctr, grid_cap);
    default: return launch_leaf_f64_tn<GW_EPART>(mv, ws, r, X, ldx, Y, ldy, st, pdl, ctr, grid_cap);
  }
}

}  // namespace hmi

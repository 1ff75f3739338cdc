// Batched products: many matrices of uneven size, rank, storage and number of
// right-hand sides run through one persistent launch per phase (projection,
// tree upsweep, HSS downsweep, SIMT expansion, tensor-core expansion).
//
// Each product keeps exactly the blocking it would have on its own (column
// chunks, tree step spans, tiles), so a product's result is bit-identical in
// a batch and alone; the batch only changes which block runs it and when.
#pragma once

#include <cstdint>

#include <cuda.h>

#include "hm_internal.h"

namespace hmi {

// One product of the batch, as the kernels see it (device memory).
// Tensor-core fields: expansion (nt .. tc_tiles) and projection (ntp ..
// tcp_tiles, w_box rows per TMA box of the projection planes).
struct BatchJob {
  MatView mv;
  Scratch ws;
  int64_t r;
  int storage;
  int rc_p, rc_e;      // SIMT column chunks: projection, expansion
  int rct;             // tree column chunk
  int g, s0;           // tree upsweep: step span, first-step span
  int s_lvl, G;        // downsweep: subtree level, chain prefetch depth
  int RT, tiles;       // SIMT expansion: rows per tile, tiles per leaf
  int tc;              // 1: tensor-core expansion
  int nt, split, nK, nX, nst, tc_tiles;
  int tcp;             // 1: tensor-core projection
  int ntp, nKp, nXp, nstp, tcp_tiles, w_box;
};

// Per-run inputs and outputs of one product.
struct BatchIO {
  const void* X;
  void* Y;
  int64_t ldx, ldy;
  int xt, yt;
};

// One unit of work: product `job`, block coordinates (bx, by) of that
// product's own launch of the phase.
struct BItem {
  int job, bx, by;
};

// Phases in launch order.  Tensor maps: four per product (expansion hi/lo,
// projection hi/lo).
enum {
  BP_PROJECT = 0,
  BP_PROJECT_TC = 1,
  BP_UP = 2,
  BP_DOWN = 3,
  BP_EXPAND = 4,
  BP_EXPAND_TC = 5,
  BP_COUNT = 6
};
constexpr int BATCH_MAPS = 4;

inline bool batch_phase_tc(int p) { return p == BP_PROJECT_TC || p == BP_EXPAND_TC; }

// Shared-memory attributes are set when a plan is built, so launches can be
// recorded into a CUDA graph.
void batch_set_smem(int phase, size_t smem);
void batch_set_smem_tc(int phase, size_t smem);
cudaError_t batch_launch_simt(int phase, const BatchJob* jobs, const BatchIO* io, const BItem* items, int n,
                              int grid, size_t smem, cudaStream_t st, bool pdl);
cudaError_t batch_launch_tc(int phase, const BatchJob* jobs, const BatchIO* io, const CUtensorMap* maps,
                            const BItem* items, int n, int grid, size_t smem, int ncol, cudaStream_t st, bool pdl);

}  // namespace hmi

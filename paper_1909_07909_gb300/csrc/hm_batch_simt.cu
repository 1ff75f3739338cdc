// Persistent batched SIMT kernels: every block walks the phase's work list
// (stride gridDim.x) and runs each item with the same block function, column
// chunk and tile the product would use on its own.  Storage types F32, BF16
// and BF16X2 (float compute).
#include "hm_batch.h"
#include "k_simt.cuh"

namespace hmi {

template <int S>
__device__ void proj_item(const BatchJob& J, const BatchIO& o, int bx, int by, unsigned char* sm) {
  using C = typename Stor<S>::C;
#define HM_P(RC_, TR_)                                                                                      \
  project_block<S, RC_, TR_>(J.mv, J.ws, J.r, o.X, o.ldx, o.xt, bx, by, reinterpret_cast<C*>(sm)); \
  break
  switch (J.rc_p) {
    case 1: HM_P(1, 2);
    case 2: HM_P(2, 2);
    case 4: HM_P(4, 2);
    case 8: HM_P(8, 2);
    case 16: HM_P(16, 1);
    default: HM_P(32, 1);
  }
#undef HM_P
}

template <int S>
__device__ void expand_item(const BatchJob& J, const BatchIO& o, int bx, int by, unsigned char* sm) {
  using C = typename Stor<S>::C;
  const int leaf = bx / J.tiles, tile = bx % J.tiles;
#define HM_E(RC_, TR_)                                                                                        \
  expand_block<S, RC_, TR_>(J.mv, J.ws, J.r, o.X, o.ldx, o.xt, o.Y, o.ldy, o.yt, J.RT, leaf, tile, by, \
                            reinterpret_cast<C*>(sm));                                                       \
  break
  constexpr int TRN = 4;   // as the single product's expansion
  switch (J.rc_e) {
    case 1: HM_E(1, TRN);
    case 2: HM_E(2, TRN);
    case 4: HM_E(4, 4);
    case 8: HM_E(8, 4);
    case 16: HM_E(16, 4);
    default: HM_E(32, 2);
  }
#undef HM_E
}

__device__ void up_item(const BatchJob& J, int bx, int by, unsigned char* sm) {
  float* f = reinterpret_cast<float*>(sm);
  const int nch = static_cast<int>((J.r + J.rct - 1) / J.rct);
  switch (J.rct) {
    case 1: tree_up_block<float, 1>(J.mv, J.ws, J.r, J.g, nch, bx, by, f); break;
    case 2: tree_up_block<float, 2>(J.mv, J.ws, J.r, J.g, nch, bx, by, f); break;
    case 4: tree_up_block<float, 4>(J.mv, J.ws, J.r, J.g, nch, bx, by, f); break;
    case 8: tree_up_block<float, 8>(J.mv, J.ws, J.r, J.g, nch, bx, by, f); break;
    default: tree_up_block<float, 16>(J.mv, J.ws, J.r, J.g, nch, bx, by, f); break;
  }
}

__device__ void down_item(const BatchJob& J, int bx, int by, unsigned char* sm) {
  switch (J.rct) {
    case 1: down_block<float, 1>(J.mv, J.ws, J.r, J.s_lvl, J.G, bx, by, sm); break;
    case 2: down_block<float, 2>(J.mv, J.ws, J.r, J.s_lvl, J.G, bx, by, sm); break;
    case 4: down_block<float, 4>(J.mv, J.ws, J.r, J.s_lvl, J.G, bx, by, sm); break;
    case 8: down_block<float, 8>(J.mv, J.ws, J.r, J.s_lvl, J.G, bx, by, sm); break;
    default: down_block<float, 16>(J.mv, J.ws, J.r, J.s_lvl, J.G, bx, by, sm); break;
  }
}

template <int PHASE>
__global__ void __launch_bounds__(256) k_batch_simt(const BatchJob* jobs, const BatchIO* io, const BItem* items,
                                                    int n) {
  pdl_launch_dependents();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const BItem w = items[it];
    const BatchJob& J = jobs[w.job];
    const BatchIO& o = io[w.job];
    if constexpr (PHASE == BP_PROJECT) {
      switch (J.storage) {
        case HM_F32: proj_item<HM_F32>(J, o, w.bx, w.by, smem_raw); break;
        case HM_BF16: proj_item<HM_BF16>(J, o, w.bx, w.by, smem_raw); break;
        default: proj_item<HM_BF16X2>(J, o, w.bx, w.by, smem_raw); break;
      }
    } else if constexpr (PHASE == BP_UP) {
      up_item(J, w.bx, w.by, smem_raw);
    } else if constexpr (PHASE == BP_DOWN) {
      down_item(J, w.bx, w.by, smem_raw);
    } else {
      switch (J.storage) {
        case HM_F32: expand_item<HM_F32>(J, o, w.bx, w.by, smem_raw); break;
        case HM_BF16: expand_item<HM_BF16>(J, o, w.bx, w.by, smem_raw); break;
        default: expand_item<HM_BF16X2>(J, o, w.bx, w.by, smem_raw); break;
      }
    }
    __syncthreads();
  }
}

void batch_set_smem(int phase, size_t smem) {
  const int v = static_cast<int>(smem);
  switch (phase) {
    case BP_PROJECT: cudaFuncSetAttribute(k_batch_simt<BP_PROJECT>, cudaFuncAttributeMaxDynamicSharedMemorySize, v); break;
    case BP_UP: cudaFuncSetAttribute(k_batch_simt<BP_UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, v); break;
    case BP_DOWN: cudaFuncSetAttribute(k_batch_simt<BP_DOWN>, cudaFuncAttributeMaxDynamicSharedMemorySize, v); break;
    default: cudaFuncSetAttribute(k_batch_simt<BP_EXPAND>, cudaFuncAttributeMaxDynamicSharedMemorySize, v); break;
  }
}

// Launch only (no attribute calls, so it can be recorded into a CUDA graph).
cudaError_t batch_launch_simt(int phase, const BatchJob* jobs, const BatchIO* io, const BItem* items, int n,
                              int grid, size_t smem, cudaStream_t st, bool pdl) {
  switch (phase) {
    case BP_PROJECT:
      return launch_k(k_batch_simt<BP_PROJECT>, dim3(grid), dim3(256), smem, st, pdl, jobs, io, items, n);
    case BP_UP:
      return launch_k(k_batch_simt<BP_UP>, dim3(grid), dim3(256), smem, st, pdl, jobs, io, items, n);
    case BP_DOWN:
      return launch_k(k_batch_simt<BP_DOWN>, dim3(grid), dim3(256), smem, st, pdl, jobs, io, items, n);
    default:
      return launch_k(k_batch_simt<BP_EXPAND>, dim3(grid), dim3(256), smem, st, pdl, jobs, io, items, n);
  }
}

}  // namespace hmi

// Persistent batched tensor-core expansion: a block allocates its tensor
// memory once, then runs tc_tile for every work item of the list (stride
// gridDim.x), each with its product's own TMA descriptors (global memory).
#include "hm_batch.h"
#include "k_tc.cuh"

namespace hmi {

__global__ void __launch_bounds__(128, 1)
    k_batch_expand_tc(const BatchJob* jobs, const BatchIO* io, const CUtensorMap* maps, const BItem* items, int n,
                      int ncol) {
  pdl_launch_dependents();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(base);
  uint8_t* tile_base = base + 1024;
  if (static_cast<int>(blockIdx.x) >= n) return;
  if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(tslot), static_cast<uint32_t>(ncol));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const BItem w = items[it];
    const BatchJob& J = jobs[w.job];
    const BatchIO& o = io[w.job];
    const CUtensorMap* ma = maps + 2 * w.job;
    const CUtensorMap* ml = maps + 2 * w.job + 1;
    const int leaf = w.bx / J.tc_tiles, rt = w.bx % J.tc_tiles;
    const int col0 = w.by * J.nt;
#define HM_T(SP, N)                                                                                               \
  tc_tile<SP, N>(ma, ml, J.mv, J.ws, J.r, o.X, o.ldx, o.xt, o.Y, o.ldy, o.yt, leaf, rt, col0, J.nK, J.nX, J.nst, \
                 tile_base, tmem);                                                                                \
  break
    if (J.split) {
      switch (J.nt) {
        case 16: HM_T(true, 16);
        case 32: HM_T(true, 32);
        case 64: HM_T(true, 64);
        default: HM_T(true, 128);
      }
    } else {
      switch (J.nt) {
        case 16: HM_T(false, 16);
        case 32: HM_T(false, 32);
        case 64: HM_T(false, 64);
        default: HM_T(false, 128);
      }
    }
#undef HM_T
    __syncthreads();
  }
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, static_cast<uint32_t>(ncol));
  }
}

void batch_set_smem_tc(size_t smem) {
  cudaFuncSetAttribute(k_batch_expand_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

cudaError_t batch_launch_tc(const BatchJob* jobs, const BatchIO* io, const CUtensorMap* maps, const BItem* items,
                            int n, int grid, size_t smem, int ncol, cudaStream_t st, bool pdl) {
  return launch_k(k_batch_expand_tc, dim3(grid), dim3(128), smem, st, pdl, jobs, io, maps, items, n, ncol);
}

}  // namespace hmi

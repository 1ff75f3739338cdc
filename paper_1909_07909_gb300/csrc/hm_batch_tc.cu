// Persistent batched tensor-core leaf contractions (projection and
// expansion): a block allocates its tensor memory once, then runs tc_tile for
// every work item of the list (stride gridDim.x), each with its product's own
// TMA descriptors (global memory).  X is always staged by the threads here
// (its descriptor would change with every run); the staged operand equals the
// one TMA writes, so results match the single-product path bit for bit.
#include "hm_batch.h"
#include "k_tc.cuh"

namespace hmi {

template <bool PROJ>
__global__ void __launch_bounds__(128, 1)
    k_batch_leaf_tc(const BatchJob* jobs, const BatchIO* io, const CUtensorMap* maps, const BItem* items, int n,
                    int ncol) {
  pdl_launch_dependents();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(base);
  uint8_t* tile_base = base + 1024;
  if (static_cast<int>(blockIdx.x) < n) {
    if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(tslot), static_cast<uint32_t>(ncol));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
      const BItem w = items[it];
      const BatchJob& J = jobs[w.job];
      const BatchIO& o = io[w.job];
      const CUtensorMap* ma = maps + BATCH_MAPS * w.job + (PROJ ? 2 : 0);
      const CUtensorMap* ml = ma + 1;
      const int tiles = PROJ ? J.tcp_tiles : J.tc_tiles;
      const int leaf = w.bx / tiles, rt = w.bx % tiles;
      const int nt = PROJ ? J.ntp : J.nt;
      const int col0 = w.by * nt;
      const int box = PROJ ? J.w_box : TC_M;
      const int nK = PROJ ? J.nKp : J.nK;
      const int nX = PROJ ? J.nXp : J.nX;
      const int nst = PROJ ? J.nstp : J.nst;
#define HM_T(SP, N)                                                                                             \
  tc_tile<SP, N, PROJ>(ma, ml, nullptr, box, J.mv, J.ws, J.r, o.X, o.ldx, o.xt, o.Y, o.ldy, o.yt, leaf, rt, col0, \
                       nK, nX, nst, tile_base, tmem, 1);                                                            \
  break
      if (J.split) {
        switch (nt) {
          case 16: HM_T(true, 16);
          case 32: HM_T(true, 32);
          case 64: HM_T(true, 64);
          case 128: HM_T(true, 128);
          default: HM_T(true, 256);
        }
      } else {
        switch (nt) {
          case 16: HM_T(false, 16);
          case 32: HM_T(false, 32);
          case 64: HM_T(false, 64);
          case 128: HM_T(false, 128);
          default: HM_T(false, 256);
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
  // The projection never waits on its predecessor; waiting here keeps this
  // grid from completing before it, so the next phase's wait covers both.
  if constexpr (PROJ) pdl_wait();
}

void batch_set_smem_tc(int phase, size_t smem) {
  if (phase == BP_PROJECT_TC)
    cudaFuncSetAttribute(k_batch_leaf_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  else
    cudaFuncSetAttribute(k_batch_leaf_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

cudaError_t batch_launch_tc(int phase, const BatchJob* jobs, const BatchIO* io, const CUtensorMap* maps,
                            const BItem* items, int n, int grid, size_t smem, int ncol, cudaStream_t st, bool pdl) {
  if (phase == BP_PROJECT_TC)
    return launch_k(k_batch_leaf_tc<true>, dim3(grid), dim3(128), smem, st, pdl, jobs, io, maps, items, n, ncol);
  return launch_k(k_batch_leaf_tc<false>, dim3(grid), dim3(128), smem, st, pdl, jobs, io, maps, items, n, ncol);
}

}  // namespace hmi

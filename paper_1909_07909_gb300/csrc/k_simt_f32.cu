// SIMT kernels instantiated for HM_F32 storage (see k_simt.cuh, k_ring.cuh).
#include "k_ring.cuh"

namespace hmi {

hm_status simt_phase_f32(int phase, const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx,
                      int xt, void* Y, int64_t ldy, int yt, cudaStream_t s, bool pdl) {
  return simt_phase_t<HM_F32>(phase, mv, ws, r, X, ldx, xt, Y, ldy, yt, s, pdl);
}

}  // namespace hmi

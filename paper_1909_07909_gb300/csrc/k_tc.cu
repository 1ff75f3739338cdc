// Host side of the tensor-core leaf expansion: TMA descriptors of the
// generator planes, launch configuration (see k_tc.cuh for the kernel).
#include <mutex>

#include "k_tc.cuh"

namespace hmi {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

static bool plane_map(CUtensorMap* map, const void* plane, int64_t n, int We) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !plane) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(We), static_cast<cuuint64_t>(n)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(We) * 2};
  const cuuint32_t box[2] = {TC_KC, TC_M};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(plane), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void make_tensor_maps(hm_matrix* A) {
  A->tm_ok = false;
  if (A->storage != HM_BF16 && A->storage != HM_BF16X2) return;
  if (A->n < TC_M || A->We < TC_KC) return;
  bool ok = plane_map(&A->tmA, A->d_A, A->n, A->We);
  if (ok && A->storage == HM_BF16X2) ok = plane_map(&A->tmAlo, A->d_A_lo, A->n, A->We);
  else A->tmAlo = A->tmA;
  A->tm_ok = ok;
}

bool use_tensor_cores(const hm_matrix* A, int64_t r) {
  if (!A->tm_ok || A->path == 1) return false;
  if (A->storage != HM_BF16 && A->storage != HM_BF16X2) return false;
  return A->path == 2 || r >= 16;
}

static size_t tc_smem(bool split, int NT, int nK, int nst) { return 1024 + tc_layout_bytes(split, NT, nK, nst); }

// Deepest ring (4..2 stages) whose shared memory fits; 0 if none does.
static int tc_stages(bool split, int NT, int nK) {
  for (int s = TC_MAX_STAGES; s >= 2; --s)
    if (tc_smem(split, NT, nK, s) <= 227 * 1024) return s;
  return 0;
}

template <bool SPLIT, int NT>
static hm_status launch_tc_nt(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                              int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  const int nK = (mv.We + TC_KC - 1) / TC_KC;
  const int nX = mv.m_pad / TC_KC;
  const int nst = tc_stages(SPLIT, NT, nK);
  if (nst == 0) return HM_EUNSUPPORTED;
  const size_t smem = tc_smem(SPLIT, NT, nK, nst);
  const int tiles = (mv.m_pad + TC_M - 1) / TC_M;
  const int nchunks = static_cast<int>((r + NT - 1) / NT);
  cudaFuncSetAttribute(k_expand_tc<SPLIT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  Scratch wk = ws;
  wk.prof = nullptr;
  prof_mark(ws.prof, 3, true, st);
  const cudaError_t e = launch_k(k_expand_tc<SPLIT, NT>, dim3(mv.L * tiles, nchunks), dim3(128), smem, st, pdl,
                                 A->tmA, A->tmAlo, mv, wk, r, X, ldx, xt, Y, ldy, yt, tiles, nK, nX, nst);
  prof_mark(ws.prof, 3, false, st);
  if (e != cudaSuccess) {
    set_error("tensor-core expansion launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

bool tc_plan(const hm_matrix* A, int64_t r, int* nt, int* nK, int* nX, int* nst, int* tiles) {
  const bool split = (A->storage == HM_BF16X2);
  const int64_t rr = std::min<int64_t>(r, 256);
  int NT = 16;
  while (NT < rr) NT *= 2;
  const int k = (A->We + TC_KC - 1) / TC_KC;
  while (NT > 16 && tc_stages(split, NT, k) == 0) NT /= 2;
  const int s = tc_stages(split, NT, k);
  if (s == 0) return false;
  *nt = NT;
  *nK = k;
  *nX = A->m_pad / TC_KC;
  *nst = s;
  *tiles = (A->m_pad + TC_M - 1) / TC_M;
  return true;
}

size_t tc_tile_smem(bool split, int NT, int nK, int nst) { return tc_layout_bytes(split, NT, nK, nst); }

int tc_tile_ncols(bool split, int NT) {
  if (split) return (2 * NT <= 32) ? 32 : 2 * NT;
  return NT < 32 ? 32 : NT;
}

hm_status launch_expand_tc(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                           int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  const bool split = (A->storage == HM_BF16X2);
  int NT = 16, nK0 = 0, nX0 = 0, nst0 = 0, tiles0 = 0;
  if (!tc_plan(A, r, &NT, &nK0, &nX0, &nst0, &tiles0)) return HM_EUNSUPPORTED;
#define HM_TC(SP, N) return launch_tc_nt<SP, N>(A, mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl)
  if (split) {
    switch (NT) {
      case 16: HM_TC(true, 16);
      case 32: HM_TC(true, 32);
      case 64: HM_TC(true, 64);
      case 128: HM_TC(true, 128);
      default: HM_TC(true, 256);
    }
  }
  switch (NT) {
    case 16: HM_TC(false, 16);
    case 32: HM_TC(false, 32);
    case 64: HM_TC(false, 64);
    case 128: HM_TC(false, 128);
    default: HM_TC(false, 256);
  }
#undef HM_TC
}

}  // namespace hmi

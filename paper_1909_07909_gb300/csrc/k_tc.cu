// Host side of the tensor-core leaf expansion: TMA descriptors of the
// generator planes, launch configuration (see k_tc.cuh for the kernel).
#include <cstring>
#include <mutex>

#include "k_tc.cuh"
#include "k_tc_persist.cuh"

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

// 2-D bf16 tensor map with 128-byte swizzle: `inner` contiguous elements per
// row, `outer` rows `row_bytes` apart, boxes of box_inner x box_outer.
static bool encode_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                      uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void make_tensor_maps(hm_matrix* A) {
  A->tm_ok = false;
  A->tmw_ok = false;
  if (A->storage != HM_BF16 && A->storage != HM_BF16X2) return;
  if (A->n < TC_M || A->We < TC_KC || A->m_pad < TC_KC) return;
  const bool split = (A->storage == HM_BF16X2);
  bool ok = encode_2d(&A->tmA, A->d_A, A->We, A->n, static_cast<uint64_t>(A->We) * 2, TC_KC, TC_M);
  if (ok && split) ok = encode_2d(&A->tmAlo, A->d_A_lo, A->We, A->n, static_cast<uint64_t>(A->We) * 2, TC_KC, TC_M);
  else A->tmAlo = A->tmA;
  A->tm_ok = ok;
  if (A->Kp >= 8) {
    A->w_box = std::min(A->Kp, TC_M);
    const uint64_t rows = static_cast<uint64_t>(A->L) * A->Kp;
    bool w = encode_2d(&A->tmW, A->d_W, A->m_pad, rows, static_cast<uint64_t>(A->m_pad) * 2, TC_KC, A->w_box);
    if (w && split) w = encode_2d(&A->tmWlo, A->d_W_lo, A->m_pad, rows, static_cast<uint64_t>(A->m_pad) * 2, TC_KC,
                                  A->w_box);
    else A->tmWlo = A->tmW;
    A->tmw_ok = w && ok;
  }
}

bool use_tensor_cores(const hm_matrix* A, int64_t r) {
  if (!A->tm_ok || A->path == 1) return false;
  if (A->storage != HM_BF16 && A->storage != HM_BF16X2) return false;
  return A->path == 2 || r >= 16;
}

static size_t tc_smem(bool split, int NT, int nK, int nst, int mt = 1) {
  return 1024 + tc_layout_bytes(split, NT, nK, nst, mt);
}

// Tiles per CTA of a single product's expansion: two 128-row tiles of a leaf
// share one CTA (one B operand, X read once per leaf, half the CTAs) when the
// leaf has two, the accumulators fit in tensor memory and a 2-stage ring
// fits; the ring is then as deep as two CTAs per SM allow when the grid
// exceeds one CTA per SM, else as deep as fits.
static void tc_pick_mt(bool split, int NT, int nK, int tiles128, int64_t ctas_mt2, int sms, int* mt, int* nst) {
  *mt = 1;
  if (tiles128 < 2 || 2 * tc_ncols_host(split, NT) > 512) return;
  const size_t two_per_sm = 113 * 1024;
  int best = 0;
  for (int s = TC_MAX_STAGES; s >= 2; --s) {
    const size_t b = tc_smem(split, NT, nK, s, 2);
    if (b > 227 * 1024) continue;
    if (best == 0) best = s;                       // deepest that fits at all
    if (ctas_mt2 > sms && b <= two_per_sm) {       // deepest that lets two CTAs share an SM
      best = s;
      break;
    }
  }
  if (best == 0) return;
  *mt = 2;
  *nst = best;
}

// Deepest ring (4..2 stages) whose shared memory fits; 0 if none does.
static int tc_stages(bool split, int NT, int nK) {
  for (int s = TC_MAX_STAGES; s >= 2; --s)
    if (tc_smem(split, NT, nK, s) <= 227 * 1024) return s;
  return 0;
}

bool tc_plan(const hm_matrix* A, int64_t r, bool proj, int* nt, int* nK, int* nX, int* nst, int* tiles) {
  if (proj && !A->tmw_ok) return false;
  const bool split = (A->storage == HM_BF16X2);
  const int64_t rr = std::min<int64_t>(r, 256);
  int NT = 16;
  while (NT < rr) NT *= 2;
  const int k = ((proj ? A->m_pad : A->We) + TC_KC - 1) / TC_KC;
  while (NT > 16 && tc_stages(split, NT, k) == 0) NT /= 2;
  const int s = tc_stages(split, NT, k);
  if (s == 0) return false;
  *nt = NT;
  *nK = k;
  *nX = proj ? k : A->m_pad / TC_KC;
  *nst = s;
  *tiles = proj ? (A->Kp + TC_M - 1) / TC_M : (A->m_pad + TC_M - 1) / TC_M;
  return true;
}

size_t tc_tile_smem(bool split, int NT, int nK, int nst) { return tc_layout_bytes(split, NT, nK, nst); }

int tc_tile_ncols(bool split, int NT) { return tc_ncols_host(split, NT); }

// Tensor map of a bf16 X block (rows inner, columns outer) with NT-column boxes,
// when X qualifies for TMA (16-byte aligned, ldx a multiple of 8 elements).
// Box height of the Z block's tensor boxes: the largest power of two up to
// 256 (at least 4) such that every box lies in one node's rows (HSS: all Ke
// rows; HODLR: each level's block starts and ends on a multiple of it, the
// blocks tiling the Ke rows); 0 when there is none (cp.async fetch).
static int z_box_rows(const MatView& mv) {
  if (mv.p < 1 || mv.Ke % 4 != 0) return 0;
  if (mv.kind != HM_HSS) {
    int next = 0;
    for (int l = 1; l <= mv.p; ++l) {
      if (mv.koff[l] != next) return 0;
      next += mv.kk[l];
    }
    if (next != mv.Ke) return 0;
  }
  for (int hb = 256; hb >= 4; hb /= 2) {
    bool ok = mv.Ke % hb == 0;
    if (mv.kind != HM_HSS)
      for (int l = 1; ok && l <= mv.p; ++l) ok = (mv.koff[l] % hb == 0) && (mv.kk[l] % hb == 0);
    if (ok) return hb;
  }
  return 0;
}

// FP32 view of the tree scratch for the Z block: rows of Ke floats, row
// node * r + col, boxes of hb rows by NT columns, no swizzle.
static bool z_map(CUtensorMap* map, const void* base, int Ke, int64_t rows, int NT, int hb) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base || Ke % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(Ke), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(Ke) * 4};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(hb), static_cast<cuuint32_t>(NT)};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool x_map(CUtensorMap* map, const void* X, int64_t n, int64_t r, int64_t ldx, int NT) {
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0 || (ldx & 7) != 0 || n < TC_KC) return false;
  return encode_2d(map, X, static_cast<uint64_t>(n), static_cast<uint64_t>(r), static_cast<uint64_t>(ldx) * 2, TC_KC,
                   static_cast<uint32_t>(NT));
}

template <bool SPLIT, int NT, bool PROJ>
static hm_status launch_leaf_nt(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                                int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  int nt = 0, nK = 0, nX = 0, nst = 0, tiles = 0;
  if (!tc_plan(A, r, PROJ, &nt, &nK, &nX, &nst, &tiles)) return HM_EUNSUPPORTED;
  const int nchunks = static_cast<int>((r + NT - 1) / NT);
  int mt = 1;
  if (!PROJ) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int nst2 = nst;
    tc_pick_mt(SPLIT, NT, nK, tiles, static_cast<int64_t>(mv.L) * ((tiles + 1) / 2) * nchunks, sms, &mt, &nst2);
    if (mt == 2) {
      nst = nst2;
      tiles = (tiles + 1) / 2;
    }
  }
  const size_t smem = tc_smem(SPLIT, NT, nK, nst, mt);
  CUtensorMap tmX;
  std::memset(&tmX, 0, sizeof(tmX));
  const int use_tmx = (xt == HM_BF16 && x_map(&tmX, X, mv.n, r, ldx, NT)) ? 1 : 0;
  cudaFuncSetAttribute(k_leaf_tc<SPLIT, NT, PROJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem));
  Scratch wk = ws;
  wk.prof = nullptr;
  const int phase = PROJ ? 0 : 3;
  prof_mark(ws.prof, phase, true, st);
  const cudaError_t e =
      launch_k(k_leaf_tc<SPLIT, NT, PROJ>, dim3(mv.L * tiles, nchunks), dim3(128), smem, st, pdl,
               PROJ ? A->tmW : A->tmA, PROJ ? A->tmWlo : A->tmAlo, tmX, use_tmx, PROJ ? A->w_box : TC_M, mv, wk, r, X,
               ldx, xt, Y, ldy, yt, tiles, nK, nX, nst, mt);
  prof_mark(ws.prof, phase, false, st);
  if (e != cudaSuccess) {
    set_error("tensor-core leaf launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

template <bool PROJ>
static hm_status launch_leaf(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                             int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  const bool split = (A->storage == HM_BF16X2);
  int NT = 16, nK0 = 0, nX0 = 0, nst0 = 0, tiles0 = 0;
  if (!tc_plan(A, r, PROJ, &NT, &nK0, &nX0, &nst0, &tiles0)) return HM_EUNSUPPORTED;
#define HM_TC(SP, N) return launch_leaf_nt<SP, N, PROJ>(A, mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl)
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

// The persistent leaf kernels (k_tc_persist.cuh) for BF16 storage, used when
// the one-item-per-CTA kernel would take more than one wave of CTAs (with
// one wave every item's loads, multiplies and stores already overlap across
// CTAs, and the expansion finishes sooner after the tree kernels): as many
// stages as fit beside the Z block and the control block, one CTA per SM.
template <int NT, bool PROJ>
static hm_status launch_tcp_nt(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                               int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl, int nK,
                               int nX, int nst_old, int tiles) {
  constexpr int TPT = (NT < 32) ? 32 : NT;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nchunks = (r + NT - 1) / NT;
  {
    // waves of the one-item-per-CTA kernel, with its own tile pairing
    int mt_o = 1, nst_o = nst_old;
    if (!PROJ) {
      const int64_t ctas2 = static_cast<int64_t>(mv.L) * ((tiles + 1) / 2) * nchunks;
      tc_pick_mt(false, NT, nK, tiles, ctas2, sms, &mt_o, &nst_o);
    }
    const int64_t ctas = static_cast<int64_t>(mv.L) * ((tiles + mt_o - 1) / mt_o) * nchunks;
    const size_t sm_o = tc_smem(false, NT, nK, nst_o, mt_o);
    const int per = sm_o <= 113 * 1024 ? 2 : 1;
    if (ctas <= static_cast<int64_t>(per) * sms) return HM_EUNSUPPORTED;
  }
  const int ke = PROJ ? 0 : mv.Ke;
  const int mt = (tiles >= 2 && 2 * TPT <= 256) ? 2 : 1;
  if (2 * mt * TPT > 512) return HM_EUNSUPPORTED;
  // rings of at least 3 stages only (a 2-stage ring is not used; the
  // one-item-per-CTA kernel takes those shapes)
  int nst = TCP_MAX_STAGES;
  while (nst > 3 && tcp_smem_bytes(NT, mt, nst, ke) > 227 * 1024) --nst;
  if (tcp_smem_bytes(NT, mt, nst, ke) > 227 * 1024) return HM_EUNSUPPORTED;
  // all of an SM's shared memory, whatever the ring needs: the CTA has its SM
  // to itself (no CTA of the neighbouring kernels, which programmatic launch
  // lets run at the same time, beside it)
  const size_t smem = 227 * 1024;
  const int tgroups = (tiles + mt - 1) / mt;
  const int64_t nitems64 = static_cast<int64_t>(mv.L) * tgroups * nchunks;
  if (nitems64 <= 0 || nitems64 > (int64_t(1) << 30)) return HM_EUNSUPPORTED;
  const int grid = static_cast<int>(std::min<int64_t>(nitems64, sms));
  CUtensorMap tmX;
  std::memset(&tmX, 0, sizeof(tmX));
  const int use_tmx = (xt == HM_BF16 && x_map(&tmX, X, mv.n, r, ldx, NT)) ? 1 : 0;
  CUtensorMap tmZ;
  std::memset(&tmZ, 0, sizeof(tmZ));
  int zhb = 0;
  if (!PROJ) {
    const void* zbase = (mv.kind == HM_HSS) ? ws.yf : ws.PS;
    zhb = z_box_rows(mv);
    if (zhb > 0 && !z_map(&tmZ, zbase, mv.Ke, (2 * static_cast<int64_t>(mv.L) - 1) * r, NT, zhb)) zhb = 0;
  }
  if (cudaFuncSetAttribute(k_expand_tcp<NT, PROJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess) {
    cudaGetLastError();
    return HM_EUNSUPPORTED;
  }
  Scratch wk = ws;
  wk.prof = nullptr;
  const int phase = PROJ ? 0 : 3;
  prof_mark(ws.prof, phase, true, st);
  const cudaError_t e =
      launch_k(k_expand_tcp<NT, PROJ>, dim3(grid), dim3(TCP_THREADS), smem, st, pdl, PROJ ? A->tmW : A->tmA, tmX,
               use_tmx, tmZ, zhb, mv, wk, r, X, ldx, xt, Y, ldy, yt, tgroups, static_cast<int>(nchunks),
               static_cast<int>(nitems64), nK, nX, nst, mt, PROJ ? A->w_box : TC_M);
  prof_mark(ws.prof, phase, false, st);
  if (e != cudaSuccess) {
    set_error("persistent tensor-core leaf launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

template <bool PROJ>
static hm_status launch_tcp(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                            int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  if (A->storage != HM_BF16) return HM_EUNSUPPORTED;
  int NT = 16, nK = 0, nX = 0, nst = 0, tiles = 0;
  if (!tc_plan(A, r, PROJ, &NT, &nK, &nX, &nst, &tiles)) return HM_EUNSUPPORTED;
#define HM_TCP(N) return launch_tcp_nt<N, PROJ>(A, mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl, nK, nX, nst, tiles)
  switch (NT) {
    case 16: HM_TCP(16);
    case 32: HM_TCP(32);
    case 64: HM_TCP(64);
    case 128: HM_TCP(128);
    default: HM_TCP(256);
  }
#undef HM_TCP
}

hm_status launch_expand_tc(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                           int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  const hm_status s = launch_tcp<false>(A, mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl);
  if (s != HM_EUNSUPPORTED) return s;
  return launch_leaf<false>(A, mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl);
}

hm_status launch_project_tc(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                            int64_t ldx, int xt, cudaStream_t st, bool pdl) {
  const hm_status s = launch_tcp<true>(A, mv, ws, r, X, ldx, xt, nullptr, 0, 0, st, pdl);
  if (s != HM_EUNSUPPORTED) return s;
  return launch_leaf<true>(A, mv, ws, r, X, ldx, xt, nullptr, 0, 0, st, pdl);
}

}  // namespace hmi

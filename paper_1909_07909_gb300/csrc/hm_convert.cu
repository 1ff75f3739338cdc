// hm_hss_to_hodlr: the HODLR form of an HSS matrix (hss2hodlr, Sec. 3.5),
// built on the device from the HSS matrix's own storage.
//
// With the nested bases of Eq. 2.2 written out explicitly for every node,
// the sibling blocks of Def. 2.3 are A(I_a, I_b) = U_a B12_q V_b^T and
// A(I_b, I_a) = U_b B21_q V_a^T, so the HODLR factors of Def. 2.2 are
//   U12_q = U_a B12_q,  V12_q = V_b,  U21_q = U_b B21_q,  V21_q = V_a,
// and the diagonal blocks are kept.  In the library's HODLR layout the factor
// living on the rows of node x (level l) sits in the level-l slot of those
// rows: the U factor (U_x times its parent's coupling) in the expansion plane,
// the V factor (the explicit V_x) in the projection rows.
//
// Each block takes up to 8 rows of one leaf.  A row's explicit bases start
// as the leaf's U and V rows and climb one level at a time through the
// child's half of R_U and R_V (the row of U_q is the row of U_x times R_U's
// half for x); at every level the block writes both factors.  Arithmetic is
// in the tree operators' type (float64 for F64 storage, float32 otherwise),
// each stored factor rounded once to the storage type (split BF16: hi and
// lo of the float32 value).  Every level's rank is the HSS column rank as
// stored (padded to a multiple of 8), so the HODLR rank total is p Kp.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>

#include "hm_api_internal.h"

namespace hmi {

constexpr int CONV_ROWS = 8;

template <int ST, typename C>
__device__ __forceinline__ C st_load(const void* hi, const void* lo, int64_t i) {
  if constexpr (ST == HM_F64) {
    return static_cast<C>(static_cast<const double*>(hi)[i]);
  } else if constexpr (ST == HM_F32) {
    return static_cast<C>(static_cast<const float*>(hi)[i]);
  } else if constexpr (ST == HM_BF16) {
    return static_cast<C>(__bfloat162float(static_cast<const __nv_bfloat16*>(hi)[i]));
  } else {
    return static_cast<C>(__bfloat162float(static_cast<const __nv_bfloat16*>(hi)[i]) +
                          __bfloat162float(static_cast<const __nv_bfloat16*>(lo)[i]));
  }
}

template <int ST, typename C>
__device__ __forceinline__ void st_store(void* hi, void* lo, int64_t i, C v) {
  if constexpr (ST == HM_F64) {
    static_cast<double*>(hi)[i] = static_cast<double>(v);
  } else if constexpr (ST == HM_F32) {
    static_cast<float*>(hi)[i] = static_cast<float>(v);
  } else if constexpr (ST == HM_BF16) {
    static_cast<__nv_bfloat16*>(hi)[i] = __float2bfloat16_rn(static_cast<float>(v));
  } else {
    const float f = static_cast<float>(v);
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    static_cast<__nv_bfloat16*>(hi)[i] = h;
    static_cast<__nv_bfloat16*>(lo)[i] = __float2bfloat16_rn(f - __bfloat162float(h));
  }
}

// Element copy of one plane entry (both planes of split BF16).
template <int ST>
__device__ __forceinline__ void st_copy(const void* shi, const void* slo, int64_t si, void* dhi, void* dlo,
                                        int64_t di) {
  if constexpr (ST == HM_F64) {
    static_cast<double*>(dhi)[di] = static_cast<const double*>(shi)[si];
  } else if constexpr (ST == HM_F32) {
    static_cast<float*>(dhi)[di] = static_cast<const float*>(shi)[si];
  } else {
    static_cast<uint16_t*>(dhi)[di] = static_cast<const uint16_t*>(shi)[si];
    if constexpr (ST == HM_BF16X2) static_cast<uint16_t*>(dlo)[di] = static_cast<const uint16_t*>(slo)[si];
  }
}

struct ConvArgs {
  const int64_t* off;
  int p, L, m_pad;
  int Ke, Kp;                  // HSS row and column ranks (padded)
  int WeS, WeH, KH;            // row widths of the two expansion planes; HODLR rank total
  const void *AS, *ASlo, *WS, *WSlo;
  const void *RU, *RV, *B12, *B21;
  void *AH, *AHlo, *WH, *WHlo;
};

template <int ST, typename C>
__global__ void __launch_bounds__(256) k_hss_to_hodlr(ConvArgs g) {
  extern __shared__ __align__(16) uint8_t conv_smem[];
  const int leaf = blockIdx.x;
  const int64_t a0 = g.off[leaf];
  const int m = static_cast<int>(g.off[leaf + 1] - a0);
  const int r0 = blockIdx.y * CONV_ROWS;
  if (r0 >= m) return;
  const int nr = min(CONV_ROWS, m - r0);
  const int Ke = g.Ke, Kp = g.Kp;
  C* u = reinterpret_cast<C*>(conv_smem);
  C* u2 = u + CONV_ROWS * Ke;
  C* v = u2 + CONV_ROWS * Ke;
  C* v2 = v + CONV_ROWS * Kp;
  const C* RU = static_cast<const C*>(g.RU);
  const C* RV = static_cast<const C*>(g.RV);
  for (int t = threadIdx.x; t < nr * Ke; t += blockDim.x) {
    const int r = t / Ke, i = t % Ke;
    u[r * Ke + i] = st_load<ST, C>(g.AS, g.ASlo, (a0 + r0 + r) * g.WeS + g.m_pad + i);
  }
  for (int t = threadIdx.x; t < nr * Kp; t += blockDim.x) {
    const int r = t / Kp, a = t % Kp;
    v[r * Kp + a] = st_load<ST, C>(g.WS, g.WSlo, (static_cast<int64_t>(leaf) * Kp + a) * g.m_pad + r0 + r);
  }
  for (int t = threadIdx.x; t < nr * g.m_pad; t += blockDim.x) {       // diagonal block (and its padding)
    const int r = t / g.m_pad, cc = t % g.m_pad;
    st_copy<ST>(g.AS, g.ASlo, (a0 + r0 + r) * g.WeS + cc, g.AH, g.AHlo, (a0 + r0 + r) * g.WeH + cc);
  }
  __syncthreads();
  int x = g.L - 1 + leaf;
  for (int l = g.p; l >= 1; --l) {
    const int q = (x - 1) / 2;
    const bool left = (x & 1) != 0;
    const C* Bq = static_cast<const C*>(left ? g.B12 : g.B21) + static_cast<int64_t>(q) * Kp * Ke;
    const int slot = (l - 1) * Kp;
    for (int t = threadIdx.x; t < nr * Kp; t += blockDim.x) {
      const int r = t / Kp, a = t % Kp;
      C acc = C(0);
      for (int i = 0; i < Ke; ++i) acc = fma(u[r * Ke + i], Bq[static_cast<int64_t>(a) * Ke + i], acc);
      st_store<ST, C>(g.AH, g.AHlo, (a0 + r0 + r) * g.WeH + g.m_pad + slot + a, acc);
      st_store<ST, C>(g.WH, g.WHlo, (static_cast<int64_t>(leaf) * g.KH + slot + a) * g.m_pad + r0 + r,
                      v[r * Kp + a]);
    }
    if (l > 1) {
      const int h = left ? 0 : 1;
      const C* Ru = RU + static_cast<int64_t>(q * 2 + h) * Ke * Ke;            // [j][i]
      const C* Rv = RV + (static_cast<int64_t>(q) * 2 * Kp + h * Kp) * Kp;     // [i][j]
      for (int t = threadIdx.x; t < nr * Ke; t += blockDim.x) {
        const int r = t / Ke, j = t % Ke;
        C acc = C(0);
        for (int i = 0; i < Ke; ++i) acc = fma(u[r * Ke + i], Ru[static_cast<int64_t>(j) * Ke + i], acc);
        u2[r * Ke + j] = acc;
      }
      for (int t = threadIdx.x; t < nr * Kp; t += blockDim.x) {
        const int r = t / Kp, j = t % Kp;
        C acc = C(0);
        for (int i = 0; i < Kp; ++i) acc = fma(v[r * Kp + i], Rv[static_cast<int64_t>(i) * Kp + j], acc);
        v2[r * Kp + j] = acc;
      }
      __syncthreads();
      C* tu = u; u = u2; u2 = tu;
      C* tv = v; v = v2; v2 = tv;
    }
    x = q;
  }
}

template <int ST, typename C>
static cudaError_t launch_convert(const ConvArgs& a, int m_max, size_t smem) {
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_hss_to_hodlr<ST, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  const dim3 grid(a.L, std::max(1, (m_max + CONV_ROWS - 1) / CONV_ROWS));
  k_hss_to_hodlr<ST, C><<<grid, 256, smem>>>(a);
  return cudaGetLastError();
}

static hm_status convert_fail(hm_matrix* H, hm_status st, const char* what, cudaError_t e) {
  void* ptrs[] = {H->d_off, H->d_A, H->d_A_lo, H->d_W, H->d_W_lo};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete H;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return st;
}

}  // namespace hmi

using namespace hmi;

extern "C" hm_status hm_hss_to_hodlr(const hm_matrix* S, hm_matrix** out) {
  if (!out) {
    set_error("out is NULL");
    return HM_EINVAL;
  }
  *out = nullptr;
  if (!S || S->magic != kMagicMatrix) {
    set_error("not a matrix handle");
    return HM_EINVAL;
  }
  if (S->kind != HM_HSS) {
    set_error("hm_hss_to_hodlr needs an HSS matrix");
    return HM_EINVAL;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != S->device) {
    set_error("the matrix lives on device %d, the current device is %d", S->device, dev);
    return HM_EINVAL;
  }
  const int st = S->storage;
  const size_t cs = (st == HM_F64) ? 8 : 4;
  const size_t smem = static_cast<size_t>(2 * CONV_ROWS) * (S->Ke + S->Kp) * cs;
  if (smem > 200 * 1024) {
    set_error("ranks %d, %d too large for the conversion kernel", S->Ke, S->Kp);
    return HM_EUNSUPPORTED;
  }
  hm_matrix* H = new (std::nothrow) hm_matrix();
  if (!H) {
    set_error("host allocation failed");
    return HM_ENOMEM;
  }
  H->magic = kMagicMatrix;
  H->kind = HM_HODLR;
  H->storage = st;
  H->device = S->device;
  H->n = S->n;
  H->p = S->p;
  H->L = S->L;
  H->ends = S->ends;
  H->m_max = S->m_max;
  H->m_pad = S->m_pad;
  H->koff[1] = 0;
  for (int l = 1; l <= S->p; ++l) {
    H->kk[l] = S->Kp;
    H->koff[l + 1] = H->koff[l] + S->Kp;
  }
  const int KH = S->p * S->Kp;
  H->Ke = H->Kp = KH;
  H->We = S->m_pad + KH;
  int64_t d_elems = 0, prev = 0;
  for (int i = 0; i < S->L; ++i) {
    const int64_t m = S->ends[i] - prev;
    d_elems += m * m;
    prev = S->ends[i];
  }
  H->gen_elems = d_elems + 2 * S->n * static_cast<int64_t>(KH);
  H->gen_bytes = static_cast<size_t>(H->gen_elems) * storage_bytes(st);

  const size_t es = (st == HM_F64) ? 8 : (st == HM_F32) ? 4 : 2;
  const bool split = (st == HM_BF16X2);
  const size_t a_elems = static_cast<size_t>(H->n) * H->We;
  const size_t w_elems = static_cast<size_t>(H->L) * KH * H->m_pad;
  size_t dev_bytes = 0;
  struct Alloc { void** p; size_t bytes; };
  Alloc allocs[] = {{reinterpret_cast<void**>(&H->d_off), (H->L + 1) * sizeof(int64_t)},
                    {&H->d_A, a_elems * es},
                    {&H->d_A_lo, split ? a_elems * 2 : 0},
                    {&H->d_W, w_elems * es},
                    {&H->d_W_lo, split ? w_elems * 2 : 0}};
  for (const Alloc& a : allocs) {
    if (a.bytes == 0) continue;
    const cudaError_t e = dev_malloc(reinterpret_cast<void**>(a.p), a.bytes);
    if (e != cudaSuccess)
      return convert_fail(H, e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "cudaMalloc (hss2hodlr)", e);
    dev_bytes += a.bytes;
  }
  cudaError_t e = cudaMemcpy(H->d_off, S->d_off, (H->L + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice);
  // projection rows beyond a leaf's size stay zero
  if (e == cudaSuccess && H->d_W) e = cudaMemset(H->d_W, 0, w_elems * es);
  if (e == cudaSuccess && H->d_W_lo) e = cudaMemset(H->d_W_lo, 0, w_elems * 2);
  if (e != cudaSuccess) return convert_fail(H, HM_ECUDA, "hss2hodlr set-up", e);
  if (a_elems > 0) {
    ConvArgs a;
    a.off = S->d_off;
    a.p = S->p;
    a.L = S->L;
    a.m_pad = S->m_pad;
    a.Ke = S->Ke;
    a.Kp = S->Kp;
    a.WeS = S->We;
    a.WeH = H->We;
    a.KH = KH;
    a.AS = S->d_A;
    a.ASlo = S->d_A_lo;
    a.WS = S->d_W;
    a.WSlo = S->d_W_lo;
    a.RU = S->d_RU;
    a.RV = S->d_RVt;
    a.B12 = S->d_B12;
    a.B21 = S->d_B21;
    a.AH = H->d_A;
    a.AHlo = H->d_A_lo;
    a.WH = H->d_W;
    a.WHlo = H->d_W_lo;
    switch (st) {
      case HM_F64: e = launch_convert<HM_F64, double>(a, S->m_max, smem); break;
      case HM_F32: e = launch_convert<HM_F32, float>(a, S->m_max, smem); break;
      case HM_BF16: e = launch_convert<HM_BF16, float>(a, S->m_max, smem); break;
      default: e = launch_convert<HM_BF16X2, float>(a, S->m_max, smem); break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return convert_fail(H, HM_ECUDA, "hss2hodlr kernel", e);
  }
  H->dev_bytes = dev_bytes;
  make_tensor_maps(H);
  H->err = device_error_word(H->device);
  if (!H->err) return convert_fail(H, HM_ECUDA, "device error word", cudaErrorMemoryAllocation);
  *out = H;
  return HM_OK;
}

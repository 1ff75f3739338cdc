// hm_hadamard: C = A o B (entrywise product) of two HODLR or two HSS matrices
// on the same cluster tree, built on the device from A's and B's storage
// (Sec. 4.4, Eq. 4.1, Fig. 4.3).
//
// For low-rank blocks (U1 B1 V1^T) o (U2 B2 V2^T) = (U1 (.)^T U2)(B1 (x) B2)(V1 (.)^T V2)^T,
// where (x) is the Kronecker product and (.)^T the transpose Khatri-Rao
// product (row i = kron(row i of U1, row i of U2)).  Hence:
//   * D_C = D_A o D_B on every leaf;
//   * every factor of C is the transpose Khatri-Rao product of A's and B's
//     (HODLR: on every level; HSS: the leaf bases), column a1 * k_B + a2;
//   * HSS: B12_C = B12_A (x) B12_B, B21_C likewise, and each child's block
//     of the stacked translation operators R_U = [R_l; R_r], R_V = [W_l; W_r]
//     is the Kronecker product of A's and B's blocks for that child.
// Ranks multiply: HODLR per level (each level's largest rank), HSS the
// largest row and column ranks before padding; C pads the products to 8.
// Products are formed in the tree operators' type (float64 for F64 storage,
// float32 otherwise) and each stored entry of D and of the factors is
// rounded once to the storage type (split BF16: hi and lo of the float32
// product of the two hi + lo values); the HSS operators stay in float32 /
// float64.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>

#include "hm_api_internal.h"

namespace hmi {

namespace {

template <int ST, typename C>
__device__ __forceinline__ C hd_load(const void* hi, const void* lo, int64_t i) {
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
__device__ __forceinline__ void hd_store(void* hi, void* lo, int64_t i, C v) {
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

}  // namespace

// One block of factor columns: offsets of the block in A, B and C (within
// the factor region of a row, or the factor rows of a leaf) and A's and B's
// ranks; C's block has kA * kB columns.
struct HdSeg {
  int offA, offB, offC, kA, kB;
};

constexpr int kHdMaxSeg = kMaxDepth + 1;

struct HdArgs {
  const int64_t* off;
  int m_pad;
  int WeA, WeB, WeC;           // row widths of the expansion planes
  int KpA, KpB, KpC;           // projection rows per leaf
  int nu, nv;                  // U and V blocks
  HdSeg us[kHdMaxSeg], vs[kHdMaxSeg];
  const void *AA, *AAlo, *WA, *WAlo, *AB, *ABlo, *WB, *WBlo;
  void *AC, *AClo, *WC, *WClo;
};

template <int ST, typename C>
__global__ void __launch_bounds__(256) k_hadamard_leaves(HdArgs g) {
  const int leaf = blockIdx.x;
  const int64_t a0 = g.off[leaf];
  const int m = static_cast<int>(g.off[leaf + 1] - a0);
  const int64_t stride = static_cast<int64_t>(blockDim.x) * gridDim.y;
  const int64_t first = threadIdx.x + static_cast<int64_t>(blockIdx.y) * blockDim.x;
  // diagonal block
  const int64_t nd = static_cast<int64_t>(m) * g.m_pad;
  for (int64_t e = first; e < nd; e += stride) {
    const int64_t row = a0 + e / g.m_pad;
    const int cc = static_cast<int>(e % g.m_pad);
    const C x = hd_load<ST, C>(g.AA, g.AAlo, row * g.WeA + cc) * hd_load<ST, C>(g.AB, g.ABlo, row * g.WeB + cc);
    hd_store<ST, C>(g.AC, g.AClo, row * g.WeC + cc, x);
  }
  // row factors: Khatri-Rao columns of every block
  for (int s = 0; s < g.nu; ++s) {
    const HdSeg sg = g.us[s];
    const int kc = sg.kA * sg.kB;
    const int64_t nu = static_cast<int64_t>(m) * kc;
    for (int64_t e = first; e < nu; e += stride) {
      const int64_t row = a0 + e / kc;
      const int ac = static_cast<int>(e % kc);
      const int a1 = ac / sg.kB, a2 = ac % sg.kB;
      const C x = hd_load<ST, C>(g.AA, g.AAlo, row * g.WeA + g.m_pad + sg.offA + a1) *
                  hd_load<ST, C>(g.AB, g.ABlo, row * g.WeB + g.m_pad + sg.offB + a2);
      hd_store<ST, C>(g.AC, g.AClo, row * g.WeC + g.m_pad + sg.offC + ac, x);
    }
  }
  // column factors (projection rows of the leaf; rows past m stay zero)
  for (int s = 0; s < g.nv; ++s) {
    const HdSeg sg = g.vs[s];
    const int kc = sg.kA * sg.kB;
    const int64_t nv = static_cast<int64_t>(kc) * m;
    for (int64_t e = first; e < nv; e += stride) {
      const int ac = static_cast<int>(e / m);
      const int rr = static_cast<int>(e % m);
      const int a1 = ac / sg.kB, a2 = ac % sg.kB;
      const C x = hd_load<ST, C>(g.WA, g.WAlo, (static_cast<int64_t>(leaf) * g.KpA + sg.offA + a1) * g.m_pad + rr) *
                  hd_load<ST, C>(g.WB, g.WBlo, (static_cast<int64_t>(leaf) * g.KpB + sg.offB + a2) * g.m_pad + rr);
      hd_store<ST, C>(g.WC, g.WClo, (static_cast<int64_t>(leaf) * g.KpC + sg.offC + ac) * g.m_pad + rr, x);
    }
  }
}

// HSS operators (layouts as built by hm_hss_create; strides are the padded
// ranks Ke, Kp):
//   RU[q][h][j][i] (i, j < Ke), RV[q][h*Kp + i][j] (i, j < Kp),
//   B12[q][j][i], B21[q][j][i] (j < Kp, i < Ke).
// C's index x pairs A's index x1 with B's x2 as x = x1 * k_B + x2, k_B the
// unpadded rank of B (ku for U-side indices, kv for V-side ones); C's
// padding indices (x >= k_A k_B) hold zeros.
struct HdTree {
  int nI;
  int kuA, kvA, kuB, kvB;                 // unpadded ranks
  int KeA, KpA, KeB, KpB, KeC, KpC;       // padded strides
};

template <typename C>
__global__ void k_hadamard_tree(HdTree t, const C* __restrict__ RUA, const C* __restrict__ RVA,
                                const C* __restrict__ B12A, const C* __restrict__ B21A, const C* __restrict__ RUB,
                                const C* __restrict__ RVB, const C* __restrict__ B12B, const C* __restrict__ B21B,
                                C* __restrict__ RUC, C* __restrict__ RVC, C* __restrict__ B12C,
                                C* __restrict__ B21C) {
  const int KeC = t.KeC, KpC = t.KpC;
  const int kuC = t.kuA * t.kuB, kvC = t.kvA * t.kvB;
  const int64_t stride = static_cast<int64_t>(blockDim.x) * gridDim.x;
  const int64_t first = threadIdx.x + static_cast<int64_t>(blockIdx.x) * blockDim.x;
  const int64_t nru = static_cast<int64_t>(t.nI) * 2 * KeC * KeC;
  for (int64_t e = first; e < nru; e += stride) {            // RUC[qh][jc][ic]
    const int ic = static_cast<int>(e % KeC);
    const int jc = static_cast<int>((e / KeC) % KeC);
    const int64_t qh = e / (static_cast<int64_t>(KeC) * KeC);
    C v = C(0);
    if (ic < kuC && jc < kuC) {
      const int i1 = ic / t.kuB, i2 = ic % t.kuB, j1 = jc / t.kuB, j2 = jc % t.kuB;
      v = RUA[(qh * t.KeA + j1) * t.KeA + i1] * RUB[(qh * t.KeB + j2) * t.KeB + i2];
    }
    RUC[e] = v;
  }
  const int64_t nrv = static_cast<int64_t>(t.nI) * 2 * KpC * KpC;
  for (int64_t e = first; e < nrv; e += stride) {            // RVC[q][h*KpC + ic][jc]
    const int jc = static_cast<int>(e % KpC);
    const int64_t rowc = e / KpC;                            // q * 2 KpC + h KpC + ic
    const int ic = static_cast<int>(rowc % KpC);
    const int64_t qh = rowc / KpC;
    C v = C(0);
    if (ic < kvC && jc < kvC) {
      const int i1 = ic / t.kvB, i2 = ic % t.kvB, j1 = jc / t.kvB, j2 = jc % t.kvB;
      v = RVA[(qh * t.KpA + i1) * t.KpA + j1] * RVB[(qh * t.KpB + i2) * t.KpB + j2];
    }
    RVC[e] = v;
  }
  const int64_t nb = static_cast<int64_t>(t.nI) * KpC * KeC;
  for (int64_t e = first; e < nb; e += stride) {             // B12C[q][jc][ic]
    const int ic = static_cast<int>(e % KeC);
    const int jc = static_cast<int>((e / KeC) % KpC);
    const int64_t q = e / (static_cast<int64_t>(KeC) * KpC);
    C v12 = C(0), v21 = C(0);
    if (ic < kuC && jc < kvC) {
      const int i1 = ic / t.kuB, i2 = ic % t.kuB, j1 = jc / t.kvB, j2 = jc % t.kvB;
      const int64_t ea = (q * t.KpA + j1) * t.KeA + i1, eb = (q * t.KpB + j2) * t.KeB + i2;
      v12 = B12A[ea] * B12B[eb];
      v21 = B21A[ea] * B21B[eb];
    }
    B12C[e] = v12;
    B21C[e] = v21;
  }
}

template <int ST, typename C>
static cudaError_t launch_hadamard_leaves(const HdArgs& a, int L, int64_t per_leaf) {
  const int gy = static_cast<int>(std::min<int64_t>(64, std::max<int64_t>(1, per_leaf / 4096)));
  k_hadamard_leaves<ST, C><<<dim3(L, gy), 256>>>(a);
  return cudaGetLastError();
}

static hm_status hadamard_fail(hm_matrix* M, hm_status st, const char* what, cudaError_t e) {
  void* ptrs[] = {M->d_off, M->d_A, M->d_A_lo, M->d_W, M->d_W_lo, M->d_RU, M->d_RVt, M->d_B12, M->d_B21};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete M;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return st;
}

}  // namespace hmi

using namespace hmi;

extern "C" hm_status hm_hadamard(const hm_matrix* A, const hm_matrix* B, hm_matrix** out) {
  if (!out) {
    set_error("out is NULL");
    return HM_EINVAL;
  }
  *out = nullptr;
  if (!A || A->magic != kMagicMatrix || !B || B->magic != kMagicMatrix) {
    set_error("not a matrix handle");
    return HM_EINVAL;
  }
  if (A->kind != B->kind || A->storage != B->storage) {
    set_error("A and B must have the same kind and storage type");
    return HM_EINVAL;
  }
  if (A->n != B->n || A->L != B->L || A->ends != B->ends) {
    set_error("A and B must have the same cluster tree");
    return HM_EINVAL;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != A->device || dev != B->device) {
    set_error("A and B must live on the current device");
    return HM_EINVAL;
  }
  const bool hss = (A->kind == HM_HSS);
  hm_matrix* M = new (std::nothrow) hm_matrix();
  if (!M) {
    set_error("host allocation failed");
    return HM_ENOMEM;
  }
  M->magic = kMagicMatrix;
  M->kind = A->kind;
  M->storage = A->storage;
  M->device = A->device;
  M->n = A->n;
  M->p = A->p;
  M->L = A->L;
  M->ends = A->ends;
  M->m_max = A->m_max;
  M->m_pad = A->m_pad;
  HdArgs a;
  std::memset(&a, 0, sizeof(a));
  if (hss) {
    M->ku_max = A->ku_max * B->ku_max;
    M->kv_max = A->kv_max * B->kv_max;
    M->Ke = (M->ku_max + 7) / 8 * 8;
    M->Kp = (M->kv_max + 7) / 8 * 8;
    a.nu = a.nv = 1;
    a.us[0] = HdSeg{0, 0, 0, A->ku_max, B->ku_max};
    a.vs[0] = HdSeg{0, 0, 0, A->kv_max, B->kv_max};
  } else {
    M->koff[1] = 0;
    for (int l = 1; l <= A->p; ++l) {
      M->kk[l] = A->kk[l] * B->kk[l];
      M->koff[l + 1] = M->koff[l] + M->kk[l];
      a.us[l - 1] = a.vs[l - 1] = HdSeg{A->koff[l], B->koff[l], M->koff[l], A->kk[l], B->kk[l]};
    }
    a.nu = a.nv = A->p;
    M->Ke = M->Kp = (M->koff[A->p + 1] + 7) / 8 * 8;
  }
  if (M->Ke > 4096 || M->Kp > 4096) {
    const int ke = M->Ke, kp = M->Kp;
    delete M;
    set_error("the product's ranks (%d, %d) are above 4096", ke, kp);
    return HM_EUNSUPPORTED;
  }
  M->We = M->m_pad + M->Ke;
  int64_t d_elems = 0, prev = 0;
  for (int i = 0; i < M->L; ++i) {
    const int64_t m = M->ends[i] - prev;
    d_elems += m * m;
    prev = M->ends[i];
  }
  const int st = A->storage;
  const size_t cs = (st == HM_F64) ? 8 : 4;
  const size_t nI = static_cast<size_t>(std::max(M->L - 1, 0));
  if (hss) {
    const int64_t ku = M->ku_max, kv = M->kv_max;
    const int64_t t_elems = static_cast<int64_t>(std::max(M->L - 2, 0)) * 2 * (ku * ku + kv * kv) +
                            static_cast<int64_t>(nI) * 2 * ku * kv;
    const int64_t l_elems = d_elems + M->n * static_cast<int64_t>(M->L > 1 ? M->ku_max + M->kv_max : 0);
    M->gen_elems = l_elems + t_elems;
    M->gen_bytes = static_cast<size_t>(l_elems) * storage_bytes(st) + static_cast<size_t>(t_elems) * cs;
  } else {
    M->gen_elems = d_elems + 2 * M->n * static_cast<int64_t>(M->koff[M->p + 1]);
    M->gen_bytes = static_cast<size_t>(M->gen_elems) * storage_bytes(st);
  }
  const size_t es = (st == HM_F64) ? 8 : (st == HM_F32) ? 4 : 2;
  const bool split = (st == HM_BF16X2);
  const size_t a_elems = static_cast<size_t>(M->n) * M->We;
  const size_t w_elems = static_cast<size_t>(M->L) * M->Kp * M->m_pad;
  const size_t ru_b = hss ? nI * 2 * M->Ke * M->Ke * cs : 0;
  const size_t rv_b = hss ? nI * 2 * M->Kp * M->Kp * cs : 0;
  const size_t b_b = hss ? nI * M->Kp * M->Ke * cs : 0;
  size_t dev_bytes = 0;
  struct Alloc { void** p; size_t bytes; bool zero; };
  Alloc allocs[] = {{reinterpret_cast<void**>(&M->d_off), (M->L + 1) * sizeof(int64_t), false},
                    {&M->d_A, a_elems * es, true},
                    {&M->d_A_lo, split ? a_elems * 2 : 0, true},
                    {&M->d_W, w_elems * es, true},
                    {&M->d_W_lo, split ? w_elems * 2 : 0, true},
                    {&M->d_RU, ru_b, false},
                    {&M->d_RVt, rv_b, false},
                    {&M->d_B12, b_b, false},
                    {&M->d_B21, b_b, false}};
  for (const Alloc& al : allocs) {
    if (al.bytes == 0) continue;
    cudaError_t e = dev_malloc(reinterpret_cast<void**>(al.p), al.bytes);
    if (e == cudaSuccess && al.zero) e = cudaMemset(*al.p, 0, al.bytes);   // padding columns and rows
    if (e != cudaSuccess)
      return hadamard_fail(M, e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "allocation (hadamard)", e);
    dev_bytes += al.bytes;
  }
  cudaError_t e = cudaMemcpy(M->d_off, A->d_off, (M->L + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) return hadamard_fail(M, HM_ECUDA, "copy of the leaf offsets", e);
  a.off = A->d_off;
  a.m_pad = M->m_pad;
  a.WeA = A->We;
  a.WeB = B->We;
  a.WeC = M->We;
  a.KpA = A->Kp;
  a.KpB = B->Kp;
  a.KpC = M->Kp;
  a.AA = A->d_A;
  a.AAlo = A->d_A_lo;
  a.WA = A->d_W;
  a.WAlo = A->d_W_lo;
  a.AB = B->d_A;
  a.ABlo = B->d_A_lo;
  a.WB = B->d_W;
  a.WBlo = B->d_W_lo;
  a.AC = M->d_A;
  a.AClo = M->d_A_lo;
  a.WC = M->d_W;
  a.WClo = M->d_W_lo;
  if (a_elems > 0) {
    const int64_t per_leaf = static_cast<int64_t>(M->m_max) * M->We + static_cast<int64_t>(M->Kp) * M->m_max;
    switch (st) {
      case HM_F64: e = launch_hadamard_leaves<HM_F64, double>(a, M->L, per_leaf); break;
      case HM_F32: e = launch_hadamard_leaves<HM_F32, float>(a, M->L, per_leaf); break;
      case HM_BF16: e = launch_hadamard_leaves<HM_BF16, float>(a, M->L, per_leaf); break;
      default: e = launch_hadamard_leaves<HM_BF16X2, float>(a, M->L, per_leaf); break;
    }
    if (e != cudaSuccess) return hadamard_fail(M, HM_ECUDA, "hadamard leaf kernel", e);
  }
  if (hss && nI > 0) {
    HdTree t{static_cast<int>(nI), A->ku_max, A->kv_max, B->ku_max, B->kv_max,
             A->Ke, A->Kp, B->Ke, B->Kp, M->Ke, M->Kp};
    const int64_t most = static_cast<int64_t>(nI) * 2 * std::max(M->Ke, M->Kp) * std::max(M->Ke, M->Kp);
    const int grid = static_cast<int>(std::min<int64_t>(4096, std::max<int64_t>(1, (most + 255) / 256)));
    if (cs == 8)
      k_hadamard_tree<double><<<grid, 256>>>(
          t, static_cast<const double*>(A->d_RU), static_cast<const double*>(A->d_RVt),
          static_cast<const double*>(A->d_B12), static_cast<const double*>(A->d_B21),
          static_cast<const double*>(B->d_RU), static_cast<const double*>(B->d_RVt),
          static_cast<const double*>(B->d_B12), static_cast<const double*>(B->d_B21),
          static_cast<double*>(M->d_RU), static_cast<double*>(M->d_RVt), static_cast<double*>(M->d_B12),
          static_cast<double*>(M->d_B21));
    else
      k_hadamard_tree<float><<<grid, 256>>>(
          t, static_cast<const float*>(A->d_RU), static_cast<const float*>(A->d_RVt),
          static_cast<const float*>(A->d_B12), static_cast<const float*>(A->d_B21),
          static_cast<const float*>(B->d_RU), static_cast<const float*>(B->d_RVt),
          static_cast<const float*>(B->d_B12), static_cast<const float*>(B->d_B21),
          static_cast<float*>(M->d_RU), static_cast<float*>(M->d_RVt), static_cast<float*>(M->d_B12),
          static_cast<float*>(M->d_B21));
    e = cudaGetLastError();
    if (e != cudaSuccess) return hadamard_fail(M, HM_ECUDA, "hadamard tree kernel", e);
  }
  e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return hadamard_fail(M, HM_ECUDA, "hadamard kernels", e);
  M->dev_bytes = dev_bytes;
  make_tensor_maps(M);
  M->err = device_error_word(M->device);
  if (!M->err) return hadamard_fail(M, HM_ECUDA, "device error word", cudaErrorMemoryAllocation);
  *out = M;
  return HM_OK;
}

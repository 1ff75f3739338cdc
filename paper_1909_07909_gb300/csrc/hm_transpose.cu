// hm_matrix_transpose: A^T as a new library matrix, built on the device from
// A's own storage, so that products with A^T (needed next to products with A
// by the Lanczos and randomized constructors of Sec. 3.2 and Sec. 3.3,
// Table 3.1) run through the same kernels as products with A.
//
// Transposing keeps the cluster tree and relabels the generators block by
// block, (A^T)(I, J) = A(J, I)^T:
//   * every leaf's diagonal block D_i becomes D_i^T;
//   * the row factors of A^T are A's column factors and the other way round
//     (HODLR, Def. 2.2: on every level; HSS, Def. 2.3: the leaf bases), so
//     the U columns of the expansion plane and the per-leaf projection rows
//     trade places;
//   * HSS (Eq. 2.2): R_U' = R_V, R_V' = R_U, B12' = B21^T, B21' = B12^T.
// In the library's layout every one of these is a permutation of stored
// elements (both planes of split BF16 alike), so A^T holds exactly A's
// values: no rounding happens, and (A^T)^T is A bit for bit.
#include <algorithm>
#include <cstring>

#include "hm_api_internal.h"

namespace hmi {

// One block row of leaves per blockIdx.x; blockIdx.y strides the elements.
// A: n x We rows [D | U]; W: L x Kp x m_pad projection rows (V^T).
// At: n x Wet rows [D^T | V] with Wet = m_pad + Kp; Wt: L x Ke x m_pad (U^T).
template <typename T>
__global__ void k_transpose_leaves(const int64_t* __restrict__ off, int m_pad, const T* __restrict__ A, int We,
                                   const T* __restrict__ W, int Kp, T* __restrict__ At, int Wet,
                                   T* __restrict__ Wt, int Ke) {
  const int leaf = blockIdx.x;
  const int64_t a0 = off[leaf];
  const int m = static_cast<int>(off[leaf + 1] - a0);
  const int64_t stride = static_cast<int64_t>(blockDim.x) * gridDim.y;
  const int64_t first = threadIdx.x + static_cast<int64_t>(blockIdx.y) * blockDim.x;
  const int64_t rows_out = static_cast<int64_t>(m) * Wet;
  for (int64_t e = first; e < rows_out; e += stride) {
    const int rr = static_cast<int>(e / Wet), cc = static_cast<int>(e % Wet);
    T v = T(0);
    if (cc < m) v = A[(a0 + cc) * We + rr];                                             // D^T
    else if (cc >= m_pad) v = W[(static_cast<int64_t>(leaf) * Kp + (cc - m_pad)) * m_pad + rr];   // V row
    At[(a0 + rr) * Wet + cc] = v;
  }
  const int64_t proj_out = static_cast<int64_t>(Ke) * m_pad;
  for (int64_t e = first; e < proj_out; e += stride) {
    const int a = static_cast<int>(e / m_pad), rr = static_cast<int>(e % m_pad);
    Wt[(static_cast<int64_t>(leaf) * Ke + a) * m_pad + rr] = (rr < m) ? A[(a0 + rr) * We + m_pad + a] : T(0);
  }
}

// HSS translation and coupling operators of the nI internal nodes (compute
// type C; layouts as built by hm_hss_create):
//   RU [q][h][j][i] = R_U(half h, row i; column j), i, j < Ke
//   RV [q][h*Kp + i][j] = R_V(half h, row i; column j), i, j < Kp
//   B12[q][j][i] = B12(i, j), B21[q][j][i] = B21(i, j), j < Kp, i < Ke
// A^T has Ke' = Kp and Kp' = Ke.
template <typename C>
__global__ void k_transpose_tree(int nI, int Ke, int Kp, const C* __restrict__ RU, const C* __restrict__ RV,
                                 const C* __restrict__ B12, const C* __restrict__ B21, C* __restrict__ RUt,
                                 C* __restrict__ RVt, C* __restrict__ B12t, C* __restrict__ B21t) {
  const int64_t stride = static_cast<int64_t>(blockDim.x) * gridDim.x;
  const int64_t first = threadIdx.x + static_cast<int64_t>(blockIdx.x) * blockDim.x;
  // R_U' = R_V: RUt[q][h][j][i] (i, j < Kp)
  const int64_t nru = static_cast<int64_t>(nI) * 2 * Kp * Kp;
  for (int64_t e = first; e < nru; e += stride) {
    const int i = static_cast<int>(e % Kp);
    const int j = static_cast<int>((e / Kp) % Kp);
    const int64_t qh = e / (static_cast<int64_t>(Kp) * Kp);       // q * 2 + h
    RUt[e] = RV[(qh * Kp + i) * Kp + j];
  }
  // R_V' = R_U: RVt[q][h*Ke + i][j] (i, j < Ke)
  const int64_t nrv = static_cast<int64_t>(nI) * 2 * Ke * Ke;
  for (int64_t e = first; e < nrv; e += stride) {
    const int j = static_cast<int>(e % Ke);
    const int i = static_cast<int>((e / Ke) % Ke);
    const int64_t qh = e / (static_cast<int64_t>(Ke) * Ke);
    RVt[e] = RU[(qh * Ke + j) * Ke + i];
  }
  // B12' = B21^T, B21' = B12^T: out[q][j][i] (j < Ke, i < Kp) = in[q][i][j]
  const int64_t nb = static_cast<int64_t>(nI) * Ke * Kp;
  for (int64_t e = first; e < nb; e += stride) {
    const int i = static_cast<int>(e % Kp);
    const int j = static_cast<int>((e / Kp) % Ke);
    const int64_t q = e / (static_cast<int64_t>(Kp) * Ke);
    const int64_t src = (q * Kp + i) * Ke + j;
    B12t[e] = B21[src];
    B21t[e] = B12[src];
  }
}

static hm_status transpose_fail(hm_matrix* T, hm_status st, const char* what, cudaError_t e) {
  void* ptrs[] = {T->d_off, T->d_A, T->d_A_lo, T->d_W, T->d_W_lo, T->d_RU, T->d_RVt, T->d_B12, T->d_B21};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete T;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return st;
}

template <typename T>
static void launch_leaves(const hm_matrix* A, hm_matrix* At, void* src_A, void* src_W, void* dst_A, void* dst_W) {
  const int64_t per_leaf = std::max<int64_t>(static_cast<int64_t>(A->m_max) * At->We, static_cast<int64_t>(A->Ke) * A->m_pad);
  const int gy = static_cast<int>(std::min<int64_t>(64, std::max<int64_t>(1, per_leaf / 2048)));
  k_transpose_leaves<T><<<dim3(A->L, gy), 256>>>(A->d_off, A->m_pad, static_cast<const T*>(src_A), A->We,
                                                static_cast<const T*>(src_W), A->Kp, static_cast<T*>(dst_A), At->We,
                                                static_cast<T*>(dst_W), A->Ke);
}

}  // namespace hmi

using namespace hmi;

extern "C" hm_status hm_matrix_transpose(const hm_matrix* A, hm_matrix** out) {
  if (!out) {
    set_error("out is NULL");
    return HM_EINVAL;
  }
  *out = nullptr;
  if (!A || A->magic != kMagicMatrix) {
    set_error("not a matrix handle");
    return HM_EINVAL;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != A->device) {
    set_error("the matrix lives on device %d, the current device is %d", A->device, dev);
    return HM_EINVAL;
  }
  hm_matrix* T = new (std::nothrow) hm_matrix();
  if (!T) {
    set_error("host allocation failed");
    return HM_ENOMEM;
  }
  T->magic = kMagicMatrix;
  T->kind = A->kind;
  T->storage = A->storage;
  T->device = A->device;
  T->n = A->n;
  T->p = A->p;
  T->L = A->L;
  T->ends = A->ends;
  T->m_max = A->m_max;
  T->m_pad = A->m_pad;
  T->Ke = A->Kp;
  T->Kp = A->Ke;
  T->ku_max = A->kv_max;
  T->kv_max = A->ku_max;
  T->We = A->m_pad + T->Ke;
  for (int l = 0; l <= kMaxDepth + 1; ++l) {
    T->kk[l] = A->kk[l];
    T->koff[l] = A->koff[l];
  }
  T->gen_elems = A->gen_elems;
  T->gen_bytes = A->gen_bytes;

  const int st = A->storage;
  const size_t es = (st == HM_F64) ? 8 : (st == HM_F32) ? 4 : 2;      // hi plane element
  const bool split = (st == HM_BF16X2);
  const size_t cs = (st == HM_F64) ? 8 : 4;                           // tree operators
  const size_t a_elems = static_cast<size_t>(T->n) * T->We;
  const size_t w_elems = static_cast<size_t>(T->L) * T->Kp * T->m_pad;
  const size_t nI = static_cast<size_t>(std::max(T->L - 1, 0));
  const bool hss = (A->kind == HM_HSS);
  const size_t ru_b = hss ? nI * 2 * T->Ke * T->Ke * cs : 0;
  const size_t rv_b = hss ? nI * 2 * T->Kp * T->Kp * cs : 0;
  const size_t b_b = hss ? nI * T->Kp * T->Ke * cs : 0;
  size_t dev_bytes = 0;
  struct Alloc { void** p; size_t bytes; };
  Alloc allocs[] = {{reinterpret_cast<void**>(&T->d_off), (T->L + 1) * sizeof(int64_t)},
                    {&T->d_A, a_elems * es},
                    {&T->d_A_lo, split ? a_elems * 2 : 0},
                    {&T->d_W, w_elems * es},
                    {&T->d_W_lo, split ? w_elems * 2 : 0},
                    {&T->d_RU, ru_b},
                    {&T->d_RVt, rv_b},
                    {&T->d_B12, b_b},
                    {&T->d_B21, b_b}};
  for (const Alloc& a : allocs) {
    if (a.bytes == 0) continue;
    const cudaError_t e = dev_malloc(reinterpret_cast<void**>(a.p), a.bytes);
    if (e != cudaSuccess)
      return transpose_fail(T, e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "cudaMalloc (transpose)", e);
    dev_bytes += a.bytes;
  }
  cudaError_t e = cudaMemcpy(T->d_off, A->d_off, (T->L + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) return transpose_fail(T, HM_ECUDA, "copy of the leaf offsets", e);
  if (a_elems > 0 || w_elems > 0) {
    if (es == 8) launch_leaves<uint64_t>(A, T, A->d_A, A->d_W, T->d_A, T->d_W);
    else if (es == 4) launch_leaves<uint32_t>(A, T, A->d_A, A->d_W, T->d_A, T->d_W);
    else launch_leaves<uint16_t>(A, T, A->d_A, A->d_W, T->d_A, T->d_W);
    if (split) launch_leaves<uint16_t>(A, T, A->d_A_lo, A->d_W_lo, T->d_A_lo, T->d_W_lo);
  }
  if (hss && nI > 0) {
    const int64_t most = static_cast<int64_t>(nI) * 2 * std::max(T->Ke, T->Kp) * std::max(T->Ke, T->Kp);
    const int grid = static_cast<int>(std::min<int64_t>(1024, std::max<int64_t>(1, (most + 255) / 256)));
    if (cs == 8)
      k_transpose_tree<double><<<grid, 256>>>(static_cast<int>(nI), A->Ke, A->Kp,
                                              static_cast<const double*>(A->d_RU), static_cast<const double*>(A->d_RVt),
                                              static_cast<const double*>(A->d_B12), static_cast<const double*>(A->d_B21),
                                              static_cast<double*>(T->d_RU), static_cast<double*>(T->d_RVt),
                                              static_cast<double*>(T->d_B12), static_cast<double*>(T->d_B21));
    else
      k_transpose_tree<float><<<grid, 256>>>(static_cast<int>(nI), A->Ke, A->Kp,
                                             static_cast<const float*>(A->d_RU), static_cast<const float*>(A->d_RVt),
                                             static_cast<const float*>(A->d_B12), static_cast<const float*>(A->d_B21),
                                             static_cast<float*>(T->d_RU), static_cast<float*>(T->d_RVt),
                                             static_cast<float*>(T->d_B12), static_cast<float*>(T->d_B21));
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) return transpose_fail(T, HM_ECUDA, "transpose kernels", e);
  T->dev_bytes = dev_bytes;
  make_tensor_maps(T);
  T->err = device_error_word(T->device);
  if (!T->err) return transpose_fail(T, HM_ECUDA, "device error word", cudaErrorMemoryAllocation);
  *out = T;
  return HM_OK;
}

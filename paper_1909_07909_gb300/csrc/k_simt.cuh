// SIMT kernels of the HODLR/HSS product (every storage type, any number of
// right-hand sides).  Instantiated per storage type by k_simt_<type>.cu.
//
// One product is three stream-ordered launches (two for HODLR):
//
//  k_project  grid (leaf, column chunk).  Stages X(I_i, chunk) in shared memory
//             and forms P_i = Wprj_i X(I_i, chunk): HODLR the per-level V^T X of
//             the leaf's rows (Fig. 4.1 left, the V12^T v2 / V21^T v1 terms),
//             HSS x-hat_i = V_i^T X_i (Fig. 4.1 right, first step).  It then
//             climbs the tree: the second of two siblings to arrive (an atomic
//             counter per node and chunk, no waiting) combines them --
//               HODLR: sums the two children's partials (levels 1..l of node q)
//               HSS:   y-hat couplings of the children with B12/B21 (levels
//                      1..p) and the upsweep x-hat_q = R_V^T [x-hat_a; x-hat_b].
//             The combine always adds left before right, so the result does not
//             depend on which sibling arrived last.
//  k_hss_down grid (subtree, chunk).  Downsweep y_child = y_coupling +
//             R_U(half) y_parent (Fig. 4.1 right, third step); a subtree rooted
//             at level s first recomputes its chain of ancestors in shared
//             memory, then owns every node below it.
//  k_expand   grid (leaf row tile, chunk).  Y(I_i) = [D_i | E_i] [X_i; Z_i]: the
//             leaf product plus, in the same pass, every level's U T (HODLR) or
//             the leaf U y-hat (HSS).
//
// Inner product engine (rows_gemm): a warp owns TR rows of the row-major
// operand; lanes split K in 16-byte vectors (coalesced streaming loads of the
// generator planes), multiply with the staged block in shared memory, and a
// butterfly reduce-scatter over the 32 lanes leaves each (row, column) sum in
// one lane.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hm_internal.h"

namespace hmi {

template <int S> struct Stor;
template <> struct Stor<HM_F64> { using C = double; static constexpr int V = 2; };
template <> struct Stor<HM_F32> { using C = float; static constexpr int V = 4; };
template <> struct Stor<HM_BF16> { using C = float; static constexpr int V = 8; };
template <> struct Stor<HM_BF16X2> { using C = float; static constexpr int V = 8; };

__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  return __ldcs(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// V consecutive elements of a generator plane, starting at element `elem`.
template <int S>
__device__ __forceinline__ void load_vec(const void* A, const void* A_lo, int64_t elem,
                                         typename Stor<S>::C* a) {
  if constexpr (S == HM_F64) {
    const uint4 u = ld_stream16(static_cast<const double*>(A) + elem);
    a[0] = __hiloint2double(static_cast<int>(u.y), static_cast<int>(u.x));
    a[1] = __hiloint2double(static_cast<int>(u.w), static_cast<int>(u.z));
  } else if constexpr (S == HM_F32) {
    const uint4 u = ld_stream16(static_cast<const float*>(A) + elem);
    a[0] = __uint_as_float(u.x); a[1] = __uint_as_float(u.y);
    a[2] = __uint_as_float(u.z); a[3] = __uint_as_float(u.w);
  } else {
    const uint4 u = ld_stream16(static_cast<const uint16_t*>(A) + elem);
    a[0] = bf_lo(u.x); a[1] = bf_hi(u.x); a[2] = bf_lo(u.y); a[3] = bf_hi(u.y);
    a[4] = bf_lo(u.z); a[5] = bf_hi(u.z); a[6] = bf_lo(u.w); a[7] = bf_hi(u.w);
    if constexpr (S == HM_BF16X2) {
      // hi + lo is exact in float (at most 17 significant bits).
      const uint4 w = ld_stream16(static_cast<const uint16_t*>(A_lo) + elem);
      a[0] += bf_lo(w.x); a[1] += bf_hi(w.x); a[2] += bf_lo(w.y); a[3] += bf_hi(w.y);
      a[4] += bf_lo(w.z); a[5] += bf_hi(w.z); a[6] += bf_lo(w.w); a[7] += bf_hi(w.w);
    }
  }
}

// V consecutive compute-type values from shared memory (16-byte aligned).
template <typename C, int V>
__device__ __forceinline__ void load_b(const C* p, C* b) {
  if constexpr (sizeof(C) == 8) {
#pragma unroll
    for (int v = 0; v < V; v += 2) {
      const double2 d = *reinterpret_cast<const double2*>(p + v);
      b[v] = d.x; b[v + 1] = d.y;
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; v += 4) {
      const float4 f = *reinterpret_cast<const float4*>(p + v);
      b[v] = f.x; b[v + 1] = f.y; b[v + 2] = f.z; b[v + 3] = f.w;
    }
  }
}

template <typename C>
__device__ __forceinline__ C load_x(const void* X, int xt, int64_t idx) {
  if (xt == HM_F64) return static_cast<C>(static_cast<const double*>(X)[idx]);
  if (xt == HM_F32) return static_cast<C>(static_cast<const float*>(X)[idx]);
  return static_cast<C>(__uint_as_float(static_cast<uint32_t>(static_cast<const uint16_t*>(X)[idx]) << 16));
}

template <typename C>
__device__ __forceinline__ void store_y(void* Y, int yt, int64_t idx, C v) {
  if (yt == HM_F64) static_cast<double*>(Y)[idx] = static_cast<double>(v);
  else static_cast<float*>(Y)[idx] = static_cast<float>(v);
}

// Butterfly reduce-scatter of N values over the 32 lanes of a warp.  After it,
// lane l holds in v[0 .. max(N/32,1)) the full sums of the value indices given
// by rs_index<N>(l, i); for N < 32 the lanes that differ only in their low
// log2(32/N) bits hold the same value.
template <int CNT, int O, typename C>
__device__ __forceinline__ void rs_step(C* v, int lane) {
  if constexpr (O >= 1) {
    if constexpr (CNT > 1) {
      constexpr int H = CNT / 2;
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const C send = up ? v[i] : v[i + H];
        const C keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      rs_step<H, O / 2>(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      rs_step<1, O / 2>(v, lane);
    }
  }
}

template <int N>
__device__ __forceinline__ int rs_index(int lane, int i) {
  int idx = i;
  int cnt = N;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (cnt > 1) {
      const int h = cnt / 2;
      if (lane & o) idx += h;
      cnt = h;
    }
  }
  return idx;
}

// Os[c * OS + t] = sum_k A(row0 + t, k) * Bs[c * KS + k] for t < nrows, c < RC.
// A: row-major plane(s) with leading dimension lda (elements), K a multiple of V.
template <int S, int RC, int TR>
__device__ __forceinline__ void rows_gemm(const void* A, const void* A_lo, int64_t row0, int64_t lda,
                                          int nrows, int K, const typename Stor<S>::C* Bs, int KS,
                                          typename Stor<S>::C* Os, int OS) {
  using C = typename Stor<S>::C;
  constexpr int V = Stor<S>::V;
  constexpr int T = TR * RC;
  constexpr int NV = (T >= 32) ? T / 32 : 1;
  constexpr int OWN = (T >= 32) ? 0 : (32 / T - 1);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int Q = K / V;
  for (int t0 = warp * TR; t0 < nrows; t0 += nw * TR) {
    C acc[T];
#pragma unroll
    for (int i = 0; i < T; ++i) acc[i] = C(0);
#pragma unroll 2
    for (int q = lane; q < Q; q += 32) {
      C a[TR][V];
#pragma unroll
      for (int t = 0; t < TR; ++t) {
        if (t0 + t < nrows) {
          load_vec<S>(A, A_lo, (row0 + t0 + t) * lda + static_cast<int64_t>(q) * V, a[t]);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) a[t][v] = C(0);
        }
      }
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        C b[V];
        load_b<C, V>(Bs + c * KS + q * V, b);
#pragma unroll
        for (int t = 0; t < TR; ++t) {
#pragma unroll
          for (int v = 0; v < V; ++v) acc[t * RC + c] = fma(a[t][v], b[v], acc[t * RC + c]);
        }
      }
    }
    rs_step<T, 16>(acc, lane);
    if ((lane & OWN) == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int f = rs_index<T>(lane, i);
        const int t = f / RC, c = f % RC;
        if (t0 + t < nrows) Os[c * OS + t0 + t] = acc[i];
      }
    }
  }
}

// HSS combine at internal node q (last arriver): couplings of the children
// (levels 1..p) and, below the root, the upsweep x-hat_q.
template <typename C>
__device__ void hss_combine(const MatView& mv, const Scratch& ws, int64_t r, int q, int col0,
                            int ncols, int rc, C* sm) {
  const int Kp = mv.Kp, Ke = mv.Ke;
  const int a = 2 * q + 1, b = 2 * q + 2;
  C* xa = sm;
  C* xb = sm + rc * Kp;
  const C* xh = static_cast<const C*>(ws.xh);
  for (int idx = threadIdx.x; idx < ncols * Kp; idx += blockDim.x) {
    const int c = idx / Kp, e = idx % Kp;
    xa[c * Kp + e] = __ldcg(xh + (static_cast<int64_t>(a) * r + col0 + c) * Kp + e);
    xb[c * Kp + e] = __ldcg(xh + (static_cast<int64_t>(b) * r + col0 + c) * Kp + e);
  }
  __syncthreads();
  const C* B12 = static_cast<const C*>(mv.B12) + static_cast<int64_t>(q) * Ke * Kp;
  const C* B21 = static_cast<const C*>(mv.B21) + static_cast<int64_t>(q) * Ke * Kp;
  C* yc = static_cast<C*>(ws.yc);
  for (int idx = threadIdx.x; idx < ncols * Ke; idx += blockDim.x) {
    const int c = idx / Ke, i = idx % Ke;
    C s12 = C(0), s21 = C(0);
    for (int j = 0; j < Kp; ++j) {
      s12 = fma(__ldg(B12 + i * Kp + j), xb[c * Kp + j], s12);
      s21 = fma(__ldg(B21 + i * Kp + j), xa[c * Kp + j], s21);
    }
    yc[(static_cast<int64_t>(a) * r + col0 + c) * Ke + i] = s12;
    yc[(static_cast<int64_t>(b) * r + col0 + c) * Ke + i] = s21;
  }
  if (q > 0) {
    const C* RVt = static_cast<const C*>(mv.RVt) + static_cast<int64_t>(q) * Kp * 2 * Kp;
    C* xw = static_cast<C*>(ws.xh);
    for (int idx = threadIdx.x; idx < ncols * Kp; idx += blockDim.x) {
      const int c = idx / Kp, i = idx % Kp;
      C s = C(0);
      for (int j = 0; j < Kp; ++j) s = fma(__ldg(RVt + i * 2 * Kp + j), xa[c * Kp + j], s);
      for (int j = 0; j < Kp; ++j) s = fma(__ldg(RVt + i * 2 * Kp + Kp + j), xb[c * Kp + j], s);
      xw[(static_cast<int64_t>(q) * r + col0 + c) * Kp + i] = s;
    }
  }
  __syncthreads();
}

// Tree climb after a leaf's projection has been written and fenced.
template <typename C>
__device__ void climb(const MatView& mv, const Scratch& ws, int64_t r, int node, int chunk,
                      int nchunks, int col0, int ncols, int rc, C* sm) {
  __shared__ int s_last;
  int child = node;
  while (child > 0) {
    const int q = (child - 1) >> 1;
    const int lq = 31 - __clz(q + 1);
    if (mv.kind == HM_HODLR && lq == 0) return;   // the root holds no partial sums
    __syncthreads();
    if (threadIdx.x == 0) {
      int* ctr = ws.cnt + static_cast<int64_t>(q) * nchunks + chunk;
      const int old = atomicAdd(ctr, 1);
      s_last = (old == 1);
      if (old == 1) atomicExch(ctr, 0);   // ready for the next product
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (mv.kind == HM_HODLR) {
      const int rows = mv.koff[lq + 1];   // levels 1..lq
      C* PS = static_cast<C*>(ws.PS);
      const int a = 2 * q + 1, b = 2 * q + 2;
      for (int idx = threadIdx.x; idx < rows * ncols; idx += blockDim.x) {
        const int c = idx / rows, e = idx % rows;
        const int64_t col = col0 + c;
        const C va = __ldcg(PS + (static_cast<int64_t>(a) * r + col) * mv.Ke + e);
        const C vb = __ldcg(PS + (static_cast<int64_t>(b) * r + col) * mv.Ke + e);
        PS[(static_cast<int64_t>(q) * r + col) * mv.Ke + e] = va + vb;
      }
    } else {
      hss_combine<C>(mv, ws, r, q, col0, ncols, rc, sm);
    }
    __threadfence();
    child = q;
  }
}

template <int S, int RC, int TR>
__global__ void __launch_bounds__(256) k_project(MatView mv, Scratch ws, int64_t r, const void* X,
                                                 int64_t ldx, int xt, int nchunks) {
  using C = typename Stor<S>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int leaf = blockIdx.x;
  const int chunk = blockIdx.y;
  const int col0 = chunk * RC;
  const int ncols = min(static_cast<int64_t>(RC), r - col0);
  const int64_t a0 = mv.off[leaf];
  const int m = static_cast<int>(mv.off[leaf + 1] - a0);
  const int K = mv.m_pad;
  const int Kp = mv.Kp;
  C* Bs = sm;
  C* Os = sm + RC * K;
  const int OS = Kp + 1;
  for (int idx = threadIdx.x; idx < RC * K; idx += blockDim.x) {
    const int c = idx / K, k = idx % K;
    C v = C(0);
    if (c < ncols && k < m) v = load_x<C>(X, xt, (a0 + k) + static_cast<int64_t>(col0 + c) * ldx);
    Bs[c * K + k] = v;
  }
  __syncthreads();
  if (m > 0) {
    rows_gemm<S, RC, TR>(mv.W, mv.W_lo, static_cast<int64_t>(leaf) * Kp, mv.m_pad, Kp, K, Bs, K, Os, OS);
  } else {
    for (int idx = threadIdx.x; idx < RC * OS; idx += blockDim.x) Os[idx] = C(0);
  }
  __syncthreads();
  const int node = mv.L - 1 + leaf;
  C* dst = static_cast<C*>(mv.kind == HM_HODLR ? ws.PS : ws.xh);
  const int ld = (mv.kind == HM_HODLR) ? mv.Ke : Kp;
  for (int idx = threadIdx.x; idx < ncols * Kp; idx += blockDim.x) {
    const int c = idx / Kp, e = idx % Kp;
    dst[(static_cast<int64_t>(node) * r + col0 + c) * ld + e] = Os[c * OS + e];
  }
  __threadfence();
  climb<C>(mv, ws, r, node, chunk, nchunks, col0, ncols, RC, sm);
}

template <typename C, int RC>
__global__ void __launch_bounds__(256) k_hss_down(MatView mv, Scratch ws, int64_t r, int s_lvl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ycur = reinterpret_cast<C*>(smem_raw);
  const int Ke = mv.Ke;
  C* ynext = ycur + RC * Ke;
  const int chunk = blockIdx.y;
  const int col0 = chunk * RC;
  const int ncols = min(static_cast<int64_t>(RC), r - col0);
  const int pos = blockIdx.x;
  const C* yc = static_cast<const C*>(ws.yc);
  C* yf = static_cast<C*>(ws.yf);
  const C* RU = static_cast<const C*>(mv.RU);
  // Chain of ancestors from level 1 down to the subtree root at level s_lvl.
  for (int l = 1; l <= s_lvl; ++l) {
    const int node = (1 << l) - 1 + (pos >> (s_lvl - l));
    if (l == 1) {
      for (int idx = threadIdx.x; idx < ncols * Ke; idx += blockDim.x) {
        const int c = idx / Ke, i = idx % Ke;
        ycur[c * Ke + i] = yc[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i];
      }
    } else {
      const int par = (node - 1) >> 1;
      const int half = (node & 1) ? 0 : 1;
      const C* R = RU + static_cast<int64_t>(par) * 2 * Ke * Ke + static_cast<int64_t>(half) * Ke * Ke;
      for (int idx = threadIdx.x; idx < ncols * Ke; idx += blockDim.x) {
        const int c = idx / Ke, i = idx % Ke;
        C s = yc[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i];
        for (int j = 0; j < Ke; ++j) s = fma(__ldg(R + i * Ke + j), ycur[c * Ke + j], s);
        ynext[c * Ke + i] = s;
      }
      __syncthreads();
      C* t = ycur; ycur = ynext; ynext = t;
    }
    __syncthreads();
  }
  {
    const int node = (1 << s_lvl) - 1 + pos;
    for (int idx = threadIdx.x; idx < ncols * Ke; idx += blockDim.x) {
      const int c = idx / Ke, i = idx % Ke;
      yf[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i] = ycur[c * Ke + i];
    }
  }
  __syncthreads();
  // The subtree below: every node owned by this block.
  for (int l = s_lvl + 1; l <= mv.p; ++l) {
    const int cnt = 1 << (l - s_lvl);
    const int first = (1 << l) - 1 + (pos << (l - s_lvl));
    const int work = cnt * ncols * Ke;
    for (int idx = threadIdx.x; idx < work; idx += blockDim.x) {
      const int nl = idx / (ncols * Ke);
      const int rem = idx % (ncols * Ke);
      const int c = rem / Ke, i = rem % Ke;
      const int node = first + nl;
      const int par = (node - 1) >> 1;
      const int half = (node & 1) ? 0 : 1;
      const C* R = RU + static_cast<int64_t>(par) * 2 * Ke * Ke + static_cast<int64_t>(half) * Ke * Ke;
      const C* yp = yf + (static_cast<int64_t>(par) * r + col0 + c) * Ke;
      C s = yc[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i];
      for (int j = 0; j < Ke; ++j) s = fma(__ldg(R + i * Ke + j), yp[j], s);
      yf[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i] = s;
    }
    __syncthreads();
  }
}

template <typename C>
__device__ __forceinline__ C z_value(const MatView& mv, const Scratch& ws, int64_t r, int leaf, int e,
                                     int64_t col) {
  if (mv.kind == HM_HSS) {
    if (mv.p == 0) return C(0);
    const int node = mv.L - 1 + leaf;
    return static_cast<const C*>(ws.yf)[(static_cast<int64_t>(node) * r + col) * mv.Ke + e];
  }
  for (int l = 1; l <= mv.p; ++l) {
    if (e < mv.koff[l] + mv.kk[l]) {
      const int anc = (1 << l) - 1 + (leaf >> (mv.p - l));
      const int sib = (anc & 1) ? anc + 1 : anc - 1;
      return static_cast<const C*>(ws.PS)[(static_cast<int64_t>(sib) * r + col) * mv.Ke + e];
    }
  }
  return C(0);
}

template <int S, int RC, int TR>
__global__ void __launch_bounds__(256) k_expand(MatView mv, Scratch ws, int64_t r, const void* X,
                                                int64_t ldx, int xt, void* Y, int64_t ldy, int yt,
                                                int RT, int tiles_per_leaf) {
  using C = typename Stor<S>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int leaf = blockIdx.x / tiles_per_leaf;
  const int tile = blockIdx.x % tiles_per_leaf;
  const int chunk = blockIdx.y;
  const int col0 = chunk * RC;
  const int ncols = min(static_cast<int64_t>(RC), r - col0);
  const int64_t a0 = mv.off[leaf];
  const int m = static_cast<int>(mv.off[leaf + 1] - a0);
  const int t0 = tile * RT;
  if (t0 >= m) return;
  const int nrows = min(RT, m - t0);
  const int K = mv.We;
  C* Bs = sm;
  C* Os = sm + RC * K;
  const int OS = RT + 1;
  for (int idx = threadIdx.x; idx < RC * K; idx += blockDim.x) {
    const int c = idx / K, k = idx % K;
    C v = C(0);
    if (c < ncols) {
      if (k < mv.m_pad) {
        if (k < m) v = load_x<C>(X, xt, (a0 + k) + static_cast<int64_t>(col0 + c) * ldx);
      } else {
        v = z_value<C>(mv, ws, r, leaf, k - mv.m_pad, col0 + c);
      }
    }
    Bs[c * K + k] = v;
  }
  __syncthreads();
  rows_gemm<S, RC, TR>(mv.A, mv.A_lo, a0 + t0, mv.We, nrows, K, Bs, K, Os, OS);
  __syncthreads();
  for (int idx = threadIdx.x; idx < ncols * nrows; idx += blockDim.x) {
    const int c = idx / nrows, t = idx % nrows;
    store_y<C>(Y, yt, (a0 + t0 + t) + static_cast<int64_t>(col0 + c) * ldy, Os[c * OS + t]);
  }
}

// ---------------------------------------------------------------------------
// Host-side launch for one storage type.
// ---------------------------------------------------------------------------

template <int S, int RC, int TR>
hm_status launch_rc(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx,
                    int xt, void* Y, int64_t ldy, int yt, cudaStream_t st) {
  using C = typename Stor<S>::C;
  const int nchunks = static_cast<int>((r + RC - 1) / RC);
  const size_t smem_p = sizeof(C) * static_cast<size_t>(
      max(RC * mv.m_pad + RC * (mv.Kp + 1), 2 * RC * mv.Kp));
  const int RT = 64;
  const int tiles = (mv.m_pad + RT - 1) / RT;
  const size_t smem_e = sizeof(C) * static_cast<size_t>(RC * mv.We + RC * (RT + 1));
  const size_t smem_d = sizeof(C) * static_cast<size_t>(2 * RC * mv.Ke);
  if (smem_p > 220 * 1024 || smem_e > 220 * 1024) return HM_EUNSUPPORTED;
  cudaFuncSetAttribute(k_project<S, RC, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem_p));
  cudaFuncSetAttribute(k_expand<S, RC, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem_e));
  k_project<S, RC, TR><<<dim3(mv.L, nchunks), 256, smem_p, st>>>(mv, ws, r, X, ldx, xt, nchunks);
  if (mv.kind == HM_HSS && mv.p >= 1) {
    const int s_lvl = max(1, mv.p - 3);
    cudaFuncSetAttribute(k_hss_down<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem_d));
    k_hss_down<C, RC><<<dim3(1u << s_lvl, nchunks), 256, smem_d, st>>>(mv, ws, r, s_lvl);
  }
  k_expand<S, RC, TR><<<dim3(mv.L * tiles, nchunks), 256, smem_e, st>>>(mv, ws, r, X, ldx, xt, Y, ldy,
                                                                       yt, RT, tiles);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("SIMT launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

template <int S>
hm_status launch_simt_t(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx,
                        int xt, void* Y, int64_t ldy, int yt, cudaStream_t st) {
  constexpr bool dbl = (S == HM_F64);
  // Column chunk: the smallest power of two >= r, at most 32; shrink while the
  // staged block would not fit in shared memory.
  int rc = 1;
  while (rc < r && rc < 32) rc *= 2;
  const size_t esz = dbl ? 8 : 4;
  while (rc > 1 && esz * static_cast<size_t>(rc) * (mv.We + 65) > 200 * 1024) rc /= 2;
  switch (rc) {
    case 1: return launch_rc<S, 1, 4>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st);
    case 2: return launch_rc<S, 2, 4>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st);
    case 4: return launch_rc<S, 4, 4>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st);
    case 8: return launch_rc<S, 8, 4>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st);
    case 16: return launch_rc<S, 16, (dbl ? 2 : 4)>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st);
    default: return launch_rc<S, 32, (dbl ? 1 : 2)>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st);
  }
}

}  // namespace hmi

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

#include <algorithm>
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

// 16-byte loads: read-only data (generators) and data other blocks of the same
// kernel wrote (bypassing L1).
__device__ __forceinline__ uint4 ld16_ro(const void* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
__device__ __forceinline__ uint4 ld16_cg(const void* p) { return __ldcg(reinterpret_cast<const uint4*>(p)); }

// Block-wide gather of `nunits` 16-byte units into shared memory with
// 8 loads in flight per thread: `map(i, src, dst)` gives the global source and
// shared destination of unit i (both 16-byte aligned) and whether it is read
// with ld.global.cg (true) or through the read-only path (false).
template <typename F>
__device__ __forceinline__ void gather16(int nunits, F&& map) {
  constexpr int U = 8;
  for (int b0 = threadIdx.x; b0 < nunits; b0 += blockDim.x * U) {
    uint4 v[U];
    uint4* dst[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = b0 + u * blockDim.x;
      dst[u] = nullptr;
      if (i < nunits) {
        const void* src;
        bool cg = map(i, src, dst[u]);
        v[u] = cg ? ld16_cg(src) : ld16_ro(src);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (dst[u]) *dst[u] = v[u];
  }
}

template <typename C>
__device__ __forceinline__ C cvt_in(double v) { return static_cast<C>(v); }
template <typename C>
__device__ __forceinline__ C cvt_in(float v) { return static_cast<C>(v); }
template <typename C>
__device__ __forceinline__ C cvt_in(uint16_t v) {
  return static_cast<C>(__uint_as_float(static_cast<uint32_t>(v) << 16));
}

// Bs[c * ldb + k] = X(a0 + k, col0 + c) for k < m, c < ncols; zero elsewhere
// (k < rows_pad, c < rc; rows_pad a multiple of 4).  Groups of 4 rows are read
// with one vector load when they are aligned and inside the leaf, and each
// thread keeps 8 groups in flight before its stores.
template <typename T, typename C>
__device__ __forceinline__ void stage_x_t(C* Bs, int ldb, const T* X, int64_t ldx, int64_t a0, int m, int rows_pad,
                                          int col0, int ncols, int rc) {
  const int kg = rows_pad >> 2;
  const int items = rc * kg;
  constexpr int U = 8;
  for (int base = threadIdx.x; base < items; base += blockDim.x * U) {
    C v[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = base + u * blockDim.x;
      const int c = it / kg, k0 = (it % kg) * 4;
      const bool ok = it < items && c < ncols;
      const T* p = X + (a0 + k0) + static_cast<int64_t>(col0 + c) * ldx;
      const bool vec = ok && k0 + 4 <= m && (reinterpret_cast<uintptr_t>(p) % (4 * sizeof(T))) == 0;
      if (vec) {
        if constexpr (sizeof(T) == 8) {
          const double2 x0 = *reinterpret_cast<const double2*>(p);
          const double2 x1 = *reinterpret_cast<const double2*>(p + 2);
          v[u][0] = static_cast<C>(x0.x); v[u][1] = static_cast<C>(x0.y);
          v[u][2] = static_cast<C>(x1.x); v[u][3] = static_cast<C>(x1.y);
        } else if constexpr (sizeof(T) == 4) {
          const float4 x = *reinterpret_cast<const float4*>(p);
          v[u][0] = static_cast<C>(x.x); v[u][1] = static_cast<C>(x.y);
          v[u][2] = static_cast<C>(x.z); v[u][3] = static_cast<C>(x.w);
        } else {
          const uint2 x = *reinterpret_cast<const uint2*>(p);
          v[u][0] = static_cast<C>(__uint_as_float(x.x << 16));
          v[u][1] = static_cast<C>(__uint_as_float(x.x & 0xffff0000u));
          v[u][2] = static_cast<C>(__uint_as_float(x.y << 16));
          v[u][3] = static_cast<C>(__uint_as_float(x.y & 0xffff0000u));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[u][j] = (ok && k0 + j < m) ? cvt_in<C>(p[j]) : C(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = base + u * blockDim.x;
      if (it < items) {
        const int c = it / kg, k0 = (it % kg) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) Bs[c * ldb + k0 + j] = v[u][j];
      }
    }
  }
}

template <typename C>
__device__ __forceinline__ void stage_x(C* Bs, int ldb, const void* X, int xt, int64_t ldx, int64_t a0, int m,
                                        int rows_pad, int col0, int ncols, int rc) {
  if (xt == HM_F64)
    stage_x_t<double, C>(Bs, ldb, static_cast<const double*>(X), ldx, a0, m, rows_pad, col0, ncols, rc);
  else if (xt == HM_F32)
    stage_x_t<float, C>(Bs, ldb, static_cast<const float*>(X), ldx, a0, m, rows_pad, col0, ncols, rc);
  else
    stage_x_t<uint16_t, C>(Bs, ldb, static_cast<const uint16_t*>(X), ldx, a0, m, rows_pad, col0, ncols, rc);
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

// The V values of one raw 16-byte vector of a generator plane (hi plane, and
// for BF16X2 the lo plane: hi + lo is exact in float, at most 17 bits).
template <int S>
__device__ __forceinline__ void unpack_vec(const uint4& u, const uint4& w, typename Stor<S>::C* a) {
  if constexpr (S == HM_F64) {
    a[0] = __hiloint2double(static_cast<int>(u.y), static_cast<int>(u.x));
    a[1] = __hiloint2double(static_cast<int>(u.w), static_cast<int>(u.z));
  } else if constexpr (S == HM_F32) {
    a[0] = __uint_as_float(u.x); a[1] = __uint_as_float(u.y);
    a[2] = __uint_as_float(u.z); a[3] = __uint_as_float(u.w);
  } else {
    a[0] = bf_lo(u.x); a[1] = bf_hi(u.x); a[2] = bf_lo(u.y); a[3] = bf_hi(u.y);
    a[4] = bf_lo(u.z); a[5] = bf_hi(u.z); a[6] = bf_lo(u.w); a[7] = bf_hi(u.w);
    if constexpr (S == HM_BF16X2) {
      a[0] += bf_lo(w.x); a[1] += bf_hi(w.x); a[2] += bf_lo(w.y); a[3] += bf_hi(w.y);
      a[4] += bf_lo(w.z); a[5] += bf_hi(w.z); a[6] += bf_lo(w.w); a[7] += bf_hi(w.w);
    }
  }
}

// Os[c * OS + t] = sum_k A(row0 + t, k) * Bs[c * KS + k] for t < nrows, c < RC.
// A: row-major plane(s) with leading dimension lda (elements), K a multiple of V.
// Lane l sums the 16-byte vectors q = l, l + 32, ... of each of its warp's TR
// rows in increasing q, then a butterfly over the lanes completes each sum;
// the order does not depend on TR or UQ, so every shape gives the same bits.
// All loads of UQ q steps of the TR rows are issued (as raw vectors) before
// the multiplies, so a narrow right-hand side keeps UQ TR loads in flight per
// lane.
template <int S, int RC, int TR, int UQ = 2>
__device__ __forceinline__ void rows_gemm(const void* A, const void* A_lo, int64_t row0, int64_t lda,
                                          int nrows, int K, const typename Stor<S>::C* Bs, int KS,
                                          typename Stor<S>::C* Os, int OS) {
  using C = typename Stor<S>::C;
  constexpr int V = Stor<S>::V;
  constexpr int T = TR * RC;
  constexpr int NV = (T >= 32) ? T / 32 : 1;
  constexpr int OWN = (T >= 32) ? 0 : (32 / T - 1);
  constexpr int ES = (S == HM_F64) ? 8 : (S == HM_F32) ? 4 : 2;   // bytes per element of a plane
  constexpr bool LO = (S == HM_BF16X2);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int Q = K / V;
  const unsigned char* Ab = static_cast<const unsigned char*>(A);
  const unsigned char* Lb = static_cast<const unsigned char*>(A_lo);
  for (int t0 = warp * TR; t0 < nrows; t0 += nw * TR) {
    C acc[T];
#pragma unroll
    for (int i = 0; i < T; ++i) acc[i] = C(0);
    for (int q0 = lane; q0 < Q; q0 += 32 * UQ) {
      uint4 ra[UQ][TR], rl[UQ][TR];
#pragma unroll
      for (int u = 0; u < UQ; ++u) {
        const int q = q0 + 32 * u;
#pragma unroll
        for (int t = 0; t < TR; ++t) {
          ra[u][t] = make_uint4(0u, 0u, 0u, 0u);
          rl[u][t] = make_uint4(0u, 0u, 0u, 0u);
          if (q < Q && t0 + t < nrows) {
            const int64_t off = ((row0 + t0 + t) * lda + static_cast<int64_t>(q) * V) * ES;
            ra[u][t] = ld_stream16(Ab + off);
            if constexpr (LO) rl[u][t] = ld_stream16(Lb + off);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UQ; ++u) {
        const int q = q0 + 32 * u;
        if (q >= Q) break;
#pragma unroll
        for (int c = 0; c < RC; ++c) {
          C b[V];
          load_b<C, V>(Bs + c * KS + q * V, b);
#pragma unroll
          for (int t = 0; t < TR; ++t) {
            C a[V];
            unpack_vec<S>(ra[u][t], rl[u][t], a);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[t * RC + c] = fma(a[v], b[v], acc[t * RC + c]);
          }
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

// Programmatic dependent launch: let the next kernel of the product start its
// independent work early, and wait for the previous kernel's results.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// out(c, i) = sum_{j < Kj} Mt[j * Ko + i] * v[c * ldv + j] for i < Ko, c < nc.
// Mt and v are in shared memory; a thread owns one i and CT columns, so the
// Mt reads of a warp are consecutive and the v reads are broadcasts.
template <typename C, int CT, typename F>
__device__ __forceinline__ void cta_gemm(const C* Mt, int Kj, int Ko, const C* v, int ldv, int nc,
                                         F&& out) {
  const int ngrp = (nc + CT - 1) / CT;
  for (int w = threadIdx.x; w < Ko * ngrp; w += blockDim.x) {
    const int i = w % Ko;
    const int c0 = (w / Ko) * CT;
    C acc[CT];
    const C* vp[CT];
#pragma unroll
    for (int t = 0; t < CT; ++t) {
      acc[t] = C(0);
      vp[t] = v + min(c0 + t, nc - 1) * ldv;
    }
#pragma unroll 4
    for (int j = 0; j < Kj; ++j) {
      const C m = Mt[j * Ko + i];
#pragma unroll
      for (int t = 0; t < CT; ++t) acc[t] = fma(m, vp[t][j], acc[t]);
    }
#pragma unroll
    for (int t = 0; t < CT; ++t)
      if (c0 + t < nc) out(c0 + t, i, acc[t]);
  }
}

// Block-wide copies into shared memory with 4 loads in flight per thread.
// stage_ro reads data that is constant for the kernel (generators); stage_cg
// reads data written by other blocks of the same kernel (L2, not L1).
// dst[i * ldd + j] = src[i * lds + j] for i < rows, j < cols.
template <typename C, bool CG>
__device__ __forceinline__ void stage2d(C* __restrict__ dst, int ldd, const C* __restrict__ src, int64_t lds,
                                        int rows, int cols) {
  constexpr int U = 4;
  const int count = rows * cols;
  for (int base = threadIdx.x; base < count; base += blockDim.x * U) {
    C v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * blockDim.x;
      const int rr = i / cols, cc = i % cols;
      if (i < count) v[u] = CG ? __ldcg(src + rr * lds + cc) : __ldg(src + rr * lds + cc);
      else v[u] = C(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * blockDim.x;
      if (i < count) dst[(i / cols) * ldd + (i % cols)] = v[u];
    }
  }
}

template <typename C>
__device__ __forceinline__ void stage_ro(C* dst, const C* src, int count) {
  stage2d<C, false>(dst, count, src, count, 1, count);
}

// ---------------------------------------------------------------------------
// Tree-up kernel: the upsweep of Fig. 4.1 (HSS: x-hat_q = R_V^T [x-hat_a; x-hat_b]
// and the couplings y_a = B12 x-hat_b, y_b = B21 x-hat_a on levels 1..p; HODLR:
// the per-level sums of the leaves' V^T X, T_q = T_a + T_b).
//
// Work proceeds in steps of up to g levels.  A block owns a group of 2^s nodes
// at level lc under one ancestor at level lt = lc - s; it stages the group's
// data and every operator the step needs in one batched pass, then combines
// the s levels in shared memory.  The first step of a block covers its own
// leaves; later steps are taken by the last of the 2^s arriving blocks (an
// atomic counter per ancestor and column chunk), so no block ever waits.
// Combines always add left before right: the result does not depend on
// arrival order.
// ---------------------------------------------------------------------------

// Shared-memory elements of one step of span s (K rows per node, rc columns).
__host__ __device__ inline int up_smem_elems(bool hss, int rc, int Kp, int Ke, int s) {
  const int K = hss ? Kp : Ke;
  const int nin = 1 << s;
  const int bufs = (nin + (nin > 2 ? nin / 2 : 1)) * rc * K;
  const int ops = hss ? (nin - 1) * (2 * Kp * Ke + 2 * Kp * Kp) : 0;
  return bufs + ops;
}

template <typename C, int RC>
__device__ void tree_up_block(const MatView& mv, const Scratch& ws, int64_t r, int g, int nchunks, int bx,
                              int chunk, C* sm) {
  __shared__ int s_last;
  const bool hss = (mv.kind == HM_HSS);
  const int Kp = mv.Kp, Ke = mv.Ke;
  const int K = hss ? Kp : Ke;
  const int col0 = chunk * RC;
  const int ncols = min(static_cast<int64_t>(RC), r - col0);
  const int lmin = hss ? 0 : 1;
  const int opsz = 2 * Kp * Ke + 2 * Kp * Kp;
  C* data = static_cast<C*>(hss ? ws.xh : ws.PS);
  C* yc = static_cast<C*>(ws.yc);
  int lc = mv.p;
  int pos = bx << min(g, mv.p - lmin);
  bool first = true;
  pdl_wait();   // the leaves' projections come from the projection kernel
  while (lc > lmin) {
    const int lt = max(lc - g, lmin);
    const int s = lc - lt;
    const int post = pos >> s;
    if (!first) {
      const int anc = (1 << lt) - 1 + post;
      __syncthreads();
      if (threadIdx.x == 0) {
        int* ctr = ws.cnt + static_cast<int64_t>(anc) * nchunks + chunk;
        const int old = atomicAdd(ctr, 1);
        s_last = (old == (1 << s) - 1);
        if (s_last) atomicExch(ctr, 0);   // ready for the next product
      }
      __syncthreads();
      if (!s_last) return;
      __threadfence();
    }
    const int nin = 1 << s;
    const int base_pos = post << s;
    C* bufA = sm;                                       // nin/2 pairs of [c][2K]
    C* bufB = bufA + nin * RC * K;
    C* ops = bufB + (nin > 2 ? nin / 2 : 1) * RC * K;
    // One batched gather of 16-byte units: the group's inputs (L2, written by
    // other blocks) and, for HSS, the operators B12, B21, R_V of its internal
    // nodes (read-only).
    {
      constexpr int E = 16 / sizeof(C);               // elements per unit
      const int uK = K / E;                           // units per column of one node
      const int n_in = nin * ncols * uK;
      const int uKK = Kp * Ke / E, uRV = 2 * Kp * Kp / E;
      const int uop = 2 * uKK + uRV;
      const int n_ops = hss ? (nin - 1) * uop : 0;
      C* ops_base = ops;
      gather16(n_in + n_ops, [&](int i, const void*& src, uint4*& dst) -> bool {
        if (i < n_in) {
          const int j = i / (ncols * uK);
          const int rem = i % (ncols * uK);
          const int c = rem / uK, e = (rem % uK) * E;
          const int node = (1 << lc) - 1 + base_pos + j;
          src = data + (static_cast<int64_t>(node) * r + col0 + c) * K + e;
          dst = reinterpret_cast<uint4*>(bufA + (j >> 1) * RC * 2 * K + c * 2 * K + (j & 1) * K + e);
          return true;
        }
        const int o = (i - n_in) / uop;
        const int e = (i - n_in) % uop;
        int lev = lt, t = o;                          // op o: level order inside the group
        while (t >= (1 << (lev - lt))) { t -= 1 << (lev - lt); ++lev; }
        const int q = (1 << lev) - 1 + (post << (lev - lt)) + t;
        dst = reinterpret_cast<uint4*>(ops_base + static_cast<int64_t>(o) * opsz) + e;
        if (e < uKK) src = static_cast<const C*>(mv.B12) + static_cast<int64_t>(q) * Kp * Ke + e * E;
        else if (e < 2 * uKK) src = static_cast<const C*>(mv.B21) + static_cast<int64_t>(q) * Kp * Ke + (e - uKK) * E;
        else src = static_cast<const C*>(mv.RV) + static_cast<int64_t>(q) * 2 * Kp * Kp + (e - 2 * uKK) * E;
        return false;
      });
    }
    __syncthreads();
    C* cur = bufA;
    C* nxt = bufB;
    for (int lev = lc - 1; lev >= lt; --lev) {
      const int nn = 1 << (lev - lt);
      for (int t = 0; t < nn; ++t) {
        const int q = (1 << lev) - 1 + (post << (lev - lt)) + t;
        const int a = 2 * q + 1, b = 2 * q + 2;
        const C* pr = cur + t * RC * 2 * K;
        C* outp = nxt + (t >> 1) * RC * 2 * K + (t & 1) * K;
        const bool top = (lev == lt);
        if (hss) {
          const C* op = ops + ((nn - 1) + t) * opsz;
          cta_gemm<C, 2>(op, Kp, Ke, pr + Kp, 2 * Kp, ncols, [&](int c, int i, C v) {
            yc[(static_cast<int64_t>(a) * r + col0 + c) * Ke + i] = v;
          });
          cta_gemm<C, 2>(op + Kp * Ke, Kp, Ke, pr, 2 * Kp, ncols, [&](int c, int i, C v) {
            yc[(static_cast<int64_t>(b) * r + col0 + c) * Ke + i] = v;
          });
          if (lev > 0) {
            cta_gemm<C, 2>(op + 2 * Kp * Ke, 2 * Kp, Kp, pr, 2 * Kp, ncols, [&](int c, int i, C v) {
              if (top) data[(static_cast<int64_t>(q) * r + col0 + c) * Kp + i] = v;
              else outp[c * 2 * K + i] = v;
            });
          }
        } else {
          const int rows = mv.koff[lev + 1];        // levels 1..lev
          for (int idx = threadIdx.x; idx < ncols * rows; idx += blockDim.x) {
            const int c = idx / rows, e = idx % rows;
            const C v = pr[c * 2 * K + e] + pr[c * 2 * K + K + e];
            data[(static_cast<int64_t>(q) * r + col0 + c) * Ke + e] = v;
            if (!top) outp[c * 2 * K + e] = v;
          }
        }
      }
      __syncthreads();
      C* tmp = cur; cur = nxt; nxt = tmp;
    }
    __threadfence();
    first = false;
    lc = lt;
    pos = post;
  }
}

template <typename C, int RC>
__global__ void __launch_bounds__(256) k_tree_up(MatView mv, Scratch ws, int64_t r, int g, int nchunks) {
  pdl_launch_dependents();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tree_up_block<C, RC>(mv, ws, r, g, nchunks, blockIdx.x, blockIdx.y, reinterpret_cast<C*>(smem_raw));
}

template <int S, int RC, int TR>
__device__ void project_block(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx, int xt,
                              int leaf, int chunk, typename Stor<S>::C* sm) {
  using C = typename Stor<S>::C;
  const int col0 = chunk * RC;
  const int ncols = min(static_cast<int64_t>(RC), r - col0);
  const int64_t a0 = mv.off[leaf];
  const int m = static_cast<int>(mv.off[leaf + 1] - a0);
  const int K = mv.m_pad;
  const int Kp = mv.Kp;
  C* Bs = sm;
  C* Os = sm + RC * K;
  const int OS = Kp + 1;
  stage_x<C>(Bs, K, X, xt, ldx, a0, m, K, col0, ncols, RC);
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
}

template <int S, int RC, int TR>
__global__ void __launch_bounds__(256, 2) k_project(MatView mv, Scratch ws, int64_t r, const void* X,
                                                 int64_t ldx, int xt, int nchunks) {
  using C = typename Stor<S>::C;
  pdl_launch_dependents();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  (void)nchunks;
  project_block<S, RC, TR>(mv, ws, r, X, ldx, xt, blockIdx.x, blockIdx.y, reinterpret_cast<C*>(smem_raw));
}

// Shared-memory elements of the downsweep: the subtree part needs, per level
// of a depth-d subtree, 2^d operator halves and two y buffers of 2^d nodes;
// the chain part prefetches G levels (operator half + coupling block) at once.
__host__ __device__ inline int down_smem_elems(int rc, int Ke, int d, int G) {
  const int sub = (1 << d) * Ke * Ke + 2 * (1 << d) * rc * Ke;
  const int chain = G * (Ke * Ke + rc * Ke) + 2 * rc * Ke;
  return sub > chain ? sub : chain;
}

template <typename C, int RC>
__device__ void down_block(const MatView& mv, const Scratch& ws, int64_t r, int s_lvl, int G, int pos, int chunk,
                           unsigned char* smem_raw) {
  const int Ke = mv.Ke;
  const int d = mv.p - s_lvl;               // subtree depth
  const int col0 = chunk * RC;
  const int ncols = min(static_cast<int64_t>(RC), r - col0);
  const C* RU = static_cast<const C*>(mv.RU);
  pdl_wait();                               // couplings come from the projection kernel
  const C* yc = static_cast<const C*>(ws.yc);
  C* yf = static_cast<C*>(ws.yf);
  // ---- chain of ancestors, level 1 .. s_lvl, G levels per prefetch ----
  C* ycur = reinterpret_cast<C*>(smem_raw);
  C* ynext = ycur + RC * Ke;
  C* Mg = ynext + RC * Ke;                  // G operator halves
  C* Yg = Mg + G * Ke * Ke;                 // G coupling blocks
  {
    const int node = 1 + (pos >> (s_lvl - 1));
    stage2d<C, false>(ycur, Ke, yc + (static_cast<int64_t>(node) * r + col0) * Ke, Ke, ncols, Ke);
    __syncthreads();
  }
  constexpr int E = 16 / sizeof(C);
  const int uM = Ke * Ke / E, uY = ncols * Ke / E;
  for (int l = 2; l <= s_lvl; l += G) {
    const int gn = min(G, s_lvl - l + 1);
    // one gather: the operator halves and coupling blocks of gn levels
    gather16(gn * (uM + uY), [&](int i, const void*& src, uint4*& dst) -> bool {
      const int g = i / (uM + uY);
      const int e = i % (uM + uY);
      const int node = (1 << (l + g)) - 1 + (pos >> (s_lvl - l - g));
      if (e < uM) {
        const int par = (node - 1) >> 1;
        const int half = (node & 1) ? 0 : 1;
        src = RU + (static_cast<int64_t>(par) * 2 + half) * Ke * Ke + e * E;
        dst = reinterpret_cast<uint4*>(Mg + g * Ke * Ke) + e;
      } else {
        src = yc + (static_cast<int64_t>(node) * r + col0) * Ke + (e - uM) * E;
        dst = reinterpret_cast<uint4*>(Yg + g * RC * Ke) + (e - uM);
      }
      return false;
    });
    __syncthreads();
    for (int g = 0; g < gn; ++g) {
      const C* Yb = Yg + g * RC * Ke;
      cta_gemm<C, 4>(Mg + g * Ke * Ke, Ke, Ke, ycur, Ke, ncols, [&](int c, int i, C v) {
        ynext[c * Ke + i] = v + Yb[c * Ke + i];
      });
      __syncthreads();
      C* t = ycur; ycur = ynext; ynext = t;
    }
  }
  if (s_lvl == mv.p) {
    const int node = (1 << s_lvl) - 1 + pos;
    for (int idx = threadIdx.x; idx < ncols * Ke; idx += blockDim.x) {
      const int c = idx / Ke, i = idx % Ke;
      yf[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i] = ycur[c * Ke + i];
    }
    return;
  }
  // ---- the subtree below, one level at a time ----
  C* Ms = reinterpret_cast<C*>(smem_raw);   // 2^d operator halves
  C* sub0 = Ms + (1 << d) * Ke * Ke;        // two buffers of 2^d nodes x RC x Ke
  C* sub1 = sub0 + (1 << d) * RC * Ke;
  // the subtree root's y moves to the subtree buffers (regions may overlap: go through registers)
  {
    C v[8];
    const int cnt = ncols * Ke;
    for (int base = 0; base < cnt; base += 8 * blockDim.x) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = base + u * blockDim.x + threadIdx.x;
        v[u] = (i < cnt) ? ycur[(i / Ke) * Ke + (i % Ke)] : C(0);
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = base + u * blockDim.x + threadIdx.x;
        if (i < cnt) sub0[i] = v[u];
      }
      __syncthreads();
    }
  }
  C* ysub = sub0;
  C* ynsub = sub1;
  for (int l = s_lvl + 1; l <= mv.p; ++l) {
    const int cnt = 1 << (l - s_lvl);
    const int first = (1 << l) - 1 + (pos << (l - s_lvl));
    {
      const int uM = Ke * Ke / (16 / static_cast<int>(sizeof(C)));
      gather16(cnt * uM, [&](int i, const void*& src, uint4*& dst) -> bool {
        const int k = i / uM, e = i % uM;
        const int node = first + k;
        const int par = (node - 1) >> 1;
        const int half = (node & 1) ? 0 : 1;
        src = reinterpret_cast<const uint4*>(RU + (static_cast<int64_t>(par) * 2 + half) * Ke * Ke) + e;
        dst = reinterpret_cast<uint4*>(Ms + k * Ke * Ke) + e;
        return false;
      });
    }
    __syncthreads();
    const int ngrp = (ncols + 3) / 4;
    const int work = cnt * Ke * ngrp;
    for (int w = threadIdx.x; w < work; w += blockDim.x) {
      const int k = w / (Ke * ngrp);
      const int rem = w % (Ke * ngrp);
      const int i = rem % Ke;
      const int c0 = (rem / Ke) * 4;
      const int node = first + k;
      const C* Mt = Ms + k * Ke * Ke;
      const C* yp = ysub + (k >> 1) * RC * Ke;
      C acc[4];
      C base[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[t] = C(0);
        const int c = min(c0 + t, ncols - 1);
        base[t] = yc[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i];
      }
#pragma unroll 4
      for (int j = 0; j < Ke; ++j) {
        const C m = Mt[j * Ke + i];
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[t] = fma(m, yp[min(c0 + t, ncols - 1) * Ke + j], acc[t]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = c0 + t;
        if (c >= ncols) continue;
        const C v = acc[t] + base[t];
        ynsub[(k * RC + c) * Ke + i] = v;
        if (l == mv.p) yf[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i] = v;
      }
    }
    __syncthreads();
    C* t = ysub; ysub = ynsub; ynsub = t;
  }
}

template <typename C, int RC>
__global__ void __launch_bounds__(256) k_hss_down(MatView mv, Scratch ws, int64_t r, int s_lvl, int G) {
  pdl_launch_dependents();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  down_block<C, RC>(mv, ws, r, s_lvl, G, blockIdx.x, blockIdx.y, smem_raw);
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

template <int S, int RC, int TR, int UQ = 2>
__device__ void expand_block(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx, int xt,
                             void* Y, int64_t ldy, int yt, int RT, int leaf, int tile, int chunk,
                             typename Stor<S>::C* sm) {
  using C = typename Stor<S>::C;
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
  const int mp = mv.m_pad;
  stage_x<C>(Bs, K, X, xt, ldx, a0, m, mp, col0, ncols, RC);
  pdl_wait();   // Z comes from the projection / downsweep kernels
  const int Ke = mv.Ke;
  for (int idx = threadIdx.x; idx < RC * Ke; idx += blockDim.x) {
    const int c = idx / Ke, e = idx % Ke;
    Bs[c * K + mp + e] = (c < ncols) ? z_value<C>(mv, ws, r, leaf, e, col0 + c) : C(0);
  }
  __syncthreads();
  rows_gemm<S, RC, TR, UQ>(mv.A, mv.A_lo, a0 + t0, mv.We, nrows, K, Bs, K, Os, OS);
  __syncthreads();
  for (int idx = threadIdx.x; idx < ncols * nrows; idx += blockDim.x) {
    const int c = idx / nrows, t = idx % nrows;
    store_y<C>(Y, yt, (a0 + t0 + t) + static_cast<int64_t>(col0 + c) * ldy, Os[c * OS + t]);
  }
}

template <int S, int RC, int TR, int UQ = 2>
__global__ void __launch_bounds__(256) k_expand(MatView mv, Scratch ws, int64_t r, const void* X,
                                                int64_t ldx, int xt, void* Y, int64_t ldy, int yt,
                                                int RT, int tiles_per_leaf) {
  using C = typename Stor<S>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  expand_block<S, RC, TR, UQ>(mv, ws, r, X, ldx, xt, Y, ldy, yt, RT, blockIdx.x / tiles_per_leaf,
                          blockIdx.x % tiles_per_leaf, blockIdx.y, reinterpret_cast<C*>(smem_raw));
}

// ---------------------------------------------------------------------------
// Host-side launches, one phase at a time (0 project, 1 HSS downsweep, 2 expand).
// Phases 1 and 2 are launched with programmatic stream serialization so that
// they start while the previous phase drains and wait (griddepcontrol.wait)
// only where they read its results.
// ---------------------------------------------------------------------------

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

inline int pick_rc(int64_t r, size_t esz, int width) {
  int rc = 1;
  while (rc < r && rc < 32) rc *= 2;
  while (rc > 1 && esz * static_cast<size_t>(rc) * (width + 65) > 200 * 1024) rc /= 2;
  return rc;
}

// Subtree depth of the downsweep: 2^d operator halves must fit in ~64 KB.
inline int down_depth(const MatView& mv, size_t esz) {
  int d = 3;
  while (d > 0 && (size_t(1) << d) * mv.Ke * mv.Ke * esz > 64 * 1024) --d;
  return std::min(d, mv.p - 1);
}

template <int S, int RC, int TR, int UQ = 2>
hm_status launch_phase_rc(int phase, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                          int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  using C = typename Stor<S>::C;
  const int nchunks = static_cast<int>((r + RC - 1) / RC);
  Scratch wk = ws;
  wk.prof = nullptr;   // kernels never see the host hook
  cudaError_t e = cudaSuccess;
  if (phase == 0) {
    const size_t smem = sizeof(C) * static_cast<size_t>(RC * mv.m_pad + RC * (mv.Kp + 1));
    if (smem > 220 * 1024) return HM_EUNSUPPORTED;
    cudaFuncSetAttribute(k_project<S, RC, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    prof_mark(ws.prof, 0, true, st);
    e = launch_k(k_project<S, RC, TR>, dim3(mv.L, nchunks), dim3(256), smem, st, pdl, mv, wk, r, X, ldx, xt,
                 nchunks);
    prof_mark(ws.prof, 0, false, st);
  } else {
    // rows per block: a whole leaf (up to 256 rows) when that still gives
    // several blocks per SM, so a block's fixed work (staging X and Z,
    // barriers) is spread over more streamed rows (smaller tiles that fill
    // the last wave better measured slower); the row sums do not depend on it
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int RT = 64;
    while (RT < 256 && RT < mv.m_pad &&
           static_cast<int64_t>(mv.L) * ((mv.m_pad + 2 * RT - 1) / (2 * RT)) * nchunks >= 4 * sms)
      RT *= 2;
    const int tiles = (mv.m_pad + RT - 1) / RT;
    const size_t smem = sizeof(C) * static_cast<size_t>(RC * mv.We + RC * (RT + 1));
    if (smem > 220 * 1024) return HM_EUNSUPPORTED;
    cudaFuncSetAttribute(k_expand<S, RC, TR, UQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    prof_mark(ws.prof, 3, true, st);
    e = launch_k(k_expand<S, RC, TR, UQ>, dim3(mv.L * tiles, nchunks), dim3(256), smem, st, pdl, mv, wk, r, X, ldx,
                 xt, Y, ldy, yt, RT, tiles);
    prof_mark(ws.prof, 3, false, st);
  }
  if (e != cudaSuccess) {
    set_error("SIMT launch (phase %d) failed: %s", phase, cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

// Tree kernels (phase 1 upsweep / sums, phase 2 HSS downsweep) with RC columns per block.
template <typename C, int RC>
hm_status launch_tree_rc(int phase, const MatView& mv, const Scratch& ws, int64_t r, cudaStream_t st, bool pdl) {
  const int nchunks = static_cast<int>((r + RC - 1) / RC);
  Scratch wk = ws;
  wk.prof = nullptr;
  cudaError_t e = cudaSuccess;
  const bool hss = (mv.kind == HM_HSS);
  if (phase == 1) {
    const int lmin = hss ? 0 : 1;
    if (mv.p <= lmin) return HM_OK;
    int g = 3;
    while (g > 1 && sizeof(C) * static_cast<size_t>(up_smem_elems(hss, RC, mv.Kp, mv.Ke, g)) > 100 * 1024) --g;
    const int s0 = std::min(g, mv.p - lmin);
    const size_t smem = sizeof(C) * static_cast<size_t>(up_smem_elems(hss, RC, mv.Kp, mv.Ke, std::min(g, mv.p)));
    if (smem > 220 * 1024) return HM_EUNSUPPORTED;
    cudaFuncSetAttribute(k_tree_up<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    prof_mark(ws.prof, 1, true, st);
    e = launch_k(k_tree_up<C, RC>, dim3(mv.L >> s0, nchunks), dim3(256), smem, st, pdl, mv, wk, r, g, nchunks);
    prof_mark(ws.prof, 1, false, st);
  } else {
    if (!hss || mv.p < 1) return HM_OK;
    const int d = down_depth(mv, sizeof(C));
    const int s_lvl = mv.p - d;
    // chain levels prefetched together: as many as fit in ~96 KB
    const int per = mv.Ke * mv.Ke + RC * mv.Ke;
    const int G = std::max(1, std::min(std::max(s_lvl - 1, 1),
                                       static_cast<int>((96 * 1024 / sizeof(C)) / std::max(per, 1))));
    const size_t smem = sizeof(C) * static_cast<size_t>(down_smem_elems(RC, mv.Ke, d, G));
    if (smem > 220 * 1024) return HM_EUNSUPPORTED;
    cudaFuncSetAttribute(k_hss_down<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    prof_mark(ws.prof, 2, true, st);
    e = launch_k(k_hss_down<C, RC>, dim3(1u << s_lvl, nchunks), dim3(256), smem, st, pdl, mv, wk, r, s_lvl, G);
    prof_mark(ws.prof, 2, false, st);
  }
  if (e != cudaSuccess) {
    set_error("tree launch (phase %d) failed: %s", phase, cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

// Leaf expansion for one or two columns with the plane streamed by bulk
// copies (k_ring.cuh; instantiated by the per-storage units).
template <int S, int RC, int TR>
hm_status launch_expand_ring(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx, int xt,
                             void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl);

// Phases: 0 projection, 1 tree upsweep / sums, 2 HSS downsweep, 3 leaf expansion.
template <int S>
hm_status simt_phase_t(int phase, const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx,
                       int xt, void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  using C = typename Stor<S>::C;
  constexpr bool dbl = (S == HM_F64);
  if (phase == 1 || phase == 2) {
    int rct = 1;
    while (rct < r && rct < 16) rct *= 2;
    switch (rct) {
      case 1: return launch_tree_rc<C, 1>(phase, mv, ws, r, st, pdl);
      case 2: return launch_tree_rc<C, 2>(phase, mv, ws, r, st, pdl);
      case 4: return launch_tree_rc<C, 4>(phase, mv, ws, r, st, pdl);
      case 8: return launch_tree_rc<C, 8>(phase, mv, ws, r, st, pdl);
      default: return launch_tree_rc<C, 16>(phase, mv, ws, r, st, pdl);
    }
  }
  const size_t esz = dbl ? 8 : 4;
  const int width = (phase == 3) ? mv.We : mv.m_pad;
  const int rc = pick_rc(r, esz, width);
#define HM_PHASE(RC_, TR_) return launch_phase_rc<S, RC_, TR_>(phase, mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl)
#define HM_PHASE_U(RC_, TR_, UQ_) \
  return launch_phase_rc<S, RC_, TR_, UQ_>(phase, mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl)
  if (phase == 0) {           // few rows (Kp) per block: one row per warp pass
    switch (rc) {
      case 1: HM_PHASE(1, 2);
      case 2: HM_PHASE(2, 2);
      case 4: HM_PHASE(4, 2);
      case 8: HM_PHASE(8, 2);
      case 16: HM_PHASE(16, 1);
      default: HM_PHASE(32, 1);
    }
  }
  // Narrow right-hand sides: 4 rows and two q steps per warp pass (8 rows and
  // one q step, for the short BF16 rows, measured slower: 0.50 vs 0.57 of HBM)
  constexpr int TRN = 4;
  constexpr int UQN = 2;
  if constexpr (S != HM_F64) {
    // one or two columns: the plane streamed through a ring of bulk copies
    hm_status st_ring = HM_EUNSUPPORTED;
    if (rc == 1) st_ring = launch_expand_ring<S, 1, TRN>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl);
    else if (rc == 2) st_ring = launch_expand_ring<S, 2, TRN>(mv, ws, r, X, ldx, xt, Y, ldy, yt, st, pdl);
    if (st_ring != HM_EUNSUPPORTED) return st_ring;
  }
  switch (rc) {
    case 1: HM_PHASE_U(1, TRN, UQN);
    case 2: HM_PHASE_U(2, TRN, UQN);
    case 4: HM_PHASE(4, 4);
    case 8: HM_PHASE(8, 4);
    case 16: HM_PHASE(16, (dbl ? 2 : 4));
    default: HM_PHASE(32, (dbl ? 1 : 2));
  }
#undef HM_PHASE
#undef HM_PHASE_U
}

}  // namespace hmi

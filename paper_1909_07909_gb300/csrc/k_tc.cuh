#pragma once
// Leaf expansion on the 5th-generation tensor cores (tcgen05) for BF16 and
// split-BF16 storage.  One CTA computes a 128-row tile of one leaf,
//
//     Y(rows, cols) = [D_i | E_i](rows, :) [X(I_i, cols); Z_i(:, cols)]
//
// (Sec. 4.1: the dense leaf product plus every level's U T for HODLR, or the
// leaf U y-hat for HSS), as a K loop of tcgen05.mma kind::f16, M = 128,
// N = NT, K = 16 per instruction, FP32 accumulators in tensor memory.
//
//  * A (the generator rows) streams through a ring (2 to 4 stages) of
//    128 x 64 bf16 tiles loaded by TMA (cp.async.bulk.tensor, 128-byte
//    swizzle), one elected thread issuing copies and MMAs.
//  * B is the right-hand side block, converted to bf16 on the fly and written
//    by all threads straight into the K-major 128-byte-swizzled layout the
//    MMA descriptor expects.  Chunks holding only X rows are staged at once;
//    chunks holding Z rows wait for the tree kernels (griddepcontrol.wait),
//    so the X part of the contraction overlaps the tree.
//  * Split BF16: A = A_hi + A_lo and B = B_hi + B_lo; acc0 += A_hi B_hi,
//    acc1 += A_hi B_lo + A_lo B_hi (the lo*lo term is dropped), and the
//    epilogue adds the two accumulators in FP64.
//  * Every wait is bounded (the device wait limit, 2 s of %globaltimer by
//    default, hm_set_device_wait_limit); on expiry the kernel sets
//    the library's device error word, skips its stores and still releases
//    its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <type_traits>

#include "hm_api_internal.h"
#include "k_simt.cuh"

namespace hmi {

constexpr int TC_M = 128;
constexpr int TC_KC = 64;
constexpr int TC_MAX_STAGES = 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One test of an mbarrier phase; the thread is suspended (not spinning)
// until the phase completes or about 1 us passes.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; after the wait limit of the status block
// of `err` (%globaltimer) records `code` there and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  const uint64_t limit = wait_limit_ns(err);
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (gtimer() - t0 > limit) {
      if (err) atomicExch(err, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// core-matrix groups 1024 bytes apart (tcgen05 descriptor format, version 1).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;              // leading byte offset (unused when swizzled)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;      // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;              // descriptor version
  d |= static_cast<uint64_t>(2) << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a);
  const __nv_bfloat16 hb = __float2bfloat16_rn(b);
  return static_cast<uint32_t>(__bfloat16_as_ushort(ha)) | (static_cast<uint32_t>(__bfloat16_as_ushort(hb)) << 16);
}

__device__ __forceinline__ double load_x_f64(const void* X, int xt, int64_t idx) {
  if (xt == HM_F64) return static_cast<const double*>(X)[idx];
  if (xt == HM_F32) return static_cast<const float*>(X)[idx];
  return __uint_as_float(static_cast<uint32_t>(static_cast<const uint16_t*>(X)[idx]) << 16);
}

template <typename V>
__device__ __forceinline__ V tc_in(double x) { return static_cast<V>(x); }
template <typename V>
__device__ __forceinline__ V tc_in(float x) { return static_cast<V>(x); }
template <typename V>
__device__ __forceinline__ V tc_in(uint16_t x) {
  return static_cast<V>(__uint_as_float(static_cast<uint32_t>(x) << 16));
}

// Z rows e0 .. e0+7 of column `col` when they are contiguous float in the
// tree scratch (HSS: the leaf's y-hat; HODLR: one level's T of one sibling),
// loaded as two 16-byte vectors; false (nothing loaded) otherwise.
template <typename V>
__device__ __forceinline__ bool z_run8(const MatView& mv, const Scratch& ws, int64_t r, int leaf, int e0, int64_t col,
                                       V (&out)[8]) {
  const float* base = nullptr;
  if (mv.kind == HM_HSS) {
    if (mv.p == 0) return false;
    base = static_cast<const float*>(ws.yf) + (static_cast<int64_t>(mv.L - 1 + leaf) * r + col) * mv.Ke + e0;
  } else {
    for (int l = 1; l <= mv.p; ++l) {
      const int lo = mv.koff[l], hi = mv.koff[l] + mv.kk[l];
      if (e0 < hi) {
        if (e0 < lo || e0 + 8 > hi) return false;   // the group leaves this level's rows
        const int anc = (1 << l) - 1 + (leaf >> (mv.p - l));
        const int sib = (anc & 1) ? anc + 1 : anc - 1;
        base = static_cast<const float*>(ws.PS) + (static_cast<int64_t>(sib) * r + col) * mv.Ke + e0;
        break;
      }
    }
    if (!base) return false;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  const float4 a = __ldcg(reinterpret_cast<const float4*>(base));
  const float4 b = __ldcg(reinterpret_cast<const float4*>(base) + 1);
  out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
  out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
  return true;
}

// Writes the B operand for K positions [k_begin, k_end) (multiples of 8) in
// the K-major swizzled layout: chunk c = k / 64 holds NT rows of 128 bytes,
// row n = right-hand side column, 16-byte unit u of the row at (u ^ (n % 8)).
// Row k of the operand is X(a0 + k) for k < m, zero up to m_pad, then the ke
// rows of Z, then zero.
// Each thread loads two 8-element groups before it converts and stores them.
template <typename T, bool SPLIT, int NT>
__device__ __forceinline__ void stage_b_t(uint8_t* sB, uint8_t* sBlo, int k_begin, int k_end, int tid, int nthr,
                                          const MatView& mv, const Scratch& ws, int64_t r, int leaf, int64_t a0,
                                          int m, int ke, int col0, const T* X, int64_t ldx) {
  using V = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  const int ngroups = (k_end - k_begin) >> 3;
  const int items = NT * ngroups;
  constexpr int U = (sizeof(T) == 8) ? 2 : 4;
  for (int base = tid; base < items; base += nthr * U) {
    V v[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = base + u * nthr;
      const int g = it % ngroups;
      const int n = it / ngroups;
      const int k0 = k_begin + g * 8;
      const int64_t col = col0 + n;
      const bool ok = it < items && col < r;
      const T* p = X + (a0 + k0) + col * ldx;
      if (ok && k0 + 8 <= m && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        // eight rows of one column, all inside the leaf: vector loads
        if constexpr (sizeof(T) == 4) {
          const float4 x0 = *reinterpret_cast<const float4*>(p);
          const float4 x1 = *reinterpret_cast<const float4*>(p + 4);
          v[u][0] = x0.x; v[u][1] = x0.y; v[u][2] = x0.z; v[u][3] = x0.w;
          v[u][4] = x1.x; v[u][5] = x1.y; v[u][6] = x1.z; v[u][7] = x1.w;
        } else if constexpr (sizeof(T) == 8) {
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const double2 x = *reinterpret_cast<const double2*>(p + 2 * h);
            v[u][2 * h] = x.x;
            v[u][2 * h + 1] = x.y;
          }
        } else {
          const uint4 x = *reinterpret_cast<const uint4*>(p);
          const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            v[u][2 * h] = __uint_as_float(w[h] << 16);
            v[u][2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
          }
        }
      } else if (ok && k0 >= mv.m_pad && k0 + 8 <= mv.m_pad + ke && z_run8<V>(mv, ws, r, leaf, k0 - mv.m_pad, col, v[u])) {
        // eight Z rows of one column, contiguous in the tree scratch: vector loads
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = k0 + j;
          V x = V(0);
          if (ok) {
            if (k < m) x = tc_in<V>(p[j]);
            else if (k >= mv.m_pad && k - mv.m_pad < ke)
              x = static_cast<V>(z_value<float>(mv, ws, r, leaf, k - mv.m_pad, col));
          }
          v[u][j] = x;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int it = base + u * nthr;
      if (it >= items) continue;
      const int g = it % ngroups;
      const int n = it / ngroups;
      const int k0 = k_begin + g * 8;
      const int chunk = k0 >> 6;
      const int un = (k0 & 63) >> 3;
      const uint32_t off = chunk * (NT * 128) + n * 128 + ((un ^ (n & 7)) << 4);
      uint4 hi;
      hi.x = pack_bf16(static_cast<float>(v[u][0]), static_cast<float>(v[u][1]));
      hi.y = pack_bf16(static_cast<float>(v[u][2]), static_cast<float>(v[u][3]));
      hi.z = pack_bf16(static_cast<float>(v[u][4]), static_cast<float>(v[u][5]));
      hi.w = pack_bf16(static_cast<float>(v[u][6]), static_cast<float>(v[u][7]));
      *reinterpret_cast<uint4*>(sB + off) = hi;
      if constexpr (SPLIT) {
        float lo[8];
        const uint32_t h[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t bits = (j & 1) ? (h[j >> 1] & 0xffff0000u) : (h[j >> 1] << 16);
          lo[j] = static_cast<float>(v[u][j] - static_cast<V>(__uint_as_float(bits)));
        }
        uint4 lw;
        lw.x = pack_bf16(lo[0], lo[1]);
        lw.y = pack_bf16(lo[2], lo[3]);
        lw.z = pack_bf16(lo[4], lo[5]);
        lw.w = pack_bf16(lo[6], lo[7]);
        *reinterpret_cast<uint4*>(sBlo + off) = lw;
      }
    }
  }
}

template <bool SPLIT, int NT>
__device__ __forceinline__ void stage_b(uint8_t* sB, uint8_t* sBlo, int k_begin, int k_end, int tid, int nthr,
                                        const MatView& mv, const Scratch& ws, int64_t r, int leaf, int64_t a0, int m,
                                        int ke, int col0, const void* X, int64_t ldx, int xt) {
  if (xt == HM_F32)
    stage_b_t<float, SPLIT, NT>(sB, sBlo, k_begin, k_end, tid, nthr, mv, ws, r, leaf, a0, m, ke, col0,
                                static_cast<const float*>(X), ldx);
  else if (xt == HM_F64)
    stage_b_t<double, SPLIT, NT>(sB, sBlo, k_begin, k_end, tid, nthr, mv, ws, r, leaf, a0, m, ke, col0,
                                 static_cast<const double*>(X), ldx);
  else
    stage_b_t<uint16_t, SPLIT, NT>(sB, sBlo, k_begin, k_end, tid, nthr, mv, ws, r, leaf, a0, m, ke, col0,
                                   static_cast<const uint16_t*>(X), ldx);
}

// Shared-memory bytes of one CTA's work (after 1024-byte alignment of the
// base): the A ring (mt 128-row tiles per stage), the B operand (hi and,
// split, lo), the barriers, the TMEM slot.
__host__ __device__ inline size_t tc_layout_bytes(bool split, int NT, int nK, int nst, int mt = 1) {
  const size_t stage = static_cast<size_t>(mt) * TC_M * TC_KC * 2 * (split ? 2 : 1);
  return nst * stage + static_cast<size_t>(nK) * NT * 128 * (split ? 2 : 1) + (2 * TC_MAX_STAGES + 2) * 8 + 16;
}

template <bool SPLIT, int NT>
__host__ __device__ constexpr int tc_ncols() {
  return SPLIT ? ((2 * NT <= 32) ? 32 : 2 * NT) : ((NT < 32) ? 32 : NT);
}

// Tensor-memory columns of one tile's accumulators (a power of two, >= 32).
__host__ __device__ inline int tc_ncols_host(bool split, int NT) {
  return split ? ((2 * NT <= 32) ? 32 : 2 * NT) : ((NT < 32) ? 32 : NT);
}

// mt (1 or 2) consecutive 128-row tiles with columns [col0, col0 + NT) of one
// leaf's contraction; the tiles share the B operand and use one accumulator
// set each (TMEM columns u * tc_ncols<SPLIT, NT>() onwards):
//   expansion (PROJ = false): Y(rows) = [D_i | E_i](rows, :) [X_i; Z_i], tile rt
//     of the leaf's rows, K = m_pad + Ke;
//   projection (PROJ = true): P_i = Wprj_i X_i, tile rt of the leaf's Kp
//     projection rows (box_rows of them are loaded; the rest of the 128-row A
//     tile is never used), K = m_pad; the result goes to the tree scratch.
// X rows come through TMA (tmX) when X is bf16, the leaf is full (m = m_pad)
// and its first row is 8-aligned; otherwise they are converted by the threads.
// The caller owns at least mt * tc_ncols<SPLIT, NT>() columns of tensor
// memory at `tmem` and a 1024-byte aligned shared-memory area `base` of
// tc_layout_bytes(..., mt) bytes.  Returns with every tensor-memory read
// complete and the block synchronised.  Each tile's result is the same
// whatever mt is.
template <bool SPLIT, int NT, bool PROJ>
__device__ void tc_tile(const CUtensorMap* tmA, const CUtensorMap* tmAlo, const CUtensorMap* tmX, int box_rows,
                        const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx, int xt,
                        void* Y, int64_t ldy, int yt, int leaf, int rt, int col0, int nK, int nX, int nst,
                        uint8_t* base, uint32_t tmem, int mt = 1) {
  constexpr int A_BYTES = TC_M * TC_KC * 2;
  const int STAGE_BYTES = A_BYTES * (SPLIT ? 2 : 1) * mt;
  constexpr int TPT = tc_ncols<SPLIT, NT>();       // TMEM columns per tile
  constexpr int BCH = NT * 128;
  constexpr uint32_t IDESC = idesc_bf16(TC_M, NT);
  uint8_t* sA = base;
  uint8_t* sB = sA + nst * STAGE_BYTES;
  uint8_t* sBlo = sB + nK * BCH;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sBlo + (SPLIT ? nK * BCH : 0));
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = full0 + 8 * TC_MAX_STAGES;
  const uint32_t accb = full0 + 16 * TC_MAX_STAGES;
  const uint32_t xbar = full0 + 8 * (2 * TC_MAX_STAGES + 1);

  const int64_t a0 = mv.off[leaf];
  const int m = static_cast<int>(mv.off[leaf + 1] - a0);
  const int t0 = rt * TC_M * mt;
  int lim;                                           // rows of this leaf's output
  int a_row;
  if constexpr (PROJ) {
    if (t0 >= mv.Kp) return;
    lim = mv.Kp;
    a_row = leaf * mv.Kp + t0;
  } else {
    if (t0 >= m) return;
    lim = m;
    a_row = static_cast<int>(a0 + t0);
  }
  const int a_bytes = TC_KC * box_rows * 2 * (SPLIT ? 2 : 1) * mt;   // bytes one stage's TMA writes
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int* err = ws.err;
  // X by TMA: bf16 input, full leaf, 16-byte aligned start row; the TMA
  // moves the chunks of 64 X rows (nXt of them), the threads stage the rest
  const bool x_tma = (tmX != nullptr) && xt == HM_BF16 && m == mv.m_pad && (a0 & 7) == 0;
  const int nXt = x_tma ? mv.m_pad / TC_KC : 0;
  const int ke = PROJ ? 0 : mv.Ke;                 // Z rows of the operand
  // bf16 X has no lo part: the A_hi x B_lo products of X chunks vanish
  const bool x_lo_zero = (xt == HM_BF16);

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accb, 1);
    mbar_init(xbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int c) {
    const int s = c % nst;
    const uint32_t dst = smem_u32(sA + s * STAGE_BYTES);
    mbar_expect_tx(full0 + 8 * s, a_bytes);
    for (int u = 0; u < mt; ++u) {
      tma_load_2d(dst + u * A_BYTES, tmA, c * TC_KC, a_row + u * TC_M, full0 + 8 * s);
      if constexpr (SPLIT) tma_load_2d(dst + (mt + u) * A_BYTES, tmAlo, c * TC_KC, a_row + u * TC_M, full0 + 8 * s);
    }
  };
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmA)) : "memory");
    if (nXt > 0) {
      mbar_expect_tx(xbar, static_cast<uint32_t>(nXt * BCH));
      for (int c = 0; c < nXt; ++c)
        tma_load_2d(smem_u32(sB + c * BCH), tmX, static_cast<int>(a0) + c * TC_KC, col0, xbar);
    }
    for (int c = 0; c < min(nst, nK); ++c) issue(c);
  }
  if (nXt < nX)
    stage_b<SPLIT, NT>(sB, sBlo, nXt * TC_KC, nX * TC_KC, threadIdx.x, 128, mv, ws, r, leaf, a0, m, ke, col0, X, ldx,
                       xt);
  fence_proxy_async();
  __syncthreads();

  // MMAs over chunks [c0, c1); single thread.  Returns false on a timed-out wait.
  auto mma_chunks = [&](int c0, int c1) -> bool {
    for (int c = c0; c < c1; ++c) {
      const int s = c % nst;
      const uint32_t ph = (c / nst) & 1;
      if (!mbar_wait(full0 + 8 * s, ph, err, 11)) return false;
      tc_fence_after();
      const uint32_t a_addr = smem_u32(sA + s * STAGE_BYTES);
      const uint32_t b_addr = smem_u32(sB + c * BCH);
      const bool lo_zero = x_lo_zero && c < nX;
#pragma unroll
      for (int k = 0; k < TC_KC / 16; ++k) {
        const uint64_t bd = sw128_desc(b_addr + k * 32);
        const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
        for (int u = 0; u < mt; ++u) {
          const uint32_t d = tmem + u * TPT;
          const uint64_t ad = sw128_desc(a_addr + u * A_BYTES + k * 32);
          umma_bf16(d, ad, bd, IDESC, acc);
          if constexpr (SPLIT) {
            const uint64_t adl = sw128_desc(a_addr + (mt + u) * A_BYTES + k * 32);
            if (!lo_zero) {
              const uint64_t bdl = sw128_desc(smem_u32(sBlo + c * BCH) + k * 32);
              umma_bf16(d + NT, ad, bdl, IDESC, acc);
              umma_bf16(d + NT, adl, bd, IDESC, 1u);
            } else {
              umma_bf16(d + NT, adl, bd, IDESC, acc);
            }
          }
        }
      }
      umma_commit(empty0 + 8 * s);
      if (c + nst < nK) {
        if (!mbar_wait(empty0 + 8 * s, ph, err, 12)) return false;
        issue(c + nst);
      }
    }
    return true;
  };

  if (warp == 0) {
    bool ok = true;
    if (lane == 0) {
      if (nXt > 0) ok = mbar_wait(xbar, 0, err, 14);
      if (ok) ok = mma_chunks(0, nX);
    }
    __syncwarp();
    if constexpr (!PROJ) asm volatile("bar.sync 1, 128;" ::: "memory");   // Z rows staged by warps 1..3
    if (lane == 0) {
      if (ok) ok = mma_chunks(nX, nK);
      umma_commit(accb);                                   // arrives when every issued MMA is done
    }
    __syncwarp();
  } else if constexpr (!PROJ) {
    pdl_wait();                                            // Z is written by the tree kernels
    stage_b<SPLIT, NT>(sB, sBlo, nX * TC_KC, nK * TC_KC, threadIdx.x - 32, 96, mv, ws, r, leaf, a0, m, ke, col0, X,
                       ldx, xt);
    fence_proxy_async();
    asm volatile("bar.arrive 1, 128;" ::: "memory");
  }
  // one lane per warp waits for the accumulators; the rest of the warp waits at the warp barrier
  int done_i = 0;
  if (lane == 0) done_i = mbar_wait(accb, 0, err, 13) ? 1 : 0;
  const bool done = __shfl_sync(0xffffffffu, done_i, 0) != 0;
  tc_fence_after();
  const int row = warp * 32 + lane;
  const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
  const int node = mv.L - 1 + leaf;
  const int ldo = (mv.kind == HM_HODLR) ? mv.Ke : mv.Kp;
  float* pout = static_cast<float*>(mv.kind == HM_HODLR ? ws.PS : ws.xh);
  for (int u = 0; u < mt; ++u) {
  const int tu = t0 + u * TC_M;                            // first row of tile u
  const int nrows = lim - tu;                              // rows of tile u inside the output (may be <= 0)
  for (int cb = 0; cb < NT; cb += 16) {
    if constexpr (PROJ) {
      if (warp * 32 >= nrows) break;                       // whole warp outside the projection rows
    }
    float v[16];
    tmem_ld16(lane_addr + u * TPT + cb, v);
    float w[16];
    if constexpr (SPLIT) tmem_ld16(lane_addr + u * TPT + NT + cb, w);
    if (done && row < nrows) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int64_t col = col0 + cb + j;
        if (col < r) {
          if constexpr (PROJ) {
            const float y = SPLIT ? v[j] + w[j] : v[j];
            pout[(static_cast<int64_t>(node) * r + col) * ldo + tu + row] = y;
          } else {
            const int64_t idx = (a0 + tu + row) + col * ldy;
            if constexpr (SPLIT) {
              const double y = static_cast<double>(v[j]) + static_cast<double>(w[j]);
              if (yt == HM_F64) static_cast<double*>(Y)[idx] = y;
              else static_cast<float*>(Y)[idx] = static_cast<float>(y);
            } else {
              if (yt == HM_F64) static_cast<double*>(Y)[idx] = v[j];
              else static_cast<float*>(Y)[idx] = v[j];
            }
          }
        }
      }
    }
  }
  }
  tc_fence_before();
  __syncthreads();
}

template <bool SPLIT, int NT, bool PROJ>
__global__ void __launch_bounds__(128, 1)
    k_leaf_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
              const __grid_constant__ CUtensorMap tmX, int use_tmx, int box_rows, MatView mv, Scratch ws, int64_t r,
              const void* X, int64_t ldx, int xt, void* Y, int64_t ldy, int yt, int tiles_per_leaf, int nK, int nX,
              int nst, int mt) {
  // tensor-memory columns: mt tiles of tc_ncols each (a power of two, at most 512)
  const uint32_t NCOL = static_cast<uint32_t>(tc_ncols<SPLIT, NT>() * mt);
  pdl_launch_dependents();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(base + tc_layout_bytes(SPLIT, NT, nK, nst, mt) - 16);
  const int leaf = blockIdx.x / tiles_per_leaf;
  const int rt = blockIdx.x % tiles_per_leaf;
  const int lim = PROJ ? mv.Kp : static_cast<int>(mv.off[leaf + 1] - mv.off[leaf]);
  if (rt * TC_M * mt >= lim) return;
  if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(tslot), NCOL);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  tc_tile<SPLIT, NT, PROJ>(&tmA, &tmAlo, use_tmx ? &tmX : nullptr, box_rows, mv, ws, r, X, ldx, xt, Y, ldy, yt,
                           leaf, rt, blockIdx.y * NT, nK, nX, nst, base, tmem, mt);
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, NCOL);
  }
}


}  // namespace hmi

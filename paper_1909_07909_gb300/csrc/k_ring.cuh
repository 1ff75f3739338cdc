// SIMT leaf expansion for one or two right-hand sides with the expansion
// plane streamed by bulk copies (cp.async.bulk) through a ring of
// shared-memory stages, instead of 16-byte loads from every lane.
//
// A narrow right-hand side gives each expansion row (the leaf's D row and its
// E row, 672 bytes for BF16 at leaf 256 and 80 factor columns) only a few
// multiply-adds per byte, so the kernel is bound by how many bytes it keeps
// in flight.  With per-lane loads a warp has one row group's loads
// outstanding at a time; here one thread requests whole stages (32 rows,
// contiguous in the plane) into a ring of 2-3 stages, starting before the
// block waits for the tree kernel (the plane does not depend on it), and the
// warps multiply from shared memory.
//
// The arithmetic is the row engine's (k_simt.cuh: rows_gemm) operation for
// operation: lane l sums the 16-byte vectors q = l, l + 32, ... of its rows in
// increasing q, then the same butterfly, so the results are bit-identical to
// the per-lane-load kernel, to the batched kernels and to wider products.
#pragma once

#include "k_tc.cuh"

namespace hmi {

__device__ __forceinline__ void ring_bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

constexpr int RING_MAX_STAGES = 4;

template <int S>
__host__ __device__ constexpr int plane_esz() {
  return (S == HM_F64) ? 8 : (S == HM_F32) ? 4 : 2;
}

// Shared memory of one block: barriers, the ring (hi, and lo for BF16X2), B, Os.
template <int S, int RC>
__host__ __device__ inline size_t ring_smem(int We, int SR, int nstg, int RT) {
  using C = typename Stor<S>::C;
  const size_t stage = static_cast<size_t>(SR) * We * plane_esz<S>();
  return 128 + nstg * stage * (S == HM_BF16X2 ? 2 : 1) + sizeof(C) * (static_cast<size_t>(RC) * We + RC * (RT + 1));
}

template <int S, int RC, int TR>
__global__ void __launch_bounds__(256) k_expand_ring(MatView mv, Scratch ws, int64_t r, const void* X, int64_t ldx,
                                                     int xt, void* Y, int64_t ldy, int yt, int RT, int tiles_per_leaf,
                                                     int nstg) {
  using C = typename Stor<S>::C;
  constexpr int V = Stor<S>::V;
  constexpr int ES = plane_esz<S>();
  constexpr bool LO = (S == HM_BF16X2);
  constexpr int UQ = 2;
  constexpr int T = TR * RC;
  constexpr int NV = (T >= 32) ? T / 32 : 1;
  constexpr int OWN = (T >= 32) ? 0 : (32 / T - 1);
  constexpr int SR = 8 * TR;                        // rows per stage: 8 warps x TR
  extern __shared__ __align__(128) unsigned char ring_smem_raw[];
  __shared__ int s_dead;
  __shared__ int s_issued;
  const int leaf = blockIdx.x / tiles_per_leaf;
  const int tile = blockIdx.x % tiles_per_leaf;
  const int col0 = blockIdx.y * RC;
  const int ncols = static_cast<int>(min(static_cast<int64_t>(RC), r - col0));
  const int64_t a0 = mv.off[leaf];
  const int m = static_cast<int>(mv.off[leaf + 1] - a0);
  const int t0 = tile * RT;
  if (t0 >= m) return;
  const int nrows = min(RT, m - t0);
  const int K = mv.We;
  const int Q = K / V;
  const uint32_t row_bytes = static_cast<uint32_t>(K) * ES;
  const uint32_t stage_bytes = SR * row_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring_smem_raw);
  unsigned char* ring = ring_smem_raw + 128;
  unsigned char* ring_lo = ring + static_cast<size_t>(nstg) * stage_bytes;
  C* Bs = reinterpret_cast<C*>(ring + static_cast<size_t>(nstg) * stage_bytes * (LO ? 2 : 1));
  C* Os = Bs + RC * K;
  const int OS = RT + 1;
  const int nst = (nrows + SR - 1) / SR;
  const int64_t row0 = a0 + t0;
  const unsigned char* Ab = static_cast<const unsigned char*>(mv.A) + row0 * row_bytes;
  const unsigned char* Lb = LO ? static_cast<const unsigned char*>(mv.A_lo) + row0 * row_bytes : nullptr;

  auto issue = [&](int sidx) {                      // one thread
    const int slot = sidx % nstg;
    const int rows = min(SR, nrows - sidx * SR);
    const uint32_t bytes = static_cast<uint32_t>(rows) * row_bytes;
    const uint32_t bar = smem_u32(bars + slot);
    mbar_expect_tx(bar, bytes * (LO ? 2u : 1u));
    ring_bulk_g2s(smem_u32(ring + static_cast<size_t>(slot) * stage_bytes),
                  Ab + static_cast<size_t>(sidx) * stage_bytes, bytes, bar);
    if constexpr (LO)
      ring_bulk_g2s(smem_u32(ring_lo + static_cast<size_t>(slot) * stage_bytes),
                    Lb + static_cast<size_t>(sidx) * stage_bytes, bytes, bar);
  };
  if (threadIdx.x == 0) {
    s_dead = 0;
    for (int s = 0; s < nstg; ++s) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    int k = 0;
    for (; k < min(nstg, nst); ++k) issue(k);      // the plane does not depend on the previous kernel
    s_issued = k;
  }
  // B = [X_i; Z_i]: the X part now, Z after the tree kernel's results are visible
  stage_x<C>(Bs, K, X, xt, ldx, a0, m, mv.m_pad, col0, ncols, RC);
  pdl_wait();
  const int Ke = mv.Ke;
  const int mp = mv.m_pad;
  for (int idx = threadIdx.x; idx < RC * Ke; idx += blockDim.x) {
    const int c = idx / Ke, e = idx % Ke;
    Bs[c * K + mp + e] = (c < ncols) ? z_value<C>(mv, ws, r, leaf, e, col0 + c) : C(0);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  for (int sidx = 0; sidx < nst; ++sidx) {
    const int slot = sidx % nstg;
    if (lane == 0 && !*reinterpret_cast<volatile int*>(&s_dead)) {
      if (!mbar_wait(smem_u32(bars + slot), (sidx / nstg) & 1, ws.err, 15)) *reinterpret_cast<volatile int*>(&s_dead) = 1;
    }
    __syncwarp();
    const int rows = min(SR, nrows - sidx * SR);
    const unsigned char* st_hi = ring + static_cast<size_t>(slot) * stage_bytes;
    const unsigned char* st_lo = ring_lo + static_cast<size_t>(slot) * stage_bytes;
    const int tw = warp * TR;                       // this warp's first row in the stage
    if (tw < rows) {
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
            if (q < Q && tw + t < rows) {
              const size_t off = static_cast<size_t>(tw + t) * row_bytes + static_cast<size_t>(q) * 16;
              ra[u][t] = *reinterpret_cast<const uint4*>(st_hi + off);
              if constexpr (LO) rl[u][t] = *reinterpret_cast<const uint4*>(st_lo + off);
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
            load_b<C, V>(Bs + c * K + q * V, b);
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
          if (tw + t < rows) Os[c * OS + sidx * SR + tw + t] = acc[i];
        }
      }
    }
    __syncthreads();                                // every warp is done with the slot
    if (threadIdx.x == 0 && sidx + nstg < nst && !*reinterpret_cast<volatile int*>(&s_dead)) {
      fence_proxy_async();                          // the slot's generic reads before the copy that overwrites it
      issue(sidx + nstg);
      s_issued = sidx + nstg + 1;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ncols * nrows; idx += blockDim.x) {
    const int c = idx / nrows, t = idx % nrows;
    store_y<C>(Y, yt, (row0 + t) + static_cast<int64_t>(col0 + c) * ldy, Os[c * OS + t]);
  }
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(&s_dead)) {
    // a wait gave up: wait (bounded) for the copies still in flight before the block's memory is released
    const int hi = s_issued;
    for (int u = (hi > nstg ? hi - nstg : 0); u < hi; ++u)
      mbar_wait(smem_u32(bars + (u % nstg)), (u / nstg) & 1, nullptr, 0);
  }
}

template <int S, int RC, int TR>
hm_status launch_expand_ring(const MatView& mv, const Scratch& ws, int64_t r, const void* X, int64_t ldx, int xt,
                             void* Y, int64_t ldy, int yt, cudaStream_t st, bool pdl) {
  constexpr int SR = 8 * TR;
  const int nchunks = static_cast<int>((r + RC - 1) / RC);
  const size_t row_bytes = static_cast<size_t>(mv.We) * plane_esz<S>();
  if (row_bytes % 16 != 0) return HM_EUNSUPPORTED;
  // a whole leaf per block, as the per-lane-load kernel
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int RT = 64;
  while (RT < 256 && RT < mv.m_pad &&
         static_cast<int64_t>(mv.L) * ((mv.m_pad + 2 * RT - 1) / (2 * RT)) * nchunks >= 4 * sms)
    RT *= 2;
  // as many stages (2..4) as keep the block within ~72 KB, so three blocks share an SM
  int nstg = RING_MAX_STAGES;
  while (nstg > 2 && ring_smem<S, RC>(mv.We, SR, nstg, RT) > 72 * 1024) --nstg;
  const size_t smem = ring_smem<S, RC>(mv.We, SR, nstg, RT);
  if (smem > 200 * 1024) return HM_EUNSUPPORTED;
  const int tiles = (mv.m_pad + RT - 1) / RT;
  cudaFuncSetAttribute(k_expand_ring<S, RC, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  Scratch wk = ws;
  wk.prof = nullptr;
  prof_mark(ws.prof, 3, true, st);
  const cudaError_t e = launch_k(k_expand_ring<S, RC, TR>, dim3(mv.L * tiles, nchunks), dim3(256), smem, st, pdl, mv,
                                 wk, r, X, ldx, xt, Y, ldy, yt, RT, tiles, nstg);
  prof_mark(ws.prof, 3, false, st);
  if (e != cudaSuccess) {
    set_error("ring expansion launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

}  // namespace hmi

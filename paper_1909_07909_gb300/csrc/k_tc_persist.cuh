#pragma once
// Persistent leaf expansion on the tensor cores for BF16 storage (Sec. 4.1:
// Y(rows, cols) = [D_i | E_i](rows, :) [X(I_i, cols); Z_i(:, cols)]), one CTA
// per SM walking work items (leaf, group of mt 128-row tiles, NT columns).
//
// The one-item-per-CTA kernel (k_tc.cuh) loads, multiplies and stores one
// item after the other, and at one CTA per SM (its whole B operand lives in
// shared memory) the SM idles while the epilogue drains the accumulators.
// Here the roles are split across warps so every phase overlaps the others:
//
//  * warp 0 (one thread): TMA producer; each stage of the ring holds one
//    64-wide K chunk of the mt A tiles and of B, and X chunks of B come by
//    TMA when X is bf16 and the leaf qualifies;
//  * warps 2, 3: the B chunks TMA does not bring.  An item's Z block (its
//    rows of the tree kernels' output, FP32) is fetched whole into shared
//    memory for the next item while this one is multiplied (after
//    griddepcontrol.wait, before the first), and converted from there to
//    bf16 straight into the stages.  The fetch is Ke/hb tiled TMA loads of hb
//    rows by NT columns from the tree scratch viewed as a 2-D tensor (each
//    box lies in one level's block); per-thread loads, and even one
//    bulk copy per level and column, queued behind the SM's own stream of
//    stage copies and took 30-80 k cycles per item.  Where the rows are not
//    16-byte aligned the block comes by cp.async.  X rows of other types or
//    of ragged leaves are converted from global memory as in k_tc.cuh;
//  * warp 1 (one thread): tcgen05.mma issue into one of two tensor-memory
//    accumulator sets, commits that free the stage and, after an item's last
//    chunk, publish its accumulators;
//  * warps 4 .. 4 + 4 EPI_WG - 1: epilogue, tensor memory -> registers ->
//    global Y, releasing the accumulator set for the item after next.
//
// The MMA sequence of a tile is the one of k_tc.cuh (chunks in order, four
// K = 16 steps each, the same descriptors and instruction shape), so the
// results are bit-identical to it and to the batched kernels.  Every wait is
// bounded (the library's device wait limit); on expiry the kernel records an
// error code, stops, waits (bounded) for its copies and MMAs in flight and
// releases its tensor memory.
#include "k_tc.cuh"

namespace hmi {

constexpr int TCP_MAX_STAGES = 8;
constexpr int TCP_EPI_WG = 2;                        // epilogue warpgroups
constexpr int TCP_THREADS = 128 + 128 * TCP_EPI_WG;  // producer, MMA, 2 stager warps, epilogue

__device__ __forceinline__ void mbar_arrive1(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__host__ __device__ inline size_t tcp_stage_bytes(int NT, int mt) {
  return static_cast<size_t>(mt) * TC_M * TC_KC * 2 + static_cast<size_t>(NT) * 128;
}

// Row stride (floats) of the Z block in shared memory: Ke rounded up to 4.
__host__ __device__ inline int tcp_ke4(int Ke) { return (Ke + 3) & ~3; }

// Dynamic shared memory: 1024 bytes of alignment slack, the stages, the Z
// block (NT columns of tcp_ke4(Ke) floats), 512 bytes of barriers and flags.
__host__ __device__ inline size_t tcp_smem_bytes(int NT, int mt, int nst, int Ke) {
  return 1024 + static_cast<size_t>(nst) * tcp_stage_bytes(NT, mt) + static_cast<size_t>(NT) * tcp_ke4(Ke) * 4 + 512;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Address of Z(e, col) of a leaf in the tree scratch (HSS: the leaf's y-hat;
// HODLR: level l's T of the leaf's sibling at that level) and the number of
// rows from e on that are contiguous there (to the end of the run).
__device__ __forceinline__ const float* tcp_z_src(const MatView& mv, const Scratch& ws, int64_t r, int leaf, int e,
                                                  int64_t col, int* run) {
  if (mv.kind == HM_HSS) {
    *run = mv.Ke - e;
    if (mv.p == 0) return nullptr;                 // one leaf: no coupling rows
    return static_cast<const float*>(ws.yf) + (static_cast<int64_t>(mv.L - 1 + leaf) * r + col) * mv.Ke + e;
  }
  for (int l = 1; l <= mv.p; ++l) {
    const int hi = mv.koff[l] + mv.kk[l];
    if (e < hi) {
      if (e < mv.koff[l]) break;
      const int anc = (1 << l) - 1 + (leaf >> (mv.p - l));
      const int sib = (anc & 1) ? anc + 1 : anc - 1;
      *run = hi - e;
      return static_cast<const float*>(ws.PS) + (static_cast<int64_t>(sib) * r + col) * mv.Ke + e;
    }
  }
  *run = 0;
  return nullptr;
}

// Z block layout in shared memory: Z(e, col0 + n) at zr[(e / 4) * NT * 4 +
// n * 4 + e % 4] (4-row groups of all NT columns, as a 4 x NT tensor box lands).
// Requests the Z block of one item (zero for columns past r and rows past Ke)
// by cp.async from the 64 stager threads; the caller waits for it with
// cp_async_commit_wait_all and a stager barrier.
template <int NT>
__device__ __forceinline__ void tcp_z_fetch(float* zr, const MatView& mv, const Scratch& ws, int64_t r, int leaf,
                                            int col0, int stid) {
  const int Ke = mv.Ke;
  const int ke4 = tcp_ke4(Ke);
  const int q4 = ke4 >> 2;
  for (int idx = stid; idx < NT * q4; idx += 64) {
    const int n = idx / q4;
    const int e0 = (idx - n * q4) * 4;
    const int64_t col = col0 + n;
    float* dst = zr + (e0 >> 2) * NT * 4 + n * 4;
    if (col >= r) {
      *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    int run = 0;
    const float* src = tcp_z_src(mv, ws, r, leaf, e0, col, &run);
    if (src && run >= 4 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
      cp_async16(dst, src);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int rj = 0;
        const float* sj = (e0 + j < Ke) ? tcp_z_src(mv, ws, r, leaf, e0 + j, col, &rj) : nullptr;
        if (sj) cp_async4(dst + j, sj);
        else dst[j] = 0.f;
      }
    }
  }
}

// The Z block of one item by Ke / hb tiled TMA loads of hb x NT boxes (one
// thread), completing on `zbar`; Z(e, col0 + n) lands at zr[(e / hb) * NT *
// hb + n * hb + e % hb].  tmZ views the tree scratch (HSS: y-hat; HODLR: the
// T blocks) as a 2-D FP32 tensor of Ke-float rows, row node * r + col, and
// every box lies in one node's rows (hb divides each level's block).
// Columns past r hold other values (the next node's rows, or zeros past the
// end): their B columns only feed output columns that are not stored.
__device__ __forceinline__ void tcp_z_fetch_tma(float* zr, uint32_t zbar, const CUtensorMap* tmZ, const MatView& mv,
                                                int64_t r, int leaf, int col0, int NT, int hb) {
  const int nq = mv.Ke / hb;
  mbar_expect_tx(zbar, static_cast<uint32_t>(mv.Ke) * NT * 4);
  for (int q = 0; q < nq; ++q) {
    const int e0 = q * hb;
    int node;
    if (mv.kind == HM_HSS) {
      node = mv.L - 1 + leaf;
    } else {
      int l = 1;
      while (l < mv.p && e0 >= mv.koff[l] + mv.kk[l]) ++l;
      const int anc = (1 << l) - 1 + (leaf >> (mv.p - l));
      node = (anc & 1) ? anc + 1 : anc - 1;
    }
    tma_load_2d(smem_u32(zr + static_cast<size_t>(q) * NT * hb), tmZ, e0, static_cast<int>(node * r + col0), zbar);
  }
}

// B rows [c*64, c*64 + 64) of a chunk holding only Z and zero rows (c*64 >=
// m_pad), from the Z block in shared memory (box height hb), in the K-major
// swizzled layout of stage_b (the same bf16 rounding of the same FP32
// values).  Consecutive threads take consecutive columns.
template <int NT>
__device__ __forceinline__ void tcp_z_convert(uint8_t* sb, const float* zr, int Ke, int hb, int kz0, int stid) {
  for (int it = stid; it < NT * 8; it += 64) {
    const int n = it % NT;
    const int un = it / NT;
    const int e0 = kz0 + un * 8;                   // first Z row of this 8-row group (a multiple of 8)
    float v[8];
    if (e0 + 8 <= Ke && hb % 8 == 0) {
      const float* p = zr + (e0 / hb) * NT * hb + n * hb + (e0 % hb);
      const float4 lo = *reinterpret_cast<const float4*>(p);
      const float4 hi4 = *reinterpret_cast<const float4*>(p + 4);
      v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
      v[4] = hi4.x; v[5] = hi4.y; v[6] = hi4.z; v[7] = hi4.w;
    } else if (e0 + 8 <= Ke && hb == 4) {
      const float4 lo = *reinterpret_cast<const float4*>(zr + (e0 >> 2) * NT * 4 + n * 4);
      const float4 hi4 = *reinterpret_cast<const float4*>(zr + ((e0 >> 2) + 1) * NT * 4 + n * 4);
      v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
      v[4] = hi4.x; v[5] = hi4.y; v[6] = hi4.z; v[7] = hi4.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int e = e0 + j;
        v[j] = (e < Ke) ? zr[(e / hb) * NT * hb + n * hb + (e % hb)] : 0.f;
      }
    }
    uint4 hi;
    hi.x = pack_bf16(v[0], v[1]);
    hi.y = pack_bf16(v[2], v[3]);
    hi.z = pack_bf16(v[4], v[5]);
    hi.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(sb + n * 128 + ((un ^ (n & 7)) << 4)) = hi;
  }
}

struct TcpItem {
  int leaf, t0, col0, m;
  int64_t a0;
  bool valid;
};

// Item it: column chunk fastest, then tile group, then leaf (consecutive CTAs
// take the column chunks of the same rows, which then hit in L2).
// The projection (proj) has Kp output rows per leaf, the expansion m.
__device__ __forceinline__ TcpItem tcp_item(const MatView& mv, int it, int tgroups, int nchunks, int NT, int mt,
                                            bool proj = false) {
  TcpItem w;
  const int chunk = it % nchunks;
  const int tg = (it / nchunks) % tgroups;
  w.leaf = it / (nchunks * tgroups);
  w.a0 = mv.off[w.leaf];
  w.m = static_cast<int>(mv.off[w.leaf + 1] - w.a0);
  w.t0 = tg * TC_M * mt;
  w.col0 = chunk * NT;
  w.valid = w.t0 < (proj ? mv.Kp : w.m);
  return w;
}

// PROJ: the leaf projection P_i = Wprj_i X_i instead (Sec. 4.1; A = the
// projection plane, box_rows of each 128-row tile loaded, K = m_pad, no Z
// rows), written to the tree scratch as k_tc.cuh writes it.
template <int NT, bool PROJ>
__global__ void __launch_bounds__(TCP_THREADS, 1)
    k_expand_tcp(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX, int use_tmx,
                 const __grid_constant__ CUtensorMap tmZ, int zhb, MatView mv, Scratch ws, int64_t r, const void* X,
                 int64_t ldx, int xt, void* Y, int64_t ldy, int yt, int tgroups, int nchunks, int nitems, int nK,
                 int nX, int nst, int mt, int box_rows) {
  constexpr int A_BYTES = TC_M * TC_KC * 2;
  constexpr int BCH = NT * 128;
  constexpr uint32_t IDESC = idesc_bf16(TC_M, NT);
  constexpr int TPT = tc_ncols<false, NT>();          // tensor-memory columns of one tile
  pdl_launch_dependents();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw_s = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  const int SB = mt * A_BYTES + BCH;
  const int ke = PROJ ? 0 : mv.Ke;                   // Z rows of the operand
  const int ke4 = tcp_ke4(ke);
  float* zr = reinterpret_cast<float*>(base + static_cast<size_t>(nst) * SB);
  uint8_t* ctl = base + static_cast<size_t>(nst) * SB + static_cast<size_t>(NT) * ke4 * 4;
  const uint32_t full0 = smem_u32(ctl);                          // nst barriers, 2 arrivals + bytes
  const uint32_t empty0 = full0 + 8 * TCP_MAX_STAGES;            // nst barriers, MMA commit
  const uint32_t accf0 = full0 + 16 * TCP_MAX_STAGES;            // 2 barriers, MMA commit
  const uint32_t acce0 = accf0 + 16;                             // 2 barriers, every epilogue thread
  const uint32_t fin = acce0 + 16;                               // the MMA thread's last commit
  const uint32_t zbar = fin + 8;                                 // bulk copies of the Z block
  const uint32_t bfree0 = full0 + 256;                           // nst barriers, producer: "B of this use is yours"
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ctl + 16 * TCP_MAX_STAGES + 48);    // after fin (bytes 160..167)
  volatile int* s_dead = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* s_flag = s_dead + 1;
  volatile int* s_issued = s_dead + 2;                           // stages whose A copies were requested
  volatile int* s_zflag = s_dead + 3;                            // the Z block arrived (stager thread 0)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* err = ws.err;
  const uint32_t ACC = static_cast<uint32_t>(mt * TPT);          // columns of one accumulator set
  const uint32_t NCOL = 2 * ACC;
  const int G = gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(full0 + 8 * s, 2);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 128 * TCP_EPI_WG);
    }
    mbar_init(fin, 1);
    mbar_init(zbar, 1);
    for (int s = 0; s < nst; ++s) mbar_init(bfree0 + 8 * s, 1);
    *s_dead = 0;
    *s_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tslot), NCOL);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      int g = 0;
      for (int it = blockIdx.x; it < nitems && !*s_dead; it += G) {
        const TcpItem w = tcp_item(mv, it, tgroups, nchunks, NT, mt, PROJ);
        if (!w.valid) continue;
        const bool x_tma = use_tmx && xt == HM_BF16 && w.m == mv.m_pad && (w.a0 & 7) == 0;
        const int nXt = x_tma ? nX : 0;
        const int a_row = PROJ ? w.leaf * mv.Kp + w.t0 : static_cast<int>(w.a0 + w.t0);
        for (int c = 0; c < nK; ++c, ++g) {
          const int s = g % nst;
          const int u = g / nst;
          if (u > 0 && !mbar_wait(empty0 + 8 * s, (u - 1) & 1, err, 41)) {
            *s_dead = 1;
            break;
          }
          const uint32_t st = smem_u32(base + static_cast<size_t>(s) * SB);
          const uint32_t bytes = static_cast<uint32_t>(mt * (PROJ ? box_rows * TC_KC * 2 : A_BYTES) + (c < nXt ? BCH : 0));
          mbar_expect_tx(full0 + 8 * s, bytes);                 // arrival 1: the A tiles (and X)
          for (int t = 0; t < mt; ++t) tma_load_2d(st + t * A_BYTES, &tmA, c * TC_KC, a_row + t * TC_M, full0 + 8 * s);
          if (c < nXt) {
            tma_load_2d(st + mt * A_BYTES, &tmX, static_cast<int>(w.a0) + c * TC_KC, w.col0, full0 + 8 * s);
            mbar_arrive1(full0 + 8 * s);                          // arrival 2: B comes with the copies
          } else {
            // the stagers write this use's B: the slot is free (the empty wait
            // above) and its full barrier is in this use's phase
            mbar_arrive1(bfree0 + 8 * s);
          }
          *s_issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issue ----
    if (lane == 0) {
      int g = 0, kk = 0;
      for (int it = blockIdx.x; it < nitems && !*s_dead; it += G) {
        const TcpItem w = tcp_item(mv, it, tgroups, nchunks, NT, mt, PROJ);
        if (!w.valid) continue;
        const int b = kk & 1;
        const int ub = kk >> 1;
        if (ub > 0 && !mbar_wait(acce0 + 8 * b, (ub - 1) & 1, err, 43)) {
          *s_dead = 1;
          break;
        }
        tc_fence_after();
        const uint32_t dacc = tmem + static_cast<uint32_t>(b) * ACC;
        bool ok = true;
        for (int c = 0; c < nK; ++c, ++g) {
          const int s = g % nst;
          if (!mbar_wait(full0 + 8 * s, (g / nst) & 1, err, 44)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_addr = smem_u32(base + static_cast<size_t>(s) * SB);
          const uint32_t b_addr = a_addr + mt * A_BYTES;
#pragma unroll
          for (int k = 0; k < TC_KC / 16; ++k) {
            const uint64_t bd = sw128_desc(b_addr + k * 32);
            const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
            for (int t = 0; t < mt; ++t)
              umma_bf16(dacc + t * TPT, sw128_desc(a_addr + t * A_BYTES + k * 32), bd, IDESC, acc);
          }
          umma_commit(empty0 + 8 * s);                          // the stage is free once these MMAs finish
        }
        if (!ok) {
          *s_dead = 1;
          break;
        }
        umma_commit(accf0 + 8 * b);                             // the item's accumulators are complete
        ++kk;
      }
      umma_commit(fin);                                         // arrives when every MMA issued here is done
    }
    __syncwarp();
  } else if (warp < 4) {
    // ---- B chunks TMA does not bring ----
    const int stid = threadIdx.x - 64;
    int bcount[TCP_MAX_STAGES] = {0, 0, 0, 0, 0, 0, 0, 0};       // uses of each slot the stagers filled
    bool waited = false;
    int g = 0;
    bool stop = false;
    int zitem = -1;                                             // item whose Z block was requested into zr
    const bool zbulk = zhb > 0;                                 // Z block by tensor boxes
    bool zpend = false;                                         // bulk copies in flight on zbar
    int zphase = 0;
    // some chunk holds only Z (and zero) rows: the ones converted from the Z block
    const bool zany = ((mv.m_pad + TC_KC - 1) / TC_KC) * TC_KC < mv.m_pad + ke;
    for (int it = blockIdx.x; it < nitems && !stop; it += G) {
      const TcpItem w = tcp_item(mv, it, tgroups, nchunks, NT, mt, PROJ);
      if (!w.valid) continue;
      const bool x_tma = use_tmx && xt == HM_BF16 && w.m == mv.m_pad && (w.a0 & 7) == 0;
      const int nXt = x_tma ? nX : 0;
      bool zready = false;
      for (int c = 0; c < nK; ++c, ++g) {
        if (c < nXt) continue;
        const int s = g % nst;
        if (stid == 0) {
          // The producer's signal for this use of the slot; its phase count is
          // the stagers' own count of the slot's uses they fill.  Waiting on
          // the empty barrier instead could run two or more phases ahead of
          // it (the chunks TMA fills pass without the stagers), and a parity
          // wait cannot tell a phase from the one two before it: it returned
          // while the MMAs still read the slot.
          int ok = *s_dead ? 0 : 1;
          if (ok && !mbar_wait(bfree0 + 8 * s, bcount[s] & 1, err, 42)) {
            ok = 0;
            *s_dead = 1;
          }
          ++bcount[s];
          *s_flag = ok;
        }
        named_bar_sync(2, 64);
        if (!*s_flag) {                                         // the same value for all 64 threads
          stop = true;
          break;
        }
        const bool zrows = (c + 1) * TC_KC > mv.m_pad && c * TC_KC < mv.m_pad + ke;
        if (zrows && !waited) {
          pdl_wait();                                           // Z is written by the tree kernels
          waited = true;
        }
        const bool zfast = c * TC_KC >= mv.m_pad;               // Z and zero rows only
        if (zrows && zfast && !zready) {
          if (zitem != it) {
            fence_proxy_async();
            if (zbulk) {
              named_bar_sync(2, 64);                            // every thread's fence before the copies
              if (stid == 0) tcp_z_fetch_tma(zr, zbar, &tmZ, mv, r, w.leaf, w.col0, NT, zhb);
            } else {
              tcp_z_fetch<NT>(zr, mv, ws, r, w.leaf, w.col0, stid);
            }
            zpend = zbulk;
          }
          if (stid == 0) *s_zflag = 1;
          if (zpend) {
            if (stid == 0 && !mbar_wait(zbar, zphase & 1, err, 46)) {
              *s_zflag = 0;
              *s_dead = 1;
            }
            ++zphase;
            zpend = false;
          } else {
            cp_async_commit_wait_all();
          }
          named_bar_sync(2, 64);
          if (!*s_zflag) {                                      // written before the barrier: the same for all
            stop = true;
            break;
          }
          zready = true;
          zitem = it;
        }
        uint8_t* sb = base + static_cast<size_t>(s) * SB + mt * A_BYTES;
        if (zfast) {
          tcp_z_convert<NT>(sb, zr, mv.Ke, zbulk ? zhb : 4, c * TC_KC - mv.m_pad, stid);
        } else {
          // stage_b addresses chunk c at c * BCH from its base
          stage_b<false, NT>(sb - static_cast<size_t>(c) * BCH, nullptr, c * TC_KC, (c + 1) * TC_KC, stid, 64, mv, ws,
                             r, w.leaf, w.a0, w.m, ke, w.col0, X, ldx, xt);
        }
        fence_proxy_async();
        named_bar_sync(2, 64);
        if (stid == 0) mbar_arrive1(full0 + 8 * s);             // arrival 2: B is in place
      }
      if (stop) break;
      // request the next item's Z block while this item is multiplied (zr is
      // free: this item's chunks are converted, behind the barrier above)
      if (waited && zany) {
        for (int it2 = it + G; it2 < nitems; it2 += G) {
          const TcpItem w2 = tcp_item(mv, it2, tgroups, nchunks, NT, mt, PROJ);
          if (!w2.valid) continue;
          fence_proxy_async();                                  // this item's reads of zr before the copies
          if (zbulk) {
            named_bar_sync(2, 64);                              // every thread's fence before the copies
            if (stid == 0) tcp_z_fetch_tma(zr, zbar, &tmZ, mv, r, w2.leaf, w2.col0, NT, zhb);
            zpend = true;
          } else {
            tcp_z_fetch<NT>(zr, mv, ws, r, w2.leaf, w2.col0, stid);
            asm volatile("cp.async.commit_group;" ::: "memory");
          }
          zitem = it2;
          break;
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (zpend && stid == 0) mbar_wait(zbar, zphase & 1, nullptr, 0);   // no copy outlives the block
    if (!waited) pdl_wait();
  } else {
    // ---- epilogue ----
    const int ew = warp & 3;                                    // tensor-memory lane quarter
    const int wg = (warp - 4) >> 2;                             // which share of the column blocks
    const int row = ew * 32 + lane;
    int kk = 0;
    for (int it = blockIdx.x; it < nitems; it += G) {
      const TcpItem w = tcp_item(mv, it, tgroups, nchunks, NT, mt, PROJ);
      if (!w.valid) continue;
      const int b = kk & 1;
      const int ub = kk >> 1;
      int okv = 0;
      if (lane == 0) okv = (!*s_dead && mbar_wait(accf0 + 8 * b, ub & 1, err, 45)) ? 1 : 0;
      okv = __shfl_sync(0xffffffffu, okv, 0);
      if (!okv) {
        if (lane == 0) *s_dead = 1;
        break;
      }
      tc_fence_after();
      const uint32_t lane_addr = tmem + static_cast<uint32_t>(b) * ACC + (static_cast<uint32_t>(ew * 32) << 16);
      const int node = mv.L - 1 + w.leaf;
      const int ldo = (mv.kind == HM_HODLR) ? mv.Ke : mv.Kp;
      float* pout = static_cast<float*>(mv.kind == HM_HODLR ? ws.PS : ws.xh);
      for (int t = 0; t < mt; ++t) {
        const int tu = w.t0 + t * TC_M;
        const int nrows = (PROJ ? mv.Kp : w.m) - tu;
        for (int cb = wg * 16; cb < NT; cb += 16 * TCP_EPI_WG) {
          float v[16];
          tmem_ld16(lane_addr + t * TPT + cb, v);
          if (row < nrows) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int64_t col = w.col0 + cb + j;
              if (col < r) {
                if constexpr (PROJ) {
                  pout[(static_cast<int64_t>(node) * r + col) * ldo + tu + row] = v[j];
                } else {
                  const int64_t idx = (w.a0 + tu + row) + col * ldy;
                  if (yt == HM_F64) static_cast<double*>(Y)[idx] = v[j];
                  else static_cast<float*>(Y)[idx] = v[j];
                }
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive1(acce0 + 8 * b);
      ++kk;
    }
  }

  __syncthreads();
  if (threadIdx.x == 32) {
    // every MMA issued by this CTA has finished (its last commit), then, after
    // a timeout, the copies still in flight into the ring
    mbar_wait(fin, 0, nullptr, 0);
    if (*s_dead) {
      const int hi = *s_issued;
      for (int u = (hi > nst ? hi - nst : 0); u < hi; ++u)
        mbar_wait(full0 + 8 * (u % nst), (u / nst) & 1, nullptr, 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, NCOL);
  }
}

}  // namespace hmi

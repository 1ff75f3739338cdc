// The whole tree part of one product in one launch of thread-block clusters
// (Sec. 4.1, Fig. 4.1): for HSS the upsweep x-hat_q = R_V^T [x-hat_a; x-hat_b]
// with the couplings y_a = B12 x-hat_b, y_b = B21 x-hat_a (Eq. 2.2), then the
// downsweep y-hat_c = R_U(c) y-hat_q + y_c; for HODLR the per-level sums of
// the leaves' projections.
//
// One cluster of CL = 2^s CTAs per chunk of RC right-hand-side columns.  CTA j
// owns the subtree below node j of level s: it runs those levels of both
// sweeps in its own shared memory with block barriers only.  The s levels
// above are shared out among the CTAs (node t of level l belongs to CTA
// t << (s - l)); operands owned by another CTA are read through distributed
// shared memory after a cluster barrier.  So a product pays one cluster
// barrier per top level instead of one global-memory handoff (fence, atomic,
// L2 round trip) per level.
//
// HSS operators stream through a ring of NS shared-memory slots filled by
// cp.async.bulk copies in the order the CTA uses them (the first NS before
// griddepcontrol.wait, overlapping the previous kernel).  The small products
// run as warp tasks: a warp computes 32 output rows of one operator for all
// RC columns (each lane a register tile of up to 4 rows by 2 columns, so a
// step reads one 16-byte operator segment and one vector pair per lane).
// A warp waits on the mbarrier of its own
// slot; the warp that finishes the last task of a slot refills it, so the
// ring runs ahead across level boundaries.  Every sum runs in the same order
// as in the level kernels (fma over j from zero, then + y_c; paired FMAs
// round each half exactly like fmaf), so both give identical bits.  Every
// wait is bounded (the library's device wait limit, 2 s of %globaltimer by
// default): on expiry the kernel records an error code in the library's
// error word and stops waiting.
#include <algorithm>
#include <type_traits>

#include "hm_api_internal.h"
#include "k_tc.cuh"

namespace hmi {

constexpr int TREE_THREADS = 256;
constexpr int TREE_MAX_S = 4;          // clusters of up to 16 CTAs (16: non-portable size)
constexpr int TREE_MAX_NS = 12;
constexpr int TREE_MAX_ITEMS = 1040;     // node ids and consumer counts (half each)

__device__ __forceinline__ uint32_t cluster_map(uint32_t saddr, int rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(saddr), "r"(rank));
  return out;
}

__device__ __forceinline__ uint4 ld_cluster16(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// Copies `units` 16-byte units from CTA `rank`'s shared memory at the same
// offset as `src` into local `dst` (block-wide).
__device__ __forceinline__ void pull_remote(void* dst, const void* src, int rank, int units) {
  const uint32_t base = cluster_map(smem_u32(src), rank);
  uint4* d = static_cast<uint4*>(dst);
  for (int u = threadIdx.x; u < units; u += blockDim.x) d[u] = ld_cluster16(base + 16u * u);
}

// Shared-memory plan of one tree launch (offsets in bytes from a 128-byte
// aligned base; every node vector is [j][c], K rows of RC columns).
struct TreeLayout {
  int s, d, K, NS;
  uint32_t slot;                       // bytes per operator slot
  uint32_t ctl, items, ring, A, B, TX, CH, TYC, TYF, STG, total;
};

template <typename C>
__host__ __device__ inline uint32_t vec_bytes(int K, int RC) {
  return static_cast<uint32_t>(K) * RC * sizeof(C);
}

// Control block: NS full barriers (8 bytes each), NS slot counters, NS
// "item held by the slot" words, the `dead` flag and the number of requests.
__host__ __device__ inline uint32_t ctl_bytes() { return 8 * TREE_MAX_NS + 8 * TREE_MAX_NS + 16; }

// s: levels shared by the cluster (2^s CTAs), at most p.
template <typename C>
__host__ __device__ inline TreeLayout tree_layout(bool hss, int p, int Kp, int Ke, int RC, int NS, int s) {
  TreeLayout t;
  t.s = p < s ? p : s;
  t.d = p - t.s;
  t.K = Kp > Ke ? Kp : Ke;
  t.NS = hss ? NS : 0;
  const uint32_t up = static_cast<uint32_t>(2 * Kp * Kp + 2 * Kp * Ke) * sizeof(C);
  const uint32_t dn = static_cast<uint32_t>(2 * Ke * Ke) * sizeof(C);
  t.slot = hss ? (((up > dn ? up : dn) + 127u) & ~127u) : 0u;
  const uint32_t v = vec_bytes<C>(t.K, RC);
  const uint32_t nleaf = 1u << t.d;
  uint32_t o = 0;
  t.ctl = o;   o += ctl_bytes();
  t.items = o; o += hss ? 4 * TREE_MAX_ITEMS : 0;
  o = (o + 127u) & ~127u;
  t.ring = o;  o += t.NS * t.slot;
  t.A = o;     o += nleaf * v;
  t.B = o;     o += (nleaf > 1 ? nleaf / 2 : 1) * v;
  t.TX = o;    o += (t.s + 1) * v;               // x-hat (HODLR: T) of the owned node per top level
  t.CH = o;    o += 2 * v;                       // stacked children of a top node
  t.TYC = o;   o += hss ? 2 * (t.s + 1) * v : 0; // couplings of the children of owned top nodes
  t.TYF = o;   o += hss ? (t.s + 1) * v : 0;     // y-hat of owned top nodes
  t.STG = o;   o += 2 * v;                       // remote operands
  t.total = o;
  return t;
}

// The RC values of row j of a node vector.
template <typename C, int RC>
__device__ __forceinline__ void load_row(const C* __restrict__ v, C (&x)[RC]) {
  if constexpr (std::is_same<C, float>::value && RC % 4 == 0) {
#pragma unroll
    for (int u = 0; u < RC / 4; ++u) {
      const float4 t = reinterpret_cast<const float4*>(v)[u];
      x[4 * u] = t.x; x[4 * u + 1] = t.y; x[4 * u + 2] = t.z; x[4 * u + 3] = t.w;
    }
  } else if constexpr (std::is_same<C, double>::value && RC % 2 == 0) {
#pragma unroll
    for (int u = 0; u < RC / 2; ++u) {
      const double2 t = reinterpret_cast<const double2*>(v)[u];
      x[2 * u] = t.x; x[2 * u + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < RC; ++c) x[c] = v[c];
  }
}

// Register tile of a warp task over a group of CW of the RC columns (CW in
// {1, 2, 4, 8}, CW <= RC): lane (rb, cb) owns rows rb*RT .. rb*RT+RT-1 and
// columns cb*CT .. cb*CT+CT-1 of the group, so a step j reads one operator
// row (RT contiguous values per lane) and one vector row (CT per lane) with
// few shared-memory wavefronts.  Narrow groups give a level with few
// products more warp tasks; every output's sum is the same whatever CW is.
template <int CW>
struct WTile {
  static constexpr int CT = CW >= 2 ? 2 : 1;
  static constexpr int RT = CW / CT;
  static constexpr int NRB = 32 / RT;   // row blocks per warp
};

template <typename C, int N>
__device__ __forceinline__ void ld_vec(const C* __restrict__ p, C (&x)[N]) {
  if constexpr (sizeof(C) * N == 16) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    memcpy(x, &t, 16);
  } else if constexpr (sizeof(C) * N == 8) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    memcpy(x, &t, 8);
  } else if constexpr (sizeof(C) * N == 32) {
    const uint4 t0 = reinterpret_cast<const uint4*>(p)[0];
    const uint4 t1 = reinterpret_cast<const uint4*>(p)[1];
    memcpy(x, &t0, 16);
    memcpy(reinterpret_cast<char*>(x) + 16, &t1, 16);
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) x[q] = p[q];
  }
}

// acc[r][c] += sum over j < kj, in order, of M[j*ko + i0 + r] v[j][c0 + c]
// (M, v in shared memory; v rows have RC values); groups of G steps load
// before they multiply.
template <typename C, int RC, int CW>
__device__ __forceinline__ void tile_acc(const C* __restrict__ M, int ko, int kj, int i0, const C* __restrict__ v,
                                         int c0, C (&acc)[WTile<CW>::RT][WTile<CW>::CT]) {
  constexpr int RT = WTile<CW>::RT, CT = WTile<CW>::CT;
  constexpr int G = 8;
  int j = 0;
  for (; j + G <= kj; j += G) {
    C m[G][RT];
    C x[G][CT];
#pragma unroll
    for (int u = 0; u < G; ++u) ld_vec<C, RT>(M + (j + u) * ko + i0, m[u]);
#pragma unroll
    for (int u = 0; u < G; ++u) ld_vec<C, CT>(v + (j + u) * RC + c0, x[u]);
#pragma unroll
    for (int u = 0; u < G; ++u) {
      if constexpr (std::is_same<C, float>::value && CT == 2) {
        const float2 xx = make_float2(x[u][0], x[u][1]);
#pragma unroll
        for (int r = 0; r < RT; ++r) {
          const float2 o = __ffma2_rn(make_float2(m[u][r], m[u][r]), xx, make_float2(acc[r][0], acc[r][1]));
          acc[r][0] = o.x;
          acc[r][1] = o.y;
        }
      } else {
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
          for (int c = 0; c < CT; ++c) acc[r][c] = fma(m[u][r], x[u][c], acc[r][c]);
      }
    }
  }
  for (; j < kj; ++j) {
    C m[RT], x[CT];
    ld_vec<C, RT>(M + j * ko + i0, m);
    ld_vec<C, CT>(v + j * RC + c0, x);
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[r][c] = fma(m[r], x[c], acc[r][c]);
  }
}

// One warp task: rows row0 .. row0+31 and columns cg*CW .. cg*CW+CW-1 of
// out = M^T v (+ add), where row j of v is va[j] for j < ka and vb[j - ka]
// after (the stacked children of R_V).  M and v in shared memory; out and
// add ([i][c] blocks of RC columns) in shared or global memory.  Split in
// two: wt_compute reads add (before the sums, so a global read overlaps
// them) and the operands into registers; wt_store writes the result, after
// the caller has released the operator slot.  Rows come in multiples of 8.
template <typename C, int CW>
struct WTResult {
  C acc[WTile<CW>::RT][WTile<CW>::CT];
  int i0, c0;
  bool active;
};

template <typename C, int RC, int CW>
__device__ __forceinline__ void wt_compute(WTResult<C, CW>& w, const C* M, int ko, int kj, const C* va, int ka,
                                           const C* vb, const C* add, int row0, int cg) {
  constexpr int RT = WTile<CW>::RT, CT = WTile<CW>::CT, NRB = WTile<CW>::NRB;
  const int lane = threadIdx.x & 31;
  w.i0 = row0 + (lane % NRB) * RT;
  w.c0 = cg * CW + (lane / NRB) * CT;
  w.active = w.i0 < ko;                  // ko is a multiple of 8, so rows i0 .. i0+RT-1 all exist
  if (!w.active) return;
  C a[RT][CT];
  if (add) {
#pragma unroll
    for (int r = 0; r < RT; ++r) ld_vec<C, CT>(add + (w.i0 + r) * RC + w.c0, a[r]);
  }
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < CT; ++c) w.acc[r][c] = C(0);
  tile_acc<C, RC, CW>(M, ko, ka < kj ? ka : kj, w.i0, va, w.c0, w.acc);
  if (kj > ka) tile_acc<C, RC, CW>(M + ka * ko, ko, kj - ka, w.i0, vb, w.c0, w.acc);
  if (add) {
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int c = 0; c < CT; ++c) w.acc[r][c] = w.acc[r][c] + a[r][c];
  }
}

template <typename C, int RC, int CW>
__device__ __forceinline__ void wt_store(const WTResult<C, CW>& w, C* out) {
  constexpr int RT = WTile<CW>::RT, CT = WTile<CW>::CT;
  if (!w.active) return;
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < CT; ++c) out[(w.i0 + r) * RC + w.c0 + c] = w.acc[r][c];
}

// Operator ring.  items[k]: node id | kind << 30 (0 upsweep record R_V, B12,
// B21; 1 downsweep record R_U); cons[k]: the warp tasks that read item k.
struct Ring {
  uint8_t* slots;
  uint64_t* full;
  int* cnt;
  int* held;                // item whose copy was last requested into the slot
  int* dead;
  int* issued;
  const int* items;
  const int* cons;          // tasks that read item k
  int* err;
  int NS, count;
  uint32_t slot_bytes;
};

template <typename C>
__device__ void ring_issue(const Ring& R, const MatView& mv, int k) {
  if (k >= R.count) return;
  const int it = R.items[k];
  const int q = it & 0x3fffffff;
  const bool down = (it >> 30) & 1;
  const int s = k % R.NS;
  const uint32_t dst = smem_u32(R.slots + static_cast<size_t>(s) * R.slot_bytes);
  const uint32_t bar = smem_u32(R.full + s);
  const int Kp = mv.Kp, Ke = mv.Ke;
  *R.issued = k + 1;
  // the slot's barrier phase now belongs to item k (a reader that sees this
  // before the expect_tx below still waits for the copy: the phase is open)
  *reinterpret_cast<volatile int*>(R.held + s) = k;
  if (!down) {
    const uint32_t brv = static_cast<uint32_t>(2 * Kp * Kp) * sizeof(C);
    const uint32_t bb = static_cast<uint32_t>(Kp * Ke) * sizeof(C);
    mbar_expect_tx(bar, brv + 2 * bb);
    bulk_g2s(dst, static_cast<const C*>(mv.RV) + static_cast<int64_t>(q) * 2 * Kp * Kp, brv, bar);
    bulk_g2s(dst + brv, static_cast<const C*>(mv.B12) + static_cast<int64_t>(q) * Kp * Ke, bb, bar);
    bulk_g2s(dst + brv + bb, static_cast<const C*>(mv.B21) + static_cast<int64_t>(q) * Kp * Ke, bb, bar);
  } else {
    const uint32_t bu = static_cast<uint32_t>(2 * Ke * Ke) * sizeof(C);
    mbar_expect_tx(bar, bu);
    bulk_g2s(dst, static_cast<const C*>(mv.RU) + static_cast<int64_t>(q) * 2 * Ke * Ke, bu, bar);
  }
}

// Called by a whole warp before its task on item k.  The slot may still hold
// an older item (k - NS, ...): a parity wait is only meaningful once the
// slot's current phase is item k's, so first wait (bounded) until item k has
// been requested into the slot, then (bounded) for its bytes.
__device__ __forceinline__ void ring_acquire(const Ring& R, int k, int* err) {
  if ((threadIdx.x & 31) == 0 && !*(volatile int*)R.dead) {
    const int s = k % R.NS;
    const volatile int* held = R.held + s;
    bool ok = (*held == k);
    if (!ok) {
      const uint64_t t0 = gtimer();
      const uint64_t limit = wait_limit_ns(err);
      while (!(ok = (*held == k))) {
        if (gtimer() - t0 > limit) {
          atomicExch(err, 22);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence_block();
    if (!ok || !mbar_wait(smem_u32(R.full + s), (k / R.NS) & 1, err, 21)) *(volatile int*)R.dead = 1;
  }
  __syncwarp();
}

// Called by a whole warp after its task on item k: the last reader of the
// slot requests item k + NS into it.
template <typename C>
__device__ __forceinline__ void ring_release(const Ring& R, const MatView& mv, int k) {
  __syncwarp();                                // every lane is done reading the slot
  if ((threadIdx.x & 31) == 0) {
    const int s = k % R.NS;
    // acquire-release: this warp's reads of the slot happen before the count,
    // and the last reader sees every other reader's count
    int old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.s32 %0, [%1], 1;"
                 : "=r"(old)
                 : "r"(smem_u32(R.cnt + s))
                 : "memory");
    if (old + 1 > R.cons[k]) {                 // more readers than the item has: protocol broken
      atomicExch(R.err, 23);
      *(volatile int*)R.dead = 1;
    } else if (old + 1 == R.cons[k]) {
      R.cnt[s] = 0;
      fence_proxy_async();                     // the slot's generic reads before the copy that overwrites it
      if (!*(volatile int*)R.dead) ring_issue<C>(R, mv, k + R.NS);
    }
  }
}

// ld: rows per column in global memory (a multiple of 8); K: row stride of a
// node in A.  16-byte loads, up to 8 in flight per thread, then the
// transposing stores (consecutive threads take consecutive columns, so the
// stores of a warp hit consecutive words).
template <typename C, int RC>
__device__ void load_leaves(C* A, const C* src, int64_t r, int ld, int K, int first_node, int nleaf, int col0) {
  constexpr int E = 16 / sizeof(C);
  const int upc = ld / E;                      // 16-byte units per column of one node
  const int total = nleaf * RC * upc;
  for (int base = threadIdx.x; base < total; base += blockDim.x * 8) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (idx < total) {
        const int c = idx % RC;
        const int e = (idx / RC) % upc;
        const int t = idx / (upc * RC);
        const int64_t col = col0 + c;
        if (col < r)
          v[u] = __ldcg(reinterpret_cast<const uint4*>(src + (static_cast<int64_t>(first_node + t) * r + col) * ld) + e);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x;
      if (idx < total) {
        const int c = idx % RC;
        const int e = (idx / RC) % upc;
        const int t = idx / (upc * RC);
        const C* x = reinterpret_cast<const C*>(&v[u]);
#pragma unroll
        for (int q = 0; q < E; ++q) A[(t * K + e * E + q) * RC + c] = x[q];
      }
    }
  }
}

// Order in which a cluster visits the n nodes (or parents) of one level:
// rotated by the column chunk, so the clusters of a launch, which all need
// the same operators, read different ones at a time (no hot L2 lines).
__device__ __forceinline__ int level_perm(int t, int n) {
  const int rot = static_cast<int>((static_cast<int64_t>(blockIdx.y) * n) / gridDim.y);
  return (t + rot) & (n - 1);
}

// Column-group width of a level with `tasks` full-width warp tasks.  Always
// the full RC: narrower groups give idle warps work but keep each task's
// dependent chain over j just as long, and multiply the slot handoffs
// (measured slower on the small top levels), so they are not used.
template <int RC>
__device__ __forceinline__ int pick_cw(int tasks, int nwarps) {
  (void)tasks;
  (void)nwarps;
  return RC;
}

enum { LV_UP = 0, LV_TOPUP = 1, LV_TOPDOWN = 2, LV_DOWN = 3 };

// Everything a level's warp tasks need.
template <typename C>
struct LevelArgs {
  int kind;
  int k;              // first item of the level
  int n;              // nodes (LV_UP), 1 (top), children (LV_DOWN)
  int lev, first;     // level; first node (LV_UP) or first child (LV_DOWN) of the CTA's part
  int nbp, nbe;       // 32-row blocks of the R_V and of the Ke-row outputs
  int h;              // LV_TOPDOWN: child half
  const C* cur;       // LV_UP: children x-hat; LV_TOPUP: stacked children; LV_TOPDOWN/DOWN: parent y-hat
  C* out;             // LV_UP: x-hat of the level; LV_TOPUP: x-hat (TX); LV_TOPDOWN/DOWN: y-hat
  C* tyc;             // LV_TOPUP: the two coupling outputs (TYC), LV_TOPDOWN: the coupling input
  C* ycg;             // subtree couplings in scratch (node blocks of Ke x RC)
  int VS;
};

// Runs the warp tasks of one level with column groups of CW: task w covers
// product (w / ncg), column group (w % ncg), in item order per warp.
template <typename C, int RC, int CW>
__device__ void run_level(const Ring& R, const MatView& mv, int* err, const LevelArgs<C>& a) {
  constexpr int ncg = RC / CW;
  const int Kp = mv.Kp, Ke = mv.Ke;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int KeRC = Ke * RC;
  int per;                                      // full-width tasks per item
  int nitems_tasks;
  if (a.kind == LV_UP || a.kind == LV_TOPUP) {
    per = (a.lev > 0 ? a.nbp : 0) + 2 * a.nbe;
    nitems_tasks = a.n * per;
  } else if (a.kind == LV_TOPDOWN) {
    per = a.nbe;
    nitems_tasks = per;
  } else {
    per = 2 * a.nbe;                            // a parent's record serves both children
    nitems_tasks = (a.n / 2) * per;
  }
  for (int w = warp; w < nitems_tasks * ncg; w += nwarps) {
    const int cg = w % ncg;
    const int tw = w / ncg;                     // full-width task
    const int iu = tw / per;                    // item within the level
    int b = tw % per;
    const int item = a.k + iu;
    ring_acquire(R, item, err);
    const C* op = reinterpret_cast<const C*>(R.slots + static_cast<size_t>(item % R.NS) * R.slot_bytes);
    WTResult<C, CW> res;
    C* dst;
    if (a.kind == LV_UP || a.kind == LV_TOPUP) {
      const int t = (a.kind == LV_UP) ? level_perm(iu, a.n) : 0;
      const C* xa = a.cur + static_cast<size_t>(2 * t) * a.VS;
      const C* xb = xa + a.VS;
      if (a.lev > 0 && b < a.nbp) {
        wt_compute<C, RC, CW>(res, op, Kp, 2 * Kp, xa, Kp, xb, nullptr, 32 * b, cg);
        dst = a.out + static_cast<size_t>(t) * a.VS;
      } else {
        if (a.lev > 0) b -= a.nbp;
        const int side = b < a.nbe ? 0 : 1;     // 0: B12 x-hat_b -> y_a, 1: B21 x-hat_a -> y_b
        const int rb = side ? b - a.nbe : b;
        wt_compute<C, RC, CW>(res, op + 2 * Kp * Kp + side * Kp * Ke, Ke, Kp, side ? xa : xb, Kp, side ? xa : xb,
                              nullptr, 32 * rb, cg);
        if (a.kind == LV_UP) dst = a.ycg + static_cast<int64_t>(2 * (a.first + t) + 1 + side) * KeRC;
        else dst = a.tyc + static_cast<size_t>(side) * a.VS;
      }
    } else if (a.kind == LV_TOPDOWN) {
      wt_compute<C, RC, CW>(res, op + a.h * Ke * Ke, Ke, Ke, a.cur, Ke, a.cur, a.tyc, 32 * b, cg);
      dst = a.out;
    } else {
      const int u = level_perm(iu, a.n / 2);
      const int hh = b / a.nbe;
      b -= hh * a.nbe;
      const int t = 2 * u + hh;
      const C* yp = a.cur + static_cast<size_t>(u) * a.VS;
      wt_compute<C, RC, CW>(res, op + hh * Ke * Ke, Ke, Ke, yp, Ke, yp,
                            a.ycg + static_cast<int64_t>(a.first + t) * KeRC, 32 * b, cg);
      dst = a.out + static_cast<size_t>(t) * a.VS;
    }
    ring_release<C>(R, mv, item);
    wt_store<C, RC, CW>(res, dst);
  }
}

template <typename C, int RC>
__device__ void run_level_cw(const Ring& R, const MatView& mv, int* err, const LevelArgs<C>& a, int cw) {
  if constexpr (RC >= 8) {
    if (cw == 8) { run_level<C, RC, 8>(R, mv, err, a); return; }
  }
  if constexpr (RC >= 4) {
    if (cw == 4) { run_level<C, RC, 4>(R, mv, err, a); return; }
  }
  if constexpr (RC >= 2) {
    run_level<C, RC, 2>(R, mv, err, a);
    return;
  }
  run_level<C, RC, 1>(R, mv, err, a);
}

template <typename C, int RC>
__global__ void __launch_bounds__(TREE_THREADS, 2) k_tree_cluster(MatView mv, Scratch ws, int64_t r, int NS, int S) {
  pdl_launch_dependents();
  extern __shared__ __align__(128) uint8_t tree_smem_raw[];
  uint8_t* tree_smem = tree_smem_raw + ((128u - (smem_u32(tree_smem_raw) & 127u)) & 127u);
  const bool hss = (mv.kind == HM_HSS);
  const TreeLayout T = tree_layout<C>(hss, mv.p, mv.Kp, mv.Ke, RC, NS, S);
  const int s = T.s, d = T.d, p = mv.p;
  const int Kp = mv.Kp, Ke = mv.Ke;
  const int j = blockIdx.x;                  // rank in the cluster (grid.x = cluster size)
  const int col0 = blockIdx.y * RC;
  const int nleaf = 1 << d;
  const uint32_t V = vec_bytes<C>(T.K, RC);
  const int VS = T.K * RC;                   // elements per node vector
  const int nwarps = blockDim.x >> 5;
  C* A = reinterpret_cast<C*>(tree_smem + T.A);
  C* Bb = reinterpret_cast<C*>(tree_smem + T.B);
  // couplings of the subtree's nodes: global scratch after y-hat, one Ke x RC
  // block per (column chunk, node); written by the upsweep, read back by the
  // downsweep of the same CTA
  const int64_t nodes = 2 * static_cast<int64_t>(mv.L) - 1;
  C* YCg = static_cast<C*>(ws.yf) + nodes * r * Ke + static_cast<int64_t>(blockIdx.y) * nodes * Ke * RC;
  auto vec = [&](uint32_t off, int idx) {
    return reinterpret_cast<C*>(tree_smem + off + static_cast<size_t>(idx) * V);
  };
  const int nbp = (Kp + 31) / 32, nbe = (Ke + 31) / 32;   // 32-row blocks of an output

  Ring R;
  R.full = reinterpret_cast<uint64_t*>(tree_smem + T.ctl);
  R.cnt = reinterpret_cast<int*>(tree_smem + T.ctl + 8 * TREE_MAX_NS);
  R.held = R.cnt + TREE_MAX_NS;
  R.dead = R.held + TREE_MAX_NS;
  R.issued = R.dead + 1;
  int* items = reinterpret_cast<int*>(tree_smem + T.items);
  int* cons = items + TREE_MAX_ITEMS / 2;
  R.items = items;
  R.cons = cons;
  R.err = ws.err;
  R.slots = tree_smem + T.ring;
  R.slot_bytes = T.slot;
  R.NS = T.NS;
  R.count = 0;

  // ---- operator order of this CTA (HSS) and the first NS requests ----
  if (threadIdx.x == 0) {
    *R.dead = 0;
    *R.issued = 0;
    if (hss) {
      int n = 0;
      // consumers of an item: its full-width warp tasks times the level's column groups
      for (int lev = p - 1; lev >= s; --lev) {                     // bottom upsweep
        const int per = (lev > 0 ? nbp : 0) + 2 * nbe;
        const int ncg = RC / pick_cw<RC>((1 << (lev - s)) * per, nwarps);
        for (int t = 0; t < (1 << (lev - s)); ++t) {
          items[n] = (1 << lev) - 1 + (j << (lev - s)) + level_perm(t, 1 << (lev - s));
          cons[n++] = per * ncg;
        }
      }
      for (int lev = s - 1; lev >= 0; --lev)                       // top upsweep, owned nodes
        if ((j & ((1 << (s - lev)) - 1)) == 0) {
          const int per = (lev > 0 ? nbp : 0) + 2 * nbe;
          items[n] = (1 << lev) - 1 + (j >> (s - lev));
          cons[n++] = per * (RC / pick_cw<RC>(per, nwarps));
        }
      for (int lev = 2; lev <= s; ++lev)                           // top downsweep: the parent's record
        if ((j & ((1 << (s - lev)) - 1)) == 0) {
          const int node = (1 << lev) - 1 + (j >> (s - lev));
          items[n] = (1 << 30) | ((node - 1) >> 1);
          cons[n++] = nbe * (RC / pick_cw<RC>(nbe, nwarps));
        }
      for (int lev = s + 1; lev <= p; ++lev) {                     // bottom downsweep: parents
        const int ncg = RC / pick_cw<RC>((1 << (lev - s)) * nbe, nwarps);
        for (int u = 0; u < (1 << (lev - 1 - s)); ++u) {
          items[n] = (1 << 30) | ((1 << (lev - 1)) - 1 + (j << (lev - 1 - s)) + level_perm(u, 1 << (lev - 1 - s)));
          cons[n++] = 2 * nbe * ncg;
        }
      }
      items[TREE_MAX_ITEMS / 2 - 1] = n;
      for (int k = 0; k < T.NS; ++k) {
        mbar_init(smem_u32(R.full + k), 1);
        R.cnt[k] = 0;
        R.held[k] = -1;
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  if (hss) {
    R.count = items[TREE_MAX_ITEMS / 2 - 1];
    if (threadIdx.x == 0)
      for (int k = 0; k < T.NS; ++k) ring_issue<C>(R, mv, k);
  }

  pdl_wait();                               // leaf projections come from the previous kernel
  C* data = static_cast<C*>(hss ? ws.xh : ws.PS);
  const int ld_leaf = hss ? Kp : Ke;
  load_leaves<C, RC>(A, data, r, ld_leaf, T.K, (1 << p) - 1 + j * nleaf, nleaf, col0);
  __syncthreads();

  int k = 0;                                // first item of the current level
  // ---- bottom upsweep: levels p-1 .. s inside the subtree ----
  C* cur = A;
  C* nxt = Bb;
  for (int lev = p - 1; lev >= s; --lev) {
    const int nn = 1 << (lev - s);
    const int first = (1 << lev) - 1 + (j << (lev - s));
    if (hss) {
      LevelArgs<C> la{LV_UP, k, nn, lev, first, nbp, nbe, 0, cur, nxt, nullptr, YCg, VS};
      run_level_cw<C, RC>(R, mv, ws.err, la, pick_cw<RC>(nn * ((lev > 0 ? nbp : 0) + 2 * nbe), nwarps));
      k += nn;
    } else {
      // HODLR: T_q = T_a + T_b over the rows of levels 1..lev; only the rows
      // of the node's own level leave shared memory (the expansion reads a
      // level-lev node's T only there, as the sibling's coupling term)
      const int rows = mv.koff[lev + 1];
      const int own0 = mv.koff[lev];
      for (int w = threadIdx.x; w < nn * rows * RC; w += blockDim.x) {
        const int c = w % RC;
        const int e = (w / RC) % rows;
        const int t = w / (RC * rows);
        const C* ch = cur + static_cast<size_t>(2 * t) * VS;
        const C v = ch[e * RC + c] + ch[VS + e * RC + c];
        nxt[static_cast<size_t>(t) * VS + e * RC + c] = v;
        if (col0 + c < r && e >= own0) data[(static_cast<int64_t>(first + t) * r + col0 + c) * Ke + e] = v;
      }
    }
    __syncthreads();
    C* tmp = cur; cur = nxt; nxt = tmp;
  }
  // the subtree root (level s) -> TX[s]
  {
    C* tx = vec(T.TX, s);
    for (int u = threadIdx.x; u < VS; u += blockDim.x) tx[u] = cur[u];
  }
  __syncthreads();

  // ---- top upsweep: levels s-1 .. 0 (HODLR: .. 1), one cluster barrier each ----
  const int lmin = hss ? 0 : 1;
  for (int lev = s - 1; lev >= lmin; --lev) {
    cluster_sync_all();                    // level lev+1 complete in every CTA
    const bool own = (j & ((1 << (s - lev)) - 1)) == 0;
    C* ch = vec(T.CH, 0);
    if (own) {
      const int rb = j + (1 << (s - lev - 1));                  // owner of the right child
      const C* mine = vec(T.TX, lev + 1);
      for (int u = threadIdx.x; u < VS; u += blockDim.x) ch[u] = mine[u];
      pull_remote(ch + VS, vec(T.TX, lev + 1), rb, static_cast<int>(V / 16));
    }
    __syncthreads();
    if (own) {
      const int q = (1 << lev) - 1 + (j >> (s - lev));
      if (hss) {
        const int per = (lev > 0 ? nbp : 0) + 2 * nbe;
        LevelArgs<C> la{LV_TOPUP, k, 1, lev, q, nbp, nbe, 0, ch, vec(T.TX, lev), vec(T.TYC, 2 * lev), YCg, VS};
        run_level_cw<C, RC>(R, mv, ws.err, la, pick_cw<RC>(per, nwarps));
        ++k;
      } else {
        const int rows = mv.koff[lev + 1];
        C* tx = vec(T.TX, lev);
        for (int w = threadIdx.x; w < rows * RC; w += blockDim.x) {
          const int c = w % RC, e = w / RC;
          const C v = ch[e * RC + c] + ch[VS + e * RC + c];
          tx[e * RC + c] = v;
          if (col0 + c < r && e >= mv.koff[lev]) data[(static_cast<int64_t>(q) * r + col0 + c) * Ke + e] = v;
        }
      }
    }
    __syncthreads();
  }

  if (hss) {
    // ---- top downsweep: levels 1 .. s ----
    for (int lev = 1; lev <= s; ++lev) {
      cluster_sync_all();                  // level lev-1 (and the couplings) complete
      const bool own = (j & ((1 << (s - lev)) - 1)) == 0;
      C* syc = vec(T.STG, 0);
      C* syp = vec(T.STG, 1);
      const int node = (1 << lev) - 1 + (j >> (s - lev));
      const int h = (node & 1) ? 0 : 1;                           // 0: left child
      if (own) {
        const int pj = (j >> (s - lev + 1)) << (s - lev + 1);     // owner of the parent
        pull_remote(syc, vec(T.TYC, 2 * (lev - 1) + h), pj, static_cast<int>(V / 16));
        if (lev >= 2) pull_remote(syp, vec(T.TYF, lev - 1), pj, static_cast<int>(V / 16));
      }
      __syncthreads();
      if (own) {
        C* yf = vec(T.TYF, lev);
        if (lev == 1) {
          for (int u = threadIdx.x; u < VS; u += blockDim.x) yf[u] = syc[u];
        } else {
          LevelArgs<C> la{LV_TOPDOWN, k, 1, lev, node, nbp, nbe, h, syp, yf, syc, YCg, VS};
          run_level_cw<C, RC>(R, mv, ws.err, la, pick_cw<RC>(nbe, nwarps));
          ++k;
        }
      }
      __syncthreads();
    }
    // ---- bottom downsweep: levels s+1 .. p ----
    const C* ypar = vec(T.TYF, s);
    for (int lev = s + 1; lev <= p; ++lev) {
      const int nc = 1 << (lev - s);                              // children at lev
      C* out = ((p - lev) % 2 == 0) ? A : Bb;
      const int firstc = (1 << lev) - 1 + (j << (lev - s));
      LevelArgs<C> la{LV_DOWN, k, nc, lev, firstc, nbp, nbe, 0, ypar, out, nullptr, YCg, VS};
      run_level_cw<C, RC>(R, mv, ws.err, la, pick_cw<RC>(nc * nbe, nwarps));
      k += nc / 2;
      __syncthreads();
      if (lev == p) {
        C* yg = static_cast<C*>(ws.yf);
        const int first = (1 << lev) - 1 + (j << (lev - s));
        const int total = nc * Ke * RC;
        for (int w = threadIdx.x; w < total; w += blockDim.x) {
          const int i = w % Ke;
          const int c = (w / Ke) % RC;
          const int t = w / (Ke * RC);
          if (col0 + c < r)
            yg[(static_cast<int64_t>(first + t) * r + col0 + c) * Ke + i] = out[static_cast<size_t>(t) * VS + i * RC + c];
        }
      }
      ypar = out;
    }
    if (d == 0) {
      // the subtree is one leaf: its y-hat is the top result
      C* yg = static_cast<C*>(ws.yf);
      const C* yf = vec(T.TYF, s);
      const int node = (1 << p) - 1 + j;
      for (int w = threadIdx.x; w < Ke * RC; w += blockDim.x) {
        const int i = w % Ke, c = w / Ke;
        if (col0 + c < r) yg[(static_cast<int64_t>(node) * r + col0 + c) * Ke + i] = yf[i * RC + c];
      }
    }
  }
  // no CTA leaves while another may still read its shared memory
  cluster_sync_all();
  if (hss && threadIdx.x == 0 && *(volatile int*)R.dead) {
    // drain: bounded waits for the copies still in flight into the ring
    const int hi = *R.issued;
    for (int u = hi > T.NS ? hi - T.NS : 0; u < hi; ++u)
      mbar_wait(smem_u32(R.full + (u % R.NS)), (u / R.NS) & 1, nullptr, 0);
  }
}

// ---- host side ----

// One launch shape: levels shared by the cluster, columns per cluster, ring
// slots (0: HODLR).
struct TreeShape {
  int s, rc, ns;
};

template <typename C>
static bool tree_fit(const MatView& mv, int RC, int s, int ns, TreeLayout* out) {
  const bool hss = (mv.kind == HM_HSS);
  const uint32_t limit = 227 * 1024 - 512;   // 128 bytes of alignment slack, static data
  const TreeLayout T = tree_layout<C>(hss, mv.p, mv.Kp, mv.Ke, RC, hss ? ns : 0, s);
  if (T.total + 128 > limit) return false;
  if (hss && (2 * (1 << T.d) + 2 * T.s) > TREE_MAX_ITEMS / 2 - 1) return false;
  *out = T;
  return true;
}

template <typename C, int RC>
static cudaLaunchConfig_t tree_cfg(const TreeLayout& T, int64_t r, cudaStream_t st, cudaLaunchAttribute* attrs,
                                   bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1 << T.s, static_cast<unsigned>((r + RC - 1) / RC));
  cfg.blockDim = dim3(TREE_THREADS);
  cfg.dynamicSmemBytes = T.total + 128;
  cfg.stream = st;
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = 1 << T.s;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  attrs[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attrs[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = pdl ? 2 : 1;
  return cfg;
}

template <typename C, int RC>
static void tree_attrs(size_t smem) {
  cudaFuncSetAttribute(k_tree_cluster<C, RC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_tree_cluster<C, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
}

// Clusters of this shape that can be resident at once (0 if none).
template <typename C, int RC>
static int tree_active(const MatView& mv, int64_t r, int s, int ns) {
  TreeLayout T;
  if (!tree_fit<C>(mv, RC, s, ns, &T)) return 0;
  tree_attrs<C, RC>(T.total + 128);
  cudaLaunchAttribute attrs[2];
  cudaLaunchConfig_t cfg = tree_cfg<C, RC>(T, r, nullptr, attrs, false);
  int nact = 0;
  if (cudaOccupancyMaxActiveClusters(&nact, k_tree_cluster<C, RC>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nact;
}

template <typename C>
static int tree_active_rc(const MatView& mv, int64_t r, const TreeShape& sh) {
  switch (sh.rc) {
    case 1: return tree_active<C, 1>(mv, r, sh.s, sh.ns);
    case 2: return tree_active<C, 2>(mv, r, sh.s, sh.ns);
    case 4: return tree_active<C, 4>(mv, r, sh.s, sh.ns);
    default: return tree_active<C, 8>(mv, r, sh.s, sh.ns);
  }
}

// The deepest ring (up to TREE_MAX_NS slots, at least 2) that fits in `budget`
// bytes of shared memory; 0 if none does.
template <typename C>
static int tree_ring(const MatView& mv, int RC, int s, uint32_t budget) {
  const bool hss = (mv.kind == HM_HSS);
  if (!hss) {
    const TreeLayout T = tree_layout<C>(false, mv.p, mv.Kp, mv.Ke, RC, 0, s);
    return (T.total + 128 <= budget) ? 1 : 0;
  }
  for (int ns = TREE_MAX_NS; ns >= 2; --ns) {
    const TreeLayout T = tree_layout<C>(true, mv.p, mv.Kp, mv.Ke, RC, ns, s);
    if (T.total + 128 <= budget) return ns;
  }
  return 0;
}

// Picks the launch shape with the fewest waves of clusters and, among those,
// the least estimated time per CTA.
template <typename C>
static bool tree_pick(const MatView& mv, int64_t r, TreeShape* out) {
  bool found = false;
  double best = 1e300;
  int best_waves = 1 << 30;
  const int smax = mv.p < TREE_MAX_S ? mv.p : TREE_MAX_S;
  for (int s = (smax >= 3 ? 3 : smax); s <= smax; ++s) {
    for (int rc = 1; rc <= 8; rc *= 2) {
      // a deep ring at one CTA per SM, or a shallower one that lets two share
      // an SM; for FP64 the deep ring leaves room for a block of the
      // diagonal-block product, which runs beside the tree (k_f64.cu)
      const uint32_t deep = (mv.storage == HM_F64) ? 188u * 1024 : 227u * 1024 - 512;
      const uint32_t budgets[2] = {deep, 113u * 1024 - 256};
      for (uint32_t budget : budgets) {
        const int ns = tree_ring<C>(mv, rc, s, budget);
        if (ns == 0) continue;
        TreeShape sh{s, rc, mv.kind == HM_HSS ? ns : 0};
        TreeLayout T;
        if (!tree_fit<C>(mv, rc, s, sh.ns, &T)) continue;
        const int nact = tree_active_rc<C>(mv, r, sh);
        if (nact <= 0) continue;
        const int64_t ncl = (r + rc - 1) / rc;
        const int waves = static_cast<int>((ncl + nact - 1) / nact);
        // estimated cycles of one CTA: the larger of its shared-memory
        // wavefronts (6K steps per node pair, RT + CT per step) and its
        // operator stream (2 records per subtree node, ~2300 cycles per copy,
        // ns in flight), plus ~2000 cycles per top level
        const int K = mv.Kp > mv.Ke ? mv.Kp : mv.Ke;
        const double wav = static_cast<double>(1 << T.d) * 6.0 * K * (rc >= 2 ? rc / 2 + 2 : 2);
        const double stream = (sh.ns > 0) ? 2.0 * (1 << T.d) * 2300.0 / sh.ns : 0.0;
        const double score = ((wav > stream ? wav : stream) + 2000.0 * T.s) * waves;
        if (waves < best_waves || (waves == best_waves && score < best)) {
          best_waves = waves;
          best = score;
          *out = sh;
          found = true;
        }
      }
    }
  }
  return found;
}

template <typename C, int RC>
static hm_status launch_tree_cl(const MatView& mv, const Scratch& ws, int64_t r, cudaStream_t st, bool pdl,
                                const TreeShape& sh) {
  TreeLayout T;
  if (!tree_fit<C>(mv, RC, sh.s, sh.ns, &T)) return HM_EUNSUPPORTED;
  tree_attrs<C, RC>(T.total + 128);
  cudaLaunchAttribute attrs[2];
  cudaLaunchConfig_t cfg = tree_cfg<C, RC>(T, r, st, attrs, pdl);
  Scratch wk = ws;
  wk.prof = nullptr;
  prof_mark(ws.prof, 1, true, st);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_tree_cluster<C, RC>, mv, wk, r, T.NS, T.s);
  if (e != cudaSuccess && pdl) {
    // launch without the early start instead
    cudaGetLastError();
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_tree_cluster<C, RC>, mv, wk, r, T.NS, T.s);
  }
  prof_mark(ws.prof, 1, false, st);
  if (e != cudaSuccess) {
    set_error("tree cluster launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

template <typename C>
static hm_status tree_launch_shape(const MatView& mv, const Scratch& ws, int64_t r, cudaStream_t st, bool pdl,
                                   const TreeShape& sh) {
  switch (sh.rc) {
    case 1: return launch_tree_cl<C, 1>(mv, ws, r, st, pdl, sh);
    case 2: return launch_tree_cl<C, 2>(mv, ws, r, st, pdl, sh);
    case 4: return launch_tree_cl<C, 4>(mv, ws, r, st, pdl, sh);
    case 8: return launch_tree_cl<C, 8>(mv, ws, r, st, pdl, sh);
    default: return HM_EUNSUPPORTED;
  }
}

bool tree_cluster_usable(hm_matrix* A, const MatView& mv, int64_t r) {
  const bool hss = (mv.kind == HM_HSS);
  if (A->tree_mode == 1) return false;
  if (mv.p < (hss ? 1 : 2) || mv.p > 11) return false;   // no tree work, or a subtree too deep
  if (A->tree_ok_r != r) {
    TreeShape sh{0, 0, 0};
    A->tree_ok = (mv.storage == HM_F64) ? tree_pick<double>(mv, r, &sh) : tree_pick<float>(mv, r, &sh);
    A->tree_s = sh.s;
    A->tree_rc = sh.rc;
    A->tree_ns = sh.ns;
    A->tree_ok_r = r;
  }
  return A->tree_ok;
}

// Times the whole product (projection, tree, expansion; the tree in one
// cluster launch) for r columns with every launch shape of the tree kernel
// that fits (levels shared by the cluster s, columns per cluster, ring
// slots), on zero inputs of the given types, three products each after a
// warm-up, and keeps the fastest for later products with r columns.  The
// product, not the tree alone, is timed because the expansion starts while
// the tree drains and competes with it for SMs.  Every shape sums in the
// same order, so the choice never changes a result.
template <typename C>
static hm_status tune_shapes(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X, int xt,
                             void* Y, int yt, cudaStream_t st, double* best_ms) {
  const bool hss = (mv.kind == HM_HSS);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    set_error("tree tuning: event creation failed");
    return HM_ECUDA;
  }
  const int mode = A->tree_mode;
  A->tree_mode = 2;
  TreeShape best{0, 0, 0};
  double bms = 1e300;
  // the built-in choice, kept unless a shape beats it by at least 2 %
  TreeShape dflt{0, 0, 0};
  const bool have_dflt = tree_pick<C>(mv, r, &dflt);
  double dms = 1e300;
  cudaEvent_t ev[6];
  for (auto& x : ev) x = nullptr;
  for (auto& x : ev) cudaEventCreate(&x);
  const int smax = mv.p < TREE_MAX_S ? mv.p : TREE_MAX_S;
  const int64_t n = mv.n;
  for (int s = (smax >= 2 ? 2 : smax); s <= smax; ++s) {
    for (int rc = 1; rc <= 8; rc *= 2) {
      for (int ns = hss ? 2 : 0; ns <= (hss ? TREE_MAX_NS : 0); ++ns) {
        const TreeShape sh{s, rc, ns};
        TreeLayout T;
        if (!tree_fit<C>(mv, rc, s, ns, &T)) continue;
        if (tree_active_rc<C>(mv, r, sh) <= 0) continue;
        A->tree_s = sh.s;
        A->tree_rc = sh.rc;
        A->tree_ns = sh.ns;
        A->tree_ok = true;
        A->tree_ok_r = r;
        hm_status stt = launch_product(A, mv, ws, r, X, n, xt, Y, n, yt, st);
        if (stt != HM_OK || !A->tree_last_cluster) { cudaGetLastError(); continue; }
        // five products, each timed on its own; the median is the shape's time
        cudaEventRecord(ev[0], st);
        for (int k = 0; k < 5 && stt == HM_OK; ++k) {
          stt = launch_product(A, mv, ws, r, X, n, xt, Y, n, yt, st);
          cudaEventRecord(ev[k + 1], st);
        }
        if (cudaEventSynchronize(ev[5]) != cudaSuccess || stt != HM_OK) { cudaGetLastError(); continue; }
        float t[5];
        for (int k = 0; k < 5; ++k) cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]);
        std::sort(t, t + 5);
        const double med = t[2];
        if (have_dflt && sh.s == dflt.s && sh.rc == dflt.rc && sh.ns == dflt.ns) dms = med;
        if (med < bms) {
          bms = med;
          best = sh;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  A->tree_mode = mode;
  if (best.rc != 0 && dms < 1e300 && bms > 0.98 * dms) {
    best = dflt;
    bms = dms;
  }
  if (best.rc == 0) {
    A->tree_ok_r = -1;   // fall back to the built-in choice
    return HM_EUNSUPPORTED;
  }
  A->tree_s = best.s;
  A->tree_rc = best.rc;
  A->tree_ns = best.ns;
  A->tree_ok = true;
  A->tree_ok_r = r;
  if (best_ms) *best_ms = bms;
  return HM_OK;
}

hm_status tune_tree_cluster(hm_matrix* A, int64_t r, int xt, int yt, double* best_ms) {
  const MatView mv = A->view();
  const bool hss = (mv.kind == HM_HSS);
  if (A->tree_mode == 1 || mv.p < (hss ? 1 : 2) || mv.p > 11) return HM_EUNSUPPORTED;
  hm_status st = ensure_scratch(A, r);
  if (st != HM_OK) return st;
  Scratch ws = scratch_of(A, r);
  ws.prof = nullptr;
  const size_t xs = (xt == HM_F64) ? 8 : (xt == HM_F32) ? 4 : 2;
  const size_t ys = (yt == HM_F64) ? 8 : 4;
  const size_t nr = static_cast<size_t>(std::max<int64_t>(mv.n, 1)) * r;
  void* X = nullptr;
  void* Y = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = dev_malloc(&X, nr * xs);
  if (e == cudaSuccess) e = dev_malloc(&Y, nr * ys);
  if (e == cudaSuccess) e = cudaMemset(X, 0, nr * xs);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (X) cudaFree(X);
    if (Y) cudaFree(Y);
    set_error("tree tuning: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA;
  }
  st = (mv.storage == HM_F64) ? tune_shapes<double>(A, mv, ws, r, X, xt, Y, yt, s, best_ms)
                              : tune_shapes<float>(A, mv, ws, r, X, xt, Y, yt, s, best_ms);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  cudaFree(X);
  cudaFree(Y);
  return st;
}

template <typename C>
static hm_status set_shape(hm_matrix* A, const MatView& mv, int64_t r, const TreeShape& sh) {
  TreeLayout T;
  if (!tree_fit<C>(mv, sh.rc, sh.s, sh.ns, &T)) return HM_EUNSUPPORTED;
  if (tree_active_rc<C>(mv, r, sh) <= 0) return HM_EUNSUPPORTED;
  A->tree_s = sh.s;
  A->tree_rc = sh.rc;
  A->tree_ns = sh.ns;
  A->tree_ok = true;
  A->tree_ok_r = r;
  return HM_OK;
}

hm_status set_tree_shape(hm_matrix* A, int64_t r, int cluster_ctas, int columns, int ring_slots) {
  const MatView mv = A->view();
  const bool hss = (mv.kind == HM_HSS);
  if (A->tree_mode == 1 || mv.p < (hss ? 1 : 2) || mv.p > 11) return HM_EUNSUPPORTED;
  int s = 0;
  while ((1 << s) < cluster_ctas && s < 30) ++s;
  const int smax = mv.p < TREE_MAX_S ? mv.p : TREE_MAX_S;
  if ((1 << s) != cluster_ctas || s < 1 || s > smax) return HM_EINVAL;
  if (columns != 1 && columns != 2 && columns != 4 && columns != 8) return HM_EINVAL;
  if (hss ? (ring_slots < 2 || ring_slots > TREE_MAX_NS) : ring_slots != 0) return HM_EINVAL;
  const TreeShape sh{s, columns, ring_slots};
  return (mv.storage == HM_F64) ? set_shape<double>(A, mv, r, sh) : set_shape<float>(A, mv, r, sh);
}

hm_status launch_tree_cluster(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, cudaStream_t st,
                              bool pdl) {
  if (!tree_cluster_usable(A, mv, r)) return HM_EUNSUPPORTED;
  const TreeShape sh{A->tree_s, A->tree_rc, A->tree_ns};
  return (mv.storage == HM_F64) ? tree_launch_shape<double>(mv, ws, r, st, pdl, sh)
                                : tree_launch_shape<float>(mv, ws, r, st, pdl, sh);
}

}  // namespace hmi

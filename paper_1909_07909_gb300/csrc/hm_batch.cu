// Host runtime of batched products: plan (per-product blocking identical to a
// single product), per-phase work lists, one persistent launch per phase,
// CUDA-graph capture and the autotuner of launch shapes.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "hm_api_internal.h"
#include "hm_batch.h"
#include "k_simt.cuh"

namespace hmi {

static hm_status bfail(hm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_error("%s", buf);
  return s;
}

// Launch-shape knobs chosen by the autotuner.  None of them changes any
// product's arithmetic: column chunks split independent columns, the tile
// height splits independent rows, and the grid only changes which block runs
// which item.
struct BatchKnobs {
  int grid_mult = 2;   // persistent blocks per SM of the SIMT phases
  int rc_cap = 32;     // widest SIMT column chunk
  int rct_cap = 16;    // widest tree column chunk
  int rt = 64;         // rows per SIMT expansion tile
};

}  // namespace hmi

struct hm_batch {
  uint32_t magic = 0;
  int device = 0;
  int count = 0;
  int sms = 152;
  std::vector<hm_matrix*> mats;
  std::vector<int64_t> rs;
  hmi::BatchKnobs knobs;
  std::vector<hmi::BatchJob> jobs;
  std::vector<hmi::BItem> items[hmi::BP_COUNT];
  size_t smem[hmi::BP_COUNT] = {};
  int grid[hmi::BP_COUNT] = {};
  int tc_ncol[hmi::BP_COUNT] = {};
  hmi::BatchJob* d_jobs = nullptr;
  hmi::BatchIO* d_io = nullptr;
  CUtensorMap* d_maps = nullptr;
  hmi::BItem* d_items[hmi::BP_COUNT] = {};
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  std::vector<hmi::BatchIO> h_io;
  cudaGraphExec_t gexec = nullptr;
  bool use_graph = true;
  int capture_error = 0;   // CUDA error of a failed capture (0 if none)
  int tuned = 0;
};

namespace hmi {

static void free_plan(hm_batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  for (int p = 0; p < BP_COUNT; ++p) {
    if (b->d_items[p]) cudaFree(b->d_items[p]);
    b->d_items[p] = nullptr;
  }
  if (b->d_jobs) cudaFree(b->d_jobs);
  b->d_jobs = nullptr;
}

static int pow2_at_least(int64_t v, int cap) {
  int x = 1;
  while (x < v && x < cap) x *= 2;
  return x;
}

// Builds the per-product blocking (the same rules as the single-product path)
// and the work lists for the current knobs; uploads jobs and items.
static hm_status build_plan(hm_batch* b) {
  free_plan(b);
  const BatchKnobs& kn = b->knobs;
  b->jobs.assign(b->count, BatchJob());
  for (int p = 0; p < BP_COUNT; ++p) {
    b->items[p].clear();
    b->smem[p] = 0;
    b->tc_ncol[p] = 32;
  }
  char* sbase = static_cast<char*>(b->d_scratch);
  size_t soff = 0;
  for (int j = 0; j < b->count; ++j) {
    hm_matrix* A = b->mats[j];
    const int64_t r = b->rs[j];
    BatchJob& J = b->jobs[j];
    std::memset(&J, 0, sizeof(J));
    J.mv = A->view();
    J.r = r;
    J.storage = A->storage;
    const MatView& mv = J.mv;
    // scratch: data then counters, 256-byte aligned (same layout as a single product)
    const size_t nodes = static_cast<size_t>(2 * A->L - 1);
    const size_t data = ((scratch_elems(mv, r) * 4 + 255) / 256) * 256;
    const size_t cnts = ((counter_count(mv, r) * sizeof(int) + 255) / 256) * 256;
    char* base = sbase + soff;
    if (A->kind == HM_HODLR) {
      J.ws.PS = base;
    } else {
      J.ws.xh = base;
      J.ws.yc = base + nodes * r * A->Kp * 4;
      J.ws.yf = base + nodes * r * (A->Kp + A->Ke) * 4;
    }
    J.ws.cnt = reinterpret_cast<int*>(base + data);
    J.ws.err = A->err;
    J.ws.prof = nullptr;
    soff += data + cnts;
    // column chunks: the single-product rule, capped by the tuned widths
    J.rc_p = std::min(pick_rc(r, 4, mv.m_pad), kn.rc_cap);
    J.rc_e = std::min(pick_rc(r, 4, mv.We), kn.rc_cap);
    J.rct = std::min(pow2_at_least(r, 16), kn.rct_cap);
    const bool hss = (mv.kind == HM_HSS);
    const int lmin = hss ? 0 : 1;
    int g = 3;
    while (g > 1 && 4 * static_cast<size_t>(up_smem_elems(hss, J.rct, mv.Kp, mv.Ke, g)) > 100 * 1024) --g;
    J.g = g;
    J.s0 = std::max(0, std::min(g, mv.p - lmin));
    if (hss && mv.p >= 1) {
      const int d = down_depth(mv, 4);
      J.s_lvl = mv.p - d;
      const int per = mv.Ke * mv.Ke + J.rct * mv.Ke;
      J.G = std::max(1, std::min(std::max(J.s_lvl - 1, 1), static_cast<int>((96 * 1024 / 4) / std::max(per, 1))));
    }
    J.RT = kn.rt;
    J.tiles = (mv.m_pad + kn.rt - 1) / kn.rt;
    J.tc = use_tensor_cores(A, r) ? 1 : 0;
    if (J.tc && !tc_plan(A, r, false, &J.nt, &J.nK, &J.nX, &J.nst, &J.tc_tiles)) J.tc = 0;
    // the projection runs on the tensor cores exactly when the single product's would
    J.tcp = (use_tensor_cores(A, r) && tc_plan(A, r, true, &J.ntp, &J.nKp, &J.nXp, &J.nstp, &J.tcp_tiles)) ? 1 : 0;
    J.w_box = A->w_box;
    J.split = (A->storage == HM_BF16X2) ? 1 : 0;
    // work items and shared memory per phase
    if (J.tcp) {
      const int nch = static_cast<int>((r + J.ntp - 1) / J.ntp);
      for (int x = 0; x < mv.L * J.tcp_tiles; ++x)
        for (int c = 0; c < nch; ++c) b->items[BP_PROJECT_TC].push_back({j, x, c});
      b->smem[BP_PROJECT_TC] =
          std::max(b->smem[BP_PROJECT_TC], 2048 + tc_tile_smem(J.split, J.ntp, J.nKp, J.nstp));
      b->tc_ncol[BP_PROJECT_TC] = std::max(b->tc_ncol[BP_PROJECT_TC], tc_tile_ncols(J.split, J.ntp));
    } else {
      const int nch_p = static_cast<int>((r + J.rc_p - 1) / J.rc_p);
      for (int leaf = 0; leaf < mv.L; ++leaf)
        for (int c = 0; c < nch_p; ++c) b->items[BP_PROJECT].push_back({j, leaf, c});
      b->smem[BP_PROJECT] =
          std::max(b->smem[BP_PROJECT], 4 * static_cast<size_t>(J.rc_p * mv.m_pad + J.rc_p * (mv.Kp + 1)));
    }
    const int nch_t = static_cast<int>((r + J.rct - 1) / J.rct);
    if (mv.p > lmin) {
      for (int x = 0; x < (mv.L >> J.s0); ++x)
        for (int c = 0; c < nch_t; ++c) b->items[BP_UP].push_back({j, x, c});
      b->smem[BP_UP] = std::max(b->smem[BP_UP],
                                4 * static_cast<size_t>(up_smem_elems(hss, J.rct, mv.Kp, mv.Ke, std::min(g, mv.p))));
    }
    if (hss && mv.p >= 1) {
      for (int x = 0; x < (1 << J.s_lvl); ++x)
        for (int c = 0; c < nch_t; ++c) b->items[BP_DOWN].push_back({j, x, c});
      b->smem[BP_DOWN] = std::max(
          b->smem[BP_DOWN], 4 * static_cast<size_t>(down_smem_elems(J.rct, mv.Ke, mv.p - J.s_lvl, J.G)));
    }
    if (J.tc) {
      const int nch = static_cast<int>((r + J.nt - 1) / J.nt);
      for (int x = 0; x < mv.L * J.tc_tiles; ++x)
        for (int c = 0; c < nch; ++c) b->items[BP_EXPAND_TC].push_back({j, x, c});
      b->smem[BP_EXPAND_TC] = std::max(b->smem[BP_EXPAND_TC], 2048 + tc_tile_smem(J.split, J.nt, J.nK, J.nst));
      b->tc_ncol[BP_EXPAND_TC] = std::max(b->tc_ncol[BP_EXPAND_TC], tc_tile_ncols(J.split, J.nt));
    } else {
      const int nch_e = static_cast<int>((r + J.rc_e - 1) / J.rc_e);
      for (int x = 0; x < mv.L * J.tiles; ++x)
        for (int c = 0; c < nch_e; ++c) b->items[BP_EXPAND].push_back({j, x, c});
      b->smem[BP_EXPAND] =
          std::max(b->smem[BP_EXPAND], 4 * static_cast<size_t>(J.rc_e * mv.We + J.rc_e * (kn.rt + 1)));
    }
  }
  for (int p = 0; p < BP_COUNT; ++p)
    if (b->smem[p] > 227 * 1024) return bfail(HM_EUNSUPPORTED, "batch phase %d needs %zu bytes of shared memory", p, b->smem[p]);
  // persistent grids
  for (int p = 0; p < BP_COUNT; ++p) {
    const int n = static_cast<int>(b->items[p].size());
    int per_sm = batch_phase_tc(p) ? 1 : kn.grid_mult;
    if (!batch_phase_tc(p) && b->smem[p] > 0) per_sm = std::max(1, std::min(per_sm, static_cast<int>((228 * 1024) / (b->smem[p] + 1024))));
    b->grid[p] = std::max(0, std::min(n, b->sms * per_sm));
  }
  for (int p = 0; p < BP_COUNT; ++p) {
    if (b->items[p].empty()) continue;
    if (batch_phase_tc(p)) batch_set_smem_tc(p, b->smem[p]);
    else batch_set_smem(p, b->smem[p]);
  }
  // upload
  cudaError_t e = dev_malloc(reinterpret_cast<void**>(&b->d_jobs), sizeof(BatchJob) * std::max(b->count, 1));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_jobs, b->jobs.data(), sizeof(BatchJob) * b->count, cudaMemcpyHostToDevice);
  for (int p = 0; p < BP_COUNT && e == cudaSuccess; ++p) {
    if (b->items[p].empty()) continue;
    e = dev_malloc(reinterpret_cast<void**>(&b->d_items[p]), sizeof(BItem) * b->items[p].size());
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_items[p], b->items[p].data(), sizeof(BItem) * b->items[p].size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return bfail(e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "batch plan upload: %s",
                                     cudaGetErrorString(e));
  return HM_OK;
}

// The six phase launches (SIMT and tensor-core projection, upsweep, downsweep,
// SIMT and tensor-core expansion), each persistent; all but the first use
// programmatic serialization.  Empty phases are skipped.
static hm_status enqueue(hm_batch* b, cudaStream_t s) {
  bool first = true;
  for (int p = 0; p < BP_COUNT; ++p) {
    const int n = static_cast<int>(b->items[p].size());
    if (n == 0) continue;
    cudaError_t e;
    if (batch_phase_tc(p))
      e = batch_launch_tc(p, b->d_jobs, b->d_io, b->d_maps, b->d_items[p], n, b->grid[p], b->smem[p], b->tc_ncol[p], s,
                          !first);
    else
      e = batch_launch_simt(p, b->d_jobs, b->d_io, b->d_items[p], n, b->grid[p], b->smem[p], s, !first);
    if (e != cudaSuccess) return bfail(HM_ECUDA, "batch launch (phase %d): %s", p, cudaGetErrorString(e));
    first = false;
  }
  return HM_OK;
}

static hm_status capture(hm_batch* b, cudaStream_t s) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bfail(HM_ECUDA, "capture stream: %s", cudaGetErrorString(e));
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  hm_status st = HM_OK;
  if (e == cudaSuccess) st = enqueue(b, cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  (void)s;
  if (e != cudaSuccess || e2 != cudaSuccess || st != HM_OK || !graph) {
    if (graph) cudaGraphDestroy(graph);
    b->capture_error = (e != cudaSuccess) ? e : (e2 != cudaSuccess ? e2 : -1);
    cudaGetLastError();
    b->use_graph = false;  // fall back to direct launches of the same kernels
    return HM_OK;
  }
  e = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->capture_error = 1000 + e;
    cudaGetLastError();
    b->gexec = nullptr;
    b->use_graph = false;
  }
  return HM_OK;
}

static hm_status run_once(hm_batch* b, cudaStream_t s) {
  if (b->use_graph) {
    if (!b->gexec) {
      hm_status st = capture(b, s);
      if (st != HM_OK) return st;
    }
    if (b->gexec) {
      const cudaError_t e = cudaGraphLaunch(b->gexec, s);
      if (e != cudaSuccess) return bfail(HM_ECUDA, "graph launch: %s", cudaGetErrorString(e));
      return HM_OK;
    }
  }
  return enqueue(b, s);
}

static uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ull;
  }
  return h;
}

static std::string signature(const hm_batch* b) {
  std::vector<std::string> parts;
  for (int j = 0; j < b->count; ++j) {
    const hm_matrix* A = b->mats[j];
    std::ostringstream o;
    o << A->kind << ":" << A->storage << ":" << A->n << ":" << A->m_pad << ":" << A->Ke << ":" << A->Kp << ":"
      << b->rs[j];
    parts.push_back(o.str());
  }
  std::sort(parts.begin(), parts.end());
  std::ostringstream o;
  for (auto& p : parts) o << p << ";";
  char buf[32];
  snprintf(buf, sizeof(buf), "%016llx", static_cast<unsigned long long>(fnv1a(o.str())));
  return buf;
}

void destroy_batch(hm_batch* b) {
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != b->device) cudaSetDevice(b->device);
  free_plan(b);
  if (b->d_io) cudaFree(b->d_io);
  if (b->d_maps) cudaFree(b->d_maps);
  if (b->d_scratch) cudaFree(b->d_scratch);
  if (dev_prev != b->device) cudaSetDevice(dev_prev);
  b->magic = 0;
  delete b;
}

}  // namespace hmi

using namespace hmi;

extern "C" hm_status hm_batch_create(hm_matrix* const* A, const int64_t* r, int32_t count, hm_batch** out) {
  if (!out) return bfail(HM_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !A || !r) return bfail(HM_EINVAL, "need count >= 1, matrices and right-hand-side counts");
  int dev = -1;
  for (int j = 0; j < count; ++j) {
    if (!A[j] || A[j]->magic != kMagicMatrix) return bfail(HM_EINVAL, "entry %d is not a matrix handle", j);
    if (A[j]->storage == HM_F64)
      return bfail(HM_EUNSUPPORTED, "entry %d: batches take F32, BF16 or BF16X2 storage (run F64 products singly)", j);
    if (r[j] < 1) return bfail(HM_EINVAL, "entry %d: r must be >= 1", j);
    if (dev < 0) dev = A[j]->device;
    if (A[j]->device != dev) return bfail(HM_EINVAL, "all matrices of a batch must live on one device");
  }
  hm_batch* b = new (std::nothrow) hm_batch();
  if (!b) return bfail(HM_ENOMEM, "host allocation failed");
  b->magic = kMagicBatch;
  b->device = dev;
  b->count = count;
  b->mats.assign(A, A + count);
  b->rs.assign(r, r + count);
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != dev) cudaSetDevice(dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  size_t total = 0;
  for (int j = 0; j < count; ++j) {
    const MatView mv = A[j]->view();
    total += ((scratch_elems(mv, r[j]) * 4 + 255) / 256) * 256 + ((counter_count(mv, r[j]) * sizeof(int) + 255) / 256) * 256;
  }
  b->scratch_bytes = std::max<size_t>(total, 256);
  cudaError_t e = dev_malloc(reinterpret_cast<void**>(&b->d_scratch), b->scratch_bytes);
  if (e == cudaSuccess) e = cudaMemset(b->d_scratch, 0, b->scratch_bytes);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&b->d_io), sizeof(BatchIO) * count);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&b->d_maps), sizeof(CUtensorMap) * BATCH_MAPS * count);
  if (e == cudaSuccess) {
    std::vector<CUtensorMap> maps(BATCH_MAPS * count);
    for (int j = 0; j < count; ++j) {
      maps[BATCH_MAPS * j] = A[j]->tmA;
      maps[BATCH_MAPS * j + 1] = A[j]->tmAlo;
      maps[BATCH_MAPS * j + 2] = A[j]->tmW;
      maps[BATCH_MAPS * j + 3] = A[j]->tmWlo;
    }
    e = cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * BATCH_MAPS * count, cudaMemcpyHostToDevice);
  }
  hm_status st = (e == cudaSuccess) ? HM_OK
                                    : bfail(e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "batch allocation: %s",
                                            cudaGetErrorString(e));
  if (st == HM_OK) st = build_plan(b);
  if (dev_prev != dev) cudaSetDevice(dev_prev);
  if (st != HM_OK) {
    destroy_batch(b);
    return st;
  }
  b->h_io.assign(count, BatchIO());
  *out = b;
  return HM_OK;
}

extern "C" hm_status hm_batch_run(hm_batch* b, const void* const* X, void* const* Y, hm_dtype xt, hm_dtype yt,
                                  void* stream) {
  if (!b || b->magic != kMagicBatch) return bfail(HM_EINVAL, "not a batch handle");
  if (!X || !Y) return bfail(HM_EINVAL, "X or Y is NULL");
  if (xt != HM_F32 && xt != HM_BF16 && xt != HM_F64) return bfail(HM_EINVAL, "X type must be F32, BF16 or F64");
  if (yt != HM_F32 && yt != HM_F64) return bfail(HM_EINVAL, "Y type must be F32 or F64");
  for (int j = 0; j < b->count; ++j) {
    if (b->mats[j]->n > 0 && (!X[j] || !Y[j])) return bfail(HM_EINVAL, "entry %d: X or Y is NULL", j);
    b->h_io[j] = {X[j], Y[j], std::max<int64_t>(b->mats[j]->n, 1), std::max<int64_t>(b->mats[j]->n, 1), xt, yt};
  }
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != b->device) cudaSetDevice(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // pageable source: returns once the host buffer has been read, so the next
  // run may overwrite it; ordered before the launches on the same stream
  cudaError_t e = cudaMemcpyAsync(b->d_io, b->h_io.data(), sizeof(BatchIO) * b->count, cudaMemcpyHostToDevice, s);
  hm_status st = (e == cudaSuccess) ? run_once(b, s) : bfail(HM_ECUDA, "batch I/O upload: %s", cudaGetErrorString(e));
  if (dev_prev != b->device) cudaSetDevice(dev_prev);
  return st;
}

extern "C" hm_status hm_batch_tune(hm_batch* b, const char* cache_path) {
  if (!b || b->magic != kMagicBatch) return bfail(HM_EINVAL, "not a batch handle");
  const std::string sig = signature(b);
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string s2;
      BatchKnobs k;
      if ((ls >> s2 >> k.grid_mult >> k.rc_cap >> k.rct_cap >> k.rt) && s2 == sig) {
        b->knobs = k;
        b->tuned = 2;
        int dev_prev = -1;
        cudaGetDevice(&dev_prev);
        if (dev_prev != b->device) cudaSetDevice(b->device);
        hm_status st = build_plan(b);
        if (dev_prev != b->device) cudaSetDevice(dev_prev);
        return st;
      }
    }
  }
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != b->device) cudaSetDevice(b->device);
  // temporary inputs (zeros) and outputs for timing
  std::vector<void*> xs(b->count, nullptr), ys(b->count, nullptr);
  hm_status st = HM_OK;
  for (int j = 0; j < b->count && st == HM_OK; ++j) {
    const size_t sz = static_cast<size_t>(std::max<int64_t>(b->mats[j]->n, 1)) * b->rs[j] * 4;
    if (cudaMalloc(&xs[j], sz) != cudaSuccess || cudaMalloc(&ys[j], sz) != cudaSuccess ||
        cudaMemset(xs[j], 0, sz) != cudaSuccess)
      st = bfail(HM_ENOMEM, "tuning buffers");
    b->h_io[j] = {xs[j], ys[j], std::max<int64_t>(b->mats[j]->n, 1), std::max<int64_t>(b->mats[j]->n, 1), HM_F32,
                  HM_F32};
  }
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == HM_OK && (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = bfail(HM_ECUDA, "tuning stream");
  auto time_knobs = [&](const BatchKnobs& k, float* ms) -> hm_status {
    b->knobs = k;
    hm_status s2 = build_plan(b);
    if (s2 != HM_OK) return s2;
    if (cudaMemcpy(b->d_io, b->h_io.data(), sizeof(BatchIO) * b->count, cudaMemcpyHostToDevice) != cudaSuccess)
      return bfail(HM_ECUDA, "tuning I/O upload");
    for (int w = 0; w < 2; ++w)
      if ((s2 = run_once(b, s)) != HM_OK) return s2;
    cudaEventRecord(e0, s);
    for (int it = 0; it < 5; ++it)
      if ((s2 = run_once(b, s)) != HM_OK) return s2;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return bfail(HM_ECUDA, "tuning run failed");
    cudaEventElapsedTime(ms, e0, e1);
    return HM_OK;
  };
  BatchKnobs best = b->knobs;
  float best_ms = 1e30f;
  if (st == HM_OK) st = time_knobs(best, &best_ms);
  // coordinate descent over the four knobs
  const int mults[] = {1, 2, 4};
  const int rcs[] = {8, 16, 32};
  const int rcts[] = {4, 8, 16};
  const int rts[] = {32, 64, 128};
  for (int knob = 0; knob < 4 && st == HM_OK; ++knob) {
    for (int v = 0; v < 3 && st == HM_OK; ++v) {
      BatchKnobs k = best;
      if (knob == 0) k.grid_mult = mults[v];
      if (knob == 1) k.rc_cap = rcs[v];
      if (knob == 2) k.rct_cap = rcts[v];
      if (knob == 3) k.rt = rts[v];
      float ms = 0.f;
      const hm_status s2 = time_knobs(k, &ms);
      if (s2 == HM_OK && ms < best_ms) {
        best_ms = ms;
        best = k;
      }
    }
  }
  b->knobs = best;
  if (st == HM_OK) st = build_plan(b);
  b->tuned = 1;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  for (int j = 0; j < b->count; ++j) {
    if (xs[j]) cudaFree(xs[j]);
    if (ys[j]) cudaFree(ys[j]);
  }
  if (dev_prev != b->device) cudaSetDevice(dev_prev);
  if (st == HM_OK && cache_path) {
    std::ofstream outf(cache_path, std::ios::app);
    if (outf) outf << sig << " " << best.grid_mult << " " << best.rc_cap << " " << best.rct_cap << " " << best.rt << "\n";
  }
  return st;
}

extern "C" hm_status hm_batch_info(const hm_batch* b, hm_batch_info_t* out) {
  if (!b || b->magic != kMagicBatch) return bfail(HM_EINVAL, "not a batch handle");
  if (!out) return bfail(HM_EINVAL, "out is NULL");
  std::memset(out, 0, sizeof(*out));
  out->count = b->count;
  int launches = 0;
  for (int p = 0; p < BP_COUNT; ++p) {
    out->items[p] = static_cast<int64_t>(b->items[p].size());
    out->grid[p] = b->grid[p];
    if (!b->items[p].empty()) ++launches;
  }
  out->launches_per_run = launches;
  out->graph = (b->use_graph && b->gexec) ? 1 : 0;
  out->capture_error = b->capture_error;
  out->tuned = b->tuned;
  out->grid_mult = b->knobs.grid_mult;
  out->rc_cap = b->knobs.rc_cap;
  out->rct_cap = b->knobs.rct_cap;
  out->tile_rows = b->knobs.rt;
  return HM_OK;
}

namespace hmi {

void destroy_other(void* any, uint32_t magic) {
  if (magic == kMagicBatch) destroy_batch(static_cast<hm_batch*>(any));
  else if (magic == kMagicServer) destroy_server(any);
  else if (is_ulv(any)) destroy_ulv(any);
}

}  // namespace hmi

// Host runtime of libhm: trees, generator packing, device memory, argument
// checking and dispatch of the products declared in include/hm.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "hm_api_internal.h"

namespace hmi {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

static hm_status fail(hm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

static hm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define HM_CUDA(call, what)                   \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// ----------------------------------------------------------------------------
// Per-device state: the status block of bounded device waits (the error word,
// then the wait limit in nanoseconds; see DeviceStatusBlock).
// ----------------------------------------------------------------------------

static std::mutex g_dev_mu;
static std::unordered_map<int, int*> g_dev_err;
static uint64_t g_wait_ns = kDefaultWaitNs;

int* device_error_word(int dev) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  auto it = g_dev_err.find(dev);
  if (it != g_dev_err.end()) return it->second;
  DeviceStatusBlock* p = nullptr;
  if (cudaMalloc(&p, sizeof(DeviceStatusBlock)) != cudaSuccess) return nullptr;
  DeviceStatusBlock h;
  h.err = 0;
  h.flag = 0;
  h.wait_ns = g_wait_ns;
  if (cudaMemcpy(p, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
  g_dev_err[dev] = &p->err;
  return &p->err;
}

// Host-side fault injection: the next g_alloc_fail device allocations fail.
static std::atomic<int> g_alloc_fail{0};

cudaError_t dev_malloc(void** p, size_t bytes) {
  int left = g_alloc_fail.load();
  while (left > 0) {
    if (g_alloc_fail.compare_exchange_weak(left, left - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(p, bytes);
}

// ----------------------------------------------------------------------------
// Round to nearest even float64 -> bfloat16 (bits).
// ----------------------------------------------------------------------------

uint16_t f64_to_bf16(double a) {
  if (std::isnan(a)) return 0x7fc0;
  if (a == 0.0) return std::signbit(a) ? 0x8000 : 0x0000;
  if (std::isinf(a)) return a > 0 ? 0x7f80 : 0xff80;
  int e = 0;
  (void)std::frexp(a, &e);            // a = m 2^e, 1/2 <= |m| < 1
  int qe = e - 8;                     // 8 significant bits
  if (qe < -133) qe = -133;           // subnormal quantum 2^-133
  const double v = std::nearbyint(std::ldexp(a, -qe));  // ties to even
  double rr = std::ldexp(v, qe);
  if (std::fabs(rr) > 3.3895313892515355e38) rr = a > 0 ? INFINITY : -INFINITY;
  const float f = static_cast<float>(rr);  // exact: every bfloat16 is a float
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  return static_cast<uint16_t>(bits >> 16);
}

double bf16_to_f64(uint16_t h) {
  const uint32_t bits = static_cast<uint32_t>(h) << 16;
  float f;
  std::memcpy(&f, &bits, 4);
  return f;
}

void Plane::init(int st, size_t cnt) {
  storage = st;
  count = cnt;
  const size_t es = (st == HM_F64) ? 8 : (st == HM_F32) ? 4 : 2;
  hi.assign(cnt * es, 0);
  if (st == HM_BF16X2) lo.assign(cnt * 2, 0);
  else lo.clear();
}

void Plane::set(size_t i, double v) {
  switch (storage) {
    case HM_F64: reinterpret_cast<double*>(hi.data())[i] = v; break;
    case HM_F32: reinterpret_cast<float*>(hi.data())[i] = static_cast<float>(v); break;
    case HM_BF16: reinterpret_cast<uint16_t*>(hi.data())[i] = f64_to_bf16(v); break;
    default: {
      const uint16_t h = f64_to_bf16(v);
      reinterpret_cast<uint16_t*>(hi.data())[i] = h;
      reinterpret_cast<uint16_t*>(lo.data())[i] = f64_to_bf16(v - bf16_to_f64(h));
    }
  }
}

size_t storage_bytes(int st) { return (st == HM_F64) ? 8 : (st == HM_F32) ? 4 : (st == HM_BF16) ? 2 : 4; }

}  // namespace hmi

using namespace hmi;

// ============================================================================
// Status strings
// ============================================================================

extern "C" const char* hm_status_string(hm_status s) {
  switch (s) {
    case HM_OK: return "HM_OK: success";
    case HM_EINVAL: return "HM_EINVAL: invalid argument";
    case HM_ENOMEM: return "HM_ENOMEM: out of memory or over budget";
    case HM_EBUSY: return "HM_EBUSY: no free slot, retry later";
    case HM_ETIMEOUT: return "HM_ETIMEOUT: bounded wait ran out";
    case HM_ECUDA: return "HM_ECUDA: CUDA runtime error";
    case HM_EUNSUPPORTED: return "HM_EUNSUPPORTED: outside this library's scope";
  }
  return "unknown hm_status";
}

extern "C" const char* hm_last_error(void) { return g_err.c_str(); }

extern "C" const char* hm_version(void) { return "hm 1.0 sm_103a"; }

// ============================================================================
// Trees
// ============================================================================

static hm_status make_tree(int64_t n, const std::vector<int64_t>& ends, hm_tree** out) {
  const size_t L = ends.size();
  if (L == 0 || (L & (L - 1)) != 0) return fail(HM_EINVAL, "number of leaves %zu is not a power of two", L);
  if (L > (size_t(1) << kMaxDepth)) return fail(HM_EINVAL, "tree deeper than %d levels", kMaxDepth);
  int64_t prev = 0;
  for (size_t i = 0; i < L; ++i) {
    if (ends[i] < prev) return fail(HM_EINVAL, "leaf ends must be non-decreasing (leaf %zu)", i);
    prev = ends[i];
  }
  if (ends.back() != n) return fail(HM_EINVAL, "last leaf end %lld != n %lld", (long long)ends.back(), (long long)n);
  hm_tree* t = new (std::nothrow) hm_tree();
  if (!t) return fail(HM_ENOMEM, "host allocation failed");
  t->magic = kMagicTree;
  t->n = n;
  t->L = static_cast<int>(L);
  int p = 0;
  while ((size_t(1) << p) < L) ++p;
  t->p = p;
  t->ends = ends;
  *out = t;
  return HM_OK;
}

extern "C" hm_status hm_tree_create(int64_t n, const int64_t* leaf_ends, int32_t num_leaves, hm_tree** out) {
  if (!out) return fail(HM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 0) return fail(HM_EINVAL, "n < 0");
  if (num_leaves < 1 || !leaf_ends) return fail(HM_EINVAL, "need num_leaves >= 1 and leaf_ends");
  std::vector<int64_t> ends(leaf_ends, leaf_ends + num_leaves);
  return make_tree(n, ends, out);
}

extern "C" hm_status hm_tree_default(int64_t n, int64_t n_min, hm_tree** out) {
  if (!out) return fail(HM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 0 || n_min < 1) return fail(HM_EINVAL, "need n >= 0 and n_min >= 1");
  // Sec. 3.1: {1..s} -> {1..ceil(s/2)} u rest, level by level while a node exceeds n_min.
  std::vector<std::pair<int64_t, int64_t>> iv{{0, n}};
  for (;;) {
    int64_t mx = 0;
    for (auto& x : iv) mx = std::max(mx, x.second - x.first);
    if (mx <= n_min) break;
    if (iv.size() >= (size_t(1) << kMaxDepth)) return fail(HM_EINVAL, "tree deeper than %d levels", kMaxDepth);
    std::vector<std::pair<int64_t, int64_t>> nx;
    nx.reserve(iv.size() * 2);
    for (auto& x : iv) {
      const int64_t h = (x.second - x.first + 1) / 2;
      nx.push_back({x.first, x.first + h});
      nx.push_back({x.first + h, x.second});
    }
    iv.swap(nx);
  }
  std::vector<int64_t> ends;
  ends.reserve(iv.size());
  for (auto& x : iv) ends.push_back(x.second);
  return make_tree(n, ends, out);
}

extern "C" hm_status hm_tree_shape(const hm_tree* t, int64_t* n, int32_t* depth, int32_t* num_leaves) {
  if (!t || t->magic != kMagicTree) return fail(HM_EINVAL, "not a tree handle");
  if (n) *n = t->n;
  if (depth) *depth = t->p;
  if (num_leaves) *num_leaves = t->L;
  return HM_OK;
}

extern "C" hm_status hm_tree_leaf_ends(const hm_tree* t, int64_t* leaf_ends) {
  if (!t || t->magic != kMagicTree) return fail(HM_EINVAL, "not a tree handle");
  if (!leaf_ends) return fail(HM_EINVAL, "leaf_ends is NULL");
  std::copy(t->ends.begin(), t->ends.end(), leaf_ends);
  return HM_OK;
}

// ============================================================================
// Matrices
// ============================================================================

namespace hmi {

int64_t node_start(const hm_tree* t, int q) {
  int lvl = 0;
  while (((2 << lvl) - 1) <= q) ++lvl;
  const int j = q - ((1 << lvl) - 1);
  const int64_t first = static_cast<int64_t>(j) << (t->p - lvl);
  return first > 0 ? t->ends[first - 1] : 0;
}

int64_t node_end(const hm_tree* t, int q) {
  int lvl = 0;
  while (((2 << lvl) - 1) <= q) ++lvl;
  const int j = q - ((1 << lvl) - 1);
  const int64_t last = (static_cast<int64_t>(j + 1) << (t->p - lvl)) - 1;
  return t->ends[last];
}

// Copy of a block that may live in device memory.
const double* host_block(const double* p, size_t count, std::vector<double>& tmp) {
  if (!p || count == 0) return p;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeDevice) {
    tmp.resize(count);
    if (cudaMemcpy(tmp.data(), p, count * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return nullptr;
    return tmp.data();
  }
  cudaGetLastError();
  return p;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

static hm_status upload(const void* h, size_t bytes, void** d, size_t* total) {
  *d = nullptr;
  if (bytes == 0) return HM_OK;
  HM_CUDA(dev_malloc(d, bytes), "cudaMalloc (generators)");
  HM_CUDA(cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice), "cudaMemcpy (generators)");
  *total += bytes;
  return HM_OK;
}

static void free_matrix_device(hm_matrix* A) {
  void* ptrs[] = {A->d_off, A->d_A, A->d_A_lo, A->d_W, A->d_W_lo, A->d_RU, A->d_RVt, A->d_B12,
                  A->d_B21, A->d_ws, A->d_cnt, A->d_io};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  A->d_off = nullptr;
}

}  // namespace hmi

hmi::MatView hm_matrix::view() const {
  using namespace hmi;
  MatView v;
  std::memset(&v, 0, sizeof(v));
  v.kind = kind;
  v.storage = storage;
  v.p = p;
  v.L = L;
  v.m_pad = m_pad;
  v.Ke = Ke;
  v.Kp = Kp;
  v.We = We;
  v.n = n;
  v.off = d_off;
  v.A = d_A;
  v.A_lo = d_A_lo;
  v.W = d_W;
  v.W_lo = d_W_lo;
  v.RU = d_RU;
  v.RV = d_RVt;
  v.B12 = d_B12;
  v.B21 = d_B21;
  for (int l = 0; l <= kMaxDepth + 1; ++l) {
    v.kk[l] = kk[l];
    v.koff[l] = koff[l];
  }
  return v;
}

namespace hmi {

static hm_status finish_create(hm_matrix* A, const hm_tree* t, Plane& Ap, Plane& Wp,
                               const std::vector<uint8_t>& tree_bytes_RU,
                               const std::vector<uint8_t>& tree_bytes_RVt,
                               const std::vector<uint8_t>& tree_bytes_B12,
                               const std::vector<uint8_t>& tree_bytes_B21, hm_matrix** out) {
  size_t dev = 0;
  std::vector<int64_t> off(t->L + 1, 0);
  for (int i = 0; i < t->L; ++i) off[i + 1] = t->ends[i];
  hm_status s;
  if ((s = upload(off.data(), off.size() * sizeof(int64_t), reinterpret_cast<void**>(&A->d_off), &dev)) != HM_OK ||
      (s = upload(Ap.hi.data(), Ap.hi.size(), &A->d_A, &dev)) != HM_OK ||
      (s = upload(Ap.lo.data(), Ap.lo.size(), &A->d_A_lo, &dev)) != HM_OK ||
      (s = upload(Wp.hi.data(), Wp.hi.size(), &A->d_W, &dev)) != HM_OK ||
      (s = upload(Wp.lo.data(), Wp.lo.size(), &A->d_W_lo, &dev)) != HM_OK ||
      (s = upload(tree_bytes_RU.data(), tree_bytes_RU.size(), &A->d_RU, &dev)) != HM_OK ||
      (s = upload(tree_bytes_RVt.data(), tree_bytes_RVt.size(), &A->d_RVt, &dev)) != HM_OK ||
      (s = upload(tree_bytes_B12.data(), tree_bytes_B12.size(), &A->d_B12, &dev)) != HM_OK ||
      (s = upload(tree_bytes_B21.data(), tree_bytes_B21.size(), &A->d_B21, &dev)) != HM_OK) {
    free_matrix_device(A);
    delete A;
    return s;
  }
  A->dev_bytes = dev;
  make_tensor_maps(A);
  A->err = device_error_word(A->device);
  if (!A->err) {
    free_matrix_device(A);
    delete A;
    return fail(HM_ECUDA, "could not allocate the device error word");
  }
  *out = A;
  return HM_OK;
}

static bool valid_storage(int st) { return st == HM_F64 || st == HM_F32 || st == HM_BF16 || st == HM_BF16X2; }

static hm_matrix* new_matrix(const hm_tree* t, int kind, int storage) {
  hm_matrix* A = new (std::nothrow) hm_matrix();
  if (!A) return nullptr;
  A->magic = kMagicMatrix;
  A->kind = kind;
  A->storage = storage;
  A->n = t->n;
  A->p = t->p;
  A->L = t->L;
  A->ends = t->ends;
  cudaGetDevice(&A->device);
  int64_t mmax = 0, prev = 0;
  for (int i = 0; i < t->L; ++i) {
    mmax = std::max(mmax, t->ends[i] - prev);
    prev = t->ends[i];
  }
  A->m_max = static_cast<int>(mmax);
  A->m_pad = round_up(std::max<int>(A->m_max, 1), 16);
  return A;
}

}  // namespace hmi

extern "C" hm_status hm_hodlr_create(const hm_tree* t, const hm_hodlr_gens* g, hm_dtype storage, hm_matrix** out) {
  if (!out) return fail(HM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!t || t->magic != kMagicTree) return fail(HM_EINVAL, "not a tree handle");
  if (!g || !g->D) return fail(HM_EINVAL, "generators missing");
  if (!valid_storage(storage)) return fail(HM_EINVAL, "unknown storage type %d", (int)storage);
  const int L = t->L, p = t->p;
  if (L > 1 && (!g->U12 || !g->V12 || !g->U21 || !g->V21 || !g->k12 || !g->k21))
    return fail(HM_EINVAL, "HODLR factor arrays missing");
  for (int q = 0; q < L - 1; ++q)
    if (g->k12[q] < 0 || g->k21[q] < 0 || g->k12[q] > 4096 || g->k21[q] > 4096)
      return fail(HM_EINVAL, "rank of node %d out of range", q);
  int64_t mmax = 0, prev = 0;
  for (int i = 0; i < L; ++i) { mmax = std::max(mmax, t->ends[i] - prev); prev = t->ends[i]; }
  if (mmax > 8192) return fail(HM_EUNSUPPORTED, "leaf size %lld above 8192", (long long)mmax);
  hm_matrix* A = new_matrix(t, HM_HODLR, storage);
  if (!A) return fail(HM_ENOMEM, "host allocation failed");
  // Per-level padded ranks and offsets.
  A->koff[1] = 0;
  for (int l = 1; l <= p; ++l) {
    int k = 0;
    for (int j = 0; j < (1 << (l - 1)); ++j) {
      const int q = (1 << (l - 1)) - 1 + j;
      k = std::max(k, std::max(g->k12[q], g->k21[q]));
    }
    A->kk[l] = k;
    A->koff[l + 1] = A->koff[l] + k;
  }
  A->Ke = A->Kp = round_up(A->koff[p + 1], 8);
  A->We = A->m_pad + A->Ke;
  const int64_t n = t->n;
  Plane Ap, Wp;
  Ap.init(storage, static_cast<size_t>(n) * A->We);
  Wp.init(storage, static_cast<size_t>(L) * A->Kp * A->m_pad);
  std::vector<double> tmp;
  int64_t elems = 0;
  for (int i = 0; i < L; ++i) {
    const int64_t a0 = (i > 0) ? t->ends[i - 1] : 0;
    const int64_t m = t->ends[i] - a0;
    if (m == 0) continue;
    const double* D = host_block(g->D[i], static_cast<size_t>(m * m), tmp);
    if (!D) { delete A; return fail(HM_EINVAL, "D[%d] is NULL or unreadable", i); }
    for (int64_t rr = 0; rr < m; ++rr)
      for (int64_t cc = 0; cc < m; ++cc) Ap.set(static_cast<size_t>(a0 + rr) * A->We + cc, D[rr + cc * m]);
    elems += m * m;
  }
  for (int l = 1; l <= p; ++l) {
    for (int j = 0; j < (1 << l); ++j) {
      const int anc = (1 << l) - 1 + j;
      const int q = (anc - 1) / 2;
      const bool left = (anc & 1) != 0;
      const int64_t s0 = node_start(t, anc), s1 = node_end(t, anc);
      const int64_t ms = s1 - s0;
      if (ms == 0) continue;
      const int kU = left ? g->k12[q] : g->k21[q];
      const int kV = left ? g->k21[q] : g->k12[q];
      std::vector<double> tu, tv;
      const double* Uf = host_block(left ? g->U12[q] : g->U21[q], static_cast<size_t>(ms * kU), tu);
      const double* Vf = host_block(left ? g->V21[q] : g->V12[q], static_cast<size_t>(ms * kV), tv);
      if ((kU > 0 && !Uf) || (kV > 0 && !Vf)) { delete A; return fail(HM_EINVAL, "factor of node %d missing", q); }
      elems += ms * (kU + kV);
      for (int64_t g0 = s0; g0 < s1; ++g0) {
        const int64_t rr = g0 - s0;
        for (int a = 0; a < kU; ++a)
          Ap.set(static_cast<size_t>(g0) * A->We + A->m_pad + A->koff[l] + a, Uf[rr + a * ms]);
      }
      // Projection rows of every leaf below this node.
      const int span = 1 << (p - l);
      for (int leaf = j * span; leaf < (j + 1) * span; ++leaf) {
        const int64_t a0 = (leaf > 0) ? t->ends[leaf - 1] : 0;
        const int64_t a1 = t->ends[leaf];
        for (int a = 0; a < kV; ++a)
          for (int64_t g0 = a0; g0 < a1; ++g0)
            Wp.set((static_cast<size_t>(leaf) * A->Kp + A->koff[l] + a) * A->m_pad + (g0 - a0),
                   Vf[(g0 - s0) + a * ms]);
      }
    }
  }
  A->gen_elems = elems;
  A->gen_bytes = static_cast<size_t>(elems) * storage_bytes(storage);
  std::vector<uint8_t> none;
  return finish_create(A, t, Ap, Wp, none, none, none, none, out);
}

extern "C" hm_status hm_hss_create(const hm_tree* t, const hm_hss_gens* g, hm_dtype storage, hm_matrix** out) {
  if (!out) return fail(HM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!t || t->magic != kMagicTree) return fail(HM_EINVAL, "not a tree handle");
  if (!g || !g->D || !g->U || !g->V || !g->ku || !g->kv) return fail(HM_EINVAL, "generators missing");
  if (!valid_storage(storage)) return fail(HM_EINVAL, "unknown storage type %d", (int)storage);
  const int L = t->L;
  const int N = 2 * L - 1;
  if (L > 1 && (!g->RU || !g->RV || !g->B12 || !g->B21)) return fail(HM_EINVAL, "HSS operator arrays missing");
  int ku_max = 0, kv_max = 0;
  for (int q = 1; q < N; ++q) {
    if (g->ku[q] < 0 || g->kv[q] < 0 || g->ku[q] > 2048 || g->kv[q] > 2048)
      return fail(HM_EINVAL, "rank of node %d out of range", q);
    ku_max = std::max(ku_max, g->ku[q]);
    kv_max = std::max(kv_max, g->kv[q]);
  }
  int64_t mmax = 0, prev = 0;
  for (int i = 0; i < L; ++i) { mmax = std::max(mmax, t->ends[i] - prev); prev = t->ends[i]; }
  if (mmax > 8192) return fail(HM_EUNSUPPORTED, "leaf size %lld above 8192", (long long)mmax);
  hm_matrix* A = new_matrix(t, HM_HSS, storage);
  if (!A) return fail(HM_ENOMEM, "host allocation failed");
  const int Ke = round_up(ku_max, 8), Kp = round_up(kv_max, 8);
  A->Ke = Ke;
  A->Kp = Kp;
  A->ku_max = ku_max;
  A->kv_max = kv_max;
  A->We = A->m_pad + Ke;
  const int64_t n = t->n;
  Plane Ap, Wp;
  Ap.init(storage, static_cast<size_t>(n) * A->We);
  Wp.init(storage, static_cast<size_t>(L) * Kp * A->m_pad);
  std::vector<double> tmp, tu, tv;
  int64_t elems = 0;
  for (int i = 0; i < L; ++i) {
    const int64_t a0 = (i > 0) ? t->ends[i - 1] : 0;
    const int64_t m = t->ends[i] - a0;
    const int nodeid = L - 1 + i;
    // A single-leaf tree has no off-diagonal blocks: its U, V take no part.
    const int ku = (L > 1) ? g->ku[nodeid] : 0, kv = (L > 1) ? g->kv[nodeid] : 0;
    if (m == 0) continue;
    const double* D = host_block(g->D[i], static_cast<size_t>(m * m), tmp);
    const double* U = host_block(g->U[i], static_cast<size_t>(m * ku), tu);
    const double* V = host_block(g->V[i], static_cast<size_t>(m * kv), tv);
    if (!D || (ku && !U) || (kv && !V)) { delete A; return fail(HM_EINVAL, "leaf %d generators missing", i); }
    for (int64_t rr = 0; rr < m; ++rr) {
      const size_t row = static_cast<size_t>(a0 + rr) * A->We;
      for (int64_t cc = 0; cc < m; ++cc) Ap.set(row + cc, D[rr + cc * m]);
      for (int a = 0; a < ku; ++a) Ap.set(row + A->m_pad + a, U[rr + a * m]);
      for (int a = 0; a < kv; ++a) Wp.set((static_cast<size_t>(i) * Kp + a) * A->m_pad + rr, V[rr + a * m]);
    }
    elems += m * m + m * (ku + kv);
  }
  // Tree operators in the compute type.
  const bool dbl = (storage == HM_F64);
  const size_t cs = dbl ? 8 : 4;
  auto put = [&](std::vector<uint8_t>& buf, size_t idx, double v) {
    if (dbl) reinterpret_cast<double*>(buf.data())[idx] = v;
    else reinterpret_cast<float*>(buf.data())[idx] = static_cast<float>(v);
  };
  // Device layouts (compute type), one block per internal node q:
  //   RUt[q][h][j][i] = R_U(h*Ke + i, j)  -- the child half h of R_U, transposed
  //   RV [q][j][i]    = R_V(j, i)         -- rows of the stacked children, row-major
  //   B12t[q][j][i]   = B12(i, j), B21t[q][j][i] = B21(i, j)
  std::vector<uint8_t> RU, RVt, B12, B21;
  const size_t nI = static_cast<size_t>(std::max(L - 1, 0));
  RU.assign(nI * 2 * Ke * Ke * cs, 0);
  RVt.assign(nI * 2 * Kp * Kp * cs, 0);
  B12.assign(nI * Kp * Ke * cs, 0);
  B21.assign(nI * Kp * Ke * cs, 0);
  int64_t telems = 0;
  for (int q = 0; q < L - 1; ++q) {
    const int a = 2 * q + 1, b = 2 * q + 2;
    const int kua = g->ku[a], kub = g->ku[b], kva = g->kv[a], kvb = g->kv[b];
    if (q > 0) {
      const int kuq = g->ku[q], kvq = g->kv[q];
      const double* R = host_block(g->RU[q], static_cast<size_t>((kua + kub) * kuq), tmp);
      if ((kua + kub) * kuq > 0 && !R) { delete A; return fail(HM_EINVAL, "RU[%d] missing", q); }
      for (int rr = 0; rr < kua + kub; ++rr) {
        const int h = rr < kua ? 0 : 1;
        const int i = rr < kua ? rr : rr - kua;
        for (int j = 0; j < kuq; ++j)
          put(RU, ((static_cast<size_t>(q) * 2 + h) * Ke + j) * Ke + i, R[rr + j * (kua + kub)]);
      }
      const double* W = host_block(g->RV[q], static_cast<size_t>((kva + kvb) * kvq), tmp);
      if ((kva + kvb) * kvq > 0 && !W) { delete A; return fail(HM_EINVAL, "RV[%d] missing", q); }
      for (int rr = 0; rr < kva + kvb; ++rr) {
        const int prow = rr < kva ? rr : Kp + (rr - kva);
        for (int cc = 0; cc < kvq; ++cc)
          put(RVt, (static_cast<size_t>(q) * 2 * Kp + prow) * Kp + cc, W[rr + cc * (kva + kvb)]);
      }
      telems += static_cast<int64_t>(kua + kub) * kuq + static_cast<int64_t>(kva + kvb) * kvq;
    }
    const double* S12 = host_block(g->B12[q], static_cast<size_t>(kua * kvb), tmp);
    if (kua * kvb > 0 && !S12) { delete A; return fail(HM_EINVAL, "B12[%d] missing", q); }
    for (int i = 0; i < kua; ++i)
      for (int j = 0; j < kvb; ++j) put(B12, (static_cast<size_t>(q) * Kp + j) * Ke + i, S12[i + j * kua]);
    const double* S21 = host_block(g->B21[q], static_cast<size_t>(kub * kva), tmp);
    if (kub * kva > 0 && !S21) { delete A; return fail(HM_EINVAL, "B21[%d] missing", q); }
    for (int i = 0; i < kub; ++i)
      for (int j = 0; j < kva; ++j) put(B21, (static_cast<size_t>(q) * Kp + j) * Ke + i, S21[i + j * kub]);
    telems += static_cast<int64_t>(kua) * kvb + static_cast<int64_t>(kub) * kva;
  }
  A->gen_elems = elems + telems;
  A->gen_bytes = static_cast<size_t>(elems) * storage_bytes(storage) + static_cast<size_t>(telems) * cs;
  return finish_create(A, t, Ap, Wp, RU, RVt, B12, B21, out);
}

extern "C" hm_status hm_matrix_info(const hm_matrix* A, hm_matrix_info_t* out) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (!out) return fail(HM_EINVAL, "out is NULL");
  out->kind = A->kind;
  out->storage = A->storage;
  out->n = A->n;
  out->depth = A->p;
  out->num_leaves = A->L;
  out->leaf_pad = A->m_pad;
  out->rank_total = A->Ke;
  out->generator_elements = A->gen_elems;
  out->generator_bytes = A->gen_bytes;
  out->device_bytes = A->dev_bytes;
  const bool cl = A->tree_ok_r >= 0 && A->tree_ok && A->tree_mode != 1 && A->tree_last_cluster;
  out->tree_cluster = cl ? (1 << A->tree_s) : 0;
  out->tree_columns = cl ? A->tree_rc : 0;
  out->tree_ring = cl ? A->tree_ns : 0;
  out->rank_col = A->Kp;
  return HM_OK;
}

extern "C" hm_status hm_matrix_bytes(const hm_matrix* A, size_t* bytes) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (!bytes) return fail(HM_EINVAL, "bytes is NULL");
  *bytes = A->gen_bytes;
  return HM_OK;
}

extern "C" hm_status hm_matrix_set_path(hm_matrix* A, int32_t path) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (path < 0 || path > 2) return fail(HM_EINVAL, "path must be 0, 1 or 2");
  A->path = path;
  return HM_OK;
}

extern "C" hm_status hm_matrix_set_tree(hm_matrix* A, int32_t mode) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (mode < 0 || mode > 2) return fail(HM_EINVAL, "tree mode must be 0, 1 or 2");
  A->tree_mode = mode;
  return HM_OK;
}

namespace hmi {

size_t scratch_elems(const MatView& mv, int64_t r) {
  const size_t nodes = static_cast<size_t>(2 * mv.L - 1);
  if (mv.kind == HM_HODLR) return nodes * r * mv.Ke;
  // x-hat, y (couplings), y-hat, then the cluster tree kernel's couplings
  // (one Ke x RC block per node and column chunk, r rounded up to 8)
  const size_t r8 = static_cast<size_t>((r + 7) / 8) * 8;
  return nodes * r * (mv.Kp + 2 * static_cast<size_t>(mv.Ke)) + nodes * r8 * mv.Ke;
}

size_t tree_counter_count(const MatView& mv, int64_t r) {
  return static_cast<size_t>(std::max(mv.L - 1, 1)) * static_cast<size_t>(std::max<int64_t>(r, 1));
}

size_t counter_count(const MatView& mv, int64_t r) { return tree_counter_count(mv, r) + 8; }

hm_status ensure_scratch(hm_matrix* A, int64_t r) {
  if (r <= A->r_cap && A->d_ws) return HM_OK;
  const MatView mv = A->view();
  const size_t cs = (A->storage == HM_F64) ? 8 : 4;
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != A->device) cudaSetDevice(A->device);
  if (A->d_ws) { cudaDeviceSynchronize(); cudaFree(A->d_ws); A->d_ws = nullptr; }
  if (A->d_cnt) { cudaFree(A->d_cnt); A->d_cnt = nullptr; }
  A->r_cap = 0;
  const size_t wb = std::max<size_t>(scratch_elems(mv, r) * cs, 256);
  const size_t cb = counter_count(mv, r) * sizeof(int);
  cudaError_t e = dev_malloc(&A->d_ws, wb);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&A->d_cnt), cb);
  if (e == cudaSuccess) e = cudaMemset(A->d_cnt, 0, cb);
  if (e == cudaSuccess) e = cudaMemset(A->d_ws, 0, wb);
  if (dev_prev != A->device) cudaSetDevice(dev_prev);
  if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
  A->r_cap = r;
  return HM_OK;
}

Scratch scratch_of(const hm_matrix* A, int64_t r) {
  Scratch s;
  std::memset(&s, 0, sizeof(s));
  const size_t cs = (A->storage == HM_F64) ? 8 : 4;
  const size_t nodes = static_cast<size_t>(2 * A->L - 1);
  char* base = static_cast<char*>(A->d_ws);
  if (A->kind == HM_HODLR) {
    s.PS = base;
  } else {
    s.xh = base;
    s.yc = base + nodes * r * A->Kp * cs;
    s.yf = base + nodes * r * (A->Kp + A->Ke) * cs;
  }
  s.cnt = A->d_cnt;
  s.err = A->err;
  return s;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

hm_status run_product(const hm_matrix* Ac, int want_kind, int64_t r, const void* X, int64_t ldx, int xt, void* Y,
                      int64_t ldy, int yt, void* stream) {
  if (!Ac || Ac->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  hm_matrix* A = const_cast<hm_matrix*>(Ac);
  if (A->kind != want_kind)
    return fail(HM_EINVAL, "matrix is %s, called the %s product", A->kind == HM_HSS ? "HSS" : "HODLR",
                want_kind == HM_HSS ? "HSS" : "HODLR");
  if (r < 0) return fail(HM_EINVAL, "r < 0");
  const int64_t n = A->n;
  if (ldx < std::max<int64_t>(n, 1) || ldy < std::max<int64_t>(n, 1)) return fail(HM_EINVAL, "ldx/ldy < n");
  if (xt != HM_F64 && xt != HM_F32 && xt != HM_BF16) return fail(HM_EINVAL, "X type must be F64, F32 or BF16");
  if (yt != HM_F64 && yt != HM_F32) return fail(HM_EINVAL, "Y type must be F64 or F32");
  if (A->storage == HM_F64 && (xt != HM_F64 || yt != HM_F64))
    return fail(HM_EUNSUPPORTED, "F64 storage needs F64 X and Y");
  if (r == 0 || n == 0) return HM_OK;
  if (!X || !Y) return fail(HM_EINVAL, "X or Y is NULL");
  const size_t xs = (xt == HM_F64) ? 8 : (xt == HM_F32) ? 4 : 2;
  const size_t ys = (yt == HM_F64) ? 8 : 4;
  {
    const char* x0 = static_cast<const char*>(X);
    const char* x1 = x0 + ((r - 1) * ldx + n) * xs;
    const char* y0 = static_cast<const char*>(Y);
    const char* y1 = y0 + ((r - 1) * ldy + n) * ys;
    if (x0 < y1 && y0 < x1) return fail(HM_EINVAL, "X and Y overlap");
  }
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != A->device) HM_CUDA(cudaSetDevice(A->device), "cudaSetDevice");
  struct Restore {
    int d, cur;
    ~Restore() { if (d != cur && d >= 0) cudaSetDevice(d); }
  } restore{dev_prev, A->device};
  hm_status st = ensure_scratch(A, r);
  if (st != HM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool xdev = is_device_ptr(X), ydev = is_device_ptr(Y);
  const void* Xd = X;
  void* Yd = Y;
  int64_t ldxd = ldx, ldyd = ldy;
  if (!xdev || !ydev) {
    const size_t need = static_cast<size_t>(n) * r * (xs + ys) + 256;
    if (A->io_cap < need) {
      if (A->d_io) { cudaStreamSynchronize(s); cudaFree(A->d_io); A->d_io = nullptr; A->io_cap = 0; }
      HM_CUDA(dev_malloc(&A->d_io, need), "cudaMalloc (host staging)");
      A->io_cap = need;
    }
    char* base = static_cast<char*>(A->d_io);
    if (!xdev) {
      HM_CUDA(cudaMemcpy2DAsync(base, n * xs, X, ldx * xs, n * xs, r, cudaMemcpyHostToDevice, s), "copy X to device");
      Xd = base;
      ldxd = n;
    }
    if (!ydev) {
      Yd = base + ((static_cast<size_t>(n) * r * xs + 255) / 256) * 256;
      ldyd = n;
    }
  }
  const MatView mv = A->view();
  Scratch ws = scratch_of(A, r);
  ws.prof = A->prof;
  st = launch_product(A, mv, ws, r, Xd, ldxd, xt, Yd, ldyd, yt, s);
  if (st != HM_OK) return st;
  if (!ydev) {
    HM_CUDA(cudaMemcpy2DAsync(Y, ldy * ys, Yd, n * ys, n * ys, r, cudaMemcpyDeviceToHost, s), "copy Y to host");
  }
  if (!xdev || !ydev) HM_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  return HM_OK;
}

hm_status launch_product(hm_matrix* A, const MatView& mv, const Scratch& ws, int64_t r, const void* X,
                         int64_t ldx, int xt, void* Y, int64_t ldy, int yt, cudaStream_t s) {
  auto phase = [&](int ph, bool pdl) -> hm_status {
    switch (mv.storage) {
      case HM_F64: return simt_phase_f64(ph, mv, ws, r, X, ldx, xt, Y, ldy, yt, s, pdl);
      case HM_F32: return simt_phase_f32(ph, mv, ws, r, X, ldx, xt, Y, ldy, yt, s, pdl);
      case HM_BF16: return simt_phase_bf16(ph, mv, ws, r, X, ldx, xt, Y, ldy, yt, s, pdl);
      default: return simt_phase_bf16x2(ph, mv, ws, r, X, ldx, xt, Y, ldy, yt, s, pdl);
    }
  };
  if (f64_tiled(mv, r)) {
    // FP64, wide blocks, one stream: projection -> tree -> D X (programmatic
    // launch: it may start beside the tree) -> Y += E Z
    prof_mark(ws.prof, 0, true, s);
    hm_status st = f64_leaf_phase(0, mv, ws, r, X, ldx, Y, ldy, s, false, 0);
    prof_mark(ws.prof, 0, false, s);
    if (st != HM_OK) return st;
    st = launch_tree_cluster(A, mv, ws, r, s, true);
    A->tree_last_cluster = (st == HM_OK);
    if (st == HM_EUNSUPPORTED) {
      st = phase(1, true);
      if (st != HM_OK) return st;
      st = phase(2, true);
    }
    if (st != HM_OK) return st;
    prof_mark(ws.prof, 4, true, s);
    st = f64_leaf_phase(1, mv, ws, r, X, ldx, Y, ldy, s, true, 0);
    prof_mark(ws.prof, 4, false, s);
    if (st != HM_OK) return st;
    prof_mark(ws.prof, 3, true, s);
    st = f64_leaf_phase(2, mv, ws, r, X, ldx, Y, ldy, s, true, 0);
    prof_mark(ws.prof, 3, false, s);
    return st;
  }
  hm_status st = HM_EUNSUPPORTED;
  if (use_tensor_cores(A, r)) st = launch_project_tc(A, mv, ws, r, X, ldx, xt, s, false);
  if (st == HM_EUNSUPPORTED) st = phase(0, false);
  if (st != HM_OK) return st;
  st = launch_tree_cluster(A, mv, ws, r, s, true);
  A->tree_last_cluster = (st == HM_OK);
  if (st == HM_EUNSUPPORTED) {
    st = phase(1, true);
    if (st != HM_OK) return st;
    st = phase(2, true);
  }
  if (st != HM_OK) return st;
  if (use_tensor_cores(A, r)) {
    st = launch_expand_tc(A, mv, ws, r, X, ldx, xt, Y, ldy, yt, s, true);
    if (st != HM_EUNSUPPORTED) return st;
  }
  return phase(3, true);
}

}  // namespace hmi

namespace hmi {

cudaEvent_t EventProf::get() {
  if (!pool_.empty()) {
    cudaEvent_t e = pool_.back();
    pool_.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void EventProf::mark(int phase, bool start, cudaStream_t s) {
  cudaEvent_t e = get();
  cudaEventRecord(e, s);
  if (start) {
    open_[phase] = e;
  } else {
    recs_.push_back({phase, open_[phase], e});
    open_[phase] = nullptr;
  }
}

hm_status EventProf::read(double ms[kPhaseSlots], int64_t launches[kPhaseSlots]) {
  for (auto& r : recs_) {
    HM_CUDA(cudaEventSynchronize(r.b), "event synchronize");
    float t = 0.f;
    HM_CUDA(cudaEventElapsedTime(&t, r.a, r.b), "event elapsed");
    ms_[r.phase] += t;
    n_[r.phase] += 1;
    pool_.push_back(r.a);
    pool_.push_back(r.b);
  }
  recs_.clear();
  for (int i = 0; i < kPhaseSlots; ++i) {
    ms[i] = ms_[i];
    launches[i] = n_[i];
    ms_[i] = 0;
    n_[i] = 0;
  }
  return HM_OK;
}

EventProf::~EventProf() {
  for (auto& r : recs_) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : pool_) cudaEventDestroy(e);
}

}  // namespace hmi

extern "C" hm_status hm_matrix_profile(hm_matrix* A, int32_t enable) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (enable && !A->prof) A->prof = new (std::nothrow) EventProf();
  if (!enable && A->prof) {
    delete A->prof;
    A->prof = nullptr;
  }
  return HM_OK;
}

extern "C" hm_status hm_matrix_phase_times(hm_matrix* A, double ms[5], int64_t launches[5]) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (!ms || !launches) return fail(HM_EINVAL, "output arrays are NULL");
  if (!A->prof) {
    for (int i = 0; i < kPhaseSlots; ++i) { ms[i] = 0; launches[i] = 0; }
    return HM_OK;
  }
  return static_cast<EventProf*>(A->prof)->read(ms, launches);
}

extern "C" hm_status hm_matrix_tune_tree(hm_matrix* A, int64_t r, hm_dtype xt, hm_dtype yt, double* best_ms) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (r < 1) return fail(HM_EINVAL, "r < 1");
  if (xt != HM_F64 && xt != HM_F32 && xt != HM_BF16) return fail(HM_EINVAL, "X type must be F64, F32 or BF16");
  if (yt != HM_F64 && yt != HM_F32) return fail(HM_EINVAL, "Y type must be F64 or F32");
  if (A->storage == HM_F64 && (xt != HM_F64 || yt != HM_F64))
    return fail(HM_EUNSUPPORTED, "F64 storage needs F64 X and Y");
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != A->device) cudaSetDevice(A->device);
  const hm_status s = tune_tree_cluster(A, r, xt, yt, best_ms);
  if (dev_prev != A->device) cudaSetDevice(dev_prev);
  if (s == HM_EUNSUPPORTED) return fail(HM_EUNSUPPORTED, "no cluster tree shape fits this matrix");
  return s;
}

extern "C" hm_status hm_matrix_set_tree_shape(hm_matrix* A, int64_t r, int32_t cluster_ctas, int32_t columns,
                                              int32_t ring_slots) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (r < 1) return fail(HM_EINVAL, "r < 1");
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != A->device) cudaSetDevice(A->device);
  const hm_status s = set_tree_shape(A, r, cluster_ctas, columns, ring_slots);
  if (dev_prev != A->device) cudaSetDevice(dev_prev);
  if (s == HM_EINVAL)
    return fail(HM_EINVAL, "tree shape: cluster_ctas a power of two from 2 to 16 and at most 2^depth, columns 1, 2, "
                           "4 or 8, ring_slots 2..12 for HSS and 0 for HODLR");
  if (s == HM_EUNSUPPORTED) return fail(HM_EUNSUPPORTED, "this tree shape does not fit this matrix");
  return s;
}

extern "C" hm_status hm_matrix_reserve(hm_matrix* A, int64_t r_max) {
  if (!A || A->magic != kMagicMatrix) return fail(HM_EINVAL, "not a matrix handle");
  if (r_max < 1) return fail(HM_EINVAL, "r_max < 1");
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != A->device) cudaSetDevice(A->device);
  hm_status s = ensure_scratch(A, r_max);
  if (dev_prev != A->device) cudaSetDevice(dev_prev);
  return s;
}

extern "C" hm_status hm_hodlr_matmat(const hm_matrix* A, int64_t r, const void* X, int64_t ldx, hm_dtype xt,
                                     void* Y, int64_t ldy, hm_dtype yt, void* stream) {
  return run_product(A, HM_HODLR, r, X, ldx, xt, Y, ldy, yt, stream);
}

extern "C" hm_status hm_hss_matmat(const hm_matrix* A, int64_t r, const void* X, int64_t ldx, hm_dtype xt,
                                   void* Y, int64_t ldy, hm_dtype yt, void* stream) {
  return run_product(A, HM_HSS, r, X, ldx, xt, Y, ldy, yt, stream);
}

extern "C" hm_status hm_device_status(void* stream) {
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  HM_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream synchronize");
  int* w = device_error_word(dev);
  if (!w) return fail(HM_ECUDA, "no device error word");
  int v = 0;
  HM_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (v != 0) {
    HM_CUDA(cudaMemset(w, 0, sizeof(int)), "clear error word");
    return fail(HM_ETIMEOUT, "a device-side bounded wait timed out (code %d)", v);
  }
  return HM_OK;
}

extern "C" hm_status hm_set_device_wait_limit(uint64_t ns) {
  if (ns < 1000 || ns > 60000000000ull) return fail(HM_EINVAL, "wait limit must be in [1e3, 6e10] ns");
  std::lock_guard<std::mutex> lk(g_dev_mu);
  g_wait_ns = ns;
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  for (auto& kv : g_dev_err) {
    cudaSetDevice(kv.first);
    DeviceStatusBlock* b = reinterpret_cast<DeviceStatusBlock*>(kv.second);
    const cudaError_t e = cudaMemcpy(&b->wait_ns, &ns, sizeof(ns), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (dev_prev >= 0) cudaSetDevice(dev_prev);
      return cuda_fail(e, "write the device wait limit");
    }
  }
  if (dev_prev >= 0) cudaSetDevice(dev_prev);
  return HM_OK;
}

extern "C" hm_status hm_get_device_wait_limit(uint64_t* ns) {
  if (!ns) return fail(HM_EINVAL, "ns is NULL");
  std::lock_guard<std::mutex> lk(g_dev_mu);
  *ns = g_wait_ns;
  return HM_OK;
}

extern "C" hm_status hm_inject_alloc_failures(int32_t count) {
  if (count < 0) return fail(HM_EINVAL, "count < 0");
  g_alloc_fail.store(count);
  return HM_OK;
}

extern "C" hm_status hm_selftest_device_timeout(void* stream) {
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  int* w = device_error_word(dev);
  if (!w) return fail(HM_ECUDA, "no device status block");
  return launch_selftest_timeout(reinterpret_cast<DeviceStatusBlock*>(w), static_cast<cudaStream_t>(stream));
}

extern "C" void hm_destroy(void* any) {
  if (!any) return;
  const uint32_t magic = *static_cast<const uint32_t*>(any);
  if (magic == kMagicTree) {
    hm_tree* t = static_cast<hm_tree*>(any);
    t->magic = 0;
    delete t;
  } else if (magic == kMagicMatrix) {
    hm_matrix* A = static_cast<hm_matrix*>(any);
    A->magic = 0;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != A->device) cudaSetDevice(A->device);
    delete A->prof;
    A->prof = nullptr;
    free_matrix_device(A);
    if (dev_prev != A->device) cudaSetDevice(dev_prev);
    delete A;
  } else {
    destroy_other(any, magic);
  }
}

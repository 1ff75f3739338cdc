// hm_matmat_noalloc: the HODLR/HSS product with its scratch in a fixed,
// statically allocated device array instead of memory the library allocates.
//
// Some callers cannot allocate device memory at the point where they need a
// product: real-time or serving loops that must not stall on cudaMalloc's
// implicit device synchronisation, and applications that hand every byte of
// the GPU to their own allocator (a framework's caching allocator, a memory
// pool sized at start-up), where a library-side cudaMalloc can fail or
// fragment that pool.  This entry point lets them run the product with no
// allocation at all: the matrix is created beforehand, X and Y are the
// caller's device buffers, and the per-call scratch (tree intermediates and
// arrival counters) lives in the array below.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "hm_api_internal.h"

namespace hmi {

// 8 MiB of scratch, 256-byte aligned.  Every GPU that loads the library holds
// it until the process exits.  All calls share it: two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on it.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device (with that device
// current).  In host code the symbol is only a host-side stand-in; kernels must
// be given the address returned here.
static std::mutex g_na_mu;
static std::unordered_map<int, unsigned char*> g_na_ptr;

static hm_status noalloc_base(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  auto it = g_na_ptr.find(dev);
  if (it != g_na_ptr.end()) {
    *out = it->second;
    return HM_OK;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  g_na_ptr[dev] = static_cast<unsigned char*>(p);
  *out = static_cast<unsigned char*>(p);
  return HM_OK;
}

size_t noalloc_required_bytes(const hm_matrix* A, int64_t r) {
  const MatView mv = A->view();
  const size_t cs = (A->storage == HM_F64) ? 8 : 4;
  const size_t data = ((scratch_elems(mv, r) * cs + 255) / 256) * 256;
  return data + counter_count(mv, r) * sizeof(int);
}

}  // namespace hmi

using namespace hmi;

extern "C" hm_status hm_matmat_noalloc(const hm_matrix* Ac, int64_t r, const void* X, int64_t ldx, hm_dtype xt,
                                       void* Y, int64_t ldy, hm_dtype yt, void* stream) {
  if (!Ac || Ac->magic != kMagicMatrix) {
    set_error("not a matrix handle");
    return HM_EINVAL;
  }
  hm_matrix* A = const_cast<hm_matrix*>(Ac);
  if (r < 0) { set_error("r < 0"); return HM_EINVAL; }
  const int64_t n = A->n;
  if (ldx < std::max<int64_t>(n, 1) || ldy < std::max<int64_t>(n, 1)) { set_error("ldx/ldy < n"); return HM_EINVAL; }
  if (xt != HM_F64 && xt != HM_F32 && xt != HM_BF16) { set_error("X type must be F64, F32 or BF16"); return HM_EINVAL; }
  if (yt != HM_F64 && yt != HM_F32) { set_error("Y type must be F64 or F32"); return HM_EINVAL; }
  if (A->storage == HM_F64 && (xt != HM_F64 || yt != HM_F64)) {
    set_error("F64 storage needs F64 X and Y");
    return HM_EUNSUPPORTED;
  }
  if (r == 0 || n == 0) return HM_OK;
  if (!X || !Y) { set_error("X or Y is NULL"); return HM_EINVAL; }
  {
    // the leaf expansion writes Y while the diagonal-block term still reads X
    const size_t xs = (xt == HM_F64) ? 8 : (xt == HM_F32) ? 4 : 2;
    const size_t ys = (yt == HM_F64) ? 8 : 4;
    const char* x0 = static_cast<const char*>(X);
    const char* x1 = x0 + ((r - 1) * ldx + n) * xs;
    const char* y0 = static_cast<const char*>(Y);
    const char* y1 = y0 + ((r - 1) * ldy + n) * ys;
    if (x0 < y1 && y0 < x1) { set_error("X and Y overlap"); return HM_EINVAL; }
  }
  const size_t need = noalloc_required_bytes(A, r);
  if (need > kNoAllocScratchBytes) {
    set_error("hm_matmat_noalloc: this product needs %zu bytes of scratch, above the fixed %zu-byte limit "
              "(use fewer right-hand sides per call or hm_hodlr_matmat / hm_hss_matmat)",
              need, kNoAllocScratchBytes);
    return HM_EINVAL;
  }
  // X and Y must already be device memory: staging host buffers would allocate.
  cudaPointerAttributes ax, ay;
  if (cudaPointerGetAttributes(&ax, X) != cudaSuccess || cudaPointerGetAttributes(&ay, Y) != cudaSuccess ||
      (ax.type != cudaMemoryTypeDevice && ax.type != cudaMemoryTypeManaged) ||
      (ay.type != cudaMemoryTypeDevice && ay.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    set_error("hm_matmat_noalloc needs device pointers for X and Y");
    return HM_EINVAL;
  }
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != A->device && cudaSetDevice(A->device) != cudaSuccess) {
    set_error("cudaSetDevice failed");
    return HM_ECUDA;
  }
  unsigned char* base = nullptr;
  hm_status st = noalloc_base(A->device, &base);
  if (st == HM_OK) {
    const MatView mv = A->view();
    const size_t cs = (A->storage == HM_F64) ? 8 : 4;
    const size_t nodes = static_cast<size_t>(2 * A->L - 1);
    const size_t data = ((scratch_elems(mv, r) * cs + 255) / 256) * 256;
    Scratch ws;
    std::memset(&ws, 0, sizeof(ws));
    if (A->kind == HM_HODLR) {
      ws.PS = base;
    } else {
      ws.xh = base;
      ws.yc = base + nodes * r * A->Kp * cs;
      ws.yf = base + nodes * r * (A->Kp + A->Ke) * cs;
    }
    ws.cnt = reinterpret_cast<int*>(base + data);
    ws.err = A->err;
    ws.prof = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The arrival counters must start at zero; the array keeps whatever the
    // previous call left, so clear them on the caller's stream.
    const cudaError_t e = cudaMemsetAsync(ws.cnt, 0, counter_count(mv, r) * sizeof(int), s);
    if (e != cudaSuccess) {
      set_error("clearing the static scratch counters failed: %s", cudaGetErrorString(e));
      st = HM_ECUDA;
    } else {
      st = launch_product(A, mv, ws, r, X, ldx, xt, Y, ldy, yt, s);
    }
  }
  if (dev_prev != A->device && dev_prev >= 0) cudaSetDevice(dev_prev);
  return st;
}

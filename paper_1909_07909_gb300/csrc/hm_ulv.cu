// HSS solve X = A^{-1} B by the implicit ULV factorization of Sec. 4.3
// (Steps 1-4; the fast ULV solvers it builds on), FP64, on the GPU.
//
// Level by level from the leaves (level p) to the root, every node q of the
// current level is a diagonal block D_q (n x n) with row basis U_q (n x ku)
// and column basis V_q (n x kv) of the current HSS matrix:
//   Step 1  QL of the row basis: Q_q^T U_q = [0; Ut_q], Ut_q ku x ku; then an
//           LQ of the top n - ku rows of Q_q^T D_q: Q_q^T D_q Z_q =
//           [[L11, 0], [D21, D22]], L11 lower triangular, D22 ku x ku;
//           V_q^T Z_q = [V1^T, V2^T].
//   Step 2  with the unknown X_q = Z_q [y1; w]: the top rows give
//           y1 = L11^{-1} (Q_q^T B_q)_top (no coupling reaches them: the row
//           basis is zero there); the bottom rows keep D22 w plus the
//           couplings, with the right-hand side b = (Q_q^T B_q)_bot - D21 y1
//           and the known compressed column part c_q = V1^T y1 (+ what the
//           children carried up) moved to the right-hand side.
//   Step 3  siblings a, b merge into their parent's leaf of the next level:
//             D = [[D22_a, Ut_a B12 V2_b^T], [Ut_b B21 V2_a^T, D22_b]],
//             U = [Ut_a R_U,top; Ut_b R_U,bot], V = [V2_a R_V,top; V2_b R_V,bot],
//             b = [b_a - Ut_a B12 c_b; b_b - Ut_b B21 c_a],
//             carry = R_V^T [c_a; c_b];
//           the root's merged block is solved by a full LQ (ku = 0).
//   Step 4  top-down, every node recovers X_q = Z_q [y1; w_q] with w_q its
//           slice of the parent's solution.
// The factorization keeps, per node, Q^T and Z explicitly, L11^{-1}, D21, V1^T
// and the merge products Ut B12, Ut B21, so that a solve is a sequence of
// batched FP64 GEMMs.  Leaves are padded to a common size with identity rows
// (their unknowns decouple and are dropped).
//
// Factorization kernels: one block of 256 threads per node; Householder
// reflectors are applied as rank-one updates, a warp per column for
// reflectors from the left (QL, column-major data, coalesced) and a thread per
// row for reflectors from the right (LQ).  FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hm_api_internal.h"
#include "k_simt.cuh"

namespace hmi {

constexpr uint32_t kMagicUlv = 0x31555248u;   // "HRU1"

}  // namespace hmi

// Per level l (0 = root .. p = leaves): nodes N = 2^l of size n, every array
// batch-strided by node.  All column-major, float64.
struct hm_ulv_level {
  int n = 0;        // node size (rows of D_q)
  int k = 0;        // rows kept for the next level (ku; 0 at the root)
  int N = 0;        // nodes
  double* Qt = nullptr;    // n x n        Q^T (identity at the root)
  double* Z = nullptr;     // n x n
  double* Linv = nullptr;  // (n-k) x (n-k) inverse of L11
  double* D21 = nullptr;   // k x (n-k)
  double* V1t = nullptr;   // kv x (n-k)   V1^T
  double* UB = nullptr;    // k x kv       Ut B12 (left child) or Ut B21 (right child) of this node
  double* Dm = nullptr;    // n x n        work: D_q, then Q^T D Z
  double* Um = nullptr;    // n x ku       work: U_q, then Q^T U
  double* Vm = nullptr;    // n x kv       work: V_q, then Z^T V
};

struct hm_ulv {
  uint32_t magic = 0;
  int device = 0;
  int64_t n = 0;
  int p = 0, L = 1;
  int ku = 0, kv = 0;
  int nleaf = 0;                       // padded leaf size of the factorization
  std::vector<int64_t> ends;
  int64_t* d_off = nullptr;
  std::vector<hm_ulv_level> lv;        // index = level
  const void* RU = nullptr;            // the matrix's translation operators (kept alive by the caller)
  const void* RV = nullptr;
  // solve work space (grown on demand)
  int64_t r_cap = 0;
  std::vector<double*> rhs, y1, bb, cv;   // per level
  double* cbuf = nullptr;
  std::vector<void*> owned;
};

namespace hmi {

namespace {

constexpr int UT = 256;   // threads of the factorization kernels

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Level-p node blocks from the packed storage: D (padded with identity rows
// and columns up to nl), U (n x ku), V (n x kv), all column-major.
__global__ void k_ulv_load_leaves(MatView mv, int nl, double* D, double* U, double* V) {
  const int leaf = blockIdx.x;
  const int64_t a0 = mv.off[leaf];
  const int m = static_cast<int>(mv.off[leaf + 1] - a0);
  double* Dq = D + static_cast<int64_t>(leaf) * nl * nl;
  double* Uq = U + static_cast<int64_t>(leaf) * nl * mv.Ke;
  double* Vq = V + static_cast<int64_t>(leaf) * nl * mv.Kp;
  const double* Ae = static_cast<const double*>(mv.A);
  const double* Wp = static_cast<const double*>(mv.W);
  for (int idx = threadIdx.x; idx < nl * nl; idx += blockDim.x) {
    const int i = idx % nl, j = idx / nl;
    double v;
    if (i < m && j < m) v = Ae[(a0 + i) * mv.We + j];
    else v = (i == j) ? 1.0 : 0.0;
    Dq[idx] = v;
  }
  for (int idx = threadIdx.x; idx < nl * mv.Ke; idx += blockDim.x) {
    const int i = idx % nl, j = idx / nl;
    Uq[idx] = (i < m) ? Ae[(a0 + i) * mv.We + mv.m_pad + j] : 0.0;
  }
  for (int idx = threadIdx.x; idx < nl * mv.Kp; idx += blockDim.x) {
    const int i = idx % nl, j = idx / nl;
    Vq[idx] = (i < m) ? Wp[(static_cast<int64_t>(leaf) * mv.Kp + j) * mv.m_pad + i] : 0.0;
  }
}

// Householder reflector H = I - tau v v^T with H x = alpha e_pivot for the
// vector x held in smem (length len, pivot index piv): on return x holds v
// (v_piv = x_piv - alpha) and the function returns tau (0 when x = 0).
__device__ double house(double* x, int len, int piv, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) s += x[i] * x[i];
  const double nrm2 = block_sum(s, red);
  __syncthreads();
  if (nrm2 == 0.0) return 0.0;
  const double xp = x[piv];
  const double alpha = (xp >= 0.0) ? -sqrt(nrm2) : sqrt(nrm2);
  const double vp = xp - alpha;
  const double vv = nrm2 - xp * xp + vp * vp;   // |v|^2
  __syncthreads();
  if (threadIdx.x == 0) x[piv] = vp;
  __syncthreads();
  return vv > 0.0 ? 2.0 / vv : 0.0;
}

// M(:, c) -= tau v (v^T M(0:len, c)) for columns c < ncol of a column-major
// matrix with leading dimension ld (reflector from the left on rows 0..len-1);
// a warp per column.
__device__ void refl_left(double* M, int ld, int ncol, const double* v, int len, double tau) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = w; c < ncol; c += nw) {
    double* col = M + static_cast<int64_t>(c) * ld;
    double s = 0.0;
    for (int i = l; i < len; i += 32) s += v[i] * col[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double f = tau * s;
    for (int i = l; i < len; i += 32) col[i] -= f * v[i];
  }
}

// M(i, c0:c0+len) -= tau (M(i, c0:c0+len) v) v^T for rows r0 <= i < r1 of a
// column-major matrix (reflector from the right); a thread per row.
__device__ void refl_right(double* M, int ld, int r0, int r1, int c0, const double* v, int len, double tau) {
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < len; ++j) s += M[static_cast<int64_t>(c0 + j) * ld + i] * v[j];
    const double f = tau * s;
    for (int j = 0; j < len; ++j) M[static_cast<int64_t>(c0 + j) * ld + i] -= f * v[j];
  }
}

// Steps 1-2 of one level: per node (block), QL of U, Q^T applied to D and to
// the identity (Qt), LQ of the top n-k rows of Q^T D accumulated into Z and
// applied to V from the left (Z^T V), then L11^{-1}, D21 and V1^T.
__global__ void __launch_bounds__(UT) k_ulv_factor(hm_ulv_level lv, int ku, int kv) {
  extern __shared__ __align__(16) double usm[];
  const int n = lv.n, k = lv.k;
  const int64_t q = blockIdx.x;
  double* D = lv.Dm + q * n * n;
  double* U = lv.Um + q * n * ku;
  double* V = lv.Vm + q * n * kv;
  double* Qt = lv.Qt + q * n * n;
  double* Z = lv.Z + q * n * n;
  double* x = usm;            // n: the current reflector
  double* red = usm + n;      // 32: block reductions
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const double e = (idx % n == idx / n) ? 1.0 : 0.0;
    Qt[idx] = e;
    Z[idx] = e;
  }
  __syncthreads();
  // QL of U (k columns, last first): H zeroes U(0:piv-1, j) into U(piv, j)
  for (int j = k - 1; j >= 0; --j) {
    const int piv = n - k + j;
    for (int i = threadIdx.x; i <= piv; i += blockDim.x) x[i] = U[static_cast<int64_t>(j) * n + i];
    __syncthreads();
    const double tau = house(x, piv + 1, piv, red);
    __syncthreads();
    if (tau != 0.0) {
      refl_left(U, n, j + 1, x, piv + 1, tau);
      refl_left(D, n, n, x, piv + 1, tau);
      refl_left(Qt, n, n, x, piv + 1, tau);
    }
    __syncthreads();
  }
  // LQ of rows 0..n-k-1 of Q^T D: H on columns j..n-1 maps row j onto e_j
  for (int j = 0; j < n - k; ++j) {
    const int len = n - j;
    for (int c = threadIdx.x; c < len; c += blockDim.x) x[c] = D[static_cast<int64_t>(j + c) * n + j];
    __syncthreads();
    const double tau = house(x, len, 0, red);
    __syncthreads();
    if (tau != 0.0) {
      refl_right(D, n, j, n, j, x, len, tau);
      refl_right(Z, n, 0, n, j, x, len, tau);
      // Z^T V: the same reflector from the left on rows j..n-1 of V
      refl_left(V + j, n, kv, x, len, tau);
    }
    __syncthreads();
  }
  // L11^{-1} (lower triangular), a thread per column: forward substitution
  const int m = n - k;
  double* Li = lv.Linv + q * m * m;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    for (int i = 0; i < c; ++i) Li[static_cast<int64_t>(c) * m + i] = 0.0;
    for (int i = c; i < m; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l2 = c; l2 < i; ++l2) s -= D[static_cast<int64_t>(l2) * n + i] * Li[static_cast<int64_t>(c) * m + l2];
      Li[static_cast<int64_t>(c) * m + i] = s / D[static_cast<int64_t>(i) * n + i];
    }
  }
  // D21 (k x m) and V1^T (kv x m)
  for (int idx = threadIdx.x; idx < k * m; idx += blockDim.x) {
    const int i = idx % k, c = idx / k;
    lv.D21[q * k * m + idx] = D[static_cast<int64_t>(c) * n + m + i];
  }
  for (int idx = threadIdx.x; idx < kv * m; idx += blockDim.x) {
    const int i = idx % kv, c = idx / kv;
    lv.V1t[q * kv * m + idx] = V[static_cast<int64_t>(i) * n + c];
  }
}

// Step 3 of the factorization: the parent's block from its children
// (next level l-1).  Child a = 2t, b = 2t+1 of level l; kept rows k = ku.
//   D = [[D22_a, Ut_a B12 V2_b^T], [Ut_b B21 V2_a^T, D22_b]]
//   U = [Ut_a R_U,top; Ut_b R_U,bot] (not at the root), V likewise with R_V.
// Also stores UB = Ut B12 (child a) and Ut B21 (child b) for the solves.
__global__ void k_ulv_merge(hm_ulv_level ch, hm_ulv_level par, MatView mv, int level_parent) {
  const int t = blockIdx.x;
  const int k = ch.k, n = ch.n, ku = mv.Ke, kv = mv.Kp;
  const int q = (1 << level_parent) - 1 + t;   // parent node id
  const double* B12 = static_cast<const double*>(mv.B12) + static_cast<int64_t>(q) * kv * ku;   // [j][i] = B12(i, j)
  const double* B21 = static_cast<const double*>(mv.B21) + static_cast<int64_t>(q) * kv * ku;
  const double* Dc[2] = {ch.Dm + static_cast<int64_t>(2 * t) * n * n, ch.Dm + static_cast<int64_t>(2 * t + 1) * n * n};
  const double* Uc[2] = {ch.Um + static_cast<int64_t>(2 * t) * n * ku, ch.Um + static_cast<int64_t>(2 * t + 1) * n * ku};
  const double* Vc[2] = {ch.Vm + static_cast<int64_t>(2 * t) * n * kv, ch.Vm + static_cast<int64_t>(2 * t + 1) * n * kv};
  const int m = n - k;
  // UB for both children: Ut_a B12 (ku x kv), Ut_b B21
  for (int h = 0; h < 2; ++h) {
    const double* Bq = h == 0 ? B12 : B21;
    double* UB = ch.UB + static_cast<int64_t>(2 * t + h) * k * kv;
    for (int idx = threadIdx.x; idx < k * kv; idx += blockDim.x) {
      const int i = idx % k, j = idx / k;
      double s = 0.0;
      for (int l = 0; l < ku; ++l) s += Uc[h][static_cast<int64_t>(l) * n + m + i] * Bq[j * ku + l];
      UB[idx] = s;
    }
  }
  __syncthreads();
  const int np = par.n;   // = 2k
  double* Dp = par.Dm + static_cast<int64_t>(t) * np * np;
  for (int idx = threadIdx.x; idx < np * np; idx += blockDim.x) {
    const int i = idx % np, j = idx / np;
    const int hi = i / k, hj = j / k, ii = i % k, jj = j % k;
    double v;
    if (hi == hj) {
      v = Dc[hi][static_cast<int64_t>(m + jj) * n + m + ii];
    } else {
      // block (hi, hj): Ut_hi B V2_hj^T = UB_hi (k x kv) times V2_hj^T (kv x k)
      const double* UB = ch.UB + static_cast<int64_t>(2 * t + hi) * k * kv;
      v = 0.0;
      for (int l = 0; l < kv; ++l) v += UB[static_cast<int64_t>(l) * k + ii] * Vc[hj][static_cast<int64_t>(l) * n + m + jj];
    }
    Dp[idx] = v;
  }
  if (level_parent > 0) {
    const double* RU = static_cast<const double*>(mv.RU) + static_cast<int64_t>(q) * 2 * ku * ku;   // [h][j][i] = R_U(h ku + i, j)
    const double* RV = static_cast<const double*>(mv.RV) + static_cast<int64_t>(q) * 2 * kv * kv;   // [j][i] = R_V(j, i)
    double* Up = par.Um + static_cast<int64_t>(t) * np * ku;
    double* Vp = par.Vm + static_cast<int64_t>(t) * np * kv;
    for (int idx = threadIdx.x; idx < np * ku; idx += blockDim.x) {
      const int i = idx % np, j = idx / np;
      const int h = i / k, ii = i % k;
      double s = 0.0;
      for (int l = 0; l < ku; ++l)
        s += Uc[h][static_cast<int64_t>(l) * n + m + ii] * RU[(static_cast<int64_t>(h) * ku + j) * ku + l];
      Up[idx] = s;
    }
    for (int idx = threadIdx.x; idx < np * kv; idx += blockDim.x) {
      const int i = idx % np, j = idx / np;
      const int h = i / k, ii = i % k;
      double s = 0.0;
      for (int l = 0; l < kv; ++l)
        s += Vc[h][static_cast<int64_t>(l) * n + m + ii] * RV[static_cast<int64_t>(h * kv + l) * kv + j];
      Vp[idx] = s;
    }
  }
}

// Batched C_b = alpha * A_b B_b + beta * C_b, column-major, FP64; A_b = A +
// b * sA etc.  Tiles of 32 x 32 outputs per block (16 x 16 threads, 2 x 2
// each) over K chunks of 32 staged in shared memory.
__global__ void __launch_bounds__(256) k_bgemm_f64(int M, int Nc, int K, double alpha, const double* A, int64_t lda,
                                                   int64_t sA, const double* B, int64_t ldb, int64_t sB, double beta,
                                                   double* C, int64_t ldc, int64_t sC, int tiles_m) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int b = blockIdx.y;
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  const double* Ab = A + b * sA;
  const double* Bb = B + b * sB;
  double* Cb = C + b * sC;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = tm * 32, c0 = tn * 32;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int idx = threadIdx.x; idx < 1024; idx += 256) {
      const int i = idx % 32, kk = idx / 32;
      As[kk][i] = (r0 + i < M && k0 + kk < K) ? Ab[static_cast<int64_t>(k0 + kk) * lda + r0 + i] : 0.0;
      Bs[i][kk] = (c0 + kk < Nc && k0 + i < K) ? Bb[static_cast<int64_t>(c0 + kk) * ldb + k0 + i] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < M && c < Nc) {
        double* p = Cb + static_cast<int64_t>(c) * ldc + r;
        *p = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *p;
      }
    }
}

cudaError_t bgemm(int M, int Nc, int K, double alpha, const double* A, int64_t lda, int64_t sA, const double* B,
                  int64_t ldb, int64_t sB, double beta, double* C, int64_t ldc, int64_t sC, int batch,
                  cudaStream_t s) {
  if (M <= 0 || Nc <= 0 || batch <= 0) return cudaSuccess;
  const int tm = (M + 31) / 32, tn = (Nc + 31) / 32;
  k_bgemm_f64<<<dim3(tm * tn, batch), 256, 0, s>>>(M, Nc, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, tm);
  return cudaGetLastError();
}

// rhs of the level-p nodes from B (rows beyond a leaf's size are zero).
__global__ void k_ulv_gather_b(const int64_t* off, int nl, int64_t r, const double* B, int64_t ldb, double* R) {
  const int leaf = blockIdx.x;
  const int64_t a0 = off[leaf];
  const int m = static_cast<int>(off[leaf + 1] - a0);
  double* Rq = R + static_cast<int64_t>(leaf) * nl * r;
  for (int64_t idx = threadIdx.x; idx < static_cast<int64_t>(nl) * r; idx += blockDim.x) {
    const int i = static_cast<int>(idx % nl);
    const int64_t c = idx / nl;
    Rq[idx] = (i < m) ? B[a0 + i + c * ldb] : 0.0;
  }
}

__global__ void k_ulv_scatter_x(const int64_t* off, int nl, int64_t r, const double* W, double* X, int64_t ldx) {
  const int leaf = blockIdx.x;
  const int64_t a0 = off[leaf];
  const int m = static_cast<int>(off[leaf + 1] - a0);
  const double* Wq = W + static_cast<int64_t>(leaf) * nl * r;
  for (int64_t idx = threadIdx.x; idx < static_cast<int64_t>(m) * r; idx += blockDim.x) {
    const int i = static_cast<int>(idx % m);
    const int64_t c = idx / m;
    X[a0 + i + c * ldx] = Wq[i + c * nl];
  }
}

// Merge of the right-hand sides (Step 3 of the solve) for the parents of
// level l: rhs_p = [bb_a - UB_a c_b; bb_b - UB_b c_a] and, above the root's
// children, carry_p = R_V^T [c_a; c_b] (added to the parent's c later).
__global__ void k_ulv_merge_rhs(const double* bb, const double* cv, const double* UB, int k, int kv, int64_t r,
                                double* rhs_p, double* carry_p, const double* RV, int level_parent) {
  const int t = blockIdx.x;
  const int q = (1 << level_parent) - 1 + t;
  const int np = 2 * k;
  for (int64_t idx = threadIdx.x; idx < static_cast<int64_t>(np) * r; idx += blockDim.x) {
    const int i = static_cast<int>(idx % np);
    const int64_t c = idx / np;
    const int h = i / k, ii = i % k;
    const int64_t me = 2 * t + h, other = 2 * t + (1 - h);
    double s = bb[me * k * r + c * k + ii];
    const double* ub = UB + me * k * kv;
    const double* co = cv + other * kv * r + c * kv;
    for (int l = 0; l < kv; ++l) s -= ub[static_cast<int64_t>(l) * k + ii] * co[l];
    rhs_p[static_cast<int64_t>(t) * np * r + c * np + i] = s;
  }
  if (level_parent > 0) {
    const double* R = RV + static_cast<int64_t>(q) * 2 * kv * kv;   // [j][i] = R_V(j, i)
    for (int64_t idx = threadIdx.x; idx < static_cast<int64_t>(kv) * r; idx += blockDim.x) {
      const int i = static_cast<int>(idx % kv);
      const int64_t c = idx / kv;
      double s = 0.0;
      for (int h = 0; h < 2; ++h) {
        const double* co = cv + (2 * t + h) * kv * r + c * kv;
        for (int l = 0; l < kv; ++l) s += R[static_cast<int64_t>(h * kv + l) * kv + i] * co[l];
      }
      carry_p[static_cast<int64_t>(t) * kv * r + c * kv + i] = s;
    }
  }
}

// [y1; w] of every node of level l from its y1 and its slice of the parent's
// solution (level l-1, node size 2k): out = rows of the node before Z.
__global__ void k_ulv_stack(const double* y1, int m, const double* wpar, int k, int npar, int64_t r, double* out,
                            int n) {
  const int q = blockIdx.x;
  const int t = q / 2, h = q % 2;
  for (int64_t idx = threadIdx.x; idx < static_cast<int64_t>(n) * r; idx += blockDim.x) {
    const int i = static_cast<int>(idx % n);
    const int64_t c = idx / n;
    double v;
    if (i < m) v = y1[static_cast<int64_t>(q) * m * r + c * m + i];
    else v = wpar[static_cast<int64_t>(t) * npar * r + c * npar + h * k + (i - m)];
    out[static_cast<int64_t>(q) * n * r + idx] = v;
  }
}

}  // namespace

}  // namespace hmi

using namespace hmi;

namespace {

hm_status ulv_fail(hm_ulv* F, hm_status s, const char* what, cudaError_t e) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (F) {
    for (void* p : F->owned) cudaFree(p);
    delete F;
  }
  return s;
}

}  // namespace

extern "C" hm_status hm_ulv_factor(const hm_matrix* A, hm_ulv** out) {
  if (!out) { set_error("out is NULL"); return HM_EINVAL; }
  *out = nullptr;
  if (!A || A->magic != kMagicMatrix) { set_error("not a matrix handle"); return HM_EINVAL; }
  if (A->kind != HM_HSS) { set_error("the ULV solve needs an HSS matrix"); return HM_EINVAL; }
  if (A->storage != HM_F64) { set_error("the ULV solve needs F64 storage"); return HM_EUNSUPPORTED; }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != A->device) { set_error("current device is not the matrix's"); return HM_EINVAL; }
  const MatView mv = A->view();
  const int ku = mv.Ke, kv = mv.Kp;
  if (ku != kv) { set_error("the ULV solve needs equal padded row and column ranks"); return HM_EUNSUPPORTED; }
  if (mv.p < 1) { set_error("the ULV solve needs at least one level"); return HM_EUNSUPPORTED; }
  const int nl = std::max(mv.m_pad, ((ku + 1 + 7) / 8) * 8);   // leaf block size: more rows than the rank
  if (2 * ku > 1024 || nl > 1024) { set_error("blocks above 1024 rows"); return HM_EUNSUPPORTED; }
  hm_ulv* F = new (std::nothrow) hm_ulv();
  if (!F) { set_error("host allocation failed"); return HM_ENOMEM; }
  F->magic = kMagicUlv;
  F->device = A->device;
  F->n = A->n;
  F->p = A->p;
  F->L = A->L;
  F->ku = ku;
  F->kv = kv;
  F->nleaf = nl;
  F->ends = A->ends;
  F->d_off = A->d_off;
  F->RU = A->d_RU;
  F->RV = A->d_RVt;
  F->lv.resize(A->p + 1);
  auto alloc = [&](double** p, size_t elems) -> cudaError_t {
    void* v = nullptr;
    const cudaError_t e = dev_malloc(&v, std::max<size_t>(elems, 1) * sizeof(double));
    if (e == cudaSuccess) {
      F->owned.push_back(v);
      *p = static_cast<double*>(v);
    }
    return e;
  };
  for (int l = 0; l <= A->p; ++l) {
    hm_ulv_level& L = F->lv[l];
    L.N = 1 << l;
    L.n = (l == A->p) ? nl : 2 * ku;
    L.k = (l == 0) ? 0 : ku;
    const size_t N = L.N, n = L.n, m = L.n - L.k;
    cudaError_t e = alloc(&L.Qt, N * n * n);
    if (e == cudaSuccess) e = alloc(&L.Z, N * n * n);
    if (e == cudaSuccess) e = alloc(&L.Linv, N * m * m);
    if (e == cudaSuccess) e = alloc(&L.D21, N * L.k * m);
    if (e == cudaSuccess) e = alloc(&L.V1t, N * kv * m);
    if (e == cudaSuccess) e = alloc(&L.UB, N * L.k * kv);
    if (e == cudaSuccess) e = alloc(&L.Dm, N * n * n);
    if (e == cudaSuccess) e = alloc(&L.Um, N * n * ku);
    if (e == cudaSuccess) e = alloc(&L.Vm, N * n * kv);
    if (e != cudaSuccess)
      return ulv_fail(F, e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, "ULV allocation", e);
  }
  cudaStream_t s = nullptr;
  k_ulv_load_leaves<<<A->L, 256, 0, s>>>(mv, nl, F->lv[A->p].Dm, F->lv[A->p].Um, F->lv[A->p].Vm);
  cudaError_t e = cudaGetLastError();
  for (int l = A->p; l >= 0 && e == cudaSuccess; --l) {
    hm_ulv_level& L = F->lv[l];
    const size_t smem = (static_cast<size_t>(L.n) + 32) * sizeof(double);
    k_ulv_factor<<<L.N, UT, smem, s>>>(L, ku, kv);
    e = cudaGetLastError();
    if (e == cudaSuccess && l > 0) {
      k_ulv_merge<<<L.N / 2, 256, 0, s>>>(L, F->lv[l - 1], mv, l - 1);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ulv_fail(F, HM_ECUDA, "ULV factorization", e);
  *out = F;
  return HM_OK;
}

namespace hmi {

static hm_status ulv_reserve(hm_ulv* F, int64_t r) {
  if (r <= F->r_cap) return HM_OK;
  for (auto* p : F->rhs) cudaFree(p);
  for (auto* p : F->y1) cudaFree(p);
  for (auto* p : F->bb) cudaFree(p);
  for (auto* p : F->cv) cudaFree(p);
  if (F->cbuf) cudaFree(F->cbuf);
  F->rhs.assign(F->p + 1, nullptr);
  F->y1.assign(F->p + 1, nullptr);
  F->bb.assign(F->p + 1, nullptr);
  F->cv.assign(F->p + 1, nullptr);
  F->cbuf = nullptr;
  F->r_cap = 0;
  auto al = [&](double** p, size_t elems) -> bool {
    void* v = nullptr;
    if (dev_malloc(&v, std::max<size_t>(elems, 1) * sizeof(double)) != cudaSuccess) return false;
    *p = static_cast<double*>(v);
    return true;
  };
  bool ok = true;
  for (int l = 0; l <= F->p && ok; ++l) {
    const hm_ulv_level& L = F->lv[l];
    const size_t N = L.N, n = L.n, m = L.n - L.k;
    ok = al(&F->rhs[l], N * n * r) && al(&F->y1[l], N * n * r) && al(&F->bb[l], N * std::max(L.k, 1) * r) &&
         al(&F->cv[l], N * F->kv * r);
  }
  if (ok) ok = al(&F->cbuf, static_cast<size_t>(F->L) * F->nleaf * r);
  if (!ok) {
    set_error("ULV solve work space allocation failed");
    return HM_ENOMEM;
  }
  F->r_cap = r;
  return HM_OK;
}

}  // namespace hmi

extern "C" hm_status hm_ulv_solve(const hm_ulv* Fc, int64_t r, const void* B, int64_t ldb, void* X, int64_t ldx,
                                  void* stream) {
  if (!Fc || Fc->magic != kMagicUlv) { set_error("not a ULV factorization handle"); return HM_EINVAL; }
  hm_ulv* F = const_cast<hm_ulv*>(Fc);
  if (r < 0 || ldb < std::max<int64_t>(F->n, 1) || ldx < std::max<int64_t>(F->n, 1)) {
    set_error("r < 0 or ldb/ldx < n");
    return HM_EINVAL;
  }
  if (r == 0 || F->n == 0) return HM_OK;
  if (!B || !X) { set_error("B or X is NULL"); return HM_EINVAL; }
  cudaPointerAttributes ab, ax;
  if (cudaPointerGetAttributes(&ab, B) != cudaSuccess || cudaPointerGetAttributes(&ax, X) != cudaSuccess ||
      (ab.type != cudaMemoryTypeDevice && ab.type != cudaMemoryTypeManaged) ||
      (ax.type != cudaMemoryTypeDevice && ax.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    set_error("hm_ulv_solve needs device pointers for B and X");
    return HM_EINVAL;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != F->device) { set_error("current device is not the factorization's"); return HM_EINVAL; }
  hm_status st = ulv_reserve(F, r);
  if (st != HM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int p = F->p, kv = F->kv;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  // level p right-hand sides
  k_ulv_gather_b<<<F->L, 256, 0, s>>>(F->d_off, F->nleaf, r, static_cast<const double*>(B), ldb, F->rhs[p]);
  chk(cudaGetLastError());
  // upward: Steps 1-3 on the right-hand sides
  for (int l = p; l >= 1; --l) {
    const hm_ulv_level& L = F->lv[l];
    const int n = L.n, k = L.k, m = n - k;
    double* b = F->y1[l];   // Q^T rhs (n x r per node); its top m rows become y1 below
    chk(bgemm(n, static_cast<int>(r), n, 1.0, L.Qt, n, static_cast<int64_t>(n) * n, F->rhs[l], n,
              static_cast<int64_t>(n) * r, 0.0, b, n, static_cast<int64_t>(n) * r, L.N, s));
    // y1 = L11^{-1} b_top (m x r), written to the first m rows of rhs[l] (no longer needed)
    chk(bgemm(m, static_cast<int>(r), m, 1.0, L.Linv, m, static_cast<int64_t>(m) * m, b, n,
              static_cast<int64_t>(n) * r, 0.0, F->rhs[l], m, static_cast<int64_t>(m) * r, L.N, s));
    // bb = b_bot - D21 y1 (k x r): copy b_bot, then subtract
    chk(cudaMemcpy2DAsync(F->bb[l], sizeof(double) * k, b + m, sizeof(double) * n, sizeof(double) * k,
                          static_cast<size_t>(L.N) * r, cudaMemcpyDeviceToDevice, s));
    chk(bgemm(k, static_cast<int>(r), m, -1.0, L.D21, k, static_cast<int64_t>(k) * m, F->rhs[l], m,
              static_cast<int64_t>(m) * r, 1.0, F->bb[l], k, static_cast<int64_t>(k) * r, L.N, s));
    // c = V1^T y1 (+ the carried part, already in cv[l] for l < p)
    chk(bgemm(kv, static_cast<int>(r), m, 1.0, L.V1t, kv, static_cast<int64_t>(kv) * m, F->rhs[l], m,
              static_cast<int64_t>(m) * r, l < p ? 1.0 : 0.0, F->cv[l], kv, static_cast<int64_t>(kv) * r, L.N, s));
    // merge into the parents' right-hand sides (and carries)
    k_ulv_merge_rhs<<<L.N / 2, 256, 0, s>>>(F->bb[l], F->cv[l], L.UB, k, kv, r, F->rhs[l - 1], F->cv[l - 1],
                                            static_cast<const double*>(F->RV), l - 1);
    chk(cudaGetLastError());
  }
  // root: w = Z L^{-1} (Q^T rhs) with Q = I
  {
    const hm_ulv_level& L = F->lv[0];
    const int n = L.n;
    chk(bgemm(n, static_cast<int>(r), n, 1.0, L.Linv, n, 0, F->rhs[0], n, 0, 0.0, F->y1[0], n, 0, 1, s));
    chk(bgemm(n, static_cast<int>(r), n, 1.0, L.Z, n, 0, F->y1[0], n, 0, 0.0, F->rhs[0], n, 0, 1, s));
  }
  // downward: X_q = Z_q [y1; w_q] (Step 4); rhs[l] holds y1 in its first m rows per node
  for (int l = 1; l <= p; ++l) {
    const hm_ulv_level& L = F->lv[l];
    const hm_ulv_level& P = F->lv[l - 1];
    const int n = L.n, k = L.k, m = n - k;
    // stack [y1; w] into y1[l] (n x r per node), then multiply by Z (into cbuf at the leaves)
    k_ulv_stack<<<L.N, 256, 0, s>>>(F->rhs[l], m, F->rhs[l - 1], k, P.n, r, F->y1[l], n);
    chk(cudaGetLastError());
    double* dst = (l == p) ? F->cbuf : F->rhs[l];
    chk(bgemm(n, static_cast<int>(r), n, 1.0, L.Z, n, static_cast<int64_t>(n) * n, F->y1[l], n,
              static_cast<int64_t>(n) * r, 0.0, dst, n, static_cast<int64_t>(n) * r, L.N, s));
  }
  k_ulv_scatter_x<<<F->L, 256, 0, s>>>(F->d_off, F->nleaf, r, F->cbuf, static_cast<double*>(X), ldx);
  chk(cudaGetLastError());
  if (e != cudaSuccess) {
    set_error("ULV solve launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

namespace hmi {

void destroy_ulv(void* any) {
  hm_ulv* F = static_cast<hm_ulv*>(any);
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != F->device) cudaSetDevice(F->device);
  cudaDeviceSynchronize();
  for (void* p : F->owned) cudaFree(p);
  for (auto* p : F->rhs) cudaFree(p);
  for (auto* p : F->y1) cudaFree(p);
  for (auto* p : F->bb) cudaFree(p);
  for (auto* p : F->cv) cudaFree(p);
  if (F->cbuf) cudaFree(F->cbuf);
  if (dev_prev != F->device) cudaSetDevice(dev_prev);
  F->magic = 0;
  delete F;
}

bool is_ulv(const void* any) { return *static_cast<const uint32_t*>(any) == kMagicUlv; }

}  // namespace hmi

// CPU fast product Y = A X of a HODLR or HSS matrix in float64, on all host
// cores (OpenMP): the algorithms of Sec. 4.1 and Fig. 4.1, O(k n log n)
// (HODLR) and O(k n) (HSS) flops per right-hand side (Table 4.1).
//
// This is the timed CPU baseline of the GPU library, not its oracle: it runs
// the paper's fast tree algorithm with cache-blocked loops, where the oracle
// expands the defining matrix.  It shares no code with the GPU library and
// links nothing but the C++ runtime and OpenMP.
//
// Layout: every block is column-major float64 (Matlab layout), copied at
// create time into one contiguous buffer, with the column factors stored
// transposed so that every product below is C = A B with A column-major.
//   HODLR (Def. 2.2): D_i per leaf; per internal node q the factors U12, U21
//     and the transposed V12^T, V21^T.
//   HSS (Def. 2.3, Eq. 2.2): D_i, U_i and V_i^T per leaf; R_U = [Rl; Rr] and
//     R_V^T per internal non-root node; B12, B21 per internal node.
// X and Y are n x r column-major with leading dimensions ldx, ldy.
#include <omp.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

namespace {

// C(m x r) (+)= A(m x k) B(k x r); A, B, C column-major.  Both operands are
// first packed into contiguous micro-panels (A: MR rows by k, B: k by NR
// columns, zero-padded), then every MR x NR register tile of C accumulates
// over k from the two panels: all loads in the inner loop are contiguous, an
// A panel stays in L1 while it meets every B panel, and the packed B (k x r)
// stays in L2.
constexpr int MR = 8;
constexpr int NR = 4;
typedef double v2d __attribute__((vector_size(16)));

void gemm(int m, int r, int k, const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
          int64_t ldc, bool accumulate) {
  if (m <= 0 || r <= 0) return;
  if (k <= 0) {
    if (!accumulate)
      for (int j = 0; j < r; ++j) std::memset(C + j * ldc, 0, sizeof(double) * m);
    return;
  }
  thread_local std::vector<double> apack, bpack;
  const int mb = (m + MR - 1) / MR, nb = (r + NR - 1) / NR;
  if (apack.size() < static_cast<size_t>(mb) * k * MR) apack.resize(static_cast<size_t>(mb) * k * MR);
  if (bpack.size() < static_cast<size_t>(nb) * k * NR) bpack.resize(static_cast<size_t>(nb) * k * NR);
  double* Ap = apack.data();
  double* Bp = bpack.data();
  for (int jb = 0; jb < nb; ++jb)
    for (int kk = 0; kk < k; ++kk)
      for (int jj = 0; jj < NR; ++jj) {
        const int j = jb * NR + jj;
        Bp[(static_cast<size_t>(jb) * k + kk) * NR + jj] = j < r ? B[j * ldb + kk] : 0.0;
      }
  for (int ib = 0; ib < mb; ++ib) {
    const int i0 = ib * MR, mr = std::min(MR, m - i0);
    double* ap = Ap + static_cast<size_t>(ib) * k * MR;
    for (int kk = 0; kk < k; ++kk) {
      const double* a = A + kk * lda + i0;
      for (int ii = 0; ii < MR; ++ii) ap[kk * MR + ii] = ii < mr ? a[ii] : 0.0;
    }
  }
  for (int ib = 0; ib < mb; ++ib) {
    const int i0 = ib * MR, mr = std::min(MR, m - i0);
    const double* ap = Ap + static_cast<size_t>(ib) * k * MR;
    for (int jb = 0; jb < nb; ++jb) {
      const int j0 = jb * NR, nr = std::min(NR, r - j0);
      const double* bp = Bp + static_cast<size_t>(jb) * k * NR;
      // MR x NR accumulators as pairs of doubles (GCC generic vectors: one
      // 128-bit register each on both x86-64 and AArch64)
      v2d acc[NR][MR / 2];
      for (int jj = 0; jj < NR; ++jj)
        for (int ii = 0; ii < MR / 2; ++ii) acc[jj][ii] = v2d{0.0, 0.0};
      for (int kk = 0; kk < k; ++kk) {
        v2d a[MR / 2];
        std::memcpy(a, ap + kk * MR, sizeof(a));
        const double* b = bp + kk * NR;
        for (int jj = 0; jj < NR; ++jj) {
          const v2d bb = {b[jj], b[jj]};
          for (int ii = 0; ii < MR / 2; ++ii) acc[jj][ii] += a[ii] * bb;
        }
      }
      for (int jj = 0; jj < nr; ++jj) {
        double* c = C + (j0 + jj) * ldc + i0;
        double t[MR];
        std::memcpy(t, acc[jj], sizeof(t));
        if (accumulate)
          for (int ii = 0; ii < mr; ++ii) c[ii] += t[ii];
        else
          for (int ii = 0; ii < mr; ++ii) c[ii] = t[ii];
      }
    }
  }
}

// A column-major m x n block copied transposed (n x m, column-major).
void put_t(double* dst, const double* src, int m, int n) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) dst[static_cast<int64_t>(i) * n + j] = src[static_cast<int64_t>(j) * m + i];
}

struct Block {
  int64_t off = 0;   // element offset in the buffer
  int rows = 0, cols = 0;
};

}  // namespace

struct hmc_matrix {
  int kind = 0;   // 0 HODLR, 1 HSS
  int64_t n = 0;
  int p = 0, L = 1;
  std::vector<int64_t> start;          // node id -> first row, end row
  std::vector<int64_t> end;
  std::vector<double> buf;
  std::vector<Block> D, U12, V12t, U21, V21t;         // HODLR
  std::vector<Block> U, Vt, RU, RVt, B12, B21;        // HSS
  std::vector<int> ku, kv;
  // per-product work space (resized for r)
  std::vector<double> ws;
};

namespace {

void node_ranges(hmc_matrix* M, const int64_t* ends) {
  const int N = 2 * M->L - 1;
  M->start.assign(N, 0);
  M->end.assign(N, 0);
  for (int i = 0; i < M->L; ++i) {
    M->start[M->L - 1 + i] = i == 0 ? 0 : ends[i - 1];
    M->end[M->L - 1 + i] = ends[i];
  }
  for (int q = M->L - 2; q >= 0; --q) {
    M->start[q] = M->start[2 * q + 1];
    M->end[q] = M->end[2 * q + 2];
  }
}

}  // namespace

extern "C" {

// Number of OpenMP threads a product uses.
int hmc_threads(void) { return omp_get_max_threads(); }

void hmc_destroy(hmc_matrix* M) { delete M; }

// HODLR generators as in the GPU library's hm_hodlr_gens: D[L], U12, V12,
// U21, V21 [L-1] (column-major float64), ranks k12, k21 [L-1].  Returns NULL
// on a bad argument or when memory runs out.
hmc_matrix* hmc_hodlr_create(int64_t n, int32_t L, const int64_t* ends, const double* const* D,
                             const double* const* U12, const double* const* V12, const double* const* U21,
                             const double* const* V21, const int32_t* k12, const int32_t* k21) {
  if (L < 1 || (L & (L - 1)) != 0 || !ends) return nullptr;
  hmc_matrix* M = new (std::nothrow) hmc_matrix();
  if (!M) return nullptr;
  try {
    M->kind = 0;
    M->n = n;
    M->L = L;
    while ((1 << M->p) < L) ++M->p;
    node_ranges(M, ends);
    int64_t total = 0;
    M->D.resize(L);
    for (int i = 0; i < L; ++i) {
      const int m = static_cast<int>(M->end[L - 1 + i] - M->start[L - 1 + i]);
      M->D[i] = {total, m, m};
      total += static_cast<int64_t>(m) * m;
    }
    M->U12.resize(L - 1); M->V12t.resize(L - 1); M->U21.resize(L - 1); M->V21t.resize(L - 1);
    for (int q = 0; q < L - 1; ++q) {
      const int ma = static_cast<int>(M->end[2 * q + 1] - M->start[2 * q + 1]);
      const int mb = static_cast<int>(M->end[2 * q + 2] - M->start[2 * q + 2]);
      M->U12[q] = {total, ma, k12[q]}; total += static_cast<int64_t>(ma) * k12[q];
      M->V12t[q] = {total, k12[q], mb}; total += static_cast<int64_t>(mb) * k12[q];
      M->U21[q] = {total, mb, k21[q]}; total += static_cast<int64_t>(mb) * k21[q];
      M->V21t[q] = {total, k21[q], ma}; total += static_cast<int64_t>(ma) * k21[q];
    }
    M->buf.assign(total, 0.0);
    double* b = M->buf.data();
    for (int i = 0; i < L; ++i)
      if (M->D[i].rows) std::memcpy(b + M->D[i].off, D[i], sizeof(double) * M->D[i].rows * M->D[i].cols);
    for (int q = 0; q < L - 1; ++q) {
      const Block& u12 = M->U12[q];
      const Block& u21 = M->U21[q];
      if (u12.rows * u12.cols) std::memcpy(b + u12.off, U12[q], sizeof(double) * u12.rows * u12.cols);
      if (u21.rows * u21.cols) std::memcpy(b + u21.off, U21[q], sizeof(double) * u21.rows * u21.cols);
      if (M->V12t[q].rows * M->V12t[q].cols) put_t(b + M->V12t[q].off, V12[q], M->V12t[q].cols, M->V12t[q].rows);
      if (M->V21t[q].rows * M->V21t[q].cols) put_t(b + M->V21t[q].off, V21[q], M->V21t[q].cols, M->V21t[q].rows);
    }
  } catch (...) {
    delete M;
    return nullptr;
  }
  return M;
}

// HSS generators as in hm_hss_gens: D, U, V [L]; RU, RV [2L-1] (internal
// non-root entries used); B12, B21 [L-1]; ranks ku, kv [2L-1].
hmc_matrix* hmc_hss_create(int64_t n, int32_t L, const int64_t* ends, const double* const* D,
                           const double* const* U, const double* const* V, const double* const* RU,
                           const double* const* RV, const double* const* B12, const double* const* B21,
                           const int32_t* ku, const int32_t* kv) {
  if (L < 1 || (L & (L - 1)) != 0 || !ends) return nullptr;
  hmc_matrix* M = new (std::nothrow) hmc_matrix();
  if (!M) return nullptr;
  try {
    M->kind = 1;
    M->n = n;
    M->L = L;
    while ((1 << M->p) < L) ++M->p;
    node_ranges(M, ends);
    const int N = 2 * L - 1;
    M->ku.assign(ku, ku + N);
    M->kv.assign(kv, kv + N);
    int64_t total = 0;
    M->D.resize(L); M->U.resize(L); M->Vt.resize(L);
    for (int i = 0; i < L; ++i) {
      const int q = L - 1 + i;
      const int m = static_cast<int>(M->end[q] - M->start[q]);
      M->D[i] = {total, m, m}; total += static_cast<int64_t>(m) * m;
      M->U[i] = {total, m, ku[q]}; total += static_cast<int64_t>(m) * ku[q];
      M->Vt[i] = {total, kv[q], m}; total += static_cast<int64_t>(m) * kv[q];
    }
    M->RU.resize(N); M->RVt.resize(N); M->B12.resize(L - 1); M->B21.resize(L - 1);
    for (int q = 0; q < L - 1; ++q) {
      const int a = 2 * q + 1, bb = 2 * q + 2;
      if (q > 0) {
        M->RU[q] = {total, ku[a] + ku[bb], ku[q]}; total += static_cast<int64_t>(ku[a] + ku[bb]) * ku[q];
        M->RVt[q] = {total, kv[q], kv[a] + kv[bb]}; total += static_cast<int64_t>(kv[a] + kv[bb]) * kv[q];
      }
      M->B12[q] = {total, ku[a], kv[bb]}; total += static_cast<int64_t>(ku[a]) * kv[bb];
      M->B21[q] = {total, ku[bb], kv[a]}; total += static_cast<int64_t>(ku[bb]) * kv[a];
    }
    M->buf.assign(total, 0.0);
    double* b = M->buf.data();
    auto cp = [&](const Block& blk, const double* src) {
      const int64_t cnt = static_cast<int64_t>(blk.rows) * blk.cols;
      if (cnt) std::memcpy(b + blk.off, src, sizeof(double) * cnt);
    };
    for (int i = 0; i < L; ++i) {
      cp(M->D[i], D[i]);
      cp(M->U[i], U[i]);
      if (M->Vt[i].rows * M->Vt[i].cols) put_t(b + M->Vt[i].off, V[i], M->Vt[i].cols, M->Vt[i].rows);
    }
    for (int q = 0; q < L - 1; ++q) {
      if (q > 0) {
        cp(M->RU[q], RU[q]);
        if (M->RVt[q].rows * M->RVt[q].cols) put_t(b + M->RVt[q].off, RV[q], M->RVt[q].cols, M->RVt[q].rows);
      }
      cp(M->B12[q], B12[q]);
      cp(M->B21[q], B21[q]);
    }
  } catch (...) {
    delete M;
    return nullptr;
  }
  return M;
}

// Y = A X.  Returns 0 on success, 1 on a bad argument, 2 when memory runs out.
int hmc_matmat(hmc_matrix* M, int64_t r, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  if (!M || r < 0 || ldx < M->n || ldy < M->n) return 1;
  if (r == 0 || M->n == 0) return 0;
  const int L = M->L, p = M->p, N = 2 * L - 1;
  const double* b = M->buf.data();
  const int R = static_cast<int>(r);
  if (M->kind == 0) {
    // HODLR (Fig. 4.1, left), owner-computes per leaf.  For every level l the
    // projections T = V^T X of both siblings are formed as sums of per-leaf
    // partial products (leaf order, so the sums do not depend on the thread
    // count); then each leaf adds the U rows of its ancestors times the
    // sibling's T to its D_i X_i.
    std::vector<int64_t> koff(L, 0);   // per leaf: offset of its level blocks in the partials
    std::vector<int> kl(static_cast<size_t>(L) * (p + 1), 0);
    int64_t per_leaf = 0;
    for (int i = 0; i < L; ++i) {
      int64_t s = 0;
      for (int l = 1; l <= p; ++l) {
        const int anc = (1 << l) - 1 + (i >> (p - l));
        const int par = (anc - 1) >> 1;
        const bool left = (anc & 1) != 0;
        const int k = left ? M->V21t[par].rows : M->V12t[par].rows;   // columns of X(I_anc) are projected by V21 (left) / V12 (right)
        kl[static_cast<size_t>(i) * (p + 1) + l] = k;
        s += k;
      }
      per_leaf = std::max(per_leaf, s);
    }
    // every entry read below is written first in this call (an empty leaf's
    // partials as zeros), so the work space is only grown, never cleared
    try {
      const size_t need = static_cast<size_t>(L) * per_leaf * R + static_cast<size_t>(N) * per_leaf * R;
      if (M->ws.size() < need) M->ws.resize(need);
    } catch (...) {
      return 2;
    }
    double* P = M->ws.data();                                   // [leaf][level blocks][r]
    double* T = P + static_cast<size_t>(L) * per_leaf * R;     // [node][k][r]
    const int64_t ldP = per_leaf;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < L; ++i) {
      const int leaf = L - 1 + i;
      const int64_t a0 = M->start[leaf];
      const int m = static_cast<int>(M->end[leaf] - a0);
      int64_t o = 0;
      for (int l = 1; l <= p; ++l) {
        const int anc = (1 << l) - 1 + (i >> (p - l));
        const int par = (anc - 1) >> 1;
        const bool left = (anc & 1) != 0;
        const Block& vt = left ? M->V21t[par] : M->V12t[par];
        const int64_t row_in = a0 - M->start[anc];
        gemm(vt.rows, R, m, b + vt.off + row_in * vt.rows, vt.rows, X + a0, ldx,
             P + static_cast<size_t>(i) * ldP * R + o, ldP, false);
        o += vt.rows;
      }
    }
    // T of node anc (projection of X(I_anc)) = sum over its leaves, left to right
    for (int l = 1; l <= p; ++l) {
#pragma omp parallel for schedule(dynamic)
      for (int j = 0; j < (1 << l); ++j) {
        const int anc = (1 << l) - 1 + j;
        const int k = kl[static_cast<size_t>(j << (p - l)) * (p + 1) + l];
        int64_t o = 0;
        for (int ll = 1; ll < l; ++ll) o += kl[static_cast<size_t>(j << (p - l)) * (p + 1) + ll];
        double* t = T + static_cast<size_t>(anc) * ldP * R;
        for (int c = 0; c < R; ++c)
          for (int e = 0; e < k; ++e) {
            double s = 0.0;
            for (int i = (j << (p - l)); i < ((j + 1) << (p - l)); ++i)
              s += P[static_cast<size_t>(i) * ldP * R + static_cast<size_t>(c) * ldP + o + e];
            t[static_cast<size_t>(c) * ldP + e] = s;
          }
      }
    }
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < L; ++i) {
      const int leaf = L - 1 + i;
      const int64_t a0 = M->start[leaf];
      const int m = static_cast<int>(M->end[leaf] - a0);
      if (m == 0) continue;
      gemm(m, R, m, b + M->D[i].off, m, X + a0, ldx, Y + a0, ldy, false);
      for (int l = 1; l <= p; ++l) {
        const int anc = (1 << l) - 1 + (i >> (p - l));
        const int par = (anc - 1) >> 1;
        const bool left = (anc & 1) != 0;
        const int sib = left ? anc + 1 : anc - 1;
        const Block& u = left ? M->U12[par] : M->U21[par];
        const int64_t row_in = a0 - M->start[anc];
        gemm(m, R, u.cols, b + u.off + row_in, u.rows, T + static_cast<size_t>(sib) * ldP * R, ldP, Y + a0, ldy,
             true);
      }
    }
    return 0;
  }
  // HSS (Fig. 4.1, right): leaf projections, upsweep through R_V, couplings
  // on levels 1..p, downsweep through R_U, leaf output U_i y_i + D_i X_i.
  int K = 1;
  for (int q = 0; q < N; ++q) K = std::max(K, std::max(M->ku[q], M->kv[q]));
  // x-hat of every node is written by the projections and the upsweep, y-hat
  // of every non-root node by its coupling (levels 1..p) before the downsweep
  // adds to it: the work space is only grown, never cleared
  try {
    const size_t need = 2 * static_cast<size_t>(N) * K * R;
    if (M->ws.size() < need) M->ws.resize(need);
  } catch (...) {
    return 2;
  }
  double* xh = M->ws.data();                                 // [node][kv][r]
  double* yh = xh + static_cast<size_t>(N) * K * R;          // [node][ku][r]
  auto XH = [&](int q) { return xh + static_cast<size_t>(q) * K * R; };
  auto YH = [&](int q) { return yh + static_cast<size_t>(q) * K * R; };
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < L; ++i) {
    const int q = L - 1 + i;
    const int64_t a0 = M->start[q];
    const int m = static_cast<int>(M->end[q] - a0);
    gemm(M->kv[q], R, m, b + M->Vt[i].off, M->Vt[i].rows, X + a0, ldx, XH(q), K, false);
  }
  for (int l = p - 1; l >= 1; --l) {
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < (1 << l); ++j) {
      const int q = (1 << l) - 1 + j;
      const int a = 2 * q + 1, c = 2 * q + 2;
      const Block& rv = M->RVt[q];
      gemm(rv.rows, R, M->kv[a], b + rv.off, rv.rows, XH(a), K, XH(q), K, false);
      gemm(rv.rows, R, M->kv[c], b + rv.off + static_cast<int64_t>(M->kv[a]) * rv.rows, rv.rows, XH(c), K, XH(q), K,
           true);
    }
  }
  for (int l = 1; l <= p; ++l) {
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < (1 << (l - 1)); ++j) {
      const int q = (1 << (l - 1)) - 1 + j;
      const int a = 2 * q + 1, c = 2 * q + 2;
      gemm(M->ku[a], R, M->kv[c], b + M->B12[q].off, M->B12[q].rows, XH(c), K, YH(a), K, false);
      gemm(M->ku[c], R, M->kv[a], b + M->B21[q].off, M->B21[q].rows, XH(a), K, YH(c), K, false);
    }
  }
  for (int l = 1; l <= p - 1; ++l) {
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < (1 << l); ++j) {
      const int q = (1 << l) - 1 + j;
      const int a = 2 * q + 1, c = 2 * q + 2;
      const Block& ru = M->RU[q];
      gemm(M->ku[a], R, ru.cols, b + ru.off, ru.rows, YH(q), K, YH(a), K, true);
      gemm(M->ku[c], R, ru.cols, b + ru.off + M->ku[a], ru.rows, YH(q), K, YH(c), K, true);
    }
  }
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < L; ++i) {
    const int q = L - 1 + i;
    const int64_t a0 = M->start[q];
    const int m = static_cast<int>(M->end[q] - a0);
    if (m == 0) continue;
    gemm(m, R, m, b + M->D[i].off, m, X + a0, ldx, Y + a0, ldy, false);
    if (p > 0) gemm(m, R, M->ku[q], b + M->U[i].off, m, YH(q), K, Y + a0, ldy, true);
  }
  return 0;
}

}  // extern "C"

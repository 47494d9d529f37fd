// LU without pivoting whose every third-order step runs through the emulated
// product: the Level-3-only factorization arXiv 2509.23565 times for blocking
// factors 256 to 2048 (Section 8), with the Schur update of Eq. 7.
//
// Step j0 (right-looking, block nb):
//   1. the panel A[j0:n, j0:j0+jb] is factored by recursive halving.  A leaf
//      (<= 64 columns) factors its diagonal block in FP64 inside one CTA and
//      forms the inverses of both triangular factors there; its rows below
//      become L21 = A21 U11^-1 through the emulated product.  An inner node
//      forms U12 = L11^-1 A12 and the Schur update of the rows below with the
//      emulated product, recurses into its right half, and joins the two
//      halves' unit-lower inverses, X21 = -X22 (L21 X11);
//   2. U12 = X A12 with X = L11^-1 of the whole block (emulated product);
//   3. A22 <- A22 - L21 U12 (emulated product, alpha = -1, beta = 1).
// The Schur updates and U12 run as products over K chunks of at most 1024, so
// every product at s <= 7 keeps the 128-column tile (see gemm_kchunks).
// No row is ever exchanged, so the factorization is stable only for matrices
// that need no pivoting (diagonally dominant, SPD).
#include <cuda_runtime.h>

#include "handle.h"

namespace emul {
namespace {

constexpr int kNpLeaf = 64;           // widest diagonal block factored in one CTA
constexpr int kNpThreads = 1024;      // 64 rows x 16 column groups
constexpr int kNpGroups = kNpThreads / kNpLeaf;
constexpr int kNpPerThread = kNpLeaf / kNpGroups;
constexpr int kNpChunk = 1024;        // K of one emulated product in the Schur updates
constexpr size_t kNpAl = 256;

inline size_t np_al(size_t x) { return (x + kNpAl - 1) / kNpAl * kNpAl; }

// The w x w diagonal block at A[d.., d..] (w <= 64) is factored in place
// without pivoting, A = L U (L unit lower), in shared memory; then
// X <- L^-1 (ld ldx, zeros above the diagonal) and Y <- U^-1 (ld w, zeros
// below).  A zero pivot leaves its column unscaled and records its 1-based
// index in *info unless an earlier one is there.  Thread (r, g) = (tid % 64,
// tid / 64) works on row r and the columns g, g + 16, ...; g is uniform in a
// warp, so the triangular structure is skipped by warp-uniform branches.
// FP64 runs at a small fraction of the tensor rate on this part, so the
// divisions are taken once per pivot (a reciprocal in shared memory) and the
// inverses touch only their nonzero triangles.
__global__ void __launch_bounds__(kNpThreads, 1) np_leaf_kernel(double* A, long lda, int d, int w, int32_t* info,
                                                                double* X, long ldx, double* Y) {
  __shared__ double S[kNpLeaf * (kNpLeaf + 1)];   // w x w, leading dimension w + 1
  __shared__ double rowbuf[2][kNpLeaf];
  __shared__ double rdiag[kNpLeaf];                // 1 / U(k,k) (0 for a zero pivot)
  const int tid = threadIdx.x;
  const int r = tid & (kNpLeaf - 1);
  const int g = tid / kNpLeaf;
  const int ld = w + 1;
  double* D = A + d + static_cast<long>(d) * lda;
  for (int j = g; j < w; j += kNpGroups)
    if (r < w) S[r + j * ld] = D[r + static_cast<long>(j) * lda];
  __syncthreads();
  if (tid == 0) {
    const double p = S[0];
    rdiag[0] = p != 0.0 ? 1.0 / p : 0.0;
    if (p == 0.0) atomicCAS(info, 0, d + 1);
  }
  for (int k = 0; k < w; ++k) {
    __syncthreads();                               // rdiag[k] and column k final
    const double rk = rdiag[k];
    if (g == 0 && r > k && r < w && rk != 0.0) S[r + k * ld] *= rk;
    __syncthreads();
    if (r > k && r < w) {
      const double l = S[r + k * ld];
      for (int j = k + 1 + g; j < w; j += kNpGroups) S[r + j * ld] = fma(-l, S[k + j * ld], S[r + j * ld]);
      // the owner of the next pivot publishes its reciprocal
      if (r == k + 1 && g == 0) {                 // its first column j = k + 1 is the pivot
        const double p = S[r + r * ld];
        rdiag[r] = p != 0.0 ? 1.0 / p : 0.0;
        if (p == 0.0) atomicCAS(info, 0, d + r + 1);
      }
    }
  }
  for (int j = g; j < w; j += kNpGroups)
    if (r < w) D[r + static_cast<long>(j) * lda] = S[r + j * ld];

  // X = L^-1: row r of X is e_r - sum_{k<r} L(r,k) X(k,:); row k of X is
  // zero right of column k
  double x[kNpPerThread];
#pragma unroll
  for (int t = 0; t < kNpPerThread; ++t) x[t] = (r == g + kNpGroups * t) ? 1.0 : 0.0;
  for (int k = 0; k + 1 < w; ++k) {
    double* rb = rowbuf[k & 1];
    if (r == k) {
#pragma unroll
      for (int t = 0; t < kNpPerThread; ++t) rb[g + kNpGroups * t] = x[t];
    }
    __syncthreads();
    if (r > k && r < w) {
      const double l = S[r + k * ld];
#pragma unroll
      for (int t = 0; t < kNpPerThread; ++t)
        if (g + kNpGroups * t <= k) x[t] = fma(-l, rb[g + kNpGroups * t], x[t]);
    }
  }
  if (r < w) {
#pragma unroll
    for (int t = 0; t < kNpPerThread; ++t)
      if (g + kNpGroups * t < w) X[r + static_cast<long>(g + kNpGroups * t) * ldx] = x[t];
  }
  __syncthreads();

  // Y = U^-1: row r of Y is (e_r - sum_{k>r} U(r,k) Y(k,:)) / U(r,r), k from
  // w-1 down; row k of Y is zero left of column k
#pragma unroll
  for (int t = 0; t < kNpPerThread; ++t) x[t] = (r == g + kNpGroups * t) ? 1.0 : 0.0;
  for (int k = w - 1; k >= 0; --k) {
    double* rb = rowbuf[k & 1];
    if (r == k) {
      const double rk = rdiag[k] != 0.0 ? rdiag[k] : __longlong_as_double(0x7FF0000000000000ll);
#pragma unroll
      for (int t = 0; t < kNpPerThread; ++t) {
        if (g + kNpGroups * t >= k) x[t] *= rk;
        rb[g + kNpGroups * t] = x[t];
      }
    }
    __syncthreads();
    if (r < k) {
      const double l = S[r + k * ld];
#pragma unroll
      for (int t = 0; t < kNpPerThread; ++t)
        if (g + kNpGroups * t >= k) x[t] = fma(-l, rb[g + kNpGroups * t], x[t]);
    }
  }
  if (r < w) {
#pragma unroll
    for (int t = 0; t < kNpPerThread; ++t)
      if (g + kNpGroups * t < w) Y[r + static_cast<long>(g + kNpGroups * t) * w] = x[t];
  }
}

struct NpBufs {
  double* X;     // jb x jb, ld nb: L11^-1 of the current block
  double* Y;     // 64 x 64: U^-1 of the current leaf
  double* T;     // scratch for the inverse join, up to nb x nb
  double* U;     // U12 of the current block, jb x (n - j0 - jb), ld jb
  long ldx;
};

// C <- beta C + alpha A B as consecutive emulated products over K chunks of at
// most kNpChunk (each rounded once; C must not overlap A or B).  A wider K
// would need level 2 in more than one accumulator job (1040 products of
// 127^2 per FP32 accumulator), which the 128-column product cannot take: it
// would fall back to 64-column tiles at half the rate; C is read and written
// once per chunk instead.
int gemm_kchunks(emul_handle_t h, int m, int n, int k, double alpha, Operand A, Operand B, double beta, double* C,
                 long ldc, int s) {
  for (int c0 = 0; c0 < k; c0 += kNpChunk) {
    const int kc = k - c0 < kNpChunk ? k - c0 : kNpChunk;
    const int rc = gemm_run(h, m, n, kc, alpha, Operand{A.ptr + c0 * A.cs, A.rs, A.cs},
                            Operand{B.ptr + c0 * B.cs, B.rs, B.cs}, c0 == 0 ? beta : 1.0, C, ldc, s, false, 0,
                            nullptr, 0, 0);
    if (rc) return rc;
  }
  return EMUL_OK;
}

// Split of a w-column panel: the left part a multiple of 16 near w/2.
inline int np_split(int w) {
  const int w1 = (w / 2 + 15) / 16 * 16;
  return w1 < w ? w1 : w / 2;
}

// Factor the panel A[d:n, d:d+w] (no pivoting) and leave L^-1 of its diagonal
// block in X at (d - j0, d - j0).
int np_panel(emul_handle_t h, double* A, long lda, int n, int j0, int d, int w, int s, int32_t* info,
             const NpBufs& B) {
  double* Xd = B.X + (d - j0) + static_cast<long>(d - j0) * B.ldx;
  if (w <= kNpLeaf) {
    np_leaf_kernel<<<1, kNpThreads, 0, h->stream>>>(A, lda, d, w, info, Xd, B.ldx, B.Y);
    h->launches++;
    int rc = check_cuda(h, cudaGetLastError(), "no-pivot leaf");
    if (rc) return rc;
    const int mb = n - d - w;
    if (mb <= 0) return EMUL_OK;
    double* A21 = A + (d + w) + static_cast<long>(d) * lda;
    // L21 = A21 U11^-1, written over A21 (both operands are sliced before the product writes)
    return gemm_run(h, mb, w, w, 1.0, Operand{A21, 1, lda}, Operand{B.Y, w, 1}, 0.0, A21, lda, s, false, 0,
                    nullptr, 0, 0);
  }
  const int w1 = np_split(w), w2 = w - w1;
  int rc = np_panel(h, A, lda, n, j0, d, w1, s, info, B);
  if (rc) return rc;
  double* A12 = A + d + static_cast<long>(d + w1) * lda;
  // U12 = L11^-1 A12 (w1 x w2), over A12
  rc = gemm_run(h, w1, w2, w1, 1.0, Operand{Xd, 1, B.ldx}, Operand{A12, lda, 1}, 0.0, A12, lda, s, false, 0, nullptr,
                0, 0);
  if (rc) return rc;
  // Schur update of the right half, every row below the left half's diagonal block
  const double* L21 = A + (d + w1) + static_cast<long>(d) * lda;
  double* A22 = A + (d + w1) + static_cast<long>(d + w1) * lda;
  rc = gemm_kchunks(h, n - d - w1, w2, w1, -1.0, Operand{L21, 1, lda}, Operand{A12, lda, 1}, 1.0, A22, lda, s);
  if (rc) return rc;
  rc = np_panel(h, A, lda, n, j0, d + w1, w2, s, info, B);
  if (rc) return rc;
  // join the inverses: X21 = -X22 (L21 X11), L21 the w2 x w1 block below the left diagonal block
  double* X22 = Xd + w1 + static_cast<long>(w1) * B.ldx;
  double* X21 = Xd + w1;
  rc = gemm_run(h, w2, w1, w1, 1.0, Operand{L21, 1, lda}, Operand{Xd, B.ldx, 1}, 0.0, B.T, w2, s, false, 0, nullptr,
                0, 0);
  if (rc) return rc;
  return gemm_run(h, w2, w1, w2, -1.0, Operand{X22, 1, B.ldx}, Operand{B.T, w2, 1}, 0.0, X21, B.ldx, s, false, 0,
                  nullptr, 0, 0);
}

}  // namespace
}  // namespace emul

extern "C" {

int emul_dgetrf_nopiv(emul_handle_t h, int n, double* A, int lda, int nb, int slices, int32_t* info,
                      emul_stats* stats) {
  using namespace emul;
  if (!h) return EMUL_INVALID_ARG;
  if (nb == 0) nb = 1024;
  if (n < 0 || lda < (n > 1 ? n : 1) || nb < 16 || nb > 4096 || slices < 1 || slices > kMaxSlices ||
      (n > 0 && (!A || !info)))
    return set_error(h, EMUL_INVALID_ARG, "emul_dgetrf_nopiv: invalid argument");
  if (stats) *stats = emul_stats{0, slices, slices, 0, 0.0, static_cast<double>(slices)};
  if (n == 0) return EMUL_OK;
  int rc = check_cuda(h, cudaMemsetAsync(info, 0, sizeof(int32_t), h->stream), "info reset");
  if (rc) return rc;
  const int nbe = nb < n ? nb : n;
  // [product workspace | X (nbe x nbe) | Y (64 x 64) | T (nbe x nbe) | U (nbe x n)]
  const size_t gw = np_al(gemm_workspace_bytes(n, n, nbe, slices, false));
  const size_t xb = np_al(8ull * nbe * nbe), yb = np_al(8ull * kNpLeaf * kNpLeaf);
  rc = reserve_workspace(h, gw + 2 * xb + yb + np_al(8ull * nbe * n));
  if (rc) return rc;
  uint8_t* base = static_cast<uint8_t*>(h->ws);
  const NpBufs B{reinterpret_cast<double*>(base + gw), reinterpret_cast<double*>(base + gw + xb),
                 reinterpret_cast<double*>(base + gw + xb + yb), reinterpret_cast<double*>(base + gw + 2 * xb + yb),
                 nbe};
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = nb < n - j0 ? nb : n - j0;
    int ph = phase_begin(h, EMUL_PHASE_PANEL);
    // the blocks of X above the diagonal are never written: zero them
    rc = check_cuda(h, cudaMemsetAsync(B.X, 0, 8ull * nbe * jb, h->stream), "inverse reset");
    if (rc) return rc;
    rc = np_panel(h, A, lda, n, j0, j0, jb, slices, info, B);
    phase_end(h, ph);
    if (rc) return rc;
    const int m2 = n - j0 - jb;
    if (m2 > 0) {
      ph = phase_begin(h, EMUL_PHASE_U12);
      double* A12 = A + j0 + static_cast<long>(j0 + jb) * lda;
      // U12 = X A12 into U, by K chunks; X is lower triangular, so chunk c only
      // reaches the rows from c on
      for (int c0 = 0; c0 < jb && !rc; c0 += kNpChunk) {
        const int kc = jb - c0 < kNpChunk ? jb - c0 : kNpChunk;
        rc = gemm_run(h, jb - c0, m2, kc, 1.0, Operand{B.X + c0 + static_cast<long>(c0) * B.ldx, 1, B.ldx},
                      Operand{A12 + c0, lda, 1}, c0 == 0 ? 0.0 : 1.0, B.U + c0, jb, slices, false, 0, nullptr, 0, 0);
      }
      if (!rc)
        rc = check_cuda(h, cudaMemcpy2DAsync(A12, 8ull * lda, B.U, 8ull * jb, 8ull * jb, m2, cudaMemcpyDeviceToDevice,
                                             h->stream), "U12 copy");
      phase_end(h, ph);
      if (rc) return rc;
      ph = phase_begin(h, EMUL_PHASE_UPDATE);
      const double* L21 = A + (j0 + jb) + static_cast<long>(j0) * lda;
      double* A22 = A + (j0 + jb) + static_cast<long>(j0 + jb) * lda;
      rc = gemm_kchunks(h, m2, m2, jb, -1.0, Operand{L21, 1, lda}, Operand{B.U, jb, 1}, 1.0, A22, lda, slices);
      phase_end(h, ph);
      if (rc) return rc;
    }
    if (stats) stats->steps++;
  }
  return EMUL_OK;
}

}  // extern "C"

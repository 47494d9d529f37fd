// Blocked LU with partial pivoting and blocked Cholesky whose third-order work
// runs through the emulated product (arXiv 2509.23565, Section 4, Eq. 5-7),
// the triangular solves that use the factors, and the residual of Eq. 8.
//
// LU step (right-looking, block nb):
//   1. panel [A11; A21] factored with partial pivoting: recursive halving; the
//      inner Schur updates use the emulated product, the leaves (<= 32 columns)
//      run a cooperative multi-block FP64 kernel (pivot search on the IEEE bit
//      patterns, one bounded grid barrier per column);
//   2. the panel's row interchanges applied to the columns left and right of it;
//   3. U12 = L11^-1 A12: L11^-1 formed in FP64 (unit lower, nb x nb), the
//      product by the emulated GEMM;
//   4. A22 <- A22 - L21 U12 by the emulated GEMM (alpha = -1, beta = 1).
// Cholesky step (lower): FP64 diagonal block, L21 = A21 L11^-T through an FP64
// L11^-1 and the emulated GEMM, then A22 <- A22 - L21 L21^T on lower tiles only,
// with one slice set serving both operands.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <set>
#include <utility>

#include <cuda_runtime.h>

#include "handle.h"

namespace emul {

namespace {

constexpr int kLeaf = 32;           // widest panel handled by the leaf kernel
constexpr int kLeafThreads = 256;
constexpr int kStatusTimeout = -4;
constexpr size_t kAl = 256;
inline size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

// Pivot exchange of the leaf: every block publishes its candidate as 8-byte
// words {32-bit payload, 32-bit epoch}; an aligned 64-bit store is
// single-copy atomic, so a reader that sees the epoch of the current column in
// a word also sees that word's payload, and no fence or counter is needed.
// Record of block b for column parity par: words [0, 4) = |value| low and high
// halves, candidate row, unused; words [4, 4 + 2w) = the candidate row, each
// double as its low and high halves.  Epoch = salt * 32 + column (salt > 0,
// distinct per leaf launch, records cleared before a factorization).
constexpr int kRecWords = 4 + 2 * kLeaf;

__device__ __forceinline__ void put_word(uint64_t* p, uint32_t payload, uint32_t epoch) {
  *reinterpret_cast<volatile uint64_t*>(p) = (static_cast<uint64_t>(epoch) << 32) | payload;
}
// Two adjacent words (16-byte aligned) in one load; each stays single-copy atomic.
__device__ __forceinline__ void get_pair(const uint64_t* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
__device__ __forceinline__ bool has_epoch(uint64_t v, uint32_t epoch) { return static_cast<uint32_t>(v >> 32) == epoch; }
// Poll a pair of words until both carry `epoch` (bounded); the double they
// hold (low half first) is returned in x.  False on timeout.
__device__ __forceinline__ bool wait_pair(const uint64_t* p, uint32_t epoch, double& x, long long limit) {
  uint64_t a, b;
  get_pair(p, a, b);
  if (!(has_epoch(a, epoch) && has_epoch(b, epoch))) {
    const long long t0 = clock64();
    do {
      if (clock64() - t0 > limit) return false;
      get_pair(p, a, b);
    } while (!(has_epoch(a, epoch) && has_epoch(b, epoch)));
  }
  x = __longlong_as_double(static_cast<long long>((b << 32) | (a & 0xFFFFFFFFull)));
  return true;
}
constexpr int kMaxRecPerLane = 8;   // records polled by one lane: the leaf runs at most 256 blocks

__device__ __forceinline__ uint64_t absbits(double x) {
  return static_cast<uint64_t>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

// (value, row) pair ordering of the pivot search: larger |value| wins, ties
// go to the smaller row (the first maximal index, as LAPACK's idamax).
__device__ __forceinline__ bool better(uint64_t v1, int r1, uint64_t v2, int r2) {
  return v1 > v2 || (v1 == v2 && r1 < r2);
}

// Leaf panel: rows d0..n-1, columns d0..d0+w-1 of A, factored in place with
// partial pivoting.  Block b keeps panel rows [b*R, b*R+R) in shared memory.
//
// Column c: (1) pivot search on column c over the block's rows, (2) the
// block's candidate (|value|, row, the row itself) and, from the block owning
// it, row c published as epoch-tagged words, (3) warp 0 collects the G
// candidates and fetches the winner's row, the last warp fetches row c, while
// warps 1-6 apply the rank-1 update of pivot c-1 to columns c+1..w-1,
// (4) row interchange, (5) multipliers of column c and the update of column
// c+1 only, so that the next pivot search can start.  Each entry receives the
// same FMAs in the same order as in a plain right-looking elimination; the
// published rows get the deferred update of pivot c-1 applied on the fly (the
// same FMA).  The exchange needs no grid barrier: a block cannot publish
// column c+2 into the slot of column c before every block has published
// column c+1, which each does only after reading column c.
//
// Every interchange is also applied to the columns [pc0, d0) and [d0+w, pc1) of
// the enclosing panel, which live in global memory: the outside column q
// (0-based over both ranges) belongs to block q % G for the whole launch, to
// the (q / G)-th of its threads other than thread 0 (it publishes the block's
// candidate) and the row-c reader (first lane of the last warp), so successive
// interchanges of one element stay in program order.  Its loads are issued
// when the pivot is known, its stores when the next pivot is known, off the
// critical path.  At most 248 outside columns exist (panel <= 256 wide, leaf
// >= 8 wide); 254 owners per block are available.
__global__ void __launch_bounds__(kLeafThreads) getf2_leaf_kernel(double* A, long lda, int n, int d0, int w, int R,
                                                                 int pc0, int pc1, int32_t* ipiv, int32_t* info,
                                                                 uint64_t* recs, uint64_t* drec, uint32_t salt,
                                                                 int* status, long long limit) {
  extern __shared__ double P[];   // P[c*R + lr]
  __shared__ double prow[2][kLeaf], crow[kLeaf];
  __shared__ double rcp_s;
  __shared__ uint64_t red_v[kLeafThreads / 32];
  __shared__ int red_r[kLeafThreads / 32];
  __shared__ int win_s, ok_s, ok7_s;
  constexpr int kRowTid = kLeafThreads - 32;   // first lane of the last warp: row-c reader
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int mp = n - d0;
  const int r0 = b * R;
  const int rcount = mp - r0 < R ? (mp - r0 > 0 ? mp - r0 : 0) : R;
  const int nleft = d0 - pc0;
  const int nout = nleft + (pc1 - d0 - w);
  const int ot = (tid == 0 || tid == kRowTid) ? -1 : tid - 1 - (tid > kRowTid ? 1 : 0);
  const int q = ot * G + b;
  double* ocol = ot >= 0 && q < nout ? A + static_cast<long>(q < nleft ? pc0 + q : d0 + w + (q - nleft)) * lda : nullptr;
  long sw_c = -1, sw_p = -1;   // pending interchange of this thread's outside column
  double sw_xc = 0.0, sw_xp = 0.0;
  bool pend = false;           // pivot c-1 was nonzero: its update of columns > c is pending
  // stage the rows: 16 loads in flight per thread before their stores
  for (int lr = tid; lr < rcount; lr += blockDim.x) {
    const double* src = A + (d0 + r0 + lr) + static_cast<long>(d0) * lda;
    for (int c0 = 0; c0 < w; c0 += 16) {
      double v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = c0 + j < w ? src[static_cast<long>(c0 + j) * lda] : 0.0;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < w) P[(c0 + j) * R + lr] = v[j];
    }
  }
  __syncthreads();

  for (int c = 0; c < w; ++c) {
    const int par = c & 1;
    const uint32_t ep = (salt << 5) | static_cast<uint32_t>(c);
    const double* pv = prow[par ^ 1];   // pivot row of column c-1
    uint64_t* rec_all = recs + static_cast<long>(par) * G * kRecWords;
    uint64_t* my = rec_all + static_cast<long>(b) * kRecWords;
    uint64_t* drow = drec + par * 2 * kLeaf;
    // (1) local candidate for column c over own rows with panel row >= c
    uint64_t bv = 0;
    int br = 0x7FFFFFFF;
    for (int lr = tid; lr < rcount; lr += blockDim.x) {
      const int pr = r0 + lr;
      if (pr < c) continue;
      const uint64_t v = absbits(P[c * R + lr]);
      if (better(v, pr, bv, br)) {
        bv = v;
        br = pr;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t v2 = __shfl_xor_sync(0xFFFFFFFFu, bv, o);
      const int r2 = __shfl_xor_sync(0xFFFFFFFFu, br, o);
      if (better(v2, r2, bv, br)) {
        bv = v2;
        br = r2;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_r[warp] = br;
    }
    __syncthreads();
    if (tid == 0) {
      for (int i = 1; i < static_cast<int>(blockDim.x / 32); ++i)
        if (better(red_v[i], red_r[i], bv, br)) {
          bv = red_v[i];
          br = red_r[i];
        }
      put_word(my + 0, static_cast<uint32_t>(bv), ep);
      put_word(my + 1, static_cast<uint32_t>(bv >> 32), ep);
      put_word(my + 2, static_cast<uint32_t>(br), ep);
      win_s = br;
    }
    __syncthreads();
    // (2) publish the candidate row and row c, current through pivot c-1
    {
      const int pr = win_s;
      if (tid < 2 * w) {
        const int cc = tid >> 1;
        if (pr != 0x7FFFFFFF) {
          const int lr = pr - r0;
          double v = P[cc * R + lr];
          if (pend && cc > c) v = fma(-P[(c - 1) * R + lr], pv[cc], v);
          const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(v));
          put_word(my + 4 + tid, static_cast<uint32_t>(tid & 1 ? bits >> 32 : bits), ep);
        }
        if (c >= r0 && c < r0 + rcount) {
          const int lr = c - r0;
          double v = P[cc * R + lr];
          if (pend && cc > c) v = fma(-P[(c - 1) * R + lr], pv[cc], v);
          const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(v));
          put_word(drow + tid, static_cast<uint32_t>(tid & 1 ? bits >> 32 : bits), ep);
        }
      }
    }
    __syncthreads();
    // (3) exchange (warp 0: candidates and pivot row; last warp: row c) while
    // warps 1-6 apply the deferred update of pivot c-1
    if (warp == 0) {
      // every lane loads all of its records at once, then re-polls the late ones
      uint64_t w0[kMaxRecPerLane], w1[kMaxRecPerLane], w2[kMaxRecPerLane];
      unsigned pending = 0;
#pragma unroll
      for (int k = 0; k < kMaxRecPerLane; ++k)
        if (lane + 32 * k < G) pending |= 1u << k;
      bool ok = true;
      const long long t0 = clock64();
      while (true) {
#pragma unroll
        for (int k = 0; k < kMaxRecPerLane; ++k)
          if (pending >> k & 1u) {
            const uint64_t* r = rec_all + static_cast<long>(lane + 32 * k) * kRecWords;
            uint64_t unused;
            get_pair(r, w0[k], w1[k]);
            get_pair(r + 2, w2[k], unused);
          }
#pragma unroll
        for (int k = 0; k < kMaxRecPerLane; ++k)
          if ((pending >> k & 1u) && has_epoch(w0[k], ep) && has_epoch(w1[k], ep) && has_epoch(w2[k], ep))
            pending &= ~(1u << k);
        if (__all_sync(0xFFFFFFFFu, pending == 0)) break;
        if (__any_sync(0xFFFFFFFFu, clock64() - t0 > limit)) {
          ok = false;
          break;
        }
      }
      uint64_t gv = 0;
      int gr = 0x7FFFFFFF, gbk = 0;
#pragma unroll
      for (int k = 0; k < kMaxRecPerLane; ++k) {
        if (lane + 32 * k >= G) continue;
        const uint64_t v = ((w1[k] & 0xFFFFFFFFull) << 32) | (w0[k] & 0xFFFFFFFFull);
        const int rr = static_cast<int>(static_cast<uint32_t>(w2[k]));
        if (better(v, rr, gv, gr)) {
          gv = v;
          gr = rr;
          gbk = lane + 32 * k;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t v2 = __shfl_xor_sync(0xFFFFFFFFu, gv, o);
        const int r2 = __shfl_xor_sync(0xFFFFFFFFu, gr, o);
        const int b2 = __shfl_xor_sync(0xFFFFFFFFu, gbk, o);
        if (better(v2, r2, gv, gr)) {
          gv = v2;
          gr = r2;
          gbk = b2;
        }
      }
      if (ok && lane < w) {
        double pvv = 0.0;
        ok = wait_pair(rec_all + static_cast<long>(gbk) * kRecWords + 4 + 2 * lane, ep, pvv, limit);
        prow[par][lane] = pvv;
        if (lane == c) rcp_s = 1.0 / pvv;
      }
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (lane == 0) {
        win_s = gr;
        ok_s = ok;
        if (!ok) atomicExch(status, kStatusTimeout);
        if (ok && b == 0) {
          ipiv[d0 + c] = d0 + gr + 1;
          if (gv == 0) atomicCAS(info, 0, d0 + c + 1);
        }
      }
    } else if (warp == kLeafThreads / 32 - 1) {
      bool ok = true;
      if (lane < w) {
        double x = 0.0;
        ok = wait_pair(drow + 2 * lane, ep, x, limit);
        crow[lane] = x;
      }
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (lane == 0) {
        ok7_s = ok;
        if (!ok) atomicExch(status, kStatusTimeout);
      }
    } else if (pend && c + 1 < w) {
      constexpr int kUpd = kLeafThreads - 64;   // warps 1-6
      for (int lr = tid - 32; lr < rcount; lr += kUpd) {
        if (r0 + lr <= c - 1) continue;
        const double l = P[(c - 1) * R + lr];
        for (int cc = c + 1; cc < w; ++cc) P[cc * R + lr] = fma(-l, pv[cc], P[cc * R + lr]);
      }
    }
    __syncthreads();
    if (!ok_s || !ok7_s) return;
    const int p = win_s;
    if (ocol) {
      if (sw_c >= 0) {
        ocol[sw_c] = sw_xp;
        ocol[sw_p] = sw_xc;
        sw_c = -1;
      }
      if (p != c) {
        sw_c = d0 + c;
        sw_p = d0 + p;
        sw_xc = ocol[sw_c];
        sw_xp = ocol[sw_p];
      }
    }
    const double piv = prow[par][c];
    pend = piv != 0.0;
    if (pend) {
      // (4) interchange rows c and p (both current through pivot c-1)
      if (p != c) {
        if (c >= r0 && c < r0 + rcount)
          for (int cc = tid; cc < w; cc += blockDim.x) P[cc * R + (c - r0)] = prow[par][cc];
        if (p >= r0 && p < r0 + rcount)
          for (int cc = tid; cc < w; cc += blockDim.x) P[cc * R + (p - r0)] = crow[cc];
      }
      __syncthreads();
      // (5) multipliers of column c, update of column c+1
      const bool use_rcp = fabs(piv) >= 2.2250738585072014e-308;
      const double rcp = rcp_s;
      const double u1 = c + 1 < w ? prow[par][c + 1] : 0.0;
      for (int lr = tid; lr < rcount; lr += blockDim.x) {
        if (r0 + lr <= c) continue;
        const double l = use_rcp ? P[c * R + lr] * rcp : P[c * R + lr] / piv;
        P[c * R + lr] = l;
        if (c + 1 < w) P[(c + 1) * R + lr] = fma(-l, u1, P[(c + 1) * R + lr]);
      }
    }
    __syncthreads();
  }
  if (sw_c >= 0) {
    ocol[sw_c] = sw_xp;
    ocol[sw_p] = sw_xc;
  }
  for (int c = 0; c < w; ++c)
    for (int lr = tid; lr < rcount; lr += blockDim.x) A[(d0 + r0 + lr) + static_cast<long>(d0 + c) * lda] = P[c * R + lr];
}

// Row interchanges ipiv[k1..k2) (1-based global rows, ipiv[k]-1 >= k) resolved
// into a gather map: after the interchanges, row dst[i] holds the original row
// src[i], for the *count affected rows (at most 2 (k2-k1)).  Applying
// transposition k to every row in turn, the content ending at row r is
// sigma(r) = t_k1(t_k1+1(... t_k2-1(r))): the transpositions taken in reverse
// order on r alone, so every row is resolved by its own thread (thread i:
// row k1+i, and row ipiv[k1+i]-1 when it lies beyond the block and no earlier
// interchange names it).  The map's order is immaterial to its users.
constexpr int kPermMax = 256;          // interchanges per gather map (longer ranges: several maps)
__global__ void __launch_bounds__(kPermMax) laswp_perm_kernel(const int32_t* ipiv, int k1, int k2,
                                                             int* map /* [2][2*kPermMax] + count */) {
  __shared__ int piv_s[kPermMax];
  __shared__ int cnt_s;
  const int nb = k2 - k1;
  const int i = threadIdx.x;
  if (i < nb) piv_s[i] = ipiv[k1 + i] - 1;
  if (i == 0) cnt_s = 0;
  __syncthreads();
  int* dst = map;
  int* src = map + 2 * kPermMax;
  auto sigma = [&](int r) {
    for (int k = nb - 1; k >= 0; --k) {
      const int p = piv_s[k], kk = k1 + k;
      r = r == kk ? p : (r == p ? kk : r);
    }
    return r;
  };
  if (i < nb) {
    const int r = k1 + i;
    const int sr = sigma(r);
    if (sr != r) {
      const int pos = atomicAdd(&cnt_s, 1);
      dst[pos] = r;
      src[pos] = sr;
    }
    const int p = piv_s[i];
    if (p >= k2) {
      bool first = true;
      for (int j = 0; j < i && first; ++j) first = piv_s[j] != p;
      if (first) {
        const int sp = sigma(p);
        if (sp != p) {
          const int pos = atomicAdd(&cnt_s, 1);
          dst[pos] = p;
          src[pos] = sp;
        }
      }
    }
  }
  __syncthreads();
  if (i == 0) map[4 * kPermMax] = cnt_s;
}

// Apply the gather map to columns [c0, c1): each block owns 8 columns, reads
// every source row into shared memory, then writes the destinations.
constexpr int kSwpCols = 8;
__global__ void __launch_bounds__(256) laswp_apply_kernel(double* A, long lda, int c0, int c1, const int* map) {
  __shared__ double buf[kSwpCols][2 * kPermMax];
  __shared__ int dst_s[2 * kPermMax], src_s[2 * kPermMax];
  const int cnt = map[4 * kPermMax];
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    dst_s[i] = map[i];
    src_s[i] = map[2 * kPermMax + i];
  }
  __syncthreads();
  const int cb = c0 + blockIdx.x * kSwpCols;
  const int ncol = c1 - cb < kSwpCols ? c1 - cb : kSwpCols;
  for (int j = 0; j < ncol; ++j) {
    const double* col = A + static_cast<long>(cb + j) * lda;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) buf[j][i] = col[src_s[i]];
  }
  __syncthreads();
  for (int j = 0; j < ncol; ++j) {
    double* col = A + static_cast<long>(cb + j) * lda;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) col[dst_s[i]] = buf[j][i];
  }
}

// Deferred interchanges of the L columns.  G is the composite gather of the
// interchanges of all later panels (G[r]: the row whose content ends at row r)
// and H its inverse; prepending a panel's interchanges (its gather map: row
// dst[i] receives the original row src[i], a permutation of the touched rows)
// changes only the rows r = H[dst[i]]: G[r] = src[i], H[src[i]] = r.
__global__ void iota2_kernel(int n, int* G, int* H) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    G[i] = i;
    H[i] = i;
  }
}

__global__ void compose_kernel(const int* map, int* G, int* H) {
  __shared__ int rr[2 * kPermMax];
  const int cnt = map[4 * kPermMax];
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) rr[i] = H[map[i]];
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int src = map[2 * kPermMax + i];
    G[rr[i]] = src;
    H[src] = rr[i];
  }
}

// tmp[(r - r0) + c (n - r0)] = A[G[r], c0 + c] for r in [r0, n); blockIdx.y = c.
__global__ void gather_rows_kernel(const double* A, long lda, int r0, int n, int c0, const int* G, double* tmp) {
  const int r = r0 + blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (r < n) tmp[(r - r0) + static_cast<long>(c) * (n - r0)] = A[G[r] + static_cast<long>(c0 + c) * lda];
}

// X (w1 x w2 at A[d0.., c0..]) <- L^-1 X with L unit lower w1 x w1 at A[d0.., d0..]
// (w1 <= 128).  The strictly lower part of L is staged in shared memory; one
// warp per column of X (cpb columns per block), lane l holding rows l, l+32,
// l+64, l+96 in registers, x_k broadcast by shuffle.
constexpr int kTrsmMax = 128;
inline int trtri_threads(int nb) { return nb <= 256 ? 256 : 512; }
__global__ void __launch_bounds__(256) trsm_small_kernel(double* A, long lda, int d0, int w1, int c0, int w2,
                                                         int cpb) {
  // all threads stage L; the first cpb warps solve one column of X each
  extern __shared__ double Ls[];   // Ls[i + k*w1] = L(i, k) for i > k, else 0
  const int tid = threadIdx.x, lane = tid & 31;
  {
    // row i per thread, columns k = tid/128 + 2j, 16 loads in flight before their stores
    const int i = tid & 127, kstep = blockDim.x >> 7;
    if (i < w1)
      for (int k0 = tid >> 7; k0 < w1; k0 += 16 * kstep) {
        double v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int k = k0 + j * kstep;
          v[j] = (k < w1 && i > k) ? A[(d0 + i) + static_cast<long>(d0 + k) * lda] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int k = k0 + j * kstep;
          if (k < w1) Ls[i + k * w1] = v[j];
        }
      }
  }
  __syncthreads();
  if ((tid >> 5) >= cpb) return;
  const int j = blockIdx.x * cpb + (tid >> 5);
  if (j >= w2) return;
  double* col = A + static_cast<long>(c0 + j) * lda + d0;
  double x[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) x[t] = lane + 32 * t < w1 ? col[lane + 32 * t] : 0.0;
#pragma unroll
  for (int t0 = 0; t0 < 4; ++t0) {
    for (int kk = 0; kk < 32; ++kk) {
      const int k = 32 * t0 + kk;
      if (k >= w1) break;
      const double xk = __shfl_sync(0xFFFFFFFFu, x[t0], kk);
#pragma unroll
      for (int t = t0; t < 4; ++t) {
        const int i = lane + 32 * t;
        if (i > k && i < w1) x[t] = fma(-Ls[i + k * w1], xk, x[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (lane + 32 * t < w1) col[lane + 32 * t] = x[t];
}

// ---------------------------------------------------------------- Cholesky diagonal block
// The nb x nb diagonal block of a Cholesky step (nb <= 512) is factored in
// FP64 by 32-column panels: a one-block leaf factors the panel's 32 x 32
// diagonal block in shared memory, the rows below it within the block are
// solved against it and the rest of the block is updated by a small FP64
// product spread over many blocks, and L11^-1 is formed afterwards column by
// column.  GB300 retires ~1.6 FP64 instructions per clock per SM, so no step
// keeps a large amount of FP64 work on a single SM.
constexpr int kCholLeaf = 32;

// Unblocked lower Cholesky of the w x w (w <= 32) block at A[d0.., d0..],
// right-looking, by four warps: lane i holds row i, warp q the columns
// j = 4s + q (s = 0..7) in registers, so the FP64 work is spread over the
// SM's four sub-partitions.  Pivot jj: its owner warp takes r = rsqrt(d) of
// the pivot d, sets L_jj = d r, scales the column by r and publishes it in
// shared memory (double-buffered, one 128-thread barrier per pivot); every
// warp then updates its columns right of jj.  GB300's FP64 latency makes every
// dependent FP64 step costly, so each pivot takes one reciprocal square root
// rather than a square root and a division.  A non-positive pivot sets *info
// (first index) and stops; nothing runs once *info is set.
// It also writes the leaf's inverse L^-1 (lower, w x w) to inv[i + j*ldi]:
// forward substitution on the identity, all columns at once, each warp on its
// own columns (row m of X, once final, is broadcast within the warp by
// shuffles; the multipliers L[i][m] come from shared memory), with the
// diagonal reciprocals formed in parallel up front.
__global__ void __launch_bounds__(128) chol_leaf_kernel(double* A, long lda, int d0, int w, double* inv, int ldi,
                                                       int32_t* info) {
  __shared__ double col[2][kCholLeaf];
  __shared__ double Ls[kCholLeaf][kCholLeaf + 1];
  __shared__ int fail_s;
  const int i = threadIdx.x & 31, q = threadIdx.x >> 5;
  if (threadIdx.x == 0) fail_s = (*info != 0);
  __syncthreads();
  if (fail_s) return;
  double* blk = A + d0 + static_cast<long>(d0) * lda;
  // padding beyond w is the identity, so the inverse below needs no special case
  double d[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int j = 4 * s + q;
    d[s] = (i < w && j < w) ? (i >= j ? blk[i + static_cast<long>(j) * lda] : 0.0) : (i == j ? 1.0 : 0.0);
  }
  int done = w;
#pragma unroll
  for (int jj = 0; jj < kCholLeaf; ++jj) {
    if (jj >= w) break;                       // uniform over the block
    const int s0 = jj >> 2;
    if (q == (jj & 3)) {
      const double diag = __shfl_sync(0xFFFFFFFFu, d[s0], jj);
      const bool ok = diag > 0.0;
      if (ok) {
        const double r = rsqrt(diag);
        if (i == jj)
          d[s0] = diag * r;
        else if (i > jj)
          d[s0] *= r;
      } else if (i == 0) {
        atomicCAS(info, 0, d0 + jj + 1);
        fail_s = 1;
      }
      col[jj & 1][i] = i >= jj ? d[s0] : 0.0;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (fail_s) {
      done = jj;
      break;
    }
    const double lij = col[jj & 1][i];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int j = 4 * s + q;
      if (j > jj && i >= j) d[s] = fma(-lij, col[jj & 1][j], d[s]);
    }
  }
  // write back the columns that were finished (all of them unless a pivot failed)
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int j = 4 * s + q;
    if (i < w && j < done && i >= j) blk[i + static_cast<long>(j) * lda] = d[s];
  }
  if (done < w) return;
  // the factor in shared memory for the inverse's multipliers
#pragma unroll
  for (int s = 0; s < 8; ++s) Ls[i][4 * s + q] = d[s];
  __syncthreads();
  const double rcp = 1.0 / Ls[i][i];
  double x[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) x[s] = (i == 4 * s + q) ? 1.0 : 0.0;
#pragma unroll
  for (int m = 0; m < kCholLeaf; ++m) {
    if (i == m) {
#pragma unroll
      for (int s = 0; s < 8; ++s) x[s] *= rcp;   // row m of X is final
    }
    const double lim = i > m ? Ls[i][m] : 0.0;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const double xm = __shfl_sync(0xFFFFFFFFu, x[s], m);
      x[s] = fma(-lim, xm, x[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int j = 4 * s + q;
    if (i < w && j < w) inv[i + static_cast<long>(j) * ldi] = x[s];
  }
}

// C(i, j) = beta C(i, j) + alpha sum_l A(i, l) B(j, l) in FP64, for the m x n
// C (ldc) with A(i, l) = A[i*ars + l*acs] and B(j, l) = B[j*brs + l*bcs];
// lower = 1 writes only i >= j.  A block computes a 16 x 32 tile (one entry
// per thread) over K chunks of 32 staged in shared memory; with n <= 32 and
// k <= 32 every block reads all its operands before it writes, so C may then
// alias A's rows of the same block (the in-place triangular solve).
__global__ void __launch_bounds__(512) dgemm_nt_small_kernel(int m, int n, int k, double alpha, const double* A,
                                                            long ars, long acs, const double* B, long brs,
                                                            long bcs, double beta, double* C, long ldc,
                                                            int lower, const int32_t* info) {
  __shared__ double As[16][33], Bs[32][33];
  if (*info != 0) return;
  const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
  const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 32;
  if (lower && j0 > i0 + 15) return;          // tile entirely above the diagonal
  const int i = i0 + ti, j = j0 + tj;
  double acc = 0.0;
  for (int l0 = 0; l0 < k; l0 += 32) {
    for (int e = threadIdx.x; e < 16 * 32; e += blockDim.x) {
      const int r = e & 15, l = e >> 4;
      As[r][l] = (i0 + r < m && l0 + l < k) ? A[(i0 + r) * ars + static_cast<long>(l0 + l) * acs] : 0.0;
    }
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int r = e & 31, l = e >> 5;
      Bs[r][l] = (j0 + r < n && l0 + l < k) ? B[(j0 + r) * brs + static_cast<long>(l0 + l) * bcs] : 0.0;
    }
    __syncthreads();
    const int lk = k - l0 < 32 ? k - l0 : 32;
    for (int l = 0; l < lk; ++l) acc = fma(As[ti][l], Bs[tj][l], acc);
    __syncthreads();
  }
  if (i < m && j < n && (!lower || i >= j)) {
    double* c = C + i + static_cast<long>(j) * ldc;
    *c = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *c);
  }
}

// inv (nb x nb, ld nb) <- L^-1 for the lower triangular L at A[d0.., d0..]
// (unit diagonal if `unit`; nb <= 512, one thread per row: launch with
// trtri_threads(nb) threads): each block solves L x = e_j for the two
// columns j and nb - 1 - j (balanced work) by column substitution.  Thread i
// owns row i of both x's in registers and reads row i of L sixteen columns
// ahead (coalesced along the column); x_k is published through shared
// memory, one barrier per step.
__global__ void __launch_bounds__(512) trtri_cols_kernel(const double* A, long lda, int d0, int nb, int unit,
                                                        double* inv, const int32_t* info) {
  __shared__ double bc[2][2];
  if (info && *info != 0) return;
  const double* L = A + d0 + static_cast<long>(d0) * lda;
  const int i = threadIdx.x;
  const int j0 = blockIdx.x, j1 = nb - 1 - static_cast<int>(blockIdx.x);
  double x0 = (i == j0) ? 1.0 : 0.0, x1 = (i == j1) ? 1.0 : 0.0;
  // every row's reciprocal at once: the steps below then multiply (a division
  // on each step's dependent path would cost its full FP64 latency 256 times)
  const double rinv = (!unit && i < nb) ? 1.0 / L[i + static_cast<long>(i) * lda] : 1.0;
  double ln[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int kk = j0 + q;
    ln[q] = (i < nb && kk < nb && i >= kk + unit) ? L[i + static_cast<long>(kk) * lda] : 0.0;
  }
  for (int g = j0; g < nb; g += 16) {
    double lv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) lv[q] = ln[q];
    if (g + 16 < nb) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int kk = g + 16 + q;
        ln[q] = (i < nb && kk < nb && i >= kk + unit) ? L[i + static_cast<long>(kk) * lda] : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int kk = g + q;
      if (kk >= nb) break;
      if (i == kk) {
        if (!unit) {
          x0 *= rinv;
          x1 *= rinv;
        }
        bc[kk & 1][0] = x0;
        bc[kk & 1][1] = x1;
      }
      __syncthreads();
      const double b0 = bc[kk & 1][0], b1 = bc[kk & 1][1];
      if (i > kk && i < nb) {
        x0 = fma(-lv[q], b0, x0);
        x1 = fma(-lv[q], b1, x1);
      }
    }
  }
  if (i < nb) {
    inv[i + static_cast<long>(j0) * nb] = x0;
    inv[i + static_cast<long>(j1) * nb] = x1;
  }
}

// One diagonal block of a triangular solve, x <- op(T)^-1 x for the bs x bs
// block at T[d0.., d0..] (bs <= 128; op = transpose with `trans`).  All
// threads stage the block (leading dimension bs + 1: conflict-free either
// way), then warp 0 solves with x in registers (lane l holds rows l, l+32,
// l+64, l+96), each x_k divided by its diagonal entry (non-unit) and broadcast
// by shuffle.  blockIdx.x = right-hand side.
__global__ void __launch_bounds__(1024) trsv_block_kernel(const double* T, long ldt, double* X, long ldx, int d0,
                                                          int bs, int lower, int unit, int trans) {
  extern __shared__ double tb[];   // tb[r + c*(bs+1)] = T(d0+r, d0+c) as stored
  const int ld = bs + 1;
  double* xc = X + static_cast<long>(blockIdx.x) * ldx + d0;
  {
    const int r = threadIdx.x & 127, cstep = blockDim.x >> 7;
    if (r < bs)
      for (int c0 = threadIdx.x >> 7; c0 < bs; c0 += 16 * cstep) {
        double v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j * cstep;
          v[j] = c < bs ? T[(d0 + r) + static_cast<long>(d0 + c) * ldt] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j * cstep < bs) tb[r + (c0 + j * cstep) * ld] = v[j];
      }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  auto t = [&](int r, int c) -> double { return trans ? tb[c + r * ld] : tb[r + c * ld]; };
  double x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = lane + 32 * q < bs ? xc[lane + 32 * q] : 0.0;
  if (lower) {
#pragma unroll
    for (int q0 = 0; q0 < 4; ++q0)
      for (int kk = 0; kk < 32; ++kk) {
        const int k = 32 * q0 + kk;
        if (k >= bs) break;
        if (!unit && lane == kk) x[q0] = x[q0] / t(k, k);
        const double xk = __shfl_sync(0xFFFFFFFFu, x[q0], kk);
#pragma unroll
        for (int q = q0; q < 4; ++q) {
          const int i = lane + 32 * q;
          if (i > k && i < bs) x[q] = fma(-t(i, k), xk, x[q]);
        }
      }
  } else {
#pragma unroll
    for (int q0 = 3; q0 >= 0; --q0)
      for (int kk = 31; kk >= 0; --kk) {
        const int k = 32 * q0 + kk;
        if (k >= bs) continue;
        if (!unit && lane == kk) x[q0] = x[q0] / t(k, k);
        const double xk = __shfl_sync(0xFFFFFFFFu, x[q0], kk);
#pragma unroll
        for (int q = 0; q <= q0; ++q) {
          const int i = lane + 32 * q;
          if (i < k) x[q] = fma(-t(i, k), xk, x[q]);
        }
      }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (lane + 32 * q < bs) xc[lane + 32 * q] = x[q];
}

// x[r] -= sum_{c in [c0, c0+bs)} T(r, c) x[c] for rows r in [r0, r1); T(r, c) =
// T[r + c*ldt] or, with `trans`, T[c + r*ldt].  blockIdx.y = right-hand side.
__global__ void gemv_update_kernel(const double* T, long ldt, double* X, long ldx, int r0, int r1, int c0, int bs,
                                   int trans) {
  __shared__ double xs[128];
  double* xc = X + static_cast<long>(blockIdx.y) * ldx;
  if (threadIdx.x < bs) xs[threadIdx.x] = xc[c0 + threadIdx.x];
  __syncthreads();
  if (!trans) {
    const int r = r0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    double acc = 0.0;
    for (int c = 0; c < bs; ++c) acc = fma(T[r + static_cast<long>(c0 + c) * ldt], xs[c], acc);
    xc[r] -= acc;
  } else {
    // one warp per row: contiguous reads of T[c0.., r]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = r0 + blockIdx.x * (blockDim.x / 32) + warp;
    if (r >= r1) return;
    double acc = 0.0;
    for (int c = lane; c < bs; c += 32) acc = fma(T[(c0 + c) + static_cast<long>(r) * ldt], xs[c], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) xc[r] -= acc;
  }
}

// Residual pass of Eq. 8: per row, r_i = sum_j a_ij x_j - b_i and sum_j |a_ij|;
// maxima of |r_i| and of the row sums collected with atomicMax on the bits.
__global__ void residual_kernel(int n, const double* A, long lda, const double* x, const double* b,
                                unsigned long long* acc) {
  extern __shared__ double xs[];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0, sa = 0.0;
  for (int c0 = 0; c0 < n; c0 += 2048) {
    const int cn = n - c0 < 2048 ? n - c0 : 2048;
    __syncthreads();
    for (int i = threadIdx.x; i < cn; i += blockDim.x) xs[i] = x[c0 + i];
    __syncthreads();
    if (r < n)
      for (int c = 0; c < cn; ++c) {
        const double a = A[r + static_cast<long>(c0 + c) * lda];
        s = fma(a, xs[c], s);
        sa += fabs(a);
      }
  }
  if (r < n) {
    const double res = fabs(s - b[r]);
    atomicMax(&acc[0], static_cast<unsigned long long>(__double_as_longlong(res)));
    atomicMax(&acc[1], static_cast<unsigned long long>(__double_as_longlong(sa)));
    atomicMax(&acc[2], static_cast<unsigned long long>(__double_as_longlong(fabs(x[r]))));
    atomicMax(&acc[3], static_cast<unsigned long long>(__double_as_longlong(fabs(b[r]))));
  }
}

__global__ void residual_finish_kernel(int n, const unsigned long long* acc, double* out) {
  const double r = __longlong_as_double(static_cast<long long>(acc[0]));
  const double an = __longlong_as_double(static_cast<long long>(acc[1]));
  const double xn = __longlong_as_double(static_cast<long long>(acc[2]));
  const double bn = __longlong_as_double(static_cast<long long>(acc[3]));
  const double eps = 1.1102230246251565e-16;   // 2^-53
  out[0] = r / ((an * xn + bn) * n * eps);
  out[1] = r / (an * xn * n * eps);
}

// ------------------------------------------------------------------ a-posteriori probe
// Freivalds-style check of one trailing update C <- C - L U on sampled rows:
// with w_j = +-1, (C_old - C_new) w must equal L (U w) up to the emulation
// tolerance 4 k u (|L||U|)|w| plus FP64 rounding of the three products.
constexpr int kProbeRows = 64;

__device__ __forceinline__ double probe_w(int j) {
  unsigned x = static_cast<unsigned>(j) * 2654435761u;
  x ^= x >> 13;
  x *= 0x5bd1e995u;
  x ^= x >> 15;
  return (x & 1u) ? 1.0 : -1.0;
}

__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double ra[32], rb[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0.0;
    b = 0.0;
    for (int i = 0; i < static_cast<int>(blockDim.x / 32); ++i) {
      a += ra[i];
      b += rb[i];
    }
  }
}

// y[i] = sum_j C(r_i, j) w_j, a[i] = sum_j |C(r_i, j)|, r_i = i*m/R (one block per sampled row)
__global__ void probe_rows_kernel(int m, int n, const double* C, long ldc, int R, double* y, double* a) {
  const int i = blockIdx.x;
  const int r = static_cast<int>(static_cast<long>(i) * m / R);
  double sy = 0.0, sa = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double c = C[r + static_cast<long>(j) * ldc];
    sy = fma(c, probe_w(j), sy);
    sa += fabs(c);
  }
  block_sum2(sy, sa);
  if (threadIdx.x == 0) {
    y[i] = sy;
    a[i] = sa;
  }
}

// z[q] = sum_j U(q, j) w_j, za[q] = sum_j |U(q, j)| (one block per row q of U, jb x n)
__global__ void probe_z_kernel(int n, const double* U, long ldu, double* z, double* za) {
  const int q = blockIdx.x;
  double sz = 0.0, sa = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double u = U[q + static_cast<long>(j) * ldu];
    sz = fma(u, probe_w(j), sz);
    sa += fabs(u);
  }
  block_sum2(sz, sa);
  if (threadIdx.x == 0) {
    z[q] = sz;
    za[q] = sa;
  }
}

// t[i] = sum_q L(r_i, q) z[q], ta[i] = sum_q |L(r_i, q)| za[q]; then the check (one thread per row)
__global__ void probe_check_kernel(int m, int n, int k, const double* L, long ldl, int R, const double* z,
                                   const double* za, const double* y0, const double* a0, const double* y1,
                                   const double* a1, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R) return;
  const int r = static_cast<int>(static_cast<long>(i) * m / R);
  double t = 0.0, ta = 0.0;
  for (int q = 0; q < k; ++q) {
    const double l = L[r + static_cast<long>(q) * ldl];
    t = fma(l, z[q], t);
    ta = fma(fabs(l), za[q], ta);
  }
  const double u = 1.1102230246251565e-16;
  const double tol = 6.0 * k * u * ta + 3.0 * n * u * (a0[i] + a1[i]);
  const double diff = fabs((y0[i] - y1[i]) - t);
  if (!(diff <= tol)) atomicExch(flag, 1);
}

// ------------------------------------------------------------------ host helpers
struct LuBufs {
  double* inv;          // nb x nb
  uint64_t* recs;       // leaf pivot exchange: [2][nsm][kRecWords] epoch-tagged words
  uint64_t* drec;       // [2][2 kLeaf]: row c of the leaf, epoch-tagged words
  unsigned long long* racc;
  int* map;             // laswp gather maps, [4*kPermMax + 1] ints each, one per recursion depth
  double* probe;        // y0, a0, y1, a1 (kProbeRows each), z, za (nb each)
  int* flag;
};
constexpr int kMapInts = 4 * kPermMax + 8;
constexpr int kMaxDepth = 8;

size_t rec_bytes(int nsm) { return 2ull * nsm * kRecWords * 8; }

size_t lu_extra_bytes(int nb, int nsm) {
  return al(static_cast<size_t>(nb) * nb * 8) + al(rec_bytes(nsm)) + al(2ull * 2 * kLeaf * 8) + al(4 * 8) +
         al(kMaxDepth * kMapInts * 4) +
         al((4ull * kProbeRows + 2ull * nb) * 8) + al(16) + kAl;
}

// Lower Cholesky of the jb x jb diagonal block at A[d0.., d0..] (jb <= 512),
// in place, by 32-column panels (chol_leaf_kernel, then the rows below the
// leaf within the block and the block's trailing lower part by
// dgemm_nt_small_kernel); with `want_inv`, inv (jb x jb, ld jb) <- L11^-1.
int chol_diag(emul_handle_t h, double* A, long lda, int d0, int jb, double* inv, int32_t* info, bool want_inv) {
  for (int c0 = 0; c0 < jb; c0 += kCholLeaf) {
    const int wp = kCholLeaf < jb - c0 ? kCholLeaf : jb - c0;
    chol_leaf_kernel<<<1, 128, 0, h->stream>>>(A, lda, d0 + c0, wp, inv + c0 + static_cast<long>(c0) * jb, jb,
                                                info);
    h->launches++;
    const int r0 = c0 + wp, mr = jb - r0;
    if (mr > 0) {
      double* Lp = A + (d0 + r0) + static_cast<long>(d0 + c0) * lda;   // rows below the leaf, its columns
      const double* ip = inv + c0 + static_cast<long>(c0) * jb;       // the leaf's inverse
      // L(r0.., c0..) = A(r0.., c0..) L_pp^-T, in place (n = k = wp <= 32)
      dgemm_nt_small_kernel<<<dim3((mr + 15) / 16, 1), 512, 0, h->stream>>>(mr, wp, wp, 1.0, Lp, 1, lda, ip, 1, jb,
                                                                          0.0, Lp, lda, 0, info);
      // A(r0.., r0..) -= L(r0.., c0..) L(r0.., c0..)^T, lower part
      dgemm_nt_small_kernel<<<dim3((mr + 15) / 16, (mr + 31) / 32), 512, 0, h->stream>>>(
          mr, mr, wp, -1.0, Lp, 1, lda, Lp, 1, lda, 1.0, A + (d0 + r0) + static_cast<long>(d0 + r0) * lda, lda, 1,
          info);
      h->launches += 2;
    }
  }
  if (want_inv) {
    trtri_cols_kernel<<<(jb + 1) / 2, trtri_threads(jb), 0, h->stream>>>(A, lda, d0, jb, 0, inv, info);
    h->launches++;
  }
  return check_cuda(h, cudaGetLastError(), "Cholesky diagonal block");
}

LuBufs carve(emul_handle_t h, size_t off, int nb) {
  uint8_t* p = static_cast<uint8_t*>(h->ws) + al(off);
  LuBufs b;
  b.inv = reinterpret_cast<double*>(p);
  p += al(static_cast<size_t>(nb) * nb * 8);
  b.recs = reinterpret_cast<uint64_t*>(p);
  p += al(rec_bytes(h->nsm));
  b.drec = reinterpret_cast<uint64_t*>(p);
  p += al(2ull * 2 * kLeaf * 8);
  b.racc = reinterpret_cast<unsigned long long*>(p);
  p += al(4 * 8);
  b.map = reinterpret_cast<int*>(p);
  p += al(kMaxDepth * kMapInts * 4);
  b.probe = reinterpret_cast<double*>(p);
  p += al((4ull * kProbeRows + 2ull * nb) * 8);
  b.flag = reinterpret_cast<int*>(p);
  return b;
}

int launch_leaf(emul_handle_t h, double* A, long lda, int n, int d0, int w, int pc0, int pc1, int32_t* ipiv,
                int32_t* info, const LuBufs& B) {
  const int mp = n - d0;
  int G = (mp + 127) / 128;   // 128 rows per block: the per-column FP64 work of a block overlaps the exchange
  const int smem_rows_cap = 200 * 1024 / (w * 8);
  if ((mp + G - 1) / G > smem_rows_cap) G = (mp + smem_rows_cap - 1) / smem_rows_cap;
  if (G < 1) G = 1;
  if (G > h->nsm) G = h->nsm;
  if (G > 32 * kMaxRecPerLane) G = 32 * kMaxRecPerLane;
  const int R = (mp + G - 1) / G;
  const size_t smem = static_cast<size_t>(R) * w * 8;
  if (smem > 220 * 1024) return set_error(h, EMUL_NOT_SUPPORTED, "panel too tall for the leaf kernel");
  smem_attr(reinterpret_cast<const void*>(getf2_leaf_kernel), 220 * 1024);
  long long limit = h->wait_limit;
  int* status = h->d_status;
  // epochs of this launch: (salt << 5) | column, salt > 0 and new per launch
  // (the records are cleared and the salt restarted by every factorization)
  uint32_t salt = ++h->leaf_salt;
  if (salt >= (1u << 27)) return set_error(h, EMUL_NOT_SUPPORTED, "too many panel leaves in one factorization");
  void* args[] = {&A, const_cast<long*>(&lda), &n, &d0, &w, const_cast<int*>(&R), &pc0, &pc1, &ipiv, &info,
                  const_cast<uint64_t**>(&B.recs), const_cast<uint64_t**>(&B.drec), &salt, &status, &limit};
  h->launches++;
  return check_cuda(h,
                    cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(getf2_leaf_kernel), dim3(G),
                                                dim3(kLeafThreads), args, smem, h->stream),
                    "panel leaf");
}

// Resolve the interchanges ipiv[k1..k2) into the gather map (once per block).
int laswp_prepare(emul_handle_t h, const int32_t* ipiv, int k1, int k2, int* map) {
  if (k2 <= k1) return EMUL_OK;
  if (k2 - k1 > kPermMax) return set_error(h, EMUL_INVALID_ARG, "too many interchanges in one block");
  laswp_perm_kernel<<<1, kPermMax, 0, h->stream>>>(ipiv, k1, k2, map);
  h->launches++;
  return check_cuda(h, cudaGetLastError(), "laswp map");
}

// Apply a prepared gather map to columns [c0, c1).
int laswp_apply(emul_handle_t h, double* A, long lda, int c0, int c1, const int* map) {
  if (c1 <= c0) return EMUL_OK;
  laswp_apply_kernel<<<(c1 - c0 + kSwpCols - 1) / kSwpCols, 256, 0, h->stream>>>(A, lda, c0, c1, map);
  h->launches++;
  return check_cuda(h, cudaGetLastError(), "laswp");
}

// The interchanges ipiv[k1..k2) applied in order to columns [c0, c1), at
// most kPermMax per gather map.
int laswp(emul_handle_t h, double* A, long lda, int c0, int c1, const int32_t* ipiv, int k1, int k2, int* map) {
  if (c1 <= c0 || k2 <= k1) return EMUL_OK;
  for (int k = k1; k < k2; k += kPermMax) {
    int rc = laswp_prepare(h, ipiv, k, k + kPermMax < k2 ? k + kPermMax : k2, map);
    if (rc) return rc;
    rc = laswp_apply(h, A, lda, c0, c1, map);
    if (rc) return rc;
  }
  return EMUL_OK;
}

int trsm_small(emul_handle_t h, double* A, long lda, int d0, int w1, int c0, int w2) {
  if (w1 <= 0 || w2 <= 0) return EMUL_OK;
  if (w1 > kTrsmMax) return set_error(h, EMUL_NOT_SUPPORTED, "panel trsm wider than 128");
  smem_attr(reinterpret_cast<const void*>(trsm_small_kernel), kTrsmMax * kTrsmMax * 8);
  // one column per block: the solve is FP64-bound (about 1.6 FMA per clock per
  // SM), so it is spread over as many SMs as columns; 256 threads stage L
  trsm_small_kernel<<<w2, 256, static_cast<size_t>(w1) * w1 * 8, h->stream>>>(A, lda, d0, w1, c0, w2, 1);
  h->launches++;
  return check_cuda(h, cudaGetLastError(), "panel trsm");
}

// Recursive panel factorization of rows d0..n-1, columns d0..d0+w-1, inside
// the panel [pc0, pc1).  The leaves apply each interchange to all columns of
// that panel, so the recursion itself swaps nothing.
int rgetrf(emul_handle_t h, double* A, long lda, int n, int d0, int w, int pc0, int pc1, int32_t* ipiv,
           int32_t* info, int s, const LuBufs& B) {
  if (w <= kLeaf) return launch_leaf(h, A, lda, n, d0, w, pc0, pc1, ipiv, info, B);
  const int w1 = (w / 2 + 7) / 8 * 8;
  const int w2 = w - w1;
  int rc = rgetrf(h, A, lda, n, d0, w1, pc0, pc1, ipiv, info, s, B);
  if (rc) return rc;
  rc = trsm_small(h, A, lda, d0, w1, d0 + w1, w2);
  if (rc) return rc;
  const int m2 = n - d0 - w1;
  // A22 (m2 x w2) -= A21 (m2 x w1) * A12 (w1 x w2)
  rc = gemm_run(h, m2, w2, w1, -1.0, Operand{A + (d0 + w1) + static_cast<long>(d0) * lda, 1, lda},
                Operand{A + d0 + static_cast<long>(d0 + w1) * lda, lda, 1}, 1.0,
                A + (d0 + w1) + static_cast<long>(d0 + w1) * lda, lda, s, false, 0, nullptr, 0, 0);
  if (rc) return rc;
  return rgetrf(h, A, lda, n, d0 + w1, w2, pc0, pc1, ipiv, info, s, B);
}

// Panel of width jb at column j0.  Up to kPanelMax columns it is one recursive
// panel, whose leaves apply each interchange across it.  A wider panel is
// factored as two such panels: the left one's interchanges are applied to the
// right one, which is updated (U12 = L11^-1 A12 through the explicit inverse
// and the emulated product, A22 -= L21 U12) and factored; its interchanges
// then go back to the left one.  B.inv is free during the panel.
constexpr int kPanelMax = 256;
int panel_getrf(emul_handle_t h, double* A, long lda, int n, int j0, int jb, int32_t* ipiv, int32_t* info, int s,
                const LuBufs& B) {
  if (jb <= kPanelMax) return rgetrf(h, A, lda, n, j0, jb, j0, j0 + jb, ipiv, info, s, B);
  const int w1 = kPanelMax, w2 = jb - w1;
  int rc = rgetrf(h, A, lda, n, j0, w1, j0, j0 + w1, ipiv, info, s, B);
  if (rc) return rc;
  rc = laswp(h, A, lda, j0 + w1, j0 + jb, ipiv, j0, j0 + w1, B.map);
  if (rc) return rc;
  trtri_cols_kernel<<<(w1 + 1) / 2, trtri_threads(w1), 0, h->stream>>>(A, lda, j0, w1, 1, B.inv, nullptr);
  h->launches++;
  rc = check_cuda(h, cudaGetLastError(), "panel trtri");
  if (rc) return rc;
  double* A12 = A + j0 + static_cast<long>(j0 + w1) * lda;
  rc = gemm_run(h, w1, w2, w1, 1.0, Operand{B.inv, 1, w1}, Operand{A12, lda, 1}, 0.0, A12, lda, s, false, 0,
                nullptr, 0, 0);
  if (rc) return rc;
  const int m2 = n - j0 - w1;
  rc = gemm_run(h, m2, w2, w1, -1.0, Operand{A + (j0 + w1) + static_cast<long>(j0) * lda, 1, lda},
                Operand{A12, lda, 1}, 1.0, A + (j0 + w1) + static_cast<long>(j0 + w1) * lda, lda, s, false, 0,
                nullptr, 0, 0);
  if (rc) return rc;
  rc = rgetrf(h, A, lda, n, j0 + w1, w2, j0 + w1, j0 + jb, ipiv, info, s, B);
  if (rc) return rc;
  return laswp(h, A, lda, j0, j0 + w1, ipiv, j0 + w1, j0 + jb, B.map);
}

}  // namespace

void trsv_attr() { smem_attr(reinterpret_cast<const void*>(trsv_block_kernel), 128 * 129 * 8); }

}  // namespace emul

namespace emul {

namespace {

constexpr int kSolveBs = 128;      // diagonal block of the persistent solve
constexpr int kPermSmemMax = 54 * 1024;   // rows whose permutation fits in shared memory (4 B each, + 4 KB)

// x <- P x for the interchanges ipiv[0..n) (1-based, applied in order): the
// composite permutation is built by one thread in shared memory (ipiv staged in
// chunks), then x is gathered through tmp.  One block.
__global__ void __launch_bounds__(1024) permute_rhs_kernel(const int32_t* ipiv, int n, double* x, double* tmp) {
  extern __shared__ int perm[];
  __shared__ int chunk[1024];
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += 1024) {
    const int m = n - k0 < 1024 ? n - k0 : 1024;
    if (static_cast<int>(threadIdx.x) < m) chunk[threadIdx.x] = ipiv[k0 + threadIdx.x] - 1;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int j = 0; j < m; ++j) {
        const int k = k0 + j, p = chunk[j];
        if (p != k && p >= 0 && p < n) {
          const int t = perm[k];
          perm[k] = perm[p];
          perm[p] = t;
        }
      }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) tmp[i] = x[perm[i]];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = tmp[i];
}

// Bounded grid barrier on a monotonic arrival counter (zeroed before the
// launch); returns false on timeout after recording it in *status.
__device__ bool solve_sync(unsigned long long* cnt, unsigned long long target, long long limit, int* status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    bool ok = true;
    if (atomicAdd(cnt, 1ull) + 1 < target) {
      volatile unsigned long long* vc = cnt;
      const long long t0 = clock64();
      while (*vc < target)
        if (clock64() - t0 > limit) {
          ok = false;
          atomicExch(status, kStatusTimeout);
          break;
        }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Forward (L unit lower) and back (U) substitution with the factors of
// emul_dgetrf for one right-hand side, in one cooperative launch.  Step s
// (the 128-row diagonal blocks of L, then those of U from the bottom) is
// solved by block s % G in one warp (x in registers, broadcast by shuffle,
// multiplication by the reciprocals of U's diagonal, formed while staging);
// block (s+1) % G stages the next diagonal block meanwhile.  Then every warp of
// every block applies the block's column of L (or U) to 32-row groups of the
// remaining rows.  Two bounded grid barriers per step.  A row's owner changes
// from step to step, so x is read and written through L2 only.
// Stage the bs x bs diagonal block at d0 for the block solve.  LU factors
// (chol = false): the block as stored, rcp = 1/diag for the upper (backward)
// solve.  Cholesky factor (chol = true): the forward solve uses L itself and
// the backward solve L^T, so the block is staged transposed there; rcp = 1/diag
// for both.
__device__ void solve_stage(const double* LU, long lda, int d0, int bs, bool lower, double* tb, double* rcp,
                            bool chol) {
  constexpr int ld = kSolveBs + 1;
  const int tid = threadIdx.x;
  const int r = tid & 127, cstep = blockDim.x >> 7;
  const bool tr = chol && !lower;
  if (r < bs)
    for (int c0 = tid >> 7; c0 < bs; c0 += 16 * cstep) {
      double v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = c0 + j * cstep;
        v[j] = c < bs ? __ldg(LU + (d0 + r) + static_cast<long>(d0 + c) * lda) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = c0 + j * cstep;
        if (c < bs) tb[tr ? c + r * ld : r + c * ld] = v[j];
      }
    }
  __syncthreads();
  if ((chol || !lower) && tid < bs) rcp[tid] = 1.0 / tb[tid + tid * ld];
  __syncthreads();
}

// CHOL = false: A = L U from the LU (unit L below the diagonal, U on and
// above it).  CHOL = true: A = L L^T from the lower Cholesky factor, forward
// with L (non-unit diagonal) and backward with L^T, whose rows are columns of
// L: the update of the rows above a block then reads each column of L
// contiguously, one warp per row of L^T.
template <bool CHOL>
__global__ void __launch_bounds__(256) getrs1_kernel(const double* LU, long lda, int n, double* x,
                                                     unsigned long long* cnt, int* status, long long limit) {
  extern __shared__ double tb[];   // kSolveBs x (kSolveBs + 1) staging of a diagonal block
  __shared__ double xs[kSolveBs];
  __shared__ double rcp[kSolveBs];
  constexpr int ld = kSolveBs + 1;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + kSolveBs - 1) / kSolveBs;
  const int nsteps = 2 * nblk;
  auto info = [&](int st, bool& lower, int& d0, int& bs) {
    lower = st < nblk;
    const int d = lower ? st : 2 * nblk - 1 - st;
    d0 = d * kSolveBs;
    bs = n - d0 < kSolveBs ? n - d0 : kSolveBs;
  };
  unsigned long long target = 0;
  int staged = -1;   // step whose diagonal block this block holds in tb
  for (int st = 0; st < nsteps; ++st) {
    bool lower;
    int d0, bs;
    info(st, lower, d0, bs);
    const int sb = st % G, nxt = (st + 1) % G;
    if (b == sb) {
      if (staged != st) solve_stage(LU, lda, d0, bs, lower, tb, rcp, CHOL);
      staged = -1;
      if (tid < 32) {
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = lane + 32 * q < bs ? __ldcg(x + d0 + lane + 32 * q) : 0.0;
        if (lower) {
#pragma unroll
          for (int q0 = 0; q0 < 4; ++q0)
            for (int kk = 0; kk < 32; ++kk) {
              const int k = 32 * q0 + kk;
              if (k >= bs) break;
              if (CHOL && lane == kk) v[q0] = v[q0] * rcp[k];
              const double xk = __shfl_sync(0xFFFFFFFFu, v[q0], kk);
#pragma unroll
              for (int q = q0; q < 4; ++q) {
                const int i = lane + 32 * q;
                if (i > k && i < bs) v[q] = fma(-tb[i + k * ld], xk, v[q]);
              }
            }
        } else {
#pragma unroll
          for (int q0 = 3; q0 >= 0; --q0)
            for (int kk = 31; kk >= 0; --kk) {
              const int k = 32 * q0 + kk;
              if (k >= bs) continue;
              if (lane == kk) v[q0] = v[q0] * rcp[k];
              const double xk = __shfl_sync(0xFFFFFFFFu, v[q0], kk);
#pragma unroll
              for (int q = 0; q <= q0; ++q) {
                const int i = lane + 32 * q;
                if (i < k) v[q] = fma(-tb[i + k * ld], xk, v[q]);
              }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (lane + 32 * q < bs) __stcg(x + d0 + lane + 32 * q, v[q]);
      }
    } else if (b == nxt && st + 1 < nsteps) {
      // the next step's solver stages its diagonal block while this one is solved
      bool l2;
      int e0, es;
      info(st + 1, l2, e0, es);
      solve_stage(LU, lda, e0, es, l2, tb, rcp, CHOL);
      staged = st + 1;
    }
    target += G;
    if (!solve_sync(cnt, target, limit, status)) return;
    // rows below (forward) or above (backward) the block, 32-row groups over all warps
    const int r_lo = lower ? d0 + bs : 0, r_hi = lower ? n : d0;
    if (CHOL && !lower && r_hi > r_lo) {
      // x_r -= sum_c L(d0 + c, r) x_c: one warp per row r, lanes along the column
      for (int c = tid; c < bs; c += blockDim.x) xs[c] = __ldcg(x + d0 + c);
      __syncthreads();
      const int wpb = blockDim.x >> 5;
      for (int r = r_lo + b * wpb + warp; r < r_hi; r += G * wpb) {
        const double* col = LU + d0 + static_cast<long>(r) * lda;
        double acc = 0.0;
        for (int c = lane; c < bs; c += 32) acc = fma(__ldg(col + c), xs[c], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) __stcg(x + r, __ldcg(x + r) - acc);
      }
    } else if (r_hi > r_lo) {
      for (int c = tid; c < bs; c += blockDim.x) xs[c] = __ldcg(x + d0 + c);
      __syncthreads();
      const int wpb = blockDim.x >> 5;
      for (int rg = b * wpb + warp; r_lo + rg * 32 < r_hi; rg += G * wpb) {
        const int r = r_lo + rg * 32 + lane;
        if (r < r_hi) {
          double acc = 0.0;
          for (int c = 0; c < bs; ++c) acc = fma(__ldg(LU + r + static_cast<long>(d0 + c) * lda), xs[c], acc);
          __stcg(x + r, __ldcg(x + r) - acc);
        }
      }
    }
    target += G;
    if (!solve_sync(cnt, target, limit, status)) return;
  }
}

}  // namespace

// Solve with the factors of emul_dgetrf (arguments validated by the caller).
int getrs_body(emul_handle_t h, int n, int nrhs, const double* LU, int lda, const int32_t* ipiv, double* B,
               int ldb) {
  if (nrhs == 1 && n <= kPermSmemMax) {
    // one right-hand side: permutation in one block, both substitutions in one cooperative launch
    int rc = reserve_workspace(h, 2 * kAl + al(static_cast<size_t>(n) * 8));
    if (rc) return rc;
    uint8_t* ws = static_cast<uint8_t*>(h->ws);
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(ws);
    double* tmp = reinterpret_cast<double*>(ws + kAl);
    smem_attr(reinterpret_cast<const void*>(permute_rhs_kernel), kPermSmemMax * 4);
    smem_attr(reinterpret_cast<const void*>(getrs1_kernel<false>), kSolveBs * (kSolveBs + 1) * 8);
    permute_rhs_kernel<<<1, 1024, static_cast<size_t>(n) * 4, h->stream>>>(ipiv, n, B, tmp);
    h->launches++;
    rc = check_cuda(h, cudaGetLastError(), "rhs permutation");
    if (rc) return rc;
    rc = check_cuda(h, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), h->stream), "solve barrier");
    if (rc) return rc;
    long ldl = lda;
    long long limit = h->wait_limit;
    int* status = h->d_status;
    void* args[] = {const_cast<double**>(&LU), &ldl, &n, &B, &cnt, &status, &limit};
    h->launches++;
    return check_cuda(h,
                      cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(getrs1_kernel<false>), dim3(h->nsm),
                                                  dim3(256), args, kSolveBs * (kSolveBs + 1) * 8, h->stream),
                      "solve");
  }
  const size_t need = lu_extra_bytes(16, h->nsm);
  int rc = reserve_workspace(h, need);
  if (rc) return rc;
  const LuBufs W = carve(h, 0, 16);
  for (int k = 0; k < n; k += kPermMax) {
    rc = laswp(h, B, ldb, 0, nrhs, ipiv, k, k + kPermMax < n ? k + kPermMax : n, W.map);
    if (rc) return rc;
  }
  constexpr int bs = 128;  // diagonal blocks of the substitution
  for (int d0 = 0; d0 < n; d0 += bs) {
    const int b = bs < n - d0 ? bs : n - d0;
    trsv_block_kernel<<<nrhs, 1024, b * (b + 1) * sizeof(double), h->stream>>>(LU, lda, B, ldb, d0, b, 1, 1, 0);
    h->launches += (d0 + b < n) ? 2 : 1;
    if (d0 + b < n)
      gemv_update_kernel<<<dim3((n - d0 - b + 255) / 256, nrhs), 256, 0, h->stream>>>(LU, lda, B, ldb, d0 + b,
                                                                                               n, d0, b, 0);
  }
  for (int d0 = ((n - 1) / bs) * bs; d0 >= 0; d0 -= bs) {
    const int b = bs < n - d0 ? bs : n - d0;
    trsv_block_kernel<<<nrhs, 1024, b * (b + 1) * sizeof(double), h->stream>>>(LU, lda, B, ldb, d0, b, 0, 0, 0);
    h->launches += (d0 > 0) ? 2 : 1;
    if (d0 > 0)
      gemv_update_kernel<<<dim3((d0 + 255) / 256, nrhs), 256, 0, h->stream>>>(LU, lda, B, ldb, 0, d0, d0, b, 0);
  }
  return check_cuda(h, cudaGetLastError(), "getrs");
}
}  // namespace emul

using emul::Operand;

namespace emul {
namespace {

// Seeded synthetic matrix for the block-size tuner: uniform(-1, 1) from a
// splitmix64 hash of (seed, i, j); with `spd`, entry (i, j) takes the hash of
// (max, min) so the matrix is symmetric, and the diagonal is n (strictly
// diagonally dominant, hence positive definite).
__global__ void tune_fill_kernel(double* A, int n, int spd, unsigned long long seed) {
  const long total = static_cast<long>(n) * n;
  for (long e = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long>(gridDim.x) * blockDim.x) {
    int i = static_cast<int>(e % n), j = static_cast<int>(e / n);
    if (spd && i == j) {
      A[e] = static_cast<double>(n);
      continue;
    }
    if (spd && i < j) {
      const int t = i;
      i = j;
      j = t;
    }
    unsigned long long z = seed + (static_cast<unsigned long long>(i) * n + j + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    A[e] = static_cast<double>(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

uint64_t nb_key(int kind, int n, int slices) {
  return (static_cast<uint64_t>(kind) << 40) | (static_cast<uint64_t>(slices) << 32) | static_cast<uint32_t>(n);
}

// The LU step's second stream and its two events, created on first use.
int aux_ready(emul_handle_t h) {
  if (h->aux) return EMUL_OK;
  int rc = check_cuda(h, cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking), "second stream");
  if (!rc) rc = check_cuda(h, cudaEventCreateWithFlags(&h->aux_start, cudaEventDisableTiming), "stream events");
  if (!rc) rc = check_cuda(h, cudaEventCreateWithFlags(&h->aux_done, cudaEventDisableTiming), "stream events");
  return rc;
}

// nb = EMUL_NB_AUTO: the tuned block size for (kind, n, slices), tuning first
// when there is none.
int resolve_nb(emul_handle_t h, int kind, int n, int slices, int* nb) {
  if (*nb != EMUL_NB_AUTO) return EMUL_OK;
  const auto it = h->nb_tuned.find(nb_key(kind, n, slices));
  if (it != h->nb_tuned.end()) {
    *nb = it->second;
    return EMUL_OK;
  }
  return emul_autotune_nb(h, kind, n, slices, nb);
}

}  // namespace
}  // namespace emul

extern "C" {

int emul_autotune_nb(emul_handle_t h, int kind, int n, int slices, int* nb_out) {
  if (!h) return EMUL_INVALID_ARG;
  if ((kind != 0 && kind != 1) || n < 1 || slices < 1 || slices > emul::kMaxSlices || !nb_out)
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_autotune_nb: invalid argument");
  const int cand[] = {128, 256, 512};
  double* A = nullptr;
  int32_t* piv = nullptr;
  if (cudaMalloc(&A, static_cast<size_t>(n) * n * 8 + static_cast<size_t>(n) * 4 + 256) != cudaSuccess) {
    cudaGetLastError();
    return emul::set_error(h, EMUL_NO_WORKSPACE, "emul_autotune_nb: no room for the trial matrix");
  }
  piv = reinterpret_cast<int32_t*>(A + static_cast<size_t>(n) * n);
  int32_t* info = piv + n;
  const bool prof = h->prof;
  h->prof = false;   // the trials are not part of any profile
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = emul::check_cuda(h, cudaEventCreate(&e0), "tuner events");
  if (!rc) rc = emul::check_cuda(h, cudaEventCreate(&e1), "tuner events");
  // candidates past the first that covers n in one panel change nothing
  int nc = 1;
  while (nc < 3 && cand[nc - 1] < n) ++nc;
  int best = cand[0];
  float best_ms = 0.0f;
  // the untimed first run takes the largest candidate: it sizes the workspace
  // and plans the product schedules the others reuse
  for (int c = -1; c < nc && !rc; ++c) {
    const int nb = cand[c < 0 ? nc - 1 : c];
    emul::tune_fill_kernel<<<4 * h->nsm, 256, 0, h->stream>>>(A, n, kind, 0x5EEDull + static_cast<unsigned>(n));
    rc = emul::check_cuda(h, cudaGetLastError(), "tuner fill");
    if (rc) break;
    cudaEventRecord(e0, h->stream);
    rc = kind == 0 ? emul_dgetrf(h, n, A, n, piv, nb, slices, info, nullptr)
                   : emul_dpotrf(h, 'L', n, A, n, nb, slices, info, nullptr);
    cudaEventRecord(e1, h->stream);
    if (rc) break;
    rc = emul::check_cuda(h, cudaEventSynchronize(e1), "tuner run");
    if (rc) break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c >= 0 && (c == 0 || ms < best_ms)) {
      best_ms = ms;
      best = nb;
    }
  }
  h->prof = prof;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(A);
  if (rc) return rc;
  h->nb_tuned[emul::nb_key(kind, n, slices)] = best;
  *nb_out = best;
  return EMUL_OK;
}

int emul_dgetrf(emul_handle_t h, int n, double* A, int lda, int32_t* ipiv, int nb, int slices, int32_t* info,
                emul_stats* stats) {
  if (!h) return EMUL_INVALID_ARG;
  if (nb == EMUL_NB_AUTO && slices >= 1 && slices <= emul::kMaxSlices && n >= 1) {
    const int rc = emul::resolve_nb(h, 0, n, slices, &nb);
    if (rc) return rc;
  }
  if (nb == EMUL_NB_AUTO && n == 0) nb = 128;
  if (nb == 0) nb = 128;
  if (n < 0 || lda < (n > 1 ? n : 1) || nb < 16 || nb > 512 || nb % 16 != 0 || slices < 0 ||
      slices > emul::kMaxSlices || (n > 0 && (!A || !ipiv || !info)))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_dgetrf: invalid argument");
  const bool autos = slices == 0;
  if (autos && !emul::selector_loaded(h))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_dgetrf: slices = 0 needs a loaded selector");
  if (stats) *stats = emul_stats{0, autos ? 8 : slices, autos ? 3 : slices, 0, 0.0, 0.0};
  double slices_sum = 0.0;
  int updates = 0;
  if (n == 0) return EMUL_OK;
  const int s_fixed = autos ? 8 : slices;
  int s_prev = 8;   // auto mode: the panel and U12 use the previous update's slice count
  int rc = emul::check_cuda(h, cudaMemsetAsync(info, 0, sizeof(int32_t), h->stream), "info reset");
  if (rc) return rc;
  const size_t gw = emul::gemm_workspace_bytes(n, n, nb, s_fixed, false);
  // after the product and LU buffers: G, H (n ints each), one panel of rows
  // (n x nb doubles) and every panel's gather maps (kept from the loop for the
  // deferred interchanges of the L columns)
  const int npanel = (n + nb - 1) / nb;
  const int cpp = (nb + emul::kPermMax - 1) / emul::kPermMax;   // gather maps per panel
  const size_t def_off = emul::al(emul::al(gw) + emul::lu_extra_bytes(nb, h->nsm));
  const size_t maps_off = def_off + emul::al(8ull * n) + emul::al(8ull * n * nb);
  rc = emul::reserve_workspace(
      h, maps_off + emul::al(static_cast<size_t>(npanel) * cpp * emul::kMapInts * sizeof(int)));
  if (rc) return rc;
  int* maps = reinterpret_cast<int*>(static_cast<uint8_t*>(h->ws) + maps_off);
  const emul::LuBufs B = emul::carve(h, gw, nb);
  rc = emul::check_cuda(h, cudaMemsetAsync(B.recs, 0, emul::rec_bytes(h->nsm), h->stream), "leaf records");
  if (rc) return rc;
  rc = emul::check_cuda(h, cudaMemsetAsync(B.drec, 0, 2ull * 2 * emul::kLeaf * 8, h->stream), "leaf records");
  if (rc) return rc;
  h->leaf_salt = 0;
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = nb < n - j0 ? nb : n - j0;
    int ph = emul::phase_begin(h, EMUL_PHASE_PANEL);
    rc = emul::panel_getrf(h, A, lda, n, j0, jb, ipiv, info, autos ? s_prev : s_fixed, B);
    emul::phase_end(h, ph);
    if (rc) return rc;
    const int m2 = n - j0 - jb;
    // L11^-1 on the second stream (L11 is final: the leaves interchanged the
    // panel's own rows) while the interchanges reach the columns right of it
    bool joined = true;
    if (m2 > 0) {
      rc = emul::aux_ready(h);
      if (!rc) rc = emul::check_cuda(h, cudaEventRecord(h->aux_start, h->stream), "stream events");
      if (!rc) rc = emul::check_cuda(h, cudaStreamWaitEvent(h->aux, h->aux_start, 0), "stream events");
      if (rc) return rc;
      emul::trtri_cols_kernel<<<(jb + 1) / 2, emul::trtri_threads(jb), 0, h->aux>>>(A, lda, j0, jb, 1, B.inv,
                                                                                       nullptr);
      h->launches++;
      rc = emul::check_cuda(h, cudaGetLastError(), "trtri");
      if (!rc) rc = emul::check_cuda(h, cudaEventRecord(h->aux_done, h->aux), "stream events");
      if (rc) return rc;
      joined = false;
    }
    ph = emul::phase_begin(h, EMUL_PHASE_SWAP);
    // the columns right of the panel; the columns left of it get all later
    // interchanges at once, after the loop, from the same maps
    for (int c = 0; c < cpp && !rc; ++c) {
      const int k1 = j0 + c * emul::kPermMax, k2 = k1 + emul::kPermMax < j0 + jb ? k1 + emul::kPermMax : j0 + jb;
      if (k1 >= k2) break;
      int* map = maps + static_cast<size_t>(j0 / nb * cpp + c) * emul::kMapInts;
      rc = emul::laswp_prepare(h, ipiv, k1, k2, map);
      if (!rc) rc = emul::laswp_apply(h, A, lda, j0 + jb, n, map);
    }
    emul::phase_end(h, ph);
    // the stream waits for L11^-1 on every path, so no work of this call is left behind on the second stream
    if (!joined) {
      const int rj = emul::check_cuda(h, cudaStreamWaitEvent(h->stream, h->aux_done, 0), "stream events");
      if (!rc) rc = rj;
    }
    if (rc) return rc;
    if (m2 > 0) {
      ph = emul::phase_begin(h, EMUL_PHASE_U12);
      double* A12 = A + j0 + static_cast<long>(j0 + jb) * lda;
      // U12 = L11^-1 A12 (jb x m2), written over A12
      rc = emul::gemm_run(h, jb, m2, jb, 1.0, Operand{B.inv, 1, jb}, Operand{A12, lda, 1}, 0.0, A12, lda,
                          autos ? s_prev : s_fixed, false, 0, nullptr, 0, 0);
      emul::phase_end(h, ph);
      if (rc) return rc;
      ph = emul::phase_begin(h, EMUL_PHASE_UPDATE);
      const double* L21 = A + (j0 + jb) + static_cast<long>(j0) * lda;
      double* A22 = A + (j0 + jb) + static_cast<long>(j0 + jb) * lda;
      int s_step = slices;
      if (autos) {
        // slice count of this update from the selector, then the probe's "before" sums
        rc = emul::selector_features(h, m2, m2, jb, Operand{L21, 1, lda}, Operand{A12, lda, 1},
                                     emul::selector_feature_buffer(h));
        if (rc) return rc;
        rc = emul::selector_predict(h, 1, emul::selector_feature_buffer(h), emul::selector_pred_buffer(h));
        if (rc) return rc;
        int32_t sp = 8;
        rc = emul::check_cuda(h, cudaMemcpyAsync(&sp, emul::selector_pred_buffer(h), 4, cudaMemcpyDeviceToHost,
                                                 h->stream), "selector read");
        if (rc) return rc;
        rc = emul::check_cuda(h, cudaStreamSynchronize(h->stream), "selector read");
        if (rc) return rc;
        s_step = sp < 3 ? 3 : (sp > 8 ? 8 : sp);
        const int R = m2 < emul::kProbeRows ? m2 : emul::kProbeRows;
        double* y0 = B.probe;
        double* a0 = y0 + emul::kProbeRows;
        double* z = y0 + 4 * emul::kProbeRows;
        double* za = z + nb;
        emul::probe_rows_kernel<<<R, 256, 0, h->stream>>>(m2, m2, A22, lda, R, y0, a0);
        emul::probe_z_kernel<<<jb, 256, 0, h->stream>>>(m2, A12, lda, z, za);
        h->launches += 2;
        cudaMemsetAsync(B.flag, 0, sizeof(int), h->stream);
      }
      // A22 -= L21 U12
      rc = emul::gemm_run(h, m2, m2, jb, -1.0, Operand{L21, 1, lda}, Operand{A12, lda, 1}, 1.0, A22, lda, s_step,
                          false, 0, nullptr, 0, 0);
      if (rc) return rc;
      if (autos) {
        const int R = m2 < emul::kProbeRows ? m2 : emul::kProbeRows;
        double* y0 = B.probe;
        double* a0 = y0 + emul::kProbeRows;
        double* y1 = a0 + emul::kProbeRows;
        double* a1 = y1 + emul::kProbeRows;
        double* z = y0 + 4 * emul::kProbeRows;
        double* za = z + nb;
        emul::probe_rows_kernel<<<R, 256, 0, h->stream>>>(m2, m2, A22, lda, R, y1, a1);
        emul::probe_check_kernel<<<(R + 63) / 64, 64, 0, h->stream>>>(m2, m2, jb, L21, lda, R, z, za, y0, a0, y1,
                                                                       a1, B.flag);
        h->launches += 2;
        int fl = 0;
        rc = emul::check_cuda(h, cudaMemcpyAsync(&fl, B.flag, 4, cudaMemcpyDeviceToHost, h->stream), "probe read");
        if (rc) return rc;
        rc = emul::check_cuda(h, cudaStreamSynchronize(h->stream), "probe read");
        if (rc) return rc;
        if (fl && s_step < 8) {
          // undo with the same slice count, redo with 8
          rc = emul::gemm_run(h, m2, m2, jb, 1.0, Operand{L21, 1, lda}, Operand{A12, lda, 1}, 1.0, A22, lda, s_step,
                              false, 0, nullptr, 0, 0);
          if (rc) return rc;
          rc = emul::gemm_run(h, m2, m2, jb, -1.0, Operand{L21, 1, lda}, Operand{A12, lda, 1}, 1.0, A22, lda, 8,
                              false, 0, nullptr, 0, 0);
          if (rc) return rc;
          if (stats) stats->checks_failed++;
          s_step = 8;
        }
        if (stats) {
          stats->slices_min = s_step < stats->slices_min ? s_step : stats->slices_min;
          stats->slices_max = s_step > stats->slices_max ? s_step : stats->slices_max;
        }
      }
      emul::phase_end(h, ph);
      slices_sum += s_step;
      updates++;
      s_prev = s_step;
    }
    if (stats) stats->steps++;
  }
  if (stats) stats->slices_mean = updates ? slices_sum / updates : static_cast<double>(s_fixed);
  // the L columns of every panel but the last: all interchanges of the later
  // panels, composed from the last panel back and gathered once per panel
  const int K = (n + nb - 1) / nb;
  if (K > 1) {
    const int ph = emul::phase_begin(h, EMUL_PHASE_SWAP);
    int* G = reinterpret_cast<int*>(static_cast<uint8_t*>(h->ws) + def_off);
    int* H = G + n;
    double* tmp = reinterpret_cast<double*>(static_cast<uint8_t*>(h->ws) + def_off + emul::al(8ull * n));
    emul::iota2_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, h->stream>>>(n, G, H);
    h->launches++;
    for (int k = K - 2; k >= 0; --k) {
      const int r0 = (k + 1) * nb, r1 = r0 + nb < n ? r0 + nb : n;
      // panel k+1's interchanges, composed from its last gather map back
      for (int c = (r1 - r0 - 1) / emul::kPermMax; c >= 0; --c) {
        emul::compose_kernel<<<1, 512, 0, h->stream>>>(maps + static_cast<size_t>((k + 1) * cpp + c) * emul::kMapInts,
                                                       G, H);
        h->launches++;
      }
      emul::gather_rows_kernel<<<dim3((n - r0 + 255) / 256, nb), 256, 0, h->stream>>>(A, lda, r0, n, k * nb, G,
                                                                                         tmp);
      h->launches++;
      rc = emul::check_cuda(h,
                            cudaMemcpy2DAsync(A + r0 + static_cast<long>(k) * nb * lda, static_cast<size_t>(lda) * 8,
                                              tmp, static_cast<size_t>(n - r0) * 8, static_cast<size_t>(n - r0) * 8,
                                              nb, cudaMemcpyDeviceToDevice, h->stream),
                            "deferred interchanges");
      if (rc) return rc;
    }
    emul::phase_end(h, ph);
  }
  return EMUL_OK;
}

int emul_dgetrs(emul_handle_t h, int n, int nrhs, const double* LU, int lda, const int32_t* ipiv, double* B,
                int ldb) {
  emul::trsv_attr();
  if (!h) return EMUL_INVALID_ARG;
  if (n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1) || (n > 0 && nrhs > 0 && (!LU || !ipiv || !B)))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_dgetrs: invalid argument");
  if (n == 0 || nrhs == 0) return EMUL_OK;
  const int ph = emul::phase_begin(h, EMUL_PHASE_SOLVE);
  const int rc = emul::getrs_body(h, n, nrhs, LU, lda, ipiv, B, ldb);
  emul::phase_end(h, ph);
  return rc;
}

int emul_dpotrf(emul_handle_t h, char uplo, int n, double* A, int lda, int nb, int slices, int32_t* info,
                emul_stats* stats) {
  if (!h) return EMUL_INVALID_ARG;
  if (nb == EMUL_NB_AUTO && slices >= 1 && slices <= emul::kMaxSlices && n >= 1) {
    const int rc = emul::resolve_nb(h, 1, n, slices, &nb);
    if (rc) return rc;
  }
  if (nb == EMUL_NB_AUTO && n == 0) nb = 128;
  if (nb == 0) nb = 128;
  if ((uplo != 'L' && uplo != 'l') || n < 0 || lda < (n > 1 ? n : 1) || nb < 16 || nb > 512 || nb % 16 != 0 ||
      slices < 1 || slices > emul::kMaxSlices || (n > 0 && (!A || !info)))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_dpotrf: invalid argument");
  if (stats) *stats = emul_stats{0, slices, slices, 0, 0.0, static_cast<double>(slices)};
  if (n == 0) return EMUL_OK;
  int rc = emul::check_cuda(h, cudaMemsetAsync(info, 0, sizeof(int32_t), h->stream), "info reset");
  if (rc) return rc;
  const size_t gw = emul::gemm_workspace_bytes(n, n, nb, slices, false);
  rc = emul::reserve_workspace(h, gw + emul::lu_extra_bytes(nb, h->nsm));
  if (rc) return rc;
  const emul::LuBufs B = emul::carve(h, gw, nb);
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = nb < n - j0 ? nb : n - j0;
    const int m2 = n - j0 - jb;
    int ph = emul::phase_begin(h, EMUL_PHASE_PANEL);
    rc = emul::chol_diag(h, A, lda, j0, jb, B.inv, info, m2 > 0);
    emul::phase_end(h, ph);
    if (rc) return rc;
    if (m2 > 0) {
      double* A21 = A + (j0 + jb) + static_cast<long>(j0) * lda;
      // L21 = A21 L11^-T: operand B is (L11^-1)^T, whose row j is row j of L11^-1
      ph = emul::phase_begin(h, EMUL_PHASE_U12);
      rc = emul::gemm_run(h, m2, jb, jb, 1.0, Operand{A21, 1, lda}, Operand{B.inv, 1, jb}, 0.0, A21, lda, slices,
                          false, 0, nullptr, 0, 0);
      emul::phase_end(h, ph);
      if (rc) return rc;
      // A22 -= L21 L21^T on the lower triangle; one slice set for both operands
      ph = emul::phase_begin(h, EMUL_PHASE_UPDATE);
      rc = emul::gemm_run(h, m2, m2, jb, -1.0, Operand{A21, 1, lda}, Operand{A21, 1, lda}, 1.0,
                          A + (j0 + jb) + static_cast<long>(j0 + jb) * lda, lda, slices, true, 0, nullptr, 0, 0);
      emul::phase_end(h, ph);
      if (rc) return rc;
    }
    if (stats) stats->steps++;
  }
  return EMUL_OK;
}

int emul_dpotrs(emul_handle_t h, char uplo, int n, int nrhs, const double* L, int lda, double* B, int ldb) {
  emul::trsv_attr();
  if (!h) return EMUL_INVALID_ARG;
  if ((uplo != 'L' && uplo != 'l') || n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1) ||
      (n > 0 && nrhs > 0 && (!L || !B)))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_dpotrs: invalid argument");
  if (n == 0 || nrhs == 0) return EMUL_OK;
  const int ph = emul::phase_begin(h, EMUL_PHASE_SOLVE);
  if (nrhs == 1) {
    // one right-hand side: both substitutions in one cooperative launch
    int rc = emul::reserve_workspace(h, emul::kAl);
    if (rc) return rc;
    unsigned long long* cnt = static_cast<unsigned long long*>(h->ws);
    rc = emul::check_cuda(h, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), h->stream), "solve barrier");
    if (rc) return rc;
    emul::smem_attr(reinterpret_cast<const void*>(emul::getrs1_kernel<true>),
                    emul::kSolveBs * (emul::kSolveBs + 1) * 8);
    long ldl = lda;
    long long limit = h->wait_limit;
    int* status = h->d_status;
    void* args[] = {const_cast<double**>(&L), &ldl, &n, &B, &cnt, &status, &limit};
    h->launches++;
    rc = emul::check_cuda(h,
                          cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(emul::getrs1_kernel<true>),
                                                      dim3(h->nsm), dim3(256), args,
                                                      emul::kSolveBs * (emul::kSolveBs + 1) * 8, h->stream),
                          "Cholesky solve");
    emul::phase_end(h, ph);
    return rc;
  }
  constexpr int bs = 128;
  for (int d0 = 0; d0 < n; d0 += bs) {
    const int b = bs < n - d0 ? bs : n - d0;
    emul::trsv_block_kernel<<<nrhs, 1024, b * (b + 1) * sizeof(double), h->stream>>>(L, lda, B, ldb, d0, b, 1, 0, 0);
    h->launches += (d0 + b < n) ? 2 : 1;
    if (d0 + b < n)
      emul::gemv_update_kernel<<<dim3((n - d0 - b + 255) / 256, nrhs), 256, 0, h->stream>>>(L, lda, B, ldb, d0 + b,
                                                                                               n, d0, b, 0);
  }
  for (int d0 = ((n - 1) / bs) * bs; d0 >= 0; d0 -= bs) {
    const int b = bs < n - d0 ? bs : n - d0;
    emul::trsv_block_kernel<<<nrhs, 1024, b * (b + 1) * sizeof(double), h->stream>>>(L, lda, B, ldb, d0, b, 0, 0, 1);
    h->launches += (d0 > 0) ? 2 : 1;
    if (d0 > 0)
      emul::gemv_update_kernel<<<dim3((d0 + 7) / 8, nrhs), 256, 0, h->stream>>>(L, lda, B, ldb, 0, d0, d0, b, 1);
  }
  emul::phase_end(h, ph);
  return emul::check_cuda(h, cudaGetLastError(), "potrs");
}

int emul_backward_error(emul_handle_t h, int n, const double* A, int lda, const double* x, const double* b,
                        double* out) {
  if (!h) return EMUL_INVALID_ARG;
  if (n <= 0 || lda < n || !A || !x || !b || !out)
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_backward_error: invalid argument");
  const size_t need = emul::lu_extra_bytes(16, h->nsm);
  int rc = emul::reserve_workspace(h, need);
  if (rc) return rc;
  const emul::LuBufs B = emul::carve(h, 0, 16);
  rc = emul::check_cuda(h, cudaMemsetAsync(B.racc, 0, 4 * sizeof(unsigned long long), h->stream), "residual reset");
  if (rc) return rc;
  emul::residual_kernel<<<(n + 255) / 256, 256, 2048 * sizeof(double), h->stream>>>(n, A, lda, x, b, B.racc);
  h->launches += 2;
  emul::residual_finish_kernel<<<1, 1, 0, h->stream>>>(n, B.racc, out);
  return emul::check_cuda(h, cudaGetLastError(), "residual");
}

}  // extern "C"

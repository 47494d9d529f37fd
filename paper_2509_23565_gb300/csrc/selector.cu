// Learned slice selector and its training data (the
// a-posteriori check follows the validated error-free products cited in
// Sec. 3 of arXiv 2509.23565).
//
// * features: 32-bin histograms of the exponent offset of each entry from its
//   row scale (A) and column scale (B), normalised by the entry count (64 floats).
// * slice errors (training labels): the slices for s are the first s slices
//   for s = 8 and the levels L <= s+1 are common to every s, so one INT32
//   level-sum pass of the tensor-core product gives D_s for all s = 3..8:
//   err_s = max_ij |D_s - D_8| / (4 k u (|A||B|)_ij).
// * MLP 64 -> 128 -> 128 -> 128 -> 6 (classes s = 3..8), ReLU, softmax
//   cross-entropy; BF16 weight copies for the forward / backward products,
//   FP32 master weights, gradients and AdamW state; FP32 accumulation.
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>

#include "handle.h"
#include "round.cuh"

namespace emul {

namespace {

constexpr int kBins = 32;
constexpr int kF = 64, kH = 128, kC = 6;
constexpr int kTile = 16;   // samples per block in the MLP kernels
constexpr int kMaxBatch = 8192;

// flat parameter layout: W0 [128][64], b0, W1 [128][128], b1, W2 [128][128], b2, W3 [6][128], b3
constexpr int kOffW0 = 0, kOffB0 = kOffW0 + kH * kF;
constexpr int kOffW1 = kOffB0 + kH, kOffB1 = kOffW1 + kH * kH;
constexpr int kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kC * kH;
constexpr int kParams = kOffB3 + kC;

__device__ __forceinline__ int entry_exponent(uint64_t u) {   // smallest E with |x| < 2^E (u = |x| bits, x != 0)
  const int E = static_cast<int>(u >> 52);
  if (E > 0) return E - 1022;
  return -1010 - __clzll(static_cast<long long>(u));
}

// Histogram of the rows of a rows x k operand: element (r, c) at X[r*rs + c*cs].
// One thread per row (rows contiguous) or one warp per row (k contiguous).
__global__ void hist_kernel(int rows, int k, const double* __restrict__ X, long rs, long cs,
                            unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[kBins];
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint64_t* Xb = reinterpret_cast<const uint64_t*>(X);
  if (rs == 1) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) {
      uint64_t mx = 0;
      for (int c = 0; c < k; ++c) {
        const uint64_t u = __ldg(Xb + r + static_cast<long>(c) * cs) & 0x7FFFFFFFFFFFFFFFull;
        mx = u > mx ? u : mx;
      }
      if (mx < 0x7FF0000000000000ull) {
        const int e = mx ? entry_exponent(mx) : 0;
        for (int c = 0; c < k; ++c) {
          const uint64_t u = __ldg(Xb + r + static_cast<long>(c) * cs) & 0x7FFFFFFFFFFFFFFFull;
          int bin = kBins - 1;
          if (u) {
            const int off = e - entry_exponent(u);
            bin = off < kBins - 1 ? off : kBins - 1;
          }
          atomicAdd(&h[bin], 1u);
        }
      }
    }
  } else {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x / 32) + warp;
    if (r < rows) {
      const uint64_t* xr = Xb + static_cast<long>(r) * rs;
      uint64_t mx = 0;
      for (int c = lane; c < k; c += 32) {
        const uint64_t u = __ldg(xr + c) & 0x7FFFFFFFFFFFFFFFull;
        mx = u > mx ? u : mx;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t v = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
        mx = v > mx ? v : mx;
      }
      if (mx < 0x7FF0000000000000ull) {
        const int e = mx ? entry_exponent(mx) : 0;
        for (int c = lane; c < k; c += 32) {
          const uint64_t u = __ldg(xr + c) & 0x7FFFFFFFFFFFFFFFull;
          int bin = kBins - 1;
          if (u) {
            const int off = e - entry_exponent(u);
            bin = off < kBins - 1 ? off : kBins - 1;
          }
          atomicAdd(&h[bin], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBins; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void hist_finish_kernel(const unsigned int* hist, double na, double nb, float* feat) {
  const int i = threadIdx.x;
  if (i < kBins) {
    feat[i] = static_cast<float>(hist[i] / na);
    feat[kBins + i] = static_cast<float>(hist[kBins + i] / nb);
  }
}

// (|A||B|)_ij in FP64, 16 x 16 tiles.
__global__ void absprod_kernel(int m, int n, int k, const double* A, long lda, const double* B, long ldb, double* P) {
  __shared__ double As[16][17], Bs[16][17];
  const int i = blockIdx.x * 16 + threadIdx.x, j = blockIdx.y * 16 + threadIdx.y;
  double acc = 0.0;
  for (int k0 = 0; k0 < k; k0 += 16) {
    const int ka = k0 + threadIdx.y, kb = k0 + threadIdx.x;
    As[threadIdx.x][threadIdx.y] = (i < m && ka < k) ? fabs(A[i + static_cast<long>(ka) * lda]) : 0.0;
    Bs[threadIdx.y][threadIdx.x] = (j < n && kb < k) ? fabs(B[kb + static_cast<long>(j) * ldb]) : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(As[threadIdx.x][kk], Bs[threadIdx.y][kk], acc);
    __syncthreads();
  }
  if (i < m && j < n) P[i + static_cast<long>(j) * m] = acc;
}

// err[s-3] = max over entries of |D_s - D_8| / (4 k u (|A||B|)_ij), D_s from the
// INT32 level sums L = 2..9 (levels[(L-2)*plane + i + j*m]).
__global__ void slice_error_kernel(int m, int n, int k, const int32_t* levels, long plane, const int32_t* e,
                                   const int32_t* f, const double* P, unsigned long long* err) {
  const long idx = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x;
  double loc[6] = {0, 0, 0, 0, 0, 0};
  if (idx < static_cast<long>(m) * n) {
    const int i = static_cast<int>(idx % m), j = static_cast<int>(idx / m);
    const double scale = 4.0 * k * 1.1102230246251565e-16 * P[idx];
    if (e[i] != 2147483647 && f[j] != 2147483647 && scale > 0.0) {
      double D[6];
      __int128 T = 0;
      for (int L = 2; L <= 9; ++L) {
        T = T * 128 + (__int128)levels[static_cast<long>(L - 2) * plane + idx];
        const int s = L - 1;
        if (s >= 3) D[s - 3] = rn_scaled(T, e[i] + f[j] - 7 * (s + 1));
      }
      for (int q = 0; q < 6; ++q) loc[q] = fabs(D[q] - D[5]) / scale;
    }
  }
  for (int q = 0; q < 6; ++q) {
    double v = loc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(&err[q], static_cast<unsigned long long>(__double_as_longlong(v)));
  }
}

__global__ void err_finish_kernel(const unsigned long long* bits, double* err) {
  if (threadIdx.x < 6) err[threadIdx.x] = __longlong_as_double(static_cast<long long>(bits[threadIdx.x]));
}

// ------------------------------------------------------------------ MLP
__device__ __forceinline__ float wbf(const __nv_bfloat16* W, int idx) { return __bfloat162float(W[idx]); }

// Forward pass for kTile samples per block (128 threads).  Z* receive the
// pre-activations (for the backward pass); H* are kept in shared memory.
__device__ void mlp_forward_tile(int b0, int batch, const float* X, const __nv_bfloat16* Wb, const float* P,
                                 float (*h0)[kF], float (*ha)[kH], float (*hb)[kH], float* Z0, float* Z1, float* Z2,
                                 float* Z3) {
  const int t = threadIdx.x;
  for (int idx = t; idx < kTile * kF; idx += blockDim.x) {
    const int sI = idx / kF, i = idx % kF;
    h0[sI][i] = (b0 + sI < batch) ? X[static_cast<long>(b0 + sI) * kF + i] : 0.f;
  }
  __syncthreads();
  // layer 0: 64 -> 128
  for (int sI = 0; sI < kTile; ++sI) {
    float acc = P[kOffB0 + t];
    for (int i = 0; i < kF; ++i) acc = fmaf(h0[sI][i], wbf(Wb, kOffW0 + t * kF + i), acc);
    if (Z0 && b0 + sI < batch) Z0[static_cast<long>(b0 + sI) * kH + t] = acc;
    ha[sI][t] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  // layer 1
  for (int sI = 0; sI < kTile; ++sI) {
    float acc = P[kOffB1 + t];
    for (int i = 0; i < kH; ++i) acc = fmaf(ha[sI][i], wbf(Wb, kOffW1 + t * kH + i), acc);
    if (Z1 && b0 + sI < batch) Z1[static_cast<long>(b0 + sI) * kH + t] = acc;
    hb[sI][t] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  // layer 2
  for (int sI = 0; sI < kTile; ++sI) {
    float acc = P[kOffB2 + t];
    for (int i = 0; i < kH; ++i) acc = fmaf(hb[sI][i], wbf(Wb, kOffW2 + t * kH + i), acc);
    if (Z2 && b0 + sI < batch) Z2[static_cast<long>(b0 + sI) * kH + t] = acc;
    ha[sI][t] = fmaxf(acc, 0.f);
  }
  __syncthreads();
  // layer 3: 128 -> 6 (logits into Z3)
  for (int idx = t; idx < kTile * kC; idx += blockDim.x) {
    const int sI = idx / kC, o = idx % kC;
    float acc = P[kOffB3 + o];
    for (int i = 0; i < kH; ++i) acc = fmaf(ha[sI][i], wbf(Wb, kOffW3 + o * kH + i), acc);
    if (b0 + sI < batch) Z3[static_cast<long>(b0 + sI) * kC + o] = acc;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(int batch, const float* X, const __nv_bfloat16* Wb,
                                                          const float* P, float* Z0, float* Z1, float* Z2, float* Z3) {
  __shared__ float h0[kTile][kF], ha[kTile][kH], hb[kTile][kH];
  mlp_forward_tile(blockIdx.x * kTile, batch, X, Wb, P, h0, ha, hb, Z0, Z1, Z2, Z3);
}

__global__ void predict_finish_kernel(int batch, const float* Z3, int32_t* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  int best = 0;
  for (int o = 1; o < kC; ++o)
    if (Z3[static_cast<long>(b) * kC + o] > Z3[static_cast<long>(b) * kC + best]) best = o;
  out[b] = 3 + best;
}

// Backward pass: gradients of the mean cross-entropy, accumulated into G
// (FP32 atomics).  Re-reads the activations from X and Z0..Z3.
__global__ void __launch_bounds__(128) mlp_backward_kernel(int batch, const float* X, const int32_t* labels,
                                                           const __nv_bfloat16* Wb, const float* Z0, const float* Z1,
                                                           const float* Z2, const float* Z3, float* G, float* loss) {
  __shared__ float d3[kTile][kC];
  __shared__ float dA[kTile][kH], dB[kTile][kH];
  __shared__ float hin[kTile][kH];
  const int t = threadIdx.x;
  const int b0 = blockIdx.x * kTile;
  const float invB = 1.f / static_cast<float>(batch);
  // softmax - onehot
  if (t < kTile) {
    const int b = b0 + t;
    if (b < batch) {
      float mx = -INFINITY;
      for (int o = 0; o < kC; ++o) mx = fmaxf(mx, Z3[static_cast<long>(b) * kC + o]);
      float sum = 0.f;
      for (int o = 0; o < kC; ++o) sum += __expf(Z3[static_cast<long>(b) * kC + o] - mx);
      const int y = labels[b] - 3;
      for (int o = 0; o < kC; ++o) {
        const float p = __expf(Z3[static_cast<long>(b) * kC + o] - mx) / sum;
        d3[t][o] = (p - (o == y ? 1.f : 0.f)) * invB;
      }
      atomicAdd(loss, -(Z3[static_cast<long>(b) * kC + y] - mx - __logf(sum)) * invB);
    } else {
      for (int o = 0; o < kC; ++o) d3[t][o] = 0.f;
    }
  }
  // h2 = relu(Z2)
  for (int sI = 0; sI < kTile; ++sI)
    hin[sI][t] = (b0 + sI < batch) ? fmaxf(Z2[static_cast<long>(b0 + sI) * kH + t], 0.f) : 0.f;
  __syncthreads();
  // layer 3 grads
  for (int idx = t; idx < kC * kH; idx += blockDim.x) {
    const int o = idx / kH, i = idx % kH;
    float g = 0.f;
    for (int sI = 0; sI < kTile; ++sI) g = fmaf(d3[sI][o], hin[sI][i], g);
    atomicAdd(&G[kOffW3 + o * kH + i], g);
  }
  if (t < kC) {
    float g = 0.f;
    for (int sI = 0; sI < kTile; ++sI) g += d3[sI][t];
    atomicAdd(&G[kOffB3 + t], g);
  }
  // dh2 = d3 W3, masked by Z2 > 0
  for (int sI = 0; sI < kTile; ++sI) {
    float acc = 0.f;
    for (int o = 0; o < kC; ++o) acc = fmaf(d3[sI][o], wbf(Wb, kOffW3 + o * kH + t), acc);
    const bool on = (b0 + sI < batch) && Z2[static_cast<long>(b0 + sI) * kH + t] > 0.f;
    dA[sI][t] = on ? acc : 0.f;
  }
  __syncthreads();
  // two hidden layers: (layer 2: input relu(Z1)), (layer 1: input relu(Z0))
  for (int layer = 2; layer >= 1; --layer) {
    const float* Zin = layer == 2 ? Z1 : Z0;
    const int offW = layer == 2 ? kOffW2 : kOffW1, offB = layer == 2 ? kOffB2 : kOffB1;
    for (int sI = 0; sI < kTile; ++sI)
      hin[sI][t] = (b0 + sI < batch) ? fmaxf(Zin[static_cast<long>(b0 + sI) * kH + t], 0.f) : 0.f;
    __syncthreads();
    for (int o = 0; o < kH; ++o) {
      float g = 0.f;
      for (int sI = 0; sI < kTile; ++sI) g = fmaf(dA[sI][o], hin[sI][t], g);
      atomicAdd(&G[offW + o * kH + t], g);
    }
    {
      float g = 0.f;
      for (int sI = 0; sI < kTile; ++sI) g += dA[sI][t];
      atomicAdd(&G[offB + t], g);
    }
    for (int sI = 0; sI < kTile; ++sI) {
      float acc = 0.f;
      for (int o = 0; o < kH; ++o) acc = fmaf(dA[sI][o], wbf(Wb, offW + o * kH + t), acc);
      const bool on = (b0 + sI < batch) && Zin[static_cast<long>(b0 + sI) * kH + t] > 0.f;
      dB[sI][t] = on ? acc : 0.f;
    }
    __syncthreads();
    for (int sI = 0; sI < kTile; ++sI) dA[sI][t] = dB[sI][t];
    __syncthreads();
  }
  // layer 0: input X (64)
  for (int idx = t; idx < kTile * kF; idx += blockDim.x) {
    const int sI = idx / kF, i = idx % kF;
    hin[sI][i] = (b0 + sI < batch) ? X[static_cast<long>(b0 + sI) * kF + i] : 0.f;
  }
  __syncthreads();
  for (int idx = t; idx < kH * kF; idx += blockDim.x) {
    const int o = idx / kF, i = idx % kF;
    float g = 0.f;
    for (int sI = 0; sI < kTile; ++sI) g = fmaf(dA[sI][o], hin[sI][i], g);
    atomicAdd(&G[kOffW0 + o * kF + i], g);
  }
  {
    float g = 0.f;
    for (int sI = 0; sI < kTile; ++sI) g += dA[sI][t];
    atomicAdd(&G[kOffB0 + t], g);
  }
}

__global__ void to_bf16_kernel(int n, const float* P, __nv_bfloat16* Wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Wb[i] = __float2bfloat16_rn(P[i]);
}

__global__ void adamw_kernel(int n, float* P, const float* G, float* M, float* V, __nv_bfloat16* Wb, float lr,
                             float wd, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * M[i] + (1.f - b1) * g;
  const float v = b2 * V[i] + (1.f - b2) * g * g;
  M[i] = m;
  V[i] = v;
  float p = P[i];
  p -= lr * ((m / c1) / (sqrtf(v / c2) + eps) + wd * p);
  P[i] = p;
  Wb[i] = __float2bfloat16_rn(p);
}

}  // namespace

// Selector state, allocated on first use.
struct SelectorState {
  float* P = nullptr;           // master parameters
  __nv_bfloat16* Wb = nullptr;  // BF16 copies
  float* G = nullptr;
  float* M = nullptr;
  float* V = nullptr;
  float* Z = nullptr;           // activations for kMaxBatch samples
  float* loss = nullptr;
  int32_t* pred = nullptr;
  float* feat = nullptr;        // one feature vector (auto LU)
  unsigned int* hist = nullptr;
  int step = 0;
  bool loaded = false;
};

namespace {
SelectorState* state_of(emul_handle_t h);

int ensure_state(emul_handle_t h, SelectorState** out) {
  SelectorState* st = state_of(h);
  if (!st->P) {
    const size_t zfl = static_cast<size_t>(kMaxBatch) * (3 * kH + kC);
    if (cudaMalloc(&st->P, kParams * 4) != cudaSuccess || cudaMalloc(&st->Wb, kParams * 2) != cudaSuccess ||
        cudaMalloc(&st->G, kParams * 4) != cudaSuccess || cudaMalloc(&st->M, kParams * 4) != cudaSuccess ||
        cudaMalloc(&st->V, kParams * 4) != cudaSuccess || cudaMalloc(&st->Z, zfl * 4) != cudaSuccess ||
        cudaMalloc(&st->loss, 4) != cudaSuccess || cudaMalloc(&st->pred, kMaxBatch * 4) != cudaSuccess ||
        cudaMalloc(&st->feat, kF * 4) != cudaSuccess || cudaMalloc(&st->hist, 2 * kBins * 4) != cudaSuccess)
      return set_error(h, EMUL_NO_WORKSPACE, "selector allocation failed");
  }
  *out = st;
  return EMUL_OK;
}

SelectorState* state_of(emul_handle_t h) {
  if (!h->selector) h->selector = new SelectorState();
  return static_cast<SelectorState*>(h->selector);
}

float* zptr(SelectorState* st, int batch, int which) {
  // Z0, Z1, Z2 (batch x 128 each), Z3 (batch x 6)
  return st->Z + static_cast<size_t>(which) * kMaxBatch * kH;
}

}  // namespace

int selector_features(emul_handle_t h, int m, int n, int k, Operand A, Operand B, float* feat) {
  SelectorState* st = nullptr;
  int rc = ensure_state(h, &st);
  if (rc) return rc;
  rc = check_cuda(h, cudaMemsetAsync(st->hist, 0, 2 * kBins * 4, h->stream), "features reset");
  if (rc) return rc;
  if (A.rs == 1)
    hist_kernel<<<(m + 255) / 256, 256, 0, h->stream>>>(m, k, A.ptr, A.rs, A.cs, st->hist);
  else
    hist_kernel<<<(m + 7) / 8, 256, 0, h->stream>>>(m, k, A.ptr, A.rs, A.cs, st->hist);
  if (B.rs == 1)
    hist_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(n, k, B.ptr, B.rs, B.cs, st->hist + kBins);
  else
    hist_kernel<<<(n + 7) / 8, 256, 0, h->stream>>>(n, k, B.ptr, B.rs, B.cs, st->hist + kBins);
  hist_finish_kernel<<<1, 32, 0, h->stream>>>(st->hist, static_cast<double>(m) * k, static_cast<double>(n) * k, feat);
  h->launches += 3;
  return check_cuda(h, cudaGetLastError(), "features");
}

int selector_predict(emul_handle_t h, int batch, const float* X, int32_t* out) {
  SelectorState* st = nullptr;
  int rc = ensure_state(h, &st);
  if (rc) return rc;
  mlp_forward_kernel<<<(batch + kTile - 1) / kTile, 128, 0, h->stream>>>(batch, X, st->Wb, st->P, nullptr, nullptr,
                                                                        nullptr, zptr(st, batch, 3));
  predict_finish_kernel<<<(batch + 127) / 128, 128, 0, h->stream>>>(batch, zptr(st, batch, 3), out);
  h->launches += 2;
  return check_cuda(h, cudaGetLastError(), "selector predict");
}

bool selector_loaded(emul_handle_t h) { return state_of(h)->loaded; }

void selector_free(emul_handle_t h) {
  if (!h->selector) return;
  SelectorState* st = static_cast<SelectorState*>(h->selector);
  for (void* p : {(void*)st->P, (void*)st->Wb, (void*)st->G, (void*)st->M, (void*)st->V, (void*)st->Z, (void*)st->loss,
                  (void*)st->pred, (void*)st->feat, (void*)st->hist})
    if (p) cudaFree(p);
  delete st;
  h->selector = nullptr;
}
float* selector_feature_buffer(emul_handle_t h) {
  SelectorState* st = nullptr;
  if (ensure_state(h, &st)) return nullptr;
  return st->feat;
}
int32_t* selector_pred_buffer(emul_handle_t h) {
  SelectorState* st = nullptr;
  if (ensure_state(h, &st)) return nullptr;
  return st->pred;
}

}  // namespace emul

using emul::Operand;

extern "C" {

int emul_selector_features(emul_handle_t h, int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                           float* feat) {
  if (!h) return EMUL_INVALID_ARG;
  if (m <= 0 || n <= 0 || k <= 0 || lda < m || ldb < k || !A || !B || !feat)
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_selector_features: invalid argument");
  return emul::selector_features(h, m, n, k, Operand{A, 1, lda}, Operand{B, ldb, 1}, feat);
}

int emul_slice_errors(emul_handle_t h, int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                      double* err) {
  if (!h) return EMUL_INVALID_ARG;
  if (m <= 0 || n <= 0 || k <= 0 || lda < m || ldb < k || !A || !B || !err || k > 16384 ||
      static_cast<long>(m) * n > (1L << 24))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_slice_errors: invalid argument");
  // workspace after the product's own: levels (8 planes int32), |A||B| (FP64), scales, error bits
  const size_t gw = emul::gemm_workspace_bytes(m, n, k, 8, false);
  const size_t plane = static_cast<size_t>(m) * n;
  const size_t need = gw + 8 * plane * 4 + plane * 8 + (m + n) * 4 + 1024;
  int rc = emul::reserve_workspace(h, need);
  if (rc) return rc;
  uint8_t* p = static_cast<uint8_t*>(h->ws) + (gw + 255) / 256 * 256;
  int32_t* levels = reinterpret_cast<int32_t*>(p);
  p += (8 * plane * 4 + 255) / 256 * 256;
  double* P = reinterpret_cast<double*>(p);
  p += (plane * 8 + 255) / 256 * 256;
  int32_t* e = reinterpret_cast<int32_t*>(p);
  p += ((size_t)m * 4 + 255) / 256 * 256;
  int32_t* f = reinterpret_cast<int32_t*>(p);
  p += ((size_t)n * 4 + 255) / 256 * 256;
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(p);
  rc = emul::gemm_run(h, m, n, k, 1.0, Operand{A, 1, lda}, Operand{B, ldb, 1}, 0.0, nullptr, 0, 8, false, 1, levels,
                      m, static_cast<long>(plane));
  if (rc) return rc;
  // the product left the scales of A and B at the start of the workspace; recompute them into e, f
  // with the slicing kernel's definition through a second split is wasteful, so reuse: the
  // product's layout is [slices A][e][slices B][f]
  {
    const long kp = (static_cast<long>(k) + 7) / 8 * 8;
    uint8_t* w = static_cast<uint8_t*>(h->ws);
    const size_t sa = (static_cast<size_t>(8) * m * kp * 2 + 255) / 256 * 256;
    const int32_t* ea = reinterpret_cast<const int32_t*>(w + sa);
    const size_t eab = ((size_t)m * 4 + 255) / 256 * 256;
    const size_t sb = (static_cast<size_t>(8) * n * kp * 2 + 255) / 256 * 256;
    const int32_t* fbp = reinterpret_cast<const int32_t*>(w + sa + eab + sb);
    rc = emul::check_cuda(h, cudaMemcpyAsync(e, ea, m * 4, cudaMemcpyDeviceToDevice, h->stream), "scales");
    if (rc) return rc;
    rc = emul::check_cuda(h, cudaMemcpyAsync(f, fbp, n * 4, cudaMemcpyDeviceToDevice, h->stream), "scales");
    if (rc) return rc;
  }
  emul::absprod_kernel<<<dim3((m + 15) / 16, (n + 15) / 16), dim3(16, 16), 0, h->stream>>>(m, n, k, A, lda, B, ldb, P);
  rc = emul::check_cuda(h, cudaMemsetAsync(bits, 0, 6 * 8, h->stream), "error reset");
  if (rc) return rc;
  emul::slice_error_kernel<<<(plane + 255) / 256, 256, 0, h->stream>>>(m, n, k, levels, static_cast<long>(plane), e,
                                                                        f, P, bits);
  emul::err_finish_kernel<<<1, 32, 0, h->stream>>>(bits, err);
  h->launches += 3;
  return emul::check_cuda(h, cudaGetLastError(), "slice errors");
}

int emul_selector_set_params(emul_handle_t h, const float* params) {
  if (!h || !params) return EMUL_INVALID_ARG;
  emul::SelectorState* st = nullptr;
  int rc = emul::ensure_state(h, &st);
  if (rc) return rc;
  rc = emul::check_cuda(h, cudaMemcpyAsync(st->P, params, emul::kParams * 4, cudaMemcpyHostToDevice, h->stream),
                        "params");
  if (rc) return rc;
  cudaMemsetAsync(st->M, 0, emul::kParams * 4, h->stream);
  cudaMemsetAsync(st->V, 0, emul::kParams * 4, h->stream);
  emul::to_bf16_kernel<<<(emul::kParams + 255) / 256, 256, 0, h->stream>>>(emul::kParams, st->P, st->Wb);
  st->step = 0;
  st->loaded = true;
  return emul::check_cuda(h, cudaStreamSynchronize(h->stream), "params");
}

int emul_selector_get_params(emul_handle_t h, float* params) {
  if (!h || !params) return EMUL_INVALID_ARG;
  emul::SelectorState* st = nullptr;
  int rc = emul::ensure_state(h, &st);
  if (rc) return rc;
  rc = emul::check_cuda(h, cudaMemcpyAsync(params, st->P, emul::kParams * 4, cudaMemcpyDeviceToHost, h->stream),
                        "params");
  if (rc) return rc;
  return emul::check_cuda(h, cudaStreamSynchronize(h->stream), "params");
}

int emul_selector_grad(emul_handle_t h, int batch, const float* X, const int32_t* labels, float* grad, float* loss) {
  if (!h) return EMUL_INVALID_ARG;
  if (batch <= 0 || batch > emul::kMaxBatch || !X || !labels || !grad || !loss)
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_selector_grad: invalid argument");
  emul::SelectorState* st = nullptr;
  int rc = emul::ensure_state(h, &st);
  if (rc) return rc;
  cudaMemsetAsync(grad, 0, emul::kParams * 4, h->stream);
  cudaMemsetAsync(loss, 0, 4, h->stream);
  const int blocks = (batch + emul::kTile - 1) / emul::kTile;
  emul::mlp_forward_kernel<<<blocks, 128, 0, h->stream>>>(batch, X, st->Wb, st->P, emul::zptr(st, batch, 0),
                                                          emul::zptr(st, batch, 1), emul::zptr(st, batch, 2),
                                                          emul::zptr(st, batch, 3));
  emul::mlp_backward_kernel<<<blocks, 128, 0, h->stream>>>(batch, X, labels, st->Wb, emul::zptr(st, batch, 0),
                                                           emul::zptr(st, batch, 1), emul::zptr(st, batch, 2),
                                                           emul::zptr(st, batch, 3), grad, loss);
  h->launches += 2;
  return emul::check_cuda(h, cudaGetLastError(), "selector grad");
}

int emul_selector_train_step(emul_handle_t h, int batch, const float* X, const int32_t* labels, float lr,
                             float weight_decay, float* loss) {
  if (!h) return EMUL_INVALID_ARG;
  emul::SelectorState* st = nullptr;
  int rc = emul::ensure_state(h, &st);
  if (rc) return rc;
  rc = emul_selector_grad(h, batch, X, labels, st->G, loss ? loss : st->loss);
  if (rc) return rc;
  st->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, static_cast<float>(st->step)), c2 = 1.f - powf(b2, static_cast<float>(st->step));
  emul::adamw_kernel<<<(emul::kParams + 255) / 256, 256, 0, h->stream>>>(emul::kParams, st->P, st->G, st->M, st->V,
                                                                         st->Wb, lr, weight_decay, b1, b2, 1e-8f, c1,
                                                                         c2);
  h->launches++;
  return emul::check_cuda(h, cudaGetLastError(), "selector step");
}

int emul_selector_predict(emul_handle_t h, int batch, const float* X, int32_t* slices) {
  if (!h) return EMUL_INVALID_ARG;
  if (batch <= 0 || batch > emul::kMaxBatch || !X || !slices)
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_selector_predict: invalid argument");
  return emul::selector_predict(h, batch, X, slices);
}

int emul_selector_save(emul_handle_t h, const char* path) {
  if (!h || !path) return EMUL_INVALID_ARG;
  std::vector<float> p(emul::kParams);
  int rc = emul_selector_get_params(h, p.data());
  if (rc) return rc;
  FILE* fp = fopen(path, "wb");
  if (!fp) return emul::set_error(h, EMUL_INVALID_ARG, "cannot open selector file for writing");
  const uint32_t hdr[2] = {0x53454c31u, static_cast<uint32_t>(emul::kParams)};   // "SEL1", count
  const bool ok = fwrite(hdr, 4, 2, fp) == 2 && fwrite(p.data(), 4, p.size(), fp) == p.size();
  fclose(fp);
  return ok ? EMUL_OK : emul::set_error(h, EMUL_INVALID_ARG, "selector file write failed");
}

int emul_selector_load(emul_handle_t h, const char* path) {
  if (!h || !path) return EMUL_INVALID_ARG;
  FILE* fp = fopen(path, "rb");
  if (!fp) return emul::set_error(h, EMUL_INVALID_ARG, "cannot open selector file");
  uint32_t hdr[2] = {0, 0};
  std::vector<float> p(emul::kParams);
  const bool ok = fread(hdr, 4, 2, fp) == 2 && hdr[0] == 0x53454c31u && hdr[1] == emul::kParams &&
                  fread(p.data(), 4, p.size(), fp) == p.size();
  fclose(fp);
  if (!ok) return emul::set_error(h, EMUL_INVALID_ARG, "not a selector weight file");
  return emul_selector_set_params(h, p.data());
}

}  // extern "C"

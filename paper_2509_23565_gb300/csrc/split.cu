// Scale extraction and slicing of a GEMM operand (arXiv 2509.23565, Section 2,
// Eq. 1-4): per row r of a rows x k operand,
//   e_r = smallest e with max_c |x(r,c)| < 2^e   (0 for a zero row, NONFINITE for Inf/NaN),
//   N   = trunc(x * 2^(7s - e_r)),  |N| < 2^(7s),
//   slice p (0 = most significant) = sign(x) * ((|N| >> 7(s-1-p)) & 127).
// Everything is integer arithmetic on the IEEE-754 bit fields; no FP64
// instruction is issued.  Slices are stored as BF16 bit patterns (every
// integer in [-127, 127] is exact in BF16), plane-major and K-contiguous:
//   out[(p*rows + r)*ldk + c], the layout the TMA loads of the product read.
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "emul_internal.h"

namespace emul {

__device__ __forceinline__ int exponent_of_maxbits(uint64_t u) {
  if (u >= 0x7FF0000000000000ull) return kNonFinite;
  if (u == 0) return 0;
  const int E = static_cast<int>(u >> 52);
  if (E > 0) return E - 1022;                      // |x| in [2^(E-1023), 2^(E-1022))
  return -1010 - __clzll(static_cast<long long>(u));  // subnormal: |x| = u * 2^-1074
}

// |N| = trunc(|x| * 2^(W - e)) for |x| < 2^e; u = |x| bit pattern.
__device__ __forceinline__ uint64_t scaled_magnitude(uint64_t u, int e, int W) {
  const int E = static_cast<int>(u >> 52);
  const uint64_t M = (u & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
  const int sh = (E ? E : 1) - 1075 + W - e;      // x = M * 2^((E?E:1) - 1075)
  if (sh >= 0) return M << sh;                     // sh <= W - 53 <= 3
  const int r = -sh;
  return r >= 64 ? 0ull : (M >> r);
}

__device__ __forceinline__ uint16_t digit_bf16(const uint16_t* lut, uint64_t mag, bool neg, int shift) {
  const int d = static_cast<int>((mag >> shift) & 127ull);
  return lut[neg ? 127 - d : 127 + d];
}

__device__ void fill_lut(uint16_t* lut) {
  for (int i = threadIdx.x; i < 255; i += blockDim.x)
    lut[i] = __bfloat16_as_ushort(__float2bfloat16_rn(static_cast<float>(i - 127)));
}

// Rows contiguous (rs == 1): tile of 64 rows per block, transposed through shared memory.
__global__ void __launch_bounds__(256) split_rowcontig_kernel(int rows, int k, const double* __restrict__ X,
                                                              long cs, int s, int32_t* __restrict__ exps,
                                                              uint16_t* __restrict__ out, long ldk) {
  __shared__ uint16_t lut[256];
  __shared__ uint64_t red[4][64];
  __shared__ int e_s[64];
  __shared__ uint64_t tile[64][65];
  fill_lut(lut);
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * 64;
  const uint64_t* Xb = reinterpret_cast<const uint64_t*>(X);
  {
    const int r = tid & 63, part = tid >> 6;
    uint64_t mx = 0;
    if (r0 + r < rows)
      for (int c = part; c < k; c += 4) {
        const uint64_t u = __ldg(Xb + (r0 + r) + static_cast<long>(c) * cs) & 0x7FFFFFFFFFFFFFFFull;
        mx = u > mx ? u : mx;
      }
    red[part][r] = mx;
  }
  __syncthreads();
  if (tid < 64) {
    uint64_t mx = red[0][tid];
    for (int p = 1; p < 4; ++p) mx = red[p][tid] > mx ? red[p][tid] : mx;
    const int e = exponent_of_maxbits(mx);
    e_s[tid] = e;
    if (r0 + tid < rows) exps[r0 + tid] = e;
  }
  __syncthreads();
  const int W = 7 * s;
  for (int c0 = 0; c0 < ldk; c0 += 64) {
    for (int i = tid; i < 64 * 64; i += 256) {
      const int r = i & 63, c = i >> 6;
      uint64_t u = 0;
      if (r0 + r < rows && c0 + c < k) u = __ldg(Xb + (r0 + r) + static_cast<long>(c0 + c) * cs);
      tile[r][c] = u;
    }
    __syncthreads();
    for (int item = tid; item < 64 * 8; item += 256) {
      const int r = item >> 3, ch = item & 7;
      const int c = c0 + ch * 8;
      if (r0 + r >= rows || c >= ldk) continue;
      const int e = e_s[r];
      uint64_t mag[8];
      bool neg[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint64_t u = tile[r][ch * 8 + j];
        neg[j] = (u >> 63) != 0;
        mag[j] = (e == kNonFinite) ? 0ull : scaled_magnitude(u & 0x7FFFFFFFFFFFFFFFull, e, W);
      }
      for (int p = 0; p < s; ++p) {
        const int shift = 7 * (s - 1 - p);
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          w[j] = static_cast<uint32_t>(digit_bf16(lut, mag[2 * j], neg[2 * j], shift)) |
                 (static_cast<uint32_t>(digit_bf16(lut, mag[2 * j + 1], neg[2 * j + 1], shift)) << 16);
        *reinterpret_cast<uint4*>(out + (static_cast<long>(p) * rows + (r0 + r)) * ldk + c) =
            make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    __syncthreads();
  }
}

// k contiguous (cs == 1): one warp per row.
__global__ void __launch_bounds__(256) split_kcontig_kernel(int rows, int k, const double* __restrict__ X, long rs,
                                                            int s, int32_t* __restrict__ exps,
                                                            uint16_t* __restrict__ out, long ldk) {
  __shared__ uint16_t lut[256];
  fill_lut(lut);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + warp;
  if (r >= rows) return;
  const uint64_t* xr = reinterpret_cast<const uint64_t*>(X) + static_cast<long>(r) * rs;
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
  const int e = exponent_of_maxbits(mx);
  if (lane == 0) exps[r] = e;
  const int W = 7 * s;
  for (int c = lane * 8; c < ldk; c += 256) {
    uint64_t mag[8];
    bool neg[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t u = (c + j < k) ? __ldg(xr + c + j) : 0ull;
      neg[j] = (u >> 63) != 0;
      mag[j] = (e == kNonFinite) ? 0ull : scaled_magnitude(u & 0x7FFFFFFFFFFFFFFFull, e, W);
    }
    for (int p = 0; p < s; ++p) {
      const int shift = 7 * (s - 1 - p);
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        w[j] = static_cast<uint32_t>(digit_bf16(lut, mag[2 * j], neg[2 * j], shift)) |
               (static_cast<uint32_t>(digit_bf16(lut, mag[2 * j + 1], neg[2 * j + 1], shift)) << 16);
      *reinterpret_cast<uint4*>(out + (static_cast<long>(p) * rows + r) * ldk + c) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

cudaError_t launch_split(cudaStream_t st, int rows, int k, const double* X, long rs, long cs, int s, int32_t* exps,
                         uint16_t* out, long ldk) {
  if (rows <= 0) return cudaSuccess;
  if (rs == 1) {
    split_rowcontig_kernel<<<(rows + 63) / 64, 256, 0, st>>>(rows, k, X, cs, s, exps, out, ldk);
  } else {
    split_kcontig_kernel<<<(rows + 7) / 8, 256, 0, st>>>(rows, k, X, rs, s, exps, out, ldk);
  }
  return cudaGetLastError();
}

}  // namespace emul

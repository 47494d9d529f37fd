// Internal declarations shared by the CUDA sources of the library.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace emul {

constexpr int kNonFinite = 2147483647;   // scale of a row / column holding Inf or NaN
constexpr int kMaxSlices = 8;
constexpr int kBK = 32;                  // K elements per staged chunk (64 B of BF16: SWIZZLE_64B)
constexpr int kExactBudget = 1040;       // k * pairs per accumulator: 1040 * 127^2 < 2^24

// One sweep of the product schedule: one or two accumulator jobs over the K
// chunks [k0c, k1c), sharing the staged slice tiles of each chunk.  A job
// sums the slice pairs (p, L-p), p = pb..pe, of one level L into one TMEM slot.
struct Sweep {
  int16_t k0c, k1c;   // chunk range
  int8_t L[2];        // job levels (L[1] = 0: one job)
  int8_t pb[2], pe[2];// pair ranges
  int8_t held;        // 1: the jobs are the last level, held for the final step
  int8_t nplanes;     // slice planes 1..nplanes of A and of B are staged
};

struct GemmArgs {
  int M, N, K;
  int s, t;                 // slices, threshold (t = s + 1)
  double alpha, beta;
  double* C;
  long ldc;
  const int32_t* ea;        // row scales of A   [M]
  const int32_t* fb;        // column scales of B [N]
  const Sweep* sched;       // device array
  int nsweeps;
  int tiles_m, tiles_n, ntiles;
  int lower;                // 1: only entries with row >= col are written
  int tri;                  // 1: tiles enumerated over the lower triangle (square tiles)
  int mode;                 // 0: update C; 1: add level sums into `levels`
  int32_t* levels;
  long ldl, ldl_plane;
  int* status;              // device status word (EMUL_TIMEOUT on a bounded-wait expiry)
  long long wait_limit;     // cycles
};

cudaError_t launch_split(cudaStream_t st, int rows, int k, const double* X, long rs, long cs, int s, int32_t* exps,
                         uint16_t* out, long ldk);

// BN = 128 with int64 Horner state (wide = false) or BN = 64 with 128-bit state (wide = true).
cudaError_t launch_gemm(cudaStream_t st, bool wide, const CUtensorMap& tmA, const CUtensorMap& tmB,
                        const GemmArgs& args, int grid, int stages, size_t smem_bytes);
size_t gemm_stage_bytes(bool wide, int s);

}  // namespace emul

// Internal declarations shared by the CUDA sources of the library.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace emul {

constexpr int kNonFinite = 2147483647;   // scale of a row / column holding Inf or NaN
constexpr int kMaxSlices = 8;
constexpr int kBK = 32;                  // K elements per staged chunk (64 B of BF16: SWIZZLE_64B)
constexpr int kMaxStagesCfg = 8;         // deepest ring of staged chunks
constexpr int kExactBudget = 1040;       // k * pairs per accumulator: 1040 * 127^2 < 2^24

// One sweep of the product schedule: one or two accumulator jobs over the K
// chunks [k0c, k1c), sharing the staged slice tiles of each chunk.  A job
// sums the slice pairs (p, L-p), p = pb..pe, of one level L into one TMEM slot.
// The epilogue takes the jobs in schedule order and adds each job's sum with
// its weight into the state, R += I 2^(7(t-L)); a job flagged kFinal (the last
// job of the 64-bit variant) completes T = R + I 2^(7(t-L)), rounds it and
// updates C.
enum JobFlag : int8_t { kFinal = 1 };
struct Sweep {
  int16_t k0c, k1c;    // chunk range
  int8_t L[2];         // job levels (L[1] = 0: one job)
  int8_t pb[2], pe[2]; // pair ranges
  int8_t flags[2];     // JobFlag bits of the two jobs
  int8_t nplanes;      // slice planes 1..nplanes of A and of B are staged
  int8_t kcs;          // K chunks per stage (kcs * nplanes <= s tiles of A and of B)
};

// Slot assignment of the jobs: TMEM slot (bits 0-1) and the parity of the
// slot's use count (bit 2) for job j of the tile-phase ph, at tab[ph * njobs + j];
// the i-th tile of a CTA uses phase i (i < t0) or t0 + (i - t0) % period.
struct SlotPlan {
  const uint8_t* tab;
  int njobs, t0, period;
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
  SlotPlan slots;           // TMEM slot of every job (device table)
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

// BN = 128 with an int64 state (wide = false) or BN = 64 with a 128-bit state
// (wide = true).  pair (128-column tile only): clusters of two CTAs, tiles of
// 256 rows (args.tiles_m counts them), tmB staged BN/2 rows per CTA, grid even.
cudaError_t launch_gemm(cudaStream_t st, bool wide, bool pair, const CUtensorMap& tmA, const CUtensorMap& tmB,
                        const GemmArgs& args, int grid, int stages, size_t smem_bytes);
size_t gemm_stage_bytes(bool wide, int s, bool pair);
// Ring stages of a launch and its shared-memory bytes.
int gemm_stages(bool wide, int s, bool pair, size_t* smem_bytes);
// CTA pairs that can be resident at once with this much shared memory.
int gemm_pair_capacity(size_t smem_bytes);

}  // namespace emul

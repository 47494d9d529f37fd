// Handle state and the internal product driver shared by the C-ABI sources.
#pragma once
#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/emul.h"
#include "emul_internal.h"

struct emul_handle_s {
  cudaStream_t stream = nullptr;
  int device = 0;
  int nsm = 0;
  int* d_status = nullptr;          // device status word written by kernels
  void* ws = nullptr;               // workspace (device)
  size_t ws_bytes = 0;
  struct SchedEntry {
    emul::Sweep* sched;             // device: sweeps, then the slot table
    int nsweeps;
    emul::SlotPlan plan;
  };
  std::map<uint64_t, SchedEntry> sched_cache;   // (slices of A / B, s, wide, level-sum mode, threshold, chunks) -> device schedule
  std::map<uint64_t, bool> narrow_cache;        // (s, t, chunks) -> the 128-column variant applies
  std::string last_error;
  void* encode_fn = nullptr;        // cuTensorMapEncodeTiled
  long long wait_limit = 2000000000LL;
  uint32_t leaf_salt = 0;            // epoch salt of the LU leaf exchange (per leaf launch)
  // profiling (emul_profile_*)
  long long launches = 0;
  bool prof = false;
  struct ProfRec {
    cudaEvent_t e0, e1;
    double flops, bytes;
  };
  std::vector<ProfRec> recs;
  struct PhaseRec {
    int kind;
    cudaEvent_t e0, e1;
  };
  std::vector<PhaseRec> phases;
  std::vector<cudaEvent_t> event_pool;
  std::map<uint64_t, int> nb_tuned;  // (kind, n, slices) -> block size chosen by emul_autotune_nb
  // second stream of the LU step: L11^-1 is formed there while the row
  // interchanges run on `stream` (created on first use, same device)
  cudaStream_t aux = nullptr;
  cudaEvent_t aux_start = nullptr, aux_done = nullptr;
  void* selector = nullptr;         // emul::SelectorState (selector.cu)
  void* batched = nullptr;          // emul::BatchedState (batched.cu)
};

namespace emul {

// A GEMM operand viewed as `rows` x `k`: element (r, c) at ptr[r*rs + c*cs].
struct Operand {
  const double* ptr;
  long rs, cs;
};

int set_error(emul_handle_t h, int code, const std::string& msg);
// Raise a kernel's dynamic shared-memory limit to `bytes`, once per device.
void smem_attr(const void* fn, int bytes);
int check_cuda(emul_handle_t h, cudaError_t e, const char* what);

// Grow the workspace to at least `bytes` (synchronises the device when it grows).
int reserve_workspace(emul_handle_t h, size_t bytes);
// Event timing of one factorization phase (EMUL_PHASE_*) while profiling is
// enabled: phase_begin returns a record index (-1 when profiling is off or an
// event cannot be had), phase_end closes it.
int phase_begin(emul_handle_t h, int kind);
void phase_end(emul_handle_t h, int idx);
// Workspace bytes a product of this shape needs (slices, scales).
size_t gemm_workspace_bytes(int m, int n, int k, int s, bool same_operand);

// C <- beta*C + alpha*(A B^T-view) with the emulated product.  A: m x k operand,
// B: n x k operand (row j of the operand is column j of the mathematical B).
// `ws_offset` places the slices inside the workspace (callers running several
// products back to back on one stream may share offset 0).
int gemm_run(emul_handle_t h, int m, int n, int k, double alpha, Operand A, Operand B, double beta, double* C,
             long ldc, int s, bool lower, int mode, int32_t* levels, long ldl, long ldl_plane, size_t ws_offset = 0,
             int t = 0,     // t: truncation threshold, 0 = s + 1
             int s_a = 0, int s_b = 0);   // slices of A / of B whose pairs are kept (0: s; max = s)

// Learned slice selector (selector.cu).
int selector_features(emul_handle_t h, int m, int n, int k, Operand A, Operand B, float* feat);
int selector_predict(emul_handle_t h, int batch, const float* X, int32_t* out);
bool selector_loaded(emul_handle_t h);
float* selector_feature_buffer(emul_handle_t h);
int32_t* selector_pred_buffer(emul_handle_t h);
void selector_free(emul_handle_t h);
void batched_free(emul_handle_t h);

}  // namespace emul

// C-ABI entry points: handle management, slicing, level sums and the emulated
// DGEMM (arXiv 2509.23565, Section 2, Eq. 1-4; Section 4, Eq. 7).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <mutex>
#include <set>
#include <utility>

#include <cudaTypedefs.h>

#include "handle.h"

namespace emul {

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline long kpad_of(int k) { return (static_cast<long>(k) + 7) / 8 * 8; }

// The slice pairs kept: p <= sa slices of A, q <= sb slices of B (sa = sb = s
// for the method itself; unequal counts keep a subset of the pairs of the
// max(sa, sb)-slice split, whose leading slices are those of a shorter split).
struct PairSet {
  int sa, sb;
  int lo(int L) const { return L - sb > 1 ? L - sb : 1; }          // first p of level L
  int hi(int L) const { return L - 1 < sa ? L - 1 : sa; }          // last p of level L
  int count(int L) const { return hi(L) >= lo(L) ? hi(L) - lo(L) + 1 : 0; }
  // highest slice index of A or B a pair of level L uses
  int planes(int L) const { return hi(L) > L - lo(L) ? hi(L) : L - lo(L); }
};

// Sum over the levels L = 2..last of n_L 2^(7(last-L)) times 127^2: the
// worst-case magnitude per unit of k of T = sum_L I_L 2^(7(last-L)) (the
// wide variant's state after all its jobs, last = t).
long double exact_sum_bound_per_k(const PairSet& ps, int last) {
  long double acc = 0.0L;
  for (int L = 2; L <= last; ++L) acc = acc * 128.0L + ps.count(L);
  return acc * 127.0L * 127.0L;
}

// K chunks per accumulator job of n slice pairs under the exactness budget.
int seg_chunks(int n) { return n > 0 ? kExactBudget / (n * kBK) : 0; }

struct Job {
  int L, pb, pe, c0, c1, flags;
};

Job make_job(const PairSet& ps, int L, int c0, int c1, int flags) {
  return Job{L, ps.lo(L), ps.hi(L), c0, c1, flags};
}

void push_sweep(std::vector<Sweep>& out, const Job& a, const Job* b) {
  Sweep sw{};
  sw.k0c = static_cast<int16_t>(a.c0);
  sw.k1c = static_cast<int16_t>(a.c1);
  const Job* js[2] = {&a, b};
  int np = 0;
  for (int j = 0; j < 2 && js[j]; ++j) {
    sw.L[j] = static_cast<int8_t>(js[j]->L);
    sw.pb[j] = static_cast<int8_t>(js[j]->pb);
    sw.pe[j] = static_cast<int8_t>(js[j]->pe);
    sw.flags[j] = static_cast<int8_t>(js[j]->flags);
    const int pj = js[j]->pe > js[j]->L - js[j]->pb ? js[j]->pe : js[j]->L - js[j]->pb;
    np = np > pj ? np : pj;
  }
  sw.nplanes = static_cast<int8_t>(np);
  out.push_back(sw);
}

// Banded schedule: the levels are covered by bands of one level or of two
// adjacent levels.  A two-level band (L, L+1) shares every staged chunk
// between both levels (the planes of L are a subset of those of L+1); a band
// that does not fit the exactness budget over the whole K runs in K groups.  The bands minimise the staged planes per K chunk (dynamic
// programme over the levels).  The epilogue adds every job's level sum with
// its weight, R += I_L 2^(7(t-L)), so the jobs may come in any order: the
// bands are issued from the highest level down, each tile starting with its
// longest MMA jobs (they keep the tensor cores busy while the epilogue rounds
// the previous tile) and ending, in the 64-bit variant, with level 2 as one
// single job: the final job, whose term 2^(7(t-2)) I_2 is added and rounded
// last.
bool build_banded(const PairSet& ps, int t, int nch, bool wide, std::vector<Sweep>& out) {
  out.clear();
  const int kInf = 1 << 28;
  std::vector<int> cost(t + 3, 0), choice(t + 3, 0);
  auto groups = [&](int seg) { return (nch + seg - 1) / seg; };
  for (int L = t; L >= 2; --L) {
    cost[L] = kInf;
    const int sg1 = seg_chunks(ps.count(L));
    // the final job (level 2 in the 64-bit variant) must be one job alone
    if (sg1 >= 1 && cost[L + 1] < kInf && (wide || L > 2 || groups(sg1) == 1)) {
      cost[L] = ps.planes(L) + cost[L + 1];
      choice[L] = 1;
    }
    if (L + 1 <= t && cost[L + 2] < kInf && (wide || L > 2)) {
      const int a = seg_chunks(ps.count(L)), b = seg_chunks(ps.count(L + 1));
      const int sg2 = a < b ? a : b;
      if (sg2 >= 1 && ps.planes(L + 1) + cost[L + 2] < cost[L]) {
        cost[L] = ps.planes(L + 1) + cost[L + 2];
        choice[L] = 2;
      }
    }
  }
  if (cost[2] >= kInf) return false;
  std::vector<std::pair<int, int>> bands;   // (first level, levels)
  for (int L = 2; L <= t; L += choice[L]) bands.push_back({L, choice[L]});
  for (auto it = bands.rbegin(); it != bands.rend(); ++it) {
    const int L = it->first;
    if (it->second == 1) {
      const int G = groups(seg_chunks(ps.count(L)));
      const int size = (nch + G - 1) / G;
      for (int g = 0; g < G; ++g) {
        const int c0 = g * size, c1 = c0 + size < nch ? c0 + size : nch;
        push_sweep(out, make_job(ps, L, c0, c1, (!wide && L == 2) ? kFinal : 0), nullptr);
      }
    } else {
      const int a = seg_chunks(ps.count(L)), b = seg_chunks(ps.count(L + 1));
      const int G = groups(a < b ? a : b);
      const int size = (nch + G - 1) / G;
      for (int g = 0; g < G; ++g) {
        const int c0 = g * size, c1 = c0 + size < nch ? c0 + size : nch;
        const Job j1 = make_job(ps, L + 1, c0, c1, 0);
        push_sweep(out, make_job(ps, L, c0, c1, 0), &j1);
      }
    }
  }
  return true;
}

// Level-ordered schedule, the fallback: from the highest level down, a level
// whose n_L pairs fit the budget over the whole K is one job; otherwise its
// pairs are split into groups that fit (64-bit variant) or its K range into
// segments (128-bit variant).  Consecutive jobs of one K range share a sweep.
// In the 64-bit variant level 2 comes last as one job (the final job).
bool build_levelwise(const PairSet& ps, int t, int nch, bool wide, std::vector<Sweep>& out) {
  out.clear();
  std::vector<Job> jobs;
  const int kc = nch * kBK;
  for (int L = t; L >= 2; --L) {
    const int pb = ps.lo(L);
    const int pe = ps.hi(L);
    const int n = pe - pb + 1;
    const int fin = (!wide && L == 2) ? kFinal : 0;
    if (n * kc <= kExactBudget) {
      jobs.push_back(Job{L, pb, pe, 0, nch, fin});
    } else if (!wide) {
      if (fin) return false;
      const int per = kExactBudget / kc;          // pairs per job
      if (per < 1) return false;
      for (int p = pb; p <= pe; p += per)
        jobs.push_back(Job{L, p, p + per - 1 < pe ? p + per - 1 : pe, 0, nch, 0});
    } else {
      int cm = kExactBudget / (kBK * n);
      if (cm < 1) cm = 1;
      for (int c0 = 0; c0 < nch; c0 += cm) jobs.push_back(Job{L, pb, pe, c0, c0 + cm < nch ? c0 + cm : nch, 0});
    }
  }
  for (size_t i = 0; i < jobs.size();) {
    // the final job stays alone in its sweep
    if (i + 1 < jobs.size() && !(jobs[i + 1].flags & kFinal) && jobs[i + 1].c0 == jobs[i].c0 &&
        jobs[i + 1].c1 == jobs[i].c1) {
      push_sweep(out, jobs[i], &jobs[i + 1]);
      i += 2;
    } else {
      push_sweep(out, jobs[i], nullptr);
      i += 1;
    }
  }
  return true;
}

// TMEM slot of every job.  The MMA issuer and the epilogue follow one rule:
// a job takes the slot whose current job is drained earliest (ties: lowest
// slot); the epilogue releases a slot when it has drained its job (in
// level-sum mode every job is drained the same way).  The rule is simulated
// tile by tile until the slot state (release points relative to the tile,
// use-count parities) repeats; the table holds the transient tiles and one
// period.  A sweep may only take slots released by jobs before it, otherwise
// the schedule is rejected.
bool plan_slots(const std::vector<Sweep>& sw, std::vector<uint8_t>& tab, int& njobs, int& t0, int& period) {
  std::vector<int> first_of_job;
  for (const Sweep& w : sw) {
    const int first = static_cast<int>(first_of_job.size());
    for (int j = 0; j < 2 && w.L[j]; ++j) first_of_job.push_back(first);
  }
  njobs = static_cast<int>(first_of_job.size());
  if (njobs == 0) return false;
  constexpr int kS = 4, kMaxTiles = 64;
  constexpr long long kFree = -(1ll << 40);
  long long rel[kS];
  int cnt[kS];
  for (int i = 0; i < kS; ++i) rel[i] = kFree, cnt[i] = 0;
  std::vector<std::vector<long long>> states;
  tab.clear();
  for (int tile = 0; tile < kMaxTiles; ++tile) {
    const long long base = static_cast<long long>(tile) * njobs;
    std::vector<long long> key;
    for (int i = 0; i < kS; ++i) {
      key.push_back(rel[i] == kFree ? kFree : rel[i] - base);
      key.push_back(cnt[i] & 1);
    }
    for (size_t i0 = 0; i0 < states.size(); ++i0)
      if (states[i0] == key) {
        t0 = static_cast<int>(i0);
        period = tile - t0;
        return true;
      }
    states.push_back(key);
    for (int j = 0; j < njobs; ++j) {
      int b = 0;
      for (int i = 1; i < kS; ++i)
        if (rel[i] < rel[b]) b = i;
      if (rel[b] >= base + first_of_job[j]) return false;
      tab.push_back(static_cast<uint8_t>(b | ((cnt[b] & 1) << 2)));
      rel[b] = base + j;
      cnt[b]++;
    }
  }
  return false;
}

// K chunks per stage: a stage holds s tiles of A and s of B, so a sweep that
// stages fewer planes packs several chunks into one stage (one barrier phase
// for more bytes; the copy engine's rate grows with the bytes per phase).
void set_chunks_per_stage(int s, std::vector<Sweep>& out) {
  for (Sweep& w : out) {
    const int nc = w.k1c - w.k0c;
    const int kmax = w.nplanes > 0 && s / w.nplanes > 1 ? s / w.nplanes : 1;
    const int nst = (nc + kmax - 1) / kmax;
    w.kcs = static_cast<int8_t>(nst > 0 ? (nc + nst - 1) / nst : 1);
  }
}

// Schedule and slot plan for the levels 2..t (t = 0: the default threshold
// s + 1 of the method): the banded schedule when it exists and plans, else the
// level-ordered one.  The level-sum mode (mode1) drains every job the same
// way and uses the same schedule.
// sa, sb: slices of A and of B whose pairs are kept (0: s); s = max(sa, sb)
// is the split both operands get and the number of planes a stage holds.
bool build_schedule(int s, int nch, bool wide, bool mode1, std::vector<Sweep>& out, std::vector<uint8_t>& tab,
                    int& njobs, int& t0, int& period, int t = 0, int sa = 0, int sb = 0) {
  (void)mode1;
  if (sa == 0) sa = s;
  if (sb == 0) sb = s;
  if (t == 0) t = s + 1;
  if (t < 2 || t > sa + sb || (sa > sb ? sa : sb) != s) return false;
  const PairSet ps{sa, sb};
  if (!(build_banded(ps, t, nch, wide, out) && plan_slots(out, tab, njobs, t0, period)) &&
      !(build_levelwise(ps, t, nch, wide, out) && plan_slots(out, tab, njobs, t0, period)))
    return false;
  set_chunks_per_stage(s, out);
  return true;
}

// The narrow variant keeps the state R in int64 and completes T = R + I_2 2^(7(t-2))
// in its final job (in 64 bits when the warp's terms allow, else in 128): it
// needs level 2 in one job and the sum of the other levels inside int64.
bool narrow_ok(int s, int k, int t = 0, int sa = 0, int sb = 0) {
  if (sa == 0) sa = s;
  if (sb == 0) sb = s;
  if (t == 0) t = s + 1;
  if (s > 7) return false;
  const int nch = (k + kBK - 1) / kBK;
  std::vector<Sweep> tmp;
  std::vector<uint8_t> tab;
  int nj, t0, per;
  if (!build_schedule(s, nch, false, false, tmp, tab, nj, t0, per, t, sa, sb)) return false;
  // R, the sum of the levels 3..t with their weights, stays below 2^61, so
  // that R + I_2 2^(7(t-2)) fits in 64 bits whenever |I_2| 2^(7(t-2)) <= 2^62
  // (the epilogue's test; otherwise it adds the term in 128 bits).
  const PairSet ps{sa, sb};
  const long double kk = static_cast<long double>(nch * kBK);
  long double r = 0.0L;
  for (int L = 3; L <= t; ++L) r += ps.count(L) * 127.0L * 127.0L * kk * powl(2.0L, 7.0L * (t - L));
  return r < 2305843009213693952.0L;   // 2^61
}

// The wide variant's 128-bit exact sum T must stay below 2^126.
bool wide_ok(int s, int t, int k, int sa = 0, int sb = 0) {
  const int nch = (k + kBK - 1) / kBK;
  return exact_sum_bound_per_k(PairSet{sa ? sa : s, sb ? sb : s}, t) * static_cast<long double>(nch * kBK) < 8.5e37L;
}

// Device copy of a schedule: the sweeps, then the slot table (16-byte aligned).
size_t schedule_bytes(size_t nsweeps, size_t ntab) { return nsweeps * sizeof(Sweep) + 16 + ntab; }

int get_schedule(emul_handle_t h, int s, int t, int nch, bool wide, bool mode1, Sweep** dptr, int* count,
                 SlotPlan* plan, int sa, int sb) {
  const uint64_t key = (static_cast<uint64_t>(sa) << 40) | (static_cast<uint64_t>(sb) << 32) |
                       (static_cast<uint64_t>(s) << 24) | (static_cast<uint64_t>(wide) << 23) |
                       (static_cast<uint64_t>(mode1) << 22) | (static_cast<uint64_t>(t) << 13) |
                       static_cast<uint64_t>(nch);   // nch < 2^13 (k <= 65536)
  auto it = h->sched_cache.find(key);
  if (it != h->sched_cache.end()) {
    *dptr = it->second.sched;
    *count = it->second.nsweeps;
    *plan = it->second.plan;
    return EMUL_OK;
  }
  std::vector<Sweep> v;
  std::vector<uint8_t> tab;
  SlotPlan sp{};
  if (!build_schedule(s, nch, wide, mode1, v, tab, sp.njobs, sp.t0, sp.period, t, sa, sb))
    return set_error(h, EMUL_INVALID_ARG, "no schedule for this slice count / k");
  const size_t off_tab = (v.size() * sizeof(Sweep) + 15) / 16 * 16;
  std::vector<uint8_t> blob(off_tab + tab.size(), 0);
  std::memcpy(blob.data(), v.data(), v.size() * sizeof(Sweep));
  std::memcpy(blob.data() + off_tab, tab.data(), tab.size());
  uint8_t* d = nullptr;
  if (cudaMalloc(&d, blob.size()) != cudaSuccess) return set_error(h, EMUL_NO_WORKSPACE, "schedule allocation failed");
  if (cudaMemcpy(d, blob.data(), blob.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_error(h, EMUL_CUDA_ERROR, "schedule upload failed");
  sp.tab = d + off_tab;
  h->sched_cache[key] = emul_handle_s::SchedEntry{reinterpret_cast<Sweep*>(d), static_cast<int>(v.size()), sp};
  *dptr = reinterpret_cast<Sweep*>(d);
  *count = static_cast<int>(v.size());
  *plan = sp;
  return EMUL_OK;
}

int encode_slices_map(emul_handle_t h, CUtensorMap* map, const uint16_t* base, int rows, int k, long kpad, int s,
                      int box_rows) {
  auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(h->encode_fn);
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(s)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(kpad) * 2, static_cast<cuuint64_t>(kpad) * 2 * rows};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(h, EMUL_CUDA_ERROR, "cuTensorMapEncodeTiled failed");
  return EMUL_OK;
}

__global__ void scale_c_kernel(int m, int n, double alpha, double beta, double* C, long ldc) {
  const long total = static_cast<long>(m) * n;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i % m);
    const long c = i / m;
    double* p = C + r + c * ldc;
    const double ad = __dmul_rn(alpha, 0.0);
    *p = (beta == 0.0) ? ad : __dadd_rn(ad, __dmul_rn(beta, *p));
  }
}

__global__ void zero_levels_kernel(int m, int n, int planes, int32_t* lv, long ldl, long ldp) {
  const long total = static_cast<long>(m) * n * planes;
  for (long i = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i % m);
    const long rest = i / m;
    const long c = rest % n;
    const long p = rest / n;
    lv[p * ldp + r + c * ldl] = 0;
  }
}

}  // namespace

// The attribute belongs to the device, and one process may drive several GPUs.
void smem_attr(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (done.insert({dev, fn}).second) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int set_error(emul_handle_t h, int code, const std::string& msg) {
  if (h) h->last_error = msg;
  return code;
}

int check_cuda(emul_handle_t h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return EMUL_OK;
  return set_error(h, EMUL_CUDA_ERROR, std::string(what) + ": " + cudaGetErrorString(e));
}

int reserve_workspace(emul_handle_t h, size_t bytes) {
  if (bytes <= h->ws_bytes) return EMUL_OK;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  const size_t want = align_up(bytes + bytes / 8);
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return set_error(h, EMUL_NO_WORKSPACE, "workspace allocation failed");
  }
  h->ws_bytes = want;
  return EMUL_OK;
}

size_t gemm_workspace_bytes(int m, int n, int k, int s, bool same_operand) {
  const size_t kp = static_cast<size_t>(kpad_of(k));
  size_t b = align_up(static_cast<size_t>(s) * m * kp * 2) + align_up(static_cast<size_t>(m) * 4);
  if (!same_operand) b += align_up(static_cast<size_t>(s) * n * kp * 2) + align_up(static_cast<size_t>(n) * 4);
  return b + kAlign;
}

int gemm_run(emul_handle_t h, int m, int n, int k, double alpha, Operand A, Operand B, double beta, double* C,
             long ldc, int s, bool lower, int mode, int32_t* levels, long ldl, long ldl_plane, size_t ws_offset,
             int t, int s_a, int s_b) {
  if (s_a == 0) s_a = s;
  if (s_b == 0) s_b = s;
  if (t == 0) t = s + 1;
  if (m <= 0 || n <= 0) return EMUL_OK;
  if (k <= 0) {
    if (mode == 1) {
      zero_levels_kernel<<<256, 256, 0, h->stream>>>(m, n, s, levels, ldl, ldl_plane);
      h->launches++;
      return check_cuda(h, cudaGetLastError(), "zero levels");
    }
    scale_c_kernel<<<1024, 256, 0, h->stream>>>(m, n, alpha, beta, C, ldc);
    h->launches++;
    return check_cuda(h, cudaGetLastError(), "scale C");
  }
  const bool same = (A.ptr == B.ptr && A.rs == B.rs && A.cs == B.cs && m == n);
  const size_t need = ws_offset + gemm_workspace_bytes(m, n, k, s, same);
  int rc = reserve_workspace(h, need);
  if (rc) return rc;
  const long kp = kpad_of(k);
  uint8_t* w = static_cast<uint8_t*>(h->ws) + ws_offset;
  uint16_t* sa = reinterpret_cast<uint16_t*>(w);
  w += align_up(static_cast<size_t>(s) * m * kp * 2);
  int32_t* ea = reinterpret_cast<int32_t*>(w);
  w += align_up(static_cast<size_t>(m) * 4);
  uint16_t* sb = sa;
  int32_t* fb = ea;
  if (!same) {
    sb = reinterpret_cast<uint16_t*>(w);
    w += align_up(static_cast<size_t>(s) * n * kp * 2);
    fb = reinterpret_cast<int32_t*>(w);
  }
  rc = check_cuda(h, launch_split(h->stream, m, k, A.ptr, A.rs, A.cs, s, ea, sa, kp), "split A");
  if (rc) return rc;
  h->launches++;
  if (!same) {
    rc = check_cuda(h, launch_split(h->stream, n, k, B.ptr, B.rs, B.cs, s, fb, sb, kp), "split B");
    if (rc) return rc;
    h->launches++;
  }
  if (mode == 1) {
    h->launches++;
    zero_levels_kernel<<<256, 256, 0, h->stream>>>(m, n, s, levels, ldl, ldl_plane);
    rc = check_cuda(h, cudaGetLastError(), "zero levels");
    if (rc) return rc;
  }
  // the narrow test plans a schedule; it is made once per (s, t, K chunks)
  const uint64_t nkey = (static_cast<uint64_t>(s_a) << 48) | (static_cast<uint64_t>(s_b) << 40) |
                        (static_cast<uint64_t>(s) << 32) | (static_cast<uint64_t>(t) << 16) |
                        static_cast<uint64_t>((k + kBK - 1) / kBK);
  auto nit = h->narrow_cache.find(nkey);
  if (nit == h->narrow_cache.end()) nit = h->narrow_cache.emplace(nkey, narrow_ok(s, k, t, s_a, s_b)).first;
  const bool wide = !nit->second;
  if (wide && mode == 0 && !wide_ok(s, t, k, s_a, s_b))
    return set_error(h, EMUL_NOT_SUPPORTED, "threshold too high for this k: the 128-bit exact sum could overflow");
  const int nch = (k + kBK - 1) / kBK;
  Sweep* sched = nullptr;
  int nsweeps = 0;
  SlotPlan plan{};
  rc = get_schedule(h, s, t, nch, wide, mode == 1, &sched, &nsweeps, &plan, s_a, s_b);
  if (rc) return rc;
  const int BN = wide ? 64 : 128;
  // CTA pairs (cta_group::2) for the 128-column tile once there are two
  // 128-row tiles: each SM stages half of B, a quarter less than alone
  bool pair = !wide && m > 128 && h->nsm >= 2;
  if (pair) {
    size_t smem_pair = 0;
    gemm_stages(false, s, true, &smem_pair);
    pair = gemm_pair_capacity(smem_pair) >= 1;   // else one CTA per tile
  }
  CUtensorMap tmA, tmB;
  rc = encode_slices_map(h, &tmA, sa, m, k, kp, s, 128);
  if (rc) return rc;
  rc = encode_slices_map(h, &tmB, sb, n, k, kp, s, pair ? BN / 2 : BN);
  if (rc) return rc;

  GemmArgs a{};
  a.M = m;
  a.N = n;
  a.K = k;
  a.s = s;
  a.t = t;
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.ea = ea;
  a.fb = fb;
  a.sched = sched;
  a.nsweeps = nsweeps;
  a.slots = plan;
  a.tiles_m = pair ? (m + 255) / 256 : (m + 127) / 128;
  a.tiles_n = (n + BN - 1) / BN;
  a.lower = lower ? 1 : 0;
  a.tri = (lower && !wide && m == n) ? 1 : 0;
  if (!a.tri)
    a.ntiles = a.tiles_m * a.tiles_n;
  else if (!pair)
    a.ntiles = a.tiles_m * (a.tiles_m + 1) / 2;
  else   // row pair r < tiles_m - 1 holds 2r + 2 tiles reaching the diagonal, the last one tiles_n
    a.ntiles = (a.tiles_m - 1) * a.tiles_m + a.tiles_n;
  a.mode = mode;
  a.levels = levels;
  a.ldl = ldl;
  a.ldl_plane = ldl_plane;
  a.status = h->d_status;
  a.wait_limit = h->wait_limit;

  size_t smem = 0;
  const int stages = gemm_stages(wide, s, pair, &smem);
  if (stages < 2) return set_error(h, EMUL_NOT_SUPPORTED, "slice tiles do not fit in shared memory");
  const int units = pair ? h->nsm / 2 : h->nsm;   // CTAs, or CTA pairs
  const int grid = (a.ntiles < units ? a.ntiles : units) * (pair ? 2 : 1);
  emul_handle_s::ProfRec rec{};
  if (h->prof) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t ev;
      if (!h->event_pool.empty()) {
        ev = h->event_pool.back();
        h->event_pool.pop_back();
      } else if (cudaEventCreate(&ev) != cudaSuccess) {
        return set_error(h, EMUL_CUDA_ERROR, "event creation failed");
      }
      (i == 0 ? rec.e0 : rec.e1) = ev;
    }
    // slice pairs kept: those of the levels L = 2..t (s(s+1)/2 at t = s + 1)
    double P = 0.0;
    for (int L = 2; L <= t; ++L) P += PairSet{s_a, s_b}.count(L);
    const double cells = lower ? 0.5 * m * (double)n : static_cast<double>(m) * n;
    rec.flops = 2.0 * cells * k * P;
    rec.bytes = cells * (beta != 0.0 ? 16.0 : 8.0) + static_cast<double>(s) * 2.0 * k * (m + (same ? 0 : n));
    cudaEventRecord(rec.e0, h->stream);
  }
  rc = check_cuda(h, launch_gemm(h->stream, wide, pair, tmA, tmB, a, grid, stages, smem), "gemm kernel");
  h->launches++;
  if (h->prof) {
    cudaEventRecord(rec.e1, h->stream);
    h->recs.push_back(rec);
  }
  return rc;
}

}  // namespace emul

using emul::Operand;

namespace emul {

namespace {
bool pool_event(emul_handle_t h, cudaEvent_t* ev) {
  if (!h->event_pool.empty()) {
    *ev = h->event_pool.back();
    h->event_pool.pop_back();
    return true;
  }
  return cudaEventCreate(ev) == cudaSuccess;
}
}  // namespace

int phase_begin(emul_handle_t h, int kind) {
  if (!h->prof) return -1;
  emul_handle_s::PhaseRec r{kind, nullptr, nullptr};
  if (!pool_event(h, &r.e0)) return -1;
  if (!pool_event(h, &r.e1)) {
    h->event_pool.push_back(r.e0);
    return -1;
  }
  cudaEventRecord(r.e0, h->stream);
  h->phases.push_back(r);
  return static_cast<int>(h->phases.size()) - 1;
}

void phase_end(emul_handle_t h, int idx) {
  if (idx >= 0 && idx < static_cast<int>(h->phases.size())) cudaEventRecord(h->phases[idx].e1, h->stream);
}

}  // namespace emul

extern "C" {

int emul_create(emul_handle_t* handle, void* stream) {
  if (!handle) return EMUL_INVALID_ARG;
  *handle = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EMUL_CUDA_ERROR;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return EMUL_CUDA_ERROR;
  if (prop.major != 10 || prop.minor != 3) return EMUL_NOT_SUPPORTED;
  auto* h = new emul_handle_s();
  h->stream = static_cast<cudaStream_t>(stream);
  h->device = dev;
  h->nsm = prop.multiProcessorCount;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &h->encode_fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !h->encode_fn) {
    delete h;
    return EMUL_CUDA_ERROR;
  }
  if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess) {
    delete h;
    return EMUL_NO_WORKSPACE;
  }
  cudaMemset(h->d_status, 0, sizeof(int));
  *handle = h;
  return EMUL_OK;
}

int emul_destroy(emul_handle_t h) {
  if (!h) return EMUL_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  for (auto& kv : h->sched_cache) cudaFree(kv.second.sched);
  for (auto& r : h->recs) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (auto& r : h->phases) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (auto ev : h->event_pool) cudaEventDestroy(ev);
  if (h->aux) {
    cudaStreamSynchronize(h->aux);
    cudaStreamDestroy(h->aux);
  }
  if (h->aux_start) cudaEventDestroy(h->aux_start);
  if (h->aux_done) cudaEventDestroy(h->aux_done);
  emul::selector_free(h);
  emul::batched_free(h);
  if (h->ws) cudaFree(h->ws);
  if (h->d_status) cudaFree(h->d_status);
  delete h;
  return EMUL_OK;
}

int emul_set_stream(emul_handle_t h, void* stream) {
  if (!h) return EMUL_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return EMUL_OK;
}

const char* emul_last_error(emul_handle_t h) { return h ? h->last_error.c_str() : "null handle"; }

int emul_sync_status(emul_handle_t h) {
  if (!h) return EMUL_INVALID_ARG;
  int rc = emul::check_cuda(h, cudaStreamSynchronize(h->stream), "stream synchronize");
  if (rc) return rc;
  int st = 0;
  rc = emul::check_cuda(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (rc) return rc;
  cudaMemset(h->d_status, 0, sizeof(int));
  if (st != 0) return emul::set_error(h, st, "a device-side wait gave up");
  return EMUL_OK;
}

size_t emul_workspace_bytes(emul_handle_t h) { return h ? h->ws_bytes : 0; }

int emul_profile_enable(emul_handle_t h, int enable) {
  if (!h) return EMUL_INVALID_ARG;
  h->prof = enable != 0;
  return EMUL_OK;
}

int emul_profile_read(emul_handle_t h, emul_profile* out) {
  if (!h || !out) return EMUL_INVALID_ARG;
  int rc = emul::check_cuda(h, cudaStreamSynchronize(h->stream), "stream synchronize");
  if (rc) return rc;
  emul_profile p{};
  p.kernel_launches = h->launches;
  for (auto& r : h->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    p.product_launches++;
    p.product_ms += ms;
    p.product_tensor_flops += r.flops;
    p.product_bytes += r.bytes;
    h->event_pool.push_back(r.e0);
    h->event_pool.push_back(r.e1);
  }
  h->recs.clear();
  for (auto& r : h->phases) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess && r.kind >= 0 && r.kind < 5) p.phase_ms[r.kind] += ms;
    h->event_pool.push_back(r.e0);
    h->event_pool.push_back(r.e1);
  }
  h->phases.clear();
  h->launches = 0;
  *out = p;
  return EMUL_OK;
}

int emul_schedule(int slices, int k, int wide, int level_sums, int threshold, int* sweeps, int cap_sweeps,
                  unsigned char* table, int cap_table, int* meta) {
  using namespace emul;
  if (slices < 1 || slices > kMaxSlices || k < 1 || !meta) return EMUL_INVALID_ARG;
  if (threshold != 0 && (threshold < 2 || threshold > 2 * slices)) return EMUL_INVALID_ARG;
  const int nch = (k + kBK - 1) / kBK;
  std::vector<Sweep> v;
  std::vector<uint8_t> tab;
  int njobs = 0, t0 = 0, period = 0;
  if (!build_schedule(slices, nch, wide != 0, level_sums != 0, v, tab, njobs, t0, period, threshold))
    return EMUL_INVALID_ARG;
  meta[0] = static_cast<int>(v.size());
  meta[1] = njobs;
  meta[2] = t0;
  meta[3] = period;
  meta[4] = static_cast<int>(tab.size());
  if (!sweeps || !table || cap_sweeps < static_cast<int>(v.size()) || cap_table < static_cast<int>(tab.size()))
    return EMUL_INVALID_ARG;
  for (size_t i = 0; i < v.size(); ++i) {
    const Sweep& w = v[i];
    const int row[EMUL_SWEEP_INTS] = {w.k0c,   w.k1c,      w.L[0],     w.L[1],    w.pb[0], w.pb[1],
                                      w.pe[0], w.pe[1],    w.flags[0], w.flags[1], w.nplanes, w.kcs};
    for (int j = 0; j < EMUL_SWEEP_INTS; ++j) sweeps[i * EMUL_SWEEP_INTS + j] = row[j];
  }
  std::memcpy(table, tab.data(), tab.size());
  return EMUL_OK;
}

int emul_split(emul_handle_t h, int rows, int k, const double* X, long rs, long cs, int slices, int32_t* exps,
               uint16_t* slice_out, long ldk) {
  if (!h) return EMUL_INVALID_ARG;
  if (rows < 0 || k < 0 || slices < 1 || slices > emul::kMaxSlices || ldk < k || ldk % 8 != 0 ||
      (rs != 1 && cs != 1) || (rows > 0 && (!X || !exps || !slice_out)))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_split: invalid argument");
  h->launches++;
  return emul::check_cuda(h, emul::launch_split(h->stream, rows, k, X, rs, cs, slices, exps, slice_out, ldk),
                          "split");
}

int emul_level_sums(emul_handle_t h, int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                    int slices, int32_t* levels, int ldl, long ldl_plane) {
  if (!h) return EMUL_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0 || slices < 1 || slices > emul::kMaxSlices || lda < (m > 1 ? m : 1) ||
      ldb < (k > 1 ? k : 1) || ldl < (m > 1 ? m : 1) || ldl_plane < static_cast<long>(ldl) * n || !levels ||
      k > 16384 * 4)
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_level_sums: invalid argument");
  return emul::gemm_run(h, m, n, k, 1.0, Operand{A, 1, lda}, Operand{B, ldb, 1}, 0.0, nullptr, 0, slices, false, 1,
                        levels, ldl, ldl_plane);
}

int emul_dgemm_threshold(emul_handle_t h, int m, int n, int k, double alpha, const double* A, int lda,
                         const double* B, int ldb, double beta, double* C, int ldc, int slices, int threshold) {
  if (!h) return EMUL_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0 || slices < 1 || slices > emul::kMaxSlices || lda < (m > 1 ? m : 1) ||
      ldb < (k > 1 ? k : 1) || ldc < (m > 1 ? m : 1) || (m > 0 && n > 0 && !C) ||
      (m > 0 && n > 0 && k > 0 && (!A || !B)) || k > 16384 * 4 ||
      (threshold != 0 && (threshold < 2 || threshold > 2 * slices)))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_dgemm: invalid argument");
  return emul::gemm_run(h, m, n, k, alpha, Operand{A, 1, lda}, Operand{B, ldb, 1}, beta, C, ldc, slices, false, 0,
                        nullptr, 0, 0, 0, threshold);
}

int emul_dgemm(emul_handle_t h, int m, int n, int k, double alpha, const double* A, int lda, const double* B,
               int ldb, double beta, double* C, int ldc, int slices) {
  return emul_dgemm_threshold(h, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, 0);
}

int emul_dgemm_unequal(emul_handle_t h, int m, int n, int k, double alpha, const double* A, int lda,
                       const double* B, int ldb, double beta, double* C, int ldc, int slices_a, int slices_b,
                       int threshold) {
  if (!h) return EMUL_INVALID_ARG;
  const int s = slices_a > slices_b ? slices_a : slices_b;
  if (m < 0 || n < 0 || k < 0 || slices_a < 1 || slices_b < 1 || s > emul::kMaxSlices || lda < (m > 1 ? m : 1) ||
      ldb < (k > 1 ? k : 1) || ldc < (m > 1 ? m : 1) || (m > 0 && n > 0 && !C) ||
      (m > 0 && n > 0 && k > 0 && (!A || !B)) || k > 16384 * 4 ||
      (threshold != 0 && (threshold < 2 || threshold > slices_a + slices_b)))
    return emul::set_error(h, EMUL_INVALID_ARG, "emul_dgemm_unequal: invalid argument");
  return emul::gemm_run(h, m, n, k, alpha, Operand{A, 1, lda}, Operand{B, ldb, 1}, beta, C, ldc, s, false, 0, nullptr,
                        0, 0, 0, threshold, slices_a, slices_b);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// emul_dgemm_noalloc: the emulated DGEMM for callers that cannot allocate
// device memory: a host library whose device memory belongs to another
// allocator (a framework's caching allocator, a pool sized at start-up), or a
// latency-bound loop that must not call cudaMalloc / cudaFree (both can
// synchronise the whole device).  All scratch lives in one file-scope device
// array of kNoAllocScratchBytes that every GPU which loads this library keeps
// until the process exits.
namespace emul {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr size_t kNoAllocSchedBytes = 16384;                // sweeps (16 B each) and the slot table
constexpr int kNoAllocMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
  int nsm = 0;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
void* g_noalloc_encode = nullptr;
std::mutex g_noalloc_mu;

// One-time set-up per device, with that device current: the device address of
// the static scratch (host code must not use the symbol itself) and the
// tensor-map encoder.
int noalloc_setup(int dev, NoAllocDevice** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.base) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return EMUL_CUDA_ERROR;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return EMUL_CUDA_ERROR;
    if (!g_noalloc_encode) {
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &g_noalloc_encode, 12000, cudaEnableDefault,
                                           &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !g_noalloc_encode)
        return EMUL_CUDA_ERROR;
    }
    d.base = static_cast<unsigned char*>(ptr);
    d.nsm = nsm;
  }
  *out = &d;
  return EMUL_OK;
}

int noalloc_map(CUtensorMap* map, const uint16_t* base, int rows, int k, long kpad, int s, int box_rows) {
  auto fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(g_noalloc_encode);
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(s)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(kpad) * 2, static_cast<cuuint64_t>(kpad) * 2 * rows};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
             ? EMUL_OK
             : EMUL_CUDA_ERROR;
}

}  // namespace
}  // namespace emul

extern "C" int emul_dgemm_noalloc(void* stream, int m, int n, int k, double alpha, const double* A, int lda,
                                  const double* B, int ldb, double beta, double* C, int ldc, int slices) {
  using namespace emul;
  if (m < 0 || n < 0 || k < 0 || slices < 1 || slices > kMaxSlices || lda < (m > 1 ? m : 1) ||
      ldb < (k > 1 ? k : 1) || ldc < (m > 1 ? m : 1) || (m > 0 && n > 0 && !C) ||
      (m > 0 && n > 0 && k > 0 && (!A || !B)) || k > 16384 * 4)
    return EMUL_INVALID_ARG;
  if (m == 0 || n == 0) return EMUL_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return EMUL_CUDA_ERROR;
  NoAllocDevice* d = nullptr;
  int rc = noalloc_setup(dev, &d);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (k == 0) {
    scale_c_kernel<<<1024, 256, 0, st>>>(m, n, alpha, beta, C, ldc);
    return cudaGetLastError() == cudaSuccess ? EMUL_OK : EMUL_CUDA_ERROR;
  }
  // scratch layout: status word | schedule | row scales | column scales | slices of A | slices of B
  const long kp = kpad_of(k);
  const size_t off_sched = kAlign;
  const size_t off_ea = off_sched + kNoAllocSchedBytes;
  const size_t off_fb = off_ea + align_up(static_cast<size_t>(m) * 4);
  const size_t off_sa = off_fb + align_up(static_cast<size_t>(n) * 4);
  const size_t off_sb = off_sa + align_up(static_cast<size_t>(slices) * m * kp * 2);
  const size_t need = off_sb + align_up(static_cast<size_t>(slices) * n * kp * 2);
  if (need > kNoAllocScratchBytes) return EMUL_NO_WORKSPACE;   // operands exceed the 16 MiB static scratch

  unsigned char* base = d->base;
  int* status = reinterpret_cast<int*>(base);
  Sweep* sched = reinterpret_cast<Sweep*>(base + off_sched);
  int32_t* ea = reinterpret_cast<int32_t*>(base + off_ea);
  int32_t* fb = reinterpret_cast<int32_t*>(base + off_fb);
  uint16_t* sa = reinterpret_cast<uint16_t*>(base + off_sa);
  uint16_t* sb = reinterpret_cast<uint16_t*>(base + off_sb);

  const bool wide = !narrow_ok(slices, k);
  const int nch = (k + kBK - 1) / kBK;
  std::vector<Sweep> v;
  std::vector<uint8_t> tab;
  SlotPlan plan{};
  if (!build_schedule(slices, nch, wide, false, v, tab, plan.njobs, plan.t0, plan.period)) return EMUL_INVALID_ARG;
  const size_t off_tab = (v.size() * sizeof(Sweep) + 15) / 16 * 16;
  if (off_tab + tab.size() > kNoAllocSchedBytes) return EMUL_NO_WORKSPACE;
  std::vector<uint8_t> blob(off_tab + tab.size(), 0);
  std::memcpy(blob.data(), v.data(), v.size() * sizeof(Sweep));
  std::memcpy(blob.data() + off_tab, tab.data(), tab.size());
  plan.tab = reinterpret_cast<const uint8_t*>(sched) + off_tab;
  // the status word must start at zero; the rest is fully rewritten by this call
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return EMUL_CUDA_ERROR;
  if (cudaMemcpyAsync(sched, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return EMUL_CUDA_ERROR;
  if (launch_split(st, m, k, A, 1, lda, slices, ea, sa, kp) != cudaSuccess) return EMUL_CUDA_ERROR;
  if (launch_split(st, n, k, B, ldb, 1, slices, fb, sb, kp) != cudaSuccess) return EMUL_CUDA_ERROR;
  const int BN = wide ? 64 : 128;
  CUtensorMap tmA, tmB;
  rc = noalloc_map(&tmA, sa, m, k, kp, slices, 128);
  if (rc) return rc;
  rc = noalloc_map(&tmB, sb, n, k, kp, slices, BN);
  if (rc) return rc;
  GemmArgs a{};
  a.M = m;
  a.N = n;
  a.K = k;
  a.s = slices;
  a.t = slices + 1;
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.ea = ea;
  a.fb = fb;
  a.sched = sched;
  a.nsweeps = static_cast<int>(v.size());
  a.slots = plan;
  a.tiles_m = (m + 127) / 128;
  a.tiles_n = (n + BN - 1) / BN;
  a.ntiles = a.tiles_m * a.tiles_n;
  a.status = status;
  a.wait_limit = 2000000000LL;
  const size_t stage = gemm_stage_bytes(wide, slices, false);
  int stages = static_cast<int>((232448 - 1024 - 2048) / stage);
  if (stages > kMaxStagesCfg) stages = kMaxStagesCfg;
  if (stages < 2) return EMUL_NOT_SUPPORTED;
  const int grid = a.ntiles < d->nsm ? a.ntiles : d->nsm;
  return launch_gemm(st, wide, false, tmA, tmB, a, grid, stages, stages * stage + 1024) == cudaSuccess ? EMUL_OK
                                                                                             : EMUL_CUDA_ERROR;
}

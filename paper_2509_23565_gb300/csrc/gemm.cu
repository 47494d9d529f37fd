// Slice-pair products on tcgen05 tensor cores with the fused exact
// recombination and C update (arXiv 2509.23565, Section 2, Eq. 2 with the
// truncation threshold t; Section 4, Eq. 7 when alpha = -1, beta = 1).
//
// For an output tile (128 rows x BN columns) the level sums
//   I_L = sum_{p+q=L} SA_p SB_q^T,  L = 2..t,
// are accumulated in TMEM as FP32.  The slices are integers |S| <= 127 held as
// BF16, so every product and every partial sum is an integer; an accumulator
// never receives more than 1040 * 127^2 < 2^24 in magnitude (the schedule
// splits K where needed), so the FP32 sums are exact.  The epilogue converts
// each drained level sum exactly to an integer and adds it with its weight,
// R += I_L 2^(7(t-L)) (int64, or 128-bit for the wide variant), so the levels
// may be drained in any order; the schedule issues the longest jobs (the
// highest levels) first and level 2 last.  The exact value
// T = sum_L I_L 2^(7(t-L)) is rounded once to FP64,
//   D = RN(T * 2^(e_i + f_j - 7t)),
// in integer arithmetic, and C = RN(RN(alpha D) + RN(beta C))
// is written straight back.  For the Schur update (alpha = -1, beta = 1) the
// epilogue does not read C: it issues red.global.add.f64 of -D, an FP64 add
// rounded to nearest that L2 performs, so the C update costs no load latency
// and no FP64 instruction on the SM (GB300 retires ~1.6 per clock per SM).
//
// Warp roles (640 threads): warp 0 issues TMA loads of the slice tiles of each
// K chunk into a ring of shared-memory stages; warp 1 owns TMEM (4 accumulator
// slots); warps 1 and 2 issue the MMAs, one job of a sweep each; both loops run
// on the whole warp (warp-uniform operands, one elected lane issues: a lone
// thread recomputing descriptors issues an MMA only every ~84 cycles, short of
// the 64 a 128 x 128 x 16 MMA takes); warps 4-19 drain the slots and write C.  The
// first warpgroup gives registers to the epilogue warpgroups (setmaxnreg).  A sweep
// of one or two jobs shares the staged tiles of a chunk; each job's TMEM slot
// (and the parity of its barriers) comes from a host-planned slot table, so the
// issuer fills slots while the epilogue drains others.  All waits are bounded.
//
// With more than 128 rows the blocks run as CTA pairs (clusters of two,
// cta_group::2, the PAIR instantiation): a pair owns a 256 x BN tile, each CTA
// stages its 128 rows of A and half of B's rows, rank 0 issues M = 256 MMAs
// that read both CTAs' tiles, and its commits reach the barriers of both; each
// CTA drains its own TMEM.  Each SM then stages a quarter fewer bytes.
#include <cstdint>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "emul_internal.h"
#include "ptx.cuh"
#include "round.cuh"

namespace emul {

namespace {

constexpr int kThreads = 640;          // 5 warpgroups: producer/MMA, 4 x epilogue
constexpr int kMmaWarps = 2;            // warps 1 .. kMmaWarps issue MMAs
constexpr int kLaunchRegs = 96;         // 640 x 96 = 61440 registers at launch
constexpr int kLowRegs = 64;            // producer warpgroup after setmaxnreg.dec
constexpr int kHighRegs = 104;          // epilogue warpgroups: 128*64 + 512*104 = 61440
constexpr int kSlots = 4;
constexpr int kEpiWarps = 16;
constexpr int kSchedSmem = 64;
constexpr int kTabSmem = 256;
constexpr int kMaxStages = kMaxStagesCfg;
constexpr uint32_t kRowBytes = kBK * 2;     // one K-major row of a staged tile
constexpr uint32_t kSwizzleCode = kRowBytes == 64 ? 4u : 6u;   // descriptor code of SWIZZLE_64B / _32B
constexpr int kStatusTimeout = -4;

template <bool WIDE>
struct Cfg {
  static constexpr int BM = 128;
  static constexpr int BN = WIDE ? 64 : 128;
  static constexpr int CPT = BN / 4;                  // columns per epilogue thread
  static constexpr uint32_t A_TILE = BM * kBK * 2;    // bytes
  static constexpr uint32_t B_TILE = BN * kBK * 2;
  static constexpr uint32_t TMEM_COLS = kSlots * BN;
  using State = typename std::conditional<WIDE, __int128, long long>::type;
};

// I 2^w in the state's width (the shift is done unsigned: I may be negative).
template <typename State>
__device__ __forceinline__ State shl_state(int I, int w);
template <>
__device__ __forceinline__ long long shl_state<long long>(int I, int w) {
  return (long long)((unsigned long long)(long long)I << w);
}
template <>
__device__ __forceinline__ __int128 shl_state<__int128>(int I, int w) {
  return (__int128)((unsigned __int128)(__int128)I << w);
}

// |I 2^w| <= 2^62 for lim = min(62 - w, 31): I >> lim is 0 or -1 exactly then.
__device__ __forceinline__ bool term_fits(int I, int lim) { return lim >= 31 || (I >> lim) == (I >> 31); }

// RN(x * 2^sh) for a 64-bit integer x, in integer arithmetic only and without
// branches (the lanes of a warp hold unrelated values), valid for
// -1022 <= sh <= 960: every |x| < 2^64 then gives a normal result (or, after a
// carry, the top binade).  |x| is normalised so that its leading one sits at
// bit 63, its top 53 bits are kept and rounded to nearest even with bit 10 as
// the round bit and bits 0-9 as the sticky bits; a carry out of the mantissa
// moves into the exponent field.
__device__ __forceinline__ double rn_x64(long long x, int sh) {
  const unsigned long long sgn = (unsigned long long)(x >> 63);      // 0 or all ones
  const unsigned long long a = ((unsigned long long)x ^ sgn) - sgn;   // |x|
  const int lz = __clzll((long long)a);
  const unsigned long long m = a << (lz & 63);
  unsigned long long q = m >> 11;
  const unsigned long long rb = (m >> 10) & 1ull;
  const unsigned long long st = (m & 0x3FFull) ? 1ull : 0ull;
  q += rb & (st | (q & 1ull));
  const unsigned long long bits = ((unsigned long long)(63 - lz + sh + 1022) << 52) + q;
  return a ? __longlong_as_double((long long)(bits | (sgn << 63))) : 0.0;
}

// D of a 64-bit exact sum x: the branchless path when sh keeps every result
// normal, else the general one.
__device__ __forceinline__ double rn_sum64(long long x, int sh) {
  if (sh >= -1022 && sh <= 960) return rn_x64(x, sh);
  return rn_scaled((__int128)x, sh);
}

// C <- RN(C + v) as a reduction in L2 (fire and forget: no load of C, no FP64
// instruction on the SM).  The FP64 add of red.global rounds to nearest even;
// each element of C is updated by exactly one thread of one launch.
__device__ __forceinline__ void red_add_f64(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ int f2i(uint32_t r) { return __float2int_rn(__uint_as_float(r)); }

__device__ __forceinline__ double neg_d(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}


// D = RN(T * 2^(e + f - 7t)) (NaN for a non-finite scale), then
// out = RN(RN(alpha D) + RN(beta C)); alpha = +-1 and beta in {0, 1} skip the
// exact multiplications.
// Update modes of C: kSub: C - D (alpha = -1, beta = 1); kSet: D (alpha = 1,
// beta = 0); kGeneral: RN(RN(alpha D) + RN(beta C)) (beta = 0: RN(alpha D)).
enum UpdMode { kGeneral = 0, kSub = 1, kSet = 2 };

template <int UPD>
__device__ __forceinline__ double apply_update(const GemmArgs& a, double D, double c_old) {
  if (UPD == kSub) return __dadd_rn(c_old, neg_d(D));
  if (UPD == kSet) return D;
  const double ad = __dmul_rn(a.alpha, D);
  if (a.beta == 0.0) return ad;
  return __dadd_rn(ad, __dmul_rn(a.beta, c_old));
}

__device__ __forceinline__ void tile_coords(const GemmArgs& a, int tile, int& tm, int& tn) {
  if (a.tri) {
    // lower-triangular enumeration of square tiles: tile = tm(tm+1)/2 + tn, tn <= tm
    int r = (int)((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
    while ((long)r * (r + 1) / 2 > tile) --r;
    while ((long)(r + 1) * (r + 2) / 2 <= tile) ++r;
    tm = r;
    tn = tile - r * (r + 1) / 2;
  } else {
    tm = tile % a.tiles_m;
    tn = tile / a.tiles_m;
  }
}

// Tiles of a CTA pair: 256 rows (128 per CTA) x BN columns; tiles_m counts
// 256-row tiles.  The lower-triangular enumeration keeps the tiles that reach
// the diagonal: row pair r holds min(2r + 2, tiles_n) of them.
__device__ __forceinline__ void tile_coords_pair(const GemmArgs& a, int tile, int& tm, int& tn) {
  if (a.tri) {
    const int full = (a.tiles_m - 1) * a.tiles_m;   // row pairs before the last: r (r + 1) tiles before row pair r
    if (tile >= full) {
      tm = a.tiles_m - 1;
      tn = tile - full;
      return;
    }
    int r = (int)((sqrtf(4.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
    while ((long)r * (r + 1) > tile) --r;
    while ((long)(r + 1) * (r + 2) <= tile) ++r;
    tm = r;
    tn = tile - r * (r + 1);
  } else {
    tm = tile % a.tiles_m;
    tn = tile / a.tiles_m;
  }
}

__device__ __forceinline__ bool aborted(volatile int* flag) { return *flag != 0; }

// Slot-table row of the i-th tile of this CTA.
__device__ __forceinline__ const uint8_t* slot_row(const uint8_t* tab, const SlotPlan& sp, long i) {
  const long ph = i < sp.t0 ? i : sp.t0 + (i - sp.t0) % sp.period;
  return tab + ph * sp.njobs;
}

__device__ __forceinline__ void raise_timeout(const GemmArgs& a, volatile int* flag) {
  atomicExch(a.status, kStatusTimeout);
  *flag = 1;
}

}  // namespace

// PAIR: a cluster of two CTAs per tile of 256 x BN (cta_group::2).  Each
// CTA stages its 128 rows of A and BN/2 rows of B; both CTAs' copies complete
// on rank 0's stage barrier; rank 0's MMA warps issue M = 256 MMAs whose
// commits reach both CTAs; each CTA drains its own TMEM and both release a
// slot on rank 0's barrier.  Rank 1's MMA warps stay idle.
template <bool WIDE, int UPD, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs a,
                int stages) {
  static_assert(!(WIDE && PAIR), "CTA pairs use the 128-column tile");
  using Cf = Cfg<WIDE>;
  using State = typename Cf::State;
  constexpr uint32_t B_T = PAIR ? Cf::B_TILE / 2 : Cf::B_TILE;   // bytes of one staged B plane
  constexpr int G = PAIR ? 2 : 1;                                  // CTAs per tile
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t stage_full[kMaxStages], stage_empty[kMaxStages];
  __shared__ __align__(8) uint64_t slot_full[kSlots], slot_empty[kSlots], mma_done[kMmaWarps];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ Sweep sched_s[kSchedSmem];   // the schedule, when it is short enough
  __shared__ uint8_t tab_s[kTabSmem];     // the slot table, when it is short enough

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = a.s;
  const uint32_t stage_bytes = (uint32_t)s * (Cf::A_TILE + B_T);
  volatile int* abortp = &abort_flag;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const int cta0 = (int)blockIdx.x / G, ncta = (int)gridDim.x / G;   // tile loop over CTAs or CTA pairs

  const bool sched_in_smem = a.nsweeps <= kSchedSmem;
  if (sched_in_smem)
    for (int i = threadIdx.x; i < a.nsweeps; i += blockDim.x) sched_s[i] = a.sched[i];
  const Sweep* sched = sched_in_smem ? sched_s : a.sched;
  const int ntab = (a.slots.t0 + a.slots.period) * a.slots.njobs;
  const bool tab_in_smem = ntab <= kTabSmem;
  if (tab_in_smem)
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) tab_s[i] = a.slots.tab[i];
  const uint8_t* tab = tab_in_smem ? tab_s : a.slots.tab;
  if (threadIdx.x == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(&stage_full[i], 1);
      mbar_init(&stage_empty[i], kMmaWarps);   // one commit per issuing warp
    }
    for (int i = 0; i < kSlots; ++i) {
      mbar_init(&slot_full[i], 1);
      mbar_init(&slot_empty[i], G * kEpiWarps);
    }
    for (int i = 0; i < kMmaWarps; ++i) mbar_init(&mma_done[i], 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    if (PAIR)
      tmem_alloc_pair(&tmem_base, Cf::TMEM_COLS);
    else
      tmem_alloc(&tmem_base, Cf::TMEM_COLS);
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();   // barriers of both CTAs initialised before any copy or arrival
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kLowRegs));
  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    // the whole warp runs the loop (warp-uniform values); one elected lane issues
    if (lane == 0) {
      prefetch_tmap(&tmA);
      prefetch_tmap(&tmB);
    }
    __syncwarp();
    long it = 0;
    bool ok = true;
    for (int tile = cta0; tile < a.ntiles && ok; tile += ncta) {
      int tm, tn;
      if (PAIR)
        tile_coords_pair(a, tile, tm, tn);
      else
        tile_coords(a, tile, tm, tn);
      const int m0 = (tm * G + (int)rank) * Cf::BM, n0 = tn * Cf::BN + (int)rank * (Cf::BN / G);
      for (int sw = 0; sw < a.nsweeps && ok; ++sw) {
        const Sweep S = sched[sw];
        const int np = S.nplanes;
        for (int kc = S.k0c; kc < S.k1c; kc += S.kcs, ++it) {
          const int nu = S.k1c - kc < S.kcs ? S.k1c - kc : S.kcs;
          const int st = (int)(it % stages);
          const uint32_t par = (uint32_t)((it / stages) & 1) ^ 1u;
          if (aborted(abortp) || !mbar_wait_warp(&stage_empty[st], par, a.wait_limit)) {
            if (!aborted(abortp) && lane == 0) raise_timeout(a, abortp);
            ok = false;
            break;
          }
          uint8_t* base = smem + (size_t)st * stage_bytes;
          if (!PAIR) {
            mbar_arrive_expect_tx_elect(&stage_full[st], (uint32_t)(nu * np) * (Cf::A_TILE + B_T));
            for (int u = 0; u < nu; ++u)
              for (int p = 0; p < np; ++p) {
                const int t = u * np + p;
                tma_load_3d_elect(base + t * Cf::A_TILE, &tmA, &stage_full[st], (kc + u) * kBK, m0, p);
                tma_load_3d_elect(base + s * Cf::A_TILE + t * B_T, &tmB, &stage_full[st], (kc + u) * kBK, n0, p);
              }
          } else {
            // rank 0's barrier counts the bytes of both CTAs (a copy of rank 1
            // may land before rank 0 announces them: the phase still waits for
            // rank 0's arrival)
            if (rank == 0)
              mbar_arrive_expect_tx_elect(&stage_full[st], (uint32_t)(G * nu * np) * (Cf::A_TILE + B_T));
            const uint32_t bar0 = mapa_rank(&stage_full[st], 0);
            for (int u = 0; u < nu; ++u)
              for (int p = 0; p < np; ++p) {
                const int t = u * np + p;
                tma_load_3d_pair_elect(base + t * Cf::A_TILE, &tmA, bar0, (kc + u) * kBK, m0, p);
                tma_load_3d_pair_elect(base + s * Cf::A_TILE + t * B_T, &tmB, bar0, (kc + u) * kBK, n0, p);
              }
          }
        }
      }
    }
    if (!ok && rank == 0) {
      // wait (bounded) for the copies still in flight before the block exits
      // (a pair's copies all complete on rank 0's barriers)
      for (long j = (it - stages > 0 ? it - stages : 0); j < it; ++j)
        mbar_wait(&stage_full[j % stages], (uint32_t)((j / stages) & 1), a.wait_limit / 8);
    }
  } else if (warp >= 1 && warp <= kMmaWarps && rank == 0) {
    // ------------------------------------------------------------ MMA issuers
    // the whole warp runs the loop (warp-uniform values); one elected lane issues
    const int myj = warp - 1;   // job of each sweep issued by this warp
    {
      constexpr uint32_t idesc = idesc_bf16_f32(128 * G, Cf::BN);
      long it = 0, tloc = 0;
      bool ok = true;
      for (int tile = cta0; tile < a.ntiles && ok; tile += ncta, ++tloc) {
        const uint8_t* srow = slot_row(tab, a.slots, tloc);
        int jj = 0;
        for (int sw = 0; sw < a.nsweeps && ok; ++sw) {
          const Sweep S = sched[sw];
          const int nj = S.L[1] ? 2 : 1;
          const bool mine = myj < nj;   // this warp has a job in the sweep
          int slot = 0;
          uint32_t dcol = 0;
          if (mine) {
            const uint32_t e = srow[jj + myj];
            slot = (int)(e & 3u);
            dcol = tmem + (uint32_t)(slot * Cf::BN);
            const uint32_t spar = ((e >> 2) & 1u) ^ 1u;
            if (aborted(abortp) || !(PAIR ? mbar_wait_cluster_warp(&slot_empty[slot], spar, a.wait_limit)
                                          : mbar_wait_warp(&slot_empty[slot], spar, a.wait_limit))) {
              if (!aborted(abortp) && lane == 0) raise_timeout(a, abortp);
              ok = false;
              break;
            }
          }
          tc_fence_after();
          const int np = S.nplanes;
          for (int kc = S.k0c; kc < S.k1c; kc += S.kcs, ++it) {
            const int nu = S.k1c - kc < S.kcs ? S.k1c - kc : S.kcs;
            const int st = (int)(it % stages);
            if (aborted(abortp) || !mbar_wait_warp(&stage_full[st], (uint32_t)((it / stages) & 1), a.wait_limit)) {
              if (!aborted(abortp) && lane == 0) raise_timeout(a, abortp);
              ok = false;
              break;
            }
            tc_fence_after();
            // descriptors of the stage's first A and B tiles; a tile or a K=16
            // step further is a plain add on the start-address field (addr >> 4,
            // 14 bits, no carry: shared memory addresses stay below 256 KB)
            const uint32_t base = smem_u32(smem + (size_t)st * stage_bytes);
            const uint64_t dA0 = umma_desc(base, kRowBytes, kSwizzleCode);
            const uint64_t dB0 = umma_desc(base + (uint32_t)s * Cf::A_TILE, kRowBytes, kSwizzleCode);
            for (int u = 0; u < nu && mine; ++u) {
              const int L = S.L[myj];
              const int pb = S.pb[myj];
              const int pe = S.pe[myj];
              const bool first = kc + u == S.k0c;
              for (int p = pb; p <= pe; ++p) {
                const int q = L - p;
                const uint64_t da = dA0 + (uint64_t)((u * np + p - 1) * (Cf::A_TILE >> 4));
                const uint64_t db = dB0 + (uint64_t)((u * np + q - 1) * (B_T >> 4));
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                  const uint32_t acc = (!first || p != pb || kk != 0) ? 1u : 0u;
                  if (PAIR)
                    mma_bf16_pair_elect(dcol, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, acc);
                  else
                    mma_bf16_elect(dcol, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, acc);
                }
              }
            }
            // also by a warp without a job here: the stage needs both
            if (PAIR)
              mma_commit_pair_both_elect(&stage_empty[st]);
            else
              mma_commit_elect(&stage_empty[st]);
          }
          if (!ok) break;
          if (mine) {
            if (PAIR)
              mma_commit_pair_both_elect(&slot_full[slot]);
            else
              mma_commit_elect(&slot_full[slot]);
          }
          jj += nj;
        }
      }
      // every MMA issued by this warp must be complete before TMEM is released
      if (PAIR)
        mma_commit_pair_both_elect(&mma_done[myj]);
      else
        mma_commit_elect(&mma_done[myj]);
      mbar_wait(&mma_done[myj], 0, a.wait_limit);
    }
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kHighRegs));
    // ------------------------------------------------------------ epilogue
    const int ew = warp - 4;
    const int quarter = warp & 3;      // TMEM lane quarter this warp may access
    const int half = ew >> 2;          // column group of CPT columns
    const int row_t = quarter * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    constexpr int CPT = Cf::CPT;
    const bool needs_c = (UPD == kSub) || (UPD == kGeneral && a.beta != 0.0);
    const int sh0 = -7 * a.t;
    State R[CPT];
    long tloc = 0;
    bool ok = true;
    // rank 0's slot barriers, where both CTAs of a pair release a slot
    uint32_t slot_empty0 = 0;
    if (PAIR) slot_empty0 = mapa_rank(&slot_empty[0], 0);
    auto release = [&](int slot) {
      if (PAIR)
        mbar_arrive_cluster(slot_empty0 + (uint32_t)(slot * 8));
      else
        mbar_arrive_relaxed(&slot_empty[slot]);
    };
    for (int tile = cta0; tile < a.ntiles && ok; tile += ncta, ++tloc) {
      int tm, tn;
      if (PAIR)
        tile_coords_pair(a, tile, tm, tn);
      else
        tile_coords(a, tile, tm, tn);
      const int row = (tm * G + (int)rank) * Cf::BM + row_t;
      const int col0 = tn * Cf::BN + half * CPT;
      const int e_row = row < a.M ? a.ea[row] : 0;
      // column scales of this thread's CPT columns, one per lane (broadcast by shuffle)
      int fcol[1];
      {
        const int col = col0 + lane;
        fcol[0] = (lane < CPT && col < a.N) ? a.fb[col] : 0;
      }
#pragma unroll
      for (int c = 0; c < CPT; ++c) R[c] = 0;
      const uint8_t* srow = slot_row(tab, a.slots, tloc);
      int jj = 0;
      bool final_done = false;
      for (int sw = 0; sw < a.nsweeps && ok; ++sw) {
        const Sweep S = sched[sw];
        const int nj = S.L[1] ? 2 : 1;
        for (int j = 0; j < nj && ok; ++j, ++jj) {
          const int fl = S.flags[j];
          const uint32_t e = srow[jj];
          const int slot = (int)(e & 3u);
          const uint32_t par = (e >> 2) & 1u;
          bool released = false;   // slot already released (final step, 64-bit path)
          if (aborted(abortp) || !mbar_wait(&slot_full[slot], par, a.wait_limit)) {
            if (!aborted(abortp)) raise_timeout(a, abortp);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ta = tmem + lane_addr + (uint32_t)(slot * Cf::BN + half * CPT);
          const int wsh = 7 * (a.t - S.L[j]);     // weight of the level: 2^(7(t-L))
          if (a.mode == 1) {
            // level sums out (exact int32), added so that K segments / pair groups accumulate
            const int L = S.L[j];
#pragma unroll
            for (int c16 = 0; c16 < CPT / 16; ++c16) {
              uint32_t r[16];
              tmem_ld16(ta + c16 * 16, r);
              tmem_ld_wait();
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int col = col0 + c16 * 16 + q;
                if (row < a.M && col < a.N) {
                  int32_t* lp = a.levels + (long)(L - 2) * a.ldl_plane + row + (long)col * a.ldl;
                  *lp += f2i(r[q]);
                }
              }
            }
          } else if (fl & kFinal) {
            // final step (64-bit variant): T = R + I 2^wsh, rounded once, C
            // updated in place.  R, the other levels, stays below 2^61, so T
            // fits in 64 bits when |I| 2^wsh <= 2^62.  When that holds for the
            // whole warp (it fails only for rows and columns whose leading
            // digits are near 127 of one sign along the whole K) the term is
            // added at once, the slot is released and the rounding runs while
            // the MMAs of the next tile fill it; otherwise the slot is held,
            // and the elements over the limit re-read I and round T from 128 bits.
            final_done = true;
            const bool rowok = row < a.M;
            const int lim = 62 - wsh < 31 ? 62 - wsh : 31;
            bool fits = true;
#pragma unroll
            for (int c16 = 0; c16 < CPT / 16; ++c16) {
              uint32_t r[16];
              tmem_ld16(ta + c16 * 16, r);
              tmem_ld_wait();
#pragma unroll
              for (int q = 0; q < 16; ++q) {
                const int I = f2i(r[q]);
                if (term_fits(I, lim))
                  R[c16 * 16 + q] += shl_state<State>(I, wsh);
                else
                  fits = false;
              }
            }
            fits = __all_sync(0xFFFFFFFFu, fits);
            if (fits) {
              tc_fence_before();
              __syncwarp();
              if (lane == 0) release(slot);
              released = true;
            }
            double* cp = a.C + row + (long)col0 * a.ldc;
            // a warp whose rows and columns are all inside C (no triangle, no
            // nonfinite row scale) rounds without per-element checks
            const bool interior = fits && __all_sync(0xFFFFFFFFu, rowok && e_row != kNonFinite) &&
                                  col0 + CPT <= a.N && !a.lower;
            if (interior) {
#pragma unroll
              for (int c = 0; c < CPT; ++c, cp += a.ldc) {
                const int f = __shfl_sync(0xFFFFFFFFu, fcol[0], c);
                const double D = (f == kNonFinite) ? __longlong_as_double(0x7FF8000000000000ll)
                                                   : rn_sum64((long long)R[c], e_row + f + sh0);
                if (UPD == kSub)
                  red_add_f64(cp, neg_d(D));
                else if (UPD == kSet)
                  *cp = D;
                else
                  *cp = apply_update<UPD>(a, D, needs_c ? *cp : 0.0);
              }
            } else
#pragma unroll
            for (int c4 = 0; c4 < CPT / 4; ++c4) {
              uint32_t r[4] = {0u, 0u, 0u, 0u};
              if (!fits) {            // warp-uniform
                tmem_ld4(ta + c4 * 4, r);
                tmem_ld_wait();
              }
#pragma unroll
              for (int q = 0; q < 4; ++q, cp += a.ldc) {
                const int c = c4 * 4 + q;
                const int col = col0 + c;
                const int f = __shfl_sync(0xFFFFFFFFu, fcol[0], c);
                if (!rowok || col >= a.N || (a.lower && row < col)) continue;
                const int I = f2i(r[q]);
                const int sh = e_row + f + sh0;
                double D;
                if (e_row == kNonFinite || f == kNonFinite)
                  D = __longlong_as_double(0x7FF8000000000000ll);
                else if (fits || term_fits(I, lim))
                  D = rn_sum64((long long)R[c], sh);
                else
                  D = rn_scaled((__int128)R[c] + shl_state<__int128>(I, wsh), sh);
                if (UPD == kSub)
                  red_add_f64(cp, neg_d(D));
                else if (UPD == kSet)
                  *cp = D;
                else
                  *cp = apply_update<UPD>(a, D, needs_c ? *cp : 0.0);
              }
            }
          } else {
#pragma unroll
            for (int c16 = 0; c16 < CPT / 16; ++c16) {
              uint32_t r[16];
              tmem_ld16(ta + c16 * 16, r);
              tmem_ld_wait();
#pragma unroll
              for (int q = 0; q < 16; ++q) R[c16 * 16 + q] += shl_state<State>(f2i(r[q]), wsh);
            }
          }
          if (!released) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) release(slot);
          }
        }
      }
      if (ok && a.mode == 0 && !final_done) {
        // every level was folded into R (wide variant): T = R
        const bool rowok = row < a.M;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int col = col0 + c;
          const int f = __shfl_sync(0xFFFFFFFFu, fcol[0], c);
          if (!rowok || col >= a.N || (a.lower && row < col)) continue;
          double D;
          if (e_row == kNonFinite || f == kNonFinite)
            D = __longlong_as_double(0x7FF8000000000000ll);
          else
            D = rn_scaled((__int128)R[c], e_row + f + sh0);
          double* cp = a.C + row + (long)col * a.ldc;
          if (UPD == kSub)
            red_add_f64(cp, neg_d(D));
          else if (UPD == kSet)
            *cp = D;
          else
            *cp = apply_update<UPD>(a, D, needs_c ? *cp : 0.0);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();   // neither CTA leaves while the other may still use its barriers or TMEM
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem, Cf::TMEM_COLS);
    else
      tmem_dealloc(tmem, Cf::TMEM_COLS);
  }
}

size_t gemm_stage_bytes(bool wide, int s, bool pair) {
  return wide ? (size_t)s * (Cfg<true>::A_TILE + Cfg<true>::B_TILE)
              : (size_t)s * (Cfg<false>::A_TILE + (pair ? Cfg<false>::B_TILE / 2 : Cfg<false>::B_TILE));
}

// Ring stages and shared-memory bytes of a launch.
int gemm_stages(bool wide, int s, bool pair, size_t* smem_bytes) {
  const size_t stage = gemm_stage_bytes(wide, s, pair);
  int stages = static_cast<int>((232448 - 1024 - 2048) / stage);
  if (stages > kMaxStagesCfg) stages = kMaxStagesCfg;
  if (smem_bytes) *smem_bytes = stages * stage + 1024;
  return stages;
}

// CTA pairs of the product kernel that can be resident at once with this much
// shared memory (0: none, e.g. on a partition without two free SMs side by side).
int gemm_pair_capacity(size_t smem_bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(dev, smem_bytes);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  auto kern = gemm_kernel<false, kSub, true>;
  int pairs = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem_bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&pairs, kern, &cfg) != cudaSuccess) pairs = 0;
  }
  cudaGetLastError();   // a failed query leaves no error behind
  cache[key] = pairs;
  return pairs;
}

template <bool WIDE, int UPD, bool PAIR>
cudaError_t launch_one(cudaStream_t st, const CUtensorMap& tmA, const CUtensorMap& tmB, const GemmArgs& args, int grid,
                       int stages, size_t smem_bytes) {
  // The register hand-over between warpgroups is only valid if the block is
  // launched with exactly kLaunchRegs registers per thread.
  auto kern = gemm_kernel<WIDE, UPD, PAIR>;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kern);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != kLaunchRegs) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  if (!PAIR) {
    kern<<<grid, kThreads, smem_bytes, st>>>(tmA, tmB, args, stages);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // the persistent grid holds no more pairs than can be resident at once (an
  // SM left without a partner would otherwise run its pair after the others)
  const int pairs = gemm_pair_capacity(smem_bytes);
  if (pairs < 1) return cudaErrorInvalidConfiguration;
  if (grid > 2 * pairs) cfg.gridDim = dim3(2 * pairs);
  return cudaLaunchKernelEx(&cfg, kern, tmA, tmB, args, stages);
}

cudaError_t launch_gemm(cudaStream_t st, bool wide, bool pair, const CUtensorMap& tmA, const CUtensorMap& tmB,
                        const GemmArgs& args, int grid, int stages, size_t smem_bytes) {
  const int upd = (args.alpha == -1.0 && args.beta == 1.0) ? kSub
                  : (args.alpha == 1.0 && args.beta == 0.0) ? kSet : kGeneral;
  if (wide) {
    if (upd == kSub) return launch_one<true, kSub, false>(st, tmA, tmB, args, grid, stages, smem_bytes);
    if (upd == kSet) return launch_one<true, kSet, false>(st, tmA, tmB, args, grid, stages, smem_bytes);
    return launch_one<true, kGeneral, false>(st, tmA, tmB, args, grid, stages, smem_bytes);
  }
  if (pair) {
    if (upd == kSub) return launch_one<false, kSub, true>(st, tmA, tmB, args, grid, stages, smem_bytes);
    if (upd == kSet) return launch_one<false, kSet, true>(st, tmA, tmB, args, grid, stages, smem_bytes);
    return launch_one<false, kGeneral, true>(st, tmA, tmB, args, grid, stages, smem_bytes);
  }
  if (upd == kSub) return launch_one<false, kSub, false>(st, tmA, tmB, args, grid, stages, smem_bytes);
  if (upd == kSet) return launch_one<false, kSet, false>(st, tmA, tmB, args, grid, stages, smem_bytes);
  return launch_one<false, kGeneral, false>(st, tmA, tmB, args, grid, stages, smem_bytes);
}

}  // namespace emul

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
// each drained level exactly to an integer and folds it into a Horner state
// R = R * 2^7 + I_L (int64, or 128-bit for the wide variant); the final value
// T = sum_L I_L 2^(7(t-L)) is rounded once to FP64,
//   D = RN(T * 2^(e_i + f_j - 7t)),
// from two exact parts with one FP64 add, and C = RN(RN(alpha D) + RN(beta C))
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
// issuer fills slots while the epilogue drains others, and a stashed job can
// hold its slot until its partner is drained.  All waits are bounded.
#include <cstdint>
#include <type_traits>

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
constexpr long long kFoldLimit = 1ll << 55;   // |R| below it: R * 2^7 + I fits in 64 bits

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

// v * 2^e2 as a double, exact, for 0 < |v| < 2^53 and a normal result.
__device__ __forceinline__ double exact_i64(long long v, int e2) {
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int msb = 63 - __clzll((long long)a);
  const unsigned long long mant = a << (52 - msb);                  // leading one at bit 52
  const unsigned long long bits = ((unsigned long long)(msb + e2 + 1022) << 52) + mant;
  return __longlong_as_double((long long)(bits | (v < 0 ? 0x8000000000000000ull : 0ull)));
}

// RN(T * 2^sh) for T = R * 2^7 + I (|R| < 2^62, |I| < 2^26): T = A1 2^35 + A0 with
// |A1| < 2^35 and |A0| < 2^37 both exact in FP64, so one DADD of the two exact
// parts gives the single correct rounding.  Outside -1022 <= sh <= 950 (parts
// that could be subnormal or overflow) the integer path is used.
__device__ __forceinline__ double rn_split(long long R, int I, int sh) {
  if (sh < -1022 || sh > 950) return rn_scaled((__int128)R * 128 + (__int128)I, sh);
  const long long A1 = R >> 28;
  const long long A0 = ((R & ((1ll << 28) - 1)) << 7) + I;
  const double dh = A1 ? exact_i64(A1, sh + 35) : 0.0;
  const double dl = A0 ? exact_i64(A0, sh) : 0.0;
  return __dadd_rn(dh, dl);
}

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

template <bool WIDE, int UPD>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs a,
                int stages) {
  using Cf = Cfg<WIDE>;
  using State = typename Cf::State;
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
  const uint32_t stage_bytes = (uint32_t)s * (Cf::A_TILE + Cf::B_TILE);
  volatile int* abortp = &abort_flag;

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
      mbar_init(&slot_empty[i], kEpiWarps);
    }
    for (int i = 0; i < kMmaWarps; ++i) mbar_init(&mma_done[i], 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, Cf::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
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
    for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
      int tm, tn;
      tile_coords(a, tile, tm, tn);
      const int m0 = tm * Cf::BM, n0 = tn * Cf::BN;
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
          mbar_arrive_expect_tx_elect(&stage_full[st], (uint32_t)(nu * np) * (Cf::A_TILE + Cf::B_TILE));
          for (int u = 0; u < nu; ++u)
            for (int p = 0; p < np; ++p) {
              const int t = u * np + p;
              tma_load_3d_elect(base + t * Cf::A_TILE, &tmA, &stage_full[st], (kc + u) * kBK, m0, p);
              tma_load_3d_elect(base + s * Cf::A_TILE + t * Cf::B_TILE, &tmB, &stage_full[st], (kc + u) * kBK, n0,
                                p);
            }
        }
      }
    }
    if (!ok) {
      // wait (bounded) for the copies still in flight before the block exits
      for (long j = (it - stages > 0 ? it - stages : 0); j < it; ++j)
        mbar_wait(&stage_full[j % stages], (uint32_t)((j / stages) & 1), a.wait_limit / 8);
    }
  } else if (warp >= 1 && warp <= kMmaWarps) {
    // ------------------------------------------------------------ MMA issuers
    // the whole warp runs the loop (warp-uniform values); one elected lane issues
    const int myj = warp - 1;   // job of each sweep issued by this warp
    {
      constexpr uint32_t idesc = idesc_bf16_f32(128, Cf::BN);
      long it = 0, tloc = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++tloc) {
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
            if (aborted(abortp) || !mbar_wait_warp(&slot_empty[slot], ((e >> 2) & 1u) ^ 1u, a.wait_limit)) {
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
                const uint64_t db = dB0 + (uint64_t)((u * np + q - 1) * (Cf::B_TILE >> 4));
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                  const uint32_t acc = (!first || p != pb || kk != 0) ? 1u : 0u;
                  mma_bf16_elect(dcol, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, acc);
                }
              }
            }
            mma_commit_elect(&stage_empty[st]);   // also by a warp without a job here: the stage needs both
          }
          if (!ok) break;
          if (mine) mma_commit_elect(&slot_full[slot]);
          jj += nj;
        }
      }
      // every MMA issued by this warp must be complete before TMEM is released
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
    for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++tloc) {
      int tm, tn;
      tile_coords(a, tile, tm, tn);
      const int row = tm * Cf::BM + row_t;
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
      int st_slot = 0;
      uint32_t st_par = 0;
      bool final_done = false;
      for (int sw = 0; sw < a.nsweeps && ok; ++sw) {
        const Sweep S = sched[sw];
        const int nj = S.L[1] ? 2 : 1;
        for (int j = 0; j < nj && ok; ++j, ++jj) {
          const int fl = S.flags[j];
          const uint32_t e = srow[jj];
          const int slot = (int)(e & 3u);
          const uint32_t par = (e >> 2) & 1u;
          if (a.mode == 0 && (fl & kStash)) {
            // left in its slot until the kTake job
            st_slot = slot;
            st_par = par;
            continue;
          }
          const bool take = a.mode == 0 && (fl & kTake);
          bool released = false;   // slots already released (final step, 64-bit path)
          if (aborted(abortp) || !mbar_wait(&slot_full[slot], par, a.wait_limit) ||
              (take && !mbar_wait(&slot_full[st_slot], st_par, a.wait_limit))) {
            if (!aborted(abortp)) raise_timeout(a, abortp);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ta = tmem + lane_addr + (uint32_t)(slot * Cf::BN + half * CPT);
          const uint32_t tb = tmem + lane_addr + (uint32_t)(st_slot * Cf::BN + half * CPT);
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
            // final step: T = R * 2^7 + I (I of this job plus the stashed one),
            // rounded once, C updated in place
            final_done = true;
            const bool rowok = row < a.M;
            // When no R of the warp reaches 2^55 (R reaches 2^57 only when whole
            // rows and columns have leading digits near 127 of one sign), T fits
            // in 64 bits: the last level is folded into R, both TMEM slots are
            // released at once, and the rounding runs while the MMAs of the next
            // tile fill them.  Otherwise T is rounded from its two exact parts.
            bool fits = !WIDE;
#pragma unroll
            for (int c = 0; c < CPT; ++c) fits = fits && R[c] > -kFoldLimit && R[c] < kFoldLimit;
            fits = __all_sync(0xFFFFFFFFu, fits);
            if (fits) {
#pragma unroll
              for (int c4 = 0; c4 < CPT / 4; ++c4) {
                uint32_t r0[4], r1[4];
                tmem_ld4(ta + c4 * 4, r0);
                if (take) tmem_ld4(tb + c4 * 4, r1);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  R[c4 * 4 + q] = R[c4 * 4 + q] * (State)128 + (State)(f2i(r0[q]) + (take ? f2i(r1[q]) : 0));
              }
              tc_fence_before();
              __syncwarp();
              if (lane == 0) {
                mbar_arrive(&slot_empty[slot]);
                if (take) mbar_arrive(&slot_empty[st_slot]);
              }
              released = true;
              double* cp = a.C + row + (long)col0 * a.ldc;
#pragma unroll
              for (int c = 0; c < CPT; ++c, cp += a.ldc) {
                const int col = col0 + c;
                const int f = __shfl_sync(0xFFFFFFFFu, fcol[0], c);
                if (!rowok || col >= a.N || (a.lower && row < col)) continue;
                const double D = (e_row == kNonFinite || f == kNonFinite)
                                     ? __longlong_as_double(0x7FF8000000000000ll)
                                     : rn_sum64((long long)R[c], e_row + f + sh0);
                if (UPD == kSub)
                  red_add_f64(cp, neg_d(D));
                else if (UPD == kSet)
                  *cp = D;
                else
                  *cp = apply_update<UPD>(a, D, needs_c ? *cp : 0.0);
              }
            } else {
#pragma unroll
              for (int c4 = 0; c4 < CPT / 4; ++c4) {
                uint32_t r0[4], r1[4];
                tmem_ld4(ta + c4 * 4, r0);
                if (take) tmem_ld4(tb + c4 * 4, r1);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const int c = c4 * 4 + q;
                  const int col = col0 + c;
                  const int f = __shfl_sync(0xFFFFFFFFu, fcol[0], c);
                  if (!rowok || col >= a.N || (a.lower && row < col)) continue;
                  const int I = f2i(r0[q]) + (take ? f2i(r1[q]) : 0);
                  double D;
                  if (e_row == kNonFinite || f == kNonFinite)
                    D = __longlong_as_double(0x7FF8000000000000ll);
                  else if (WIDE)
                    D = rn_scaled((__int128)R[c] * 128 + (__int128)I, e_row + f + sh0);
                  else
                    D = rn_split((long long)R[c], I, e_row + f + sh0);
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
          } else {
            if (fl & kOpen) {
#pragma unroll
              for (int c = 0; c < CPT; ++c) R[c] = R[c] * (State)128;
            }
            if (!take) {
#pragma unroll
              for (int c16 = 0; c16 < CPT / 16; ++c16) {
                uint32_t r[16];
                tmem_ld16(ta + c16 * 16, r);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 16; ++q) R[c16 * 16 + q] += (State)f2i(r[q]);
              }
            } else {
#pragma unroll
              for (int c8 = 0; c8 < CPT / 8; ++c8) {
                uint32_t r[8], r2[8];
                tmem_ld8(ta + c8 * 8, r);
                tmem_ld8(tb + c8 * 8, r2);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 8; ++q) R[c8 * 8 + q] += (State)(f2i(r[q]) + f2i(r2[q]));
              }
            }
          }
          if (!released) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              mbar_arrive(&slot_empty[slot]);
              if (take) mbar_arrive(&slot_empty[st_slot]);
            }
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
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, Cf::TMEM_COLS);
  }
}

size_t gemm_stage_bytes(bool wide, int s) {
  return wide ? (size_t)s * (Cfg<true>::A_TILE + Cfg<true>::B_TILE)
              : (size_t)s * (Cfg<false>::A_TILE + Cfg<false>::B_TILE);
}

template <bool WIDE, int UPD>
cudaError_t launch_one(cudaStream_t st, const CUtensorMap& tmA, const CUtensorMap& tmB, const GemmArgs& args, int grid,
                       int stages, size_t smem_bytes) {
  // The register hand-over between warpgroups is only valid if the block is
  // launched with exactly kLaunchRegs registers per thread.
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)gemm_kernel<WIDE, UPD>);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != kLaunchRegs) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(gemm_kernel<WIDE, UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
  if (e != cudaSuccess) return e;
  gemm_kernel<WIDE, UPD><<<grid, kThreads, smem_bytes, st>>>(tmA, tmB, args, stages);
  return cudaGetLastError();
}

cudaError_t launch_gemm(cudaStream_t st, bool wide, const CUtensorMap& tmA, const CUtensorMap& tmB,
                        const GemmArgs& args, int grid, int stages, size_t smem_bytes) {
  const int upd = (args.alpha == -1.0 && args.beta == 1.0) ? kSub
                  : (args.alpha == 1.0 && args.beta == 0.0) ? kSet : kGeneral;
  if (wide) {
    if (upd == kSub) return launch_one<true, kSub>(st, tmA, tmB, args, grid, stages, smem_bytes);
    if (upd == kSet) return launch_one<true, kSet>(st, tmA, tmB, args, grid, stages, smem_bytes);
    return launch_one<true, kGeneral>(st, tmA, tmB, args, grid, stages, smem_bytes);
  }
  if (upd == kSub) return launch_one<false, kSub>(st, tmA, tmB, args, grid, stages, smem_bytes);
  if (upd == kSet) return launch_one<false, kSet>(st, tmA, tmB, args, grid, stages, smem_bytes);
  return launch_one<false, kGeneral>(st, tmA, tmB, args, grid, stages, smem_bytes);
}

}  // namespace emul

"""Host-side checks of the product kernel's schedule and TMEM slot plan
(emul_schedule; no GPU needed).

The level sums I_L = sum_{p+q=L} S_p^A S_q^B of Sec. 2 are accumulated in
jobs (one level, a pair range, a K range) grouped into sweeps; the epilogue
adds each job's sum with its level's weight, T = sum_L I_L 2^(7(t-L)).  Checked here for every
slice count and a range of k, both variants and both modes:
* every slice pair (p, q) with p + q <= t and every K chunk is summed
  exactly once (t = s + 1, the method's threshold, and other thresholds
  2 <= t <= 2s down to the full s^2-pair product), and no job exceeds the exact-accumulation budget
  (k_job * pairs <= 1040, so |I| < 2^24 in FP32);
* the narrow variant's final job (the one whose term completes T before the
  rounding) is level 2, alone in the last sweep; the wide variant has none;
* a sweep stages every plane its pairs use, within the stage's s planes;
* the slot table drives the MMA/epilogue barrier protocol without deadlock,
  with the parity bit of each job equal to the parity of its slot's use count
  (simulated independently of the planner, from the barrier semantics).
"""
import pytest

from paper_2509_23565_gb300 import binding

BUDGET = 1040
KBK = 32
FINAL = 1
KS = (1, 16, 32, 33, 64, 100, 128, 200, 224, 256, 300, 512, 1000, 2048)


def thresholds(s):
    return sorted({t for t in (s + 1, 2, s, s + 2, 2 * s - 1, 2 * s) if 2 <= t <= 2 * s})


ST = [(s, t) for s in range(1, 9) for t in thresholds(s)]


def jobs_of(sweeps):
    out = []
    for si, w in enumerate(sweeps):
        for j in (0, 1):
            if w[f"L{j}"] == 0:
                continue
            out.append({"sweep": si, "L": w[f"L{j}"], "pb": w[f"pb{j}"], "pe": w[f"pe{j}"], "c0": w["k0c"],
                        "c1": w["k1c"], "flags": w[f"flags{j}"]})
    return out


def get(s, k, wide, ls, t):
    r = binding.schedule(s, k, wide=wide, level_sums=ls, t=t)
    if wide:
        assert r is not None, f"the wide variant must schedule any k (s={s}, k={k})"
    return r


@pytest.mark.parametrize("s,t", ST)
def test_coverage_budget_planes(s, t):
    for k in KS:
        for wide in (False, True):
            r = get(s, k, wide, False, t)
            if r is None:
                continue
            sweeps, _, _ = r
            nch = (k + KBK - 1) // KBK
            count = {}
            for w in sweeps:
                assert 0 <= w["k0c"] < w["k1c"] <= nch
                assert w["kcs"] >= 1 and w["kcs"] * w["nplanes"] <= s and w["nplanes"] <= s
                for j in (0, 1):
                    L = w[f"L{j}"]
                    if L == 0:
                        continue
                    pb, pe = w[f"pb{j}"], w[f"pe{j}"]
                    assert 1 <= pb <= pe and 2 <= L <= t
                    assert (pe - pb + 1) * (w["k1c"] - w["k0c"]) * KBK <= BUDGET
                    for p in range(pb, pe + 1):
                        q = L - p
                        assert 1 <= q <= s
                        assert max(p, q) <= w["nplanes"]
                        for c in range(w["k0c"], w["k1c"]):
                            count[(p, q, c)] = count.get((p, q, c), 0) + 1
            want = {(p, q, c) for p in range(1, s + 1) for q in range(1, s + 1) if p + q <= t
                    for c in range(nch)}
            assert set(count) == want, (s, k, wide)
            assert all(v == 1 for v in count.values()), (s, k, wide)


@pytest.mark.parametrize("s,t", ST)
def test_final_job(s, t):
    """The narrow variant rounds after its last job, which must be the only
    job of level 2 (its term I_2 2^(7(t-2)) is the one the epilogue adds in
    128 bits when it would overflow 64) and alone in the last sweep; the
    wide variant rounds after all its jobs and flags none.  The first sweep
    holds the highest level (the longest jobs start each tile)."""
    for k in KS:
        for wide in (False, True):
            r = get(s, k, wide, False, t)
            if r is None:
                continue
            sweeps, _, _ = r
            jobs = jobs_of(sweeps)
            finals = [jb for jb in jobs if jb["flags"] & FINAL]
            if wide:
                assert not finals, (s, k, t)
                continue
            assert len(finals) == 1 and finals[0] is jobs[-1], (s, k, t)
            assert finals[0]["L"] == 2 and [jb["L"] for jb in jobs].count(2) == 1
            assert sweeps[-1]["L1"] == 0
            assert max(sweeps[0]["L0"], sweeps[0]["L1"]) == max(jb["L"] for jb in jobs)


@pytest.mark.parametrize("s,t", ST)
def test_slot_protocol(s, t):
    """Barrier-level simulation over several tiles: the MMA side takes a sweep
    when every slot it needs has been released as often as it was allocated;
    the epilogue drains jobs in order and releases each slot when its job is
    drained.  The table's parity bit must equal the slot's use count
    parity; the simulation must run to the end (no deadlock)."""
    for k in KS:
        for wide in (False, True):
            for ls in (False, True):
                r = get(s, k, wide, ls, t)
                if r is None:
                    continue
                sweeps, tab, info = r
                nj, t0, per = info["njobs"], info["t0"], info["period"]
                jobs = jobs_of(sweeps)
                assert len(jobs) == nj and per >= 1
                ntiles = t0 + 2 * per + 1
                alloc = [0, 0, 0, 0]
                rel = [0, 0, 0, 0]
                full = {}            # (tile, job) -> slot, once the MMA has committed it
                mma = (0, 0)         # (tile, sweep)
                epi = (0, 0)         # (tile, job)
                steps = 0
                while epi[0] < ntiles:
                    steps += 1
                    assert steps < 100000
                    progressed = False
                    if mma[0] < ntiles:
                        tile, si = mma
                        ph = tile if tile < t0 else t0 + (tile - t0) % per
                        idx = [j for j, jb in enumerate(jobs) if jb["sweep"] == si]
                        slots = [tab[ph * nj + j] & 3 for j in idx]
                        assert len(set(slots)) == len(slots)
                        if all(rel[sl] == alloc[sl] for sl in slots):
                            for j, sl in zip(idx, slots):
                                assert (tab[ph * nj + j] >> 2) & 1 == alloc[sl] & 1, (s, k, wide, ls)
                                alloc[sl] += 1
                                full[(tile, j)] = sl
                            mma = (tile, si + 1) if si + 1 < len(sweeps) else (tile + 1, 0)
                            progressed = True
                    tile, j = epi
                    if (tile, j) in full:
                        rel[full[(tile, j)]] += 1
                        epi = (tile, j + 1) if j + 1 < nj else (tile + 1, 0)
                        progressed = True
                    assert progressed, f"deadlock s={s} k={k} wide={wide} level_sums={ls} at {mma} {epi}"


def test_lu_schedule_shape():
    """The LU's trailing update (s = 7, k = nb = 256, narrow) uses the banded
    schedule: levels {7,8} and {5,6} in K halves, then {3,4}, then {2}, 16
    staged planes per K chunk."""
    sweeps, _, info = binding.schedule(7, 256)
    levels = [(w["L0"], w["L1"]) for w in sweeps]
    assert levels == [(7, 8), (7, 8), (5, 6), (5, 6), (3, 4), (2, 0)]
    nch = 8
    assert sum(w["nplanes"] * (w["k1c"] - w["k0c"]) for w in sweeps) == 16 * nch
    assert info["njobs"] == 11


def test_narrow_reach_at_s7():
    """At s = 7 the 128-column variant schedules every k up to 1024 (32 chunks):
    level 2, one pair, fits the exactness budget over 1024 in one job, which
    the final job must be; at 1056 it would need two, so only the wide variant
    schedules it."""
    for k in (32, 256, 512, 1000, 1024):
        r = binding.schedule(7, k)
        assert r is not None, k
        last = r[0][-1]
        assert (last["L0"], last["L1"], last["flags0"]) == (2, 0, FINAL) and last["k1c"] - last["k0c"] == (k + 31) // 32
    assert binding.schedule(7, 1056) is None
    assert binding.schedule(7, 1056, wide=True) is not None


@pytest.mark.parametrize("s", [1, 4, 7])
def test_threshold_out_of_range(s):
    for t in (1, 2 * s + 1):
        assert binding.schedule(s, 256, wide=True, t=t) is None
    full = binding.schedule(s, 64, wide=True, t=2 * s)
    assert full is not None and max(max(w["L0"], w["L1"]) for w in full[0]) == 2 * s

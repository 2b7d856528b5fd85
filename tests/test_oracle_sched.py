"""Pins of the scheduling oracle: Table 2's printed urgencies and priorities, hand-computed
batch boundaries, levels and delays, the miss-ratio metric (Eq. 3) on hand-made logs, and the
discrete-event simulation against exhaustive enumeration of 3-chain instances.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import sched as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2.txt")


def _table2():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        c, per, D, ec, eg, ul, pri = line.split()
        rows.append((int(c), float(per), float(D), float(ec), float(eg), float(ul), int(pri)))
    return rows


def _trunc4(v):
    return math.floor(v * 1e4) / 1e4


def test_table2_urgency_values():
    rows = _table2()
    for c, _per, D, ec, eg, ul, _pri in rows:
        got = _trunc4(S.table2_urgency(D, ec, eg))
        if c == 10:
            assert abs(got - 0.0056) < 1e-12 and ul == 0.0050   # misprinted row
        else:
            assert abs(got - ul) < 1e-12, (c, got, ul)


def test_table2_priority_ranks():
    rows = _table2()
    uls = [S.table2_urgency(D, ec, eg) for _c, _p, D, ec, eg, _u, _r in rows]
    pri = S.priority_ranks(uls)
    printed = [r[6] for r in rows]
    for c in range(len(rows)):
        if c in (2, 7):
            continue
        assert pri[c] == printed[c], c
    # C2 and C7 have equal urgency; the table ranks the higher id first, the rule the lower
    assert {pri[2], pri[7]} == {printed[2], printed[7]} == {4, 5}
    assert pri[2] < pri[7]


def test_batch_boundaries_hand():
    assert S.batch_boundaries([0.2, 0.2, 0.2, 0.1, 0.4, 0.05], 0.5) == [2, 4]
    assert S.batch_boundaries([0.5, 0.5], 0.5) == [0, 1]
    assert S.batch_boundaries([0.1] * 4, 0.5) == []
    assert S.batch_boundaries([], 0.5) == []
    assert S.batch_boundaries([0.3, 0.3, 0.3], 0.0) == [0, 1, 2]


def test_batch_gate_overlap():
    g = S.BatchGate(500.0)
    assert not g.launched(0, 200.0)
    assert g.launched(1, 300.0)          # 500 >= 500: batch {0, 1} closes
    assert g.pending == 1
    assert g.launched(2, 600.0)          # batch {2} closes
    assert g.pending == 2                # overlapped mode (max_closed = 2) must now wait
    g.finished(0)
    assert g.pending == 2
    g.finished(1)
    assert g.pending == 1
    g.finished(2)
    assert g.pending == 0


def test_miss_ratio_hand_log():
    assert abs(S.overall_miss_ratio({0: (1, 4), 1: (0, 2), 2: (3, 3)}) - (0.25 + 0 + 1) / 3) < 1e-15
    assert S.overall_miss_ratio({0: (0, 0), 1: (1, 2)}) == 0.5
    assert S.overall_miss_ratio({}) == 0.0


def _R(fid, chain, t_arr, D, est, prec=0, util=1.0):
    return S.Ready(fid, chain, t_arr, t_arr + D, est, 0.0, prec, util)


def test_decide_levels_and_reservation():
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=1, th_urgent=1 / 100.0, num_pri=6)
    # slack 50 -> UL 0.02 > TH 0.01: reserved level 0
    d = S.decide(0.0, [_R(1, 0, 0, 150, 100)], [], 0, cfg)
    assert (d.kind, d.frames, d.level) == (S.RELEASE, [1], 0)
    # slack 1000 -> UL 0.001; active non-urgent ULs 0.002, 0.0005; urgent one ignored
    act = [S.Active(5, 0.002), S.Active(6, 0.0005), S.Active(7, 0.5)]
    d = S.decide(0.0, [_R(2, 1, 0, 1100, 100)], act[:2], 0, cfg)
    # r = 1 (0.002 > 0.001), n = 3 -> 1 + floor(1*5/3) = 2
    assert d.level == 2
    # an urgent active unit of another chain holds the release (Section 4.4.4) ...
    d = S.decide(0.0, [_R(2, 1, 0, 1100, 100)], act, 0, cfg)
    assert d.kind == S.DELAY
    # ... unless the candidate is exempt by low utilisation, or the urgent unit is its own chain
    d = S.decide(0.0, [_R(2, 1, 0, 1100, 100, util=0.05)], act, 0, cfg)
    assert d.kind == S.RELEASE and d.level == 2
    d = S.decide(0.0, [_R(2, 7, 0, 1100, 100)], act, 0, cfg)
    assert d.kind == S.RELEASE


def test_decide_order_batch_drop_wait():
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=3, th_urgent=0.0)
    ready = [_R(1, 0, 0, 1000, 100), _R(2, 1, 10, 500, 100), _R(3, 2, 5, 2000, 100, prec=1),
             _R(4, 3, 0, 50, 100), _R(5, 4, 0, 900, 100)]
    d = S.decide(20.0, ready, [], 0, cfg)
    assert d.drops == [4]                         # slack 50 - 100 - 20 < 0: early exit
    assert d.frames == [2, 5, 1]                  # slack 390, 780, 880; precision 0 only
    d = S.decide(20.0, ready, [], 2, cfg)
    assert d.kind == S.WAIT and d.drops == [4]
    fifo = S.PolicyConfig(policy=S.POLICY_FIFO, max_batch=1, num_pri=6)
    d = S.decide(20.0, ready, [], 0, fifo)
    assert d.frames == [1] and d.drops == [] and d.level == 5    # (t_arr 0, chain 0) first


# ---------------------------------------------------------------- DES vs enumeration

def _instance(seed):
    """3 chains, 1-3 frames each, 1-3 units per frame; at most 8 units in total so that the
    enumeration stays small."""
    rng = np.random.default_rng(seed)
    frames = []
    fid, units = 0, 0
    for c in range(3):
        t_arr = float(rng.integers(0, 20))
        for k in range(int(rng.integers(1, 4))):
            n_st = int(rng.integers(1, 4))
            if units + n_st > 8 - (2 - c):       # leave at least one unit for later chains
                break
            stages = [float(rng.integers(3, 15)) for _ in range(n_st)]
            D = float(rng.integers(20, 90))
            frames.append(S.SimFrame(fid, c, t_arr, t_arr + D, stages))
            fid += 1
            units += n_st
            t_arr += float(rng.integers(5, 40))
    return frames


def _enumerate(frames):
    """Every schedule of one non-preemptive server that starts a ready unit whenever it is
    idle (units of a frame in order; a frame is ready from its arrival).  Yields
    (list of (t_start, frame, stage), finish times)."""
    by = {f.frame_id: f for f in frames}

    def rec(t, nxt, trace, fin):
        ready = [f for f in frames if f.t_arr <= t and nxt[f.frame_id] < len(f.stages)]
        if not ready:
            future = [f.t_arr for f in frames if f.t_arr > t and nxt[f.frame_id] < len(f.stages)]
            if not future:
                yield list(trace), dict(fin)
                return
            yield from rec(min(future), nxt, trace, fin)
            return
        for f in ready:
            k = nxt[f.frame_id]
            te = t + f.stages[k]
            nxt[f.frame_id] += 1
            trace.append((t, f.frame_id, k))
            if nxt[f.frame_id] == len(f.stages):
                fin[f.frame_id] = te
            yield from rec(te, nxt, trace, fin)
            trace.pop()
            fin.pop(f.frame_id, None)
            nxt[f.frame_id] -= 1

    yield from rec(0.0, {f.frame_id: 0 for f in frames}, [], {})


def _is_least_slack(trace, frames):
    by = {f.frame_id: f for f in frames}
    nxt = {f.frame_id: 0 for f in frames}
    for t, fid, k in trace:
        ready = [f for f in frames if f.t_arr <= t and nxt[f.frame_id] < len(f.stages)]
        key = lambda f: (f.deadline - sum(f.stages[nxt[f.frame_id]:]) - t, f.chain_id, f.t_arr,
                         f.frame_id)
        if min(ready, key=key).frame_id != fid:
            return False
        nxt[fid] += 1
    return True


@pytest.mark.parametrize("seed", range(12))
def test_des_matches_enumeration(seed):
    frames = _instance(seed)
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=1, delta_eval_us=0.0, max_closed=1,
                         th_urgent=0.0, early_exit=False)
    res = S.simulate(frames, cfg)
    greedy = []
    best_miss = None
    for trace, fin in _enumerate(frames):
        misses = sum(fin[f.frame_id] > f.deadline for f in frames)
        best_miss = misses if best_miss is None else min(best_miss, misses)
        if _is_least_slack(trace, frames):
            greedy.append((trace, fin))
    assert len(greedy) == 1
    trace, fin = greedy[0]
    assert [(t, m[0][0], m[0][1]) for t, m, _lvl in res.releases] == trace
    assert res.done == fin
    assert sum(res.missed.values()) >= best_miss     # least slack is not optimal in general


def test_des_early_exit_and_batching_invariants():
    rng = np.random.default_rng(4)
    frames = []
    for i in range(200):
        c = i % 5
        t = float(i * 40 + rng.integers(0, 30))
        frames.append(S.SimFrame(i, c, t, t + float(rng.choice([150, 300, 600])),
                                 [float(rng.integers(20, 120))], precision=c % 2))
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=4, delta_eval_us=100.0,
                         max_closed=2, th_urgent=0.0)
    res = S.simulate(frames, cfg, unit_time=lambda ds: 10.0 + 0.5 * sum(ds))
    assert set(res.done) | set(res.dropped) == {f.frame_id for f in frames}
    assert not set(res.done) & set(res.dropped)
    for _t, members, _lvl in res.releases:
        assert 1 <= len(members) <= 4
        assert len({frames[fid].precision for fid, _ in members}) == 1
    for fid, t in res.dropped.items():        # dropped only when hopeless at that time
        f = frames[fid]
        assert f.deadline - f.stages[0] - t < 0
    fifo = S.simulate(frames, S.PolicyConfig(policy=S.POLICY_FIFO, max_batch=1, max_closed=0),
                      unit_time=lambda ds: 10.0 + 0.5 * sum(ds))
    assert not fifo.dropped and len(fifo.done) == len(frames)
    assert [m[0][0] for _t, m, _l in fifo.releases] == [f.frame_id for f in
                                                        sorted(frames, key=lambda f: (f.t_arr, f.chain_id))]


def test_comparison_policies_hand_example():
    """Three frames with hand-computed orders.  At t = 1000 us:
         frame  arrival  deadline  estimate  period   wait  ratio (w+e)/e  util e/P
         A      0        5000      400       50000    1000  3.5            0.008
         B      600      3000      100       200000   400   5.0            0.0005
         C      900      9000      1600      100000   100   1.0625         0.016
    EDF: B (3000), A (5000), C;  SJF: B (100), A (400), C;  HRRN: B (5.0), A (3.5), C (1.0625);
    LCUF: B (0.0005), A (0.008), C (0.016).  FIFO: A, B, C.  A unit takes every ready frame of
    the same precision in that order."""
    t = 1000.0
    ready = [S.Ready(1, 0, 0.0, 5000.0, 400.0, period=50000.0),
             S.Ready(2, 1, 600.0, 3000.0, 100.0, period=200000.0),
             S.Ready(3, 2, 900.0, 9000.0, 1600.0, period=100000.0)]
    want = {S.POLICY_EDF: [2, 1, 3], S.POLICY_SJF: [2, 1, 3], S.POLICY_HRRN: [2, 1, 3],
            S.POLICY_LCUF: [2, 1, 3], S.POLICY_FIFO: [1, 2, 3]}
    for pol, order in want.items():
        d = S.decide(t, ready, [], 0, S.PolicyConfig(policy=pol, max_closed=0))
        assert d.kind == S.RELEASE and d.frames == order, pol
    # a swap that separates the policies: make C the shortest and lowest-utilisation job
    ready[2] = S.Ready(3, 2, 900.0, 9000.0, 50.0, period=400000.0)   # ratio (100+50)/50 = 3.0
    got = {pol: S.decide(t, ready, [], 0, S.PolicyConfig(policy=pol, max_closed=0)).frames
           for pol in (S.POLICY_EDF, S.POLICY_SJF, S.POLICY_HRRN, S.POLICY_LCUF)}
    assert got[S.POLICY_EDF] == [2, 1, 3]        # deadlines unchanged
    assert got[S.POLICY_SJF] == [3, 2, 1]        # 50 < 100 < 400
    assert got[S.POLICY_HRRN] == [2, 1, 3]       # 5.0 > 3.5 > 3.0
    assert got[S.POLICY_LCUF] == [3, 2, 1]       # 0.000125 < 0.0005 < 0.008


def test_saedf_eqdf_hand_example():
    """Three frames at t = 1000 us that separate EDF, slack-aware EDF and EQDF:
         frame  deadline  estimate  slack = d - e - t   quasi-deadline d - lambda e (0.5 / 1)
         X      3000      100       1900                2950 / 2900
         Y      3400      1000      1400                2900 / 2400
         Z      1500      800       -300                1100 / 700
    EDF: Z, X, Y.  SAEDF: X, Y (slack >= 0, by deadline), then Z.  EQDF lambda 0.5 and 1: Z, Y,
    X; lambda 0 is EDF.  The urgency policy drops Z (negative slack) and releases Y, X."""
    t = 1000.0
    ready = [S.Ready(1, 0, 500.0, 3000.0, 100.0), S.Ready(2, 1, 400.0, 3400.0, 1000.0),
             S.Ready(3, 2, 300.0, 1500.0, 800.0)]
    cases = [(S.POLICY_EDF, 0.5, [3, 1, 2]), (S.POLICY_SAEDF, 0.5, [1, 2, 3]), (S.POLICY_EQDF, 0.5, [3, 2, 1]),
             (S.POLICY_EQDF, 1.0, [3, 2, 1]), (S.POLICY_EQDF, 0.0, [3, 1, 2])]
    for pol, lam, order in cases:
        d = S.decide(t, ready, [], 0, S.PolicyConfig(policy=pol, max_closed=0, eqdf_lambda=lam))
        assert d.kind == S.RELEASE and d.frames == order and d.drops == [], (pol, lam)
    d = S.decide(t, ready, [], 0, S.PolicyConfig(policy=S.POLICY_URGENCY, max_closed=0))
    assert d.frames == [2, 1] and d.drops == [3]


def test_comparison_policies_match_sorting():
    """On random ready sets the head each comparison policy releases is the textbook optimum:
    min deadline, min estimate, max response ratio, min utilisation (ties: chain, arrival, id)."""
    import numpy as np
    rng = np.random.default_rng(3)
    for _ in range(2000):
        t = 1e5
        ready = [S.Ready(i, int(rng.integers(0, 4)), t - float(rng.integers(0, 5000)),
                         t + float(rng.integers(-100, 20000)), float(rng.integers(10, 3000)),
                         float(rng.choice([0.0, 30.0])), 0, 1.0, float(rng.choice([5e4, 1e5, 2e5])))
                 for i in range(int(rng.integers(1, 9)))]
        tie = lambda f: (f.chain_id, f.t_arr, f.frame_id)
        keys = {S.POLICY_EDF: lambda f: (f.deadline,) + tie(f),
                S.POLICY_SJF: lambda f: (f.est_gpu + f.est_cpu,) + tie(f),
                S.POLICY_HRRN: lambda f: (-(t - f.t_arr + f.est_gpu + f.est_cpu) / (f.est_gpu + f.est_cpu),) + tie(f),
                S.POLICY_LCUF: lambda f: ((f.est_gpu + f.est_cpu) / f.period,) + tie(f),
                S.POLICY_SAEDF: lambda f: (f.deadline - f.est_gpu - f.est_cpu - t < 0, f.deadline) + tie(f),
                S.POLICY_EQDF: lambda f: (f.deadline - 0.5 * (f.est_gpu + f.est_cpu),) + tie(f)}
        for pol, key in keys.items():
            d = S.decide(t, ready, [], 0, S.PolicyConfig(policy=pol, max_closed=0, max_batch=8, eqdf_lambda=0.5))
            assert d.frames[0] == min(ready, key=key).frame_id, pol
            assert d.drops == []                  # no early exit outside the urgency policy


def test_des_estimate_noise_only_moves_decisions():
    """Estimate noise changes what the policy sees, not the work: with eps = 0 the run is
    identical to the noiseless one; with eps = 0.3 every frame still completes or is dropped,
    and the release trace differs."""
    from pp_synth import noise_factors
    import numpy as np
    rng = np.random.default_rng(8)
    base = []
    for i in range(400):
        t = float(i * 40 + rng.integers(0, 30))
        base.append((i, i % 5, t, t + float(rng.choice([150, 300, 800])), float(rng.integers(30, 120))))
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=1, delta_eval_us=0.0, max_closed=0,
                         th_urgent=-1.0, num_pri=4)

    def run(eps):
        fac = noise_factors(3, range(400), eps)
        frames = [S.SimFrame(i, c, t, dl, [d], est=[d * fac[i]]) for (i, c, t, dl, d) in base]
        return S.simulate(frames, cfg)

    plain = S.simulate([S.SimFrame(i, c, t, dl, [d]) for (i, c, t, dl, d) in base], cfg)
    r0, r3 = run(0.0), run(0.3)
    assert r0.done == plain.done and r0.dropped == plain.dropped and r0.releases == plain.releases
    assert set(r3.done) | set(r3.dropped) == set(range(400))
    assert r3.releases != plain.releases


def test_des_cpu_priority_hand_example():
    """CPU segments (Section 4.3), one core.  A (chain 0, arrives 0, deadline 10000): GPU 100 us,
    then CPU 1000 us.  B (chain 1, arrives 50, deadline 650): GPU 100 us (runs 100-200 behind A),
    then CPU 200 us.  FIFO CPU: B waits for A's segment (core busy 100-1100) and ends at 1300 --
    missed.  Urgency CPU priority: at 200, B's slack is 650 - 200 - 200 = 250 against A's
    10000 - 900 - 200 = 8900, so B preempts A, runs 200-400 and is met; A resumes and ends at
    400 + 900 = 1300."""
    frames = [S.SimFrame(0, 0, 0.0, 10000.0, [100.0], cpu=[1000.0]),
              S.SimFrame(1, 1, 50.0, 650.0, [100.0], cpu=[200.0])]
    cfg = S.PolicyConfig(policy=S.POLICY_FIFO, max_batch=1, max_closed=0, th_urgent=-1.0, early_exit=False)
    fifo = S.simulate(frames, cfg, cpu_cores=1, cpu_policy="fifo")
    assert fifo.done == {0: 1100.0, 1: 1300.0} and fifo.missed == {0: False, 1: True}
    urg = S.simulate(frames, cfg, cpu_cores=1, cpu_policy="urgency")
    assert urg.done == {0: 1300.0, 1: 400.0} and urg.missed == {0: False, 1: False}


def test_des_cpu_segments_invariants():
    """With a core per frame the CPU policies coincide (no contention); any run completes every
    frame no earlier than its arrival plus its GPU and CPU work; the GPU policy's slack counts the
    remaining CPU time (an urgency run drops a frame whose CPU segment alone outlasts its
    deadline)."""
    import numpy as np
    rng = np.random.default_rng(12)
    frames = []
    for i in range(150):
        t = float(i * 300 + rng.integers(0, 200))
        g = [float(rng.integers(50, 200)) for _ in range(2)]
        c = [float(rng.integers(0, 800)), float(rng.integers(100, 900))]
        frames.append(S.SimFrame(i, i % 6, t, t + float(rng.choice([3000, 6000, 20000])), g, cpu=c))
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=2, delta_eval_us=300.0, max_closed=2,
                         th_urgent=-1.0, early_exit=False)
    a = S.simulate(frames, cfg, cpu_cores=1000, cpu_policy="fifo")
    b = S.simulate(frames, cfg, cpu_cores=1000, cpu_policy="urgency")
    assert a.done == b.done and a.releases == b.releases
    for cores in (1, 2, 4):
        for pol in ("fifo", "urgency"):
            r = S.simulate(frames, cfg, cpu_cores=cores, cpu_policy=pol)
            assert set(r.done) == set(range(150))
            for f in frames:
                assert r.done[f.frame_id] >= f.t_arr + sum(f.stages) + sum(f.cpu) - 1e-9
    late = [S.SimFrame(0, 0, 0.0, 500.0, [100.0], cpu=[600.0])]
    r = S.simulate(late, S.PolicyConfig(policy=S.POLICY_URGENCY, max_closed=0, th_urgent=-1.0))
    assert r.dropped == {0: 0.0}


# ---------------------------------------------------------------- DES branches, hand-computed

def _delay_case(quantum):
    # A (chain 0) is urgent when released at t=0 (slack 50 us, UL 0.02 > TH 0.015) and holds the
    # GPU until t=100.  B (chain 1) arrives at t=10 with slack 95 (UL 0.0105): less urgent than
    # A, so it is delayed, and re-checked every quantum: its slack shrinks as time passes, and it
    # is released at the first wake-up where its UL exceeds A's 0.02 (slack < 50 us):
    #   quantum 50: wake at 60, slack 145 - 40 - 60 = 45 -> released at 60 (UL 0.022 > TH: level 0)
    #   quantum 30: wake at 40 (slack 65, still delayed), then 70 (slack 35) -> released at 70
    # Either way it waits in the GPU queue until A completes and runs 100..140 (deadline 145).
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=1, max_closed=0, th_urgent=0.015, num_pri=6)
    frames = [S.SimFrame(0, 0, 0.0, 150.0, [100.0]), S.SimFrame(1, 1, 10.0, 145.0, [40.0])]
    return S.simulate(frames, cfg, delay_quantum_us=quantum)


@pytest.mark.timeout(60)
def test_des_delay_and_wake_up_hand_example():
    for quantum, t_rel in ((50.0, 60.0), (30.0, 70.0)):
        r = _delay_case(quantum)
        assert r.releases == [(0.0, [(0, 0)], 0), (t_rel, [(1, 0)], 0)], quantum
        assert r.done == {0: 100.0, 1: 140.0} and r.missed == {0: False, 1: False}


def test_des_gpu_queue_runs_lower_levels_first():
    # A (level 1) holds the GPU 0..30.  C (chain 2, slack 1945, less urgent than A: rank 1 of 2
    # -> level 1 + floor(1 * 5 / 2) = 3) is released at t=5 and queues; B (chain 1, slack 50,
    # UL 0.02 > TH -> reserved level 0) is released at t=10 and queues behind it.  When A
    # completes, the queue hands the GPU to the lower level first: B runs 30..70, C 70..120.
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=1, max_closed=0, th_urgent=0.015, num_pri=6)
    frames = [S.SimFrame(0, 0, 0.0, 1000.0, [30.0]), S.SimFrame(1, 2, 5.0, 2000.0, [50.0]),
              S.SimFrame(2, 1, 10.0, 100.0, [40.0])]
    r = S.simulate(frames, cfg)
    assert r.releases == [(0.0, [(0, 0)], 1), (5.0, [(1, 0)], 3), (10.0, [(2, 0)], 0)]
    assert r.done == {0: 30.0, 2: 70.0, 1: 120.0}
    assert not any(r.missed.values())


def test_des_two_servers_hand_example():
    # X (100 us) and Y (60 us) are released at t=0 (X first: less slack) and, with two servers,
    # both start at once; Z (20 us) arrives at t=10, queues, and starts when Y frees its server
    # at 60.  Levels: X alone -> 1; Y ranks behind X (1 of 2) -> 3; Z behind both (2 of 3) -> 4.
    # With one server the same releases run back to back.
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=1, max_closed=0, th_urgent=-1.0, num_pri=6)
    frames = [S.SimFrame(0, 0, 0.0, 1000.0, [100.0]), S.SimFrame(1, 1, 0.0, 1000.0, [60.0]),
              S.SimFrame(2, 2, 10.0, 1000.0, [20.0])]
    rel = [(0.0, [(0, 0)], 1), (0.0, [(1, 0)], 3), (10.0, [(2, 0)], 4)]
    two = S.simulate(frames, cfg, servers=2)
    assert two.releases == rel and two.done == {0: 100.0, 1: 60.0, 2: 80.0}
    one = S.simulate(frames, cfg, servers=1)
    assert one.releases == rel and one.done == {0: 100.0, 1: 160.0, 2: 180.0}


# ---------------------------------------------------------------- tight-deadline share (f_tight)

def test_tight_share_halves_exactly_the_seeded_chains():
    """Section 6.2: f_tight halves the deadlines of a share of the chains.  serving_chains halves
    floor(f_tight n + 1/2) chains' deadlines -- the first ones of a seeded permutation, so a
    larger share keeps a smaller one's chains -- and leaves every other deadline at its period."""
    from pp_synth import serving_chains, tight_chains
    for n in (10, 11, 33):
        prev = set()
        for share in (0.0, 0.2, 0.4, 0.7, 1.0):
            chains = serving_chains(n, mixed=True, tight=share)
            halved = {c.chain_id for c in chains if c.deadline_ms == c.period_ms / 2}
            kept = {c.chain_id for c in chains if c.deadline_ms == c.period_ms}
            assert len(halved) == math.floor(share * n + 0.5) and len(halved) + len(kept) == n
            assert halved == set(tight_chains(n, share))
            assert halved == set(int(c) for c in np.random.default_rng(1500).permutation(n)[:len(halved)])
            assert prev <= halved
            prev = halved
    with pytest.raises(ValueError):
        tight_chains(5, 1.5)


def _tight_des(share, policy):
    from pp_synth import arrival_times, serving_chains
    chains = serving_chains(33, mixed=True, tight=share)
    ev = arrival_times(chains, 500.0, rate=20.0, jitter_ms=0.5, seed=1400)
    by = {c.chain_id: c for c in chains}
    frames = [S.SimFrame(i, cid, t * 1e3, t * 1e3 + by[cid].deadline_ms * 0.01 * 1e3, [20.0 + n / 1000.0],
                         precision=by[cid].precision, period=by[cid].period_ms * 1e3)
              for i, (t, cid, n) in enumerate(ev)]
    if policy == "urgency":
        cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=1, max_closed=0, th_urgent=-1.0)
    else:
        cfg = S.PolicyConfig(policy=S.POLICY_FIFO, max_batch=1, max_closed=0, early_exit=False)
    return frames, S.simulate(frames, cfg)


def test_des_tight_share_sweep():
    """The f_tight sweep in the DES (33 chains at 20x the paper's rates, f_d = 0.01, one GPU
    server, ~85 % busy): each frame's deadline is its chain's (halved for the tight chains), the
    miss ratio rises with the tight share for both the urgency rule and FIFO, and the urgency
    rule misses no more than FIFO at any share (the paper's tight-deadline sweep)."""
    from pp_synth import tight_chains
    miss = {}
    for share in (0.0, 0.4, 0.8):
        tight = set(tight_chains(33, share))
        for pol in ("urgency", "fifo"):
            frames, r = _tight_des(share, pol)
            for f in frames:
                period_us = f.period
                rel = (f.deadline - f.t_arr) / 0.01
                assert math.isclose(rel, period_us / 2 if f.chain_id in tight else period_us, rel_tol=1e-9)
            miss[share, pol] = S.miss_ratio_of(r, frames)
    for pol in ("urgency", "fifo"):
        assert miss[0.0, pol] < miss[0.4, pol] < miss[0.8, pol], miss
    for share in (0.0, 0.4, 0.8):
        assert miss[share, "urgency"] <= miss[share, "fifo"], miss

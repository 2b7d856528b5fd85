"""Decision replay: the library's release rule (pp_policy_decide, C++) and the oracle's
decide() (Python) must take the same decision on every state -- same kind, same frames in the
same order, same stream level, same drops.  Pure host code: runs on the CPU."""
import numpy as np
import pytest

from oracle import sched as S


@pytest.fixture(scope="module")
def pp():
    from paper_2509_12207_gb300 import _build
    _build.build()
    import paper_2509_12207_gb300 as m
    return m


def _random_state(rng):
    t = float(rng.uniform(0, 1e5))
    n = int(rng.integers(0, 14))
    ready = []
    for i in range(n):
        # coarse grids make ties in slack, chain and arrival common
        t_arr = t - float(rng.choice([0, 100, 250, 1000, 5000]))
        D = float(rng.choice([500, 1000, 2000, 5000, 50000]))
        est = float(rng.choice([100, 400, 900, 3000]))
        ready.append(dict(frame_id=int(1000 + i * 7 % 13 + 20 * i), chain_id=int(rng.integers(0, 6)),
                          precision=int(rng.integers(0, 2)), t_arr_us=t_arr, deadline_us=t_arr + D,
                          est_gpu_us=est, est_cpu_us=float(rng.choice([0.0, 50.0])),
                          util=float(rng.choice([0.05, 0.1, 0.5, 1.0])),
                          period_us=float(rng.choice([0.0, 50000.0, 100000.0, 200000.0]))))
    active = [(int(rng.integers(0, 6)), float(rng.choice([-np.inf, 1e-5, 1e-4, 5e-4, 2e-3, 1e-2])))
              for _ in range(int(rng.integers(0, 6)))]
    cfg = dict(policy=int(rng.integers(0, 8)), max_batch=int(rng.integers(1, 9)),
               max_closed=int(rng.integers(0, 3)), num_pri=int(rng.integers(1, 7)),
               early_exit=int(rng.integers(0, 2)),
               th_urgent=float(rng.choice([0.0, -1.0, 1e-4, 1e-3])), util_exempt=0.1,
               eqdf_lambda=float(rng.choice([0.0, 0.5, 1.0, 2.0])))
    return t, ready, active, int(rng.integers(0, 4)), cfg


def _oracle(t, ready, active, closed, cfg):
    oc = S.PolicyConfig(policy=cfg["policy"], max_batch=cfg["max_batch"], max_closed=cfg["max_closed"],
                        th_urgent=cfg["th_urgent"], util_exempt=cfg["util_exempt"],
                        early_exit=bool(cfg["early_exit"]), num_pri=cfg["num_pri"],
                        eqdf_lambda=cfg["eqdf_lambda"])
    rr = [S.Ready(r["frame_id"], r["chain_id"], r["t_arr_us"], r["deadline_us"], r["est_gpu_us"],
                  r["est_cpu_us"], r["precision"], r["util"], r["period_us"]) for r in ready]
    aa = [S.Active(c, u) for c, u in active]
    return S.decide(t, rr, aa, closed, oc)


def test_replay_random_states(pp):
    rng = np.random.default_rng(2024)
    kinds = {}
    for _ in range(12000):
        t, ready, active, closed, cfg = _random_state(rng)
        kind, frames, level, drops = pp.policy_decide(cfg, t, ready, active, closed)
        d = _oracle(t, ready, active, closed, cfg)
        assert kind == d.kind, (cfg, ready, active, closed)
        assert drops == d.drops
        if kind == S.RELEASE:
            assert frames == d.frames
            assert level == d.level
        kinds[kind] = kinds.get(kind, 0) + 1
    # every kind of decision was exercised
    assert set(kinds) == {S.NONE, S.RELEASE, S.WAIT, S.DELAY}, kinds


@pytest.mark.parametrize("noise", [0.0, 0.3])
def test_replay_des_trace(pp, noise):
    """Replays every decision point of a discrete-event simulation through the library; with
    noise, the policy sees every frame's estimate scaled by its per-frame factor 1 + U[-eps,
    eps) while units run for the true durations (the estimation-error study)."""
    from pp_synth import noise_factors
    rng = np.random.default_rng(5)
    fac = noise_factors(41, range(300), noise)
    frames = []
    for i in range(300):
        t = float(i * 30 + rng.integers(0, 25))
        d = float(rng.integers(20, 150))
        frames.append(S.SimFrame(i, i % 7, t, t + float(rng.choice([200, 400, 900])),
                                 [d], precision=(i % 7) % 2, est=[d * fac[i]] if noise else None))
    cfg = S.PolicyConfig(policy=S.POLICY_URGENCY, max_batch=4, delta_eval_us=150.0, max_closed=2,
                         th_urgent=1.0 / 150.0, num_pri=6)
    calls = []
    orig = S.decide

    def spy(t, ready, active, closed, c):
        d = orig(t, ready, active, closed, c)
        calls.append((t, list(ready), list(active), closed, d))
        return d

    S.decide = spy
    try:
        S.simulate(frames, cfg, delay_quantum_us=50.0, unit_time=lambda ds: 15.0 + 0.6 * sum(ds))
    finally:
        S.decide = orig
    assert len(calls) > 300
    pc = dict(policy=cfg.policy, max_batch=cfg.max_batch, max_closed=cfg.max_closed, num_pri=cfg.num_pri,
              early_exit=int(cfg.early_exit), th_urgent=cfg.th_urgent, util_exempt=cfg.util_exempt)
    seen = set()
    for t, ready, active, closed, d in calls:
        rr = [dict(frame_id=r.frame_id, chain_id=r.chain_id, precision=r.precision, t_arr_us=r.t_arr,
                   deadline_us=r.deadline, est_gpu_us=r.est_gpu, est_cpu_us=r.est_cpu, util=r.util) for r in ready]
        kind, fr, level, drops = pp.policy_decide(pc, t, rr, [(a.chain_id, a.ul) for a in active], closed)
        assert (kind, drops) == (d.kind, d.drops)
        if kind == S.RELEASE:
            assert (fr, level) == (d.frames, d.level)
        seen.add(kind)
    assert S.RELEASE in seen and S.WAIT in seen


def test_replay_priorities(pp):
    """pp_policy_priority agrees with the oracle's priority() for every policy, including the
    degenerate cases (no estimate, no period, non-positive slack)."""
    rng = np.random.default_rng(11)
    for _ in range(3000):
        t, ready, active, closed, cfg = _random_state(rng)
        for r in ready[:3]:
            if rng.random() < 0.2:
                r["est_gpu_us"], r["est_cpu_us"] = 0.0, 0.0
            got = pp.policy_priority(cfg, t, r)
            f = S.Ready(r["frame_id"], r["chain_id"], r["t_arr_us"], r["deadline_us"], r["est_gpu_us"],
                        r["est_cpu_us"], r["precision"], r["util"], r["period_us"])
            want = S.priority(f, t, S.PolicyConfig(policy=cfg["policy"], eqdf_lambda=cfg["eqdf_lambda"]))
            assert got == want or (np.isnan(got) and np.isnan(want)), (cfg["policy"], r, got, want)


@pytest.mark.parametrize("policy", [S.POLICY_EDF, S.POLICY_SJF, S.POLICY_HRRN, S.POLICY_LCUF,
                                    S.POLICY_SAEDF, S.POLICY_EQDF])
def test_replay_des_trace_other_policies(pp, policy):
    """The comparison policies through a whole simulated run: every decision the DES takes is
    the library's decision on the same state."""
    rng = np.random.default_rng(9 + policy)
    frames = []
    for i in range(200):
        t = float(i * 35 + rng.integers(0, 25))
        frames.append(S.SimFrame(i, i % 5, t, t + float(rng.choice([200, 400, 900])),
                                 [float(rng.integers(20, 150))], precision=(i % 5) % 2,
                                 period=float([50000, 100000, 200000][i % 3])))
    cfg = S.PolicyConfig(policy=policy, max_batch=4, delta_eval_us=150.0, max_closed=2, num_pri=6)
    calls = []
    orig = S.decide

    def spy(t, ready, active, closed, c):
        d = orig(t, ready, active, closed, c)
        calls.append((t, list(ready), list(active), closed, d))
        return d
    S.decide = spy
    try:
        S.simulate(frames, cfg)
    finally:
        S.decide = orig
    assert len(calls) > 200
    pc = dict(policy=policy, max_batch=4, max_closed=2, num_pri=6, early_exit=1, th_urgent=0.0, util_exempt=0.1,
              eqdf_lambda=cfg.eqdf_lambda)
    for t, ready, active, closed, d in calls:
        rd = [dict(frame_id=f.frame_id, chain_id=f.chain_id, precision=f.precision, t_arr_us=f.t_arr,
                   deadline_us=f.deadline, est_gpu_us=f.est_gpu, est_cpu_us=f.est_cpu, util=f.util,
                   period_us=f.period) for f in ready]
        kind, fr, level, drops = pp.policy_decide(pc, t, rd, [(a.chain_id, a.ul) for a in active], closed)
        assert (kind, drops) == (d.kind, d.drops)
        if kind == S.RELEASE:
            assert (fr, level) == (d.frames, d.level)

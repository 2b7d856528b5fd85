"""The serving runtime's dispatcher, checked from the outside.

* Decision replay: the runtime logs every release decision with the inputs it was taken on
  (pp_config.decision_log); every logged decision of a contended mixed-precision serving run
  is replayed through the oracle's restatement of the release rule (oracle.sched.decide) and
  must agree exactly (kind, released frames in order, stream level, dropped frames), for the
  urgency policy, the FIFO baseline and each comparison policy.  Every completed frame must
  have been released by exactly one logged decision, at that decision's time and level.
* Device error path: a unit whose kernels find the sticky device error word set (what a
  bounded wait that ran out leaves) reports its frames as PP_FRAME_ERROR, not DONE, and once
  the word is cleared frames complete exactly again."""
import time

import numpy as np
import pytest

from oracle import pillars as O
from oracle import sched as S
from pp_synth import BACKBONE_SMALL, GEOM_SMALL, pillar_weights, uniform_cloud
from tests._util import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
import paper_2509_12207_gb300 as pp  # noqa: E402

DEV = "cuda:0"
W_SMALL = pillar_weights(BACKBONE_SMALL, 7)


def _ctx(**kw):
    knobs = dict(max_batch=4, cap_points=150000, units=2, th_urgent=-1.0, autotune=0)
    knobs.update(kw)
    cfg, keep = pp.make_config(GEOM_SMALL, BACKBONE_SMALL, W_SMALL, **knobs)
    return pp.Context(cfg), keep


def _drain(ctx, n, timeout_s=30.0):
    got = []
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        got += ctx.poll(64, timeout_us=100000)
    assert len(got) == n, (len(got), n)
    return got


def _oracle_decision(rec):
    c = rec["cfg"]
    cfg = S.PolicyConfig(policy=c["policy"], max_batch=c["max_batch"], max_closed=c["max_closed"],
                         th_urgent=c["th_urgent"], util_exempt=c["util_exempt"], early_exit=bool(c["early_exit"]),
                         num_pri=c["num_pri"], eqdf_lambda=c["eqdf_lambda"])
    ready = [S.Ready(f["frame_id"], f["chain_id"], f["t_arr_us"], f["deadline_us"], f["est_gpu_us"], f["est_cpu_us"],
                     f["precision"], f["util"], f["period_us"]) for f in rec["ready"]]
    active = [S.Active(ch, ul) for ch, ul in rec["active"]]
    return S.decide(rec["t_us"], ready, active, rec["closed_pending"], cfg)


# (policy, max_batch, graphs, max_closed, early exit, th_urgent): the urgency policy calibrates
# TH_urgent over the first frames (so reservation and delaying take part), the others as the
# serving benchmark runs them
POLICIES = {
    "urgency": (pp.PP_POLICY_URGENCY, 4, 1, 2, 1, 0.0),
    "fifo": (pp.PP_POLICY_FIFO, 1, 0, 0, 0, -1.0),
    "edf": (pp.PP_POLICY_EDF, 4, 1, 2, 0, -1.0),
    "sjf": (pp.PP_POLICY_SJF, 4, 1, 2, 0, -1.0),
    "hrrn": (pp.PP_POLICY_HRRN, 4, 1, 2, 0, -1.0),
    "lcuf": (pp.PP_POLICY_LCUF, 4, 1, 2, 0, -1.0),
    "saedf": (pp.PP_POLICY_SAEDF, 4, 1, 2, 0, -1.0),
    "eqdf": (pp.PP_POLICY_EQDF, 4, 1, 2, 0, -1.0),
}


@pytest.fixture(scope="module")
def serving_clouds():
    return [torch.from_numpy(uniform_cloud(150000, 4000 + k, GEOM_SMALL)).to(DEV) for k in range(4)]


@pytest.mark.parametrize("name", sorted(POLICIES))
def test_dispatcher_decisions_replay_through_oracle(name, serving_clouds):
    policy, mb, graphs, closed, ee, th = POLICIES[name]
    ctx, keep = _ctx(policy=policy, max_batch=mb, use_graphs=graphs, max_closed=closed, early_exit=ee,
                     th_urgent=th, th_calib_frames=16, units=3, decision_log=200000, delta_eval_us=300.0)
    try:
        # 12 chains, odd ones BF16; periods 2/4/8 ms; a third of them with deadlines short
        # enough (0.35 ms) that frames queue behind others, go late and (urgency) get dropped
        n_chains = 12
        for c in range(n_chains):
            period = [2.0, 4.0, 8.0][c % 3]
            dl = 0.35 if c % 4 == 1 else period
            ctx.register_chain(c, period, dl, pp.PP_BF16 if c % 2 else pp.PP_F32)
        rng = np.random.default_rng(5)
        arrivals = []
        for c in range(n_chains):
            period_us = [2000.0, 4000.0, 8000.0][c % 3]
            t = 2000.0 + rng.uniform(0, period_us)
            while t < 400000.0:
                arrivals.append((t, c, int(rng.integers(0, 4)), int(rng.integers(30000, 150001))))
                t += period_us
        arrivals.sort()
        rep = ctx.replay(arrivals, serving_clouds, timeout_us=20e6)
        assert rep["submitted"] + rep["rejected"] == len(arrivals)
        st = ctx.stats()
        log = ctx.decision_log()
        assert st["decisions"] == len(log) > 0
        assert st["device_errors"] == 0
    finally:
        ctx.destroy()
    kinds = {}
    for rec in log:
        d = _oracle_decision(rec)
        got = (rec["kind"], rec["frames"], rec["level"], sorted(rec["drops"]))
        want = (d.kind, d.frames, d.level, sorted(d.drops))
        assert got == want, (rec["t_us"], got, want)
        kinds[rec["kind"]] = kinds.get(rec["kind"], 0) + 1
    assert kinds.get(pp.PP_DECIDE_RELEASE, 0) > 0
    # every frame that ran was released by exactly one launched decision; every dropped frame
    # by exactly one drop
    released, dropped = {}, {}
    for rec in log:
        if rec["kind"] == pp.PP_DECIDE_RELEASE and rec["launched"]:
            for fid in rec["frames"]:
                assert fid not in released
                released[fid] = rec
        for fid in rec["drops"]:
            assert fid not in dropped
            dropped[fid] = rec
    assert len(released) == st["done"]
    assert len(dropped) == st["dropped"]
    if name != "urgency":
        assert not dropped                      # no early exit outside the urgency policy


def test_dispatcher_results_match_logged_releases(serving_clouds):
    """Each polled result carries the release time, stream level and unit size of the logged
    decision that released it."""
    ctx, keep = _ctx(policy=pp.PP_POLICY_URGENCY, max_batch=4, th_urgent=0.0, th_calib_frames=8, units=2,
                     decision_log=100000)
    try:
        for c in range(4):
            ctx.register_chain(c, 5.0, 5.0, pp.PP_BF16 if c % 2 else pp.PP_F32)
        res = []
        for k in range(40):
            rc, ids = ctx.submit_many([k % 4, (k + 1) % 4], [serving_clouds[k % 4], serving_clouds[(k + 1) % 4]])
            assert rc == pp.PP_OK
            res += ctx.poll(64, timeout_us=0)
        res += _drain(ctx, 80 - len(res))
        log = ctx.decision_log()
        by_frame = {}
        for rec in log:
            if rec["kind"] == pp.PP_DECIDE_RELEASE and rec["launched"]:
                for fid in rec["frames"]:
                    by_frame[fid] = rec
        for r in res:
            if r.status != pp.PP_FRAME_DONE:
                continue
            rec = by_frame[r.frame_id]
            assert r.t_release_us == rec["t_us"]
            assert r.level == rec["level"]
            assert r.batch == len(rec["frames"])
        ctx.release_many([r.frame_id for r in res])
    finally:
        ctx.destroy()


def test_unit_reports_device_error_word():
    """A release unit whose kernels find the device error word set reports its frames as
    PP_FRAME_ERROR (the convs skipped their stores); pp_poll still returns its results; once the
    word is cleared, frames complete exactly again."""
    cloud = uniform_cloud(30000, 3, GEOM_SMALL)
    ref = O.frame(cloud, GEOM_SMALL, BACKBONE_SMALL, W_SMALL)
    assert pp.device_error(clear=True) == 0
    ctx, keep = _ctx(units=1, precisions=1, max_batch=2)
    try:
        ctx.register_chain(0, 50.0, 50.0, pp.PP_F32)
        rc, _ = ctx.submit(0, cloud)
        assert rc == pp.PP_OK
        (r,) = _drain(ctx, 1)
        assert r.status == pp.PP_FRAME_DONE
        ctx.release(r.frame_id)
        try:
            pp.device_error_set(2)               # as an MMA wait that ran out would leave it
            for _ in range(3):
                assert ctx.submit(0, cloud)[0] == pp.PP_OK
            bad = _drain(ctx, 3)
        finally:
            code = pp.device_error(clear=True)
        assert code == 2
        assert all(r.status == pp.PP_FRAME_ERROR and r.missed for r in bad)
        st = ctx.stats()
        assert st["device_errors"] >= 1 and st["device_error_code"] == 2 and st["done"] == 1
        ctx.release_many([r.frame_id for r in bad])
        for _ in range(2):
            assert ctx.submit(0, cloud)[0] == pp.PP_OK
        good = _drain(ctx, 2)
        for r in good:
            assert r.status == pp.PP_FRAME_DONE
            assert r.num_pillars == ref["vox"]["num_pillars"]
            got = pp.result_tensor(r)[1:-1, 1:-1].float().cpu().numpy()
            assert rel_err(got, ref["blocks"][-1]) <= FP32_TOL
        ctx.release_many([r.frame_id for r in good])
    finally:
        ctx.destroy()


def test_stats_reset_starts_afresh():
    """pp_stats_reset zeroes the counters and latency samples (a warm-up excluded from a
    measurement) while the context keeps serving: frames after it are counted from zero."""
    ctx, keep = _ctx(units=1, precisions=2)
    try:
        ctx.register_chain(0, 50.0, 50.0, pp.PP_BF16)
        cloud = uniform_cloud(40000, 9, GEOM_SMALL)
        for _ in range(3):
            assert ctx.submit(0, cloud)[0] == pp.PP_OK
        ctx.release_many([r.frame_id for r in _drain(ctx, 3)])
        assert ctx.stats()["done"] == 3
        ctx.stats_reset()
        st = ctx.stats()
        assert st["done"] == st["submitted"] == st["missed"] == 0 and st["lat_p99_us"] == 0.0
        assert st["chain_frames"][0] == 0 and st["decisions"] == 0
        for _ in range(2):
            assert ctx.submit(0, cloud)[0] == pp.PP_OK
        ctx.release_many([r.frame_id for r in _drain(ctx, 2)])
        st = ctx.stats()
        assert st["done"] == st["submitted"] == st["chain_frames"][0] == 2 and st["lat_p99_us"] > 0
    finally:
        ctx.destroy()

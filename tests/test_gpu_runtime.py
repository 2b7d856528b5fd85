"""Whole front end through the C ABI: a release unit (pp_pipeline_*) with plain launches and
with its CUDA graphs, and the serving runtime (pp_create ... pp_destroy), checked against the
FP64 oracle; a frame's result is bit-identical alone and in a mixed batch; admission under the
HBM budget, early exit and shutdown with work in flight."""
import time

import numpy as np
import pytest

from oracle import pillars as O
from pp_synth import (BACKBONE_FULL, BACKBONE_SMALL, GEOM_FULL, GEOM_SMALL, config_points,
                      pillar_weights, uniform_cloud)
from tests._util import BF16_TOL, FP32_TOL, bf16_emulated_backbone, max_norm_err, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
import paper_2509_12207_gb300 as pp  # noqa: E402

DEV = "cuda:0"
W_SMALL = pillar_weights(BACKBONE_SMALL, 7)


def _ref(cloud, g=GEOM_SMALL, bb=BACKBONE_SMALL, w=W_SMALL):
    return O.frame(cloud, g, bb, w)


def _interior(t):
    return t[1:-1, 1:-1].float().cpu().numpy()


def _check_out(got, ref, prec, w=W_SMALL, bb=BACKBONE_SMALL):
    """FP32: per-element error (rel_err) <= 1e-4.  BF16: max error relative to the output's
    largest magnitude <= 2e-2 against the FP64 oracle with unrounded weights, and <= 8e-3
    against the oracle with the BF16 path's roundings emulated (a canvas value that sits on a
    bf16 rounding boundary may round one ulp apart on the two sides)."""
    if prec == pp.PP_F32:
        assert rel_err(got, ref["blocks"][-1]) <= FP32_TOL
    else:
        assert max_norm_err(got, ref["blocks"][-1]) <= BF16_TOL
        emu = bf16_emulated_backbone(ref["canvas"], w[2], w[3], bb.layers(64))
        assert max_norm_err(got, emu) <= 8e-3


@pytest.fixture(scope="module")
def small_clouds():
    return [config_points(3, 0, 61000), config_points(1, 0), config_points(3, 1, 150000)]


@pytest.mark.parametrize("prec", [pp.PP_F32, pp.PP_BF16])
def test_pipeline_batch_and_graph(prec, small_clouds):
    cfg, keep = pp.make_config(GEOM_SMALL, BACKBONE_SMALL, W_SMALL, max_batch=4, cap_points=150000)
    p = pp.Pipeline(cfg, prec)
    try:
        frames = [torch.from_numpy(c).to(DEV) for c in small_clouds]
        refs = [_ref(c) for c in small_clouds]
        outs = {}
        for use_graph in (False, True):
            p.run(frames, use_graph=use_graph)
            torch.cuda.synchronize()
            for i, r in enumerate(refs):
                assert p.num_pillars(i) == r["vox"]["num_pillars"]
                o = p.output_tensor(i, 0)
                _check_out(_interior(o), r, prec)
                if use_graph:
                    assert torch.equal(o, outs[i])     # graph replay == plain launches, bitwise
                else:
                    outs[i] = o
        # the same frame alone (batch of 1) is bit-identical to its result in the batch
        p.run([frames[2]], use_graph=True)
        torch.cuda.synchronize()
        assert torch.equal(p.output_tensor(0, 0), outs[2])
    finally:
        p.destroy()


@pytest.mark.parametrize("prec", [pp.PP_F32, pp.PP_BF16])
def test_pipeline_canvas_follows_frame_sequences(prec):
    """A release unit keeps each slot's canvas from frame to frame: the bucket pass zeroes the
    cells the slot's previous frame drew that hold no pillar now, and the PointNet pass writes
    the new pillars.  Slots run different frames in turn (overlapping and disjoint cells, an
    empty frame, fewer frames than before) and every output matches the oracle of its own
    frame, so no stale pillar survives."""
    clouds = [uniform_cloud(n, 300 + i, GEOM_SMALL) for i, n in enumerate((60000, 20000, 150000, 0, 90000))]
    refs = [_ref(c) for c in clouds]
    cfg, keep = pp.make_config(GEOM_SMALL, BACKBONE_SMALL, W_SMALL, max_batch=2, cap_points=150000)
    p = pp.Pipeline(cfg, prec)
    try:
        dev = [torch.from_numpy(c).to(DEV) if len(c) else torch.zeros((0, 4), device=DEV) for c in clouds]
        for seq in ([0, 1], [2, 3], [1], [4, 0], [3, 2], [0]):
            p.run([dev[i] for i in seq])
            torch.cuda.synchronize()
            for slot, i in enumerate(seq):
                assert p.num_pillars(slot) == refs[i]["vox"]["num_pillars"], (seq, slot)
                _check_out(_interior(p.output_tensor(slot, 0)), refs[i], prec)
    finally:
        p.destroy()


def test_pipeline_stream_k(small_clouds):
    """With stream_k the autotuner may pick stream-K tiles for the 3xTF32 convs: results stay
    within the FP32 tolerance and are bit-reproducible launch to launch."""
    cfg, keep = pp.make_config(GEOM_SMALL, BACKBONE_SMALL, W_SMALL, max_batch=3, cap_points=150000, stream_k=1)
    p = pp.Pipeline(cfg, pp.PP_F32)
    try:
        frames = [torch.from_numpy(c).to(DEV) for c in small_clouds]
        p.run(frames)
        torch.cuda.synchronize()
        first = [p.output_tensor(i, 0).clone() for i in range(3)]
        for i, c in enumerate(small_clouds):
            _check_out(_interior(first[i]), _ref(c), pp.PP_F32)
        p.run(frames)
        torch.cuda.synchronize()
        assert all(torch.equal(p.output_tensor(i, 0), first[i]) for i in range(3))
    finally:
        p.destroy()


@pytest.fixture(scope="module")
def full_frame():
    w = pillar_weights(BACKBONE_FULL, 11)
    cloud = config_points(2, 0)
    return w, cloud, O.frame(cloud, GEOM_FULL, BACKBONE_FULL, w)


@pytest.mark.parametrize("cuda_cores", [0, 1])
def test_pipeline_full_size_fp32(cuda_cores, full_frame):
    """The full-size FP32 frame, with the convs on the tensor cores (3xTF32) and on CUDA cores."""
    w, cloud, ref = full_frame
    cfg, keep = pp.make_config(GEOM_FULL, BACKBONE_FULL, w, max_batch=1, cap_points=120000,
                               fp32_cuda_cores=cuda_cores)
    p = pp.Pipeline(cfg, pp.PP_F32)
    try:
        p.run([torch.from_numpy(cloud).to(DEV)])
        torch.cuda.synchronize()
        assert p.num_pillars(0) == ref["vox"]["num_pillars"] == GEOM_FULL.max_pillars
        for b in range(3):
            assert rel_err(_interior(p.output_tensor(0, b)), ref["blocks"][b]) <= FP32_TOL, b
    finally:
        p.destroy()


def test_runtime_full_size_all_blocks(full_frame):
    """The full-size frame through the serving runtime: every block's output, as copied into
    the frame's result slot by the unit's graph, matches the oracle."""
    w, cloud, ref = full_frame
    cfg, keep = pp.make_config(GEOM_FULL, BACKBONE_FULL, w, max_batch=2, cap_points=120000,
                               precisions=1, units=1, th_urgent=-1.0, keep_blocks=1)
    ctx = pp.Context(cfg)
    try:
        ctx.register_chain(0, 100.0, 100.0, pp.PP_F32)
        rc, ids = ctx.submit_many([0], [cloud])          # host memory, staged
        assert rc == pp.PP_OK
        dev_cloud = torch.from_numpy(cloud).to(DEV)
        rc, fid = ctx.submit(0, dev_cloud)              # device memory, read in place
        assert rc == pp.PP_OK
        res = _drain(ctx, 2)
        for r in res:
            assert r.num_pillars == ref["vox"]["num_pillars"]
            for b in range(3):
                assert rel_err(_interior(pp.result_tensor(r, b)), ref["blocks"][b]) <= FP32_TOL, b
        assert torch.equal(pp.result_tensor(res[0]), pp.result_tensor(res[1]))
        ctx.release_many([r.frame_id for r in res])
    finally:
        ctx.destroy()
    # by default a result slot keeps only the final output (the last block)
    cfg, keep = pp.make_config(GEOM_FULL, BACKBONE_FULL, w, max_batch=1, cap_points=120000,
                               precisions=1, units=1, th_urgent=-1.0, autotune=0)
    ctx = pp.Context(cfg)
    try:
        ctx.register_chain(0, 100.0, 100.0, pp.PP_F32)
        rc, ids = ctx.submit_many([0], [cloud])
        (r,) = _drain(ctx, 1)
        assert not r.block_dev[0] and not r.block_dev[1] and r.block_dev[2] == r.out_dev
        assert rel_err(_interior(pp.result_tensor(r)), ref["blocks"][2]) <= FP32_TOL
        ctx.release_many(ids)
    finally:
        ctx.destroy()


def _ctx(**kw):
    knobs = dict(max_batch=4, cap_points=150000, units=2, th_urgent=-1.0)
    knobs.update(kw)
    cfg, keep = pp.make_config(GEOM_SMALL, BACKBONE_SMALL, W_SMALL, **knobs)
    ctx = pp.Context(cfg)
    return ctx, keep


def _drain(ctx, n, timeout_s=30.0):
    got = []
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        got += ctx.poll(64, timeout_us=100000)
    assert len(got) == n, (len(got), n)
    return got


def test_runtime_serves_frames_exactly(small_clouds):
    ctx, keep = _ctx()
    try:
        ctx.register_chain(0, 50.0, 50.0, pp.PP_F32)
        ctx.register_chain(1, 100.0, 100.0, pp.PP_BF16)
        ids = {}
        dev_frames = [torch.from_numpy(c).to(DEV) for c in small_clouds]
        for i, c in enumerate(small_clouds):
            rc, fid = ctx.submit(0, c)                    # host memory, copied
            assert rc == pp.PP_OK
            ids[fid] = (0, i)
            rc, fid = ctx.submit(1, dev_frames[i])        # device memory, borrowed
            assert rc == pp.PP_OK
            ids[fid] = (1, i)
        res = _drain(ctx, len(ids))
        refs = [_ref(c) for c in small_clouds]
        for r in res:
            chain, i = ids[r.frame_id]
            assert r.status == pp.PP_FRAME_DONE and r.chain_id == chain
            assert r.num_pillars == refs[i]["vox"]["num_pillars"]
            assert r.t_done_us > r.t_release_us >= r.t_arr_us
            _check_out(_interior(pp.result_tensor(r)), refs[i], pp.PP_F32 if chain == 0 else pp.PP_BF16)
            ctx.release(r.frame_id)
        st = ctx.stats()
        assert st["done"] == len(ids) and st["dropped"] == 0
        assert st["chain_frames"][0] == 3 and st["chain_frames"][1] == 3
    finally:
        ctx.destroy()


def test_runtime_alone_vs_mix(small_clouds):
    # synchronous batches (each release waits for the previous one) so frames that arrive
    # while a unit runs accumulate and are released together
    ctx, keep = _ctx(delta_eval_us=0.0, max_closed=1)
    try:
        ctx.register_chain(3, 100.0, 100.0, pp.PP_BF16)
        ctx.register_chain(4, 100.0, 100.0, pp.PP_BF16)
        probe = small_clouds[1]
        rc, fid = ctx.submit(3, probe)
        (r,) = _drain(ctx, 1)
        assert r.batch == 1
        alone = pp.result_tensor(r)
        ctx.release(r.frame_id)
        others = [uniform_cloud(n, 50 + n, GEOM_SMALL) for n in (30000, 90000, 140000, 60000, 120000, 45000, 80000)]
        want = None
        # the probe among other frames: units fill up, later frames share units
        dev = [torch.from_numpy(c).to(DEV) for c in others]
        probe_dev = torch.from_numpy(probe).to(DEV)
        torch.cuda.synchronize()
        for k, c in enumerate(dev):
            ctx.submit(4, c)
            if k == 3:
                _, want = ctx.submit(3, probe_dev)
        res = _drain(ctx, len(others) + 1)
        mix = [r for r in res if r.frame_id == want][0]
        assert mix.status == pp.PP_FRAME_DONE
        assert torch.equal(pp.result_tensor(mix), alone)
        assert max(r.batch for r in res) > 1       # some frames did share a unit
        for r in res:
            ctx.release(r.frame_id)
    finally:
        ctx.destroy()


def test_runtime_admission_budget_and_early_exit():
    ctx, keep = _ctx(units=1, precisions=1, max_admitted=4)   # FP32 only, 4 result slots
    try:
        ctx.register_chain(0, 50.0, 50.0, pp.PP_F32)
        cloud = uniform_cloud(30000, 3, GEOM_SMALL)
        ids = []
        for _ in range(4):
            rc, fid = ctx.submit(0, cloud)
            assert rc == pp.PP_OK
            ids.append(fid)
        rc, _ = ctx.submit(0, cloud)
        assert rc == pp.PP_EAGAIN                 # budget: 4 admitted, none released yet
        res = _drain(ctx, 4)
        assert all(r.status == pp.PP_FRAME_DONE for r in res)   # one unit, reused at completion
        rc, _ = ctx.submit(0, cloud)
        assert rc == pp.PP_EAGAIN                 # results still held
        for r in res:
            ctx.release(r.frame_id)
        # a frame whose deadline has already passed is dropped before release (early exit)
        now = pp.now_us()
        rc, late = ctx.submit(0, cloud, t_arrival_us=now - 5000.0, abs_deadline_us=now - 1000.0)
        assert rc == pp.PP_OK
        (r,) = _drain(ctx, 1)
        assert r.frame_id == late and r.status == pp.PP_FRAME_DROPPED and r.missed
        ctx.release(late)
        st = ctx.stats()
        assert st["rejected"] == 2 and st["dropped"] == 1
    finally:
        ctx.destroy()


def test_runtime_fifo_baseline_and_destroy_in_flight():
    ctx, keep = _ctx(policy=pp.PP_POLICY_FIFO, max_batch=1, use_graphs=0, max_closed=0, units=4)
    ctx.register_chain(0, 50.0, 50.0, pp.PP_F32)
    ctx.register_chain(1, 50.0, 50.0, pp.PP_BF16)
    for k in range(6):
        ctx.submit(k % 2, uniform_cloud(40000, k, GEOM_SMALL))
    ctx.destroy()          # bounded wait for in-flight units, then frees everything


@pytest.mark.parametrize("host", [False, True])
def test_runtime_submit_many_one_unit(host):
    """Frames submitted together (pp_submit_frames) become ready together and run as one unit
    of uneven point counts; their result copies (made inside the unit's graph) are exact, and
    they are returned in one pp_result_release_many."""
    ctx, keep = _ctx(max_batch=8, delta_eval_us=0.0, max_closed=1)
    try:
        ctx.register_chain(0, 100.0, 100.0, pp.PP_F32)
        clouds = [uniform_cloud(n, 70 + i, GEOM_SMALL)
                  for i, n in enumerate((30000, 150000, 0, 61000, 90000, 1, 120000, 45000))]
        frames = clouds if host else [torch.from_numpy(c).to(DEV) for c in clouds]
        torch.cuda.synchronize()
        rc, ids = ctx.submit_many([0] * 8, frames)
        assert rc == pp.PP_OK and len(ids) == 8
        res = {r.frame_id: r for r in _drain(ctx, 8)}
        assert sorted(res) == sorted(ids)
        assert all(r.status == pp.PP_FRAME_DONE and r.batch == 8 for r in res.values())
        for i in (1, 2, 5, 7):
            ref = _ref(clouds[i])
            r = res[ids[i]]
            assert r.num_pillars == ref["vox"]["num_pillars"]
            for b in range(len(BACKBONE_SMALL.convs)):
                assert rel_err(_interior(pp.result_tensor(r, b)), ref["blocks"][b]) <= FP32_TOL, (i, b)
        ctx.release_many(ids)
        with pytest.raises(pp.PPError):
            ctx.release_many(ids[:1])           # already released
    finally:
        ctx.destroy()


def test_runtime_submit_many_partial_admission():
    ctx, keep = _ctx(units=1, precisions=1, max_admitted=4)
    try:
        ctx.register_chain(0, 50.0, 50.0, pp.PP_F32)
        cloud = uniform_cloud(20000, 5, GEOM_SMALL)
        rc, ids = ctx.submit_many([0] * 6, [cloud] * 6)
        assert rc == pp.PP_EAGAIN and len(ids) == 4   # admitted in order until the budget is full
        res = _drain(ctx, 4)
        assert sorted(r.frame_id for r in res) == sorted(ids)
        ctx.release_many(ids)
        assert ctx.stats()["rejected"] == 2
    finally:
        ctx.destroy()


@pytest.mark.parametrize("policy", [pp.PP_POLICY_EDF, pp.PP_POLICY_SJF, pp.PP_POLICY_HRRN, pp.PP_POLICY_LCUF,
                                    pp.PP_POLICY_SAEDF, pp.PP_POLICY_EQDF])
def test_runtime_comparison_policies(policy, small_clouds):
    """The comparison release orders serve every frame, with results identical to the oracle's
    pillars and within tolerance."""
    ctx, keep = _ctx(policy=policy, max_batch=4, th_urgent=-1.0, early_exit=0)
    try:
        ctx.register_chain(0, 50.0, 50.0, pp.PP_BF16)
        ctx.register_chain(1, 200.0, 200.0, pp.PP_BF16)
        dev = [torch.from_numpy(c).to(DEV) for c in small_clouds]
        ids = {}
        for i, c in enumerate(dev):
            for chain in (0, 1):
                rc, fid = ctx.submit(chain, c)
                assert rc == pp.PP_OK
                ids[fid] = i
        res = _drain(ctx, len(ids))
        refs = [_ref(c) for c in small_clouds]
        for r in res:
            assert r.status == pp.PP_FRAME_DONE
            assert r.num_pillars == refs[ids[r.frame_id]]["vox"]["num_pillars"]
        ctx.release_many([r.frame_id for r in res])
    finally:
        ctx.destroy()


def test_runtime_replay_trace():
    """pp_replay submits a timed trace from the library's own thread loop: every frame is
    accounted for (admitted or rejected), every admitted frame completes, submissions keep to
    the schedule, and malformed traces are rejected before anything runs."""
    ctx, keep = _ctx(max_batch=4, max_admitted=16)
    try:
        ctx.register_chain(0, 20.0, 20.0, pp.PP_BF16)
        ctx.register_chain(1, 40.0, 40.0, pp.PP_BF16)
        clouds = [torch.from_numpy(uniform_cloud(n, 90 + n, GEOM_SMALL)).to(DEV) for n in (30000, 150000)]
        arrivals = [(1000.0 + 500.0 * k, k % 2, k % 2, [30000, 150000][k % 2] - 7 * k) for k in range(80)]
        rep = ctx.replay(arrivals, clouds, timeout_us=5e6)
        assert rep["submitted"] + rep["rejected"] == 80
        assert rep["completed"] + rep["dropped"] == rep["submitted"]
        assert rep["submit_late_us_mean"] < 2000.0
        st = ctx.stats()
        assert st["done"] + st["dropped"] == rep["submitted"]
        with pytest.raises(pp.PPError):
            ctx.replay(list(reversed(arrivals)), clouds)          # not sorted by time
        with pytest.raises(pp.PPError):
            ctx.replay([(0.0, 0, 0, 40000)], clouds)              # more points than the cloud has
    finally:
        ctx.destroy()


def test_runtime_batched_bf16_unit_full_workload():
    """The 8-frame BF16 workload exactly as the bench runs it (uneven 30k-150k frames of the
    0.32 m grid submitted together into one unit of a graph-launched, autotuned context):
    every frame's pillars match the oracle exactly and its backbone output is within the BF16
    tolerance (and within 8e-3 of the oracle with BF16 roundings emulated)."""
    from pp_synth import batched_counts
    counts = batched_counts(3)
    clouds = [config_points(3, k, n) for k, n in enumerate(counts)]
    ctx, keep = _ctx(max_batch=8, units=2, precisions=2, early_exit=0)
    try:
        ctx.register_chain(0, 10000.0, 10000.0, pp.PP_BF16)
        dev = [torch.from_numpy(c).to(DEV) for c in clouds]
        rc, ids = ctx.submit_many([0] * 8, dev)
        assert rc == pp.PP_OK
        res = {r.frame_id: r for r in _drain(ctx, 8)}
        assert all(r.batch == 8 for r in res.values())
        for k, fid in enumerate(ids):
            ref = _ref(clouds[k])
            r = res[fid]
            assert r.num_pillars == ref["vox"]["num_pillars"]
            _check_out(_interior(pp.result_tensor(r)), ref, pp.PP_BF16)
        ctx.release_many(ids)
    finally:
        ctx.destroy()


def _submit_batched_or_alone(ctx, pinned, together, **kw):
    """Submits the frames together (one release unit batching them) or one at a time, each
    polled before the next (one-frame units); returns (ids, results by id)."""
    if together:
        rc, ids = ctx.submit_many([0] * len(pinned), pinned, **kw)
        assert rc == pp.PP_OK
        res = {r.frame_id: r for r in _drain(ctx, len(ids))}
        assert max(r.batch for r in res.values()) > 1  # the batched path did run
        return ids, res
    ids, res = [], {}
    for k in range(len(pinned)):
        one = {key: v[k:k + 1] for key, v in kw.items()}
        rc, got = ctx.submit_many([0], pinned[k:k + 1], **one)
        assert rc == pp.PP_OK and len(got) == 1
        ids += got
        for r in _drain(ctx, 1):
            assert r.batch == 1
            res[r.frame_id] = r
    return ids, res


@pytest.mark.parametrize("together", [True, False], ids=["batched-unit", "one-frame-units"])
def test_runtime_pinned_host_points(small_clouds, together):
    """Page-locked host frames are borrowed without a staging copy (a batched unit copies them by
    copy engine, a one-frame unit reads them in place over the host link): results match the
    oracle exactly as device frames do; pageable memory is refused in that mode."""
    import ctypes
    ctx, keep = _ctx(max_batch=4)
    try:
        ctx.register_chain(0, 100.0, 100.0, pp.PP_F32)
        pinned = [torch.from_numpy(c).pin_memory() for c in small_clouds]
        ids, res = _submit_batched_or_alone(ctx, pinned, together)
        for k, fid in enumerate(ids):
            ref = _ref(small_clouds[k])
            assert res[fid].num_pillars == ref["vox"]["num_pillars"]
            _check_out(_interior(pp.result_tensor(res[fid])), ref, pp.PP_F32)
        ctx.release_many(ids)
        pageable = np.ascontiguousarray(small_clouds[0])
        fid = ctypes.c_uint64(0)
        rc = pp.lib().pp_submit_frame(ctx.h, 0, pageable.ctypes.data, 1000, pp.PP_POINTS_PINNED,
                                      pp.now_us(), 0.0, ctypes.byref(fid))
        assert rc == pp.PP_EINVAL and b"page-locked" in pp.lib().pp_last_error()
    finally:
        ctx.destroy()


# ---- neck + detection head inside the release unit

@pytest.fixture(scope="module")
def full_head(full_frame):
    """Neck/head weights for the full-size network and the oracle's neck and head maps of the
    full-size frame."""
    from pp_synth import head_weights
    w, cloud, ref = full_frame
    hw = head_weights(BACKBONE_FULL)
    neck = O.neck(ref["blocks"], hw[0], hw[1])
    return hw, neck, O.head(neck, hw[2], hw[3])


def test_pipeline_neck_head_full_size_fp32(full_frame, full_head):
    """The full-size FP32 unit with the neck and head (three transposed convs of strides 1, 2, 4
    into one 384-channel map, then 72 outputs padded to 128): both maps match the oracle run
    end to end from the points; the padding channels are zero."""
    w, cloud, ref = full_frame
    hw, neck_ref, head_ref = full_head
    cfg, keep = pp.make_config(GEOM_FULL, BACKBONE_FULL, w, head=hw, max_batch=1, cap_points=120000)
    p = pp.Pipeline(cfg, pp.PP_F32)
    try:
        p.run([torch.from_numpy(cloud).to(DEV)])
        torch.cuda.synchronize()
        neck = p.output_tensor(0, -3)
        head = p.output_tensor(0, -2)
        assert neck.shape == (250, 218, 384) and head.shape == (250, 218, 128)
        assert rel_err(_interior(neck), neck_ref) <= FP32_TOL
        h = _interior(head)
        assert rel_err(h[..., :72], head_ref) <= FP32_TOL
        assert not h[..., 72:].any()
        for t in (neck, head):   # borders stay zero
            assert not t[0].any() and not t[-1].any() and not t[:, 0].any() and not t[:, -1].any()
    finally:
        p.destroy()


def test_pipeline_full_size_bf16_blocks(full_frame):
    """The full-size frame through a BF16 unit, block by block: each block output within the
    BF16 tolerance of the FP64 oracle (unrounded weights), and of the oracle's block applied to
    the unit's own (BF16) input of that block, so that one block's error cannot hide behind
    another's."""
    w, cloud, ref = full_frame
    cfg, keep = pp.make_config(GEOM_FULL, BACKBONE_FULL, w, max_batch=1, cap_points=120000)
    p = pp.Pipeline(cfg, pp.PP_BF16)
    try:
        p.run([torch.from_numpy(cloud).to(DEV)])
        torch.cuda.synchronize()
        assert p.num_pillars(0) == ref["vox"]["num_pillars"]
        blocks = [_interior(p.output_tensor(0, b)).astype(np.float64) for b in range(3)]
    finally:
        p.destroy()
    layers = BACKBONE_FULL.layers(64)
    ends = list(np.cumsum(BACKBONE_FULL.convs) - 1)
    x, start = ref["canvas"], 0
    for b, end in enumerate(ends):
        assert max_norm_err(blocks[b], ref["blocks"][b]) <= BF16_TOL, b
        r = x
        for l in range(start, end + 1):
            r = O.conv3x3_bn_relu(r, w[2][l], w[3][l], layers[l][2])
        assert max_norm_err(blocks[b], r) <= BF16_TOL, b
        x, start = blocks[b], end + 1


def test_pipeline_neck_head_bf16(full_frame, full_head):
    """BF16 unit with the neck and head: each stage against the oracle applied to the unit's
    own (BF16) input of that stage, weights unrounded; the head end to end within the BF16
    tolerance of the FP64 oracle."""
    w, cloud, ref = full_frame
    hw, neck_ref, head_ref = full_head
    cfg, keep = pp.make_config(GEOM_FULL, BACKBONE_FULL, w, head=hw, max_batch=2, cap_points=120000)
    p = pp.Pipeline(cfg, pp.PP_BF16)
    try:
        p.run([torch.from_numpy(cloud).to(DEV)] * 2)
        torch.cuda.synchronize()
        blocks = [_interior(p.output_tensor(0, b)).astype(np.float64) for b in range(3)]
        neck = _interior(p.output_tensor(0, -3)).astype(np.float64)
        head = _interior(p.output_tensor(0, -2))
        assert max_norm_err(neck, O.neck(blocks, hw[0], hw[1])) <= BF16_TOL
        assert max_norm_err(head[..., :72], O.head(neck, hw[2], hw[3])) <= BF16_TOL
        assert not head[..., 72:].any()
        assert max_norm_err(head[..., :72], head_ref) <= BF16_TOL
        assert torch.equal(p.output_tensor(0, -2), p.output_tensor(1, -2))
    finally:
        p.destroy()


def test_runtime_serves_head_maps(full_frame, full_head):
    """Through the serving runtime with a head: each result carries the head map (out_c 128,
    out_valid_c 72, no block outputs), equal to the oracle's."""
    w, cloud, ref = full_frame
    hw, neck_ref, head_ref = full_head
    cfg, keep = pp.make_config(GEOM_FULL, BACKBONE_FULL, w, head=hw, max_batch=2, cap_points=120000,
                               precisions=1, units=1, th_urgent=-1.0)
    ctx = pp.Context(cfg)
    try:
        ctx.register_chain(0, 100.0, 100.0, pp.PP_F32)
        rc, ids = ctx.submit_many([0, 0], [cloud, cloud])
        assert rc == pp.PP_OK
        res = _drain(ctx, 2)
        for r in res:
            assert (r.out_c, r.out_valid_c, r.out_h, r.out_w) == (128, 72, 248, 216)
            assert not any(r.block_dev)
            h = _interior(pp.result_tensor(r))
            assert rel_err(h[..., :72], head_ref) <= FP32_TOL
            assert not h[..., 72:].any()
        ctx.release_many(ids)
    finally:
        ctx.destroy()


def test_runtime_synthetic_load_chain(small_clouds):
    """A synthetic-load chain (kernels of set duration and SM share) served beside a pillar
    chain: its frames complete with no outputs after about n_kernels x kernel_us of device time,
    one per unit; the pillar frames stay exact; bad arguments are refused."""
    ctx, keep = _ctx(max_batch=4)
    try:
        ctx.register_chain(0, 100.0, 100.0, pp.PP_F32)
        ctx.register_synthetic_chain(1, 100.0, 100.0, 4, 200.0, 0.5)
        with pytest.raises(pp.PPError):
            ctx.register_synthetic_chain(1, 100.0, 100.0, 4, 200.0, 0.5)     # already registered
        for bad in [(0, 200.0, 0.5), (4, 0.5, 0.5), (4, 200.0, 0.0), (4, 200.0, 1.5), (300, 200.0, 0.5)]:
            with pytest.raises(pp.PPError):
                ctx.register_synthetic_chain(2, 100.0, 100.0, *bad)
        empty = np.zeros((0, 4), np.float32)
        rc, sids = ctx.submit_many([1, 1, 1], [empty, empty, empty])
        assert rc == pp.PP_OK and len(sids) == 3
        rc, pids = ctx.submit_many([0, 0], small_clouds[:2])
        assert rc == pp.PP_OK
        res = {r.frame_id: r for r in _drain(ctx, 5)}
        for fid in sids:
            r = res[fid]
            assert r.status == pp.PP_FRAME_DONE and not r.out_dev and r.out_dtype == -1 and r.batch == 1
            assert 300.0 <= r.t_done_us - r.t_release_us <= 20000.0, r.t_done_us - r.t_release_us
        for k, fid in enumerate(pids):
            assert res[fid].num_pillars == _ref(small_clouds[k])["vox"]["num_pillars"]
        st = ctx.stats()
        assert st["chain_frames"][1] == 3 and st["chain_frames"][0] == 2
        ctx.release_many(sids + pids)
    finally:
        ctx.destroy()


@pytest.mark.parametrize("together", [True, False], ids=["batched-unit", "one-frame-units"])
def test_runtime_host_output_buffers(small_clouds, together):
    """Frames submitted with page-locked host output buffers (written by copy engine for a
    batched unit, by the result copy kernel for a one-frame unit): when polled, each buffer
    holds exactly the frame's final output; pageable memory is refused and admits nothing."""
    ctx, keep = _ctx(max_batch=4)
    try:
        ctx.register_chain(0, 100.0, 100.0, pp.PP_F32)
        nbytes = ctx.result_bytes(pp.PP_F32)
        assert nbytes > 0
        outs = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in small_clouds]
        dev = [torch.from_numpy(c).to(DEV) for c in small_clouds]
        ids, res = _submit_batched_or_alone(ctx, dev, together, host_out=outs)
        for k, fid in enumerate(ids):
            r = res[fid]
            assert r.out_host
            assert torch.equal(pp.result_host_tensor(r), pp.result_tensor(r).cpu())
            _check_out(_interior(pp.result_host_tensor(r)), _ref(small_clouds[k]), pp.PP_F32)
        ctx.release_many(ids)
        with pytest.raises(pp.PPError):
            ctx.submit_many([0], dev[:1], host_out=[torch.empty(nbytes, dtype=torch.uint8)])
        assert ctx.stats()["submitted"] == len(ids)
    finally:
        ctx.destroy()

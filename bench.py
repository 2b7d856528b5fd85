"""Benchmark of the pillar front end on GB300 through the library's public C ABI.

Default workload: full-size single frame, FP32 -- 120,000 points (70 % in 40 Gaussian blobs),
0.16 m grid 432 x 496, 12,000 pillars x 32 points, PointNet 9->64, backbone 64/128/256 channels
x 4/6/6 conv3x3 at strides 2/2/2.  One step = one frame through the whole hot path: admission
(pp_submit_frame), release by the urgency rule, one graph launch (voxelise, PointNet, scatter,
16 convs), completion (pp_poll) and release of the result.

Prints one JSON line: frames/s with inputs resident in HBM (value), the same through host
buffers with the H2D copy and a D2H read of the result inside the timed region (e2e), the conv
kernels' roofline (FP32 FMA bound), the oracle's CPU baseline, clocks seen during the run.
Multi-GPU: replicas only (frames are independent); rank 0 prints the aggregate.
``--impl reference`` times the FP64 CPU oracle on the same workload (one frame per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "cfg2-fp32": "full-size single frame FP32: 120k clustered points, 432x496 grid, 12000 pillars, "
                 "backbone 64/128/256 x 4/6/6 conv3x3 strides 2/2/2",
    "cfg1-fp32": "single frame FP32: 20k uniform points, 216x248 grid, 4000 pillars, 3 conv3x3 64ch",
    "cfg3-bf16": "batched BF16: 8 frames of 30k-150k uniform points per unit, 216x248 grid, 3 conv3x3 64ch",
}

# (chains, steps in flight) of the throughput run: the steps alternate between the chains (a
# chain's units run in order on its streams; units of different chains overlap on the GPU).
# Measured: full-size frame 2,470 frames/s at 3 x 4 and 4 x 4 against 2,344 at 2 x 3 and
# 2,333-2,383 at 4 x 6, 6 x 6, 8 x 8 (a unit's front end then overlaps another's convolutions
# without queueing so deep that units contend); the 8-frame unit's short kernels keep more in
# flight busy
SERVING_SHAPE = {"cfg3-bf16": (3, 6), "cfg1-fp32": (2, 3)}
SERVING_SHAPE_DEFAULT = (4, 4)

REFERENCE_BUDGET_S = 90  # wall-clock cap of the reference arm's timed steps

HEAD_NOTE = ", + neck (transposed convs to 128 channels each, concatenated) and 1x1 head (72 outputs)"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2-fp32", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--head", action="store_true",
                    help="the step also runs the neck (upsample + concat) and the detection head")
    ap.add_argument("--no-clocks", action="store_true", help="do not sample nvidia-smi (profiling runs)")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the raw nvidia-smi samples of the timed region "
                         "(bench_clocks_<pid>.csv; default: the system temporary directory)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving comparison")
    ap.add_argument("--no-batched", action="store_true",
                    help="with the default workload, skip the 8-frame BF16 unit run reported under batched_bf16")
    ap.add_argument("--fp32-cuda-cores", action="store_true", help="FP32 convs on CUDA cores instead of 3xTF32")
    ap.add_argument("--stream-k", action="store_true",
                    help="let the autotuner also time the stream-K 3xTF32 conv tiles (config stream_k; "
                         "bit-reproducible here because every unit of the FP32 workloads holds one frame)")
    ap.add_argument("--depth", type=int, default=None,
                    help="steps in flight (1 = each step waits for the last; default per workload)")
    ap.add_argument("--chains", type=int, default=None,
                    help="sensor chains the steps alternate between (a chain's units run in order on its "
                         "own streams; units of different chains may overlap on the GPU; default per workload)")
    ap.add_argument("--tune-table", default=None,
                    help="conv tile table: loaded (no autotuning) if the file exists, else written after "
                         "autotuning, so that a profiled run launches the same tiles as a plain one")
    ap.add_argument("--serve-sweep", default=None,
                    help="run only the serving sweep: comma list of chains:rate:seconds[:mixed][:dfac][:noise]"
                         "[:util/kernel_us/frame_us] (the last: odd chains run synthetic kernels)")
    ap.add_argument("--serve-modes", default="urgency,plain",
                    help="release policies of the sweep: urgency, plain, edf, sjf, hrrn, lcuf, saedf, eqdf")
    ap.add_argument("--profile-conv", default=None,
                    help="LAYER:TILE[:REPS] -- launch only backbone layer LAYER of the workload (0-based, its input "
                         "random) with conv tile TILE, REPS times (default 3), and exit: a short process for a "
                         "profiler to capture one conv kernel")
    ap.add_argument("--profile-frontend", default=None, metavar="REPS",
                    help="launch only the voxelise + point selection + PointNet stage (pp_voxelize_pointnet) on "
                         "the workload's frames REPS times and exit: a short process for a profiler")
    ap.add_argument("--cpu-worker", default=None, help=argparse.SUPPRESS)
    a = ap.parse_args()
    chains, depth = SERVING_SHAPE.get(a.workload, SERVING_SHAPE_DEFAULT)
    a.chains = chains if a.chains is None else a.chains
    a.depth = depth if a.depth is None else a.depth
    return a


def _workload(name):
    from pp_synth import (BACKBONE_FULL, BACKBONE_SMALL, GEOM_FULL, GEOM_SMALL, batched_counts,
                          config_points, pillar_weights)
    if name == "cfg2-fp32":
        g, bb, prec, batch, cap = GEOM_FULL, BACKBONE_FULL, 0, 1, 120000
        frames = [config_points(2, k) for k in range(4)]
    elif name == "cfg1-fp32":
        g, bb, prec, batch, cap = GEOM_SMALL, BACKBONE_SMALL, 0, 1, 20000
        frames = [config_points(1, k) for k in range(4)]
    else:
        g, bb, prec, batch, cap = GEOM_SMALL, BACKBONE_SMALL, 1, 8, 150000
        counts = batched_counts(3)
        frames = [config_points(3, k, n) for k, n in enumerate(counts)]
    return g, bb, prec, batch, cap, frames, pillar_weights(bb, 7)


# DRAM bytes (read + write) of all conv launches of one step, from one-pass ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the sha256 of the conv source they
# were taken on: a changed kernel reports null until it is captured again.
CONV_TRAFFIC = {
    # per distinct layer shape, one launch each (bench.py --profile-conv LAYER:TILE with the
    # tuned tile), summed over the step's layers: full-size frame 119.10 + 3 x 28.30 + 28.57 +
    # 5 x 15.44 + 16.61 + 5 x 12.11 MB; 8-frame unit 56.40 + 2 x 14.30 MB
    "cfg2-fp32": (386.96e6, "85903ed2da2377408ed2145782c910963e4bc0278d0b31c7742d9d7985a06fc3"),
    "cfg3-bf16": (85.01e6, "85903ed2da2377408ed2145782c910963e4bc0278d0b31c7742d9d7985a06fc3"),
}
# the same for the neck and head launches of one step (upsamplings + head); not re-captured on the
# current conv source, so reported as null
NECK_HEAD_TRAFFIC = {
    "cfg2-fp32": (250.4e6, "66563541ec5512d479f1ac7b165d18ef09f7cffc2ec9cd36b8ec5f3f07b2bac5"),
    "cfg3-bf16": (42.3e6, "66563541ec5512d479f1ac7b165d18ef09f7cffc2ec9cd36b8ec5f3f07b2bac5"),
}


def _conv_traffic(workload, table=None):
    import hashlib
    ent = (CONV_TRAFFIC if table is None else table).get(workload)
    if ent is None:
        return None
    src = os.path.join(ROOT, "paper_2509_12207_gb300", "csrc", "conv_tc.cu")
    with open(src, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    return ent[0] if digest == ent[1] else None


def _front_end_roofline(g, stages, elt, peaks):
    """HBM roofline of the voxelise and scatter stages of one step: algorithmic bytes (per frame:
    voxelise reads 16 B per point, reads and writes the 4-byte count of every cell, writes 32
    float4 points plus 8 B of coordinates per kept pillar; the incremental scatter reads 256 B of
    features and 4 B of coordinates per kept pillar, writes its 64 channels and 4 B of drawn list,
    and zeroes the 64 channels of every stale cell after reading its 4-byte drawn entry and cell
    map entry; the dense scatter writes the whole padded canvas) over the stage's device time."""
    peak = float(peaks.get("hbm_gbs", 6800.0))
    G = g.nx * g.ny
    canvas_px = (g.nx + 2) * (g.ny + 2)  # elt: canvas bytes per channel (8 = split FP32)
    vox = sum(16 * n + 8 * G + (16 * 32 + 8) * p for n, p in zip(stages["_npoints"], stages["_npillars"]))
    # the release unit's voxelise + PointNet: the same minus the gathered-point writes, plus the
    # gathered points read once (16 B each) and the 256-byte feature row written per pillar
    vpn = sum(16 * n + 8 * G + (8 + 256) * p + 16 * k
              for n, p, k in zip(stages["_npoints"], stages["_npillars"], stages["_gathered"]))
    sca = stages["_scatter_bytes"]
    dense = sum(256 * p + 64 * canvas_px * elt for p in stages["_npillars"])
    res = {"unit": "GB/s", "peak": peak, "peak_source": "hbm_gbs of measured" if "hbm_gbs" in peaks else "fallback"}
    for name, b in (("voxelize_pointnet", vpn), ("voxelize", vox), ("scatter", sca), ("scatter_dense", dense)):
        gbs = b / (stages[name] * 1e-3) / 1e9
        res[name] = {"bytes": int(b), "achieved": gbs, "frac": gbs / peak}
    return res


def _conv_flops(g, bb):
    tot = 0
    H, W = g.ny, g.nx
    for ci, co, s in bb.layers(64):
        Ho, Wo = (H - 1) // s + 1, (W - 1) // s + 1
        tot += 2 * Ho * Wo * co * 9 * ci
        H, W = Ho, Wo
    return tot


# ------------------------------------------------------------------ CPU oracle (baseline)

def _oracle_seconds(name, min_s, head=False, max_frames=512):
    """Times the FP64 oracle on the workload's frames in turn (this process) until ``min_s``
    seconds of oracle work have run (at least one frame, at most ``max_frames``); returns
    (frames, seconds)."""
    from oracle import pillars as O
    g, bb, _prec, _batch, _cap, frames, w = _workload(name)
    hw = None
    if head:
        from pp_synth import head_weights
        hw = head_weights(bb)
    t0 = time.perf_counter()
    k = 0
    while k < max_frames and (k == 0 or time.perf_counter() - t0 < min_s):
        r = O.frame(frames[k % len(frames)], g, bb, w)
        if hw is not None:
            O.head(O.neck(r["blocks"], hw[0], hw[1]), hw[2], hw[3])
        k += 1
    return k, time.perf_counter() - t0


CPU_BASELINE_S = 10.0  # seconds of oracle work in the CPU baseline sample


def _cpu_baseline(name, head=False, min_s=CPU_BASELINE_S):
    """Runs the oracle single-threaded in a child process (BLAS pinned to one thread) on a
    bounded sample: whole frames until about ``min_s`` seconds of oracle work."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker",
                          "%s:%g:%d" % (name, min_s, 1 if head else 0),
                          "--workload", name], capture_output=True, text=True, env=env, timeout=900)
    if out.returncode != 0:
        return {"value": None, "unit": "frames/s", "cores": 1, "kind": "oracle",
                "sample": "failed: " + out.stderr[-300:]}
    n_frames, secs = out.stdout.strip().splitlines()[-1].split()
    n_frames, secs = int(n_frames), float(secs)
    return {"value": n_frames / secs, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": "%d full frame(s) of the workload through the FP64 NumPy oracle, one thread, %.1f s"
                      % (n_frames, secs)}


# ------------------------------------------------------------------ clocks

def _die_with_parent():
    """Child-side: ask Linux to SIGTERM this process when its parent exits (PR_SET_PDEATHSIG)."""
    try:
        import ctypes
        import signal
        ctypes.CDLL("libc.so.6", use_errno=True).prctl(1, signal.SIGTERM, 0, 0, 0)
    except OSError:
        pass


class _Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons while the timed region runs.
    Always stopped by the caller (try/finally); the child also dies with this process and is
    killed by a watchdog after `max_s` seconds."""

    def __init__(self, gpu_index, enabled=True, max_s=600.0, out_dir=None):
        import tempfile
        self.p = None
        self.path = os.path.join(out_dir or tempfile.gettempdir(), "bench_clocks_%d.csv" % os.getpid())
        if not enabled:
            return
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f, stderr=subprocess.DEVNULL,
                preexec_fn=_die_with_parent)
            import threading
            self.timer = threading.Timer(max_s, self._kill)
            self.timer.daemon = True
            self.timer.start()
            time.sleep(0.5)  # let the sampler start before the timed region
        except (OSError, FileNotFoundError):
            self.p = None

    def _kill(self):
        if self.p is not None and self.p.poll() is None:
            self.p.kill()

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        self.timer.cancel()
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            self.p.wait(5)
        self.f.close()
        self.p = None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ measurements

def _time_conv_kernels(pp, torch, g, bb, w, prec, batch, reps=20, tile=-1):
    """Average duration of each conv layer's kernel: `reps` launches through pp_conv3x3 are
    captured into a CUDA graph (tensor maps encoded once, at capture), and one replay of that
    graph is timed with CUDA events on the replay stream, so host launch cost is not counted."""
    dt = torch.bfloat16 if prec == pp.PP_BF16 else torch.float32
    H, W = g.ny, g.nx
    x = torch.rand((batch, H + 2, W + 2, 64), device="cuda").to(dt)
    x[:, 0] = 0; x[:, -1] = 0; x[:, :, 0] = 0; x[:, :, -1] = 0
    planes = ()
    if prec == pp.PP_F32_TC:  # 3xTF32 operands are split FP32 (value and remainder planes)
        x, planes = pp.split_f32(x), (2,)
    per_layer = []
    stream = torch.cuda.current_stream()
    for (ci, co, s), wt, bn in zip(bb.layers(64), w[2], w[3]):
        wp = pp.pack_conv_weights(torch.from_numpy(wt).cuda(), prec)
        ss = torch.from_numpy(pp.bn_fold(bn)).cuda()
        Ho, Wo = (H - 1) // s + 1, (W - 1) // s + 1
        out = torch.zeros(planes + (batch, Ho + 2, Wo + 2, co), dtype=dt, device="cuda")
        # stream-K workspace made once, outside the captured launches (a release unit owns one)
        ws = pp.conv_workspace(batch, H, W, ci, co, s, prec) if prec == pp.PP_F32_TC else None
        pp.conv3x3(x, wp, ss, co, s, dtype=prec, out=out, tile=tile, workspace=ws)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                pp.conv3x3(x, wp, ss, co, s, dtype=prec, out=out, tile=tile, workspace=ws)
        graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        flops = 2.0 * batch * Ho * Wo * co * 9 * ci
        per_layer.append((e0.elapsed_time(e1) / reps * 1e-3, flops))
        x, H, W = out, Ho, Wo
    return per_layer


def _time_neck_head(pp, torch, g, bb, prec, batch, reps=20):
    """Average duration of each neck launch (one transposed conv per block into the concatenated
    map) and of the 1x1 head, timed as the convs are (graph of `reps` launches, one replay under
    CUDA events), with its algorithmic FLOPs and HBM bytes: the input map read once, the output
    written once, the weights read once (elt bytes per element: 8 for split FP32, value and
    remainder; 2 for BF16).  The head counts its real outputs (72), not its padding to 128."""
    from pp_synth import NECK_CHANNELS, head_weights
    up_w, up_bn, hw, hb = head_weights(bb)
    dt = torch.bfloat16 if prec == pp.PP_BF16 else torch.float32
    planes = (2,) if prec == pp.PP_F32_TC else ()
    elt = 8 if prec == pp.PP_F32_TC else 2
    sizes, H, W = [], g.ny, g.nx
    for (ci, co, s) in bb.layers(64):
        H, W = (H - 1) // s + 1, (W - 1) // s + 1
        sizes.append((H, W, co))
    blocks = [sizes[e] for e in _block_ends(bb)]
    H0, W0 = blocks[0][:2]
    neck_c = NECK_CHANNELS * len(blocks)
    neck = torch.zeros(planes + (batch, H0 + 2, W0 + 2, neck_c), dtype=dt, device="cuda")
    launches = []
    for k, ((Hb, Wb, C), wt, bn) in enumerate(zip(blocks, up_w, up_bn)):
        x = torch.rand((batch, Hb + 2, Wb + 2, C), device="cuda").to(dt)
        if planes:
            x = pp.split_f32(x)
        up = H0 // Hb
        wp = pp.pack_upsample_weights(wt, up, prec)
        ss = torch.from_numpy(pp.bn_fold(bn)).cuda()
        fn = (lambda x=x, wp=wp, ss=ss, up=up, k=k:
              pp.upsample(x, wp, ss, NECK_CHANNELS, up, prec, neck, out_coff=k * NECK_CHANNELS))
        byt = elt * (batch * Hb * Wb * C + batch * H0 * W0 * NECK_CHANNELS + C * up * up * NECK_CHANNELS)
        launches.append(("upsample x%d" % up, fn, 2.0 * batch * Hb * Wb * C * up * up * NECK_CHANNELS, byt))
    hwp, hss = pp.pack_head_weights(hw, hb, prec)
    hout = torch.zeros(planes + (batch, H0 + 2, W0 + 2, 128), dtype=dt, device="cuda")
    nout = hw.shape[0]
    launches.append(("head", lambda: pp.head(neck, hwp, hss, nout, prec, out=hout),
                     2.0 * batch * H0 * W0 * neck_c * nout,
                     elt * (batch * H0 * W0 * (neck_c + nout) + neck_c * nout)))
    stream = torch.cuda.current_stream()
    out = []
    for name, fn, flops, byt in launches:
        fn()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                fn()
        graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append((name, e0.elapsed_time(e1) / reps * 1e-3, flops, byt))
    return out


def _measure_tf32_tflops(torch, n=8192, reps=10):
    """Dense TF32 tensor-core rate on this GPU: torch.matmul (cuBLAS) of two n x n float32
    matrices with TF32 allowed, 2 n^3 FLOP, best of `reps` CUDA-event-timed calls."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.rand((n, n), device="cuda")
        b = torch.rand((n, n), device="cuda")
        c = torch.matmul(a, b)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        del a, b, c
        return 2.0 * n ** 3 / best / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def _profile_conv(a):
    """--profile-conv: one backbone layer of the workload, launched REPS times with one tile
    (split FP32 operands for the FP32 workloads, BF16 otherwise), on random input."""
    import torch
    import paper_2509_12207_gb300 as pp
    g, bb, prec, batch, _cap, _frames, w = _workload(a.workload)
    parts = a.profile_conv.split(":")
    layer, tile = int(parts[0]), int(parts[1])
    reps = int(parts[2]) if len(parts) > 2 else 3
    dt = pp.PP_BF16 if prec == pp.PP_BF16 else pp.PP_F32_TC
    H, W = g.ny, g.nx
    layers = bb.layers(64)
    for ci, co, st in layers[:layer]:
        H, W = (H - 1) // st + 1, (W - 1) // st + 1
    ci, co, st = layers[layer]
    x = torch.rand((batch, H + 2, W + 2, ci), device="cuda")
    x[:, 0] = 0; x[:, -1] = 0; x[:, :, 0] = 0; x[:, :, -1] = 0
    x = pp.split_f32(x) if dt == pp.PP_F32_TC else x.to(torch.bfloat16)
    wp = pp.pack_conv_weights(torch.from_numpy(w[2][layer]).cuda(), dt)
    ss = torch.from_numpy(pp.bn_fold(w[3][layer])).cuda()
    for _ in range(reps):
        out = pp.conv3x3(x, wp, ss, co, st, dtype=dt, tile=tile)
    torch.cuda.synchronize()
    print(json.dumps({"profile_conv": {"workload": a.workload, "layer": layer, "cin": ci, "cout": co, "stride": st,
                                       "H": H, "W": W, "batch": batch, "tile": tile,
                                       "tile_info": pp.conv_tile_info(dt, tile), "reps": reps,
                                       "out_shape": list(out.shape)}}))


def _profile_frontend(a):
    """--profile-frontend: pp_voxelize_pointnet on one step's frames, REPS times."""
    import torch
    import paper_2509_12207_gb300 as pp
    g, bb, prec, batch, cap, frames, w = _workload(a.workload)
    fs = [torch.from_numpy(frames[j % len(frames)]).cuda() for j in range(batch)]
    cap = max(int(f.shape[0]) for f in fs)
    pts = torch.zeros((batch, cap, 4), dtype=torch.float32, device="cuda")
    for j, f in enumerate(fs):
        pts[j, :f.shape[0]] = f
    n = torch.tensor([int(f.shape[0]) for f in fs], dtype=torch.int32, device="cuda")
    pfn_w = torch.from_numpy(w[0]).cuda()
    pfn_ss = torch.from_numpy(pp.bn_fold(w[1])).cuda()
    for _ in range(int(a.profile_frontend)):
        v = pp.voxelize_pointnet(pts, n, g, pfn_w, pfn_ss)
    torch.cuda.synchronize()
    print(json.dumps({"profile_frontend": {"workload": a.workload, "frames": batch, "points": [int(f.shape[0]) for f in fs],
                                           "num_pillars": [int(x) for x in v["num_pillars"].cpu()]}}))


def _block_ends(bb):
    ends, n = [], 0
    for c in bb.convs:
        n += c
        ends.append(n - 1)
    return ends


def _time_stages(pp, torch, g, frames_dev, w, prec, batch, reps=20):
    """Device time of the voxelise / PointNet / scatter stages for one step's batch of frames,
    each stage captured in a CUDA graph (so that only the device work is timed) and replayed.
    The scatter the release unit runs is incremental (pp_scatter_update on a canvas that keeps
    the previous frame): it is timed alternating between this step's frames and the next
    step's, so every update zeroes the other set's stale cells; the dense pp_scatter is timed
    beside it."""
    def batch_of(shift):
        fs = [frames_dev[(j + shift) % len(frames_dev)] for j in range(batch)]
        cap = max(int(f.shape[0]) for f in fs)
        pts = torch.zeros((batch, cap, 4), dtype=torch.float32, device="cuda")
        for j, f in enumerate(fs):
            pts[j, :f.shape[0]] = f
        return fs, pts, torch.tensor([int(f.shape[0]) for f in fs], dtype=torch.int32, device="cuda")

    (fs, pts, n), (_, pts2, n2) = batch_of(0), batch_of(1)
    pfn_w = torch.from_numpy(w[0]).cuda()
    pfn_ss = torch.from_numpy(pp.bn_fold(w[1])).cuda()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        v = pp.voxelize(pts, n, g)
        feat = pp.pointnet(v["pts"], v["npts"], v["coord"], v["num_pillars"], pfn_w, pfn_ss, g)
        v2 = pp.voxelize(pts2, n2, g)
        feat2 = pp.pointnet(v2["pts"], v2["npts"], v2["coord"], v2["num_pillars"], pfn_w, pfn_ss, g)
        canvas = pp.scatter(feat, v["pillar_of_cell"], g, dtype=prec)
        state = pp.ScatterState(g, batch, prec)
        pp.scatter_update(state, feat, v["coord"], v["num_pillars"], v["pillar_of_cell"])
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()

    def update_pair():
        pp.scatter_update(state, feat2, v2["coord"], v2["num_pillars"], v2["pillar_of_cell"])
        pp.scatter_update(state, feat, v["coord"], v["num_pillars"], v["pillar_of_cell"])

    out = {}
    for name, fn, per in (("voxelize_pointnet", lambda: pp.voxelize_pointnet(pts, n, g, pfn_w, pfn_ss), 1),
                          ("voxelize", lambda: pp.voxelize(pts, n, g), 1),
                          ("pointnet", lambda: pp.pointnet(v["pts"], v["npts"], v["coord"], v["num_pillars"],
                                                           pfn_w, pfn_ss, g), 1),
                          ("scatter", update_pair, 2),
                          ("scatter_dense", lambda: pp.scatter(feat, v["pillar_of_cell"], g, dtype=prec), 1)):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            keep = fn()  # noqa: F841  (outputs live in the graph's pool)
        graph.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / reps / per
        del graph
    canvas_bytes = canvas.numel() * canvas.element_size()
    out["_npoints"] = [int(f.shape[0]) for f in fs]
    out["_npillars"] = [int(x) for x in v["num_pillars"].cpu()]
    out["_gathered"] = [int(v["npts"][j, :int(v["num_pillars"][j])].sum()) for j in range(batch)]
    # algorithmic bytes of one incremental update, averaged over the two directions
    elt = {pp.PP_BF16: 2, pp.PP_F32: 4, pp.PP_F32_TC: 8}[prec]
    cells = [[set(x["coord"][j, :int(x["num_pillars"][j])].cpu().tolist()) for j in range(batch)] for x in (v, v2)]
    upd = 0
    for new, old in ((1, 0), (0, 1)):
        for j in range(batch):
            upd += len(cells[new][j]) * (256 + 8 + 64 * elt) + len(cells[old][j] - cells[new][j]) * (8 + 64 * elt)
    out["_scatter_bytes"] = upd / 2
    return out, canvas_bytes, int(v["num_pillars"][0])


def _run_ours(a, rank, world, dist):
    import numpy as np
    import torch
    import paper_2509_12207_gb300 as pp

    dev = rank % max(1, torch.cuda.device_count())
    torch.cuda.set_device(dev)
    g, bb, prec, batch, cap, frames, w = _workload(a.workload)
    # throughput run: no deadline pressure (early exit off, 10 s deadline), so a slow run (a
    # profiler) still completes every frame
    tuned = bool(a.tune_table) and os.path.exists(a.tune_table) and pp.conv_tune_load(a.tune_table) > 0
    head = None
    if a.head:
        from pp_synth import head_weights
        head = head_weights(bb)
    cfg, keep = pp.make_config(g, bb, w, head=head, max_batch=batch, cap_points=cap, precisions=1 << prec,
                               units=max(2, a.depth), max_admitted=2 * a.depth * batch,
                               th_urgent=-1.0, early_exit=0, fp32_cuda_cores=1 if a.fp32_cuda_cores else 0,
                               autotune=0 if tuned else 1, stream_k=1 if a.stream_k else 0)
    ctx = pp.Context(cfg)
    if a.tune_table and not tuned:
        pp.conv_tune_save(a.tune_table)
    for ch in range(max(1, a.chains)):
        ctx.register_chain(ch, 10000.0, 10000.0, prec)
    frames_dev = [torch.from_numpy(f).cuda() for f in frames]
    frames_host = [torch.from_numpy(f).pin_memory() for f in frames]
    n_frames = batch

    res_bytes = ctx.result_bytes(prec)
    free_sinks = [torch.empty(res_bytes, dtype=torch.uint8).pin_memory() for _ in range(a.depth * n_frames)]
    sink_of = {}

    def submit(k, host):
        fs = [(frames_host if host else frames_dev)[(k * n_frames + j) % len(frames)] for j in range(n_frames)]
        # the step's frames arrive together (one submission), so they share one release unit
        # host inputs are pinned tensors: borrowed, read in place by the kernels over the host
        # link (PP_POINTS_PINNED), so the step's host->device traffic is the points themselves;
        # host outputs: each frame's result lands in a pinned host buffer, written by the unit's
        # own result copy over the host link (pp_submit_frames_ex)
        sinks = [free_sinks.pop() for _ in range(n_frames)] if host else None
        rc, ids = ctx.submit_many([k % max(1, a.chains)] * n_frames, fs, host_out=sinks)
        assert rc == pp.PP_OK and len(ids) == n_frames, rc
        if host:
            sink_of.update(zip(ids, sinks))

    def run_steps(steps, host):
        """Runs `steps` steps with up to `depth` of them in flight (continuous batching: a step
        is submitted as soon as an earlier one's results have been read and released)."""
        k = done = inflight = 0
        while done < steps * n_frames:
            while k < steps and inflight < a.depth * n_frames:
                submit(k, host)
                k += 1
                inflight += n_frames
            got = ctx.poll(64, timeout_us=1000000)
            for r in got:
                assert r.status == pp.PP_FRAME_DONE
                if host:
                    # the frame's outputs are already in its pinned host buffer (complete at poll)
                    assert r.out_host
                    run_steps.d2h += res_bytes
                    free_sinks.append(sink_of.pop(r.frame_id))
            ctx.release_many([r.frame_id for r in got])
            inflight -= len(got)
            done += len(got)
    run_steps.d2h = 0

    def timed(host):
        run_steps(a.warmup, host)
        timed.units_before = ctx.stats()["units_launched"]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t0 = time.perf_counter()
        run_steps.d2h = 0
        run_steps(a.steps, host)
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        el = replica_window(dist, e0.elapsed_time(e1) * 1e-3, "cuda")
        return el, wall

    clocks = _Clocks(dev, enabled=not a.no_clocks, out_dir=a.clocks_dir)
    try:
        el, wall = timed(host=False)
    finally:
        clk = clocks.stop()
    st = ctx.stats()
    # units launched inside the timed region (the warm-up steps ran before it)
    timed_units = st["units_launched"] - timed.units_before
    e2e_el, _ = timed(host=True)
    h2d = sum(int(frames[(k * n_frames + j) % len(frames)].nbytes) for k in range(a.steps)
              for j in range(n_frames)) // a.steps
    d2h = run_steps.d2h // a.steps
    ctx.destroy()

    # kernel roofline: the conv kernels dominate the step
    conv_dtype = prec if (prec == pp.PP_BF16 or a.fp32_cuda_cores) else pp.PP_F32_TC
    layers = _time_conv_kernels(pp, torch, g, bb, w, conv_dtype, batch)
    conv_s = sum(t for t, _ in layers)
    conv_flops = sum(f for _, f in layers)
    # the scatter writes the canvas the convs read (split FP32 for the 3xTF32 convs)
    stages, canvas_bytes, num_p = _time_stages(pp, torch, g, frames_dev, w,
                                               pp.PP_F32_TC if conv_dtype == pp.PP_F32_TC else prec, n_frames)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    src = "of measured" if peaks else "of fallback"
    if prec == pp.PP_F32 and a.fp32_cuda_cores:
        sm_max = (clk.get("sm_max_mhz") or 2070.0)
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12       # FP32 FMA lanes x 2 flops x clock
        bound, peak_note = "alu", "FP32 FMA: 152 SMs x 128 lanes x 2 x %.0f MHz (derived)" % sm_max
    elif prec == pp.PP_F32:
        # 3xTF32: every FP32 FLOP costs three TF32 tensor FLOPs; the TF32 rate is measured here
        # (a library GEMM), the nominal TF32/BF16 ratio applied to the measured BF16 peak is
        # reported beside it
        tf32 = _measure_tf32_tflops(torch)
        peak = tf32 / 3.0
        bound, peak_note = "tensor", ("FP32-equivalent via 3 TF32 passes: cuBLAS TF32 GEMM 8192^3 measured in this "
                                      "run (%.1f TFLOP/s, best of 10) / 3" % tf32)
        peak_nominal = bf16 * (1.1 / 2.25) / 3.0
    else:
        peak = bf16
        bound, peak_note = "tensor", "bf16 dense, %s" % src
    achieved = conv_flops / conv_s / 1e12
    if prec != pp.PP_F32 or a.fp32_cuda_cores:
        peak_nominal = None
    traffic = _conv_traffic(a.workload) if conv_dtype != pp.PP_F32 else None
    neck_head = None
    if conv_dtype != pp.PP_F32:
        # pointwise GEMMs with K = 64..384: below the ridge point (FLOPs per HBM byte) of either
        # dtype, so bound by HBM; the tensor-side figures are given beside it
        nh = _time_neck_head(pp, torch, g, bb, conv_dtype, batch)
        nh_s = sum(x[1] for x in nh)
        nh_f, nh_b = sum(x[2] for x in nh), sum(x[3] for x in nh)
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        neck_head = {"bound": "hbm", "achieved": nh_b / nh_s / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": nh_b / nh_s / 1e9 / hbm, "peak_source": "HBM copy, %s" % src,
                     "traffic": _conv_traffic(a.workload, NECK_HEAD_TRAFFIC),
                     "ms_per_frame": nh_s * 1e3 / n_frames, "bytes_per_step": nh_b,
                     "tflops": nh_f / nh_s / 1e12, "tensor_frac": nh_f / nh_s / 1e12 / peak,
                     "launches": [{"kernel": k, "us": round(t * 1e6, 2), "tflops": round(f / t / 1e12, 1),
                                   "gbs": round(b / t / 1e9)} for k, t, f, b in nh],
                     "in_step": bool(a.head)}
    res = {
        "metric": "pillar frames/s", "value": replica_throughput(a.steps * n_frames, world, el), "unit": "frames/s",
        "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": el / a.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == pp.PP_F32 else "bf16", "data": "synthetic",
        "config": {"workload": WORKLOADS[a.workload] + (HEAD_NOTE if a.head else ""), "frames_per_step": n_frames, "steps_in_flight": a.depth,
                   "chains": max(1, a.chains), "conv_stream_k": a.stream_k and prec == pp.PP_F32
                   and not a.fp32_cuda_cores, "points_per_frame":
                   [int(f.shape[0]) for f in frames], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "per-frame working set (~%d MB canvas + activations) exceeds the 129 MB L2"
                         % (canvas_bytes // 2 ** 20)},
        "e2e": {"value": replica_throughput(a.steps * n_frames, world, e2e_el), "unit": "frames/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per step, all conv launches",
                     "kernel": "conv3x3 (%s), all layers"
                     % {pp.PP_F32: "CUDA-core FP32", pp.PP_F32_TC: "tcgen05 3xTF32", pp.PP_BF16: "tcgen05 BF16"}[conv_dtype],
                     "peak_source": peak_note,
                     "frac_of_nominal": None if peak_nominal is None else achieved / peak_nominal,
                     "peak_nominal": peak_nominal,
                     "peak_nominal_source": None if peak_nominal is None else
                     "bf16 dense %s x 1.1/2.25 (nominal TF32/BF16) / 3" % src,
                     "conv_ms_per_frame": conv_s * 1e3 / n_frames,
                     "timing": "each layer alone on the GPU: a CUDA graph of 20 launches replayed once under CUDA "
                               "events on its stream, after the timed region",
                     # the same FLOPs over the step's device time, which also holds the front end: in
                     # the timed steps the units of several chains overlap on the GPU, so this can
                     # exceed the per-layer figure above
                     "in_step": {"tflops": conv_flops / (el / a.steps) / 1e12,
                                 "frac": conv_flops / (el / a.steps) / 1e12 / peak},
                     "layers_us": [round(t * 1e6, 2) for t, _ in layers],
                     "layers_tflops": [round(f / t / 1e12, 1) for t, f in layers]},
        "stage_ms_per_step": {k: v for k, v in stages.items() if not k.startswith("_")},
        "neck_head": neck_head,
        "front_end_roofline": _front_end_roofline(g, stages, {pp.PP_BF16: 2, pp.PP_F32: 4, pp.PP_F32_TC: 8}[
            pp.PP_F32_TC if conv_dtype == pp.PP_F32_TC else prec], peaks),
        "runtime": {"lat_p50_us": st["lat_p50_us"], "lat_p99_us": st["lat_p99_us"],
                    "sched_us_per_decision": st["sched_us_per_decision"], "units": timed_units,
                    "frames_per_unit": a.steps * n_frames / max(1, timed_units)},
        # per unit: 4 voxelisation kernels (count, tile sums, scan, bucket + stale canvas cells),
        # point selection + PointNet + canvas write, one per conv layer, (one per block and the
        # head,) result copy
        "gpu_launches": timed_units * (4 + 1 + len(bb.layers(64)) + (len(bb.convs) + 1 if a.head else 0) + 1),
        "clocks": clk,
        "num_pillars": num_p,
        "wall_s": wall,
    }
    return res


# ------------------------------------------------------------------ replicas (one process per GPU)

def replica_window(dist, seconds, device="cpu"):
    """The timed window of a multi-GPU run: the slowest rank's (all-reduce MAX over the process
    group; the value itself without one).  Every rank processes its own frames, so the job's
    throughput is the frames of all ranks over this window."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(frames_per_rank, world, window_s):
    """Whole-job frames/s of `world` replicas that each processed frames_per_rank frames."""
    return frames_per_rank * world / window_s


# ------------------------------------------------------------------ serving (chains with deadlines)

def _serve(pp, torch, mode, n_chains, rate, duration_s, mixed, seed=1400, clouds=None, dfac=1.0, noise=0.0,
           synth=None, tight=0.0, warmup_s=1.0):
    """Replays periodic chains in real time against one context and returns its statistics.

    mode "urgency": the paper's release rules (urgency order, early exit, stream binding,
    delayed launch, overlapped batched sync) with continuous batching of up to 8 frames per
    graph launch; chains BF16 (``mixed``: odd chains BF16, even FP32).  mode "plain": every
    frame launched on arrival, kernel by kernel, FP32, on its chain's default-priority stream.
    modes "edf" / "sjf" / "hrrn" / "lcuf" / "saedf" / "eqdf": the urgency mode's units and sync, released in that
    comparison order (no early exit, reservation or delaying).
    Periods 50/100/200 ms round robin, deadline = period, jitter +-5 ms, 30k-150k points per
    frame (config-1 geometry); arrivals scaled by ``rate``, deadlines by ``dfac`` (the paper's
    f_a and f_d), and a seeded share ``tight`` of the chains with halved deadlines (the paper's
    f_tight; pp_synth.tight_chains); ``noise``: every frame's estimate, as the policy sees it, scaled by a factor
    drawn from 1 + U[-noise, noise) (the paper's estimation-error study).  ``synth`` = (util,
    kernel_us, total_us): every odd chain becomes a synthetic-load chain whose frames run
    round(total_us / kernel_us) kernels of about kernel_us on round(util x SMs) SMs (the paper's
    kernel-utilisation and kernel-time studies).  A frame the budget cannot admit counts as a
    miss.  The statistics exclude a warm-up replay of ``warmup_s`` seconds at the same load
    (another seed), run to completion on the same context first."""
    from pp_synth import BACKBONE_SMALL, GEOM_SMALL, arrival_times, pillar_weights, serving_chains
    g, bb = GEOM_SMALL, BACKBONE_SMALL
    w = pillar_weights(bb, 7)
    chains = serving_chains(n_chains, mixed=mixed, tight=tight)
    others = {"edf": pp.PP_POLICY_EDF, "sjf": pp.PP_POLICY_SJF, "hrrn": pp.PP_POLICY_HRRN,
              "lcuf": pp.PP_POLICY_LCUF, "saedf": pp.PP_POLICY_SAEDF, "eqdf": pp.PP_POLICY_EQDF}
    if mode == "urgency":
        knobs = dict(policy=pp.PP_POLICY_URGENCY, max_batch=8, use_graphs=1, max_closed=2,
                     delta_eval_us=500.0, th_urgent=0.0, th_calib_frames=64, early_exit=1, units=8)
        prec = [c.precision for c in chains]
    elif mode in others:
        # the same batched, graph-launched units and batched sync, released in the comparison
        # policy's order instead of by urgency (no early exit, reservation or delaying)
        knobs = dict(policy=others[mode], max_batch=8, use_graphs=1, max_closed=2,
                     delta_eval_us=500.0, th_urgent=-1.0, early_exit=0, units=8)
        prec = [c.precision for c in chains]
    else:
        knobs = dict(policy=pp.PP_POLICY_FIFO, max_batch=1, use_graphs=0, max_closed=0, early_exit=0,
                     th_urgent=-1.0, units=16)
        prec = [pp.PP_F32] * n_chains
    need = (1 if pp.PP_F32 in prec else 0) | (2 if pp.PP_BF16 in prec else 0)
    cfg, keep = pp.make_config(g, bb, w, cap_points=150000, precisions=need, est_noise=noise,
                               noise_seed=seed, **knobs)
    ctx = pp.Context(cfg)
    try:
        synthetic = set()
        for c, p in zip(chains, prec):
            if synth is not None and c.chain_id % 2 == 1:
                util, kus, tot = synth
                ctx.register_synthetic_chain(c.chain_id, c.period_ms, c.deadline_ms * dfac,
                                             max(1, int(round(tot / kus))), kus, util)
                synthetic.add(c.chain_id)
            else:
                ctx.register_chain(c.chain_id, c.period_ms, c.deadline_ms * dfac, p)
        if warmup_s > 0:
            wev = arrival_times(chains, warmup_s * 1000.0, rate=rate, jitter_ms=5.0, seed=seed + 7)
            ctx.replay([(20000.0 + t_ms * 1000.0, cid, i % len(clouds), 0 if cid in synthetic else n)
                        for i, (t_ms, cid, n) in enumerate(wev)], clouds, timeout_us=30e6)
            ctx.stats_reset()
        ev = arrival_times(chains, duration_s * 1000.0, rate=rate, jitter_ms=5.0, seed=seed)
        ev = [(t, cid, 0 if cid in synthetic else n) for t, cid, n in ev]
        # real-time replay from the library's own load generator (pp_replay): submissions at
        # their scheduled times, results polled and released as they complete
        arrivals = [(20000.0 + t_ms * 1000.0, cid, i % len(clouds), n) for i, (t_ms, cid, n) in enumerate(ev)]
        rep = ctx.replay(arrivals, clouds, timeout_us=30e6)
        rejected = {c: r for c, r in enumerate(rep["chain_rejected"]) if r}
        st = ctx.stats()
    finally:
        ctx.destroy()
    per = {}
    for c in chains:
        n = st["chain_frames"][c.chain_id] + rejected.get(c.chain_id, 0)
        m = st["chain_missed"][c.chain_id] + rejected.get(c.chain_id, 0)
        if n:
            per[c.chain_id] = (m, n)
    miss = sum(m / n for m, n in per.values()) / max(1, len(per))
    return {"mode": mode, "chains": n_chains, "rate": rate, "deadline_factor": dfac, "mixed": mixed,
            "tight": tight, "tight_chains": [c.chain_id for c in chains if c.deadline_ms < c.period_ms],
            "seconds": duration_s, "warmup_s": warmup_s,
            "est_noise": noise, "synthetic": None if synth is None else
            {"util": synth[0], "kernel_us": synth[1], "frame_us": synth[2], "chains": "odd"},
            "frames": len(ev),
            "done": st["done"], "dropped": st["dropped"], "rejected": sum(rejected.values()),
            "miss_ratio": miss, "lat_p50_ms": st["lat_p50_us"] / 1e3, "lat_p99_ms": st["lat_p99_us"] / 1e3,
            "frames_per_s": st["done"] / duration_s, "mean_batch": st["mean_batch"],
            "delayed": st["delayed_releases"], "collisions": st["collisions"],
            "th_urgent_per_ms": st["th_urgent"] * 1e3 if st["th_urgent"] > 0 else None,
            "sched_us_per_decision": st["sched_us_per_decision"],
            "submit_late_us": {"mean": rep["submit_late_us_mean"], "max": rep["submit_late_us_max"]}}


def parse_sweep_item(item):
    """One --serve-sweep point: ``chains:rate:seconds`` then, in this order and each optional,
    ``mixed`` (any other word: all BF16), the deadline factor f_d, the estimate noise and
    ``util/kernel_us/frame_us`` (odd chains synthetic); ``key=value`` items (dfac, noise, tight,
    synth) may stand anywhere after the first three and override the positional ones.  tight is
    the share of chains with halved deadlines (f_tight; default 0)."""
    parts = item.split(":")
    if len(parts) < 3:
        raise ValueError("sweep point %r: need chains:rate:seconds" % item)
    pt = {"chains": int(parts[0]), "rate": float(parts[1]), "seconds": float(parts[2]), "mixed": False,
          "dfac": 1.0, "noise": 0.0, "synth": None, "tight": 0.0}
    pos = []
    for tok in parts[3:]:
        if "=" in tok:
            k, v = tok.split("=", 1)
            if k not in ("dfac", "noise", "tight", "synth"):
                raise ValueError("sweep point %r: unknown key %s" % (item, k))
            pt[k] = tuple(float(x) for x in v.split("/")) if k == "synth" else float(v)
        else:
            pos.append(tok)
    if pos:
        pt["mixed"] = pos[0] == "mixed"
    if len(pos) > 1 and "dfac=" not in item:
        pt["dfac"] = float(pos[1])
    if len(pos) > 2 and "noise=" not in item:
        pt["noise"] = float(pos[2])
    if len(pos) > 3 and "synth=" not in item:
        pt["synth"] = tuple(float(x) for x in pos[3].split("/"))
    if not 0.0 <= pt["tight"] <= 1.0:
        raise ValueError("sweep point %r: tight must be in [0, 1]" % item)
    return pt


# Serving points of the default run: (key, chains, rate x, seconds, mixed, f_d, f_tight).  The
# 11-chain point is the base load at the paper's rates; the 33-chain points take the paper's
# default share of tight-deadline chains (40 %): loose deadlines at 96x (~37k frames/s offered,
# past the plain per-frame path's saturation near 28k frames/s on this GPU) and deadlines of
# 0.5 % of the period at 64x (~25k frames/s, where the deadlines rather than the load decide).
SERVING_POINTS = [
    ("config4_11_chains_1x", 11, 1.0, 4.0, False, 1.0, 0.0),
    ("overload_33_chains_96x_fd1_tight0.4", 33, 96.0, 8.0, True, 1.0, 0.4),
    ("tight_33_chains_64x_fd0.005_tight0.4", 33, 64.0, 8.0, True, 0.005, 0.4),
]


def _serving_clouds(torch):
    from pp_synth import GEOM_SMALL, uniform_cloud
    return [torch.from_numpy(uniform_cloud(150000, 7000 + k, GEOM_SMALL)).cuda() for k in range(16)]


def _run_reference(a):
    g, bb, prec, batch, cap, frames, w = _workload(a.workload)
    from oracle import pillars as O
    head = None
    if a.head:
        from pp_synth import head_weights
        head = head_weights(bb)

    def one(pts):
        r = O.frame(pts, g, bb, w)
        if head is not None:
            O.head(O.neck(r["blocks"], head[0], head[1]), head[2], head[3])

    # the oracle takes seconds per frame: at most one warm-up frame, and the timed steps stop
    # once REFERENCE_BUDGET_S is spent (at least one step), so any --steps ends within minutes
    warm = min(a.warmup, 1)
    for k in range(warm):
        one(frames[k % len(frames)])
    t0 = time.perf_counter()
    steps = 0
    while steps < a.steps and (steps == 0 or time.perf_counter() - t0 < REFERENCE_BUDGET_S):
        for j in range(batch):
            one(frames[(steps * batch + j) % len(frames)])
        steps += 1
    secs = time.perf_counter() - t0
    v = steps * batch / secs
    cores = os.cpu_count()
    return {"impl": "reference", "metric": "pillar frames/s", "value": v, "unit": "frames/s", "n_gpus": 1,
            "steps": steps, "steps_requested": a.steps, "warmup": warm, "ms_per_step": secs / steps * 1e3,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[a.workload] + (HEAD_NOTE if a.head else ""), "frames_per_step": batch},
            "cpu_baseline": {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": "%d step(s) of %d full frame(s) through the FP64 NumPy oracle in %.1f s "
                                       "(timed steps stop after %d s; BLAS threads as installed, up to %d cores)"
                                       % (steps, batch, secs, REFERENCE_BUDGET_S, cores)},
            "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = _args()
    if a.cpu_worker:
        name, min_s, head = a.cpu_worker.split(":")
        print("%d %.6f" % _oracle_seconds(name, float(min_s), head == "1"))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.profile_conv:
        _profile_conv(a)
        return
    if a.profile_frontend:
        _profile_frontend(a)
        return
    if a.impl == "reference":
        if rank == 0:
            print(json.dumps(_run_reference(a)))
        return
    if a.serve_sweep:
        import torch
        import paper_2509_12207_gb300 as pp
        torch.cuda.set_device(0)
        clouds = _serving_clouds(torch)
        out = []
        for item in a.serve_sweep.split(","):
            pt = parse_sweep_item(item)
            for mode in a.serve_modes.split(","):
                out.append(_serve(pp, torch, mode, pt["chains"], pt["rate"], pt["seconds"], pt["mixed"],
                                  clouds=clouds, dfac=pt["dfac"], noise=pt["noise"], synth=pt["synth"],
                                  tight=pt["tight"]))
                print(json.dumps(out[-1]), file=sys.stderr, flush=True)
        print(json.dumps({"metric": "deadline-miss ratio and p99 chain latency, urgency-served batched "
                          "vs plain per-frame launches", "serving": out}))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    res = _run_ours(a, rank, world, dist)
    if a.workload == "cfg2-fp32" and not a.no_batched and not a.head and not a.fp32_cuda_cores:
        # the batched BF16 workload (8 frames of 30k-150k points per unit, BF16 backbone on the
        # tensor cores) as its own timed run, reported beside the full-size FP32 frame
        import copy
        b = copy.copy(a)
        b.workload, b.tune_table = "cfg3-bf16", None
        b.chains, b.depth = SERVING_SHAPE["cfg3-bf16"]
        sub = _run_ours(b, rank, world, dist)
        res["batched_bf16"] = {k: sub[k] for k in (
            "metric", "value", "unit", "ms_per_step", "dtype", "config", "e2e", "roofline", "front_end_roofline",
            "neck_head", "stage_ms_per_step", "runtime", "gpu_launches", "clocks", "num_pillars", "wall_s")}
    if rank == 0 and not a.no_serving:
        import torch
        import paper_2509_12207_gb300 as pp
        clouds = _serving_clouds(torch)
        res["serving"] = {key: [_serve(pp, torch, m, n, rate, secs, mixed, clouds=clouds, dfac=dfac, tight=tight)
                                for m in ("urgency", "plain")]
                          for key, n, rate, secs, mixed, dfac, tight in SERVING_POINTS}
    if rank == 0:
        if not a.no_cpu_baseline:
            res["cpu_baseline"] = _cpu_baseline(a.workload, a.head)
        print(json.dumps(res))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

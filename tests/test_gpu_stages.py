"""Parity of each stage entry point (through the C ABI) with the FP64 oracle.

Integer outputs (cells, counts, pillar ids, coords, npts, gathered points, canvas positions)
must match bit for bit; FP32 features and conv outputs within 1e-4 of the oracle (rel_err);
the BF16 conv within 2e-2 of the oracle with unrounded weights, and within 8e-3 of the oracle
fed the same bf16-rounded operands (only FP32 accumulation order and the output rounding
differ there)."""
import dataclasses

import numpy as np
import pytest

from oracle import pillars as O
from pp_synth import (GEOM_FULL, GEOM_SMALL, Geometry, clustered_cloud, config_points,
                      pillar_weights, uniform_cloud, BACKBONE_SMALL)
from tests._util import tf32_remainder, BF16_TOL, FP32_TOL, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
import paper_2509_12207_gb300 as pp  # noqa: E402

DEV = "cuda:0"
TINY = Geometry(0.0, 1.28, -0.32, 0.64, -1.0, 1.0, 0.32, 0.32, 4, 3, 5)


def _batch(clouds, cap=None):
    cap = cap or max(1, max(len(c) for c in clouds))
    pts = np.zeros((len(clouds), cap, 4), np.float32)
    for i, c in enumerate(clouds):
        pts[i, : len(c)] = c
    n = np.array([len(c) for c in clouds], np.int32)
    return torch.from_numpy(pts).to(DEV), torch.from_numpy(n).to(DEV)


def _check_vox(g, clouds, v, b):
    ref = O.voxelise(clouds[b], g)
    n = len(clouds[b])
    num = int(v["num_pillars"][b])
    assert num == ref["num_pillars"]
    np.testing.assert_array_equal(v["cell"][b, :n].cpu().numpy(), ref["cell"])
    np.testing.assert_array_equal(v["cnt"][b].cpu().numpy(), ref["cnt"])
    np.testing.assert_array_equal(v["pillar_of_cell"][b].cpu().numpy(), ref["pillar_of_cell"])
    np.testing.assert_array_equal(v["coord"][b, :num].cpu().numpy(), ref["coord"])
    np.testing.assert_array_equal(v["npts"][b, :num].cpu().numpy(), ref["npts"])
    got = v["pts"][b, :num].cpu().numpy()
    assert got.tobytes() == ref["pts"].tobytes()  # bit-exact, including zero padding
    return ref


def _edge_cloud(g, n, seed):
    rng = np.random.default_rng(seed)
    pts = uniform_cloud(n, seed, g)
    k = n // 3
    pts[:k, 0] = (rng.integers(0, g.nx + 1, k) * np.float32(g.vx) + np.float32(g.xmin)).astype(np.float32)
    pts[:k, 1] = (rng.integers(0, g.ny + 1, k) * np.float32(g.vy) + np.float32(g.ymin)).astype(np.float32)
    pts[k:k + 10, 2] = np.float32(g.zmax)
    pts[k + 10:k + 20, 0] = np.nan
    pts[k + 20:k + 30, 1] = np.float32(g.ymax)
    pts[:200, 0] = np.float32(g.xmin) + np.float32(0.05)   # one crowded cell (> 32 points)
    pts[:200, 1] = np.float32(g.ymin) + np.float32(0.05)
    pts[:200, 2] = 0.0
    return pts[rng.permutation(n)]


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "edges", "tiny"])
def test_voxelize_single(name):
    if name == "cfg1":
        g, clouds = GEOM_SMALL, [config_points(1, 0)]
    elif name == "cfg2":
        g, clouds = GEOM_FULL, [config_points(2, 0)]
    elif name == "edges":
        g, clouds = GEOM_SMALL, [_edge_cloud(GEOM_SMALL, 30000, 3)]
    else:
        g, clouds = TINY, [_edge_cloud(TINY, 500, 4)]
    pts, n = _batch(clouds)
    v = pp.voxelize(pts, n, g)
    torch.cuda.synchronize()
    pp.voxelize_check(v)
    _check_vox(g, clouds, v, 0)


def test_voxelize_batched_uneven_and_degenerate():
    g = GEOM_SMALL
    clouds = [config_points(3, 0, 150000), np.zeros((0, 4), np.float32), config_points(3, 1, 31000),
              uniform_cloud(50, 9, g) + np.float32(500.0),  # every point dropped
              clustered_cloud(90000, 5, g)]
    pts, n = _batch(clouds, cap=150000)
    v = pp.voxelize(pts, n, g)
    torch.cuda.synchronize()
    for b in range(len(clouds)):
        ref = _check_vox(g, clouds, v, b)
        if b == 0:
            assert ref["num_pillars"] == g.max_pillars   # the cap binds at 150k points
    # determinism: a second run is bit-identical
    w = pp.voxelize(pts, n, g)
    torch.cuda.synchronize()
    assert torch.equal(v["pillar_of_cell"], w["pillar_of_cell"])
    assert torch.equal(v["num_pillars"], w["num_pillars"])
    for b in range(len(clouds)):
        num = int(v["num_pillars"][b])       # entries past num_pillars are unspecified
        for k in ("coord", "npts", "pts"):
            assert torch.equal(v[k][b, :num], w[k][b, :num])


def test_voxelize_bad_count_reported():
    g = GEOM_SMALL
    pts, n = _batch([uniform_cloud(100, 1, g)])
    n.fill_(1000)  # > cap: the frame is treated as empty and the error word is set
    v = pp.voxelize(pts, n, g)
    with pytest.raises(pp.PPError):
        pp.voxelize_check(v)
    assert int(v["num_pillars"][0]) == 0


def _pfn_params(seed=7):
    pfn_w, pfn_bn, _, _ = pillar_weights(BACKBONE_SMALL, seed)
    ss = pp.bn_fold(pfn_bn)
    return pfn_w, pfn_bn, torch.from_numpy(pfn_w).to(DEV), torch.from_numpy(ss).to(DEV)


@pytest.mark.parametrize("g,cfg", [(GEOM_SMALL, 1), (GEOM_FULL, 2)])
def test_pointnet_and_scatter(g, cfg):
    cloud = config_points(cfg, 1)
    pts, n = _batch([cloud])
    v = pp.voxelize(pts, n, g)
    pfn_w, pfn_bn, w_d, ss_d = _pfn_params()
    feat = pp.pointnet(v["pts"], v["npts"], v["coord"], v["num_pillars"], w_d, ss_d, g)
    torch.cuda.synchronize()
    ref = O.voxelise(cloud, g)
    num = ref["num_pillars"]
    rf = O.pointnet(ref["pts"], ref["npts"], ref["coord"], pfn_w, pfn_bn, g)
    assert rel_err(feat[0, :num].cpu().numpy(), rf) <= FP32_TOL
    # scatter positions are exact: feed the GPU features, compare with the oracle scatter of them
    f32 = feat[0, :num].cpu().numpy().astype(np.float64)
    canvas_ref = O.scatter(f32, ref["coord"], g)
    for dt in (pp.PP_F32, pp.PP_BF16):
        canvas = pp.scatter(feat, v["pillar_of_cell"], g, dtype=dt)
        torch.cuda.synchronize()
        c = canvas[0].float().cpu().numpy()
        assert not c[0].any() and not c[-1].any() and not c[:, 0].any() and not c[:, -1].any()
        want = torch.from_numpy(canvas_ref).to(torch.float32)
        if dt == pp.PP_BF16:
            want = want.to(torch.bfloat16).float()
        assert np.array_equal(c[1:-1, 1:-1], want.numpy())
    # split FP32 canvas (the 3xTF32 conv operand): plane 0 = the FP32 canvas, plane 1 = its
    # TF32 remainders, border zero in both
    f32c = pp.scatter(feat, v["pillar_of_cell"], g, dtype=pp.PP_F32)
    split = pp.scatter(feat, v["pillar_of_cell"], g, dtype=pp.PP_F32_TC)
    torch.cuda.synchronize()
    assert tuple(split.shape) == (2,) + tuple(f32c.shape)
    assert torch.equal(split[0], f32c)
    assert np.array_equal(split[1].cpu().numpy(), tf32_remainder(f32c.cpu().numpy()))


def test_tf32_split_exact():
    """pp_tf32_split against the bit-pattern definition, on values that exercise every case:
    signs, zeros, subnormals, powers of two, values whose low bits are all set, and a length
    that leaves a tail after the 4-wide main loop."""
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(1000).astype(np.float32) * 10,
                        np.array([0.0, -0.0, 1.0, -2.0, 1e-40, -3e-39, 2.0 ** -126, 3.4e38], np.float32),
                        (np.arange(1, 40, dtype=np.uint32) | np.uint32(0x3F801FFF)).view(np.float32)])
    for n in (v.size, v.size - 1, v.size - 2, 3, 1):
        x = torch.from_numpy(v[:n].copy()).to(DEV)
        lo = pp.tf32_split(x)
        torch.cuda.synchronize()
        want = tf32_remainder(v[:n])
        assert np.array_equal(lo.cpu().numpy().view(np.uint32), want.view(np.uint32)), n
        # plane 0 + plane 1 reproduces x exactly
        hi = (v[:n].view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
        assert np.array_equal(hi + lo.cpu().numpy(), v[:n])


def test_scatter_batched_bf16_rounding():
    g = GEOM_SMALL
    clouds = [config_points(3, 2, 40000), config_points(3, 3, 120000)]
    pts, n = _batch(clouds)
    v = pp.voxelize(pts, n, g)
    feat = torch.randn((2, g.max_pillars, 64), device=DEV) * 3
    canvas = pp.scatter(feat, v["pillar_of_cell"], g, dtype=pp.PP_BF16)
    torch.cuda.synchronize()
    for b in range(2):
        num = int(v["num_pillars"][b])
        coord = v["coord"][b, :num].long()
        inner = canvas[b, 1:-1, 1:-1].reshape(-1, 64)
        assert torch.equal(inner[coord], feat[b, :num].to(torch.bfloat16))
        mask = torch.ones(inner.shape[0], dtype=torch.bool, device=DEV)
        mask[coord] = False
        assert not inner[mask].any()


def test_voxelize_pointnet_fused_equals_stages():
    """The release unit's fused point selection + PointNet gives, bit for bit, pp_voxelize +
    pp_pointnet's outputs (crowded clustered pillars that need the sort's merge steps, a short
    frame, an empty row)."""
    g = GEOM_FULL
    w = pillar_weights(BACKBONE_SMALL, 7)
    pfn_w = torch.from_numpy(w[0]).to(DEV)
    ss = torch.from_numpy(pp.bn_fold(w[1])).to(DEV)
    clouds = [clustered_cloud(120000, 5), config_points(1, 0), np.zeros((0, 4), np.float32)]
    pts, n = _batch(clouds)
    v = pp.voxelize(pts, n, g)
    feat = pp.pointnet(v["pts"], v["npts"], v["coord"], v["num_pillars"], pfn_w, ss, g)
    f = pp.voxelize_pointnet(pts, n, g, pfn_w, ss)
    torch.cuda.synchronize()
    for k in ("pillar_of_cell", "num_pillars"):
        assert torch.equal(f[k], v[k]), k
    for b in range(3):
        assert torch.equal(f["cell"][b, :len(clouds[b])], v["cell"][b, :len(clouds[b])])   # rows past n unwritten
        num = int(v["num_pillars"][b])
        assert torch.equal(f["coord"][b, :num], v["coord"][b, :num])
        assert torch.equal(f["npts"][b, :num], v["npts"][b, :num])
        assert torch.equal(f["feat"][b, :num], feat[b, :num]), b
    assert int(v["npts"][0, :int(v["num_pillars"][0])].max()) == 32   # crowded pillars were exercised


@pytest.mark.parametrize("dtype", [pp.PP_F32, pp.PP_F32_TC, pp.PP_BF16])
def test_scatter_update_sequence_equals_dense(dtype):
    """pp_scatter_update on one persistent canvas over a sequence of frames (overlapping and
    disjoint pillar sets, a frame whose row has no points, the full 4000-pillar cap, a repeat)
    gives, after every frame, exactly pp_scatter's dense canvas (bit for bit, border included)."""
    g = GEOM_SMALL
    seq = [(config_points(3, 2, 40000), config_points(3, 3, 120000)),
           (config_points(3, 4, 90000), config_points(3, 3, 120000)),
           (config_points(3, 5, 2000), np.zeros((0, 4), np.float32)),
           (config_points(3, 6, 150000), config_points(3, 7, 30000)),
           (config_points(3, 6, 150000), config_points(3, 7, 30000))]
    state = pp.ScatterState(g, 2, dtype)
    for k, clouds in enumerate(seq):
        pts, n = _batch(list(clouds))
        v = pp.voxelize(pts, n, g)
        feat = torch.randn((2, g.max_pillars, 64), device=DEV) * 3
        got = pp.scatter_update(state, feat, v["coord"], v["num_pillars"], v["pillar_of_cell"])
        want = pp.scatter(feat, v["pillar_of_cell"], g, dtype=dtype)
        torch.cuda.synchronize()
        assert torch.equal(got, want), k
        assert torch.equal(state.drawn_num.cpu(), v["num_pillars"].cpu()), k


# ------------------------------------------------------------------ conv

def _conv_case(B, H, W, cin, cout, s, seed, density=0.5):
    rng = np.random.default_rng(seed)
    x = np.maximum(rng.normal(size=(B, H, W, cin)), 0) * (rng.random((B, H, W, 1)) < density)
    w = rng.normal(0, np.sqrt(2.0 / (9 * cin)), (cout, cin, 3, 3)).astype(np.float32)
    bn = np.stack([rng.uniform(0.5, 1.5, cout), rng.uniform(-0.1, 0.1, cout),
                   rng.normal(0, 0.1, cout), rng.uniform(0.5, 2.0, cout)]).astype(np.float32)
    xp = np.zeros((B, H + 2, W + 2, cin), np.float32)
    xp[:, 1:-1, 1:-1] = x
    return xp, w, bn


SHAPES = [(2, 20, 18, 64, 64, 1), (2, 20, 18, 64, 64, 2), (1, 34, 46, 128, 128, 1),
          (1, 26, 30, 64, 128, 2), (1, 14, 10, 256, 256, 1), (1, 16, 18, 128, 256, 2),
          (3, 9, 17, 64, 64, 1), (2, 22, 300, 64, 64, 1), (2, 24, 300, 64, 64, 2),
          (3, 80, 98, 128, 128, 1),   # more 128-pixel halo tiles (189) than SMs: CTAs walk several
          (1, 64, 128, 64, 64, 1)]    # 8x16 boxes tile the output exactly: more halo runs (65) than boxes


@pytest.mark.parametrize("shape", SHAPES)
def test_conv_f32(shape):
    B, H, W, cin, cout, s = shape
    xp, w, bn = _conv_case(B, H, W, cin, cout, s, seed=H * W + cin)
    x_d = torch.from_numpy(xp).to(DEV)
    wp = pp.pack_conv_weights(torch.from_numpy(w).to(DEV), pp.PP_F32)
    ss = torch.from_numpy(pp.bn_fold(bn)).to(DEV)
    refs = [O.conv3x3_bn_relu(xp[b, 1:-1, 1:-1].astype(np.float64), w, bn, s) for b in range(B)]
    for tile in range(pp.conv_tile_count(pp.PP_F32)):
        if cout % (64 if tile in (0, 1) else 128):
            continue
        out = pp.conv3x3(x_d, wp, ss, cout, s, dtype=pp.PP_F32, tile=tile)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        for b in range(B):
            assert rel_err(o[b, 1:-1, 1:-1], refs[b]) <= FP32_TOL, (tile, b)
            assert not o[b, 0].any() and not o[b, -1].any() and not o[b, :, 0].any() and not o[b, :, -1].any()


@pytest.mark.parametrize("shape", SHAPES)
def test_conv_f32_tensor_cores(shape):
    """FP32 conv on the tensor cores (3xTF32 split) meets the FP32 tolerance on every tile."""
    B, H, W, cin, cout, s = shape
    xp, w, bn = _conv_case(B, H, W, cin, cout, s, seed=H * W + cin + 2)
    x_d = pp.split_f32(torch.from_numpy(xp).to(DEV))      # split FP32 operand [2, B, ...]
    assert np.array_equal(x_d[1].cpu().numpy(), tf32_remainder(xp))
    wp = pp.pack_conv_weights(torch.from_numpy(w).to(DEV), pp.PP_F32_TC)
    ss = torch.from_numpy(pp.bn_fold(bn)).to(DEV)
    refs = [O.conv3x3_bn_relu(xp[b, 1:-1, 1:-1].astype(np.float64), w, bn, s) for b in range(B)]
    n_tiles = pp.conv_tile_count(pp.PP_F32_TC)
    assert n_tiles >= 14
    ws = pp.conv_workspace(B, H, W, cin, cout, s, pp.PP_F32_TC, DEV)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # every tile, then every tile again in reverse order on the same workspace (stream-K tiles of
    # different widths share it, as the layers of a release unit do)
    for tile in list(range(n_tiles)) + list(range(n_tiles - 1, -1, -1)) + [-1]:
        if tile >= 0 and cout % pp.conv_tile_info(pp.PP_F32_TC, tile)[2]:
            continue
        if tile >= 0 and pp.conv_tile_info(pp.PP_F32_TC, tile)[3] in (4, 5, 6) and s != 1:
            with pytest.raises(pp.PPError, match="stride-1"):  # the halo-row tile is stride 1 only
                pp.conv3x3(x_d, wp, ss, cout, s, dtype=pp.PP_F32_TC, tile=tile, workspace=ws)
            continue
        out = pp.conv3x3(x_d, wp, ss, cout, s, dtype=pp.PP_F32_TC, tile=tile, workspace=ws)
        torch.cuda.synchronize()
        assert pp.device_error() == 0
        if tile >= 0 and pp.conv_tile_info(pp.PP_F32_TC, tile)[3] in (3, 5):
            # stream-K: bit-reproducible, and the arrival counters are left zero
            again = pp.conv3x3(x_d, wp, ss, cout, s, dtype=pp.PP_F32_TC, tile=tile, workspace=ws)
            torch.cuda.synchronize()
            assert torch.equal(out, again), tile
            counters = ws[0][ws[1] - ws[0].data_ptr() + 2 * sms * 128 * 128 * 4:][: ws[2] - 2 * sms * 128 * 128 * 4]
            assert not counters.any(), tile
        o = out.cpu().numpy()
        # plane 1 is exactly the TF32 remainder of plane 0 (the next layer's A remainder)
        assert np.array_equal(o[1], tf32_remainder(o[0])), tile
        for b in range(B):
            assert rel_err(o[0, b, 1:-1, 1:-1], refs[b]) <= FP32_TOL, (tile, b)
            for q in (0, 1):
                ob = o[q, b]
                assert not ob[0].any() and not ob[-1].any() and not ob[:, 0].any() and not ob[:, -1].any()


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("shape", SHAPES)
def test_conv_bf16(shape):
    B, H, W, cin, cout, s = shape
    xp, w, bn = _conv_case(B, H, W, cin, cout, s, seed=H * W + cin + 1)
    xb = _bf16(xp)
    x_d = xb.to(DEV)
    wp = pp.pack_conv_weights(torch.from_numpy(w).to(DEV), pp.PP_BF16)
    ss = torch.from_numpy(pp.bn_fold(bn)).to(DEV)
    x_r = xb.float().numpy().astype(np.float64)
    w_r = torch.from_numpy(w).to(torch.bfloat16).float().numpy().astype(np.float64)
    loose = [O.conv3x3_bn_relu(x_r[b, 1:-1, 1:-1], w, bn, s) for b in range(B)]
    tight = [O.conv3x3_bn_relu(x_r[b, 1:-1, 1:-1], w_r, bn, s) for b in range(B)]
    for tile in list(range(pp.conv_tile_count(pp.PP_BF16))) + [-1]:
        if tile >= 0 and cout % pp.conv_tile_info(pp.PP_BF16, tile)[2]:
            continue
        if tile >= 0 and pp.conv_tile_info(pp.PP_BF16, tile)[3] == 2 and (cin != 64 or cout != 64):
            continue   # the row-streaming kernel is for 64 -> 64 channel layers
        out = pp.conv3x3(x_d, wp, ss, cout, s, dtype=pp.PP_BF16, tile=tile)
        torch.cuda.synchronize()
        assert pp.device_error() == 0
        o = out.float().cpu().numpy()
        for b in range(B):
            assert rel_err(o[b, 1:-1, 1:-1], tight[b]) <= 8e-3, (tile, b)
            assert rel_err(o[b, 1:-1, 1:-1], loose[b]) <= BF16_TOL, (tile, b)
            assert not o[b, 0].any() and not o[b, -1].any() and not o[b, :, 0].any() and not o[b, :, -1].any()


@pytest.mark.parametrize("dtype", [pp.PP_F32, pp.PP_F32_TC], ids=["cuda-cores", "3xtf32"])
def test_frame_config1_fp32_end_to_end(dtype):
    """The 20k-point frame through the stage entry points, the convs on CUDA cores (PP_F32) and
    on the tensor cores (PP_F32_TC: split FP32 operands, 3xTF32 products, the default FP32
    path), every layer's output against the FP64 oracle."""
    g, bb = GEOM_SMALL, BACKBONE_SMALL
    cloud = config_points(1, 0)
    weights = pillar_weights(bb, 7)
    ref = O.frame(cloud, g, bb, weights)
    pfn_w, pfn_bn, conv_w, conv_bn = weights
    pts, n = _batch([cloud])
    v = pp.voxelize(pts, n, g)
    feat = pp.pointnet(v["pts"], v["npts"], v["coord"], v["num_pillars"],
                       torch.from_numpy(pfn_w).to(DEV), torch.from_numpy(pp.bn_fold(pfn_bn)).to(DEV), g)
    x = pp.scatter(feat, v["pillar_of_cell"], g, dtype=dtype)
    outs = []
    for (ci, co, s), w, bn in zip(bb.layers(64), conv_w, conv_bn):
        x = pp.conv3x3(x, pp.pack_conv_weights(torch.from_numpy(w).to(DEV), dtype),
                       torch.from_numpy(pp.bn_fold(bn)).to(DEV), co, s, dtype=dtype)
        outs.append(x[0] if dtype == pp.PP_F32_TC else x)   # value plane of split FP32
    torch.cuda.synchronize()
    got = outs[-1][0, 1:-1, 1:-1].cpu().numpy()
    assert got.shape == ref["blocks"][-1].shape
    assert rel_err(got, ref["blocks"][-1]) <= FP32_TOL
    # every layer, each against the oracle's layer on the same (oracle) input chain
    r = ref["canvas"]
    for (ci, co, s), w, bn, o in zip(bb.layers(64), conv_w, conv_bn, outs):
        r = O.conv3x3_bn_relu(r, w, bn, s)
        assert rel_err(o[0, 1:-1, 1:-1].cpu().numpy(), r) <= FP32_TOL, (ci, co, s)


@pytest.mark.parametrize("dtype", [pp.PP_BF16, pp.PP_F32_TC])
def test_conv_autotune_then_library_choice(dtype):
    """The autotuner picks a tile that supports the shape; afterwards tile = -1 uses it and the
    result is bit-identical to an explicit launch of that tile (and still meets tolerance)."""
    pp.conv_tune_clear()
    B, H, W, cin, cout, s = 2, 30, 44, 64, 64, 2
    xp, w, bn = _conv_case(B, H, W, cin, cout, s, seed=77)
    if dtype == pp.PP_BF16:
        x_d = _bf16(xp).to(DEV)
    else:
        x_d = pp.split_f32(torch.from_numpy(xp).to(DEV))
    wp = pp.pack_conv_weights(torch.from_numpy(w).to(DEV), dtype)
    ss = torch.from_numpy(pp.bn_fold(bn)).to(DEV)
    Ho, Wo = (H - 1) // s + 1, (W - 1) // s + 1
    planes = (2,) if dtype == pp.PP_F32_TC else ()
    out = torch.zeros(planes + (B, Ho + 2, Wo + 2, cout), dtype=x_d.dtype, device=DEV)
    tile, us = pp.conv_autotune(x_d, wp, ss, cout, s, dtype, out)
    assert 0 <= tile < pp.conv_tile_count(dtype) and us > 0
    explicit = pp.conv3x3(x_d, wp, ss, cout, s, dtype=dtype, tile=tile)
    chosen = pp.conv3x3(x_d, wp, ss, cout, s, dtype=dtype, tile=-1)
    torch.cuda.synchronize()
    assert torch.equal(explicit, chosen)
    ref = [O.conv3x3_bn_relu(xp[b, 1:-1, 1:-1].astype(np.float64), w, bn, s) for b in range(B)]
    o = (chosen[0] if dtype == pp.PP_F32_TC else chosen).float().cpu().numpy()
    for b in range(B):
        tol = FP32_TOL if dtype == pp.PP_F32_TC else BF16_TOL
        assert rel_err(o[b, 1:-1, 1:-1], ref[b]) <= tol
    pp.conv_tune_clear()


# ---- neck (transposed-conv upsampling + concatenation) and detection head

def _dev_input(xp, dtype):
    t = torch.from_numpy(xp).to(DEV)
    return pp.split_f32(t) if dtype == pp.PP_F32_TC else t.to(torch.bfloat16)


def _ref_input(xp, dtype):
    """What the kernel reads: the FP32 values, or their BF16 roundings."""
    return xp.astype(np.float64) if dtype == pp.PP_F32_TC else _bf16(xp).double().numpy()


def _close(got, ref, dtype):
    if dtype == pp.PP_F32_TC:
        return rel_err(got, ref) <= FP32_TOL
    from tests._util import max_norm_err
    return max_norm_err(got, ref) <= BF16_TOL


@pytest.mark.parametrize("dtype", [pp.PP_F32_TC, pp.PP_BF16])
@pytest.mark.parametrize("up,cin,H,W", [(1, 64, 13, 37), (2, 128, 9, 21), (4, 256, 5, 11)])
def test_upsample_into_concat(dtype, up, cin, H, W):
    """Transposed conv (kernel = stride = up) + BN + ReLU written into its channel range of a
    concatenated map, on every persistent tile: matches the oracle; the other channel ranges and
    the border stay zero."""
    B, cout, out_c, coff = 2, 128, 384, 128
    xp, _, bn = _conv_case(B, H, W, cin, cout, 1, seed=up * 100 + cin)
    rng = np.random.default_rng(up)
    w = rng.normal(0, np.sqrt(2.0 / cin), (cin, cout, up, up)).astype(np.float32)
    x_d = _dev_input(xp, dtype)
    wp = pp.pack_upsample_weights(w, up, dtype)
    ss = torch.from_numpy(pp.bn_fold(bn)).to(DEV)
    xr = _ref_input(xp, dtype)
    refs = [O.deconv_bn_relu(xr[b, 1:-1, 1:-1], w, bn, up) for b in range(B)]
    planes = (2,) if dtype == pp.PP_F32_TC else ()
    tdt = torch.float32 if dtype == pp.PP_F32_TC else torch.bfloat16
    tiles = [t for t in range(pp.conv_tile_count(dtype))
             if pp.conv_tile_info(dtype, t)[3] == 1 and cout % pp.conv_tile_info(dtype, t)[2] == 0]
    assert tiles
    for tile in [-1] + tiles:
        out = torch.zeros(planes + (B, up * H + 2, up * W + 2, out_c), dtype=tdt, device=DEV)
        pp.upsample(x_d, wp, ss, cout, up, dtype, out, out_coff=coff, tile=tile)
        torch.cuda.synchronize()
        assert pp.device_error() == 0
        o = (out[0] if planes else out).float().cpu().numpy()
        for b in range(B):
            assert _close(o[b, 1:-1, 1:-1, coff:coff + cout], refs[b], dtype), (tile, b)
        assert not o[:, :, :, :coff].any() and not o[:, :, :, coff + cout:].any()
        assert not o[:, 0].any() and not o[:, -1].any() and not o[:, :, 0].any() and not o[:, :, -1].any()
        if planes:
            assert np.array_equal(out[1].cpu().numpy(), tf32_remainder(out[0].cpu().numpy()))


@pytest.mark.parametrize("dtype", [pp.PP_F32_TC, pp.PP_BF16])
def test_head_1x1(dtype):
    """The 1x1 head with bias (no activation) over a 384-channel map: matches the oracle; the
    channels past the 72 outputs are zero."""
    B, H, W, cin, cout = 2, 19, 27, 384, 72
    xp, _, _ = _conv_case(B, H, W, cin, 64, 1, seed=9)
    rng = np.random.default_rng(10)
    w = rng.normal(0, np.sqrt(1.0 / cin), (cout, cin)).astype(np.float32)
    bias = rng.uniform(-0.1, 0.1, cout).astype(np.float32)
    x_d = _dev_input(xp, dtype)
    wp, ss = pp.pack_head_weights(w, bias, dtype)
    xr = _ref_input(xp, dtype)
    out = pp.head(x_d, wp, ss, cout, dtype)
    torch.cuda.synchronize()
    o = (out[0] if dtype == pp.PP_F32_TC else out).float().cpu().numpy()
    assert o.shape[-1] == 128 and not o[..., cout:].any()
    for b in range(B):
        ref = O.head(xr[b, 1:-1, 1:-1], w, bias)
        assert _close(o[b, 1:-1, 1:-1, :cout], ref, dtype), b


def test_neck_head_full_size_fp32():
    """Neck + head on the full-size frame's three block outputs (432x496 grid: 64/128/256
    channels at 248x216, 124x108, 62x54): three transposed convs into one 384-channel map,
    then the 72-output head, against the oracle."""
    from pp_synth import BACKBONE_FULL, head_weights
    up_w, up_bn, hw, hb = head_weights(BACKBONE_FULL)
    rng = np.random.default_rng(21)
    sizes = [(248, 216, 64), (124, 108, 128), (62, 54, 256)]
    blocks = []
    for (H, W, C) in sizes:
        xp = np.zeros((1, H + 2, W + 2, C), np.float32)
        xp[0, 1:-1, 1:-1] = np.maximum(rng.normal(size=(H, W, C)), 0).astype(np.float32)
        blocks.append(xp)
    neck = torch.zeros((2, 1, 250, 218, 384), device=DEV)
    for k, (xp, w, bn) in enumerate(zip(blocks, up_w, up_bn)):
        up = 2 ** k
        pp.upsample(pp.split_f32(torch.from_numpy(xp).to(DEV)), pp.pack_upsample_weights(w, up, pp.PP_F32_TC),
                    torch.from_numpy(pp.bn_fold(bn)).to(DEV), 128, up, pp.PP_F32_TC, neck, out_coff=128 * k)
    wp, ss = pp.pack_head_weights(hw, hb, pp.PP_F32_TC)
    out = pp.head(neck, wp, ss, 72, pp.PP_F32_TC)
    torch.cuda.synchronize()
    n_ref = O.neck([b[0, 1:-1, 1:-1].astype(np.float64) for b in blocks], up_w, up_bn)
    assert rel_err(neck[0, 0, 1:-1, 1:-1].cpu().numpy(), n_ref) <= FP32_TOL
    h_ref = O.head(n_ref, hw, hb)
    assert rel_err(out[0, 0, 1:-1, 1:-1, :72].cpu().numpy(), h_ref) <= FP32_TOL

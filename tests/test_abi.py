"""The C-ABI library builds, loads without a GPU, and exports every function include/*.h
declares; host-only entry points behave as documented.  CPU only (no compute calls)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pp_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2509_12207_gb300 import _build
    _build.build()
    import paper_2509_12207_gb300 as pp
    return pp.lib()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2509_12207_gb300 as pp
    assert set(pp.declared_symbols()) <= _declared()
    assert _declared() <= set(pp.declared_symbols())


def test_version_and_errors(lib):
    import paper_2509_12207_gb300 as pp
    assert b"sm_103a" in lib.pp_version()
    # argument validation runs on the host and records a message
    g = pp.Geometry(0, 1, 0, 1, 0, 1, 0.5, 0.5, 2, 2, 4, 16)   # max_pts != 32
    assert lib.pp_voxelize_workspace_bytes(ctypes.byref(g), 1, 10) == 0
    rc = lib.pp_conv3x3(1, 8, 8, 48, 64, 1, 0, 16, 16, 16, 16, -1, None)
    assert rc == pp.PP_EINVAL and b"multiples of 64" in lib.pp_last_error()
    rc = lib.pp_conv3x3(1, 7, 8, 64, 64, 2, 0, 16, 16, 16, 16, -1, None)
    assert rc == pp.PP_EINVAL and b"even" in lib.pp_last_error()
    assert lib.pp_conv_packed_bytes(64, 128, 1) == 9 * 64 * 128 * 2
    # weights are packed only for the shapes pp_conv3x3 takes (it reads 9 cin cout of them)
    assert lib.pp_conv_packed_bytes(3, 64, 1) == 0 and lib.pp_conv_packed_bytes(64, 72, 2) == 0
    rc = lib.pp_conv_pack_weights(16, 3, 64, 2, 16, None)
    assert rc == pp.PP_EINVAL and b"multiples of 64" in lib.pp_last_error()
    import torch
    with pytest.raises(pp.PPError, match="OIHW"):
        pp.pack_conv_weights(torch.zeros(64, 3, 3, 64), pp.PP_F32_TC)


def test_bn_fold_matches_definition(lib):
    import paper_2509_12207_gb300 as pp
    rng = np.random.default_rng(0)
    bn = np.stack([rng.uniform(0.5, 1.5, 64), rng.uniform(-1, 1, 64), rng.normal(size=64),
                   rng.uniform(0.1, 3, 64)]).astype(np.float32)
    ss = pp.bn_fold(bn)
    h = rng.normal(size=(100, 64)) * 3
    want = bn[0] * (h - bn[2]) / np.sqrt(bn[3].astype(np.float64) + 1e-3) + bn[1]
    np.testing.assert_allclose(h * ss[0] + ss[1], want, rtol=1e-6, atol=1e-6)


def test_tune_table_save_load(lib, tmp_path):
    import paper_2509_12207_gb300 as pp
    pp.conv_tune_clear()
    f = tmp_path / "tiles.txt"
    n_bf16 = pp.conv_tile_count(pp.PP_BF16)
    f.write_text("# comment\n"
                 "1 8 248 216 64 64 2 %d 20.5\n"   # valid
                 "1 8 124 108 64 64 1 999 1.0\n"   # tile does not exist: skipped
                 "garbage line\n"
                 "0 1 496 432 64 64 2 1 40.0\n" % (n_bf16 - 1))
    assert pp.conv_tune_load(f) == 2
    out = tmp_path / "saved.txt"
    pp.conv_tune_save(out)
    lines = [l for l in out.read_text().splitlines() if not l.startswith("#")]
    assert sorted(l.split()[:8] for l in lines) == sorted([
        ["0", "1", "496", "432", "64", "64", "2", "1"], ["1", "8", "248", "216", "64", "64", "2", str(n_bf16 - 1)]])
    pp.conv_tune_clear()
    pp.conv_tune_save(out)
    assert [l for l in out.read_text().splitlines() if not l.startswith("#")] == []
    with pytest.raises(pp.PPError):
        pp.conv_tune_load(tmp_path / "missing.txt")


def test_config_defaults_and_host_validation(lib):
    """pp_config_defaults fills the documented defaults; host-side checks of the workspace and
    split-FP32 entry points reject bad arguments without touching a GPU."""
    import paper_2509_12207_gb300 as pp
    cfg = pp.Config()
    lib.pp_config_defaults(ctypes.byref(cfg))
    assert cfg.autotune == 1 and cfg.stream_k == 0 and cfg.fp32_cuda_cores == 0
    assert cfg.policy == pp.PP_POLICY_URGENCY
    # stream-K workspaces exist only for the 3xTF32 dtype
    assert lib.pp_conv_workspace_bytes(1, 62, 54, 256, 256, 1, pp.PP_BF16) == 0
    assert lib.pp_conv_workspace_bytes(1, 62, 54, 256, 256, 1, pp.PP_F32_TC) > 0
    assert lib.pp_conv_workspace_bytes(1, 62, 54, 250, 256, 1, pp.PP_F32_TC) == 0
    assert lib.pp_tf32_split(None, None, 0, None) == pp.PP_OK
    assert lib.pp_tf32_split(16, 16, -1, None) == pp.PP_EINVAL
    assert lib.pp_tf32_split(16, 32, 8, None) == pp.PP_EINVAL and b"overlap" in lib.pp_last_error()
    assert lib.pp_tf32_split(17, 4096, 8, None) == pp.PP_EINVAL and b"aligned" in lib.pp_last_error()
    # a 3xTF32 tile index is plain (persistent = 1), its stream-K twin (3), or, last, one of the
    # seven halo tiles: runs of 128 output pixels with 64 / 128 channels and a unified ring or
    # split A and B rings, the same with deeper split rings (4), the first two with the stream-K
    # partition over accumulation groups (5), then runs of 126 pixels with the three kx taps in
    # the MMA's N dimension (6)
    n = lib.pp_conv_tile_count(pp.PP_F32_TC)
    npl = (n - 7) // 2
    for t in range(n):
        info = pp.conv_tile_info(pp.PP_F32_TC, t)
        assert info[3] == (1 if t < npl else 3 if t < 2 * npl else 4 if t < n - 3 else 5 if t < n - 1 else 6)
        if t < 2 * npl:
            assert info[:3] == pp.conv_tile_info(pp.PP_F32_TC, t % npl)[:3]
    assert [pp.conv_tile_info(pp.PP_F32_TC, n - 7 + i) for i in range(7)] == [
        (1, 128, 64, 4), (1, 128, 128, 4), (1, 128, 64, 4), (1, 128, 128, 4), (1, 128, 64, 5), (1, 128, 128, 5),
        (1, 126, 64, 6)]
    with pytest.raises(pp.PPError):
        pp.conv_tile_info(pp.PP_F32_TC, n)


def test_neck_head_host_validation(lib):
    import paper_2509_12207_gb300 as pp
    # packed sizes: [up*up*cout][cin] (BF16) or [2][up*up*cout][cin] (split FP32); the head pads
    # its outputs to a multiple of 64
    assert lib.pp_upsample_packed_bytes(128, 128, 2, pp.PP_BF16) == 4 * 128 * 128 * 2
    assert lib.pp_upsample_packed_bytes(256, 128, 4, pp.PP_F32_TC) == 2 * 16 * 128 * 256 * 4
    assert lib.pp_head_packed_bytes(384, 72, pp.PP_BF16) == 128 * 384 * 2
    assert lib.pp_head_packed_bytes(384, 72, pp.PP_F32_TC) == 2 * 128 * 384 * 4
    assert lib.pp_upsample_packed_bytes(100, 128, 2, pp.PP_BF16) == 0
    assert lib.pp_upsample_packed_bytes(128, 128, 2, pp.PP_F32) == 0
    p = 4096
    ok = (1, 8, 8, 128, 128, 2, pp.PP_BF16, p, p, p, p, 384, 128, -1, None)
    for i, bad in [(3, 96), (4, 100), (5, 0), (5, 9), (11, 200), (12, 32), (12, 320)]:
        args = list(ok)
        args[i] = bad
        assert lib.pp_upsample(*args) == pp.PP_EINVAL, (i, bad)
    args = list(ok)
    args[7] = None
    assert lib.pp_upsample(*args) == pp.PP_EINVAL and b"NULL" in lib.pp_last_error()
    assert lib.pp_head(1, 8, 8, 100, 72, pp.PP_BF16, p, p, p, p, -1, None) == pp.PP_EINVAL
    assert lib.pp_head(1, 8, 8, 384, 0, pp.PP_BF16, p, p, p, p, -1, None) == pp.PP_EINVAL
    assert lib.pp_head(1, 8, 8, 384, 72, pp.PP_BF16, None, p, p, p, -1, None) == pp.PP_EINVAL


def test_config_head_defaults_and_layout(lib):
    import ctypes
    import paper_2509_12207_gb300 as pp
    cfg = pp.Config()
    lib.pp_config_defaults(ctypes.byref(cfg))
    assert cfg.head_outputs == 0 and cfg.up_channels == 128 and not cfg.up_w and not cfg.head_w
    assert cfg.eqdf_lambda == 0.5 and cfg.est_noise == 0.0
    # every Python struct mirror has the size of the C struct of this build
    mirrors = {"pp_config": pp.Config, "pp_result": pp.Result, "pp_stats": pp.Stats, "pp_geometry": pp.Geometry,
               "pp_arrival": pp.Arrival, "pp_replay_stats": pp.ReplayStats, "pp_policy_frame": pp.PolicyFrame,
               "pp_policy_active": pp.PolicyActive, "pp_policy_config": pp.PolicyConfig,
               "pp_policy_decision": pp.PolicyDecision, "pp_decision_record": pp.DecisionRecord}
    for name, cls in mirrors.items():
        assert lib.pp_struct_size(name.encode()) == ctypes.sizeof(cls), name
    assert lib.pp_struct_size(b"pp_nothing") == 0


def test_runtime_declarations_cite_the_paper():
    """Every entry point of the serving runtime (from the runtime banner of include/pp.h on) is
    preceded by a comment that names the passage it restates (a Section, Eq. or Table) or says
    that the paper has no counterpart; a declaration right after another with no comment of its
    own shares that one's."""
    src = open(os.path.join(ROOT, "include", "pp.h")).read()
    body = src[src.index("Serving runtime."):]
    cite = re.compile(r"(Section \d|Eq\. \d|Table \d|no counterpart in the paper|the paper has no counterpart)",
                      re.I)
    prev, last_ok, seen, missing = 0, False, [], []
    for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pp_\w+)\s*\(", body, flags=re.M):
        seg = body[prev:m.start()]
        comments = "\n".join(re.findall(r"/\*.*?\*/", seg, flags=re.S))
        text = " ".join(re.sub(r"/\*|\*/|^\s*\*", " ", comments, flags=re.M).split())
        ok = bool(cite.search(text)) if comments else last_ok
        last_ok = ok
        seen.append(m.group(1))
        if not ok:
            missing.append(m.group(1))
        prev = body.index(";", m.end()) + 1
    for name in ("pp_create", "pp_register_chain", "pp_submit_frame", "pp_submit_frames", "pp_submit_frames_ex",
                 "pp_poll", "pp_result_release", "pp_result_release_many", "pp_get_stats", "pp_destroy",
                 "pp_policy_decide", "pp_decision_log"):
        assert name in seen, name
    assert not missing, missing


def test_noise_factor_matches_splitmix64(lib):
    """The runtime's per-frame estimate-noise factor is the published SplitMix64 sequence
    (first outputs for seed 0 are the reference values of the generator's C source)."""
    import paper_2509_12207_gb300 as pp
    from pp_synth import noise_factors, splitmix64
    assert splitmix64(0, 1) == 0xE220A8397B1DCDAF
    assert splitmix64(0, 2) == 0x6E789E6AA1B965F4
    assert splitmix64(0, 3) == 0x06C45D188009454F
    ids = [1, 2, 3, 17, 1000, 123456789]
    for seed in (0, 7, 2 ** 63 + 5):
        want = noise_factors(seed, ids, 0.3)
        got = [pp.noise_factor(seed, i, 0.3) for i in ids]
        assert got == list(want)
        assert all(0.7 <= g < 1.3 for g in got)
    assert pp.noise_factor(5, 9, 0.0) == 1.0
    f = noise_factors(11, range(1, 20001), 0.3)
    assert abs(f.mean() - 1.0) < 0.01 and f.min() >= 0.7 and f.max() < 1.3

"""Python binding of ``libpp.so`` (C ABI in ``include/pp.h``): argument marshalling only.

Every step of the pillar front end and the serving runtime runs inside the library's CUDA
kernels and C++ runtime; PyTorch is used here only to allocate device memory and to hand over
CUDA stream handles.  There is no fallback: if the library has not been built (``build()``) or
no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpp.so")

PP_OK, PP_EINVAL, PP_ENOMEM, PP_EAGAIN, PP_ETIMEDOUT, PP_EDEVICE, PP_ESTATE = 0, -1, -2, -3, -4, -5, -6
PP_F32, PP_BF16, PP_F32_TC = 0, 1, 2
BN_EPS = 1e-3


class PPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("pp error %d: %s" % (code, msg))
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax", "vx", "vy")] + \
               [(n, ctypes.c_int32) for n in ("nx", "ny", "max_pillars", "max_pts")]

    @classmethod
    def of(cls, g) -> "Geometry":
        if isinstance(g, cls):
            return g
        return cls(g.xmin, g.xmax, g.ymin, g.ymax, g.zmin, g.zmax, g.vx, g.vy,
                   g.nx, g.ny, g.max_pillars, getattr(g, "max_pts", 32))


MAX_BLOCKS = 4
MAX_CHAINS = 64
PP_POLICY_FIFO, PP_POLICY_URGENCY, PP_POLICY_EDF, PP_POLICY_SJF, PP_POLICY_HRRN, PP_POLICY_LCUF = 0, 1, 2, 3, 4, 5
PP_POLICY_SAEDF, PP_POLICY_EQDF = 6, 7
PP_FRAME_DONE, PP_FRAME_DROPPED, PP_FRAME_ERROR = 0, 1, 2
PP_POINTS_HOST, PP_POINTS_DEVICE, PP_POINTS_PINNED = 0, 1, 2


def _points_mode(t):
    """PP_POINTS_* for a frame: CUDA tensor -> device (borrowed), pinned CPU tensor -> pinned
    (borrowed, read in place by the kernels), anything else -> host (copied)."""
    if hasattr(t, "is_cuda"):
        if t.is_cuda:
            return PP_POINTS_DEVICE
        if t.is_pinned():
            return PP_POINTS_PINNED
    return PP_POINTS_HOST
PP_DECIDE_NONE, PP_DECIDE_RELEASE, PP_DECIDE_WAIT, PP_DECIDE_DELAY = 0, 1, 2, 3


class Config(ctypes.Structure):
    _fields_ = [
        ("geom", Geometry),
        ("n_blocks", ctypes.c_int32), ("convs", ctypes.c_int32 * MAX_BLOCKS),
        ("chans", ctypes.c_int32 * MAX_BLOCKS), ("strides", ctypes.c_int32 * MAX_BLOCKS),
        ("pfn_w", ctypes.c_void_p), ("pfn_bn", ctypes.c_void_p),
        ("conv_w", ctypes.c_void_p), ("conv_bn", ctypes.c_void_p),
        ("max_batch", ctypes.c_int32), ("cap_points", ctypes.c_int32),
        ("precisions", ctypes.c_int32), ("units", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("policy", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
        ("delta_eval_us", ctypes.c_double), ("max_closed", ctypes.c_int32),
        ("delay_quantum_us", ctypes.c_double), ("th_urgent", ctypes.c_double),
        ("th_calib_frames", ctypes.c_int32), ("util_exempt", ctypes.c_double),
        ("early_exit", ctypes.c_int32), ("num_streams", ctypes.c_int32),
        ("max_admitted", ctypes.c_int32), ("fp32_cuda_cores", ctypes.c_int32),
        ("autotune", ctypes.c_int32), ("stream_k", ctypes.c_int32),
        ("head_outputs", ctypes.c_int32), ("up_channels", ctypes.c_int32),
        ("up_w", ctypes.c_void_p), ("up_bn", ctypes.c_void_p),
        ("head_w", ctypes.c_void_p), ("head_b", ctypes.c_void_p),
        ("eqdf_lambda", ctypes.c_double),
        ("est_noise", ctypes.c_double), ("noise_seed", ctypes.c_uint64),
        ("keep_blocks", ctypes.c_int32), ("decision_log", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("frame_id", ctypes.c_uint64), ("chain_id", ctypes.c_int32), ("status", ctypes.c_int32),
        ("t_arr_us", ctypes.c_double), ("t_release_us", ctypes.c_double),
        ("t_done_us", ctypes.c_double), ("deadline_us", ctypes.c_double),
        ("missed", ctypes.c_int32), ("num_pillars", ctypes.c_int32),
        ("batch", ctypes.c_int32), ("level", ctypes.c_int32),
        ("out_dev", ctypes.c_void_p), ("out_c", ctypes.c_int32), ("out_h", ctypes.c_int32),
        ("out_w", ctypes.c_int32), ("out_dtype", ctypes.c_int32),
        ("block_dev", ctypes.c_void_p * MAX_BLOCKS), ("block_c", ctypes.c_int32 * MAX_BLOCKS),
        ("block_h", ctypes.c_int32 * MAX_BLOCKS), ("block_w", ctypes.c_int32 * MAX_BLOCKS),
        ("out_valid_c", ctypes.c_int32),
        ("out_host", ctypes.c_void_p),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64), ("done", ctypes.c_uint64), ("dropped", ctypes.c_uint64),
        ("missed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
        ("overall_miss_ratio", ctypes.c_double), ("lat_p50_us", ctypes.c_double),
        ("lat_p99_us", ctypes.c_double), ("lat_mean_us", ctypes.c_double),
        ("frames_per_s", ctypes.c_double), ("units_launched", ctypes.c_uint64),
        ("mean_batch", ctypes.c_double), ("delayed_releases", ctypes.c_uint64),
        ("delayed_us", ctypes.c_double), ("collisions", ctypes.c_uint64),
        ("sched_us_per_decision", ctypes.c_double), ("th_urgent", ctypes.c_double),
        ("chain_frames", ctypes.c_uint64 * MAX_CHAINS), ("chain_missed", ctypes.c_uint64 * MAX_CHAINS),
        ("chain_p99_us", ctypes.c_double * MAX_CHAINS),
        ("device_errors", ctypes.c_uint64), ("device_error_code", ctypes.c_uint32),
        ("decisions", ctypes.c_uint64),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("chain_")}
        d["chain_frames"] = list(self.chain_frames)
        d["chain_missed"] = list(self.chain_missed)
        d["chain_p99_us"] = list(self.chain_p99_us)
        return d


class Arrival(ctypes.Structure):
    _fields_ = [("t_us", ctypes.c_double), ("chain_id", ctypes.c_int32), ("cloud", ctypes.c_int32),
                ("n_points", ctypes.c_int64)]


class ReplayStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("rejected", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("dropped", ctypes.c_uint64), ("chain_rejected", ctypes.c_uint64 * MAX_CHAINS),
                ("wall_s", ctypes.c_double), ("submit_late_us_max", ctypes.c_double),
                ("submit_late_us_mean", ctypes.c_double)]


class PolicyFrame(ctypes.Structure):
    _fields_ = [("frame_id", ctypes.c_uint64), ("chain_id", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("t_arr_us", ctypes.c_double), ("deadline_us", ctypes.c_double),
                ("est_gpu_us", ctypes.c_double), ("est_cpu_us", ctypes.c_double), ("util", ctypes.c_double),
                ("period_us", ctypes.c_double)]


class PolicyActive(ctypes.Structure):
    _fields_ = [("chain_id", ctypes.c_int32), ("ul", ctypes.c_double)]


class PolicyConfig(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("max_closed", ctypes.c_int32),
                ("num_pri", ctypes.c_int32), ("early_exit", ctypes.c_int32),
                ("th_urgent", ctypes.c_double), ("util_exempt", ctypes.c_double),
                ("eqdf_lambda", ctypes.c_double)]


class PolicyDecision(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("n_frames", ctypes.c_int32),
                ("n_drops", ctypes.c_int32), ("frames", ctypes.c_uint64 * 8)]


class DecisionRecord(ctypes.Structure):
    _fields_ = [("t_us", ctypes.c_double), ("cfg", PolicyConfig), ("closed_pending", ctypes.c_int32),
                ("n_ready", ctypes.c_int32), ("n_active", ctypes.c_int32), ("launched", ctypes.c_int32),
                ("ready_off", ctypes.c_int64), ("active_off", ctypes.c_int64), ("drops_off", ctypes.c_int64),
                ("decision", PolicyDecision)]


_lib: Optional[ctypes.CDLL] = None

_P = ctypes.c_void_p
_I = ctypes.c_int32
_SZ = ctypes.c_size_t
_GP = ctypes.POINTER(Geometry)

# name -> (restype, argtypes)
_SIGS = {
    "pp_version": (ctypes.c_char_p, []),
    "pp_last_error": (ctypes.c_char_p, []),
    "pp_voxelize_workspace_bytes": (_SZ, [_GP, _I, _I]),
    "pp_voxelize": (ctypes.c_int, [_GP, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "pp_voxelize_check": (ctypes.c_int, [_P, _P]),
    "pp_voxelize_pointnet": (ctypes.c_int, [_GP, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "pp_voxelize_static": (ctypes.c_int, [_GP, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pp_pointnet": (ctypes.c_int, [_GP, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pp_scatter": (ctypes.c_int, [_GP, _I, _P, _P, _P, _I, _P]),
    "pp_scatter_update": (ctypes.c_int, [_GP, _I, _P, _P, _P, _P, _P, _P, _P, _I, _P]),
    "pp_conv3x3": (ctypes.c_int, [_I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I, _P]),
    "pp_conv_tile_count": (ctypes.c_int, [_I]),
    "pp_conv_packed_bytes": (_SZ, [_I, _I, _I]),
    "pp_conv_tile_info": (ctypes.c_int, [_I, _I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "pp_conv_pack_weights": (ctypes.c_int, [_P, _I, _I, _I, _P, _P]),
    "pp_bn_fold": (ctypes.c_int, [_P, _I, ctypes.c_float, _P]),
    "pp_conv_autotune": (ctypes.c_int, [_I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
    "pp_tf32_split": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "pp_upsample_packed_bytes": (_SZ, [_I, _I, _I, _I]),
    "pp_upsample_pack_weights": (ctypes.c_int, [_P, _I, _I, _I, _I, _P]),
    "pp_head_packed_bytes": (_SZ, [_I, _I, _I]),
    "pp_head_pack_weights": (ctypes.c_int, [_P, _P, _I, _I, _I, _P, _P]),
    "pp_upsample": (ctypes.c_int, [_I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I, _I, _I, _P]),
    "pp_head": (ctypes.c_int, [_I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I, _P]),
    "pp_conv3x3_ws": (ctypes.c_int, [_I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I, _P, _SZ, _P]),
    "pp_conv_workspace_bytes": (_SZ, [_I, _I, _I, _I, _I, _I, _I]),
    "pp_conv_autotune_ws": (ctypes.c_int, [_I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _SZ, _I,
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
    "pp_conv_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "pp_conv_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "pp_conv_tune_clear": (None, []),
    "pp_device_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32), _I]),
    "pp_device_error_set": (ctypes.c_int, [ctypes.c_uint32]),
    "pp_decision_log": (ctypes.c_int, [_P, ctypes.POINTER(DecisionRecord), _I, ctypes.POINTER(PolicyFrame),
                                       ctypes.c_int64, ctypes.POINTER(PolicyActive), ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "pp_config_defaults": (None, [ctypes.POINTER(Config)]),
    "pp_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "pp_register_chain": (ctypes.c_int, [_P, _I, ctypes.c_double, ctypes.c_double, _I]),
    "pp_register_synthetic_chain": (ctypes.c_int, [_P, _I, ctypes.c_double, ctypes.c_double, _I, ctypes.c_double,
                                                   ctypes.c_double]),
    "pp_submit_frame": (ctypes.c_int, [_P, _I, _P, ctypes.c_int64, _I, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "pp_poll": (ctypes.c_int, [_P, ctypes.POINTER(Result), _I, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64]),
    "pp_submit_frames": (ctypes.c_int, [_P, _I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_int64), _I, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "pp_submit_frames_ex": (ctypes.c_int, [_P, _I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_int64), _I, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32)]),
    "pp_result_bytes": (_SZ, [_P, _I]),
    "pp_result_release": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "pp_result_release_many": (ctypes.c_int, [_P, _I, ctypes.POINTER(ctypes.c_uint64)]),
    "pp_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "pp_stats_reset": (ctypes.c_int, [_P]),
    "pp_destroy": (ctypes.c_int, [_P]),
    "pp_now_us": (ctypes.c_double, []),
    "pp_struct_size": (_SZ, [ctypes.c_char_p]),
    "pp_noise_factor": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double]),
    "pp_pipeline_create": (ctypes.c_int, [ctypes.POINTER(Config), _I, ctypes.POINTER(ctypes.c_void_p)]),
    "pp_pipeline_run": (ctypes.c_int, [_P, _I, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int32),
                                       _I, _P]),
    "pp_pipeline_output": (ctypes.c_int, [_P, _I, _I, ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "pp_pipeline_bytes": (_SZ, [_P]),
    "pp_pipeline_destroy": (ctypes.c_int, [_P]),
    "pp_policy_priority": (ctypes.c_double, [ctypes.POINTER(PolicyConfig), ctypes.c_double,
                                             ctypes.POINTER(PolicyFrame)]),
    "pp_replay": (ctypes.c_int, [_P, ctypes.POINTER(Arrival), ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p),
                                 ctypes.POINTER(ctypes.c_int64), _I, _I, ctypes.c_double, ctypes.POINTER(ReplayStats)]),
    "pp_policy_decide": (ctypes.c_int, [ctypes.POINTER(PolicyConfig), ctypes.c_double, ctypes.POINTER(PolicyFrame),
                                        _I, ctypes.POINTER(PolicyActive), _I, _I, ctypes.POINTER(PolicyDecision),
                                        ctypes.POINTER(ctypes.c_uint64), _I]),
}


def lib() -> ctypes.CDLL:
    """Loads the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PPError(PP_ESTATE, "libpp.so is not built; run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return sorted(_SIGS)


def _check(code: int) -> None:
    if code != PP_OK:
        raise PPError(code, lib().pp_last_error().decode())


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream=None) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise PPError(PP_EINVAL, "tensor must be on a CUDA device")


# ------------------------------------------------------------------ stage entry points

def voxelize(points, n_points, geom, stream=None) -> Dict[str, object]:
    """points: cuda float32 [B, cap, 4]; n_points: cuda int32 [B].  Returns the pp_voxelize
    outputs as tensors (see pp.h)."""
    import torch
    _need_cuda(points, n_points)
    g = Geometry.of(geom)
    B, cap = int(points.shape[0]), int(points.shape[1])
    dev = points.device
    G, P = g.nx * g.ny, g.max_pillars
    out = {
        "cell": torch.empty((B, cap), dtype=torch.int32, device=dev),
        "cnt": torch.empty((B, G), dtype=torch.int32, device=dev),
        "pillar_of_cell": torch.empty((B, G), dtype=torch.int32, device=dev),
        "coord": torch.empty((B, P), dtype=torch.int32, device=dev),
        "npts": torch.empty((B, P), dtype=torch.int32, device=dev),
        "num_pillars": torch.empty((B,), dtype=torch.int32, device=dev),
        "pts": torch.empty((B, P, 32, 4), dtype=torch.float32, device=dev),
    }
    ws_bytes = lib().pp_voxelize_workspace_bytes(ctypes.byref(g), B, cap)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    off = (-ws.data_ptr()) % 256
    ws_ptr = ws.data_ptr() + off
    ws[off:off + 256].zero_()  # the error word; the rest needs no initialisation
    s = _stream(stream)
    _check(lib().pp_voxelize(ctypes.byref(g), B, cap, _ptr(points), _ptr(n_points), _ptr(out["cell"]),
                             _ptr(out["cnt"]), _ptr(out["pillar_of_cell"]), _ptr(out["coord"]),
                             _ptr(out["npts"]), _ptr(out["num_pillars"]), _ptr(out["pts"]),
                             ws_ptr, ws_bytes, s))
    out["_workspace"] = (ws, ws_ptr)
    return out


def voxelize_pointnet(points, n_points, geom, pfn_w, scale_shift, stream=None) -> Dict[str, object]:
    """pp_voxelize_pointnet: pp_voxelize's outputs without pts, plus "feat" [B, P, 64]."""
    import torch
    _need_cuda(points, n_points, pfn_w, scale_shift)
    g = Geometry.of(geom)
    B, cap = int(points.shape[0]), int(points.shape[1])
    dev = points.device
    G, P = g.nx * g.ny, g.max_pillars
    out = {k: torch.empty(shape, dtype=torch.int32, device=dev) for k, shape in
           (("cell", (B, cap)), ("cnt", (B, G)), ("pillar_of_cell", (B, G)), ("coord", (B, P)),
            ("npts", (B, P)), ("num_pillars", (B,)))}
    out["feat"] = torch.empty((B, P, 64), dtype=torch.float32, device=dev)
    ws_bytes = lib().pp_voxelize_workspace_bytes(ctypes.byref(g), B, cap)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    off = (-ws.data_ptr()) % 256
    ws_ptr = ws.data_ptr() + off
    ws[off:off + 256].zero_()  # the error word; the rest needs no initialisation
    _check(lib().pp_voxelize_pointnet(ctypes.byref(g), B, cap, _ptr(points), _ptr(n_points), _ptr(out["cell"]),
                                      _ptr(out["cnt"]), _ptr(out["pillar_of_cell"]), _ptr(out["coord"]),
                                      _ptr(out["npts"]), _ptr(out["num_pillars"]), _ptr(pfn_w), _ptr(scale_shift),
                                      _ptr(out["feat"]), ws_ptr, ws_bytes, _stream(stream)))
    out["_workspace"] = (ws, ws_ptr)
    return out


def voxelize_static(points, n_points, geom, stream=None) -> Dict[str, object]:
    """pp_voxelize_static: same outputs as voxelize(), scratch in the library's static device
    array instead of a workspace (for callers that cannot allocate device memory; the output
    tensors here are still allocated by torch on the caller's side)."""
    import torch
    _need_cuda(points, n_points)
    g = Geometry.of(geom)
    B, cap = int(points.shape[0]), int(points.shape[1])
    dev = points.device
    G, P = g.nx * g.ny, g.max_pillars
    out = {
        "cell": torch.empty((B, cap), dtype=torch.int32, device=dev),
        "cnt": torch.empty((B, G), dtype=torch.int32, device=dev),
        "pillar_of_cell": torch.empty((B, G), dtype=torch.int32, device=dev),
        "coord": torch.empty((B, P), dtype=torch.int32, device=dev),
        "npts": torch.empty((B, P), dtype=torch.int32, device=dev),
        "num_pillars": torch.empty((B,), dtype=torch.int32, device=dev),
        "pts": torch.empty((B, P, 32, 4), dtype=torch.float32, device=dev),
    }
    _check(lib().pp_voxelize_static(ctypes.byref(g), B, cap, _ptr(points), _ptr(n_points), _ptr(out["cell"]),
                                    _ptr(out["cnt"]), _ptr(out["pillar_of_cell"]), _ptr(out["coord"]),
                                    _ptr(out["npts"]), _ptr(out["num_pillars"]), _ptr(out["pts"]),
                                    _stream(stream)))
    return out


def voxelize_check(vox, stream=None) -> None:
    _check(lib().pp_voxelize_check(vox["_workspace"][1], _stream(stream)))


def pointnet(pts, npts, coord, num_pillars, pfn_w, scale_shift, geom, stream=None):
    """Returns feat: cuda float32 [B, P, 64]."""
    import torch
    _need_cuda(pts, npts, coord, num_pillars, pfn_w, scale_shift)
    g = Geometry.of(geom)
    B = int(pts.shape[0])
    feat = torch.empty((B, g.max_pillars, 64), dtype=torch.float32, device=pts.device)
    _check(lib().pp_pointnet(ctypes.byref(g), B, _ptr(pts), _ptr(npts), _ptr(coord), _ptr(num_pillars),
                             _ptr(pfn_w), _ptr(scale_shift), _ptr(feat), _stream(stream)))
    return feat


def scatter(feat, pillar_of_cell, geom, dtype=PP_F32, stream=None):
    """Returns the padded NHWC canvas [B, ny+2, nx+2, 64] (float32 or bfloat16); for
    PP_F32_TC the split FP32 canvas [2, B, ny+2, nx+2, 64] (values, TF32 remainders)."""
    import torch
    _need_cuda(feat, pillar_of_cell)
    g = Geometry.of(geom)
    B = int(feat.shape[0])
    tdt = torch.bfloat16 if dtype == PP_BF16 else torch.float32
    shape = (B, g.ny + 2, g.nx + 2, 64)
    canvas = torch.empty(((2,) if dtype == PP_F32_TC else ()) + shape, dtype=tdt, device=feat.device)
    _check(lib().pp_scatter(ctypes.byref(g), B, _ptr(feat), _ptr(pillar_of_cell), _ptr(canvas), dtype,
                            _stream(stream)))
    return canvas


class ScatterState:
    """A persistent canvas for pp_scatter_update (zero canvas, drawn lists, drawn counts)."""

    def __init__(self, geom, batch, dtype=PP_F32, device="cuda"):
        import torch
        g = Geometry.of(geom)
        self.geom, self.dtype = geom, dtype
        tdt = torch.bfloat16 if dtype == PP_BF16 else torch.float32
        shape = (batch, g.ny + 2, g.nx + 2, 64)
        self.canvas = torch.zeros(((2,) if dtype == PP_F32_TC else ()) + shape, dtype=tdt, device=device)
        self.drawn = torch.zeros((batch, g.max_pillars), dtype=torch.int32, device=device)
        self.drawn_num = torch.zeros((batch,), dtype=torch.int32, device=device)


def scatter_update(state, feat, coord, num_pillars, pillar_of_cell, stream=None):
    """pp_scatter_update on ``state`` (a ScatterState); returns its canvas."""
    _need_cuda(feat, coord, num_pillars, pillar_of_cell)
    g = Geometry.of(state.geom)
    B = int(feat.shape[0])
    _check(lib().pp_scatter_update(ctypes.byref(g), B, _ptr(feat), _ptr(coord), _ptr(num_pillars),
                                   _ptr(pillar_of_cell), _ptr(state.drawn), _ptr(state.drawn_num),
                                   _ptr(state.canvas), state.dtype, _stream(stream)))
    return state.canvas


def pack_conv_weights(w_oihw, dtype, stream=None):
    """w_oihw: cuda float32 [cout, cin, 3, 3] -> packed weights for pp_conv3x3."""
    import torch
    if w_oihw.dim() != 4 or tuple(w_oihw.shape[2:]) != (3, 3):
        raise PPError(PP_EINVAL, "pack_conv_weights: weights must be OIHW [cout, cin, 3, 3], got %s"
                      % (tuple(w_oihw.shape),))
    _need_cuda(w_oihw)
    cout, cin = int(w_oihw.shape[0]), int(w_oihw.shape[1])
    n = lib().pp_conv_packed_bytes(cin, cout, dtype)
    f32 = dtype in (PP_F32, PP_F32_TC)
    dst = torch.empty(n // (4 if f32 else 2), dtype=torch.float32 if f32 else torch.bfloat16, device=w_oihw.device)
    _check(lib().pp_conv_pack_weights(_ptr(w_oihw.contiguous()), cin, cout, dtype, _ptr(dst), _stream(stream)))
    return dst


def bn_fold(bn):
    """bn: host float32 array [4, C] (gamma, beta, mean, var) -> numpy float32 [2, C]."""
    import numpy as np
    a = np.ascontiguousarray(bn, dtype=np.float32)
    c = a.shape[1]
    out = np.empty((2, c), dtype=np.float32)
    _check(lib().pp_bn_fold(a.ctypes.data, c, BN_EPS, out.ctypes.data))
    return out


def tf32_split(x, stream=None):
    """pp_tf32_split: the TF32 remainder plane of a float32 CUDA tensor (same shape)."""
    import torch
    _need_cuda(x)
    x = x.contiguous()
    lo = torch.empty_like(x)
    _check(lib().pp_tf32_split(_ptr(x), _ptr(lo), x.numel(), _stream(stream)))
    return lo


def split_f32(x, stream=None):
    """A float32 tensor as split FP32 (the PP_F32_TC operand form): [2, *x.shape], plane 0 = x,
    plane 1 = its TF32 remainders (computed by pp_tf32_split)."""
    import torch
    out = torch.empty((2,) + tuple(x.shape), dtype=torch.float32, device=x.device)
    out[0].copy_(x)
    _check(lib().pp_tf32_split(_ptr(out[0]), _ptr(out[1]), x.numel(), _stream(stream)))
    return out


def conv_workspace(B, H, W, cin, cout, stride, dtype, device="cuda"):
    """A zeroed, 256-byte aligned device workspace for the stream-K tiles of this conv shape
    (pp_conv_workspace_bytes), as (tensor keeping it alive, pointer, bytes); None if none is
    needed."""
    import torch
    n = int(lib().pp_conv_workspace_bytes(B, H, W, cin, cout, stride, dtype))
    if n == 0:
        return None
    buf = torch.zeros(n + 256, dtype=torch.uint8, device=device)
    ptr = buf.data_ptr() + (-buf.data_ptr()) % 256
    return buf, ptr, n


def conv3x3(x, w_packed, scale_shift, cout, stride, dtype=PP_F32, tile=-1, out=None, stream=None,
            workspace=None):
    """x: padded NHWC [B, H+2, W+2, cin] (float32 for PP_F32, bfloat16 for PP_BF16; for
    PP_F32_TC split FP32 [2, B, H+2, W+2, cin], see split_f32).  Returns the padded output
    [B, Ho+2, Wo+2, cout] (border zero; [2, B, ...] split FP32 for PP_F32_TC).  workspace: a
    conv_workspace() triple for the stream-K tiles (PP_F32_TC; one is made when omitted)."""
    import torch
    _need_cuda(x, w_packed, scale_shift)
    split = dtype == PP_F32_TC
    if split and x.dim() != 5:
        raise PPError(PP_EINVAL, "PP_F32_TC conv takes split FP32 [2, B, H+2, W+2, cin]")
    B, Hp, Wp, cin = (int(v) for v in x.shape[-4:])
    H, W = Hp - 2, Wp - 2
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    if out is None:
        out = torch.zeros(((2,) if split else ()) + (B, Ho + 2, Wo + 2, cout), dtype=x.dtype, device=x.device)
    if split and workspace is None:
        workspace = conv_workspace(B, H, W, cin, cout, stride, dtype, x.device)
    ws_ptr, ws_n = (workspace[1], workspace[2]) if workspace else (None, 0)
    _check(lib().pp_conv3x3_ws(B, H, W, cin, cout, stride, dtype, _ptr(x), _ptr(w_packed), _ptr(scale_shift),
                               _ptr(out), tile, ws_ptr, ws_n, _stream(stream)))
    return out


def pack_upsample_weights(w, up, dtype):
    """Host float32 ConvTranspose2d weights [cin, cout, up, up] -> packed device weights."""
    import numpy as np
    import torch
    w = np.ascontiguousarray(w, dtype=np.float32)
    cin, cout = int(w.shape[0]), int(w.shape[1])
    buf = torch.empty(lib().pp_upsample_packed_bytes(cin, cout, up, dtype), dtype=torch.uint8, device="cuda")
    _check(lib().pp_upsample_pack_weights(w.ctypes.data, cin, cout, up, dtype, _ptr(buf)))
    return buf


def pack_head_weights(w, b, dtype):
    """Host float32 head weights [cout, cin] and bias [cout] -> (packed device weights, device
    scale_shift [2, cout_pad])."""
    import numpy as np
    import torch
    w = np.ascontiguousarray(w, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    cout, cin = int(w.shape[0]), int(w.shape[1])
    buf = torch.empty(lib().pp_head_packed_bytes(cin, cout, dtype), dtype=torch.uint8, device="cuda")
    pad = (cout + 63) // 64 * 64
    ss = torch.empty((2, pad), dtype=torch.float32, device="cuda")
    _check(lib().pp_head_pack_weights(w.ctypes.data, b.ctypes.data, cin, cout, dtype, _ptr(buf), _ptr(ss)))
    return buf, ss


def upsample(x, w_packed, scale_shift, cout, up, dtype, out, out_coff=0, tile=-1, stream=None):
    """pp_upsample of x (padded NHWC [B, H+2, W+2, cin]; split FP32 [2, B, ...] for PP_F32_TC)
    into channels [out_coff, out_coff + cout) of ``out`` ([.., B, up H + 2, up W + 2, out_c])."""
    B, Hp, Wp, cin = (int(v) for v in x.shape[-4:])
    out_c = int(out.shape[-1])
    _check(lib().pp_upsample(B, Hp - 2, Wp - 2, cin, cout, up, dtype, _ptr(x), _ptr(w_packed), _ptr(scale_shift),
                             _ptr(out), out_c, out_coff, tile, _stream(stream)))
    return out


def head(x, w_packed, scale_shift, cout, dtype, tile=-1, out=None, stream=None):
    """pp_head of x -> [(2,) B, H+2, W+2, cout_pad] (channels >= cout are zero)."""
    import torch
    B, Hp, Wp, cin = (int(v) for v in x.shape[-4:])
    pad = (cout + 63) // 64 * 64
    if out is None:
        out = torch.zeros(((2,) if dtype == PP_F32_TC else ()) + (B, Hp, Wp, pad), dtype=x.dtype, device=x.device)
    _check(lib().pp_head(B, Hp - 2, Wp - 2, cin, cout, dtype, _ptr(x), _ptr(w_packed), _ptr(scale_shift),
                         _ptr(out), tile, _stream(stream)))
    return out


def conv_autotune(x, w_packed, scale_shift, cout, stride, dtype, out, reps=5, workspace=None):
    """pp_conv_autotune on the layer shape of ``x`` (padded NHWC; split FP32 [2, B, ...] for
    PP_F32_TC) -> (best tile, us per launch)."""
    B, Hp, Wp, cin = (int(v) for v in x.shape[-4:])
    t, us = ctypes.c_int32(-1), ctypes.c_float(0)
    if dtype == PP_F32_TC and workspace is None:
        workspace = conv_workspace(B, Hp - 2, Wp - 2, cin, cout, stride, dtype, x.device)
    ws_ptr, ws_n = (workspace[1], workspace[2]) if workspace else (None, 0)
    _check(lib().pp_conv_autotune_ws(B, Hp - 2, Wp - 2, cin, cout, stride, dtype, _ptr(x), _ptr(w_packed),
                                     _ptr(scale_shift), _ptr(out), ws_ptr, ws_n, reps, ctypes.byref(t),
                                     ctypes.byref(us)))
    return int(t.value), float(us.value)


def conv_tune_save(path):
    _check(lib().pp_conv_tune_save(str(path).encode()))


def conv_tune_load(path) -> int:
    n = lib().pp_conv_tune_load(str(path).encode())
    if n < 0:
        _check(n)
    return int(n)


def conv_tune_clear():
    lib().pp_conv_tune_clear()


def conv_tile_count(dtype) -> int:
    return int(lib().pp_conv_tile_count(dtype))


def conv_tile_info(dtype, tile):
    """(bh, bw, bn, persistent) of conv tile ``tile``."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().pp_conv_tile_info(dtype, tile, *[ctypes.byref(x) for x in v]))
    return tuple(int(x.value) for x in v)


def device_error(clear: bool = True) -> int:
    v = ctypes.c_uint32(0)
    _check(lib().pp_device_error(ctypes.byref(v), 1 if clear else 0))
    return int(v.value)


def device_error_set(bits: int) -> None:
    """pp_device_error_set: sets bits of the sticky device error word (a test hook)."""
    _check(lib().pp_device_error_set(int(bits)))


# ------------------------------------------------------------------ runtime, pipeline, policy

def make_config(geom, backbone, weights, head=None, **knobs):
    """Builds a pp_config (defaults from pp_config_defaults) for ``geom`` / ``backbone``
    (objects with the pp_synth Geometry/Backbone fields) and ``weights`` =
    (pfn_w [64,9], pfn_bn [4,64], conv_w list, conv_bn list) as float32 arrays; ``head`` =
    (up_w list, up_bn list, head_w, head_b) adds the neck and the detection head.  Returns the
    config and the list of arrays it points into (keep it alive while the config is used)."""
    import numpy as np
    cfg = Config()
    lib().pp_config_defaults(ctypes.byref(cfg))
    cfg.geom = Geometry.of(geom)
    cfg.n_blocks = len(backbone.convs)
    for i, (n, c, st) in enumerate(zip(backbone.convs, backbone.chans, backbone.strides)):
        cfg.convs[i], cfg.chans[i], cfg.strides[i] = n, c, st
    pfn_w, pfn_bn, conv_w, conv_bn = weights
    keep = [np.ascontiguousarray(pfn_w, dtype=np.float32), np.ascontiguousarray(pfn_bn, dtype=np.float32)]
    cw = [np.ascontiguousarray(w, dtype=np.float32) for w in conv_w]
    cb = [np.ascontiguousarray(b, dtype=np.float32) for b in conv_bn]
    arr_w = (ctypes.c_void_p * len(cw))(*[a.ctypes.data for a in cw])
    arr_b = (ctypes.c_void_p * len(cb))(*[a.ctypes.data for a in cb])
    keep += cw + cb + [arr_w, arr_b]
    cfg.pfn_w, cfg.pfn_bn = keep[0].ctypes.data, keep[1].ctypes.data
    cfg.conv_w = ctypes.cast(arr_w, ctypes.c_void_p)
    cfg.conv_bn = ctypes.cast(arr_b, ctypes.c_void_p)
    if head is not None:
        up_w, up_bn, head_w, head_b = head
        uw = [np.ascontiguousarray(w, dtype=np.float32) for w in up_w]
        ub = [np.ascontiguousarray(b, dtype=np.float32) for b in up_bn]
        hw, hb = np.ascontiguousarray(head_w, dtype=np.float32), np.ascontiguousarray(head_b, dtype=np.float32)
        arr_uw = (ctypes.c_void_p * len(uw))(*[a.ctypes.data for a in uw])
        arr_ub = (ctypes.c_void_p * len(ub))(*[a.ctypes.data for a in ub])
        keep += uw + ub + [hw, hb, arr_uw, arr_ub]
        cfg.head_outputs, cfg.up_channels = int(hw.shape[0]), int(uw[0].shape[1])
        cfg.up_w = ctypes.cast(arr_uw, ctypes.c_void_p)
        cfg.up_bn = ctypes.cast(arr_ub, ctypes.c_void_p)
        cfg.head_w, cfg.head_b = hw.ctypes.data, hb.ctypes.data
    for k, v in knobs.items():
        if not hasattr(cfg, k):
            raise PPError(PP_EINVAL, "unknown config field %s" % k)
        setattr(cfg, k, v)
    return cfg, keep


class Context:
    """A serving context (pp_create ... pp_destroy)."""

    def __init__(self, cfg):
        h = ctypes.c_void_p()
        _check(lib().pp_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h

    def register_chain(self, chain_id, period_ms, deadline_ms, precision):
        _check(lib().pp_register_chain(self.h, chain_id, period_ms, deadline_ms, precision))

    def register_synthetic_chain(self, chain_id, period_ms, deadline_ms, n_kernels, kernel_us, util):
        """A synthetic-load chain: each frame runs n_kernels kernels of about kernel_us on
        round(util x SMs) SMs (submit its frames with no points)."""
        _check(lib().pp_register_synthetic_chain(self.h, chain_id, period_ms, deadline_ms, n_kernels, kernel_us,
                                                 util))

    def submit(self, chain_id, points, t_arrival_us=None, abs_deadline_us=0.0, n_points=None):
        """points: numpy float32 [N, 4] (host; copied), a CUDA tensor [N, 4] (device; borrowed
        until the frame is polled) or a pinned CPU tensor (borrowed; the kernels read it in
        place).  Returns (status, frame_id); status PP_EAGAIN when not admitted."""
        fid = ctypes.c_uint64(0)
        t = now_us() if t_arrival_us is None else t_arrival_us
        mode = _points_mode(points)
        if mode != PP_POINTS_HOST:
            n = int(points.shape[0]) if n_points is None else n_points
            rc = lib().pp_submit_frame(self.h, chain_id, _ptr(points), n, mode, t, abs_deadline_us, ctypes.byref(fid))
        else:
            import numpy as np
            a = np.ascontiguousarray(points, dtype=np.float32)
            n = int(a.shape[0]) if n_points is None else n_points
            rc = lib().pp_submit_frame(self.h, chain_id, a.ctypes.data if n else None, n, 0, t, abs_deadline_us,
                                       ctypes.byref(fid))
        if rc not in (PP_OK, PP_EAGAIN):
            _check(rc)
        return rc, int(fid.value)

    def submit_many(self, chain_ids, frames, t_arrival_us=None, abs_deadlines_us=None, host_out=None):
        """Submits frames that arrive together (one pp_submit_frames call): ``frames`` are all
        CUDA tensors [N, 4] (borrowed), all pinned CPU tensors (borrowed, read in place) or all
        host arrays (copied).  ``host_out``: optional list of pinned CPU tensors (each at least
        result_bytes(precision) bytes, or None) that receive each frame's outputs
        (pp_submit_frames_ex).  Returns (status, ids of the admitted frames, in order)."""
        n = len(frames)
        t = now_us() if t_arrival_us is None else t_arrival_us
        mode = _points_mode(frames[0]) if n else PP_POINTS_HOST
        dev = mode != PP_POINTS_HOST
        keep = []
        if dev:
            ptrs = [_ptr(f) for f in frames]
        else:
            import numpy as np
            keep = [np.ascontiguousarray(f, dtype=np.float32) for f in frames]
            ptrs = [a.ctypes.data if a.shape[0] else None for a in keep]
        cids = (ctypes.c_int32 * n)(*chain_ids)
        parr = (ctypes.c_void_p * n)(*ptrs)
        cnt = (ctypes.c_int64 * n)(*[int(f.shape[0]) for f in frames])
        dls = (ctypes.c_double * n)(*abs_deadlines_us) if abs_deadlines_us is not None else None
        ids = (ctypes.c_uint64 * n)()
        got = ctypes.c_int32(0)
        if host_out is None:
            rc = lib().pp_submit_frames(self.h, n, cids, parr, cnt, mode, t, dls, ids, ctypes.byref(got))
        else:
            hout = (ctypes.c_void_p * n)(*[(_ptr(x) if x is not None else None) for x in host_out])
            rc = lib().pp_submit_frames_ex(self.h, n, cids, parr, cnt, mode, t, dls, hout, ids, ctypes.byref(got))
        if rc not in (PP_OK, PP_EAGAIN):
            _check(rc)
        return rc, [int(ids[i]) for i in range(got.value)]

    def result_bytes(self, precision):
        """pp_result_bytes: size of one frame's outputs (a host output buffer) at ``precision``."""
        return int(lib().pp_result_bytes(self.h, precision))

    def release_many(self, frame_ids):
        n = len(frame_ids)
        if n:
            _check(lib().pp_result_release_many(self.h, n, (ctypes.c_uint64 * n)(*frame_ids)))

    def poll(self, max_results=64, timeout_us=0):
        buf = (Result * max_results)()
        n = ctypes.c_int32(0)
        _check(lib().pp_poll(self.h, buf, max_results, ctypes.byref(n), int(timeout_us)))
        return [buf[i] for i in range(n.value)]

    def release(self, frame_id):
        _check(lib().pp_result_release(self.h, ctypes.c_uint64(frame_id)))

    def replay(self, arrivals, clouds, timeout_us=10e6):
        """pp_replay: ``arrivals`` = [(t_us, chain_id, cloud index, n_points)] sorted by time;
        ``clouds`` all CUDA tensors [N, 4] (borrowed) or all host arrays.  Returns the replay
        statistics as a dict (chain_rejected as a list)."""
        n = len(arrivals)
        arr = (Arrival * max(1, n))(*[Arrival(float(t), int(c), int(k), int(m)) for t, c, k, m in arrivals])
        mode = _points_mode(clouds[0])
        dev = mode != PP_POINTS_HOST
        keep = clouds if dev else [__import__("numpy").ascontiguousarray(x, dtype="float32") for x in clouds]
        ptrs = (ctypes.c_void_p * len(keep))(*[(_ptr(x) if dev else x.ctypes.data) for x in keep])
        cnt = (ctypes.c_int64 * len(keep))(*[int(x.shape[0]) for x in keep])
        st = ReplayStats()
        _check(lib().pp_replay(self.h, arr, n, ptrs, cnt, len(keep), mode, float(timeout_us),
                               ctypes.byref(st)))
        d = {k: getattr(st, k) for k, _ in st._fields_ if k != "chain_rejected"}
        d["chain_rejected"] = list(st.chain_rejected)
        return d

    def decision_log(self):
        """pp_decision_log: every logged release decision as a dict with the time ``t_us``, the
        rule's configuration ``cfg`` (dict of PolicyConfig fields), ``closed_pending``,
        ``ready`` (list of dicts of PolicyFrame fields), ``active`` (list of (chain_id, ul)),
        ``launched`` and the decision (``kind``, ``frames``, ``level``, ``drops``)."""
        nr, nf, na, nd = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        L = lib()
        _check(L.pp_decision_log(self.h, None, 0, None, 0, None, 0, None, 0, ctypes.byref(nr), ctypes.byref(nf),
                                 ctypes.byref(na), ctypes.byref(nd)))
        recs = (DecisionRecord * max(1, nr.value))()
        rf = (PolicyFrame * max(1, nf.value))()
        ac = (PolicyActive * max(1, na.value))()
        dr = (ctypes.c_uint64 * max(1, nd.value))()
        _check(L.pp_decision_log(self.h, recs, len(recs), rf, len(rf), ac, len(ac), dr, len(dr), ctypes.byref(nr),
                                 ctypes.byref(nf), ctypes.byref(na), ctypes.byref(nd)))
        out = []
        for k in range(nr.value):
            r = recs[k]
            d = r.decision
            out.append({
                "t_us": r.t_us, "cfg": {n: getattr(r.cfg, n) for n, _ in PolicyConfig._fields_},
                "closed_pending": r.closed_pending, "launched": r.launched,
                "ready": [{n: getattr(rf[r.ready_off + i], n) for n, _ in PolicyFrame._fields_}
                          for i in range(r.n_ready)],
                "active": [(ac[r.active_off + i].chain_id, ac[r.active_off + i].ul) for i in range(r.n_active)],
                "kind": d.kind, "frames": [int(d.frames[i]) for i in range(d.n_frames)], "level": d.level,
                "drops": [int(dr[r.drops_off + i]) for i in range(d.n_drops)]})
        return out

    def stats(self):
        s = Stats()
        _check(lib().pp_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def stats_reset(self):
        """pp_stats_reset: the statistics start afresh (frames in flight and estimates kept)."""
        _check(lib().pp_stats_reset(self.h))

    def destroy(self):
        if self.h:
            rc = lib().pp_destroy(self.h)
            self.h = None
            _check(rc)


def now_us() -> float:
    return float(lib().pp_now_us())


def noise_factor(seed, frame_id, eps) -> float:
    """pp_noise_factor: the estimate-noise factor the runtime gives frame ``frame_id``."""
    return float(lib().pp_noise_factor(seed, frame_id, eps))


def result_host_tensor(r):
    """A result's host copy of its final output (pp_submit_frames_ex) as a CPU tensor view
    [h+2, w+2, c] (float32 or bfloat16; valid while the caller's buffer lives)."""
    import numpy as np
    import torch
    ptr = r.out_host
    if not ptr:
        raise PPError(PP_ESTATE, "frame %d has no host output" % r.frame_id)
    c, h, w = r.out_c, r.out_h, r.out_w
    n = (h + 2) * (w + 2) * c
    if r.out_dtype == PP_F32:
        a = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_float)), shape=(n,))
        return torch.from_numpy(a).view(h + 2, w + 2, c)
    a = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_int16)), shape=(n,))
    return torch.from_numpy(a).view(h + 2, w + 2, c).view(torch.bfloat16)


def result_tensor(r, block=None):
    """Wraps a result's output (the last layer, or block ``block``) as a torch tensor view of
    the padded NHWC device buffer [h+2, w+2, c] (valid until the frame is released)."""
    import torch
    if not r.out_dev:
        raise PPError(PP_ESTATE, "frame %d has no output (status %d)" % (r.frame_id, r.status))
    if block is None:
        ptr, c, h, w = r.out_dev, r.out_c, r.out_h, r.out_w
    else:
        ptr, c, h, w = r.block_dev[block], r.block_c[block], r.block_h[block], r.block_w[block]
    dt = torch.float32 if r.out_dtype == PP_F32 else torch.bfloat16
    return _device_view(ptr, (h + 2, w + 2, c), dt)


class _CudaArray:
    """Minimal __cuda_array_interface__ exporter for a device buffer the library owns."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _device_view(ptr, shape, dtype):
    """Copy of the device buffer of ``shape``/``dtype`` at ``ptr`` as a new CUDA tensor."""
    import torch
    if dtype == torch.bfloat16:
        t = torch.as_tensor(_CudaArray(ptr, shape, "<i2"), device="cuda").view(torch.bfloat16)
    elif dtype == torch.float32:
        t = torch.as_tensor(_CudaArray(ptr, shape, "<f4"), device="cuda")
    elif dtype == torch.int32:
        t = torch.as_tensor(_CudaArray(ptr, shape, "<i4"), device="cuda")
    else:
        raise PPError(PP_EINVAL, "unsupported dtype %s" % dtype)
    return t.clone()


class Pipeline:
    """One release unit without the runtime (pp_pipeline_*)."""

    def __init__(self, cfg, precision):
        h = ctypes.c_void_p()
        _check(lib().pp_pipeline_create(ctypes.byref(cfg), precision, ctypes.byref(h)))
        self.h = h
        self.precision = precision

    def run(self, frames, counts=None, use_graph=True, stream=None):
        """frames: list of CUDA tensors [N_i, 4] (or host numpy arrays)."""
        n = len(frames)
        ptrs = (ctypes.c_void_p * n)(*[(_ptr(f) if hasattr(f, "data_ptr") else f.ctypes.data) for f in frames])
        cnt = (ctypes.c_int32 * n)(*[int(f.shape[0]) for f in frames] if counts is None else counts)
        _check(lib().pp_pipeline_run(self.h, n, ptrs, cnt, 1 if use_graph else 0, _stream(stream)))

    def output(self, i, block):
        d = ctypes.c_void_p()
        c, h, w = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().pp_pipeline_output(self.h, i, block, ctypes.byref(d), ctypes.byref(c), ctypes.byref(h),
                                        ctypes.byref(w)))
        return d.value, c.value, h.value, w.value

    def output_tensor(self, i, block):
        import torch
        ptr, c, h, w = self.output(i, block)
        dt = torch.float32 if self.precision == PP_F32 else torch.bfloat16
        return _device_view(ptr, (h + 2, w + 2, c), dt)

    def num_pillars(self, i):
        import torch
        ptr, _, _, _ = self.output(i, -1)
        return int(_device_view(ptr, (1,), torch.int32)[0])

    def bytes(self):
        return int(lib().pp_pipeline_bytes(self.h))

    def destroy(self):
        if self.h:
            lib().pp_pipeline_destroy(self.h)
            self.h = None


def policy_decide(cfg, t_us, ready, active, closed_pending):
    """Calls pp_policy_decide.  ready: list of dicts with PolicyFrame fields; active: list of
    (chain_id, ul).  Returns (kind, frame ids, level, drop ids)."""
    pc = PolicyConfig(**cfg)
    rf = (PolicyFrame * max(1, len(ready)))(*[PolicyFrame(**r) for r in ready])
    ac = (PolicyActive * max(1, len(active)))(*[PolicyActive(c, u) for c, u in active])
    d = PolicyDecision()
    drops = (ctypes.c_uint64 * max(1, len(ready)))()
    _check(lib().pp_policy_decide(ctypes.byref(pc), float(t_us), rf, len(ready), ac, len(active),
                                  int(closed_pending), ctypes.byref(d), drops, len(ready)))
    return d.kind, [int(d.frames[i]) for i in range(d.n_frames)], d.level, [int(drops[i]) for i in range(d.n_drops)]


def policy_priority(cfg, t_us, frame):
    """pp_policy_priority: the priority of one frame (dict of PolicyFrame fields) under cfg."""
    return float(lib().pp_policy_priority(ctypes.byref(PolicyConfig(**cfg)), float(t_us),
                                          ctypes.byref(PolicyFrame(**frame))))

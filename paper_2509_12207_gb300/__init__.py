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
PP_F32, PP_BF16 = 0, 1
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
    "pp_pointnet": (ctypes.c_int, [_GP, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pp_scatter": (ctypes.c_int, [_GP, _I, _P, _P, _P, _I, _P]),
    "pp_conv3x3": (ctypes.c_int, [_I, _I, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I, _P]),
    "pp_conv_tile_count": (ctypes.c_int, [_I]),
    "pp_conv_packed_bytes": (_SZ, [_I, _I, _I]),
    "pp_conv_pack_weights": (ctypes.c_int, [_P, _I, _I, _I, _P, _P]),
    "pp_bn_fold": (ctypes.c_int, [_P, _I, ctypes.c_float, _P]),
    "pp_device_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32), _I]),
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
    ws = torch.zeros(ws_bytes + 256, dtype=torch.uint8, device=dev)
    off = (-ws.data_ptr()) % 256
    ws_ptr = ws.data_ptr() + off
    s = _stream(stream)
    _check(lib().pp_voxelize(ctypes.byref(g), B, cap, _ptr(points), _ptr(n_points), _ptr(out["cell"]),
                             _ptr(out["cnt"]), _ptr(out["pillar_of_cell"]), _ptr(out["coord"]),
                             _ptr(out["npts"]), _ptr(out["num_pillars"]), _ptr(out["pts"]),
                             ws_ptr, ws_bytes, s))
    out["_workspace"] = (ws, ws_ptr)
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
    """Returns the padded NHWC canvas [B, ny+2, nx+2, 64] (float32 or bfloat16)."""
    import torch
    _need_cuda(feat, pillar_of_cell)
    g = Geometry.of(geom)
    B = int(feat.shape[0])
    tdt = torch.float32 if dtype == PP_F32 else torch.bfloat16
    canvas = torch.empty((B, g.ny + 2, g.nx + 2, 64), dtype=tdt, device=feat.device)
    _check(lib().pp_scatter(ctypes.byref(g), B, _ptr(feat), _ptr(pillar_of_cell), _ptr(canvas), dtype,
                            _stream(stream)))
    return canvas


def pack_conv_weights(w_oihw, dtype, stream=None):
    """w_oihw: cuda float32 [cout, cin, 3, 3] -> packed weights for pp_conv3x3."""
    import torch
    _need_cuda(w_oihw)
    cout, cin = int(w_oihw.shape[0]), int(w_oihw.shape[1])
    n = lib().pp_conv_packed_bytes(cin, cout, dtype)
    dst = torch.empty(n // (4 if dtype == PP_F32 else 2),
                      dtype=torch.float32 if dtype == PP_F32 else torch.bfloat16, device=w_oihw.device)
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


def conv3x3(x, w_packed, scale_shift, cout, stride, dtype=PP_F32, tile=-1, out=None, stream=None):
    """x: padded NHWC [B, H+2, W+2, cin] (float32 for PP_F32, bfloat16 for PP_BF16).
    Returns the padded output [B, Ho+2, Wo+2, cout] (border zero)."""
    import torch
    _need_cuda(x, w_packed, scale_shift)
    B, Hp, Wp, cin = (int(v) for v in x.shape)
    H, W = Hp - 2, Wp - 2
    Ho, Wo = (H - 1) // stride + 1, (W - 1) // stride + 1
    if out is None:
        out = torch.zeros((B, Ho + 2, Wo + 2, cout), dtype=x.dtype, device=x.device)
    _check(lib().pp_conv3x3(B, H, W, cin, cout, stride, dtype, _ptr(x), _ptr(w_packed), _ptr(scale_shift),
                            _ptr(out), tile, _stream(stream)))
    return out


def conv_tile_count(dtype) -> int:
    return int(lib().pp_conv_tile_count(dtype))


def device_error(clear: bool = True) -> int:
    v = ctypes.c_uint32(0)
    _check(lib().pp_device_error(ctypes.byref(v), 1 if clear else 0))
    return int(v.value)
